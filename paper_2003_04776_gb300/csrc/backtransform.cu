// backtransform.cu -- eigenvectors of the original pencil (Section 1): with
// (A, B) = (Q S Z^T, Q T Z^T) reduced to the real Schur pencil (S, T), a right
// eigenvector v of (S, T) gives x = Z v for (A, B); likewise x = Z v with
// (A, B) = (Q S Z^H, Q T Z^H) for a complex Schur pencil (ZGEMM below).  X = Z V is one FP64 GEMM
// (cuBLAS, natively or by its fixed-point emulation on the tensor cores);
// every eigenvector is then normalised so that its entry of largest modulus
// is exactly 1, with the same rule as the solve's post-pass.
#include <cublas_v2.h>

#include "common.cuh"
#include "cplx.cuh"

namespace pevc {

int bt_handle(void** h, cudaStream_t s) {
  if (!*h) {
    cublasHandle_t c = nullptr;
    if (cublasCreate(&c) != CUBLAS_STATUS_SUCCESS) return PEVC_ERR_CUDA;
    *h = c;
  }
  return cublasSetStream(static_cast<cublasHandle_t>(*h), s) == CUBLAS_STATUS_SUCCESS ? 0 : PEVC_ERR_CUDA;
}

void bt_handle_destroy(void* h) {
  if (h) cublasDestroy(static_cast<cublasHandle_t>(h));
}

// X = Z V (n x m, all column-major FP64).
int bt_gemm(void* h, bool emulated, int n, int m, const double* Z, int ldz, const double* V, int ldv, double* X,
            int ldx) {
  cublasHandle_t c = static_cast<cublasHandle_t>(h);
  const double one = 1.0, zero = 0.0;
  if (!emulated)
    return cublasDgemm(c, CUBLAS_OP_N, CUBLAS_OP_N, n, m, n, &one, Z, ldz, V, ldv, &zero, X, ldx) ==
                   CUBLAS_STATUS_SUCCESS
               ? 0
               : PEVC_ERR_CUDA;
  if (cublasSetEmulationStrategy(c, CUBLAS_EMULATION_STRATEGY_EAGER) != CUBLAS_STATUS_SUCCESS)
    return PEVC_ERR_UNSUPPORTED;
  const cublasStatus_t r = cublasGemmEx(c, CUBLAS_OP_N, CUBLAS_OP_N, n, m, n, &one, Z, CUDA_R_64F, ldz, V,
                                        CUDA_R_64F, ldv, &zero, X, CUDA_R_64F, ldx,
                                        CUBLAS_COMPUTE_64F_EMULATED_FIXEDPOINT, CUBLAS_GEMM_DEFAULT);
  cublasSetEmulationStrategy(c, CUBLAS_EMULATION_STRATEGY_DEFAULT);
  if (r == CUBLAS_STATUS_NOT_SUPPORTED) return PEVC_ERR_UNSUPPORTED;
  return r == CUBLAS_STATUS_SUCCESS ? 0 : PEVC_ERR_CUDA;
}

struct BtBest {
  unsigned long long v;   // magnitude key: the bits of |x|, or of the modulus hypot(re, im)
  int i;
};

__device__ __forceinline__ BtBest bt_better(BtBest a, BtBest b) {
  return (b.v > a.v || (b.v == a.v && b.i < a.i)) ? b : a;
}

// One CTA per eigenvector (a real column, or the first column of a pair).
__global__ void __launch_bounds__(256) k_bt_normalise(double* X, int ldx, int n, const signed char* kind) {
  const int q = blockIdx.x;
  const int kd = kind[q];
  if (kd == 2) return;
  const bool pair = kd == 1;
  double* x0 = X + (size_t)q * ldx;
  double* x1 = pair ? x0 + ldx : nullptr;
  const int tid = threadIdx.x;
  __shared__ BtBest s_red[8];
  // the entry of largest modulus (first index on ties)
  BtBest best{0ull, 0x7fffffff};
  for (int r = tid; r < n; r += blockDim.x) {
    const double vr = x0[r];
    // the modulus itself, not its square: a square overflows above 2^511 and
    // would make every large entry tie (unnormalised columns reach 2^1022)
    const unsigned long long key = pair ? abs_key(hypot(vr, x1[r])) : abs_key(vr);
    best = bt_better(best, BtBest{key, r});
  }
  for (int o = 16; o > 0; o >>= 1) {
    BtBest other{(unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)best.v, o),
                 __shfl_xor_sync(0xffffffffu, best.i, o)};
    best = bt_better(best, other);
  }
  if ((tid & 31) == 0) s_red[tid >> 5] = best;
  __syncthreads();
  if (tid == 0) {
    BtBest b = s_red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = bt_better(b, s_red[w]);
    s_red[0] = b;
  }
  __syncthreads();
  best = s_red[0];
  if (!best.v) return;   // an all-zero vector stays zero
  const int istar = best.i;
  const double dr = x0[istar], di = pair ? x1[istar] : 0.0;
  // 1 / d for a real vector; conj(d) / |d|^2 for a complex one, with d scaled
  // by 2^-e (e the exponent bound of its larger part) so |d|^2 cannot overflow
  const int e = exp_ub(max_nonneg(fabs(dr), fabs(di)));
  const double sr = pow2_scale(dr, -e), si = pow2_scale(di, -e);
  const double s2 = 1.0 / fma(sr, sr, si * si);
  const double nr = sr * s2, ni = si * s2;
  __syncthreads();   // every thread has read x[istar]
  for (int r = tid; r < n; r += blockDim.x) {
    if (pair) {
      const double vr = x0[r], vi = x1[r];
      double zr = pow2_scale(fma(vr, nr, vi * ni), -e), zi = pow2_scale(fma(vi, nr, -(vr * ni)), -e);
      if (r == istar) { zr = 1.0; zi = 0.0; }
      x0[r] = zr;
      x1[r] = zi;
    } else {
      x0[r] = (r == istar) ? 1.0 : x0[r] / dr;
    }
  }
}

// Complex eigenvectors (interleaved complex128 columns), one CTA per column:
// the entry of largest modulus (first index on ties) becomes exactly 1.
__global__ void __launch_bounds__(256) k_bt_normalise_c(double* X, int ldx, int n) {
  const int q = blockIdx.x;
  double* x = X + 2 * (size_t)q * ldx;
  const int tid = threadIdx.x;
  __shared__ BtBest s_red[8];
  BtBest best{0ull, 0x7fffffff};
  for (int r = tid; r < n; r += blockDim.x) {
    const double vr = x[2 * r], vi = x[2 * r + 1];
    best = bt_better(best, BtBest{abs_key(hypot(vr, vi)), r});   // the modulus: its square could overflow
  }
  for (int o = 16; o > 0; o >>= 1) {
    BtBest other{(unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)best.v, o),
                 __shfl_xor_sync(0xffffffffu, best.i, o)};
    best = bt_better(best, other);
  }
  if ((tid & 31) == 0) s_red[tid >> 5] = best;
  __syncthreads();
  if (tid == 0) {
    BtBest b = s_red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = bt_better(b, s_red[w]);
    s_red[0] = b;
  }
  __syncthreads();
  best = s_red[0];
  if (!best.v) return;   // an all-zero vector stays zero
  const int istar = best.i;
  const double dr = x[2 * istar], di = x[2 * istar + 1];
  // z / d = z conj(d') / |d'|^2 * 2^-e with d' = 2^-e d, so |d'|^2 cannot overflow
  const int e = exp_ub(max_nonneg(fabs(dr), fabs(di)));
  const double sr = pow2_scale(dr, -e), si = pow2_scale(di, -e);
  const double s2 = 1.0 / fma(sr, sr, si * si);
  const double nr = sr * s2, ni = si * s2;
  __syncthreads();   // every thread has read x[istar]
  for (int r = tid; r < n; r += blockDim.x) {
    const double vr = x[2 * r], vi = x[2 * r + 1];
    double zr = pow2_scale(fma(vr, nr, vi * ni), -e), zi = pow2_scale(fma(vi, nr, -(vr * ni)), -e);
    if (r == istar) { zr = 1.0; zi = 0.0; }
    x[2 * r] = zr;
    x[2 * r + 1] = zi;
  }
}

// X = Z V for complex128 column-major arrays (cuBLAS ZGEMM).
int bt_zgemm(void* h, int n, int m, const double* Z, int ldz, const double* V, int ldv, double* X, int ldx) {
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
  return cublasZgemm(static_cast<cublasHandle_t>(h), CUBLAS_OP_N, CUBLAS_OP_N, n, m, n, &one,
                     reinterpret_cast<const cuDoubleComplex*>(Z), ldz, reinterpret_cast<const cuDoubleComplex*>(V),
                     ldv, &zero, reinterpret_cast<cuDoubleComplex*>(X), ldx) == CUBLAS_STATUS_SUCCESS
             ? 0
             : PEVC_ERR_CUDA;
}

cudaError_t launch_bt_normalise_c(double* X, int ldx, int n, int m, cudaStream_t s) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  k_bt_normalise_c<<<m, 256, 0, s>>>(X, ldx, n);
  return cudaGetLastError();
}

cudaError_t launch_bt_normalise(double* X, int ldx, int n, int m, const signed char* kind, cudaStream_t s) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  k_bt_normalise<<<m, 256, 0, s>>>(X, ldx, n, kind);
  return cudaGetLastError();
}

}  // namespace pevc

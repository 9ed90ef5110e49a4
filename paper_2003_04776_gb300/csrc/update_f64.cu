// update_f64.cu -- kernel 2 of Section 3 in FP64 on the tensor cores (DMMA,
// mma.sync m8n8k4 f64): the robust left update
//     Y_kj <- 2^sY Y_kj - [S_ki  T_ki] * 2^sX [X D ; -X B]
// for every tile k < i and column tile j >= i of stage i, with X = Y_ij.
//
// Before the product every column is consolidated (Algorithm 3: gamma =
// min(alpha_X, alpha_Y), i.e. the larger exponent) and protected
// (ProtectUpdate with ||Y||, ||[S_ki T_ki]||_inf and ||X''||), and the right
// update X'' = [X D; -X B] (Algorithm 2) is kept below Omega; the scale
// factors are applied on the fly instead of rescaling X and Y in place.  The
// epilogue writes the new per-column maxima (the norm bookkeeping of
// Section 4).
#include "common.cuh"

namespace pevc {

constexpr int kUpdCols = 32;   // output columns per CTA
constexpr int kUpdK = 16;      // K chunk

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

// mode 0: stage i, tiles k < i, j >= i, X = tile (i, j) of (Xsrc, exX, nrmX).
// mode 1: the diagonal-tile term of a residual: k = i = blockIdx.y, j >= k,
//         with the quasi-triangular part of [S_kk T_kk] only.
__global__ void __launch_bounds__(256) k_update_f64(Problem P, int i_stage, int k_lo, int mode,
                                                    const double* __restrict__ Xsrc, const int* __restrict__ exX,
                                                    const double* __restrict__ nrmX) {
  const int nsub = P.tb / kUpdCols;
  const int k = k_lo + (int)blockIdx.y;
  const int i = (mode == 0) ? i_stage : k;
  const int j = ((mode == 0) ? i_stage : 0) + (int)blockIdx.x / nsub;
  if (j < i) return;
  const int sub = (int)blockIdx.x % nsub;
  const int cs = P.cstart[j], ce = P.cstart[j + 1];
  const int c0 = cs + sub * kUpdCols;
  if (c0 >= ce) return;
  const int nc = min(kUpdCols, ce - c0);
  const int rk0 = P.toff[k], hk = P.toff[k + 1] - rk0;
  const int ri0 = P.toff[i], hi = P.toff[i + 1] - ri0;
  const int K = 2 * hi;
  double* Yt = tile_ptr(P, k, j);
  const double* Xt = Xsrc + tri_index(i, j) * (long long)P.tb * P.tb;
  const int tb = P.tb;
  const int tid = threadIdx.x;

  __shared__ double As[kUpdK][kMaxTile + 4];
  __shared__ double Bs[kUpdK][kUpdCols + 4];
  __shared__ int s_sY[kUpdCols], s_sX[kUpdCols], s_e[kUpdCols], s_on[kUpdCols], s_yz[kUpdCols];
  __shared__ int s_kind[kUpdCols];
  __shared__ double s_a[kUpdCols], s_b[kUpdCols], s_beta[kUpdCols], s_nrm[kUpdCols];
  __shared__ int s_any;

  if (tid == 0) s_any = 0;
  __syncthreads();
  if (tid < kUpdCols) {
    int on = 0, sY = 0, sX = 0, en = 0;
    bool yz = true;
    if (tid < nc) {
      const int q = c0 + tid;
      on = update_scales(P, exX, nrmX, k, i, q, sY, sX, en, yz) ? 1 : 0;
      const int kd = P.kind[q];
      const int cc = (kd == 2) ? P.ccol[q] - 1 : P.ccol[q];
      s_kind[tid] = kd;
      s_a[tid] = P.ca[cc];
      s_b[tid] = P.cb[cc];
      s_beta[tid] = P.cbeta[cc];
    }
    s_on[tid] = on;
    s_sY[tid] = sY;
    s_sX[tid] = sX;
    s_e[tid] = en;
    s_yz[tid] = yz ? 1 : 0;
    s_nrm[tid] = 0.0;
    if (on) atomicOr(&s_any, 1);
  }
  __syncthreads();
  if (!s_any) return;

  const int warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t4 = lane & 3;
  const int wr = warp & 3, wc = warp >> 2;
  double acc[4][2][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) { acc[a][b][0] = 0.0; acc[a][b][1] = 0.0; }

  for (int kb = 0; kb < K; kb += kUpdK) {
    for (int idx = tid; idx < kUpdK * kMaxTile; idx += 256) {
      const int kk = idx / kMaxTile, row = idx % kMaxTile;
      const int kap = kb + kk;
      double v = 0.0;
      if (row < hk && kap < K) {
        const int gr = rk0 + row, gc = ri0 + (kap < hi ? kap : kap - hi);
        bool ok = true;
        if (mode == 1) ok = (kap < hi) ? (gc >= gr || (gc == gr - 1 && P.blk[gr] == 2)) : (gc >= gr);
        if (ok) v = (kap < hi) ? P.S[(size_t)gc * P.lds + gr] : P.T[(size_t)gc * P.ldt + gr];
      }
      As[kk][row] = v;
    }
    for (int idx = tid; idx < kUpdK * kUpdCols; idx += 256) {
      const int kk = idx / kUpdCols, col = idx % kUpdCols;
      const int kap = kb + kk;
      double v = 0.0;
      if (col < nc && kap < K && s_on[col]) {
        const int lq = c0 + col - cs;
        const int sx = s_sX[col];
        const int kd = s_kind[col];
        if (kap < hi) {
          v = s_beta[col] * pow2_scale(Xt[(size_t)lq * tb + kap], sx);
        } else {
          const int kp = kap - hi;
          const double a = s_a[col], b = s_b[col];
          if (kd == 0) {
            v = -a * pow2_scale(Xt[(size_t)lq * tb + kp], sx);
          } else if (kd == 1) {
            const double xr = pow2_scale(Xt[(size_t)lq * tb + kp], sx);
            const double xi = pow2_scale(Xt[(size_t)(lq + 1) * tb + kp], sx);
            v = -(a * xr - b * xi);
          } else {
            const double xr = pow2_scale(Xt[(size_t)(lq - 1) * tb + kp], sx);
            const double xi = pow2_scale(Xt[(size_t)lq * tb + kp], sx);
            v = -(b * xr + a * xi);
          }
        }
      }
      Bs[kk][col] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kUpdK; kk += 4) {
      // mode 1: [S_kk T_kk] is quasi-triangular (S_rc = 0 for c < r - 1,
      // T_rc = 0 for c < r), so a K step whose four columns all lie left of
      // the warp's first row (32 wr) minus one multiplies zeros only: the
      // warp skips it (warp-uniform; the same sums, without the zero terms)
      if (mode == 1) {
        const int kap = kb + kk + 3;                          // the step's last K index
        const int c = kap < hi ? kap : kap - hi;              // its local column in S or T
        if (kap < K && (kap < hi ? c < 32 * wr - 1 : (kb + kk >= hi && c < 32 * wr - 1))) continue;
      }
      double af[4], bf[2];
#pragma unroll
      for (int a = 0; a < 4; ++a) af[a] = As[kk + t4][32 * wr + 8 * a + g];
#pragma unroll
      for (int b = 0; b < 2; ++b) bf[b] = Bs[kk + t4][16 * wc + 8 * b + g];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) dmma(acc[a][b][0], acc[a][b][1], af[a], bf[b]);
    }
    __syncthreads();
  }

  // epilogue: Y <- 2^sY Y - acc, column maxima
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int row = 32 * wr + 8 * a + g;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int col = 16 * wc + 8 * b + 2 * t4 + e;
        if (row < hk && col < nc && s_on[col]) {
          const size_t off = (size_t)(c0 + col - cs) * tb + row;
          const double yold = s_yz[col] ? 0.0 : pow2_scale(Yt[off], s_sY[col]);
          const double ynew = yold - acc[a][b][e];
          Yt[off] = ynew;
          if (ynew != 0.0) atomic_max_nonneg(&s_nrm[col], fabs(ynew));
        }
      }
    }
  }
  __syncthreads();
  if (tid < nc && s_on[tid]) {
    const long long idx = (long long)k * P.m + c0 + tid;
    P.nrm[idx] = s_nrm[tid];
    P.ex[idx] = s_e[tid];   // kept even for an all-zero column so a pair's exponents agree
  }
}

cudaError_t launch_update_f64(const Problem& P, int i, int k_lo, int k_hi, cudaStream_t s) {
  if (k_hi <= k_lo) return cudaSuccess;
  const int nsub = P.tb / kUpdCols;
  dim3 grid((P.M - i) * nsub, k_hi - k_lo);
  k_update_f64<<<grid, 256, 0, s>>>(P, i, k_lo, 0, P.Y, P.ex, P.nrm);
  return cudaGetLastError();
}

cudaError_t launch_diag_residual_f64(const Problem& P, const double* Xsrc, const int* exX, const double* nrmX,
                                     cudaStream_t s) {
  if (P.M <= 0) return cudaSuccess;
  const int nsub = P.tb / kUpdCols;
  dim3 grid(P.M * nsub, P.M);
  k_update_f64<<<grid, 256, 0, s>>>(P, 0, 0, 1, Xsrc, exX, nrmX);
  return cudaGetLastError();
}

}  // namespace pevc

// post.cu -- post-processing task of Section 5.2: enforce one consistent
// scaling per eigenvector.  The tiles of a column carry different exponents
// (augmented tiles, Section 4); each column is consolidated to the exponent
// of its largest represented entry (an exact power-of-two rescaling, up to
// underflow of entries that are negligible against the largest), then
// normalised so its entry of largest modulus is exactly 1, and written to
// V_out with zeros below the eigenvector's block.
//
// After consolidation the largest entry has modulus in [1, 2) (the reference
// exponent is that of the largest represented magnitude), so the argmax works
// on squared moduli as integer keys and the normalisation multiplies by the
// reciprocal of the pivot computed once per column: one or two FP64
// operations per element instead of a division.
#include "common.cuh"

namespace pevc {

struct BestIdx {
  unsigned long long v;   // key of the squared modulus (non-negative doubles order like their bits)
  int i;
};

__device__ __forceinline__ BestIdx better(BestIdx a, BestIdx b) {
  if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
  return a;
}

// Column tile of output column q (cstart is non-decreasing).
__device__ __forceinline__ int col_tile(const Problem& P, int q) {
  int lo = 0, hi = P.M - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.cstart[mid] <= q) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(256) k_post(Problem P, double* __restrict__ V, int ldv,
                                              int32_t* __restrict__ scale, int normalise) {
  const int q = blockIdx.x;
  const int kd = P.kind[q];
  if (kd == 2) return;
  const bool pair = kd == 1;
  const int j = col_tile(P, q);
  const int lq = q - P.cstart[j];
  const int c0 = P.ccol[q];
  const int last = c0 + (pair ? 1 : 0);   // last row of the eigenvector's block
  const int m = P.m, tb = P.tb;
  const int tid = threadIdx.x;
  __shared__ int s_eref;
  __shared__ BestIdx s_red[8];
  __shared__ int s_ered[8];

  // 1. reference exponent: the largest represented magnitude over the tiles
  int eref = INT32_MIN;
  for (int k = tid; k <= j; k += blockDim.x) {
    const long long idx = (long long)k * m + q;
    const double nv = pair ? max_nonneg(P.nrm[idx], P.nrm[idx + 1]) : P.nrm[idx];
    if (abs_key(nv)) eref = max(eref, P.ex[idx] + ilogb_key(abs_key(nv)));
  }
  for (int o = 16; o > 0; o >>= 1) eref = max(eref, __shfl_xor_sync(0xffffffffu, eref, o));
  if ((tid & 31) == 0) s_ered[tid >> 5] = eref;
  __syncthreads();
  if (tid == 0) {
    int e = s_ered[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) e = max(e, s_ered[w]);
    s_eref = e;
  }
  __syncthreads();
  eref = s_eref;

  // 2. the entry of largest modulus (first index on ties)
  BestIdx best{0ull, 0x7fffffff};
  for (int k = 0; k <= j; ++k) {
    const long long idx = (long long)k * m + q;
    const double nv = pair ? max_nonneg(P.nrm[idx], P.nrm[idx + 1]) : P.nrm[idx];
    if (!abs_key(nv)) continue;
    const int sh = P.ex[idx] - eref;
    const int r0 = P.toff[k], h = min(P.toff[k + 1], last + 1) - r0;
    const double* Yt = tile_ptr(P, k, j);
    for (int r = tid; r < h; r += blockDim.x) {
      const double vr = pow2_scale(Yt[(size_t)lq * tb + r], sh);
      double mg2;
      if (pair) {
        const double vi = pow2_scale(Yt[(size_t)(lq + 1) * tb + r], sh);
        mg2 = fma(vr, vr, vi * vi);
      } else {
        mg2 = vr * vr;
      }
      best = better(best, BestIdx{abs_key(mg2), r0 + r});
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    BestIdx other{(unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)best.v, o),
                  __shfl_xor_sync(0xffffffffu, best.i, o)};
    best = better(best, other);
  }
  if ((tid & 31) == 0) s_red[tid >> 5] = best;
  __syncthreads();
  if (tid == 0) {
    BestIdx b = s_red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = better(b, s_red[w]);
    s_red[0] = b;
  }
  __syncthreads();
  best = s_red[0];
  const int istar = best.i;

  // value at istar (consolidated), and the normalising factors: 1 / d for
  // a real column, conj(d) / |d|^2 for a pair (|d| in [1, 2))
  double dr = 1.0, di = 0.0;
  if (best.v) {
    int k = 0;
    while (k < j && P.toff[k + 1] <= istar) ++k;
    const long long idx = (long long)k * m + q;
    const int sh = P.ex[idx] - eref;
    const double* Yt = tile_ptr(P, k, j);
    const int r = istar - P.toff[k];
    dr = pow2_scale(Yt[(size_t)lq * tb + r], sh);
    if (pair) di = pow2_scale(Yt[(size_t)(lq + 1) * tb + r], sh);
  }
  const double s2 = 1.0 / fma(dr, dr, di * di);
  const double nr = pair ? dr * s2 : 1.0 / dr, ni = di * s2;

  // 3. write the column(s)
  double* v0 = V + (size_t)q * ldv;
  double* v1 = pair ? V + (size_t)(q + 1) * ldv : nullptr;
  for (int k = 0; k <= j; ++k) {
    const long long idx = (long long)k * m + q;
    const double nv = pair ? max_nonneg(P.nrm[idx], P.nrm[idx + 1]) : P.nrm[idx];
    const bool nz = abs_key(nv) != 0;
    const int r0 = P.toff[k], h = min(P.toff[k + 1], last + 1) - r0;
    const int sh = nz ? P.ex[idx] - eref : 0;
    const double* Yt = tile_ptr(P, k, j);
    for (int r = tid; r < h; r += blockDim.x) {
      double vr = 0.0, vi = 0.0;
      if (nz) {
        vr = pow2_scale(Yt[(size_t)lq * tb + r], sh);
        if (pair) vi = pow2_scale(Yt[(size_t)(lq + 1) * tb + r], sh);
      }
      if (normalise && best.v) {
        if (pair) {
          const double zr = fma(vr, nr, vi * ni), zi = fma(vi, nr, -(vr * ni));
          vr = zr;
          vi = zi;
        } else {
          vr = vr * nr;
        }
        if (r0 + r == istar) { vr = 1.0; vi = 0.0; }
      }
      v0[r0 + r] = vr;
      if (pair) v1[r0 + r] = vi;
    }
  }
  for (int r = last + 1 + tid; r < P.n; r += blockDim.x) {
    v0[r] = 0.0;
    if (pair) v1[r] = 0.0;
  }
  if (tid == 0) {
    int32_t sc = eref;
    if (normalise && best.v) sc = eref + ilogb_key(abs_key(pair ? hypot(dr, di) : dr));
    scale[q] = sc;
    if (pair) scale[q + 1] = sc;
  }
}

cudaError_t launch_post(const Problem& P, double* V, int ldv, int32_t* scale, bool normalise,
                        cudaStream_t s) {
  if (P.m <= 0) return cudaSuccess;
  k_post<<<P.m, 256, 0, s>>>(P, V, ldv, scale, normalise ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace pevc

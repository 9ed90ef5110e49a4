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
// on integer keys (the magnitude bits of a real entry, of the squared modulus
// of a complex one) and the normalisation multiplies by the reciprocal of the
// pivot computed once per column: one FP64 operation per real element, three
// per complex one, instead of a division; the power-of-two consolidation is
// integer arithmetic.
#include "common.cuh"

namespace pevc {

struct BestIdx {
  unsigned long long v;   // magnitude key: bits of |v| (real) or of |v|^2 (complex); non-negative doubles order like their bits
  int i;
};

__device__ __forceinline__ BestIdx better(BestIdx a, BestIdx b) {
  if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
  return a;
}

// x * 2^e on the two 32-bit halves for a normal x with a normal result (and
// for e == 0); the library path otherwise (zero, subnormal, out of range).
// Only the exponent field is tested: a test of the whole magnitude against
// zero would be compiled into an FP64 comparison for every element.
__device__ __forceinline__ double scale2(double x, int e) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const int E = (hi >> 20) & 0x7ff;
  const int En = E + e;
  if (E != 0 && E != 0x7ff && En > 0 && En < 0x7ff) return __hiloint2double(hi + (e << 20), lo);
  if (e == 0) return x;
  return ldexp(x, e);
}

// Magnitude key of a double (its bit pattern without the sign), assembled
// from the two 32-bit halves.
__device__ __forceinline__ unsigned long long mag_key(double x) {
  return ((unsigned long long)((unsigned)__double2hiint(x) & 0x7fffffffu) << 32) | (unsigned)__double2loint(x);
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

constexpr int kPostTiles = 256;        // tiles of a column staged at once
constexpr int kNoTile = INT32_MIN;     // a tile whose column segment is all zero

// Per tile k in [kb, ke) of output column q: x = exponent shift to the
// reference exponent (kNoTile for an all-zero segment), y = first row, z =
// rows of the eigenvector's support in the tile.  Synchronises the CTA before
// and after.
__device__ __forceinline__ void stage_tiles(const Problem& P, int q, bool pair, int last, int eref, int kb, int ke,
                                            int4* s_tile) {
  __syncthreads();
  for (int k = kb + (int)threadIdx.x; k < ke; k += blockDim.x) {
    const long long idx = (long long)k * P.m + q;
    const double nv = pair ? max_nonneg(P.nrm[idx], P.nrm[idx + 1]) : P.nrm[idx];
    const int r0 = P.toff[k], h = min(P.toff[k + 1], last + 1) - r0;
    s_tile[k - kb] = make_int4(abs_key(nv) ? P.ex[idx] - eref : kNoTile, r0, max(h, 0), 0);
  }
  __syncthreads();
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
  __shared__ int4 s_tile[kPostTiles];

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

  // 2. the entry of largest modulus (first index on ties), and 3. the
  //    written column(s).  Both passes run over the flattened (tile, row)
  //    index space of the column in chunks of kPostTiles tiles, with the
  //    per-tile shift and row range staged in shared memory, and four rows
  //    per thread in flight.
  BestIdx best{0ull, 0x7fffffff};
  for (int kb = 0; kb <= j; kb += kPostTiles) {
    const int ke = min(j + 1, kb + kPostTiles);
    stage_tiles(P, q, pair, last, eref, kb, ke, s_tile);
    const int nflat = (ke - kb) * tb;
    for (int f0 = tid; f0 < nflat; f0 += 4 * (int)blockDim.x) {
      double vr[4], vi[4];
      int row[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int f = f0 + u * (int)blockDim.x;
        row[u] = -1;
        vr[u] = vi[u] = 0.0;
        if (f < nflat) {
          const int kk = f / tb, r = f - kk * tb;
          const int4 ti = s_tile[kk];
          if (r < ti.z && ti.x != kNoTile) {
            const double* Yt = tile_ptr(P, kb + kk, j);
            vr[u] = Yt[(size_t)lq * tb + r];
            if (pair) vi[u] = Yt[(size_t)(lq + 1) * tb + r];
            row[u] = ti.y + r;
            vr[u] = scale2(vr[u], ti.x);
            if (pair) vi[u] = scale2(vi[u], ti.x);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (row[u] < 0) continue;
        // real columns compare |v| by its magnitude bits; pairs the squared modulus
        const unsigned long long key = pair ? mag_key(fma(vr[u], vr[u], vi[u] * vi[u])) : mag_key(vr[u]);
        best = better(best, BestIdx{key, row[u]});
      }
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
  const bool norm = normalise && best.v;

  double* v0 = V + (size_t)q * ldv;
  double* v1 = pair ? V + (size_t)(q + 1) * ldv : nullptr;
  for (int kb = 0; kb <= j; kb += kPostTiles) {
    const int ke = min(j + 1, kb + kPostTiles);
    stage_tiles(P, q, pair, last, eref, kb, ke, s_tile);
    const int nflat = (ke - kb) * tb;
    for (int f0 = tid; f0 < nflat; f0 += 4 * (int)blockDim.x) {
      double vr[4], vi[4];
      int row[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int f = f0 + u * (int)blockDim.x;
        row[u] = -1;
        vr[u] = vi[u] = 0.0;
        if (f < nflat) {
          const int kk = f / tb, r = f - kk * tb;
          const int4 ti = s_tile[kk];
          if (r < ti.z) {
            row[u] = ti.y + r;
            if (ti.x != kNoTile) {
              const double* Yt = tile_ptr(P, kb + kk, j);
              vr[u] = scale2(Yt[(size_t)lq * tb + r], ti.x);
              if (pair) vi[u] = scale2(Yt[(size_t)(lq + 1) * tb + r], ti.x);
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (row[u] < 0) continue;
        double xr = vr[u], xi = vi[u];
        if (norm) {
          if (pair) {
            const double zr = fma(xr, nr, xi * ni), zi = fma(xi, nr, -(xr * ni));
            xr = zr;
            xi = zi;
          } else {
            xr = xr * nr;
          }
          if (row[u] == istar) { xr = 1.0; xi = 0.0; }
        }
        v0[row[u]] = xr;
        if (pair) v1[row[u]] = xi;
      }
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

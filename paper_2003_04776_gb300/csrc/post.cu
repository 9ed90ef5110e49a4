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
  int i;                  // row
  int k;                  // its row tile
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

// One CTA per output column (a pair's two columns together).  The column's
// tiles are staged kPostTiles at a time (shift to the reference exponent,
// first row, rows of the eigenvector's support, and whether the tile can
// hold the entry of largest modulus); warps take tiles in turn and lanes
// the rows of a tile, so every load and store is a contiguous run.  Y is
// read once for the written column plus once for the few candidate tiles of
// the argmax: the largest represented magnitude of the column is at least
// 2^eref, so a tile whose own largest magnitude is below 2^(eref - 1) (times
// sqrt 2 for the modulus of a pair) cannot hold it.
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
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (int)(blockDim.x >> 5);
  __shared__ int s_eref;
  __shared__ BestIdx s_red[8];
  __shared__ int s_ered[8];
  __shared__ int4 s_tile[kPostTiles];     // shift (kNoTile: all zero), first row, rows, candidate

  // 1. reference exponent: the largest represented magnitude over the tiles
  int eref = INT32_MIN;
  for (int k = tid; k <= j; k += blockDim.x) {
    const long long idx = (long long)k * m + q;
    const double nv = pair ? max_nonneg(P.nrm[idx], P.nrm[idx + 1]) : P.nrm[idx];
    if (abs_key(nv)) eref = max(eref, P.ex[idx] + ilogb_key(abs_key(nv)));
  }
  for (int o = 16; o > 0; o >>= 1) eref = max(eref, __shfl_xor_sync(0xffffffffu, eref, o));
  if (lane == 0) s_ered[warp] = eref;
  __syncthreads();
  if (tid == 0) {
    int e = s_ered[0];
    for (int w = 1; w < nw; ++w) e = max(e, s_ered[w]);
    s_eref = e;
  }
  __syncthreads();
  eref = s_eref;

  auto stage = [&](int kb, int ke) {
    __syncthreads();
    for (int k = kb + tid; k < ke; k += blockDim.x) {
      const long long idx = (long long)k * m + q;
      const double nv = pair ? max_nonneg(P.nrm[idx], P.nrm[idx + 1]) : P.nrm[idx];
      const int r0 = P.toff[k], h = min(P.toff[k + 1], last + 1) - r0;
      const bool nz = abs_key(nv) != 0;
      const int top = nz ? P.ex[idx] + ilogb_key(abs_key(nv)) : INT32_MIN;
      s_tile[k - kb] = make_int4(nz ? P.ex[idx] - eref : kNoTile, r0, max(h, 0), top >= eref - 1 ? 1 : 0);
    }
    __syncthreads();
  };

  // 2. the entry of largest modulus (first index on ties), over the
  //    candidate tiles
  BestIdx best{0ull, 0x7fffffff, 0};
  for (int kb = 0; kb <= j; kb += kPostTiles) {
    const int ke = min(j + 1, kb + kPostTiles);
    stage(kb, ke);
    for (int kk = warp; kk < ke - kb; kk += nw) {
      const int4 ti = s_tile[kk];
      if (!ti.w) continue;
      const double* Yt = tile_ptr(P, kb + kk, j);
      for (int r = lane; r < ti.z; r += 32) {
        const double vr = scale2(Yt[(size_t)lq * tb + r], ti.x);
        const double vi = pair ? scale2(Yt[(size_t)(lq + 1) * tb + r], ti.x) : 0.0;
        // real columns compare |v| by its magnitude bits; pairs the squared modulus
        const unsigned long long key = pair ? mag_key(fma(vr, vr, vi * vi)) : mag_key(vr);
        best = better(best, BestIdx{key, ti.y + r, kb + kk});
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    BestIdx other{(unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)best.v, o),
                  __shfl_xor_sync(0xffffffffu, best.i, o), __shfl_xor_sync(0xffffffffu, best.k, o)};
    best = better(best, other);
  }
  if (lane == 0) s_red[warp] = best;
  __syncthreads();
  if (tid == 0) {
    BestIdx b = s_red[0];
    for (int w = 1; w < nw; ++w) b = better(b, s_red[w]);
    s_red[0] = b;
  }
  __syncthreads();
  best = s_red[0];
  const int istar = best.i;

  // value at istar (consolidated), and the normalising factors: 1 / d for
  // a real column, conj(d) / |d|^2 for a pair (|d| in [1, 2))
  double dr = 1.0, di = 0.0;
  if (best.v) {
    const int k = best.k;
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

  // 3. the written column(s)
  double* v0 = V + (size_t)q * ldv;
  double* v1 = pair ? V + (size_t)(q + 1) * ldv : nullptr;
  for (int kb = 0; kb <= j; kb += kPostTiles) {
    const int ke = min(j + 1, kb + kPostTiles);
    if (kb > 0) stage(kb, ke);
    for (int kk = warp; kk < ke - kb; kk += nw) {
      const int4 ti = s_tile[kk];
      const double* Yt = tile_ptr(P, kb + kk, j);
      for (int r = lane; r < ti.z; r += 32) {
        double xr = 0.0, xi = 0.0;
        if (ti.x != kNoTile) {
          xr = scale2(Yt[(size_t)lq * tb + r], ti.x);
          if (pair) xi = scale2(Yt[(size_t)(lq + 1) * tb + r], ti.x);
        }
        const int row = ti.y + r;
        if (norm) {
          if (pair) {
            const double zr = fma(xr, nr, xi * ni), zi = fma(xi, nr, -(xr * ni));
            xr = zr;
            xi = zi;
          } else {
            xr = xr * nr;
          }
          if (row == istar) { xr = 1.0; xi = 0.0; }
        }
        v0[row] = xr;
        if (pair) v1[row] = xi;
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

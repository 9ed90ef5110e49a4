// cplx.cu -- eigenvectors of a complex pencil in generalized Schur form, the
// extension to complex data types of Section 7.  S and T are upper triangular
// with complex entries; every diagonal entry c gives the eigenvalue (alpha_c,
// beta_c) = (S_cc, T_cc) and the eigenvector x with x_c = 1, x_i = 0 below c and
// (beta S - alpha T) x = 0.  There are no 2x2 blocks, so the robust blocked
// backward substitution of Section 3 (Algorithm 1) runs with 1x1 steps only,
// in complex FP64 arithmetic:
//
//   init     the right-hand sides Y[0:c, c] = -(beta S - alpha T)[0:c, c] and
//            the unit tips, written straight into the output columns;
//   stage i  (bottom-up over the tile rows) the diagonal solve of tile i for
//            every column whose tip is in tile i or below (kernel 3; the tip
//            tile itself is kernel 1), then the left update
//                Y_kj <- Y_kj - (beta S_ki - alpha T_ki) X_ij    for k < i
//            (kernel 2) as one complex GEMM per tile pair,
//                Y_kj <- Y_kj - S_ki (beta X_ij) + T_ki (alpha X_ij);
//   post     consolidation of every column to one power of two and
//            normalisation.
//
// Every tile segment of a column carries its own power-of-two exponent (the
// augmented tiles of Section 4).  Divisions are guarded by ProtectDivision,
// the in-tile and left updates by ProtectUpdate, and before a left update the
// two segments are consolidated to the larger exponent and the right update
// [beta X; alpha X] is kept below Omega (Algorithms 2 and 3).  Magnitudes are
// |re| + |im|, which is submultiplicative for complex products, so the real
// bounds carry over.  The left update needs the infinity norms (maximum row
// sums of magnitudes) of every tile of S and T above the diagonal.
//
// FP64 FMA and the FP64 tensor path run at about the same rate on this GPU,
// so the update is a register-tiled SIMT complex GEMM in FP64.
#include <algorithm>

#include "common.cuh"
#include "cplx.cuh"

namespace pevc {

namespace {

constexpr int kCxTile = 64;              // tile order
constexpr int kCxTri = kCxTile * (kCxTile + 1) / 2;
constexpr int kCxNone = -(1 << 28);      // exponent bound of a zero magnitude
constexpr int kCxUpdCols = 32;           // columns per update CTA
constexpr int kCxUpdK = 8;               // K chunk of the update
constexpr int kCxDiagWarps = 8;          // columns per diagonal-solve CTA

__device__ __forceinline__ double2 ld2(const double* p) {
  return *reinterpret_cast<const double2*>(p);
}
__device__ __forceinline__ void st2(double* p, double2 v) { *reinterpret_cast<double2*>(p) = v; }

// m = beta s - alpha t
__device__ __forceinline__ double2 pencil_entry(double2 be, double2 al, double2 s, double2 t) {
  double2 m;
  m.x = (be.x * s.x - be.y * s.y) - (al.x * t.x - al.y * t.y);
  m.y = (be.x * s.y + be.y * s.x) - (al.x * t.y + al.y * t.x);
  return m;
}

// Smallest E with v < 2^E for v >= 0 (kCxNone for v = 0).
__device__ __forceinline__ int eab(double v) {
  const unsigned long long k = abs_key(v);
  return k ? ilogb_key(k) + 1 : kCxNone;
}

// An exponent bound of |re| + |im| from the two parts' exponent fields
// (integer instructions only): |re| + |im| <= 2 max(|re|, |im|).
__device__ __forceinline__ int cexp_ub(double2 z) { return max(exp_ub(z.x), exp_ub(z.y)) + 1; }

__device__ __forceinline__ double2 cscale(double2 z, int e) {
  return make_double2(pow2_scale(z.x, e), pow2_scale(z.y, e));
}

__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long k) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, k, o);
    k = v > k ? v : k;
  }
  return k;
}

// ---------------------------------------------------------------------------
// Pre-pass.
// ---------------------------------------------------------------------------

// Largest magnitude over the upper triangles of S and T (one CTA per column);
// an Inf or NaN sets kStNonfinite.
__global__ void __launch_bounds__(256) k_cx_scan(const double* __restrict__ S, int lds,
                                                 const double* __restrict__ T, int ldt, int n,
                                                 double* __restrict__ gmax, unsigned* __restrict__ status) {
  const int j = blockIdx.x;
  unsigned long long key = 0;
  bool bad = false;
  for (int r = threadIdx.x; r <= j; r += blockDim.x) {
    const double2 s = ld2(S + 2 * ((size_t)j * lds + r));
    const double2 t = ld2(T + 2 * ((size_t)j * ldt + r));
    const double ms = cmag(s.x, s.y), mt = cmag(t.x, t.y);
    if (!isfinite(ms) || !isfinite(mt)) {
      bad = true;
      continue;
    }
    const unsigned long long a = abs_key(ms), b = abs_key(mt);
    key = max(key, max(a, b));
  }
  key = warp_max_key(key);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStNonfinite);
  if ((threadIdx.x & 31) == 0 && key) atomicMax(reinterpret_cast<unsigned long long*>(gmax), key);
}

// (alpha, beta) of every selected column, pre-scaled by 2^-sigma so that
// max(|beta|, |alpha|) * max|S, T| <= 2^1000 (the eigenvector is unchanged).
__global__ void k_cx_eig(const double* __restrict__ S, int lds, const double* __restrict__ T, int ldt,
                         const int* __restrict__ ccol, int m, const double* __restrict__ gmax,
                         double* __restrict__ alpha, double* __restrict__ beta, unsigned* __restrict__ status) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m) return;
  const int c = ccol[q];
  const double2 a = ld2(S + 2 * ((size_t)c * lds + c));
  const double2 b = ld2(T + 2 * ((size_t)c * ldt + c));
  const double coef = max_nonneg(cmag(a.x, a.y), cmag(b.x, b.y));
  const double mx = *gmax;
  int sg = 0;
  if (abs_key(coef) && abs_key(mx)) sg = max(0, eab(coef) + eab(mx) - kPrescaleExp);
  if (!abs_key(coef)) atomicOr(status, kStIndefinite);
  st2(alpha + 2 * q, cscale(a, -sg));
  st2(beta + 2 * q, cscale(b, -sg));
}

// Infinity norms (maximum row sums of |re| + |im|) of the tiles (k, i), k < i,
// of S and T: one CTA of kCxTile threads per tile, a thread per row.
__global__ void __launch_bounds__(kCxTile) k_cx_tilenorms(const double* __restrict__ S, int lds,
                                                         const double* __restrict__ T, int ldt, int n, int ldm,
                                                         double* __restrict__ tnS, double* __restrict__ tnT) {
  const int i = blockIdx.x, k = blockIdx.y;
  if (k >= i) return;
  __shared__ unsigned long long s_max[2];
  if (threadIdx.x < 2) s_max[threadIdx.x] = 0;
  __syncthreads();
  const int r = k * kCxTile + threadIdx.x;           // tile k < i is a full tile
  const int c0 = i * kCxTile, c1 = min(n, c0 + kCxTile);
  double rs = 0.0, rt = 0.0;
  for (int c = c0; c < c1; ++c) {
    const double2 s = ld2(S + 2 * ((size_t)c * lds + r));
    const double2 t = ld2(T + 2 * ((size_t)c * ldt + r));
    rs += cmag(s.x, s.y);
    rt += cmag(t.x, t.y);
  }
  const unsigned long long ks = warp_max_key(abs_key(rs)), kt = warp_max_key(abs_key(rt));
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&s_max[0], ks);
    atomicMax(&s_max[1], kt);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    tnS[(size_t)k * ldm + i] = __longlong_as_double((long long)s_max[0]);
    tnT[(size_t)k * ldm + i] = __longlong_as_double((long long)s_max[1]);
  }
}

// Right-hand sides and unit tips of every selected column, with exponent 0
// and the magnitude maximum of every tile segment (one CTA per column, a warp
// per tile segment).  Only the tip's own tile gets the tip's column,
// -(beta S - alpha T)[r, c] for rows r < c there (kernel 1 solves the diagonal
// tile alone); the tiles above start from zero and receive the tip's
// contribution, with the rest of the tile's solution, through the left
// update of the tip's stage.  Rows of the tip's tile below the tip are zero.
__global__ void __launch_bounds__(256) k_cx_init(const double* __restrict__ S, int lds,
                                                 const double* __restrict__ T, int ldt, int n,
                                                 const int* __restrict__ ccol, const double* __restrict__ alpha,
                                                 const double* __restrict__ beta, double* __restrict__ V, int ldv,
                                                 int* __restrict__ ex, double* __restrict__ nrm, int lde) {
  const int q = blockIdx.x;
  const int c = ccol[q];
  const int jt = c / kCxTile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double2 al = ld2(alpha + 2 * q), be = ld2(beta + 2 * q);
  double* v = V + 2 * (size_t)q * ldv;
  for (int k = warp; k <= jt; k += 8) {
    const int r0 = k * kCxTile, r1 = min(n, r0 + kCxTile);
    unsigned long long key = 0;
    for (int r = r0 + lane; r < r1; r += 32) {
      double2 y;
      if (k < jt) {
        y = make_double2(0.0, 0.0);
      } else if (r < c) {
        const double2 mm = pencil_entry(be, al, ld2(S + 2 * ((size_t)c * lds + r)), ld2(T + 2 * ((size_t)c * ldt + r)));
        y = make_double2(-mm.x, -mm.y);
      } else {
        y = make_double2(r == c ? 1.0 : 0.0, 0.0);
      }
      st2(v + 2 * r, y);
      key = max(key, abs_key(cmag(y.x, y.y)));
    }
    key = warp_max_key(key);
    if (lane == 0) {
      ex[(size_t)k * lde + q] = 0;
      nrm[(size_t)k * lde + q] = __longlong_as_double((long long)key);
    }
  }
}

// ---------------------------------------------------------------------------
// Kernel 1/3: diagonal-tile solves of stage i, one warp per column.
// ---------------------------------------------------------------------------

// Column r of the packed upper triangle starts at r (r + 1) / 2.
__device__ __forceinline__ int tri_off(int r) { return (r * (r + 1)) >> 1; }

__global__ void __launch_bounds__(32 * kCxDiagWarps) k_cx_diag(
    int i, const double* __restrict__ S, int lds, const double* __restrict__ T, int ldt, int n,
    const int* __restrict__ ccol, int q0, int m, const double* __restrict__ alpha,
    const double* __restrict__ beta, double* __restrict__ V, int ldv, int* __restrict__ ex,
    double* __restrict__ nrm, int lde) {
  extern __shared__ double2 s_dyn[];
  double2* s_S = s_dyn;                    // packed upper triangle of S_ii
  double2* s_T = s_dyn + kCxTri;           // and of T_ii
  __shared__ double s_cS[kCxTile], s_cT[kCxTile];   // max |entry| above the diagonal, per column

  const int ri0 = i * kCxTile;
  const int hi = min(kCxTile, n - ri0);
  for (int e = threadIdx.x; e < kCxTri; e += blockDim.x) {
    // column r, row l of the packed triangle
    int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (tri_off(r) > e) --r;
    while (tri_off(r + 1) <= e) ++r;
    const int l = e - tri_off(r);
    double2 s = make_double2(0.0, 0.0), t = make_double2(0.0, 0.0);
    if (r < hi) {
      s = ld2(S + 2 * ((size_t)(ri0 + r) * lds + ri0 + l));
      t = ld2(T + 2 * ((size_t)(ri0 + r) * ldt + ri0 + l));
    }
    s_S[e] = s;
    s_T[e] = t;
  }
  __syncthreads();
  if (threadIdx.x < kCxTile) {
    const int r = threadIdx.x;
    unsigned long long ks = 0, kt = 0;
    for (int l = 0; l < r; ++l) {
      const double2 s = s_S[tri_off(r) + l], t = s_T[tri_off(r) + l];
      ks = max(ks, abs_key(cmag(s.x, s.y)));
      kt = max(kt, abs_key(cmag(t.x, t.y)));
    }
    s_cS[r] = __longlong_as_double((long long)ks);
    s_cT[r] = __longlong_as_double((long long)kt);
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = q0 + blockIdx.x * kCxDiagWarps + warp;
  if (q >= m) return;                      // warp-uniform; no block barrier follows
  const int c = ccol[q];
  const int top = (c < ri0 + hi) ? c - ri0 - 1 : hi - 1;   // last row to solve (the tip's tile stops above it)
  const double2 al = ld2(alpha + 2 * q), be = ld2(beta + 2 * q);
  const double mal = cmag(al.x, al.y), mbe = cmag(be.x, be.y);

  // Per-row pivot reciprocals and update bounds, lane-parallel: rows lane and
  // lane + 32.  Pivots below smin = max(u (|beta||S_ll| + |alpha||T_ll|),
  // DBL_MIN) are raised to smin (the perturbation of Section 5.2).
  double2 rp[2];
  int erp[2], et[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int l = lane + 32 * h;
    rp[h] = make_double2(0.0, 0.0);
    erp[h] = kCxNone;
    et[h] = kCxNone;
    if (l < hi) {
      const double2 s = s_S[tri_off(l) + l], t = s_T[tri_off(l) + l];
      double2 piv = pencil_entry(be, al, s, t);
      const double smin = fmax(0x1p-53 * (mbe * cmag(s.x, s.y) + mal * cmag(t.x, t.y)), 0x1p-1022);   // DBL_MIN
      if (cmag(piv.x, piv.y) < smin) piv = make_double2(smin, 0.0);
      crecip(piv.x, piv.y, rp[h].x, rp[h].y);
      erp[h] = cexp_ub(rp[h]);
      et[h] = eab(mbe * s_cS[l] + mal * s_cT[l]);
    }
  }

  double* v = V + 2 * ((size_t)q * ldv + ri0);
  double2 y[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int l = lane + 32 * h;
    y[h] = (l < hi) ? ld2(v + 2 * l) : make_double2(0.0, 0.0);
  }
  int e = ex[(size_t)i * lde + q];

  for (int r = top; r >= 0; --r) {
    const int h = r >> 5, src = r & 31;
    double2 yr;
    yr.x = __shfl_sync(0xffffffffu, h ? y[1].x : y[0].x, src);
    yr.y = __shfl_sync(0xffffffffu, h ? y[1].y : y[0].y, src);
    double2 rr;
    rr.x = __shfl_sync(0xffffffffu, h ? rp[1].x : rp[0].x, src);
    rr.y = __shfl_sync(0xffffffffu, h ? rp[1].y : rp[0].y, src);
    const int er = __shfl_sync(0xffffffffu, h ? erp[1] : erp[0], src);
    const int etr = __shfl_sync(0xffffffffu, h ? et[1] : et[0], src);
    // ProtectDivision: |y_r / p_r| <= |y_r| |1/p_r| < 2^(ey + er) must stay below Omega
    const int kd = cexp_ub(yr) + er + 1 - kOmegaExp;
    if (kd > 0) {                          // uniform: every lane holds y_r
      y[0] = cscale(y[0], -kd);
      y[1] = cscale(y[1], -kd);
      yr = cscale(yr, -kd);
      e += kd;
    }
    double2 x;
    cmul(yr.x, yr.y, rr.x, rr.y, x.x, x.y);
    if (r > 0) {
      // ProtectUpdate(max |y_l| over l < r, |beta| cS_r + |alpha| cT_r, |x_r|)
      int eyl = kCxNone;
      if (lane < r) eyl = cexp_ub(y[0]);
      if (lane + 32 < r) eyl = max(eyl, cexp_ub(y[1]));
      eyl = __reduce_max_sync(0xffffffffu, eyl);
      const int etx = (etr == kCxNone) ? kCxNone : etr + cexp_ub(x);
      const int ku = max(eyl, etx) + 1 - kOmegaExp;
      if (ku > 0) {
        y[0] = cscale(y[0], -ku);
        y[1] = cscale(y[1], -ku);
        x = cscale(x, -ku);
        e += ku;
      }
    }
    if (lane == src) {                     // explicit halves: no dynamic register index
      if (h) y[1] = x;
      else y[0] = x;
    }
    if (r > 0) {
      const int base = tri_off(r);
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int l = lane + 32 * hh;
        if (l < r) {
          const double2 mm = pencil_entry(be, al, s_S[base + l], s_T[base + l]);
          y[hh].x -= mm.x * x.x - mm.y * x.y;
          y[hh].y -= mm.x * x.y + mm.y * x.x;
        }
      }
    }
  }

  unsigned long long key = 0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int l = lane + 32 * h;
    if (l < hi) {
      st2(v + 2 * l, y[h]);
      key = max(key, abs_key(cmag(y[h].x, y[h].y)));
    }
  }
  key = warp_max_key(key);
  if (lane == 0) {
    ex[(size_t)i * lde + q] = e;
    nrm[(size_t)i * lde + q] = __longlong_as_double((long long)key);
  }
}

// ---------------------------------------------------------------------------
// Kernel 2: left updates of stage i, one CTA per (tile k < i, 32 columns).
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_cx_update(
    int i, const double* __restrict__ S, int lds, const double* __restrict__ T, int ldt, int n, int q0, int m,
    const double* __restrict__ alpha, const double* __restrict__ beta, double* __restrict__ V, int ldv,
    int* __restrict__ ex, double* __restrict__ nrm, int lde, const double* __restrict__ tnS,
    const double* __restrict__ tnT, int ldm) {
  const int k = blockIdx.y;
  const int qb = q0 + blockIdx.x * kCxUpdCols;
  const int ri0 = i * kCxTile, hi = min(kCxTile, n - ri0);
  const int rk0 = k * kCxTile;             // tile k < i is full
  const int tid = threadIdx.x;

  __shared__ double2 sA[2][kCxUpdK][kCxTile];       // S_ki, T_ki chunk
  __shared__ double2 sB[2][kCxUpdK][kCxUpdCols];    // beta X'', alpha X''
  __shared__ int s_fY[kCxUpdCols], s_fX[kCxUpdCols], s_on[kCxUpdCols];
  __shared__ double2 s_al[kCxUpdCols], s_be[kCxUpdCols];
  __shared__ unsigned long long s_max[kCxUpdCols];

  if (tid < kCxUpdCols) {
    const int q = qb + tid;
    int on = 0, fY = 0, fX = 0, enew = 0;
    if (q < m) {
      const int eY = ex[(size_t)k * lde + q], eX = ex[(size_t)i * lde + q];
      const double nY = nrm[(size_t)k * lde + q], nX = nrm[(size_t)i * lde + q];
      if (abs_key(nX)) {
        on = 1;
        const bool yz = !abs_key(nY);
        const int E = yz ? eX : max(eY, eX);
        const double2 al = ld2(alpha + 2 * q), be = ld2(beta + 2 * q);
        // right update [beta X; alpha X] below Omega: 2^-kr max(|beta|, |alpha|) |X| <= Omega
        const int ea = eab(max_nonneg(cmag(al.x, al.y), cmag(be.x, be.y)));
        const int exn = eab(nX) + eX - E;
        const int kr = max(0, ea + exn + 1 - kOmegaExp);
        const int ex2 = ea + exn - kr;
        // ProtectUpdate(|Y|, ||[S_ki T_ki]||_inf, |X''|), all on exponent bounds
        const double tS = tnS[(size_t)k * ldm + i], tT = tnT[(size_t)k * ldm + i];
        const int et = eab(tS + tT);
        const int eyn = yz ? kCxNone : eab(nY) + eY - E - kr;
        const int top = max(eyn, et == kCxNone ? kCxNone : et + ex2);
        const int kp = max(0, top + 1 - kOmegaExp);
        fY = eY - E - kr - kp;
        fX = eX - E - kr - kp;
        enew = E + kr + kp;
        s_al[tid] = al;
        s_be[tid] = be;
      }
    }
    s_on[tid] = on;
    s_fY[tid] = fY;
    s_fX[tid] = fX;
    s_max[tid] = 0;
    if (on) ex[(size_t)k * lde + q] = enew;   // read above by this thread only
  }
  __syncthreads();

  const int tx = tid & 7, ty = tid >> 3;    // columns tx + 8 u, rows ty and ty + 32
  double2 acc[2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[a][u] = make_double2(0.0, 0.0);

  for (int kk0 = 0; kk0 < hi; kk0 += kCxUpdK) {
    // A chunk: kCxUpdK columns of S_ki and T_ki (64 rows each)
    for (int e = tid; e < 2 * kCxUpdK * kCxTile; e += 256) {
      const int which = e / (kCxUpdK * kCxTile);
      const int rem = e % (kCxUpdK * kCxTile);
      const int kc = rem / kCxTile, row = rem % kCxTile;
      const int col = ri0 + kk0 + kc;
      double2 a = make_double2(0.0, 0.0);
      if (kk0 + kc < hi) a = ld2((which ? T : S) + 2 * ((size_t)col * (which ? ldt : lds) + rk0 + row));
      sA[which][kc][row] = a;
    }
    // B chunk: X'' = 2^fX X scaled by beta and by alpha
    {
      const int kc = tid / kCxUpdCols, j = tid % kCxUpdCols;   // 8 x 32 = 256 elements
      const int q = qb + j;
      double2 b1 = make_double2(0.0, 0.0), b2 = b1;
      if (s_on[j] && kk0 + kc < hi) {
        const double2 x = cscale(ld2(V + 2 * ((size_t)q * ldv + ri0 + kk0 + kc)), s_fX[j]);
        const double2 be = s_be[j], al = s_al[j];
        cmul(be.x, be.y, x.x, x.y, b1.x, b1.y);
        cmul(al.x, al.y, x.x, x.y, b2.x, b2.y);
      }
      sB[0][kc][j] = b1;
      sB[1][kc][j] = b2;
    }
    __syncthreads();
#pragma unroll
    for (int kc = 0; kc < kCxUpdK; ++kc) {
      double2 as[2], at[2], b1[4], b2[4];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        as[a] = sA[0][kc][ty + 32 * a];
        at[a] = sA[1][kc][ty + 32 * a];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        b1[u] = sB[0][kc][tx + 8 * u];
        b2[u] = sB[1][kc][tx + 8 * u];
      }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          // acc += S b1 - T b2
          acc[a][u].x = fma(as[a].x, b1[u].x, acc[a][u].x);
          acc[a][u].x = fma(-as[a].y, b1[u].y, acc[a][u].x);
          acc[a][u].y = fma(as[a].x, b1[u].y, acc[a][u].y);
          acc[a][u].y = fma(as[a].y, b1[u].x, acc[a][u].y);
          acc[a][u].x = fma(-at[a].x, b2[u].x, acc[a][u].x);
          acc[a][u].x = fma(at[a].y, b2[u].y, acc[a][u].x);
          acc[a][u].y = fma(-at[a].x, b2[u].y, acc[a][u].y);
          acc[a][u].y = fma(-at[a].y, b2[u].x, acc[a][u].y);
        }
    }
    __syncthreads();
  }

  // Epilogue: Y <- 2^fY Y - acc, and the new segment maxima.
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int j = tx + 8 * u;
    if (!s_on[j]) continue;
    const int q = qb + j;
    unsigned long long key = 0;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      double* p = V + 2 * ((size_t)q * ldv + rk0 + ty + 32 * a);
      const double2 yv = cscale(ld2(p), s_fY[j]);
      const double2 nv = make_double2(yv.x - acc[a][u].x, yv.y - acc[a][u].y);
      st2(p, nv);
      key = max(key, abs_key(cmag(nv.x, nv.y)));
    }
    atomicMax(&s_max[j], key);
  }
  __syncthreads();
  if (tid < kCxUpdCols && s_on[tid])
    nrm[(size_t)k * lde + qb + tid] = __longlong_as_double((long long)s_max[tid]);
}

// ---------------------------------------------------------------------------
// Post-pass: one power of two per column, then normalisation.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_cx_post(int n, const int* __restrict__ ccol, double* __restrict__ V, int ldv,
                                                 const int* __restrict__ ex, const double* __restrict__ nrm, int lde,
                                                 int32_t* __restrict__ scale, int normalise) {
  const int q = blockIdx.x;
  const int c = ccol[q];
  const int jt = c / kCxTile;
  const int tid = threadIdx.x;
  __shared__ int s_E;
  __shared__ double s_best[256];
  __shared__ int s_idx[256];
  if (tid == 0) {
    int E = INT32_MIN;
    for (int k = 0; k <= jt; ++k)
      if (abs_key(nrm[(size_t)k * lde + q])) E = max(E, ex[(size_t)k * lde + q]);
    s_E = (E == INT32_MIN) ? 0 : E;
  }
  __syncthreads();
  const int E = s_E;
  double* v = V + 2 * (size_t)q * ldv;
  double best = -1.0;
  int bidx = 0;
  for (int r = tid; r <= c; r += 256) {
    const int k = r / kCxTile;
    const double2 z = cscale(ld2(v + 2 * r), ex[(size_t)k * lde + q] - E);
    st2(v + 2 * r, z);
    const double mz = hypot(z.x, z.y);
    if (mz > best) {                       // rows visited in increasing order: first index wins
      best = mz;
      bidx = r;
    }
  }
  s_best[tid] = best;
  s_idx[tid] = bidx;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o) {
      const double b2 = s_best[tid + o];
      const int i2 = s_idx[tid + o];
      if (b2 > s_best[tid] || (b2 == s_best[tid] && i2 < s_idx[tid])) {
        s_best[tid] = b2;
        s_idx[tid] = i2;
      }
    }
    __syncthreads();
  }
  const int istar = s_idx[0];
  const double bmax = s_best[0];
  if (normalise && bmax > 0.0) {
    const double2 d = ld2(v + 2 * istar);   // written above by this block; visible after the barriers
    __syncthreads();                         // every thread has read d before it is overwritten
    for (int r = tid; r <= c; r += 256) {
      double2 z = ld2(v + 2 * r);
      double2 o;
      if (r == istar) {
        o = make_double2(1.0, 0.0);
      } else {
        cdiv(z.x, z.y, d.x, d.y, o.x, o.y);
      }
      st2(v + 2 * r, o);
    }
    if (tid == 0) scale[q] = E + ilogb(bmax);
  } else if (tid == 0) {
    scale[q] = E;
  }
  for (int r = c + 1 + tid; r < n; r += 256) st2(v + 2 * r, make_double2(0.0, 0.0));
}

// ---------------------------------------------------------------------------
// Left eigenvectors: u^H (beta S - alpha T) = 0 is (beta S - alpha T)^H u = 0,
// and with J the reversal permutation J (beta S - alpha T)^H J = conj(beta) S'
// - conj(alpha) T' for the upper triangular (S', T') = (J S^H J, J T^H J), whose
// diagonal entry n-1-c is (conj(alpha_c), conj(beta_c)).  So J u is the right
// eigenvector of (S', T') at entry n-1-c.
// ---------------------------------------------------------------------------

// B(i, j) = conj(A(n-1-j, n-1-i)), B column-major with leading dimension n:
// 32 x 32 tiles through shared memory, coalesced on both sides.
__global__ void __launch_bounds__(256) k_cx_flip_ct(const double* __restrict__ A, int lda, int n,
                                                    double* __restrict__ B) {
  __shared__ double2 tile[32][33];
  const int bi = blockIdx.x, bj = blockIdx.y, tx = threadIdx.x, ty = threadIdx.y;
  const int rbase = n - 32 * bj - 32;    // rows of A feeding B's columns 32 bj .. 32 bj + 31
  const int cbase = n - 32 * bi - 32;    // columns of A feeding B's rows 32 bi .. 32 bi + 31
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = rbase + tx, c = cbase + ty + 8 * k;
    if (r >= 0 && c >= 0) tile[ty + 8 * k][tx] = ld2(A + 2 * ((size_t)c * lda + r));
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = 32 * bi + tx, j = 32 * bj + ty + 8 * k;
    if (i < n && j < n) {
      const double2 z = tile[31 - tx][31 - ty - 8 * k];
      st2(B + 2 * ((size_t)j * n + i), make_double2(z.x, -z.y));
    }
  }
}

__global__ void k_cx_flip_sel(const int32_t* __restrict__ sel, int n, int32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = sel[n - 1 - i];
}

// Reverses the n x m array V (leading dimension ldv) in place as one
// sequence in column-major order: element (r, q) trades places with
// (n-1-r, m-1-q), which reverses the rows and the column order at once.
// scale[0 .. m) is reversed as well.
__global__ void __launch_bounds__(256) k_cx_reverse(double* __restrict__ V, int ldv, int n, int m,
                                                    int32_t* __restrict__ scale) {
  const long long half = ((long long)n * m) >> 1;
  const long long L = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (L < half) {
    const int q = (int)(L / n), r = (int)(L % n);
    double* a = V + 2 * ((size_t)q * ldv + r);
    double* b = V + 2 * ((size_t)(m - 1 - q) * ldv + (n - 1 - r));
    const double2 za = ld2(a), zb = ld2(b);
    st2(a, zb);
    st2(b, za);
  }
  if (L < (m >> 1)) {
    const int t = scale[L];
    scale[L] = scale[m - 1 - L];
    scale[m - 1 - L] = t;
  }
}

int cx_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? PEVC_ERR_NOMEM : PEVC_ERR_CUDA; }

#define CXK(call)                                  \
  do {                                             \
    cudaError_t _e = (call);                       \
    if (_e != cudaSuccess) return cx_fail(_e);     \
  } while (0)

template <class Tp>
int cx_alloc(Tp** p, size_t count) {
  if (cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(Tp)) != cudaSuccess) {
    *p = nullptr;
    return PEVC_ERR_NOMEM;
  }
  return 0;
}

}  // namespace

struct CplxWork {
  int n_max = 0, Mmax = 0;
  double* alpha = nullptr;
  double* beta = nullptr;
  int* ccol = nullptr;
  int* ex = nullptr;
  double* nrm = nullptr;
  double* tnS = nullptr;
  double* tnT = nullptr;
  double* gmax = nullptr;
  unsigned* status = nullptr;
  int32_t* h_sel = nullptr;
  int* h_ccol = nullptr;
  unsigned* h_status = nullptr;
  // left eigenvectors: the flipped conjugate-transposed pencil and selection
  // (allocated by the first left solve)
  double* lS = nullptr;
  double* lT = nullptr;
  int32_t* lsel = nullptr;
};

void cplx_free(CplxWork* w) {
  if (!w) return;
  void* dev[] = {w->alpha, w->beta, w->ccol, w->ex, w->nrm, w->tnS, w->tnT, w->gmax, w->status,
                 w->lS, w->lT, w->lsel};
  for (void* d : dev)
    if (d) cudaFree(d);
  void* host[] = {w->h_sel, w->h_ccol, w->h_status};
  for (void* h : host)
    if (h) cudaFreeHost(h);
  delete w;
}

static int cplx_alloc(CplxWork** out, int n_max) {
  CplxWork* w = new CplxWork;
  w->n_max = n_max;
  w->Mmax = (n_max + kCxTile - 1) / kCxTile;
  const size_t nm = (size_t)std::max(n_max, 1), M = (size_t)std::max(w->Mmax, 1);
  int rc = cx_alloc(&w->alpha, 2 * nm);
  rc = rc ? rc : cx_alloc(&w->beta, 2 * nm);
  rc = rc ? rc : cx_alloc(&w->ccol, nm);
  rc = rc ? rc : cx_alloc(&w->ex, M * nm);
  rc = rc ? rc : cx_alloc(&w->nrm, M * nm);
  rc = rc ? rc : cx_alloc(&w->tnS, M * M);
  rc = rc ? rc : cx_alloc(&w->tnT, M * M);
  rc = rc ? rc : cx_alloc(&w->gmax, 1);
  rc = rc ? rc : cx_alloc(&w->status, 1);
  if (!rc && cudaMallocHost(reinterpret_cast<void**>(&w->h_sel), nm * sizeof(int32_t)) != cudaSuccess) rc = PEVC_ERR_NOMEM;
  if (!rc && cudaMallocHost(reinterpret_cast<void**>(&w->h_ccol), nm * sizeof(int)) != cudaSuccess) rc = PEVC_ERR_NOMEM;
  if (!rc && cudaMallocHost(reinterpret_cast<void**>(&w->h_status), sizeof(unsigned)) != cudaSuccess) rc = PEVC_ERR_NOMEM;
  if (!rc) {
    const int smem = 2 * kCxTri * (int)sizeof(double2);
    if (cudaFuncSetAttribute(k_cx_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
      rc = PEVC_ERR_CUDA;
  }
  if (rc) {
    cplx_free(w);
    return rc;
  }
  *out = w;
  return 0;
}

int cplx_solve(CplxWork** wp, int n_max, cudaStream_t s, const double* S, int lds, const double* T, int ldt, int n,
               const int32_t* select, double* V, int ldv, int32_t* scale, int* m_out, bool normalise) {
  *m_out = 0;
  if (n == 0) return 0;
  if (!*wp) {
    const int rc = cplx_alloc(wp, n_max);
    if (rc) return rc;
  }
  CplxWork* w = *wp;
  const int M = (n + kCxTile - 1) / kCxTile;
  int m = 0;
  if (select) {
    CXK(cudaMemcpyAsync(w->h_sel, select, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CXK(cudaStreamSynchronize(s));
    for (int c = 0; c < n; ++c)
      if (w->h_sel[c]) w->h_ccol[m++] = c;
  } else {
    for (int c = 0; c < n; ++c) w->h_ccol[m++] = c;
  }
  CXK(cudaMemsetAsync(w->gmax, 0, sizeof(double), s));
  CXK(cudaMemsetAsync(w->status, 0, sizeof(unsigned), s));
  if (m) CXK(cudaMemcpyAsync(w->ccol, w->h_ccol, (size_t)m * sizeof(int), cudaMemcpyHostToDevice, s));
  k_cx_scan<<<n, 256, 0, s>>>(S, lds, T, ldt, n, w->gmax, w->status);
  CXK(cudaGetLastError());
  if (m) {
    k_cx_eig<<<(m + 255) / 256, 256, 0, s>>>(S, lds, T, ldt, w->ccol, m, w->gmax, w->alpha, w->beta, w->status);
    CXK(cudaGetLastError());
  }
  CXK(cudaMemcpyAsync(w->h_status, w->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CXK(cudaStreamSynchronize(s));
  const unsigned st = *w->h_status;
  if (st & kStNonfinite) return PEVC_ERR_NONFINITE;
  if (st & kStIndefinite) return PEVC_ERR_INDEFINITE;
  *m_out = m;
  if (m == 0) return 0;

  const int lde = w->n_max, ldm = w->Mmax;
  if (M > 1) {
    k_cx_tilenorms<<<dim3(M, M - 1), kCxTile, 0, s>>>(S, lds, T, ldt, n, ldm, w->tnS, w->tnT);
    CXK(cudaGetLastError());
  }
  k_cx_init<<<m, 256, 0, s>>>(S, lds, T, ldt, n, w->ccol, w->alpha, w->beta, V, ldv, w->ex, w->nrm, lde);
  CXK(cudaGetLastError());
  const int smem = 2 * kCxTri * (int)sizeof(double2);
  int q0 = m;
  for (int i = M - 1; i >= 0; --i) {
    // first selected column whose tip is in tile i or below (ccol ascends)
    while (q0 > 0 && w->h_ccol[q0 - 1] >= i * kCxTile) --q0;
    const int act = m - q0;
    if (act == 0) continue;
    k_cx_diag<<<(act + kCxDiagWarps - 1) / kCxDiagWarps, 32 * kCxDiagWarps, smem, s>>>(
        i, S, lds, T, ldt, n, w->ccol, q0, m, w->alpha, w->beta, V, ldv, w->ex, w->nrm, lde);
    CXK(cudaGetLastError());
    if (i > 0) {
      k_cx_update<<<dim3((act + kCxUpdCols - 1) / kCxUpdCols, i), 256, 0, s>>>(
          i, S, lds, T, ldt, n, q0, m, w->alpha, w->beta, V, ldv, w->ex, w->nrm, lde, w->tnS, w->tnT, ldm);
      CXK(cudaGetLastError());
    }
  }
  k_cx_post<<<m, 256, 0, s>>>(n, w->ccol, V, ldv, w->ex, w->nrm, lde, scale, normalise ? 1 : 0);
  CXK(cudaGetLastError());
  CXK(cudaStreamSynchronize(s));
  return 0;
}

int cplx_solve_left(CplxWork** wp, int n_max, cudaStream_t s, const double* S, int lds, const double* T, int ldt,
                    int n, const int32_t* select, double* U, int ldu, int32_t* scale, int* m_out, bool normalise) {
  *m_out = 0;
  if (n == 0) return 0;
  if (!*wp) {
    const int rc = cplx_alloc(wp, n_max);
    if (rc) return rc;
  }
  CplxWork* w = *wp;
  if (!w->lS) {
    const size_t nn = (size_t)std::max(n_max, 1) * std::max(n_max, 1);
    int rc = cx_alloc(&w->lS, 2 * nn);
    rc = rc ? rc : cx_alloc(&w->lT, 2 * nn);
    rc = rc ? rc : cx_alloc(&w->lsel, (size_t)std::max(n_max, 1));
    if (rc) return rc;
  }
  const dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
  k_cx_flip_ct<<<grid, block, 0, s>>>(S, lds, n, w->lS);
  CXK(cudaGetLastError());
  k_cx_flip_ct<<<grid, block, 0, s>>>(T, ldt, n, w->lT);
  CXK(cudaGetLastError());
  if (select) {
    k_cx_flip_sel<<<(n + 255) / 256, 256, 0, s>>>(select, n, w->lsel);
    CXK(cudaGetLastError());
  }
  const int rc = cplx_solve(wp, n_max, s, w->lS, n, w->lT, n, n, select ? w->lsel : nullptr, U, ldu, scale, m_out,
                            normalise);
  if (rc) return rc;
  const int m = *m_out;
  const long long half = (long long)n * m / 2;   // >= m / 2, the scale pairs
  if (half > 0) {
    k_cx_reverse<<<(unsigned)((half + 255) / 256), 256, 0, s>>>(U, ldu, n, m, scale);
    CXK(cudaGetLastError());
  }
  CXK(cudaStreamSynchronize(s));
  return 0;
}

}  // namespace pevc

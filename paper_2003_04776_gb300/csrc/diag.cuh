// diag.cuh -- device helpers of the diagonal-tile solves (kernels 1 and 3 of
// Section 3 with ProtectDivision / ProtectUpdate of Section 4): the staged
// diagonal blocks, the right-hand-side-independent factors of 1x1 and 2x2
// blocks, and one block step of one eigenvector.
#pragma once

#include "common.cuh"

namespace pevc {

constexpr double kUlp = 0x1p-53;

// Shared memory of one diagonal-tile task (a chunk of at most CB columns of a
// tile of order <= kMaxTile), in one struct so that a persistent kernel can
// overlay it with the memory of its other tasks.
template <int CB>
struct DiagSmem {
  double2 PQ[2][CB];                 // per block column, per column: (P, Q)
  double a[CB], b[CB], beta[CB], y[CB];   // per unit (eigenvector)
  double W[2][CB], piv[2][CB];
  // the diagonal tile's 1x1 / 2x2 blocks and column bounds, read by the
  // up-front factors only (the complex tips are computed with them);
  // afterwards the same memory holds the current block's S and T columns
  union {
    struct {
      double Sd[kMaxTile][2], Td[kMaxTile][2], tcS[kMaxTile], tcT[kMaxTile];
    } blk;
    double nc[4][kMaxTile];
  } ov;
  double tipw[CB][4];                // a complex pair's tip: re, im of its two rows (tip mode)
  // right-hand-side-independent factors per (block, unit): 1x1 blocks the
  // inverted pivot (1 double real, 2 complex), 2x2 blocks the LU factors
  // (4 doubles real, 8 complex) -- at most 2 doubles per row and column
  double pre[2 * kMaxTile * CB];
  short te[kMaxTile][CB];            // ProtectUpdate's t per (block, unit) as a power-of-two bound: t < 2^te
  unsigned long long key[CB];        // column maxima
  int lc[CB];                        // local column of chunk column t
  int tip[CB], e[CB], act[CB];       // per unit
  int sh[CB], anysh;                 // per column
  int boff[kMaxTile];                // offset of a block's factors in pre
  int nb, n1;
  short bs[kMaxTile];
  short ep[kMaxTile][CB];            // ilogb of the pivot (or u22) magnitude
  unsigned char bz[kMaxTile];
  unsigned char bord[kMaxTile];      // block indices, the 1x1 blocks first
  unsigned char pf[kMaxTile][CB];    // 2x2 pivot position pi | pj << 1
};

struct ColStep {
  double P[2][2];   // [block col][pair member]: beta * w
  double Q[2][2];   //                          : Re/Im of alpha * w
  double W[2][2];   // new stored values of the block rows
  int shift;
};

// The tile's diagonal blocks, staged in shared memory: for local row r,
// Sd[r][c] = S[r, bs(r) + c] and Td[r][c] = T[r, bs(r) + c] for the (one or
// two) columns c of its block; tcS / tcT are the column-segment maxima above
// each column's block inside the tile (the t of ProtectUpdate).
struct DiagBlocks {
  const double (*Sd)[2];
  const double (*Td)[2];
  const double* tcS;
  const double* tcT;
};

// 2^e for -1022 <= e <= 1023, assembled from the exponent field: the bound
// ProtectUpdate's t is kept as (t < 2^e, stored as e in 16 bits).  With the
// pre-scaling (|beta| max|S|, (|a| + |b|) max|T| <= 2^1000) t stays below
// 2^1002, so 2^e is finite; it is at most twice t (times 2^-1022 for t = 0).
__device__ __forceinline__ double pow2_bound(int e) { return __hiloint2double((e + 1023) << 20, 0); }

__device__ __forceinline__ double upd_norm(const DiagBlocks& D, int li0, int sz, double beta, double amag) {
  double t = fabs(beta) * D.tcS[li0] + amag * D.tcT[li0];
  if (sz == 2) t += fabs(beta) * D.tcS[li0 + 1] + amag * D.tcT[li0 + 1];
  return t;
}

// Twice the largest of |x|, |y| (an upper bound of |x| + |y|), by integer
// arithmetic on the exponent field; requires max(|x|, |y|) < 2^1023.
__device__ __forceinline__ double twice_max_abs(unsigned long long key) {
  return __longlong_as_double((long long)(key + (1ull << 52)));
}

// Entry (p, q) of a 2x2 array held in four registers (no local-memory array
// for a runtime index).
__device__ __forceinline__ double pick2(double m00, double m01, double m10, double m11, int p, int q) {
  return p ? (q ? m11 : m10) : (q ? m01 : m00);
}

// The right-hand-side-independent part of the robust 2x2 solve of a real
// eigenvalue, (beta S_bb - a T_bb) x = r: Gaussian elimination with complete
// pivoting, pivots below smin raised to smin (the DLALN2 principle of Section
// 5.2).  f = {1/piv, l, m[pi][oj]/piv, 1/u22}; ep = ilogb |u22|; pf = pi | pj << 1.
// The two quotients by the pivot are products with its reciprocal; with
// complete pivoting both are at most 1 in magnitude.
__device__ __forceinline__ void real2_factor(const DiagBlocks& D, int li0, double a, double beta, double* f,
                                             short& ep, unsigned char& pf) {
  double m[2][2];
  double sm = 0.0, tm = 0.0;
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const double s = D.Sd[li0 + p][q], t = D.Td[li0 + p][q];
      m[p][q] = beta * s - a * t;
      sm = max_nonneg(sm, fabs(s));
      tm = max_nonneg(tm, fabs(t));
    }
  const double smin = max_nonneg(kUlp * (fabs(beta) * sm + fabs(a) * tm), 0x1p-1022);
  int pi = 0, pj = 0;
  unsigned long long big = abs_key(m[0][0]);
  if (abs_key(m[0][1]) > big) { big = abs_key(m[0][1]); pi = 0; pj = 1; }
  if (abs_key(m[1][0]) > big) { big = abs_key(m[1][0]); pi = 1; pj = 0; }
  if (abs_key(m[1][1]) > big) { big = abs_key(m[1][1]); pi = 1; pj = 1; }
  if (big < abs_key(smin)) {
    m[0][0] = smin; m[0][1] = 0.0; m[1][0] = 0.0; m[1][1] = smin;
    pi = 0; pj = 0;
  }
  const int oi = 1 - pi, oj = 1 - pj;
  const double piv = pick2(m[0][0], m[0][1], m[1][0], m[1][1], pi, pj);
  const double m_oi_pj = pick2(m[0][0], m[0][1], m[1][0], m[1][1], oi, pj);
  const double m_pi_oj = pick2(m[0][0], m[0][1], m[1][0], m[1][1], pi, oj);
  const double m_oi_oj = pick2(m[0][0], m[0][1], m[1][0], m[1][1], oi, oj);
  const double ipiv = 1.0 / piv;
  const double l = m_oi_pj * ipiv;
  const double g = m_pi_oj * ipiv;
  double u22 = m_oi_oj - l * m_pi_oj;
  if (abs_key(u22) < abs_key(smin)) u22 = copysign(smin, u22);
  f[0] = ipiv;
  f[1] = l;
  f[2] = g;
  f[3] = 1.0 / u22;
  ep = (short)ilogb_key(abs_key(u22));
  pf = (unsigned char)(pi | (pj << 1));
}

// Complex counterpart (alpha = a + i b): f = {l, 1/u22, 1/piv, m[pi][oj]/piv}
// as (re, im) pairs; ep = ilogb(|Re u22| + |Im u22|).  Two complex
// reciprocals; the quotients by the pivot are products with its reciprocal.
__device__ __forceinline__ void cplx2_factor(const DiagBlocks& D, int li0, double a, double b, double beta, double* f,
                                             short& ep, unsigned char& pf) {
  const double amag = fabs(a) + fabs(b);
  double mr[2][2], mi[2][2];
  double sm = 0.0, tm = 0.0;
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const double s = D.Sd[li0 + p][q], t = D.Td[li0 + p][q];
      mr[p][q] = beta * s - a * t;
      mi[p][q] = -b * t;
      sm = max_nonneg(sm, fabs(s));
      tm = max_nonneg(tm, fabs(t));
    }
  const double smin = max_nonneg(kUlp * (fabs(beta) * sm + amag * tm), 0x1p-1022);
  int pi = 0, pj = 0;
  double big = -1.0;
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if (cmag(mr[p][q], mi[p][q]) > big) { big = cmag(mr[p][q], mi[p][q]); pi = p; pj = q; }
  if (big < smin) {
    mr[0][0] = smin; mr[0][1] = 0.0; mr[1][0] = 0.0; mr[1][1] = smin;
    mi[0][0] = 0.0; mi[0][1] = 0.0; mi[1][0] = 0.0; mi[1][1] = 0.0;
    pi = 0; pj = 0;
  }
  const int oi = 1 - pi, oj = 1 - pj;
#define PEVC_PICK(A, p, q) pick2(A[0][0], A[0][1], A[1][0], A[1][1], p, q)
  const double pvr = PEVC_PICK(mr, pi, pj), pvi = PEVC_PICK(mi, pi, pj);
  const double a1r = PEVC_PICK(mr, oi, pj), a1i = PEVC_PICK(mi, oi, pj);
  const double a2r = PEVC_PICK(mr, pi, oj), a2i = PEVC_PICK(mi, pi, oj);
  const double a3r = PEVC_PICK(mr, oi, oj), a3i = PEVC_PICK(mi, oi, oj);
#undef PEVC_PICK
  double ipr, ipi;
  crecip(pvr, pvi, ipr, ipi);
  double lr, li, gr, gi;
  cmul(a1r, a1i, ipr, ipi, lr, li);
  cmul(a2r, a2i, ipr, ipi, gr, gi);
  double ur = a3r - (lr * a2r - li * a2i);
  double ui = a3i - (lr * a2i + li * a2r);
  if (cmag(ur, ui) < smin) { ur = smin; ui = 0.0; }
  f[0] = lr;
  f[1] = li;
  crecip(ur, ui, f[2], f[3]);
  f[4] = ipr;
  f[5] = ipi;
  f[6] = gr;
  f[7] = gi;
  ep = (short)ilogb_key(abs_key(cmag(ur, ui)));
  pf = (unsigned char)(pi | (pj << 1));
}

// Tip of a complex pair: a null vector of M = beta S_jj - alpha T_jj,
// scaled so that its entry of largest modulus is exactly 1.
__device__ __forceinline__ void cplx_tip(const DiagBlocks& D, int li0, double a, double b, double beta,
                                         double& w0r, double& w0i, double& w1r, double& w1i) {
  double mr[2][2], mi[2][2];
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const double s = D.Sd[li0 + p][q], t = D.Td[li0 + p][q];
      mr[p][q] = beta * s - a * t;
      mi[p][q] = -b * t;
    }
  // (-m01, m00) is orthogonal to row 0, (m11, -m10) to row 1; both span ker M.
  double ur[2] = {-mr[0][1], mr[0][0]}, ui[2] = {-mi[0][1], mi[0][0]};
  double vr[2] = {mr[1][1], -mr[1][0]}, vi[2] = {mi[1][1], -mi[1][0]};
  const double nu = fmax(cmag(ur[0], ui[0]), cmag(ur[1], ui[1]));
  const double nv = fmax(cmag(vr[0], vi[0]), cmag(vr[1], vi[1]));
  if (nv > nu) { ur[0] = vr[0]; ur[1] = vr[1]; ui[0] = vi[0]; ui[1] = vi[1]; }
  const int big = (hypot(ur[1], ui[1]) > hypot(ur[0], ui[0])) ? 1 : 0;
  double zr[2], zi[2];
  cdiv(ur[0], ui[0], ur[big], ui[big], zr[0], zi[0]);
  cdiv(ur[1], ui[1], ur[big], ui[big], zr[1], zi[1]);
  zr[big] = 1.0;
  zi[big] = 0.0;
  w0r = zr[0]; w0i = zi[0]; w1r = zr[1]; w1i = zi[1];
}

// Phase A of one block step for one eigenvector (unit u): the right-hand-side-
// dependent part of the robust 1x1 / 2x2 solve and its protection.  piv holds
// the block rows' current values (the unit's columns t0c, t0c + 1); y, active
// and e are the unit's running bound, activity and exponent (updated); tipw
// is a complex pair's tip (cplx_tip, computed up front).
template <int CB>
__device__ __forceinline__ ColStep unit_step(const double* tipw, int mode, bool tips, int i0, int tip, int li0,
                                             int sz, bool has_above, bool pairs, int t0c, int u, double a,
                                             double b, double beta, double tn, int ep, const double* f, int pf,
                                             const double (*piv)[CB], double& y, bool& active, int& e) {
  ColStep st;
  st.shift = 0;
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int v = 0; v < 2; ++v) { st.P[x][v] = 0.0; st.Q[x][v] = 0.0; st.W[x][v] = 0.0; }
  if (mode == kDiagTip && i0 == tip) {
    // kernel 1: the tip, then the protect for the update of the rows above
    active = true;
    double w[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    if (!pairs) w[0][0] = 1.0;
    else {
      w[0][0] = tipw[0];
      w[0][1] = tipw[1];
      w[1][0] = tipw[2];
      w[1][1] = tipw[3];
    }
    const double x = fmax(cmag(w[0][0], w[0][1]), cmag(w[1][0], w[1][1]));
    const int ku = has_above ? protect_update(0.0, tn, x) : 0;
#pragma unroll
    for (int xx = 0; xx < 2; ++xx)
#pragma unroll
      for (int v = 0; v < 2; ++v) w[xx][v] = ku ? pow2_scale(w[xx][v], -ku) : w[xx][v];
    y = has_above ? tn * pow2_scale(x, -ku) : 0.0;
#pragma unroll
    for (int xx = 0; xx < 2; ++xx) {
      st.W[xx][0] = w[xx][0]; st.W[xx][1] = w[xx][1];
      st.P[xx][0] = beta * w[xx][0]; st.P[xx][1] = beta * w[xx][1];
      st.Q[xx][0] = a * w[xx][0] - b * w[xx][1];
      st.Q[xx][1] = a * w[xx][1] + b * w[xx][0];
    }
    e = ku;
  } else if (tips && i0 >= tip) {
    // below a tip, and (correction) at the tip block itself, the column
    // is zero: W, P, Q stay 0 and nothing is scaled
  } else if (active) {
    if (sz == 1 && !pairs) {
      // w = r / p as r * (1/p); ProtectDivision against |p| >= 2^ep
      double r = piv[0][t0c];
      int kd = exp_ub(r) - ep - kOmegaExp;
      kd = kd > 0 ? kd : 0;
      if (kd) { r = pow2_scale(r, -kd); y = pow2_scale(y, -kd); }
      double w = r * f[u];
      const int ku = has_above ? protect_update_ub(y, tn, w) : 0;
      if (ku) { w = pow2_scale(w, -ku); y = pow2_scale(y, -ku); }
      if (has_above) y = fma(tn, fabs(w), y);
      st.shift = kd + ku;
      st.W[0][0] = w;
      st.P[0][0] = beta * w;
      st.Q[0][0] = a * w;
    } else if (sz == 1) {
      // complex: |r| <= |Re r| + |Im r| < 2^(ilogb(max) + 2); the
      // quotient by p may grow by one more factor 2 (|p| >= cmag(p)/2)
      double rr = piv[0][t0c], ri = piv[0][t0c + 1];
      int kd = max(exp_ub(rr), exp_ub(ri)) + 2 - ep - kOmegaExp;
      kd = kd > 0 ? kd : 0;
      if (kd) { rr = pow2_scale(rr, -kd); ri = pow2_scale(ri, -kd); y = pow2_scale(y, -kd); }
      const double ir = f[2 * u], ii = f[2 * u + 1];
      double wr = fma(rr, ir, -ri * ii), wi = fma(rr, ii, ri * ir);
      const double x2 = twice_max_abs(max(abs_key(wr), abs_key(wi)));   // >= |Re w| + |Im w|
      const int ku = has_above ? protect_update_ub(y, tn, x2) : 0;
      double x2s = x2;
      if (ku) { wr = pow2_scale(wr, -ku); wi = pow2_scale(wi, -ku); x2s = pow2_scale(x2, -ku); y = pow2_scale(y, -ku); }
      if (has_above) y = fma(tn, x2s, y);
      st.shift = kd + ku;
      st.W[0][0] = wr; st.W[0][1] = wi;
      st.P[0][0] = beta * wr; st.P[0][1] = beta * wi;
      st.Q[0][0] = fma(a, wr, -b * wi); st.Q[0][1] = fma(a, wi, b * wr);
    } else if (!pairs) {
      // real 2x2 block: forward / back substitution with the factors
      const double* g = f + 4 * u;
      const int pi = pf & 1, pj = pf >> 1;
      double r0v = piv[0][t0c], r1v = piv[1][t0c];
      int kd = max(exp_ub(r0v), exp_ub(r1v)) + 5 - ep - kOmegaExp;
      kd = kd > 0 ? kd : 0;
      if (kd) { r0v = pow2_scale(r0v, -kd); r1v = pow2_scale(r1v, -kd); y = pow2_scale(y, -kd); }
      const double rp = pi ? r1v : r0v, ro = pi ? r0v : r1v;
      const double xo = fma(-g[1], rp, ro) * g[3];
      const double xp = fma(-g[2], xo, rp * g[0]);
      double w0 = pj ? xo : xp, w1 = pj ? xp : xo;
      const double x = max_nonneg(fabs(w0), fabs(w1));
      const int ku = has_above ? protect_update_ub(y, tn, x) : 0;
      double xs = x;
      if (ku) { w0 = pow2_scale(w0, -ku); w1 = pow2_scale(w1, -ku); xs = pow2_scale(x, -ku); y = pow2_scale(y, -ku); }
      if (has_above) y = fma(tn, xs, y);
      st.shift = kd + ku;
      st.W[0][0] = w0; st.W[1][0] = w1;
      st.P[0][0] = beta * w0; st.P[1][0] = beta * w1;
      st.Q[0][0] = a * w0; st.Q[1][0] = a * w1;
    } else {
      // complex 2x2 block
      const double* g = f + 8 * u;
      const int pi = pf & 1, pj = pf >> 1;
      double r0r = piv[0][t0c], r0i = piv[0][t0c + 1], r1r = piv[1][t0c], r1i = piv[1][t0c + 1];
      int kd = max(max(exp_ub(r0r), exp_ub(r0i)), max(exp_ub(r1r), exp_ub(r1i))) + 6 - ep - kOmegaExp;
      kd = kd > 0 ? kd : 0;
      if (kd) {
        r0r = pow2_scale(r0r, -kd); r0i = pow2_scale(r0i, -kd);
        r1r = pow2_scale(r1r, -kd); r1i = pow2_scale(r1i, -kd);
        y = pow2_scale(y, -kd);
      }
      const double rpr = pi ? r1r : r0r, rpi = pi ? r1i : r0i;
      const double ror = pi ? r0r : r1r, roi = pi ? r0i : r1i;
      const double lre = g[0], lim = g[1];
      const double er = fma(-lre, rpr, fma(lim, rpi, ror));
      const double ei = fma(-lre, rpi, fma(-lim, rpr, roi));
      const double xor_ = fma(er, g[2], -ei * g[3]), xoi = fma(er, g[3], ei * g[2]);
      const double q1r = fma(rpr, g[4], -rpi * g[5]), q1i = fma(rpr, g[5], rpi * g[4]);
      const double xpr = fma(-g[6], xor_, fma(g[7], xoi, q1r));
      const double xpi = fma(-g[6], xoi, fma(-g[7], xor_, q1i));
      double w0r, w0i, w1r, w1i;
      if (pj == 0) { w0r = xpr; w0i = xpi; w1r = xor_; w1i = xoi; }
      else         { w0r = xor_; w0i = xoi; w1r = xpr; w1i = xpi; }
      const double x2 = twice_max_abs(max(max(abs_key(w0r), abs_key(w0i)), max(abs_key(w1r), abs_key(w1i))));
      const int ku = has_above ? protect_update_ub(y, tn, x2) : 0;
      double x2s = x2;
      if (ku) {
        w0r = pow2_scale(w0r, -ku); w0i = pow2_scale(w0i, -ku);
        w1r = pow2_scale(w1r, -ku); w1i = pow2_scale(w1i, -ku);
        x2s = pow2_scale(x2, -ku); y = pow2_scale(y, -ku);
      }
      if (has_above) y = fma(tn, x2s, y);
      st.shift = kd + ku;
      st.W[0][0] = w0r; st.W[0][1] = w0i; st.W[1][0] = w1r; st.W[1][1] = w1i;
      st.P[0][0] = beta * w0r; st.P[0][1] = beta * w0i;
      st.P[1][0] = beta * w1r; st.P[1][1] = beta * w1i;
      st.Q[0][0] = fma(a, w0r, -b * w0i); st.Q[0][1] = fma(a, w0i, b * w0r);
      st.Q[1][0] = fma(a, w1r, -b * w1i); st.Q[1][1] = fma(a, w1i, b * w1r);
    }
    e += st.shift;
  }
  return st;
}


// Phase A of one 2x2 block step of complex pairs in a right-hand-side solve
// (kernel 3), taken by a whole warp: each unit (at most 4) gets 8 lanes, and
// the independent products of its 2x2 solve and of P = beta w, Q = alpha w
// are spread over them, so that the step issues 9 FP64 warp instructions
// instead of 29 on one lane (a warp issues its FP64 instructions one at a
// time).  Each value is computed with the same operations as in unit_step.
// Writes the unit's P, Q, W, shift, running bound y and exponent e; returns
// whether any unit shifted.  All 32 lanes call it.
template <int CB>
__device__ __forceinline__ bool pair2_step_warp(int lane, int nu, int li0, const double (*piv)[CB],
                                                const double* f, const short* ep_row, const unsigned char* pf_row,
                                                const short* te_row, const double* s_a, const double* s_b,
                                                const double* s_beta, double* s_y, int* s_e, const int* s_act,
                                                int* s_sh, double2 (*s_PQ)[CB], double (*s_W)[CB]) {
  const int u = lane >> 3, j = lane & 7, base = lane & ~7;
  const bool mine = u < nu;
  const int uu = mine ? u : 0;
  const int t0c = 2 * uu;
  const bool has_above = li0 > 0;
  const double a = s_a[uu], b = s_b[uu], beta = s_beta[uu];
  const double tn = pow2_bound(te_row[uu]);
  double y = s_y[uu];
  const int ep = ep_row[uu];
  const bool active = mine && s_act[uu];
  const unsigned full = 0xffffffffu;
  int shift = 0;
  double* pq0 = reinterpret_cast<double*>(&s_PQ[0][t0c]);   // P(t0c), Q(t0c), P(t0c + 1), Q(t0c + 1)
  double* pq1 = reinterpret_cast<double*>(&s_PQ[1][t0c]);
  const int j4 = j & 3;
  const double* g = f + 8 * uu;
  const int pf = pf_row[uu];
  const int pi = pf & 1, pj = pf >> 1;
  double r0r = piv[0][t0c], r0i = piv[0][t0c + 1], r1r = piv[1][t0c], r1i = piv[1][t0c + 1];
  int kd = max(max(exp_ub(r0r), exp_ub(r0i)), max(exp_ub(r1r), exp_ub(r1i))) + 6 - ep - kOmegaExp;
  kd = kd > 0 ? kd : 0;
  if (kd) {
    r0r = pow2_scale(r0r, -kd); r0i = pow2_scale(r0i, -kd);
    r1r = pow2_scale(r1r, -kd); r1i = pow2_scale(r1i, -kd);
    y = pow2_scale(y, -kd);
  }
  const double rpr = pi ? r1r : r0r, rpi = pi ? r1i : r0i;
  const double ror = pi ? r0r : r1r, roi = pi ? r0i : r1i;
  const double lre = g[0], lim = g[1];
  // lanes j4 = 0..3: Re e, Im e (e = ro - l rp), Re q, Im q (q = rp / piv)
  const double A1 = j4 < 2 ? -lre : rpr;
  const double B1 = j4 == 0 ? rpr : (j4 == 1 ? rpi : (j4 == 2 ? g[4] : g[5]));
  const double C1 = j4 == 0 ? lim : (j4 == 1 ? -lim : (j4 == 2 ? -rpi : rpi));
  const double D1 = j4 == 0 ? rpi : (j4 == 1 ? rpr : (j4 == 2 ? g[5] : g[4]));
  const double E1 = j4 == 0 ? ror : (j4 == 1 ? roi : -0.0);
  const double v1 = fma(A1, B1, fma(C1, D1, E1));
  const double er = __shfl_sync(full, v1, base), ei = __shfl_sync(full, v1, base + 1);
  const double q1r = __shfl_sync(full, v1, base + 2), q1i = __shfl_sync(full, v1, base + 3);
  // even lanes Re xo, odd lanes Im xo (xo = e / u22)
  const bool ev = (j & 1) == 0;
  const double v2 = fma(er, ev ? g[2] : g[3], (ev ? -ei : ei) * (ev ? g[3] : g[2]));
  const double xor_ = __shfl_sync(full, v2, base), xoi = __shfl_sync(full, v2, base + 1);
  // even lanes Re xp, odd lanes Im xp (xp = q - (m / piv) xo)
  const double v3 = fma(-g[6], ev ? xor_ : xoi, fma(ev ? g[7] : -g[7], ev ? xoi : xor_, ev ? q1r : q1i));
  const double xpr = __shfl_sync(full, v3, base), xpi = __shfl_sync(full, v3, base + 1);
  double w0r, w0i, w1r, w1i;
  if (pj == 0) { w0r = xpr; w0i = xpi; w1r = xor_; w1i = xoi; }
  else         { w0r = xor_; w0i = xoi; w1r = xpr; w1i = xpi; }
  const double x2 = twice_max_abs(max(max(abs_key(w0r), abs_key(w0i)), max(abs_key(w1r), abs_key(w1i))));
  const int ku = has_above ? protect_update_ub(y, tn, x2) : 0;
  double x2s = x2;
  if (ku) {
    w0r = pow2_scale(w0r, -ku); w0i = pow2_scale(w0i, -ku);
    w1r = pow2_scale(w1r, -ku); w1i = pow2_scale(w1i, -ku);
    x2s = pow2_scale(x2, -ku); y = pow2_scale(y, -ku);
  }
  // lanes 0..7: block column xc = j / 4; P re, P im, Q re, Q im
  const int xc = j >> 2;
  const double wr = xc ? w1r : w0r, wi = xc ? w1i : w0i;
  const double A4 = j4 < 2 ? beta : a;
  const double B4 = (j4 == 0 || j4 == 2) ? wr : wi;
  const double C4 = j4 < 2 ? -0.0 : (j4 == 2 ? -b : b);
  const double D4 = j4 < 2 ? 1.0 : (j4 == 2 ? wi : wr);
  const double v = fma(A4, B4, C4 * D4);
  if (active) {
    shift = kd + ku;
    double* pq = xc ? pq1 : pq0;
    pq[(j4 & 1) * 2 + (j4 >> 1)] = v;
    if (j == 0) {
      s_W[0][t0c] = w0r; s_W[0][t0c + 1] = w0i; s_W[1][t0c] = w1r; s_W[1][t0c + 1] = w1i;
      s_sh[t0c] = shift; s_sh[t0c + 1] = shift; s_e[uu] += shift;
      s_y[uu] = has_above ? fma(tn, x2s, y) : y;
    }
  } else if (mine && j == 0) {
    pq0[0] = pq0[1] = pq0[2] = pq0[3] = 0.0;
    pq1[0] = pq1[1] = pq1[2] = pq1[3] = 0.0;
    s_W[0][t0c] = s_W[0][t0c + 1] = s_W[1][t0c] = s_W[1][t0c + 1] = 0.0;
    s_sh[t0c] = 0; s_sh[t0c + 1] = 0;
  }
  return __any_sync(full, shift != 0);
}

}  // namespace pevc

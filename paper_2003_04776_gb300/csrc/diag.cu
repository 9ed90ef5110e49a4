// diag.cu -- diagonal-tile kernel: kernel 1 (tips, the eigenvectors of a
// small Schur pencil) and kernel 3 (the small solves S_ii Z D - T_ii Z B = Y_ij)
// of Section 3, made robust with ProtectDivision / ProtectUpdate (Section 4).
//
// One CTA owns one tile (i, j) and a chunk of at most CB (+1, so a complex
// pair is never split) of its columns.  Thread r holds row r of the chunk in
// registers.  The 1x1 / 2x2 blocks of S_ii are processed bottom-up; for every
// block the column threads solve the block (real or complex, Gaussian
// elimination with complete pivoting for 2x2, pivots below smin raised to
// smin -- the DLALN2 principle of Section 5.2) and pick the power-of-two scale
// that keeps the division and the following column update below Omega; then
// all row threads apply the scale and the rank-1/rank-2 column update
//   y_r <- 2^-k y_r - (S_{r,blk} (beta w) - T_{r,blk} (alpha w)).
// Every tile column carries its own exponent (an augmented tile column).
#include "common.cuh"

namespace pevc {

constexpr double kUlp = 0x1p-53;

struct ColStep {
  double P[2][2];   // [block col][pair member]: beta * w
  double Q[2][2];   //                          : Re/Im of alpha * w
  double W[2][2];   // new stored values of the block rows
  int shift;
};

// t of ProtectUpdate for the block's columns: |beta| ||S_col|| + |alpha| ||T_col||.
__device__ __forceinline__ double upd_norm(const Problem& P, int i0, int sz, double beta, double amag) {
  double t = fabs(beta) * P.tcS[i0] + amag * P.tcT[i0];
  if (sz == 2) t += fabs(beta) * P.tcS[i0 + 1] + amag * P.tcT[i0 + 1];
  return t;
}

// Robust solve of one block for a real eigenvalue.  r[] are the block rows'
// right-hand sides (already in the column's current scale); y is the bound on
// the rows above.  Returns the values and the total scale shift.
__device__ void real_block(const Problem& P, int i0, int sz, bool has_above, double a, double beta,
                           double r0, double r1, double& y, ColStep& out) {
  const double* S = P.S;
  const double* T = P.T;
  const size_t lds = P.lds, ldt = P.ldt;
  double w0, w1 = 0.0;
  int kd;
  if (sz == 1) {
    const double s = S[i0 * lds + i0], t = T[i0 * ldt + i0];
    double p = beta * s - a * t;
    const double smin = fmax(kUlp * (fabs(beta) * fabs(s) + fabs(a) * fabs(t)), 0x1p-1022);
    if (fabs(p) < smin) p = copysign(smin, p);
    kd = protect_division(fabs(r0), 0, fabs(p));
    if (kd) { r0 = pow2_scale(r0, -kd); y = pow2_scale(y, -kd); }
    w0 = r0 / p;
  } else {
    double m[2][2];
    double sm = 0.0, tm = 0.0;
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const double s = S[(i0 + q) * lds + i0 + p], t = T[(i0 + q) * ldt + i0 + p];
        m[p][q] = beta * s - a * t;
        sm = fmax(sm, fabs(s));
        tm = fmax(tm, fabs(t));
      }
    const double smin = fmax(kUlp * (fabs(beta) * sm + fabs(a) * tm), 0x1p-1022);
    int pi = 0, pj = 0;
    double big = fabs(m[0][0]);
    if (fabs(m[0][1]) > big) { big = fabs(m[0][1]); pi = 0; pj = 1; }
    if (fabs(m[1][0]) > big) { big = fabs(m[1][0]); pi = 1; pj = 0; }
    if (fabs(m[1][1]) > big) { big = fabs(m[1][1]); pi = 1; pj = 1; }
    if (big < smin) {
      m[0][0] = smin; m[0][1] = 0.0; m[1][0] = 0.0; m[1][1] = smin;
      pi = 0; pj = 0;
    }
    const int oi = 1 - pi, oj = 1 - pj;
    const double piv = m[pi][pj];
    const double l = m[oi][pj] / piv;
    double u22 = m[oi][oj] - l * m[pi][oj];
    if (fabs(u22) < smin) u22 = copysign(smin, u22);
    kd = protect_division(fmax(fabs(r0), fabs(r1)), 5, fabs(u22));
    if (kd) { r0 = pow2_scale(r0, -kd); r1 = pow2_scale(r1, -kd); y = pow2_scale(y, -kd); }
    const double rp = pi ? r1 : r0, ro = pi ? r0 : r1;
    const double xo = (ro - l * rp) / u22;
    const double xp = rp / piv - (m[pi][oj] / piv) * xo;
    w0 = oj ? xp : xo;
    w1 = oj ? xo : xp;
  }
  int ku = 0;
  const double tn = upd_norm(P, i0, sz, beta, fabs(a));
  const double x = fmax(fabs(w0), fabs(w1));
  if (has_above) ku = protect_update(y, tn, x);
  if (ku) { w0 = pow2_scale(w0, -ku); w1 = pow2_scale(w1, -ku); }
  if (has_above) y = pow2_scale(y, -ku) + tn * pow2_scale(x, -ku);
  out.shift = kd + ku;
  out.W[0][0] = w0; out.W[1][0] = w1;
  out.P[0][0] = beta * w0; out.P[1][0] = beta * w1;
  out.Q[0][0] = a * w0; out.Q[1][0] = a * w1;
}

// Complex counterpart for alpha = a + i b (a complex pair's two columns).
__device__ void cplx_block(const Problem& P, int i0, int sz, bool has_above, double a, double b,
                           double beta, double r0r, double r0i, double r1r, double r1i, double& y,
                           ColStep& out) {
  const double* S = P.S;
  const double* T = P.T;
  const size_t lds = P.lds, ldt = P.ldt;
  const double amag = fabs(a) + fabs(b);
  double w0r, w0i, w1r = 0.0, w1i = 0.0;
  int kd;
  if (sz == 1) {
    const double s = S[i0 * lds + i0], t = T[i0 * ldt + i0];
    double pr = beta * s - a * t, pim = -b * t;
    const double smin = fmax(kUlp * (fabs(beta) * fabs(s) + amag * fabs(t)), 0x1p-1022);
    if (cmag(pr, pim) < smin) { pr = smin; pim = 0.0; }
    kd = protect_division(cmag(r0r, r0i), 1, cmag(pr, pim));
    if (kd) { r0r = pow2_scale(r0r, -kd); r0i = pow2_scale(r0i, -kd); y = pow2_scale(y, -kd); }
    cdiv(r0r, r0i, pr, pim, w0r, w0i);
  } else {
    double mr[2][2], mi[2][2];
    double sm = 0.0, tm = 0.0;
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const double s = S[(i0 + q) * lds + i0 + p], t = T[(i0 + q) * ldt + i0 + p];
        mr[p][q] = beta * s - a * t;
        mi[p][q] = -b * t;
        sm = fmax(sm, fabs(s));
        tm = fmax(tm, fabs(t));
      }
    const double smin = fmax(kUlp * (fabs(beta) * sm + amag * tm), 0x1p-1022);
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
    double lr, li;
    cdiv(mr[oi][pj], mi[oi][pj], mr[pi][pj], mi[pi][pj], lr, li);
    double ur = mr[oi][oj] - (lr * mr[pi][oj] - li * mi[pi][oj]);
    double ui = mi[oi][oj] - (lr * mi[pi][oj] + li * mr[pi][oj]);
    if (cmag(ur, ui) < smin) { ur = smin; ui = 0.0; }
    kd = protect_division(fmax(cmag(r0r, r0i), cmag(r1r, r1i)), 5, cmag(ur, ui));
    if (kd) {
      r0r = pow2_scale(r0r, -kd); r0i = pow2_scale(r0i, -kd);
      r1r = pow2_scale(r1r, -kd); r1i = pow2_scale(r1i, -kd);
      y = pow2_scale(y, -kd);
    }
    const double rpr = pi ? r1r : r0r, rpi = pi ? r1i : r0i;
    const double ror = pi ? r0r : r1r, roi = pi ? r0i : r1i;
    const double er = ror - (lr * rpr - li * rpi), ei = roi - (lr * rpi + li * rpr);
    double xor_, xoi, q1r, q1i, q2r, q2i;
    cdiv(er, ei, ur, ui, xor_, xoi);
    cdiv(rpr, rpi, mr[pi][pj], mi[pi][pj], q1r, q1i);
    cdiv(mr[pi][oj], mi[pi][oj], mr[pi][pj], mi[pi][pj], q2r, q2i);
    const double xpr = q1r - (q2r * xor_ - q2i * xoi);
    const double xpi = q1i - (q2r * xoi + q2i * xor_);
    if (oj) { w0r = xpr; w0i = xpi; w1r = xor_; w1i = xoi; }
    else    { w0r = xor_; w0i = xoi; w1r = xpr; w1i = xpi; }
  }
  int ku = 0;
  const double tn = upd_norm(P, i0, sz, beta, amag);
  const double x = fmax(cmag(w0r, w0i), cmag(w1r, w1i));
  if (has_above) ku = protect_update(y, tn, x);
  if (ku) {
    w0r = pow2_scale(w0r, -ku); w0i = pow2_scale(w0i, -ku);
    w1r = pow2_scale(w1r, -ku); w1i = pow2_scale(w1i, -ku);
  }
  if (has_above) y = pow2_scale(y, -ku) + tn * pow2_scale(x, -ku);
  out.shift = kd + ku;
  out.W[0][0] = w0r; out.W[0][1] = w0i; out.W[1][0] = w1r; out.W[1][1] = w1i;
  out.P[0][0] = beta * w0r; out.P[0][1] = beta * w0i;
  out.P[1][0] = beta * w1r; out.P[1][1] = beta * w1i;
  out.Q[0][0] = a * w0r - b * w0i; out.Q[0][1] = a * w0i + b * w0r;
  out.Q[1][0] = a * w1r - b * w1i; out.Q[1][1] = a * w1i + b * w1r;
}

// Tip of a complex pair: a null vector of M = beta S_jj - alpha T_jj,
// scaled so that its entry of largest modulus is exactly 1.
__device__ void cplx_tip(const Problem& P, int i0, double a, double b, double beta,
                         double& w0r, double& w0i, double& w1r, double& w1i) {
  const double* S = P.S;
  const double* T = P.T;
  const size_t lds = P.lds, ldt = P.ldt;
  double mr[2][2], mi[2][2];
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const double s = S[(i0 + q) * lds + i0 + p], t = T[(i0 + q) * ldt + i0 + p];
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

template <int CB>
__global__ void __launch_bounds__(kMaxTile) k_diag(Problem P, int i_row, int mode) {
  const bool tips = mode != kDiagSolve;          // one CTA row per diagonal tile
  constexpr int NC = CB + 1;
  const int j = tips ? (int)blockIdx.y : i_row + 1 + (int)blockIdx.y;
  const int i = tips ? j : i_row;
  const int cs = P.cstart[j], ce = P.cstart[j + 1];
  int q0 = cs + (int)blockIdx.x * CB;
  if (q0 >= ce) return;
  int q1 = min(ce, q0 + CB);
  if (P.kind[q0] == 2) ++q0;
  if (q1 < ce && P.kind[q1] == 2) ++q1;
  const int nq = q1 - q0;
  if (nq <= 0) return;
  const int r0 = P.toff[i], h = P.toff[i + 1] - r0;
  const int lr = threadIdx.x;
  double* Yt = tile_ptr(P, i, j);
  const int m = P.m;

  __shared__ double s_a[NC], s_b[NC], s_beta[NC], s_y[NC], s_nrm[NC];
  __shared__ int s_kind[NC], s_tip[NC], s_e[NC], s_act[NC], s_sh[NC];
  __shared__ double s_piv[2][NC], s_P[2][NC], s_Q[2][NC], s_W[2][NC];

  if (lr < nq) {
    const int q = q0 + lr;
    const int c = P.ccol[q];
    const int kd = P.kind[q];
    const int c0 = (kd == 2) ? c - 1 : c;
    s_kind[lr] = kd;
    s_tip[lr] = c0;
    s_a[lr] = P.ca[c0];
    s_b[lr] = P.cb[c0];
    s_beta[lr] = P.cbeta[c0];
    s_nrm[lr] = 0.0;
    s_sh[lr] = 0;
    if (mode == kDiagTip) {
      s_act[lr] = 0;
      s_e[lr] = 0;
      s_y[lr] = 0.0;
    } else {
      const long long base = (long long)i * m;
      double nv = P.nrm[base + q];
      if (kd == 1) nv = fmax(nv, P.nrm[base + q + 1]);
      if (kd == 2) nv = fmax(nv, P.nrm[base + q - 1]);
      s_act[lr] = nv > 0.0;
      s_e[lr] = P.ex[base + q];
      s_y[lr] = nv;
    }
  }
  __syncthreads();

  double vals[NC];
#pragma unroll
  for (int t = 0; t < NC; ++t) {
    vals[t] = 0.0;
    if (mode != kDiagTip && t < nq && lr < h && s_act[t]) vals[t] = Yt[(size_t)(q0 - cs + t) * P.tb + lr];
  }

  int rr = r0 + h - 1;
  while (rr >= r0) {
    const int i0 = (P.blk[rr] == 2) ? rr - 1 : rr;
    const int sz = rr - i0 + 1;
    const int li0 = i0 - r0;
    if (lr >= li0 && lr < li0 + sz) {
#pragma unroll
      for (int t = 0; t < NC; ++t)
        if (t < nq) s_piv[lr - li0][t] = vals[t];
    }
    __syncthreads();
    if (lr < nq) {
      const int t = lr;
      const int kd = s_kind[t];
      if (kd != 2) {
        const int tip = s_tip[t];
        const bool has_above = li0 > 0;
        ColStep st;
        st.shift = 0;
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v) { st.P[u][v] = 0.0; st.Q[u][v] = 0.0; st.W[u][v] = 0.0; }
        double y = s_y[t];
        bool active = s_act[t];
        const bool at_or_below_tip = tips && i0 >= tip;
        if (mode == kDiagTip && i0 == tip) {
          // kernel 1: the tip, then the protect for the update of the rows above
          active = true;
          const double a = s_a[t], b = s_b[t], beta = s_beta[t];
          double w[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
          double amag = fabs(a) + fabs(b);
          if (kd == 0) w[0][0] = 1.0;
          else cplx_tip(P, i0, a, b, beta, w[0][0], w[0][1], w[1][0], w[1][1]);
          const double tn = upd_norm(P, i0, sz, beta, amag);
          const double x = fmax(cmag(w[0][0], w[0][1]), cmag(w[1][0], w[1][1]));
          int ku = has_above ? protect_update(0.0, tn, x) : 0;
#pragma unroll
          for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 2; ++v) w[u][v] = ku ? pow2_scale(w[u][v], -ku) : w[u][v];
          y = has_above ? tn * pow2_scale(x, -ku) : 0.0;
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            st.W[u][0] = w[u][0]; st.W[u][1] = w[u][1];
            st.P[u][0] = beta * w[u][0]; st.P[u][1] = beta * w[u][1];
            st.Q[u][0] = a * w[u][0] - b * w[u][1];
            st.Q[u][1] = a * w[u][1] + b * w[u][0];
          }
          s_e[t] = ku;
        } else if (at_or_below_tip) {
          // below a tip, and (correction) at the tip block itself, the column
          // is zero: W, P, Q stay 0 and nothing is scaled
        } else if (active) {
          const double a = s_a[t], b = s_b[t], beta = s_beta[t];
          if (kd == 0) {
            real_block(P, i0, sz, has_above, a, beta, s_piv[0][t], sz == 2 ? s_piv[1][t] : 0.0, y, st);
          } else {
            cplx_block(P, i0, sz, has_above, a, b, beta, s_piv[0][t], s_piv[0][t + 1],
                       sz == 2 ? s_piv[1][t] : 0.0, sz == 2 ? s_piv[1][t + 1] : 0.0, y, st);
          }
          s_e[t] += st.shift;
        }
        s_act[t] = active;
        s_y[t] = y;
        s_sh[t] = st.shift;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          s_P[u][t] = st.P[u][0]; s_Q[u][t] = st.Q[u][0]; s_W[u][t] = st.W[u][0];
        }
        if (kd == 1) {
          s_act[t + 1] = active;
          s_e[t + 1] = s_e[t];
          s_sh[t + 1] = st.shift;
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            s_P[u][t + 1] = st.P[u][1]; s_Q[u][t + 1] = st.Q[u][1]; s_W[u][t + 1] = st.W[u][1];
          }
        }
      }
    }
    __syncthreads();
    if (lr < h) {
      double s0 = 0.0, t0 = 0.0, s1 = 0.0, t1 = 0.0;
      const bool above = lr < li0;
      if (above) {
        s0 = P.S[(size_t)i0 * P.lds + r0 + lr];
        t0 = P.T[(size_t)i0 * P.ldt + r0 + lr];
        if (sz == 2) {
          s1 = P.S[(size_t)(i0 + 1) * P.lds + r0 + lr];
          t1 = P.T[(size_t)(i0 + 1) * P.ldt + r0 + lr];
        }
      }
      const bool inblk = lr >= li0 && lr < li0 + sz;
#pragma unroll
      for (int t = 0; t < NC; ++t) {
        if (t >= nq) break;
        const int sh = s_sh[t];
        double v = vals[t];
        if (sh) v = pow2_scale(v, -sh);
        if (inblk) {
          v = s_W[lr - li0][t];
        } else if (above) {
          v = fma(-s0, s_P[0][t], v);
          v = fma(t0, s_Q[0][t], v);
          if (sz == 2) {
            v = fma(-s1, s_P[1][t], v);
            v = fma(t1, s_Q[1][t], v);
          }
        }
        vals[t] = v;
      }
    }
    rr = i0 - 1;
  }

  // write back the solved tile columns and their augmented exponents / norms
  if (lr < h) {
#pragma unroll
    for (int t = 0; t < NC; ++t) {
      if (t >= nq) break;
      if (tips || s_act[t]) Yt[(size_t)(q0 - cs + t) * P.tb + lr] = vals[t];
    }
  }
#pragma unroll
  for (int t = 0; t < NC; ++t) {
    if (t >= nq) break;
    double v = (lr < h) ? fabs(vals[t]) : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((lr & 31) == 0 && v > 0.0) atomic_max_nonneg(&s_nrm[t], v);
  }
  __syncthreads();
  if (lr < nq) {
    const long long idx = (long long)i * m + q0 + lr;
    if (tips || s_act[lr]) {
      P.nrm[idx] = s_nrm[lr];
      P.ex[idx] = s_e[lr];    // kept even for an all-zero column so a pair's exponents agree
    }
  }
}

constexpr int kDiagCB = 16;

cudaError_t launch_diag(const Problem& P, int i, int mode, cudaStream_t s) {
  const int chunks = (P.tb + kDiagCB - 1) / kDiagCB;
  const int ntiles = (mode != kDiagSolve) ? P.M : (P.M - 1 - i);
  if (ntiles <= 0) return cudaSuccess;
  dim3 grid(chunks, ntiles);
  k_diag<kDiagCB><<<grid, kMaxTile, 0, s>>>(P, i, mode);
  return cudaGetLastError();
}

}  // namespace pevc

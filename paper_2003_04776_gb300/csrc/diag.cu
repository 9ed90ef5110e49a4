// diag.cu -- diagonal-tile kernel: kernel 1 (tips, the eigenvectors of a
// small Schur pencil) and kernel 3 (the small solves S_ii Z D - T_ii Z B = Y_ij)
// of Section 3, made robust with ProtectDivision / ProtectUpdate (Section 4).
//
// One CTA owns one tile (i, j) and a chunk of at most CB columns that are all
// real or all complex pairs (so the per-block pivot work is never divergent).
// Thread r holds row r of the chunk in registers.  The 1x1 / 2x2 blocks of
// S_ii are processed bottom-up; for every block the column threads solve the
// block (real or complex; Gaussian elimination with complete pivoting for
// 2x2, pivots below smin raised to smin -- the DLALN2 principle of Section
// 5.2) and pick the power-of-two scale that keeps the division and the
// following column update below Omega; then all row threads apply the scale
// and the rank-1/rank-2 column update
//   y_r <- 2^-k y_r - (S_{r,blk} (beta w) - T_{r,blk} (alpha w)).
// Every tile column carries its own exponent (an augmented tile column).
//
// FP64 instructions are scarce on this GPU, so everything that does not depend
// on the right-hand side is taken off the sequential block chain: the
// diagonal blocks' entries and column norms are staged in shared memory, and
// the pivots of all 1x1 blocks are inverted up front by all threads in
// parallel; the step itself is then a multiplication, integer exponent logic
// for the protection, and the rank update.
#include "common.cuh"

namespace pevc {

constexpr double kUlp = 0x1p-53;

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

__device__ __forceinline__ double upd_norm(const DiagBlocks& D, int li0, int sz, double beta, double amag) {
  double t = fabs(beta) * D.tcS[li0] + amag * D.tcT[li0];
  if (sz == 2) t += fabs(beta) * D.tcS[li0 + 1] + amag * D.tcT[li0 + 1];
  return t;
}

// Robust 2x2 solve for a real eigenvalue: (beta S_bb - a T_bb) x = r, r in
// the column's current scale; y bounds the rows above.
__device__ __forceinline__ void real_block2(const DiagBlocks& D, int li0, bool has_above, double a, double beta,
                                            double r0, double r1, double& y, ColStep& out) {
  double m[2][2];
  double sm = 0.0, tm = 0.0;
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const double s = D.Sd[li0 + p][q], t = D.Td[li0 + p][q];
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
  const int kd = protect_division(fmax(fabs(r0), fabs(r1)), 5, fabs(u22));
  if (kd) { r0 = pow2_scale(r0, -kd); r1 = pow2_scale(r1, -kd); y = pow2_scale(y, -kd); }
  const double rp = pi ? r1 : r0, ro = pi ? r0 : r1;
  const double xo = (ro - l * rp) / u22;
  const double xp = rp / piv - (m[pi][oj] / piv) * xo;
  double w0 = oj ? xp : xo, w1 = oj ? xo : xp;
  int ku = 0;
  const double tn = upd_norm(D, li0, 2, beta, fabs(a));
  const double x = fmax(fabs(w0), fabs(w1));
  if (has_above) ku = protect_update(y, tn, x);
  if (ku) { w0 = pow2_scale(w0, -ku); w1 = pow2_scale(w1, -ku); }
  if (has_above) y = pow2_scale(y, -ku) + tn * pow2_scale(x, -ku);
  out.shift = kd + ku;
  out.W[0][0] = w0; out.W[1][0] = w1;
  out.P[0][0] = beta * w0; out.P[1][0] = beta * w1;
  out.Q[0][0] = a * w0; out.Q[1][0] = a * w1;
}

// Complex 2x2 counterpart (alpha = a + i b).
__device__ __forceinline__ void cplx_block2(const DiagBlocks& D, int li0, bool has_above, double a, double b,
                                            double beta, double r0r, double r0i, double r1r, double r1i, double& y,
                                            ColStep& out) {
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
  const int kd = protect_division(fmax(cmag(r0r, r0i), cmag(r1r, r1i)), 5, cmag(ur, ui));
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
  double w0r, w0i, w1r, w1i;
  if (oj) { w0r = xpr; w0i = xpi; w1r = xor_; w1i = xoi; }
  else    { w0r = xor_; w0i = xoi; w1r = xpr; w1i = xpi; }
  int ku = 0;
  const double tn = upd_norm(D, li0, 2, beta, amag);
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

template <int CB>
__global__ void __launch_bounds__(kMaxTile) k_diag(Problem P, int i_row, int mode) {
  const bool tips = mode != kDiagSolve;          // one CTA row per diagonal tile
  const int j = tips ? (int)blockIdx.y : i_row + 1 + (int)blockIdx.y;
  const int i = tips ? j : i_row;
  const int chunk = P.dchunk_first[j] + (int)blockIdx.x;
  if (chunk >= P.dchunk_first[j + 1]) return;
  const int cs = P.cstart[j];
  const int pos0 = P.dchunk_pos[chunk];
  const int nq = P.dchunk_cnt[chunk];                       // columns of this chunk (<= CB)
  const bool pairs = P.kind[cs + P.dperm[pos0]] != 0;       // all complex pairs, or all real
  const int nu = pairs ? nq / 2 : nq;                       // eigenvectors (units) of the chunk
  const int r0 = P.toff[i], h = P.toff[i + 1] - r0;
  const int lr = threadIdx.x;
  double* Yt = tile_ptr(P, i, j);
  const int m = P.m;

  __shared__ int s_lc[CB];                                  // local column of chunk column t
  __shared__ double s_a[CB], s_b[CB], s_beta[CB], s_y[CB];  // per unit
  __shared__ int s_tip[CB], s_e[CB], s_act[CB];             // per unit
  __shared__ int s_sh[CB], s_anysh;                         // per column
  __shared__ double2 s_PQ[2][CB];                           // per block column, per column: (P, Q)
  __shared__ double s_W[2][CB], s_piv[2][CB];
  __shared__ short s_bs[kMaxTile];
  __shared__ unsigned char s_bz[kMaxTile];
  __shared__ int s_nb;
  __shared__ double s_Sd[kMaxTile][2], s_Td[kMaxTile][2], s_tcS[kMaxTile], s_tcT[kMaxTile];
  __shared__ double s_inv[kMaxTile][CB];                    // 1x1 pivots inverted: real [b][u], complex [b][2u..2u+1]
  __shared__ double s_tn[kMaxTile][CB];                     // ProtectUpdate's t per (block, unit)
  __shared__ short s_ep[kMaxTile][CB];                      // ilogb of |pivot| per (block, unit)
  __shared__ unsigned long long s_key[CB];

  // ---- stage column constants, the diagonal blocks and the block list
  if (lr < nq) {
    s_lc[lr] = P.dperm[pos0 + lr];
    s_sh[lr] = 0;
    s_key[lr] = 0ull;
  }
  __syncthreads();
  if (lr < nu) {
    const int t = pairs ? 2 * lr : lr;
    const int q = cs + s_lc[t];
    const int c0 = P.ccol[q];                               // first row of the eigenvector's block
    s_tip[lr] = c0;
    s_a[lr] = P.ca[c0];
    s_b[lr] = P.cb[c0];
    s_beta[lr] = P.cbeta[c0];
    if (mode == kDiagTip) {
      s_act[lr] = 0;
      s_e[lr] = 0;
      s_y[lr] = 0.0;
    } else {
      const long long base = (long long)i * m;
      double nv = P.nrm[base + q];
      if (pairs) nv = fmax(nv, P.nrm[base + q + 1]);
      s_act[lr] = nv > 0.0;
      s_e[lr] = P.ex[base + q];
      s_y[lr] = nv;
    }
  }
  if (lr < h) {
    const int gr = r0 + lr;
    const int bs = (P.blk[gr] == 2) ? gr - 1 : gr;
    const bool two = P.blk[gr] != 0;
    s_Sd[lr][0] = P.S[(size_t)bs * P.lds + gr];
    s_Td[lr][0] = P.T[(size_t)bs * P.ldt + gr];
    s_Sd[lr][1] = two ? P.S[(size_t)(bs + 1) * P.lds + gr] : 0.0;
    s_Td[lr][1] = two ? P.T[(size_t)(bs + 1) * P.ldt + gr] : 0.0;
    s_tcS[lr] = P.tcS[gr];
    s_tcT[lr] = P.tcT[gr];
  }
  if (lr == 0) {
    int nb = 0;
    for (int rr = h - 1; rr >= 0;) {
      const int st = (P.blk[r0 + rr] == 2) ? rr - 1 : rr;
      s_bs[nb] = (short)st;
      s_bz[nb] = (unsigned char)(rr - st + 1);
      ++nb;
      rr = st - 1;
    }
    s_nb = nb;
  }
  __syncthreads();
  const DiagBlocks D{s_Sd, s_Td, s_tcS, s_tcT};
  const int nb = s_nb;

  // ---- invert the pivots of every 1x1 block for every unit, in parallel
  for (int item = lr; item < nb * nu; item += blockDim.x) {
    const int bidx = item / nu, u = item % nu;
    if (s_bz[bidx] != 1) continue;
    const int li = s_bs[bidx];
    const double s = s_Sd[li][0], t = s_Td[li][0];
    const double a = s_a[u], b = s_b[u], beta = s_beta[u];
    if (!pairs) {
      double p = beta * s - a * t;
      const double smin = fmax(kUlp * (fabs(beta) * fabs(s) + fabs(a) * fabs(t)), 0x1p-1022);
      if (fabs(p) < smin) p = copysign(smin, p);
      s_inv[bidx][u] = 1.0 / p;
      s_ep[bidx][u] = (short)ilogb(p);
      s_tn[bidx][u] = fabs(beta) * s_tcS[li] + fabs(a) * s_tcT[li];
    } else {
      double pr = beta * s - a * t, pim = -b * t;
      const double amag = fabs(a) + fabs(b);
      const double smin = fmax(kUlp * (fabs(beta) * fabs(s) + amag * fabs(t)), 0x1p-1022);
      if (cmag(pr, pim) < smin) { pr = smin; pim = 0.0; }
      double ir, ii;
      cdiv(1.0, 0.0, pr, pim, ir, ii);
      s_inv[bidx][2 * u] = ir;
      s_inv[bidx][2 * u + 1] = ii;
      s_ep[bidx][u] = (short)ilogb(cmag(pr, pim));
      s_tn[bidx][u] = fabs(beta) * s_tcS[li] + amag * s_tcT[li];
    }
  }

  double vals[CB];
#pragma unroll
  for (int t = 0; t < CB; ++t) {
    vals[t] = 0.0;
    if (mode != kDiagTip && t < nq && lr < h && s_act[pairs ? t / 2 : t])
      vals[t] = Yt[(size_t)s_lc[t] * P.tb + lr];
  }
  __syncthreads();

  // S/T entries of the next block's columns for this thread's row (prefetched)
  double nS0 = 0.0, nT0 = 0.0, nS1 = 0.0, nT1 = 0.0;
  {
    const int li0 = s_bs[0], sz = s_bz[0];
    if (lr < li0) {
      nS0 = P.S[(size_t)(r0 + li0) * P.lds + r0 + lr];
      nT0 = P.T[(size_t)(r0 + li0) * P.ldt + r0 + lr];
      if (sz == 2) {
        nS1 = P.S[(size_t)(r0 + li0 + 1) * P.lds + r0 + lr];
        nT1 = P.T[(size_t)(r0 + li0 + 1) * P.ldt + r0 + lr];
      }
    }
  }

  for (int bidx = 0; bidx < nb; ++bidx) {
    const int li0 = s_bs[bidx], sz = s_bz[bidx];
    const int i0 = r0 + li0;
    if (lr >= li0 && lr < li0 + sz) {
#pragma unroll
      for (int t = 0; t < CB; ++t)
        if (t < nq) s_piv[lr - li0][t] = vals[t];
    }
    __syncthreads();
    // ---- phase A: one lane of warp 0 per unit solves the block
    if (lr < 32) {
      int myshift = 0;
      if (lr < nu) {
        const int u = lr;
        const int t0c = pairs ? 2 * u : u;
        const int tip = s_tip[u];
        const bool has_above = li0 > 0;
        const double a = s_a[u], b = s_b[u], beta = s_beta[u];
        ColStep st;
        st.shift = 0;
#pragma unroll
        for (int x = 0; x < 2; ++x)
#pragma unroll
          for (int v = 0; v < 2; ++v) { st.P[x][v] = 0.0; st.Q[x][v] = 0.0; st.W[x][v] = 0.0; }
        double y = s_y[u];
        bool active = s_act[u];
        if (mode == kDiagTip && i0 == tip) {
          // kernel 1: the tip, then the protect for the update of the rows above
          active = true;
          double w[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
          const double amag = fabs(a) + fabs(b);
          if (!pairs) w[0][0] = 1.0;
          else cplx_tip(D, li0, a, b, beta, w[0][0], w[0][1], w[1][0], w[1][1]);
          const double tn = upd_norm(D, li0, sz, beta, amag);
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
          s_e[u] = ku;
        } else if (tips && i0 >= tip) {
          // below a tip, and (correction) at the tip block itself, the column
          // is zero: W, P, Q stay 0 and nothing is scaled
        } else if (active) {
          if (sz == 1) {
            // precomputed inverse pivot: w = r / p as r * (1/p)
            const double tn = s_tn[bidx][u];
            const int ep = s_ep[bidx][u];
            if (!pairs) {
              double r = s_piv[0][t0c];
              int kd = 0;
              if (r != 0.0) { kd = exp_above(fabs(r)) - ep - kOmegaExp; kd = kd > 0 ? kd : 0; }
              if (kd) { r = pow2_scale(r, -kd); y = pow2_scale(y, -kd); }
              double w = r * s_inv[bidx][u];
              const int ku = has_above ? protect_update(y, tn, fabs(w)) : 0;
              if (ku) w = pow2_scale(w, -ku);
              if (has_above) y = pow2_scale(y, -ku) + tn * fabs(w);
              st.shift = kd + ku;
              st.W[0][0] = w;
              st.P[0][0] = beta * w;
              st.Q[0][0] = a * w;
            } else {
              double rr = s_piv[0][t0c], ri = s_piv[0][t0c + 1];
              const double mg = cmag(rr, ri);
              int kd = 0;
              if (mg > 0.0) { kd = exp_above(mg) + 1 - ep - kOmegaExp; kd = kd > 0 ? kd : 0; }
              if (kd) { rr = pow2_scale(rr, -kd); ri = pow2_scale(ri, -kd); y = pow2_scale(y, -kd); }
              const double ir = s_inv[bidx][2 * u], ii = s_inv[bidx][2 * u + 1];
              double wr = rr * ir - ri * ii, wi = rr * ii + ri * ir;
              const int ku = has_above ? protect_update(y, tn, cmag(wr, wi)) : 0;
              if (ku) { wr = pow2_scale(wr, -ku); wi = pow2_scale(wi, -ku); }
              if (has_above) y = pow2_scale(y, -ku) + tn * cmag(wr, wi);
              st.shift = kd + ku;
              st.W[0][0] = wr; st.W[0][1] = wi;
              st.P[0][0] = beta * wr; st.P[0][1] = beta * wi;
              st.Q[0][0] = a * wr - b * wi; st.Q[0][1] = a * wi + b * wr;
            }
          } else if (!pairs) {
            real_block2(D, li0, has_above, a, beta, s_piv[0][t0c], s_piv[1][t0c], y, st);
          } else {
            cplx_block2(D, li0, has_above, a, b, beta, s_piv[0][t0c], s_piv[0][t0c + 1], s_piv[1][t0c],
                        s_piv[1][t0c + 1], y, st);
          }
          s_e[u] += st.shift;
        }
        s_act[u] = active;
        s_y[u] = y;
        myshift = st.shift;
        const int ncols = pairs ? 2 : 1;
        for (int mm = 0; mm < ncols; ++mm) {
          s_sh[t0c + mm] = st.shift;
#pragma unroll
          for (int x = 0; x < 2; ++x) {
            s_PQ[x][t0c + mm] = make_double2(st.P[x][mm], st.Q[x][mm]);
            s_W[x][t0c + mm] = st.W[x][mm];
          }
        }
      }
      const bool anysh = __any_sync(0xffffffffu, myshift != 0);
      if (lr == 0) s_anysh = anysh ? 1 : 0;
    }
    __syncthreads();
    // ---- phase B: every row applies the scale and the rank update
    const double cS0 = nS0, cT0 = nT0, cS1 = nS1, cT1 = nT1;
    if (bidx + 1 < nb) {   // prefetch the next block's columns
      const int ln = s_bs[bidx + 1], szn = s_bz[bidx + 1];
      nS0 = nT0 = nS1 = nT1 = 0.0;
      if (lr < ln) {
        nS0 = P.S[(size_t)(r0 + ln) * P.lds + r0 + lr];
        nT0 = P.T[(size_t)(r0 + ln) * P.ldt + r0 + lr];
        if (szn == 2) {
          nS1 = P.S[(size_t)(r0 + ln + 1) * P.lds + r0 + lr];
          nT1 = P.T[(size_t)(r0 + ln + 1) * P.ldt + r0 + lr];
        }
      }
    }
    if (lr < h) {
      if (s_anysh) {
#pragma unroll
        for (int t = 0; t < CB; ++t)
          if (t < nq && s_sh[t]) vals[t] = pow2_scale(vals[t], -s_sh[t]);
      }
      if (lr >= li0 && lr < li0 + sz) {
#pragma unroll
        for (int t = 0; t < CB; ++t)
          if (t < nq) vals[t] = s_W[lr - li0][t];
      } else if (lr < li0) {
        if (sz == 1) {
#pragma unroll
          for (int t = 0; t < CB; ++t) {
            if (t < nq) {
              const double2 pq = s_PQ[0][t];
              vals[t] = fma(cT0, pq.y, fma(-cS0, pq.x, vals[t]));
            }
          }
        } else {
#pragma unroll
          for (int t = 0; t < CB; ++t) {
            if (t < nq) {
              const double2 pq0 = s_PQ[0][t], pq1 = s_PQ[1][t];
              vals[t] = fma(cT1, pq1.y, fma(-cS1, pq1.x, fma(cT0, pq0.y, fma(-cS0, pq0.x, vals[t]))));
            }
          }
        }
      }
    }
  }

  // write back the solved tile columns and their augmented exponents / norms
#pragma unroll
  for (int t = 0; t < CB; ++t) {
    if (t < nq) {
      const bool wr = tips || s_act[pairs ? t / 2 : t];
      if (lr < h && wr) Yt[(size_t)s_lc[t] * P.tb + lr] = vals[t];
      unsigned long long key = (lr < h) ? abs_key(vals[t]) : 0ull;
      for (int o = 16; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o));
      if ((lr & 31) == 0 && key) atomicMax(&s_key[t], key);
    }
  }
  __syncthreads();
  if (lr < nq) {
    const int u = pairs ? lr / 2 : lr;
    if (tips || s_act[u]) {
      const long long idx = (long long)i * m + cs + s_lc[lr];
      P.nrm[idx] = __longlong_as_double((long long)s_key[lr]);
      P.ex[idx] = s_e[u];     // kept even for an all-zero column so a pair's exponents agree
    }
  }
}

constexpr int kDiagCB = 16;

cudaError_t launch_diag(const Problem& P, int i, int mode, cudaStream_t s) {
  const int ntiles = (mode != kDiagSolve) ? P.M : (P.M - 1 - i);
  if (ntiles <= 0 || P.dchunk_max <= 0) return cudaSuccess;
  dim3 grid(P.dchunk_max, ntiles);
  k_diag<kDiagCB><<<grid, kMaxTile, 0, s>>>(P, i, mode);
  return cudaGetLastError();
}

}  // namespace pevc

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

// Twice the largest of |x|, |y| (an upper bound of |x| + |y|), by integer
// arithmetic on the exponent field; requires max(|x|, |y|) < 2^1023.
__device__ __forceinline__ double twice_max_abs(unsigned long long key) {
  return __longlong_as_double((long long)(key + (1ull << 52)));
}

// The right-hand-side-independent part of the robust 2x2 solve of a real
// eigenvalue, (beta S_bb - a T_bb) x = r: Gaussian elimination with complete
// pivoting, pivots below smin raised to smin (the DLALN2 principle of Section
// 5.2).  f = {1/piv, l, m[pi][oj]/piv, 1/u22}; ep = ilogb |u22|; pf = pi | pj << 1.
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
  f[0] = 1.0 / piv;
  f[1] = l;
  f[2] = m[pi][oj] / piv;
  f[3] = 1.0 / u22;
  ep = (short)ilogb_key(abs_key(u22));
  pf = (unsigned char)(pi | (pj << 1));
}

// Complex counterpart (alpha = a + i b): f = {l, 1/u22, 1/piv, m[pi][oj]/piv}
// as (re, im) pairs; ep = ilogb(|Re u22| + |Im u22|).
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
  f[0] = lr;
  f[1] = li;
  cdiv(1.0, 0.0, ur, ui, f[2], f[3]);
  cdiv(1.0, 0.0, mr[pi][pj], mi[pi][pj], f[4], f[5]);
  cdiv(mr[pi][oj], mi[pi][oj], mr[pi][pj], mi[pi][pj], f[6], f[7]);
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

template <int CB>
__global__ void __launch_bounds__(kMaxTile, 5) k_diag(Problem P, int i_row, int mode) {
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
  __shared__ int s_boff[kMaxTile];                          // offset of a block's factors in s_pre
  __shared__ int s_nb;
  __shared__ double s_Sd[kMaxTile][2], s_Td[kMaxTile][2], s_tcS[kMaxTile], s_tcT[kMaxTile];
  // right-hand-side-independent factors per (block, unit): 1x1 blocks the
  // inverted pivot (1 double real, 2 complex), 2x2 blocks the LU factors
  // (4 doubles real, 8 complex) -- at most 2 doubles per row and column
  __shared__ double s_pre[2 * kMaxTile * CB];
  __shared__ double s_tn[kMaxTile][CB];                     // ProtectUpdate's t per (block, unit)
  __shared__ short s_ep[kMaxTile][CB];                      // ilogb of the pivot (or u22) magnitude
  __shared__ unsigned char s_pf[kMaxTile][CB];              // 2x2 pivot position pi | pj << 1
  __shared__ unsigned long long s_key[CB];

  // one CTA per launch brings the diagonal tile's S and T columns into L2:
  // every CTA of the launch walks the same columns, in step (prefetch
  // addresses stay inside each column segment)
  if (blockIdx.x == 0 && blockIdx.y == 0 && lr < h) {
    const int lines = (8 * h + 127) / 128;
    const double* sc = P.S + (size_t)(r0 + lr) * P.lds + r0;
    const double* tc = P.T + (size_t)(r0 + lr) * P.ldt + r0;
    for (int q = 0; q <= lines; ++q) {
      const int off = min(16 * q, h - 1);                    // in doubles: 128 bytes per line
      asm volatile("prefetch.global.L2 [%0];\n" ::"l"(sc + off));
      asm volatile("prefetch.global.L2 [%0];\n" ::"l"(tc + off));
    }
  }
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
      if (pairs) nv = max_nonneg(nv, P.nrm[base + q + 1]);
      s_act[lr] = abs_key(nv) != 0;
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
    int nb = 0, off = 0;
    for (int rr = h - 1; rr >= 0;) {
      const int st = (P.blk[r0 + rr] == 2) ? rr - 1 : rr;
      const int sz = rr - st + 1;
      s_bs[nb] = (short)st;
      s_bz[nb] = (unsigned char)sz;
      s_boff[nb] = off;
      off += (sz == 1 ? 1 : 4) * (pairs ? 2 : 1) * nu;
      ++nb;
      rr = st - 1;
    }
    s_nb = nb;
  }
  __syncthreads();
  const DiagBlocks D{s_Sd, s_Td, s_tcS, s_tcT};
  const int nb = s_nb;

  // ---- everything that does not depend on the right-hand side, for every
  //      (block, unit) in parallel: pivots, factors, ProtectUpdate's t
  for (int item = lr; item < nb * nu; item += blockDim.x) {
    const int bidx = item / nu, u = item % nu;
    const int li = s_bs[bidx], sz = s_bz[bidx];
    const double a = s_a[u], b = s_b[u], beta = s_beta[u];
    const double amag = fabs(a) + fabs(b);
    double* f = s_pre + s_boff[bidx];
    s_tn[bidx][u] = upd_norm(D, li, sz, beta, amag);
    if (sz == 1) {
      const double s = s_Sd[li][0], t = s_Td[li][0];
      if (!pairs) {
        double p = beta * s - a * t;
        const double smin = fmax(kUlp * (fabs(beta) * fabs(s) + fabs(a) * fabs(t)), 0x1p-1022);
        if (fabs(p) < smin) p = copysign(smin, p);
        f[u] = 1.0 / p;
        s_ep[bidx][u] = (short)ilogb_key(abs_key(p));
      } else {
        double pr = beta * s - a * t, pim = -b * t;
        const double smin = fmax(kUlp * (fabs(beta) * fabs(s) + amag * fabs(t)), 0x1p-1022);
        if (cmag(pr, pim) < smin) { pr = smin; pim = 0.0; }
        cdiv(1.0, 0.0, pr, pim, f[2 * u], f[2 * u + 1]);
        s_ep[bidx][u] = (short)ilogb_key(abs_key(cmag(pr, pim)));
      }
      s_pf[bidx][u] = 0;
    } else if (!pairs) {
      real2_factor(D, li, a, beta, f + 4 * u, s_ep[bidx][u], s_pf[bidx][u]);
    } else {
      cplx2_factor(D, li, a, b, beta, f + 8 * u, s_ep[bidx][u], s_pf[bidx][u]);
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
    // ---- phase A: one lane of warp 0 per unit solves the block; only the
    //      right-hand-side-dependent arithmetic is left here
    if (lr < 32) {
      int myshift = 0;
      if (lr < nu) {
        const int u = lr;
        const int t0c = pairs ? 2 * u : u;
        const int tip = s_tip[u];
        const bool has_above = li0 > 0;
        const double a = s_a[u], b = s_b[u], beta = s_beta[u];
        const double tn = s_tn[bidx][u];
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
          if (!pairs) w[0][0] = 1.0;
          else cplx_tip(D, li0, a, b, beta, w[0][0], w[0][1], w[1][0], w[1][1]);
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
          const int ep = s_ep[bidx][u];
          const double* f = s_pre + s_boff[bidx];
          if (sz == 1 && !pairs) {
            // w = r / p as r * (1/p); ProtectDivision against |p| >= 2^ep
            double r = s_piv[0][t0c];
            const unsigned long long rb = abs_key(r);
            int kd = rb ? ilogb_key(rb) + 1 - ep - kOmegaExp : 0;
            kd = kd > 0 ? kd : 0;
            if (kd) { r = pow2_scale(r, -kd); y = pow2_scale(y, -kd); }
            double w = r * f[u];
            const int ku = has_above ? protect_update(y, tn, fabs(w)) : 0;
            if (ku) w = pow2_scale(w, -ku);
            if (has_above) y = fma(tn, fabs(w), pow2_scale(y, -ku));
            st.shift = kd + ku;
            st.W[0][0] = w;
            st.P[0][0] = beta * w;
            st.Q[0][0] = a * w;
          } else if (sz == 1) {
            // complex: |r| <= |Re r| + |Im r| < 2^(ilogb(max) + 2); the
            // quotient by p may grow by one more factor 2 (|p| >= cmag(p)/2)
            double rr = s_piv[0][t0c], ri = s_piv[0][t0c + 1];
            const unsigned long long rb = max(abs_key(rr), abs_key(ri));
            int kd = rb ? ilogb_key(rb) + 3 - ep - kOmegaExp : 0;
            kd = kd > 0 ? kd : 0;
            if (kd) { rr = pow2_scale(rr, -kd); ri = pow2_scale(ri, -kd); y = pow2_scale(y, -kd); }
            const double ir = f[2 * u], ii = f[2 * u + 1];
            double wr = fma(rr, ir, -ri * ii), wi = fma(rr, ii, ri * ir);
            const double x2 = twice_max_abs(max(abs_key(wr), abs_key(wi)));   // >= |Re w| + |Im w|
            const int ku = has_above ? protect_update(y, tn, x2) : 0;
            if (ku) { wr = pow2_scale(wr, -ku); wi = pow2_scale(wi, -ku); }
            if (has_above) y = fma(tn, pow2_scale(x2, -ku), pow2_scale(y, -ku));
            st.shift = kd + ku;
            st.W[0][0] = wr; st.W[0][1] = wi;
            st.P[0][0] = beta * wr; st.P[0][1] = beta * wi;
            st.Q[0][0] = fma(a, wr, -b * wi); st.Q[0][1] = fma(a, wi, b * wr);
          } else if (!pairs) {
            // real 2x2 block: forward / back substitution with the factors
            const double* g = f + 4 * u;
            const int pf = s_pf[bidx][u], pi = pf & 1, pj = pf >> 1;
            double r0v = s_piv[0][t0c], r1v = s_piv[1][t0c];
            const unsigned long long rb = max(abs_key(r0v), abs_key(r1v));
            int kd = rb ? ilogb_key(rb) + 1 + 5 - ep - kOmegaExp : 0;
            kd = kd > 0 ? kd : 0;
            if (kd) { r0v = pow2_scale(r0v, -kd); r1v = pow2_scale(r1v, -kd); y = pow2_scale(y, -kd); }
            const double rp = pi ? r1v : r0v, ro = pi ? r0v : r1v;
            const double xo = fma(-g[1], rp, ro) * g[3];
            const double xp = fma(-g[2], xo, rp * g[0]);
            double w0 = pj ? xo : xp, w1 = pj ? xp : xo;
            const double x = max_nonneg(fabs(w0), fabs(w1));
            const int ku = has_above ? protect_update(y, tn, x) : 0;
            if (ku) { w0 = pow2_scale(w0, -ku); w1 = pow2_scale(w1, -ku); }
            if (has_above) y = fma(tn, pow2_scale(x, -ku), pow2_scale(y, -ku));
            st.shift = kd + ku;
            st.W[0][0] = w0; st.W[1][0] = w1;
            st.P[0][0] = beta * w0; st.P[1][0] = beta * w1;
            st.Q[0][0] = a * w0; st.Q[1][0] = a * w1;
          } else {
            // complex 2x2 block
            const double* g = f + 8 * u;
            const int pf = s_pf[bidx][u], pi = pf & 1, pj = pf >> 1;
            double r0r = s_piv[0][t0c], r0i = s_piv[0][t0c + 1], r1r = s_piv[1][t0c], r1i = s_piv[1][t0c + 1];
            const unsigned long long rb =
                max(max(abs_key(r0r), abs_key(r0i)), max(abs_key(r1r), abs_key(r1i)));
            int kd = rb ? ilogb_key(rb) + 2 + 5 - ep - kOmegaExp : 0;
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
            const int ku = has_above ? protect_update(y, tn, x2) : 0;
            if (ku) {
              w0r = pow2_scale(w0r, -ku); w0i = pow2_scale(w0i, -ku);
              w1r = pow2_scale(w1r, -ku); w1i = pow2_scale(w1i, -ku);
            }
            if (has_above) y = fma(tn, pow2_scale(x2, -ku), pow2_scale(y, -ku));
            st.shift = kd + ku;
            st.W[0][0] = w0r; st.W[0][1] = w0i; st.W[1][0] = w1r; st.W[1][1] = w1i;
            st.P[0][0] = beta * w0r; st.P[0][1] = beta * w0i;
            st.P[1][0] = beta * w1r; st.P[1][1] = beta * w1i;
            st.Q[0][0] = fma(a, w0r, -b * w0i); st.Q[0][1] = fma(a, w0i, b * w0r);
            st.Q[1][0] = fma(a, w1r, -b * w1i); st.Q[1][1] = fma(a, w1i, b * w1r);
          }
          s_e[u] += st.shift;
        }
        s_act[u] = active;
        s_y[u] = y;
        myshift = st.shift;
        const int ncols = pairs ? 2 : 1;
#pragma unroll
        for (int mm = 0; mm < 2; ++mm) {
          if (mm >= ncols) break;
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

cudaError_t launch_diag(const Problem& P, int i, int mode, cudaStream_t s) {
  const int ntiles = (mode != kDiagSolve) ? P.M : (P.M - 1 - i);
  if (ntiles <= 0 || P.dchunk_max <= 0) return cudaSuccess;
  dim3 grid(P.dchunk_max, ntiles);
  k_diag<kDiagChunk><<<grid, kMaxTile, 0, s>>>(P, i, mode);
  return cudaGetLastError();
}

}  // namespace pevc

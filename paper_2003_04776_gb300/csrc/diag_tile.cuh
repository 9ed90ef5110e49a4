// diag_tile.cuh -- one diagonal-tile task (kernels 1 and 3 of Section 3), shared
// by the per-stage kernel k_diag (diag.cu) and the persistent scheduler
// (dag.cu): kernel 1 (tips, the eigenvectors of a small Schur pencil) and
// kernel 3 (the small solves S_ii Z D - T_ii Z B = Y_ij) of Section 3, made
// robust with ProtectDivision / ProtectUpdate (Section 4).
//
// One CTA owns one tile (i, j) and a chunk of at most CB columns that are all
// real or all complex pairs (so the per-block pivot work is never divergent).
// Thread lr holds column lr % CB of the chunk at the rows congruent to lr / CB
// modulo 128 / CB, in registers.  The 1x1 / 2x2 blocks of S_ii are processed
// bottom-up; for every block the solve of each eigenvector (real or complex;
// Gaussian elimination with complete pivoting for 2x2, pivots below smin
// raised to smin -- the DLALN2 principle of Section 5.2) picks the power-of-
// two scale that keeps the division and the following column update below
// Omega; then all threads apply the scale and the rank-1/rank-2 update
//   y_r <- 2^-k y_r - (S_{r,blk} (beta w) - T_{r,blk} (alpha w))
// of the rows above the block.  Every tile column carries its own exponent
// (an augmented tile column).
//
// FP64 instructions are scarce on this GPU (the SM's FP64 unit takes 16
// cycles per warp instruction, and a warp issues them one at a time), so
// everything that does not depend on the right-hand side is taken off the
// sequential block chain and computed up front by all threads (inverted
// pivots, 2x2 LU factors with one reciprocal per pivot, ProtectUpdate's t; the
// 1x1 and the 2x2 blocks in separate warp-uniform passes).  A step is then a
// few multiplications, the protection's integer exponent logic on the high
// words, and the rank update; the 2x2 blocks of complex pairs spread their
// step over eight lanes per eigenvector.
#pragma once

#include "diag.cuh"

namespace pevc {

// One diagonal-tile task: tile (i, j) (i == j for the tips), column chunk
// `chunk` (an index into the chunk lists), solved by the 128 threads of the
// calling CTA in the shared memory sm.  pa_warp picks the warp of the block
// solves; with prefetch the CTA also brings the diagonal tile's S and T
// columns into L2 for the other chunks of the row.
template <int CB>
__device__ __forceinline__ void diag_tile(const Problem& P, int i, int j, int chunk, int mode, int pa_warp,
                                          bool prefetch, DiagSmem<CB>& sm) {
  const bool tips = mode != kDiagSolve;
  const int cs = P.cstart[j];
  const int pos0 = P.dchunk_pos[chunk];
  const int nq = P.dchunk_cnt[chunk];                       // columns of this chunk (<= CB)
  const bool pairs = P.kind[cs + P.dperm[pos0]] != 0;       // all complex pairs, or all real
  const int nu = pairs ? nq / 2 : nq;                       // eigenvectors (units) of the chunk
  const int r0 = P.toff[i], h = P.toff[i + 1] - r0;
  const int lr = threadIdx.x;
  double* Yt = tile_ptr(P, i, j);
  const int m = P.m;

  auto& s_lc = sm.lc;
  auto& s_a = sm.a;
  auto& s_b = sm.b;
  auto& s_beta = sm.beta;
  auto& s_y = sm.y;
  auto& s_tip = sm.tip;
  auto& s_e = sm.e;
  auto& s_act = sm.act;
  auto& s_sh = sm.sh;
  auto& s_anysh = sm.anysh;
  auto& s_PQ = sm.PQ;
  auto& s_W = sm.W;
  auto& s_piv = sm.piv;
  auto& s_bs = sm.bs;
  auto& s_bz = sm.bz;
  auto& s_boff = sm.boff;
  auto& s_nb = sm.nb;
  auto& s_n1 = sm.n1;
  auto& s_bord = sm.bord;
  auto& s_Sd = sm.ov.blk.Sd;
  auto& s_Td = sm.ov.blk.Td;
  auto& s_tcS = sm.ov.blk.tcS;
  auto& s_tcT = sm.ov.blk.tcT;
  auto& s_pre = sm.pre;
  auto& s_te = sm.te;
  auto& s_ep = sm.ep;
  auto& s_pf = sm.pf;
  auto& s_key = sm.key;
  auto& s_nc = sm.ov.nc;

  // one CTA per launch brings the diagonal tile's S and T columns into L2:
  // every CTA of the launch walks the same columns, in step (prefetch
  // addresses stay inside each column segment)
  if (prefetch && lr < h) {
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
    int n1 = 0;
    for (int q = 0; q < nb; ++q)
      if (s_bz[q] == 1) s_bord[n1++] = (unsigned char)q;
    s_n1 = n1;
    int q2 = n1;
    for (int q = 0; q < nb; ++q)
      if (s_bz[q] == 2) s_bord[q2++] = (unsigned char)q;
  }
  __syncthreads();
  const DiagBlocks D{s_Sd, s_Td, s_tcS, s_tcT};
  const int nb = s_nb;

  // ---- everything that does not depend on the right-hand side, for every
  //      (block, unit) in parallel: pivots, factors, ProtectUpdate's t.  The
  //      1x1 blocks come first and the 2x2 blocks after them, so that a warp
  //      takes one kind of block at a time
  const int n1 = s_n1;
  for (int item = lr; item < nb * nu; item += blockDim.x) {
    const int bidx = s_bord[item / nu], u = item % nu;
    const bool one = item < n1 * nu;
    const int li = s_bs[bidx];
    const double a = s_a[u], b = s_b[u], beta = s_beta[u];
    const double amag = fabs(a) + fabs(b);
    double* f = s_pre + s_boff[bidx];
    s_te[bidx][u] = (short)exp_ub(upd_norm(D, li, one ? 1 : 2, beta, amag));
    if (one) {
      const double s = s_Sd[li][0], t = s_Td[li][0];
      if (!pairs) {
        double p = beta * s - a * t;
        const double smin = max_nonneg(kUlp * (fabs(beta) * fabs(s) + fabs(a) * fabs(t)), 0x1p-1022);
        if (abs_key(p) < abs_key(smin)) p = copysign(smin, p);
        f[u] = 1.0 / p;
        s_ep[bidx][u] = (short)ilogb_key(abs_key(p));
      } else {
        double pr = beta * s - a * t, pim = -b * t;
        const double smin = max_nonneg(kUlp * (fabs(beta) * fabs(s) + amag * fabs(t)), 0x1p-1022);
        const double pm = cmag(pr, pim);
        if (abs_key(pm) < abs_key(smin)) { pr = smin; pim = 0.0; }
        crecip(pr, pim, f[2 * u], f[2 * u + 1]);
        s_ep[bidx][u] = (short)ilogb_key(abs_key(abs_key(pm) < abs_key(smin) ? smin : pm));
      }
      s_pf[bidx][u] = 0;
    } else if (!pairs) {
      real2_factor(D, li, a, beta, f + 4 * u, s_ep[bidx][u], s_pf[bidx][u]);
    } else {
      cplx2_factor(D, li, a, b, beta, f + 8 * u, s_ep[bidx][u], s_pf[bidx][u]);
    }
  }

  // the complex tips (kernel 1 on a pair's own 2x2 block), from the staged
  // blocks while they are still in shared memory
  if (mode == kDiagTip && pairs && lr < nu) {
    const int li = s_tip[lr] - r0;
    cplx_tip(D, li, s_a[lr], s_b[lr], s_beta[lr], sm.tipw[lr][0], sm.tipw[lr][1], sm.tipw[lr][2], sm.tipw[lr][3]);
  }

  // ---- element ownership: thread lr holds column t = lr % CB of the chunk at
  //      rows g + NG k (g = lr / CB, k < CB).  A warp then covers CB columns of
  //      32 / CB interleaved row groups, so the rows above a block -- the only
  //      rows with rank-update work -- are spread evenly over the four warps
  //      at every step (a warp issues its FP64 instructions one at a time, so
  //      a step lasts as long as its busiest warp)
  constexpr int NG = kMaxTile / CB;
  const int t = lr % CB, g = lr / CB;
  const bool tcol = t < nq;
  double vals[CB];
#pragma unroll
  for (int k = 0; k < CB; ++k) {
    const int r = g + NG * k;
    vals[k] = 0.0;
    if (mode != kDiagTip && tcol && r < h && s_act[pairs ? t / 2 : t]) vals[k] = Yt[(size_t)s_lc[t] * P.tb + r];
  }
  // the current block's S and T columns (the rows above it) are staged in
  // shared memory (s_nc, over the diagonal blocks' memory, free once the
  // factors and tips above are computed): loaded into registers during the
  // step before, stored after the step's first barrier (every thread has then
  // finished the previous step's rank update, the only reader)
  __syncthreads();
  {
    const int li0 = s_bs[0], sz = s_bz[0];
    if (lr < li0) {
      s_nc[0][lr] = P.S[(size_t)(r0 + li0) * P.lds + r0 + lr];
      s_nc[1][lr] = P.T[(size_t)(r0 + li0) * P.ldt + r0 + lr];
      if (sz == 2) {
        s_nc[2][lr] = P.S[(size_t)(r0 + li0 + 1) * P.lds + r0 + lr];
        s_nc[3][lr] = P.T[(size_t)(r0 + li0 + 1) * P.ldt + r0 + lr];
      }
    }
  }
  __syncthreads();

  double nS0 = 0.0, nT0 = 0.0, nS1 = 0.0, nT1 = 0.0;   // the next block's columns, in flight
  for (int bidx = 0; bidx < nb; ++bidx) {
    const int li0 = s_bs[bidx], sz = s_bz[bidx];
    const int i0 = r0 + li0;
    if (tcol) {
#pragma unroll
      for (int k = 0; k < CB; ++k) {
        const int r = g + NG * k;
        if (r >= li0 && r < li0 + sz) s_piv[r - li0][t] = vals[k];
      }
    }
    __syncthreads();
    if (bidx > 0 && lr < li0) {
      s_nc[0][lr] = nS0;
      s_nc[1][lr] = nT0;
      s_nc[2][lr] = nS1;
      s_nc[3][lr] = nT1;
    }
    const int ln = (bidx + 1 < nb) ? s_bs[bidx + 1] : 0, szn = (bidx + 1 < nb) ? s_bz[bidx + 1] : 1;
    if (lr < ln) {
      nS0 = P.S[(size_t)(r0 + ln) * P.lds + r0 + lr];
      nT0 = P.T[(size_t)(r0 + ln) * P.ldt + r0 + lr];
      nS1 = 0.0;
      nT1 = 0.0;
      if (szn == 2) {
        nS1 = P.S[(size_t)(r0 + ln + 1) * P.lds + r0 + lr];
        nT1 = P.T[(size_t)(r0 + ln + 1) * P.ldt + r0 + lr];
      }
    }
    // ---- phase A: the block's solve for every unit; only the
    //      right-hand-side-dependent arithmetic is left here (the 2x2
    //      blocks of complex pairs in a right-hand-side solve take eight
    //      lanes per unit, everything else one)
    if ((lr >> 5) == pa_warp && mode == kDiagSolve && pairs && sz == 2) {
      const bool anysh = pair2_step_warp<CB>(lr & 31, nu, li0, s_piv, s_pre + s_boff[bidx], s_ep[bidx],
                                            s_pf[bidx], s_te[bidx], s_a, s_b, s_beta, s_y, s_e, s_act, s_sh,
                                            s_PQ, s_W);
      if ((lr & 31) == 0) s_anysh = anysh ? 1 : 0;
    } else if ((lr >> 5) == pa_warp) {
      const int u = lr & 31;
      int myshift = 0;
      if (u < nu) {
        const int t0c = pairs ? 2 * u : u;
        const int tip = s_tip[u];
        const bool has_above = li0 > 0;
        const double a = s_a[u], b = s_b[u], beta = s_beta[u];
        const double tn = pow2_bound(s_te[bidx][u]);
        double y = s_y[u];
        bool active = s_act[u];
        int e = s_e[u];
        const ColStep st = unit_step<CB>(sm.tipw[u], mode, tips, i0, tip, li0, sz, has_above, pairs, t0c, u, a, b, beta, tn,
                                         s_ep[bidx][u], s_pre + s_boff[bidx], s_pf[bidx][u], s_piv, y, active, e);
        s_e[u] = e;
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
      if (u == 0) s_anysh = anysh ? 1 : 0;
    }
    __syncthreads();
    // ---- phase B: the scale and the rank update of the rows above, the
    //      solved values into the block rows
    if (tcol) {
      if (s_anysh) {
        const int sh = s_sh[t];
        if (sh) {
#pragma unroll
          for (int k = 0; k < CB; ++k) vals[k] = pow2_scale(vals[k], -sh);
        }
      }
      // row steps k run while the warp's first row group is above the block
      // (a warp-uniform exit, so no FP64 instruction is issued for a step
      // without work); lanes past the block's first row keep their values
      const double (*cn)[kMaxTile] = s_nc;
      const double2 pq0 = s_PQ[0][t];
      const int wg = (lr >> 5) * (32 / CB);
      // the S, T entries of row step k + 1 are read from shared memory
      // before the FMAs of step k (rows below 128 always: in bounds), so
      // their latency hides behind the FP64 instructions
      if (sz == 1) {
        double c0 = cn[0][g], c1 = cn[1][g];
#pragma unroll
        for (int k = 0; k < CB; ++k) {
          double d0 = 0.0, d1 = 0.0;
          if (k + 1 < CB) { d0 = cn[0][g + NG * (k + 1)]; d1 = cn[1][g + NG * (k + 1)]; }
          if (wg + NG * k >= li0) break;
          const int r = g + NG * k;
          const double v = fma(c1, pq0.y, fma(-c0, pq0.x, vals[k]));
          vals[k] = r < li0 ? v : vals[k];
          c0 = d0;
          c1 = d1;
        }
      } else {
        const double2 pq1 = s_PQ[1][t];
        double c0 = cn[0][g], c1 = cn[1][g], c2 = cn[2][g], c3 = cn[3][g];
#pragma unroll
        for (int k = 0; k < CB; ++k) {
          double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
          if (k + 1 < CB) {
            const int rn = g + NG * (k + 1);
            d0 = cn[0][rn]; d1 = cn[1][rn]; d2 = cn[2][rn]; d3 = cn[3][rn];
          }
          if (wg + NG * k >= li0) break;
          const int r = g + NG * k;
          const double v = fma(c3, pq1.y, fma(-c2, pq1.x, fma(c1, pq0.y, fma(-c0, pq0.x, vals[k]))));
          vals[k] = r < li0 ? v : vals[k];
          c0 = d0; c1 = d1; c2 = d2; c3 = d3;
        }
      }
#pragma unroll
      for (int k = 0; k < CB; ++k) {
        const int r = g + NG * k;
        if (r >= li0 && r < li0 + sz) vals[k] = s_W[r - li0][t];
      }
    }
  }

  // write back the solved tile columns and their augmented exponents / norms
  unsigned long long key = 0ull;
  if (tcol) {
    const bool wr = tips || s_act[pairs ? t / 2 : t];
#pragma unroll
    for (int k = 0; k < CB; ++k) {
      const int r = g + NG * k;
      if (r < h) {
        if (wr) Yt[(size_t)s_lc[t] * P.tb + r] = vals[k];
        key = max(key, abs_key(vals[k]));
      }
    }
  }
  // lanes lr, lr ^ CB, lr ^ 2CB, ... of a warp share the column
#pragma unroll
  for (int o = CB; o < 32; o <<= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o));
  if ((lr & 31) < CB && tcol && key) atomicMax(&s_key[t], key);
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

}  // namespace pevc

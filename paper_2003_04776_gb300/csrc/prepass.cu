// prepass.cu -- the pre-processing tasks of Section 5.2: infinity norms of
// all super-diagonal tiles of S and T, the column-segment norms needed by the
// robust diagonal solves, the finiteness check of every entry that is read,
// the eigenvalue pairs (alpha, beta) of the diagonal blocks (Section 2) and
// their power-of-two pre-scaling (Section 4, last paragraph).
#include "common.cuh"

namespace pevc {

__global__ void k_gather_subdiag(const double* __restrict__ S, int lds, int n, double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i + 1 < n) out[i] = S[(size_t)i * lds + i + 1];
}

cudaError_t launch_gather_subdiag(const double* S, int lds, int n, double* out, cudaStream_t s) {
  if (n < 2) return cudaSuccess;
  k_gather_subdiag<<<(n + 255) / 256, 256, 0, s>>>(S, lds, n, out);
  return cudaGetLastError();
}

__device__ __forceinline__ void block_reduce_max2(double& a, double& b, double* red) {
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) { red[w] = a; red[32 + w] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < nw; ++q) { a = fmax(a, red[q]); b = fmax(b, red[32 + q]); }
  }
}

// An upper bound of 2^-32 |x| from the key of |x| (finite): exact for
// |x| >= 2^-990, the smallest normal number below that.
__device__ __forceinline__ double scaled_down32(unsigned long long key) {
  const unsigned long long e = key >> 52;
  const unsigned long long b = e > 32 ? key - (32ull << 52) : (key ? 0x0010000000000000ull : 0ull);
  return __longlong_as_double((long long)b);
}

// One CTA per tile pair (k, l), k <= l.  Off-diagonal tiles: exponent bound
// of ||[S_kl T_kl]||_inf.  Diagonal tiles: tcS/tcT column-segment maxima.
// lfix >= 0: the tiles (k, lfix) of one column block, k = blockIdx.x.
__global__ void __launch_bounds__(128) k_tilenorms(Problem P, int lfix) {
  __shared__ double red[64];
  const long long x = blockIdx.x;
  int l = lfix, k = (int)x;
  if (lfix < 0) {
    l = (int)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
    while ((long long)l * (l + 1) / 2 > x) --l;
    while ((long long)(l + 1) * (l + 2) / 2 <= x) ++l;
    k = (int)(x - (long long)l * (l + 1) / 2);
  }
  const int rk0 = P.toff[k], hk = P.toff[k + 1] - rk0;
  const int cl0 = P.toff[l], hl = P.toff[l + 1] - cl0;
  const double* S = P.S;
  const double* T = P.T;
  bool finite = true;
  double amax = 0.0, rs = 0.0;
  if (k < l) {
    // integer keys for the maximum and the finiteness test; the row sums of
    // 2^-32 |x| (kept from overflowing) accumulate upper bounds formed on the
    // exponent field, so only the two additions use the FP64 pipe
    const int r = threadIdx.x;
    if (r < hk) {
      unsigned long long key = 0, bad = 0;
      double rs0 = 0.0, rs1 = 0.0;
#pragma unroll 8
      for (int c = 0; c < hl; ++c) {
        const unsigned long long ks = abs_key(S[(size_t)(cl0 + c) * P.lds + rk0 + r]);
        const unsigned long long kt = abs_key(T[(size_t)(cl0 + c) * P.ldt + rk0 + r]);
        bad |= (ks >= 0x7ff0000000000000ull) | (kt >= 0x7ff0000000000000ull);
        key = max(key, max(ks, kt));
        rs0 += scaled_down32(ks);
        rs1 += scaled_down32(kt);
      }
      finite = !bad;
      amax = __longlong_as_double((long long)key);
      rs = rs0 + rs1;
    }
  } else {
    const int c = threadIdx.x;
    if (c < hl) {
      const int gc = cl0 + c;
      const int bs = (P.blk[gc] == 2) ? gc - 1 : gc;
      const int last = (P.blk[gc] == 1) ? gc + 1 : gc;    // subdiagonal entry of a 2x2 block
      double ms = 0.0, mt = 0.0;
      for (int r = cl0; r <= last; ++r) {
        const double s = fabs(S[(size_t)gc * P.lds + r]);
        const double t = fabs(T[(size_t)gc * P.ldt + r]);
        finite = finite && isfinite(s) && isfinite(t);
        amax = fmax(amax, fmax(s, t));
        if (r < bs) { ms = fmax(ms, s); mt = fmax(mt, t); }
      }
      P.tcS[gc] = ms;
      P.tcT[gc] = mt;
    }
    // row sums of the quasi-triangular diagonal tile (row r reads S[r, r-1]
    // when r is the second row of a 2x2 block)
    const int r = threadIdx.x;
    if (r < hl) {
      const int gr = cl0 + r;
      const int c_first = (P.blk[gr] == 2) ? gr - 1 : gr;
      for (int gc = c_first; gc < cl0 + hl; ++gc) {
        rs += scaled_down32(abs_key(S[(size_t)gc * P.lds + gr]));
        if (gc >= gr) rs += scaled_down32(abs_key(T[(size_t)gc * P.ldt + gr]));
      }
    }
  }
  if (!finite) atomicOr(P.status, kStNonfinite);
  block_reduce_max2(amax, rs, red);
  if (threadIdx.x == 0) {
    if (isfinite(amax)) atomic_max_nonneg(P.gmax, amax);
    P.EA[k * P.M + l] = (rs > 0.0 && isfinite(rs)) ? exp_above(rs) + 33 : -(1 << 28);
  }
}

// Eigenvalue pair of the block starting at each diagonal position in
// [c_begin, c_end), plus the structural checks of a standardised real Schur
// form.  spec (may be null): the pre-scale was taken from the maximum of the
// column blocks seen so far; spec[0] receives that maximum and spec[1] (an
// int) the largest exponent bound of the pairs' coefficients, for the check
// against the final maximum.
__global__ void k_eigpairs(Problem P, int c_begin, int c_end, double* spec) {
  const int c = c_begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (spec && blockIdx.x == 0 && threadIdx.x == 0) spec[0] = *P.gmax;
  if (c >= c_end || P.blk[c] == 2) return;
  const double* S = P.S;
  const double* T = P.T;
  const int lds = P.lds, ldt = P.ldt;
  double a, b, beta;
  if (P.blk[c] == 0) {
    a = S[(size_t)c * lds + c];
    beta = T[(size_t)c * ldt + c];
    b = 0.0;
    if (signbit(beta)) { a = -a; beta = -beta; }
  } else {
    const double s11 = S[(size_t)c * lds + c], s21 = S[(size_t)c * lds + c + 1];
    const double s12 = S[(size_t)(c + 1) * lds + c], s22 = S[(size_t)(c + 1) * lds + c + 1];
    const double t1 = T[(size_t)c * ldt + c], t2 = T[(size_t)(c + 1) * ldt + c + 1];
    const double t12 = T[(size_t)(c + 1) * ldt + c], t21 = T[(size_t)c * ldt + c + 1];
    if (t12 != 0.0 || t21 != 0.0 || !(t1 > 0.0) || !(t2 > 0.0)) {
      atomicOr(P.status, kStNotSchur);
      return;
    }
    // det(S_jj - lambda diag(t1, t2)) = 0: lambda = mid +- sqrt(half^2 + prod)
    const double g1 = s11 / t1, g2 = s22 / t2;
    const double mid = 0.5 * (g1 + g2), half = 0.5 * (g1 - g2);
    const double prod = (s12 / t1) * (s21 / t2);
    const double negdisc = -(half * half + prod);
    if (!(negdisc > 0.0)) {
      atomicOr(P.status, isfinite(negdisc) ? kStNotSchur : kStNonfinite);
      return;
    }
    a = mid;
    b = sqrt(negdisc);
    beta = 1.0;
    if (!isfinite(a) || !isfinite(b)) {
      atomicOr(P.status, kStNonfinite);
      return;
    }
  }
  // pre-scaling of the pair so that max(|beta|, |a|+|b|) * max|S,T| <= 2^1000
  const double coef = fmax(fabs(beta), fabs(a) + fabs(b));
  const double gm = *P.gmax;
  if (spec && coef > 0.0) atomicMax(reinterpret_cast<int*>(spec + 1), exp_above(coef));
  if (coef > 0.0 && gm > 0.0) {
    const int k = exp_above(coef) + exp_above(gm) - kPrescaleExp;
    if (k > 0) { a = ldexp(a, -k); b = ldexp(b, -k); beta = ldexp(beta, -k); }
  }
  const int sz = (P.blk[c] == 1) ? 2 : 1;
  for (int r = c; r < c + sz; ++r) { P.ca[r] = a; P.cb[r] = b; P.cbeta[r] = beta; }
}

cudaError_t launch_prepass(const Problem& P, cudaStream_t s) {
  const long long tiles = (long long)P.M * (P.M + 1) / 2;
  if (tiles > 0) k_tilenorms<<<(unsigned)tiles, 128, 0, s>>>(P, -1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (P.n > 0) k_eigpairs<<<(P.n + 127) / 128, 128, 0, s>>>(P, 0, P.n, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_prepass_block(const Problem& P, int l, int c_begin, int c_end, double* spec, cudaStream_t s) {
  k_tilenorms<<<(unsigned)(l + 1), 128, 0, s>>>(P, l);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (c_end > c_begin) k_eigpairs<<<(c_end - c_begin + 127) / 128, 128, 0, s>>>(P, c_begin, c_end, spec);
  return cudaGetLastError();
}

// Augmented state before the first task: every tile column is zero
// (exponent kExpZero, norm 0) (what & 1); indefinite selected eigenvalues are
// flagged (what & 2).
__global__ void k_init_state(Problem P, int what) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)P.M * P.m;
  if ((what & 1) && idx < total) {
    P.ex[idx] = kExpZero;
    P.nrm[idx] = 0.0;
  }
  if ((what & 2) && idx < P.m) {
    const int c = P.ccol[idx];
    if (P.kind[idx] == 0 && P.ca[c] == 0.0 && P.cbeta[c] == 0.0) atomicOr(P.status, kStIndefinite);
  }
}

cudaError_t launch_init_state(const Problem& P, cudaStream_t s, int what) {
  const long long total = (long long)P.M * P.m > P.m ? (long long)P.M * P.m : P.m;
  if (total <= 0) return cudaSuccess;
  k_init_state<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(P, what);
  return cudaGetLastError();
}

}  // namespace pevc

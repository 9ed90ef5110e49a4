// common.cuh -- internal definitions of the pevc CUDA library (sm_103a).
//
// Robustness arithmetic of Section 4 of Kjelgaard Mikkelsen & Myllykoski
// (PPAM 2019): every stored tile column is an augmented column <alpha, x>
// with alpha = 2^-e kept as a signed 32-bit exponent e (Section 5), so the
// represented value is 2^e * x.  Omega = 2^1022.  All scale factors are
// powers of two, so applying them is exact up to underflow.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pevc.h"

namespace pevc {

constexpr int kOmegaExp = 1022;        // Omega = 2^1022
constexpr int kPrescaleExp = 1000;     // |beta| max|S|, (|a|+|b|) max|T| <= 2^1000
constexpr int kExpZero = -(1 << 29);   // exponent of a tile column that is still zero
constexpr int kMaxTile = 128;          // largest tile order
constexpr int kDiagChunk = 8;          // columns per diagonal-solve CTA (even: pairs stay whole)

// Device status bits (reduced to a PEVC_ERR_* value on the host).
constexpr unsigned kStNotSchur = 1u;
constexpr unsigned kStNonfinite = 2u;
constexpr unsigned kStIndefinite = 4u;
constexpr unsigned kStTimeout = 8u;

// FP64 instructions are scarce on this GPU (a warp instruction occupies a
// sub-partition's FP64 unit for tens of cycles), so exponent extraction,
// comparisons and maxima of non-negative values work on the IEEE-754 bit
// patterns with integer instructions.

// |x| as an ordered integer key (non-negative doubles order like their bits).
__device__ __forceinline__ unsigned long long abs_key(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// floor(log2 v) for the key a = abs_key(v) of a finite v != 0: the biased
// exponent field for normal numbers, the position of the leading mantissa
// bit for subnormals.
__device__ __forceinline__ int ilogb_key(unsigned long long a) {
  const int E = (int)(a >> 52);
  return E ? E - 1023 : (63 - __clzll((long long)a)) - 1074;
}

// Smallest E with |v| < 2^E for finite v != 0.
__device__ __forceinline__ int exp_above(double v) { return ilogb_key(abs_key(v)) + 1; }

// Larger of two non-negative doubles, by an unsigned maximum of their
// magnitude bit patterns (a signed comparison of the raw patterns would be
// compiled into an FP64 maximum, an instruction on the scarce FP64 pipe).
__device__ __forceinline__ double max_nonneg(double x, double y) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  const unsigned long long b = (unsigned long long)__double_as_longlong(y) & 0x7fffffffffffffffull;
  return __longlong_as_double((long long)(a > b ? a : b));
}

// ProtectUpdate (Section 4, property 2) on exponent bounds: y, t, x >= 0 and
// finite.  k >= 0 with 2^-k (y + t x) <= Omega.
__device__ __forceinline__ int protect_update(double y, double t, double x) {
  const unsigned long long yb = abs_key(y), tb = abs_key(t), xb = abs_key(x);
  int top = INT32_MIN / 4;
  if (yb) top = ilogb_key(yb) + 1;
  if (tb && xb) top = max(top, ilogb_key(tb) + ilogb_key(xb) + 2);
  int k = top + 1 - kOmegaExp;
  return k > 0 ? k : 0;
}

// Exponent upper bound |x| < 2^exp_ub(x) of a finite x, read from the high
// word's exponent field with 32-bit integer instructions (zero and
// subnormal x give -1022).  For a normal x it is ilogb(x) + 1.
__device__ __forceinline__ int exp_ub(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) - 1022; }

// ProtectUpdate on the exp_ub bounds (the block-step form): zero arguments
// count as 2^-1022, which can only raise k, and never does unless the other
// term is below 2^-1022 times Omega.
__device__ __forceinline__ int protect_update_ub(double y, double t, double x) {
  const int top = max(exp_ub(y), exp_ub(t) + exp_ub(x));
  const int k = top + 1 - kOmegaExp;
  return k > 0 ? k : 0;
}

// Same bound when t is already given as an exponent bound (t < 2^et).
__device__ __forceinline__ int protect_update_e(int ey_or_min, int etx_or_min) {
  int top = max(ey_or_min, etx_or_min);
  int k = top + 1 - kOmegaExp;
  return k > 0 ? k : 0;
}

// ProtectDivision (Section 4, property 1) for the numerator bound 2^sh * b
// and denominator magnitude t > 0: k >= 0 with 2^-k 2^sh b <= t Omega.
__device__ __forceinline__ int protect_division(double b, int sh, double t) {
  const unsigned long long bb = abs_key(b);
  if (!bb) return 0;
  int k = ilogb_key(bb) + 1 + sh - ilogb_key(abs_key(t)) - kOmegaExp;   // t >= 2^ilogb(t)
  return k > 0 ? k : 0;
}

// Complex quotient (pr + i pi) = (ar + i ai) / (br + i bi): Smith (1962),
// with Baudin & Smith's (2012) regrouping when the divisor-part ratio
// underflows to zero.
__device__ __forceinline__ void cdiv(double ar, double ai, double br, double bi,
                                     double& pr, double& pi) {
  if (fabs(br) >= fabs(bi)) {
    const double rho = bi / br;
    const double den = br + bi * rho;
    if (rho != 0.0) {
      pr = (ar + ai * rho) / den;
      pi = (ai - ar * rho) / den;
    } else {
      pr = (ar + bi * (ai / br)) / den;
      pi = (ai - bi * (ar / br)) / den;
    }
  } else {
    const double rho = br / bi;
    const double den = bi + br * rho;
    if (rho != 0.0) {
      pr = (ar * rho + ai) / den;
      pi = (ai * rho - ar) / den;
    } else {
      pr = (br * (ar / bi) + ai) / den;
      pi = (br * (ai / bi) - ar) / den;
    }
  }
}

// Complex reciprocal (pr + i pi) = 1 / (br + i bi): Smith's quotient above
// with the numerator 1, so that it takes two divisions instead of three (the
// second quotient is a product with the reciprocal of the denominator).
__device__ __forceinline__ void crecip(double br, double bi, double& pr, double& pi) {
  if (fabs(br) >= fabs(bi)) {
    const double rho = bi / br;
    const double inv = 1.0 / (br + bi * rho);
    pr = inv;
    pi = (rho != 0.0) ? -rho * inv : -(bi * inv) * inv;
  } else {
    const double rho = br / bi;
    const double inv = 1.0 / (bi + br * rho);
    pr = (rho != 0.0) ? rho * inv : (br * inv) * inv;
    pi = -inv;
  }
}

// (pr + i pi) = (ar + i ai) (br + i bi)
__device__ __forceinline__ void cmul(double ar, double ai, double br, double bi, double& pr, double& pi) {
  pr = fma(ar, br, -(ai * bi));
  pi = fma(ar, bi, ai * br);
}

__device__ __forceinline__ double cmag(double re, double im) { return fabs(re) + fabs(im); }

// x * 2^e, exact up to underflow/overflow like ldexp.  Normal results are
// formed by adding e to the exponent field with integer arithmetic (FP64
// instructions are scarce on this GPU); zero, subnormal and out-of-range
// cases take the library path.
__device__ __forceinline__ double pow2_scale(double x, int e) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  const int En = E + e;
  if (E != 0 && E != 0x7ff && En > 0 && En < 0x7ff) return __longlong_as_double(b + ((long long)e << 52));
  if (e == 0 || x == 0.0) return x;
  return ldexp(x, e);
}

// Branch-free fast paths of the two epilogue scalings (straight-line integer
// code, so that the independent elements of a block overlap their FP64
// latencies).  slow is set when an input is subnormal or a result leaves the
// normal range; the caller then recomputes with the exact helpers.
//   i64_scaled_fast: t * 2^e rounded to nearest (ties to even), |t| < 2^63
__device__ __forceinline__ double i64_scaled_fast(long long t, int e, bool& slow) {
  const unsigned long long sgn = (unsigned long long)t & (1ull << 63);
  const unsigned long long mag = t < 0 ? 0ull - (unsigned long long)t : (unsigned long long)t;
  const int lz = __clzll((long long)(mag | 1ull));
  const unsigned long long mm = mag << lz;
  unsigned long long mant = mm >> 11;
  const unsigned long long rest = mm & 0x7ffull;
  mant += (unsigned long long)((rest > 0x400ull) | ((rest == 0x400ull) & (unsigned)(mant & 1ull)));
  const unsigned long long carry = mant >> 53;
  mant >>= carry;
  const int E = 1086 - lz + e + (int)carry;
  slow |= (mag != 0) & ((E <= 0) | (E >= 2047));
  const unsigned long long bits = sgn | ((unsigned long long)(E & 0x7ff) << 52) | (mant & ((1ull << 52) - 1));
  return __longlong_as_double((long long)(mag ? bits : 0ull));
}
//   pow2_scale_fast: y * 2^s for a normal or zero y, on the two 32-bit
//   halves (a zero test of the whole magnitude would be compiled into an
//   FP64 comparison, an instruction on the scarce FP64 pipe)
__device__ __forceinline__ double pow2_scale_fast(double y, int sh, bool& slow) {
  const int hi = __double2hiint(y), lo = __double2loint(y);
  const int E = (hi >> 20) & 0x7ff;
  const int En = E + sh;
  const bool zs = E == 0;   // zero or subnormal
  slow |= (zs & (((hi & 0xfffff) | lo) != 0)) | (!zs & ((En <= 0) | (En >= 2047)));
  return zs ? y : __hiloint2double(hi + (sh << 20), lo);
}

// t * 2^e rounded to nearest (ties to even), for |t| < 2^63: the IEEE-754
// fields are assembled with integer instructions (a 64-bit integer to FP64
// conversion is a slow instruction on this GPU).  Results outside the normal
// range take the library path.
__device__ __forceinline__ double i64_scaled(long long t, int e) {
  if (t == 0) return 0.0;
  const unsigned long long sgn = t < 0 ? (1ull << 63) : 0ull;
  unsigned long long m = t < 0 ? 0ull - (unsigned long long)t : (unsigned long long)t;
  const int lz = __clzll((long long)m);
  m <<= lz;                                   // leading one at bit 63
  unsigned long long mant = m >> 11;          // 53 significant bits
  const unsigned long long rest = m & 0x7ffull;
  if (rest > 0x400ull || (rest == 0x400ull && (mant & 1ull))) ++mant;
  int E = 1023 + 63 - lz + e;
  if (mant >> 53) { mant >>= 1; ++E; }
  if (E <= 0 || E >= 2047) return ldexp((double)t, e);
  return __longlong_as_double((long long)(sgn | ((unsigned long long)E << 52) | (mant & ((1ull << 52) - 1))));
}

// Largest of non-negative doubles via their bit patterns (monotone for x >= 0).
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), __double_as_longlong(v));
}

// Packed index of tile (k, j), k <= j, in the upper triangle of tiles.
__host__ __device__ __forceinline__ long long tri_index(int k, int j) {
  return (long long)j * (j + 1) / 2 + k;
}

// Everything a kernel needs to know about one pencil and its workspace.
struct Problem {
  // inputs
  const double* S;
  const double* T;
  int lds, ldt, n;
  // structure (device copies of host-computed arrays)
  const signed char* blk;   // [n]  0 = 1x1, 1 = first row of 2x2, 2 = second row
  const int* toff;          // [M+1] row offsets of the tiles
  const int* cstart;        // [M+1] first output column of each column tile
  const int* ccol;          // [m]   diagonal position of each output column
  const signed char* kind;  // [m]   0 real, 1 Re of a pair, 2 Im of a pair
  int M, m, tb;             // tile count, output columns, tile storage order
  // eigenvalues per output column (pre-scaled)
  double* ca;
  double* cb;
  double* cbeta;
  // norms
  int* EA;                  // [M*M] ||[S_kl T_kl]||_inf < 2^EA[k*M+l], k <= l
  double* tcS;              // [n] max |S_rc| over rows r of c's tile above c's block
  double* tcT;              // [n]
  double* gmax;             // [1] max |entry| of S, T over what is read
  // augmented tiles
  double* Y;                // tiles (k <= j), tb x tb column-major each
  int* ex;                  // [M*m] exponent of column q in row tile k
  double* nrm;              // [M*m] max |stored| of column q in row tile k
  unsigned* status;         // device status bits
  // diagonal-kernel column chunks: real columns and complex pairs grouped
  // apart, so one CTA's pivot work is never divergent
  const int* dperm;         // [m] local column (within its column tile) at every position
  const int* dchunk_pos;    // first position of each chunk
  const int* dchunk_cnt;    // columns in each chunk
  const int* dchunk_first;  // [M+1] first chunk of each column tile
  int dchunk_max;           // most chunks in one column tile
};

__device__ __forceinline__ double* tile_ptr(const Problem& P, int k, int j) {
  return P.Y + tri_index(k, j) * (long long)P.tb * P.tb;
}

// Per-column consolidation + protection of the update of Y_kj (target P) by
// X = tile (i, j) whose exponents / norms are exX / nrmX (Algorithms 2 and 3):
// returns false when X'' is zero (nothing to do).  sY, sX shift the stored Y
// and X to the new common exponent enew.
__device__ __forceinline__ bool update_scales(const Problem& P, const int* exX, const double* nrmX,
                                              int k, int i, int q, int& sY, int& sX, int& enew,
                                              bool& yzero) {
  const int m = P.m;
  const int kd = P.kind[q];
  const int partner = (kd == 1) ? q + 1 : (kd == 2 ? q - 1 : q);
  const long long bk = (long long)k * m, bi = (long long)i * m;
  const double nY = max_nonneg(P.nrm[bk + q], P.nrm[bk + partner]);
  const double nX = max_nonneg(nrmX[bi + q], nrmX[bi + partner]);
  const int c0 = (kd == 2) ? P.ccol[q] - 1 : P.ccol[q];
  const double cB = max_nonneg(fabs(P.cbeta[c0]), fabs(P.ca[c0]) + fabs(P.cb[c0]));
  yzero = abs_key(nY) == 0;
  if (abs_key(nX) == 0 || abs_key(cB) == 0) return false;
  const int eY = P.ex[bk + q], eX = exX[bi + q];
  const int e0 = yzero ? eX : max(eY, eX);
  const int xb = exp_above(cB) + exp_above(nX) + eX - e0;          // ||X''|| < 2^xb at e0
  const int top_y = yzero ? INT32_MIN / 4 : exp_above(nY) + eY - e0;
  int kp = protect_update_e(top_y, P.EA[k * P.M + i] + xb);       // Algorithm 3
  const int kr = xb - kOmegaExp;                                   // Algorithm 2: ||X''|| <= Omega
  if (kr > kp) kp = kr;
  enew = e0 + kp;
  sY = yzero ? 0 : eY - enew;
  sX = eX - enew;
  return true;
}

// Per-launch CUDA-event timing on the solve's stream (host side).  Kinds:
// 0 update, 1 diagonal solve, 2 slicing of X, 3 everything else.
struct Profiler {
  bool on = false;
  int cap = 0, used = 0;
  cudaEvent_t* ev = nullptr;   // 2 * cap events
  int* kind = nullptr;
  double* flops = nullptr;
  int launches = 0;
  int pending_kind = 3;
  void reset() { used = 0; launches = 0; }
  void begin(cudaStream_t s) {
    ++launches;
    if (on && used < cap) cudaEventRecord(ev[2 * used], s);
  }
  void end(cudaStream_t s, int k, double f) {
    if (on && used < cap) {
      cudaEventRecord(ev[2 * used + 1], s);
      kind[used] = k;
      flops[used] = f;
      ++used;
    }
  }
};

// Diagonal-tile kernel modes.
constexpr int kDiagSolve = 0;     // kernel 3: tiles (i, j), j > i, right-hand side from Y
constexpr int kDiagTip = 1;       // kernel 1: tiles (j, j), unit tips, zero right-hand side
constexpr int kDiagTipCorr = 2;   // tiles (j, j) of a correction: zero tips, right-hand side from Y

// ---- launchers (one translation unit each) ----
cudaError_t launch_prepass(const Problem& P, cudaStream_t s);
// The pre-pass of one column block l (tiles (k, l), eigenvalues of the
// diagonal positions [c_begin, c_end)), for a solve whose inputs arrive by
// column blocks; spec: see k_eigpairs.
cudaError_t launch_prepass_block(const Problem& P, int l, int c_begin, int c_end, double* spec, cudaStream_t s);
cudaError_t launch_init_state(const Problem& P, cudaStream_t s, int what = 3);
cudaError_t launch_diag(const Problem& P, int i, int mode, cudaStream_t s);
// The tips (mode kDiagTip) of one diagonal tile j.
cudaError_t launch_diag_tile(const Problem& P, int j, int mode, cudaStream_t s);
cudaError_t launch_update_f64(const Problem& P, int i, int k_lo, int k_hi, cudaStream_t s);
cudaError_t launch_diag_residual_f64(const Problem& P, const double* Xsrc, const int* exX, const double* nrmX,
                                     cudaStream_t s);
cudaError_t launch_post(const Problem& P, double* V, int ldv, int32_t* scale, bool normalise,
                        cudaStream_t s);
cudaError_t launch_gather_subdiag(const double* S, int lds, int n, double* out, cudaStream_t s);
// back-transformation X = Z V (backtransform.cu)
int bt_handle(void** h, cudaStream_t s);
void bt_handle_destroy(void* h);
int bt_gemm(void* h, bool emulated, int n, int m, const double* Z, int ldz, const double* V, int ldv, double* X,
            int ldx);
cudaError_t launch_bt_normalise(double* X, int ldx, int n, int m, const signed char* kind, cudaStream_t s);
// left eigenvectors through the flipped transposed pencil (left.cu)
cudaError_t launch_flip_transpose(const double* A, int lda, int n, double* B, cudaStream_t s);
cudaError_t launch_flip_select(const int32_t* sel, int n, int32_t* out, cudaStream_t s);
cudaError_t launch_left_out(const double* Vp, int n, int m, const signed char* kind, const int32_t* scp, double* U,
                            int ldu, int32_t* scale, cudaStream_t s);

}  // namespace pevc

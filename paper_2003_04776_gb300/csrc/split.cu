// split.cu -- split-precision updates (Section 3, kernel 2) and the residual
// correction sweep.
//
// Slicing (Ozaki-style, exact): every row r of a tile [S_kl T_kl] is written
// as 2^e_r * sum_p s_p 2^(-7-8p) and every column q of X'' = [X D; -X B] as
// 2^F_q * sum_q t_q 2^(-7-8q), with integer slices |s|, |t| <= 128 that BF16
// holds exactly.  A slice product is an integer below 2^14, so the FP32
// tensor-core accumulation of K = 2 tb <= 256 terms is exact for the slice
// levels l = p + q <= 2 (the levels above contribute below 2^-24 of the
// result).  Each level has its own FP32 accumulator; the FP64 epilogue
// recombines them, applies the power-of-two scales of the augmented tiles
// (Algorithms 2 and 3 of Section 4: consolidation to a common exponent,
// ProtectUpdate) and writes the new column maxima (Section 4 norm
// bookkeeping).
//
// The power-of-two column scales of the augmented tiles are what makes the
// slices exact: X'' is scaled by 2^-F_q, a per-column exponent the augmented
// representation already carries.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>

#include "sched.cuh"
#include "split.cuh"

namespace pevc {

__device__ __forceinline__ void tile_pair(long long x, int& k, int& l) {
  int ll = (int)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
  while ((long long)ll * (ll + 1) / 2 > x) --ll;
  while ((long long)(ll + 1) * (ll + 2) / 2 <= x) ++ll;
  l = ll;
  k = (int)(x - (long long)ll * (ll + 1) / 2);
}

__device__ __forceinline__ int col_tile_of(const Problem& P, int q) {
  int lo = 0, hi = P.M - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.cstart[mid] <= q) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Slices of v relative to 2^e (|v| < 2^e): the balanced base-2^DB digits of
// the integer round(v 2^(B - e)), B = (DB - 1) + DB (NS - 1), so that
//   v 2^-e = sum_p d_p 2^(-(DB - 1) - DB p) + O(2^-B-1),   |d_p| <= 2^(DB - 1):
// DB = 8 for BF16 slices (|d| <= 128, 8 significant bits), DB = 4 for FP8
// E4M3 slices (|d| <= 8, 4 significant bits).  Integer arithmetic on the
// binary64 fields only (exact).
template <int NS, int DB = 8>
__device__ __forceinline__ void int_slices(double v, int e, int (&d)[NS]) {
  constexpr int B = (DB - 1) + DB * (NS - 1);
  constexpr long long R = 1ll << DB, H = R / 2;
  const long long bits = __double_as_longlong(v);
  const int E = (int)((bits >> 52) & 0x7ff);
  long long mant = bits & ((1ll << 52) - 1);
  if (E != 0) mant |= 1ll << 52;
  const int Eeff = E != 0 ? E : 1;
  const int sh = Eeff - 1075 + B - e;
  long long q;
  if (mant == 0) {
    q = 0;
  } else if (sh >= 0) {
    q = mant << sh;
  } else if (-sh >= 60) {
    q = 0;
  } else {
    const int r = -sh;
    q = (mant + (1ll << (r - 1))) >> r;
  }
  if (bits < 0) q = -q;
#pragma unroll
  for (int p = NS - 1; p >= 1; --p) {
    const int dp = (int)(((q + H) & (R - 1)) - H);
    d[p] = dp;
    q = (q - dp) >> DB;
  }
  d[0] = (int)q;
}

__device__ __forceinline__ __nv_bfloat16 small_int_bf16(int x) { return __float2bfloat16_rn((float)x); }

// The FP8 E4M3 byte of an integer |x| <= 15 (exact: 4 significant bits),
// assembled from the fields: sign, biased exponent (bias 7), 3 mantissa bits.
__device__ __forceinline__ unsigned char small_int_e4m3(int x) {
  const unsigned a = (unsigned)(x < 0 ? -x : x);
  if (a == 0) return 0;
  const int E = 31 - __clz((int)a);                   // floor(log2 a), 0..3
  const unsigned m = (a << (3 - E)) & 7u;
  return (unsigned char)(((x < 0) ? 0x80u : 0u) | ((unsigned)(E + 7) << 3) | m);
}

// The slice storage of the two formats: BF16 (8-bit digits) or FP8 E4M3
// (4-bit digits).
template <bool FP8>
struct Slice;
template <>
struct Slice<false> {
  using T = __nv_bfloat16;
  static constexpr int DB = 8;
  __device__ static T enc(int x) { return small_int_bf16(x); }
};
template <>
struct Slice<true> {
  using T = unsigned char;
  static constexpr int DB = 4;
  __device__ static T enc(int x) { return small_int_e4m3(x); }
};

// ---------------------------------------------------------------- A slices

// One CTA per half tile (64 rows of tile (k, l)), so that the tiles the
// resident CTAs hold between the row maxima and the slicing stay in L2.
constexpr int kSplitARows = 64;

template <int NS, bool FP8 = false>
__global__ void __launch_bounds__(256) k_split_A(Problem P, typename Slice<FP8>::T* __restrict__ As,
                                                 int* __restrict__ eA, int ns, int lfix) {
  using E = typename Slice<FP8>::T;
  int k = (int)(blockIdx.x >> 1), l = lfix;   // lfix >= 0: the tiles (k, lfix) of one column block
  if (lfix < 0) tile_pair(blockIdx.x >> 1, k, l);
  const int tb = P.tb, K2 = 2 * tb;
  const int rbase = (int)(blockIdx.x & 1) * kSplitARows;   // first local row of this half
  const int rk0 = P.toff[k], hk = P.toff[k + 1] - rk0;
  const int cl0 = P.toff[l], hl = P.toff[l + 1] - cl0;
  const long long tri = tri_index(k, l);
  __shared__ int s_e[kSplitARows];
  __shared__ unsigned long long s_part[4][kSplitARows];
  const double* S = P.S;
  const double* T = P.T;
  const int tid = threadIdx.x;
  if (rbase >= tb) return;
  // row maxima: four threads per row, each over a quarter of [S_kl T_kl]
  {
    const int rr = tid % kSplitARows, part = tid / kSplitARows;
    const int r = rbase + rr;
    unsigned long long key = 0;
    if (r < hk) {
      const int gr = rk0 + r;
      const bool isT = part >= 2;
      const int cb = (part & 1) * (tb / 2), ce = min(hl, cb + tb / 2);
      const int first = (k == l) ? (isT ? gr - cl0 : max(0, gr - cl0 - (P.blk[gr] == 2 ? 1 : 0))) : 0;
      const double* src = isT ? T : S;
      const int ld = isT ? P.ldt : P.lds;
#pragma unroll 4
      for (int c = max(cb, first); c < ce; ++c) key = max(key, abs_key(src[(size_t)(cl0 + c) * ld + gr]));
    }
    s_part[part][rr] = key;
  }
  __syncthreads();
  if (tid < kSplitARows) {
    const int r = rbase + tid;
    const unsigned long long key = max(max(s_part[0][tid], s_part[1][tid]), max(s_part[2][tid], s_part[3][tid]));
    const int e = key ? exp_above(__longlong_as_double((long long)key)) : 0;
    s_e[tid] = e;
    if (r < tb) eA[tri * tb + r] = e;
  }
  __syncthreads();
  const int groups = K2 / 8;
  const int rows = min(kSplitARows, tb - rbase);
  for (int item = tid; item < rows * groups; item += blockDim.x) {
    const int rr = item % rows, g = item / rows;
    const int r = rbase + rr;
    const int gr = rk0 + r;
    int sl[8][NS];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int kap = 8 * g + u;
      const bool isT = kap >= tb;
      const int c = isT ? kap - tb : kap;
      double v = 0.0;
      if (r < hk && c < hl) {
        const int gc = cl0 + c;
        bool ok = true;
        if (k == l) ok = isT ? (gc >= gr) : (gc >= gr || (gc == gr - 1 && P.blk[gr] == 2));
        if (ok) v = isT ? T[(size_t)gc * P.ldt + gr] : S[(size_t)gc * P.lds + gr];
      }
      int_slices<NS, Slice<FP8>::DB>(v, s_e[rr], sl[u]);
    }
#pragma unroll
    for (int p = 0; p < NS; ++p) {
      __align__(16) E pk[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) pk[u] = Slice<FP8>::enc(sl[u][p]);
      E* dst = As + ((tri * ns + p) * tb + r) * (long long)K2 + 8 * g;
      if (FP8) *reinterpret_cast<uint2*>(dst) = *reinterpret_cast<const uint2*>(pk);
      else *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(pk);
    }
  }
}

// ---------------------------------------------------------------- X slices

// X'' = [beta x ; -(alpha x)] of tile row i for output columns q >= q_begin,
// from the augmented tiles (Ysrc, exsrc, nrmsrc).  One warp per column.
template <int NS, bool FP8 = false>
__global__ void __launch_bounds__(256) k_split_X(Problem P, int i, int q_begin, const double* __restrict__ Ysrc,
                                                 const double* __restrict__ nrmsrc,
                                                 typename Slice<FP8>::T* __restrict__ Xs, int* __restrict__ F, int ns,
                                                 int mstride) {
  using T = typename Slice<FP8>::T;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = q_begin + blockIdx.x * 8 + warp;
  if (q >= P.m) return;
  const int tb = P.tb, K2 = 2 * tb, m = P.m;
  const int kd = P.kind[q];
  const int c0 = (kd == 2) ? P.ccol[q] - 1 : P.ccol[q];
  const double a = P.ca[c0], b = P.cb[c0], beta = P.cbeta[c0];
  const int j = col_tile_of(P, q);
  const int lq = q - P.cstart[j];
  const double* Xt = Ysrc + tri_index(i, j) * (long long)tb * tb;
  const long long base = (long long)i * m;
  double nx = nrmsrc[base + q];
  if (kd == 1) nx = fmax(nx, nrmsrc[base + q + 1]);
  if (kd == 2) nx = fmax(nx, nrmsrc[base + q - 1]);
  const int hi = P.toff[i + 1] - P.toff[i];
  constexpr int U = kMaxTile / 32;
  double top[U], bot[U];
  double mx = 0.0;
  unsigned long long key = 0;
  const int g = (nx > 0.0) ? exp_above(nx) : 0;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int kap = lane + 32 * u;
    double own = 0.0, oth = 0.0;
    if (nx > 0.0 && kap < hi) {
      own = pow2_scale(Xt[(size_t)lq * tb + kap], -g);
      if (kd == 1) oth = pow2_scale(Xt[(size_t)(lq + 1) * tb + kap], -g);
      if (kd == 2) oth = pow2_scale(Xt[(size_t)(lq - 1) * tb + kap], -g);
    }
    top[u] = beta * own;
    if (kd == 0) bot[u] = -(a * own);
    else if (kd == 1) bot[u] = -(a * own - b * oth);     // own = Re x, oth = Im x
    else bot[u] = -(b * oth + a * own);                 // own = Im x, oth = Re x
    key = max(key, max(abs_key(top[u]), abs_key(bot[u])));
  }
  for (int o = 16; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o));
  mx = __longlong_as_double((long long)key);
  const int f = (mx > 0.0) ? exp_above(mx) : 0;
  if (lane == 0) F[q] = (mx > 0.0) ? g + f : kExpZero;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int kap = lane + 32 * u;
    if (kap >= tb) continue;
    int st[NS], sb[NS];
    int_slices<NS, Slice<FP8>::DB>(top[u], f, st);
    int_slices<NS, Slice<FP8>::DB>(bot[u], f, sb);
#pragma unroll
    for (int p = 0; p < NS; ++p) {
      T* xrow = Xs + ((long long)p * mstride + q) * K2;
      xrow[kap] = Slice<FP8>::enc(st[p]);
      xrow[tb + kap] = Slice<FP8>::enc(sb[p]);
    }
  }
}

// ------------------------------------------------------------- the update

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldmatrix_x4(unsigned (&r)[4], const void* smem) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// D = A B + C for a 16x32 E4M3 A (row) and a 32x8 E4M3 B (col), FP32
// accumulators: four E4M3 values per register, the fragment layout of
// mma.m16n8k16 with each 16-bit element replaced by two consecutive 8-bit
// ones (so ldmatrix of the bytes as 16-bit pairs gives the fragments).
__device__ __forceinline__ void mma_fp8(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int kSplitRows = 128;
constexpr int kSplitCols = 32;

// K chunk per pipeline stage (elements): BF16 32 for up to 3 slices, 16 for 5
// (so that two CTAs fit in shared memory and one CTA's epilogue overlaps the
// other's MMAs); FP8 32 (one K step of the m16n8k32 MMA).
template <int NS, bool FP8 = false>
__host__ __device__ constexpr int split_kc() { return FP8 ? 32 : (NS >= 5 ? 16 : 32); }
// padded smem row (elements): 16 bytes more, so ldmatrix is conflict-free
template <int NS, bool FP8 = false>
__host__ __device__ constexpr int split_ld() { return split_kc<NS, FP8>() + (FP8 ? 16 : 8); }

template <int NS, bool FP8 = false>
constexpr int split_smem_bytes() {
  return 2 * NS * (kSplitRows + kSplitCols) * split_ld<NS, FP8>() * (FP8 ? 1 : 2);
}

// Y_kj <- 2^sY Y_kj - 2^sX [S_ki T_ki] X''_ij for k_lo <= k < k_lo + gridDim.y, j >= i.
template <int NS, int L, bool FP8 = false>
__global__ void __launch_bounds__(256, 2) k_update_split(Problem P, int i, int k_lo, const int* __restrict__ exX,
                                                         const double* __restrict__ nrmX,
                                                         const typename Slice<FP8>::T* __restrict__ As,
                                                         const int* __restrict__ eA,
                                                         const typename Slice<FP8>::T* __restrict__ Xs,
                                                         const int* __restrict__ F, int ns, int mstride) {
  using T = typename Slice<FP8>::T;
  constexpr int DB = Slice<FP8>::DB;                  // bits per digit
  constexpr int E16 = 16 / (int)sizeof(T);            // elements per 16 bytes
  constexpr int KSTEP = FP8 ? 32 : 16;                // K of one mma.sync
  constexpr int KC = split_kc<NS, FP8>();
  constexpr int LD = split_ld<NS, FP8>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sA = reinterpret_cast<T*>(smem_raw);             // [2][NS][128][LD]
  T* sB = sA + 2 * NS * kSplitRows * LD;              // [2][NS][32][LD]
  const int tb = P.tb, K2 = 2 * tb;
  const int nsub = tb / kSplitCols;
  const int j = i + (int)blockIdx.x / nsub;
  const int sub = (int)blockIdx.x % nsub;
  const int k = k_lo + (int)blockIdx.y;
  const int cs = P.cstart[j], ce = P.cstart[j + 1];
  const int c0 = cs + sub * kSplitCols;
  if (c0 >= ce) return;
  const int nc = min(kSplitCols, ce - c0);
  const int rk0 = P.toff[k], hk = P.toff[k + 1] - rk0;
  double* Yt = tile_ptr(P, k, j);
  const long long tri = tri_index(k, i);
  const int tid = threadIdx.x;

  __shared__ int s_sY[kSplitCols], s_sc[kSplitCols], s_e[kSplitCols], s_on[kSplitCols], s_yz[kSplitCols];
  __shared__ unsigned long long s_key[kSplitCols];
  __shared__ int s_eA[kSplitRows];
  __shared__ int s_any;
  if (tid == 0) s_any = 0;
  __syncthreads();
  if (tid < kSplitCols) {
    int on = 0, sY = 0, sX = 0, en = 0;
    bool yz = true;
    if (tid < nc) {
      const int q = c0 + tid;
      on = update_scales(P, exX, nrmX, k, i, q, sY, sX, en, yz) ? 1 : 0;
      if (on && F[q] == kExpZero) on = 0;
      s_sc[tid] = on ? F[q] - 2 * (DB - 1) - DB * (L - 1) + sX : 0;
    }
    s_on[tid] = on;
    s_sY[tid] = sY;
    s_e[tid] = en;
    s_yz[tid] = yz ? 1 : 0;
    s_key[tid] = 0ull;
    if (on) atomicOr(&s_any, 1);
  }
  if (tid < kSplitRows) s_eA[tid] = (tid < tb) ? eA[tri * tb + tid] : 0;
  __syncthreads();
  if (!s_any) return;

  // slices are stored K-contiguous: [slice][row or column][K]
  const T* Abase = As + tri * ns * (long long)tb * K2;
  auto load_stage = [&](int st, int kb) {
    T* a_dst = sA + st * NS * kSplitRows * LD;
    T* b_dst = sB + st * NS * kSplitCols * LD;
    constexpr int chunks = KC / E16;                      // 16-byte pieces per row
    for (int idx = tid; idx < NS * kSplitRows * chunks; idx += 256) {
      const int c16 = idx % chunks, r = (idx / chunks) % kSplitRows, p = idx / (chunks * kSplitRows);
      const bool valid = r < tb;
      const T* src = Abase + ((long long)p * tb + (valid ? r : 0)) * K2 + kb + E16 * c16;
      cp_async16(a_dst + (p * kSplitRows + r) * LD + E16 * c16, src, valid);
    }
    for (int idx = tid; idx < NS * kSplitCols * chunks; idx += 256) {
      const int c16 = idx % chunks, col = (idx / chunks) % kSplitCols, p = idx / (chunks * kSplitCols);
      const bool valid = col < nc;
      const T* src = Xs + ((long long)p * mstride + c0 + (valid ? col : 0)) * K2 + kb + E16 * c16;
      cp_async16(b_dst + (p * kSplitCols + col) * LD + E16 * c16, src, valid);
    }
  };

  const int warp = tid >> 5, lane = tid & 31;
  const int wr = warp & 3, wc = warp >> 2;
  float acc[L][2][2][4];
#pragma unroll
  for (int s = 0; s < L; ++s)
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[s][a][b][e] = 0.0f;

  const int nchunks = K2 / KC;
  load_stage(0, 0);
  cp_async_commit();
  for (int ch = 0; ch < nchunks; ++ch) {
    const int st = ch & 1;
    if (ch + 1 < nchunks) load_stage(st ^ 1, (ch + 1) * KC);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const T* a_s = sA + st * NS * kSplitRows * LD;
    const T* b_s = sB + st * NS * kSplitCols * LD;
#pragma unroll
    for (int kk = 0; kk < KC; kk += KSTEP) {
      unsigned bf[NS][4];
#pragma unroll
      for (int q = 0; q < NS; ++q)
        ldmatrix_x4(bf[q], b_s + (q * kSplitCols + 16 * wc + (lane & 7) + ((lane >> 4) << 3)) * LD + kk +
                               ((lane >> 3) & 1) * E16);
#pragma unroll
      for (int p = 0; p < NS; ++p) {
        unsigned af[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
          ldmatrix_x4(af[mt], a_s + (p * kSplitRows + 32 * wr + 16 * mt + (lane & 15)) * LD + kk + (lane >> 4) * E16);
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          if (p + q < L) {
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
              if (FP8) {
                mma_fp8(acc[p + q][mt][0], af[mt], bf[q][0], bf[q][1]);
                mma_fp8(acc[p + q][mt][1], af[mt], bf[q][2], bf[q][3]);
              } else {
                mma_bf16(acc[p + q][mt][0], af[mt], bf[q][0], bf[q][1]);
                mma_bf16(acc[p + q][mt][1], af[mt], bf[q][2], bf[q][3]);
              }
            }
          }
        }
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();

  // epilogue: recombine the (integer-valued) levels exactly as one integer,
  // one conversion to FP64, power-of-two scales by exponent arithmetic, one
  // FP64 subtraction per element; column maxima by integer keys
  const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int col = 16 * wc + 8 * nt + 2 * t4 + e;
      const bool con = col < nc && s_on[col];
      unsigned long long key = 0;
      if (con) {
        const int sY = s_sY[col], sc = s_sc[col];
        const bool yz = s_yz[col] != 0;
        double* ycol = Yt + (size_t)(c0 + col - cs) * tb;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int row = 32 * wr + 16 * mt + g + 8 * h;
            if (row < hk) {
              long long t = 0;
#pragma unroll
              for (int s = 0; s < L; ++s) t = (t << DB) + (long long)__float2int_rn(acc[s][mt][nt][2 * h + e]);
              const double prod = i64_scaled(t, s_eA[row] + sc);
              const double yold = yz ? 0.0 : pow2_scale(ycol[row], sY);
              const double ynew = yold - prod;
              ycol[row] = ynew;
              key = max(key, abs_key(ynew));
            }
          }
      }
      // reduce over the 8 lanes (g) that share this column
      key = max(key, __shfl_xor_sync(0xffffffffu, key, 4));
      key = max(key, __shfl_xor_sync(0xffffffffu, key, 8));
      key = max(key, __shfl_xor_sync(0xffffffffu, key, 16));
      if (con && g == 0 && key) atomicMax(&s_key[col], key);
    }
  __syncthreads();
  if (tid < nc && s_on[tid]) {
    const long long idx = (long long)k * P.m + c0 + tid;
    P.nrm[idx] = __longlong_as_double((long long)s_key[tid]);
    P.ex[idx] = s_e[tid];
  }
}

// V (first pass) += delta (correction), per tile column, at a common exponent.
__global__ void __launch_bounds__(256) k_combine(Problem P, const double* __restrict__ Y2,
                                                 const int* __restrict__ ex2, const double* __restrict__ nrm2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.y * 8 + warp;
  const int k = blockIdx.x;
  if (q >= P.m) return;
  const int j = col_tile_of(P, q);
  if (k > j) return;
  const int m = P.m, tb = P.tb;
  const int kd = P.kind[q];
  const int partner = (kd == 1) ? q + 1 : (kd == 2 ? q - 1 : q);
  const long long idx = (long long)k * m + q;
  const long long pidx = (long long)k * m + partner;
  const double n1 = fmax(P.nrm[idx], P.nrm[pidx]);
  const double n2 = fmax(nrm2[idx], nrm2[pidx]);
  if (!(n2 > 0.0)) return;
  const int lq = q - P.cstart[j];
  double* Vt = tile_ptr(P, k, j) + (size_t)lq * tb;
  const double* Dt = Y2 + tri_index(k, j) * (long long)tb * tb + (size_t)lq * tb;
  const int h = P.toff[k + 1] - P.toff[k];
  const int e1 = P.ex[idx], e2 = ex2[idx];
  const int e = (n1 > 0.0) ? max(e1, e2) + 1 : e2;
  double mx = 0.0;
  for (int r = lane; r < h; r += 32) {
    const double v = (n1 > 0.0 ? pow2_scale(Vt[r], e1 - e) : 0.0) + pow2_scale(Dt[r], e2 - e);
    Vt[r] = v;
    mx = fmax(mx, fabs(v));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    P.nrm[idx] = mx;
    P.ex[idx] = e;
  }
}

constexpr int kSweepBig = 1 << 20;   // a sweep that changed a column beyond measure

// Convergence of the correction sweeps: how much the sweep just made
// (V <- V + delta) changed each eigenvector as returned, i.e. normalised by
// its largest entry V(m).  To first order that change is
//     (delta - g V) / V(m),   g = delta(m) / V(m),
// so the part of delta along V itself -- large when an error made near the
// bottom of a column grew upward with the eigenvector's own growth -- does
// not count, as it does not change the normalised vector.  A pair's complex
// vector is measured as one (complex g).  Values are taken relative to 2^E,
// E the binary exponent of the column's largest tile maximum; the maximum
// over columns of floor(log2 max_i |change(i)|) into *out (which starts below
// any value).  One warp per real eigenvector or pair.
__global__ void __launch_bounds__(256) k_sweep_change(Problem P, const double* __restrict__ Y2,
                                                      const int* __restrict__ ex2, int* __restrict__ out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.x * 8 + warp;
  if (q >= P.m) return;
  const int kd = P.kind[q];
  if (kd == 2) return;                       // the pair's first column measures both
  const bool pr = kd == 1;
  const int j = col_tile_of(P, q);
  const int lq = q - P.cstart[j], tb = P.tb, m = P.m;
  // the tile with the largest entry (per-tile maxima at their exponents)
  int E = INT32_MIN, ks = 0;
  for (int k = lane; k <= j; k += 32) {
    const long long idx = (long long)k * m + q;
    const unsigned long long k0 = abs_key(P.nrm[idx]), k1 = pr ? abs_key(P.nrm[idx + 1]) : 0ull;
    int e = INT32_MIN;
    if (k0) e = P.ex[idx] + ilogb_key(k0);
    if (k1) e = max(e, P.ex[idx + 1] + ilogb_key(k1));
    if (e > E) { E = e; ks = k; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const int e2 = __shfl_xor_sync(0xffffffffu, E, o), k2 = __shfl_xor_sync(0xffffffffu, ks, o);
    if (e2 > E || (e2 == E && k2 < ks)) { E = e2; ks = k2; }
  }
  if (E == INT32_MIN) return;                // V is zero: nothing to measure
  // V and delta of column c at tile k, row r, relative to 2^E
  auto vat = [&](int c, int k, int r) {
    return pow2_scale(tile_ptr(P, k, j)[(size_t)(lq + c) * tb + r], P.ex[(long long)k * m + q + c] - E);
  };
  auto dat = [&](int c, int k, int r) {
    const double* Dt = Y2 + tri_index(k, j) * (long long)tb * tb;
    return pow2_scale(Dt[(size_t)(lq + c) * tb + r], ex2[(long long)k * m + q + c] - E);
  };
  // the largest entry of that tile (modulus bound |Re| + |Im| for a pair)
  const int hs = P.toff[ks + 1] - P.toff[ks];
  unsigned long long best = 0;
  int rm = 0;
  for (int r = lane; r < hs; r += 32) {
    const double x = pr ? cmag(vat(0, ks, r), vat(1, ks, r)) : fabs(vat(0, ks, r));
    const unsigned long long kx = abs_key(x);
    if (kx > best) { best = kx; rm = r; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long b2 = __shfl_xor_sync(0xffffffffu, best, o);
    const int r2 = __shfl_xor_sync(0xffffffffu, rm, o);
    if (b2 > best || (b2 == best && r2 < rm)) { best = b2; rm = r2; }
  }
  if (!best) return;
  // g = delta(m) / V(m)
  double gr, gi = 0.0;
  double vmr = vat(0, ks, rm), vmi = pr ? vat(1, ks, rm) : 0.0;
  const double dmr = dat(0, ks, rm), dmi = pr ? dat(1, ks, rm) : 0.0;
  if (!pr) {
    gr = dmr / vmr;
  } else {
    const double den = vmr * vmr + vmi * vmi;
    gr = (dmr * vmr + dmi * vmi) / den;
    gi = (dmi * vmr - dmr * vmi) / den;
  }
  // max_i |delta(i) - g V(i)| over the column's tiles, relative to |V(m)|
  double mx = 0.0;
  for (int k = 0; k <= j; ++k) {
    const int h = P.toff[k + 1] - P.toff[k];
    for (int r = lane; r < h; r += 32) {
      const double vr = vat(0, k, r), dr = dat(0, k, r);
      double c;
      if (!pr) {
        c = fabs(fma(-gr, vr, dr));
      } else {
        const double vi = vat(1, k, r), di = dat(1, k, r);
        c = cmag(dr - (gr * vr - gi * vi), di - (gr * vi + gi * vr));
      }
      mx = fmax(mx, c);
    }
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0 && mx > 0.0) {
    const double vm = pr ? cmag(vmr, vmi) : fabs(vmr);
    const double rel = mx / vm;
    const unsigned long long kr = abs_key(rel);
    atomicMax(out, (rel < 0x1p1000) ? ilogb_key(kr) : kSweepBig);   // NaN or huge: count as large
  }
}

// ------------------------------------------------------------------ host

int split_alloc(SplitWorkspace& w, int n_max, int tb, int Mmax, int prec) {
  w.tb = tb;
  w.n_max = std::max(n_max, 1);
  w.Mmax = Mmax;
  w.ns = kMaxSlices;
  w.tiles = (size_t)Mmax * (Mmax + 1) / 2;
  auto al = [](void** p, size_t bytes) { return cudaMalloc(p, bytes > 0 ? bytes : 16); };
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = al((void**)&w.As, w.tiles * w.ns * (size_t)tb * 2 * tb * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = al((void**)&w.eA, w.tiles * (size_t)tb * sizeof(int));
  if (e == cudaSuccess) e = al((void**)&w.Xs, (size_t)w.ns * w.n_max * 2 * tb * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = al((void**)&w.F, (size_t)w.n_max * sizeof(int));
  if (e == cudaSuccess) e = al((void**)&w.d_sweep, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&w.h_sweep, sizeof(int));
  if (e == cudaSuccess) e = al((void**)&w.Y2, w.tiles * (size_t)tb * tb * sizeof(double));
  if (e == cudaSuccess) e = al((void**)&w.ex2, (size_t)Mmax * w.n_max * sizeof(int));
  if (e == cudaSuccess) e = al((void**)&w.nrm2, (size_t)Mmax * w.n_max * sizeof(double));
  w.fp8 = prec == PEVC_SPLIT_FP8X4;
  if (w.fp8) {
    if (e == cudaSuccess) e = al((void**)&w.As8, w.tiles * 4 * (size_t)tb * 2 * tb);
    if (e == cudaSuccess) e = al((void**)&w.Xs8, (size_t)4 * w.n_max * 2 * tb);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_update_split<4, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               split_smem_bytes<4, true>());
  }
  if (e == cudaSuccess) {
    cudaError_t a1 = cudaFuncSetAttribute(k_update_split<3, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          split_smem_bytes<3>());
    cudaError_t a2 = cudaFuncSetAttribute(k_update_split<5, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          split_smem_bytes<5>());
    e = (a1 != cudaSuccess) ? a1 : a2;
  }
  w.max_chunks = w.n_max / 48 + Mmax + 1;
  if (e == cudaSuccess) e = al((void**)&w.chunk_c0_48, (size_t)w.max_chunks * sizeof(int));
  if (e == cudaSuccess) e = al((void**)&w.chunk_j_48, (size_t)w.max_chunks * sizeof(int));
  if (e == cudaSuccess) e = al((void**)&w.chunk_c0_64, (size_t)w.max_chunks * sizeof(int));
  if (e == cudaSuccess) e = al((void**)&w.chunk_j_64, (size_t)w.max_chunks * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&w.h_chunk_first48, (size_t)(Mmax + 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&w.h_chunk_first64, (size_t)(Mmax + 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&w.h_chunks, (size_t)4 * w.max_chunks * sizeof(int));
  if (e == cudaSuccess) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&w.nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  if (e == cudaSuccess && update_tc_setup() != 0) e = cudaErrorInvalidValue;
  if (e == cudaSuccess && make_tensor_maps(w) != 0) e = cudaErrorInvalidValue;
  {
    // update kernel for tiles of order 128: tcgen05 (default) or mma.sync
    // (PEVC_UPDATE_KERNEL=mma); other tile orders always take mma.sync
    const char* sel = getenv("PEVC_UPDATE_KERNEL");
    w.use_tc = !(sel && sel[0] == 'm');
  }
  w.on = e == cudaSuccess;
  if (e != cudaSuccess) {
    split_free(w);
    return e == cudaErrorMemoryAllocation ? PEVC_ERR_NOMEM : PEVC_ERR_CUDA;
  }
  return 0;
}

void split_free(SplitWorkspace& w) {
  void* ptrs[] = {w.As, w.eA, w.Xs, w.F, w.d_sweep, w.Y2, w.ex2, w.nrm2, w.chunk_c0_48, w.chunk_j_48, w.chunk_c0_64, w.chunk_j_64,
                  w.As8, w.Xs8};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  void* hp[] = {w.h_chunk_first48, w.h_chunk_first64, w.h_chunks, w.h_sweep};
  for (void* p : hp)
    if (p) cudaFreeHost(p);
  w.chunk_c0_48 = w.chunk_j_48 = w.chunk_c0_64 = w.chunk_j_64 = nullptr;
  w.h_chunk_first48 = w.h_chunk_first64 = w.h_chunks = nullptr;
  w.d_sweep = w.h_sweep = nullptr;
  w.As = nullptr;
  w.As8 = nullptr;
  w.Xs8 = nullptr;
  w.eA = nullptr;
  w.Xs = nullptr;
  w.F = nullptr;
  w.Y2 = nullptr;
  w.ex2 = nullptr;
  w.nrm2 = nullptr;
  w.on = false;
}

constexpr int kMaxSweeps = 6;      // adaptive correction sweeps: at most
constexpr int kSweepTarget = -30;  // stop once the predicted error is below 2^-30 of V

SplitConfig split_config(int prec, bool correction) {
  SplitConfig c;
  if (prec == PEVC_SPLIT_BF16X5) {
    c.ns1 = 5;
    c.levels1 = 5;
    c.correction = false;
  } else if (prec == PEVC_SPLIT_FP8X4) {
    // four FP8 E4M3 slices of 4-bit digits (about 15 bits) and the levels
    // p + q < 4 (10 products); the residual of the correction sweeps in
    // BF16x5.  A sweep multiplies the error by about the pass's own relative
    // error (2^-15 times the substitution's growth, measured 1/30 to 1/200),
    // so one sweep leaves errors up to 1e-5 on pencils of order 1000: the
    // sweeps repeat (iterative refinement) until the predicted error is
    // below 2^kSweepTarget, at most kMaxSweeps times
    c.ns1 = 4;
    c.levels1 = 4;
    c.fp8 = true;
    c.correction = correction;
    c.sweeps = kMaxSweeps;
    c.adaptive = true;
  } else {
    c.ns1 = 3;
    c.levels1 = 3;
    c.correction = correction;
  }
  c.ns_res = 5;
  c.levels_res = 5;
  // tuning override: a fixed sweep count (1 to kMaxSweeps)
  if (const char* sw = getenv("PEVC_SWEEPS")) {
    c.sweeps = std::min(std::max(atoi(sw), 1), kMaxSweeps);
    c.adaptive = false;
  }
  return c;
}

namespace {

int products(int ns, int levels) {
  int c = 0;
  for (int p = 0; p < ns; ++p)
    for (int q = 0; q < ns; ++q)
      if (p + q < levels) ++c;
  return c;
}

cudaError_t launch_split_A(const Problem& P, SplitWorkspace& w, int ns, cudaStream_t s) {
  const long long tiles = (long long)P.M * (P.M + 1) / 2;
  if (tiles <= 0) return cudaSuccess;
  if (ns == 5) k_split_A<5><<<(unsigned)(2 * tiles), 256, 0, s>>>(P, w.As, w.eA, w.ns, -1);
  else k_split_A<3><<<(unsigned)(2 * tiles), 256, 0, s>>>(P, w.As, w.eA, w.ns, -1);
  return cudaGetLastError();
}

cudaError_t split_A_block(const Problem& P, SplitWorkspace& w, int l, int ns, cudaStream_t s) {
  if (ns == 5) k_split_A<5><<<(unsigned)(2 * (l + 1)), 256, 0, s>>>(P, w.As, w.eA, w.ns, l);
  else k_split_A<3><<<(unsigned)(2 * (l + 1)), 256, 0, s>>>(P, w.As, w.eA, w.ns, l);
  return cudaGetLastError();
}

cudaError_t launch_split_X(const Problem& P, SplitWorkspace& w, int i, int q_begin, const double* Ysrc,
                           const double* nrmsrc, int ns, cudaStream_t s) {
  const int cols = P.m - q_begin;
  if (cols <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((cols + 7) / 8);
  if (ns == 5) k_split_X<5><<<blocks, 256, 0, s>>>(P, i, q_begin, Ysrc, nrmsrc, w.Xs, w.F, w.ns, w.n_max);
  else k_split_X<3><<<blocks, 256, 0, s>>>(P, i, q_begin, Ysrc, nrmsrc, w.Xs, w.F, w.ns, w.n_max);
  return cudaGetLastError();
}

// The FP8 E4M3 slices (four 4-bit digits) of [S T] and of X'', and the
// update from them: tcgen05 kind::f8f6f4 for tiles of order 128, else
// mma.sync m16n8k32.
cudaError_t launch_split_A8(const Problem& P, SplitWorkspace& w, cudaStream_t s) {
  const long long tiles = (long long)P.M * (P.M + 1) / 2;
  if (tiles <= 0) return cudaSuccess;
  k_split_A<4, true><<<(unsigned)(2 * tiles), 256, 0, s>>>(P, w.As8, w.eA, 4, -1);
  return cudaGetLastError();
}

cudaError_t launch_split_X8(const Problem& P, SplitWorkspace& w, int i, int q_begin, const double* Ysrc,
                            const double* nrmsrc, cudaStream_t s) {
  const int cols = P.m - q_begin;
  if (cols <= 0) return cudaSuccess;
  k_split_X<4, true><<<(unsigned)((cols + 7) / 8), 256, 0, s>>>(P, i, q_begin, Ysrc, nrmsrc, w.Xs8, w.F, 4, w.n_max);
  return cudaGetLastError();
}

// ftz: a correction sweep's update (products below the normal range flushed,
// see update_tc.cu)
cudaError_t launch_update_split8(const Problem& P, SplitWorkspace& w, int i, int k_lo, int k_hi, const int* exX,
                                 const double* nrmX, cudaStream_t s, bool ftz = false) {
  if (k_hi <= k_lo) return cudaSuccess;
  if (w.use_tc && w.tc_ok) return launch_update_tc(P, w, i, k_lo, k_hi, exX, nrmX, 4, 4, true, s, ftz);
  const int nsub = P.tb / kSplitCols;
  dim3 grid((P.M - i) * nsub, k_hi - k_lo);
  k_update_split<4, 4, true><<<grid, 256, split_smem_bytes<4, true>(), s>>>(P, i, k_lo, exX, nrmX, w.As8, w.eA,
                                                                            w.Xs8, w.F, 4, w.n_max);
  return cudaGetLastError();
}

cudaError_t launch_update_split(const Problem& P, SplitWorkspace& w, int i, int k_lo, int k_hi, const int* exX,
                                const double* nrmX, int ns, int levels, cudaStream_t s, bool ftz = false) {
  if (k_hi <= k_lo) return cudaSuccess;
  if (w.use_tc && w.tc_ok) return launch_update_tc(P, w, i, k_lo, k_hi, exX, nrmX, ns, levels, false, s, ftz);
  const int nsub = P.tb / kSplitCols;
  dim3 grid((P.M - i) * nsub, k_hi - k_lo);
  if (ns == 5 && levels == 5)
    k_update_split<5, 5><<<grid, 256, split_smem_bytes<5>(), s>>>(P, i, k_lo, exX, nrmX, w.As, w.eA, w.Xs, w.F,
                                                                  w.ns, w.n_max);
  else
    k_update_split<3, 3><<<grid, 256, split_smem_bytes<3>(), s>>>(P, i, k_lo, exX, nrmX, w.As, w.eA, w.Xs, w.F,
                                                                  w.ns, w.n_max);
  return cudaGetLastError();
}


// One bottom-up pass of the task graph over the augmented tiles of P: tips
// (or tip corrections), then per block row the diagonal solves and the sliced
// updates of everything above, walked with lookahead (sched.cuh).
struct SplitOps : StageOps {
  const Problem& P;
  SplitWorkspace& w;
  const HostStructure& hs;
  int tip_mode, ns, levels, prods;
  Profiler& prof;
  bool fp8;   // FP8 E4M3 slices (four 4-bit digits), else BF16
  SplitOps(const Problem& P_, SplitWorkspace& w_, const HostStructure& hs_, int tip_mode_, int ns_, int levels_,
           Profiler& prof_, bool fp8_ = false)
      : P(P_), w(w_), hs(hs_), tip_mode(tip_mode_), ns(ns_), levels(levels_), prods(products(ns_, levels_)),
        prof(prof_), fp8(fp8_) {}
  cudaError_t tips(cudaStream_t s) override {
    prof.begin(s);
    cudaError_t e = launch_diag(P, 0, tip_mode, s);
    prof.end(s, 1, 0.0);
    return e;
  }
  cudaError_t diag(int i, cudaStream_t s) override {
    prof.begin(s);
    cudaError_t e = launch_diag(P, i, kDiagSolve, s);
    prof.end(s, 1, 0.0);
    return e;
  }
  cudaError_t prep(int i, cudaStream_t s) override {
    prof.begin(s);
    cudaError_t e = fp8 ? launch_split_X8(P, w, i, hs.cstart[i], P.Y, P.nrm, s)
                        : launch_split_X(P, w, i, hs.cstart[i], P.Y, P.nrm, ns, s);
    prof.end(s, 2, 0.0);
    return e;
  }
  cudaError_t update(int i, int k_lo, int k_hi, cudaStream_t s) override {
    const double rows = hs.toff[k_hi] - hs.toff[k_lo], cols = P.m - hs.cstart[i];
    const double K = 2.0 * (hs.toff[i + 1] - hs.toff[i]);
    prof.begin(s);
    const bool ftz = tip_mode == kDiagTipCorr;   // the correction pass of a sweep
    cudaError_t e = fp8 ? launch_update_split8(P, w, i, k_lo, k_hi, P.ex, P.nrm, s, ftz)
                        : launch_update_split(P, w, i, k_lo, k_hi, P.ex, P.nrm, ns, levels, s, ftz);
    // E4M3 products at half weight: the tensor cores' FP8 rate is twice
    // their BF16 rate, so every pass is counted in BF16-equivalent flops
    prof.end(s, 0, 2.0 * rows * cols * K * prods * (fp8 ? 0.5 : 1.0));
    return e;
  }
};

#define SCK(call)                                              \
  do {                                                         \
    cudaError_t _e = (call);                                   \
    if (_e != cudaSuccess) return PEVC_ERR_CUDA;               \
  } while (0)

}  // namespace

cudaError_t launch_split_A_block(const Problem& P, SplitWorkspace& w, int l, int ns, cudaStream_t s) {
  return split_A_block(P, w, l, ns, s);
}

int split_prepare(SplitWorkspace& w, const Problem& P, const HostStructure& hs, cudaStream_t s) {
  if (!w.on) return PEVC_ERR_UNSUPPORTED;
  if (w.use_tc && w.tc_ok) {
    // output column chunks (width 48 and 64) inside every column tile
    int* h48c = w.h_chunks;
    int* h48j = h48c + w.max_chunks;
    int* h64c = h48j + w.max_chunks;
    int* h64j = h64c + w.max_chunks;
    int n48 = 0, n64 = 0;
    for (int j = 0; j < P.M; ++j) {
      w.h_chunk_first48[j] = n48;
      w.h_chunk_first64[j] = n64;
      for (int c = hs.cstart[j]; c < hs.cstart[j + 1]; c += 48) { h48c[n48] = c; h48j[n48] = j; ++n48; }
      for (int c = hs.cstart[j]; c < hs.cstart[j + 1]; c += 64) { h64c[n64] = c; h64j[n64] = j; ++n64; }
    }
    w.h_chunk_first48[P.M] = n48;
    w.h_chunk_first64[P.M] = n64;
    if (n48 > w.max_chunks || n64 > w.max_chunks) return PEVC_ERR_CUDA;
    SCK(cudaMemcpyAsync(w.chunk_c0_48, h48c, (size_t)n48 * sizeof(int), cudaMemcpyHostToDevice, s));
    SCK(cudaMemcpyAsync(w.chunk_j_48, h48j, (size_t)n48 * sizeof(int), cudaMemcpyHostToDevice, s));
    SCK(cudaMemcpyAsync(w.chunk_c0_64, h64c, (size_t)n64 * sizeof(int), cudaMemcpyHostToDevice, s));
    SCK(cudaMemcpyAsync(w.chunk_j_64, h64j, (size_t)n64 * sizeof(int), cudaMemcpyHostToDevice, s));
  }
  return 0;
}

int split_solve(SplitWorkspace& w, const Problem& P, const HostStructure& hs, const SplitConfig& cfg,
                cudaStream_t s, const SchedContext& sc, Profiler& prof, cudaEvent_t ev_dag, cudaEvent_t ev_corr,
                Arrivals* arr) {
  if (!w.on) return PEVC_ERR_UNSUPPORTED;
  if (arr && (cfg.correction || cfg.fp8)) return PEVC_ERR_UNSUPPORTED;
  if (!arr) {
    const int rc = split_prepare(w, P, hs, s);
    if (rc) return rc;
  }
  // BF16 slices of [S T] for the solve passes (BF16 plans) and the residual
  // (5 slices); FP8 slices for the solve passes of FP8 plans
  const int ns_a = cfg.fp8 ? cfg.ns_res : (cfg.correction ? std::max(cfg.ns1, cfg.ns_res) : cfg.ns1);
  if (!arr) {
    if (cfg.fp8) {
      if (!w.fp8) return PEVC_ERR_UNSUPPORTED;
      prof.begin(s);
      SCK(launch_split_A8(P, w, s));
      prof.end(s, 3, 0.0);
    }
    if (!cfg.fp8 || cfg.correction) {
      prof.begin(s);
      SCK(launch_split_A(P, w, ns_a == 5 ? 5 : 3, s));
      prof.end(s, 3, 0.0);
    }
    SplitOps ops(P, w, hs, kDiagTip, cfg.ns1, cfg.levels1, prof, cfg.fp8);
    SCK(walk_dag(P.M, ops, s, sc.aux, sc.ev, sc.lookahead));
  } else {
    // column block i's arrival work (pre-pass, slices, tips) is the caller's
    struct StreamedOps : SplitOps {
      Arrivals* arr;
      StreamedOps(const Problem& P_, SplitWorkspace& w_, const HostStructure& hs_, const SplitConfig& cfg_,
                  Profiler& prof_, Arrivals* arr_)
          : SplitOps(P_, w_, hs_, kDiagTip, cfg_.ns1, cfg_.levels1, prof_), arr(arr_) {}
      cudaError_t tips(cudaStream_t) override { return cudaSuccess; }   // tile by tile, on arrival
      cudaError_t arrive(int l, cudaStream_t st) override { return arr->arrive(l, st); }
    } ops(P, w, hs, cfg, prof, arr);
    SCK(walk_dag(P.M, ops, s, sc.aux, sc.ev, sc.lookahead));
  }
  SCK(cudaEventRecord(ev_dag, s));
  w.last_sweeps = 0;
  int prev = 0;   // the previous sweep's size (adaptive sweeps)
  for (int sweep = 0; cfg.correction && sweep < cfg.sweeps; ++sweep) {
    // residual R = (S V D - T V B) of the current V (the first pass, or the
    // previous sweep's sum), accumulated tile row by tile row into the
    // correction tiles as -R (including the diagonal tiles)
    Problem P2 = P;
    P2.Y = w.Y2;
    P2.ex = w.ex2;
    P2.nrm = w.nrm2;
    prof.begin(s);
    SCK(launch_init_state(P2, s));
    prof.end(s, 3, 0.0);
    // diagonal tiles in FP64: a tile column of V spans a range of ~2^64 in
    // magnitude, so fixed-point slices relative to its largest entry would
    // lose the small entries that the rows near its bottom depend on
    prof.begin(s);
    SCK(launch_diag_residual_f64(P2, P.Y, P.ex, P.nrm, s));
    prof.end(s, 3, 0.0);
    // off-diagonal tiles (l > k) as exact slice products: every X'' entry is
    // below the rows it updates, so slice truncation is relative to smaller
    // magnitudes than the result's
    const int prods = products(cfg.ns_res, cfg.levels_res);
    for (int l = 1; l < P.M; ++l) {
      prof.begin(s);
      SCK(launch_split_X(P, w, l, hs.cstart[l], P.Y, P.nrm, cfg.ns_res, s));
      prof.end(s, 2, 0.0);
      const double rows = hs.toff[l], cols = P.m - hs.cstart[l], K = 2.0 * (hs.toff[l + 1] - hs.toff[l]);
      prof.begin(s);
      SCK(launch_update_split(P2, w, l, 0, l, P.ex, P.nrm, cfg.ns_res, cfg.levels_res, s, true));
      prof.end(s, 0, 2.0 * rows * cols * K * prods);
    }
    // the correction: same graph, zero tips, right-hand side -R
    {
      SplitOps ops(P2, w, hs, kDiagTipCorr, cfg.ns1, cfg.levels1, prof, cfg.fp8);
      SCK(walk_dag(P.M, ops, s, sc.aux, sc.ev, sc.lookahead));
    }
    prof.begin(s);
    dim3 grid(P.M, (P.m + 7) / 8);
    k_combine<<<grid, 256, 0, s>>>(P, w.Y2, w.ex2, w.nrm2);
    SCK(cudaGetLastError());
    prof.end(s, 3, 0.0);
    ++w.last_sweeps;
    if (cfg.adaptive && sweep + 1 < cfg.sweeps) {
      // r = log2 of the largest change this sweep made to a normalised
      // eigenvector, about the error it had before the sweep; the error
      // after it is about r times the contraction, estimated from the last
      // two sweeps (the host waits for the sweep to finish to read r)
      prof.begin(s);
      SCK(cudaMemsetAsync(w.d_sweep, 0x80, sizeof(int), s));
      k_sweep_change<<<(unsigned)((P.m + 7) / 8), 256, 0, s>>>(P, w.Y2, w.ex2, w.d_sweep);
      SCK(cudaGetLastError());
      prof.end(s, 3, 0.0);
      SCK(cudaMemcpyAsync(w.h_sweep, w.d_sweep, sizeof(int), cudaMemcpyDeviceToHost, s));
      SCK(cudaStreamSynchronize(s));
      const int r = *w.h_sweep;
      const int predicted = sweep > 0 ? r + std::min(0, r - prev) : r;
      if (predicted <= kSweepTarget) break;
      prev = r;
    }
  }
  SCK(cudaEventRecord(ev_corr, s));
  return 0;
}


// ----------------------------------------------- back-transformation X = Z V
//
// Section 1: with (A, B) = (Q S Z^T, Q T Z^T), x = Z v is an eigenvector of
// (A, B).  The product runs as exact BF16 slice products, like the updates:
// every row r of Z is sliced (kBtSlices slices of 8 bits) per chunk of kBtK
// columns relative to its own exponent bound in that chunk, every column c of V per chunk of kBtK rows
// likewise, so that the products of one chunk accumulate exactly in FP32 per
// slice level; the chunks' recombined values are summed in FP64.  Chunks of
// V below a column block's last non-zero row (V is quasi-triangular) are
// skipped.

constexpr int kBtK = 256;          // K chunk with exact FP32 level sums
constexpr int kBtRows = 32;        // rows of Z sliced by one CTA
constexpr int kBtSlices = 6;       // 48 bits per operand: entries of X within about 2^-47 of sum |Z_rk V_kc|

// Last non-zero row + 1 of every column of V (one warp per column).
__global__ void __launch_bounds__(256) k_bt_heights(const double* __restrict__ V, int ldv, int n, int m,
                                                    int* __restrict__ h) {
  const int q = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (q >= m) return;
  const double* v = V + (size_t)q * ldv;
  int last = 0;
  for (int r = lane; r < n; r += 32)
    if (abs_key(v[r]) != 0) last = r + 1;
  for (int o = 16; o > 0; o >>= 1) last = max(last, __shfl_xor_sync(0xffffffffu, last, o));
  if (lane == 0) h[q] = last;
}

// Z slices: Zs[kc][p][r][kBtK] (K-contiguous per row), eZ[kc][r].  One CTA
// per (32 rows, chunk): thread t reads row t % 32 at 32 consecutive chunk
// columns (a warp reads 32 consecutive rows of a column: coalesced).
template <int NS>
__global__ void __launch_bounds__(256) k_bt_slice_Z(const double* __restrict__ Z, int ldz, int n,
                                                    __nv_bfloat16* __restrict__ Zs, int* __restrict__ eZ) {
  const int kc = blockIdx.y;
  const int rr = threadIdx.x % kBtRows, part = threadIdx.x / kBtRows;   // 8 parts of 32 columns
  const int r = blockIdx.x * kBtRows + rr;
  const int k0 = kc * kBtK + part * 32;
  __shared__ unsigned long long s_key[8][kBtRows];
  double v[32];
  unsigned long long key = 0;
#pragma unroll
  for (int t = 0; t < 32; ++t) {
    v[t] = (r < n && k0 + t < n) ? Z[(size_t)(k0 + t) * ldz + r] : 0.0;
    key = max(key, abs_key(v[t]));
  }
  s_key[part][rr] = key;
  __syncthreads();
  unsigned long long km = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) km = max(km, s_key[q][rr]);
  const int e = km ? exp_above(__longlong_as_double((long long)km)) : 0;
  if (r >= n) return;
  if (part == 0) eZ[(size_t)kc * n + r] = e;
  __nv_bfloat16* dst = Zs + (((size_t)kc * NS) * n + r) * kBtK + part * 32;
#pragma unroll
  for (int t = 0; t < 32; ++t) {
    int d[NS];
    int_slices<NS>(v[t], e, d);
#pragma unroll
    for (int p = 0; p < NS; ++p) dst[(size_t)p * n * kBtK + t] = small_int_bf16(d[p]);
  }
}

// V slices: Vs[kc][p][c][kBtK] (K-contiguous per column), eV[kc][c]; one warp
// per (column, chunk), each lane 8 consecutive rows.  Chunks at or below the
// column's height are all zero (exponent 0).
template <int NS>
__global__ void __launch_bounds__(256) k_bt_slice_V(const double* __restrict__ V, int ldv, int n, int m,
                                                    __nv_bfloat16* __restrict__ Vs, int* __restrict__ eV) {
  const int q = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  const int kc = blockIdx.y;
  if (q >= m) return;
  const int r0 = kc * kBtK + lane * 8;
  double v[8];
  unsigned long long key = 0;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    v[t] = (r0 + t < n) ? V[(size_t)q * ldv + r0 + t] : 0.0;
    key = max(key, abs_key(v[t]));
  }
  for (int o = 16; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o));
  const int e = key ? exp_above(__longlong_as_double((long long)key)) : 0;
  if (lane == 0) eV[(size_t)kc * m + q] = e;
  __nv_bfloat16* dst = Vs + (((size_t)kc * NS) * m + q) * kBtK + lane * 8;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    int d[NS];
    int_slices<NS>(v[t], e, d);
#pragma unroll
    for (int p = 0; p < NS; ++p) dst[(size_t)p * m * kBtK + t] = small_int_bf16(d[p]);
  }
}


// X[rows of this CTA, columns of this CTA] = Z V: a pipeline of K stages of
// KC over the chunks the column block needs (cp.async double buffering, BF16
// mma.sync with one FP32 accumulator per slice level); at the end of every
// chunk the levels are recombined exactly as one integer and added, scaled by
// the row's and the column's exponents of that chunk, to FP64 accumulators.
template <int NS, int L>
__global__ void __launch_bounds__(256, 1) k_bt_gemm(const __nv_bfloat16* __restrict__ Zs, const int* __restrict__ eZ,
                                                     const __nv_bfloat16* __restrict__ Vs,
                                                     const int* __restrict__ eV, const int* __restrict__ h, int n,
                                                     int m, double* __restrict__ X, int ldx) {
  constexpr int KC = split_kc<NS>();
  constexpr int LD = split_ld<NS>();
  constexpr int per_chunk = kBtK / KC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(smem_raw);    // [2][NS][128][LD]
  __nv_bfloat16* sB = sA + 2 * NS * kSplitRows * LD;                 // [2][NS][32][LD]
  const int c0 = blockIdx.x * kSplitCols, r0 = blockIdx.y * kSplitRows;
  const int tid = threadIdx.x;
  __shared__ int s_nk;
  if (tid < 32) {
    int hh = (c0 + tid < m) ? h[c0 + tid] : 0;
    for (int o = 16; o > 0; o >>= 1) hh = max(hh, __shfl_xor_sync(0xffffffffu, hh, o));
    if (tid == 0) s_nk = (hh + kBtK - 1) / kBtK;
  }
  __syncthreads();
  const int nk = s_nk;

  auto load_stage = [&](int st, int idx) {
    const int kc = idx / per_chunk, kb = (idx % per_chunk) * KC;
    __nv_bfloat16* a_dst = sA + st * NS * kSplitRows * LD;
    __nv_bfloat16* b_dst = sB + st * NS * kSplitCols * LD;
    constexpr int chunks = KC / 8;                        // 16-byte pieces per row
    for (int q = tid; q < NS * kSplitRows * chunks; q += 256) {
      const int c16 = q % chunks, r = (q / chunks) % kSplitRows, p = q / (chunks * kSplitRows);
      const bool valid = r0 + r < n;
      const __nv_bfloat16* src = Zs + (((size_t)kc * NS + p) * n + (valid ? r0 + r : 0)) * kBtK + kb + 8 * c16;
      cp_async16(a_dst + (p * kSplitRows + r) * LD + 8 * c16, src, valid);
    }
    for (int q = tid; q < NS * kSplitCols * chunks; q += 256) {
      const int c16 = q % chunks, col = (q / chunks) % kSplitCols, p = q / (chunks * kSplitCols);
      const bool valid = c0 + col < m;
      const __nv_bfloat16* src = Vs + (((size_t)kc * NS + p) * m + (valid ? c0 + col : 0)) * kBtK + kb + 8 * c16;
      cp_async16(b_dst + (p * kSplitCols + col) * LD + 8 * c16, src, valid);
    }
  };

  const int warp = tid >> 5, lane = tid & 31;
  const int wr = warp & 3, wc = warp >> 2;
  const int g = lane >> 2, t4 = lane & 3;
  float acc[L][2][2][4];
  double out[2][2][2][2];   // [mt][nt][h][e]
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int hh = 0; hh < 2; ++hh)
#pragma unroll
        for (int e = 0; e < 2; ++e) out[mt][nt][hh][e] = 0.0;
  auto zero_levels = [&]() {
#pragma unroll
    for (int s = 0; s < L; ++s)
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[s][a][b][e] = 0.0f;
  };
  zero_levels();

  const int nst = nk * per_chunk;
  if (nst > 0) load_stage(0, 0);
  cp_async_commit();
  for (int idx = 0; idx < nst; ++idx) {
    const int st = idx & 1;
    if (idx + 1 < nst) load_stage(st ^ 1, idx + 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const __nv_bfloat16* a_s = sA + st * NS * kSplitRows * LD;
    const __nv_bfloat16* b_s = sB + st * NS * kSplitCols * LD;
#pragma unroll
    for (int kk = 0; kk < KC; kk += 16) {
      unsigned bf[NS][4];
#pragma unroll
      for (int q = 0; q < NS; ++q)
        ldmatrix_x4(bf[q], b_s + (q * kSplitCols + 16 * wc + (lane & 7) + ((lane >> 4) << 3)) * LD + kk +
                               ((lane >> 3) & 1) * 8);
#pragma unroll
      for (int p = 0; p < NS; ++p) {
        unsigned af[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
          ldmatrix_x4(af[mt], a_s + (p * kSplitRows + 32 * wr + 16 * mt + (lane & 15)) * LD + kk + (lane >> 4) * 8);
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          if (p + q < L) {
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
              mma_bf16(acc[p + q][mt][0], af[mt], bf[q][0], bf[q][1]);
              mma_bf16(acc[p + q][mt][1], af[mt], bf[q][2], bf[q][3]);
            }
          }
        }
      }
    }
    __syncthreads();
    if ((idx + 1) % per_chunk == 0) {
      // the chunk is complete: its exact level sums, scaled, into FP64
      const int kc = idx / per_chunk;
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int row = r0 + 32 * wr + 16 * mt + g + 8 * hh;
          const int ez = row < n ? eZ[(size_t)kc * n + row] : 0;
#pragma unroll
          for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const int col = c0 + 16 * wc + 8 * nt + 2 * t4 + e;
              const int ev = col < m ? eV[(size_t)kc * m + col] : 0;
              long long t = 0;
#pragma unroll
              for (int s = 0; s < L; ++s) t = (t << 8) + (long long)__float2int_rn(acc[s][mt][nt][2 * hh + e]);
              out[mt][nt][hh][e] += i64_scaled(t, ez + ev - 14 - 8 * (L - 1));
            }
        }
      zero_levels();
    }
  }
  cp_async_wait<0>();
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int row = r0 + 32 * wr + 16 * mt + g + 8 * hh;
      if (row >= n) continue;
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int col = c0 + 16 * wc + 8 * nt + 2 * t4 + e;
          if (col < m) X[(size_t)col * ldx + row] = out[mt][nt][hh][e];
        }
    }
}

// Workspace of the split back-transformation (slices and exponents of Z and
// V, column heights), for orders up to n_max.
size_t bt_split_bytes(int n_max) {
  const size_t nkc = (size_t)(std::max(n_max, 1) + kBtK - 1) / kBtK, n = (size_t)std::max(n_max, 1);
  return 2 * (nkc * kBtSlices * n * kBtK * sizeof(__nv_bfloat16)) + 2 * nkc * n * sizeof(int) + n * sizeof(int) +
         6 * 256;
}

// X = Z V (n x m, column-major FP64) with the split GEMM above; ws holds
// bt_split_bytes(n) bytes (256-byte aligned).
cudaError_t launch_bt_split(const double* Z, int ldz, int n, const double* V, int ldv, int m, double* X, int ldx,
                            unsigned char* ws, cudaStream_t s) {
  if (n <= 0 || m <= 0) return cudaSuccess;
  constexpr int NS = kBtSlices;
  const int nkc = (n + kBtK - 1) / kBtK;
  auto take = [&](size_t bytes) {
    unsigned char* q = ws;
    ws += (bytes + 255) / 256 * 256;
    return q;
  };
  __nv_bfloat16* Zs = (__nv_bfloat16*)take((size_t)nkc * NS * n * kBtK * sizeof(__nv_bfloat16));
  __nv_bfloat16* Vs = (__nv_bfloat16*)take((size_t)nkc * NS * m * kBtK * sizeof(__nv_bfloat16));
  int* eZ = (int*)take((size_t)nkc * n * sizeof(int));
  int* eV = (int*)take((size_t)nkc * m * sizeof(int));
  int* h = (int*)take((size_t)m * sizeof(int));
  k_bt_heights<<<(m + 7) / 8, 256, 0, s>>>(V, ldv, n, m, h);
  k_bt_slice_Z<NS><<<dim3((n + kBtRows - 1) / kBtRows, nkc), 256, 0, s>>>(Z, ldz, n, Zs, eZ);
  k_bt_slice_V<NS><<<dim3((m + 7) / 8, nkc), 256, 0, s>>>(V, ldv, n, m, Vs, eV);
  const int smem = split_smem_bytes<NS>();
  cudaError_t e = cudaFuncSetAttribute(k_bt_gemm<NS, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_bt_gemm<NS, NS><<<dim3((m + kSplitCols - 1) / kSplitCols, (n + kSplitRows - 1) / kSplitRows), 256, smem, s>>>(
      Zs, eZ, Vs, eV, h, n, m, X, ldx);
  return cudaGetLastError();
}

}  // namespace pevc

// update_tc.cu -- the split-precision update (Section 3, kernel 2) on the
// fifth-generation tensor cores, fed by TMA:
//     Y_kj <- 2^sY Y_kj - 2^sX [S_ki T_ki] X''_ij,   k in [k_lo, k_hi), j >= i,
// with [S_ki T_ki] and X'' given as exact integer slices (split.cu): BF16
// (8-bit digits) or FP8 E4M3 (4-bit digits).
//
// Persistent CTA (one per SM) of nineteen warps:
//   warp 0     TMA producer: per K block of 128 bytes (64 BF16 or 128 E4M3
//              elements) one 3-D box with every slice of
//              the A row tile and one with every slice of the X'' column
//              chunk (rows of 128 bytes, 128-byte swizzle), landing directly
//              in the K-major layout the MMA reads; a ring of shared-memory
//              stages with full / empty mbarriers;
//   warp 1     tensor-memory owner and MMA issuer: the slice products p x q
//              with p + q < L of one A slice p are one tcgen05.mma (M = 128,
//              N = (L - p) NCOL over the stacked X'' slices, K = 32 bytes:
//              16 BF16 (kind::f16) or 32 E4M3 (kind::f8f6f4), FP32 out)
//              whose consecutive NCOL-column blocks are the level
//              accumulators p .. L - 1;
//              the level accumulators of an output tile live in one of two
//              tensor-memory buffers;
//   warps 2-17 two epilogue groups of eight warps (two per tensor-memory
//              lane quarter, each with half of the tile's columns); group g
//              takes every other output tile and owns buffer g, so one group's
//              epilogue overlaps the MMAs of the next tile and the other
//              group's epilogue;
//   warp 18    column-scale producer: the per-column scales of the CTA's
//              output tiles, up to four tiles ahead, into a ring of shared-
//              memory slots (full / empty mbarriers), and each tile's Y chunk
//              (contiguous in HBM) prefetched into L2.
// Epilogue, per element: exact integer recombination of the levels, its
// rounding to FP64 with the augmented-tile scale applied (Algorithms 2 and 3
// of Section 4; half the elements of a block by the int64 -> FP64 conversion
// and exponent arithmetic, half by integer assembly of the binary64 fields,
// so that the FP64 and integer pipes share the work), one FP64 subtraction;
// new column maxima (rounded-up 32-bit keys) by one warp reduction per column.
// Every wait is bounded (SM clock cycles): a wait that runs out sets
// PEVC_ERR_TIMEOUT in the status word and the CTA winds down: every role runs
// out of bounded waits, the producer waits (bounded) for the loads it issued,
// the MMA issuer for the MMAs it issued, and tensor memory is freed.
#include <cuda.h>

#include "split.cuh"
#include "tc.cuh"

namespace pevc {

constexpr int kTcRows = 128;                 // M of every MMA: one row tile
constexpr int kTcRowBytes = 128;             // K per pipeline stage: one 128-byte swizzle row
constexpr long long kTcWait = 4000000000LL;  // bounded waits: about 2 s of SM clock
constexpr int kTcEpiWarps = 8;               // warps per epilogue group: two per lane quarter
constexpr int kTcColBlock = 4;               // columns per epilogue step
constexpr int kTcScalesWarp = 2 + 2 * kTcEpiWarps;       // the column-scales producer
constexpr int kTcThreads = 32 * (kTcScalesWarp + 1);   // producer, MMA issuer, two epilogue groups, scales
constexpr int kTcRing = 4;                              // column-scale slots (output tiles ahead)
// (nineteen warps: one SM sub-partition holds five of them, so its 16K
// registers cap a thread at 96)

template <int NS, int NCOL>
struct TcGeom {
  static constexpr int a_slice = kTcRows * kTcRowBytes;   // bytes of one A slice per stage (1024-multiple)
  static constexpr int b_slice = NCOL * kTcRowBytes;      // bytes of one X'' slice per stage (1024-multiple)
  static constexpr int stage = NS * (a_slice + b_slice);
  static constexpr int stages = (225 * 1024) / stage < 4 ? (225 * 1024) / stage : 4;
  static constexpr int smem = stages * stage + 1024 + 256;   // + alignment slack, mbarriers, TMEM address
};

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(mbar))
      : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(mbar)), "r"(bytes));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(mbar)));
}
// Bulk prefetch of a contiguous global range into L2 (16-byte aligned, size a
// multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}
// Named barrier of one epilogue group (ids 1 and 2).
__device__ __forceinline__ void group_barrier(int g) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(1 + g), "n"(32 * kTcEpiWarps));
}

struct TmTiles {
  const int* chunk_c0;   // first output column of every column chunk (global list)
  const int* chunk_j;    // its column tile
  int chunk_first;       // first chunk of column tile i
  int nchunks;           // chunks of column tiles >= i
  int k_lo, nk;
};

// Per-column data of an output tile: x = shift of the stored Y, y = shift of
// the product (without the row exponent), z = flags (1 = column updated,
// 2 = Y still zero), w = the column's new exponent.
template <int L, int NCOL, int DB>
__device__ __forceinline__ void tile_scales(const Problem& P, int i, const TmTiles& tt, int t, const int* exX,
                                            const double* nrmX, const int* F, int col, int4* out) {
  const int k = tt.k_lo + t / tt.nchunks;
  const int ch = tt.chunk_first + t % tt.nchunks;
  const int j = tt.chunk_j[ch];
  const int c0 = tt.chunk_c0[ch];
  const int nc = min(NCOL, P.cstart[j + 1] - c0);
  int on = 0, sY = 0, sX = 0, en = 0, sc = 0;
  bool yz = true;
  if (col < nc) {
    const int q = c0 + col;
    on = update_scales(P, exX, nrmX, k, i, q, sY, sX, en, yz) ? 1 : 0;
    if (on && F[q] == kExpZero) on = 0;
    sc = on ? F[q] - 2 * (DB - 1) - DB * (L - 1) + sX : 0;
  }
  *out = make_int4(sY, sc, on | (yz ? 2 : 0), en);
}

// The Y columns an output tile updates: a contiguous range of its tile.
template <int NCOL>
__device__ __forceinline__ void tile_y_range(const Problem& P, const TmTiles& tt, int t, const double*& y,
                                             uint32_t& bytes) {
  const int k = tt.k_lo + t / tt.nchunks;
  const int ch = tt.chunk_first + t % tt.nchunks;
  const int j = tt.chunk_j[ch];
  const int c0 = tt.chunk_c0[ch];
  const int nc = min(NCOL, P.cstart[j + 1] - c0);
  y = tile_ptr(P, k, j) + (size_t)(c0 - P.cstart[j]) * P.tb;
  bytes = (uint32_t)(nc * P.tb * sizeof(double));
}

// The scaled product t * 2^e of an update, as i64_scaled_fast and
// pow2_scale_fast form it, except that a product whose stored magnitude falls
// below the normal range is flushed to a zero of its sign instead of sending
// the block to the exact path.  Such products arise in the correction pass,
// where a tile Y2(k) holds the residual of row k at the scale of that row's
// own terms, while the corrections of rows i far below k are smaller by the
// eigenvector's growth over i - k tiles; below 2^-1022 of the tile's scale
// they cannot change a stored value of the tile.  Overflow still takes the
// exact path.  Used by the correction sweeps' updates (template flag FTZ); the
// first pass keeps the plain fast paths (its products never underflow: every
// update into a tile is at least as large as the tile's stored values).
__device__ __forceinline__ double i64_scaled_ftz(long long t, int e, bool& slow) {
  const unsigned long long sgn = (unsigned long long)t & (1ull << 63);
  const unsigned long long mag = t < 0 ? 0ull - (unsigned long long)t : (unsigned long long)t;
  const int lz = __clzll((long long)(mag | 1ull));
  const int E = 1086 - lz + e;                 // before rounding; rounding adds at most one
  bool sl = false;
  const double r = i64_scaled_fast(t, e, sl);
  slow |= sl & (E > 0);
  return (mag != 0 && E <= 0) ? __longlong_as_double((long long)sgn) : r;
}
// y * 2^s for y = (double)t (a normal number or zero), flushed like i64_scaled_ftz
__device__ __forceinline__ double pow2_scale_ftz(double y, int sh, bool& slow) {
  const int hi = __double2hiint(y);
  const int E = (hi >> 20) & 0x7ff;
  const bool under = E != 0 && E + sh <= 0;
  bool sl = false;
  const double r = pow2_scale_fast(y, sh, sl);
  slow |= sl & !under;
  return under ? __hiloint2double(hi & (int)0x80000000, 0) : r;
}

// Upper 32 bits of |x|'s bit pattern, rounded up: non-negative doubles order
// like these keys, and the double they stand for is an upper bound of |x|
// (within 2^-20 relative), which is all the norm bookkeeping needs.
__device__ __forceinline__ unsigned key32(double x) {
  return (unsigned)((abs_key(x) + 0xffffffffull) >> 32);
}

template <int NS, int L, int NCOL, bool FP8 = false, bool FTZ = false>
__global__ void __maxnreg__(96) k_update_tc(Problem P, int i, TmTiles tt, const int* __restrict__ exX,
                                                             const double* __restrict__ nrmX,
                                                             const int* __restrict__ eA, const int* __restrict__ F,
                                                             int ns, const __grid_constant__ CUtensorMap tmA,
                                                             const __grid_constant__ CUtensorMap tmB) {
  static_assert(NCOL % 16 == 0 && 2 * L * NCOL <= 512, "two level-accumulator buffers must fit tensor memory");
  static_assert(NS >= L && L <= 5 && L * NCOL <= 256, "one MMA per A slice covers at most N = 256 columns");
  using G = TcGeom<NS, NCOL>;
  constexpr int DB = FP8 ? 4 : 8;                 // bits per slice digit
  constexpr int KE = FP8 ? 128 : 64;              // K elements per stage (one 128-byte row)
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // swizzle atoms need 1024-byte aligned stage bases
  unsigned char* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + G::stages * G::stage);
  uint64_t* empty = full + G::stages;
  uint64_t* tfull = empty + G::stages;   // [2] accumulator buffer complete
  uint64_t* tempty = tfull + 2;          // [2] accumulator buffer drained (its group's warps arrive)
  uint64_t* drain = tempty + 2;          // MMAs in flight completed (failure path only)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

  __shared__ int4 s_col[kTcRing][NCOL];            // column scales of the next output tiles (a ring)
  __shared__ uint64_t s_sfull[kTcRing], s_sempty[kTcRing];
  __shared__ unsigned s_key[2][4][NCOL];           // per group and lane quarter: column maxima (upper 32 bits)
  __shared__ int s_fail, s_stop[2];
  volatile int* fail = &s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tb = P.tb;
  const int nks = 2 * tb / KE;
  const int total = tt.nk * tt.nchunks;
  constexpr uint32_t kCols = 512;
  constexpr uint32_t kTx = (uint32_t)G::stage;

  if (tid == 0) {
    for (int s = 0; s < G::stages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], kTcEpiWarps); }
    mbar_init(drain, 1);
    for (int r = 0; r < kTcRing; ++r) { mbar_init(&s_sfull[r], 1); mbar_init(&s_sempty[r], 1); }
    s_fail = 0;
    s_stop[0] = s_stop[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  if (warp == 1) tc_alloc(tmem_slot, kCols);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0, used = 0, last_ph = 0;   // per stage: loaded at least once, parity of its last load
      for (int t = blockIdx.x; t < total && !*fail; t += gridDim.x) {
        const int k = tt.k_lo + t / tt.nchunks;
        const int ch = tt.chunk_first + t % tt.nchunks;
        const int c0 = tt.chunk_c0[ch];
        const int a_plane = (int)(tri_index(k, i) * ns);
        for (int kk = 0; kk < nks; ++kk) {
          if (!mbar_wait_cycles(&empty[s], ph ^ 1u, kTcWait)) { *fail = 1; break; }
          mbar_expect_tx(&full[s], kTx);
          unsigned char* dst = smem + s * G::stage;
          tma_load_3d(dst, &tmA, kk * KE, 0, a_plane, &full[s]);
          tma_load_3d(dst + NS * G::a_slice, &tmB, kk * KE, c0, 0, &full[s]);
          used |= 1u << s;
          last_ph = (last_ph & ~(1u << s)) | (ph << s);
          if (++s == G::stages) { s = 0; ph ^= 1u; }
        }
      }
      // after a failure, the loads already issued land before shared memory
      // is released (a load the MMA warp consumed has completed its phase,
      // so its wait returns at once)
      if (*fail)
        for (int q = 0; q < G::stages; ++q)
          if (used & (1u << q)) mbar_wait_cycles(&full[q], (last_ph >> q) & 1u, kTcWait);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      int s = 0, it = 0;
      uint32_t ph = 0;
      for (int t = blockIdx.x; t < total && !*fail; t += gridDim.x, ++it) {
        const int buf = it & 1;
        if (!mbar_wait_cycles(&tempty[buf], ((it >> 1) & 1) ^ 1u, kTcWait)) { *fail = 1; break; }
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(buf * L * NCOL);
        for (int kk = 0; kk < nks; ++kk) {
          if (!mbar_wait_cycles(&full[s], ph, kTcWait)) { *fail = 1; break; }
          tc_fence_after();
          const uint32_t base = smem_addr(smem + s * G::stage);
          const uint64_t ad = smem_desc_sw128(base, 1024);
          const uint64_t bd = smem_desc_sw128(base + NS * G::a_slice, 1024);
          // one MMA per A slice p: the X'' slices q < L - p are consecutive
          // NCOL-row blocks of the stage and the level accumulators
          // consecutive NCOL-column blocks of the buffer, so A_p times the
          // stacked slices lands every product p x q in level p + q
          // K steps of 32 bytes inside the swizzled row
#pragma unroll
          for (int k32 = 0; k32 < kTcRowBytes / 32; ++k32)
#pragma unroll
            for (int p = 0; p < NS && p < L; ++p) {
              constexpr int kNq[5] = {NS < L ? NS : L, NS < L - 1 ? NS : L - 1, NS < L - 2 ? NS : L - 2,
                                      NS < L - 3 ? NS : L - 3, NS < L - 4 ? NS : L - 4};
              const uint64_t a_p = ad + (uint64_t)((p * G::a_slice + 32 * k32) >> 4);
              const uint64_t b_k = bd + (uint64_t)((32 * k32) >> 4);
              const uint32_t accum = (kk | k32 | p) ? 1u : 0u;
              if constexpr (FP8)
                tc_mma_e4m3(acc + (uint32_t)(p * NCOL), a_p, b_k, idesc_e4m3_f32(kTcRows, kNq[p] * NCOL), accum);
              else
                tc_mma_bf16(acc + (uint32_t)(p * NCOL), a_p, b_k, idesc_bf16_f32(kTcRows, kNq[p] * NCOL), accum);
            }
          tc_commit(&empty[s]);             // frees the stage once these MMAs completed
          if (++s == G::stages) { s = 0; ph ^= 1u; }
        }
        if (*fail) break;
        tc_commit(&tfull[buf]);             // the tile's accumulators are complete
      }
      // after a failure, every MMA already issued completes before tensor
      // memory is freed: one more commit, to its own barrier, and a bounded wait
      if (*fail) {
        tc_commit(drain);
        mbar_wait_cycles(drain, 0u, kTcWait);
      }
    }
  } else if (warp == kTcScalesWarp) {
    // -------------------------------------------------------------- scales
    // per output tile of this CTA, in order: the column scales into the next
    // ring slot (a chain of dependent global loads, kept off the epilogue
    // groups) and the tile's Y chunk into L2
    for (int it = 0;; ++it) {
      const int t = blockIdx.x + it * (int)gridDim.x;
      if (t >= total || __any_sync(0xffffffffu, *fail != 0)) break;   // warp-uniform exits
      const int rs = it % kTcRing;
      if (!__all_sync(0xffffffffu, mbar_wait_cycles(&s_sempty[rs], (uint32_t)((it / kTcRing) & 1) ^ 1u, kTcWait))) {
        *fail = 1;
        break;
      }
      for (int c = lane; c < NCOL; c += 32) tile_scales<L, NCOL, DB>(P, i, tt, t, exX, nrmX, F, c, &s_col[rs][c]);
      if (lane == 0) {
        const double* yp;
        uint32_t yb;
        tile_y_range<NCOL>(P, tt, t, yp, yb);
        prefetch_l2(yp, yb);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&s_sfull[rs]);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    constexpr int CW = kTcColBlock;
    constexpr int HALF = NCOL / 2;                    // columns of one warp
    const int ew = warp - 2;
    const int g = ew / kTcEpiWarps;                   // group: every other tile, buffer g
    const int et = tid - 64 - 32 * kTcEpiWarps * g;   // thread index within the group
    const int quarter = warp & 3;                     // tensor-memory lane quarter of this warp
    const int half = (ew >> 2) & 1;                   // which half of the tile's columns
    const int row = 32 * quarter + lane;
    const int cbeg = half * HALF;
    int it = g;
    int t = blockIdx.x + it * (int)gridDim.x;
    for (; t < total; it += 2, t = blockIdx.x + it * (int)gridDim.x) {
      const int rs = it % kTcRing;
      // a wait that runs out skips the tile's work but still passes both
      // group barriers below, where the group stops together
      const bool sok = mbar_wait_cycles(&s_sfull[rs], (uint32_t)((it / kTcRing) & 1), kTcWait);
      if (!sok) *fail = 1;
      const int4* scol = s_col[rs];
      const int k = tt.k_lo + t / tt.nchunks;
      const int ch = tt.chunk_first + t % tt.nchunks;
      const int j = tt.chunk_j[ch];
      const int c0 = tt.chunk_c0[ch];
      const int cs = P.cstart[j];
      const int nc = min(NCOL, P.cstart[j + 1] - c0);
      const int hk = P.toff[k + 1] - P.toff[k];
      const bool rowok = row < hk;
      double* ycol = tile_ptr(P, k, j) + (size_t)(c0 - cs) * tb + row;   // column col at ycol[col * tb]
      const int erow = rowok ? eA[tri_index(k, i) * tb + row] : 0;
      // this row's Y in the warp's first block: loads in flight while the MMAs run
      double yv[CW];
#pragma unroll
      for (int u = 0; u < CW; ++u) {
        const int col = cbeg + u;
        const int4 cd = scol[col];
        yv[u] = (rowok && col < nc && cd.z == 1) ? ycol[(size_t)col * tb] : 0.0;
      }
      // warp-uniform, since the work below synchronises the warp
      const bool ok = __all_sync(0xffffffffu, sok && mbar_wait_cycles(&tfull[g], (uint32_t)((it >> 1) & 1), kTcWait));
      if (!ok) *fail = 1;
      tc_fence_after();
      if (ok) {
        const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(g * L * NCOL);
#pragma unroll 1
        for (int cb = cbeg; cb < cbeg + HALF; cb += CW) {
          uint32_t lv[L][CW];
#pragma unroll
          for (int s = 0; s < L; ++s) tc_ld4(lane_base + (uint32_t)(s * NCOL + cb), lv[s]);
          tc_wait_ld();
          if (cb + CW == cbeg + HALF) {
            // this warp's part of the buffer is drained: once every warp of
            // the group arrived, the MMAs of the group's next tile may start
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[g]);
          }
          double yn[CW];
#pragma unroll
          for (int u = 0; u < CW; ++u) {
            yn[u] = 0.0;
            if (cb + CW < cbeg + HALF) {
              const int col = cb + CW + u;
              const int4 cd = scol[col];
              if (rowok && col < nc && cd.z == 1) yn[u] = ycol[(size_t)col * tb];
            }
          }
          // straight-line fast path over the block's elements; the exact
          // path only when a value leaves the normal range
          double ynew[CW];
          bool act[CW];
          bool slow = false;
          // the shifts of the stored Y are per column, so this test is the
          // same on every lane: most blocks keep Y's exponents and skip them
          bool shy = false;
#pragma unroll
          for (int u = 0; u < CW; ++u) shy |= scol[cb + u].x != 0;
#pragma unroll
          for (int u = 0; u < CW; ++u) {
            const int col = cb + u;
            const int4 cd = scol[col];
            act[u] = (cd.z & 1) && rowok && col < nc;
            long long tv = 0;
#pragma unroll
            for (int s = 0; s < L; ++s)
              tv += (long long)__float2int_rn(__uint_as_float(lv[s][u])) * (1ll << (DB * (L - 1 - s)));
            bool sl = false;
            // half the elements convert on the FP64 pipe, half by integer
            // assembly of the binary64 fields (the same rounded value), so
            // that neither pipe alone bounds the block
            double prod;
            if constexpr (FTZ)
              prod = (u & 2) ? i64_scaled_ftz(tv, erow + cd.y, sl) : pow2_scale_ftz((double)tv, erow + cd.y, sl);
            else
              prod = (u & 2) ? i64_scaled_fast(tv, erow + cd.y, sl) : pow2_scale_fast((double)tv, erow + cd.y, sl);
            double yold = yv[u];
            if (shy) yold = pow2_scale_fast(yv[u], cd.x, sl);
            if (cd.z & 2) yold = 0.0;
            slow |= act[u] & sl;
            ynew[u] = yold - prod;
          }
          if (__any_sync(0xffffffffu, slow)) {
#pragma unroll
            for (int u = 0; u < CW; ++u) {
              const int4 cd = scol[cb + u];
              long long tv = 0;
#pragma unroll
              for (int s = 0; s < L; ++s) tv = (tv << DB) + (long long)__float2int_rn(__uint_as_float(lv[s][u]));
              const double prod = pow2_scale((double)tv, erow + cd.y);
              const double yold = (cd.z & 2) ? 0.0 : pow2_scale(yv[u], cd.x);
              if (act[u]) ynew[u] = yold - prod;
            }
          }
          unsigned key[CW];
#pragma unroll
          for (int u = 0; u < CW; ++u) {
            if (act[u]) ycol[(size_t)(cb + u) * tb] = ynew[u];
            key[u] = act[u] ? key32(ynew[u]) : 0u;
          }
          // column maxima over the warp's 32 rows: one warp reduction each
#pragma unroll
          for (int u = 0; u < CW; ++u) {
            const unsigned cm = __reduce_max_sync(0xffffffffu, key[u]);
            if (lane == 0) s_key[g][quarter][cb + u] = cm;
          }
#pragma unroll
          for (int u = 0; u < CW; ++u) yv[u] = yn[u];
        }
      }
      group_barrier(g);
      // new norms and exponents of the tile's columns
      if (et < NCOL) {
        const int4 cd = scol[et];
        if (ok && et < nc && (cd.z & 1)) {
          const long long idx = (long long)k * P.m + c0 + et;
          const unsigned km = max(max(s_key[g][0][et], s_key[g][1][et]), max(s_key[g][2][et], s_key[g][3][et]));
          P.nrm[idx] = __longlong_as_double((long long)km << 32);
          P.ex[idx] = cd.w;
        }
      }
      if (et == 0) s_stop[g] = *fail;
      group_barrier(g);
      if (et == 0) mbar_arrive(&s_sempty[rs]);   // the slot may take a later tile's scales
      if (s_stop[g]) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*fail && tid == 0) atomicOr(P.status, kStTimeout);
  if (warp == 1) {
    tc_fence_after();
    tc_dealloc(tmem, kCols);
  }
}

// ------------------------------------------------------------------ host

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

int update_tc_setup() {
  cudaError_t a = cudaFuncSetAttribute(k_update_tc<5, 5, 48>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       TcGeom<5, 48>::smem);
  cudaError_t b = cudaFuncSetAttribute(k_update_tc<3, 3, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       TcGeom<3, 64>::smem);
  cudaError_t c = cudaFuncSetAttribute(k_update_tc<4, 4, 64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       TcGeom<4, 64>::smem);
  // the correction sweeps' instantiations (underflowing products flushed)
  cudaError_t d = cudaFuncSetAttribute(k_update_tc<5, 5, 48, false, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, TcGeom<5, 48>::smem);
  cudaError_t e = cudaFuncSetAttribute(k_update_tc<3, 3, 64, false, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, TcGeom<3, 64>::smem);
  cudaError_t f = cudaFuncSetAttribute(k_update_tc<4, 4, 64, true, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, TcGeom<4, 64>::smem);
  return (a == cudaSuccess && b == cudaSuccess && c == cudaSuccess && d == cudaSuccess && e == cudaSuccess &&
          f == cudaSuccess && encode_fn())
             ? 0
             : PEVC_ERR_CUDA;
}

// Tensor maps over the K-contiguous slice buffers (one K block of 128 bytes =
// one 128-byte swizzle row per box row, every slice of the operand in one box):
//   A: [tile * ns + slice][row][2 tb]  -> dims {2tb, tb, tiles*ns}, box {64, 128, NS}
//   B: [slice][column][2 tb]           -> dims {2tb, n_max, ns},    box {64, NCOL, NS}
// and, for FP8 plans, over the E4M3 slices (four, bytes):
//   A: [tile * 4 + slice][row][2 tb]   -> dims {2tb, tb, tiles*4},  box {128, 128, 4}
//   B: [slice][column][2 tb]           -> dims {2tb, n_max, 4},     box {128, 64, 4}
int make_tensor_maps(SplitWorkspace& w) {
  w.tc_ok = false;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return PEVC_ERR_CUDA;
  if (w.tb != kTcRows) return 0;   // the tensor-core update handles tiles of order 128 only
  const cuuint64_t tb = (cuuint64_t)w.tb, K2 = (cuuint64_t)(2 * w.tb);
  cuuint32_t es[3] = {1, 1, 1};
  for (int v = 0; v < 2; ++v) {
    const cuuint32_t nsl = v == 0 ? 5 : 3;
    cuuint64_t dims[3] = {K2, tb, (cuuint64_t)(w.tiles * w.ns)};
    cuuint64_t strides[2] = {K2 * 2, tb * K2 * 2};
    cuuint32_t box[3] = {(cuuint32_t)(kTcRowBytes / 2), (cuuint32_t)kTcRows, nsl};
    if (enc(reinterpret_cast<CUtensorMap*>(v == 0 ? w.tmA : w.tmA3), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, w.As, dims,
            strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return PEVC_ERR_CUDA;
  }
  for (int v = 0; v < 2; ++v) {
    const cuuint32_t ncol = v == 0 ? 48 : 64, nsl = v == 0 ? 5 : 3;
    cuuint64_t dims[3] = {K2, (cuuint64_t)w.n_max, (cuuint64_t)w.ns};
    cuuint64_t strides[2] = {K2 * 2, (cuuint64_t)w.n_max * K2 * 2};
    cuuint32_t box[3] = {(cuuint32_t)(kTcRowBytes / 2), ncol, nsl};
    if (enc(reinterpret_cast<CUtensorMap*>(v == 0 ? w.tmB48 : w.tmB64), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, w.Xs,
            dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return PEVC_ERR_CUDA;
  }
  if (w.fp8) {
    cuuint64_t adims[3] = {K2, tb, (cuuint64_t)(w.tiles * 4)};
    cuuint64_t astrides[2] = {K2, tb * K2};
    cuuint32_t abox[3] = {(cuuint32_t)kTcRowBytes, (cuuint32_t)kTcRows, 4};
    if (enc(reinterpret_cast<CUtensorMap*>(w.tmA8), CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, w.As8, adims, astrides, abox,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return PEVC_ERR_CUDA;
    cuuint64_t bdims[3] = {K2, (cuuint64_t)w.n_max, 4};
    cuuint64_t bstrides[2] = {K2, (cuuint64_t)w.n_max * K2};
    cuuint32_t bbox[3] = {(cuuint32_t)kTcRowBytes, 64, 4};
    if (enc(reinterpret_cast<CUtensorMap*>(w.tmB64_8), CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, w.Xs8, bdims, bstrides,
            bbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return PEVC_ERR_CUDA;
  }
  w.tc_ok = true;
  return 0;
}

cudaError_t launch_update_tc(const Problem& P, const SplitWorkspace& w, int i, int k_lo, int k_hi, const int* exX,
                             const double* nrmX, int ns, int levels, bool fp8, cudaStream_t s, bool ftz) {
  if (k_hi <= k_lo) return cudaSuccess;
  const bool five = !fp8 && ns == 5 && levels == 5;
  const int* first = five ? w.h_chunk_first48 : w.h_chunk_first64;
  TmTiles tt;
  tt.chunk_c0 = five ? w.chunk_c0_48 : w.chunk_c0_64;
  tt.chunk_j = five ? w.chunk_j_48 : w.chunk_j_64;
  tt.chunk_first = first[i];
  tt.nchunks = first[P.M] - first[i];
  tt.k_lo = k_lo;
  tt.nk = k_hi - k_lo;
  const int total = tt.nk * tt.nchunks;
  if (total <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)(total < w.nsm ? total : w.nsm);
  if (fp8) {
    const CUtensorMap& mA = *reinterpret_cast<const CUtensorMap*>(w.tmA8);
    const CUtensorMap& mB = *reinterpret_cast<const CUtensorMap*>(w.tmB64_8);
    if (ftz)
      k_update_tc<4, 4, 64, true, true><<<grid, kTcThreads, TcGeom<4, 64>::smem, s>>>(P, i, tt, exX, nrmX, w.eA, w.F,
                                                                                     4, mA, mB);
    else
      k_update_tc<4, 4, 64, true><<<grid, kTcThreads, TcGeom<4, 64>::smem, s>>>(P, i, tt, exX, nrmX, w.eA, w.F, 4, mA,
                                                                               mB);
  } else if (five) {
    const CUtensorMap& mA = *reinterpret_cast<const CUtensorMap*>(w.tmA);
    const CUtensorMap& mB = *reinterpret_cast<const CUtensorMap*>(w.tmB48);
    if (ftz)
      k_update_tc<5, 5, 48, false, true><<<grid, kTcThreads, TcGeom<5, 48>::smem, s>>>(P, i, tt, exX, nrmX, w.eA, w.F,
                                                                                      w.ns, mA, mB);
    else
      k_update_tc<5, 5, 48><<<grid, kTcThreads, TcGeom<5, 48>::smem, s>>>(P, i, tt, exX, nrmX, w.eA, w.F, w.ns, mA, mB);
  } else {
    const CUtensorMap& mA = *reinterpret_cast<const CUtensorMap*>(w.tmA3);
    const CUtensorMap& mB = *reinterpret_cast<const CUtensorMap*>(w.tmB64);
    if (ftz)
      k_update_tc<3, 3, 64, false, true><<<grid, kTcThreads, TcGeom<3, 64>::smem, s>>>(P, i, tt, exX, nrmX, w.eA, w.F,
                                                                                      w.ns, mA, mB);
    else
      k_update_tc<3, 3, 64><<<grid, kTcThreads, TcGeom<3, 64>::smem, s>>>(P, i, tt, exX, nrmX, w.eA, w.F, w.ns, mA, mB);
  }
  return cudaGetLastError();
}

}  // namespace pevc

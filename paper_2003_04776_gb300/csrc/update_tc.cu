// update_tc.cu -- the split-precision update (Section 3, kernel 2) on the
// fifth-generation tensor cores, fed by TMA:
//     Y_kj <- 2^sY Y_kj - 2^sX [S_ki T_ki] X''_ij,   k in [k_lo, k_hi), j >= i,
// with [S_ki T_ki] and X'' given as exact BF16 slices (split.cu).
//
// Persistent, warp-specialised CTA of 6 warps:
//   warp 0   TMA producer: 3-D tensor-map boxes (8 elements x rows x K groups)
//            land directly in the canonical K-major core-matrix layout;
//   warp 1   tensor-memory owner and MMA issuer: every slice product p x q
//            with p + q < L is a tcgen05.mma (M=128, N=NCOL, K=16, BF16 in,
//            FP32 out) into the accumulator of its level p + q;
//   warps 2-5 epilogue: tcgen05.ld of the level accumulators, exact integer
//            recombination, augmented-tile scales (Algorithms 2 and 3 of
//            Section 4), one FP64 conversion and one FP64 subtraction per
//            element, new column maxima.
// Shared-memory stages form an mbarrier ring (full / empty); the level
// accumulators are double-buffered in tensor memory so that the epilogue of
// one output tile overlaps the MMAs of the next.  Every wait is bounded: a
// wait that runs out sets PEVC_ERR_TIMEOUT in the status word and the CTA
// winds down (all roles run out of bounded waits, tensor memory is freed).
#include <cuda.h>

#include "split.cuh"
#include "tc.cuh"

namespace pevc {

constexpr int kTmRows = 128;
constexpr int kTmKc = 32;                        // K per stage
constexpr int kTmGroups = kTmKc / 8;             // core-matrix columns per stage
constexpr int kTmLboA = kTmRows * 16;            // bytes between K-adjacent core matrices of A
constexpr int kTmSbo = 128;                      // bytes between M/N-adjacent core matrices
constexpr long kTmWait = 1L << 22;

template <int NS, int NCOL>
struct TmGeom {
  static constexpr int lbo_b = NCOL * 16;
  static constexpr int slice_a = kTmGroups * kTmLboA;
  static constexpr int slice_b = kTmGroups * lbo_b;
  static constexpr int stage = NS * (slice_a + slice_b);
  static constexpr int stages = (NS >= 5) ? 3 : 4;
  static constexpr int smem = stages * stage + 1024;   // + barriers
};

template <int L, int NCOL>
__host__ __device__ constexpr uint32_t tm_tmem_cols() {
  return (2 * L * NCOL <= 128) ? 128 : (2 * L * NCOL <= 256) ? 256 : 512;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(mbar))
      : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(mbar)), "r"(bytes));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(mbar)));
}
__device__ __forceinline__ void epi_barrier() { asm volatile("bar.sync 1, 128;\n" ::); }

struct TmTiles {
  const int* chunk_c0;   // first output column of every column chunk (global list)
  const int* chunk_j;    // its column tile
  int chunk_first;       // first chunk of column tile i
  int nchunks;           // chunks of column tiles >= i
  int k_lo, nk;
};

template <int NS, int L, int NCOL>
__global__ void __launch_bounds__(192, 1) k_update_tma(Problem P, int i, TmTiles tt, const int* __restrict__ exX,
                                                       const double* __restrict__ nrmX, const int* __restrict__ eA,
                                                       const int* __restrict__ F, int ns,
                                                       const __grid_constant__ CUtensorMap tmA,
                                                       const __grid_constant__ CUtensorMap tmB) {
  using G = TmGeom<NS, NCOL>;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + G::stages * G::stage);
  uint64_t* empty = full + G::stages;
  uint64_t* tfull = empty + G::stages;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);

  __shared__ int s_on[2][NCOL], s_sY[2][NCOL], s_sc[2][NCOL], s_e[2][NCOL], s_yz[2][NCOL];
  __shared__ unsigned long long s_key[2][NCOL];
  __shared__ int s_fail, s_stop;
  volatile int* fail = &s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tb = P.tb, K2 = 2 * tb;
  const int nkc = K2 / kTmKc;
  const int total = tt.nk * tt.nchunks;
  constexpr uint32_t kCols = tm_tmem_cols<L, NCOL>();
  constexpr uint32_t kTx = (uint32_t)G::stage;

  if (tid == 0) {
    for (int s = 0; s < G::stages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], 4); }
    s_fail = 0;
    s_stop = 0;
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
      uint32_t ph = 0;
      for (int t = blockIdx.x; t < total && !*fail; t += gridDim.x) {
        const int k = tt.k_lo + t / tt.nchunks;
        const int ch = tt.chunk_first + t % tt.nchunks;
        const int c0 = tt.chunk_c0[ch];
        const int a_plane = (int)(tri_index(k, i) * ns);
        for (int kc = 0; kc < nkc; ++kc) {
          if (!mbar_wait_bounded(&empty[s], ph ^ 1u, kTmWait)) { *fail = 1; break; }
          mbar_expect_tx(&full[s], kTx);
          unsigned char* a_dst = smem + s * G::stage;
          unsigned char* b_dst = a_dst + NS * G::slice_a;
          for (int p = 0; p < NS; ++p) {
            tma_load_4d(a_dst + p * G::slice_a, &tmA, 0, 0, kc * kTmGroups, a_plane + p, &full[s]);
            tma_load_4d(b_dst + p * G::slice_b, &tmB, 0, c0, kc * kTmGroups, p, &full[s]);
          }
          if (++s == G::stages) { s = 0; ph ^= 1u; }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(kTmRows, NCOL);
      int s = 0, buf = 0;
      uint32_t ph = 0, aph = 0;
      for (int t = blockIdx.x; t < total && !*fail; t += gridDim.x) {
        if (!mbar_wait_bounded(&tempty[buf], aph ^ 1u, kTmWait)) { *fail = 1; break; }
        tc_fence_after();
        const uint32_t acc0 = tmem + (uint32_t)(buf * L * NCOL);
        uint32_t started = 0;
        for (int kc = 0; kc < nkc; ++kc) {
          if (!mbar_wait_bounded(&full[s], ph, kTmWait)) { *fail = 1; break; }
          tc_fence_after();
          const uint32_t a_base = smem_addr(smem + s * G::stage);
          const uint32_t b_base = a_base + NS * G::slice_a;
#pragma unroll
          for (int kk = 0; kk < kTmKc / 16; ++kk)
#pragma unroll
            for (int p = 0; p < NS; ++p)
#pragma unroll
              for (int q = 0; q < NS; ++q)
                if (p + q < L) {
                  const uint64_t ad = smem_desc(a_base + p * G::slice_a + kk * 2 * kTmLboA, kTmLboA, kTmSbo);
                  const uint64_t bd = smem_desc(b_base + q * G::slice_b + kk * 2 * G::lbo_b, G::lbo_b, kTmSbo);
                  tc_mma_bf16(acc0 + (uint32_t)((p + q) * NCOL), ad, bd, idesc, (started >> (p + q)) & 1u);
                  started |= 1u << (p + q);
                }
          tc_commit(&empty[s]);             // frees the stage once these MMAs completed
          if (++s == G::stages) { s = 0; ph ^= 1u; }
        }
        if (*fail) break;
        tc_commit(&tfull[buf]);             // the tile's accumulators are complete
        buf ^= 1;
        if (buf == 0) aph ^= 1u;
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int et = tid - 64;                          // 0..127
    const int quarter = warp & 3;                     // tensor-memory lane quarter of this warp
    const int row = 32 * quarter + lane;
    int buf = 0;
    uint32_t aph = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
      // a uniform stop decision for the four epilogue warps
      if (et == 0) s_stop = *fail;
      epi_barrier();
      if (s_stop) break;
      const int k = tt.k_lo + t / tt.nchunks;
      const int ch = tt.chunk_first + t % tt.nchunks;
      const int j = tt.chunk_j[ch];
      const int c0 = tt.chunk_c0[ch];
      const int cs = P.cstart[j];
      const int nc = min(NCOL, P.cstart[j + 1] - c0);
      const int rk0 = P.toff[k], hk = P.toff[k + 1] - rk0;
      double* Yt = tile_ptr(P, k, j);
      // per-column consolidation + protection while the MMAs run
      if (et < NCOL) {
        int on = 0, sY = 0, sX = 0, en = 0;
        bool yz = true;
        if (et < nc) {
          const int q = c0 + et;
          on = update_scales(P, exX, nrmX, k, i, q, sY, sX, en, yz) ? 1 : 0;
          if (on && F[q] == kExpZero) on = 0;
          s_sc[buf][et] = on ? F[q] - 14 - 8 * (L - 1) + sX : 0;
        }
        s_on[buf][et] = on;
        s_sY[buf][et] = sY;
        s_e[buf][et] = en;
        s_yz[buf][et] = yz ? 1 : 0;
        s_key[buf][et] = 0ull;
      }
      const int erow = (row < tb) ? eA[tri_index(k, i) * tb + row] : 0;
      epi_barrier();
      // this thread's row of Y for every column of the tile, loaded (all
      // loads in flight at once) while the tile's MMAs run
      double yv[NCOL];
#pragma unroll
      for (int col = 0; col < NCOL; ++col) {
        yv[col] = 0.0;
        if (col < nc && row < hk && s_on[buf][col] && !s_yz[buf][col])
          yv[col] = Yt[(size_t)(c0 + col - cs) * tb + row];
      }
      const bool ok = mbar_wait_bounded(&tfull[buf], aph, kTmWait);
      if (!ok) *fail = 1;
      tc_fence_after();
      if (ok) {
        const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(buf * L * NCOL);
#pragma unroll
        for (int cb = 0; cb < NCOL; cb += 16) {
          uint32_t lv[L][16];
#pragma unroll
          for (int s = 0; s < L; ++s) tc_ld16(lane_base + (uint32_t)(s * NCOL + cb), lv[s]);
          tc_wait_ld();
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int col = cb + u;
            const bool con = col < nc && s_on[buf][col];
            unsigned long long key = 0;
            if (con && row < hk) {
              long long tv = 0;
#pragma unroll
              for (int s = 0; s < L; ++s) tv = (tv << 8) + (long long)__float2int_rn(__uint_as_float(lv[s][u]));
              const double prod = pow2_scale((double)tv, erow + s_sc[buf][col]);
              const double yold = pow2_scale(yv[col], s_sY[buf][col]);
              const double ynew = yold - prod;
              Yt[(size_t)(c0 + col - cs) * tb + row] = ynew;
              key = abs_key(ynew);
            }
            if (con) {
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o));
              if (lane == 0 && key) atomicMax(&s_key[buf][col], key);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
      epi_barrier();
      if (ok && et < nc && s_on[buf][et]) {
        const long long idx = (long long)k * P.m + c0 + et;
        P.nrm[idx] = __longlong_as_double((long long)s_key[buf][et]);
        P.ex[idx] = s_e[buf][et];
      }
      buf ^= 1;
      if (buf == 0) aph ^= 1u;
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
  cudaError_t a = cudaFuncSetAttribute(k_update_tma<5, 5, 48>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       TmGeom<5, 48>::smem);
  cudaError_t b = cudaFuncSetAttribute(k_update_tma<3, 3, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       TmGeom<3, 64>::smem);
  return (a == cudaSuccess && b == cudaSuccess && encode_fn()) ? 0 : PEVC_ERR_CUDA;
}

// Tensor maps over the core-matrix-major slice buffers:
//   A: [tile * ns + slice][K group][row][8]  -> dims {8, tb, 2tb/8, tiles*ns}, box {8, 128, 4, 1}
//   B: [slice][K group][column][8]           -> dims {8, n_max, 2tb/8, ns},    box {8, NCOL, 4, 1}
int make_tensor_maps(SplitWorkspace& w) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return PEVC_ERR_CUDA;
  const cuuint64_t tb = (cuuint64_t)w.tb, kg = (cuuint64_t)(2 * w.tb / 8);
  {
    cuuint64_t dims[4] = {8, tb, kg, (cuuint64_t)(w.tiles * w.ns)};
    cuuint64_t strides[3] = {16, tb * 16, kg * tb * 16};
    cuuint32_t box[4] = {8, (cuuint32_t)kTmRows, (cuuint32_t)kTmGroups, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    if (enc(reinterpret_cast<CUtensorMap*>(w.tmA), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, w.As, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return PEVC_ERR_CUDA;
  }
  for (int v = 0; v < 2; ++v) {
    const cuuint32_t ncol = v == 0 ? 48 : 64;
    cuuint64_t dims[4] = {8, (cuuint64_t)w.n_max, kg, (cuuint64_t)w.ns};
    cuuint64_t strides[3] = {16, (cuuint64_t)w.n_max * 16, kg * (cuuint64_t)w.n_max * 16};
    cuuint32_t box[4] = {8, ncol, (cuuint32_t)kTmGroups, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    if (enc(reinterpret_cast<CUtensorMap*>(v == 0 ? w.tmB48 : w.tmB64), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, w.Xs,
            dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return PEVC_ERR_CUDA;
  }
  return 0;
}

cudaError_t launch_update_tc(const Problem& P, const SplitWorkspace& w, int i, int k_lo, int k_hi, const int* exX,
                             const double* nrmX, int ns, int levels, cudaStream_t s) {
  if (k_hi <= k_lo) return cudaSuccess;
  const bool five = (ns == 5 && levels == 5);
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
  const CUtensorMap& mA = *reinterpret_cast<const CUtensorMap*>(w.tmA);
  if (five) {
    const CUtensorMap& mB = *reinterpret_cast<const CUtensorMap*>(w.tmB48);
    k_update_tma<5, 5, 48><<<grid, 192, TmGeom<5, 48>::smem, s>>>(P, i, tt, exX, nrmX, w.eA, w.F, w.ns, mA, mB);
  } else {
    const CUtensorMap& mB = *reinterpret_cast<const CUtensorMap*>(w.tmB64);
    k_update_tma<3, 3, 64><<<grid, 192, TmGeom<3, 64>::smem, s>>>(P, i, tt, exX, nrmX, w.eA, w.F, w.ns, mA, mB);
  }
  return cudaGetLastError();
}

}  // namespace pevc

// update_tc.cu -- the split-precision update (Section 3, kernel 2) on the
// fifth-generation tensor cores:
//     Y_kj <- 2^sY Y_kj - 2^sX [S_ki T_ki] X''_ij,   k in [k_lo, k_hi), j >= i,
// with [S_ki T_ki] and X'' given as exact BF16 slices (split.cu).  One CTA
// (4 warps) owns 128 rows x 64 columns.  Every slice product p x q with
// p + q < L is a tcgen05.mma (M=128, N=64, K=16, BF16 in, FP32 out) into the
// accumulator of its level p + q, held in tensor memory; one thread issues the
// MMAs, cp.async double-buffers the K chunks in the canonical K-major layout,
// an mbarrier per buffer reports MMA completion (every wait is bounded and
// reports PEVC_ERR_TIMEOUT through the status word).  The epilogue reads the
// level accumulators with tcgen05.ld, combines them exactly as one integer and
// applies the augmented-tile scales (Algorithms 2 and 3 of Section 4) with
// one FP64 conversion and one FP64 subtraction per element.
#include "split.cuh"
#include "tc.cuh"

namespace pevc {

constexpr int kTcRows = 128;
constexpr int kTcCols = 64;
constexpr int kTcKc = 32;                              // K per pipeline stage
constexpr int kTcLboA = (kTcRows / 8) * 128;           // bytes between K-adjacent core matrices (A)
constexpr int kTcLboB = (kTcCols / 8) * 128;           // (B)
constexpr int kTcSbo = 128;                            // bytes between M/N-adjacent core matrices
constexpr int kTcSliceA = (kTcKc / 8) * kTcLboA;       // one slice of one stage
constexpr int kTcSliceB = (kTcKc / 8) * kTcLboB;
constexpr long kTcWaitLimit = 1L << 22;

template <int NS>
__host__ __device__ constexpr int tc_stage_bytes() { return NS * (kTcSliceA + kTcSliceB); }
template <int NS>
__host__ __device__ constexpr int tc_smem_bytes() { return 2 * tc_stage_bytes<NS>(); }
template <int L>
__host__ __device__ constexpr uint32_t tc_tmem_cols() {
  return (L * kTcCols <= 32) ? 32 : (L * kTcCols <= 64) ? 64 : (L * kTcCols <= 128) ? 128 : (L * kTcCols <= 256) ? 256 : 512;
}

template <int NS, int L>
__global__ void __launch_bounds__(128) k_update_tc(Problem P, int i, int k_lo, const int* __restrict__ exX,
                                                   const double* __restrict__ nrmX,
                                                   const __nv_bfloat16* __restrict__ As,
                                                   const int* __restrict__ eA,
                                                   const __nv_bfloat16* __restrict__ Xs,
                                                   const int* __restrict__ F, int ns, int mstride) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tb = P.tb, K2 = 2 * tb;
  const int nsub = (tb + kTcCols - 1) / kTcCols;
  const int j = i + (int)blockIdx.x / nsub;
  const int sub = (int)blockIdx.x % nsub;
  const int k = k_lo + (int)blockIdx.y;
  const int cs = P.cstart[j], ce = P.cstart[j + 1];
  const int c0 = cs + sub * kTcCols;
  if (c0 >= ce) return;
  const int nc = min(kTcCols, ce - c0);
  const int rk0 = P.toff[k], hk = P.toff[k + 1] - rk0;
  double* Yt = tile_ptr(P, k, j);
  const long long tri = tri_index(k, i);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  __shared__ int s_sY[kTcCols], s_sc[kTcCols], s_e[kTcCols], s_on[kTcCols], s_yz[kTcCols];
  __shared__ unsigned long long s_key[kTcCols];
  __shared__ int s_eA[kTcRows];
  __shared__ int s_any, s_fail;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mbar[2];

  if (tid == 0) { s_any = 0; s_fail = 0; }
  __syncthreads();
  if (tid < kTcCols) {
    int on = 0, sY = 0, sX = 0, en = 0;
    bool yz = true;
    if (tid < nc) {
      const int q = c0 + tid;
      on = update_scales(P, exX, nrmX, k, i, q, sY, sX, en, yz) ? 1 : 0;
      if (on && F[q] == kExpZero) on = 0;
      s_sc[tid] = on ? F[q] - 14 - 8 * (L - 1) + sX : 0;
    }
    s_on[tid] = on;
    s_sY[tid] = sY;
    s_e[tid] = en;
    s_yz[tid] = yz ? 1 : 0;
    s_key[tid] = 0ull;
    if (on) atomicOr(&s_any, 1);
  }
  s_eA[tid] = (tid < tb) ? eA[tri * tb + tid] : 0;
  __syncthreads();
  if (!s_any) return;

  constexpr uint32_t kCols = tc_tmem_cols<L>();
  if (warp == 0) tc_alloc(&s_tmem, kCols);
  if (tid == 0) {
    mbar_init(&s_mbar[0], 1);
    mbar_init(&s_mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  const __nv_bfloat16* Abase = As + tri * ns * (long long)tb * K2;
  auto load_stage = [&](int st, int kb) {
    unsigned char* a_dst = smem + st * tc_stage_bytes<NS>();
    unsigned char* b_dst = a_dst + NS * kTcSliceA;
    constexpr int groups = kTcKc / 8;
    for (int idx = tid; idx < NS * kTcRows * groups; idx += 128) {
      const int g = idx % groups, r = (idx / groups) % kTcRows, p = idx / (groups * kTcRows);
      const bool valid = r < tb;
      const __nv_bfloat16* src = Abase + ((long long)p * tb + (valid ? r : 0)) * K2 + kb + 8 * g;
      cp_async16_zfill(a_dst + p * kTcSliceA + g * kTcLboA + (r >> 3) * kTcSbo + (r & 7) * 16, src, valid);
    }
    for (int idx = tid; idx < NS * kTcCols * groups; idx += 128) {
      const int g = idx % groups, col = (idx / groups) % kTcCols, p = idx / (groups * kTcCols);
      const bool valid = col < nc;
      const __nv_bfloat16* src = Xs + ((long long)p * mstride + c0 + (valid ? col : 0)) * K2 + kb + 8 * g;
      cp_async16_zfill(b_dst + p * kTcSliceB + g * kTcLboB + (col >> 3) * kTcSbo + (col & 7) * 16, src, valid);
    }
  };

  constexpr uint32_t idesc = idesc_bf16_f32(kTcRows, kTcCols);
  const int nchunks = K2 / kTcKc;
  uint32_t started = 0;   // levels whose accumulator already holds data (issuing thread only)
  bool ok = true;
  load_stage(0, 0);
  cp_async_commit_group();
  for (int ch = 0; ch < nchunks && ok; ++ch) {
    const int st = ch & 1;
    if (ch + 1 < nchunks) {
      if (ch >= 1) {   // the buffer of chunk ch+1 was read by the MMAs of chunk ch-1
        if (!mbar_wait_bounded(&s_mbar[st ^ 1], ((ch - 1) >> 1) & 1, kTcWaitLimit)) {
          atomicExch(&s_fail, 1);
        }
      }
      load_stage(st ^ 1, (ch + 1) * kTcKc);
    }
    cp_async_commit_group();
    cp_async_wait_group<1>();
    fence_async_smem();
    __syncthreads();
    if (s_fail) { ok = false; break; }
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a_base = smem_addr(smem + st * tc_stage_bytes<NS>());
      const uint32_t b_base = a_base + NS * kTcSliceA;
#pragma unroll
      for (int kk = 0; kk < kTcKc / 16; ++kk) {
#pragma unroll
        for (int p = 0; p < NS; ++p)
#pragma unroll
          for (int q = 0; q < NS; ++q) {
            if (p + q < L) {
              const int s = p + q;
              const uint64_t ad = smem_desc(a_base + p * kTcSliceA + kk * 2 * kTcLboA, kTcLboA, kTcSbo);
              const uint64_t bd = smem_desc(b_base + q * kTcSliceB + kk * 2 * kTcLboB, kTcLboB, kTcSbo);
              tc_mma_bf16(tmem + s * kTcCols, ad, bd, idesc, (started >> s) & 1u);
              started |= 1u << s;
            }
          }
      }
      tc_commit(&s_mbar[st]);
    }
  }
  cp_async_wait_group<0>();
  if (ok) {
    const int last = nchunks - 1;
    if (!mbar_wait_bounded(&s_mbar[last & 1], (last >> 1) & 1, kTcWaitLimit)) atomicExch(&s_fail, 1);
  }
  tc_fence_after();
  __syncthreads();
  const bool good = ok && !s_fail;

  if (good) {
    const int row = 32 * warp + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    for (int cb = 0; cb < kTcCols; cb += 16) {
      uint32_t lv[L][16];
#pragma unroll
      for (int s = 0; s < L; ++s) tc_ld16(lane_base + s * kTcCols + cb, lv[s]);
      tc_wait_ld();
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int col = cb + u;
        unsigned long long key = 0;
        const bool con = col < nc && s_on[col];
        if (con && row < hk) {
          long long t = 0;
#pragma unroll
          for (int s = 0; s < L; ++s) t = (t << 8) + (long long)__float2int_rn(__uint_as_float(lv[s][u]));
          double* ycol = Yt + (size_t)(c0 + col - cs) * tb;
          const double prod = pow2_scale((double)t, s_eA[row] + s_sc[col]);
          const double yold = s_yz[col] ? 0.0 : pow2_scale(ycol[row], s_sY[col]);
          const double ynew = yold - prod;
          ycol[row] = ynew;
          key = abs_key(ynew);
        }
        if (con) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) key = max(key, __shfl_xor_sync(0xffffffffu, key, o));
          if (lane == 0 && key) atomicMax(&s_key[col], key);
        }
      }
    }
  } else if (tid == 0) {
    atomicOr(P.status, kStTimeout);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, kCols);
  if (good && tid < nc && s_on[tid]) {
    const long long idx = (long long)k * P.m + c0 + tid;
    P.nrm[idx] = __longlong_as_double((long long)s_key[tid]);
    P.ex[idx] = s_e[tid];
  }
}

int update_tc_setup() {
  cudaError_t a = cudaFuncSetAttribute(k_update_tc<3, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       tc_smem_bytes<3>());
  cudaError_t b = cudaFuncSetAttribute(k_update_tc<5, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       tc_smem_bytes<5>());
  return (a == cudaSuccess && b == cudaSuccess) ? 0 : PEVC_ERR_CUDA;
}

cudaError_t launch_update_tc(const Problem& P, const SplitWorkspace& w, int i, int k_lo, int k_hi, const int* exX,
                             const double* nrmX, int ns, int levels, cudaStream_t s) {
  if (k_hi <= k_lo) return cudaSuccess;
  const int nsub = (P.tb + kTcCols - 1) / kTcCols;
  dim3 grid((P.M - i) * nsub, k_hi - k_lo);
  if (ns == 5 && levels == 5)
    k_update_tc<5, 5><<<grid, 128, tc_smem_bytes<5>(), s>>>(P, i, k_lo, exX, nrmX, w.As, w.eA, w.Xs, w.F, w.ns,
                                                             w.n_max);
  else
    k_update_tc<3, 3><<<grid, 128, tc_smem_bytes<3>(), s>>>(P, i, k_lo, exX, nrmX, w.As, w.eA, w.Xs, w.F, w.ns,
                                                             w.n_max);
  return cudaGetLastError();
}

}  // namespace pevc

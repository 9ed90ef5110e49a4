// cuda_runtime.h stand-in for the kernel emulation tests -- TEST INFRASTRUCTURE.
//
// Compiles the library's CUDA C++ kernel sources as host C++ and runs them on
// a model of the CUDA thread model: one host thread per thread of a block
// (blocks of a grid run one after another), std::barrier for
// __syncthreads, per-warp exchange slots for shuffles, votes and reductions,
// CTA-wide statics for __shared__, host memory for device memory, and
// synchronous stream operations (launches run in program order, which every
// stream and event dependency of the library respects).  Math functions are
// the host's.  The PTX the library uses outside its tcgen05 kernel is
// modelled from its documented semantics: mma.sync m8n8k4 f64 and m16n8k16
// bf16 (fragment layouts), ldmatrix.x4, cp.async (completed at once), and the
// mbarrier operations and clock64 of the bounded-wait self-test.  The tcgen05
// / TMA update is not covered.  Nothing in the library uses this file.
#pragma once
#include <math.h>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <cfloat>
#include <atomic>
#include <barrier>
#include <memory>
#include <thread>
#include <vector>

#define __host__
#define __device__
#define __global__
#define __forceinline__ inline
#define __launch_bounds__(...)
#define __shared__ static

typedef int cudaError_t;
enum { cudaSuccess = 0, cudaErrorInvalidValue = 1, cudaErrorMemoryAllocation = 2 };
typedef void* cudaStream_t;
typedef void* cudaEvent_t;
enum cudaMemcpyKind { cudaMemcpyHostToDevice, cudaMemcpyDeviceToHost, cudaMemcpyDeviceToDevice };
enum cudaFuncAttribute { cudaFuncAttributeMaxDynamicSharedMemorySize };
struct double2 { double x, y; };
inline double2 make_double2(double x, double y) { return {x, y}; }
struct dim3 {
  unsigned x, y, z;
  dim3(unsigned a = 1, unsigned b = 1, unsigned c = 1) : x(a), y(b), z(c) {}
};
struct uint3 { unsigned x, y, z; };
struct int4 { int x, y, z, w; };
inline int4 make_int4(int x, int y, int z, int w) { return {x, y, z, w}; }

inline cudaError_t cudaEventRecord(cudaEvent_t, cudaStream_t) { return 0; }
inline cudaError_t cudaGetLastError() { return 0; }
inline cudaError_t cudaStreamSynchronize(cudaStream_t) { return 0; }
inline cudaError_t cudaMemcpyAsync(void* d, const void* s, size_t b, cudaMemcpyKind, cudaStream_t) {
  memcpy(d, s, b);
  return 0;
}
inline cudaError_t cudaMemcpy2DAsync(void* d, size_t dp, const void* s, size_t sp, size_t w, size_t h,
                                     cudaMemcpyKind, cudaStream_t) {
  for (size_t r = 0; r < h; ++r) memcpy((char*)d + r * dp, (const char*)s + r * sp, w);
  return 0;
}
inline cudaError_t cudaMemsetAsync(void* d, int v, size_t b, cudaStream_t) {
  memset(d, v, b);
  return 0;
}
// Every device or pinned-host allocation the library makes is counted, so
// that a test can show an entry point allocates nothing.
inline std::atomic<long long> g_emu_allocs{0};
inline cudaError_t cudaMalloc(void** p, size_t b) {
  g_emu_allocs.fetch_add(1);
  *p = calloc(b ? b : 1, 1);
  return *p ? 0 : cudaErrorMemoryAllocation;
}
inline cudaError_t cudaMallocHost(void** p, size_t b) { return cudaMalloc(p, b); }
template <class T>
inline cudaError_t cudaMalloc(T** p, size_t b) { return cudaMalloc(reinterpret_cast<void**>(p), b); }
template <class T>
inline cudaError_t cudaMallocHost(T** p, size_t b) { return cudaMalloc(reinterpret_cast<void**>(p), b); }
inline cudaError_t cudaFree(void* p) { free(p); return 0; }
inline cudaError_t cudaFreeHost(void* p) { free(p); return 0; }
template <class F>
inline cudaError_t cudaFuncSetAttribute(F, cudaFuncAttribute, int) { return 0; }

namespace emu {
struct Warp {
  std::barrier<> bar{32};
  uint64_t slot[32];
};
struct Cta {
  std::barrier<>* bar;
};
inline thread_local uint3 tIdx, bIdx;
inline thread_local dim3 bDim, gDim;
inline thread_local Warp* warp = nullptr;
inline thread_local int lane = 0;
inline thread_local Cta* cta = nullptr;
inline thread_local unsigned char* dyn_smem = nullptr;

template <class T>
inline T shfl(T v, int src) {
  static_assert(sizeof(T) <= 8);
  uint64_t b = 0;
  memcpy(&b, &v, sizeof(T));
  warp->slot[lane] = b;
  warp->bar.arrive_and_wait();
  const uint64_t r = warp->slot[src & 31];
  warp->bar.arrive_and_wait();
  T out;
  memcpy(&out, &r, sizeof(T));
  return out;
}

template <class K, class... A>
void launch(K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t, A... args) {
  // one host thread per CUDA thread of a block, reused for every block of the
  // grid in turn (blocks run one after another; a barrier separates them)
  const int nt = (int)(block.x * block.y * block.z);
  const long long nb = (long long)grid.x * grid.y * grid.z;
  if (nt <= 0 || nb <= 0) return;
  std::vector<unsigned char> dyn(smem ? smem : 16);
  std::barrier<> bar(nt);
  Cta c{&bar};
  std::vector<std::unique_ptr<Warp>> ws((nt + 31) / 32);
  for (auto& w : ws) w.reset(new Warp);
  std::vector<std::thread> th;
  th.reserve(nt);
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      tIdx = uint3{(unsigned)(t % block.x), (unsigned)((t / block.x) % block.y), (unsigned)(t / (block.x * block.y))};
      bDim = block;
      gDim = grid;
      warp = ws[t / 32].get();
      lane = t % 32;
      cta = &c;
      dyn_smem = dyn.data();
      for (long long b = 0; b < nb; ++b) {
        bIdx = uint3{(unsigned)(b % grid.x), (unsigned)((b / grid.x) % grid.y), (unsigned)(b / ((long long)grid.x * grid.y))};
        kernel(args...);
        bar.arrive_and_wait();   // the block's shared memory is reused by the next block
      }
    });
  for (auto& x : th) x.join();
}
}  // namespace emu

#define threadIdx emu::tIdx
#define blockIdx emu::bIdx
#define blockDim emu::bDim
#define gridDim emu::gDim

inline void __syncthreads() { emu::cta->bar->arrive_and_wait(); }
template <class T>
inline T __shfl_sync(unsigned, T v, int src) { return emu::shfl(v, src & 31); }
template <class T>
inline T __shfl_xor_sync(unsigned, T v, int o) { return emu::shfl(v, emu::lane ^ o); }
inline int __reduce_max_sync(unsigned, int v) {
  int best = v;
  for (int l = 0; l < 32; ++l) best = std::max(best, emu::shfl(v, l));
  return best;
}
inline int __any_sync(unsigned, int p) {
  int r = 0;
  for (int l = 0; l < 32; ++l) r |= emu::shfl(p ? 1 : 0, l);
  return r;
}
inline int __all_sync(unsigned, int p) {
  int r = 1;
  for (int l = 0; l < 32; ++l) r &= emu::shfl(p ? 1 : 0, l);
  return r;
}

inline long long __double_as_longlong(double d) { long long r; memcpy(&r, &d, 8); return r; }
inline double __longlong_as_double(long long l) { double r; memcpy(&r, &l, 8); return r; }
inline int __double2hiint(double d) { return (int)((unsigned long long)__double_as_longlong(d) >> 32); }
inline int __double2loint(double d) { return (int)(uint32_t)__double_as_longlong(d); }
inline double __hiloint2double(int hi, int lo) {
  return __longlong_as_double((long long)(((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo));
}
inline int __clzll(long long x) { return x ? __builtin_clzll((unsigned long long)x) : 64; }
inline int __clz(int x) { return x ? __builtin_clz((unsigned)x) : 32; }
template <class T>
inline T max(T a, T b) { return a > b ? a : b; }
template <class T>
inline T min(T a, T b) { return a < b ? a : b; }
inline unsigned atomicOr(unsigned* a, unsigned v) { return std::atomic_ref<unsigned>(*a).fetch_or(v); }
inline int atomicOr(int* a, int v) { return std::atomic_ref<int>(*a).fetch_or(v); }
inline int atomicAdd(int* a, int v) { return std::atomic_ref<int>(*a).fetch_add(v); }
inline int atomicExch(int* a, int v) { return std::atomic_ref<int>(*a).exchange(v); }
inline void __threadfence() { std::atomic_thread_fence(std::memory_order_seq_cst); }
inline void __nanosleep(unsigned) {}
inline unsigned atomicAdd(unsigned* a, unsigned v) { return std::atomic_ref<unsigned>(*a).fetch_add(v); }
inline int atomicMax(int* a, int v) {
  std::atomic_ref<int> r(*a);
  int cur = r.load();
  while (cur < v && !r.compare_exchange_weak(cur, v)) {}
  return cur;
}
inline unsigned long long atomicMax(unsigned long long* a, unsigned long long v) {
  std::atomic_ref<unsigned long long> r(*a);
  unsigned long long cur = r.load();
  while (cur < v && !r.compare_exchange_weak(cur, v)) {}
  return cur;
}

// ---- additions for the real-pencil path ----
#define __align__(n) __attribute__((aligned(n)))
enum { cudaStreamNonBlocking = 1, cudaEventDisableTiming = 2 };
enum cudaDeviceAttr { cudaDevAttrMultiProcessorCount };
inline cudaError_t cudaSetDevice(int) { return 0; }
inline cudaError_t cudaGetDevice(int* d) { *d = 0; return 0; }
inline cudaError_t cudaDeviceGetAttribute(int* v, cudaDeviceAttr, int) { *v = 152; return 0; }
inline cudaError_t cudaStreamCreateWithFlags(cudaStream_t* s, unsigned) { *s = (void*)0x1; return 0; }
inline cudaError_t cudaStreamDestroy(cudaStream_t) { return 0; }
inline cudaError_t cudaStreamWaitEvent(cudaStream_t, cudaEvent_t, unsigned = 0) { return 0; }
inline cudaError_t cudaEventCreate(cudaEvent_t* e) { *e = (void*)0x1; return 0; }
inline cudaError_t cudaEventCreateWithFlags(cudaEvent_t* e, unsigned) { *e = (void*)0x1; return 0; }
inline cudaError_t cudaEventDestroy(cudaEvent_t) { return 0; }
inline cudaError_t cudaEventElapsedTime(float* ms, cudaEvent_t, cudaEvent_t) { *ms = 0.f; return 0; }
template <class T>
inline cudaError_t cudaGetSymbolAddress(void** p, T& sym) { *p = (void*)&sym; return 0; }

namespace emu {
inline void allgather(double v, double (&out)[32]) {
  uint64_t b;
  memcpy(&b, &v, 8);
  warp->slot[lane] = b;
  warp->bar.arrive_and_wait();
  for (int l = 0; l < 32; ++l) memcpy(&out[l], &warp->slot[l], 8);
  warp->bar.arrive_and_wait();
}
// mma.sync.m8n8k4 row.col f64: A 8x4 from lane row*4 + k, B 4x8 from lane
// col*4 + k, C/D at row = lane >> 2, cols 2 (lane & 3) + {0, 1}.
inline void dmma_m8n8k4(double& c0, double& c1, double a, double b) {
  double A[32], B[32];
  allgather(a, A);
  allgather(b, B);
  const int row = lane >> 2, col0 = (lane & 3) * 2;
  double acc0 = c0, acc1 = c1;
  for (int k = 0; k < 4; ++k) {
    acc0 = fma(A[row * 4 + k], B[col0 * 4 + k], acc0);
    acc1 = fma(A[row * 4 + k], B[(col0 + 1) * 4 + k], acc1);
  }
  c0 = acc0;
  c1 = acc1;
}
}  // namespace emu

// ---- mbarrier and clock model for the bounded-wait self-test ----
// An mbarrier word holds {expected count, pending count, phase}; an arrival
// that completes the phase flips its parity and rearms the count, and
// try_wait.parity(p) succeeds once the phase with parity p has completed.
#include <chrono>
namespace emu {
inline void mbar_init(uint64_t* m, uint32_t count) { *m = ((uint64_t)count << 32) | ((uint64_t)count << 1); }
inline void mbar_arrive(uint64_t* m) {
  std::atomic_ref<uint64_t> r(*m);
  uint64_t cur = r.load(), nxt;
  do {
    const uint64_t cnt = cur >> 32, pend = (cur >> 1) & 0x7fffffffu, ph = cur & 1u;
    nxt = pend > 1 ? (cnt << 32) | ((pend - 1) << 1) | ph : (cnt << 32) | (cnt << 1) | (ph ^ 1u);
  } while (!r.compare_exchange_weak(cur, nxt));
}
inline bool mbar_try_wait(uint64_t* m, uint32_t parity) {
  return (std::atomic_ref<uint64_t>(*m).load() & 1u) != parity;
}
}  // namespace emu
inline long long clock64() {
  // about 2 GHz, the order of this GPU's SM clock
  return (long long)(std::chrono::duration_cast<std::chrono::nanoseconds>(
                         std::chrono::steady_clock::now().time_since_epoch()).count() * 2);
}

// ---- the split path's PTX: cp.async, ldmatrix.x4 and mma.sync m16n8k16 bf16 ----
struct uint4 { unsigned x, y, z, w; };
struct uint2 { unsigned x, y; };
inline size_t __cvta_generic_to_shared(const void* p) { return (size_t)p; }
inline int __float2int_rn(float f) { return (int)lrintf(f); }
namespace emu {
// cp.async of 16 bytes with zero fill, completed at once (the waits become no-ops)
inline void cp_async16(void* smem, const void* gmem, bool valid) {
  if (valid) memcpy(smem, gmem, 16);
  else memset(smem, 0, 16);
}
// ldmatrix.sync.aligned.m8n8.x4.b16: lanes 8i .. 8i+7 give the row addresses
// of matrix i; lane L receives, from each matrix i, the 32-bit pair of
// elements 2 (L % 4), 2 (L % 4) + 1 of row L / 4.
inline void ldmatrix_x4(unsigned (&r)[4], const void* row_addr) {
  const uint64_t mine = (uint64_t)(size_t)row_addr;
  uint64_t addr[32];
  warp->slot[lane] = mine;
  warp->bar.arrive_and_wait();
  for (int l = 0; l < 32; ++l) addr[l] = warp->slot[l];
  warp->bar.arrive_and_wait();
  for (int i = 0; i < 4; ++i)
    memcpy(&r[i], reinterpret_cast<const unsigned char*>((size_t)addr[8 * i + lane / 4]) + 4 * (lane % 4), 4);
}
inline float bf16_lo(unsigned w) { const unsigned b = w << 16; float f; memcpy(&f, &b, 4); return f; }
inline float bf16_hi(unsigned w) { const unsigned b = w & 0xffff0000u; float f; memcpy(&f, &b, 4); return f; }
// mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 (g = lane / 4, t = lane % 4):
//   A regs (row, k pair): {g, 2t}, {g+8, 2t}, {g, 2t+8}, {g+8, 2t+8};
//   B regs (k pair, col): {2t, g}, {2t+8, g};  C: rows g, g+8, cols 2t, 2t+1.
// The split path's products are exact integers below 2^24, so the order of
// the FP32 additions does not matter.
inline void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  unsigned A[32][4], B[32][2];
  for (int q = 0; q < 4; ++q) {
    warp->slot[lane] = a[q];
    warp->bar.arrive_and_wait();
    for (int l = 0; l < 32; ++l) A[l][q] = (unsigned)warp->slot[l];
    warp->bar.arrive_and_wait();
  }
  for (int q = 0; q < 2; ++q) {
    warp->slot[lane] = q ? b1 : b0;
    warp->bar.arrive_and_wait();
    for (int l = 0; l < 32; ++l) B[l][q] = (unsigned)warp->slot[l];
    warp->bar.arrive_and_wait();
  }
  auto a_el = [&](int row, int k) {
    const int l = (row % 8) * 4 + (k % 8) / 2, q = row / 8 + 2 * (k / 8);
    return (k & 1) ? bf16_hi(A[l][q]) : bf16_lo(A[l][q]);
  };
  auto b_el = [&](int k, int col) {
    const int l = col * 4 + (k % 8) / 2, q = k / 8;
    return (k & 1) ? bf16_hi(B[l][q]) : bf16_lo(B[l][q]);
  };
  const int g = lane >> 2, t = lane & 3;
  for (int e = 0; e < 4; ++e) {
    const int row = g + 8 * (e >> 1), col = 2 * t + (e & 1);
    float acc = c[e];
    for (int k = 0; k < 16; ++k) acc += a_el(row, k) * b_el(k, col);
    c[e] = acc;
  }
}
// E4M3 byte to float: sign, 4-bit exponent (bias 7; 0 = subnormal), 3-bit
// mantissa (exponent 15 with mantissa 7 is NaN, never produced by the slices).
inline float e4m3_value(unsigned b) {
  const int sgn = (b >> 7) & 1, E = (b >> 3) & 15, m = b & 7;
  const float mag = E ? std::ldexp(1.0f + m / 8.0f, E - 7) : std::ldexp(m / 8.0f, -6);
  return sgn ? -mag : mag;
}
// mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 (g = lane / 4, t = lane % 4),
// four bytes per register, element k of a register at byte k % 4:
//   A regs (row, k quad): {g, 4t}, {g+8, 4t}, {g, 4t+16}, {g+8, 4t+16};
//   B regs (k quad, col): {4t, g}, {4t+16, g};  C as m16n8k16.
inline void mma_e4m3(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  unsigned A[32][4], B[32][2];
  for (int q = 0; q < 4; ++q) {
    warp->slot[lane] = a[q];
    warp->bar.arrive_and_wait();
    for (int l = 0; l < 32; ++l) A[l][q] = (unsigned)warp->slot[l];
    warp->bar.arrive_and_wait();
  }
  for (int q = 0; q < 2; ++q) {
    warp->slot[lane] = q ? b1 : b0;
    warp->bar.arrive_and_wait();
    for (int l = 0; l < 32; ++l) B[l][q] = (unsigned)warp->slot[l];
    warp->bar.arrive_and_wait();
  }
  auto a_el = [&](int row, int k) {
    const int l = (row % 8) * 4 + (k % 16) / 4, q = row / 8 + 2 * (k / 16);
    return e4m3_value((A[l][q] >> (8 * (k % 4))) & 0xffu);
  };
  auto b_el = [&](int k, int col) {
    const int l = col * 4 + (k % 16) / 4, q = k / 16;
    return e4m3_value((B[l][q] >> (8 * (k % 4))) & 0xffu);
  };
  const int g = lane >> 2, t = lane & 3;
  for (int e = 0; e < 4; ++e) {
    const int row = g + 8 * (e >> 1), col = 2 * t + (e & 1);
    float acc = c[e];
    for (int k = 0; k < 32; ++k) acc += a_el(row, k) * b_el(k, col);
    c[e] = acc;
  }
}
}  // namespace emu


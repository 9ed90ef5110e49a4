// split.cuh -- split-precision path: kernel 2 of Section 3 (the updates
// Y <- Y - (S X D - T X B)) as exact products of BF16 slices on the tensor
// cores, with FP32 accumulation per slice level and an FP64 epilogue, and the
// FP64-faithful residual correction sweep.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace pevc {

constexpr int kMaxSlices = 5;

struct SplitConfig {
  int ns1 = 3, levels1 = 3;      // slices / levels of the solve passes
  int ns_res = 5, levels_res = 5;  // slices / levels of the residual
  bool correction = true;
  int sweeps = 1;                  // correction sweeps (iterative refinement) when correction is on:
                                   // the count, or with `adaptive` the most
  bool adaptive = false;           // stop once the correction has converged
  bool fp8 = false;                // solve passes on FP8 E4M3 slices (4-bit digits)
};

struct SplitWorkspace {
  bool on = false;
  int tb = 0, n_max = 0, Mmax = 0, ns = 0;
  size_t tiles = 0;
  __nv_bfloat16* As = nullptr;   // [tile (k<=l)][slice][tb][2 tb]   row slices of [S_kl T_kl]
  int* eA = nullptr;             // [tile (k<=l)][tb]                row exponents
  __nv_bfloat16* Xs = nullptr;   // [slice][n_max][2 tb]             column slices of X''
  bool fp8 = false;              // FP8 plans: the E4M3 slices below
  unsigned char* As8 = nullptr;  // [tile (k<=l)][4][tb][2 tb]       E4M3 row slices of [S_kl T_kl]
  unsigned char* Xs8 = nullptr;  // [4][n_max][2 tb]                 E4M3 column slices of X''
  int* F = nullptr;              // [n_max]                          column exponents of X''
  int* d_sweep = nullptr;        // device int: size of the last correction (log2, relative to V)
  int* h_sweep = nullptr;        // pinned host copy of it
  int last_sweeps = 0;           // correction sweeps the last solve ran
  double* Y2 = nullptr;          // correction tiles
  int* ex2 = nullptr;
  double* nrm2 = nullptr;
  bool use_tc = true;            // tcgen05 update kernel (else the mma.sync one)
  bool tc_ok = false;            // tensor maps built (tiles of order 128)
  int nsm = 0;
  // TMA tensor maps over As and Xs (CUtensorMap storage: 128 bytes, 64-aligned):
  // A boxes of 5 and 3 slices, X'' boxes of 48 columns x 5 slices and 64 x 3
  alignas(64) unsigned char tmA[128];
  alignas(64) unsigned char tmA3[128];
  alignas(64) unsigned char tmB48[128];
  alignas(64) unsigned char tmB64[128];
  // FP8 plans: E4M3 A boxes of 4 slices, X'' boxes of 64 columns x 4 slices
  alignas(64) unsigned char tmA8[128];
  alignas(64) unsigned char tmB64_8[128];
  // output column chunks of width 48 / 64 inside each column tile (per solve)
  int* chunk_c0_48 = nullptr;
  int* chunk_j_48 = nullptr;
  int* chunk_c0_64 = nullptr;
  int* chunk_j_64 = nullptr;
  int* h_chunk_first48 = nullptr;   // host [Mmax + 1]
  int* h_chunk_first64 = nullptr;
  int* h_chunks = nullptr;          // host staging
  int max_chunks = 0;
};

// Host copies of the structure, for launch shapes and work counts.
struct HostStructure {
  const int* toff;
  const int* cstart;
};

struct SchedContext {
  cudaStream_t aux = nullptr;   // second stream for the lookahead solves
  cudaEvent_t* ev = nullptr;    // 2 * Mmax events
  bool lookahead = true;
};

int split_alloc(SplitWorkspace& w, int n_max, int tb, int Mmax, int prec);
int update_tc_setup();
int make_tensor_maps(SplitWorkspace& w);
cudaError_t launch_update_tc(const Problem& P, const SplitWorkspace& w, int i, int k_lo, int k_hi, const int* exX,
                             const double* nrmX, int ns, int levels, bool fp8, cudaStream_t s, bool ftz = false);
void split_free(SplitWorkspace& w);
SplitConfig split_config(int prec, bool correction);
// Inputs that arrive by column blocks (pevc_solve_host): arrive(i) orders
// what follows after column block i's copy and arrival work (pre-pass,
// slices of [S T], tips).
struct Arrivals {
  virtual ~Arrivals() = default;
  virtual cudaError_t arrive(int l, cudaStream_t s) = 0;
};
cudaError_t launch_split_A_block(const Problem& P, SplitWorkspace& w, int l, int ns, cudaStream_t s);
// The output column chunks of the tcgen05 update, built from the structure
// and uploaded on s (small copies: a streamed solve issues them before its
// blocks of S and T, which the copy engine would otherwise take first).
int split_prepare(SplitWorkspace& w, const Problem& P, const HostStructure& hs, cudaStream_t s);
// arr: null, or the arrivals of a streamed solve (no correction sweep), which
// then slice [S T] and run the tips block by block; the caller has run
// split_prepare.
int split_solve(SplitWorkspace& w, const Problem& P, const HostStructure& hs, const SplitConfig& cfg,
                cudaStream_t s, const SchedContext& sc, Profiler& prof, cudaEvent_t ev_dag, cudaEvent_t ev_corr,
                Arrivals* arr = nullptr);

// Back-transformation X = Z V as exact BF16 slice products (6 slices per
// operand, chunks of 256 along K summed in FP64); the workspace ws holds
// bt_split_bytes(n) bytes.
size_t bt_split_bytes(int n_max);
cudaError_t launch_bt_split(const double* Z, int ldz, int n, const double* V, int ldv, int m, double* X, int ldx,
                            unsigned char* ws, cudaStream_t s);

}  // namespace pevc

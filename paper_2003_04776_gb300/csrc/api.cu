// api.cu -- the C ABI (include/pevc.h): plans, argument checks, the host-side
// structure analysis (1x1 / 2x2 blocks, tile partition, output columns) and
// the stage loop that walks the task graph of Algorithm 1 bottom-up.
//
// Task graph (Section 3, Algorithm 1; Section 5.3): for every block column j
// a tip task on tile (j, j), then for i = j-1 .. 0 the updates of all tiles
// above from tile (i+1, j) and the solve of tile (i, j).  The graph is the
// disjoint union of one sub-graph per block column; here all block columns
// advance together, one block row per stage from the bottom up:
//   stage i:  solve tiles (i, j), j > i   ->   update tiles (k, j), k < i <= j
// so every [S_ki T_ki] tile row panel is read once per stage for all columns.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "autotune.cuh"
#include "common.cuh"
#include "cplx.cuh"
#include "dag.cuh"
#include "sched.cuh"
#include "split.cuh"

namespace pevc {
// Bounded-wait self-test (watchdog.cu).
cudaError_t launch_watchdog_probe(unsigned* status, int withhold, long long cycles, cudaStream_t s);
}  // namespace pevc

using namespace pevc;

struct pevc_plan_s {
  int dev = 0, nsm = 0;
  int n_max = 0, batch_max = 1, prec = PEVC_FP64, tb = 64;
  unsigned flags = 0;
  cudaStream_t stream = nullptr;
  int Mmax = 0;
  // device workspace
  double* Y = nullptr;
  int* ex = nullptr;
  double* nrm = nullptr;
  int* EA = nullptr;
  double* tcS = nullptr;
  double* tcT = nullptr;
  double* gmax = nullptr;
  double* ca = nullptr;
  double* cb = nullptr;
  double* cbeta = nullptr;
  signed char* blk = nullptr;
  int* toff = nullptr;
  int* cstart = nullptr;
  int* ccol = nullptr;
  signed char* kind = nullptr;
  unsigned* status = nullptr;
  double* subd = nullptr;
  int* dperm = nullptr;      // diagonal-kernel chunks (see Problem)
  int* dcpos = nullptr;
  int* dccnt = nullptr;
  int* dcfirst = nullptr;
  // pinned host staging
  double* h_subd = nullptr;
  int32_t* h_sel = nullptr;
  signed char* h_blk = nullptr;
  int* h_toff = nullptr;
  int* h_cstart = nullptr;
  int* h_ccol = nullptr;
  signed char* h_kind = nullptr;
  unsigned* h_status = nullptr;
  int* h_dperm = nullptr;
  int* h_dcpos = nullptr;
  int* h_dccnt = nullptr;
  int* h_dcfirst = nullptr;
  int dchunk_max = 0;
  cudaEvent_t ev[6] = {};
  double stats[8] = {};
  SplitWorkspace split;
  Profiler prof;
  double kprof[12] = {};
  cudaStream_t aux = nullptr;
  cudaEvent_t* sev = nullptr;   // 2 * Mmax scheduling events
  bool lookahead = true;
  // batched solves: child plans (own workspace and stream each) run pencils
  // concurrently
  int nchild = 0;
  pevc_plan_s* child[8] = {};
  cudaStream_t cstream[8] = {};
  cudaEvent_t bev = nullptr;     // the children wait for the plan's stream
  unsigned* h_bstatus = nullptr; // pinned [batch_max] status words
  // back-transformation: cuBLAS handle, the column count of the last solve
  // (whose column kinds are in kind), caller-given kinds
  void* blas = nullptr;
  int last_m = -1;
  signed char* bt_kind = nullptr;
  signed char* h_bt_kind = nullptr;
  unsigned char* bt_ws = nullptr;   // split back-transformation workspace (first call)
  size_t bt_ws_bytes = 0;
  // left eigenvectors: the flipped transposed pencil, its selection, its
  // solve's output (allocated by the first pevc_solve_left)
  double* lS = nullptr;
  double* lT = nullptr;
  double* lV = nullptr;
  int32_t* lsel = nullptr;
  int32_t* lsc = nullptr;
  // complex pencils (allocated by the first pevc_solve_cplx)
  CplxWork* cx = nullptr;
  // solves from host memory (allocated by the first pevc_solve_host): device
  // copies of S and T, the output and its scales (leading dimension n_max),
  // the copy stream with one event per column block, the pre-scale record per
  // column block (the maximum seen so far, the largest coefficient exponent)
  // and the bytes the last call copied each way
  double* hS = nullptr;
  double* hT = nullptr;
  double* hV = nullptr;
  int32_t* hsc = nullptr;
  cudaStream_t hstream = nullptr;
  cudaStream_t astream = nullptr;   // the blocks' arrival work (pre-pass, slices, tips)
  cudaEvent_t* hev = nullptr;       // [Mmax] block l copied
  cudaEvent_t* aev = nullptr;       // [Mmax] block l's arrival work done
  cudaEvent_t hstart = nullptr;
  cudaEvent_t hinit = nullptr;
  double* hspec = nullptr;
  double* h_hspec = nullptr;
  long long host_bytes[2] = {0, 0};
  // device-side task-graph scheduler (dag.cuh), the walk of FP64 plans:
  // the pencil record, the task list, the ready counters, the update
  // sub-chunks and the ticket / abort pair
  bool dag = false;
  DagPencil* d_pen = nullptr;
  DagPencil* h_pen = nullptr;
  int4* d_tasks = nullptr;
  int4* h_tasks = nullptr;
  long long task_cap = 0;
  int* d_cnt = nullptr;
  size_t cnt_cap = 0;
  int* d_sub = nullptr;
  int* h_sub = nullptr;
  int sub_cap = 0;
  int* d_ticket = nullptr;
  // batched solves of FP64 plans on the scheduler: every pencil's workspace,
  // structure, counters and record are slices of these pools (bdag)
  bool bdag = false;
  unsigned char* b_work = nullptr;      // augmented tiles, exponents, norms, eigenvalues
  size_t b_work_bytes = 0;
  unsigned char* b_strc = nullptr;      // structure arrays (device) ...
  unsigned char* h_b_strc = nullptr;    // ... and their pinned host copy
  size_t b_strc_bytes = 0;
  int* b_cnt = nullptr;                 // ready counters
  size_t b_cnt_ints = 0;
  double* b_subd = nullptr;             // subdiagonals [batch_max * n_max]
  double* h_b_subd = nullptr;
  int32_t* h_b_sel = nullptr;           // selections [batch_max * n_max]
  unsigned* b_status = nullptr;         // [batch_max]
  double* b_gmax = nullptr;             // [batch_max]
  DagPencil* b_pen = nullptr;           // [batch_max]
  DagPencil* h_b_pen = nullptr;
  int4* b_tasks = nullptr;
  int4* h_b_tasks = nullptr;
  long long b_task_cap = 0;
  // the candidates timed by PEVC_AUTOTUNE: {tile, prec, stage walk, ms}
  std::vector<std::array<double, 4>> tune_log;
};

namespace {

int cuda_fail(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return PEVC_ERR_NOMEM;
  return PEVC_ERR_CUDA;
}

#define CK(call)                                \
  do {                                          \
    cudaError_t _e = (call);                    \
    if (_e != cudaSuccess) return cuda_fail(_e); \
  } while (0)

int status_from_bits(unsigned bits) {
  if (bits & kStNonfinite) return PEVC_ERR_NONFINITE;
  if (bits & kStNotSchur) return PEVC_ERR_NOT_SCHUR;
  if (bits & kStIndefinite) return PEVC_ERR_INDEFINITE;
  if (bits & kStTimeout) return PEVC_ERR_TIMEOUT;
  return PEVC_SUCCESS;
}

// Default tile order (PEVC_AUTOTUNE measures instead).  FP64: small pencils
// want small tiles (enough tiles to fill the GPU, short diagonal solves),
// large ones the largest (fewer stages, larger updates).  Split precisions:
// always 128, the tcgen05 update's order; the split paths' componentwise
// error also grows as the tiles shrink (the diagonal tiles are solved in
// FP64, the rest goes through the slices: on the batched workload's worst
// vectors 2e-13 .. 3e-9 at order 128 against 1e-8 .. 8e-7 at 32 and 64).
int choose_tile(int n_max, int prec) {
  if (prec != PEVC_FP64) return 128;
  if (n_max <= 256) return 32;
  if (n_max <= 1024) return 64;
  return 128;
}

// Default walk of FP64 plans (PEVC_AUTOTUNE measures instead): the device-side
// scheduler for batches, where it runs every pencil's graph in one launch
// (1210 against 903 pencils/s on the batched workload); the stage walk for
// single pencils, where its 256-thread update kernel keeps the FP64 pipe
// busier than the scheduler's 128-thread update tasks (n = 4000: 56 against
// 67 ms; n = 20000: 5.26 against 5.81 s).
bool default_dag(int, int batch_max) { return batch_max > 1; }

template <typename Tp>
int dalloc(Tp** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(Tp));
  return e == cudaSuccess ? 0 : cuda_fail(e);
}

template <typename Tp>
int halloc(Tp** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMallocHost((void**)p, count * sizeof(Tp));
  return e == cudaSuccess ? 0 : cuda_fail(e);
}

void free_plan(pevc_plan_t p) {
  if (!p) return;
  for (int c = 0; c < 8; ++c) {
    if (p->child[c]) free_plan(p->child[c]);
    if (p->cstream[c]) cudaStreamDestroy(p->cstream[c]);
  }
  if (p->bev) cudaEventDestroy(p->bev);
  if (p->h_bstatus) cudaFreeHost(p->h_bstatus);
  void* dev[] = {p->Y, p->ex, p->nrm, p->EA, p->tcS, p->tcT, p->gmax, p->ca, p->cb, p->cbeta,
                 p->blk, p->toff, p->cstart, p->ccol, p->kind, p->status, p->subd,
                 p->dperm, p->dcpos, p->dccnt, p->dcfirst};
  for (void* d : dev)
    if (d) cudaFree(d);
  void* host[] = {p->h_subd, p->h_sel, p->h_blk, p->h_toff, p->h_cstart, p->h_ccol, p->h_kind, p->h_status,
                  p->h_dperm, p->h_dcpos, p->h_dccnt, p->h_dcfirst};
  for (void* h : host)
    if (h) cudaFreeHost(h);
  for (auto& e : p->ev)
    if (e) cudaEventDestroy(e);
  if (p->prof.ev) {
    for (int q = 0; q < 2 * p->prof.cap; ++q) cudaEventDestroy(p->prof.ev[q]);
    delete[] p->prof.ev;
    delete[] p->prof.kind;
    delete[] p->prof.flops;
  }
  split_free(p->split);
  if (p->sev) {
    for (int q = 0; q < 2 * p->Mmax; ++q)
      if (p->sev[q]) cudaEventDestroy(p->sev[q]);
    delete[] p->sev;
  }
  if (p->aux) cudaStreamDestroy(p->aux);
  bt_handle_destroy(p->blas);
  void* ldev[] = {p->lS, p->lT, p->lV, p->lsel, p->lsc};
  for (void* d : ldev)
    if (d) cudaFree(d);
  cplx_free(p->cx);
  void* bd[] = {p->b_work, p->b_strc, p->b_cnt, p->b_subd, p->b_status, p->b_gmax, p->b_pen, p->b_tasks};
  for (void* d : bd)
    if (d) cudaFree(d);
  void* bh[] = {p->h_b_strc, p->h_b_subd, p->h_b_sel, p->h_b_pen, p->h_b_tasks};
  for (void* h : bh)
    if (h) cudaFreeHost(h);
  void* dagd[] = {p->d_pen, p->d_tasks, p->d_cnt, p->d_sub, p->d_ticket};
  for (void* d : dagd)
    if (d) cudaFree(d);
  void* dagh[] = {p->h_pen, p->h_tasks, p->h_sub};
  for (void* h : dagh)
    if (h) cudaFreeHost(h);
  void* hdev[] = {p->hS, p->hT, p->hV, p->hsc, p->hspec};
  for (void* d : hdev)
    if (d) cudaFree(d);
  if (p->h_hspec) cudaFreeHost(p->h_hspec);
  for (cudaEvent_t* evs : {p->hev, p->aev}) {
    if (!evs) continue;
    for (int q = 0; q < p->Mmax; ++q)
      if (evs[q]) cudaEventDestroy(evs[q]);
    delete[] evs;
  }
  if (p->hstart) cudaEventDestroy(p->hstart);
  if (p->hinit) cudaEventDestroy(p->hinit);
  if (p->hstream) cudaStreamDestroy(p->hstream);
  if (p->astream) cudaStreamDestroy(p->astream);
  if (p->bt_kind) cudaFree(p->bt_kind);
  if (p->bt_ws) cudaFree(p->bt_ws);
  if (p->h_bt_kind) cudaFreeHost(p->h_bt_kind);
  delete p;
}

struct Structure {
  int M = 0, m = 0, nchunks = 0;
};

// Host-side structure analysis: block pattern from the subdiagonal, tile
// partition (Section 5.1: tiles of order tb, moved down by one row where a
// boundary would split a 2x2 block), and the output columns grouped by the
// row tile of their block (the column partition conforms to the row one).
int analyse(pevc_plan_t p, int n, bool has_sel, Structure& st) {
  for (int i = 0; i + 1 < n; ++i)
    if (!std::isfinite(p->h_subd[i])) return PEVC_ERR_NONFINITE;
  for (int i = 0; i < n; ++i) p->h_blk[i] = 0;
  for (int i = 0; i + 1 < n; ++i) {
    if (p->h_subd[i] != 0.0) {
      if (p->h_blk[i] != 0) return PEVC_ERR_NOT_SCHUR;
      p->h_blk[i] = 1;
      p->h_blk[i + 1] = 2;
    }
  }
  int M = 0;
  p->h_toff[0] = 0;
  int off = 0;
  while (off < n) {
    int nxt = std::min(off + p->tb, n);
    if (nxt < n && p->h_blk[nxt] == 2) --nxt;
    if (M + 1 >= p->Mmax) return PEVC_ERR_CUDA;   // cannot happen: Mmax bounds ceil(n/(tb-1))
    p->h_toff[++M] = nxt;
    off = nxt;
  }
  int m = 0, tile = 0;
  for (int j = 0; j <= M; ++j) p->h_cstart[j] = 0;
  for (int c = 0; c < n; ++c) {
    if (p->h_blk[c] == 2) continue;
    const int sz = (p->h_blk[c] == 1) ? 2 : 1;
    while (c >= p->h_toff[tile + 1]) {
      ++tile;
      p->h_cstart[tile] = m;
    }
    bool sel = !has_sel || p->h_sel[c] != 0 || (sz == 2 && p->h_sel[c + 1] != 0);
    if (!sel) continue;
    for (int u = 0; u < sz; ++u) {
      p->h_ccol[m] = c + u;
      p->h_kind[m] = (signed char)(sz == 1 ? 0 : 1 + u);
      ++m;
    }
  }
  while (tile < M) {
    ++tile;
    p->h_cstart[tile] = m;
  }
  st.M = M;
  st.m = m;
  // diagonal-kernel chunks: per column tile, real columns first, then the
  // complex pairs; chunks of at most kDiagChunk columns, never mixing the
  // two kinds
  const int kCB = kDiagChunk;
  int nch = 0, maxc = 0;
  for (int j = 0; j < M; ++j) {
    p->h_dcfirst[j] = nch;
    const int cs = p->h_cstart[j], ce = p->h_cstart[j + 1];
    int pos = cs;
    for (int q = cs; q < ce; ++q)
      if (p->h_kind[q] == 0) p->h_dperm[pos++] = q - cs;
    const int nreal = pos - cs;
    for (int q = cs; q < ce; ++q)
      if (p->h_kind[q] != 0) p->h_dperm[pos++] = q - cs;
    for (int s0 = 0; s0 < nreal; s0 += kCB) {
      p->h_dcpos[nch] = cs + s0;
      p->h_dccnt[nch] = std::min(kCB, nreal - s0);
      ++nch;
    }
    for (int s0 = nreal; s0 < ce - cs; s0 += kCB) {   // kCB is even: pairs stay whole
      p->h_dcpos[nch] = cs + s0;
      p->h_dccnt[nch] = std::min(kCB, ce - cs - s0);
      ++nch;
    }
    maxc = std::max(maxc, nch - p->h_dcfirst[j]);
  }
  p->h_dcfirst[M] = nch;
  p->dchunk_max = maxc;
  st.nchunks = nch;
  return 0;
}

Problem make_problem(pevc_plan_t p, const double* S, int lds, const double* T, int ldt, int n,
                     const Structure& st) {
  Problem P;
  P.S = S;
  P.T = T;
  P.lds = lds;
  P.ldt = ldt;
  P.n = n;
  P.blk = p->blk;
  P.toff = p->toff;
  P.cstart = p->cstart;
  P.ccol = p->ccol;
  P.kind = p->kind;
  P.M = st.M;
  P.m = st.m;
  P.tb = p->tb;
  P.ca = p->ca;
  P.cb = p->cb;
  P.cbeta = p->cbeta;
  P.EA = p->EA;
  P.tcS = p->tcS;
  P.tcT = p->tcT;
  P.gmax = p->gmax;
  P.Y = p->Y;
  P.ex = p->ex;
  P.nrm = p->nrm;
  P.status = p->status;
  P.dperm = p->dperm;
  P.dchunk_pos = p->dcpos;
  P.dchunk_cnt = p->dccnt;
  P.dchunk_first = p->dcfirst;
  P.dchunk_max = p->dchunk_max;
  return P;
}

int read_status(pevc_plan_t p, unsigned* bits) {
  CK(cudaMemcpyAsync(p->h_status, p->status, sizeof(unsigned), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  *bits = *p->h_status;
  return 0;
}

// Phase 1 of a solve: the subdiagonal (block structure) and the selection to
// the host, stream-ordered and asynchronous.
int structure_begin(pevc_plan_t p, const double* S, int lds, int n, const int32_t* sel) {
  cudaStream_t s = p->stream;
  p->prof.begin(s);
  CK(launch_gather_subdiag(S, lds, n, p->subd, s));
  p->prof.end(s, 3, 0.0);
  if (n > 1) CK(cudaMemcpyAsync(p->h_subd, p->subd, (size_t)(n - 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (sel) CK(cudaMemcpyAsync(p->h_sel, sel, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  return 0;
}

// Phase 2: wait for phase 1 (and everything before it on the plan's stream)
// and analyse the structure on the host.
int structure_end(pevc_plan_t p, int n, bool has_sel, Structure& st) {
  CK(cudaStreamSynchronize(p->stream));
  return analyse(p, n, has_sel, st);
}

// Bound of every dependence wait of the scheduler, in SM clock cycles (about
// 5 s at 2 GHz: far above any wait of a walk that progresses).
constexpr long long kDagWaitCycles = 10000000000LL;

// The task graph of one pencil on the device (dag.cuh): update sub-chunks and
// the task list in walk order, built here from the host structure; ready
// counters zeroed; one persistent launch.
int dag_enqueue(pevc_plan_t p, const Problem& P, const Structure& st, cudaStream_t s) {
  const int M = st.M;
  int* h_first = p->h_sub;
  int* h_c0 = h_first + (p->Mmax + 1);
  int* h_nc = h_c0 + p->sub_cap;
  int nsub_max = 0;
  const int ns = dag_subchunks(M, p->h_cstart, p->h_kind, h_first, h_c0, h_nc, p->sub_cap, &nsub_max);
  if (ns < 0) return PEVC_ERR_CUDA;
  const int cap = (int)std::min<long long>(p->task_cap, INT32_MAX);
  int cnt = dag_stage_tasks(0, M, M, p->h_dcfirst, h_first, p->h_tasks, 0, cap);
  double flops = 0.0;
  for (int i = M - 1; i >= 1 && cnt >= 0; --i) {
    cnt = dag_stage_tasks(0, M, i, p->h_dcfirst, h_first, p->h_tasks, cnt, cap);
    flops += 2.0 * p->h_toff[i] * (double)(P.m - p->h_cstart[i]) * 2.0 * (p->h_toff[i + 1] - p->h_toff[i]);
  }
  if (cnt < 0) return PEVC_ERR_CUDA;
  const size_t tiles = (size_t)M * (M + 1) / 2;
  nsub_max = std::max(nsub_max, 1);
  if (tiles * (2 + (size_t)nsub_max) > p->cnt_cap) return PEVC_ERR_CUDA;
  DagPencil& hp = *p->h_pen;
  hp.P = P;
  hp.dcnt = p->d_cnt;
  hp.utile = p->d_cnt + tiles;
  hp.usub = p->d_cnt + 2 * tiles;
  hp.sub_first = p->d_sub;
  hp.sub_c0 = p->d_sub + (p->Mmax + 1);
  hp.sub_nc = p->d_sub + (p->Mmax + 1) + p->sub_cap;
  hp.nsub_max = nsub_max;
  CK(cudaMemcpyAsync(p->d_sub, h_first, (size_t)(M + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  if (ns > 0) {
    CK(cudaMemcpyAsync((void*)hp.sub_c0, h_c0, (size_t)ns * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync((void*)hp.sub_nc, h_nc, (size_t)ns * sizeof(int), cudaMemcpyHostToDevice, s));
  }
  CK(cudaMemcpyAsync(p->d_tasks, p->h_tasks, (size_t)cnt * sizeof(int4), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(p->d_pen, p->h_pen, sizeof(DagPencil), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(p->d_cnt, 0, tiles * (2 + (size_t)nsub_max) * sizeof(int), s));
  CK(cudaMemsetAsync(p->d_ticket, 0, 2 * sizeof(int), s));
  p->prof.begin(s);
  CK(launch_dag(p->d_pen, p->d_tasks, cnt, p->d_ticket, p->d_ticket + 1, kDagWaitCycles, dag_grid(p->nsm), s));
  p->prof.end(s, 0, flops);
  return 0;
}

// ---- batched solves on the scheduler: per-pencil slices of the pools ----

// Slice sizes for a pencil of order n, from bounds that hold whatever its
// block structure (M <= the tile-count bound of the order; m <= n): bytes of
// workspace, bytes of structure, ready counters.
struct SliceSize {
  size_t work = 0, strc = 0, cnt = 0;
};

size_t r256(size_t x) { return (x + 255) / 256 * 256; }
int slice_mmax(int n, int tb) { return (std::max(n, 1) + tb - 2) / (tb - 1) + 1; }

SliceSize slice_size(int n, int tb) {
  const size_t nn = (size_t)std::max(n, 1), Mb = (size_t)slice_mmax(n, tb), tiles = Mb * (Mb + 1) / 2;
  const size_t nsb = (size_t)dag_nsub_bound(tb);
  SliceSize z;
  z.work = r256(tiles * tb * tb * sizeof(double)) + r256(Mb * nn * sizeof(int)) + r256(Mb * nn * sizeof(double)) +
           r256(Mb * Mb * sizeof(int)) + 5 * r256(nn * sizeof(double));
  z.strc = 2 * r256(nn) + 4 * r256((Mb + 1) * sizeof(int)) + 2 * r256(nn * sizeof(int)) +
           2 * r256((nn + Mb) * sizeof(int)) + 2 * r256(Mb * nsb * sizeof(int));
  z.cnt = tiles * (2 + nsb);
  return z;
}

// One pencil of a batch: a plan view whose workspace pointers are its slices
// (device work, device structure, host structure mirror, counters), so that
// analyse() and make_problem() serve it unchanged.
struct BatchPencil {
  pevc_plan_s v;           // a view: every pointer is borrowed
  int* sub_first = nullptr;  // host mirror of the sub-chunks ...
  int* sub_c0 = nullptr;
  int* sub_nc = nullptr;
  int* d_sub_first = nullptr;  // ... and the device slices
  int* d_sub_c0 = nullptr;
  int* d_sub_nc = nullptr;
  int* cnt = nullptr;
  int nsub_max = 1;
  Structure st;
  size_t strc_off = 0;
};

void bind_slice(pevc_plan_t p, int b, int n, size_t work_off, size_t strc_off, size_t cnt_off, BatchPencil& bp) {
  pevc_plan_s& v = bp.v;
  const size_t nn = (size_t)std::max(n, 1);
  const int Mb = slice_mmax(n, p->tb);
  const size_t tiles = (size_t)Mb * (Mb + 1) / 2, nsb = (size_t)dag_nsub_bound(p->tb);
  v.n_max = n;
  v.prec = PEVC_FP64;
  v.tb = p->tb;
  v.flags = p->flags;
  v.stream = p->stream;
  v.Mmax = Mb;
  v.nsm = p->nsm;
  unsigned char* w = p->b_work + work_off;
  auto take = [&](size_t bytes) {
    unsigned char* q = w;
    w += r256(bytes);
    return q;
  };
  v.Y = (double*)take(tiles * p->tb * p->tb * sizeof(double));
  v.ex = (int*)take((size_t)Mb * nn * sizeof(int));
  v.nrm = (double*)take((size_t)Mb * nn * sizeof(double));
  v.EA = (int*)take((size_t)Mb * Mb * sizeof(int));
  v.tcS = (double*)take(nn * sizeof(double));
  v.tcT = (double*)take(nn * sizeof(double));
  v.ca = (double*)take(nn * sizeof(double));
  v.cb = (double*)take(nn * sizeof(double));
  v.cbeta = (double*)take(nn * sizeof(double));
  v.gmax = p->b_gmax + b;
  v.status = p->b_status + b;
  // structure: the same offsets in the device pool and its host mirror
  size_t o = strc_off;
  auto both = [&](size_t bytes, void** dev, void** host) {
    *dev = p->b_strc + o;
    *host = p->h_b_strc + o;
    o += r256(bytes);
  };
  both(nn, (void**)&v.blk, (void**)&v.h_blk);
  both(nn, (void**)&v.kind, (void**)&v.h_kind);
  both((Mb + 1) * sizeof(int), (void**)&v.toff, (void**)&v.h_toff);
  both((Mb + 1) * sizeof(int), (void**)&v.cstart, (void**)&v.h_cstart);
  both((Mb + 1) * sizeof(int), (void**)&v.dcfirst, (void**)&v.h_dcfirst);
  both((Mb + 1) * sizeof(int), (void**)&bp.d_sub_first, (void**)&bp.sub_first);
  both(nn * sizeof(int), (void**)&v.ccol, (void**)&v.h_ccol);
  both(nn * sizeof(int), (void**)&v.dperm, (void**)&v.h_dperm);
  both((nn + Mb) * sizeof(int), (void**)&v.dcpos, (void**)&v.h_dcpos);
  both((nn + Mb) * sizeof(int), (void**)&v.dccnt, (void**)&v.h_dccnt);
  both((size_t)Mb * nsb * sizeof(int), (void**)&bp.d_sub_c0, (void**)&bp.sub_c0);
  both((size_t)Mb * nsb * sizeof(int), (void**)&bp.d_sub_nc, (void**)&bp.sub_nc);
  v.h_subd = p->h_b_subd + (size_t)b * p->n_max;
  v.subd = p->b_subd + (size_t)b * p->n_max;
  v.h_sel = p->h_b_sel + (size_t)b * p->n_max;
  bp.cnt = p->b_cnt + cnt_off;
  bp.strc_off = strc_off;
  (void)tiles;
}

// Phase 3: everything else, stream-ordered.  With check_prepass the call reads
// the status after the pre-pass and returns early for a bad pencil; without it
// the whole graph is enqueued and the status is read once at the end (the
// kernels run to completion on any input: their loops depend only on the
// structure).
int solve_enqueue(pevc_plan_t p, const double* S, int lds, const double* T, int ldt, int n, double* V, int ldv,
                  int32_t* scale, const Structure& st, bool check_prepass) {
  cudaStream_t s = p->stream;
  // structure to the device, pre-processing tasks
  CK(cudaMemcpyAsync(p->blk, p->h_blk, (size_t)n, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(p->toff, p->h_toff, (size_t)(st.M + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(p->cstart, p->h_cstart, (size_t)(st.M + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  if (st.m > 0) {
    CK(cudaMemcpyAsync(p->ccol, p->h_ccol, (size_t)st.m * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p->kind, p->h_kind, (size_t)st.m, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p->dperm, p->h_dperm, (size_t)st.m * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p->dcpos, p->h_dcpos, (size_t)st.nchunks * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p->dccnt, p->h_dccnt, (size_t)st.nchunks * sizeof(int), cudaMemcpyHostToDevice, s));
  }
  CK(cudaMemcpyAsync(p->dcfirst, p->h_dcfirst, (size_t)(st.M + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(p->status, 0, sizeof(unsigned), s));
  CK(cudaMemsetAsync(p->gmax, 0, sizeof(double), s));
  Problem P = make_problem(p, S, lds, T, ldt, n, st);
  p->prof.begin(s);
  CK(launch_prepass(P, s));
  p->prof.end(s, 3, 0.0);
  ++p->prof.launches;   // the prepass is two kernels
  if (check_prepass) {
    unsigned bits = 0;
    int rc = read_status(p, &bits);
    if (rc) return rc;
    if (bits) return status_from_bits(bits);
  }
  CK(cudaEventRecord(p->ev[1], s));
  if (st.m == 0) {
    CK(cudaEventRecord(p->ev[2], s));
    CK(cudaEventRecord(p->ev[3], s));
    CK(cudaEventRecord(p->ev[4], s));
    return 0;
  }
  p->prof.begin(s);
  CK(launch_init_state(P, s));
  p->prof.end(s, 3, 0.0);
  // the task graph, bottom-up by block row
  SchedContext sc{p->aux, p->sev, p->lookahead};
  if (p->prec == PEVC_FP64) {
    struct F64Ops : StageOps {
      const Problem& P;
      pevc_plan_t p;
      F64Ops(const Problem& P_, pevc_plan_t p_) : P(P_), p(p_) {}
      cudaError_t tips(cudaStream_t st) override {
        p->prof.begin(st);
        cudaError_t e = launch_diag(P, 0, kDiagTip, st);
        p->prof.end(st, 1, 0.0);
        return e;
      }
      cudaError_t diag(int i, cudaStream_t st) override {
        p->prof.begin(st);
        cudaError_t e = launch_diag(P, i, kDiagSolve, st);
        p->prof.end(st, 1, 0.0);
        return e;
      }
      cudaError_t prep(int, cudaStream_t) override { return cudaSuccess; }
      cudaError_t update(int i, int k_lo, int k_hi, cudaStream_t st) override {
        const double rows = p->h_toff[k_hi] - p->h_toff[k_lo], cols = P.m - p->h_cstart[i];
        const double K = 2.0 * (p->h_toff[i + 1] - p->h_toff[i]);
        p->prof.begin(st);
        cudaError_t e = launch_update_f64(P, i, k_lo, k_hi, st);
        p->prof.end(st, 0, 2.0 * rows * cols * K);
        return e;
      }
    } ops(P, p);
    if (p->dag) {
      int rc = dag_enqueue(p, P, st, s);
      if (rc) return rc;
    } else {
      CK(walk_dag(st.M, ops, s, sc.aux, sc.ev, sc.lookahead));
    }
    CK(cudaEventRecord(p->ev[2], s));
    CK(cudaEventRecord(p->ev[3], s));
  } else {
    HostStructure hs{p->h_toff, p->h_cstart};
    SplitConfig cfg = split_config(p->prec, (p->flags & PEVC_NO_CORRECTION) == 0);
    int rc = split_solve(p->split, P, hs, cfg, s, sc, p->prof, p->ev[2], p->ev[3]);
    if (rc) return rc;
  }
  // post-processing: consistent scaling and normalisation
  p->prof.begin(s);
  CK(launch_post(P, V, ldv, scale, (p->flags & PEVC_NO_NORMALISE) == 0, s));
  p->prof.end(s, 3, 0.0);
  CK(cudaEventRecord(p->ev[4], s));
  return 0;
}

int solve_one(pevc_plan_t p, const double* S, int lds, const double* T, int ldt, int n,
              const int32_t* sel, double* V, int ldv, int32_t* scale, int* m_out) {
  cudaStream_t s = p->stream;
  *m_out = 0;
  for (double& x : p->stats) x = 0.0;
  if (n == 0) return 0;
  p->prof.reset();
  CK(cudaEventRecord(p->ev[0], s));
  // 1. block structure and selection to the host
  int rc = structure_begin(p, S, lds, n, sel);
  if (rc) return rc;
  Structure st;
  if ((rc = structure_end(p, n, sel != nullptr, st))) return rc;
  *m_out = st.m;
  p->last_m = st.m;
  // 2. pre-processing, the task graph, post-processing
  if ((rc = solve_enqueue(p, S, lds, T, ldt, n, V, ldv, scale, st, true))) return rc;
  unsigned bits = 0;
  if ((rc = read_status(p, &bits))) return rc;
  float ms[4] = {0, 0, 0, 0};
  cudaEventElapsedTime(&ms[0], p->ev[0], p->ev[4]);
  cudaEventElapsedTime(&ms[1], p->ev[0], p->ev[1]);
  cudaEventElapsedTime(&ms[2], p->ev[1], p->ev[2]);
  cudaEventElapsedTime(&ms[3], p->ev[2], p->ev[3]);
  p->stats[0] = ms[0];
  p->stats[1] = ms[1];
  p->stats[2] = ms[2];
  p->stats[3] = ms[3];
  float post = 0.0f;
  cudaEventElapsedTime(&post, p->ev[3], p->ev[4]);
  p->stats[4] = post;
  p->stats[5] = st.M;
  p->stats[6] = p->prof.launches;
  p->stats[7] = p->prec == PEVC_FP64 ? (p->dag ? 1.0 : 0.0) : (double)p->split.last_sweeps;
  for (double& x : p->kprof) x = 0.0;
  for (int q = 0; q < p->prof.used; ++q) {
    float t = 0.0f;
    cudaEventElapsedTime(&t, p->prof.ev[2 * q], p->prof.ev[2 * q + 1]);
    const int k = p->prof.kind[q];
    p->kprof[3 * k] += t;
    p->kprof[3 * k + 1] += 1.0;
    p->kprof[3 * k + 2] += p->prof.flops[q];
  }
  return status_from_bits(bits);
}

// Argument checks of one pencil (pevc_solve's codes).
int check_args(int n_max, const double* S, int lds, const double* T, int ldt, int n, const double* V, int ldv,
               const int32_t* scale) {
  if (n < 0 || n > n_max) return -6;
  if (n > 0 && !S) return -2;
  if (lds < std::max(n, 1)) return -3;
  if (n > 0 && !T) return -4;
  if (ldt < std::max(n, 1)) return -5;
  if (n > 0 && !V) return -8;
  if (ldv < std::max(n, 1)) return -9;
  if (n > 0 && !scale) return -10;
  return 0;
}

// ---- solves from host memory, with the inputs streamed in by column blocks
//
// S and T are copied to the plan's device copies column block by column
// block from the right (the order in which the bottom-up walk needs them),
// each block's rows 0 .. (end of the block) only -- the tiles on and above the
// diagonal, everything the method reads -- on a copy stream, one event per
// block.  Stage i of the walk waits for block i, whose pre-pass (tile norms,
// eigenvalues), slices and tips run on its arrival, so the copies overlap the
// solve.  The eigenvalues' pre-scale (every (alpha, beta) scaled by a power of
// two when max(|beta|, |a| + |b|) max|S, T| would exceed 2^1000) is taken from
// the maximum of the blocks seen so far; once all have arrived the pre-scale
// of every block is checked against the final maximum, and the rare solve
// whose pre-scale would change is run again on the device copies.

int host_alloc(pevc_plan_t p) {
  if (p->hS) return 0;
  const size_t nn = (size_t)p->n_max * p->n_max;
  int rc = dalloc(&p->hS, nn);
  rc = rc ? rc : dalloc(&p->hT, nn);
  rc = rc ? rc : dalloc(&p->hV, nn);
  rc = rc ? rc : dalloc(&p->hsc, (size_t)p->n_max);
  rc = rc ? rc : dalloc(&p->hspec, 2 * (size_t)p->Mmax);
  rc = rc ? rc : halloc(&p->h_hspec, 2 * (size_t)p->Mmax);
  if (rc) return rc;
  CK(cudaStreamCreateWithFlags(&p->hstream, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&p->astream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&p->hstart, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&p->hinit, cudaEventDisableTiming));
  p->hev = new (std::nothrow) cudaEvent_t[p->Mmax]();
  p->aev = new (std::nothrow) cudaEvent_t[p->Mmax]();
  if (!p->hev || !p->aev) return PEVC_ERR_NOMEM;
  for (int q = 0; q < p->Mmax; ++q) {
    CK(cudaEventCreateWithFlags(&p->hev[q], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&p->aev[q], cudaEventDisableTiming));
  }
  return 0;
}

// The arrival work of every column block, enqueued up front on the arrival
// stream (after the zeroed state, hinit): per block, from the right, wait for
// its copy, then its pre-pass (tile norms, eigenvalues), its slices (split
// plans) and the tips of its diagonal tile; aev[l] marks it done.  The walk's
// stage l waits for aev[l] alone, so the tips of the blocks to come run beside
// the stages before them.  (Tiles and columns these write are not touched by
// those stages: the tips write tile (l, l) and its columns' state, the stages
// before l update tiles (k, j) with j > l.)
int enqueue_arrivals(pevc_plan_t p, const Problem& P, int ns) {
  cudaStream_t a = p->astream;
  CK(cudaStreamWaitEvent(a, p->hinit, 0));
  for (int l = P.M - 1; l >= 0; --l) {
    CK(cudaStreamWaitEvent(a, p->hev[l], 0));
    p->prof.begin(a);
    CK(launch_prepass_block(P, l, p->h_toff[l], p->h_toff[l + 1], p->hspec + 2 * l, a));
    p->prof.end(a, 3, 0.0);
    ++p->prof.launches;   // two kernels
    if (ns) {
      p->prof.begin(a);
      CK(launch_split_A_block(P, p->split, l, ns, a));
      p->prof.end(a, 3, 0.0);
    }
    p->prof.begin(a);
    CK(launch_diag_tile(P, l, kDiagTip, a));
    p->prof.end(a, 1, 0.0);
    CK(cudaEventRecord(p->aev[l], a));
  }
  return 0;
}

struct HostArrivals : Arrivals {
  pevc_plan_t p;
  explicit HostArrivals(pevc_plan_t p_) : p(p_) {}
  cudaError_t arrive(int l, cudaStream_t s) override { return cudaStreamWaitEvent(s, p->aev[l], 0); }
};

int solve_host(pevc_plan_t p, const double* S, int lds, const double* T, int ldt, int n, const int32_t* sel,
               double* V, int ldv, int32_t* scale, int* m_out) {
  cudaStream_t s = p->stream;
  *m_out = 0;
  for (double& x : p->stats) x = 0.0;
  p->host_bytes[0] = p->host_bytes[1] = 0;
  if (n == 0) return 0;
  int rc = host_alloc(p);
  if (rc) return rc;
  p->prof.reset();
  CK(cudaEventRecord(p->ev[0], s));
  // 1. block structure and selection, read on the host
  for (int c = 0; c + 1 < n; ++c) p->h_subd[c] = S[(size_t)c * lds + c + 1];
  if (sel) std::memcpy(p->h_sel, sel, (size_t)n * sizeof(int32_t));
  Structure st;
  if ((rc = analyse(p, n, sel != nullptr, st))) return rc;
  *m_out = st.m;
  p->last_m = st.m;
  const int M = st.M, ldd = p->n_max;
  // the rows of V below each column tile's last row are zero: host threads
  // write them while the GPU works, and only the rows above come back
  std::vector<std::thread> zero;
  {
    const int nt = (int)std::min<unsigned>(8u, std::max(1u, std::thread::hardware_concurrency() / 2));
    const int m = st.m;
    for (int t = 0; t < nt && m > 0; ++t)
      zero.emplace_back([p, V, ldv, n, M, m, nt, t] {
        int j = 0;
        for (int q = (int)((long long)m * t / nt); q < (int)((long long)m * (t + 1) / nt); ++q) {
          while (j + 1 < M && p->h_cstart[j + 1] <= q) ++j;
          const int r0 = p->h_toff[j + 1];
          if (r0 < n) std::memset(V + (size_t)q * ldv + r0, 0, (size_t)(n - r0) * sizeof(double));
        }
      });
  }
  struct Joiner {
    std::vector<std::thread>& t;
    ~Joiner() {
      for (auto& x : t)
        if (x.joinable()) x.join();
    }
  } joiner{zero};
  // split plans with the correction sweep (which reads every block at once) or
  // FP8 slices take the whole copy first
  const SplitConfig scfg = split_config(p->prec, (p->flags & PEVC_NO_CORRECTION) == 0);
  const bool streamed = p->prec == PEVC_FP64 || !(scfg.correction || scfg.fp8);
  if (streamed) {
    // the structure (and every other small host-to-device copy of the solve)
    // first: the copy engine takes the copies in the order they are issued,
    // so these must not queue behind the blocks of S and T
    cudaStream_t ss = s;
    // structure to the device
    CK(cudaMemcpyAsync(p->blk, p->h_blk, (size_t)n, cudaMemcpyHostToDevice, ss));
    CK(cudaMemcpyAsync(p->toff, p->h_toff, (size_t)(M + 1) * sizeof(int), cudaMemcpyHostToDevice, ss));
    CK(cudaMemcpyAsync(p->cstart, p->h_cstart, (size_t)(M + 1) * sizeof(int), cudaMemcpyHostToDevice, ss));
    if (st.m > 0) {
      CK(cudaMemcpyAsync(p->ccol, p->h_ccol, (size_t)st.m * sizeof(int), cudaMemcpyHostToDevice, ss));
      CK(cudaMemcpyAsync(p->kind, p->h_kind, (size_t)st.m, cudaMemcpyHostToDevice, ss));
      CK(cudaMemcpyAsync(p->dperm, p->h_dperm, (size_t)st.m * sizeof(int), cudaMemcpyHostToDevice, ss));
      CK(cudaMemcpyAsync(p->dcpos, p->h_dcpos, (size_t)st.nchunks * sizeof(int), cudaMemcpyHostToDevice, ss));
      CK(cudaMemcpyAsync(p->dccnt, p->h_dccnt, (size_t)st.nchunks * sizeof(int), cudaMemcpyHostToDevice, ss));
    }
    CK(cudaMemcpyAsync(p->dcfirst, p->h_dcfirst, (size_t)(M + 1) * sizeof(int), cudaMemcpyHostToDevice, ss));
    CK(cudaMemsetAsync(p->status, 0, sizeof(unsigned), ss));
    CK(cudaMemsetAsync(p->gmax, 0, sizeof(double), ss));
    for (int l = 0; l < M; ++l) {
      p->h_hspec[2 * l] = 0.0;
      const int lowest = INT32_MIN;
      std::memcpy(&p->h_hspec[2 * l + 1], &lowest, sizeof(int));
    }
    CK(cudaMemcpyAsync(p->hspec, p->h_hspec, 2 * (size_t)M * sizeof(double), cudaMemcpyHostToDevice, ss));
    if (p->prec != PEVC_FP64 && st.m > 0) {
      HostStructure hs{p->h_toff, p->h_cstart};
      if ((rc = split_prepare(p->split, make_problem(p, p->hS, ldd, p->hT, ldd, n, st), hs, ss))) return rc;
    }
    // the zeroed augmented state, before the copies are issued
    CK(cudaEventRecord(p->ev[1], ss));
    if (st.m > 0) {
      p->prof.begin(ss);
      CK(launch_init_state(make_problem(p, p->hS, ldd, p->hT, ldd, n, st), ss, 1));
      p->prof.end(ss, 3, 0.0);
      CK(cudaEventRecord(p->hinit, ss));
    }
  }
  // 2. the copies, column blocks from the right, after the plan's earlier
  //    work (which may still read the device copies)
  CK(cudaEventRecord(p->hstart, s));
  CK(cudaStreamWaitEvent(p->hstream, p->hstart, 0));
  for (int l = M - 1; l >= 0; --l) {
    const int c0 = p->h_toff[l], c1 = p->h_toff[l + 1];
    const size_t w = (size_t)c1 * sizeof(double);
    CK(cudaMemcpy2DAsync(p->hS + (size_t)c0 * ldd, (size_t)ldd * sizeof(double), S + (size_t)c0 * lds,
                         (size_t)lds * sizeof(double), w, (size_t)(c1 - c0), cudaMemcpyHostToDevice, p->hstream));
    CK(cudaMemcpy2DAsync(p->hT + (size_t)c0 * ldd, (size_t)ldd * sizeof(double), T + (size_t)c0 * ldt,
                         (size_t)ldt * sizeof(double), w, (size_t)(c1 - c0), cudaMemcpyHostToDevice, p->hstream));
    CK(cudaEventRecord(p->hev[l], p->hstream));
    p->host_bytes[0] += 2 * (long long)w * (c1 - c0);
  }
  // 3. the solve on the device copies, each stage after its column block
  if (!streamed) {
    // the correction sweep reads every block at the start: the whole copy first
    for (int l = 0; l < M; ++l) CK(cudaStreamWaitEvent(s, p->hev[l], 0));
    if ((rc = solve_enqueue(p, p->hS, ldd, p->hT, ldd, n, p->hV, ldd, p->hsc, st, false))) return rc;
  } else {
    cudaStream_t ss = s;
    Problem P = make_problem(p, p->hS, ldd, p->hT, ldd, n, st);
    if (st.m > 0) {
      int ns = 0;
      if (p->prec != PEVC_FP64) ns = split_config(p->prec, false).ns1 == 5 ? 5 : 3;
      if ((rc = enqueue_arrivals(p, P, ns))) return rc;
      HostArrivals arr(p);
      SchedContext sc{p->aux, p->sev, p->lookahead};
      if (p->prec == PEVC_FP64) {
        struct F64Streamed : StageOps {
          const Problem& P;
          pevc_plan_t p;
          Arrivals& arr;
          F64Streamed(const Problem& P_, pevc_plan_t p_, Arrivals& a_) : P(P_), p(p_), arr(a_) {}
          cudaError_t arrive(int l, cudaStream_t st) override { return arr.arrive(l, st); }
          cudaError_t tips(cudaStream_t) override { return cudaSuccess; }   // tile by tile, on arrival
          cudaError_t diag(int i, cudaStream_t st) override {
            p->prof.begin(st);
            cudaError_t e = launch_diag(P, i, kDiagSolve, st);
            p->prof.end(st, 1, 0.0);
            return e;
          }
          cudaError_t prep(int, cudaStream_t) override { return cudaSuccess; }
          cudaError_t update(int i, int k_lo, int k_hi, cudaStream_t st) override {
            const double rows = p->h_toff[k_hi] - p->h_toff[k_lo], cols = P.m - p->h_cstart[i];
            const double K = 2.0 * (p->h_toff[i + 1] - p->h_toff[i]);
            p->prof.begin(st);
            cudaError_t e = launch_update_f64(P, i, k_lo, k_hi, st);
            p->prof.end(st, 0, 2.0 * rows * cols * K);
            return e;
          }
        } ops(P, p, arr);
        CK(walk_dag(M, ops, ss, sc.aux, sc.ev, sc.lookahead));
        CK(cudaEventRecord(p->ev[2], ss));
        CK(cudaEventRecord(p->ev[3], ss));
      } else {
        HostStructure hs{p->h_toff, p->h_cstart};
        SplitConfig cfg = split_config(p->prec, false);
        if ((rc = split_solve(p->split, P, hs, cfg, ss, sc, p->prof, p->ev[2], p->ev[3], &arr))) return rc;
      }
      // every eigenvalue is known now: the indefinite-eigenvalue check
      p->prof.begin(ss);
      CK(launch_init_state(P, ss, 2));
      p->prof.end(ss, 3, 0.0);
      p->prof.begin(ss);
      CK(launch_post(P, p->hV, ldd, p->hsc, (p->flags & PEVC_NO_NORMALISE) == 0, ss));
      p->prof.end(ss, 3, 0.0);
    } else {
      for (int l = 0; l < M; ++l) CK(cudaStreamWaitEvent(ss, p->hev[l], 0));
      CK(cudaEventRecord(p->ev[2], ss));
      CK(cudaEventRecord(p->ev[3], ss));
    }
    CK(cudaEventRecord(p->ev[4], ss));
    // the pre-scale check: every block's pre-scale against the final maximum
    CK(cudaMemcpyAsync(p->h_hspec, p->hspec, 2 * (size_t)M * sizeof(double), cudaMemcpyDeviceToHost, ss));
    CK(cudaMemcpyAsync(p->h_subd, p->gmax, sizeof(double), cudaMemcpyDeviceToHost, ss));
    CK(cudaStreamSynchronize(ss));
    const double gfin = p->h_subd[0];
    bool redo = false;
    for (int l = 0; l < M && st.m > 0; ++l) {
      int ec = 0;
      std::memcpy(&ec, &p->h_hspec[2 * l + 1], sizeof(int));
      const double gu = p->h_hspec[2 * l];
      if (ec == INT32_MIN || !(gfin > 0.0)) continue;
      const int ef = std::ilogb(gfin) + 1, eu = gu > 0.0 ? std::ilogb(gu) + 1 : INT32_MIN / 2;
      // the pre-scale of a pair is max(0, e_coef + e_max - 1000): it differs
      // only where the final one is positive and the maxima differ
      if (ef != eu && ec + ef - kPrescaleExp > 0) redo = true;
    }
    if (redo) {
      if ((rc = solve_enqueue(p, p->hS, ldd, p->hT, ldd, n, p->hV, ldd, p->hsc, st, false))) return rc;
    }
  }
  // 4. the result to the host: per column tile j the rows above the end of
  //    row tile j (the zeros below are written by the host threads, joined
  //    first so that no two writers share the buffer at once)
  for (auto& x : zero) x.join();
  if (st.m > 0) {
    long long bytes = 0;
    for (int j = 0; j < M; ++j) {
      const int q0 = p->h_cstart[j], q1 = p->h_cstart[j + 1], rows = p->h_toff[j + 1];
      if (q1 <= q0) continue;
      CK(cudaMemcpy2DAsync(V + (size_t)q0 * ldv, (size_t)ldv * sizeof(double), p->hV + (size_t)q0 * ldd,
                           (size_t)ldd * sizeof(double), (size_t)rows * sizeof(double), (size_t)(q1 - q0),
                           cudaMemcpyDeviceToHost, s));
      bytes += (long long)rows * (q1 - q0) * (long long)sizeof(double);
    }
    CK(cudaMemcpyAsync(scale, p->hsc, (size_t)st.m * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    p->host_bytes[1] = bytes + (long long)st.m * sizeof(int32_t);
  }
  CK(cudaEventRecord(p->ev[5], s));
  unsigned bits = 0;
  if ((rc = read_status(p, &bits))) return rc;
  float ms[4] = {0, 0, 0, 0};
  cudaEventElapsedTime(&ms[0], p->ev[0], p->ev[5]);
  cudaEventElapsedTime(&ms[1], p->ev[0], p->ev[1]);
  cudaEventElapsedTime(&ms[2], p->ev[1], p->ev[2]);
  cudaEventElapsedTime(&ms[3], p->ev[2], p->ev[3]);
  p->stats[0] = ms[0];
  p->stats[1] = ms[1];
  p->stats[2] = ms[2];
  p->stats[3] = ms[3];
  float post = 0.0f;
  cudaEventElapsedTime(&post, p->ev[3], p->ev[4]);
  p->stats[4] = post;
  p->stats[5] = M;
  p->stats[6] = p->prof.launches;
  p->stats[7] = p->prec == PEVC_FP64 ? 0.0 : (double)p->split.last_sweeps;
  for (double& x : p->kprof) x = 0.0;
  for (int q = 0; q < p->prof.used; ++q) {
    float t = 0.0f;
    cudaEventElapsedTime(&t, p->prof.ev[2 * q], p->prof.ev[2 * q + 1]);
    const int k = p->prof.kind[q];
    p->kprof[3 * k] += t;
    p->kprof[3 * k + 1] += 1.0;
    p->kprof[3 * k + 2] += p->prof.flops[q];
  }
  return status_from_bits(bits);
}

// A batch of an FP64 plan on the device scheduler: pencils are packed into
// waves whose slices fit the pools (one wave for most batches); per wave the
// host reads every pencil's block structure at once, builds one task list
// that interleaves the pencils' stages by depth (the bottom stage of every
// pencil first, so that all pencils advance together and the large ones keep
// the GPU busy at the end), and the whole wave is one persistent launch
// between the per-pencil pre- and post-passes.  Statuses are read once per wave.
int solve_batched_dag(pevc_plan_t p, int count, const double* const* S, const int* lds, const double* const* T,
                      const int* ldt, const int* n, const int32_t* const* select, double* const* V_out,
                      const int* ldv, int32_t* const* scale_out, int* m_out, int* status) {
  cudaStream_t s = p->stream;
  std::vector<BatchPencil> bp(count > 0 ? count : 1);
  std::vector<char> live(count > 0 ? count : 1, 0);
  const int cap = (int)std::min<long long>(p->b_task_cap, INT32_MAX);
  int b0 = 0;
  while (b0 < count) {
    size_t wo = 0, so = 0, co = 0;
    int b1 = b0;
    for (; b1 < count; ++b1) {
      m_out[b1] = 0;
      status[b1] = check_args(p->n_max, S[b1], lds[b1], T[b1], ldt[b1], n[b1], V_out[b1], ldv[b1], scale_out[b1]);
      live[b1] = 0;
      if (status[b1] || n[b1] == 0) continue;
      const SliceSize z = slice_size(n[b1], p->tb);
      if (wo + z.work > p->b_work_bytes || so + z.strc > p->b_strc_bytes || co + z.cnt > p->b_cnt_ints) {
        if (b1 == b0) return PEVC_ERR_CUDA;   // cannot happen: the pools hold one pencil of order n_max
        break;
      }
      bind_slice(p, b1, n[b1], wo, so, co, bp[b1]);
      live[b1] = 1;
      wo += z.work;
      so += z.strc;
      co += z.cnt;
    }
    // 1. every pencil's subdiagonal (and selection) to the host
    for (int b = b0; b < b1; ++b) {
      if (!live[b]) continue;
      CK(launch_gather_subdiag(S[b], lds[b], n[b], bp[b].v.subd, s));
      if (select && select[b])
        CK(cudaMemcpyAsync(bp[b].v.h_sel, select[b], (size_t)n[b] * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaMemcpyAsync(p->h_b_subd + (size_t)b0 * p->n_max, p->b_subd + (size_t)b0 * p->n_max,
                       (size_t)(b1 - b0) * p->n_max * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // 2. structure, sub-chunks, records
    int maxM = 0;
    for (int b = b0; b < b1; ++b) {
      if (!live[b]) continue;
      BatchPencil& q = bp[b];
      int rc = analyse(&q.v, n[b], select && select[b], q.st);
      int nsm = 0;
      if (!rc && dag_subchunks(q.st.M, q.v.h_cstart, q.v.h_kind, q.sub_first, q.sub_c0, q.sub_nc,
                               q.v.Mmax * dag_nsub_bound(p->tb), &nsm) < 0)
        rc = PEVC_ERR_CUDA;
      if (rc) {
        status[b] = rc;
        live[b] = 0;
        continue;
      }
      q.nsub_max = std::max(nsm, 1);
      m_out[b] = q.st.m;
      maxM = std::max(maxM, q.st.M);
      const size_t tiles = (size_t)q.st.M * (q.st.M + 1) / 2;
      DagPencil& D = p->h_b_pen[b - b0];
      D.P = make_problem(&q.v, S[b], lds[b], T[b], ldt[b], n[b], q.st);
      D.dcnt = q.cnt;
      D.utile = q.cnt + tiles;
      D.usub = q.cnt + 2 * tiles;
      D.sub_first = q.d_sub_first;
      D.sub_c0 = q.d_sub_c0;
      D.sub_nc = q.d_sub_nc;
      D.nsub_max = q.nsub_max;
    }
    // 3. the wave's task list: stage by stage from the bottom, every pencil's
    //    stage of the same depth together
    int cnt = 0;
    for (int d = 0; d < maxM && cnt >= 0; ++d)
      for (int b = b0; b < b1 && cnt >= 0; ++b) {
        if (!live[b]) continue;
        const int M = bp[b].st.M, stage = d == 0 ? M : M - d;
        if (d > 0 && stage < 1) continue;
        cnt = dag_stage_tasks(b - b0, M, stage, bp[b].v.h_dcfirst, bp[b].sub_first, p->h_b_tasks, cnt, cap);
      }
    if (cnt < 0) return PEVC_ERR_CUDA;
    // 4. structure, records and tasks to the device; counters, statuses and
    //    running maxima zeroed
    if (so) CK(cudaMemcpyAsync(p->b_strc, p->h_b_strc, so, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p->b_pen, p->h_b_pen, (size_t)(b1 - b0) * sizeof(DagPencil), cudaMemcpyHostToDevice, s));
    if (cnt) CK(cudaMemcpyAsync(p->b_tasks, p->h_b_tasks, (size_t)cnt * sizeof(int4), cudaMemcpyHostToDevice, s));
    if (co) CK(cudaMemsetAsync(p->b_cnt, 0, co * sizeof(int), s));
    CK(cudaMemsetAsync(p->b_status + b0, 0, (size_t)(b1 - b0) * sizeof(unsigned), s));
    CK(cudaMemsetAsync(p->b_gmax + b0, 0, (size_t)(b1 - b0) * sizeof(double), s));
    CK(cudaMemsetAsync(p->d_ticket, 0, 2 * sizeof(int), s));
    // 5. pre-passes, the walk, post-passes
    for (int b = b0; b < b1; ++b) {
      if (!live[b]) continue;
      const Problem& P = p->h_b_pen[b - b0].P;
      CK(launch_prepass(P, s));
      if (bp[b].st.m > 0) CK(launch_init_state(P, s));
    }
    CK(launch_dag(p->b_pen, p->b_tasks, cnt, p->d_ticket, p->d_ticket + 1, kDagWaitCycles, dag_grid(p->nsm), s));
    for (int b = b0; b < b1; ++b) {
      if (!live[b] || bp[b].st.m == 0) continue;
      CK(launch_post(p->h_b_pen[b - b0].P, V_out[b], ldv[b], scale_out[b], (p->flags & PEVC_NO_NORMALISE) == 0, s));
    }
    // 6. statuses (the host buffers of this wave are free again after this)
    CK(cudaMemcpyAsync(p->h_bstatus + b0, p->b_status + b0, (size_t)(b1 - b0) * sizeof(unsigned),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int b = b0; b < b1; ++b)
      if (live[b]) status[b] = status_from_bits(p->h_bstatus[b]);
    b0 = b1;
  }
  return 0;
}

// A batch on the child plans: pencil b runs on child b % nchild (its own
// workspace and stream), so up to nchild pencils are in flight at once.  Per
// wave the host reads every child's block structure, then enqueues each
// pencil's whole graph without waiting; the status words come back with the
// last synchronisation.
int solve_batched(pevc_plan_t p, int count, const double* const* S, const int* lds, const double* const* T,
                  const int* ldt, const int* n, const int32_t* const* select, double* const* V_out,
                  const int* ldv, int32_t* const* scale_out, int* m_out, int* status) {
  const int K = p->nchild;
  CK(cudaEventRecord(p->bev, p->stream));   // the batch follows the work already on the plan's stream
  for (int c = 0; c < K; ++c) CK(cudaStreamWaitEvent(p->child[c]->stream, p->bev, 0));
  std::vector<char> pending(count > 0 ? count : 1, 0);
  for (int w = 0; w < count; w += K) {
    const int nb = std::min(K, count - w);
    for (int c = 0; c < nb; ++c) {
      const int b = w + c;
      m_out[b] = 0;
      status[b] = check_args(p->n_max, S[b], lds[b], T[b], ldt[b], n[b], V_out[b], ldv[b], scale_out[b]);
      if (status[b] || n[b] == 0) continue;
      const int32_t* sel = select ? select[b] : nullptr;
      status[b] = structure_begin(p->child[c], S[b], lds[b], n[b], sel);
      pending[b] = status[b] == 0;
    }
    for (int c = 0; c < nb; ++c) {
      const int b = w + c;
      if (!pending[b]) continue;
      pevc_plan_t q = p->child[c];
      Structure st;
      const int32_t* sel = select ? select[b] : nullptr;
      int rc = structure_end(q, n[b], sel != nullptr, st);
      if (!rc) {
        m_out[b] = st.m;
        rc = solve_enqueue(q, S[b], lds[b], T[b], ldt[b], n[b], V_out[b], ldv[b], scale_out[b], st, false);
      }
      if (!rc && cudaMemcpyAsync(&p->h_bstatus[b], q->status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                 q->stream) != cudaSuccess)
        rc = PEVC_ERR_CUDA;
      if (rc) {
        status[b] = rc;
        pending[b] = 0;
        if (rc == PEVC_ERR_CUDA) return PEVC_ERR_CUDA;
      }
    }
  }
  for (int c = 0; c < K; ++c) CK(cudaStreamSynchronize(p->child[c]->stream));
  for (int b = 0; b < count; ++b)
    if (pending[b]) status[b] = status_from_bits(p->h_bstatus[b]);
  return 0;
}

}  // namespace

extern "C" {

int pevc_plan(pevc_plan_t* plan, int n_max, int batch_max, int prec, int tile, unsigned flags,
              void* stream) {
  if (!plan) return -1;
  *plan = nullptr;
  if (n_max < 0) return -2;
  if (batch_max < 1) return -3;
  if (prec != PEVC_FP64 && prec != PEVC_SPLIT_BF16X3 && prec != PEVC_SPLIT_FP8X4 && prec != PEVC_SPLIT_BF16X5)
    return -4;
  if (tile != 0 && tile != 32 && tile != 64 && tile != 96 && tile != 128) return -5;
  if (flags & ~(PEVC_NO_NORMALISE | PEVC_NO_CORRECTION | PEVC_STAGE_WALK | PEVC_DEVICE_WALK | PEVC_AUTOTUNE))
    return -6;
  if ((flags & PEVC_STAGE_WALK) && (flags & PEVC_DEVICE_WALK)) return -6;
  std::vector<std::array<double, 4>> tune_log;
  if (flags & PEVC_AUTOTUNE) {
    int t = 0, q = 0;
    unsigned walk = 0;
    const int rc = autotune_pick(n_max, prec, tile, flags & ~PEVC_AUTOTUNE, stream, &t, &q, &walk, &tune_log);
    if (rc) return rc;
    tile = t;
    prec = q;
    flags = (flags & ~(PEVC_STAGE_WALK | PEVC_DEVICE_WALK | PEVC_AUTOTUNE)) | walk;
  }
  pevc_plan_t p = new (std::nothrow) pevc_plan_s();
  if (!p) return PEVC_ERR_NOMEM;
  p->tune_log = std::move(tune_log);
  p->n_max = n_max;
  p->batch_max = batch_max;
  p->prec = prec;
  p->flags = flags;
  p->stream = (cudaStream_t)stream;
  p->tb = tile ? tile : choose_tile(n_max, prec);
  if (cudaGetDevice(&p->dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->dev) != cudaSuccess) {
    delete p;
    return PEVC_ERR_CUDA;
  }
  const int nm = std::max(n_max, 1);
  p->Mmax = (nm + p->tb - 2) / (p->tb - 1) + 1;
  const size_t M = (size_t)p->Mmax;
  int rc = 0;
  rc = rc ? rc : dalloc(&p->Y, M * (M + 1) / 2 * (size_t)p->tb * p->tb);
  rc = rc ? rc : dalloc(&p->ex, M * nm);
  rc = rc ? rc : dalloc(&p->nrm, M * nm);
  rc = rc ? rc : dalloc(&p->EA, M * M);
  rc = rc ? rc : dalloc(&p->tcS, nm);
  rc = rc ? rc : dalloc(&p->tcT, nm);
  rc = rc ? rc : dalloc(&p->gmax, 1);
  rc = rc ? rc : dalloc(&p->ca, nm);
  rc = rc ? rc : dalloc(&p->cb, nm);
  rc = rc ? rc : dalloc(&p->cbeta, nm);
  rc = rc ? rc : dalloc(&p->blk, nm);
  rc = rc ? rc : dalloc(&p->toff, M + 1);
  rc = rc ? rc : dalloc(&p->cstart, M + 1);
  rc = rc ? rc : dalloc(&p->ccol, nm);
  rc = rc ? rc : dalloc(&p->kind, nm);
  rc = rc ? rc : dalloc(&p->status, 1);
  rc = rc ? rc : dalloc(&p->subd, nm);
  rc = rc ? rc : dalloc(&p->dperm, nm);
  rc = rc ? rc : dalloc(&p->dcpos, nm + M);
  rc = rc ? rc : dalloc(&p->dccnt, nm + M);
  rc = rc ? rc : dalloc(&p->dcfirst, M + 1);
  rc = rc ? rc : halloc(&p->h_dperm, nm);
  rc = rc ? rc : halloc(&p->h_dcpos, nm + M);
  rc = rc ? rc : halloc(&p->h_dccnt, nm + M);
  rc = rc ? rc : halloc(&p->h_dcfirst, M + 1);
  rc = rc ? rc : halloc(&p->h_subd, nm);
  rc = rc ? rc : halloc(&p->h_sel, nm);
  rc = rc ? rc : halloc(&p->h_blk, nm);
  rc = rc ? rc : halloc(&p->h_toff, M + 1);
  rc = rc ? rc : halloc(&p->h_cstart, M + 1);
  rc = rc ? rc : halloc(&p->h_ccol, nm);
  rc = rc ? rc : halloc(&p->h_kind, nm);
  rc = rc ? rc : halloc(&p->h_status, 1);
  for (auto& e : p->ev)
    if (!rc && cudaEventCreate(&e) != cudaSuccess) rc = PEVC_ERR_CUDA;
  if (!rc && cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking) != cudaSuccess) rc = PEVC_ERR_CUDA;
  {
    // The stages run strictly in order on the plan's stream; PEVC_LOOKAHEAD=1
    // moves the solves of the next block row to a second stream (they overlap
    // the rest of the update; measured slower on GB300 once the update fills
    // every SM, so it is off by default).
    const char* la = getenv("PEVC_LOOKAHEAD");
    p->lookahead = la && la[0] == '1';
  }
  if (!rc) {
    p->sev = new (std::nothrow) cudaEvent_t[2 * p->Mmax]();
    if (!p->sev) rc = PEVC_ERR_NOMEM;
    for (int q = 0; !rc && q < 2 * p->Mmax; ++q)
      if (cudaEventCreateWithFlags(&p->sev[q], cudaEventDisableTiming) != cudaSuccess) rc = PEVC_ERR_CUDA;
  }
  if (!rc && prec != PEVC_FP64) rc = split_alloc(p->split, n_max, p->tb, p->Mmax, prec);
  if (!rc) {
    // the scheduler: FP64 plans walk the task graph on the device unless
    // PEVC_SCHED=stage asks for the stage walk; every plan keeps the small
    // records of the scheduler's self-test
    const char* sch = getenv("PEVC_SCHED");
    bool dag = default_dag(n_max, batch_max);
    if (flags & PEVC_DEVICE_WALK) dag = true;
    if (flags & PEVC_STAGE_WALK) dag = false;
    if (sch) dag = sch[0] == 'd';       // PEVC_SCHED=dag | stage overrides, for comparisons
    p->dag = prec == PEVC_FP64 && dag;
    const size_t tiles = M * (M + 1) / 2;
    const int nsb = dag_nsub_bound(p->tb);
    p->task_cap = p->dag ? dag_task_bound(p->Mmax, p->tb) : 1;
    p->cnt_cap = p->dag ? tiles * (size_t)(2 + nsb) : 1;
    p->sub_cap = p->Mmax * nsb;
    rc = rc ? rc : dalloc(&p->d_pen, 1);
    rc = rc ? rc : halloc(&p->h_pen, 1);
    rc = rc ? rc : dalloc(&p->d_tasks, (size_t)p->task_cap);
    rc = rc ? rc : halloc(&p->h_tasks, (size_t)p->task_cap);
    rc = rc ? rc : dalloc(&p->d_cnt, p->cnt_cap);
    rc = rc ? rc : dalloc(&p->d_sub, (size_t)(p->Mmax + 1) + 2 * (size_t)p->sub_cap);
    rc = rc ? rc : halloc(&p->h_sub, (size_t)(p->Mmax + 1) + 2 * (size_t)p->sub_cap);
    rc = rc ? rc : dalloc(&p->d_ticket, 2);
  }
  if (!rc && batch_max > 1 && p->dag) {
    // batches on the scheduler: pools that hold the slices of many pencils
    // (workspace: a budget of the larger of about 6 GB and eight pencils of
    // order n_max, or PEVC_BATCH_BYTES, packed by each pencil's own order, so
    // that a batch of small pencils runs as one wave; structure, counters and
    // records for all batch_max pencils)
    const SliceSize z = slice_size(n_max, p->tb);
    const char* bb = getenv("PEVC_BATCH_BYTES");
    const double budget = bb ? atof(bb) : std::max(6e9, 8.0 * (double)z.work);
    const size_t k = std::min<size_t>((size_t)batch_max, std::max<size_t>(1, (size_t)(budget / (double)z.work)));
    const size_t B = (size_t)batch_max;
    p->bdag = true;
    p->b_work_bytes = k * z.work;
    p->b_strc_bytes = B * z.strc;
    p->b_cnt_ints = B * z.cnt;
    p->b_task_cap = (long long)B * dag_task_bound(slice_mmax(n_max, p->tb), p->tb);
    rc = rc ? rc : dalloc(&p->b_work, p->b_work_bytes);
    rc = rc ? rc : dalloc(&p->b_strc, p->b_strc_bytes);
    rc = rc ? rc : halloc(&p->h_b_strc, p->b_strc_bytes);
    rc = rc ? rc : dalloc(&p->b_cnt, p->b_cnt_ints);
    rc = rc ? rc : dalloc(&p->b_subd, B * nm);
    rc = rc ? rc : halloc(&p->h_b_subd, B * nm);
    rc = rc ? rc : halloc(&p->h_b_sel, B * nm);
    rc = rc ? rc : dalloc(&p->b_status, B);
    rc = rc ? rc : dalloc(&p->b_gmax, B);
    rc = rc ? rc : dalloc(&p->b_pen, B);
    rc = rc ? rc : halloc(&p->h_b_pen, B);
    rc = rc ? rc : dalloc(&p->b_tasks, (size_t)p->b_task_cap);
    rc = rc ? rc : halloc(&p->h_b_tasks, (size_t)p->b_task_cap);
    rc = rc ? rc : halloc(&p->h_bstatus, B);
  } else if (!rc && batch_max > 1) {
    // child plans for concurrent pencils, as many as about 4 GB of workspace
    // allows (at most 8)
    const double tiles = (double)p->Mmax * (p->Mmax + 1) / 2.0 * (double)p->tb * p->tb;
    const double bytes = tiles * (prec == PEVC_FP64 ? 8.0 : 36.0) + 64.0 * nm;
    int k = (int)(4e9 / bytes);
    k = std::max(1, std::min(k, std::min(batch_max, 8)));
    rc = halloc(&p->h_bstatus, (size_t)batch_max);
    if (!rc && cudaEventCreateWithFlags(&p->bev, cudaEventDisableTiming) != cudaSuccess) rc = PEVC_ERR_CUDA;
    for (int c = 0; !rc && c < k; ++c) {
      if (cudaStreamCreateWithFlags(&p->cstream[c], cudaStreamNonBlocking) != cudaSuccess) {
        rc = PEVC_ERR_CUDA;
        break;
      }
      rc = pevc_plan(&p->child[c], n_max, 1, prec, p->tb, flags, p->cstream[c]);
      if (!rc) p->nchild = c + 1;
    }
  }
  if (rc) {
    free_plan(p);
    return rc;
  }
  *plan = p;
  return 0;
}

int pevc_solve(pevc_plan_t plan, const double* S, int lds, const double* T, int ldt, int n,
               const int32_t* select, double* V_out, int ldv, int32_t* scale_out, int* m_out) {
  if (!plan) return -1;
  if (n < 0 || n > plan->n_max) return -6;
  if (n > 0 && !S) return -2;
  if (lds < std::max(n, 1)) return -3;
  if (n > 0 && !T) return -4;
  if (ldt < std::max(n, 1)) return -5;
  if (n > 0 && !V_out) return -8;
  if (ldv < std::max(n, 1)) return -9;
  if (n > 0 && !scale_out) return -10;
  if (!m_out) return -11;
  return solve_one(plan, S, lds, T, ldt, n, select, V_out, ldv, scale_out, m_out);
}

int pevc_solve_host(pevc_plan_t plan, const double* S, int lds, const double* T, int ldt, int n,
                    const int32_t* select, double* V_out, int ldv, int32_t* scale_out, int* m_out) {
  if (!plan) return -1;
  if (n < 0 || n > plan->n_max) return -6;
  if (n > 0 && !S) return -2;
  if (lds < std::max(n, 1)) return -3;
  if (n > 0 && !T) return -4;
  if (ldt < std::max(n, 1)) return -5;
  if (n > 0 && !V_out) return -8;
  if (ldv < std::max(n, 1)) return -9;
  if (n > 0 && !scale_out) return -10;
  if (!m_out) return -11;
  return solve_host(plan, S, lds, T, ldt, n, select, V_out, ldv, scale_out, m_out);
}

int pevc_last_host_bytes(pevc_plan_t plan, long long* out) {
  if (!plan) return -1;
  if (!out) return -2;
  out[0] = plan->host_bytes[0];
  out[1] = plan->host_bytes[1];
  return 0;
}

int pevc_solve_batched(pevc_plan_t plan, int count, const double* const* S, const int* lds,
                       const double* const* T, const int* ldt, const int* n,
                       const int32_t* const* select, double* const* V_out, const int* ldv,
                       int32_t* const* scale_out, int* m_out, int* status) {
  if (!plan) return -1;
  if (count < 0 || count > plan->batch_max) return -2;
  if (count > 0 && (!S || !lds || !T || !ldt || !n || !V_out || !ldv || !scale_out || !m_out || !status))
    return -3;
  plan->last_m = -1;   // the plan's column kinds no longer describe one solve
  if (plan->bdag)
    return solve_batched_dag(plan, count, S, lds, T, ldt, n, select, V_out, ldv, scale_out, m_out, status);
  if (plan->nchild > 0)
    return solve_batched(plan, count, S, lds, T, ldt, n, select, V_out, ldv, scale_out, m_out, status);
  for (int b = 0; b < count; ++b) {
    status[b] = pevc_solve(plan, S[b], lds[b], T[b], ldt[b], n[b], select ? select[b] : nullptr,
                           V_out[b], ldv[b], scale_out[b], &m_out[b]);
    if (status[b] == PEVC_ERR_CUDA) return PEVC_ERR_CUDA;
  }
  return 0;
}

int pevc_backtransform(pevc_plan_t plan, const double* Z, int ldz, int n, const double* V, int ldv, int m,
                       const int* kinds, double* X, int ldx, unsigned flags) {
  if (!plan) return -1;
  if (n < 0 || n > plan->n_max) return -4;
  const int ld_min = n > 1 ? n : 1;
  if (!Z && n > 0) return -2;
  if (ldz < ld_min) return -3;
  if (!V && m > 0) return -5;
  if (ldv < ld_min) return -6;
  if (m < 0 || m > n) return -7;
  if (!X && m > 0) return -9;
  if (ldx < ld_min) return -10;
  if (flags & ~(PEVC_NO_NORMALISE | PEVC_BT_EMULATED | PEVC_BT_CUBLAS)) return -11;
  const signed char* dkind = plan->kind;
  if (kinds) {
    for (int q = 0; q < m; ++q) {
      const int k = kinds[q];
      if (k < 0 || k > 2 || (k == 1 && (q + 1 >= m || kinds[q + 1] != 2)) || (k == 2 && (q == 0 || kinds[q - 1] != 1)))
        return -8;
    }
  } else if (m > 0 && plan->last_m != m) {
    return -8;
  }
  if (n == 0 || m == 0) return 0;
  if (cudaSetDevice(plan->dev) != cudaSuccess) return PEVC_ERR_CUDA;
  if (kinds && !(flags & PEVC_NO_NORMALISE)) {
    if (!plan->bt_kind && cudaMalloc(&plan->bt_kind, (size_t)plan->n_max) != cudaSuccess) return PEVC_ERR_NOMEM;
    if (!plan->h_bt_kind && cudaMallocHost(&plan->h_bt_kind, (size_t)plan->n_max) != cudaSuccess)
      return PEVC_ERR_NOMEM;
    CK(cudaStreamSynchronize(plan->stream));   // the staging buffer may still feed an earlier copy
    for (int q = 0; q < m; ++q) plan->h_bt_kind[q] = (signed char)kinds[q];
    CK(cudaMemcpyAsync(plan->bt_kind, plan->h_bt_kind, (size_t)m, cudaMemcpyHostToDevice, plan->stream));
    dkind = plan->bt_kind;
  }
  if (flags & (PEVC_BT_CUBLAS | PEVC_BT_EMULATED)) {
    int rc = bt_handle(&plan->blas, plan->stream);
    if (rc) return rc;
    if ((rc = bt_gemm(plan->blas, (flags & PEVC_BT_EMULATED) != 0, n, m, Z, ldz, V, ldv, X, ldx))) return rc;
  } else {
    // the library's split GEMM; its workspace comes with the first call
    if (!plan->bt_ws) {
      plan->bt_ws_bytes = bt_split_bytes(plan->n_max);
      if (cudaMalloc(&plan->bt_ws, plan->bt_ws_bytes) != cudaSuccess) {
        plan->bt_ws = nullptr;
        return PEVC_ERR_NOMEM;
      }
    }
    CK(launch_bt_split(Z, ldz, n, V, ldv, m, X, ldx, plan->bt_ws, plan->stream));
  }
  if (!(flags & PEVC_NO_NORMALISE)) CK(launch_bt_normalise(X, ldx, n, m, dkind, plan->stream));
  CK(cudaStreamSynchronize(plan->stream));
  return 0;
}

int pevc_backtransform_cplx(pevc_plan_t plan, const double* Z, int ldz, int n, const double* V, int ldv, int m,
                            double* X, int ldx, unsigned flags) {
  if (!plan) return -1;
  if (n < 0 || n > plan->n_max) return -4;
  const int ld_min = n > 1 ? n : 1;
  if (!Z && n > 0) return -2;
  if (ldz < ld_min) return -3;
  if (!V && m > 0) return -5;
  if (ldv < ld_min) return -6;
  if (m < 0 || m > n) return -7;
  if (!X && m > 0) return -8;
  if (ldx < ld_min) return -9;
  if (flags & ~PEVC_NO_NORMALISE) return -10;
  if ((uintptr_t)Z & 15u) return -2;
  if ((uintptr_t)V & 15u) return -5;
  if ((uintptr_t)X & 15u) return -8;
  if (n == 0 || m == 0) return 0;
  if (cudaSetDevice(plan->dev) != cudaSuccess) return PEVC_ERR_CUDA;
  int rc = bt_handle(&plan->blas, plan->stream);
  if (rc) return rc;
  if ((rc = bt_zgemm(plan->blas, n, m, Z, ldz, V, ldv, X, ldx))) return rc;
  if (!(flags & PEVC_NO_NORMALISE)) CK(launch_bt_normalise_c(X, ldx, n, m, plan->stream));
  CK(cudaStreamSynchronize(plan->stream));
  return 0;
}

int pevc_solve_left(pevc_plan_t plan, const double* S, int lds, const double* T, int ldt, int n,
                    const int32_t* select, double* U_out, int ldu, int32_t* scale_out, int* m_out) {
  if (!plan) return -1;
  if (n < 0 || n > plan->n_max) return -6;
  if (n > 0 && !S) return -2;
  if (lds < std::max(n, 1)) return -3;
  if (n > 0 && !T) return -4;
  if (ldt < std::max(n, 1)) return -5;
  if (n > 0 && !U_out) return -8;
  if (ldu < std::max(n, 1)) return -9;
  if (n > 0 && !scale_out) return -10;
  if (!m_out) return -11;
  *m_out = 0;
  if (n == 0) return 0;
  pevc_plan_t p = plan;
  if (cudaSetDevice(p->dev) != cudaSuccess) return PEVC_ERR_CUDA;
  if (!p->lS) {
    const size_t nn = (size_t)p->n_max * p->n_max;
    int rc = dalloc(&p->lS, nn);
    rc = rc ? rc : dalloc(&p->lT, nn);
    rc = rc ? rc : dalloc(&p->lV, nn);
    rc = rc ? rc : dalloc(&p->lsel, (size_t)p->n_max);
    rc = rc ? rc : dalloc(&p->lsc, (size_t)p->n_max);
    if (rc) return rc;
  }
  cudaStream_t s = p->stream;
  CK(launch_flip_transpose(S, lds, n, p->lS, s));
  CK(launch_flip_transpose(T, ldt, n, p->lT, s));
  if (select) CK(launch_flip_select(select, n, p->lsel, s));
  int rc = solve_one(p, p->lS, n, p->lT, n, n, select ? p->lsel : nullptr, p->lV, n, p->lsc, m_out);
  p->last_m = -1;   // the plan's column kinds describe the flipped pencil
  if (rc) return rc;
  CK(launch_left_out(p->lV, n, *m_out, p->kind, p->lsc, U_out, ldu, scale_out, s));
  CK(cudaStreamSynchronize(s));
  return 0;
}

namespace {

// Arguments shared by the complex solves (numbered as in the ABI, the plan
// first): 0 when they are valid, else -i.  complex128 elements are read and
// written as 16-byte pairs, so S, T and the output must be 16-byte aligned.
int cplx_args(pevc_plan_t plan, const double* S, int lds, const double* T, int ldt, int n, const double* out,
              int ldo, const int32_t* scale_out, const int* m_out) {
  if (!plan) return -1;
  if (n < 0 || n > plan->n_max) return -6;
  if (n > 0 && !S) return -2;
  if (lds < std::max(n, 1)) return -3;
  if (n > 0 && !T) return -4;
  if (ldt < std::max(n, 1)) return -5;
  if (n > 0 && !out) return -8;
  if (ldo < std::max(n, 1)) return -9;
  if (n > 0 && !scale_out) return -10;
  if (!m_out) return -11;
  if (n > 0 && ((uintptr_t)S & 15u)) return -2;
  if (n > 0 && ((uintptr_t)T & 15u)) return -4;
  if (n > 0 && ((uintptr_t)out & 15u)) return -8;
  return 0;
}

}  // namespace

int pevc_solve_cplx(pevc_plan_t plan, const double* S, int lds, const double* T, int ldt, int n,
                    const int32_t* select, double* V_out, int ldv, int32_t* scale_out, int* m_out) {
  const int bad = cplx_args(plan, S, lds, T, ldt, n, V_out, ldv, scale_out, m_out);
  if (bad) return bad;
  *m_out = 0;
  if (n == 0) return 0;
  if (cudaSetDevice(plan->dev) != cudaSuccess) return PEVC_ERR_CUDA;
  return cplx_solve(&plan->cx, plan->n_max, plan->stream, S, lds, T, ldt, n, select, V_out, ldv, scale_out, m_out,
                    !(plan->flags & PEVC_NO_NORMALISE));
}

int pevc_solve_cplx_left(pevc_plan_t plan, const double* S, int lds, const double* T, int ldt, int n,
                         const int32_t* select, double* U_out, int ldu, int32_t* scale_out, int* m_out) {
  const int bad = cplx_args(plan, S, lds, T, ldt, n, U_out, ldu, scale_out, m_out);
  if (bad) return bad;
  *m_out = 0;
  if (n == 0) return 0;
  if (cudaSetDevice(plan->dev) != cudaSuccess) return PEVC_ERR_CUDA;
  return cplx_solve_left(&plan->cx, plan->n_max, plan->stream, S, lds, T, ldt, n, select, U_out, ldu, scale_out,
                         m_out, !(plan->flags & PEVC_NO_NORMALISE));
}

int pevc_watchdog_selftest(pevc_plan_t plan, int withhold, long long cycles) {
  if (!plan) return -1;
  if (withhold != 0 && withhold != 1) return -2;
  if (cycles <= 0 || cycles > 4000000000LL) return -3;   // at most about 2 s of SM clock
  if (cudaSetDevice(plan->dev) != cudaSuccess) return PEVC_ERR_CUDA;
  CK(cudaMemsetAsync(plan->status, 0, sizeof(unsigned), plan->stream));
  CK(launch_watchdog_probe(plan->status, withhold, cycles, plan->stream));
  unsigned bits = 0;
  const int rc = read_status(plan, &bits);
  if (rc) return rc;
  return (bits & kStTimeout) ? PEVC_ERR_TIMEOUT : 0;
}

int pevc_scheduler_selftest(pevc_plan_t plan, int withhold, long long cycles) {
  if (!plan) return -1;
  if (withhold != 0 && withhold != 1) return -2;
  if (cycles <= 0 || cycles > 4000000000LL) return -3;   // at most about 2 s of SM clock
  if (cudaSetDevice(plan->dev) != cudaSuccess) return PEVC_ERR_CUDA;
  // a pencil record whose only use is the probe's counter and status word
  DagPencil& hp = *plan->h_pen;
  hp = DagPencil{};
  hp.P.status = plan->status;
  hp.dcnt = plan->d_cnt;
  cudaStream_t s = plan->stream;
  CK(cudaMemsetAsync(plan->status, 0, sizeof(unsigned), s));
  CK(cudaMemcpyAsync(plan->d_pen, plan->h_pen, sizeof(DagPencil), cudaMemcpyHostToDevice, s));
  CK(launch_dag_selftest(plan->d_pen, plan->d_tasks, plan->d_ticket, plan->d_ticket + 1, withhold, cycles, s));
  unsigned bits = 0;
  const int rc = read_status(plan, &bits);
  if (rc) return rc;
  return (bits & kStTimeout) ? PEVC_ERR_TIMEOUT : 0;
}

int pevc_destroy(pevc_plan_t plan) {
  if (!plan) return 0;
  cudaStreamSynchronize(plan->stream);
  free_plan(plan);
  return 0;
}

const char* pevc_strerror(int code) {
  switch (code) {
    case PEVC_SUCCESS: return "success";
    case PEVC_ERR_NOT_SCHUR: return "pencil is not in standardised real Schur form";
    case PEVC_ERR_NONFINITE: return "Inf or NaN in the input";
    case PEVC_ERR_INDEFINITE: return "indefinite eigenvalue (alpha = beta = 0) selected";
    case PEVC_ERR_TIMEOUT: return "a bounded device wait timed out";
    case PEVC_ERR_CUDA: return "CUDA runtime error";
    case PEVC_ERR_NOMEM: return "out of memory";
    case PEVC_ERR_UNSUPPORTED: return "unsupported feature";
    case PEVC_ERR_TOO_LARGE: return "order above PEVC_STATIC_N_MAX for pevc_solve_static";
    default: return code < 0 ? "invalid argument" : "unknown status";
  }
}

int pevc_plan_info(pevc_plan_t plan, int* info) {
  if (!plan) return -1;
  if (!info) return -2;
  info[0] = plan->tb;
  info[1] = plan->prec;
  info[2] = plan->n_max;
  info[3] = plan->batch_max;
  info[4] = (int)plan->flags;
  info[5] = plan->nsm;
  info[6] = plan->prec == PEVC_FP64 ? 0 : (plan->prec == PEVC_SPLIT_BF16X5 ? 5 : (plan->prec == PEVC_SPLIT_BF16X3 ? 3 : 4));
  {
    const SplitConfig c = split_config(plan->prec, (plan->flags & PEVC_NO_CORRECTION) == 0);
    info[7] = (plan->prec != PEVC_FP64 && c.correction) ? c.sweeps : 0;
  }
  return 0;
}

int pevc_autotune_log(pevc_plan_t plan, double* out, int cap) {
  if (!plan) return -1;
  if (!out && cap > 0) return -2;
  const int k = (int)plan->tune_log.size();
  for (int q = 0; q < k && q < cap; ++q)
    for (int x = 0; x < 4; ++x) out[4 * q + x] = plan->tune_log[q][x];
  return k;
}

int pevc_set_profile(pevc_plan_t plan, int on) {
  if (!plan) return -1;
  Profiler& pr = plan->prof;
  if (on && !pr.ev) {
    const int cap = 8192;
    pr.ev = new (std::nothrow) cudaEvent_t[2 * cap];
    pr.kind = new (std::nothrow) int[cap];
    pr.flops = new (std::nothrow) double[cap];
    if (!pr.ev || !pr.kind || !pr.flops) return PEVC_ERR_NOMEM;
    for (int q = 0; q < 2 * cap; ++q)
      if (cudaEventCreate(&pr.ev[q]) != cudaSuccess) return PEVC_ERR_CUDA;
    pr.cap = cap;
  }
  pr.on = on != 0;
  return 0;
}

int pevc_kernel_profile(pevc_plan_t plan, double* out) {
  if (!plan) return -1;
  if (!out) return -2;
  for (int q = 0; q < 12; ++q) out[q] = plan->kprof[q];
  return 0;
}

int pevc_last_stats(pevc_plan_t plan, double* stats) {
  if (!plan) return -1;
  if (!stats) return -2;
  for (int q = 0; q < 8; ++q) stats[q] = plan->stats[q];
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// pevc_solve_static: the FP64 solve of small pencils for callers that cannot
// allocate device memory.  Every piece of device workspace lives in one
// file-scope array; the host-side structure arrays live on the caller's
// stack.  The kernels and their order are those of an FP64 plan whose n_max
// equals the call's n (same tile order, stages walked strictly in order).

namespace {

constexpr int kStaticNMax = PEVC_STATIC_N_MAX;
constexpr int kStaticMaxDevices = 64;

constexpr size_t static_round(size_t x) { return (x + 255) / 256 * 256; }
constexpr int static_mmax(int n, int tb) { return ((n < 1 ? 1 : n) + tb - 2) / (tb - 1) + 1; }

// Byte offsets of the workspace pieces inside the scratch array, each on a
// 256-byte boundary; bytes = the total.
struct StaticLayout {
  size_t Y = 0, ex = 0, nrm = 0, EA = 0, tcS = 0, tcT = 0, gmax = 0, ca = 0, cb = 0, cbeta = 0, blk = 0,
         toff = 0, cstart = 0, ccol = 0, kind = 0, status = 0, subd = 0, dperm = 0, dcpos = 0, dccnt = 0,
         dcfirst = 0, bytes = 0;
};

constexpr StaticLayout static_layout(int n, int tb) {
  StaticLayout L;
  const size_t nm = n < 1 ? 1 : (size_t)n;
  const size_t M = (size_t)static_mmax(n, tb);
  size_t o = 0;
  L.Y = o;       o = static_round(o + M * (M + 1) / 2 * (size_t)tb * tb * sizeof(double));
  L.ex = o;      o = static_round(o + M * nm * sizeof(int));
  L.nrm = o;     o = static_round(o + M * nm * sizeof(double));
  L.EA = o;      o = static_round(o + M * M * sizeof(int));
  L.tcS = o;     o = static_round(o + nm * sizeof(double));
  L.tcT = o;     o = static_round(o + nm * sizeof(double));
  L.gmax = o;    o = static_round(o + sizeof(double));
  L.ca = o;      o = static_round(o + nm * sizeof(double));
  L.cb = o;      o = static_round(o + nm * sizeof(double));
  L.cbeta = o;   o = static_round(o + nm * sizeof(double));
  L.blk = o;     o = static_round(o + nm);
  L.toff = o;    o = static_round(o + (M + 1) * sizeof(int));
  L.cstart = o;  o = static_round(o + (M + 1) * sizeof(int));
  L.ccol = o;    o = static_round(o + nm * sizeof(int));
  L.kind = o;    o = static_round(o + nm);
  L.status = o;  o = static_round(o + sizeof(unsigned));
  L.subd = o;    o = static_round(o + nm * sizeof(double));
  L.dperm = o;   o = static_round(o + nm * sizeof(int));
  L.dcpos = o;   o = static_round(o + (nm + M) * sizeof(int));
  L.dccnt = o;   o = static_round(o + (nm + M) * sizeof(int));
  L.dcfirst = o; o = static_round(o + (M + 1) * sizeof(int));
  L.bytes = o;
  return L;
}

// The FP64 tile choice is 32 up to order 256 and 64 up to order 1024, so the
// largest layout below the maximum order is one of these two.
constexpr size_t static_max(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kStaticBytes = static_max(static_layout(256, 32).bytes, static_layout(kStaticNMax, 64).bytes);
constexpr int kStaticMMax = static_mmax(256, 32) > static_mmax(kStaticNMax, 64) ? static_mmax(256, 32)
                                                                                 : static_mmax(kStaticNMax, 64);
static_assert(kStaticNMax <= 1024, "the static entry point assumes the FP64 tile choice of orders <= 1024");

}  // namespace

// The scratch array: in host code this name only stands for the device
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

namespace {

std::mutex g_static_mutex;
void* g_static_addr[kStaticMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does this set-up).
int static_scratch(unsigned char** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticMaxDevices) return PEVC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_addr[dev]) {
    void* ptr = nullptr;
    CK(cudaGetSymbolAddress(&ptr, g_static_scratch));
    if (!ptr) return PEVC_ERR_CUDA;
    g_static_addr[dev] = ptr;
  }
  *out = (unsigned char*)g_static_addr[dev];
  return 0;
}

// Host copies of the structure for one call (on the caller's stack).
struct StaticHost {
  double subd[kStaticNMax];
  int32_t sel[kStaticNMax];
  signed char blk[kStaticNMax];
  signed char kind[kStaticNMax];
  int ccol[kStaticNMax];
  int dperm[kStaticNMax];
  int dcpos[kStaticNMax + kStaticMMax];
  int dccnt[kStaticNMax + kStaticMMax];
  int toff[kStaticMMax + 1];
  int cstart[kStaticMMax + 1];
  int dcfirst[kStaticMMax + 1];
  unsigned status;
};

struct StaticF64Ops : StageOps {
  const Problem& P;
  explicit StaticF64Ops(const Problem& P_) : P(P_) {}
  cudaError_t tips(cudaStream_t st) override { return launch_diag(P, 0, kDiagTip, st); }
  cudaError_t diag(int i, cudaStream_t st) override { return launch_diag(P, i, kDiagSolve, st); }
  cudaError_t prep(int, cudaStream_t) override { return cudaSuccess; }
  cudaError_t update(int i, int k_lo, int k_hi, cudaStream_t st) override {
    return launch_update_f64(P, i, k_lo, k_hi, st);
  }
};

int solve_static(const double* S, int lds, const double* T, int ldt, int n, const int32_t* sel, double* V,
                 int ldv, int32_t* scale, int* m_out, unsigned flags, cudaStream_t s) {
  *m_out = 0;
  unsigned char* base = nullptr;
  int rc = static_scratch(&base);
  if (rc) return rc;
  if (n == 0) return 0;
  const int tb = choose_tile(n, PEVC_FP64);
  const StaticLayout L = static_layout(n, tb);
  if (L.bytes > kStaticBytes) return PEVC_ERR_TOO_LARGE;
  StaticHost h;
  pevc_plan_s p;   // a view: every pointer below is borrowed, nothing is freed
  p.n_max = n;
  p.prec = PEVC_FP64;
  p.tb = tb;
  p.flags = flags;
  p.stream = s;
  p.Mmax = static_mmax(n, tb);
  p.lookahead = false;
  p.Y = (double*)(base + L.Y);
  p.ex = (int*)(base + L.ex);
  p.nrm = (double*)(base + L.nrm);
  p.EA = (int*)(base + L.EA);
  p.tcS = (double*)(base + L.tcS);
  p.tcT = (double*)(base + L.tcT);
  p.gmax = (double*)(base + L.gmax);
  p.ca = (double*)(base + L.ca);
  p.cb = (double*)(base + L.cb);
  p.cbeta = (double*)(base + L.cbeta);
  p.blk = (signed char*)(base + L.blk);
  p.toff = (int*)(base + L.toff);
  p.cstart = (int*)(base + L.cstart);
  p.ccol = (int*)(base + L.ccol);
  p.kind = (signed char*)(base + L.kind);
  p.status = (unsigned*)(base + L.status);
  p.subd = (double*)(base + L.subd);
  p.dperm = (int*)(base + L.dperm);
  p.dcpos = (int*)(base + L.dcpos);
  p.dccnt = (int*)(base + L.dccnt);
  p.dcfirst = (int*)(base + L.dcfirst);
  p.h_subd = h.subd;
  p.h_sel = h.sel;
  p.h_blk = h.blk;
  p.h_toff = h.toff;
  p.h_cstart = h.cstart;
  p.h_ccol = h.ccol;
  p.h_kind = h.kind;
  p.h_status = &h.status;
  p.h_dperm = h.dperm;
  p.h_dcpos = h.dcpos;
  p.h_dccnt = h.dccnt;
  p.h_dcfirst = h.dcfirst;

  // 1. block structure and selection to the host (pageable copies on s)
  CK(launch_gather_subdiag(S, lds, n, p.subd, s));
  if (n > 1) CK(cudaMemcpyAsync(p.h_subd, p.subd, (size_t)(n - 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (sel) CK(cudaMemcpyAsync(p.h_sel, sel, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  Structure st;
  if ((rc = analyse(&p, n, sel != nullptr, st))) return rc;
  *m_out = st.m;
  // 2. structure to the device; the status word and the running maximum
  //    must start at zero (the array keeps the previous call's contents)
  CK(cudaMemcpyAsync(p.blk, p.h_blk, (size_t)n, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(p.toff, p.h_toff, (size_t)(st.M + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(p.cstart, p.h_cstart, (size_t)(st.M + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  if (st.m > 0) {
    CK(cudaMemcpyAsync(p.ccol, p.h_ccol, (size_t)st.m * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p.kind, p.h_kind, (size_t)st.m, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p.dperm, p.h_dperm, (size_t)st.m * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p.dcpos, p.h_dcpos, (size_t)st.nchunks * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(p.dccnt, p.h_dccnt, (size_t)st.nchunks * sizeof(int), cudaMemcpyHostToDevice, s));
  }
  CK(cudaMemcpyAsync(p.dcfirst, p.h_dcfirst, (size_t)(st.M + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(p.status, 0, sizeof(unsigned), s));
  CK(cudaMemsetAsync(p.gmax, 0, sizeof(double), s));
  Problem P = make_problem(&p, S, lds, T, ldt, n, st);
  CK(launch_prepass(P, s));
  unsigned bits = 0;
  if ((rc = read_status(&p, &bits))) return rc;
  if (bits) return status_from_bits(bits);
  if (st.m > 0) {
    // 3. the task graph, bottom-up by block row; 4. post-processing
    CK(launch_init_state(P, s));
    StaticF64Ops ops(P);
    CK(walk_dag(st.M, ops, s, nullptr, nullptr, false));
    CK(launch_post(P, V, ldv, scale, (flags & PEVC_NO_NORMALISE) == 0, s));
  }
  if ((rc = read_status(&p, &bits))) return rc;
  return status_from_bits(bits);
}

}  // namespace

extern "C" int pevc_solve_static(const double* S, int lds, const double* T, int ldt, int n,
                                 const int32_t* select, double* V_out, int ldv, int32_t* scale_out, int* m_out,
                                 unsigned flags, void* stream) {
  if (n < 0) return -5;
  if (n > kStaticNMax) return PEVC_ERR_TOO_LARGE;
  if (n > 0 && !S) return -1;
  if (lds < std::max(n, 1)) return -2;
  if (n > 0 && !T) return -3;
  if (ldt < std::max(n, 1)) return -4;
  if (n > 0 && !V_out) return -7;
  if (ldv < std::max(n, 1)) return -8;
  if (n > 0 && !scale_out) return -9;
  if (!m_out) return -10;
  if (flags & ~PEVC_NO_NORMALISE) return -11;
  return solve_static(S, lds, T, ldt, n, select, V_out, ldv, scale_out, m_out, flags, (cudaStream_t)stream);
}

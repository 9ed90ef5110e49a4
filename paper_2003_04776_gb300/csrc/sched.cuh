// sched.cuh -- the walk of the task graph of Algorithm 1 (Section 3), shared
// by the FP64 and the split-precision passes.
//
// The graph is the disjoint union of one sub-graph per block column
// (Section 5.3): a tip task on (j, j), then for i = j-1 .. 0 the updates of
// every tile above from tile (i+1, j) and the solve of tile (i, j).  The
// solves of row i and the update from row i read column block i of S and T
// (and blocks right of it), so when the inputs arrive by column blocks from
// the right, arrive(i) before that work orders it after its inputs.  All block
// columns advance together, one block row per stage, bottom-up.  With
// lookahead, stage i first updates only tile row i-1 -- the row whose solves
// are on the critical path -- then the solves of row i-1 run on a second
// stream while the rest of stage i's update (tile rows < i-1) runs on the
// first: FP64 diagonal solves and tensor-core updates overlap on different
// pipes, and data dependences are carried by events (the solves of row i-1
// touch only tiles (i-1, j); the rest of the update touches rows < i-1).
#pragma once

#include "common.cuh"

namespace pevc {

struct StageOps {
  virtual ~StageOps() = default;
  // stage i is about to run: what it needs of column block i of S and T
  // (for inputs that arrive by column blocks; nothing otherwise)
  virtual cudaError_t arrive(int, cudaStream_t) { return cudaSuccess; }
  virtual cudaError_t tips(cudaStream_t s) = 0;                 // kernel 1 on every (j, j)
  virtual cudaError_t diag(int i, cudaStream_t s) = 0;          // kernel 3 on (i, j), j > i
  virtual cudaError_t prep(int i, cudaStream_t s) = 0;          // operand preparation of row i
  virtual cudaError_t update(int i, int k_lo, int k_hi, cudaStream_t s) = 0;  // kernel 2: rows [k_lo, k_hi)
};

// events: 2*M events owned by the caller.
inline cudaError_t walk_dag(int M, StageOps& ops, cudaStream_t main, cudaStream_t aux, cudaEvent_t* ev,
                            bool lookahead) {
  cudaError_t e;
  if ((e = ops.tips(main)) != cudaSuccess) return e;
  if (!lookahead || !aux) {
    for (int i = M - 1; i >= 0; --i) {
      if ((e = ops.arrive(i, main)) != cudaSuccess) return e;
      if (i < M - 1 && (e = ops.diag(i, main)) != cudaSuccess) return e;
      if (i > 0) {
        if ((e = ops.prep(i, main)) != cudaSuccess) return e;
        if ((e = ops.update(i, 0, i, main)) != cudaSuccess) return e;
      }
    }
    return cudaSuccess;
  }
  if ((e = ops.arrive(M - 1, main)) != cudaSuccess) return e;
  for (int i = M - 1; i >= 1; --i) {
    cudaEvent_t ev_upd = ev[2 * i], ev_diag = ev[2 * i + 1];
    if ((e = ops.arrive(i - 1, main)) != cudaSuccess) return e;
    if ((e = ops.prep(i, main)) != cudaSuccess) return e;
    if ((e = ops.update(i, i - 1, i, main)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ev_upd, main)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(aux, ev_upd, 0)) != cudaSuccess) return e;
    if ((e = ops.diag(i - 1, aux)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ev_diag, aux)) != cudaSuccess) return e;
    if (i - 1 > 0 && (e = ops.update(i, 0, i - 1, main)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(main, ev_diag, 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace pevc

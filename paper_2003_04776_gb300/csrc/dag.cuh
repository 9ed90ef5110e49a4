// dag.cuh -- the device-side scheduler of the task graph of Algorithm 1
// (Section 3; the graph of Section 5.3 is the disjoint union of one sub-graph
// per block column).
//
// One persistent kernel (k_dag) runs every task of one or several pencils.
// Its CTAs take tasks from one list in a fixed order with an atomic ticket
// and wait, thread 0 alone and bounded in SM clock cycles, for the task's
// dependences on per-tile ready counters in global memory:
//   TIP  (j, c)       kernel 1 on chunk c of tile (j, j)              no dependence
//   DIAG (i, j, c)    kernel 3 on chunk c of tile (i, j), i < j       every update into (i, j) applied
//   UPD  (k, i, j, s) kernel 2: sub-chunk s of Y_kj from X = Y_ij,    every chunk of (i, j) solved, and
//                     k < i <= j                                      the update from source i + 1 into
//                                                                     (k, j, s) applied (updates land
//                                                                     in descending source order, the
//                                                                     order of the stage walk, so the
//                                                                     result is deterministic)
// The list is a topological order (every dependence of a task lies before
// it), so the CTA holding the earliest unfinished task never waits and the
// walk always progresses, with no need for all CTAs to be resident at once.
// A column chain runs ahead as soon as its own dependences are met: the solves
// of a block row overlap the updates of the rows above, and the partial last
// wave of one stage fills with the next stage's ready tasks.  A wait that runs
// out sets kStTimeout in the pencil's status word and an abort flag that ends
// every CTA's walk.
//
// Sub-chunks of the update (at most kDagSubCols output columns) never split a
// complex pair, so both columns of a pair take their consolidation scale from
// the same norms.
#pragma once

#include "common.cuh"

namespace pevc {

constexpr int kDagSubCols = 32;   // output columns of one update task
constexpr int kTaskTip = 0, kTaskDiag = 1, kTaskUpd = 2;

// Everything the scheduler needs about one pencil: its problem and workspace,
// the ready counters (zeroed before every solve) and the update sub-chunks.
struct DagPencil {
  Problem P;
  int* dcnt;                // [M(M+1)/2] chunks of tile (i, j) solved (tri_index)
  int* utile;               // [M(M+1)/2] updates (source, sub-chunk) applied to tile (k, j)
  int* usub;                // [M(M+1)/2 * nsub_max] sources applied to sub-chunk s of tile (k, j)
  const int* sub_first;     // [M+1] first sub-chunk of column tile j
  const int* sub_c0;        // first output column of each sub-chunk
  const int* sub_nc;        // its column count (<= kDagSubCols)
  int nsub_max;             // most sub-chunks in one column tile
};

// A task: x = pencil | type << 24; y = i (UPD: k); z = j;
// w = chunk (TIP, DIAG: index into the pencil's chunk lists) or
//     i << 8 | s (UPD: source tile row and sub-chunk within column tile j).
__host__ __device__ __forceinline__ int4 dag_task(int pencil, int type, int y, int z, int w) {
  return make_int4(pencil | (type << 24), y, z, w);
}

// Host: sub-chunks of every column tile (widths <= kDagSubCols, never ending
// between the two columns of a pair).  kind: [m] column kinds; cstart: [M+1].
// Writes sub_first[M+1], sub_c0[], sub_nc[] and returns the sub-chunk count
// (or -1 if it would exceed cap); nsub_max receives the most in one tile.
int dag_subchunks(int M, const int* cstart, const signed char* kind, int* sub_first, int* sub_c0, int* sub_nc,
                  int cap, int* nsub_max);

// Host: appends the tasks of stage i of one pencil (i = M: the tips) to out,
// in the walk order: the updates from tile row i, row i - 1 first (the rows
// the next solves wait for), then the solves of row i - 1.  A CTA that takes a
// solve finds its updates done or nearly so, and the solves of one stage
// overlap the last updates of the stage before and the first of the next.
// Returns the new task count or -1 past cap.
int dag_stage_tasks(int pencil, int M, int stage, const int* dchunk_first, const int* sub_first, int4* out,
                    int count, int cap);

// Upper bound of the task count of one pencil with M tiles of order tb.
long long dag_task_bound(int M, int tb);
int dag_nsub_bound(int tb);

// One persistent launch over tasks[0, ntasks) of the pencils pens[] (device
// array).  ticket and abort (device ints) must be zero; grid = CTAs to run.
cudaError_t launch_dag(const DagPencil* pens, const int4* tasks, int ntasks, int* ticket, int* abort_flag,
                       long long wait_cycles, int grid, cudaStream_t s);
int dag_grid(int nsm);    // CTAs of a full wave of k_dag

// Test of the scheduler's bounded wait: one task whose dependence nothing
// satisfies (withhold != 0) or an empty dependence; status gets kStTimeout
// when the wait runs out.
cudaError_t launch_dag_selftest(DagPencil* pen, int4* tasks, int* ticket, int* abort_flag, int withhold,
                                long long cycles, cudaStream_t s);

}  // namespace pevc

// dag.cu -- the device-side scheduler (dag.cuh): one persistent kernel walks
// the task graph of Algorithm 1 (Section 3) for one or several pencils,
// running the diagonal-tile tasks (kernels 1 and 3, diag.cuh) and the FP64
// tensor-core updates (kernel 2 with Algorithms 2 and 3 of Section 4) as they
// become ready.
#include "dag.cuh"
#include "diag_tile.cuh"

namespace pevc {

// ------------------------------------------------------------------ host

int dag_nsub_bound(int tb) {
  // every sub-chunk but the last of a tile has at least kDagSubCols - 1 columns
  return (tb + kDagSubCols - 2) / (kDagSubCols - 1);
}

long long dag_task_bound(int M, int tb) {
  const long long Ml = M;
  const long long tiles = Ml * (Ml + 1) / 2;
  const long long chunks_per_tile = tb / kDiagChunk + 2;     // real columns and pairs chunked apart
  const long long upd = (Ml * Ml * Ml - Ml) / 6 * dag_nsub_bound(tb);   // sum over i of i (M - i)
  return tiles * chunks_per_tile + upd;
}

int dag_subchunks(int M, const int* cstart, const signed char* kind, int* sub_first, int* sub_c0, int* sub_nc,
                  int cap, int* nsub_max) {
  int ns = 0, most = 0;
  for (int j = 0; j < M; ++j) {
    sub_first[j] = ns;
    const int ce = cstart[j + 1];
    for (int c = cstart[j]; c < ce;) {
      int w = ce - c < kDagSubCols ? ce - c : kDagSubCols;
      if (c + w < ce && kind[c + w - 1] == 1) --w;        // the pair's second column is the next sub-chunk's first
      if (ns >= cap) return -1;
      sub_c0[ns] = c;
      sub_nc[ns] = w;
      ++ns;
      c += w;
    }
    most = ns - sub_first[j] > most ? ns - sub_first[j] : most;
  }
  sub_first[M] = ns;
  *nsub_max = most;
  return ns;
}

int dag_stage_tasks(int pencil, int M, int stage, const int* dchunk_first, const int* sub_first, int4* out,
                    int count, int cap) {
  auto push = [&](int4 t) {
    if (count < 0 || count >= cap) {
      count = -1;
      return;
    }
    out[count++] = t;
  };
  if (stage >= M) {                       // the tips: kernel 1 on every diagonal tile
    for (int j = 0; j < M; ++j)
      for (int c = dchunk_first[j]; c < dchunk_first[j + 1]; ++c) push(dag_task(pencil, kTaskTip, j, j, c));
    return count;
  }
  const int i = stage;                    // source tile row of this stage's updates
  if (i < 1) return count;
  auto updates = [&](int k) {
    for (int j = i; j < M; ++j)
      for (int s = 0; s < sub_first[j + 1] - sub_first[j]; ++s) push(dag_task(pencil, kTaskUpd, k, j, i << 8 | s));
  };
  for (int k = i - 1; k >= 0; --k) updates(k);   // row i - 1 first: its solves come next
  for (int j = i; j < M; ++j)             // the solves of row i - 1 (every update into them is then applied)
    for (int c = dchunk_first[j]; c < dchunk_first[j + 1]; ++c) push(dag_task(pencil, kTaskDiag, i - 1, j, c));
  return count;
}

int dag_grid(int nsm) { return 5 * nsm; }   // the kernel's residency: five 128-thread CTAs per SM

// ---------------------------------------------------------------- device

constexpr int kDagUpdK = 16;              // K chunk of the update's shared-memory staging

struct UpdSmem {
  double As[kDagUpdK][kMaxTile + 4];      // [S_ki T_ki] K chunk
  double Bs[kDagUpdK][kDagSubCols + 4];   // X'' K chunk
  double a[kDagSubCols], b[kDagSubCols], beta[kDagSubCols], nrm[kDagSubCols];
  int sY[kDagSubCols], sX[kDagSubCols], e[kDagSubCols], on[kDagSubCols], yz[kDagSubCols], kind[kDagSubCols];
  int any;
};

template <int CB>
union DagSmem {
  DiagSmem<CB> d;
  UpdSmem u;
};

__device__ __forceinline__ void dag_dmma(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

// Kernel 2 on one sub-chunk: Y_kj[:, c0 .. c0+nc) <- 2^sY Y - [S_ki T_ki] 2^sX X''
// with X'' = [X D ; -X B] (Algorithm 2) and per-column consolidation and
// ProtectUpdate (Algorithm 3, update_scales), in FP64 on the tensor cores
// (DMMA m8n8k4).  Four warps, each 32 rows x 32 columns of the output.
__device__ __forceinline__ void upd_task(const Problem& P, int k, int i, int j, int c0, int nc, UpdSmem& sm) {
  const int cs = P.cstart[j];
  const int rk0 = P.toff[k], hk = P.toff[k + 1] - rk0;
  const int ri0 = P.toff[i], hi = P.toff[i + 1] - ri0;
  const int K = 2 * hi;
  const int tb = P.tb;
  double* Yt = tile_ptr(P, k, j);
  const double* Xt = tile_ptr(P, i, j);
  const int tid = threadIdx.x;

  if (tid == 0) sm.any = 0;
  __syncthreads();
  if (tid < kDagSubCols) {
    int on = 0, sY = 0, sX = 0, en = 0;
    bool yz = true;
    if (tid < nc) {
      const int q = c0 + tid;
      on = update_scales(P, P.ex, P.nrm, k, i, q, sY, sX, en, yz) ? 1 : 0;
      const int kd = P.kind[q];
      const int cc = (kd == 2) ? P.ccol[q] - 1 : P.ccol[q];
      sm.kind[tid] = kd;
      sm.a[tid] = P.ca[cc];
      sm.b[tid] = P.cb[cc];
      sm.beta[tid] = P.cbeta[cc];
    }
    sm.on[tid] = on;
    sm.sY[tid] = sY;
    sm.sX[tid] = sX;
    sm.e[tid] = en;
    sm.yz[tid] = yz ? 1 : 0;
    sm.nrm[tid] = 0.0;
    if (on) atomicOr(&sm.any, 1);
  }
  __syncthreads();
  if (!sm.any) return;                    // uniform: nothing of X'' is non-zero

  const int warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t4 = lane & 3;
  double acc[4][4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc[a][b][0] = 0.0; acc[a][b][1] = 0.0; }

  for (int kb = 0; kb < K; kb += kDagUpdK) {
    for (int idx = tid; idx < kDagUpdK * kMaxTile; idx += kMaxTile) {
      const int kk = idx / kMaxTile, row = idx % kMaxTile;
      const int kap = kb + kk;
      double v = 0.0;
      if (row < hk && kap < K) {
        const int gr = rk0 + row, gc = ri0 + (kap < hi ? kap : kap - hi);
        v = (kap < hi) ? P.S[(size_t)gc * P.lds + gr] : P.T[(size_t)gc * P.ldt + gr];
      }
      sm.As[kk][row] = v;
    }
    for (int idx = tid; idx < kDagUpdK * kDagSubCols; idx += kMaxTile) {
      const int kk = idx / kDagSubCols, col = idx % kDagSubCols;
      const int kap = kb + kk;
      double v = 0.0;
      if (col < nc && kap < K && sm.on[col]) {
        const int lq = c0 + col - cs;
        const int sx = sm.sX[col];
        const int kd = sm.kind[col];
        if (kap < hi) {
          v = sm.beta[col] * pow2_scale(Xt[(size_t)lq * tb + kap], sx);
        } else {
          const int kp = kap - hi;
          const double a = sm.a[col], b = sm.b[col];
          if (kd == 0) {
            v = -a * pow2_scale(Xt[(size_t)lq * tb + kp], sx);
          } else if (kd == 1) {
            const double xr = pow2_scale(Xt[(size_t)lq * tb + kp], sx);
            const double xi = pow2_scale(Xt[(size_t)(lq + 1) * tb + kp], sx);
            v = -(a * xr - b * xi);
          } else {
            const double xr = pow2_scale(Xt[(size_t)(lq - 1) * tb + kp], sx);
            const double xi = pow2_scale(Xt[(size_t)lq * tb + kp], sx);
            v = -(b * xr + a * xi);
          }
        }
      }
      sm.Bs[kk][col] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kDagUpdK; kk += 4) {
      double af[4], bf[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) af[a] = sm.As[kk + t4][32 * warp + 8 * a + g];
#pragma unroll
      for (int b = 0; b < 4; ++b) bf[b] = sm.Bs[kk + t4][8 * b + g];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) dag_dmma(acc[a][b][0], acc[a][b][1], af[a], bf[b]);
    }
    __syncthreads();
  }

  // epilogue: Y <- 2^sY Y - acc, column maxima
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int row = 32 * warp + 8 * a + g;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int col = 8 * b + 2 * t4 + e;
        if (row < hk && col < nc && sm.on[col]) {
          const size_t off = (size_t)(c0 + col - cs) * tb + row;
          const double yold = sm.yz[col] ? 0.0 : pow2_scale(Yt[off], sm.sY[col]);
          const double ynew = yold - acc[a][b][e];
          Yt[off] = ynew;
          if (ynew != 0.0) atomic_max_nonneg(&sm.nrm[col], fabs(ynew));
        }
      }
    }
  }
  __syncthreads();
  if (tid < nc && sm.on[tid]) {
    const long long idx = (long long)k * P.m + c0 + tid;
    P.nrm[idx] = sm.nrm[tid];
    P.ex[idx] = sm.e[tid];   // kept even for an all-zero column so a pair's exponents agree
  }
}

// A counter read that bypasses the SM's L1 (another SM wrote it).
__device__ __forceinline__ int dag_load(const int* p) { return *(const volatile int*)p; }

// Thread 0: waits until the task's dependences are met, bounded by `cycles`
// SM clock cycles; false when the wait ran out (the pencil's status word gets
// kStTimeout and every CTA is told to stop) or another CTA gave up.
__device__ bool dag_wait(const DagPencil& D, int4 task, int type, int* abort_flag, long long cycles) {
  const int* c1 = nullptr;
  const int* c2 = nullptr;
  int t1 = 0, t2 = 0;
  const Problem& P = D.P;
  const int j = task.z;
  if (type == kTaskDiag) {
    const int i = task.y;
    c1 = &D.utile[tri_index(i, j)];
    t1 = (j - i) * (D.sub_first[j + 1] - D.sub_first[j]);
  } else if (type == kTaskUpd) {
    const int k = task.y, i = task.w >> 8, s = task.w & 255;
    c1 = &D.dcnt[tri_index(i, j)];
    t1 = P.dchunk_first[j + 1] - P.dchunk_first[j];
    c2 = &D.usub[tri_index(k, j) * D.nsub_max + s];
    t2 = j - i;
  } else if (type != kTaskTip) {           // the self-test's probe: one counter, target 1
    c1 = D.dcnt;
    t1 = 1;
  }
  if (!c1) return dag_load(abort_flag) == 0;
  const long long t0 = clock64();
  for (;;) {
    if (dag_load(c1) >= t1 && (!c2 || dag_load(c2) >= t2)) return true;
    if (dag_load(abort_flag)) return false;
    if (clock64() - t0 > cycles) {
      atomicOr(P.status, kStTimeout);
      atomicExch(abort_flag, 1);
      return false;
    }
    __nanosleep(100);
  }
}

// Thread 0, after the task's writes (all threads, then a barrier): publish
// them and count the task as done.
__device__ __forceinline__ void dag_signal(const DagPencil& D, int4 task, int type) {
  __threadfence();
  if (type == kTaskUpd) {
    const int k = task.y, j = task.z, s = task.w & 255;
    atomicAdd(&D.usub[tri_index(k, j) * D.nsub_max + s], 1);
    atomicAdd(&D.utile[tri_index(k, j)], 1);
  } else if (type == kTaskTip || type == kTaskDiag) {
    atomicAdd(&D.dcnt[tri_index(task.y, task.z)], 1);
  }
}

template <int CB>
__global__ void __launch_bounds__(kMaxTile, 5) k_dag(const DagPencil* __restrict__ pens,
                                                      const int4* __restrict__ tasks, int ntasks, int* ticket,
                                                      int* abort_flag, long long wait_cycles) {
  __shared__ DagSmem<CB> sm;
  __shared__ int s_t, s_ok;
  for (;;) {
    if (threadIdx.x == 0) s_t = dag_load(abort_flag) ? ntasks : atomicAdd(ticket, 1);
    __syncthreads();
    const int t = s_t;
    if (t >= ntasks) break;                // uniform
    const int4 task = tasks[t];
    const int type = task.x >> 24;
    const DagPencil& D = pens[task.x & 0xffffff];
    if (threadIdx.x == 0) {
      s_ok = dag_wait(D, task, type, abort_flag, wait_cycles) ? 1 : 0;
      __threadfence();
    }
    __syncthreads();
    if (!s_ok) break;                      // uniform
    __threadfence();                       // every thread reads what the dependences wrote
    if (type == kTaskUpd) {
      const int sidx = D.sub_first[task.z] + (task.w & 255);
      upd_task(D.P, task.y, task.w >> 8, task.z, D.sub_c0[sidx], D.sub_nc[sidx], sm.u);
    } else if (type == kTaskTip || type == kTaskDiag) {
      const int i = task.y, j = task.z, chunk = task.w;
      const bool pf = type == kTaskDiag && j == i + 1 && chunk == D.P.dchunk_first[j];
      diag_tile<CB>(D.P, i, j, chunk, type == kTaskTip ? kDiagTip : kDiagSolve, (t + (int)blockIdx.x) & 3, pf,
                    sm.d);
    }
    __syncthreads();
    if (threadIdx.x == 0) dag_signal(D, task, type);
  }
}

cudaError_t launch_dag(const DagPencil* pens, const int4* tasks, int ntasks, int* ticket, int* abort_flag,
                       long long wait_cycles, int grid, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  if (grid > ntasks) grid = ntasks;
  k_dag<kDiagChunk><<<grid, kMaxTile, 0, s>>>(pens, tasks, ntasks, ticket, abort_flag, wait_cycles);
  return cudaGetLastError();
}

// The bounded wait of the scheduler, exercised without a fault: one probe
// task whose counter (pen->dcnt[0]) is set to its target by a one-thread
// kernel before the walk, or left at zero (withhold) so that the wait runs
// out after `cycles` SM clock cycles.
__global__ void k_dag_probe_setup(DagPencil* pen, int4* tasks, int* ticket, int* abort_flag, int withhold) {
  *ticket = 0;
  *abort_flag = 0;
  pen->dcnt[0] = withhold ? 0 : 1;
  tasks[0] = dag_task(0, 3, 0, 0, 0);
}

cudaError_t launch_dag_selftest(DagPencil* pen, int4* tasks, int* ticket, int* abort_flag, int withhold,
                                long long cycles, cudaStream_t s) {
  k_dag_probe_setup<<<1, 1, 0, s>>>(pen, tasks, ticket, abort_flag, withhold);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_dag(pen, tasks, 1, ticket, abort_flag, cycles, 1, s);
}

}  // namespace pevc

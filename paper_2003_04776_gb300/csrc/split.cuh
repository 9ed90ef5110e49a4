// split.cuh -- split-precision update path (Ozaki-style slices, Section 3's
// kernel 2 on BF16 / FP8 tensor cores) and the FP64 residual correction.
#pragma once

#include "common.cuh"

namespace pevc {

struct SplitWorkspace {
  bool on = false;
};

int split_alloc(SplitWorkspace& w, int n_max, int tb, int Mmax, int prec);
void split_free(SplitWorkspace& w);
int split_solve(SplitWorkspace& w, const Problem& P, int prec, bool correct, cudaStream_t s,
                cudaEvent_t ev_dag, cudaEvent_t ev_corr, int* nupd, int* ndiag);

}  // namespace pevc

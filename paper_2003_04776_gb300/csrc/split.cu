#include "split.cuh"

namespace pevc {

int split_alloc(SplitWorkspace& w, int, int, int, int) { w.on = false; return PEVC_ERR_UNSUPPORTED; }
void split_free(SplitWorkspace& w) { w.on = false; }
int split_solve(SplitWorkspace&, const Problem&, int, bool, cudaStream_t, cudaEvent_t, cudaEvent_t,
                int*, int*) {
  return PEVC_ERR_UNSUPPORTED;
}

}  // namespace pevc

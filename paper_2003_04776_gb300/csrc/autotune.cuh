// autotune.cuh -- the plan-time autotuner (autotune.cu).
#pragma once

#include <array>
#include <vector>

#include "common.cuh"

namespace pevc {

// Times one solve of every candidate setting on a synthetic pencil and returns
// the fastest: the tile order (when tile is 0; else the given one; split
// plans try only 128), the precision (split plans: BF16x5 or BF16x3 with the
// correction sweep; FP64 plans keep FP64) and the walk flag (split plans: 0;
// FP64: PEVC_DEVICE_WALK or PEVC_STAGE_WALK).  log receives
// {tile, prec, stage walk, ms} per candidate.  Cached per device, order,
// precision family, tile and flags for the life of the process.  Returns 0 or
// a PEVC_ERR_* code.
int autotune_pick(int n_max, int prec, int tile, unsigned flags, void* stream, int* tile_out, int* prec_out,
                  unsigned* walk_out, std::vector<std::array<double, 4>>* log);

}  // namespace pevc

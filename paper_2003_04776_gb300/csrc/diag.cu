// diag.cu -- diagonal-tile kernel launched once per stage: kernel 1 (tips)
// and kernel 3 (the small solves S_ii Z D - T_ii Z B = Y_ij) of Section 3,
// one CTA per (tile, column chunk), each running diag_tile (diag_tile.cuh).
#include "diag_tile.cuh"

namespace pevc {

template <int CB>
__global__ void __launch_bounds__(kMaxTile, 6) k_diag(Problem P, int i_row, int mode) {
  __shared__ DiagSmem<CB> sm;
  const bool tips = mode != kDiagSolve;          // one CTA row per diagonal tile from i_row
  const int j = tips ? i_row + (int)blockIdx.y : i_row + 1 + (int)blockIdx.y;
  const int i = tips ? j : i_row;
  const int chunk = P.dchunk_first[j] + (int)blockIdx.x;
  if (chunk >= P.dchunk_first[j + 1]) return;
  // pa_warp spreads the block solves over the sub-partitions; one CTA per
  // launch prefetches the diagonal tile's columns
  diag_tile<CB>(P, i, j, chunk, mode, (int)(blockIdx.x + blockIdx.y) & 3, blockIdx.x == 0 && blockIdx.y == 0, sm);
}

cudaError_t launch_diag(const Problem& P, int i, int mode, cudaStream_t s) {
  const int ntiles = (mode != kDiagSolve) ? P.M : (P.M - 1 - i);
  if (ntiles <= 0 || P.dchunk_max <= 0) return cudaSuccess;
  dim3 grid(P.dchunk_max, ntiles);
  k_diag<kDiagChunk><<<grid, kMaxTile, 0, s>>>(P, mode != kDiagSolve ? 0 : i, mode);
  return cudaGetLastError();
}

cudaError_t launch_diag_tile(const Problem& P, int j, int mode, cudaStream_t s) {
  if (P.dchunk_max <= 0) return cudaSuccess;
  dim3 grid(P.dchunk_max, 1);
  k_diag<kDiagChunk><<<grid, kMaxTile, 0, s>>>(P, j, mode);
  return cudaGetLastError();
}

}  // namespace pevc

// left.cu -- left eigenvectors through the right-eigenvector solve.
//
// A left eigenvector u of the real Schur pencil (S, T), u^H (beta S - alpha T)
// = 0, satisfies (beta S^T - conj(alpha) T^T) u = 0.  With J the reversal
// permutation, (S', T') = (J S^T J, J T^T J) is again a standardised real Schur
// pencil (its 1x1 and 2x2 blocks are those of (S, T) in reverse order, T' is
// diagonal inside the 2x2 blocks), and J u is its right eigenvector for
// conj(alpha).  The solve of (S', T') returns, for a complex pair, the vector z'
// for the eigenvalue with positive imaginary part, so u = J conj(z'): rows in
// reverse order, the imaginary column negated, and the columns back in the
// order of S's diagonal.  These kernels do the two permutations.
#include "common.cuh"

namespace pevc {

// B(i, j) = A(n-1-j, n-1-i) for i, j < n (B column-major with leading
// dimension n): 32 x 32 tiles through shared memory, coalesced on both sides.
__global__ void __launch_bounds__(256) k_flip_transpose(const double* __restrict__ A, int lda, int n,
                                                        double* __restrict__ B) {
  __shared__ double tile[32][33];
  const int bi = blockIdx.x, bj = blockIdx.y, tx = threadIdx.x, ty = threadIdx.y;
  const int rbase = n - 32 * bj - 32;   // rows of A feeding B's columns 32 bj .. 32 bj + 31
  const int cbase = n - 32 * bi - 32;   // columns of A feeding B's rows 32 bi .. 32 bi + 31
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = rbase + tx, c = cbase + ty + 8 * k;
    if (r >= 0 && c >= 0) tile[ty + 8 * k][tx] = A[(size_t)c * lda + r];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = 32 * bi + tx, j = 32 * bj + ty + 8 * k;
    if (i < n && j < n) B[(size_t)j * n + i] = tile[31 - tx][31 - ty - 8 * k];
  }
}

__global__ void k_flip_select(const int32_t* __restrict__ sel, int n, int32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = sel[n - 1 - i];
}

// Column q of the flipped solve's output goes to column m-1-q (a real
// eigenvector), m-2-q (the real part of a pair) or m-q (its imaginary part,
// negated), with its rows reversed.
__global__ void __launch_bounds__(256) k_left_out(const double* __restrict__ Vp, int n, int m,
                                                  const signed char* __restrict__ kind,
                                                  const int32_t* __restrict__ scp, double* __restrict__ U, int ldu,
                                                  int32_t* __restrict__ scale) {
  const int q = blockIdx.x;
  const int kd = kind[q];
  const int oc = kd == 0 ? m - 1 - q : (kd == 1 ? m - 2 - q : m - q);
  const long long flip = kd == 2 ? (long long)0x8000000000000000ull : 0ll;   // sign bit
  const double* v = Vp + (size_t)q * n;
  double* u = U + (size_t)oc * ldu;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    u[i] = __longlong_as_double(__double_as_longlong(v[n - 1 - i]) ^ flip);
  if (threadIdx.x == 0) scale[oc] = scp[q];
}

cudaError_t launch_flip_transpose(const double* A, int lda, int n, double* B, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
  k_flip_transpose<<<grid, block, 0, s>>>(A, lda, n, B);
  return cudaGetLastError();
}

cudaError_t launch_flip_select(const int32_t* sel, int n, int32_t* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_flip_select<<<(n + 255) / 256, 256, 0, s>>>(sel, n, out);
  return cudaGetLastError();
}

cudaError_t launch_left_out(const double* Vp, int n, int m, const signed char* kind, const int32_t* scp, double* U,
                            int ldu, int32_t* scale, cudaStream_t s) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  k_left_out<<<m, 256, 0, s>>>(Vp, n, m, kind, scp, U, ldu, scale);
  return cudaGetLastError();
}

}  // namespace pevc

// cplx.cuh -- host interface of the complex-pencil solve (cplx.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pevc {

// Workspace owned by a plan, allocated by the first complex solve for orders
// up to n_max; the caller's output V is the working array.
struct CplxWork;
void cplx_free(CplxWork* w);
int cplx_solve(CplxWork** w, int n_max, cudaStream_t s, const double* S, int lds, const double* T, int ldt, int n,
               const int32_t* select, double* V, int ldv, int32_t* scale, int* m_out, bool normalise);
// Left eigenvectors through the flipped conjugate-transposed pencil.
int cplx_solve_left(CplxWork** w, int n_max, cudaStream_t s, const double* S, int lds, const double* T, int ldt,
                    int n, const int32_t* select, double* U, int ldu, int32_t* scale, int* m_out, bool normalise);

// Back-transformation of complex eigenvectors (backtransform.cu).
int bt_zgemm(void* h, int n, int m, const double* Z, int ldz, const double* V, int ldv, double* X, int ldx);
cudaError_t launch_bt_normalise_c(double* X, int ldx, int n, int m, cudaStream_t s);

}  // namespace pevc

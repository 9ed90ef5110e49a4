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

}  // namespace pevc

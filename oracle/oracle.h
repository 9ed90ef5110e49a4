/*
 * oracle.h -- declarations of the plain FP64 CPU oracle (test infrastructure
 * only; the CUDA library neither includes nor links this file).
 *
 * Matrices are column-major binary64.  Status values: 0 success, -i for an
 * invalid i-th argument, positive values for the conditions below.
 */
#ifndef PEVC_ORACLE_H
#define PEVC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_ERR_NOT_SCHUR 1    /* 2x2 block with real eigenvalues, or T_jj not diagonal/positive */
#define ORC_ERR_NONFINITE 2    /* Inf or NaN in the parts of S, T that are read */
#define ORC_ERR_INDEFINITE 3   /* alpha = beta = 0 for a selected 1x1 block */
#define ORC_ERR_NOMEM 6

#define ORC_FLAG_NO_NORMALISE 1   /* return 2^e-scaled vectors and e instead of normalised ones */
#define ORC_FLAG_PLAIN 2          /* no scaling, no smin: the non-robust substitution */

int orc_protect_upd(double y, double t, double x);
int orc_protect_div(double b, double t);
void orc_cdiv(double ar, double ai, double br, double bi, double *qr, double *qi);
int orc_blocks(int n, const double *S, int lds, const double *T, int ldt, signed char *blk);
int orc_eigpairs(int n, const double *S, int lds, const double *T, int ldt,
                 const signed char *blk, double *a, double *b, double *beta, int *sigma);
int orc_evc(int n, const double *S, int lds, const double *T, int ldt, const int *select,
            int flags, double *V, int ldv, int32_t *scale, int *m_out, int nthreads);
/* Complex pencils: S, T, V interleaved (re, im) complex128, leading
 * dimensions in complex elements; alpha, beta interleaved complex[n]. */
int orc_eigpairs_cplx(int n, const double *S, int lds, const double *T, int ldt,
                      double *alpha, double *beta, int *sigma);
int orc_evc_cplx(int n, const double *S, int lds, const double *T, int ldt, const int *select,
                 int flags, double *V, int ldv, int32_t *scale, int *m_out, int nthreads);
int orc_version(void);

#ifdef __cplusplus
}
#endif
#endif

/*
 * pevc.h -- C ABI of the GB300 library for robust generalized eigenvectors
 * of a real pencil (S, T) in generalized real Schur form.
 *
 * Method: Kjelgaard Mikkelsen & Myllykoski, "Parallel Robust Computation of
 * Generalized Eigenvectors of Matrix Pencils" (PPAM 2019).  The library solves
 * the homogeneous matrix equation S V D - T V B = 0 (Section 2.2) for all or
 * selected eigenvectors with the blocked algorithm of Section 3 (Algorithm 1),
 * made robust against overflow with augmented tiles -- a tile plus one
 * power-of-two scale per eigenvector column -- and scale consolidation before
 * every update (Section 4, Algorithms 2 and 3).
 *
 * Conventions shared by every entry point
 *   - Matrices are binary64, column-major, with a leading dimension ld >= n.
 *   - S is upper quasi-triangular with 1x1 and 2x2 diagonal blocks (a 2x2
 *     block starts at row i when S[i+1,i] != 0); T is upper triangular and
 *     each 2x2 diagonal block of T is diagonal with positive entries (the
 *     standardised real Schur form of Section 2).  Entries strictly below the
 *     first subdiagonal of S and below the diagonal of T are never read.
 *   - Eigenvalues follow Section 2: (alpha, beta), alpha = a + i b, beta >= 0;
 *     a 1x1 block gives (S_cc, T_cc), a 2x2 block gives beta = 1 and the root
 *     a + i b, b > 0, of det(S_jj - lambda T_jj) = 0.  beta = 0 is an infinite
 *     eigenvalue; alpha = beta = 0 is the indefinite case (an error when
 *     selected).
 *   - Output columns: a real eigenvalue gives one column, a complex pair two
 *     consecutive columns (Re z, Im z) of the eigenvector z of a + i b with
 *     b > 0 (the Lemma of Section 2.1).  Without a selection column c belongs
 *     to diagonal position c and V is upper quasi-triangular; with a selection
 *     the selected eigenvectors are packed in diagonal order.  Selecting
 *     either row of a 2x2 block selects the pair (Section 5: the subset is
 *     closed under complex conjugation).  Rows below an eigenvector's block
 *     are written as zero.
 *   - Normalisation (default): every vector is divided by its entry of
 *     largest modulus (first index on ties), so that entry is exactly 1.
 *     scale_out[c] is then the binary exponent of that entry's magnitude
 *     relative to a tip of unit largest modulus, i.e. log2 of the growth.
 *     With PEVC_NO_NORMALISE the columns are returned consolidated to one
 *     power of two per column: the eigenvector is 2^scale_out[c] * V[:,c]
 *     (the augmented representation of Section 4 with alpha = 2^-scale).
 *   - Status: 0 success; -i means argument i is invalid (LAPACK INFO style,
 *     counting the plan as argument 1); positive values are the PEVC_ERR_*
 *     codes below.  On error V_out is unspecified.  No entry point aborts or
 *     traps; device-side conditions are reported through the status.
 */
#ifndef PEVC_H
#define PEVC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pevc_plan_s *pevc_plan_t;

/* Arithmetic of the bulk updates (kernel 2 of Section 3). */
#define PEVC_FP64 0          /* FP64 tensor-core updates (DMMA)                      */
#define PEVC_SPLIT_BF16X3 1  /* BF16 x3 slice products + FP64 residual correction   */
#define PEVC_SPLIT_FP8X4 2   /* FP8 E4M3 x4 slice products + residual corrections   */
#define PEVC_SPLIT_BF16X5 3  /* BF16 x5 slice products in one pass (no correction)   */

/* Plan / solve flags. */
#define PEVC_NO_NORMALISE 1u   /* return consolidated columns and exponents      */
#define PEVC_NO_CORRECTION 2u  /* split precisions: skip the correction sweeps   */
#define PEVC_BT_EMULATED 4u    /* pevc_backtransform: FP64 GEMM by fixed-point emulation */
#define PEVC_STAGE_WALK 8u     /* FP64 plans: walk the task graph stage by stage from the host
                                  instead of the device-side scheduler                    */
#define PEVC_AUTOTUNE 16u      /* pevc_plan: choose the settings by timing (see pevc_plan) */
#define PEVC_DEVICE_WALK 32u   /* FP64 plans: the device-side scheduler whatever the order   */
#define PEVC_BT_CUBLAS 64u     /* pevc_backtransform: cuBLAS FP64 GEMM instead of the library's
                                  split GEMM                                               */

/* Status codes. */
#define PEVC_SUCCESS 0
#define PEVC_ERR_NOT_SCHUR 1    /* 2x2 block with real eigenvalues, adjacent 2x2 blocks,
                                   or a 2x2 block of T that is not diagonal and positive */
#define PEVC_ERR_NONFINITE 2    /* Inf or NaN among the entries of S or T that are read */
#define PEVC_ERR_INDEFINITE 3   /* alpha = beta = 0 for a selected eigenvalue (Section 2) */
#define PEVC_ERR_TIMEOUT 4      /* a bounded device wait ran out                         */
#define PEVC_ERR_CUDA 5         /* a CUDA runtime call failed                            */
#define PEVC_ERR_NOMEM 6        /* device or pinned host allocation failed               */
#define PEVC_ERR_UNSUPPORTED 7  /* a requested feature is not available in this build    */
#define PEVC_ERR_TOO_LARGE 8    /* n above PEVC_STATIC_N_MAX in pevc_solve_static         */

/* Largest order accepted by pevc_solve_static. */
#define PEVC_STATIC_N_MAX 512

/*
 * pevc_plan -- create a plan that owns all device workspace for pencils of
 * order up to n_max (and batches of up to batch_max pencils).
 *   plan       out: the new plan (NULL on failure)
 *   n_max      largest order a solve will use, >= 0
 *   batch_max  largest batch count for pevc_solve_batched, >= 1
 *   prec       PEVC_FP64, PEVC_SPLIT_BF16X3, PEVC_SPLIT_FP8X4 or PEVC_SPLIT_BF16X5
 *   tile       tile order (Section 5.1: tiles of S, T and V are conformal; a
 *              tile boundary never splits a 2x2 block); 0 lets the library
 *              choose (from n_max and prec, or by timing with PEVC_AUTOTUNE);
 *              otherwise 32, 64, 96 or 128
 *   flags      PEVC_NO_NORMALISE | PEVC_NO_CORRECTION | PEVC_STAGE_WALK |
 *              PEVC_DEVICE_WALK | PEVC_AUTOTUNE.  FP64 plans walk the task
 *              graph with the device-side scheduler (one persistent launch,
 *              Section 3 and Section 5.3) for batches, stage by stage from the
 *              host for single pencils; the walk flags force one (not both).  Split plans use the stage walk (their tcgen05
 *              update needs a whole SM per CTA).  With PEVC_AUTOTUNE the plan
 *              times one solve of
 *              each candidate setting on a synthetic pencil of order n_max
 *              (made on the device: 2x2 blocks on two thirds of the diagonal,
 *              uniform off-diagonal entries) and keeps the fastest: for the
 *              split precisions the split depth (BF16x5 in one pass, or
 *              BF16x3 or FP8x4 plus the correction sweep), whichever of the
 *              three prec names, at tile order 128 (or the given one); for FP64 the tile
 *              order among 64, 96 and 128 (32 too up to order 512) when tile
 *              is 0, and the walk; FP64 plans time orders above 8192 on a
 *              pencil of order 8192.  The
 *              winner is cached per device, order and precision family for
 *              later plans of this process; pevc_plan_info reports it and
 *              pevc_autotune_log the times.  The timing needs about 2 n_max^2
 *              doubles more of device memory while the plan is made.
 *   stream     cudaStream_t (as void*) on which every solve is ordered; NULL
 *              is the legacy default stream
 * The plan allocates with cudaMalloc; pevc_solve itself allocates nothing.
 * Returns 0, -i, PEVC_ERR_NOMEM or PEVC_ERR_CUDA.
 */
int pevc_plan(pevc_plan_t *plan, int n_max, int batch_max, int prec, int tile,
              unsigned flags, void *stream);

/*
 * pevc_solve -- all (select == NULL) or the selected eigenvectors of (S, T).
 *   plan       a plan with n <= n_max
 *   S, lds     device, n x n, read only (never modified; pre-scaling is done
 *              on the eigenvalue pairs, which leaves the eigenvectors fixed)
 *   T, ldt     device, n x n, read only
 *   n          order, 0 <= n <= n_max
 *   select     device int32[n] or NULL; nonzero selects an eigenvalue
 *   V_out, ldv device, n x m_out, written (caller-owned; n x n suffices)
 *   scale_out  device int32[m_out], written
 *   m_out      host: number of columns written
 * Stream-ordered on the plan's stream; the call reads the block structure
 * back to the host once and synchronises on return (m_out and the status are
 * final when it returns); PEVC_SPLIT_FP8X4 plans also wait after each
 * correction sweep, to read how much it changed the eigenvectors.
 * Deterministic: equal inputs give bitwise-equal outputs.
 */
int pevc_solve(pevc_plan_t plan, const double *S, int lds, const double *T, int ldt, int n,
               const int32_t *select, double *V_out, int ldv, int32_t *scale_out, int *m_out);

/*
 * pevc_solve_host -- pevc_solve on HOST memory: S, T (read), select (may be
 * NULL), V_out and scale_out (written) are host arrays, with the leading
 * dimensions and codes of pevc_solve.  The method reads only the tiles on and
 * above the block diagonal of S and T (Section 3: the tiles (k, l), k <= l),
 * and its bottom-up walk needs column block l of S and T only from stage l
 * on; so the call copies, for every column block l from the last to the
 * first, rows 0 .. (last row of block l) of its columns, on a copy stream of
 * the plan's own, and stage l waits for block l alone: the copies overlap the
 * solve, and the lower triangles are never copied.  The eigenvalues' pre-
 * scaling (Section 4) takes the maximum of the blocks seen so far; if the
 * final maximum would change a pre-scale (only for entries near 2^1000), the
 * solve is run again on the copied data.  The first call allocates the
 * device copies of S, T and V (3 n_max^2 doubles) and the copy stream; pinned
 * host arrays give the fastest copies.  Ordered after the work on the plan's
 * stream; synchronises on return.  Returns pevc_solve's codes.
 */
int pevc_solve_host(pevc_plan_t plan, const double *S, int lds, const double *T, int ldt, int n,
                    const int32_t *select, double *V_out, int ldv, int32_t *scale_out, int *m_out);

/*
 * pevc_last_host_bytes -- bytes the last pevc_solve_host call copied:
 *   out  host long long[2]: {host to device, device to host}
 * Returns 0, -1 (plan NULL) or -2 (out NULL).
 */
int pevc_last_host_bytes(pevc_plan_t plan, long long *out);

/*
 * pevc_solve_batched -- count independent pencils of (possibly) different
 * orders, each as in pevc_solve.  Pointer arguments are host arrays of
 * length count holding device pointers (select[i] may be NULL, select itself
 * may be NULL for "all"); lds, ldt, n, ldv are host int arrays.  m_out and
 * status are host int arrays of length count: status[i] is pencil i's own
 * status, so one bad pencil does not stop the others.  Every n[i] must be
 * <= n_max and count <= batch_max.  Returns 0 when the arguments are valid
 * and every pencil was processed (check status[]), else -i or a PEVC_ERR_*.
 * A plan made with batch_max > 1 owns up to 8 child workspaces with their own
 * streams (as many as about 4 GB allows) and runs that many pencils at once;
 * the batch is ordered after the work already on the plan's stream and the
 * call synchronises on return.
 */
int pevc_solve_batched(pevc_plan_t plan, int count,
                       const double *const *S, const int *lds,
                       const double *const *T, const int *ldt, const int *n,
                       const int32_t *const *select, double *const *V_out, const int *ldv,
                       int32_t *const *scale_out, int *m_out, int *status);

/* pevc_destroy -- free a plan and its workspace (NULL is accepted). */
int pevc_destroy(pevc_plan_t plan);

/* pevc_strerror -- static text for a status value. */
const char *pevc_strerror(int code);

/*
 * pevc_plan_info -- the plan's resolved settings (after autotuning).
 *   info  host int[8]: {tile, prec, n_max, batch_max, flags, device SM count,
 *                       slices per operand (0 for FP64), correction sweeps
 *                       (the most: FP8x4 repeats them until they converge)}
 */
int pevc_plan_info(pevc_plan_t plan, int *info);

/*
 * pevc_autotune_log -- the candidates a PEVC_AUTOTUNE plan timed (or whose
 * times it took from the process's cache), in the order they were tried.
 *   out   host double[4 * cap]: per candidate {tile, prec, stage walk (0/1),
 *         milliseconds of one solve of the synthetic pencil}
 * Returns the number of candidates (at most cap are written; 0 for a plan
 * made without PEVC_AUTOTUNE), or -1 for a NULL plan, -2 for a NULL out.
 */
int pevc_autotune_log(pevc_plan_t plan, double *out, int cap);

/*
 * pevc_last_stats -- host double[8] timing/work figures of the last solve on
 * this plan: {total ms (device, CUDA events), prepass ms, first-pass ms,
 * correction ms, postpass ms, tiles M, kernel launches, and for FP64 plans
 * the scheduler (1: the task graph walked on the device by one persistent
 * launch, 0: stage by stage from the host), for split plans the correction
 * sweeps the solve ran}.
 */
int pevc_last_stats(pevc_plan_t plan, double *stats);

/*
 * pevc_set_profile -- on != 0 records a CUDA event pair around every kernel
 * launch of later solves on the plan's stream (a few microseconds per
 * launch); 0 switches it off (the default).
 */
int pevc_set_profile(pevc_plan_t plan, int on);

/*
 * pevc_kernel_profile -- per-kernel-kind totals of the last profiled solve.
 *   out  host double[12]: for kind = update, diagonal solve, slicing, other:
 *        {milliseconds, launches, tensor-core flops} at out[3*kind .. 3*kind+2]
 *        (flops count every slice product: 2 * rows * cols * K * products).
 */
int pevc_kernel_profile(pevc_plan_t plan, double *out);

/*
 * pevc_solve_static -- pevc_solve in FP64 for pencils of order n <=
 * PEVC_STATIC_N_MAX without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- code that runs where a device allocation could block or fail
 * at a bad moment (inside a real-time or latency-bounded loop, under a
 * caller's own memory pool or allocation budget, or in a plugin whose host
 * forbids allocating) -- and that cannot keep a plan alive.
 *   S, lds, T, ldt, n, select, V_out, ldv, scale_out, m_out
 *              as in pevc_solve (device pointers owned by the caller; m_out
 *              is host memory)
 *   flags      0 or PEVC_NO_NORMALISE
 *   stream     cudaStream_t (as void*) on which the work is ordered
 * Workspace: one file-scope device array of just under 2 MiB (the
 * workspace of an order-512 FP64 solve), which every GPU that loads the
 * library holds until the process exits; host-side structure arrays (about
 * 16 KB) live on the calling thread's stack.  The call allocates nothing:
 * no cudaMalloc, cudaFree, cudaMallocHost or allocating library routine; its
 * host copies go through pageable memory.
 * Set-up: the first call on a device, with that device current, looks up the
 * array's device address (cudaGetSymbolAddress) once; make that first call
 * before any stream capture on the device (a call with n = 0 does only the
 * set-up).
 * Sharing: every call on a device uses the same array, which keeps the last
 * call's contents (the call clears what must start at zero itself).  Calls
 * whose GPU work overlaps -- on different streams, or from different host
 * threads -- race on the array and give wrong results; order them on one
 * stream or serialise them.  The call synchronises on return, like
 * pevc_solve, and its kernels and tile order are those of an FP64 plan with
 * n_max = n, so its output equals that plan's.
 * Returns 0, -i (argument i invalid, counting S as argument 1),
 * PEVC_ERR_TOO_LARGE when n > PEVC_STATIC_N_MAX, or a status of pevc_solve.
 */
int pevc_solve_static(const double *S, int lds, const double *T, int ldt, int n,
                      const int32_t *select, double *V_out, int ldv, int32_t *scale_out, int *m_out,
                      unsigned flags, void *stream);

/*
 * pevc_backtransform -- eigenvectors of the original pencil (Section 1).
 * With (A, B) = (Q S Z^T, Q T Z^T) the pencil before its reduction to the
 * real Schur pencil (S, T), a right eigenvector v of (S, T) gives the right
 * eigenvector x = Z v of (A, B) for the same eigenvalue.  Computes X = Z V for
 * the m columns of V as pevc_solve writes them, on the plan's stream, as
 * exact BF16 slice products on the tensor cores: every row of Z and every
 * column of V is split, per chunk of 256 along the inner dimension and
 * relative to its own power-of-two bound in that chunk, into six 8-bit
 * slices; the chunk's products sum exactly in FP32 per slice level and the
 * chunks' values are summed in FP64, so each entry of X carries an error of
 * at most about 2^-46 of sum over chunks of (the chunk's largest |Z_rk|) times
 * sum |V_kc| plus (the chunk's largest |V_kc|) times sum |Z_rk| (chunks of V below a column's last
 * non-zero row are skipped: V from a solve is quasi-triangular).  With
 * PEVC_BT_CUBLAS or PEVC_BT_EMULATED it is cuBLAS's FP64 GEMM instead.  Then,
 * unless PEVC_NO_NORMALISE, the call scales every eigenvector
 * (a real column, or the real and imaginary columns of a complex pair taken
 * as one complex vector) so that its entry of largest modulus is exactly 1
 * (the first such entry on ties; an all-zero vector stays zero).
 *   plan       a plan with n <= n_max
 *   Z, ldz     device, column-major n x n, ldz >= n; read-only
 *   n          order of the pencil
 *   V, ldv     device, column-major n x m, ldv >= n; read-only
 *   m          number of columns of V (0 <= m <= n)
 *   kinds      host int[m]: 0 a real eigenvector's column, 1 and 2 the real
 *              and imaginary columns of a complex pair (a 1 is always
 *              followed by a 2); or NULL for the columns of the plan's last
 *              pevc_solve (m must then equal that solve's column count)
 *   X, ldx     device, column-major n x m, ldx >= n, caller-allocated; must
 *              not overlap Z or V
 *   flags      PEVC_NO_NORMALISE | PEVC_BT_CUBLAS | PEVC_BT_EMULATED (cuBLAS's
 *              fixed-point emulation of the FP64 GEMM on the tensor cores)
 * The first call allocates the split GEMM's workspace (about 24 n_max^2
 * bytes) or, with the cuBLAS flags, the plan's cuBLAS handle, and, with kinds
 * given, a device copy of them (n_max bytes); the call synchronises the
 * plan's stream before returning.
 * Returns 0, -i (argument i invalid, counting the plan as argument 1),
 * PEVC_ERR_UNSUPPORTED (emulation not available), PEVC_ERR_NOMEM or
 * PEVC_ERR_CUDA (a CUDA or cuBLAS call failed).
 */
int pevc_backtransform(pevc_plan_t plan, const double *Z, int ldz, int n, const double *V, int ldv, int m,
                       const int *kinds, double *X, int ldx, unsigned flags);

/*
 * pevc_solve_left -- left eigenvectors of the real Schur pencil (S, T): for
 * every selected eigenvalue alpha / beta, u != 0 with u^H (beta S - alpha T) = 0
 * (the paper names left eigenvectors as future work, Section 7).  u is the
 * right eigenvector, for conj(alpha), of (S^T, T^T); with J the reversal
 * permutation, (J S^T J, J T^T J) is again a standardised real Schur pencil, so
 * the call forms it, runs pevc_solve's robust solve on it, and reverses the
 * rows back.
 *   S, lds, T, ldt, n, select, scale_out, m_out
 *              as in pevc_solve (select marks diagonal positions of S)
 *   U_out, ldu device, column-major n x m, caller-allocated: the columns in
 *              the order of S's diagonal, a complex pair as (Re u, Im u) for
 *              the eigenvalue with positive imaginary part; u is zero above
 *              its diagonal block, and normalised like pevc_solve's columns
 *              (entry of largest modulus exactly 1) unless the plan was made
 *              with PEVC_NO_NORMALISE, in which case scale_out[c] = e means
 *              the represented vector is 2^e U_out[:, c]
 * Workspace: the first call allocates three n_max x n_max FP64 arrays and two
 * int32[n_max] arrays on the plan (the flipped pencil and its solve); later
 * calls allocate nothing.  The call synchronises on return.
 * Returns 0, -i (argument i invalid, counting the plan as argument 1), or a
 * status of pevc_solve (which then refers to the same blocks of S and T).
 */
int pevc_solve_left(pevc_plan_t plan, const double *S, int lds, const double *T, int ldt, int n,
                    const int32_t *select, double *U_out, int ldu, int32_t *scale_out, int *m_out);

/*
 * pevc_solve_cplx -- eigenvectors of a complex pencil in generalized
 * (complex) Schur form, the extension to complex data types that the paper
 * names in Section 7.  S and T are upper triangular with complex entries;
 * diagonal entry c gives the eigenvalue (alpha_c, beta_c) = (S_cc, T_cc) and
 * the eigenvector x with x_c = 1 before normalisation, x_i = 0 for i > c and
 * (beta_c S - alpha_c T) x = 0.  The robust blocked substitution of
 * pevc_solve runs with complex arithmetic and no 2x2 blocks (tiles of order
 * 64, FP64 throughout, whatever the plan's precision).
 *   S, lds     device, n x n complex128 (interleaved re, im; cuDoubleComplex
 *              layout), column-major, lds >= n counted in complex elements,
 *              16-byte aligned; entries below the diagonal are never read
 *   T, ldt     the same for T
 *   n          order, 0 <= n <= the plan's n_max
 *   select     device int32[n] or NULL; nonzero selects diagonal entry c
 *   V_out, ldv device, n x m complex128, column-major, caller-allocated and
 *              16-byte aligned: one column per selected entry, in diagonal
 *              order; zero below the tip; normalised like pevc_solve's
 *              columns (entry of largest modulus exactly 1 + 0i) unless the
 *              plan was made with PEVC_NO_NORMALISE (then the eigenvector is
 *              2^scale_out[c] V_out[:, c])
 *   scale_out  device int32[m], written
 *   m_out      host: number of columns written
 * Workspace: the first call allocates about 12 n_max (n_max / 64 + 3) bytes
 * of device memory on the plan (a power-of-two exponent and a magnitude per
 * tile segment of every column); V_out itself is the working array.  The call reads the
 * selection back to the host, synchronises once after the input scan and
 * again on return.
 * Returns 0, -i (argument i invalid, counting the plan as argument 1; a
 * misaligned S, T or V_out counts as invalid), PEVC_ERR_NONFINITE,
 * PEVC_ERR_INDEFINITE (S_cc = T_cc = 0 for a selected c), PEVC_ERR_NOMEM or
 * PEVC_ERR_CUDA.
 */
int pevc_solve_cplx(pevc_plan_t plan, const double *S, int lds, const double *T, int ldt, int n,
                    const int32_t *select, double *V_out, int ldv, int32_t *scale_out, int *m_out);

/*
 * pevc_solve_cplx_left -- left eigenvectors of a complex triangular pencil:
 * for every selected diagonal entry c, u != 0 with u^H (beta_c S - alpha_c T)
 * = 0 (left eigenvectors and complex data are both future work in Section 7).
 * With J the reversal permutation, J (beta S - alpha T)^H J = conj(beta) S' -
 * conj(alpha) T' for (S', T') = (J S^H J, J T^H J), again upper triangular, so
 * J u is pevc_solve_cplx's eigenvector of (S', T') at entry n-1-c: the call
 * forms (S', T') in plan workspace, solves, and reverses rows and columns.
 *   arguments  as in pevc_solve_cplx; U_out holds one column per selected
 *              entry in the order of S's diagonal, zero above the entry,
 *              normalised so the entry of largest modulus is exactly 1 + 0i
 *              (the last such entry on ties) unless the plan was made with
 *              PEVC_NO_NORMALISE
 * Workspace: the first call allocates two n_max x n_max complex128 arrays and
 * an int32[n_max] array on the plan, besides pevc_solve_cplx's workspace.
 * Returns as pevc_solve_cplx.
 */
int pevc_solve_cplx_left(pevc_plan_t plan, const double *S, int lds, const double *T, int ldt, int n,
                         const int32_t *select, double *U_out, int ldu, int32_t *scale_out, int *m_out);

/*
 * pevc_backtransform_cplx -- eigenvectors of the original complex pencil:
 * with (A, B) = (Q S Z^H, Q T Z^H) the complex QZ reduction of (A, B), an
 * eigenvector v of the triangular (S, T) gives x = Z v for (A, B) (Section 1,
 * for complex data).  X = Z V is one complex FP64 GEMM (cuBLAS ZGEMM on the
 * plan's stream); then, unless PEVC_NO_NORMALISE, every column is scaled so
 * that its entry of largest modulus (the first on ties) is exactly 1 + 0i.
 *   Z, ldz     device, n x n complex128, column-major, 16-byte aligned
 *   n          order, <= the plan's n_max
 *   V, ldv     device, n x m complex128 (pevc_solve_cplx's output)
 *   m          0 <= m <= n
 *   X, ldx     device, n x m complex128, caller-allocated, not overlapping Z
 *              or V
 *   flags      0 or PEVC_NO_NORMALISE
 * The first call creates the plan's cuBLAS handle.  Synchronises on return.
 * Returns 0, -i (argument i invalid, counting the plan as argument 1) or
 * PEVC_ERR_CUDA.
 */
int pevc_backtransform_cplx(pevc_plan_t plan, const double *Z, int ldz, int n, const double *V, int ldv, int m,
                            double *X, int ldx, unsigned flags);

/*
 * pevc_watchdog_selftest -- exercises the bounded device waits.  Every wait
 * inside the library's kernels is bounded in SM clock cycles; when a bound
 * runs out the kernel records a timeout in the plan's status word and
 * returns, the call reports PEVC_ERR_TIMEOUT and the CUDA context stays
 * usable.  This call runs one such wait (an mbarrier wait, as in the
 * tensor-core update) on the plan's stream.
 *   withhold  0: the awaited arrival happens first, the wait completes
 *             1: the arrival is withheld, the wait gives up after `cycles`
 *   cycles    the bound, 0 < cycles <= 4e9 (about 2 s of SM clock)
 * Synchronises on return.  Returns 0 (wait completed), PEVC_ERR_TIMEOUT (the
 * bound ran out), -i for an invalid argument or PEVC_ERR_CUDA.
 */
int pevc_watchdog_selftest(pevc_plan_t plan, int withhold, long long cycles);

/*
 * pevc_scheduler_selftest -- exercises the bounded dependence wait of the
 * device-side task-graph scheduler (the persistent walk of Algorithm 1's task
 * graph, Section 3 and Section 5.3, that FP64 plans use): one walk of a
 * one-task list whose task waits on a ready counter.
 *   withhold  0: the counter is set first, the task runs at once
 *             1: nothing sets it; the wait gives up after `cycles`, records
 *                a timeout in the plan's status word and ends the walk
 *   cycles    the bound, 0 < cycles <= 4e9 (about 2 s of SM clock)
 * Synchronises on return.  Returns 0, PEVC_ERR_TIMEOUT (the bound ran out),
 * -i for an invalid argument or PEVC_ERR_CUDA.  The plan stays usable.
 */
int pevc_scheduler_selftest(pevc_plan_t plan, int withhold, long long cycles);

#ifdef __cplusplus
}
#endif
#endif /* PEVC_H */

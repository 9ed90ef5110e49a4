/*
 * oracle.c -- plain FP64 CPU oracle for the robust computation of the
 * generalized eigenvectors of a real Schur pencil (S, T).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this code.  It shares no code, header,
 * table or helper with the CUDA library; the two are written independently
 * from the paper (Kjelgaard Mikkelsen & Myllykoski, "Parallel Robust
 * Computation of Generalized Eigenvectors of Matrix Pencils", PPAM 2019).
 *
 * What it computes (Section 2, the "tall" equation and its Lemma):
 *   for each selected diagonal block j of S (1x1 at row c, or 2x2 at rows
 *   c, c+1) with eigenvalue (alpha_j, beta_j), alpha_j = a_j + i b_j, the
 *   vector v != 0 with v_i = 0 below the block and (beta_j S - alpha_j T) v = 0.
 *   A real eigenvalue gives one real column; a complex pair gives the two
 *   columns (Re z, Im z) of the eigenvector z for a_j + i b_j, b_j > 0.
 *
 * How: one eigenvector at a time, by column-oriented backward substitution
 * with dynamic scaling, the scalar method that the paper attributes to
 * LAPACK's xTGEVC (Section 1) and to Anderson's xLATRS principles
 * (Section 4).  Every division is guarded by ProtectDivision and every
 * linear update by ProtectUpdate (Section 4, properties 1 and 2); the scale
 * factors are powers of two, accumulated in a signed 32-bit exponent
 * (Section 5: Zazamoukh's scaling factors are signed 32-bit integers).
 *
 * Readings of points the paper leaves open:
 *   - Omega = 2^1022.  ProtectUpdate / ProtectDivision return a power of two
 *     2^-k, with k from exponent bounds (frexp); they satisfy the properties
 *     of Section 4 but may scale by up to 8x more than the minimum.
 *   - (alpha, beta): 1x1 block -> (S_cc, T_cc), sign chosen so beta >= 0;
 *     2x2 block (T_jj diagonal, positive) -> beta = 1, alpha = p + i q from
 *     the quadratic det(S_jj - lambda T_jj) = 0, q > 0.
 *   - Pre-scaling (Section 4, last paragraph; Section 5.2): instead of
 *     scaling S and T, (alpha, beta) of each eigenvalue is scaled by a power
 *     of two so that max(|beta|, |a|+|b|) * max|S,T entries| <= 2^1000.  The
 *     operator beta S - alpha T is then scaled by the same power of two and
 *     its null vector is unchanged.
 *   - Near-singular pivots: smin = max(u * (|beta| max|S_ii| + |alpha| max|T_ii|),
 *     DBL_MIN) over the entries of the diagonal block itself (u = 2^-53).
 *   - Complex magnitudes are bounded by |re| + |im|.
 *   - Output: each vector is divided by its entry of largest modulus (first
 *     index on ties), so that entry is exactly 1; scale[c] = e + ilogb(|max|),
 *     the binary exponent of the growth relative to a unit tip.
 *
 * Complex pencils (orc_evc_cplx, at the end of this file): the same
 * substitution for complex triangular (S, T) with 1x1 steps only.
 *
 * All arithmetic is IEEE binary64 with round-to-nearest; the build uses
 * -ffp-contract=off so no fused multiply-add changes the rounding.
 */
#include <float.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "oracle.h"

#define OMEGA_EXP 1022         /* Omega = 2^1022 */
#define PRESCALE_EXP 1000      /* |beta| max|S| and |alpha| max|T| are kept below 2^1000 */
#define ULP 0x1p-53            /* unit roundoff u */

#define SE(i, j) S[(size_t)(j) * (size_t)lds + (size_t)(i)]
#define TE(i, j) T[(size_t)(j) * (size_t)ldt + (size_t)(i)]

/* ------------------------------------------------------------------------ */
/* Scalar robustness primitives (Section 4).                                  */
/* ------------------------------------------------------------------------ */

/* Smallest E with v < 2^E, for finite v > 0. */
static int exp_above(double v)
{
    int e;
    frexp(v, &e);           /* v = m 2^e, m in [1/2, 1) */
    return e;
}

/* ProtectUpdate (Section 4, property 2): y = ||Y||, t = ||T||, x = ||X||, all
 * finite and >= 0.  Returns k >= 0 such that 2^-k (y + t x) <= Omega. */
int orc_protect_upd(double y, double t, double x)
{
    const int NONE = INT_MIN / 4;
    int ey = (y > 0.0) ? exp_above(y) : NONE;
    int etx = (t > 0.0 && x > 0.0) ? exp_above(t) + exp_above(x) : NONE;
    int top = (ey > etx ? ey : etx);
    if (top == NONE)
        return 0;
    int k = top + 1 - OMEGA_EXP;       /* y + t x < 2^(top+1) */
    return k > 0 ? k : 0;
}

/* ProtectDivision (Section 4, property 1): b >= 0 bounds |numerator|, t > 0
 * is |denominator|.  Returns k >= 0 such that 2^-k b <= t Omega. */
int orc_protect_div(double b, double t)
{
    if (!(b > 0.0))
        return 0;
    int eb = exp_above(b);             /* b < 2^eb */
    int et;
    frexp(t, &et);                     /* t >= 2^(et-1) */
    int k = eb - (et - 1) - OMEGA_EXP;
    return k > 0 ? k : 0;
}

/* ProtectDivision for the numerator bound 2^sh * b, evaluated without forming
 * 2^sh * b (which may exceed the binary64 range). */
static int protect_div_sh(double b, int sh, double t)
{
    if (!(b > 0.0))
        return 0;
    int et;
    frexp(t, &et);
    int k = exp_above(b) + sh - (et - 1) - OMEGA_EXP;
    return k > 0 ? k : 0;
}

/* Complex division q = a / b (b != 0): Smith's algorithm (1962) with the
 * refinement of Baudin and Smith (2012, "A robust complex division in
 * Scilab") for the case where the ratio of the divisor's parts underflows. */
void orc_cdiv(double ar, double ai, double br, double bi, double *qr, double *qi)
{
    if (fabs(bi) <= fabs(br)) {
        double r = bi / br;
        double t = 1.0 / (br + bi * r);
        if (r != 0.0) {
            *qr = (ar + ai * r) * t;
            *qi = (ai - ar * r) * t;
        } else {
            *qr = (ar + bi * (ai / br)) * t;
            *qi = (ai - bi * (ar / br)) * t;
        }
    } else {
        double r = br / bi;
        double t = 1.0 / (bi + br * r);
        if (r != 0.0) {
            *qr = (ar * r + ai) * t;
            *qi = (ai * r - ar) * t;
        } else {
            *qr = (br * (ar / bi) + ai) * t;
            *qi = (br * (ai / bi) - ar) * t;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Structure and eigenvalues (Section 2).                                     */
/* ------------------------------------------------------------------------ */

/* blk[i] = 0 for a 1x1 block, 1 for the first and 2 for the second row of a
 * 2x2 block.  A 2x2 block starts at i when S[i+1,i] != 0. */
int orc_blocks(int n, const double *S, int lds, const double *T, int ldt, signed char *blk)
{
    for (int i = 0; i < n; ++i)
        blk[i] = 0;
    for (int i = 0; i + 1 < n; ++i) {
        if (SE(i + 1, i) != 0.0) {
            if (blk[i] != 0)
                return ORC_ERR_NOT_SCHUR;       /* two adjacent subdiagonal entries */
            blk[i] = 1;
            blk[i + 1] = 2;
        }
    }
    (void)T;
    (void)ldt;
    return 0;
}

/* Largest |entry| over the parts of S and T that the method reads: the upper
 * triangles plus the subdiagonal entries inside 2x2 blocks.  Returns
 * ORC_ERR_NONFINITE if any of those entries is Inf or NaN. */
static int upper_maxabs(int n, const double *S, int lds, const double *T, int ldt,
                        const signed char *blk, double *mx)
{
    double m = 0.0;
    for (int j = 0; j < n; ++j) {
        int last = (j + 1 < n && blk[j] == 1) ? j + 1 : j;
        for (int i = 0; i <= last; ++i) {
            double s = fabs(SE(i, j)), t = fabs(TE(i, j));
            if (!isfinite(s) || !isfinite(t))
                return ORC_ERR_NONFINITE;
            if (s > m) m = s;
            if (t > m) m = t;
        }
    }
    *mx = m;
    return 0;
}

/* (a, b, beta) of every block, written at each of its rows, plus the
 * power-of-two pre-scaling exponent sigma (the pair is scaled by 2^-sigma). */
int orc_eigpairs(int n, const double *S, int lds, const double *T, int ldt,
                 const signed char *blk, double *a, double *b, double *beta, int *sigma)
{
    double mx;
    int st = upper_maxabs(n, S, lds, T, ldt, blk, &mx);
    if (st)
        return st;
    for (int c = 0; c < n; ++c) {
        if (blk[c] == 2)
            continue;
        double ac, bc, betac;
        if (blk[c] == 0) {
            ac = SE(c, c);
            betac = TE(c, c);
            bc = 0.0;
            if (betac < 0.0 || (betac == 0.0 && signbit(betac))) {
                ac = -ac;
                betac = -betac;
            }
        } else {
            double t1 = TE(c, c), t2 = TE(c + 1, c + 1);
            if (TE(c, c + 1) != 0.0 || TE(c + 1, c) != 0.0 || !(t1 > 0.0) || !(t2 > 0.0))
                return ORC_ERR_NOT_SCHUR;
            /* det(S_jj - lambda T_jj) = 0 with T_jj = diag(t1, t2):
             * lambda = p +- sqrt(d^2 + w), p = (u1+u2)/2, d = (u1-u2)/2,
             * u1 = s11/t1, u2 = s22/t2, w = (s12/t1)(s21/t2). */
            double u1 = SE(c, c) / t1, u2 = SE(c + 1, c + 1) / t2;
            double p = 0.5 * (u1 + u2), d = 0.5 * (u1 - u2);
            double w = (SE(c, c + 1) / t1) * (SE(c + 1, c) / t2);
            double q2 = -(d * d + w);
            if (!(q2 > 0.0))
                return ORC_ERR_NOT_SCHUR;      /* a 2x2 block with real eigenvalues */
            ac = p;
            bc = sqrt(q2);
            betac = 1.0;
            if (!isfinite(ac) || !isfinite(bc))
                return ORC_ERR_NONFINITE;
        }
        /* pre-scaling: max(|beta|, |a|+|b|) * mx <= 2^PRESCALE_EXP */
        int sg = 0;
        double coef = fmax(fabs(betac), fabs(ac) + fabs(bc));
        if (coef > 0.0 && mx > 0.0) {
            int k = exp_above(coef) + exp_above(mx) - PRESCALE_EXP;
            if (k > 0)
                sg = k;
        }
        if (sg) {
            ac = ldexp(ac, -sg);
            bc = ldexp(bc, -sg);
            betac = ldexp(betac, -sg);
        }
        int sz = (blk[c] == 1) ? 2 : 1;
        for (int r = c; r < c + sz; ++r) {
            a[r] = ac;
            b[r] = bc;
            beta[r] = betac;
            if (sigma)
                sigma[r] = sg;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One eigenvector by robust backward substitution.                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n;
    const double *S;
    int lds;
    const double *T;
    int ldt;
    const signed char *blk;
    const double *a, *b, *beta;
    const double *cS, *cT;   /* max |S_rk|, |T_rk| over the rows r above the block of column k */
} pencil_t;

static void scale_all(double *wr, double *wi, int len, double *rr, double *ri, int rlen, int k)
{
    for (int i = 0; i < len; ++i) {
        wr[i] = ldexp(wr[i], -k);
        if (wi) wi[i] = ldexp(wi[i], -k);
    }
    for (int i = 0; i < rlen; ++i) {
        rr[i] = ldexp(rr[i], -k);
        if (ri) ri[i] = ldexp(ri[i], -k);
    }
}

static double mag(double re, double im) { return fabs(re) + fabs(im); }

/* Solve the real 1x1 or 2x2 system (beta S_bb - a T_bb) x = r for the block
 * at rows i0 .. i0+sz-1 (real eigenvalue: b = 0).  Gaussian elimination with
 * complete pivoting for 2x2 (the DLALN2 principle that Section 5.2 names),
 * pivots below smin raised to smin, ProtectDivision before dividing. */
static void solve_real_block(const pencil_t *P, int i0, int sz, double a, double beta,
                             double *w, int len, double *r, int rlen, int *e, int robust)
{
    const double *S = P->S, *T = P->T;
    const int lds = P->lds, ldt = P->ldt;
    if (sz == 1) {
        double piv = beta * SE(i0, i0) - a * TE(i0, i0);
        if (robust) {
            double smin = fmax(ULP * (fabs(beta) * fabs(SE(i0, i0)) + fabs(a) * fabs(TE(i0, i0))), DBL_MIN);
            if (fabs(piv) < smin)
                piv = (piv < 0.0) ? -smin : smin;
            int k = orc_protect_div(fabs(r[i0]), fabs(piv));
            if (k) {
                scale_all(w, NULL, len, r, NULL, rlen, k);
                *e += k;
            }
        }
        w[i0] = r[i0] / piv;
        return;
    }
    double m[2][2], smax = 0.0, tmax = 0.0;
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) {
            m[p][q] = beta * SE(i0 + p, i0 + q) - a * TE(i0 + p, i0 + q);
            smax = fmax(smax, fabs(SE(i0 + p, i0 + q)));
            tmax = fmax(tmax, fabs(TE(i0 + p, i0 + q)));
        }
    double smin = fmax(ULP * (fabs(beta) * smax + fabs(a) * tmax), DBL_MIN);
    int pi = 0, pj = 0;
    double best = -1.0;
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q)
            if (fabs(m[p][q]) > best) {
                best = fabs(m[p][q]);
                pi = p;
                pj = q;
            }
    if (robust && best < smin) {
        m[0][0] = smin; m[0][1] = 0.0; m[1][0] = 0.0; m[1][1] = smin;
        pi = 0;
        pj = 0;
    }
    int oi = 1 - pi, oj = 1 - pj;
    double l = m[oi][pj] / m[pi][pj];
    double u22 = m[oi][oj] - l * m[pi][oj];
    if (robust) {
        if (fabs(u22) < smin)
            u22 = (u22 < 0.0) ? -smin : smin;
        double rn = fmax(fabs(r[i0]), fabs(r[i0 + 1]));
        int k = protect_div_sh(rn, 5, fabs(u22));
        if (k) {
            scale_all(w, NULL, len, r, NULL, rlen, k);
            *e += k;
        }
    }
    double rp = r[i0 + pi];
    double ro = r[i0 + oi] - l * rp;
    double xo = ro / u22;
    double xp = rp / m[pi][pj] - (m[pi][oj] / m[pi][pj]) * xo;
    w[i0 + oj] = xo;
    w[i0 + pj] = xp;
}

/* Complex counterpart for a complex eigenvalue alpha = a + i b. */
static void solve_cplx_block(const pencil_t *P, int i0, int sz, double a, double b, double beta,
                             double *wr, double *wi, int len, double *rr, double *ri, int rlen,
                             int *e, int robust)
{
    const double *S = P->S, *T = P->T;
    const int lds = P->lds, ldt = P->ldt;
    const double amag = fabs(a) + fabs(b);
    if (sz == 1) {
        double pr = beta * SE(i0, i0) - a * TE(i0, i0);
        double pim = -b * TE(i0, i0);
        if (robust) {
            double smin = fmax(ULP * (fabs(beta) * fabs(SE(i0, i0)) + amag * fabs(TE(i0, i0))), DBL_MIN);
            if (mag(pr, pim) < smin) {
                pr = smin;
                pim = 0.0;
            }
            int k = protect_div_sh(mag(rr[i0], ri[i0]), 1, mag(pr, pim));
            if (k) {
                scale_all(wr, wi, len, rr, ri, rlen, k);
                *e += k;
            }
        }
        orc_cdiv(rr[i0], ri[i0], pr, pim, &wr[i0], &wi[i0]);
        return;
    }
    double mr[2][2], mi[2][2], smax = 0.0, tmax = 0.0;
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) {
            mr[p][q] = beta * SE(i0 + p, i0 + q) - a * TE(i0 + p, i0 + q);
            mi[p][q] = -b * TE(i0 + p, i0 + q);
            smax = fmax(smax, fabs(SE(i0 + p, i0 + q)));
            tmax = fmax(tmax, fabs(TE(i0 + p, i0 + q)));
        }
    double smin = fmax(ULP * (fabs(beta) * smax + amag * tmax), DBL_MIN);
    int pi = 0, pj = 0;
    double best = -1.0;
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q)
            if (mag(mr[p][q], mi[p][q]) > best) {
                best = mag(mr[p][q], mi[p][q]);
                pi = p;
                pj = q;
            }
    if (robust && best < smin) {
        mr[0][0] = smin; mr[0][1] = 0.0; mr[1][0] = 0.0; mr[1][1] = smin;
        mi[0][0] = 0.0; mi[0][1] = 0.0; mi[1][0] = 0.0; mi[1][1] = 0.0;
        pi = 0;
        pj = 0;
    }
    int oi = 1 - pi, oj = 1 - pj;
    double lr, li;
    orc_cdiv(mr[oi][pj], mi[oi][pj], mr[pi][pj], mi[pi][pj], &lr, &li);
    /* u22 = m[oi][oj] - l * m[pi][oj] */
    double ur = mr[oi][oj] - (lr * mr[pi][oj] - li * mi[pi][oj]);
    double ui = mi[oi][oj] - (lr * mi[pi][oj] + li * mr[pi][oj]);
    if (robust) {
        if (mag(ur, ui) < smin) {
            ur = smin;
            ui = 0.0;
        }
        double rn = fmax(mag(rr[i0], ri[i0]), mag(rr[i0 + 1], ri[i0 + 1]));
        int k = protect_div_sh(rn, 5, mag(ur, ui));
        if (k) {
            scale_all(wr, wi, len, rr, ri, rlen, k);
            *e += k;
        }
    }
    double rpr = rr[i0 + pi], rpi = ri[i0 + pi];
    double ror = rr[i0 + oi] - (lr * rpr - li * rpi);
    double roi = ri[i0 + oi] - (lr * rpi + li * rpr);
    double xor_, xoi;
    orc_cdiv(ror, roi, ur, ui, &xor_, &xoi);
    double t1r, t1i, t2r, t2i;
    orc_cdiv(rpr, rpi, mr[pi][pj], mi[pi][pj], &t1r, &t1i);
    orc_cdiv(mr[pi][oj], mi[pi][oj], mr[pi][pj], mi[pi][pj], &t2r, &t2i);
    wr[i0 + oj] = xor_;
    wi[i0 + oj] = xoi;
    wr[i0 + pj] = t1r - (t2r * xor_ - t2i * xoi);
    wi[i0 + pj] = t1i - (t2r * xoi + t2i * xor_);
}

/* The vector of the block whose first row is c, unnormalised: on return
 * w[0 .. c+sz-1] (wi for a complex pair) and the exponent e represent the
 * eigenvector 2^e w relative to a tip of unit largest modulus. */
static int evc_block(const pencil_t *P, int c, double *wr, double *wi, int *e_out, int robust)
{
    const double *S = P->S, *T = P->T;
    const int lds = P->lds, ldt = P->ldt;
    const signed char *blk = P->blk;
    const int sz = (blk[c] == 1) ? 2 : 1;
    const double a = P->a[c], b = P->b[c], beta = P->beta[c];
    const int cplx = (sz == 2);
    const int len = c + sz;
    const double amag = fabs(a) + fabs(b);
    int e = 0;

    if (!cplx && a == 0.0 && beta == 0.0)
        return ORC_ERR_INDEFINITE;

    double *rr = (double *)calloc((size_t)(c > 0 ? c : 1), sizeof(double));
    double *ri = cplx ? (double *)calloc((size_t)(c > 0 ? c : 1), sizeof(double)) : NULL;
    if (!rr || (cplx && !ri)) {
        free(rr);
        free(ri);
        return ORC_ERR_NOMEM;
    }
    for (int i = 0; i < len; ++i) {
        wr[i] = 0.0;
        if (cplx) wi[i] = 0.0;
    }

    /* Tip: the eigenvector of the diagonal block itself (kernel 1 of
     * Section 3). */
    if (!cplx) {
        wr[c] = 1.0;
    } else {
        double mr[2][2], mi[2][2];
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) {
                mr[p][q] = beta * SE(c + p, c + q) - a * TE(c + p, c + q);
                mi[p][q] = -b * TE(c + p, c + q);
            }
        /* M is singular: (-m01, m00) and (m11, -m10) both span its kernel. */
        double v1r[2] = {-mr[0][1], mr[0][0]}, v1i[2] = {-mi[0][1], mi[0][0]};
        double v2r[2] = {mr[1][1], -mr[1][0]}, v2i[2] = {mi[1][1], -mi[1][0]};
        double n1 = fmax(mag(v1r[0], v1i[0]), mag(v1r[1], v1i[1]));
        double n2 = fmax(mag(v2r[0], v2i[0]), mag(v2r[1], v2i[1]));
        double *vr = (n1 >= n2) ? v1r : v2r, *vi = (n1 >= n2) ? v1i : v2i;
        int big = (hypot(vr[1], vi[1]) > hypot(vr[0], vi[0])) ? 1 : 0;
        double dr = vr[big], di = vi[big];
        for (int q = 0; q < 2; ++q)
            orc_cdiv(vr[q], vi[q], dr, di, &wr[c + q], &wi[c + q]);
        wr[c + big] = 1.0;
        wi[c + big] = 0.0;
    }

    /* Right-hand side for the rows above the tip: r = -(beta S - alpha T) w_tip. */
    if (c > 0) {
        double t = 0.0, x = 0.0;
        for (int q = 0; q < sz; ++q) {
            t += fabs(beta) * P->cS[c + q] + amag * P->cT[c + q];
            x = fmax(x, cplx ? mag(wr[c + q], wi[c + q]) : fabs(wr[c + q]));
        }
        if (robust) {
            int k = orc_protect_upd(0.0, t, x);
            if (k) {
                scale_all(wr, cplx ? wi : NULL, len, rr, ri, 0, k);
                e += k;
            }
        }
        for (int q = 0; q < sz; ++q) {
            int k = c + q;
            for (int i = 0; i < c; ++i) {
                double mrk = beta * SE(i, k) - a * TE(i, k);
                if (!cplx) {
                    rr[i] -= mrk * wr[k];
                } else {
                    double mik = -b * TE(i, k);
                    rr[i] -= mrk * wr[k] - mik * wi[k];
                    ri[i] -= mrk * wi[k] + mik * wr[k];
                }
            }
        }
    }

    /* Backward substitution over the blocks above the tip (kernel 3 of
     * Section 3, one column at a time). */
    int i = c - 1;
    while (i >= 0) {
        int i0 = (blk[i] == 2) ? i - 1 : i;
        int szi = i - i0 + 1;
        if (!cplx)
            solve_real_block(P, i0, szi, a, beta, wr, len, rr, c, &e, robust);
        else
            solve_cplx_block(P, i0, szi, a, b, beta, wr, wi, len, rr, ri, c, &e, robust);
        if (i0 > 0) {
            if (robust) {
                double y = 0.0, t = 0.0, x = 0.0;
                for (int r = 0; r < i0; ++r)
                    y = fmax(y, cplx ? mag(rr[r], ri[r]) : fabs(rr[r]));
                for (int q = 0; q < szi; ++q) {
                    t += fabs(beta) * P->cS[i0 + q] + amag * P->cT[i0 + q];
                    x = fmax(x, cplx ? mag(wr[i0 + q], wi[i0 + q]) : fabs(wr[i0 + q]));
                }
                int k = orc_protect_upd(y, t, x);
                if (k) {
                    scale_all(wr, cplx ? wi : NULL, len, rr, ri, c, k);
                    e += k;
                }
            }
            for (int q = 0; q < szi; ++q) {
                int k = i0 + q;
                for (int r = 0; r < i0; ++r) {
                    double mrk = beta * SE(r, k) - a * TE(r, k);
                    if (!cplx) {
                        rr[r] -= mrk * wr[k];
                    } else {
                        double mik = -b * TE(r, k);
                        rr[r] -= mrk * wr[k] - mik * wi[k];
                        ri[r] -= mrk * wi[k] + mik * wr[k];
                    }
                }
            }
        }
        i = i0 - 1;
    }
    free(rr);
    free(ri);
    *e_out = e;
    return 0;
}

/* Column norms above each block: cS[k] = max_{r < start(k)} |S_rk|. */
static void column_norms(int n, const double *S, int lds, const double *T, int ldt,
                         const signed char *blk, double *cS, double *cT)
{
    for (int k = 0; k < n; ++k) {
        int start = (blk[k] == 2) ? k - 1 : k;
        double ms = 0.0, mt = 0.0;
        for (int r = 0; r < start; ++r) {
            ms = fmax(ms, fabs(SE(r, k)));
            mt = fmax(mt, fabs(TE(r, k)));
        }
        cS[k] = ms;
        cT[k] = mt;
    }
}

/* ------------------------------------------------------------------------ */
/* Public driver.                                                             */
/* ------------------------------------------------------------------------ */

int orc_evc(int n, const double *S, int lds, const double *T, int ldt, const int *select,
            int flags, double *V, int ldv, int32_t *scale, int *m_out, int nthreads)
{
    if (n < 0) return -1;
    if (n > 0 && !S) return -2;
    if (lds < (n > 1 ? n : 1)) return -3;
    if (n > 0 && !T) return -4;
    if (ldt < (n > 1 ? n : 1)) return -5;
    if (n > 0 && !V) return -8;
    if (ldv < (n > 1 ? n : 1)) return -9;
    if (!m_out) return -11;
    *m_out = 0;
    if (n == 0)
        return 0;

    signed char *blk = (signed char *)malloc((size_t)n);
    double *a = (double *)malloc((size_t)n * sizeof(double));
    double *b = (double *)malloc((size_t)n * sizeof(double));
    double *beta = (double *)malloc((size_t)n * sizeof(double));
    double *cS = (double *)malloc((size_t)n * sizeof(double));
    double *cT = (double *)malloc((size_t)n * sizeof(double));
    int *outcol = (int *)malloc((size_t)n * sizeof(int));
    int status = 0;
    if (!blk || !a || !b || !beta || !cS || !cT || !outcol) {
        status = ORC_ERR_NOMEM;
        goto done;
    }
    status = orc_blocks(n, S, lds, T, ldt, blk);
    if (status) goto done;
    status = orc_eigpairs(n, S, lds, T, ldt, blk, a, b, beta, NULL);
    if (status) goto done;
    column_norms(n, S, lds, T, ldt, blk, cS, cT);

    /* Output column of each selected block (a pair is selected when either of
     * its rows is; closure under conjugation, Section 5). */
    int m = 0;
    for (int c = 0; c < n; ++c) {
        outcol[c] = -1;
        if (blk[c] == 2) continue;
        int sz = (blk[c] == 1) ? 2 : 1;
        int sel = !select || select[c] || (sz == 2 && select[c + 1]);
        if (sel) {
            outcol[c] = select ? m : c;
            m += sz;
        }
    }
    *m_out = select ? m : n;

    pencil_t P = {n, S, lds, T, ldt, blk, a, b, beta, cS, cT};
    const int robust = !(flags & ORC_FLAG_PLAIN);
    const int normalise = !(flags & ORC_FLAG_NO_NORMALISE);
    int nt = nthreads > 0 ? nthreads : 1;
    (void)nt;

#pragma omp parallel num_threads(nt)
    {
        double *wr = (double *)malloc((size_t)n * sizeof(double));
        double *wi = (double *)malloc((size_t)n * sizeof(double));
        int local = (!wr || !wi) ? ORC_ERR_NOMEM : 0;
#pragma omp for schedule(dynamic, 1)
        for (int c = n - 1; c >= 0; --c) {
            if (outcol[c] < 0 || local) continue;
            int sz = (blk[c] == 1) ? 2 : 1;
            int e = 0;
            int st = evc_block(&P, c, wr, sz == 2 ? wi : NULL, &e, robust);
            if (st) {
                local = st;
                continue;
            }
            int len = c + sz, oc = outcol[c];
            double *v0 = V + (size_t)oc * (size_t)ldv;
            double *v1 = (sz == 2) ? V + (size_t)(oc + 1) * (size_t)ldv : NULL;
            int32_t sc = e;
            if (normalise) {
                int istar = 0;
                double best = -1.0;
                for (int r = 0; r < len; ++r) {
                    double mr = (sz == 2) ? hypot(wr[r], wi[r]) : fabs(wr[r]);
                    if (mr > best) {
                        best = mr;
                        istar = r;
                    }
                }
                if (best > 0.0)
                    sc = e + ilogb(best);
                if (sz == 1) {
                    double d = wr[istar];
                    for (int r = 0; r < len; ++r)
                        v0[r] = wr[r] / d;
                    v0[istar] = 1.0;
                } else {
                    double dr = wr[istar], di = wi[istar];
                    for (int r = 0; r < len; ++r)
                        orc_cdiv(wr[r], wi[r], dr, di, &v0[r], &v1[r]);
                    v0[istar] = 1.0;
                    v1[istar] = 0.0;
                }
            } else {
                for (int r = 0; r < len; ++r) {
                    v0[r] = wr[r];
                    if (sz == 2) v1[r] = wi[r];
                }
            }
            for (int r = len; r < n; ++r) {
                v0[r] = 0.0;
                if (sz == 2) v1[r] = 0.0;
            }
            if (scale) {
                scale[oc] = sc;
                if (sz == 2) scale[oc + 1] = sc;
            }
        }
#pragma omp critical
        {
            if (local && !status) status = local;
        }
        free(wr);
        free(wi);
    }
    if (!select) {
        /* unselected positions cannot exist without a selection */
    }
done:
    free(blk);
    free(a);
    free(b);
    free(beta);
    free(cS);
    free(cT);
    free(outcol);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Complex pencils (Section 7, the extension to complex data types).          */
/* ------------------------------------------------------------------------ */

/* A complex pencil (S, T) in generalized complex Schur form: both upper
 * triangular, entries stored interleaved (re, im) in column-major order with
 * leading dimensions counted in complex elements.  There are no 2x2 blocks:
 * every diagonal entry gives one eigenvalue (alpha, beta) = (S_cc, T_cc),
 * both complex, and one eigenvector x with x_c = 1, x_i = 0 below c and
 * (beta S - alpha T) x = 0.  The substitution is the scalar method above with
 * complex arithmetic throughout; magnitudes are bounded by |re| + |im|, which
 * is submultiplicative for complex products, so ProtectUpdate's bound
 * ||Y|| + ||T|| ||X|| covers the complex update. */

#define CSR(i, j) S[2 * ((size_t)(j) * (size_t)lds + (size_t)(i))]
#define CSI(i, j) S[2 * ((size_t)(j) * (size_t)lds + (size_t)(i)) + 1]
#define CTR(i, j) T[2 * ((size_t)(j) * (size_t)ldt + (size_t)(i))]
#define CTI(i, j) T[2 * ((size_t)(j) * (size_t)ldt + (size_t)(i)) + 1]

/* (alpha, beta) of every diagonal entry, scaled by 2^-sigma so that
 * max(|beta|, |alpha|) * max|S, T entries| <= 2^PRESCALE_EXP (magnitudes
 * |re| + |im|).  Returns ORC_ERR_NONFINITE if an entry of the upper
 * triangles is Inf or NaN. */
int orc_eigpairs_cplx(int n, const double *S, int lds, const double *T, int ldt,
                      double *alpha, double *beta, int *sigma)
{
    double mx = 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i <= j; ++i) {
            double ms = mag(CSR(i, j), CSI(i, j)), mt = mag(CTR(i, j), CTI(i, j));
            if (!isfinite(ms) || !isfinite(mt))
                return ORC_ERR_NONFINITE;
            mx = fmax(mx, fmax(ms, mt));
        }
    for (int c = 0; c < n; ++c) {
        double ar = CSR(c, c), ai = CSI(c, c), br = CTR(c, c), bi = CTI(c, c);
        int sg = 0;
        double coef = fmax(mag(br, bi), mag(ar, ai));
        if (coef > 0.0 && mx > 0.0) {
            int k = exp_above(coef) + exp_above(mx) - PRESCALE_EXP;
            if (k > 0)
                sg = k;
        }
        alpha[2 * c] = ldexp(ar, -sg);
        alpha[2 * c + 1] = ldexp(ai, -sg);
        beta[2 * c] = ldexp(br, -sg);
        beta[2 * c + 1] = ldexp(bi, -sg);
        if (sigma)
            sigma[c] = sg;
    }
    return 0;
}

/* m = beta * s - alpha * t for complex scalars. */
static void cpencil(double br, double bi, double ar, double ai, double sr, double si, double tr, double ti,
                    double *mr, double *mi)
{
    *mr = (br * sr - bi * si) - (ar * tr - ai * ti);
    *mi = (br * si + bi * sr) - (ar * ti + ai * tr);
}

/* The eigenvector of diagonal entry c: on return w[0 .. c] (re, im
 * interleaved) and e represent 2^e w relative to the unit tip w_c = 1. */
static int evc_cplx_one(int n, const double *S, int lds, const double *T, int ldt, const double *alpha,
                        const double *beta, const double *cS, const double *cT, int c, double *w, double *r,
                        int *e_out, int robust)
{
    (void)n;
    const double ar = alpha[2 * c], ai = alpha[2 * c + 1], br = beta[2 * c], bi = beta[2 * c + 1];
    const double amag = mag(ar, ai), bmag = mag(br, bi);
    if (amag == 0.0 && bmag == 0.0)
        return ORC_ERR_INDEFINITE;
    int e = 0;
    for (int i = 0; i <= c; ++i) {
        w[2 * i] = 0.0;
        w[2 * i + 1] = 0.0;
    }
    w[2 * c] = 1.0;
    for (int i = 0; i < c; ++i) {
        r[2 * i] = 0.0;
        r[2 * i + 1] = 0.0;
    }
    /* r = -(beta S - alpha T)[0:c, c] * w_c (the tip is 1) */
    if (c > 0) {
        if (robust) {
            int k = orc_protect_upd(0.0, bmag * cS[c] + amag * cT[c], 1.0);
            if (k) {
                scale_all(w, NULL, 2 * (c + 1), r, NULL, 0, k);
                e += k;
            }
        }
        const double xr = w[2 * c], xi = w[2 * c + 1];
        for (int i = 0; i < c; ++i) {
            double mr, mi;
            cpencil(br, bi, ar, ai, CSR(i, c), CSI(i, c), CTR(i, c), CTI(i, c), &mr, &mi);
            r[2 * i] -= mr * xr - mi * xi;
            r[2 * i + 1] -= mr * xi + mi * xr;
        }
    }
    for (int i = c - 1; i >= 0; --i) {
        double pr, pim;
        cpencil(br, bi, ar, ai, CSR(i, i), CSI(i, i), CTR(i, i), CTI(i, i), &pr, &pim);
        if (robust) {
            double smin = fmax(ULP * (bmag * mag(CSR(i, i), CSI(i, i)) + amag * mag(CTR(i, i), CTI(i, i))),
                               DBL_MIN);
            if (mag(pr, pim) < smin) {
                pr = smin;
                pim = 0.0;
            }
            /* |q|_1 <= 2 |a|_1 / |b|_1 for q = a / b, hence the factor 2^1 */
            int k = protect_div_sh(mag(r[2 * i], r[2 * i + 1]), 1, mag(pr, pim));
            if (k) {
                scale_all(w, NULL, 2 * (c + 1), r, NULL, 2 * c, k);
                e += k;
            }
        }
        orc_cdiv(r[2 * i], r[2 * i + 1], pr, pim, &w[2 * i], &w[2 * i + 1]);
        if (i > 0) {
            const double xr = w[2 * i], xi = w[2 * i + 1];
            if (robust) {
                double y = 0.0;
                for (int q = 0; q < i; ++q)
                    y = fmax(y, mag(r[2 * q], r[2 * q + 1]));
                int k = orc_protect_upd(y, bmag * cS[i] + amag * cT[i], mag(xr, xi));
                if (k) {
                    scale_all(w, NULL, 2 * (c + 1), r, NULL, 2 * c, k);
                    e += k;
                }
            }
            const double yr = w[2 * i], yi = w[2 * i + 1];
            for (int q = 0; q < i; ++q) {
                double mr, mi;
                cpencil(br, bi, ar, ai, CSR(q, i), CSI(q, i), CTR(q, i), CTI(q, i), &mr, &mi);
                r[2 * q] -= mr * yr - mi * yi;
                r[2 * q + 1] -= mr * yi + mi * yr;
            }
        }
    }
    *e_out = e;
    return 0;
}

int orc_evc_cplx(int n, const double *S, int lds, const double *T, int ldt, const int *select, int flags,
                 double *V, int ldv, int32_t *scale, int *m_out, int nthreads)
{
    if (n < 0) return -1;
    if (n > 0 && !S) return -2;
    if (lds < (n > 1 ? n : 1)) return -3;
    if (n > 0 && !T) return -4;
    if (ldt < (n > 1 ? n : 1)) return -5;
    if (n > 0 && !V) return -8;
    if (ldv < (n > 1 ? n : 1)) return -9;
    if (!m_out) return -11;
    *m_out = 0;
    if (n == 0)
        return 0;
    double *alpha = (double *)malloc((size_t)n * 2 * sizeof(double));
    double *beta = (double *)malloc((size_t)n * 2 * sizeof(double));
    double *cS = (double *)malloc((size_t)n * sizeof(double));
    double *cT = (double *)malloc((size_t)n * sizeof(double));
    int *outcol = (int *)malloc((size_t)n * sizeof(int));
    int status = 0;
    if (!alpha || !beta || !cS || !cT || !outcol) {
        status = ORC_ERR_NOMEM;
        goto done;
    }
    status = orc_eigpairs_cplx(n, S, lds, T, ldt, alpha, beta, NULL);
    if (status) goto done;
    /* cS[k] = max_{r < k} |S_rk|, cT likewise */
    for (int k = 0; k < n; ++k) {
        double ms = 0.0, mt = 0.0;
        for (int q = 0; q < k; ++q) {
            ms = fmax(ms, mag(CSR(q, k), CSI(q, k)));
            mt = fmax(mt, mag(CTR(q, k), CTI(q, k)));
        }
        cS[k] = ms;
        cT[k] = mt;
    }
    int m = 0;
    for (int c = 0; c < n; ++c) {
        outcol[c] = (!select || select[c]) ? m : -1;
        if (outcol[c] >= 0) ++m;
    }
    *m_out = m;
    const int robust = !(flags & ORC_FLAG_PLAIN);
    const int normalise = !(flags & ORC_FLAG_NO_NORMALISE);
    int nt = nthreads > 0 ? nthreads : 1;
    (void)nt;

#pragma omp parallel num_threads(nt)
    {
        double *w = (double *)malloc((size_t)n * 2 * sizeof(double));
        double *r = (double *)malloc((size_t)n * 2 * sizeof(double));
        int local = (!w || !r) ? ORC_ERR_NOMEM : 0;
#pragma omp for schedule(dynamic, 1)
        for (int c = n - 1; c >= 0; --c) {
            if (outcol[c] < 0 || local) continue;
            int e = 0;
            int st = evc_cplx_one(n, S, lds, T, ldt, alpha, beta, cS, cT, c, w, r, &e, robust);
            if (st) {
                local = st;
                continue;
            }
            double *v = V + 2 * (size_t)outcol[c] * (size_t)ldv;
            int32_t sc = e;
            if (normalise) {
                int istar = 0;
                double best = -1.0;
                for (int i = 0; i <= c; ++i) {
                    double mi = hypot(w[2 * i], w[2 * i + 1]);
                    if (mi > best) {
                        best = mi;
                        istar = i;
                    }
                }
                if (best > 0.0)
                    sc = e + ilogb(best);
                const double dr = w[2 * istar], di = w[2 * istar + 1];
                for (int i = 0; i <= c; ++i)
                    orc_cdiv(w[2 * i], w[2 * i + 1], dr, di, &v[2 * i], &v[2 * i + 1]);
                v[2 * istar] = 1.0;
                v[2 * istar + 1] = 0.0;
            } else {
                for (int i = 0; i <= c; ++i) {
                    v[2 * i] = w[2 * i];
                    v[2 * i + 1] = w[2 * i + 1];
                }
            }
            for (int i = c + 1; i < n; ++i) {
                v[2 * i] = 0.0;
                v[2 * i + 1] = 0.0;
            }
            if (scale)
                scale[outcol[c]] = sc;
        }
#pragma omp critical
        {
            if (local && !status) status = local;
        }
        free(w);
        free(r);
    }
done:
    free(alpha);
    free(beta);
    free(cS);
    free(cT);
    free(outcol);
    return status;
}

int orc_version(void) { return 1; }

/*
 * Plain FP64 CPU oracle for ALS-WR / ALS-NCG (Winlaw, Hynes, Caterini,
 * De Sterck, "Algorithmic Acceleration of Parallel ALS for Collaborative
 * Filtering", arXiv 1508.03110).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or constant with the CUDA path.
 *
 * Everything is double precision and written as the paper states it, row by
 * row, with no blocking or fusion:
 *   - loss            Eq. (1), §II
 *   - gradient        §III-A (the expanded derivative) and §V-C "Gradient
 *                     Evaluation"
 *   - per-row solve   Eq. (3) (users) and Eq. (4) (items), by a textbook
 *                     column (gaxpy) Cholesky factorisation, Golub & Van Loan
 *   - one ALS sweep   Algorithm 1 loop body: all u_i, then all m_j
 *   - line-search polynomial Q(alpha) coefficients, §V-C "Line Search & Loss
 *                     Function Evaluation"
 *
 * Data layout: the iterate x is Eq. (5) flattened: n_u rows u_i of n_f values,
 * then n_m rows m_j of n_f values (row-major, no padding).  Ratings come as a
 * by-user list (uptr/uidx/uval, items of each user ascending) and a by-item
 * list (mptr/midx/mval, users of each item ascending).
 *
 * Reductions: every row's scalar term is stored in a per-row array and the
 * array is then summed serially in row order, so results are bit-identical for
 * any OpenMP thread count.
 *
 * Empty rows (n_ui = 0 or n_mj = 0): the row does not enter f, its Gram matrix
 * is the zero matrix and Eq. (3)/(4) is singular.  Reading used here: the
 * solve sets that row to zero; its gradient is zero.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n_u, n_m;
    int32_t n_f;
    double lambda;
    const int64_t *uptr; const int32_t *uidx; const double *uval; /* by user */
    const int64_t *mptr; const int32_t *midx; const double *mval; /* by item */
} orc_problem;

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static double dot(const double *a, const double *b, int n) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

static double ordered_sum(const double *t, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += t[i];
    return s;
}

/* ---------------------------------------------------------------------------
 * Eq. (1): L = sum_{(i,j) in I} (r_ij - u_i.m_j)^2
 *            + lambda (sum_i n_ui |u_i|^2 + sum_j n_mj |m_j|^2)
 * ------------------------------------------------------------------------- */
double orc_loss(const orc_problem *P, const double *X) {
    const int nf = P->n_f;
    const double *U = X, *M = X + P->n_u * (int64_t)nf;
    const int64_t nrow = P->n_u + P->n_m;
    double *term = (double *)malloc(sizeof(double) * (size_t)(nrow > 0 ? nrow : 1));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < P->n_u; ++i) {
        const double *u = U + i * nf;
        const int64_t n = P->uptr[i + 1] - P->uptr[i];
        double s = 0.0;
        for (int64_t e = P->uptr[i]; e < P->uptr[i + 1]; ++e) {
            const double r = P->uval[e] - dot(u, M + (int64_t)P->uidx[e] * nf, nf);
            s += r * r;
        }
        term[i] = s + P->lambda * (double)n * dot(u, u, nf);
    }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < P->n_m; ++j) {
        const double *m = M + j * nf;
        const int64_t n = P->mptr[j + 1] - P->mptr[j];
        term[P->n_u + j] = P->lambda * (double)n * dot(m, m, nf);
    }
    const double f = ordered_sum(term, nrow);
    free(term);
    return f;
}

/* ---------------------------------------------------------------------------
 * Gradient (§III-A expansion; §V-C "Gradient Evaluation"):
 *   dL/du_i = 2 lambda n_ui u_i + 2 sum_{j in I_i} (u_i.m_j - r_ij) m_j
 *   dL/dm_j = 2 lambda n_mj m_j + 2 sum_{i in I_j} (u_i.m_j - r_ij) u_i
 * ------------------------------------------------------------------------- */
void orc_grad(const orc_problem *P, const double *X, double *G) {
    const int nf = P->n_f;
    const double *U = X, *M = X + P->n_u * (int64_t)nf;
    double *GU = G, *GM = G + P->n_u * (int64_t)nf;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < P->n_u; ++i) {
        const double *u = U + i * nf;
        double *g = GU + i * nf;
        const int64_t n = P->uptr[i + 1] - P->uptr[i];
        for (int k = 0; k < nf; ++k) g[k] = 2.0 * P->lambda * (double)n * u[k];
        for (int64_t e = P->uptr[i]; e < P->uptr[i + 1]; ++e) {
            const double *m = M + (int64_t)P->uidx[e] * nf;
            const double d = dot(u, m, nf) - P->uval[e];
            for (int k = 0; k < nf; ++k) g[k] += 2.0 * d * m[k];
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < P->n_m; ++j) {
        const double *m = M + j * nf;
        double *g = GM + j * nf;
        const int64_t n = P->mptr[j + 1] - P->mptr[j];
        for (int k = 0; k < nf; ++k) g[k] = 2.0 * P->lambda * (double)n * m[k];
        for (int64_t e = P->mptr[j]; e < P->mptr[j + 1]; ++e) {
            const double *u = U + (int64_t)P->midx[e] * nf;
            const double d = dot(u, m, nf) - P->mval[e];
            for (int k = 0; k < nf; ++k) g[k] += 2.0 * d * u[k];
        }
    }
}

/* ---------------------------------------------------------------------------
 * Textbook Cholesky solve of a symmetric positive definite n x n system
 * A x = b (A row-major, only its lower triangle is read).  Column-oriented
 * ("gaxpy") Cholesky, Golub & Van Loan: for each column j, subtract the
 * contributions of the already-finished columns, then divide by the square
 * root of the pivot.  Then L y = b forwards and L^T x = y backwards.
 * Returns 0 on success, -1 if a pivot is not positive.  L is scratch (n*n).
 * ------------------------------------------------------------------------- */
int orc_chol_solve(int n, const double *A, const double *b, double *x, double *L) {
    for (int j = 0; j < n; ++j) {
        for (int i = j; i < n; ++i) {
            double v = A[i * n + j];
            for (int k = 0; k < j; ++k) v -= L[i * n + k] * L[j * n + k];
            if (i == j) {
                if (!(v > 0.0)) return -1;
                L[j * n + j] = sqrt(v);
            } else {
                L[i * n + j] = v / L[j * n + j];
            }
        }
    }
    for (int i = 0; i < n; ++i) {          /* forward: L y = b */
        double v = b[i];
        for (int k = 0; k < i; ++k) v -= L[i * n + k] * x[k];
        x[i] = v / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {     /* backward: L^T x = y */
        double v = x[i];
        for (int k = i + 1; k < n; ++k) v -= L[k * n + i] * x[k];
        x[i] = v / L[i * n + i];
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * One row of Eq. (3) / Eq. (4): given the n fixed-side vectors F[idx[e]] and
 * the ratings val[e] of this row,
 *   A = sum_e F_e F_e^T + lambda * n * I,   v = sum_e val_e F_e,   out = A^-1 v.
 * Returns 0, or -1 if A is not positive definite.  Empty rows give zero.
 * ------------------------------------------------------------------------- */
int orc_solve_row(int nf, double lambda, int64_t n, const int32_t *idx,
                  const double *val, const double *F, double *out, double *work) {
    double *A = work, *v = work + nf * nf, *L = work + nf * nf + nf;
    if (n == 0) {
        for (int k = 0; k < nf; ++k) out[k] = 0.0;
        return 0;
    }
    memset(A, 0, sizeof(double) * (size_t)(nf * nf));
    memset(v, 0, sizeof(double) * (size_t)nf);
    for (int64_t e = 0; e < n; ++e) {
        const double *f = F + (int64_t)idx[e] * nf;
        for (int a = 0; a < nf; ++a) {
            for (int b = 0; b < nf; ++b) A[a * nf + b] += f[a] * f[b];
            v[a] += val[e] * f[a];
        }
    }
    for (int a = 0; a < nf; ++a) A[a * nf + a] += lambda * (double)n;
    return orc_chol_solve(nf, A, v, out, L);
}

/* Half of Algorithm 1: all u_i from Eq. (3) with M fixed (side 0), or all m_j
 * from Eq. (4) with U fixed (side 1).  F is the fixed factor block, OUT the
 * solved block.  Returns the number of rows whose matrix was not SPD. */
int64_t orc_half_sweep(const orc_problem *P, int side, const double *F, double *OUT) {
    const int nf = P->n_f;
    const int64_t nrow = side == 0 ? P->n_u : P->n_m;
    const int64_t *ptr = side == 0 ? P->uptr : P->mptr;
    const int32_t *idx = side == 0 ? P->uidx : P->midx;
    const double *val = side == 0 ? P->uval : P->mval;
    int64_t bad = 0;
#pragma omp parallel reduction(+ : bad)
    {
        double *work = (double *)malloc(sizeof(double) * (size_t)(2 * nf * nf + nf));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < nrow; ++i) {
            if (orc_solve_row(nf, P->lambda, ptr[i + 1] - ptr[i], idx + ptr[i], val + ptr[i],
                              F, OUT + i * nf, work) != 0)
                bad += 1;
        }
        free(work);
    }
    return bad;
}

/* The same solve for a chosen subset of rows only (rows[q] of side 0/1);
 * OUT[q] receives that row.  Used to check sampled rows of large problems. */
int64_t orc_solve_rows(const orc_problem *P, int side, const double *F, int64_t nsel,
                       const int64_t *rows, double *OUT) {
    const int nf = P->n_f;
    const int64_t *ptr = side == 0 ? P->uptr : P->mptr;
    const int32_t *idx = side == 0 ? P->uidx : P->midx;
    const double *val = side == 0 ? P->uval : P->mval;
    int64_t bad = 0;
#pragma omp parallel reduction(+ : bad)
    {
        double *work = (double *)malloc(sizeof(double) * (size_t)(2 * nf * nf + nf));
#pragma omp for schedule(static)
        for (int64_t q = 0; q < nsel; ++q) {
            const int64_t i = rows[q];
            if (orc_solve_row(nf, P->lambda, ptr[i + 1] - ptr[i], idx + ptr[i], val + ptr[i], F,
                              OUT + q * nf, work) != 0)
                bad += 1;
        }
        free(work);
    }
    return bad;
}

/* P(x) = one ALS iteration, Algorithm 1 loop body: the U block of XBAR from
 * the M block of X, then the M block of XBAR from the new U block. */
int64_t orc_sweep(const orc_problem *P, const double *X, double *XBAR) {
    const int64_t off = P->n_u * (int64_t)P->n_f;
    int64_t bad = orc_half_sweep(P, 0, X + off, XBAR);
    bad += orc_half_sweep(P, 1, XBAR, XBAR + off);
    return bad;
}

/* ---------------------------------------------------------------------------
 * §V-C: Q(alpha) = f(x + alpha p) = sum_{n=0..4} c_n alpha^n.
 * With u = x_u + alpha p_u and m = x_m + alpha p_m, each rating contributes
 *   (r - u.m)^2 = (e0 - alpha a - alpha^2 b)^2,
 *   e0 = r - x_u.x_m,  a = x_u.p_m + p_u.x_m,  b = p_u.p_m,
 * i.e. e0^2, -2 e0 a, a^2 - 2 e0 b, 2 a b, b^2 for alpha^0..alpha^4, and each
 * row contributes lambda n (|x|^2 + 2 alpha x.p + alpha^2 |p|^2).
 * ------------------------------------------------------------------------- */
void orc_ls_coeffs(const orc_problem *P, const double *X, const double *PD, double c[5]) {
    const int nf = P->n_f;
    const int64_t off = P->n_u * (int64_t)nf, nrow = P->n_u + P->n_m;
    double *term = (double *)malloc(sizeof(double) * (size_t)(5 * (nrow > 0 ? nrow : 1)));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < P->n_u; ++i) {
        const double *xu = X + i * nf, *pu = PD + i * nf;
        double t[5] = {0, 0, 0, 0, 0};
        for (int64_t e = P->uptr[i]; e < P->uptr[i + 1]; ++e) {
            const int64_t j = P->uidx[e];
            const double *xm = X + off + j * nf, *pm = PD + off + j * nf;
            const double e0 = P->uval[e] - dot(xu, xm, nf);
            const double a = dot(xu, pm, nf) + dot(pu, xm, nf);
            const double b = dot(pu, pm, nf);
            t[0] += e0 * e0;
            t[1] += -2.0 * e0 * a;
            t[2] += a * a - 2.0 * e0 * b;
            t[3] += 2.0 * a * b;
            t[4] += b * b;
        }
        const double ln = P->lambda * (double)(P->uptr[i + 1] - P->uptr[i]);
        t[0] += ln * dot(xu, xu, nf);
        t[1] += ln * 2.0 * dot(xu, pu, nf);
        t[2] += ln * dot(pu, pu, nf);
        for (int n = 0; n < 5; ++n) term[n * nrow + i] = t[n];
    }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < P->n_m; ++j) {
        const double *xm = X + off + j * nf, *pm = PD + off + j * nf;
        const double ln = P->lambda * (double)(P->mptr[j + 1] - P->mptr[j]);
        term[0 * nrow + P->n_u + j] = ln * dot(xm, xm, nf);
        term[1 * nrow + P->n_u + j] = ln * 2.0 * dot(xm, pm, nf);
        term[2 * nrow + P->n_u + j] = ln * dot(pm, pm, nf);
        term[3 * nrow + P->n_u + j] = 0.0;
        term[4 * nrow + P->n_u + j] = 0.0;
    }
    for (int n = 0; n < 5; ++n) c[n] = ordered_sum(term + n * nrow, nrow);
    free(term);
}

/* Fold-in of new users against a fixed M (Eq. (3) for rows that are not in R):
 * request q has ratings idx/val[req_ptr[q] .. req_ptr[q+1]).  Returns the
 * number of requests whose matrix was not SPD. */
int64_t orc_foldin(int nf, double lambda, int64_t n_req, const int64_t *req_ptr,
                   const int32_t *idx, const double *val, const double *M, double *OUT) {
    int64_t bad = 0;
#pragma omp parallel reduction(+ : bad)
    {
        double *work = (double *)malloc(sizeof(double) * (size_t)(2 * nf * nf + nf));
#pragma omp for schedule(static)
        for (int64_t q = 0; q < n_req; ++q) {
            if (orc_solve_row(nf, lambda, req_ptr[q + 1] - req_ptr[q], idx + req_ptr[q],
                              val + req_ptr[q], M, OUT + q * nf, work) != 0)
                bad += 1;
        }
        free(work);
    }
    return bad;
}

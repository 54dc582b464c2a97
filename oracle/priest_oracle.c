/*
 * priest_oracle.c -- plain FP64 CPU oracle for PRIEST (arXiv 2309.08235).
 *
 * TEST INFRASTRUCTURE ONLY: see priest_oracle.h.  Everything here is written
 * for a reader checking it against the paper: dense matrices, plain loops,
 * trigonometric targets exactly as the paper's polar form writes them, a
 * literal block-by-block F^T product, and a dense KKT solved by LU with
 * partial pivoting.  No blocking, fusion or algebraic shortcut.
 *
 * Readings of points the paper leaves open (each is also listed in the
 * repository's design notes):
 *   - The right-hand side of the shared KKT system carries +rho F^T e
 *     (stationarity of eq. lagrange; eq. matrix_vec prints a minus sign).
 *   - The multiplier step uses the e rebuilt from the current iterate
 *     (eq. fixed_point_1: h(xi_bar^k, lambda^k) returns e^{k+1} and
 *     lambda^{k+1}), and the full e = [e_tilde; tau - s].
 *   - xi_bar^0 = Pi_A(xi), lambda^0 = 0 unless a warm start is given.
 *   - beta of an (a, a, b) ellipsoid is taken in the axis-scaled frame,
 *     beta = atan2(sqrt(dx^2+dy^2)/a, dz/b); d is then the exact argmin of
 *     the Lagrangian given (alpha, beta), clipped to d >= 1.
 *   - atan2(0, 0) = 0 for degenerate directions.
 *   - Refit weights exp(-(c_aug - delta)/gamma) (eq. update_covariance prints
 *     a positive exponent, which would favour the worst samples).
 *   - r is the 2-norm of the full stacked residual; c_1 the summed squared
 *     acceleration; c_aug = c_1 + r.
 */
#include "priest_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ----------------------------------------------------------------------- */
/* Bernstein basis (eq. parametrized; the paper says only "polynomial";     */
/* Bernstein of the stated degree is used).                                 */
/* ----------------------------------------------------------------------- */

static double binom(int n, int k)
{
    double c = 1.0;
    int i;
    if (k < 0 || k > n) return 0.0;
    for (i = 1; i <= k; ++i) c = c * (double)(n - k + i) / (double)i;
    return c;
}

static double ipow(double x, int e)
{
    double p = 1.0;
    int i;
    for (i = 0; i < e; ++i) p *= x;
    return p;
}

/* B_{j,m}(tau) = C(m, j) tau^j (1 - tau)^(m - j); zero outside 0 <= j <= m. */
static double bern(int m, int j, double tau)
{
    if (m < 0 || j < 0 || j > m) return 0.0;
    return binom(m, j) * ipow(tau, j) * ipow(1.0 - tau, m - j);
}

int orc_basis(int degree, int n_p, double horizon, double *P, double *Pd, double *Pdd)
{
    int n = degree, nv = degree + 1, k, j;
    if (degree < 2 || n_p < 2 || !(horizon > 0.0)) return -1;
    for (k = 0; k < n_p; ++k) {
        double tau = (double)k / (double)(n_p - 1);
        for (j = 0; j < nv; ++j) {
            /* d/dtau B_{j,n} = n (B_{j-1,n-1} - B_{j,n-1});
             * d2/dtau2 B_{j,n} = n (n-1) (B_{j-2,n-2} - 2 B_{j-1,n-2} + B_{j,n-2});
             * dt = T_h dtau. */
            double d1 = n * (bern(n - 1, j - 1, tau) - bern(n - 1, j, tau));
            double d2 = n * (n - 1) *
                        (bern(n - 2, j - 2, tau) - 2.0 * bern(n - 2, j - 1, tau) + bern(n - 2, j, tau));
            P[k * nv + j] = bern(n, j, tau);
            Pd[k * nv + j] = d1 / horizon;
            Pdd[k * nv + j] = d2 / (horizon * horizon);
        }
    }
    return 0;
}

/* ----------------------------------------------------------------------- */
/* Problem checks and the equality block A xi = b_eq (Sec. II-A.2).         */
/* ----------------------------------------------------------------------- */

static int check_problem(const orc_problem *pr)
{
    int j;
    if (!pr) return -1;
    if (pr->dims != 2 && pr->dims != 3) return -1;
    if (pr->degree < 5 || pr->degree > 15) return -1;
    if (pr->n_p < 2) return -1;
    if (!(pr->horizon > 0.0) || !(pr->rho > 0.0)) return -1;
    if (!(pr->vmax > 0.0) || !(pr->amax > 0.0)) return -1;
    if (pr->n_obs < 0) return -1;
    if (pr->bc_final_mask < 0 || pr->bc_final_mask > 7) return -1;
    if (pr->n_obs > 0 && (!pr->center || !pr->vel || !pr->semi)) return -1;
    for (j = 0; j < pr->n_obs; ++j) {
        if (!(pr->semi[2 * j] > 0.0)) return -1;
        if (pr->dims == 3 && !(pr->semi[2 * j + 1] > 0.0)) return -1;
    }
    return 0;
}

static int n_eq_rows(const orc_problem *pr)
{
    int q, n = 3;
    for (q = 0; q < 3; ++q)
        if (pr->bc_final_mask & (1 << q)) ++n;
    return n;
}

int orc_equality(const orc_problem *pr, double *A, double *b)
{
    int nv, np, neq, row, q, j, ax;
    double *P, *Pd, *Pdd;
    const double *rows0[3], *rowsf[3];
    if (check_problem(pr)) return -1;
    nv = pr->degree + 1;
    np = pr->n_p;
    neq = n_eq_rows(pr);
    P = (double *)malloc(sizeof(double) * np * nv * 3);
    if (!P) return -2;
    Pd = P + np * nv;
    Pdd = Pd + np * nv;
    orc_basis(pr->degree, np, pr->horizon, P, Pd, Pdd);
    /* first rows: P_0, Pd_0, Pdd_0; last rows: P_{-1}, Pd_{-1}, Pdd_{-1} */
    rows0[0] = P;
    rows0[1] = Pd;
    rows0[2] = Pdd;
    rowsf[0] = P + (np - 1) * nv;
    rowsf[1] = Pd + (np - 1) * nv;
    rowsf[2] = Pdd + (np - 1) * nv;
    row = 0;
    for (q = 0; q < 3; ++q, ++row) {
        for (j = 0; j < nv; ++j) A[row * nv + j] = rows0[q][j];
        for (ax = 0; ax < pr->dims; ++ax) b[ax * neq + row] = pr->b0[ax][q];
    }
    for (q = 0; q < 3; ++q) {
        if (!(pr->bc_final_mask & (1 << q))) continue;
        for (j = 0; j < nv; ++j) A[row * nv + j] = rowsf[q][j];
        for (ax = 0; ax < pr->dims; ++ax) b[ax * neq + row] = pr->bf[ax][q];
        ++row;
    }
    free(P);
    return neq;
}

/* ----------------------------------------------------------------------- */
/* KKT matrix of eq. matrix_vec, per axis.  F (eq. f_e, and G of eq.        */
/* bound_con) is block diagonal over the axes with the same block, so every */
/* axis has the same KKT matrix.  F^T F is summed over the stacked blocks:  */
/* n_obs copies of P (F_o), then Pd, Pdd, then -P and P for the bounds.     */
/* ----------------------------------------------------------------------- */

static void add_gram(int np, int nv, const double *B, double sign_sq, double *H)
{
    int i, j, t;
    for (i = 0; i < nv; ++i)
        for (j = 0; j < nv; ++j) {
            double s = 0.0;
            for (t = 0; t < np; ++t) s += B[t * nv + i] * B[t * nv + j];
            H[i * nv + j] += sign_sq * s;
        }
}

int orc_kkt_matrix(const orc_problem *pr, double *K)
{
    int nv, np, neq, n, i, j, o;
    double *P, *Pd, *Pdd, *A, *b, *FtF;
    if (check_problem(pr)) return -1;
    nv = pr->degree + 1;
    np = pr->n_p;
    neq = n_eq_rows(pr);
    n = nv + neq;
    P = (double *)malloc(sizeof(double) * (np * nv * 3 + neq * nv + 3 * neq + nv * nv));
    if (!P) return -2;
    Pd = P + np * nv;
    Pdd = Pd + np * nv;
    A = Pdd + np * nv;
    b = A + neq * nv;
    FtF = b + 3 * neq;
    orc_basis(pr->degree, np, pr->horizon, P, Pd, Pdd);
    orc_equality(pr, A, b);
    memset(FtF, 0, sizeof(double) * nv * nv);
    for (o = 0; o < pr->n_obs; ++o) add_gram(np, nv, P, 1.0, FtF); /* F_o: P stacked n_obs times */
    add_gram(np, nv, Pd, 1.0, FtF);
    add_gram(np, nv, Pdd, 1.0, FtF);
    if (pr->use_bounds) {
        add_gram(np, nv, P, 1.0, FtF); /* (-P)^T (-P) */
        add_gram(np, nv, P, 1.0, FtF); /* P^T P */
    }
    for (i = 0; i < n * n; ++i) K[i] = 0.0;
    for (i = 0; i < nv; ++i)
        for (j = 0; j < nv; ++j) K[i * n + j] = (i == j ? 1.0 : 0.0) + pr->rho * FtF[i * nv + j];
    for (i = 0; i < neq; ++i)
        for (j = 0; j < nv; ++j) {
            K[(nv + i) * n + j] = A[i * nv + j];
            K[j * n + (nv + i)] = A[i * nv + j];
        }
    free(P);
    return n;
}

/* LU factorisation with partial pivoting, in place; perm records row swaps. */
static int lu_factor(int n, double *M, int *perm)
{
    int i, j, k;
    for (i = 0; i < n; ++i) perm[i] = i;
    for (k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(M[k * n + k]);
        for (i = k + 1; i < n; ++i)
            if (fabs(M[i * n + k]) > best) {
                best = fabs(M[i * n + k]);
                p = i;
            }
        if (!(best > 0.0)) return -6;
        if (p != k) {
            int tmp = perm[k];
            perm[k] = perm[p];
            perm[p] = tmp;
            for (j = 0; j < n; ++j) {
                double t = M[k * n + j];
                M[k * n + j] = M[p * n + j];
                M[p * n + j] = t;
            }
        }
        for (i = k + 1; i < n; ++i) {
            double f = M[i * n + k] / M[k * n + k];
            M[i * n + k] = f;
            for (j = k + 1; j < n; ++j) M[i * n + j] -= f * M[k * n + j];
        }
    }
    return 0;
}

static void lu_solve(int n, const double *LU, const int *perm, const double *rhs, double *x)
{
    int i, j;
    double *y = (double *)malloc(sizeof(double) * n);
    for (i = 0; i < n; ++i) {
        double s = rhs[perm[i]];
        for (j = 0; j < i; ++j) s -= LU[i * n + j] * y[j];
        y[i] = s;
    }
    for (i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (j = i + 1; j < n; ++j) s -= LU[i * n + j] * x[j];
        x[i] = s / LU[i * n + i];
    }
    free(y);
}

/* ----------------------------------------------------------------------- */
/* Closed-form alpha / beta / d updates (Appendix).                         */
/* ----------------------------------------------------------------------- */

void orc_obstacle_polar(int dims, const double *pos, const double *o, double a, double b,
                        double *alpha, double *beta, double *d, double *e)
{
    double dx = pos[0] - o[0], dy = pos[1] - o[1], dz = (dims == 3) ? pos[2] - o[2] : 0.0;
    double al, be, ux, uy, uz, dd;
    /* eq. comp_alpha: the xy cross-section is a circle of radius a, so the
     * minimising azimuth is the line-of-sight angle. */
    al = atan2(dy, dx);
    if (dims == 3) {
        /* eq. comp_beta, axis-scaled frame. */
        be = atan2(sqrt(dx * dx + dy * dy) / a, dz / b);
        ux = a * cos(al) * sin(be);
        uy = a * sin(al) * sin(be);
        uz = b * cos(be);
    } else {
        be = 0.5 * ORC_PI;
        ux = a * cos(al);
        uy = a * sin(al);
        uz = 0.0;
    }
    /* eq. comp_d: minimise || Delta - d u ||^2 over d, then clip to d >= 1
     * (d_min = 1, d_max = inf for obstacle blocks). */
    dd = (ux * dx + uy * dy + uz * dz) / (ux * ux + uy * uy + uz * uz);
    if (dd < 1.0) dd = 1.0;
    *alpha = al;
    *beta = be;
    *d = dd;
    e[0] = o[0] + dd * ux;
    e[1] = o[1] + dd * uy;
    if (dims == 3) e[2] = o[2] + dd * uz;
}

void orc_bound_polar(int dims, const double *v, double vmax,
                     double *alpha, double *beta, double *d, double *e)
{
    double al, be, ux, uy, uz, dd;
    al = atan2(v[1], v[0]);
    if (dims == 3) {
        be = atan2(sqrt(v[0] * v[0] + v[1] * v[1]), v[2]);
        ux = vmax * cos(al) * sin(be);
        uy = vmax * sin(al) * sin(be);
        uz = vmax * cos(be);
    } else {
        be = 0.5 * ORC_PI;
        ux = vmax * cos(al);
        uy = vmax * sin(al);
        uz = 0.0;
    }
    dd = (ux * v[0] + uy * v[1] + (dims == 3 ? uz * v[2] : 0.0)) / (ux * ux + uy * uy + uz * uz);
    if (dd < 0.0) dd = 0.0; /* d_min = 0 */
    if (dd > 1.0) dd = 1.0; /* d_max = 1 */
    *alpha = al;
    *beta = be;
    *d = dd;
    e[0] = dd * ux;
    e[1] = dd * uy;
    if (dims == 3) e[2] = dd * uz;
}

/* ----------------------------------------------------------------------- */
/* Projection: alternating minimisation (Appendix eqs. comp_alpha..zeta).   */
/* ----------------------------------------------------------------------- */

typedef struct {
    int dims, nv, np, neq, nk, no;
    double *P, *Pd, *Pdd, *A, *b, *KLU, *tk;
    int *perm;
} orc_ws;

static int ws_init(const orc_problem *pr, orc_ws *w)
{
    int i;
    memset(w, 0, sizeof(*w));
    if (check_problem(pr)) return -1;
    w->dims = pr->dims;
    w->nv = pr->degree + 1;
    w->np = pr->n_p;
    w->neq = n_eq_rows(pr);
    w->nk = w->nv + w->neq;
    w->no = pr->n_obs;
    w->P = (double *)malloc(sizeof(double) * (3 * w->np * w->nv + w->neq * w->nv + 3 * w->neq +
                                              w->nk * w->nk + w->np));
    w->perm = (int *)malloc(sizeof(int) * w->nk);
    if (!w->P || !w->perm) return -2;
    w->Pd = w->P + w->np * w->nv;
    w->Pdd = w->Pd + w->np * w->nv;
    w->A = w->Pdd + w->np * w->nv;
    w->b = w->A + w->neq * w->nv;
    w->KLU = w->b + 3 * w->neq;
    w->tk = w->KLU + w->nk * w->nk;
    orc_basis(pr->degree, w->np, pr->horizon, w->P, w->Pd, w->Pdd);
    orc_equality(pr, w->A, w->b);
    orc_kkt_matrix(pr, w->KLU);
    if (lu_factor(w->nk, w->KLU, w->perm)) return -6;
    for (i = 0; i < w->np; ++i) w->tk[i] = pr->horizon * (double)i / (double)(w->np - 1);
    return 0;
}

static void ws_free(orc_ws *w)
{
    free(w->P);
    free(w->perm);
}

/* Solve the per-axis KKT system [[H, A^T], [A, 0]] [c; nu] = [rhs; b_axis]. */
static void kkt_solve_axis(const orc_ws *w, int ax, const double *rhs, double *c)
{
    int i;
    double *r = (double *)malloc(sizeof(double) * 2 * w->nk);
    double *x = r + w->nk;
    for (i = 0; i < w->nv; ++i) r[i] = rhs[i];
    for (i = 0; i < w->neq; ++i) r[w->nv + i] = w->b[ax * w->neq + i];
    lu_solve(w->nk, w->KLU, w->perm, r, x);
    for (i = 0; i < w->nv; ++i) c[i] = x[i];
    free(r);
}

/* Pi_A: min 1/2 ||c - xi||^2 s.t. A c = b, per axis, via [[I, A^T], [A, 0]]. */
static void project_eq_axis(const orc_ws *w, int ax, const double *xi, double *c)
{
    int n = w->nv + w->neq, i, j;
    double *M = (double *)malloc(sizeof(double) * (n * n + 2 * n));
    double *r = M + n * n, *x = r + n;
    int *perm = (int *)malloc(sizeof(int) * n);
    for (i = 0; i < n * n; ++i) M[i] = 0.0;
    for (i = 0; i < w->nv; ++i) M[i * n + i] = 1.0;
    for (i = 0; i < w->neq; ++i)
        for (j = 0; j < w->nv; ++j) {
            M[(w->nv + i) * n + j] = w->A[i * w->nv + j];
            M[j * n + (w->nv + i)] = w->A[i * w->nv + j];
        }
    lu_factor(n, M, perm);
    for (i = 0; i < w->nv; ++i) r[i] = xi[i];
    for (i = 0; i < w->neq; ++i) r[w->nv + i] = w->b[ax * w->neq + i];
    lu_solve(n, M, perm, r, x);
    for (i = 0; i < w->nv; ++i) c[i] = x[i];
    free(M);
    free(perm);
}

/* Position / velocity / acceleration of every axis at every time stamp. */
static void eval_traj(const orc_ws *w, const double *c, double *pos, double *vel, double *acc)
{
    int ax, t, j;
    for (ax = 0; ax < w->dims; ++ax)
        for (t = 0; t < w->np; ++t) {
            double p = 0.0, v = 0.0, a = 0.0;
            for (j = 0; j < w->nv; ++j) {
                double cj = c[ax * w->nv + j];
                p += w->P[t * w->nv + j] * cj;
                v += w->Pd[t * w->nv + j] * cj;
                a += w->Pdd[t * w->nv + j] * cj;
            }
            pos[t * 3 + ax] = p;
            vel[t * 3 + ax] = v;
            acc[t * 3 + ax] = a;
        }
}

/* One AM iteration for one sample: xb (xi_bar^k -> xi_bar^{k+1}) and lam
 * (lambda^k -> lambda^{k+1}) in place. */
static void am_iteration(const orc_problem *pr, const orc_ws *w, const double *xi, double *xb,
                         double *lam, double *scratch)
{
    int dims = w->dims, nv = w->nv, np = w->np, no = w->no;
    int t, j, ax, col;
    double *pos = scratch, *vel = pos + 3 * np, *acc = vel + 3 * np;
    double *eo = acc + 3 * np;      /* n_obs x np x 3 obstacle targets */
    double *ev = eo + 3 * np * no;  /* np x 3 */
    double *ea = ev + 3 * np;       /* np x 3 */
    double *elo = ea + 3 * np;      /* np x 3 bound targets, rows -P */
    double *ehi = elo + 3 * np;     /* np x 3 bound targets, rows +P */
    double rhs[16];
    double al, be, dd, o[3], e[3];

    eval_traj(w, xb, pos, vel, acc);

    /* alpha, beta, d and the rebuilt e^{k+1} (eqs. comp_alpha..comp_d, obtain_e) */
    for (j = 0; j < no; ++j)
        for (t = 0; t < np; ++t) {
            for (ax = 0; ax < dims; ++ax)
                o[ax] = pr->center[j * dims + ax] + pr->vel[j * dims + ax] * w->tk[t];
            orc_obstacle_polar(dims, pos + 3 * t, o, pr->semi[2 * j], pr->semi[2 * j + 1], &al, &be,
                               &dd, e);
            for (ax = 0; ax < dims; ++ax) eo[(j * np + t) * 3 + ax] = e[ax];
        }
    for (t = 0; t < np; ++t) {
        orc_bound_polar(dims, vel + 3 * t, pr->vmax, &al, &be, &dd, ev + 3 * t);
        orc_bound_polar(dims, acc + 3 * t, pr->amax, &al, &be, &dd, ea + 3 * t);
    }
    if (pr->use_bounds) {
        /* s^{k+1} = max(0, -G xi_bar^k + tau), e_b = tau - s; G = [-P; P],
         * tau = [-s_min; s_max] (Appendix, slack step and eq. obtain_e). */
        for (t = 0; t < np; ++t)
            for (ax = 0; ax < dims; ++ax) {
                double x = pos[3 * t + ax];
                double s_lo = (-pr->smin[ax]) - (-x);
                double s_hi = pr->smax[ax] - x;
                if (s_lo < 0.0) s_lo = 0.0;
                if (s_hi < 0.0) s_hi = 0.0;
                elo[3 * t + ax] = -pr->smin[ax] - s_lo;
                ehi[3 * t + ax] = pr->smax[ax] - s_hi;
            }
    }

    for (ax = 0; ax < dims; ++ax) {
        /* eq. lag: lambda^{k+1} = lambda^k - rho F^T (F xi_bar^k - e^{k+1}),
         * F^T applied block by block over the stacked rows of eq. f_e. */
        for (col = 0; col < nv; ++col) {
            double g = 0.0, fte = 0.0;
            for (j = 0; j < no; ++j)
                for (t = 0; t < np; ++t) {
                    double f = w->P[t * nv + col];
                    g += f * (pos[3 * t + ax] - eo[(j * np + t) * 3 + ax]);
                    fte += f * eo[(j * np + t) * 3 + ax];
                }
            for (t = 0; t < np; ++t) {
                g += w->Pd[t * nv + col] * (vel[3 * t + ax] - ev[3 * t + ax]);
                fte += w->Pd[t * nv + col] * ev[3 * t + ax];
                g += w->Pdd[t * nv + col] * (acc[3 * t + ax] - ea[3 * t + ax]);
                fte += w->Pdd[t * nv + col] * ea[3 * t + ax];
            }
            if (pr->use_bounds)
                for (t = 0; t < np; ++t) {
                    double f = w->P[t * nv + col];
                    g += (-f) * ((-pos[3 * t + ax]) - elo[3 * t + ax]);
                    fte += (-f) * elo[3 * t + ax];
                    g += f * (pos[3 * t + ax] - ehi[3 * t + ax]);
                    fte += f * ehi[3 * t + ax];
                }
            lam[ax * nv + col] -= pr->rho * g;
            /* eta of eq. matrix_vec: xi + lambda^{k+1} + rho F^T e^{k+1} */
            rhs[col] = xi[ax * nv + col] + lam[ax * nv + col] + pr->rho * fte;
        }
        /* eq. comp_zeta / affine_trans: the shared equality-constrained QP. */
        kkt_solve_axis(w, ax, rhs, xb + ax * nv);
    }
}

int orc_project_eq(const orc_problem *pr, int N, const double *xi, double *out)
{
    orc_ws w;
    int i, ax, D, rc = ws_init(pr, &w);
    if (rc) {
        ws_free(&w);
        return rc;
    }
    D = w.dims * w.nv;
    for (i = 0; i < N; ++i)
        for (ax = 0; ax < w.dims; ++ax)
            project_eq_axis(&w, ax, xi + (size_t)i * D + ax * w.nv, out + (size_t)i * D + ax * w.nv);
    ws_free(&w);
    return 0;
}

int orc_project(const orc_problem *pr, int K, int N, const double *xi, const double *xi_bar0,
                double *lambda_io, double *xi_bar_out)
{
    orc_ws w;
    int i, k, ax, D, rc = ws_init(pr, &w);
    double *scratch, *lam;
    if (rc || K < 0 || N < 0) {
        ws_free(&w);
        return rc ? rc : -1;
    }
    D = w.dims * w.nv;
    scratch = (double *)malloc(sizeof(double) * (3 * w.np * (7 + w.no) + 16));
    lam = (double *)malloc(sizeof(double) * (D + 1));
    if (!scratch || !lam) {
        free(scratch);
        free(lam);
        ws_free(&w);
        return -2;
    }
    for (i = 0; i < N; ++i) {
        const double *x = xi + (size_t)i * D;
        double *xb = xi_bar_out + (size_t)i * D;
        int d;
        if (xi_bar0)
            for (d = 0; d < D; ++d) xb[d] = xi_bar0[(size_t)i * D + d];
        else
            for (ax = 0; ax < w.dims; ++ax) project_eq_axis(&w, ax, x + ax * w.nv, xb + ax * w.nv);
        for (d = 0; d < D; ++d) lam[d] = lambda_io ? lambda_io[(size_t)i * D + d] : 0.0;
        for (k = 0; k < K; ++k) am_iteration(pr, &w, x, xb, lam, scratch);
        if (lambda_io)
            for (d = 0; d < D; ++d) lambda_io[(size_t)i * D + d] = lam[d];
    }
    free(scratch);
    free(lam);
    ws_free(&w);
    return 0;
}

/* ----------------------------------------------------------------------- */
/* Residual and cost (Alg. 1 lines "compute the residuals", "evaluate").    */
/* ----------------------------------------------------------------------- */

/* c_1 contribution of one time stamp.  Point-to-point benchmark: |a|^2.
 * BARN-style cost (acceleration, curvature and path-following penalties):
 * w_acc |a|^2 + w_curv kappa^2 + w_path d^2, kappa = |v x a| /
 * (|v|^2 + eps^2)^(3/2) (the curvature of the path, regularised where the
 * robot is at rest), d = distance from the point to its projection on the
 * straight start-goal segment (clamped to the segment). */
static double point_cost(const orc_problem *pr, int dims, const double *p, const double *v, const double *a)
{
    double a2 = 0.0, v2 = 0.0, c2, den, s[3] = {0, 0, 0}, u[3] = {0, 0, 0}, len = 0.0, lam = 0.0, d2 = 0.0;
    int ax;
    for (ax = 0; ax < dims; ++ax) {
        a2 += a[ax] * a[ax];
        v2 += v[ax] * v[ax];
    }
    if (pr->cost_kind != 1) return a2;
    /* |v x a|^2 */
    if (dims == 2) {
        const double cz = v[0] * a[1] - v[1] * a[0];
        c2 = cz * cz;
    } else {
        const double cx = v[1] * a[2] - v[2] * a[1], cy = v[2] * a[0] - v[0] * a[2], cz = v[0] * a[1] - v[1] * a[0];
        c2 = cx * cx + cy * cy + cz * cz;
    }
    den = v2 + pr->curv_eps * pr->curv_eps;
    /* kappa^2 = |v x a|^2 / den^3 */
    for (ax = 0; ax < dims; ++ax) {
        s[ax] = pr->b0[ax][0];
        u[ax] = pr->bf[ax][0] - pr->b0[ax][0];
        len += u[ax] * u[ax];
    }
    len = sqrt(len);
    if (len > 0.0) {
        for (ax = 0; ax < dims; ++ax) {
            u[ax] /= len;
            lam += (p[ax] - s[ax]) * u[ax];
        }
        if (lam < 0.0) lam = 0.0;
        if (lam > len) lam = len;
    }
    for (ax = 0; ax < dims; ++ax) {
        const double e = p[ax] - s[ax] - lam * u[ax];
        d2 += e * e;
    }
    return pr->w_acc * a2 + pr->w_curv * c2 / (den * den * den) + pr->w_path * d2;
}

int orc_residual_cost(const orc_problem *pr, int N, const double *xi_bar, double *r, double *c1)
{
    orc_ws w;
    int i, j, t, ax, D, rc = ws_init(pr, &w);
    double *pos, *vel, *acc;
    if (rc) {
        ws_free(&w);
        return rc;
    }
    D = w.dims * w.nv;
    pos = (double *)malloc(sizeof(double) * 9 * w.np);
    vel = pos + 3 * w.np;
    acc = vel + 3 * w.np;
    for (i = 0; i < N; ++i) {
        double r2 = 0.0, cost = 0.0;
        eval_traj(&w, xi_bar + (size_t)i * D, pos, vel, acc);
        for (t = 0; t < w.np; ++t) {
            double v2 = 0.0, a2 = 0.0, nv_, na_;
            /* obstacle blocks: residual = Delta (1 - d / rho_s) with
             * d = max(1, rho_s); norm = max(0, 1/rho_s - 1) ||Delta||. */
            for (j = 0; j < w.no; ++j) {
                double dl[3] = {0.0, 0.0, 0.0}, rs2 = 0.0, n2 = 0.0, a = pr->semi[2 * j],
                       b = pr->semi[2 * j + 1];
                for (ax = 0; ax < w.dims; ++ax) {
                    double o = pr->center[j * w.dims + ax] + pr->vel[j * w.dims + ax] * w.tk[t];
                    double s = (ax == 2) ? b : a;
                    dl[ax] = pos[3 * t + ax] - o;
                    rs2 += (dl[ax] / s) * (dl[ax] / s);
                    n2 += dl[ax] * dl[ax];
                }
                if (rs2 >= 1.0) continue;
                if (rs2 == 0.0) {
                    /* degenerate direction: alpha = beta = 0 -> target on +x (2-D) / +z (3-D) */
                    double s = (w.dims == 3) ? b : a;
                    r2 += s * s;
                } else {
                    double f = 1.0 / sqrt(rs2) - 1.0;
                    r2 += f * f * n2;
                }
            }
            for (ax = 0; ax < w.dims; ++ax) {
                v2 += vel[3 * t + ax] * vel[3 * t + ax];
                a2 += acc[3 * t + ax] * acc[3 * t + ax];
            }
            nv_ = sqrt(v2);
            na_ = sqrt(a2);
            if (nv_ > pr->vmax) r2 += (nv_ - pr->vmax) * (nv_ - pr->vmax);
            if (na_ > pr->amax) r2 += (na_ - pr->amax) * (na_ - pr->amax);
            if (pr->use_bounds)
                for (ax = 0; ax < w.dims; ++ax) {
                    double x = pos[3 * t + ax];
                    if (x < pr->smin[ax]) r2 += (pr->smin[ax] - x) * (pr->smin[ax] - x);
                    if (x > pr->smax[ax]) r2 += (x - pr->smax[ax]) * (x - pr->smax[ax]);
                }
            cost += point_cost(pr, w.dims, pos + 3 * t, vel + 3 * t, acc + 3 * t);
        }
        if (r) r[i] = sqrt(r2);
        if (c1) c1[i] = cost;
    }
    free(pos);
    ws_free(&w);
    return 0;
}

int orc_residual_stacked(const orc_problem *pr, int N, const double *xi_bar, double *r)
{
    orc_ws w;
    int i, j, t, ax, D, rc = ws_init(pr, &w);
    double *pos, *vel, *acc, al, be, dd, o[3], e[3];
    if (rc) {
        ws_free(&w);
        return rc;
    }
    D = w.dims * w.nv;
    pos = (double *)malloc(sizeof(double) * 9 * w.np);
    vel = pos + 3 * w.np;
    acc = vel + 3 * w.np;
    for (i = 0; i < N; ++i) {
        double r2 = 0.0;
        eval_traj(&w, xi_bar + (size_t)i * D, pos, vel, acc);
        for (t = 0; t < w.np; ++t) {
            for (j = 0; j < w.no; ++j) {
                for (ax = 0; ax < w.dims; ++ax)
                    o[ax] = pr->center[j * w.dims + ax] + pr->vel[j * w.dims + ax] * w.tk[t];
                orc_obstacle_polar(w.dims, pos + 3 * t, o, pr->semi[2 * j], pr->semi[2 * j + 1],
                                   &al, &be, &dd, e);
                for (ax = 0; ax < w.dims; ++ax)
                    r2 += (pos[3 * t + ax] - e[ax]) * (pos[3 * t + ax] - e[ax]);
            }
            orc_bound_polar(w.dims, vel + 3 * t, pr->vmax, &al, &be, &dd, e);
            for (ax = 0; ax < w.dims; ++ax) r2 += (vel[3 * t + ax] - e[ax]) * (vel[3 * t + ax] - e[ax]);
            orc_bound_polar(w.dims, acc + 3 * t, pr->amax, &al, &be, &dd, e);
            for (ax = 0; ax < w.dims; ++ax) r2 += (acc[3 * t + ax] - e[ax]) * (acc[3 * t + ax] - e[ax]);
            if (pr->use_bounds)
                for (ax = 0; ax < w.dims; ++ax) {
                    double x = pos[3 * t + ax];
                    double s_lo = x - pr->smin[ax], s_hi = pr->smax[ax] - x;
                    double res_lo, res_hi;
                    if (s_lo < 0.0) s_lo = 0.0;
                    if (s_hi < 0.0) s_hi = 0.0;
                    /* G xi - (tau - s) for the -P and +P rows */
                    res_lo = (-x) - (-pr->smin[ax] - s_lo);
                    res_hi = x - (pr->smax[ax] - s_hi);
                    r2 += res_lo * res_lo + res_hi * res_hi;
                }
        }
        r[i] = sqrt(r2);
    }
    free(pos);
    ws_free(&w);
    return 0;
}

/* ----------------------------------------------------------------------- */
/* Selections (Alg. 1): sort by (key, index) ascending.                     */
/* ----------------------------------------------------------------------- */

typedef struct {
    double key;
    int idx;
} keyed;

static int keyed_cmp(const void *pa, const void *pb)
{
    const keyed *a = (const keyed *)pa, *b = (const keyed *)pb;
    /* NaN keys order after every number */
    int na = isnan(a->key), nb = isnan(b->key);
    if (na != nb) return na - nb;
    if (!na && a->key < b->key) return -1;
    if (!na && a->key > b->key) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

int orc_select(int N, const double *r, const double *c_aug, int n_proj, int n_elite,
               int *proj_idx, int *elite_idx)
{
    keyed *k;
    int i;
    if (N <= 0 || n_proj <= 0 || n_proj > N || n_elite <= 0 || n_elite > n_proj) return -1;
    k = (keyed *)malloc(sizeof(keyed) * N);
    for (i = 0; i < N; ++i) {
        k[i].key = r[i];
        k[i].idx = i;
    }
    qsort(k, N, sizeof(keyed), keyed_cmp);
    if (proj_idx)
        for (i = 0; i < n_proj; ++i) proj_idx[i] = k[i].idx;
    for (i = 0; i < n_proj; ++i) k[i].key = c_aug[k[i].idx];
    qsort(k, n_proj, sizeof(keyed), keyed_cmp);
    for (i = 0; i < n_elite; ++i) elite_idx[i] = k[i].idx;
    free(k);
    return 0;
}

/* ----------------------------------------------------------------------- */
/* Distribution update (eqs. update_mean, update_covariance).               */
/* ----------------------------------------------------------------------- */

int orc_refit(int D, int n_elite, const double *elites, const double *c_aug,
              double sigma_lr, double gamma, double *mu, double *cov)
{
    int m, i, j;
    double delta, sw = 0.0;
    double *w, *mnew;
    if (D <= 0 || n_elite <= 0 || !(gamma > 0.0)) return -1;
    w = (double *)malloc(sizeof(double) * (n_elite + D));
    mnew = w + n_elite;
    delta = c_aug[0];
    for (m = 1; m < n_elite; ++m)
        if (c_aug[m] < delta) delta = c_aug[m];
    for (m = 0; m < n_elite; ++m) {
        w[m] = exp(-(c_aug[m] - delta) / gamma);
        sw += w[m];
    }
    for (i = 0; i < D; ++i) {
        double s = 0.0;
        for (m = 0; m < n_elite; ++m) s += w[m] * elites[(size_t)m * D + i];
        mnew[i] = (1.0 - sigma_lr) * mu[i] + sigma_lr * s / sw;
    }
    for (i = 0; i < D; ++i)
        for (j = 0; j < D; ++j) {
            double s = 0.0;
            for (m = 0; m < n_elite; ++m)
                s += w[m] * (elites[(size_t)m * D + i] - mnew[i]) * (elites[(size_t)m * D + j] - mnew[j]);
            cov[i * D + j] = (1.0 - sigma_lr) * cov[i * D + j] + sigma_lr * s / sw;
        }
    for (i = 0; i < D; ++i) mu[i] = mnew[i];
    free(w);
    return 0;
}

int orc_cholesky(int D, const double *S, double *L)
{
    int i, j, k;
    for (i = 0; i < D * D; ++i) L[i] = 0.0;
    for (j = 0; j < D; ++j) {
        double s = S[j * D + j];
        for (k = 0; k < j; ++k) s -= L[j * D + k] * L[j * D + k];
        if (!(s > 0.0)) return -6;
        L[j * D + j] = sqrt(s);
        for (i = j + 1; i < D; ++i) {
            double t = S[i * D + j];
            for (k = 0; k < j; ++k) t -= L[i * D + k] * L[j * D + k];
            L[i * D + j] = t / L[j * D + j];
        }
    }
    return 0;
}

/* ----------------------------------------------------------------------- */
/* Host Gaussian stream.  SplitMix64 (Steele, Lea, Flood, OOPSLA 2014):     */
/* state += 0x9E3779B97F4A7C15, output = the published 64-bit finaliser.    */
/* Uniform u = (x >> 11) * 2^-53 in [0, 1); Box-Muller on (1 - u1, u2).     */
/* ----------------------------------------------------------------------- */

static uint64_t sm64_next(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void orc_rng_normal(uint64_t seed, int64_t count, double *out)
{
    uint64_t s = seed;
    int64_t i = 0;
    while (i < count) {
        double u1 = (double)(sm64_next(&s) >> 11) * (1.0 / 9007199254740992.0);
        double u2 = (double)(sm64_next(&s) >> 11) * (1.0 / 9007199254740992.0);
        double rad = sqrt(-2.0 * log(1.0 - u1));
        double th = 2.0 * ORC_PI * u2;
        out[i++] = rad * cos(th);
        if (i < count) out[i++] = rad * sin(th);
    }
}

int orc_default_mean(const orc_problem *pr, double *mu)
{
    int ax, k, nv;
    if (check_problem(pr)) return -1;
    nv = pr->degree + 1;
    for (ax = 0; ax < pr->dims; ++ax)
        for (k = 0; k < nv; ++k)
            mu[ax * nv + k] = pr->b0[ax][0] + (pr->bf[ax][0] - pr->b0[ax][0]) * (double)k / (double)pr->degree;
    return 0;
}

/* ----------------------------------------------------------------------- */
/* Alg. 1.                                                                  */
/* ----------------------------------------------------------------------- */

int orc_plan(const orc_problem *pr, const orc_cem *cem, const double *mu0, const double *cov0,
             const double *z, uint64_t seed, double *best, double *best_r, double *best_caug,
             double *mu_out, double *cov_out, int *elite_out)
{
    return orc_plan_warm(pr, cem, mu0, cov0, NULL, z, seed, best, best_r, best_caug, mu_out, cov_out, elite_out,
                         NULL);
}

int orc_plan_warm(const orc_problem *pr, const orc_cem *cem, const double *mu0, const double *cov0,
                  const double *lam0, const double *z, uint64_t seed, double *best, double *best_r,
                  double *best_caug, double *mu_out, double *cov_out, int *elite_out, double *lam_out)
{
    int D, N, L, l, i, j, k, rc;
    double *mu, *cov, *Lc, *Sh, *xi, *xb, *r, *c1, *caug, *zz = NULL, *el, *elc, *lam;
    int *eidx;
    if (check_problem(pr) || !cem) return -1;
    N = cem->n_samples;
    L = cem->cem_iters;
    if (N <= 0 || L <= 0 || cem->proj_iters < 0 || cem->n_proj <= 0 || cem->n_proj > N ||
        cem->n_elite <= 0 || cem->n_elite > cem->n_proj)
        return -1;
    D = pr->dims * (pr->degree + 1);
    mu = (double *)malloc(sizeof(double) * (2 * D + 3 * D * D + 3 * (size_t)N * D + 3 * N +
                                            (size_t)cem->n_elite * (D + 1)));
    eidx = (int *)malloc(sizeof(int) * cem->n_elite);
    if (!mu || !eidx) return -2;
    cov = mu + D;
    Lc = cov + D * D;
    Sh = Lc + D * D;
    xi = Sh + D * D;
    xb = xi + (size_t)N * D;
    r = xb + (size_t)N * D;
    c1 = r + N;
    caug = c1 + N;
    el = caug + N;
    elc = el + (size_t)cem->n_elite * D;
    lam = elc + cem->n_elite;
    if (mu0)
        for (i = 0; i < D; ++i) mu[i] = mu0[i];
    else
        orc_default_mean(pr, mu);
    for (i = 0; i < D * D; ++i) cov[i] = cov0 ? cov0[i] : 0.0;
    if (!cov0)
        for (i = 0; i < D; ++i) cov[i * D + i] = cem->init_std * cem->init_std;
    if (!z) {
        zz = (double *)malloc(sizeof(double) * (size_t)L * N * D);
        orc_rng_normal(seed, (int64_t)L * N * D, zz);
        z = zz;
    }
    rc = 0;
    for (l = 0; l < L && rc == 0; ++l) {
        /* Alg. 1: draw N_b samples from N(mu, Sigma) through a Cholesky factor
         * of Sigma + eps I (eps relative to the mean variance). */
        double tr = 0.0, eps;
        for (i = 0; i < D; ++i) tr += cov[i * D + i];
        eps = cem->chol_eps * tr / (double)D;
        for (i = 0; i < D * D; ++i) Sh[i] = cov[i];
        for (i = 0; i < D; ++i) Sh[i * D + i] += eps;
        rc = orc_cholesky(D, Sh, Lc);
        if (rc) break;
        for (i = 0; i < N; ++i) {
            const double *zi = z + ((size_t)l * N + i) * D;
            for (j = 0; j < D; ++j) {
                double s = mu[j];
                for (k = 0; k <= j; ++k) s += Lc[j * D + k] * zi[k];
                xi[(size_t)i * D + j] = s;
            }
        }
        /* projection (lambda^0 = 0, or the warm start in the first CEM
         * iteration), residuals, cost */
        for (i = 0; i < N * D; ++i) lam[i] = (l == 0 && lam0) ? lam0[i] : 0.0;
        rc = orc_project(pr, cem->proj_iters, N, xi, NULL, lam, xb);
        if (rc) break;
        if (l == L - 1 && lam_out)
            for (i = 0; i < N * D; ++i) lam_out[i] = lam[i];
        orc_residual_cost(pr, N, xb, r, c1);
        for (i = 0; i < N; ++i) caug[i] = c1[i] + r[i];
        rc = orc_select(N, r, caug, cem->n_proj, cem->n_elite, NULL, eidx);
        if (rc) break;
        for (i = 0; i < cem->n_elite; ++i) {
            for (j = 0; j < D; ++j) el[(size_t)i * D + j] = xb[(size_t)eidx[i] * D + j];
            elc[i] = caug[eidx[i]];
        }
        rc = orc_refit(D, cem->n_elite, el, elc, cem->sigma_lr, cem->gamma, mu, cov);
    }
    if (rc == 0) {
        /* Alg. 1 return: the member of the last EliteSet with the lowest c_aug */
        for (j = 0; j < D; ++j) best[j] = xb[(size_t)eidx[0] * D + j];
        if (best_r) *best_r = r[eidx[0]];
        if (best_caug) *best_caug = caug[eidx[0]];
        if (mu_out)
            for (j = 0; j < D; ++j) mu_out[j] = mu[j];
        if (cov_out)
            for (j = 0; j < D * D; ++j) cov_out[j] = cov[j];
        if (elite_out)
            for (j = 0; j < cem->n_elite; ++j) elite_out[j] = eidx[j];
    }
    free(zz);
    free(mu);
    free(eidx);
    return rc;
}

/* ----------------------------------------------------------------------- */
/* D-PRIEST (Sec. D-PRIEST, Fig. fig_decentralized).                        */
/* ----------------------------------------------------------------------- */

/* Default means of the M distributions: the straight-line coefficients
 * with every interior coefficient (k = 1 .. n-1) moved by
 * (j - (M-1)/2) * spread along the unit normal of the start-goal line
 * (2-D: the line rotated by +90 degrees; 3-D: the horizontal normal; x when
 * that is undefined).  The trajectory then bows sideways by that amount
 * times (1 - B_0 - B_n), zero at both ends. */
int orc_multi_default_means(const orc_problem *pr, int M, double spread, double *mu)
{
    int D, nv, j, ax, k;
    double d[3] = {0, 0, 0}, nrm[3] = {0, 0, 0}, h;
    if (check_problem(pr) || M < 1) return -1;
    nv = pr->degree + 1;
    D = pr->dims * nv;
    for (ax = 0; ax < pr->dims; ++ax) d[ax] = pr->bf[ax][0] - pr->b0[ax][0];
    h = sqrt(d[0] * d[0] + d[1] * d[1]);
    if (h > 1e-12) {
        nrm[0] = -d[1] / h;
        nrm[1] = d[0] / h;
    } else {
        nrm[0] = 1.0;
    }
    for (j = 0; j < M; ++j) {
        const double off = ((double)j - 0.5 * (double)(M - 1)) * spread;
        double *m = mu + (size_t)j * D;
        orc_default_mean(pr, m);
        for (ax = 0; ax < pr->dims; ++ax)
            for (k = 1; k < pr->degree; ++k) m[ax * nv + k] += off * nrm[ax];
    }
    return 0;
}

/* D-PRIEST: M distributions (mu_j, Sigma_j), N_b / M samples each, stacked
 * row-wise (rows j * N_b/M .. are distribution j's), one projection of all
 * rows, then per distribution the residual / cost, ConstraintEliteSet of
 * N_proj / M, EliteSet of N_elite / M and the refit; after L iterations the
 * best elite of each distribution, and over them the lowest c_aug (ties:
 * the lower j).  z: L x N_b x D (row j * N_b/M + i at iteration l) or NULL
 * for the stream seeded by `seed`. */
int orc_plan_multi(const orc_problem *pr, const orc_cem *cem, int M, const double *mu0, const double *cov0,
                   const double *z, uint64_t seed, double *best, double *best_caug, int *best_dist,
                   double *dist_best, double *dist_r, double *dist_caug, double *mu_out)
{
    int D, N, L, nj, npj, nej, l, i, j, k, q, rc = 0;
    double *mu, *cov, *Lc, *Sh, *xi, *xb, *r, *c1, *caug, *zz = NULL, *el, *elc, *bcaug;
    int *eidx, *bidx;
    if (check_problem(pr) || !cem || M < 1) return -1;
    N = cem->n_samples;
    L = cem->cem_iters;
    if (N <= 0 || N % M || L <= 0 || cem->proj_iters < 0) return -1;
    nj = N / M;
    npj = cem->n_proj / M > 0 ? cem->n_proj / M : 1;
    nej = cem->n_elite / M > 0 ? cem->n_elite / M : 1;
    if (npj > nj || nej > npj) return -1;
    D = pr->dims * (pr->degree + 1);
    mu = (double *)malloc(sizeof(double) * ((size_t)M * (D + 2 * D * D) + D * D + 2 * (size_t)N * D + 3 * N +
                                            (size_t)nej * (D + 1) + M));
    eidx = (int *)malloc(sizeof(int) * ((size_t)M * nej + M));
    if (!mu || !eidx) return -2;
    cov = mu + (size_t)M * D;
    Lc = cov + (size_t)M * D * D;
    Sh = Lc + (size_t)M * D * D;
    xi = Sh + D * D;
    xb = xi + (size_t)N * D;
    r = xb + (size_t)N * D;
    c1 = r + N;
    caug = c1 + N;
    el = caug + N;
    elc = el + (size_t)nej * D;
    bcaug = elc + nej;
    bidx = eidx + (size_t)M * nej;
    if (mu0)
        for (i = 0; i < M * D; ++i) mu[i] = mu0[i];
    else
        orc_multi_default_means(pr, M, 2.0 * cem->init_std, mu);
    for (j = 0; j < M; ++j)
        for (i = 0; i < D * D; ++i)
            cov[(size_t)j * D * D + i] = cov0 ? cov0[(size_t)j * D * D + i]
                                              : ((i / D == i % D) ? cem->init_std * cem->init_std : 0.0);
    if (!z) {
        zz = (double *)malloc(sizeof(double) * (size_t)L * N * D);
        orc_rng_normal(seed, (int64_t)L * N * D, zz);
        z = zz;
    }
    for (l = 0; l < L && rc == 0; ++l) {
        /* samples of every distribution, stacked row-wise */
        for (j = 0; j < M && rc == 0; ++j) {
            const double *cj = cov + (size_t)j * D * D;
            double *Lj = Lc + (size_t)j * D * D, tr = 0.0, eps;
            for (i = 0; i < D; ++i) tr += cj[i * D + i];
            eps = cem->chol_eps * tr / (double)D;
            for (i = 0; i < D * D; ++i) Sh[i] = cj[i];
            for (i = 0; i < D; ++i) Sh[i * D + i] += eps;
            rc = orc_cholesky(D, Sh, Lj);
            for (i = 0; i < nj && rc == 0; ++i) {
                const int row = j * nj + i;
                const double *zi = z + ((size_t)l * N + row) * D;
                for (k = 0; k < D; ++k) {
                    double s = mu[(size_t)j * D + k];
                    for (q = 0; q <= k; ++q) s += Lj[k * D + q] * zi[q];
                    xi[(size_t)row * D + k] = s;
                }
            }
        }
        if (rc) break;
        /* one projection of all rows */
        rc = orc_project(pr, cem->proj_iters, N, xi, NULL, NULL, xb);
        if (rc) break;
        orc_residual_cost(pr, N, xb, r, c1);
        for (i = 0; i < N; ++i) caug[i] = c1[i] + r[i];
        /* per distribution: selections and refit */
        for (j = 0; j < M && rc == 0; ++j) {
            int *ej = eidx + (size_t)j * nej;
            rc = orc_select(nj, r + (size_t)j * nj, caug + (size_t)j * nj, npj, nej, NULL, ej);
            if (rc) break;
            for (i = 0; i < nej; ++i) {
                for (k = 0; k < D; ++k) el[(size_t)i * D + k] = xb[((size_t)j * nj + ej[i]) * D + k];
                elc[i] = caug[(size_t)j * nj + ej[i]];
            }
            rc = orc_refit(D, nej, el, elc, cem->sigma_lr, cem->gamma, mu + (size_t)j * D, cov + (size_t)j * D * D);
            bidx[j] = j * nj + ej[0];
            bcaug[j] = caug[bidx[j]];
        }
    }
    if (rc == 0) {
        int jb = 0;
        for (j = 1; j < M; ++j)
            if (bcaug[j] < bcaug[jb]) jb = j;
        for (k = 0; k < D; ++k) best[k] = xb[(size_t)bidx[jb] * D + k];
        if (best_caug) *best_caug = bcaug[jb];
        if (best_dist) *best_dist = jb;
        for (j = 0; j < M; ++j) {
            if (dist_best)
                for (k = 0; k < D; ++k) dist_best[(size_t)j * D + k] = xb[(size_t)bidx[j] * D + k];
            if (dist_r) dist_r[j] = r[bidx[j]];
            if (dist_caug) dist_caug[j] = bcaug[j];
        }
        if (mu_out)
            for (i = 0; i < M * D; ++i) mu_out[i] = mu[i];
    }
    free(zz);
    free(mu);
    free(eidx);
    return rc;
}

/*
 * Plain FP64 CPU oracle for the Wilson-Dirac operator and the CG solvers on
 * its normal equations.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg load this code.  It shares nothing with the CUDA library:
 * no headers, no tables, no helpers.
 *
 * Everything here is written from the paper's definitions, as literally as
 * possible, with full 4x4 spin matrices (no half-spinor trick, no blocking):
 *
 *   Section 2.1, Eq. (1): the Dirac operator.  The hopping term is written with
 *   -kappa:
 *     (D psi)(n) = psi(n) - kappa sum_mu [ b+_mu(n) (1 - gamma_mu) U_mu(n) psi(n+mu)
 *                                        + b-_mu(n) (1 + gamma_mu) U_mu(n-mu)^dag psi(n-mu) ]
 *   The paper prints +kappa; on lattices with even extents the two signs are
 *   unitarily equivalent through eps(n) = (-1)^(x+y+z+t), and the -kappa form
 *   is what the library implements.  Eq. (3): P(+-mu) = 1 +- gamma_mu, the
 *   forward hop carries P(-mu), the backward hop P(+mu).
 *   b+_3(n) = -1 when n_t = T-1, b-_3(n) = -1 when n_t = 0 (antiperiodic time
 *   direction, section 2.3: "periodic or antiperiodic boundary conditions");
 *   every other b is +1.  The stored links are never modified.
 *   The argument of U^dag in the backward term is U_mu(n - mu) (the printed
 *   equation drops the direction index).
 *
 *   D^dag is written as the literal adjoint of that matrix (projectors swapped):
 *     (D^dag psi)(n) = psi(n) - kappa sum_mu [ b+_mu(n) (1 + gamma_mu) U_mu(n) psi(n+mu)
 *                                            + b-_mu(n) (1 - gamma_mu) U_mu(n-mu)^dag psi(n-mu) ]
 *   The tests check it against gamma5 D gamma5 (section 2.2).
 *
 *   Appendix A: the gamma matrices, copied as data below.
 *
 *   Section 2.2: Conjugate Gradient.  The printed listing solves D D^dag y = eta
 *   and then forms psi = D^dag y (CGNE); it writes norms where squared norms
 *   belong and its first residual omits a D^dag.  Both repaired forms are here:
 *   CGNR (D^dag D x = D^dag b) and CGNE (D D^dag y = b, x = D^dag y), each the
 *   textbook Hestenes-Stiefel iteration with squared norms.
 *
 * Layouts (canonical): links U[mu][n][A][B] (4 x V x 3 x 3 complex), spinors
 * psi[n][alpha][A] (V x 4 x 3 complex); site n = x + Lx*(y + Ly*(z + Lz*t)).
 *
 * All sums are naive, in FP64, in site order.  The site loop of the operator
 * may run on several OpenMP threads; each output site is written by exactly
 * one thread, so the result does not depend on the thread count.
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Appendix A (conventions): gamma_0 .. gamma_3, row-major 4x4. */
static const cplx GAMMA[4][4][4] = {
    {{0, 0, 0, I}, {0, 0, I, 0}, {0, -I, 0, 0}, {-I, 0, 0, 0}},
    {{0, 0, 0, -1}, {0, 0, 1, 0}, {0, 1, 0, 0}, {-1, 0, 0, 0}},
    {{0, 0, I, 0}, {0, 0, 0, -I}, {-I, 0, 0, 0}, {0, I, 0, 0}},
    {{0, 0, 1, 0}, {0, 0, 0, 1}, {1, 0, 0, 0}, {0, 1, 0, 0}},
};
/* Appendix A: gamma_5. */
static const cplx GAMMA5[4][4] = {
    {1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, -1, 0}, {0, 0, 0, -1}};

/* Copies of the tables, so the tests can check them against the paper. */
void oracle_gamma(int mu, double *out32)
{
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            cplx g = (mu == 5) ? GAMMA5[a][b] : GAMMA[mu][a][b];
            out32[2 * (4 * a + b)] = creal(g);
            out32[2 * (4 * a + b) + 1] = cimag(g);
        }
}

static size_t volume(const int L[4])
{
    return (size_t)L[0] * L[1] * L[2] * L[3];
}

static void coords(const int L[4], size_t n, int c[4])
{
    for (int mu = 0; mu < 4; ++mu) {
        c[mu] = (int)(n % (size_t)L[mu]);
        n /= (size_t)L[mu];
    }
}

static size_t index_of(const int L[4], const int c[4])
{
    return (size_t)c[0] + (size_t)L[0] * ((size_t)c[1] + (size_t)L[1] * ((size_t)c[2] + (size_t)L[2] * (size_t)c[3]));
}

static const cplx *link(const cplx *U, const int L[4], int mu, size_t n)
{
    return U + ((size_t)mu * volume(L) + n) * 9;
}

/*
 * One output site of D (sign = +1) or D^dag (sign = -1):
 *   forward hop projector  1 - sign*gamma_mu
 *   backward hop projector 1 + sign*gamma_mu
 */
static void apply_site(const int L[4], int antiperiodic_t, double kappa, const cplx *U, const cplx *psi, int sign,
                       size_t n, cplx *out /* 12 */)
{
    cplx hop[4][3];
    memset(hop, 0, sizeof(hop));
    int c[4];
    coords(L, n, c);
    for (int mu = 0; mu < 4; ++mu) {
        /* forward neighbour n + mu */
        int cf[4] = {c[0], c[1], c[2], c[3]};
        cf[mu] = (c[mu] + 1) % L[mu];
        size_t nf = index_of(L, cf);
        double bf = (mu == 3 && antiperiodic_t && c[3] == L[3] - 1) ? -1.0 : 1.0;
        /* backward neighbour n - mu */
        int cb[4] = {c[0], c[1], c[2], c[3]};
        cb[mu] = (c[mu] + L[mu] - 1) % L[mu];
        size_t nb = index_of(L, cb);
        double bb = (mu == 3 && antiperiodic_t && c[3] == 0) ? -1.0 : 1.0;

        const cplx *Uf = link(U, L, mu, n);  /* U_mu(n) */
        const cplx *Ub = link(U, L, mu, nb); /* U_mu(n - mu) */
        const cplx *pf = psi + nf * 12;
        const cplx *pb = psi + nb * 12;

        for (int alpha = 0; alpha < 4; ++alpha)
            for (int A = 0; A < 3; ++A) {
                cplx s = 0;
                for (int beta = 0; beta < 4; ++beta) {
                    cplx Pf = (alpha == beta ? 1.0 : 0.0) - sign * GAMMA[mu][alpha][beta];
                    cplx Pb = (alpha == beta ? 1.0 : 0.0) + sign * GAMMA[mu][alpha][beta];
                    for (int B = 0; B < 3; ++B) {
                        s += bf * Pf * Uf[3 * A + B] * pf[3 * beta + B];
                        s += bb * Pb * conj(Ub[3 * B + A]) * pb[3 * beta + B];
                    }
                }
                hop[alpha][A] += s;
            }
    }
    const cplx *p0 = psi + n * 12;
    for (int alpha = 0; alpha < 4; ++alpha)
        for (int A = 0; A < 3; ++A)
            out[3 * alpha + A] = p0[3 * alpha + A] - kappa * hop[alpha][A];
}

static int g_threads = 1;

void oracle_set_threads(int n)
{
    g_threads = n > 0 ? n : 1;
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return g_threads;
#else
    return 1;
#endif
}

/* out = D psi (dagger = 0) or D^dag psi (dagger = 1).  out must not alias psi. */
void oracle_wilson_apply(const int L[4], int antiperiodic_t, double kappa, const cplx *U, const cplx *psi, cplx *out,
                         int dagger)
{
    const long long V = (long long)volume(L);
    const int sign = dagger ? -1 : 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
    for (long long n = 0; n < V; ++n)
        apply_site(L, antiperiodic_t, kappa, U, psi, sign, (size_t)n, out + (size_t)n * 12);
}

/* The operator at a list of sites only: out[k*12 ..] = (D psi)(sites[k]). */
void oracle_wilson_apply_sites(const int L[4], int antiperiodic_t, double kappa, const cplx *U, const cplx *psi,
                               int dagger, const long long *sites, long long nsites, cplx *out)
{
    const int sign = dagger ? -1 : 1;
    for (long long k = 0; k < nsites; ++k)
        apply_site(L, antiperiodic_t, kappa, U, psi, sign, (size_t)sites[k], out + (size_t)k * 12);
}

/* ---- FP64 vector helpers for the solvers (plain loops, site order) ---- */

static double norm2(const cplx *a, size_t N)
{
    double s = 0.0;
    for (size_t i = 0; i < N; ++i)
        s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

/* out = D^dag D psi, using tmp for D psi */
void oracle_normal_apply(const int L[4], int antiperiodic_t, double kappa, const cplx *U, const cplx *psi,
                         cplx *out, cplx *tmp)
{
    oracle_wilson_apply(L, antiperiodic_t, kappa, U, psi, tmp, 0);
    oracle_wilson_apply(L, antiperiodic_t, kappa, U, tmp, out, 1);
}

typedef struct {
    int iters;
    int converged;
    double iter_resid;      /* last iterated ||r|| / ||rhs|| of the normal system */
    double true_normal_rel; /* recomputed ||D^dag(b - D x)|| / ||D^dag b|| */
    double true_rel;        /* recomputed ||b - D x|| / ||b|| */
} oracle_cg_info;

static void true_residuals(const int L[4], int ap, double kappa, const cplx *U, const cplx *b, const cplx *x,
                           size_t N, oracle_cg_info *info)
{
    cplx *Dx = malloc(N * sizeof(cplx));
    cplx *e = malloc(N * sizeof(cplx));
    cplx *Ddb = malloc(N * sizeof(cplx));
    cplx *De = malloc(N * sizeof(cplx));
    oracle_wilson_apply(L, ap, kappa, U, x, Dx, 0);
    for (size_t i = 0; i < N; ++i)
        e[i] = b[i] - Dx[i];
    oracle_wilson_apply(L, ap, kappa, U, b, Ddb, 1);
    oracle_wilson_apply(L, ap, kappa, U, e, De, 1);
    double nb = norm2(b, N), ne = norm2(e, N), ndb = norm2(Ddb, N), nde = norm2(De, N);
    info->true_rel = nb > 0 ? sqrt(ne / nb) : sqrt(ne);
    info->true_normal_rel = ndb > 0 ? sqrt(nde / ndb) : sqrt(nde);
    free(Dx);
    free(e);
    free(Ddb);
    free(De);
}

/*
 * CGNR: solve D^dag D x = D^dag b (section 2.2, normal equations; the
 * Hestenes-Stiefel iteration with squared norms).
 *   x = x0; r = D^dag b - D^dag D x; p = r; rho = |r|^2
 *   loop: q = D p; alpha = rho / |q|^2; x += alpha p; r -= alpha D^dag q
 *         rho' = |r|^2; stop when sqrt(rho') <= tol |D^dag b|
 *         beta = rho' / rho; p = r + beta p; rho = rho'
 * x holds x0 on entry (zeros for the default start) and the solution on exit.
 */
int oracle_cgnr(const int L[4], int ap, double kappa, const cplx *U, const cplx *b, cplx *x, double tol,
                int max_iter, oracle_cg_info *info)
{
    const size_t N = volume(L) * 12;
    cplx *r = malloc(N * sizeof(cplx)), *p = malloc(N * sizeof(cplx)), *q = malloc(N * sizeof(cplx));
    cplx *t = malloc(N * sizeof(cplx)), *db = malloc(N * sizeof(cplx));
    oracle_wilson_apply(L, ap, kappa, U, b, db, 1);
    oracle_normal_apply(L, ap, kappa, U, x, r, t);
    for (size_t i = 0; i < N; ++i) {
        r[i] = db[i] - r[i];
        p[i] = r[i];
    }
    const double ndb = sqrt(norm2(db, N));
    double rho = norm2(r, N);
    int k = 0, conv = sqrt(rho) <= tol * ndb;
    while (!conv && k < max_iter) {
        oracle_wilson_apply(L, ap, kappa, U, p, q, 0);
        double alpha = rho / norm2(q, N);
        oracle_wilson_apply(L, ap, kappa, U, q, t, 1);
        for (size_t i = 0; i < N; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * t[i];
        }
        double rho1 = norm2(r, N);
        ++k;
        if (sqrt(rho1) <= tol * ndb)
            conv = 1;
        double beta = rho1 / rho;
        for (size_t i = 0; i < N; ++i)
            p[i] = r[i] + beta * p[i];
        rho = rho1;
    }
    info->iters = k;
    info->converged = conv;
    info->iter_resid = ndb > 0 ? sqrt(rho) / ndb : sqrt(rho);
    true_residuals(L, ap, kappa, U, b, x, N, info);
    free(r);
    free(p);
    free(q);
    free(t);
    free(db);
    return conv ? 0 : 1;
}

/*
 * CGNE, the form the paper's listing implements (section 2.2): solve
 * D D^dag y = b, then x = D^dag y.
 *   y = 0; r = b; p = r; rho = |r|^2
 *   loop: q = D^dag p; alpha = rho / |q|^2; y += alpha p; r -= alpha D q
 *         rho' = |r|^2; stop when sqrt(rho') <= tol |b|
 *         beta = rho' / rho; p = r + beta p; rho = rho'
 *   x = D^dag y
 * Here r = b - D D^dag y = b - D x is the residual of D x = b itself.
 */
int oracle_cgne(const int L[4], int ap, double kappa, const cplx *U, const cplx *b, cplx *x, double tol,
                int max_iter, oracle_cg_info *info)
{
    const size_t N = volume(L) * 12;
    cplx *y = calloc(N, sizeof(cplx)), *r = malloc(N * sizeof(cplx)), *p = malloc(N * sizeof(cplx));
    cplx *q = malloc(N * sizeof(cplx)), *t = malloc(N * sizeof(cplx));
    for (size_t i = 0; i < N; ++i) {
        r[i] = b[i];
        p[i] = r[i];
    }
    const double nb = sqrt(norm2(b, N));
    double rho = norm2(r, N);
    int k = 0, conv = sqrt(rho) <= tol * nb;
    while (!conv && k < max_iter) {
        oracle_wilson_apply(L, ap, kappa, U, p, q, 1);
        double alpha = rho / norm2(q, N);
        oracle_wilson_apply(L, ap, kappa, U, q, t, 0);
        for (size_t i = 0; i < N; ++i) {
            y[i] += alpha * p[i];
            r[i] -= alpha * t[i];
        }
        double rho1 = norm2(r, N);
        ++k;
        if (sqrt(rho1) <= tol * nb)
            conv = 1;
        double beta = rho1 / rho;
        for (size_t i = 0; i < N; ++i)
            p[i] = r[i] + beta * p[i];
        rho = rho1;
    }
    oracle_wilson_apply(L, ap, kappa, U, y, x, 1);
    info->iters = k;
    info->converged = conv;
    info->iter_resid = nb > 0 ? sqrt(rho) / nb : sqrt(rho);
    true_residuals(L, ap, kappa, U, b, x, N, info);
    free(y);
    free(r);
    free(p);
    free(q);
    free(t);
    return conv ? 0 : 1;
}

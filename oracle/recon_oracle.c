/*
 * recon_oracle.c -- plain, slow, double-precision CPU oracle for the hot path of
 * "Scalable network reconstruction in subquadratic time" (T. P. Peixoto,
 * arXiv:2401.01404).
 *
 * THIS IS TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU
 * baseline of the benchmark load it. The product (the CUDA library) never
 * calls it, links it or includes anything from here, and this file includes
 * nothing from the product: the two share no code, header or constant.
 *
 * What it computes, and where the paper defines it:
 *   - Ising pseudo-likelihood objective with Laplace prior (App. A, the
 *     pseudolikelihood product and the Laplace prior P(W|lambda)).
 *   - Multivariate Gaussian pseudo-likelihood objective (App. A, Gaussian
 *     pseudolikelihood with theta_i = 1/sqrt(W_ii)).
 *   - The pair "distance" d(i,j) = -max_{W_ij} pi(W) of Algorithm 2, returned
 *     as the gain max_w pi(W_ij <- w) - pi(W) (the ranking is the same because
 *     pi(W) is fixed while pairs are ranked).  The 1-D maximisation is done by
 *     bisection on the subgradient, the element-wise method Sec. II suggests.
 *   - The coordinate updates of Algorithm 1 / Algorithm 2 with the tracked
 *     neighbour sums m_i of App. A, and the update of the extra per-node
 *     parameters theta "alongside W" (App. A).
 *   - Exhaustive m-best pairs, exact k-nearest neighbours, NNDescent
 *     (Algorithm 4) and FindBest (Algorithm 3), all over a given dense
 *     distance matrix.
 *
 * Conventions.  X is node-major: X[i*M + m] is node i in sample m (the paper's
 * X is N x M with one column per sample, Sec. II).  W is a dense symmetric
 * N x N matrix; its diagonal is not a coupling and is ignored (the Gaussian
 * diagonal is carried separately as s2[i] = theta_i^2 = 1/W_ii).  All
 * arithmetic is double.  phi[i*M+m] = h_i + sum_{j != i} W_ij x_j^m is the
 * Ising local field; mu[i*M+m] = sum_{j != i} W_ij x_j^m is the Gaussian
 * neighbour sum m_i of App. A.
 *
 * Parity status: every function here is pinned by the not-gpu tests (closed
 * forms, brute force, invariants); the NNDescent trajectory is random and is
 * compared only through recall and iteration statistics.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* 1-D maximisation by bisection                                             */
/* ------------------------------------------------------------------------ */

/* Derivative of the smooth (likelihood) part of a concave 1-D objective,
 * as a function of the new value w of the coordinate. Strictly decreasing. */
typedef double (*deriv_fn)(double w, const void *ctx);

/* argmax_w  S(w) - lambda*|w|  over |w| <= wmax, for S concave with derivative
 * D = S'.  w = 0 is optimal iff 0 lies in the subgradient D(0) - lambda*[-1,1],
 * i.e. |D(0)| <= lambda.  Otherwise the optimum lies on the side of sign(D(0))
 * and solves D(w) = lambda*sign(w); it is bracketed by doubling and then
 * bisected to a relative width of 1e-13. */
static double argmax_l1(deriv_fn D, const void *ctx, double lambda, double wmax)
{
    double d0 = D(0.0, ctx);
    if (fabs(d0) <= lambda)
        return 0.0;
    double sgn = d0 > 0 ? 1.0 : -1.0;
    /* g(u) = sgn*D(sgn*u) - lambda, decreasing in u >= 0, g(0) > 0 */
#define G_OF(u) (sgn * D(sgn * (u), ctx) - lambda)
    double lo = 0.0, hi = wmax < 1.0 ? wmax : 1.0;
    while (G_OF(hi) > 0) {
        if (hi >= wmax)
            return sgn * wmax; /* the optimum is beyond the clamp */
        lo = hi;
        hi = 2 * hi < wmax ? 2 * hi : wmax;
    }
    for (int it = 0; it < 400 && hi - lo > 1e-13 * (hi > 1.0 ? hi : 1.0); ++it) {
        double mid = 0.5 * (lo + hi);
        if (G_OF(mid) > 0)
            lo = mid;
        else
            hi = mid;
    }
#undef G_OF
    return sgn * 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------ */
/* Ising model (App. A)                                                      */
/* ------------------------------------------------------------------------ */

/* log(2 cosh z) = log(e^z + e^-z), written so that it does not overflow. */
static double log2cosh(double z)
{
    double a = fabs(z);
    return a + log1p(exp(-2.0 * a));
}

/* phi_i^m = h_i + sum_{j != i} W_ij x_j^m, from scratch (App. A). */
void orc_ising_phi(int N, int M, const int8_t *X, const double *h, const double *W, double *phi)
{
    for (int i = 0; i < N; ++i)
        for (int m = 0; m < M; ++m) {
            double s = h[i];
            for (int j = 0; j < N; ++j)
                if (j != i && W[(int64_t)i * N + j] != 0.0)
                    s += W[(int64_t)i * N + j] * X[(int64_t)j * M + m];
            phi[(int64_t)i * M + m] = s;
        }
}

/* log pi(W, h) up to a constant: the log pseudo-likelihood
 * sum_m sum_i [x_i phi_i - log 2cosh phi_i] plus the Laplace log-prior
 * -lambda sum_{i<j} |W_ij| (App. A; the constant sum log(lambda/2) is dropped). */
double orc_ising_objective(int N, int M, const int8_t *X, const double *h, const double *W, double lambda)
{
    double *phi = (double *)malloc(sizeof(double) * (size_t)N * M);
    orc_ising_phi(N, M, X, h, W, phi);
    double ll = 0.0;
    for (int i = 0; i < N; ++i)
        for (int m = 0; m < M; ++m) {
            double z = phi[(int64_t)i * M + m];
            ll += X[(int64_t)i * M + m] * z - log2cosh(z);
        }
    free(phi);
    double pen = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j)
            pen += fabs(W[(int64_t)i * N + j]);
    return ll - lambda * pen;
}

typedef struct {
    int M;
    const int8_t *xi, *xj;
    const double *phi_i, *phi_j;
    double w_old;
} ising_pair_ctx;

/* Change of the pseudo-log-likelihood when W_ij moves from w_old to w.  Only
 * the conditionals of i and j contain W_ij; their fields move by
 * (w - w_old) x_j and (w - w_old) x_i.  The difference is taken sample by
 * sample, before summing. */
static double ising_pair_dll(const ising_pair_ctx *c, double w)
{
    double dw = w - c->w_old, s = 0.0;
    for (int m = 0; m < c->M; ++m) {
        double xi = c->xi[m], xj = c->xj[m];
        double pi0 = c->phi_i[m], pj0 = c->phi_j[m];
        double pi1 = pi0 + dw * xj, pj1 = pj0 + dw * xi;
        double now = xi * pi1 - log2cosh(pi1) + xj * pj1 - log2cosh(pj1);
        double before = xi * pi0 - log2cosh(pi0) + xj * pj0 - log2cosh(pj0);
        s += now - before;
    }
    return s;
}

/* d/dw of ising_pair_dll: sum_m [x_i x_j - x_j tanh(phi_i') + x_j x_i - x_i tanh(phi_j')]. */
static double ising_pair_deriv(double w, const void *vc)
{
    const ising_pair_ctx *c = (const ising_pair_ctx *)vc;
    double dw = w - c->w_old, s = 0.0;
    for (int m = 0; m < c->M; ++m) {
        double xi = c->xi[m], xj = c->xj[m];
        double pi1 = c->phi_i[m] + dw * xj, pj1 = c->phi_j[m] + dw * xi;
        s += xj * (xi - tanh(pi1)) + xi * (xj - tanh(pj1));
    }
    return s;
}

/* Gain of the best single-coupling update of pair (i,j):
 *   max_w pi(W_ij <- w) - pi(W) = max_w [dll(w) - lambda|w| + lambda|W_ij|],
 * with |w| <= w_clamp.  d(i,j) of Algorithm 2 is minus this gain.  Returns the
 * gain and writes the maximiser. */
double orc_ising_pair_gain(int M, const int8_t *xi, const int8_t *xj, const double *phi_i,
                           const double *phi_j, double w_old, double lambda, double w_clamp,
                           double *w_star)
{
    ising_pair_ctx c = {M, xi, xj, phi_i, phi_j, w_old};
    double w = argmax_l1(ising_pair_deriv, &c, lambda, w_clamp);
    if (w_star)
        *w_star = w;
    return ising_pair_dll(&c, w) - lambda * fabs(w) + lambda * fabs(w_old);
}

/* Scores a list of pairs (OpenMP over pairs: the paper's own CPU
 * parallelisation of independent pair evaluations, App. B). */
void orc_ising_score_pairs(int N, int M, const int8_t *X, const double *phi, const double *W,
                           double lambda, double w_clamp, int64_t P, const int32_t *pairs,
                           double *gain, double *w_star, int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
#endif
    for (int64_t p = 0; p < P; ++p) {
        int i = pairs[2 * p], j = pairs[2 * p + 1];
        double ws = 0.0;
        gain[p] = orc_ising_pair_gain(M, X + (int64_t)i * M, X + (int64_t)j * M, phi + (int64_t)i * M,
                                      phi + (int64_t)j * M, W[(int64_t)i * N + j], lambda, w_clamp,
                                      &ws);
        if (w_star)
            w_star[p] = ws;
    }
    (void)nthreads;
}

/* Same, for pairs whose current coupling is given explicitly (W_ij = wcur[p])
 * and whose field rows are given; used at sizes where a dense W does not fit. */
void orc_ising_score_pairs_rows(int M, const int8_t *X, const double *phi, double lambda,
                                double w_clamp, int64_t P, const int32_t *pairs,
                                const double *wcur, double *gain, double *w_star, int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
#endif
    for (int64_t p = 0; p < P; ++p) {
        int i = pairs[2 * p], j = pairs[2 * p + 1];
        double ws = 0.0;
        gain[p] = orc_ising_pair_gain(M, X + (int64_t)i * M, X + (int64_t)j * M, phi + (int64_t)i * M,
                                      phi + (int64_t)j * M, wcur ? wcur[p] : 0.0, lambda, w_clamp,
                                      &ws);
        if (w_star)
            w_star[p] = ws;
    }
    (void)nthreads;
}

/* Applies the coordinate updates of Algorithm 2 (and Algorithm 1) to the pairs,
 * one after the other in the given order: W_ij <- argmax, then the tracked
 * fields of i and j move by (W_ij' - W_ij) x_j and (W_ij' - W_ij) x_i (App. A).
 * Returns Delta = sum |W_ij' - W_ij|. */
double orc_ising_update_pairs(int N, int M, const int8_t *X, double *phi, double *W, double lambda,
                              double w_clamp, int64_t P, const int32_t *pairs)
{
    double delta = 0.0;
    for (int64_t p = 0; p < P; ++p) {
        int i = pairs[2 * p], j = pairs[2 * p + 1];
        double w_old = W[(int64_t)i * N + j], w_new = 0.0;
        orc_ising_pair_gain(M, X + (int64_t)i * M, X + (int64_t)j * M, phi + (int64_t)i * M,
                            phi + (int64_t)j * M, w_old, lambda, w_clamp, &w_new);
        double dw = w_new - w_old;
        for (int m = 0; m < M; ++m) {
            phi[(int64_t)i * M + m] += dw * X[(int64_t)j * M + m];
            phi[(int64_t)j * M + m] += dw * X[(int64_t)i * M + m];
        }
        W[(int64_t)i * N + j] = w_new;
        W[(int64_t)j * N + i] = w_new;
        delta += fabs(dw);
    }
    return delta;
}

typedef struct {
    int M;
    const int8_t *x;
    const double *phi;
    double h_old;
} ising_field_ctx;

/* d/dh of sum_m [x phi - log 2cosh phi] with phi = phi_old + (h - h_old). */
static double ising_field_deriv(double h, const void *vc)
{
    const ising_field_ctx *c = (const ising_field_ctx *)vc;
    double s = 0.0;
    for (int m = 0; m < c->M; ++m)
        s += c->x[m] - tanh(c->phi[m] + (h - c->h_old));
    return s;
}

/* Optimises every local field h_i in turn (the extra per-node parameters theta
 * that App. A updates alongside W; they carry no prior), moving phi_i with it.
 * Returns sum |h_i' - h_i|. */
double orc_ising_field_sweep(int N, int M, const int8_t *X, double *phi, double *h, double h_clamp)
{
    double delta = 0.0;
    for (int i = 0; i < N; ++i) {
        ising_field_ctx c = {M, X + (int64_t)i * M, phi + (int64_t)i * M, h[i]};
        double hn = argmax_l1(ising_field_deriv, &c, 0.0, h_clamp);
        double dh = hn - h[i];
        for (int m = 0; m < M; ++m)
            phi[(int64_t)i * M + m] += dh;
        h[i] = hn;
        delta += fabs(dh);
    }
    return delta;
}

/* ------------------------------------------------------------------------ */
/* Multivariate Gaussian model (App. A)                                      */
/* ------------------------------------------------------------------------ */

static const double LOG_2PI = 1.83787706640934548356;

/* mu_i^m = sum_{j != i} W_ij x_j^m, the tracked neighbour sum of App. A. */
void orc_gauss_mu(int N, int M, const double *X, const double *W, double *mu)
{
    for (int i = 0; i < N; ++i)
        for (int m = 0; m < M; ++m) {
            double s = 0.0;
            for (int j = 0; j < N; ++j)
                if (j != i && W[(int64_t)i * N + j] != 0.0)
                    s += W[(int64_t)i * N + j] * X[(int64_t)j * M + m];
            mu[(int64_t)i * M + m] = s;
        }
}

/* log of one Gaussian conditional: x_i | rest ~ Normal(-theta_i^2 mu_i, theta_i^2),
 * with s2 = theta_i^2 = 1/W_ii. */
static double gauss_logcond(double x, double mu, double s2)
{
    double r = x + s2 * mu;
    return -r * r / (2.0 * s2) - 0.5 * log(s2) - 0.5 * LOG_2PI;
}

/* log pseudo-likelihood plus Laplace log-prior on the off-diagonal (App. A). */
double orc_gauss_objective(int N, int M, const double *X, const double *s2, const double *W, double lambda)
{
    double *mu = (double *)malloc(sizeof(double) * (size_t)N * M);
    orc_gauss_mu(N, M, X, W, mu);
    double ll = 0.0;
    for (int i = 0; i < N; ++i)
        for (int m = 0; m < M; ++m)
            ll += gauss_logcond(X[(int64_t)i * M + m], mu[(int64_t)i * M + m], s2[i]);
    free(mu);
    double pen = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j)
            pen += fabs(W[(int64_t)i * N + j]);
    return ll - lambda * pen;
}

typedef struct {
    int M;
    const double *xi, *xj, *mu_i, *mu_j;
    double s2i, s2j, w_old;
} gauss_pair_ctx;

static double gauss_pair_dll(const gauss_pair_ctx *c, double w)
{
    double dw = w - c->w_old, s = 0.0;
    for (int m = 0; m < c->M; ++m) {
        double xi = c->xi[m], xj = c->xj[m];
        double now = gauss_logcond(xi, c->mu_i[m] + dw * xj, c->s2i) +
                     gauss_logcond(xj, c->mu_j[m] + dw * xi, c->s2j);
        double before = gauss_logcond(xi, c->mu_i[m], c->s2i) + gauss_logcond(xj, c->mu_j[m], c->s2j);
        s += now - before;
    }
    return s;
}

/* d/dw: sum_m -[(x_i + s2_i mu_i') x_j + (x_j + s2_j mu_j') x_i]. */
static double gauss_pair_deriv(double w, const void *vc)
{
    const gauss_pair_ctx *c = (const gauss_pair_ctx *)vc;
    double dw = w - c->w_old, s = 0.0;
    for (int m = 0; m < c->M; ++m) {
        double xi = c->xi[m], xj = c->xj[m];
        s -= (xi + c->s2i * (c->mu_i[m] + dw * xj)) * xj + (xj + c->s2j * (c->mu_j[m] + dw * xi)) * xi;
    }
    return s;
}

double orc_gauss_pair_gain(int M, const double *xi, const double *xj, const double *mu_i,
                           const double *mu_j, double s2i, double s2j, double w_old, double lambda,
                           double w_clamp, double *w_star)
{
    gauss_pair_ctx c = {M, xi, xj, mu_i, mu_j, s2i, s2j, w_old};
    double w = argmax_l1(gauss_pair_deriv, &c, lambda, w_clamp);
    if (w_star)
        *w_star = w;
    return gauss_pair_dll(&c, w) - lambda * fabs(w) + lambda * fabs(w_old);
}

void orc_gauss_score_pairs(int N, int M, const double *X, const double *mu, const double *s2,
                           const double *W, double lambda, double w_clamp, int64_t P,
                           const int32_t *pairs, const double *wcur, double *gain, double *w_star,
                           int nthreads)
{
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
#endif
    for (int64_t p = 0; p < P; ++p) {
        int i = pairs[2 * p], j = pairs[2 * p + 1];
        double w_old = W ? W[(int64_t)i * N + j] : (wcur ? wcur[p] : 0.0);
        double ws = 0.0;
        gain[p] = orc_gauss_pair_gain(M, X + (int64_t)i * M, X + (int64_t)j * M, mu + (int64_t)i * M,
                                      mu + (int64_t)j * M, s2[i], s2[j], w_old, lambda, w_clamp, &ws);
        if (w_star)
            w_star[p] = ws;
    }
    (void)nthreads;
}

double orc_gauss_update_pairs(int N, int M, const double *X, double *mu, const double *s2, double *W,
                              double lambda, double w_clamp, int64_t P, const int32_t *pairs)
{
    double delta = 0.0;
    for (int64_t p = 0; p < P; ++p) {
        int i = pairs[2 * p], j = pairs[2 * p + 1];
        double w_old = W[(int64_t)i * N + j], w_new = 0.0;
        orc_gauss_pair_gain(M, X + (int64_t)i * M, X + (int64_t)j * M, mu + (int64_t)i * M,
                            mu + (int64_t)j * M, s2[i], s2[j], w_old, lambda, w_clamp, &w_new);
        double dw = w_new - w_old;
        for (int m = 0; m < M; ++m) {
            mu[(int64_t)i * M + m] += dw * X[(int64_t)j * M + m];
            mu[(int64_t)j * M + m] += dw * X[(int64_t)i * M + m];
        }
        W[(int64_t)i * N + j] = w_new;
        W[(int64_t)j * N + i] = w_new;
        delta += fabs(dw);
    }
    return delta;
}

typedef struct {
    int M;
    const double *x, *mu;
} gauss_diag_ctx;

/* d/du of sum_m log Normal(x | -u mu, u) with u = theta_i^2, written per sample
 * as the derivative of -(x + u mu)^2/(2u) - (1/2) log u. */
static double gauss_diag_deriv(double u, const gauss_diag_ctx *c)
{
    double s = 0.0;
    for (int m = 0; m < c->M; ++m) {
        double x = c->x[m], mu = c->mu[m], r = x + u * mu;
        s += -r * mu / u + r * r / (2.0 * u * u) - 0.5 / u;
    }
    return s;
}

/* Optimises every theta_i^2 in turn (the diagonal of W carries no prior; App. A
 * updates theta alongside W).  The derivative is positive near u = 0 and
 * negative for large u, with a single root, found by doubling and bisection.
 * Returns sum |u' - u|. */
double orc_gauss_diag_sweep(int N, int M, const double *X, const double *mu, double *s2)
{
    double delta = 0.0;
    for (int i = 0; i < N; ++i) {
        gauss_diag_ctx c = {M, X + (int64_t)i * M, mu + (int64_t)i * M};
        double lo = 0.0, hi = 1.0;
        while (gauss_diag_deriv(hi, &c) > 0) {
            lo = hi;
            hi *= 2.0;
        }
        for (int it = 0; it < 400 && hi - lo > 1e-15 * hi; ++it) {
            double mid = 0.5 * (lo + hi);
            if (gauss_diag_deriv(mid, &c) > 0)
                lo = mid;
            else
                hi = mid;
        }
        double un = 0.5 * (lo + hi);
        delta += fabs(un - s2[i]);
        s2[i] = un;
    }
    return delta;
}

/* ------------------------------------------------------------------------ */
/* Searches over a given dense distance matrix D (n x n, symmetric)          */
/* ------------------------------------------------------------------------ */

/* Total order used everywhere the paper breaks ties "arbitrarily" (Fig. 1):
 * by d, then by the smaller, then the larger node id, then by direction. */
typedef struct {
    double d;
    int32_t a, b; /* directed edge a -> b (for pairs: a < b) */
} edge_t;

static int edge_cmp(const void *pa, const void *pb)
{
    const edge_t *x = (const edge_t *)pa, *y = (const edge_t *)pb;
    if (x->d != y->d)
        return x->d < y->d ? -1 : 1;
    int xl = x->a < x->b ? x->a : x->b, yl = y->a < y->b ? y->a : y->b;
    if (xl != yl)
        return xl < yl ? -1 : 1;
    int xh = x->a < x->b ? x->b : x->a, yh = y->a < y->b ? y->b : y->a;
    if (xh != yh)
        return xh < yh ? -1 : 1;
    if (x->a != y->a)
        return x->a < y->a ? -1 : 1;
    return 0;
}

#define DIST(D, N, i, j) ((D)[(int64_t)(i) * (N) + (j)])

/* m best pairs of S by exhaustive search (Algorithm 3, base case).  Writes up
 * to m pairs (global ids, a < b) in ascending order; returns how many. */
int64_t orc_exhaustive_best(int N, const double *D, int nS, const int32_t *S, int64_t m, int32_t *out)
{
    int64_t n = (int64_t)nS * (nS - 1) / 2, q = 0;
    edge_t *e = (edge_t *)malloc(sizeof(edge_t) * (size_t)(n > 0 ? n : 1));
    for (int x = 0; x < nS; ++x)
        for (int y = x + 1; y < nS; ++y) {
            int a = S[x] < S[y] ? S[x] : S[y], b = S[x] < S[y] ? S[y] : S[x];
            e[q].d = DIST(D, N, a, b);
            e[q].a = a;
            e[q].b = b;
            ++q;
        }
    qsort(e, (size_t)q, sizeof(edge_t), edge_cmp);
    int64_t r = q < m ? q : m;
    for (int64_t p = 0; p < r; ++p) {
        out[2 * p] = e[p].a;
        out[2 * p + 1] = e[p].b;
    }
    free(e);
    return r;
}

/* Exact k nearest neighbours of every node of S among S (the KNN problem that
 * Algorithm 3 delegates to FindKNN), by sorting all candidates by (d, id).
 * G is nS x k of global ids. */
void orc_exact_knn(int N, const double *D, int nS, const int32_t *S, int k, int32_t *G)
{
    edge_t *e = (edge_t *)malloc(sizeof(edge_t) * (size_t)(nS > 1 ? nS : 1));
    for (int x = 0; x < nS; ++x) {
        int q = 0;
        for (int y = 0; y < nS; ++y)
            if (y != x) {
                e[q].d = DIST(D, N, S[x], S[y]);
                e[q].a = S[x];
                e[q].b = S[y];
                ++q;
            }
        qsort(e, (size_t)q, sizeof(edge_t), edge_cmp);
        for (int r = 0; r < k; ++r)
            G[(int64_t)x * k + r] = r < q ? e[r].b : -1;
    }
    free(e);
}

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the oracle's own
 * counter-based stream for the random choices of NNDescent. */
static uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

static int in_list(const int32_t *l, int k, int32_t v)
{
    for (int r = 0; r < k; ++r)
        if (l[r] == v)
            return 1;
    return 0;
}

/* NNDescent (Algorithm 4) over the node set S, written as the algorithm reads:
 * a random k-out digraph; then repeatedly, with G' a copy of G and U the
 * undirected version of G, every second neighbour v of every node i (through
 * U) replaces the worst entry u_hat of i's list in G' when d(i,v) < d(i,u_hat);
 * Delta counts replacements; stop when Delta/(k|S|) < eps.
 * Readings where the paper is silent: the initial k out-neighbours are
 * distinct and differ from i; U(i) is out(i) together with at most in_cap
 * in-neighbours per node, sampled uniformly afresh each iteration (the "first k
 * neighbours" cap of Sec. III); ties in the worst entry go to the largest
 * (d, id).  G (nS x k, global ids) is the result; returns iterations used. */
int orc_nndescent(int N, const double *D, int nS, const int32_t *S, int k, double eps, int max_iters,
                  int in_cap, uint64_t seed, int32_t *G, int64_t *replacements)
{
    /* local index of each global id */
    int32_t *loc = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    for (int v = 0; v < N; ++v)
        loc[v] = -1;
    for (int x = 0; x < nS; ++x)
        loc[S[x]] = x;
    int32_t *Gl = (int32_t *)malloc(sizeof(int32_t) * (size_t)nS * k);  /* G, local ids */
    int32_t *Gn = (int32_t *)malloc(sizeof(int32_t) * (size_t)nS * k);  /* G' */
    /* random k distinct out-neighbours != i */
    for (int x = 0; x < nS; ++x) {
        int q = 0;
        uint64_t ctr = 0;
        while (q < k) {
            uint64_t r = splitmix64(seed ^ splitmix64(((uint64_t)x << 32) ^ ctr++));
            int y = (int)(r % (uint64_t)nS);
            if (y == x || in_list(Gl + (int64_t)x * k, q, y))
                continue;
            Gl[(int64_t)x * k + q++] = y;
        }
    }
    int deg_cap = k + in_cap;
    int32_t *U = (int32_t *)malloc(sizeof(int32_t) * (size_t)nS * deg_cap);
    int *Udeg = (int *)malloc(sizeof(int) * (size_t)nS);
    int *indeg = (int *)malloc(sizeof(int) * (size_t)nS);
    int64_t *inoff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nS + 1));
    int32_t *insrc = (int32_t *)malloc(sizeof(int32_t) * (size_t)nS * k);
    uint64_t *prio = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nS * k);
    int iters = 0;
    int64_t total = 0;
    for (iters = 0; iters < max_iters;) {
        ++iters;
        memcpy(Gn, Gl, sizeof(int32_t) * (size_t)nS * k);
        /* U = undirected version of G */
        for (int x = 0; x < nS; ++x)
            indeg[x] = 0;
        for (int64_t e = 0; e < (int64_t)nS * k; ++e)
            indeg[Gl[e]]++;
        inoff[0] = 0;
        for (int x = 0; x < nS; ++x)
            inoff[x + 1] = inoff[x] + indeg[x];
        for (int x = 0; x < nS; ++x)
            indeg[x] = 0;
        for (int x = 0; x < nS; ++x)
            for (int r = 0; r < k; ++r) {
                int y = Gl[(int64_t)x * k + r];
                insrc[inoff[y] + indeg[y]++] = x;
            }
        for (int x = 0; x < nS; ++x) {
            int d = 0;
            for (int r = 0; r < k; ++r)
                U[(int64_t)x * deg_cap + d++] = Gl[(int64_t)x * k + r];
            /* in-neighbours: keep the in_cap with the smallest random priority */
            int64_t b = inoff[x];
            int n_in = indeg[x];
            for (int q = 0; q < n_in; ++q)
                prio[b + q] = splitmix64(seed ^ splitmix64(((uint64_t)iters << 40) ^
                                                           ((uint64_t)x << 20) ^ (uint64_t)insrc[b + q]));
            int take = n_in < in_cap ? n_in : in_cap;
            for (int q = 0; q < take; ++q) { /* partial selection sort by priority */
                int best = q;
                for (int z = q + 1; z < n_in; ++z)
                    if (prio[b + z] < prio[b + best])
                        best = z;
                uint64_t tp = prio[b + q];
                prio[b + q] = prio[b + best];
                prio[b + best] = tp;
                int32_t ts = insrc[b + q];
                insrc[b + q] = insrc[b + best];
                insrc[b + best] = ts;
                int y = insrc[b + q];
                if (!in_list(U + (int64_t)x * deg_cap, d, y))
                    U[(int64_t)x * deg_cap + d++] = y;
            }
            Udeg[x] = d;
        }
        int64_t delta = 0;
        for (int x = 0; x < nS; ++x) {
            int32_t *gi = Gn + (int64_t)x * k;
            for (int a = 0; a < Udeg[x]; ++a) {
                int y = U[(int64_t)x * deg_cap + a];
                for (int c = 0; c < Udeg[y]; ++c) {
                    int v = U[(int64_t)y * deg_cap + c];
                    if (v == x || in_list(gi, k, v))
                        continue;
                    /* the worst entry of i's list in G' */
                    int worst = 0;
                    for (int r = 1; r < k; ++r) {
                        double dr = DIST(D, N, S[x], S[gi[r]]), dw = DIST(D, N, S[x], S[gi[worst]]);
                        if (dr > dw || (dr == dw && S[gi[r]] > S[gi[worst]]))
                            worst = r;
                    }
                    if (DIST(D, N, S[x], S[v]) < DIST(D, N, S[x], S[gi[worst]])) {
                        gi[worst] = v;
                        ++delta;
                    }
                }
            }
        }
        memcpy(Gl, Gn, sizeof(int32_t) * (size_t)nS * k);
        total += delta;
        if ((double)delta / ((double)k * nS) < eps)
            break;
    }
    for (int64_t e = 0; e < (int64_t)nS * k; ++e)
        G[e] = S[Gl[e]];
    if (replacements)
        *replacements = total;
    free(loc);
    free(Gl);
    free(Gn);
    free(U);
    free(Udeg);
    free(indeg);
    free(inoff);
    free(insrc);
    free(prio);
    return iters;
}

/* Bookkeeping of one FindBest call, for the tests of Sec. III's invariants. */
typedef struct {
    int levels;                 /* recursion levels that ran a KNN search */
    int64_t level_size[64];     /* |S_t| at each level (the last one is exhaustive) */
    int64_t level_D[64];        /* |D| at each KNN level */
    int level_k[64];            /* k_t used at each KNN level */
    int64_t knn_iters;          /* total NNDescent iterations */
} orc_findbest_stats;

static int64_t findbest_rec(int N, const double *D, int nS, const int32_t *S, int64_t m, int knn_exact,
                            int k_min, double eps, int max_iters, int in_cap, uint64_t seed, int depth,
                            int32_t *out, orc_findbest_stats *st)
{
    if (depth < 64)
        st->level_size[depth] = nS;
    if ((int64_t)nS * nS <= 4 * m) {
        st->levels = depth;
        return orc_exhaustive_best(N, D, nS, S, m, out);
    }
    /* k = ceil(4m/|S|), raised to the configured k (reading of the paper's k) */
    int64_t k64 = (4 * m + nS - 1) / nS;
    if (k64 < k_min)
        k64 = k_min;
    if (k64 > nS - 1)
        k64 = nS - 1;
    int k = (int)k64;
    int32_t *G = (int32_t *)malloc(sizeof(int32_t) * (size_t)nS * k);
    if (knn_exact)
        orc_exact_knn(N, D, nS, S, k, G);
    else
        st->knn_iters += orc_nndescent(N, D, nS, S, k, eps, max_iters, in_cap,
                                       splitmix64(seed + (uint64_t)depth), G, NULL);
    /* D+ = the 2m directed edges of G with the smallest d */
    int64_t nE = (int64_t)nS * k;
    edge_t *E = (edge_t *)malloc(sizeof(edge_t) * (size_t)nE);
    for (int x = 0; x < nS; ++x)
        for (int r = 0; r < k; ++r) {
            int64_t e = (int64_t)x * k + r;
            E[e].a = S[x];
            E[e].b = G[e];
            E[e].d = DIST(D, N, S[x], G[e]);
        }
    qsort(E, (size_t)nE, sizeof(edge_t), edge_cmp);
    int64_t nDp = nE < 2 * m ? nE : 2 * m;
    /* D = unique undirected pairs of D+ (as an N x N membership mask) */
    uint8_t *inD = (uint8_t *)calloc((size_t)N * N, 1);
    int64_t nD = 0;
    edge_t *Dset = (edge_t *)malloc(sizeof(edge_t) * (size_t)(nDp > 0 ? nDp : 1));
    for (int64_t p = 0; p < nDp; ++p) {
        int a = E[p].a < E[p].b ? E[p].a : E[p].b, b = E[p].a < E[p].b ? E[p].b : E[p].a;
        if (!inD[(int64_t)a * N + b]) {
            inD[(int64_t)a * N + b] = 1;
            Dset[nD].a = a;
            Dset[nD].b = b;
            Dset[nD].d = E[p].d;
            ++nD;
        }
    }
    if (depth < 64) {
        st->level_D[depth] = nD;
        st->level_k[depth] = k;
    }
    /* S' = nodes whose every out-edge in G is in D */
    int32_t *S2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)nS);
    int nS2 = 0;
    for (int x = 0; x < nS; ++x) {
        int all = 1;
        for (int r = 0; r < k; ++r) {
            int a = S[x], b = G[(int64_t)x * k + r];
            int lo = a < b ? a : b, hi = a < b ? b : a;
            if (!inD[(int64_t)lo * N + hi]) {
                all = 0;
                break;
            }
        }
        if (all)
            S2[nS2++] = S[x];
    }
    int32_t *sub = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 2));
    int64_t nsub = findbest_rec(N, D, nS2, S2, m, knn_exact, k_min, eps, max_iters, in_cap, seed,
                                depth + 1, sub, st);
    /* m best pairs of D u D' */
    edge_t *U = (edge_t *)malloc(sizeof(edge_t) * (size_t)(nD + nsub + 1));
    int64_t nU = 0;
    for (int64_t p = 0; p < nD; ++p)
        U[nU++] = Dset[p];
    for (int64_t p = 0; p < nsub; ++p) {
        int a = sub[2 * p], b = sub[2 * p + 1];
        if (inD[(int64_t)a * N + b])
            continue;
        U[nU].a = a;
        U[nU].b = b;
        U[nU].d = DIST(D, N, a, b);
        ++nU;
    }
    qsort(U, (size_t)nU, sizeof(edge_t), edge_cmp);
    int64_t r = nU < m ? nU : m;
    for (int64_t p = 0; p < r; ++p) {
        out[2 * p] = U[p].a;
        out[2 * p + 1] = U[p].b;
    }
    free(G);
    free(E);
    free(inD);
    free(Dset);
    free(S2);
    free(sub);
    free(U);
    return r;
}

/* FindBest(m, S, d) of Algorithm 3 over a dense distance matrix, with either
 * the exact KNN (knn_exact = 1) or NNDescent (Algorithm 4) as FindKNN.  Writes
 * up to m pairs (a < b, ascending d) into out[2m]; returns the count. */
int64_t orc_findbest(int N, const double *D, int nS, const int32_t *S, int64_t m, int knn_exact,
                     int k_min, double eps, int max_iters, int in_cap, uint64_t seed, int32_t *out,
                     orc_findbest_stats *st)
{
    orc_findbest_stats local;
    if (!st)
        st = &local;
    memset(st, 0, sizeof(*st));
    return findbest_rec(N, D, nS, S, m, knn_exact, k_min, eps, max_iters, in_cap, seed, 0, out, st);
}

int orc_nthreads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

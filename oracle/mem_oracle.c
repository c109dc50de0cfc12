/*
 * mem_oracle.c -- FP64 CPU oracle for the 35-moment maximal-entropy moment
 * method (MEM) of arXiv 2303.02898, "Stabilizing the Maximal Entropy Moment
 * Method for Rarefied Gas Dynamics at Single-Precision".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * __graft_entry__.smoke() and the CPU-baseline / reference arm of bench.py may
 * load it.  It shares no code, table or constant generator with the CUDA
 * library, and it never reads anything the CUDA library produced as an
 * expected value.
 *
 * Everything is FP64, dense, in the order the paper states it:
 *   - tensor Gauss-Hermite rule (Golub-Welsch: eigen-decomposition of the
 *     Jacobi matrix of the probabilists' Hermite polynomials);
 *   - the 35 orthonormal Hermite-product statistics phi_i(ubar) of total
 *     degree <= 4 in 3D velocity (Appendix B, orthonormal form of Eq.
 *     "Sufficient 35", extended from the 1D cylindrical set to full 3D);
 *   - the canonical-form moment map with the log-sum-exp partition function
 *     (Eqs. "Numerical integration moments" and "MLE optimization goal log sum
 *     exp", Section 3.1);
 *   - Algorithm 1 (modified Newton with a multiple of the identity, Armijo
 *     backtracking), objective/gradient/Hessian of Appendix C;
 *   - the translation/dilation gauge and its change-of-gauge matrix
 *     (Eqs. "Sufficient 35 ortho", "Change gauge M F", "Hermite parameters");
 *   - characteristic speed = spectral radius of dF/dM (Eq. "The lax F");
 *   - ES-BGK source (Appendix A), local Lax-Friedrichs, Lax-Wendroff and FLIC
 *     finite-volume updates with neighbour gauge transforms and Strang-split
 *     collision (Algorithm 2);
 *   - the paper's nine-statistic system for axisymmetric flow (Eq. "Sufficient
 *     35"): Algorithm 1, flux and characteristic speed on its statistics;
 *   - Rankine-Hugoniot states (Appendix D).
 *
 * Parity status: every function below has a pin in tests/test_oracle_pins.py
 * (closed forms, invariants, brute force).  The paper's figures print no
 * values, so nothing is pinned to a figure.
 *
 * Conventions (readings of the paper):
 *   - M_i(g) = int phi_i((u-w)/s) f(u) d^3u, the moments in the cell's gauge
 *     g = (w_x,w_y,w_z,s_x,s_y,s_z); M_0 = n.
 *   - beta_0 = n; beta_1..34 are the natural parameters relative to the
 *     Gauss-Hermite base measure: f ~ n exp(-|ubar|^2/2 + sum_{i>=1} beta_i
 *     phi_i(ubar)).  This is an exact re-parameterisation of the paper's
 *     Lebesgue-measure beta (|ubar|^2/2 lies in the span of the statistics):
 *     objective differences, gradient and Hessian are identical, so Algorithm
 *     1 takes identical steps.  beta = 0 is the Maxwellian of the gauge.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NP 35      /* number of statistics, total degree <= 4 in 3D */
#define NMAXQ 64   /* largest 1D Gauss-Hermite order supported */

/* ------------------------------------------------------------------------ */
/* Multi-index table: statistic k <-> (a,b,c), a+b+c <= 4.  Ordered by total
 * degree, then a descending, then b descending. */
static int g_idx[NP][3];
static int g_idx_ready = 0;

static void build_index(void) {
    if (g_idx_ready) return;
    int k = 0;
    for (int d = 0; d <= 4; ++d)
        for (int a = d; a >= 0; --a)
            for (int b = d - a; b >= 0; --b) {
                g_idx[k][0] = a; g_idx[k][1] = b; g_idx[k][2] = d - a - b; ++k;
            }
    g_idx_ready = 1;
}

void or_basis_index(int *abc) {
    build_index();
    for (int k = 0; k < NP; ++k) for (int j = 0; j < 3; ++j) abc[3 * k + j] = g_idx[k][j];
}

int or_index_of(int a, int b, int c) {
    build_index();
    for (int k = 0; k < NP; ++k)
        if (g_idx[k][0] == a && g_idx[k][1] == b && g_idx[k][2] == c) return k;
    return -1;
}

/* Orthonormal probabilists' Hermite values he_0..he_kmax at x:
 * He_{k+1} = x He_k - k He_{k-1}; he_k = He_k / sqrt(k!). */
static void hermite_on(double x, int kmax, double *he) {
    double Hm1 = 0.0, H = 1.0, fact = 1.0;
    he[0] = 1.0;
    for (int k = 0; k < kmax; ++k) {
        double Hp = x * H - k * Hm1;
        Hm1 = H; H = Hp;
        fact *= (double)(k + 1);
        he[k + 1] = H / sqrt(fact);
    }
}

/* phi_i(ubar) for all 35 statistics. */
void or_phi(const double *u, double *phi) {
    build_index();
    double hx[5], hy[5], hz[5];
    hermite_on(u[0], 4, hx); hermite_on(u[1], 4, hy); hermite_on(u[2], 4, hz);
    for (int k = 0; k < NP; ++k) phi[k] = hx[g_idx[k][0]] * hy[g_idx[k][1]] * hz[g_idx[k][2]];
}

/* ------------------------------------------------------------------------ */
/* Dense symmetric eigen-decomposition by cyclic Jacobi rotations (textbook,
 * FP64).  a is n x n row-major and is destroyed; eigenvalues to ev, the
 * eigenvectors (columns) to v if v != NULL. */
static void jacobi_eigen(int n, double *a, double *ev, double *v) {
    if (v) { for (int i = 0; i < n * n; ++i) v[i] = 0.0; for (int i = 0; i < n; ++i) v[i * n + i] = 1.0; }
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < n; ++p) {
            diag += a[p * n + p] * a[p * n + p];
            for (int q = p + 1; q < n; ++q) off += a[p * n + q] * a[p * n + q];
        }
        if (off <= 1e-30 * (diag + 1e-300)) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = a[p * n + q];
                if (fabs(apq) < 1e-300) continue;
                double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) { /* columns p,q */
                    double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = c * akp - s * akq;
                    a[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) { /* rows p,q */
                    double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = c * apk - s * aqk;
                    a[q * n + k] = s * apk + c * aqk;
                }
                if (v)
                    for (int k = 0; k < n; ++k) {
                        double vkp = v[k * n + p], vkq = v[k * n + q];
                        v[k * n + p] = c * vkp - s * vkq;
                        v[k * n + q] = s * vkp + c * vkq;
                    }
            }
    }
    for (int i = 0; i < n; ++i) ev[i] = a[i * n + i];
}

/* Gauss-Hermite rule for the standard normal weight (probabilists'), by
 * Golub-Welsch: nodes = eigenvalues of the Jacobi matrix with off-diagonal
 * sqrt(k), weights = squared first eigenvector components (sum to 1).
 * Returns 0 on success. */
int or_gh_rule(int n, double *x, double *w) {
    if (n < 1 || n > NMAXQ) return -1;
    double *J = calloc((size_t)n * n, sizeof(double)), *V = calloc((size_t)n * n, sizeof(double));
    double ev[NMAXQ];
    for (int k = 0; k + 1 < n; ++k) J[k * n + k + 1] = J[(k + 1) * n + k] = sqrt((double)(k + 1));
    jacobi_eigen(n, J, ev, V);
    int order[NMAXQ];
    for (int i = 0; i < n; ++i) order[i] = i;
    for (int i = 0; i < n; ++i) /* sort ascending */
        for (int j = i + 1; j < n; ++j)
            if (ev[order[j]] < ev[order[i]]) { int t = order[i]; order[i] = order[j]; order[j] = t; }
    double sw = 0.0;
    for (int i = 0; i < n; ++i) { x[i] = ev[order[i]]; w[i] = V[0 * n + order[i]] * V[0 * n + order[i]]; sw += w[i]; }
    for (int i = 0; i < n; ++i) w[i] /= sw;
    free(J); free(V);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Quadrature rule cache: tensor n^3 nodes ubar_q, log w_q, phi(ubar_q). */
typedef struct { int n, Q, phys; double *u; double *logw; double *phi; } rule_t;
static rule_t g_rules[NMAXQ + 1];

/* Block Gauss-Legendre tensor rules on a box in the gauge frame (rule ids
 * 100..115, registered by or_set_box_rule).  Per axis, [-L, L] is split into
 * nb equal blocks with ng Legendre points each; the Gaussian base measure is
 * folded into the weights, w_i = w^GL_i exp(-x_i^2/2) / sqrt(2 pi), so beta
 * keeps its meaning (beta = 0 is the gauge's Maxwellian, up to truncation). */
static rule_t g_box_rules[16];

static void gl_rule(int n, double *x, double *w) {
    /* Golub-Welsch for Legendre on [-1, 1]: off-diagonal k / sqrt(4k^2 - 1). */
    double *J = calloc((size_t)n * n, sizeof(double)), *V = calloc((size_t)n * n, sizeof(double)), ev[64];
    for (int k = 1; k < n; ++k) J[(k - 1) * n + k] = J[k * n + k - 1] = k / sqrt(4.0 * k * k - 1.0);
    jacobi_eigen(n, J, ev, V);
    int order[64];
    for (int i = 0; i < n; ++i) order[i] = i;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (ev[order[j]] < ev[order[i]]) { int t = order[i]; order[i] = order[j]; order[j] = t; }
    for (int i = 0; i < n; ++i) { x[i] = ev[order[i]]; w[i] = 2.0 * V[order[i]] * V[order[i]]; }
    free(J); free(V);
}

int or_set_box_rule(int id, int nbx, int nbr, int ng, double Lx, double Lr) {
    if (id < 100 || id > 115 || ng < 1 || ng > 16 || nbx < 1 || nbr < 1 || nbx * ng > 256 || nbr * ng > 256) return -1;
    rule_t *r = &g_box_rules[id - 100];
    if (r->Q) { free(r->u); free(r->logw); free(r->phi); r->Q = 0; }
    double gx[16], gw[16];
    gl_rule(ng, gx, gw);
    double ax[3][256], aw[3][256];
    int na[3];
    for (int a = 0; a < 3; ++a) {
        int nb = a == 0 ? nbx : nbr;
        double L = a == 0 ? Lx : Lr, h = 2.0 * L / nb;
        na[a] = nb * ng;
        for (int b = 0; b < nb; ++b)
            for (int i = 0; i < ng; ++i) {
                double x = -L + h * (b + 0.5 * (gx[i] + 1.0));
                ax[a][b * ng + i] = x;
                aw[a][b * ng + i] = 0.5 * h * gw[i] * exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
            }
    }
    int Q = na[0] * na[1] * na[2];
    double *u = malloc(sizeof(double) * 3 * Q), *lw = malloc(sizeof(double) * Q), *ph = malloc(sizeof(double) * NP * (size_t)Q);
    int q = 0;
    for (int i = 0; i < na[0]; ++i) for (int j = 0; j < na[1]; ++j) for (int k = 0; k < na[2]; ++k, ++q) {
        u[3 * q] = ax[0][i]; u[3 * q + 1] = ax[1][j]; u[3 * q + 2] = ax[2][k];
        lw[q] = log(aw[0][i]) + log(aw[1][j]) + log(aw[2][k]);
        or_phi(&u[3 * q], &ph[(size_t)NP * q]);
    }
    r->n = -1; r->u = u; r->logw = lw; r->phi = ph; r->Q = Q;
    return Q;
}

/* Velocity-space rules (rule ids 200..215, registered by
 * or_set_velocity_rule): the nodes are fixed in the lab frame, as in the
 * paper's shock computations (Section 3.1, Eq. "Numerical integration", with
 * the integration domain (u_x, u_r) in [a_x, b_x] x [0, b_r] of Appendix D).
 * u_x: [a_x, b_x] in nbx equal blocks of ng Gauss-Legendre points; u_r:
 * [0, b_r] in nbr equal blocks of ng Gauss-Legendre points with the polar
 * weight u_r; azimuth: K equispaced angles 2 pi k / K (trapezoid, exact for
 * trigonometric polynomials of degree < K).  Nodes u_q = (u_x, u_r cos t,
 * u_r sin t), weights w_q (no base measure).  In a cell of gauge g the rule
 * is used through ubar_q = (u_q - w) / s with log weight
 * log w_q - |ubar_q|^2 / 2, so that beta keeps its meaning (relative to the
 * gauge's Gaussian; constant factors cancel in Z). */
static rule_t g_vel_rules[16];

int or_set_velocity_rule(int id, double ax, double bx, int nbx, double br, int nbr, int ng, int K) {
    if (id < 200 || id > 215 || ng < 1 || ng > 16 || nbx < 1 || nbr < 1 || K < 1 || nbx * ng > 512 ||
        nbr * ng > 512 || K > 64 || !(bx > ax) || !(br > 0.0))
        return -1;
    rule_t *r = &g_vel_rules[id - 200];
    if (r->Q) { free(r->u); free(r->logw); r->Q = 0; }
    double gx[16], gw[16];
    gl_rule(ng, gx, gw);
    int nx = nbx * ng, nr = nbr * ng, Q = nx * nr * K;
    double *u = malloc(sizeof(double) * 3 * Q), *lw = malloc(sizeof(double) * Q);
    double hx = (bx - ax) / nbx, hr = br / nbr;
    int q = 0;
    for (int bi = 0; bi < nbx; ++bi) for (int i = 0; i < ng; ++i) {
        double x = ax + hx * (bi + 0.5 * (gx[i] + 1.0)), wx = 0.5 * hx * gw[i];
        for (int bj = 0; bj < nbr; ++bj) for (int j = 0; j < ng; ++j) {
            double rr = hr * (bj + 0.5 * (gx[j] + 1.0)), wr = 0.5 * hr * gw[j] * rr;
            for (int k = 0; k < K; ++k, ++q) {
                double t = 2.0 * M_PI * k / K;
                u[3 * q] = x; u[3 * q + 1] = rr * cos(t); u[3 * q + 2] = rr * sin(t);
                lw[q] = log(wx) + log(wr) + log(2.0 * M_PI / K);
            }
        }
    }
    r->n = -2; r->phys = 1; r->u = u; r->logw = lw; r->phi = NULL; r->Q = Q;
    return Q;
}

/* Node q of rule r seen from a cell of gauge g: ubar, log weight and the
 * statistics (phi points into the table for gauge-frame rules, else into
 * buf). */
static const double *rule_node(const rule_t *r, const double *g, int q, double *ub, double *lw, double *buf) {
    if (!r->phys) {
        ub[0] = r->u[3 * q]; ub[1] = r->u[3 * q + 1]; ub[2] = r->u[3 * q + 2];
        *lw = r->logw[q];
        return &r->phi[(size_t)NP * q];
    }
    for (int a = 0; a < 3; ++a) ub[a] = (r->u[3 * q + a] - g[a]) / g[3 + a];
    *lw = r->logw[q] - 0.5 * (ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
    or_phi(ub, buf);
    return buf;
}

static const rule_t *get_rule(int n) {
    if (n >= 100 && n <= 115) return g_box_rules[n - 100].Q ? &g_box_rules[n - 100] : NULL;
    if (n >= 200 && n <= 215) return g_vel_rules[n - 200].Q ? &g_vel_rules[n - 200] : NULL;
    if (n < 1 || n > NMAXQ) return NULL;
    rule_t *r = &g_rules[n];
    if (r->Q) return r;
    #pragma omp critical(or_rule_init)
    {
        if (!r->Q) {
            double x[NMAXQ], w[NMAXQ];
            or_gh_rule(n, x, w);
            int Q = n * n * n;
            double *u = malloc(sizeof(double) * 3 * Q), *lw = malloc(sizeof(double) * Q), *ph = malloc(sizeof(double) * NP * Q);
            for (int i = 0; i < n; ++i) for (int j = 0; j < n; ++j) for (int k = 0; k < n; ++k) {
                int q = (i * n + j) * n + k;
                u[3 * q] = x[i]; u[3 * q + 1] = x[j]; u[3 * q + 2] = x[k];
                lw[q] = log(w[i]) + log(w[j]) + log(w[k]);
                or_phi(&u[3 * q], &ph[NP * q]);
            }
            r->n = n; r->u = u; r->logw = lw; r->phi = ph;
            #pragma omp flush
            r->Q = Q;
        }
    }
    return r;
}

int or_rule_is_velocity(int n) {
    const rule_t *r = get_rule(n);
    return r ? r->phys : -1;
}

int or_rule_nodes(int n, double *u, double *logw) {
    const rule_t *r = get_rule(n);
    if (!r) return -1;
    memcpy(u, r->u, sizeof(double) * 3 * r->Q);
    memcpy(logw, r->logw, sizeof(double) * r->Q);
    return r->Q;
}

/* ------------------------------------------------------------------------ */
/* Forward map beta -> expectations under the discrete canonical-form
 * distribution sigma_q = w_q exp(beta.phi_q - log Z)  (Section 3.1, Eqs.
 * "Numerical integration moments" and the log-sum-exp form of log Z).
 * Outputs (any may be NULL): logZ; m[i] = E phi_i; S[i][j] = E phi_i phi_j;
 * X[i] = E ubar_x phi_i; XS[i][j] = E ubar_x phi_i phi_j. */
void or_expect(int order, const double *g, const double *beta, double *logZ, double *m, double *S, double *X,
               double *XS) {
    const rule_t *r = get_rule(order);
    int Q = r->Q;
    double *e = malloc(sizeof(double) * Q);
    double emax = -INFINITY, ub[3], lw, buf[NP];
    for (int q = 0; q < Q; ++q) {
        const double *ph = rule_node(r, g, q, ub, &lw, buf);
        double s = lw;
        for (int i = 1; i < NP; ++i) s += beta[i] * ph[i];
        e[q] = s;
        if (s > emax) emax = s;
    }
    double Z = 0.0;
    for (int q = 0; q < Q; ++q) { e[q] = exp(e[q] - emax); Z += e[q]; }
    if (logZ) *logZ = emax + log(Z);
    if (m) memset(m, 0, sizeof(double) * NP);
    if (S) memset(S, 0, sizeof(double) * NP * NP);
    if (X) memset(X, 0, sizeof(double) * NP);
    if (XS) memset(XS, 0, sizeof(double) * NP * NP);
    for (int q = 0; q < Q; ++q) {
        double sg = e[q] / Z;
        const double *ph = rule_node(r, g, q, ub, &lw, buf);
        double ux = ub[0];
        for (int i = 0; i < NP; ++i) {
            if (m) m[i] += sg * ph[i];
            if (X) X[i] += sg * ux * ph[i];
            if (S || XS)
                for (int j = 0; j <= i; ++j) {
                    double p = sg * ph[i] * ph[j];
                    if (S) S[i * NP + j] += p;
                    if (XS) XS[i * NP + j] += ux * p;
                }
        }
    }
    for (int i = 0; i < NP; ++i)
        for (int j = i + 1; j < NP; ++j) {
            if (S) S[i * NP + j] = S[j * NP + i];
            if (XS) XS[i * NP + j] = XS[j * NP + i];
        }
    free(e);
}

/* Objective of Appendix C, Eq. "MLE optimization goal", with beta_0 = n held
 * at its minimiser: L = log Z - sum_{i>=1} beta_i M_i / n. */
double or_objective(int order, const double *g, const double *beta, const double *M) {
    double lz;
    or_expect(order, g, beta, &lz, NULL, NULL, NULL, NULL);
    double s = 0.0;
    for (int i = 1; i < NP; ++i) s += beta[i] * M[i] / M[0];
    return lz - s;
}

/* Relative moment residual ||E phi(beta) - M/n||_2 / ||M/n||_2 (acceptance
 * measure of the solve; slot 0 contributes 0 by construction). */
double or_residual(int order, const double *g, const double *beta, const double *M) {
    double m[NP];
    or_expect(order, g, beta, NULL, m, NULL, NULL, NULL);
    double num = 0.0, den = 0.0;
    for (int i = 0; i < NP; ++i) {
        double t = M[i] / M[0];
        den += t * t;
        if (i) num += (m[i] - t) * (m[i] - t);
    }
    return sqrt(num / den);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (Section 3.2): Newton's method modified by adding a multiple of
 * the identity, with backtracking line search on a relaxed Armijo test. */
typedef struct {
    double tol;        /* convergence tolerance on res (1e-8) */
    int maxI;          /* iteration limit (500, as in every experiment) */
    double lambda0;    /* first identity multiple (1e-3) */
    double lambda_mul; /* growth per failed factorisation (10) */
    int max_lambda;    /* cap on lambda retries (reading: unbounded in paper) */
    double c;          /* Armijo slope factor (5e-4) */
    double atol, rtol; /* Armijo floating-point slack (5e-6, 5e-5) */
    int maxT;          /* line-search trials are s = 0..maxT (25) */
    double alpha_min;  /* stagnation exit alpha <= 1e-6 */
    int final_step;    /* 1: apply the last computed Newton step on res <= tol
                          (an extension; 0, Algorithm 1's own order, is the
                          default) */
} or_opts;

enum {
    ST_CONVERGED = 1, ST_STAGNATED = 2, ST_MAXITER = 4, ST_NONFINITE = 8,
    ST_LAMBDA = 16, ST_LAMBDA_CAP = 32, ST_BADINPUT = 64
};

static void default_opts(or_opts *o) {
    o->tol = 1e-8; o->maxI = 500; o->lambda0 = 1e-3; o->lambda_mul = 10.0; o->max_lambda = 20;
    o->c = 5e-4; o->atol = 5e-6; o->rtol = 5e-5; o->maxT = 25; o->alpha_min = 1e-6;
    o->final_step = 0;
}

/* Standard Cholesky of the n x n matrix A + shift*I (row-major); fails on a
 * pivot that is not positive and finite.  L is lower triangular. */
static int cholesky(int n, const double *A, double shift, double *L) {
    for (int i = 0; i < n * n; ++i) L[i] = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j] + shift;
        for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
        if (!(d > 0.0) || !isfinite(d)) return 1;
        double ljj = sqrt(d);
        L[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = s / ljj;
        }
    }
    return 0;
}

static void solve_lower(int n, const double *L, const double *b, double *x) {
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i * n + k] * x[k];
        x[i] = s / L[i * n + i];
    }
}

static void solve_upper_T(int n, const double *L, const double *b, double *x) { /* L^T x = b */
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
        x[i] = s / L[i * n + i];
    }
}

/* Solve one cell.  M[35] (M_0 = n), beta[35] in: warm start (slots 1..34),
 * out: solution with beta_0 = n.  Returns status bits; *iters = loop count;
 * *res_out = last res; *lam_out = largest identity multiple used. */
int or_solve(int order, const double *g, const double *M, double *beta, const double *optv, int *iters, double *res_out,
             double *lam_out) {
    or_opts o; default_opts(&o);
    if (optv) { o.tol = optv[0]; o.maxI = (int)optv[1]; o.final_step = optv[2] != 0.0; }
    const int D = NP - 1;
    double n = M[0];
    int st = 0;
    if (!(n > 0.0) || !isfinite(n)) { if (iters) *iters = 0; return ST_BADINPUT; }
    for (int i = 0; i < NP; ++i) if (!isfinite(M[i]) || !isfinite(beta[i])) { if (iters) *iters = 0; return ST_BADINPUT; }
    double b[NP], db[NP] = {0}, G[NP] = {0}, m[NP], S[NP * NP], H[34 * 34], Lh[34 * 34], wv[34], rhs[34], trial[NP];
    memcpy(b, beta, sizeof(b));
    b[0] = n;
    double Lcur = or_objective(order, g, b, M);
    int it = 0, conv = 0;
    double res = INFINITY, lam_used = 0.0, alpha = 1.0;
    while (!conv && it <= o.maxI) {
        /* BackTrackingLineSearch: alpha = 2 -> halve before each trial. */
        alpha = 2.0;
        int s = 0, sat = 0;
        while (!sat && s <= o.maxT) {
            if (!sat) alpha *= 0.5;
            for (int i = 0; i < NP; ++i) trial[i] = b[i] + alpha * db[i];
            trial[0] = n;
            double Lt = or_objective(order, g, trial, M);
            double LD = Lcur - Lt, gd = 0.0;
            for (int i = 1; i < NP; ++i) gd += G[i] * alpha * db[i];
            double gradD = -o.c * gd;
            sat = (LD - gradD) >= -(o.atol + o.rtol * fabs(LD));
            s += 1;
        }
        for (int i = 1; i < NP; ++i) b[i] += alpha * db[i];
        Lcur = or_objective(order, g, b, M);
        /* Hessian and gradient of L at beta (Appendix C). */
        or_expect(order, g, b, NULL, m, S, NULL, NULL);
        for (int i = 1; i < NP; ++i) G[i] = m[i] - M[i] / n;
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) H[i * D + j] = S[(i + 1) * NP + (j + 1)] - m[i + 1] * m[j + 1];
        /* Cholesky, adding lambda*I until it succeeds. */
        double lambda = o.lambda0;
        int fail = cholesky(D, H, 0.0, Lh), tries = 0;
        while (fail) {
            if (tries >= o.max_lambda) break;
            fail = cholesky(D, H, lambda, Lh);
            st |= ST_LAMBDA;
            if (lambda > lam_used) lam_used = lambda;
            lambda *= o.lambda_mul;
            ++tries;
        }
        if (fail) { st |= ST_LAMBDA_CAP | ST_NONFINITE; ++it; break; }
        for (int i = 0; i < D; ++i) rhs[i] = -G[i + 1];
        solve_lower(D, Lh, rhs, wv);
        double dx[34];
        solve_upper_T(D, Lh, wv, dx);
        db[0] = 0.0;
        for (int i = 0; i < D; ++i) db[i + 1] = dx[i];
        double dg = 0.0;
        for (int i = 1; i < NP; ++i) dg += db[i] * G[i];
        res = 0.5 * fabs(dg);
        if (!isfinite(res)) { st |= ST_NONFINITE; ++it; break; }
        if (res <= o.tol) st |= ST_CONVERGED;
        if (alpha <= o.alpha_min) st |= ST_STAGNATED;
        conv = (res <= o.tol) || (alpha <= o.alpha_min);
        ++it;
    }
    if (!conv && !(st & ST_NONFINITE)) st |= ST_MAXITER;
    /* Algorithm 1 returns beta without the direction computed in the last
     * pass (final_step = 0, the default).  The decrement res = |dbeta.grad|/2
     * <= tol bounds the objective error, not the moment residual
     * (|grad|^2 <= 2 res lambda_max(H)); final_step = 1, an extension,
     * applies that last Newton step when the loop stops on res <= tol. */
    if (o.final_step && (st & ST_CONVERGED))
        for (int i = 1; i < NP; ++i) b[i] += db[i];
    memcpy(beta, b, sizeof(b));
    beta[0] = n;
    if (iters) *iters = it;
    if (res_out) *res_out = res;
    if (lam_out) *lam_out = lam_used;
    return st;
}

void or_solve_batch(int order, int64_t B, const double *g, const double *M, double *beta, int *status, int *iters,
                    const double *optv, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    get_rule(order);
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t c = 0; c < B; ++c) {
        int it = 0;
        int st = or_solve(order, g ? &g[6 * c] : NULL, &M[NP * c], &beta[NP * c], optv, &it, NULL, NULL);
        if (status) status[c] = st;
        if (iters) iters[c] = it;
    }
}

/* ------------------------------------------------------------------------ */
/* Change of gauge (Eq. "Change gauge M F").  For g = (w, s) and g' = (w', s'),
 * ubar' = a*ubar + b per axis with a = s/s', b = (w - w')/s'.  T(g', g) maps
 * M(g) -> M(g'): phi_i(ubar') = sum_j T_ij phi_j(ubar).  Built here by going
 * through monomials: he_a(y) = sum_k H[a][k] y^k, y^k by the binomial theorem,
 * x^j = sum_d E[j][d] he_d(x) with E = H^{-1}. */
static void hermite_monomial_coeffs(double H[5][5]) {
    double He[5][5] = {{0}};
    He[0][0] = 1.0;
    He[1][1] = 1.0;
    for (int k = 1; k < 4; ++k)
        for (int p = 0; p < 5; ++p) {
            double v = -k * He[k - 1][p];
            if (p > 0) v += He[k][p - 1];
            He[k + 1][p] = v;
        }
    double fact = 1.0;
    for (int a = 0; a < 5; ++a) {
        if (a > 0) fact *= a;
        for (int p = 0; p < 5; ++p) H[a][p] = He[a][p] / sqrt(fact);
    }
}

static void axis_map(double a, double b, double t[5][5]) {
    double H[5][5], E[5][5] = {{0}};
    hermite_monomial_coeffs(H);
    /* E = H^{-1}, lower triangular, by forward substitution on columns. */
    for (int col = 0; col < 5; ++col)
        for (int r = 0; r < 5; ++r) {
            double s = (r == col) ? 1.0 : 0.0;
            for (int k = 0; k < r; ++k) s -= H[r][k] * E[k][col];
            E[r][col] = s / H[r][r];
        }
    /* x^j in he: x^j = sum_d Einv[j][d] he_d  where Einv = E (since H maps he->x^p
       coefficients: he = H x  => x = E he). */
    double C[5][5] = {{0}};
    for (int k = 0; k < 5; ++k) { C[k][0] = 1.0; for (int j = 1; j <= k; ++j) C[k][j] = C[k - 1][j - 1] + (j <= k - 1 ? C[k - 1][j] : 0.0); }
    for (int A = 0; A < 5; ++A)
        for (int d = 0; d < 5; ++d) {
            double s = 0.0;
            for (int k = 0; k <= A; ++k)          /* he_A(y) = sum_k H[A][k] y^k */
                for (int j = 0; j <= k; ++j)      /* y^k = sum_j C(k,j) a^j b^(k-j) x^j */
                    s += H[A][k] * C[k][j] * pow(a, j) * pow(b, k - j) * E[j][d];
            t[A][d] = s;
        }
}

void or_gauge_T(const double *g_to, const double *g_from, double *T) {
    build_index();
    double t[3][5][5];
    for (int ax = 0; ax < 3; ++ax) {
        double a = g_from[3 + ax] / g_to[3 + ax];
        double b = (g_from[ax] - g_to[ax]) / g_to[3 + ax];
        axis_map(a, b, t[ax]);
    }
    for (int i = 0; i < NP; ++i)
        for (int j = 0; j < NP; ++j)
            T[i * NP + j] = t[0][g_idx[i][0]][g_idx[j][0]] * t[1][g_idx[i][1]][g_idx[j][1]] * t[2][g_idx[i][2]][g_idx[j][2]];
}

static void matvec35(const double *T, const double *x, double *y) {
    for (int i = 0; i < NP; ++i) { double s = 0.0; for (int j = 0; j < NP; ++j) s += T[i * NP + j] * x[j]; y[i] = s; }
}

/* Hermite gauge of the distribution with moments M in gauge g (Eqs. "Hermite
 * parameters", "Hermite parameters in moments"): mean velocity and variance.
 * axisym = 1 is the 1D-shock form (w_y = w_z = 0, s_y = s_z = s_r with
 * s_r^2 = (<u_y^2> + <u_z^2>)/2); axisym = 0 takes each axis on its own. */
void or_hermite_gauge(const double *M, const double *g, int axisym, double *gH) {
    double n = M[0];
    double mean[3], ex2[3];
    for (int ax = 0; ax < 3; ++ax) {
        int e1[3] = {0, 0, 0}, e2[3] = {0, 0, 0};
        e1[ax] = 1; e2[ax] = 2;
        double m1 = M[or_index_of(e1[0], e1[1], e1[2])] / n;            /* E ubar */
        double m2 = sqrt(2.0) * M[or_index_of(e2[0], e2[1], e2[2])] / n + 1.0; /* E ubar^2 */
        mean[ax] = g[ax] + g[3 + ax] * m1;                              /* E u */
        ex2[ax] = g[ax] * g[ax] + 2.0 * g[ax] * g[3 + ax] * m1 + g[3 + ax] * g[3 + ax] * m2; /* E u^2 */
    }
    if (axisym) {
        gH[0] = mean[0]; gH[1] = 0.0; gH[2] = 0.0;
        gH[3] = sqrt(ex2[0] - mean[0] * mean[0]);
        double sr = sqrt(0.5 * (ex2[1] + ex2[2]));
        gH[4] = sr; gH[5] = sr;
    } else {
        for (int ax = 0; ax < 3; ++ax) { gH[ax] = mean[ax]; gH[3 + ax] = sqrt(ex2[ax] - mean[ax] * mean[ax]); }
    }
}

void or_transform_M(const double *g_to, const double *g_from, const double *M, double *Mout) {
    double T[NP * NP];
    or_gauge_T(g_to, g_from, T);
    matvec35(T, M, Mout);
}

/* beta (Gauss-Hermite base measure) from gauge g_from to g_to.  With
 * c = coefficients of -|ubar|^2/2 in the basis, the Lebesgue parameters are
 * beta + c and transform with T(g_from, g_to)^T (Eq. "Change gauge M F"). */
void or_transform_beta(const double *g_to, const double *g_from, const double *beta, double *bout) {
    double T[NP * NP], bl[NP], c[NP] = {0};
    int i200 = or_index_of(2, 0, 0), i020 = or_index_of(0, 2, 0), i002 = or_index_of(0, 0, 2);
    c[i200] = c[i020] = c[i002] = -1.0 / sqrt(2.0);
    or_gauge_T(g_from, g_to, T);
    for (int j = 0; j < NP; ++j) bl[j] = (j ? beta[j] + c[j] : 0.0);
    for (int i = 1; i < NP; ++i) {
        double s = 0.0;
        for (int j = 1; j < NP; ++j) s += T[j * NP + i] * bl[j];
        bout[i] = s - c[i];
    }
    bout[0] = beta[0];
}

/* ------------------------------------------------------------------------ */
/* Flux (Eq. "The ME equation", subeq. 3) and characteristic speed (Eq. "The
 * lax F"): F_i = n (w_x E phi_i + s_x E ubar_x phi_i); the eigenvalues of
 * dF/dM are the generalised eigenvalues of (d F/d alpha, d M/d alpha) =
 * n (E u_x phi phi^T, E phi phi^T) over all 35 statistics.  Whitened with the
 * Cholesky factor of E phi phi^T and diagonalised by Jacobi. */
void or_flux(int order, const double *beta, const double *g, double n, double *F, double *speed, double *lmin, double *lmax) {
    double m[NP], S[NP * NP], X[NP], XS[NP * NP];
    or_expect(order, g, beta, NULL, m, S, X, XS);
    if (F) for (int i = 0; i < NP; ++i) F[i] = n * (g[0] * m[i] + g[3] * X[i]);
    if (speed || lmin || lmax) {
        double L[NP * NP], C[NP * NP], tmp[NP * NP], ev[NP];
        if (cholesky(NP, S, 0.0, L)) {
            /* E phi phi^T numerically singular: the pencil has no reliable
             * spectrum (the failure mode the paper reports for over-refined
             * Mach-10 meshes).  Fall back to the Rayleigh-quotient bound over
             * the nodes, max_q |w_x + s_x ubar_x,q|. */
            const rule_t *r = get_rule(order);
            double a = INFINITY, b = -INFINITY;
            for (int q = 0; q < r->Q; ++q) {
                double ux = r->phys ? r->u[3 * q] : g[0] + g[3] * r->u[3 * q];
                if (ux < a) a = ux;
                if (ux > b) b = ux;
            }
            if (lmin) *lmin = a;
            if (lmax) *lmax = b;
            if (speed) *speed = fmax(fabs(a), fabs(b));
            return;
        }
        /* tmp = L^{-1} XS  (column by column), C = tmp L^{-T} */
        for (int col = 0; col < NP; ++col) {
            double bcol[NP], xcol[NP];
            for (int i = 0; i < NP; ++i) bcol[i] = XS[i * NP + col];
            solve_lower(NP, L, bcol, xcol);
            for (int i = 0; i < NP; ++i) tmp[i * NP + col] = xcol[i];
        }
        for (int row = 0; row < NP; ++row) {
            double brow[NP], xrow[NP];
            for (int i = 0; i < NP; ++i) brow[i] = tmp[row * NP + i];
            solve_lower(NP, L, brow, xrow);
            for (int i = 0; i < NP; ++i) C[row * NP + i] = xrow[i];
        }
        for (int i = 0; i < NP; ++i) for (int j = i + 1; j < NP; ++j) {
            double avg = 0.5 * (C[i * NP + j] + C[j * NP + i]);
            C[i * NP + j] = C[j * NP + i] = avg;
        }
        jacobi_eigen(NP, C, ev, NULL);
        double mu_lo = ev[0], mu_hi = ev[0];
        for (int i = 1; i < NP; ++i) { if (ev[i] < mu_lo) mu_lo = ev[i]; if (ev[i] > mu_hi) mu_hi = ev[i]; }
        double a = g[0] + g[3] * mu_lo, b = g[0] + g[3] * mu_hi;
        if (lmin) *lmin = a;
        if (lmax) *lmax = b;
        if (speed) *speed = fmax(fabs(a), fabs(b));
    }
}

/* ------------------------------------------------------------------------ */
/* Condition diagnostic (Section 4, Fig. 7: condition number of the moment
 * Jacobian dM/dbeta = n H, Eq. "moments vs parameter jacob").  The estimate
 * is the ratio of the largest to the smallest pivot L_kk^2 of the Cholesky
 * factorisation of the n x n SPD matrix A: every pivot is a diagonal entry of
 * a Schur complement, so it lies between the extreme eigenvalues and the
 * ratio never exceeds cond(A).  Returns -1 if A is not positive definite. */
double or_pivot_ratio(int n, const double *A) {
    double *L = malloc(sizeof(double) * n * n);
    double r = -1.0;
    if (!cholesky(n, A, 0.0, L)) {
        double mn = INFINITY, mx = 0.0;
        for (int k = 0; k < n; ++k) {
            const double d = L[k * n + k] * L[k * n + k];
            if (d < mn) mn = d;
            if (d > mx) mx = d;
        }
        r = mx / mn;
    }
    free(L);
    return r;
}

/* The estimate for one cell: H = Cov(phi_1..34) at beta (Appendix C). */
double or_cond_estimate(int order, const double *g, const double *beta) {
    double m[NP], S[NP * NP], H[34 * 34];
    or_expect(order, g, beta, NULL, m, S, NULL, NULL);
    for (int i = 0; i < 34; ++i)
        for (int j = 0; j < 34; ++j) H[i * 34 + j] = S[(i + 1) * NP + (j + 1)] - m[i + 1] * m[j + 1];
    return or_pivot_ratio(34, H);
}

/* ------------------------------------------------------------------------ */
/* ES-BGK target moments (Appendix A, Eq. "The ES BGK model"): Gaussian with
 * the cell's density and mean velocity and covariance
 * Sigma = T/Pr I + (1 - 1/Pr) P/n, expressed in the cell's gauge g.  The
 * Gaussian expectation of each statistic is taken with a 5-point-per-axis
 * Gauss-Hermite rule in whitened coordinates (exact for degree <= 9). */
static void central_moments(const double *M, const double *g, double *mean_u, double *P_over_n) {
    double n = M[0], mb[3], E2[3][3];
    for (int a = 0; a < 3; ++a) {
        int e[3] = {0, 0, 0}; e[a] = 1;
        mb[a] = M[or_index_of(e[0], e[1], e[2])] / n;
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            int e[3] = {0, 0, 0};
            if (a == b) { e[a] = 2; E2[a][b] = sqrt(2.0) * M[or_index_of(e[0], e[1], e[2])] / n + 1.0; }
            else { e[a] = 1; e[b] = 1; E2[a][b] = M[or_index_of(e[0], e[1], e[2])] / n; }
        }
    for (int a = 0; a < 3; ++a) mean_u[a] = g[a] + g[3 + a] * mb[a];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) P_over_n[3 * a + b] = g[3 + a] * g[3 + b] * (E2[a][b] - mb[a] * mb[b]);
}

void or_macro(const double *M, const double *g, double *out /* n, v[3], T, P/n[9] */) {
    double v[3], P[9];
    central_moments(M, g, v, P);
    out[0] = M[0];
    for (int a = 0; a < 3; ++a) out[1 + a] = v[a];
    out[4] = (P[0] + P[4] + P[8]) / 3.0;
    for (int k = 0; k < 9; ++k) out[5 + k] = P[k];
}

void or_gaussian_moments(const double *mean_bar, const double *cov_bar, double n, double *Mout) {
    double x[5], w[5], Lc[9];
    or_gh_rule(5, x, w);
    cholesky(3, cov_bar, 0.0, Lc);
    for (int i = 0; i < NP; ++i) Mout[i] = 0.0;
    for (int i = 0; i < 5; ++i) for (int j = 0; j < 5; ++j) for (int k = 0; k < 5; ++k) {
        double z[3] = {x[i], x[j], x[k]}, u[3], ph[NP];
        for (int a = 0; a < 3; ++a) { u[a] = mean_bar[a]; for (int b = 0; b <= a; ++b) u[a] += Lc[3 * a + b] * z[b]; }
        or_phi(u, ph);
        double ww = w[i] * w[j] * w[k];
        for (int p = 0; p < NP; ++p) Mout[p] += n * ww * ph[p];
    }
}

void or_esbgk(const double *M, const double *g, double Pr, double *Mt) {
    double n = M[0], v[3], P[9];
    central_moments(M, g, v, P);
    double T = (P[0] + P[4] + P[8]) / 3.0;
    double mb[3], cb[9];
    for (int a = 0; a < 3; ++a) mb[a] = (v[a] - g[a]) / g[3 + a];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double sig = (a == b ? T / Pr : 0.0) + (1.0 - 1.0 / Pr) * P[3 * a + b];
            cb[3 * a + b] = sig / (g[3 + a] * g[3 + b]);
        }
    or_gaussian_moments(mb, cb, n, Mt);
}

/* ------------------------------------------------------------------------ */
/* Rankine-Hugoniot jump (Appendix D, Eq. "RH condition"). */
void or_rh(double mach, double gamma, double *rho_ratio, double *T_ratio) {
    double M2 = mach * mach;
    *rho_ratio = (gamma + 1.0) * M2 / ((gamma - 1.0) * M2 + 2.0);
    *T_ratio = (2.0 * gamma * M2 - (gamma - 1.0)) * ((gamma - 1.0) * M2 + 2.0) / ((gamma + 1.0) * (gamma + 1.0) * M2);
}

/* ------------------------------------------------------------------------ */
/* One time step of Algorithm 2 on a 1D mesh of N interior cells plus one
 * Dirichlet ghost cell on each side (slots 0 and N+1).  State arrays are
 * (N+2) x 35 (M, beta) and (N+2) x 6 (g); speed (N+2) holds on entry the
 * characteristic speeds of the previous Transport (they set dt) and on exit
 * this Transport's speeds.
 *   dt = cfl * dx / max(speed_prev)
 *   Collision(dt/2) -> Transport(dt) [Newton, flux, neighbour gauge, LF, FV]
 *   -> Collision(dt/2) -> Hermite gauge and transform of M, beta.
 * relax_coef: tau = relax_coef / n (Maxwell molecules with mu ~ T).
 * out[0] = dt, out[1] = max new speed, out[2] = max |d rho| over the step. */
static void collide(double *M, const double *g, double dt, double Pr, double relax_coef) {
    double Mt[NP];
    or_esbgk(M, g, Pr, Mt);
    double tau = relax_coef / M[0];
    double r = dt / tau;
    for (int i = 0; i < NP; ++i) M[i] = (1.0 - r) * M[i] + r * Mt[i];
}

/* Numerical flux at the interface between cells a = c - 1 + side and
 * b = c + side, everything in the gauge g(c) of the cell being updated
 * (Eq. "The lax F convert" moves the neighbours there):
 *   scheme 0: local Lax-Friedrichs, Eq. "The lax F";
 *   scheme 1: two-step Lax-Wendroff, Eq. "The lax W": the interface moments
 *     M(n - 1/2) = (M_a + M_b)/2 + dt/(2 dx) (F_a - F_b), their parameters by
 *     Algorithm 1 and the flux of those parameters.  The solve runs in the
 *     Hermite gauge of the interface moments (cold start, beta = 0 there)
 *     and the flux is moved back to g(c): the maximum-entropy density of a
 *     moment vector does not depend on the gauge it is written in;
 *   scheme 2: FLIC, Eq. "The FLIC": F^LF + phi(r) (F^LW - F^LF) statistic by
 *     statistic with the van Leer limiter phi(r) = (r + |r|)/(1 + r) and
 *     r = (M_a - M_{a-1}) / (M_b - M_a) in g(c).  The statistics are the nine
 *     of the paper's 1D system (Eq. "Sufficient 35"), written as orthonormal
 *     combinations psi_j = v_j . phi of the 3D Hermite products (see
 *     flic_basis); each moment or flux vector x enters through v_j . x, and
 *     the blended part is sum_j phi_j (v_j . (F^LW - F^LF)) v_j.  Directions
 *     outside their span vanish for an axisymmetric flow and keep F^LF.  A
 *     zero denominator is read as r = 0 (first order there), phi = 0 at
 *     r = -1 (the printed form is 0/0 there), and cell a - 1 before the
 *     first cell is the ghost cell itself (r = 0).
 * An interface whose solve fails (non-finite, lambda cap, bad input, maxI
 * passes without meeting tol) or whose flux is not finite takes F^LF.  Interface solves add their status bits to
 * *ist. */
/* The nine statistics of the 1D system (Eq. "Sufficient 35": 1, u_x,
 * (u_x^2 - 1)/sqrt2, u_r^2/2 - 1, He_3(u_x)/sqrt6, He_4(u_x)/sqrt24,
 * u_r^4/8 - u_r^2 + 1, u_x (u_r^2 - 2)/2, (u_x^2 - 1)(u_r^2 - 2)/(2 sqrt2);
 * the eighth is printed with u_r^2 - 1, which is neither orthogonal to u_x
 * nor of unit norm under the Gaussian: read as u_r^2 - 2)
 * as unit vectors over the 3D orthonormal Hermite products, from
 * y^2 + z^2 = He_2(y) + He_2(z) + 2 and
 * (y^2 + z^2)^2 = He_4(y) + He_4(z) + 2 He_2(y) He_2(z) + 8 (He_2(y) + He_2(z)) + 8. */
static void flic_basis(double v[9][NP]) {
    memset(v, 0, sizeof(double) * 9 * NP);
    const double r2 = sqrt(0.5), q = sqrt(24.0) / 8.0;
    v[0][or_index_of(0, 0, 0)] = 1.0;
    v[1][or_index_of(1, 0, 0)] = 1.0;
    v[2][or_index_of(2, 0, 0)] = 1.0;
    v[3][or_index_of(0, 2, 0)] = v[3][or_index_of(0, 0, 2)] = r2;
    v[4][or_index_of(3, 0, 0)] = 1.0;
    v[5][or_index_of(4, 0, 0)] = 1.0;
    v[6][or_index_of(0, 4, 0)] = v[6][or_index_of(0, 0, 4)] = q;
    v[6][or_index_of(0, 2, 2)] = 0.5;
    v[7][or_index_of(1, 2, 0)] = v[7][or_index_of(1, 0, 2)] = r2;
    v[8][or_index_of(2, 2, 0)] = v[8][or_index_of(2, 0, 2)] = r2;
}

void or_flic_basis(double *v) { flic_basis((double (*)[NP])v); }

/* ------------------------------------------------------------------------ */
/* The paper's own system for axisymmetric 1D flow: the nine statistics
 * psi_j = v_j . phi of Eq. "Sufficient 35" with natural parameters alpha_j,
 * f ~ n exp(-|ubar|^2/2 + sum_{j>=1} alpha_j psi_j(ubar)), i.e. the 35-product
 * parameters beta = sum_j alpha_j v_j (alpha_0 = beta_0 = n).  Every integrand
 * here depends on (u_x, u_r) only, so a velocity-space rule with one azimuth
 * (K = 1) integrates it exactly in the angle. */
static void axi_beta(const double v[9][NP], const double *a, double *beta) {
    for (int i = 0; i < NP; ++i) beta[i] = 0.0;
    for (int j = 0; j < 9; ++j)
        for (int i = 0; i < NP; ++i) beta[i] += a[j] * v[j][i];
}

/* Algorithm 1 on the nine statistics: M9 = (n, psi moments), alpha [9]
 * in (start) / out (solution, alpha_0 = n).  Same steps and options as
 * or_solve, over the eight unknowns alpha_1..alpha_8. */
int or_solve_axi(int order, const double *g, const double *M9, double *alpha, const double *optv, int *iters,
                 double *res_out) {
    or_opts o; default_opts(&o);
    if (optv) { o.tol = optv[0]; o.maxI = (int)optv[1]; o.final_step = optv[2] != 0.0; }
    const int D = 8;
    double v[9][NP];
    flic_basis(v);
    const double n = M9[0];
    int st = 0;
    if (!(n > 0.0) || !isfinite(n)) { if (iters) *iters = 0; return ST_BADINPUT; }
    for (int j = 0; j < 9; ++j) if (!isfinite(M9[j]) || !isfinite(alpha[j])) { if (iters) *iters = 0; return ST_BADINPUT; }
    /* v_j . Ms = M9_j, so or_objective(beta(alpha), Ms) = log Z - sum_j alpha_j M9_j / n */
    double Ms[NP];
    axi_beta(v, M9, Ms);
    double a[9], da[9] = {0}, G[9] = {0}, b[NP], tr[9], m[NP], S[NP * NP], H[64], Lh[64], wv[8], rhs[8], dx[8];
    memcpy(a, alpha, sizeof(a));
    a[0] = n;
    axi_beta(v, a, b);
    double Lcur = or_objective(order, g, b, Ms);
    int it = 0, conv = 0;
    double res = INFINITY, step = 1.0;
    while (!conv && it <= o.maxI) {
        step = 2.0;
        int s = 0, sat = 0;
        while (!sat && s <= o.maxT) {
            step *= 0.5;
            for (int j = 0; j < 9; ++j) tr[j] = a[j] + step * da[j];
            tr[0] = n;
            axi_beta(v, tr, b);
            const double Lt = or_objective(order, g, b, Ms);
            double gd = 0.0;
            for (int j = 1; j < 9; ++j) gd += G[j] * step * da[j];
            const double LD = Lcur - Lt;
            sat = (LD - (-o.c * gd)) >= -(o.atol + o.rtol * fabs(LD));
            s += 1;
        }
        for (int j = 1; j < 9; ++j) a[j] += step * da[j];
        axi_beta(v, a, b);
        Lcur = or_objective(order, g, b, Ms);
        or_expect(order, g, b, NULL, m, S, NULL, NULL);
        double mj[9];
        for (int j = 0; j < 9; ++j) {
            mj[j] = 0.0;
            for (int i = 0; i < NP; ++i) mj[j] += v[j][i] * m[i];
        }
        for (int j = 1; j < 9; ++j) G[j] = mj[j] - M9[j] / n;
        for (int p = 0; p < D; ++p)
            for (int q = 0; q < D; ++q) {
                double e = 0.0;
                for (int i = 0; i < NP; ++i)
                    for (int k = 0; k < NP; ++k) e += v[p + 1][i] * S[i * NP + k] * v[q + 1][k];
                H[p * D + q] = e - mj[p + 1] * mj[q + 1];
            }
        double lambda = o.lambda0;
        int fail = cholesky(D, H, 0.0, Lh), tries = 0;
        while (fail) {
            if (tries >= o.max_lambda) break;
            fail = cholesky(D, H, lambda, Lh);
            st |= ST_LAMBDA;
            lambda *= o.lambda_mul;
            ++tries;
        }
        if (fail) { st |= ST_LAMBDA_CAP | ST_NONFINITE; ++it; break; }
        for (int p = 0; p < D; ++p) rhs[p] = -G[p + 1];
        solve_lower(D, Lh, rhs, wv);
        solve_upper_T(D, Lh, wv, dx);
        da[0] = 0.0;
        for (int p = 0; p < D; ++p) da[p + 1] = dx[p];
        double dg = 0.0;
        for (int j = 1; j < 9; ++j) dg += da[j] * G[j];
        res = 0.5 * fabs(dg);
        if (!isfinite(res)) { st |= ST_NONFINITE; ++it; break; }
        if (res <= o.tol) st |= ST_CONVERGED;
        if (step <= o.alpha_min) st |= ST_STAGNATED;
        conv = (res <= o.tol) || (step <= o.alpha_min);
        ++it;
    }
    if (!conv && !(st & ST_NONFINITE)) st |= ST_MAXITER;
    if (o.final_step && (st & ST_CONVERGED))
        for (int j = 1; j < 9; ++j) a[j] += da[j];
    memcpy(alpha, a, sizeof(a));
    alpha[0] = n;
    if (iters) *iters = it;
    if (res_out) *res_out = res;
    return st;
}

/* Flux of the nine moments, F9_j = v_j . F (F as in or_flux), and the
 * characteristic speed of the nine-statistic system: the spectral radius of
 * the 9 x 9 pencil (E[ubar_x psi psi^T], E[psi psi^T]) scaled by the gauge,
 * as the paper states it for its statistics (Eq. "The lax F"). */
void or_flux_axi(int order, const double *alpha, const double *g, double n, double *F9, double *speed) {
    double v[9][NP], b[NP], m[NP], S[NP * NP], X[NP], XS[NP * NP];
    flic_basis(v);
    double a[9];
    memcpy(a, alpha, sizeof(a));
    a[0] = n;
    axi_beta(v, a, b);
    or_expect(order, g, b, NULL, m, S, X, XS);
    for (int j = 0; j < 9; ++j) {
        double em = 0.0, ex = 0.0;
        for (int i = 0; i < NP; ++i) { em += v[j][i] * m[i]; ex += v[j][i] * X[i]; }
        if (F9) F9[j] = n * (g[0] * em + g[3] * ex);
    }
    if (!speed) return;
    double A[81], B[81], L[81], C[81], tmp[81], ev[9];
    for (int p = 0; p < 9; ++p)
        for (int q = 0; q < 9; ++q) {
            double ea = 0.0, eb = 0.0;
            for (int i = 0; i < NP; ++i)
                for (int k = 0; k < NP; ++k) {
                    ea += v[p][i] * XS[i * NP + k] * v[q][k];
                    eb += v[p][i] * S[i * NP + k] * v[q][k];
                }
            A[p * 9 + q] = ea;
            B[p * 9 + q] = eb;
        }
    if (cholesky(9, B, 0.0, L)) { *speed = NAN; return; }
    for (int col = 0; col < 9; ++col) {
        double bc[9], xc[9];
        for (int i = 0; i < 9; ++i) bc[i] = A[i * 9 + col];
        solve_lower(9, L, bc, xc);
        for (int i = 0; i < 9; ++i) tmp[i * 9 + col] = xc[i];
    }
    for (int row = 0; row < 9; ++row) {
        double br[9], xr[9];
        for (int i = 0; i < 9; ++i) br[i] = tmp[row * 9 + i];
        solve_lower(9, L, br, xr);
        for (int i = 0; i < 9; ++i) C[row * 9 + i] = xr[i];
    }
    for (int i = 0; i < 9; ++i)
        for (int j = i + 1; j < 9; ++j) C[i * 9 + j] = C[j * 9 + i] = 0.5 * (C[i * 9 + j] + C[j * 9 + i]);
    jacobi_eigen(9, C, ev, NULL);
    double lo = ev[0], hi = ev[0];
    for (int i = 1; i < 9; ++i) { if (ev[i] < lo) lo = ev[i]; if (ev[i] > hi) hi = ev[i]; }
    *speed = fmax(fabs(g[0] + g[3] * lo), fabs(g[0] + g[3] * hi));
}

/* Which system the shock step solves (Algorithm 2 on either set of
 * statistics): 35 (default) the Hermite products; 9 the paper's nine
 * statistics of axisymmetric flow (Appendix B), through or_solve_axi and
 * or_flux_axi.  The state stays the 35 moments and parameters: for an
 * axisymmetric flow they lie in the span of the orthonormal v_j, so
 * M9_j = v_j . M, alpha_j = v_j . beta, beta = sum_j alpha_j v_j and
 * F = sum_j F9_j v_j; the characteristic speed is the nine-statistic one. */
static int g_shock_stats = 35;
void or_set_shock_stats(int stats) { g_shock_stats = stats == 9 ? 9 : 35; }

static int shock_solve(int order, const double *g, const double *M, double *beta, const double *optv, int *it) {
    if (g_shock_stats != 9) return or_solve(order, g, M, beta, optv, it, NULL, NULL);
    double v[9][NP], M9[9], a[9];
    flic_basis(v);
    for (int j = 0; j < 9; ++j) {
        M9[j] = 0.0;
        a[j] = 0.0;
        for (int i = 0; i < NP; ++i) { M9[j] += v[j][i] * M[i]; a[j] += v[j][i] * beta[i]; }
    }
    const int st = or_solve_axi(order, g, M9, a, optv, it, NULL);
    axi_beta(v, a, beta);
    return st;
}

static void shock_flux(int order, const double *beta, const double *g, double n, double *F, double *speed) {
    if (g_shock_stats != 9) {
        or_flux(order, beta, g, n, F, speed, NULL, NULL);
        return;
    }
    double v[9][NP], a[9], F9[9];
    flic_basis(v);
    for (int j = 0; j < 9; ++j) {
        a[j] = 0.0;
        for (int i = 0; i < NP; ++i) a[j] += v[j][i] * beta[i];
    }
    or_flux_axi(order, a, g, n, F9, speed);
    for (int i = 0; i < NP; ++i) {
        F[i] = 0.0;
        for (int j = 0; j < 9; ++j) F[i] += F9[j] * v[j][i];
    }
}

/* Which ratio sets the FLIC limiter.  Eq. "The FLIC" writes the limiter
 * phi_{n-1/2} without a statistic index but its ratio r with the moments
 * M_i.  0 (default): one phi_j per statistic of the nine; 1: one phi per
 * interface, the smallest of the nine statistics' phi_j, from ratios taken
 * in the interface's Hermite gauge (both neighbours then use the same phi,
 * and the scheme stays conservative); 2: one phi per interface from the
 * number density M_0.  The limiter multiplies the nine statistics'
 * components of F^LW - F^LF. */
static int g_flic_mode = 0;
void or_set_flic_limiter(int mode) { g_flic_mode = (mode >= 0 && mode <= 2) ? mode : 0; }

static double dot35(const double *a, const double *b) {
    double s = 0.0;
    for (int i = 0; i < NP; ++i) s += a[i] * b[i];
    return s;
}

static void interface_flux(int order, int scheme, int c, int side, const double *M, const double *F, const double *g,
                           const double *speed, double dtdx, const double *optv, double *flux, int *ist) {
    const int a = c - 1 + side, b = c + side;
    double T[NP * NP], Ma[NP], Mb[NP], Fa[NP], Fb[NP], flf[NP];
    or_gauge_T(&g[6 * c], &g[6 * a], T);
    matvec35(T, &M[NP * a], Ma); matvec35(T, &F[NP * a], Fa);
    or_gauge_T(&g[6 * c], &g[6 * b], T);
    matvec35(T, &M[NP * b], Mb); matvec35(T, &F[NP * b], Fb);
    const double lam = fmax(speed[a], speed[b]);
    for (int i = 0; i < NP; ++i) flf[i] = 0.5 * (Fa[i] + Fb[i]) + 0.5 * lam * (Ma[i] - Mb[i]);
    if (scheme == 0) {
        memcpy(flux, flf, sizeof(flf));
        return;
    }
    double MI[NP], gI[6], MH[NP], bI[NP], FI[NP], flw[NP];
    for (int i = 0; i < NP; ++i) MI[i] = 0.5 * (Ma[i] + Mb[i]) + 0.5 * dtdx * (Fa[i] - Fb[i]);
    or_hermite_gauge(MI, &g[6 * c], 1, gI);
    or_transform_M(gI, &g[6 * c], MI, MH);
    memset(bI, 0, sizeof(bI));
    bI[0] = MH[0];
    int it = 0;
    const int sI = shock_solve(order, gI, MH, bI, optv, &it);
    *ist |= sI;
    shock_flux(order, bI, gI, MH[0], FI, NULL);
    int ok = (sI & (ST_NONFINITE | ST_LAMBDA_CAP | ST_BADINPUT | ST_MAXITER)) == 0;
    for (int i = 0; i < NP; ++i) ok = ok && isfinite(FI[i]);
    if (!ok) {
        memcpy(flux, flf, sizeof(flf));
        return;
    }
    or_gauge_T(&g[6 * c], gI, T);
    matvec35(T, FI, flw);
    if (scheme == 1) {
        memcpy(flux, flw, sizeof(flw));
        return;
    }
    const int aa = a > 0 ? a - 1 : a;
    double Maa[NP];
    or_gauge_T(&g[6 * c], &g[6 * aa], T);
    matvec35(T, &M[NP * aa], Maa);
    double v[9][NP], D[NP];
    flic_basis(v);
    for (int i = 0; i < NP; ++i) {
        D[i] = flw[i] - flf[i];
        flux[i] = flf[i];
    }
    /* Mode 1 (the smallest phi per interface): its ratios are taken in the
     * interface's own Hermite gauge gI, which both neighbours share, so the
     * two sides of the interface use the same phi and the scheme stays
     * conservative; modes 0 and 2 take them in the updated cell's gauge
     * g(c), as every quantity of cell c. */
    const double *ra = Ma, *raa = Maa, *rb = Mb;
    double MaI[NP], MaaI[NP], MbI[NP];
    if (g_flic_mode == 1) {
        or_gauge_T(gI, &g[6 * a], T); matvec35(T, &M[NP * a], MaI);
        or_gauge_T(gI, &g[6 * aa], T); matvec35(T, &M[NP * aa], MaaI);
        or_gauge_T(gI, &g[6 * b], T); matvec35(T, &M[NP * b], MbI);
        ra = MaI; raa = MaaI; rb = MbI;
    }
    double phis[9];
    for (int j = 0; j < 9; ++j) {
        const double num = dot35(v[j], ra) - dot35(v[j], raa), den = dot35(v[j], rb) - dot35(v[j], ra);
        const double r = den != 0.0 ? num / den : 0.0;
        /* (r + |r|)/(1 + r): 0 for r <= 0 (also at r = -1, where the printed
         * form is 0/0), 2r/(1 + r) = 2/(1 + 1/r) for r > 0 (2 as r -> inf) */
        phis[j] = r > 0.0 ? 2.0 / (1.0 + 1.0 / r) : 0.0;
    }
    if (g_flic_mode != 0) {
        /* one limiter per interface */
        double phi = phis[0];
        if (g_flic_mode == 1)
            for (int j = 1; j < 9; ++j) phi = fmin(phi, phis[j]);
        for (int j = 0; j < 9; ++j) phis[j] = phi;
    }
    for (int j = 0; j < 9; ++j) {
        const double phi = phis[j];
        if (phi == 0.0) continue;
        const double d = phi * dot35(v[j], D);
        for (int i = 0; i < NP; ++i) flux[i] += d * v[j][i];
    }
}

/* The interface flux above for cells c - 1 + side and c + side of the arrays
 * M, F, g, speed (cell c - 2 + side must exist or be the first cell);
 * returns the interface solve's status bits (0 for scheme 0). */
int or_interface_flux(int order, int scheme, int c, int side, const double *M, const double *F, const double *g,
                      const double *speed, double dtdx, const double *optv, double *flux) {
    get_rule(order);
    int ist = 0;
    interface_flux(order, scheme, c, side, M, F, g, speed, dtdx, optv, flux, &ist);
    return ist;
}

void or_shock_step(int order, int N, double dx, double cfl, double Pr, double relax_coef,
                   double *M, double *beta, double *g, double *speed, int *status, int *iters,
                   const double *optv, int nthreads, double *out, double *cond, int scheme, int *iface_status) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    get_rule(order);
    int NT = N + 2;
    double smax = 0.0;
    for (int c = 0; c < NT; ++c) if (speed[c] > smax) smax = speed[c];
    double dt = cfl * dx / smax;
    double *rho0 = malloc(sizeof(double) * NT), *F = malloc(sizeof(double) * NP * NT), *Mn = malloc(sizeof(double) * NP * NT);
    for (int c = 0; c < NT; ++c) rho0[c] = M[NP * c];
    #pragma omp parallel for schedule(dynamic, 1)
    for (int c = 1; c <= N; ++c) {
        collide(&M[NP * c], &g[6 * c], 0.5 * dt, Pr, relax_coef);
        int it = 0;
        int st = shock_solve(order, &g[6 * c], &M[NP * c], &beta[NP * c], optv, &it);
        if (status) status[c] = st;
        if (iters) iters[c] = it;
        if (cond) cond[c] = or_cond_estimate(order, &g[6 * c], &beta[NP * c]);
    }
    #pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < NT; ++c) {
        double bb[NP];
        memcpy(bb, &beta[NP * c], sizeof(bb));
        if (c == 0 || c == N + 1) for (int i = 0; i < NP; ++i) bb[i] = 0.0;
        shock_flux(order, bb, &g[6 * c], M[NP * c], &F[NP * c], &speed[c]);
    }
    #pragma omp parallel for schedule(dynamic, 1)
    for (int c = 1; c <= N; ++c) {
        double fl[NP], fr[NP];
        int ist = 0;
        interface_flux(order, scheme, c, 0, M, F, g, speed, dt / dx, optv, fl, &ist);
        interface_flux(order, scheme, c, 1, M, F, g, speed, dt / dx, optv, fr, &ist);
        for (int i = 0; i < NP; ++i) Mn[NP * c + i] = M[NP * c + i] + dt / dx * (fl[i] - fr[i]);
        if (iface_status) iface_status[c] = ist;
    }
    double dmax = 0.0, snew = 0.0;
    for (int c = 0; c < NT; ++c) if (speed[c] > snew) snew = speed[c];
    #pragma omp parallel for schedule(static) reduction(max:dmax)
    for (int c = 1; c <= N; ++c) {
        double *Mc = &Mn[NP * c];
        collide(Mc, &g[6 * c], 0.5 * dt, Pr, relax_coef);
        double gH[6], bt[NP];
        or_hermite_gauge(Mc, &g[6 * c], 1, gH);
        or_transform_M(gH, &g[6 * c], Mc, &M[NP * c]);
        or_transform_beta(gH, &g[6 * c], &beta[NP * c], bt);
        memcpy(&beta[NP * c], bt, sizeof(bt));
        memcpy(&g[6 * c], gH, sizeof(gH));
        double d = fabs(M[NP * c] - rho0[c]);
        if (d > dmax) dmax = d;
    }
    out[0] = dt; out[1] = snew; out[2] = dmax;
    free(rho0); free(F); free(Mn);
}

/* Flux and speed of a batch of cells (used to prime the first step's dt). */
void or_flux_batch(int order, int64_t B, const double *M, const double *beta, const double *g, double *F, double *speed, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    get_rule(order);
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < B; ++c)
        or_flux(order, &beta[NP * c], &g[6 * c], M[NP * c], F ? &F[NP * c] : NULL, speed ? &speed[c] : NULL, NULL, NULL);
}

/* ------------------------------------------------------------------------ */
/* Synthetic solve targets: the moments, in the distribution's own Hermite
 * gauge (per-axis), of p(c) ~ exp(-|c|^2/2 + sum_k a_k c^k - sum_k b_k c^k),
 * c = (u - v)/sqrt(T): a = 10 cubic coefficients in the multi-index order of
 * the degree-3 statistics, b = 6 coefficients of c_x^4, c_y^4, c_z^4,
 * c_x^2 c_y^2, c_x^2 c_z^2, c_y^2 c_z^2.  Density n = 1.  The expectations use
 * a tensor Gauss-Hermite rule of the given order in c. */
void or_target_moments(int order, const double *v, double T, const double *a, const double *b, double *M, double *gH) {
    build_index();
    const rule_t *r = get_rule(order);
    int Q = r->Q;
    double *e = malloc(sizeof(double) * Q), *p = malloc(sizeof(double) * Q);
    static const int quart[6][3] = {{4, 0, 0}, {0, 4, 0}, {0, 0, 4}, {2, 2, 0}, {2, 0, 2}, {0, 2, 2}};
    /* The rule is re-centred on the distribution: c = mu + sc * z with z on
     * the Gauss-Hermite nodes, so the integrand p(c(z)) / N(z) is smooth and
     * the rule converges fast.  Three passes refine (mu, sc) to the mean and
     * standard deviation of c; the last frame is the Hermite gauge. */
    double mu[3] = {0, 0, 0}, sc[3] = {1, 1, 1};
    for (int pass = 0; pass < 4; ++pass) {
        double emax = -INFINITY;
        for (int q = 0; q < Q; ++q) {
            const double *z = &r->u[3 * q];
            double c[3];
            for (int ax = 0; ax < 3; ++ax) c[ax] = mu[ax] + sc[ax] * z[ax];
            double ex = r->logw[q] + 0.5 * (z[0] * z[0] + z[1] * z[1] + z[2] * z[2]);
            ex -= 0.5 * (c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
            double pw[3][5];
            for (int ax = 0; ax < 3; ++ax) { pw[ax][0] = 1.0; for (int e = 1; e < 5; ++e) pw[ax][e] = pw[ax][e - 1] * c[ax]; }
            for (int k = 0; k < 10; ++k) {
                int *ix = g_idx[10 + k];
                ex += a[k] * pw[0][ix[0]] * pw[1][ix[1]] * pw[2][ix[2]];
            }
            for (int k = 0; k < 6; ++k) ex -= b[k] * pw[0][quart[k][0]] * pw[1][quart[k][1]] * pw[2][quart[k][2]];
            e[q] = ex;
            if (ex > emax) emax = ex;
        }
        double Z = 0.0;
        for (int q = 0; q < Q; ++q) { p[q] = exp(e[q] - emax); Z += p[q]; }
        for (int q = 0; q < Q; ++q) p[q] /= Z;
        double mean[3] = {0, 0, 0}, var[3] = {0, 0, 0};
        for (int q = 0; q < Q; ++q) for (int ax = 0; ax < 3; ++ax) mean[ax] += p[q] * (mu[ax] + sc[ax] * r->u[3 * q + ax]);
        for (int q = 0; q < Q; ++q) for (int ax = 0; ax < 3; ++ax) {
            double d = mu[ax] + sc[ax] * r->u[3 * q + ax] - mean[ax];
            var[ax] += p[q] * d * d;
        }
        if (pass == 3) {
            /* Hermite gauge in u = v + sqrt(T) c, and the moments there. */
            for (int ax = 0; ax < 3; ++ax) { gH[ax] = v[ax] + sqrt(T) * mean[ax]; gH[3 + ax] = sqrt(T * var[ax]); }
            for (int i = 0; i < NP; ++i) M[i] = 0.0;
            for (int q = 0; q < Q; ++q) {
                double ub[3], ph[NP];
                for (int ax = 0; ax < 3; ++ax) ub[ax] = (v[ax] + sqrt(T) * (mu[ax] + sc[ax] * r->u[3 * q + ax]) - gH[ax]) / gH[3 + ax];
                or_phi(ub, ph);
                for (int i = 0; i < NP; ++i) M[i] += p[q] * ph[i];
            }
        }
        for (int ax = 0; ax < 3; ++ax) { mu[ax] = mean[ax]; sc[ax] = sqrt(var[ax]); }
    }
    free(e); free(p);
}

void or_target_batch(int order, int64_t B, const double *v, const double *T, const double *a, const double *b, double *M, double *gH, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    get_rule(order);
    #pragma omp parallel for schedule(dynamic, 8)
    for (int64_t c = 0; c < B; ++c)
        or_target_moments(order, &v[3 * c], T[c], &a[10 * c], &b[6 * c], &M[NP * c], &gH[6 * c]);
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

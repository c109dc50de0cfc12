// shock.cu -- time steps of Algorithm 2 on 1D normal shocks (Appendix D),
// for one problem or a packed batch of independent problems.
//
// One step, every problem p of the batch at once:
//   dt_p = cfl dx_p / max speed of p's previous transport       (k_dt)
//   Collision(dt_p/2), ES-BGK, Eq. "source update"               (k_collide)
//   Transport(dt_p): Newton (fused or plain back-end), flux and speed,
//     neighbour gauge transform + local Lax-Friedrichs + finite volume
//     (Eqs. "The lax F", "The lax F convert", "The ME equation fvm 2")
//                                                                (k_stencil)
//     or, for Lax-Wendroff / FLIC problems, the interface moments of Eq.
//     "The lax W" in their Hermite gauge (k_iface_state), Newton and flux
//     at every interface, then the LW or FLIC fluxes + finite volume
//                                                                (k_stencil2)
//   Collision(dt_p/2)                                            (k_collide)
//   Hermite gauge and transform of M and beta                    (k_regauge)
// Problem p owns the contiguous cells [off_p, off_p + N_p + 2): a Dirichlet
// ghost cell at each end holding the Rankine-Hugoniot Maxwellian in its own
// Hermite gauge (beta = 0, never updated) and N_p interior cells.  Every
// kernel works per cell and every reduction per problem, so a problem's
// result does not depend on which other problems share the batch.  All
// per-step scalars live in device memory, so a step can be captured in a
// CUDA graph when the fused Newton back-end is used.
#include <math.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "shock.h"

using namespace mem;

namespace {

// Hermite-product expectations of the Gaussian N(mu, S) in the gauge frame:
// E[He_a(x) He_b(y) He_c(z)] equals the moment of a formal Gaussian with
// mean mu and covariance K = S - I, built by the recursion
//   m_{alpha + e_i} = mu_i m_alpha + sum_j alpha_j K_ij m_{alpha - e_j}.
template <typename R>
__host__ __device__ __forceinline__ void gaussian_hermite(const R mu[3], const R K[3][3], R n, R *out) {
    R m[NP];
    m[0] = 1;
#pragma unroll
    for (int k = 1; k < NP; ++k) {
        const int al[3] = {exp_a(k), exp_b(k), exp_c(k)};
        const int i = al[0] > 0 ? 0 : (al[1] > 0 ? 1 : 2);
        int be[3] = {al[0], al[1], al[2]};
        be[i] -= 1;
        R v = mu[i] * m[idx3(be[0], be[1], be[2])];
#pragma unroll
        for (int j = 0; j < 3; ++j)
            if (be[j] > 0) {
                int g2[3] = {be[0], be[1], be[2]};
                g2[j] -= 1;
                v += (R)be[j] * K[i][j] * m[idx3(g2[0], g2[1], g2[2])];
            }
        m[k] = v;
    }
    const R fact[5] = {1, 1, 2, 6, 24};
#pragma unroll
    for (int k = 0; k < NP; ++k) out[k] = n * m[k] / sqrt(fact[exp_a(k)] * fact[exp_b(k)] * fact[exp_c(k)]);
}

// ES-BGK target (Appendix A): Gaussian with the cell's n and mean velocity and
// covariance Sigma = T/Pr I + (1 - 1/Pr) P/n, in the cell's gauge.
__device__ __forceinline__ void esbgk_target(const float *M, const float *g, float Pr, float *Mt) {
    const float n = M[0];
    const int i1[3] = {idx3(1, 0, 0), idx3(0, 1, 0), idx3(0, 0, 1)};
    float mb[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) mb[a] = M[i1[a]] / n;
    float E2[3][3];
    E2[0][0] = 1.41421356f * M[idx3(2, 0, 0)] / n + 1.f;
    E2[1][1] = 1.41421356f * M[idx3(0, 2, 0)] / n + 1.f;
    E2[2][2] = 1.41421356f * M[idx3(0, 0, 2)] / n + 1.f;
    E2[0][1] = E2[1][0] = M[idx3(1, 1, 0)] / n;
    E2[0][2] = E2[2][0] = M[idx3(1, 0, 1)] / n;
    E2[1][2] = E2[2][1] = M[idx3(0, 1, 1)] / n;
    float P[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) P[a][b] = g[3 + a] * g[3 + b] * (E2[a][b] - mb[a] * mb[b]);
    const float T = (P[0][0] + P[1][1] + P[2][2]) / 3.f;
    float K[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float sig = (a == b ? T / Pr : 0.f) + (1.f - 1.f / Pr) * P[a][b];
            K[a][b] = sig / (g[3 + a] * g[3 + b]) - (a == b ? 1.f : 0.f);
        }
    gaussian_hermite<float>(mb, K, n, Mt);
}

// Cells per block of the stencil-type kernels below.  Each block moves its
// rows of the row-major state arrays between HBM and shared memory with
// consecutive threads on consecutive floats (coalesced), and each thread
// computes one cell from shared memory.
constexpr int SB = 64;

// Rows [r0, r0 + N) of a row-major array of W floats per row into shared
// memory (row pitch W); rows outside [0, NT) are left unset.  Unrolled so
// that sixteen loads per thread are in flight together.
template <int W, int N>
__device__ __forceinline__ void stage_in(float *dst, const float *src, int r0, int NT) {
    constexpr int CNT = W * N, IT = (CNT + SB - 1) / SB, U = 16;
    const int lo = (max(r0, 0) - r0) * W, hi = (min(r0 + N, NT) - r0) * W;
    const float *s = src + (ptrdiff_t)r0 * W;
#pragma unroll
    for (int j0 = 0; j0 < IT; j0 += U) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = threadIdx.x + (j0 + u) * SB;
            v[u] = (j0 + u < IT && t >= lo && t < hi) ? s[t] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = threadIdx.x + (j0 + u) * SB;
            if (j0 + u < IT && t < CNT) dst[t] = v[u];
        }
    }
}

// Rows [r0, r0 + N) back from shared memory, only those whose live flag
// (shared memory, one per row) is set and that lie below NT.
template <int W, int N>
__device__ __forceinline__ void stage_out(float *dst, const float *src, int r0, int NT, const unsigned char *live) {
    constexpr int CNT = W * N, IT = (CNT + SB - 1) / SB;
    const int hi = (min(r0 + N, NT) - r0) * W;
    float *d = dst + (ptrdiff_t)r0 * W;
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        const int t = threadIdx.x + j * SB;
        if (t < hi && live[t / W]) d[t] = src[t];
    }
}

__global__ void __launch_bounds__(SB) k_collide(float *__restrict__ M, const float *__restrict__ g,
                                                const int *__restrict__ pid, const unsigned char *__restrict__ interior,
                                                const ShockProb *__restrict__ prm, const ShockScalars *__restrict__ sc,
                                                int NT, float frac, float *rho0) {
    __shared__ float sM[SB * NP], sg[SB * 6];
    __shared__ unsigned char sl[SB];
    const int c0 = blockIdx.x * SB, c = c0 + threadIdx.x;
    stage_in<NP, SB>(sM, M, c0, NT);
    stage_in<6, SB>(sg, g, c0, NT);
    const bool live = c < NT && interior[c];
    sl[threadIdx.x] = live;
    __syncthreads();
    if (live) {
        const int p = pid[c];
        float *row = sM + threadIdx.x * NP;
        float m[NP], gg[6], mt[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) m[k] = row[k];
#pragma unroll
        for (int k = 0; k < 6; ++k) gg[k] = sg[threadIdx.x * 6 + k];
        if (rho0) rho0[c] = m[0];
        esbgk_target(m, gg, prm[p].Pr, mt);
        const float r = frac * sc[p].dt * m[0] / prm[p].relax;  // dt' / tau, tau = relax / n
#pragma unroll
        for (int k = 0; k < NP; ++k) row[k] = (1.f - r) * m[k] + r * mt[k];
    }
    __syncthreads();
    stage_out<NP, SB>(M, sM, c0, NT, sl);
}

// Local Lax-Friedrichs finite-volume update of interior cell c in its own
// gauge: M_c += dt/dx (F^LF_{c-1/2} - F^LF_{c+1/2}), neighbours moved to g_c.
// Arguments are the rows of cells c - 1, c, c + 1 (M, F, gauge) and their
// speeds; out receives the updated row.  One compiled copy serves k_stencil
// (rows in shared memory) and the LF problems of k_stencil2 (rows in HBM), so
// a problem's result does not depend on the schemes of the batch it shares.
__device__ __noinline__ void lf_update(const float *Ml, const float *M0, const float *Mr, const float *Fl,
                                       const float *F0, const float *Fr, const float *gl_, const float *g0_,
                                       const float *gr_, float sl, float s0, float sr, float *out, float r) {
    float g0[6], gl[6], gr[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        g0[k] = g0_[k];
        gl[k] = gl_[k];
        gr[k] = gr_[k];
    }
    const float ll = fmaxf(sl, s0), lr = fmaxf(s0, sr);
    float acc[NP], x[NP], y[NP];
    AxisMap T[3];
    // F^LF_{c-1/2} - F^LF_{c+1/2} = 0.5(Fl + F0) + 0.5 ll (Ml - M0) - 0.5(F0 + Fr) - 0.5 lr (M0 - Mr)
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = -0.5f * (ll + lr) * M0[k];
    gauge_maps(g0, gl, T);
#pragma unroll
    for (int k = 0; k < NP; ++k) x[k] = Ml[k];
    apply_T(T, x, y);
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] += 0.5f * ll * y[k];
#pragma unroll
    for (int k = 0; k < NP; ++k) x[k] = Fl[k];
    apply_T(T, x, y);
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] += 0.5f * y[k];
    gauge_maps(g0, gr, T);
#pragma unroll
    for (int k = 0; k < NP; ++k) x[k] = Mr[k];
    apply_T(T, x, y);
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] += 0.5f * lr * y[k];
#pragma unroll
    for (int k = 0; k < NP; ++k) x[k] = Fr[k];
    apply_T(T, x, y);
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] -= 0.5f * y[k];
#pragma unroll
    for (int k = 0; k < NP; ++k) out[k] = M0[k] + r * acc[k];
}

// LF step of every interior cell: rows c0 - 1 .. c0 + SB of M, F, g and
// speed staged in shared memory, the updated rows staged and stored back.
__global__ void __launch_bounds__(SB) k_stencil(const float *__restrict__ M, const float *__restrict__ F,
                                                const float *__restrict__ g, const float *__restrict__ speed,
                                                float *__restrict__ Mn, const int *__restrict__ pid,
                                                const unsigned char *__restrict__ interior,
                                                const ShockProb *__restrict__ prm,
                                                const ShockScalars *__restrict__ sc, int NT) {
    __shared__ float sM[(SB + 2) * NP], sF[(SB + 2) * NP], sg[(SB + 2) * 6], ss[SB + 2], sO[SB * NP];
    __shared__ unsigned char sl[SB];
    const int c0 = blockIdx.x * SB, c = c0 + threadIdx.x;
    stage_in<NP, SB + 2>(sM, M, c0 - 1, NT);
    stage_in<NP, SB + 2>(sF, F, c0 - 1, NT);
    stage_in<6, SB + 2>(sg, g, c0 - 1, NT);
    stage_in<1, SB + 2>(ss, speed, c0 - 1, NT);
    // an interior cell's neighbours are cells of its own problem (or its ghosts)
    const bool live = c < NT && interior[c];
    sl[threadIdx.x] = live;
    __syncthreads();
    if (live) {
        const int p = pid[c], i = threadIdx.x + 1;  // row of c in the staged arrays
        lf_update(sM + (i - 1) * NP, sM + i * NP, sM + (i + 1) * NP, sF + (i - 1) * NP, sF + i * NP,
                  sF + (i + 1) * NP, sg + (i - 1) * 6, sg + i * 6, sg + (i + 1) * 6, ss[i - 1], ss[i], ss[i + 1],
                  sO + threadIdx.x * NP, sc[p].dt / prm[p].dx);
    }
    __syncthreads();
    stage_out<NP, SB>(Mn, sO, c0, NT, sl);
}

// Status bits of an interface solve whose parameters are not used: the
// solve stopped (non-finite values, lambda cap), its input was bad, or it
// ran out of passes without meeting tol.
constexpr int IFACE_FAILED = MEM_ST_NONFINITE | MEM_ST_LAMBDA_CAP | MEM_ST_BADINPUT | MEM_ST_MAXITER;

// Interface moments of Eq. "The lax W" between cells c - 1 and c (iface[c]
// set), formed in the gauge of cell c and moved to their own Hermite gauge
// (axisymmetric form).  The Newton start is the interface's parameters of
// the previous step carried to the new gauge (the density they describe),
// or beta = 0 there where that solve failed.  Entries without an interface
// get a copy of cell c, so that every row the solver and the flux kernel see
// is valid.
__global__ void __launch_bounds__(128) k_iface_state(const float *__restrict__ M, const float *__restrict__ F,
                                                     const float *__restrict__ g, const float *__restrict__ beta,
                                                     float *__restrict__ MI, float *__restrict__ gI,
                                                     float *__restrict__ betaI,
                                                     const int32_t *__restrict__ statusI,
                                                     const unsigned char *__restrict__ iface,
                                                     const int *__restrict__ pid, const ShockProb *__restrict__ prm,
                                                     const ShockScalars *__restrict__ sc, int NT) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= NT) return;
    if (!iface[c]) {
        for (int k = 0; k < NP; ++k) {
            MI[(size_t)c * NP + k] = M[(size_t)c * NP + k];
            betaI[(size_t)c * NP + k] = beta[(size_t)c * NP + k];
        }
        for (int k = 0; k < 6; ++k) gI[(size_t)c * 6 + k] = g[(size_t)c * 6 + k];
        return;
    }
    const int p = pid[c];
    const float h = 0.5f * sc[p].dt / prm[p].dx;
    float gb[6], ga[6], gh[6], m[NP], x[NP], y[NP];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        gb[k] = g[(size_t)c * 6 + k];
        ga[k] = g[(size_t)(c - 1) * 6 + k];
    }
    AxisMap T[3];
    gauge_maps(gb, ga, T);
    // M(n - 1/2) = (M_a + M_b)/2 + dt/(2 dx) (F_a - F_b), a = c - 1, b = c
#pragma unroll
    for (int k = 0; k < NP; ++k) x[k] = M[(size_t)(c - 1) * NP + k];
    apply_T(T, x, y);
#pragma unroll
    for (int k = 0; k < NP; ++k) m[k] = 0.5f * (y[k] + M[(size_t)c * NP + k]);
#pragma unroll
    for (int k = 0; k < NP; ++k) x[k] = F[(size_t)(c - 1) * NP + k];
    apply_T(T, x, y);
#pragma unroll
    for (int k = 0; k < NP; ++k) m[k] += h * (y[k] - F[(size_t)c * NP + k]);
    hermite_gauge(m, gb, 1, gh);
    gauge_maps(gh, gb, T);
    apply_T(T, m, y);
    // warm start: previous parameters (gauge gI[c]) carried to gh
    float gp[6], bp[NP];
    bool ok = (statusI[c] & IFACE_FAILED) == 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) gp[k] = gI[(size_t)c * 6 + k];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        bp[k] = betaI[(size_t)c * NP + k];
        ok = ok && isfinite(bp[k]);
    }
    transform_beta(gh, gp, bp, m);
#pragma unroll
    for (int k = 1; k < NP; ++k) ok = ok && isfinite(m[k]);
    // carried parameters, or beta = 0 (the gauge's Maxwellian) as a whole
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        MI[(size_t)c * NP + k] = y[k];
        betaI[(size_t)c * NP + k] = k == 0 ? y[0] : (ok ? m[k] : 0.f);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) gI[(size_t)c * 6 + k] = gh[k];
}

// The nine statistics of the paper's 1D system (Eq. "Sufficient 35": 1, u_x,
// (u_x^2-1)/sqrt2, u_r^2/2-1, He_3(u_x)/sqrt6, He_4(u_x)/sqrt24,
// u_r^4/8-u_r^2+1, u_x(u_r^2-2)/2, (u_x^2-1)(u_r^2-2)/(2 sqrt2)) are unit
// vectors v_j over the 3D Hermite products; project9 gives v_j . x and
// add9 adds sum_j c_j v_j.  FLIC limits these nine; the other directions
// vanish for an axisymmetric flow, and a per-product limiter there only
// amplifies FP32 noise in y <-> z symmetric pairs.
constexpr float FL_R2 = 0.70710678118654752f;  // 1/sqrt2
constexpr float FL_Q = 0.61237243569579452f;   // sqrt(24)/8

__device__ __forceinline__ void project9(const float *x, float *q) {
    q[0] = x[idx3(0, 0, 0)];
    q[1] = x[idx3(1, 0, 0)];
    q[2] = x[idx3(2, 0, 0)];
    q[3] = FL_R2 * (x[idx3(0, 2, 0)] + x[idx3(0, 0, 2)]);
    q[4] = x[idx3(3, 0, 0)];
    q[5] = x[idx3(4, 0, 0)];
    q[6] = FL_Q * (x[idx3(0, 4, 0)] + x[idx3(0, 0, 4)]) + 0.5f * x[idx3(0, 2, 2)];
    q[7] = FL_R2 * (x[idx3(1, 2, 0)] + x[idx3(1, 0, 2)]);
    q[8] = FL_R2 * (x[idx3(2, 2, 0)] + x[idx3(2, 0, 2)]);
}

__device__ __forceinline__ void add9(float *f, const float *c) {
    f[idx3(0, 0, 0)] += c[0];
    f[idx3(1, 0, 0)] += c[1];
    f[idx3(2, 0, 0)] += c[2];
    f[idx3(0, 2, 0)] += FL_R2 * c[3];
    f[idx3(0, 0, 2)] += FL_R2 * c[3];
    f[idx3(3, 0, 0)] += c[4];
    f[idx3(4, 0, 0)] += c[5];
    f[idx3(0, 4, 0)] += FL_Q * c[6];
    f[idx3(0, 0, 4)] += FL_Q * c[6];
    f[idx3(0, 2, 2)] += 0.5f * c[6];
    f[idx3(1, 2, 0)] += FL_R2 * c[7];
    f[idx3(1, 0, 2)] += FL_R2 * c[7];
    f[idx3(2, 2, 0)] += FL_R2 * c[8];
    f[idx3(2, 0, 2)] += FL_R2 * c[8];
}

// Finite-volume update of interior cell c with Lax-Wendroff or FLIC fluxes
// (per problem; LF problems of a mixed batch take the LF flux), everything in
// the gauge g(c).  At the interface between cells a and b = a + 1:
//   F^LF = (F_a + F_b)/2 + lambda/2 (M_a - M_b), Eq. "The lax F";
//   F^LW = T(g(c), g_I) F(beta_I; g_I), the interface solve's flux;
//   FLIC: F^LF + sum_j phi_j (v_j . (F^LW - F^LF)) v_j over the nine 1D
//   statistics (project9) with the van Leer limiter phi(r) = (r + |r|)/(1 + r),
//   r_j = v_j . (M_a - M_{a-1}) / v_j . (M_b - M_a); r = 0 where the
//   denominator is 0, phi = 0 for r <= 0 (also r = -1, where the printed form
//   is 0/0), and the ghost cell standing in for the cell before the first one.
//   flic = 0 (default): one phi_j per statistic; flic = 1: one phi per
//   interface, the smallest phi_j with the ratios taken in the interface's
//   Hermite gauge (the same phi on both sides: conservative); flic = 2: the
//   density's phi for all (the printed phi_{n-1/2} carries no statistic
//   index, its ratio is written with the moments M_i).
// An interface whose Newton solve failed (IFACE_FAILED) or whose flux is not
// finite takes F^LF.
__global__ void __launch_bounds__(128) k_stencil2(const float *__restrict__ M, const float *__restrict__ F,
                                                  const float *__restrict__ g, const float *__restrict__ speed,
                                                  const float *__restrict__ FI, const float *__restrict__ gI,
                                                  const int32_t *__restrict__ statusI,
                                                  float *__restrict__ Mn, const int *__restrict__ pid,
                                                  const unsigned char *__restrict__ interior,
                                                  const ShockProb *__restrict__ prm,
                                                  const ShockScalars *__restrict__ sc, int NT) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= NT || !interior[c]) return;
    const int p = pid[c];
    const int scheme = prm[p].scheme, off = prm[p].off;
    if (scheme == MEM_SCHEME_LF) {
        lf_update(M + (size_t)(c - 1) * NP, M + (size_t)c * NP, M + (size_t)(c + 1) * NP, F + (size_t)(c - 1) * NP,
                  F + (size_t)c * NP, F + (size_t)(c + 1) * NP, g + (size_t)(c - 1) * 6, g + (size_t)c * 6,
                  g + (size_t)(c + 1) * 6, speed[c - 1], speed[c], speed[c + 1], Mn + (size_t)c * NP,
                  sc[p].dt / prm[p].dx);
        return;
    }
    float g0[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) g0[k] = g[(size_t)c * 6 + k];
    float acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = 0.f;
    for (int side = 0; side < 2; ++side) {
        const int a = c - 1 + side, b = c + side;
        float ma[NP], mb[NP], f[NP], x[NP], y[NP], gn[6];
        AxisMap T[3];
        // M_a, M_b in g(c) (one of them is cell c itself)
#pragma unroll
        for (int k = 0; k < 6; ++k) gn[k] = g[(size_t)(side ? b : a) * 6 + k];
        gauge_maps(g0, gn, T);
#pragma unroll
        for (int k = 0; k < NP; ++k) x[k] = M[(size_t)(side ? b : a) * NP + k];
        apply_T(T, x, y);
        const float lam = fmaxf(speed[a], speed[b]);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float own = M[(size_t)c * NP + k];
            ma[k] = side ? own : y[k];
            mb[k] = side ? y[k] : own;
            f[k] = 0.5f * lam * (ma[k] - mb[k]) + 0.5f * F[(size_t)c * NP + k];
        }
#pragma unroll
        for (int k = 0; k < NP; ++k) x[k] = F[(size_t)(side ? b : a) * NP + k];
        apply_T(T, x, y);
#pragma unroll
        for (int k = 0; k < NP; ++k) f[k] += 0.5f * y[k];
        bool lw_ok = (statusI[b] & IFACE_FAILED) == 0;
        if (lw_ok) {
            float w[NP];
#pragma unroll
            for (int k = 0; k < 6; ++k) gn[k] = gI[(size_t)b * 6 + k];
            gauge_maps(g0, gn, T);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                x[k] = FI[(size_t)b * NP + k];
                lw_ok = lw_ok && isfinite(x[k]);
            }
            apply_T(T, x, w);
            if (lw_ok && scheme == MEM_SCHEME_LW) {
#pragma unroll
                for (int k = 0; k < NP; ++k) f[k] = w[k];
            } else if (lw_ok) {
                const int aa = a - 1 >= off ? a - 1 : a;
#pragma unroll
                for (int k = 0; k < 6; ++k) gn[k] = g[(size_t)aa * 6 + k];
                gauge_maps(g0, gn, T);
#pragma unroll
                for (int k = 0; k < NP; ++k) x[k] = M[(size_t)aa * NP + k];
                apply_T(T, x, y);
                float qaa[9], qa[9], qb[9], qd[9];
                project9(y, qaa);
                project9(ma, qa);
                project9(mb, qb);
#pragma unroll
                for (int k = 0; k < NP; ++k) w[k] -= f[k];
                project9(w, qd);
                const int mode = prm[p].flic;
                if (mode == 1) {
                    // the ratios in the interface's Hermite gauge, which both
                    // neighbours share (one phi for both sides)
                    float gi[6];
#pragma unroll
                    for (int k = 0; k < 6; ++k) gi[k] = gI[(size_t)b * 6 + k];
                    auto in_gi = [&](int cc, float *q) {
#pragma unroll
                        for (int k = 0; k < 6; ++k) gn[k] = g[(size_t)cc * 6 + k];
                        gauge_maps(gi, gn, T);
#pragma unroll
                        for (int k = 0; k < NP; ++k) x[k] = M[(size_t)cc * NP + k];
                        apply_T(T, x, y);
                        project9(y, q);
                    };
                    in_gi(aa, qaa);
                    in_gi(a, qa);
                    in_gi(b, qb);
                }
                float phi[9], pmin = 2.f;
#pragma unroll
                for (int j = 0; j < 9; ++j) {
                    const float num = qa[j] - qaa[j], den = qb[j] - qa[j];
                    const float r = den != 0.f ? num / den : 0.f;
                    phi[j] = r > 0.f ? 2.f / (1.f + 1.f / r) : 0.f;
                    pmin = fminf(pmin, phi[j]);
                }
#pragma unroll
                for (int j = 0; j < 9; ++j) qd[j] *= mode == 0 ? phi[j] : (mode == 2 ? phi[0] : pmin);
                add9(f, qd);
            }
        }
#pragma unroll
        for (int k = 0; k < NP; ++k) acc[k] += side ? -f[k] : f[k];
    }
    const float r = sc[p].dt / prm[p].dx;
#pragma unroll
    for (int k = 0; k < NP; ++k) Mn[(size_t)c * NP + k] = M[(size_t)c * NP + k] + r * acc[k];
}

__global__ void __launch_bounds__(SB) k_regauge(const float *__restrict__ Mn, float *__restrict__ M,
                                                float *__restrict__ beta, float *__restrict__ g,
                                                const float *__restrict__ rho0, const int *__restrict__ pid,
                                                const unsigned char *__restrict__ interior, ShockScalars *sc, int NT) {
    __shared__ float sM[SB * NP], sB[SB * NP], sg[SB * 6];
    __shared__ unsigned char sl[SB];
    const int c0 = blockIdx.x * SB, c = c0 + threadIdx.x;
    stage_in<NP, SB>(sM, Mn, c0, NT);
    stage_in<NP, SB>(sB, beta, c0, NT);
    stage_in<6, SB>(sg, g, c0, NT);
    const bool live = c < NT && interior[c];
    sl[threadIdx.x] = live;
    __syncthreads();
    unsigned dv = 0u;
    int key = -1;
    if (live) {
        float *mrow = sM + threadIdx.x * NP, *brow = sB + threadIdx.x * NP, *grow = sg + threadIdx.x * 6;
        float m[NP], gg[6], gh[6], y[NP], b[NP], bo[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) { m[k] = mrow[k]; b[k] = brow[k]; }
#pragma unroll
        for (int k = 0; k < 6; ++k) gg[k] = grow[k];
        hermite_gauge(m, gg, 1, gh);
        AxisMap T[3];
        gauge_maps(gh, gg, T);
        apply_T(T, m, y);
        transform_beta(gh, gg, b, bo);
        bo[0] = y[0];
#pragma unroll
        for (int k = 0; k < NP; ++k) { mrow[k] = y[k]; brow[k] = bo[k]; }
#pragma unroll
        for (int k = 0; k < 6; ++k) grow[k] = gh[k];
        key = pid[c];
        dv = __float_as_uint(fabsf(y[0] - rho0[c]));
    }
    // the steady metric: one atomic per problem and warp (non-negative
    // floats order like their bit patterns)
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    dv = __reduce_max_sync(grp, dv);
    if (key >= 0 && (int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicMax(&sc[key].steady_bits, dv);
    __syncthreads();
    stage_out<NP, SB>(M, sM, c0, NT, sl);
    stage_out<NP, SB>(beta, sB, c0, NT, sl);
    stage_out<6, SB>(g, sg, c0, NT, sl);
}

// dt_p = cfl dx_p / max speed over problem p's cells (ghosts included); one
// block per problem.
__global__ void k_dt(const float *__restrict__ speed, const ShockProb *__restrict__ prm, ShockScalars *sc) {
    __shared__ float red[32];
    const ShockProb pr = prm[blockIdx.x];
    float m = 0.f;
    for (int c = threadIdx.x; c < pr.n + 2; c += blockDim.x) m = fmaxf(m, speed[pr.off + c]);
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        float r = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.f;
        r = warp_max(r);
        if (threadIdx.x == 0) {
            ShockScalars &s = sc[blockIdx.x];
            const float dt = pr.cfl_dx / r;
            if (pr.t_end > 0.0 && s.t + (double)dt >= pr.t_end) {
                // cut to end at t_end (dt = 0 once there)
                s.dt = (float)fmax(pr.t_end - s.t, 0.0);
                s.t = fmax(s.t, pr.t_end);
            } else {
                s.dt = dt;
                s.t += (double)dt;
            }
            s.steps += 1;
            s.steady_bits = 0u;
        }
    }
}

void rh_states(const mem_shock_params &p, double &n_dn, double &T_dn, double &v_up, double &v_dn) {
    const double g = p.gamma, M2 = p.mach * p.mach;
    const double r = (g + 1.0) * M2 / ((g - 1.0) * M2 + 2.0);
    const double t = (2.0 * g * M2 - (g - 1.0)) * ((g - 1.0) * M2 + 2.0) / ((g + 1.0) * (g + 1.0) * M2);
    v_up = sqrt(g) * p.mach;
    n_dn = r;
    T_dn = t;
    v_dn = v_up / r;
}

}  // namespace

// ---------------------------------------------------------------------------
namespace mem_host {

bool shock_params_valid(const mem_shock_params &p) {
    return p.ncells >= 1 && p.xr > p.xl && p.mach >= 1.0 && p.cfl > 0 && p.Pr > 0.5 && p.gamma > 1.0 && p.kn > 0 &&
           (p.ic == 0 || p.ic == 1) && p.maxI >= 0 && (p.impl == MEM_IMPL_PLAIN || p.impl == MEM_IMPL_FUSED) &&
           p.na > 0 && p.nb > 0 && p.nr > 0 && p.scheme >= MEM_SCHEME_LF && p.scheme <= MEM_SCHEME_FLIC &&
           (p.ic == 0 || p.thickness > 0) && p.t_end >= 0.0 && (p.stats == 35 || p.stats == 9) &&
           p.flic_limiter >= 0 && p.flic_limiter <= 2;
}

// Device bytes per packed cell, the interface arrays of Lax-Wendroff / FLIC
// problems included (an upper bound for LF-only batches).
size_t batch_bytes_per_cell(const mem_ctx *ctx) {
    const size_t work = ctx->vel ? (size_t)MEM_MU_STRIDE : (size_t)ctx->Q + MEM_NCOL_FLUX;
    const size_t iface = sizeof(float) * (3 * NP + 6 + 1) + sizeof(int32_t) * 2 + 1;
    return sizeof(float) * (5 * NP + 6 + 3 + work) + sizeof(int32_t) * 3 + 1 + iface;
}

// Integration domain of a velocity-space rule for one problem (Appendix D):
// n_a, n_b, n_r thermal speeds beyond the up- and downstream Maxwellians.
static void shock_domain(const mem_shock_params &p, double *dom) {
    double n_dn, T_dn, v_up, v_dn;
    rh_states(p, n_dn, T_dn, v_up, v_dn);
    const double c_up = 1.0, c_dn = sqrt(T_dn);
    const double ax = std::min(v_dn - p.na * c_dn, v_up - p.na * c_up);
    const double bx = std::max(v_up + p.nb * c_up, v_dn + p.nb * c_dn);
    const double br = std::max(p.nr * c_up, p.nr * c_dn);
    dom[0] = ax;
    dom[1] = bx;
    dom[2] = br;
    dom[3] = 0.0;
}

void batch_free(ShockBatch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    void *ptrs[] = {b->M, b->beta, b->g, b->speed, b->F, b->Mn, b->rho0, b->sigma, b->mom, b->status, b->iters,
                    b->pid, b->interior, b->prm, b->sc, b->mu, b->dom, b->cond, b->MI, b->betaI, b->gI,
                    b->FI, b->speedI, b->statusI, b->itersI, b->iface};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete b;
}

// Initial state of one problem into host arrays at cell offset `off`.
// ic 0: a step at x = 0 between the Rankine-Hugoniot Maxwellians, each cell in
// its own Hermite gauge (M = n e_0, beta = 0).  ic 1: Appendix D, Eq. "Mx
// ini": the two Maxwellians' moments blended with a tanh profile of
// thickness parameter `thickness`; the blend is a two-Gaussian mixture whose
// moments are written in its own (axisymmetric) Hermite gauge.
static void set_ic(const mem_shock_params &p, const ShockProb &pr, double thickness, float *hM, float *hb, float *hg) {
    double n_dn, T_dn, v_up, v_dn;
    rh_states(p, n_dn, T_dn, v_up, v_dn);
    const double n_up = 1.0, T_up = 1.0;
    const int NT = pr.n + 2;
    for (int c = 0; c < NT; ++c) {
        const double x = p.xl + (c - 0.5) * pr.dx;
        float *M = hM + (size_t)(pr.off + c) * NP, *b = hb + (size_t)(pr.off + c) * NP, *g = hg + (size_t)(pr.off + c) * 6;
        for (int k = 0; k < NP; ++k) { M[k] = 0.f; b[k] = 0.f; }
        const bool ghost = c == 0 || c == NT - 1;
        if (p.ic == 0 || ghost) {
            const bool up = x < 0.0;
            const double n = up ? n_up : n_dn, T = up ? T_up : T_dn, v = up ? v_up : v_dn;
            M[0] = (float)n;
            b[0] = (float)n;
            g[0] = (float)v;
            g[1] = g[2] = 0.f;
            g[3] = g[4] = g[5] = (float)sqrt(T);
            continue;
        }
        const double h = 0.5 * thickness;
        const double w = (tanh(x / h) - tanh(p.xl / h)) / (tanh(p.xr / h) - tanh(p.xl / h));
        const double a0 = (1.0 - w) * n_up, a1 = w * n_dn, n = a0 + a1;
        const double v = (a0 * v_up + a1 * v_dn) / n;
        const double ex2 = (a0 * (T_up + v_up * v_up) + a1 * (T_dn + v_dn * v_dn)) / n;
        const double sx = sqrt(ex2 - v * v), sr = sqrt((a0 * T_up + a1 * T_dn) / n);
        const double gg[6] = {v, 0.0, 0.0, sx, sr, sr};
        double acc[NP] = {0.0};
        const double comp[2][3] = {{a0, v_up, T_up}, {a1, v_dn, T_dn}};
        for (int q = 0; q < 2; ++q) {
            const double mu[3] = {(comp[q][1] - gg[0]) / gg[3], 0.0, 0.0};
            double K[3][3] = {{comp[q][2] / (sx * sx) - 1.0, 0, 0}, {0, comp[q][2] / (sr * sr) - 1.0, 0},
                              {0, 0, comp[q][2] / (sr * sr) - 1.0}};
            double mq[NP];
            gaussian_hermite<double>(mu, K, comp[q][0], mq);
            for (int k = 0; k < NP; ++k) acc[k] += mq[k];
        }
        for (int k = 0; k < NP; ++k) M[k] = (float)acc[k];
        b[0] = (float)n;
        for (int k = 0; k < 6; ++k) g[k] = (float)gg[k];
    }
}

int batch_create(mem_ctx *ctx, const mem_shock_params *ps, int P, ShockBatch **out) {
    *out = nullptr;
    if (P < 1) return MEM_EINVAL;
    for (int i = 0; i < P; ++i)
        if (!shock_params_valid(ps[i]) || (ctx->vel && ps[i].impl != MEM_IMPL_FUSED)) return MEM_EINVAL;
    ShockBatch *b = new ShockBatch();
    b->ctx = ctx;
    b->P = P;
    b->params.assign(ps, ps + P);
    int off = 0;
    for (int i = 0; i < P; ++i) {
        ShockProb pr;
        double n_dn, T_dn, v_up, v_dn;
        rh_states(ps[i], n_dn, T_dn, v_up, v_dn);
        pr.off = off;
        pr.n = ps[i].ncells;
        pr.dx = (float)((ps[i].xr - ps[i].xl) / ps[i].ncells);
        pr.cfl_dx = (float)(ps[i].cfl * (ps[i].xr - ps[i].xl) / ps[i].ncells);
        pr.Pr = (float)ps[i].Pr;
        // Maxwell molecules (Appendix A) with upstream Knudsen number kn:
        // mu = kn sqrt(2/pi) T, tau = mu / (Pr n T) = relax / n.
        pr.relax = (float)(ps[i].kn * sqrt(2.0 / 3.14159265358979323846) / ps[i].Pr);
        pr.drho = (float)(n_dn - 1.0);
        pr.scheme = ps[i].scheme;
        pr.flic = ps[i].flic_limiter;
        pr.t_end = ps[i].t_end;
        b->second_order |= ps[i].scheme != MEM_SCHEME_LF;
        b->hprm.push_back(pr);
        off += pr.n + 2;
    }
    b->NT = off;
    const size_t NT = (size_t)off;
    const int Q = ctx->Q;
    auto alloc = [&](void **ptr, size_t bytes) { return cudaMalloc(ptr, bytes) == cudaSuccess; };
    // Flux work space: moment rows (velocity-space rule) or the plain path's
    // sigma and moment columns (Gauss-Hermite rule).
    const bool work_ok = ctx->vel ? alloc((void **)&b->mu, sizeof(float) * NT * MEM_MU_STRIDE) &&
                                        alloc((void **)&b->dom, sizeof(float) * DOM_REC * P) &&
                                        alloc((void **)&b->cond, sizeof(float) * NT)
                                  : alloc((void **)&b->sigma, sizeof(float) * NT * (size_t)Q) &&
                                        alloc((void **)&b->mom, sizeof(float) * NT * (size_t)MEM_NCOL_FLUX);
    bool ok = work_ok && alloc((void **)&b->M, sizeof(float) * NT * NP) && alloc((void **)&b->beta, sizeof(float) * NT * NP) &&
              alloc((void **)&b->g, sizeof(float) * NT * 6) && alloc((void **)&b->speed, sizeof(float) * NT) &&
              alloc((void **)&b->F, sizeof(float) * NT * NP) && alloc((void **)&b->Mn, sizeof(float) * NT * NP) &&
              alloc((void **)&b->rho0, sizeof(float) * NT) &&
              alloc((void **)&b->status, sizeof(int32_t) * NT) && alloc((void **)&b->iters, sizeof(int32_t) * NT) &&
              alloc((void **)&b->pid, sizeof(int) * NT) && alloc((void **)&b->interior, NT) &&
              alloc((void **)&b->prm, sizeof(ShockProb) * P) && alloc((void **)&b->sc, sizeof(ShockScalars) * P);
    if (ok && b->second_order)
        ok = alloc((void **)&b->MI, sizeof(float) * NT * NP) && alloc((void **)&b->betaI, sizeof(float) * NT * NP) &&
             alloc((void **)&b->gI, sizeof(float) * NT * 6) && alloc((void **)&b->FI, sizeof(float) * NT * NP) &&
             alloc((void **)&b->speedI, sizeof(float) * NT) && alloc((void **)&b->statusI, sizeof(int32_t) * NT) &&
             alloc((void **)&b->itersI, sizeof(int32_t) * NT) && alloc((void **)&b->iface, NT);
    if (!ok) { cudaGetLastError(); batch_free(b); return MEM_ENOMEM; }
    std::vector<float> hM(NT * NP), hb(NT * NP), hg(NT * 6);
    std::vector<int> hpid(NT);
    std::vector<unsigned char> hint(NT), hif(NT, 0);
    for (int i = 0; i < P; ++i) {
        const ShockProb &pr = b->hprm[i];
        set_ic(ps[i], pr, ps[i].thickness, hM.data(), hb.data(), hg.data());
        for (int c = 0; c < pr.n + 2; ++c) {
            hpid[pr.off + c] = i;
            hint[pr.off + c] = (c > 0 && c < pr.n + 1) ? 1 : 0;
            hif[pr.off + c] = (c > 0 && pr.scheme != MEM_SCHEME_LF) ? 1 : 0;
        }
    }
    std::vector<float> hbI(NT * NP, 0.f);
    if (b->second_order &&
        (cudaMemcpy(b->iface, hif.data(), NT, cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(b->betaI, hbI.data(), sizeof(float) * hbI.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(b->gI, hg.data(), sizeof(float) * hg.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemset(b->statusI, 0, sizeof(int32_t) * NT) != cudaSuccess ||
         cudaMemset(b->itersI, 0, sizeof(int32_t) * NT) != cudaSuccess)) {
        batch_free(b);
        return MEM_ECUDA;
    }
    std::vector<ShockScalars> hsc(P);
    memset(hsc.data(), 0, sizeof(ShockScalars) * P);
    if (cudaMemcpy(b->M, hM.data(), sizeof(float) * hM.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->beta, hb.data(), sizeof(float) * hb.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->g, hg.data(), sizeof(float) * hg.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->pid, hpid.data(), sizeof(int) * NT, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->interior, hint.data(), NT, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->prm, b->hprm.data(), sizeof(ShockProb) * P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->sc, hsc.data(), sizeof(ShockScalars) * P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->status, 0, sizeof(int32_t) * NT) != cudaSuccess ||
        cudaMemset(b->iters, 0, sizeof(int32_t) * NT) != cudaSuccess) {
        batch_free(b);
        return MEM_ECUDA;
    }
    if (ctx->vel) {
        std::vector<float> hdom(DOM_REC * (size_t)P);
        for (int i = 0; i < P; ++i) {
            double d[4];
            shock_domain(ps[i], d);
            dom_record(d[0], d[1], d[2], ctx->nbx, ctx->nbr, &hdom[DOM_REC * (size_t)i]);
        }
        if (cudaMemcpy(b->dom, hdom.data(), sizeof(float) * hdom.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(b->cond, 0, sizeof(float) * NT) != cudaSuccess) {
            batch_free(b);
            return MEM_ECUDA;
        }
    }
    // Natural parameters of the initial state (the tanh blend is not a
    // Maxwellian), then the characteristic speeds that set the first dt.
    int rc = MEM_OK;
    const bool nine = ps[0].stats == 9;
    bool any_tanh = false;
    for (int i = 0; i < P; ++i) any_tanh |= ps[i].ic == 1;
    if (any_tanh) {
        mem_solve_opts o;
        mem_solve_opts_default(&o);
        o.tol = ps[0].tol;
        o.maxI = ps[0].maxI;
        rc = (ctx->vel && nine)
                 ? axi_run(ctx, b->M, b->beta, b->g, b->status, b->iters, nullptr, nullptr, b->pid, b->dom,
                           (int64_t)NT, o, true, 0, b->interior)
             : ctx->vel ? vel_run(ctx, b->M, b->beta, b->g, b->status, b->iters, nullptr, b->pid, b->dom, (int64_t)NT,
                                  o, true, 0, b->interior)
                        : solve_fused(ctx, b->M, b->beta, b->status, b->iters, (int64_t)NT, o, 0, b->interior);
    }
    if (!rc && ctx->vel && nine) {
        mem_solve_opts o;
        mem_solve_opts_default(&o);
        rc = axi_run(ctx, b->M, b->beta, b->g, nullptr, nullptr, b->F, b->speed, b->pid, b->dom, (int64_t)NT, o, false,
                     0);
    } else if (!rc && ctx->vel) {
        mem_solve_opts o;
        mem_solve_opts_default(&o);
        rc = vel_run(ctx, b->M, b->beta, b->g, nullptr, nullptr, b->mu, b->pid, b->dom, (int64_t)NT, o, false, 0);
        if (!rc) rc = flux_from_mu(ctx, b->mu, b->M, b->g, b->F, b->speed, (int64_t)NT, 0, true);
    } else if (!rc) rc = (ps[0].impl == MEM_IMPL_FUSED && flux_fused_available(ctx))
                      ? flux_fused(ctx, b->M, b->beta, b->g, b->F, b->speed, (int64_t)NT, 0, true)
                      : flux_bufs(ctx, b->M, b->beta, b->g, b->F, b->speed, (int64_t)NT, b->sigma, b->mom, 0);
    if (rc || cudaDeviceSynchronize() != cudaSuccess) { batch_free(b); return rc ? rc : MEM_ECUDA; }
    *out = b;
    return MEM_OK;
}

int batch_enqueue_step(ShockBatch *b, cudaStream_t st) {
    const int NT = b->NT;
    const unsigned nb = (unsigned)((NT + 127) / 128), nsb = (unsigned)((NT + SB - 1) / SB);
    k_dt<<<b->P, 256, 0, st>>>(b->speed, b->prm, b->sc);
    k_collide<<<nsb, SB, 0, st>>>(b->M, b->g, b->pid, b->interior, b->prm, b->sc, NT, 0.5f, b->rho0);
    const mem_shock_params &p0 = b->params[0];
    mem_solve_opts o;
    mem_solve_opts_default(&o);
    o.impl = p0.impl;
    o.tol = p0.tol;
    o.maxI = p0.maxI;
    int rc;
    const bool nine = p0.stats == 9;
    if (b->ctx->vel && nine) {
        // the paper's nine-statistic system: solve, flux and speed in one
        // launch (ghost cells: flux and speed only)
        rc = axi_run(b->ctx, b->M, b->beta, b->g, b->status, b->iters, b->F, b->speed, b->pid, b->dom, NT, o, true, st,
                     b->interior, b->cond);
    } else if (b->ctx->vel) {
        // Velocity-space rule: the solve kernel also leaves the moments of
        // degree <= 9 at the new beta (ghost cells included), and the speed
        // kernel reads them.
        rc = vel_run(b->ctx, b->M, b->beta, b->g, b->status, b->iters, b->mu, b->pid, b->dom, NT, o, true, st,
                     b->interior, b->cond);
        if (!rc) rc = flux_from_mu(b->ctx, b->mu, b->M, b->g, b->F, b->speed, NT, st, true);
    } else {
    rc = (o.impl == MEM_IMPL_PLAIN)
                 ? solve_plain(b->ctx, b->M, b->beta, b->status, b->iters, NT, o, st, b->interior)
                 : solve_fused(b->ctx, b->M, b->beta, b->status, b->iters, NT, o, st, b->interior);
    if (rc) return rc;
    rc = (o.impl == MEM_IMPL_FUSED && flux_fused_available(b->ctx))
             ? flux_fused(b->ctx, b->M, b->beta, b->g, b->F, b->speed, NT, st, true)
             : flux_bufs(b->ctx, b->M, b->beta, b->g, b->F, b->speed, NT, b->sigma, b->mom, st);
    }
    if (rc) return rc;
    if (b->second_order) {
        // Lax-Wendroff / FLIC: one more Newton solve and flux per interface,
        // in the interface's Hermite gauge (no speeds needed there).
        k_iface_state<<<nb, 128, 0, st>>>(b->M, b->F, b->g, b->beta, b->MI, b->gI, b->betaI, b->statusI, b->iface,
                                          b->pid, b->prm, b->sc, NT);
        if (b->ctx->vel && nine) {
            rc = axi_run(b->ctx, b->MI, b->betaI, b->gI, b->statusI, b->itersI, b->FI, nullptr, b->pid, b->dom, NT, o,
                         true, st, b->iface);
        } else if (b->ctx->vel) {
            rc = vel_run(b->ctx, b->MI, b->betaI, b->gI, b->statusI, b->itersI, b->mu, b->pid, b->dom, NT, o, true, st,
                         b->iface);
            if (!rc) rc = flux_from_mu(b->ctx, b->mu, b->MI, b->gI, b->FI, nullptr, NT, st, true);
        } else if (o.impl == MEM_IMPL_PLAIN) {
            rc = solve_plain(b->ctx, b->MI, b->betaI, b->statusI, b->itersI, NT, o, st, b->iface);
            if (!rc) rc = flux_bufs(b->ctx, b->MI, b->betaI, b->gI, b->FI, b->speedI, NT, b->sigma, b->mom, st);
        } else {
            rc = solve_fused(b->ctx, b->MI, b->betaI, b->statusI, b->itersI, NT, o, st, b->iface);
            if (!rc)
                rc = flux_fused_available(b->ctx)
                         ? flux_fused(b->ctx, b->MI, b->betaI, b->gI, b->FI, nullptr, NT, st, true)
                         : flux_bufs(b->ctx, b->MI, b->betaI, b->gI, b->FI, b->speedI, NT, b->sigma, b->mom, st);
        }
        if (rc) return rc;
        k_stencil2<<<nb, 128, 0, st>>>(b->M, b->F, b->g, b->speed, b->FI, b->gI, b->statusI, b->Mn, b->pid,
                                       b->interior, b->prm, b->sc, NT);
    } else
        k_stencil<<<nsb, SB, 0, st>>>(b->M, b->F, b->g, b->speed, b->Mn, b->pid, b->interior, b->prm, b->sc, NT);
    k_collide<<<nsb, SB, 0, st>>>(b->Mn, b->g, b->pid, b->interior, b->prm, b->sc, NT, 0.5f, nullptr);
    k_regauge<<<nsb, SB, 0, st>>>(b->Mn, b->M, b->beta, b->g, b->rho0, b->pid, b->interior, b->sc, NT);
    MEM_CUDA_TRY(cudaGetLastError());
    return MEM_OK;
}

// Host profiles of problem i (Appendix A definitions, m = k_B = 1).
int batch_profiles(ShockBatch *b, int i, float *M_host, float *g_host, float *beta_host, float *rho, float *ux,
                   float *T, float *sxx, float *qx, double *t_out, int *steps_out) {
    if (i < 0 || i >= b->P) return MEM_EINVAL;
    const ShockProb &pr = b->hprm[i];
    const int N = pr.n, NT = N + 2;
    std::vector<float> hM((size_t)NT * NP), hg((size_t)NT * 6);
    MEM_CUDA_TRY(cudaDeviceSynchronize());
    MEM_CUDA_TRY(cudaMemcpy(hM.data(), b->M + (size_t)pr.off * NP, sizeof(float) * hM.size(), cudaMemcpyDeviceToHost));
    MEM_CUDA_TRY(cudaMemcpy(hg.data(), b->g + (size_t)pr.off * 6, sizeof(float) * hg.size(), cudaMemcpyDeviceToHost));
    if (M_host) memcpy(M_host, hM.data(), sizeof(float) * hM.size());
    if (g_host) memcpy(g_host, hg.data(), sizeof(float) * hg.size());
    if (beta_host)
        MEM_CUDA_TRY(cudaMemcpy(beta_host, b->beta + (size_t)pr.off * NP, sizeof(float) * NT * NP, cudaMemcpyDeviceToHost));
    if (t_out || steps_out) {
        ShockScalars h;
        MEM_CUDA_TRY(cudaMemcpy(&h, b->sc + i, sizeof(h), cudaMemcpyDeviceToHost));
        if (t_out) *t_out = h.t;
        if (steps_out) *steps_out = h.steps;
    }
    for (int c = 0; c < N; ++c) {
        const float *m = &hM[(size_t)(c + 1) * NP];
        const float *gg = &hg[(size_t)(c + 1) * 6];
        const double n = m[0];
        double mb[3], E2[3];
        const int i1[3] = {idx3(1, 0, 0), idx3(0, 1, 0), idx3(0, 0, 1)};
        const int i2[3] = {idx3(2, 0, 0), idx3(0, 2, 0), idx3(0, 0, 2)};
        for (int a = 0; a < 3; ++a) { mb[a] = m[i1[a]] / n; E2[a] = sqrt(2.0) * m[i2[a]] / n + 1.0; }
        double var[3];
        for (int a = 0; a < 3; ++a) var[a] = gg[3 + a] * gg[3 + a] * (E2[a] - mb[a] * mb[a]);
        const double Tc = (var[0] + var[1] + var[2]) / 3.0;
        if (rho) rho[c] = (float)n;
        if (ux) ux[c] = (float)(gg[0] + gg[3] * mb[0]);
        if (T) T[c] = (float)Tc;
        if (sxx) sxx[c] = (float)(n * (var[0] - Tc));
        if (qx) {
            // q_x = n/2 sum_b E[c_x c_b^2], c = u - v, from raw moments of ubar.
            const double X = mb[0], X2 = E2[0], X3 = sqrt(6.0) * m[idx3(3, 0, 0)] / n + 3.0 * X;
            double q = gg[3] * gg[3] * gg[3] * (X3 - 3.0 * X * X2 + 2.0 * X * X * X);
            const int iy[2] = {idx3(1, 1, 0), idx3(1, 0, 1)}, iy2[2] = {idx3(1, 2, 0), idx3(1, 0, 2)};
            for (int bb = 1; bb < 3; ++bb) {
                const double Y = mb[bb], Y2 = E2[bb], XY = m[iy[bb - 1]] / n;
                const double XY2 = sqrt(2.0) * m[iy2[bb - 1]] / n + X;
                q += gg[3] * gg[3 + bb] * gg[3 + bb] * (XY2 - 2.0 * Y * XY - X * Y2 + 2.0 * X * Y * Y);
            }
            qx[c] = (float)(0.5 * n * q);
        }
    }
    return MEM_OK;
}

int batch_read_scalars(ShockBatch *b, std::vector<ShockScalars> &out, cudaStream_t st) {
    out.resize(b->P);
    MEM_CUDA_TRY(cudaMemcpyAsync(out.data(), b->sc, sizeof(ShockScalars) * b->P, cudaMemcpyDeviceToHost, st));
    MEM_CUDA_TRY(cudaStreamSynchronize(st));
    return MEM_OK;
}

}  // namespace mem_host

// ---------------------------------------------------------------------------
// C ABI: one problem (mem_shock_init) or a packed batch (mem_shock_init_batch).
struct mem_shock {
    mem_host::ShockBatch *b = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
};

extern "C" {

int mem_shock_condition(mem_shock *s, int problem, double *max_cond) {
    if (!s || !max_cond) return MEM_EINVAL;
    mem_host::ShockBatch *b = s->b;
    if (problem < 0 || problem >= b->P) return MEM_EINVAL;
    if (!b->cond) return MEM_EINVAL;  // a Gauss-Hermite context records no estimate
    const ShockProb &pr = b->hprm[problem];
    std::vector<float> h((size_t)pr.n);
    MEM_CUDA_TRY(cudaDeviceSynchronize());
    MEM_CUDA_TRY(cudaMemcpy(h.data(), b->cond + pr.off + 1, sizeof(float) * pr.n, cudaMemcpyDeviceToHost));
    double m = 0.0;
    for (float v : h) m = fmax(m, (double)v);
    *max_cond = m;
    return MEM_OK;
}

int mem_shock_domain(const mem_shock_params *p, double *domain) {
    if (!p || !domain || !mem_host::shock_params_valid(*p)) return MEM_EINVAL;
    double d[4];
    mem_host::shock_domain(*p, d);
    domain[0] = d[0];
    domain[1] = d[1];
    domain[2] = d[2];
    return MEM_OK;
}

void mem_shock_params_default(mem_shock_params *p) {
    p->mach = 1.5;
    p->ncells = 64;
    p->xl = -20.0;
    p->xr = 20.0;
    p->cfl = 0.5;
    p->Pr = 2.0 / 3.0;
    p->gamma = 5.0 / 3.0;
    p->kn = 1.0;
    p->ic = 0;
    p->impl = MEM_IMPL_FUSED;
    p->graph = 1;
    p->tol = 1e-8f;
    p->maxI = 500;
    p->na = p->nb = p->nr = 5.0;
    p->scheme = MEM_SCHEME_LF;
    p->thickness = 15.7;
    p->t_end = 0.0;
    p->stats = 35;
    p->flic_limiter = 0;
}

void mem_shock_free(mem_shock *s) {
    if (!s) return;
    cudaDeviceSynchronize();
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->graph) cudaGraphDestroy(s->graph);
    mem_host::batch_free(s->b);
    delete s;
}

int mem_shock_init_batch(mem_ctx *ctx, const mem_shock_params *ps, int nprob, mem_shock **out) {
    if (!ctx || !ps || !out || nprob < 1) return MEM_EINVAL;
    for (int i = 1; i < nprob; ++i)
        if (ps[i].impl != ps[0].impl || ps[i].tol != ps[0].tol || ps[i].maxI != ps[0].maxI ||
            ps[i].stats != ps[0].stats)
            return MEM_EINVAL;
    *out = nullptr;
    mem_host::ShockBatch *b = nullptr;
    int rc = mem_host::batch_create(ctx, ps, nprob, &b);
    if (rc) return rc;
    mem_shock *s = new mem_shock();
    s->b = b;
    *out = s;
    return MEM_OK;
}

int mem_shock_init(mem_ctx *ctx, const mem_shock_params *p, mem_shock **out) {
    if (!p) return MEM_EINVAL;
    return mem_shock_init_batch(ctx, p, 1, out);
}

int mem_shock_num_problems(const mem_shock *s) { return s ? s->b->P : 0; }

int mem_shock_step(mem_shock *s, int nsteps, double *steady_metric, void *stream) {
    if (!s || nsteps < 0) return MEM_EINVAL;
    mem_host::ShockBatch *b = s->b;
    cudaStream_t st = (cudaStream_t)stream;
    const bool use_graph = b->params[0].graph && b->params[0].impl == MEM_IMPL_FUSED;
    if (use_graph && !s->gexec && nsteps > 0) {
        // Capture one step.  The legacy default stream cannot be captured, so
        // capture on a private stream; the first step runs uncaptured (the
        // fused kernel sets its shared-memory limit on first use).
        cudaStream_t cap = st;
        bool own = false;
        if (!cap) {
            MEM_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            own = true;
        }
        int rc = mem_host::batch_enqueue_step(b, st);
        if (rc) return rc;
        --nsteps;
        MEM_CUDA_TRY(cudaStreamSynchronize(st));
        MEM_CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        rc = mem_host::batch_enqueue_step(b, cap);
        cudaGraph_t gph = nullptr;
        cudaError_t e = cudaStreamEndCapture(cap, &gph);
        if (own) cudaStreamDestroy(cap);
        if (rc || e != cudaSuccess) { if (gph) cudaGraphDestroy(gph); return rc ? rc : MEM_ECUDA; }
        s->graph = gph;
        MEM_CUDA_TRY(cudaGraphInstantiate(&s->gexec, gph, 0));
    }
    for (int k = 0; k < nsteps; ++k) {
        if (use_graph) MEM_CUDA_TRY(cudaGraphLaunch(s->gexec, st));
        else {
            int rc = mem_host::batch_enqueue_step(b, st);
            if (rc) return rc;
        }
    }
    if (steady_metric) {
        std::vector<ShockScalars> h;
        int rc = mem_host::batch_read_scalars(b, h, st);
        if (rc) return rc;
        double worst = 0.0;
        for (int i = 0; i < b->P; ++i) {
            float d;
            memcpy(&d, &h[i].steady_bits, sizeof(d));
            worst = fmax(worst, (double)d / b->hprm[i].drho);
        }
        *steady_metric = worst;
    }
    return MEM_OK;
}

int mem_shock_get_interfaces(mem_shock *s, float *MI, float *betaI, float *gI, float *FI, int32_t *status,
                             int32_t *iters) {
    if (!s || !s->b->second_order) return MEM_EINVAL;
    const mem_host::ShockBatch *b = s->b;
    const size_t NT = (size_t)b->NT;
    MEM_CUDA_TRY(cudaDeviceSynchronize());
    if (MI) MEM_CUDA_TRY(cudaMemcpy(MI, b->MI, sizeof(float) * NT * NP, cudaMemcpyDeviceToHost));
    if (betaI) MEM_CUDA_TRY(cudaMemcpy(betaI, b->betaI, sizeof(float) * NT * NP, cudaMemcpyDeviceToHost));
    if (gI) MEM_CUDA_TRY(cudaMemcpy(gI, b->gI, sizeof(float) * NT * 6, cudaMemcpyDeviceToHost));
    if (FI) MEM_CUDA_TRY(cudaMemcpy(FI, b->FI, sizeof(float) * NT * NP, cudaMemcpyDeviceToHost));
    if (status) MEM_CUDA_TRY(cudaMemcpy(status, b->statusI, sizeof(int32_t) * NT, cudaMemcpyDeviceToHost));
    if (iters) MEM_CUDA_TRY(cudaMemcpy(iters, b->itersI, sizeof(int32_t) * NT, cudaMemcpyDeviceToHost));
    return MEM_OK;
}

int mem_shock_device_state(mem_shock *s, float **M, float **beta, float **g, float **speed, int32_t **status,
                           int32_t **iters) {
    if (!s) return MEM_EINVAL;
    mem_host::ShockBatch *b = s->b;
    if (M) *M = b->M;
    if (beta) *beta = b->beta;
    if (g) *g = b->g;
    if (speed) *speed = b->speed;
    if (status) *status = b->status;
    if (iters) *iters = b->iters;
    return MEM_OK;
}

int mem_shock_get(mem_shock *s, float *M_host, float *g_host, float *beta_host, float *rho, float *ux, float *T,
                  float *sxx, float *qx, double *t_out) {
    if (!s) return MEM_EINVAL;
    return mem_host::batch_profiles(s->b, 0, M_host, g_host, beta_host, rho, ux, T, sxx, qx, t_out, nullptr);
}

int mem_shock_get_problem(mem_shock *s, int problem, float *rho, float *ux, float *T, float *sxx, float *qx,
                          double *t_out, int32_t *steps_out) {
    if (!s) return MEM_EINVAL;
    int steps = 0;
    int rc = mem_host::batch_profiles(s->b, problem, nullptr, nullptr, nullptr, rho, ux, T, sxx, qx, t_out, &steps);
    if (steps_out) *steps_out = steps;
    return rc;
}

}  // extern "C"

// shock.cu -- one time step of Algorithm 2 on a 1D normal shock (Appendix D):
//   dt = cfl dx / max speed            (k_dt, device-side, previous transport)
//   Collision(dt/2)                    (k_collide, ES-BGK, Eq. "source update")
//   Transport(dt): Newton (mem_solve), flux and speed (mem_flux),
//                  neighbour gauge transform + local Lax-Friedrichs + finite
//                  volume (k_stencil, Eqs. "The lax F", "The lax F convert",
//                  "The ME equation fvm 2")
//   Collision(dt/2)                    (k_collide)
//   Hermite gauge, transform of M and beta (k_regauge).
// Cells 0 and N+1 are Dirichlet ghost cells holding the Rankine-Hugoniot
// Maxwellians in their own Hermite gauge (beta = 0); they are never updated.
// All per-step scalars live in device memory, so the whole step can be
// captured in a CUDA graph when the fused Newton back-end is used.
#include <math.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "ctx.h"

using namespace mem;

struct ShockScalars {
    float dt;
    unsigned int steady_bits;  // max |d rho| as float bits (non-negative)
    double t;
    int steps;
};

struct mem_shock {
    mem_ctx *ctx = nullptr;
    mem_shock_params p;
    int N = 0;
    double dx = 0.0, n_up = 1, T_up = 1, v_up = 0, n_dn = 1, T_dn = 1, v_dn = 0;
    float relax = 0.f;  // tau = relax / n
    float *M = nullptr, *beta = nullptr, *g = nullptr, *speed = nullptr, *F = nullptr, *Mn = nullptr;
    float *rho0 = nullptr, *sigma = nullptr, *mom = nullptr;
    int32_t *status = nullptr, *iters = nullptr;
    ShockScalars *sc = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
};

namespace {

// Hermite-product expectations of the Gaussian N(mu, S) in the gauge frame:
// E[He_a(x) He_b(y) He_c(z)] equals the moment of a formal Gaussian with
// mean mu and covariance K = S - I, built by the recursion
//   m_{alpha + e_i} = mu_i m_alpha + sum_j alpha_j K_ij m_{alpha - e_j}.
__device__ __forceinline__ void gaussian_hermite(const float mu[3], const float K[3][3], float n, float *out) {
    float m[NP];
    m[0] = 1.f;
#pragma unroll
    for (int k = 1; k < NP; ++k) {
        const int al[3] = {exp_a(k), exp_b(k), exp_c(k)};
        const int i = al[0] > 0 ? 0 : (al[1] > 0 ? 1 : 2);
        int be[3] = {al[0], al[1], al[2]};
        be[i] -= 1;
        float v = mu[i] * m[idx3(be[0], be[1], be[2])];
#pragma unroll
        for (int j = 0; j < 3; ++j)
            if (be[j] > 0) {
                int g2[3] = {be[0], be[1], be[2]};
                g2[j] -= 1;
                v += (float)be[j] * K[i][j] * m[idx3(g2[0], g2[1], g2[2])];
            }
        m[k] = v;
    }
    const float fact[5] = {1.f, 1.f, 2.f, 6.f, 24.f};
#pragma unroll
    for (int k = 0; k < NP; ++k) out[k] = n * m[k] * rsqrtf(fact[exp_a(k)] * fact[exp_b(k)] * fact[exp_c(k)]);
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
    float P[3][3], T = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) P[a][b] = g[3 + a] * g[3 + b] * (E2[a][b] - mb[a] * mb[b]);
    T = (P[0][0] + P[1][1] + P[2][2]) / 3.f;
    float K[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float sig = (a == b ? T / Pr : 0.f) + (1.f - 1.f / Pr) * P[a][b];
            K[a][b] = sig / (g[3 + a] * g[3 + b]) - (a == b ? 1.f : 0.f);
        }
    gaussian_hermite(mb, K, n, Mt);
}

__global__ void k_collide(float *__restrict__ M, const float *__restrict__ g, int N, const ShockScalars *sc, float frac,
                          float Pr, float relax, float *rho0) {
    const int c = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    if (c > N) return;
    float m[NP], gg[6], mt[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) m[k] = M[(size_t)c * NP + k];
#pragma unroll
    for (int k = 0; k < 6; ++k) gg[k] = g[(size_t)c * 6 + k];
    if (rho0) rho0[c] = m[0];
    esbgk_target(m, gg, Pr, mt);
    const float r = frac * sc->dt * m[0] / relax;  // dt' / tau
#pragma unroll
    for (int k = 0; k < NP; ++k) M[(size_t)c * NP + k] = (1.f - r) * m[k] + r * mt[k];
}

// Local Lax-Friedrichs finite-volume update in the cell's own gauge.
__global__ void __launch_bounds__(128) k_stencil(const float *__restrict__ M, const float *__restrict__ F,
                                                 const float *__restrict__ g, const float *__restrict__ speed,
                                                 float *__restrict__ Mn, int N, float dx, const ShockScalars *sc) {
    const int c = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    if (c > N) return;
    float g0[6], gl[6], gr[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        g0[k] = g[(size_t)c * 6 + k];
        gl[k] = g[(size_t)(c - 1) * 6 + k];
        gr[k] = g[(size_t)(c + 1) * 6 + k];
    }
    const float s0 = speed[c], ll = fmaxf(speed[c - 1], s0), lr = fmaxf(s0, speed[c + 1]);
    const float r = sc->dt / dx;
    float acc[NP], x[NP], y[NP];
    AxisMap T[3];
    // own cell: F0 - F0 cancels; diffusion terms -0.5 (ll + lr) M0
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = -0.5f * (ll + lr) * M[(size_t)c * NP + k];
    gauge_maps(g0, gl, T);
#pragma unroll
    for (int k = 0; k < NP; ++k) x[k] = M[(size_t)(c - 1) * NP + k];
    apply_T(T, x, y);
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] += 0.5f * ll * y[k];
#pragma unroll
    for (int k = 0; k < NP; ++k) x[k] = F[(size_t)(c - 1) * NP + k];
    apply_T(T, x, y);
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] += 0.5f * y[k];
    gauge_maps(g0, gr, T);
#pragma unroll
    for (int k = 0; k < NP; ++k) x[k] = M[(size_t)(c + 1) * NP + k];
    apply_T(T, x, y);
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] += 0.5f * lr * y[k];
#pragma unroll
    for (int k = 0; k < NP; ++k) x[k] = F[(size_t)(c + 1) * NP + k];
    apply_T(T, x, y);
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] -= 0.5f * y[k];
    // F^LF_{c-1/2} - F^LF_{c+1/2} = 0.5(Fl + F0) + 0.5 ll (Ml - M0) - 0.5(F0 + Fr) - 0.5 lr (M0 - Mr)
#pragma unroll
    for (int k = 0; k < NP; ++k) Mn[(size_t)c * NP + k] = M[(size_t)c * NP + k] + r * acc[k];
}

__global__ void k_regauge(const float *__restrict__ Mn, float *__restrict__ M, float *__restrict__ beta,
                          float *__restrict__ g, const float *__restrict__ rho0, int N, ShockScalars *sc) {
    const int c = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    if (c > N) return;
    float m[NP], gg[6], gh[6], y[NP], b[NP], bo[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) { m[k] = Mn[(size_t)c * NP + k]; b[k] = beta[(size_t)c * NP + k]; }
#pragma unroll
    for (int k = 0; k < 6; ++k) gg[k] = g[(size_t)c * 6 + k];
    hermite_gauge(m, gg, 1, gh);
    AxisMap T[3];
    gauge_maps(gh, gg, T);
    apply_T(T, m, y);
    transform_beta(gh, gg, b, bo);
#pragma unroll
    for (int k = 0; k < NP; ++k) { M[(size_t)c * NP + k] = y[k]; beta[(size_t)c * NP + k] = bo[k]; }
    bo[0] = y[0];
    beta[(size_t)c * NP] = y[0];
#pragma unroll
    for (int k = 0; k < 6; ++k) g[(size_t)c * 6 + k] = gh[k];
    const float d = fabsf(y[0] - rho0[c]);
    atomicMax(&sc->steady_bits, __float_as_uint(d));
}

// dt = cfl dx / max speed over all cells (incl. ghosts); one block.
__global__ void k_dt(const float *__restrict__ speed, int NT, float cfl_dx, ShockScalars *sc) {
    __shared__ float red[32];
    float m = 0.f;
    for (int c = threadIdx.x; c < NT; c += blockDim.x) m = fmaxf(m, speed[c]);
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        float r = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.f;
        r = warp_max(r);
        if (threadIdx.x == 0) {
            const float dt = cfl_dx / r;
            sc->dt = dt;
            sc->t += (double)dt;
            sc->steps += 1;
            sc->steady_bits = 0u;
        }
    }
}

int enqueue_step(mem_shock *s, cudaStream_t st) {
    const int N = s->N, NT = N + 2;
    const unsigned nb = (unsigned)((N + 127) / 128);
    k_dt<<<1, 1024, 0, st>>>(s->speed, NT, (float)(s->p.cfl * s->dx), s->sc);
    k_collide<<<nb, 128, 0, st>>>(s->M, s->g, N, s->sc, 0.5f, (float)s->p.Pr, s->relax, s->rho0);
    mem_solve_opts o;
    mem_solve_opts_default(&o);
    o.impl = s->p.impl;
    o.tol = s->p.tol;
    o.maxI = s->p.maxI;
    int rc = (o.impl == MEM_IMPL_PLAIN)
                 ? mem_host::solve_plain(s->ctx, s->M + NP, s->beta + NP, s->status + 1, s->iters + 1, N, o, st)
                 : mem_host::solve_fused(s->ctx, s->M + NP, s->beta + NP, s->status + 1, s->iters + 1, N, o, st);
    if (rc) return rc;
    rc = mem_host::flux_bufs(s->ctx, s->M, s->beta, s->g, s->F, s->speed, NT, s->sigma, s->mom, st);
    if (rc) return rc;
    k_stencil<<<nb, 128, 0, st>>>(s->M, s->F, s->g, s->speed, s->Mn, N, (float)s->dx, s->sc);
    k_collide<<<nb, 128, 0, st>>>(s->Mn, s->g, N, s->sc, 0.5f, (float)s->p.Pr, s->relax, nullptr);
    k_regauge<<<nb, 128, 0, st>>>(s->Mn, s->M, s->beta, s->g, s->rho0, N, s->sc);
    MEM_CUDA_TRY(cudaGetLastError());
    return MEM_OK;
}

}  // namespace

extern "C" {

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
}

void mem_shock_free(mem_shock *s) {
    if (!s) return;
    cudaDeviceSynchronize();
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->graph) cudaGraphDestroy(s->graph);
    void *ptrs[] = {s->M, s->beta, s->g, s->speed, s->F, s->Mn, s->rho0, s->sigma, s->mom, s->status, s->iters, s->sc};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete s;
}

int mem_shock_init(mem_ctx *ctx, const mem_shock_params *p, mem_shock **out) {
    if (!ctx || !p || !out || p->ncells < 1 || !(p->xr > p->xl) || !(p->mach >= 1.0) || !(p->cfl > 0) ||
        !(p->Pr > 0.5) || !(p->gamma > 1.0) || !(p->kn > 0) || p->ic != 0)
        return MEM_EINVAL;
    *out = nullptr;
    mem_shock *s = new mem_shock();
    s->ctx = ctx;
    s->p = *p;
    const int N = p->ncells, NT = N + 2;
    s->N = N;
    s->dx = (p->xr - p->xl) / N;
    // Rankine-Hugoniot states (Appendix D), m = k_B = 1, n_- = T_- = 1.
    const double g = p->gamma, M2 = p->mach * p->mach;
    const double r = (g + 1.0) * M2 / ((g - 1.0) * M2 + 2.0);
    const double t = (2.0 * g * M2 - (g - 1.0)) * ((g - 1.0) * M2 + 2.0) / ((g + 1.0) * (g + 1.0) * M2);
    s->v_up = sqrt(g) * p->mach;
    s->n_dn = r;
    s->T_dn = t;
    s->v_dn = s->v_up / r;
    // Maxwell molecules, Kn = 1: mu = kn sqrt(2/pi) T and tau = mu / (Pr n T).
    s->relax = (float)(p->kn * sqrt(2.0 / 3.14159265358979323846) / p->Pr);
    auto alloc = [&](void **ptr, size_t bytes) { return cudaMalloc(ptr, bytes) == cudaSuccess; };
    const int Q = ctx->Q;
    bool ok = alloc((void **)&s->M, sizeof(float) * NT * NP) && alloc((void **)&s->beta, sizeof(float) * NT * NP) &&
              alloc((void **)&s->g, sizeof(float) * NT * 6) && alloc((void **)&s->speed, sizeof(float) * NT) &&
              alloc((void **)&s->F, sizeof(float) * NT * NP) && alloc((void **)&s->Mn, sizeof(float) * NT * NP) &&
              alloc((void **)&s->rho0, sizeof(float) * NT) && alloc((void **)&s->sigma, sizeof(float) * NT * (size_t)Q) &&
              alloc((void **)&s->mom, sizeof(float) * NT * (size_t)MEM_NCOL_FLUX) &&
              alloc((void **)&s->status, sizeof(int32_t) * NT) && alloc((void **)&s->iters, sizeof(int32_t) * NT) &&
              alloc((void **)&s->sc, sizeof(ShockScalars));
    if (!ok) { cudaGetLastError(); mem_shock_free(s); return MEM_ENOMEM; }
    // Initial condition: a step at x = 0 between the RH Maxwellians, each cell
    // in its own Hermite gauge (M = n e_0, beta = 0).
    std::vector<float> hM((size_t)NT * NP, 0.f), hb((size_t)NT * NP, 0.f), hg((size_t)NT * 6, 0.f);
    for (int c = 0; c < NT; ++c) {
        const double x = p->xl + (c - 0.5) * s->dx;
        const bool up = x < 0.0;
        const double n = up ? s->n_up : s->n_dn, T = up ? s->T_up : s->T_dn, v = up ? s->v_up : s->v_dn;
        hM[(size_t)c * NP] = (float)n;
        hb[(size_t)c * NP] = (float)n;
        hg[(size_t)c * 6 + 0] = (float)v;
        hg[(size_t)c * 6 + 3] = hg[(size_t)c * 6 + 4] = hg[(size_t)c * 6 + 5] = (float)sqrt(T);
    }
    ShockScalars z;
    memset(&z, 0, sizeof(z));
    if (cudaMemcpy(s->M, hM.data(), sizeof(float) * hM.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->beta, hb.data(), sizeof(float) * hb.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->g, hg.data(), sizeof(float) * hg.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(s->sc, &z, sizeof(z), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(s->status, 0, sizeof(int32_t) * NT) != cudaSuccess ||
        cudaMemset(s->iters, 0, sizeof(int32_t) * NT) != cudaSuccess) {
        mem_shock_free(s);
        return MEM_ECUDA;
    }
    // Prime the characteristic speeds of the initial state (they set dt of the
    // first step).
    int rc = mem_host::flux_bufs(ctx, s->M, s->beta, s->g, s->F, s->speed, NT, s->sigma, s->mom, 0);
    if (rc || cudaDeviceSynchronize() != cudaSuccess) { mem_shock_free(s); return rc ? rc : MEM_ECUDA; }
    *out = s;
    return MEM_OK;
}

int mem_shock_step(mem_shock *s, int nsteps, double *steady_metric, void *stream) {
    if (!s || nsteps < 0) return MEM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const bool use_graph = s->p.graph && s->p.impl == MEM_IMPL_FUSED;
    if (use_graph && !s->gexec && nsteps > 0) {
        // Capture one step.  The legacy default stream cannot be captured.
        cudaStream_t cap = st;
        bool own = false;
        if (!cap) {
            MEM_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            own = true;
        }
        // The first launch of the fused kernel sets its shared-memory limit;
        // do it outside the capture.
        int rc = enqueue_step(s, cap);
        if (rc) return rc;
        --nsteps;
        MEM_CUDA_TRY(cudaStreamSynchronize(cap));
        MEM_CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_step(s, cap);
        cudaGraph_t gph = nullptr;
        cudaError_t e = cudaStreamEndCapture(cap, &gph);
        if (rc || e != cudaSuccess) { if (gph) cudaGraphDestroy(gph); return rc ? rc : MEM_ECUDA; }
        s->graph = gph;
        MEM_CUDA_TRY(cudaGraphInstantiate(&s->gexec, gph, 0));
        if (own) cudaStreamDestroy(cap);
    }
    for (int k = 0; k < nsteps; ++k) {
        if (use_graph) MEM_CUDA_TRY(cudaGraphLaunch(s->gexec, st));
        else {
            int rc = enqueue_step(s, st);
            if (rc) return rc;
        }
    }
    if (steady_metric) {
        ShockScalars h;
        MEM_CUDA_TRY(cudaMemcpyAsync(&h, s->sc, sizeof(h), cudaMemcpyDeviceToHost, st));
        MEM_CUDA_TRY(cudaStreamSynchronize(st));
        float d;
        memcpy(&d, &h.steady_bits, sizeof(d));
        *steady_metric = (double)d / (s->n_dn - s->n_up);
    }
    return MEM_OK;
}

int mem_shock_device_state(mem_shock *s, float **M, float **beta, float **g, float **speed, int32_t **status,
                           int32_t **iters) {
    if (!s) return MEM_EINVAL;
    if (M) *M = s->M;
    if (beta) *beta = s->beta;
    if (g) *g = s->g;
    if (speed) *speed = s->speed;
    if (status) *status = s->status;
    if (iters) *iters = s->iters;
    return MEM_OK;
}

int mem_shock_get(mem_shock *s, float *M_host, float *g_host, float *beta_host, float *rho, float *ux, float *T,
                  float *sxx, float *qx, double *t_out) {
    if (!s) return MEM_EINVAL;
    const int N = s->N, NT = N + 2;
    std::vector<float> hM((size_t)NT * NP), hg((size_t)NT * 6);
    MEM_CUDA_TRY(cudaDeviceSynchronize());
    MEM_CUDA_TRY(cudaMemcpy(hM.data(), s->M, sizeof(float) * hM.size(), cudaMemcpyDeviceToHost));
    MEM_CUDA_TRY(cudaMemcpy(hg.data(), s->g, sizeof(float) * hg.size(), cudaMemcpyDeviceToHost));
    if (M_host) memcpy(M_host, hM.data(), sizeof(float) * hM.size());
    if (g_host) memcpy(g_host, hg.data(), sizeof(float) * hg.size());
    if (beta_host) MEM_CUDA_TRY(cudaMemcpy(beta_host, s->beta, sizeof(float) * NT * NP, cudaMemcpyDeviceToHost));
    if (t_out) {
        ShockScalars h;
        MEM_CUDA_TRY(cudaMemcpy(&h, s->sc, sizeof(h), cudaMemcpyDeviceToHost));
        *t_out = h.t;
    }
    // Macroscopic profiles (Appendix A definitions, m = k_B = 1) from the
    // moments in each cell's gauge.
    for (int i = 0; i < N; ++i) {
        const float *m = &hM[(size_t)(i + 1) * NP];
        const float *gg = &hg[(size_t)(i + 1) * 6];
        const double n = m[0];
        double mb[3], E2[3];
        const int i1[3] = {idx3(1, 0, 0), idx3(0, 1, 0), idx3(0, 0, 1)};
        const int i2[3] = {idx3(2, 0, 0), idx3(0, 2, 0), idx3(0, 0, 2)};
        for (int a = 0; a < 3; ++a) { mb[a] = m[i1[a]] / n; E2[a] = sqrt(2.0) * m[i2[a]] / n + 1.0; }
        double var[3];
        for (int a = 0; a < 3; ++a) var[a] = gg[3 + a] * gg[3 + a] * (E2[a] - mb[a] * mb[a]);
        const double Tc = (var[0] + var[1] + var[2]) / 3.0;
        if (rho) rho[i] = (float)n;
        if (ux) ux[i] = (float)(gg[0] + gg[3] * mb[0]);
        if (T) T[i] = (float)Tc;
        if (sxx) sxx[i] = (float)(n * (var[0] - Tc));
        if (qx) {
            // q_x = n/2 sum_b E[c_x c_b^2], c = u - v, from raw moments of ubar.
            const double X = mb[0], X2 = E2[0], X3 = sqrt(6.0) * m[idx3(3, 0, 0)] / n + 3.0 * X;
            double q = gg[3] * gg[3] * gg[3] * (X3 - 3.0 * X * X2 + 2.0 * X * X * X);
            const int iy[2] = {idx3(1, 1, 0), idx3(1, 0, 1)}, iy2[2] = {idx3(1, 2, 0), idx3(1, 0, 2)};
            for (int b = 1; b < 3; ++b) {
                const double Y = mb[b], Y2 = E2[b], XY = m[iy[b - 1]] / n;
                const double XY2 = sqrt(2.0) * m[iy2[b - 1]] / n + X;
                q += gg[3] * gg[3 + b] * gg[3 + b] * (XY2 - 2.0 * Y * XY - X * Y2 + 2.0 * X * Y * Y);
            }
            qx[i] = (float)(0.5 * n * q);
        }
    }
    return MEM_OK;
}

}  // extern "C"

// ctx.h -- the library context and the internal interfaces between the
// translation units (host side).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "mem.h"

#define MEM_NCOL_SOLVE 630   // [phi_0..34 | phi_i phi_j, 1 <= j <= i <= 34 packed]
#define MEM_NCOL_FLUX 1330   // [phi | ubar_x phi | phi phi^T packed (630) | ubar_x phi phi^T packed (630)]
#define MEM_HE_STRIDE 16     // he_0..he_9 per 1D node, padded
#define MEM_MU_STRIDE 224    // moment row: mu_abc (a+b+c <= 9, 220) | u_x node range (2) | pad

// Launch shape of a persistent warp-per-cell kernel: warps per block (2, 4
// or 8) and a cap on resident blocks per SM (0: as many as fit).
struct mem_launch_cfg {
    int warps = 4;
    int blocks_per_sm = 0;
};

struct mem_ctx {
    int device = 0;
    mem_launch_cfg cfg_fused, cfg_axi;  // set by the autotuner (mem_tune / mem_set_launch)
    int n1d = 0;  // nodes per axis
    int Q = 0;    // n1d^3
    std::vector<double> x1d, w1d;   // 1D Gauss-Hermite rule (probabilists', weights sum to 1)
    // Device tables (constant after mem_init).
    float *d_phiT = nullptr;       // [35][Q]   phi_k(ubar_q)
    float *d_logw = nullptr;       // [Q]       log w_q
    float *d_tab_solve = nullptr;  // [Q][630]
    float *d_tab_flux = nullptr;   // [Q][1330]
    float *d_he1d = nullptr;       // [n1d][16] he_0..he_9 at the 1D nodes
    float *d_x1d = nullptr;        // [n1d]
    float *d_logw1d = nullptr;     // [n1d]
    int *d_lin_off = nullptr;      // [596]  Hessian-term offsets (packed i>=j>=1)
    int2 *d_lin_terms = nullptr;   // (mu index, coefficient bits) per term
    int n_lin_terms = 0;
    int2 *d_hess_slots = nullptr;  // [n_hess_slots][32] per-lane Hessian term sequences
    int n_hess_slots = 0;
    int2 *d_hess_slots128 = nullptr;  // [n_hess_slots128][128] the same terms over 128 lanes (block per cell)
    int n_hess_slots128 = 0;
    int2 *d_hr_slots = nullptr;  // Hessian terms in rounds of 32 entries (warp per cell), see build_hess_rounds
    int *d_hr_rounds = nullptr;  // [n_hess_rounds] terms per round
    int *d_hr_ent = nullptr;     // [n_hess_rounds][32] destination (i | j << 8) or -1
    int n_hess_rounds = 0;
    int2 *d_flux_slots = nullptr;  // [n_flux_slots][32] E[phi phi^T] and E[ubar_x phi phi^T] terms
    int n_flux_slots = 0;
    int2 *d_axi_slots = nullptr;   // [n_axi_slots][32] the same, parity blocks of axisymmetric cells
    int n_axi_slots = 0;
    int *d_xlin_off = nullptr;     // [631]  flux-Jacobian terms (packed i>=j>=0)
    int2 *d_xlin_terms = nullptr;
    float xmax = 0.f;              // largest 1D node
    float *d_tc_tab = nullptr;     // tensor-core contraction tables (mixed back-end), [704][Q] row-major
    CUtensorMap tm_tab48, tm_tab208, tm_tab192;  // their tensor maps: boxes of 48, 208, 192 rows x 32 nodes
    double *d_phiT64 = nullptr;    // [35][Q] phi_k(ubar_q) in FP64 (residual recompute)
    double *d_logw64 = nullptr;    // [Q] log w_q in FP64
    // Velocity-space rule (mem_init_velocity): nodes fixed in the lab frame.
    int vel = 0;                             // 1: velocity-space context (no gauge-frame tables)
    int nbx = 0, nbr = 0, ng = 0, K = 0;     // blocks in u_x, blocks in u_r, points per block, azimuths
    int nx = 0, npt = 0;                     // nodes in u_x; points of the transverse plane
    double dom[3] = {0, 0, 0};               // default domain (a_x, b_x, b_r)
    float2 *d_vt2 = nullptr;  // [nx] x | [npt] y | [npt] z node offsets in block widths, as float pairs (hi, lo)
    float *d_vtf = nullptr;   // [nx] log w^GL of each x node | [nr] log(w^GL t_r / K) of each radial node
    float *d_dom0 = nullptr;                 // the default domain as a domain record (dom_record)
    int2 *d_axi_terms = nullptr;             // nine-statistic system: linearisation terms (mu index, coef)
    int *d_axi_toff = nullptr;               // [91] term offsets of E[psi psi^T] and E[ubar_x psi psi^T]
    // Scratch owned by the context (plain solver, flux at orders without a
    // fused kernel, velocity-space flux), allocated once when the context is
    // created.  Calls that use it are ordered on the GPU through scratch_ev
    // (recorded after each use, waited on before the next, whatever the
    // stream), and mu serialises their enqueueing.
    std::mutex mu;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    cudaEvent_t scratch_ev = nullptr;
    bool scratch_ev_live = false;
};

namespace mem_host {
int reserve_scratch(mem_ctx *ctx, size_t bytes);                     // at context creation only
int scratch_begin(mem_ctx *ctx, size_t bytes, cudaStream_t st);       // with ctx->mu held
void scratch_end(mem_ctx *ctx, cudaStream_t st);                      // with ctx->mu held
size_t plain_scratch_bytes(int Q);                                    // plain / mixed solve, one chunk
bool tc_available(const mem_ctx *ctx);
// Domain record of a velocity-space rule (what its kernels read per cell, all
// FP32): a_x, the block widths h_x = (b_x - a_x) / nbx and h_r = b_r / nbr as
// float pairs (hi, lo); two unused slots.
constexpr int DOM_REC = 8;
void dom_record(double ax, double bx, double br, int nbx, int nbr, float *rec);
int build_tc_tables(mem_ctx *ctx, const std::vector<double> &phi);
size_t tc_sigma_floats(int Q, int64_t cells);
int tc_contract(mem_ctx *ctx, const float *a_hi, const float *a_lo, int64_t rows, float *mom, int n, int *err,
                cudaStream_t st);
int residual64(mem_ctx *ctx, const float *M, const float *beta, const int32_t *status, int32_t mask, double *res,
               int32_t *status_out, double accept, int64_t B, cudaStream_t st);
size_t flux_scratch_bytes(int Q);                                     // dense flux, one chunk
int gh_rule(int n, std::vector<double> &x, std::vector<double> &w);
int solve_plain(mem_ctx *ctx, const float *M, float *beta, int32_t *status, int32_t *iters, int64_t B,
                const mem_solve_opts &o, cudaStream_t st, const unsigned char *active = nullptr);
int solve_mixed(mem_ctx *ctx, const float *M, float *beta, int32_t *status, int32_t *iters, int64_t B,
                const mem_solve_opts &o, cudaStream_t st, const unsigned char *active = nullptr);
int solve_fused(mem_ctx *ctx, const float *M, float *beta, int32_t *status, int32_t *iters, int64_t B,
                const mem_solve_opts &o, cudaStream_t st, const unsigned char *active = nullptr);
int flux(mem_ctx *ctx, const float *M, const float *beta, const float *g, float *F, float *speed, int64_t B,
         cudaStream_t st);
int flux_bufs(mem_ctx *ctx, const float *M, const float *beta, const float *g, float *F, float *speed, int64_t B,
              float *sigma, float *mom, cudaStream_t st);
int flux_fused(mem_ctx *ctx, const float *M, const float *beta, const float *g, float *F, float *speed,
               int64_t B, cudaStream_t st, bool axisym);
bool flux_fused_available(const mem_ctx *ctx);
int flux_from_mu(mem_ctx *ctx, const float *mu, const float *M, const float *g, float *F, float *speed, int64_t B,
                 cudaStream_t st, bool axisym);
int vel_run(mem_ctx *ctx, const float *M, float *beta, const float *g, int32_t *status, int32_t *iters, float *mu,
            const int *pid, const float *dom, int64_t B, const mem_solve_opts &o, bool solve, cudaStream_t st,
            const unsigned char *active = nullptr, float *cond = nullptr);
size_t vel_smem_bytes(int nx, int npt);
int build_axi_tables(mem_ctx *ctx);
int axi_occupancy(mem_ctx *ctx, int W, int *per_sm);
int fused_occupancy(mem_ctx *ctx, int W, int *per_sm);
int axi_run(mem_ctx *ctx, const float *M, float *beta, const float *g, int32_t *status, int32_t *iters, float *F,
            float *speed, const int *pid, const float *dom, int64_t B, const mem_solve_opts &o, bool solve,
            cudaStream_t st, const unsigned char *active = nullptr, float *cond = nullptr);
int gl_rule(int n, std::vector<double> &x, std::vector<double> &w);
int gauge_hermite(mem_ctx *ctx, const float *M_in, const float *g_in, float *g_out, float *M_out,
                  float *beta_inout, int64_t B, int axisym, cudaStream_t st);
int gauge_transform(const float *g_to, const float *g_from, const float *M_in, float *M_out, int64_t B,
                    cudaStream_t st);
int targets(mem_ctx *ctx, int gen_order, const float *v, const float *T, const float *a, const float *b,
            float *M_out, float *g_out, int64_t B, cudaStream_t st);
}  // namespace mem_host

#define MEM_CUDA_TRY(x)                                   \
    do {                                                  \
        cudaError_t e__ = (x);                            \
        if (e__ != cudaSuccess) return MEM_ECUDA;         \
    } while (0)

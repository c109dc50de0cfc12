// shock.h -- packed batch of independent 1D shock problems (host side).
#pragma once

#include <vector>

#include "ctx.h"

// Per-problem constants (device copy in ShockBatch::prm).
struct ShockProb {
    int off;       // first cell (left ghost) of the problem in the packed arrays
    int n;         // interior cells
    float dx;      // cell width
    float cfl_dx;  // cfl * dx
    float Pr;      // Prandtl number of the ES-BGK model
    float relax;   // tau = relax / n
    float drho;    // rho_+ - rho_- (normalises the steady-state metric)
    int scheme;    // interface flux, MEM_SCHEME_*
    int flic;      // FLIC limiter: 0 per statistic, 1 smallest of the nine (interface gauge), 2 density
    double t_end;  // > 0: simulated time at which the problem stops
};

// Per-problem step scalars (device).
struct ShockScalars {
    float dt;
    unsigned int steady_bits;  // max |d rho| of the last step, float bits (non-negative)
    double t;                  // simulated time
    int steps;
    int pad;
};

namespace mem_host {

struct ShockBatch {
    mem_ctx *ctx = nullptr;
    int P = 0;   // problems
    int NT = 0;  // packed cells, ghosts included
    std::vector<mem_shock_params> params;
    std::vector<ShockProb> hprm;
    float *M = nullptr, *beta = nullptr, *g = nullptr, *speed = nullptr, *F = nullptr, *Mn = nullptr;
    float *rho0 = nullptr, *sigma = nullptr, *mom = nullptr;
    float *mu = nullptr;      // [NT][MEM_MU_STRIDE] moment rows (velocity-space rule)
    float *dom = nullptr;     // [P][DOM_REC] integration domain record per problem (velocity-space rule)
    float *cond = nullptr;    // [NT] pivot-ratio condition estimate of each cell's last solve (velocity-space rule)
    int32_t *status = nullptr, *iters = nullptr;
    // Interfaces (Lax-Wendroff / FLIC problems only): entry c is the interface
    // between cells c - 1 and c of one problem (iface[c] set), in its own
    // Hermite gauge; other entries hold a copy of cell c so every row is valid.
    bool second_order = false;
    float *MI = nullptr, *betaI = nullptr, *gI = nullptr, *FI = nullptr, *speedI = nullptr;
    int32_t *statusI = nullptr, *itersI = nullptr;
    unsigned char *iface = nullptr;
    int *pid = nullptr;
    unsigned char *interior = nullptr;
    ShockProb *prm = nullptr;
    ShockScalars *sc = nullptr;
};

bool shock_params_valid(const mem_shock_params &p);
size_t batch_bytes_per_cell(const mem_ctx *ctx);
int batch_create(mem_ctx *ctx, const mem_shock_params *ps, int P, ShockBatch **out);
void batch_free(ShockBatch *b);
int batch_enqueue_step(ShockBatch *b, cudaStream_t st);
int batch_profiles(ShockBatch *b, int i, float *M_host, float *g_host, float *beta_host, float *rho, float *ux,
                   float *T, float *sxx, float *qx, double *t_out, int *steps_out);
int batch_read_scalars(ShockBatch *b, std::vector<ShockScalars> &out, cudaStream_t st);

}  // namespace mem_host

// tune.cu -- the autotuner of the persistent warp-per-cell kernels: for the
// fused Gauss-Hermite solve and the nine-statistic velocity-space solve it
// times every candidate launch shape (2, 4 or 8 warps per block; the
// resident blocks per SM at, 3/4 of and 1/2 of the occupancy limit) on the
// caller's own batch with CUDA events, keeps the fastest in the context and
// reports every candidate.  A cell's arithmetic does not depend on the launch
// shape (one warp computes one cell, whatever block it sits in), so the
// choice changes the time only, never a result.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "ctx.h"

extern "C" {

int mem_set_launch(mem_ctx *ctx, int kernel, int warps, int blocks_per_sm) {
    if (!ctx || (warps != 2 && warps != 4 && warps != 8) || blocks_per_sm < 0 || blocks_per_sm > 64) return MEM_EINVAL;
    if (kernel == MEM_TUNE_FUSED && !ctx->vel) ctx->cfg_fused = {warps, blocks_per_sm};
    else if (kernel == MEM_TUNE_AXI && ctx->vel) ctx->cfg_axi = {warps, blocks_per_sm};
    else return MEM_EINVAL;
    return MEM_OK;
}

int mem_get_launch(const mem_ctx *ctx, int kernel, int32_t *warps, int32_t *blocks_per_sm) {
    if (!ctx || !warps || !blocks_per_sm) return MEM_EINVAL;
    const mem_launch_cfg *c = kernel == MEM_TUNE_FUSED ? &ctx->cfg_fused : kernel == MEM_TUNE_AXI ? &ctx->cfg_axi : nullptr;
    if (!c) return MEM_EINVAL;
    *warps = c->warps;
    *blocks_per_sm = c->blocks_per_sm;
    return MEM_OK;
}

int mem_tune(mem_ctx *ctx, int kernel, const float *M, const float *beta0, const float *gauge, int64_t B, int reps,
             const mem_solve_opts *opts, mem_tune_report *out, void *stream) {
    if (!ctx || !M || !beta0 || !out || B <= 0 || reps < 1 || reps > 16) return MEM_EINVAL;
    if (kernel == MEM_TUNE_FUSED ? (ctx->vel || (ctx->n1d != 8 && ctx->n1d != 12))
                                 : (kernel != MEM_TUNE_AXI || !ctx->vel || !gauge))
        return MEM_EINVAL;
    mem_solve_opts o;
    mem_solve_opts_default(&o);
    if (opts) o = *opts;
    o.impl = MEM_IMPL_FUSED;
    cudaStream_t st = (cudaStream_t)stream;
    mem_launch_cfg &cfg = kernel == MEM_TUNE_FUSED ? ctx->cfg_fused : ctx->cfg_axi;
    const mem_launch_cfg saved = cfg;
    // candidates: the default first
    std::vector<mem_launch_cfg> cand = {{4, 0}};
    for (int W : {2, 4, 8}) {
        int per_sm = 0;
        const int rc = kernel == MEM_TUNE_FUSED ? mem_host::fused_occupancy(ctx, W, &per_sm)
                                                : mem_host::axi_occupancy(ctx, W, &per_sm);
        if (rc || per_sm < 1) continue;
        for (int b : {per_sm, (3 * per_sm + 3) / 4, (per_sm + 1) / 2}) {
            const mem_launch_cfg c{W, b};
            bool seen = false;
            for (auto &x : cand) seen |= (x.warps == c.warps && (x.blocks_per_sm == c.blocks_per_sm ||
                                                                 (x.blocks_per_sm == 0 && b == per_sm)));
            if (!seen && (int)cand.size() < 16) cand.push_back(c);
        }
    }
    // the tuner's own working memory (it runs at set-up, not in a hot loop)
    float *beta = nullptr;
    if (cudaMalloc(&beta, sizeof(float) * (size_t)B * NP) != cudaSuccess) {
        cudaGetLastError();
        return MEM_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MEM_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = MEM_ECUDA;
    memset(out, 0, sizeof(*out));
    float best = 1e30f;
    for (size_t i = 0; i < cand.size() && !rc; ++i) {
        cfg = cand[i];
        float t_best = 1e30f;
        for (int r = 0; r < reps + 1 && !rc; ++r) {  // the first run warms up
            if (cudaMemcpyAsync(beta, beta0, sizeof(float) * (size_t)B * NP, cudaMemcpyDeviceToDevice, st) !=
                    cudaSuccess ||
                cudaEventRecord(e0, st) != cudaSuccess) {
                rc = MEM_ECUDA;
                break;
            }
            rc = kernel == MEM_TUNE_FUSED
                     ? mem_host::solve_fused(ctx, M, beta, nullptr, nullptr, B, o, st)
                     : mem_host::axi_run(ctx, M, beta, gauge, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, B,
                                         o, true, st);
            float ms = 0.f;
            if (!rc && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = MEM_ECUDA;
            if (!rc && r > 0) t_best = std::min(t_best, ms);
        }
        if (rc) break;
        out->warps[i] = cfg.warps;
        out->blocks_per_sm[i] = cfg.blocks_per_sm;
        out->ms[i] = t_best;
        out->n = (int32_t)(i + 1);
        if (i == 0) out->default_ms = t_best;
        if (t_best < best) {
            best = t_best;
            out->best = (int32_t)i;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(beta);
    cfg = rc ? saved : cand[out->best];
    return rc;
}

}  // extern "C"

// ---- the tuning table on disk: one line per (device, rule, kernel),
// "device<TAB>rule<TAB>kernel<TAB>warps<TAB>blocks_per_sm".
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

namespace {

std::string rule_key(const mem_ctx *ctx) {
    char b[96];
    if (ctx->vel) snprintf(b, sizeof b, "vel%dx%dx%dx%d", ctx->nbx, ctx->nbr, ctx->ng, ctx->K);
    else snprintf(b, sizeof b, "gh%d", ctx->n1d);
    return b;
}

std::string device_key(const mem_ctx *ctx) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, ctx->device) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string s(p.name);
    for (char &ch : s)
        if (ch == '\t' || ch == '\n') ch = ' ';
    return s;
}

int tuned_kernel(const mem_ctx *ctx) { return ctx->vel ? MEM_TUNE_AXI : MEM_TUNE_FUSED; }

}  // namespace

extern "C" {

int mem_tune_save(const mem_ctx *ctx, const char *path) {
    if (!ctx || !path) return MEM_EINVAL;
    const std::string dev = device_key(ctx), rule = rule_key(ctx);
    const int kernel = tuned_kernel(ctx);
    const mem_launch_cfg &c = ctx->vel ? ctx->cfg_axi : ctx->cfg_fused;
    std::vector<std::string> keep;
    if (FILE *f = fopen(path, "r")) {
        char line[512];
        while (fgets(line, sizeof line, f)) {
            char d[256] = {0}, r[96] = {0};
            int k = -1, w = 0, b = 0;
            const bool same = sscanf(line, "%255[^\t]\t%95[^\t]\t%d\t%d\t%d", d, r, &k, &w, &b) == 5 && dev == d &&
                              rule == r && k == kernel;
            if (!same && strchr(line, '\t')) keep.push_back(line);
        }
        fclose(f);
    }
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return MEM_EINVAL;
    for (const std::string &l : keep) fputs(l.c_str(), f);
    fprintf(f, "%s\t%s\t%d\t%d\t%d\n", dev.c_str(), rule.c_str(), kernel, c.warps, c.blocks_per_sm);
    const bool ok = fclose(f) == 0 && rename(tmp.c_str(), path) == 0;
    return ok ? MEM_OK : MEM_EINVAL;
}

int mem_tune_load(mem_ctx *ctx, const char *path) {
    if (!ctx || !path) return MEM_EINVAL;
    FILE *f = fopen(path, "r");
    if (!f) return MEM_EINVAL;
    const std::string dev = device_key(ctx), rule = rule_key(ctx);
    const int kernel = tuned_kernel(ctx);
    int found = 0;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        char d[256] = {0}, r[96] = {0};
        int k = -1, w = 0, b = 0;
        if (sscanf(line, "%255[^\t]\t%95[^\t]\t%d\t%d\t%d", d, r, &k, &w, &b) == 5 && dev == d && rule == r &&
            k == kernel && mem_set_launch(ctx, kernel, w, b) == MEM_OK)
            found = 1;  // the last matching line wins
    }
    fclose(f);
    return found ? MEM_OK : MEM_ENOTFOUND;
}

}  // extern "C"

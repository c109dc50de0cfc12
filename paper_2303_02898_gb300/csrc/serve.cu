// serve.cu -- continuous batching of shock solves with device-resident state.
//
// Requests queue on the host.  Admitted requests live in one packed batch on
// the device (their M, beta, gauge and speeds stay resident between steps);
// every device iteration advances all of them by one Algorithm 2 time step,
// each with its own dt.  After each progress call, problems that reached the
// steady-state test (or their step cap) are retired -- their profiles copied
// to the host -- and queued requests are admitted while the cell and
// device-memory budgets allow.  Membership changes repack the batch:
// surviving problems' state is copied device-to-device into the new layout,
// so a problem's trajectory does not depend on who else is resident.  Each
// packed batch's time step is captured once in a CUDA graph (after one
// uncaptured step) and replayed for every step until the membership changes.
#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <mutex>
#include <string.h>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "shock.h"

using namespace mem;
using mem_host::ShockBatch;

namespace {
double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t id;
    mem_shock_params p;
    double t_submit;
    int steps;  // time steps taken so far
};

struct Done {
    mem_shock_result r;
    std::vector<float> rho, ux, T;
};
}  // namespace

struct mem_server {
    mem_ctx *ctx = nullptr;
    size_t budget = 0;
    int max_cells = 0;
    double steady_tol = 1e-6;
    int max_steps = 0;
    std::deque<Req> queue;
    std::vector<Req> resident;  // batch order
    ShockBatch *batch = nullptr;
    std::map<uint64_t, Done> done;
    uint64_t next_id = 1;
    int stats = 0;  // statistics system of every request (the first request's)
    cudaGraph_t graph = nullptr;      // one time step of the current batch
    cudaGraphExec_t gexec = nullptr;
    std::mutex mu;
};

namespace {

size_t cells_of(const std::vector<Req> &v) {
    size_t c = 0;
    for (auto &r : v) c += (size_t)r.p.ncells + 2;
    return c;
}

void drop_graph(mem_server *sv) {
    if (sv->gexec) cudaGraphExecDestroy(sv->gexec);
    if (sv->graph) cudaGraphDestroy(sv->graph);
    sv->gexec = nullptr;
    sv->graph = nullptr;
}

// k time steps of the resident batch: the first step of a new batch runs
// uncaptured (kernels set their launch attributes on first use), then one
// step is captured on a private stream and replayed.
int step_batch(mem_server *sv, int k, cudaStream_t st) {
    if (k <= 0) return MEM_OK;
    if (!sv->gexec) {
        int rc = mem_host::batch_enqueue_step(sv->batch, st);
        if (rc) return rc;
        if (--k == 0) return MEM_OK;
        MEM_CUDA_TRY(cudaStreamSynchronize(st));
        cudaStream_t cap;
        MEM_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rc = mem_host::batch_enqueue_step(sv->batch, cap);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(cap, &g);
            if (e == cudaSuccess && !rc) {
                sv->graph = g;
                e = cudaGraphInstantiate(&sv->gexec, g, 0);
                if (e != cudaSuccess) sv->gexec = nullptr;
            } else if (g) {
                cudaGraphDestroy(g);
            }
        }
        cudaStreamDestroy(cap);
        if (rc) return rc;
        if (e != cudaSuccess) {
            cudaGetLastError();
            drop_graph(sv);
            return MEM_ECUDA;
        }
    }
    for (int i = 0; i < k; ++i) MEM_CUDA_TRY(cudaGraphLaunch(sv->gexec, st));
    return MEM_OK;
}

// Retire every resident problem with error code rc (their device state is
// gone); queued requests stay queued.
void fail_resident(mem_server *sv, int rc) {
    const double t = now_s();
    for (auto &r : sv->resident) {
        Done dn;
        memset(&dn.r, 0, sizeof(dn.r));
        dn.r.status = rc;
        dn.r.steps = r.steps;
        dn.r.ncells = r.p.ncells;
        dn.r.latency_s = t - r.t_submit;
        sv->done[r.id] = std::move(dn);
    }
    sv->resident.clear();
}

// Rebuild the packed batch for the current resident list; problems that were
// already resident keep their state (copied device to device).
int rebuild(mem_server *sv, const std::vector<Req> &old_list, cudaStream_t st) {
    drop_graph(sv);
    ShockBatch *old = sv->batch;
    sv->batch = nullptr;
    if (sv->resident.empty()) {
        mem_host::batch_free(old);
        return MEM_OK;
    }
    std::vector<mem_shock_params> ps;
    for (auto &r : sv->resident) ps.push_back(r.p);
    ShockBatch *nb = nullptr;
    int rc = mem_host::batch_create(sv->ctx, ps.data(), (int)ps.size(), &nb);
    if (rc) {
        mem_host::batch_free(old);
        fail_resident(sv, rc);
        return rc;
    }
    if (old) {
        std::map<uint64_t, int> where;
        for (int i = 0; i < (int)old_list.size(); ++i) where[old_list[i].id] = i;
        cudaError_t e = cudaSuccess;
        auto cp = [&](void *dst, const void *src, size_t bytes) {
            if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
        };
        for (int i = 0; i < (int)sv->resident.size(); ++i) {
            auto it = where.find(sv->resident[i].id);
            if (it == where.end()) continue;
            const ShockProb &src = old->hprm[it->second], &dst = nb->hprm[i];
            const size_t nc = (size_t)src.n + 2;
            cp(nb->M + (size_t)dst.off * NP, old->M + (size_t)src.off * NP, sizeof(float) * nc * NP);
            cp(nb->beta + (size_t)dst.off * NP, old->beta + (size_t)src.off * NP, sizeof(float) * nc * NP);
            cp(nb->g + (size_t)dst.off * 6, old->g + (size_t)src.off * 6, sizeof(float) * nc * 6);
            cp(nb->speed + dst.off, old->speed + src.off, sizeof(float) * nc);
            cp(nb->status + dst.off, old->status + src.off, sizeof(int32_t) * nc);
            cp(nb->iters + dst.off, old->iters + src.off, sizeof(int32_t) * nc);
            cp(nb->sc + i, old->sc + it->second, sizeof(ShockScalars));
            if (src.scheme != MEM_SCHEME_LF) {
                // the interface solves' warm starts (Lax-Wendroff / FLIC)
                cp(nb->betaI + (size_t)dst.off * NP, old->betaI + (size_t)src.off * NP, sizeof(float) * nc * NP);
                cp(nb->gI + (size_t)dst.off * 6, old->gI + (size_t)src.off * 6, sizeof(float) * nc * 6);
                cp(nb->statusI + dst.off, old->statusI + src.off, sizeof(int32_t) * nc);
                cp(nb->itersI + dst.off, old->itersI + src.off, sizeof(int32_t) * nc);
            }
        }
        const cudaError_t es = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = es;
        mem_host::batch_free(old);
        if (e != cudaSuccess) {
            // neither batch survives a failed copy: the resident problems
            // are retired with the error, and the server stays consistent
            cudaGetLastError();
            mem_host::batch_free(nb);
            fail_resident(sv, MEM_ECUDA);
            return MEM_ECUDA;
        }
    }
    sv->batch = nb;
    return MEM_OK;
}

bool admit(mem_server *sv) {
    bool changed = false;
    size_t cells = cells_of(sv->resident);
    const size_t per = mem_host::batch_bytes_per_cell(sv->ctx);
    while (!sv->queue.empty()) {
        const size_t c = (size_t)sv->queue.front().p.ncells + 2;
        if (cells + c > (size_t)sv->max_cells || (cells + c) * per > sv->budget) break;
        sv->resident.push_back(sv->queue.front());
        sv->queue.pop_front();
        cells += c;
        changed = true;
    }
    return changed;
}

}  // namespace

extern "C" {

int mem_serve_create(mem_ctx *ctx, size_t hbm_budget_bytes, int32_t max_cells, double steady_tol, int32_t max_steps,
                     mem_server **out) {
    if (!ctx || !out || max_cells < 3 || max_steps < 1 || !(steady_tol > 0) || hbm_budget_bytes == 0) return MEM_EINVAL;
    mem_server *sv = new mem_server();
    sv->ctx = ctx;
    sv->budget = hbm_budget_bytes;
    sv->max_cells = max_cells;
    sv->steady_tol = steady_tol;
    sv->max_steps = max_steps;
    *out = sv;
    return MEM_OK;
}

int mem_serve_submit(mem_server *sv, const mem_shock_params *p, uint64_t *req_id) {
    if (!sv || !p || !req_id) return MEM_EINVAL;
    mem_shock_params q = *p;
    q.impl = MEM_IMPL_FUSED;  // one Newton back-end for the whole batch
    q.graph = 0;
    q.tol = 1e-8f;
    q.maxI = 500;
    if (!mem_host::shock_params_valid(q)) return MEM_EINVAL;
    const size_t c = (size_t)q.ncells + 2;
    if (c > (size_t)sv->max_cells || c * mem_host::batch_bytes_per_cell(sv->ctx) > sv->budget) return MEM_EBUSY;
    std::lock_guard<std::mutex> lock(sv->mu);
    if (!sv->stats) sv->stats = q.stats;
    if (q.stats != sv->stats) return MEM_EINVAL;  // one statistics system per batch
    Req r;
    r.id = sv->next_id++;
    r.p = q;
    r.t_submit = now_s();
    r.steps = 0;
    sv->queue.push_back(r);
    *req_id = r.id;
    return MEM_OK;
}

int mem_serve_progress(mem_server *sv, int iters, void *stream) {
    if (!sv || iters < 0) return MEM_EINVAL;
    std::lock_guard<std::mutex> lock(sv->mu);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<Req> before = sv->resident;
    if (admit(sv) || (!sv->batch && !sv->resident.empty())) {
        int rc = rebuild(sv, before, st);
        if (rc) return rc;
    }
    int remaining = iters;
    while (remaining > 0 && sv->batch) {
        // run no resident problem past its step cap
        int k = remaining;
        for (auto &r : sv->resident) k = std::min(k, sv->max_steps - r.steps);
        k = std::max(k, 0);
        {
            int rc = step_batch(sv, k, st);
            if (rc) return rc;
        }
        for (auto &r : sv->resident) r.steps += k;
        remaining -= std::max(k, 1);
        std::vector<ShockScalars> h;
        int rc = mem_host::batch_read_scalars(sv->batch, h, st);
        if (rc) return rc;
        const double t = now_s();
        std::vector<Req> keep;
        for (int i = 0; i < sv->batch->P; ++i) {
            float d;
            memcpy(&d, &h[i].steady_bits, sizeof(d));
            const double metric = (double)d / sv->batch->hprm[i].drho;
            const bool steady = h[i].steps >= 2 && metric < sv->steady_tol;
            if (!steady && h[i].steps < sv->max_steps) {
                keep.push_back(sv->resident[i]);
                continue;
            }
            Done dn;
            const int N = sv->batch->hprm[i].n;
            dn.rho.resize(N);
            dn.ux.resize(N);
            dn.T.resize(N);
            double tsim = 0.0;
            int steps = 0;
            rc = mem_host::batch_profiles(sv->batch, i, nullptr, nullptr, nullptr, dn.rho.data(), dn.ux.data(),
                                          dn.T.data(), nullptr, nullptr, &tsim, &steps);
            if (rc) return rc;
            dn.r.status = MEM_OK;
            dn.r.steps = steps;
            dn.r.ncells = N;
            dn.r.steady = steady ? 1 : 0;
            dn.r.sim_time = tsim;
            dn.r.latency_s = t - sv->resident[i].t_submit;
            sv->done[sv->resident[i].id] = std::move(dn);
        }
        if (keep.size() != sv->resident.size()) {
            before = sv->resident;
            sv->resident = keep;
            admit(sv);
            rc = rebuild(sv, before, st);
            if (rc) return rc;
        }
    }
    return MEM_OK;
}

int mem_serve_poll(mem_server *sv, uint64_t req_id, mem_shock_result *res, float *rho, float *ux, float *T) {
    if (!sv) return MEM_EINVAL;
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->done.find(req_id);
    if (it != sv->done.end()) {
        if (res) *res = it->second.r;
        const size_t N = it->second.rho.size();
        if (rho) memcpy(rho, it->second.rho.data(), sizeof(float) * N);
        if (ux) memcpy(ux, it->second.ux.data(), sizeof(float) * N);
        if (T) memcpy(T, it->second.T.data(), sizeof(float) * N);
        return MEM_OK;
    }
    for (auto &r : sv->queue)
        if (r.id == req_id) {
            if (res) { memset(res, 0, sizeof(*res)); res->status = MEM_PENDING; res->ncells = r.p.ncells; }
            return MEM_PENDING;
        }
    for (auto &r : sv->resident)
        if (r.id == req_id) {
            if (res) { memset(res, 0, sizeof(*res)); res->status = MEM_PENDING; res->ncells = r.p.ncells; }
            return MEM_PENDING;
        }
    return MEM_ENOTFOUND;
}

int mem_serve_stats(mem_server *sv, int32_t *queued, int32_t *resident, int32_t *resident_cells, int32_t *completed) {
    if (!sv) return MEM_EINVAL;
    std::lock_guard<std::mutex> lock(sv->mu);
    if (queued) *queued = (int32_t)sv->queue.size();
    if (resident) *resident = (int32_t)sv->resident.size();
    if (resident_cells) *resident_cells = (int32_t)cells_of(sv->resident);
    if (completed) *completed = (int32_t)sv->done.size();
    return MEM_OK;
}

void mem_serve_destroy(mem_server *sv) {
    if (!sv) return;
    drop_graph(sv);
    mem_host::batch_free(sv->batch);
    delete sv;
}

}  // extern "C"

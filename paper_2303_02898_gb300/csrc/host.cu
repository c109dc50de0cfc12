// host.cu -- mem_solve_host: Algorithm 1 (Section 3.2) on moments that live
// in host memory.  The batch streams through the device in chunks: while the
// fused kernel solves chunk i on the caller's stream, a copy stream brings
// chunk i + 1 in and takes chunk i - 1 out, so the host <-> device traffic
// hides behind the solves.  The staging buffers are two slots in the
// context's scratch.
#include <algorithm>

#include "common.cuh"
#include "ctx.h"

namespace {

constexpr int64_t HOST_CHUNK = 1 << 18;  // cells per chunk

struct Slot {
    float *M, *beta;
    int32_t *status, *iters;
};

size_t slot_bytes(int64_t C) {
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return 2 * up(sizeof(float) * (size_t)C * NP) + 2 * up(sizeof(int32_t) * (size_t)C);
}

Slot carve(char *base, int64_t C) {
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    Slot s;
    s.M = (float *)base;
    base += up(sizeof(float) * (size_t)C * NP);
    s.beta = (float *)base;
    base += up(sizeof(float) * (size_t)C * NP);
    s.status = (int32_t *)base;
    base += up(sizeof(int32_t) * (size_t)C);
    s.iters = (int32_t *)base;
    return s;
}

}  // namespace

extern "C" int mem_solve_host(mem_ctx *ctx, const float *M_host, float *beta_host, int32_t *status_host,
                              int32_t *iters_host, int64_t B, int warm, const mem_solve_opts *opts, void *stream) {
    if (!ctx || B < 0) return MEM_EINVAL;
    if (B == 0) return MEM_OK;
    if (!M_host || !beta_host || ctx->vel) return MEM_EINVAL;
    mem_solve_opts o;
    mem_solve_opts_default(&o);
    if (opts) o = *opts;
    if (o.maxI < 0 || o.maxT < 0 || o.maxT > 60 || o.max_lambda < 0 || o.max_lambda > 60) return MEM_EINVAL;
    // the fused back-end needs no scratch of its own, so the staging slots can use it
    if (o.impl != MEM_IMPL_FUSED || (ctx->n1d != 8 && ctx->n1d != 12)) return MEM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    MEM_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone) return MEM_EINVAL;

    std::lock_guard<std::mutex> lock(ctx->mu);
    const int64_t C = std::min<int64_t>(B, HOST_CHUNK);
    const size_t sb = slot_bytes(C);
    int rc = mem_host::scratch_begin(ctx, 2 * sb, st);
    if (rc) return rc;
    Slot slot[2] = {carve((char *)ctx->scratch, C), carve((char *)ctx->scratch + sb, C)};

    cudaStream_t cs = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_solved[2] = {nullptr, nullptr}, ev_out = nullptr, ev_start = nullptr;
    auto cleanup = [&]() {
        for (int s = 0; s < 2; ++s) {
            if (ev_in[s]) cudaEventDestroy(ev_in[s]);
            if (ev_solved[s]) cudaEventDestroy(ev_solved[s]);
        }
        if (ev_out) cudaEventDestroy(ev_out);
        if (ev_start) cudaEventDestroy(ev_start);
        if (cs) cudaStreamDestroy(cs);  // released once its work is done
    };
    auto fail = [&](int code) {
        cudaGetLastError();
        cleanup();
        return code;
    };
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return fail(MEM_ECUDA);
    for (int s = 0; s < 2; ++s)
        if (cudaEventCreateWithFlags(&ev_in[s], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev_solved[s], cudaEventDisableTiming) != cudaSuccess)
            return fail(MEM_ECUDA);
    if (cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming) != cudaSuccess)
        return fail(MEM_ECUDA);
    // the copy stream starts after what the caller's stream holds (the
    // previous user of the scratch included)
    if (cudaEventRecord(ev_start, st) != cudaSuccess || cudaStreamWaitEvent(cs, ev_start, 0) != cudaSuccess)
        return fail(MEM_ECUDA);

    const int64_t nchunks = (B + C - 1) / C;
    auto bring_in = [&](int64_t i) -> bool {
        const Slot &s = slot[i & 1];
        const int64_t c0 = i * C, n = std::min<int64_t>(C, B - c0);
        if (cudaMemcpyAsync(s.M, M_host + c0 * NP, sizeof(float) * (size_t)n * NP, cudaMemcpyHostToDevice, cs) !=
            cudaSuccess)
            return false;
        if (warm) {
            if (cudaMemcpyAsync(s.beta, beta_host + c0 * NP, sizeof(float) * (size_t)n * NP, cudaMemcpyHostToDevice,
                                cs) != cudaSuccess)
                return false;
        } else if (cudaMemsetAsync(s.beta, 0, sizeof(float) * (size_t)n * NP, cs) != cudaSuccess) {
            return false;
        }
        return cudaEventRecord(ev_in[i & 1], cs) == cudaSuccess;
    };
    auto take_out = [&](int64_t i) -> bool {
        const Slot &s = slot[i & 1];
        const int64_t c0 = i * C, n = std::min<int64_t>(C, B - c0);
        if (cudaStreamWaitEvent(cs, ev_solved[i & 1], 0) != cudaSuccess) return false;
        if (cudaMemcpyAsync(beta_host + c0 * NP, s.beta, sizeof(float) * (size_t)n * NP, cudaMemcpyDeviceToHost,
                            cs) != cudaSuccess)
            return false;
        if (status_host && cudaMemcpyAsync(status_host + c0, s.status, sizeof(int32_t) * (size_t)n,
                                           cudaMemcpyDeviceToHost, cs) != cudaSuccess)
            return false;
        if (iters_host && cudaMemcpyAsync(iters_host + c0, s.iters, sizeof(int32_t) * (size_t)n,
                                          cudaMemcpyDeviceToHost, cs) != cudaSuccess)
            return false;
        return true;
    };
    // copy-stream order: in 0, in 1, out 0, in 2, out 1, ...: chunk i + 2
    // reuses chunk i's slot only after chunk i's results have left it
    if (!bring_in(0)) return fail(MEM_ECUDA);
    for (int64_t i = 0; i < nchunks; ++i) {
        if (i + 1 < nchunks && !bring_in(i + 1)) return fail(MEM_ECUDA);
        const Slot &s = slot[i & 1];
        const int64_t n = std::min<int64_t>(C, B - i * C);
        if (cudaStreamWaitEvent(st, ev_in[i & 1], 0) != cudaSuccess) return fail(MEM_ECUDA);
        rc = mem_host::solve_fused(ctx, s.M, s.beta, s.status, s.iters, n, o, st);
        if (rc) return fail(rc);
        if (cudaEventRecord(ev_solved[i & 1], st) != cudaSuccess) return fail(MEM_ECUDA);
        if (!take_out(i)) return fail(MEM_ECUDA);
    }
    // the call is complete on the caller's stream once the last results are out
    if (cudaEventRecord(ev_out, cs) != cudaSuccess || cudaStreamWaitEvent(st, ev_out, 0) != cudaSuccess)
        return fail(MEM_ECUDA);
    mem_host::scratch_end(ctx, st);
    cleanup();
    return MEM_OK;
}

// gauge.cu -- Hermite gauge and change-of-gauge kernels (Section 3.3,
// Eqs. "Hermite parameters", "Change gauge M F"), one thread per cell.
#include "common.cuh"
#include "ctx.h"

using namespace mem;

namespace {

__global__ void k_gauge_hermite(const float *__restrict__ M_in, const float *__restrict__ g_in, float *g_out,
                                float *M_out, float *beta, int64_t B, int axisym) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= B) return;
    float m[NP], g[6], gh[6], y[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) m[k] = M_in[c * NP + k];
#pragma unroll
    for (int k = 0; k < 6; ++k) g[k] = g_in[c * 6 + k];
    hermite_gauge(m, g, axisym, gh);
    AxisMap T[3];
    gauge_maps(gh, g, T);
    apply_T(T, m, y);
    if (beta) {
        float b[NP], bo[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) b[k] = beta[c * NP + k];
        transform_beta(gh, g, b, bo);
#pragma unroll
        for (int k = 0; k < NP; ++k) beta[c * NP + k] = bo[k];
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) M_out[c * NP + k] = y[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) g_out[c * 6 + k] = gh[k];
}

__global__ void k_gauge_transform(const float *__restrict__ g_to, const float *__restrict__ g_from,
                                  const float *M_in, float *M_out, int64_t B) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= B) return;
    float m[NP], y[NP], gt[6], gf[6];
#pragma unroll
    for (int k = 0; k < NP; ++k) m[k] = M_in[c * NP + k];
#pragma unroll
    for (int k = 0; k < 6; ++k) { gt[k] = g_to[c * 6 + k]; gf[k] = g_from[c * 6 + k]; }
    AxisMap T[3];
    gauge_maps(gt, gf, T);
    apply_T(T, m, y);
#pragma unroll
    for (int k = 0; k < NP; ++k) M_out[c * NP + k] = y[k];
}

}  // namespace

namespace mem_host {

int gauge_hermite(mem_ctx *, const float *M_in, const float *g_in, float *g_out, float *M_out, float *beta_inout,
                  int64_t B, int axisym, cudaStream_t st) {
    k_gauge_hermite<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(M_in, g_in, g_out, M_out, beta_inout, B, axisym);
    MEM_CUDA_TRY(cudaGetLastError());
    return MEM_OK;
}

int gauge_transform(const float *g_to, const float *g_from, const float *M_in, float *M_out, int64_t B,
                    cudaStream_t st) {
    k_gauge_transform<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(g_to, g_from, M_in, M_out, B);
    MEM_CUDA_TRY(cudaGetLastError());
    return MEM_OK;
}

}  // namespace mem_host

// sumfact.cuh -- sum-factorised evaluation on the tensor Gauss-Hermite grid
// (nodes (x_i, x_j, x_k), fixed in the gauge frame): one warp per cell, lane l
// owning the node lines (j, k) = p with p = l + 32 r.
#pragma once

#include "common.cuh"
#include "ctx.h"

namespace mem {

constexpr int LDH = 35;

__host__ __device__ constexpr int ceil_div(int a, int b) { return (a + b - 1) / b; }

template <int N>
struct FusedCfg {
    static constexpr int P = N * N;              // node lines (j, k)
    static constexpr int R = ceil_div(P, 32);    // lines per lane
    static constexpr int NODES = R * N;          // nodes per lane
    static constexpr int S1 = 9 * P;             // stage-x output
    static constexpr int T2 = 45 * N;            // stage-y output
    static constexpr int WORK = (S1 + T2) > (NP1 * LDH) ? (S1 + T2) : (NP1 * LDH);
    // per-warp floats: beta, dbeta, M/n, grad, rhs, mu(165) + work
    static constexpr int WARP_FLOATS = 5 * 36 + 168 + WORK;
};

// Exponent contribution of a parameter vector v (slots 1..34) on the lane's
// nodes: out[r*N + i] = sum_a he_a(x_i) u_a(line r).  add_logw adds log w_q.
// v is read once into registers; each 1D table row he(x_i) once per node i.
template <int N>
__device__ __forceinline__ void exponent(const float *v, const float *he, const float *lw, int lane, bool add_logw,
                                         float (&out)[FusedCfg<N>::NODES]) {
    using C = FusedCfg<N>;
    float vr[NP];
#pragma unroll
    for (int k = 1; k < NP; ++k) vr[k] = v[k];
    float u[C::R][5], lwjk[C::R];
    bool live[C::R];
#pragma unroll
    for (int r = 0; r < C::R; ++r) {
        const int p = lane + 32 * r;
        live[r] = p < C::P;
        const int j = live[r] ? p / N : 0, k = live[r] ? p % N : 0;
        float hy[5], hz[5];
#pragma unroll
        for (int a = 0; a < 5; ++a) { hy[a] = he[j * MEM_HE_STRIDE + a]; hz[a] = he[k * MEM_HE_STRIDE + a]; }
#pragma unroll
        for (int a = 0; a <= 4; ++a) {
            float acc = 0.f;
#pragma unroll
            for (int b = 0; a + b <= 4; ++b) {
                float inner = 0.f;
#pragma unroll
                for (int c = 0; a + b + c <= 4; ++c)
                    if (a + b + c > 0) inner += vr[idx3(a, b, c)] * hz[c];
                acc += inner * hy[b];
            }
            u[r][a] = acc;
        }
        lwjk[r] = add_logw ? lw[j] + lw[k] : 0.f;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float hx[5];
#pragma unroll
        for (int a = 0; a < 5; ++a) hx[a] = he[i * MEM_HE_STRIDE + a];
        const float lwi = add_logw ? lw[i] : 0.f;
#pragma unroll
        for (int r = 0; r < C::R; ++r) {
            float e = lwjk[r] + lwi;
#pragma unroll
            for (int a = 0; a <= 4; ++a) e += u[r][a] * hx[a];
            out[r * N + i] = live[r] ? e : (add_logw ? -INFINITY : 0.f);
        }
    }
}

}  // namespace mem

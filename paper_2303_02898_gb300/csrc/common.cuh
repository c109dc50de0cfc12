// common.cuh -- device helpers shared by the kernels of the MEM library.
//
// Statistics are orthonormal Hermite products phi_(a,b,c) = he_a(x) he_b(y)
// he_c(z), he_k = He_k / sqrt(k!), ordered by total degree d, then a
// descending, then b descending.  With this order the index of (a,b,c) is
//     idx = d(d+1)(d+2)/6 + (b+c)(b+c+1)/2 + c,   d = a + b + c,
// which also enumerates the higher-degree Hermite products used for the
// Hessian and flux-Jacobian moments (165 of degree <= 8, 220 of degree <= 9).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mem.h"

#define NP 35
#define NP1 34

namespace mem {

__host__ __device__ constexpr int tri3(int d) { return d * (d + 1) * (d + 2) / 6; }
__host__ __device__ constexpr int idx3(int a, int b, int c) {
    return tri3(a + b + c) + (b + c) * (b + c + 1) / 2 + c;
}
// Decode statistic k into (a, b, c).
__host__ __device__ constexpr int deg_of(int k) {
    int d = 0;
    while (tri3(d + 1) <= k) ++d;
    return d;
}
__host__ __device__ constexpr int exp_a(int k) {
    int d = deg_of(k), p = k - tri3(d), j = 0;
    while ((j + 1) * (j + 2) / 2 <= p) ++j;
    return d - j;
}
__host__ __device__ constexpr int exp_c(int k) {
    int d = deg_of(k), p = k - tri3(d), j = 0;
    while ((j + 1) * (j + 2) / 2 <= p) ++j;
    return p - j * (j + 1) / 2;
}
__host__ __device__ constexpr int exp_b(int k) { return deg_of(k) - exp_a(k) - exp_c(k); }

static_assert(idx3(1, 0, 0) == 1 && idx3(0, 0, 1) == 3 && idx3(2, 0, 0) == 4 && idx3(0, 0, 2) == 9, "order");
static_assert(idx3(0, 0, 4) == 34 && tri3(5) == 35 && tri3(9) == 165 && tri3(10) == 220, "counts");
static_assert(exp_a(5) == 1 && exp_b(5) == 1 && exp_c(5) == 0, "decode");

// Orthonormal Hermite values he_0..he_K at x (He_{k+1} = x He_k - k He_{k-1}).
template <int K>
__device__ __forceinline__ void hermite_vals(float x, float (&h)[K + 1]) {
    float hm1 = 0.f, hc = 1.f;
    h[0] = 1.f;
    float inv = 1.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float hp = x * hc - (float)k * hm1;
        hm1 = hc;
        hc = hp;
        inv *= rsqrtf((float)(k + 1));
        h[k + 1] = hc * inv;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---------------------------------------------------------------------------
// Change of gauge.  For g -> g' the frames are related per axis by
// ubar' = s ubar + t with s = s_g / s_g', t = (w_g - w_g') / s_g'.  The
// coefficients of he_A(s x + t) in he_d(x) follow from the Appell property
// He_A(y + t) = sum_j C(A,j) t^(A-j) He_j(y) and the multiplication theorem
// He_j(s x) = sum_i s^(j-2i) (s^2-1)^i j! / ((j-2i)! i! 2^i) He_(j-2i)(x):
//   tmap[A][d] = sqrt(d!/A!) sum_{j>=d, j-d even} C(A,j) t^(A-j) s^d
//                ((s^2-1)/2)^((j-d)/2) j! / (d! ((j-d)/2)!).
// tmap is lower triangular (d <= A <= 4).
struct AxisMap {
    float m[5][5];
};

__host__ __device__ inline void axis_map(float s, float t, AxisMap &T) {
    const float fact[5] = {1.f, 1.f, 2.f, 6.f, 24.f};
    const float binom[5][5] = {{1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
    float tp[5], sp[5], hp[3];
    tp[0] = 1.f;
    sp[0] = 1.f;
    for (int i = 1; i < 5; ++i) { tp[i] = tp[i - 1] * t; sp[i] = sp[i - 1] * s; }
    const float h = 0.5f * (s * s - 1.f);
    hp[0] = 1.f; hp[1] = h; hp[2] = h * h;
    for (int A = 0; A < 5; ++A)
        for (int d = 0; d < 5; ++d) {
            float acc = 0.f;
            if (d <= A) {
                for (int j = d; j <= A; j += 2) {
                    int i = (j - d) / 2;
                    acc += binom[A][j] * tp[A - j] * sp[d] * hp[i] * fact[j] / (fact[d] * fact[i]);
                }
                acc *= sqrtf(fact[d] / fact[A]);
            }
            T.m[A][d] = acc;
        }
}

// Per-axis maps for T(g_to, g_from): M(g_to) = T M(g_from).
__host__ __device__ inline void gauge_maps(const float *g_to, const float *g_from, AxisMap (&T)[3]) {
    for (int ax = 0; ax < 3; ++ax) {
        float s = g_from[3 + ax] / g_to[3 + ax];
        float t = (g_from[ax] - g_to[ax]) / g_to[3 + ax];
        axis_map(s, t, T[ax]);
    }
}

// y = T x with T = tx (x) ty (x) tz restricted to total degree <= 4, applied
// axis by axis (each factor is lower triangular, so degree never grows).
__device__ __forceinline__ void apply_T(const AxisMap (&T)[3], const float *x, float *y) {
    float u[NP], v[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {  // along x: u_(a,b,c) = sum_{d<=a} tx[a][d] x_(d,b,c)
        const int a = exp_a(k), b = exp_b(k), c = exp_c(k);
        float acc = 0.f;
#pragma unroll
        for (int d = 0; d <= a; ++d) acc += T[0].m[a][d] * x[idx3(d, b, c)];
        u[k] = acc;
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int a = exp_a(k), b = exp_b(k), c = exp_c(k);
        float acc = 0.f;
#pragma unroll
        for (int e = 0; e <= b; ++e) acc += T[1].m[b][e] * u[idx3(a, e, c)];
        v[k] = acc;
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int a = exp_a(k), b = exp_b(k), c = exp_c(k);
        float acc = 0.f;
#pragma unroll
        for (int f = 0; f <= c; ++f) acc += T[2].m[c][f] * v[idx3(a, b, f)];
        y[k] = acc;
    }
}

// y = T^T x (each factor transposed: sum over a >= d).
__device__ __forceinline__ void apply_TT(const AxisMap (&T)[3], const float *x, float *y) {
    float u[NP], v[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int d = exp_a(k), b = exp_b(k), c = exp_c(k);
        float acc = 0.f;
#pragma unroll
        for (int a = d; a + b + c <= 4; ++a) acc += T[0].m[a][d] * x[idx3(a, b, c)];
        u[k] = acc;
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int a = exp_a(k), e = exp_b(k), c = exp_c(k);
        float acc = 0.f;
#pragma unroll
        for (int b = e; a + b + c <= 4; ++b) acc += T[1].m[b][e] * u[idx3(a, b, c)];
        v[k] = acc;
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int a = exp_a(k), b = exp_b(k), f = exp_c(k);
        float acc = 0.f;
#pragma unroll
        for (int c = f; a + b + c <= 4; ++c) acc += T[2].m[c][f] * v[idx3(a, b, c)];
        y[k] = acc;
    }
}

// Hermite gauge of moments M in gauge g (Eq. "Hermite parameters"): per-axis
// mean and standard deviation of u, or the axisymmetric 1D-shock form.
__device__ __forceinline__ void hermite_gauge(const float *M, const float *g, int axisym, float *gH) {
    const float n = M[0];
    float mean[3], ex2[3];
    const int i1[3] = {idx3(1, 0, 0), idx3(0, 1, 0), idx3(0, 0, 1)};
    const int i2[3] = {idx3(2, 0, 0), idx3(0, 2, 0), idx3(0, 0, 2)};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        float m1 = M[i1[ax]] / n;                       // E ubar
        float m2 = 1.41421356f * M[i2[ax]] / n + 1.f;    // E ubar^2
        float w = g[ax], s = g[3 + ax];
        mean[ax] = w + s * m1;
        // variance of u about its mean: s^2 (E ubar^2 - (E ubar)^2)
        ex2[ax] = s * s * (m2 - m1 * m1);
    }
    if (axisym) {
        gH[0] = mean[0]; gH[1] = 0.f; gH[2] = 0.f;
        gH[3] = sqrtf(ex2[0]);
        // s_r^2 = (<u_y^2> + <u_z^2>)/2 with raw second moments
        float sr2 = 0.5f * (ex2[1] + mean[1] * mean[1] + ex2[2] + mean[2] * mean[2]);
        gH[4] = gH[5] = sqrtf(sr2);
    } else {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) { gH[ax] = mean[ax]; gH[3 + ax] = sqrtf(ex2[ax]); }
    }
}

// Carry beta (Gauss-Hermite base measure) from gauge g_from to g_to:
// beta^L = beta + c with c = -(1/sqrt 2) on the three (2,0,0)-type slots is
// the Lebesgue-measure parameter, which maps with T(g_from, g_to)^T.
__device__ __forceinline__ void transform_beta(const float *g_to, const float *g_from, const float *beta, float *out) {
    AxisMap T[3];
    gauge_maps(g_from, g_to, T);
    float bl[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) bl[k] = k ? beta[k] : 0.f;
    const float c = -0.70710678f;
    bl[idx3(2, 0, 0)] += c; bl[idx3(0, 2, 0)] += c; bl[idx3(0, 0, 2)] += c;
    apply_TT(T, bl, out);
    out[idx3(2, 0, 0)] -= c; out[idx3(0, 2, 0)] -= c; out[idx3(0, 0, 2)] -= c;
    out[0] = beta[0];
}

}  // namespace mem

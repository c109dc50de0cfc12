// plain.cu -- the plain FP32 back-end: one kernel per stage of Algorithm 1,
// dense statistics tables, a host loop over Newton passes.  It is the
// baseline the fused back-end is measured against, and the flux/speed path
// (which needs the dense E[phi phi^T] and E[u_x phi phi^T]).
//
// Per Newton pass, over the cells still active:
//   k_linesearch  backtracking Armijo search on the objective (Algorithm 1,
//                 BackTrackingLineSearch / ArmijoCondition), update of beta,
//                 and sigma_q at the new beta (Section 3.1, log-sum-exp);
//   k_sgemm       [cells x Q] x [Q x 630] -> E phi, E phi_i phi_j (packed);
//   k_newton      gradient, Hessian = covariance (Appendix C), Cholesky with
//                 lambda*I retries, two triangular solves, decrement, status.
#include <float.h>

#include "common.cuh"
#include "ctx.h"
#include "linalg.cuh"
#include "sumfact.cuh"

using namespace mem;

namespace {

__device__ __forceinline__ float tc_round(float x) {  // to TF32, nearest (ties away)
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

constexpr int BLK = 256;
constexpr int MAXJ = 16;  // nodes per thread: Q <= 4096
constexpr int CHUNK = 1 << 16;

__device__ __forceinline__ float block_reduce_max(float v, float *red) {
    v = warp_max(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    float r = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : -INFINITY;
    if (w == 0) r = warp_max(r);
    if (threadIdx.x == 0) red[0] = r;
    __syncthreads();
    return red[0];
}

__device__ __forceinline__ float block_reduce_sum(float v, float *red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    float r = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.f;
    if (w == 0) r = warp_sum(r);
    if (threadIdx.x == 0) red[0] = r;
    __syncthreads();
    return red[0];
}

struct PlainState {
    float *sigma;  // [CHUNK][Q] (mixed back-end: TF32 hi part, rows padded to whole tiles of 128)
    float *sig_lo; // mixed back-end: TF32 lo part, same layout
    float *mom;    // [CHUNK][630]
    float *db;     // [CHUNK][35]
    float *G;      // [CHUNK][35]
    float *Lcur;   // [CHUNK]
    float *alpha;  // [CHUNK]
    int *it;       // [CHUNK]
    int *st;       // [CHUNK]
    int *act0, *act1;  // [CHUNK]
    int *cnt;      // [2]
    int *err;      // [1] mixed back-end: a tensor-core wait timed out
};

__global__ void k_init(const float *__restrict__ M, float *__restrict__ beta, int n, PlainState S,
                       int32_t *status, int32_t *iters, const unsigned char *active) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    if (active && !active[c]) return;
    const float *m = M + (size_t)c * NP;
    float *b = beta + (size_t)c * NP;
    bool bad = !(m[0] > 0.f) || !isfinite(m[0]);
    for (int k = 0; k < NP; ++k) bad |= !isfinite(m[k]) || (k > 0 && !isfinite(b[k]));
    S.it[c] = 0;
    for (int k = 0; k < NP; ++k) { S.db[(size_t)c * NP + k] = 0.f; S.G[(size_t)c * NP + k] = 0.f; }
    S.Lcur[c] = NAN;
    if (bad) {
        S.st[c] = MEM_ST_BADINPUT;
        if (status) status[c] = MEM_ST_BADINPUT;
        if (iters) iters[c] = 0;
        return;
    }
    S.st[c] = 0;
    b[0] = m[0];
    const int slot = atomicAdd(&S.cnt[0], 1);
    S.act0[slot] = c;
}

// One block per active cell.  Nodes q = tid + 256 j.  The exponent of the
// trial point beta + alpha dbeta is e_beta + alpha e_dbeta (both computed once).
__global__ void __launch_bounds__(BLK) k_linesearch(const int *__restrict__ act, const float *__restrict__ M,
                                                    float *__restrict__ beta, PlainState S,
                                                    const float *__restrict__ phiT, const float *__restrict__ logw,
                                                    int Q, mem_solve_opts o) {
    __shared__ float sb[NP], sd[NP], sm[NP], sg[NP], red[32], sc[4];
    const int slot = blockIdx.x, c = act[slot], tid = threadIdx.x;
    const float *Mc = M + (size_t)c * NP;
    float *bc = beta + (size_t)c * NP;
    if (tid < NP) {
        const float n = Mc[0];
        sb[tid] = tid ? bc[tid] : 0.f;
        sd[tid] = tid ? S.db[(size_t)c * NP + tid] : 0.f;
        sg[tid] = tid ? S.G[(size_t)c * NP + tid] : 0.f;
        sm[tid] = tid ? Mc[tid] / n : 0.f;
    }
    __syncthreads();
    if (tid == 0) {
        float gd = 0.f, mb = 0.f, md = 0.f;
        for (int k = 1; k < NP; ++k) { gd += sg[k] * sd[k]; mb += sb[k] * sm[k]; md += sd[k] * sm[k]; }
        sc[0] = gd; sc[1] = mb; sc[2] = md;
    }
    float eb[MAXJ], ed[MAXJ];
    const int nj = (Q + BLK - 1) / BLK;
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) {
        eb[j] = -INFINITY;
        ed[j] = 0.f;
        const int q = tid + j * BLK;
        if (j < nj && q < Q) {
            float s = logw[q], d = 0.f;
            for (int k = 1; k < NP; ++k) {
                const float p = phiT[(size_t)k * Q + q];
                s += sb[k] * p;
                d += sd[k] * p;
            }
            eb[j] = s;
            ed[j] = d;
        }
    }
    __syncthreads();
    const float gd = sc[0], mb = sc[1], md = sc[2];
    float Lcur = S.Lcur[c];
    if (isnan(Lcur)) {  // first pass: objective at the start point
        float mx = -INFINITY;
#pragma unroll
        for (int j = 0; j < MAXJ; ++j) mx = fmaxf(mx, eb[j]);
        mx = block_reduce_max(mx, red);
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < MAXJ; ++j) s += (j < nj) ? __expf(eb[j] - mx) : 0.f;
        s = block_reduce_sum(s, red);
        Lcur = mx + logf(s) - mb;
    }
    float alpha = 2.f, Lt = NAN, mx = 0.f, Z = 1.f;
    bool sat = false;
    for (int s = 0; !sat && s <= o.maxT; ++s) {
        alpha *= 0.5f;
        float m = -INFINITY;
#pragma unroll
        for (int j = 0; j < MAXJ; ++j) m = fmaxf(m, eb[j] + alpha * ed[j]);
        mx = block_reduce_max(m, red);
        float z = 0.f;
#pragma unroll
        for (int j = 0; j < MAXJ; ++j) z += (j < nj) ? __expf(eb[j] + alpha * ed[j] - mx) : 0.f;
        Z = block_reduce_sum(z, red);
        Lt = mx + logf(Z) - (mb + alpha * md);
        const float LD = Lcur - Lt, gradD = -o.c_armijo * alpha * gd;
        sat = (LD - gradD) >= -(o.atol + o.rtol * fabsf(LD));
    }
    const float invZ = 1.f / Z;
    {
        float *sig = S.sigma + (size_t)slot * Q;
#pragma unroll
        for (int j = 0; j < MAXJ; ++j) {
            const int q = tid + j * BLK;
            if (j < nj && q < Q) sig[q] = __expf(eb[j] + alpha * ed[j] - mx) * invZ;
        }
    }
    if (tid >= 1 && tid < NP) bc[tid] = sb[tid] + alpha * sd[tid];
    if (tid == 0) { S.Lcur[c] = Lt; S.alpha[c] = alpha; }
}

// The line search of the mixed back-end, one warp per active cell: the same
// steps as k_linesearch (exponents at beta and dbeta, Armijo backtracking,
// sigma of the accepted point), with the exponents sum-factorised on the
// tensor Gauss-Hermite grid (nodes q = i N^2 + p, lane l owning the node
// lines p = l + 32 r: the order of the dense tables) and sigma written as a
// TF32 hi row and a TF32 lo row (sigma = hi + lo to about 2^-22), 32
// consecutive nodes per warp store.  Persistent: resident blocks whose warps
// loop over the active cells.
template <int N>
__global__ void __launch_bounds__(128) k_linesearch_sf(const int *__restrict__ act, int nact,
                                                       const float *__restrict__ M, float *__restrict__ beta,
                                                       PlainState S, const float *__restrict__ he1d,
                                                       const float *__restrict__ logw1d, mem_solve_opts o) {
    using C = FusedCfg<N>;
    constexpr int Q = N * N * N;
    __shared__ float s_he[N * MEM_HE_STRIDE], s_lw[16];
    __shared__ float sv[4][4][36];
    for (int t = threadIdx.x; t < N * MEM_HE_STRIDE; t += blockDim.x) s_he[t] = he1d[t];
    for (int t = threadIdx.x; t < N; t += blockDim.x) s_lw[t] = logw1d[t];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // persistent: each warp takes active cells gridDim.x * 4 apart
    for (int slot = blockIdx.x * 4 + w; slot < nact; slot += gridDim.x * 4) {
        const int c = act[slot];
        const float *Mc = M + (size_t)c * NP;
        float *bc = beta + (size_t)c * NP;
        float *sb = sv[w][0], *sd = sv[w][1], *sg = sv[w][2], *sm = sv[w][3];
        const float n = Mc[0];
        for (int k = lane; k < NP; k += 32) {
            sb[k] = k ? bc[k] : 0.f;
            sd[k] = k ? S.db[(size_t)c * NP + k] : 0.f;
            sg[k] = k ? S.G[(size_t)c * NP + k] : 0.f;
            sm[k] = k ? Mc[k] / n : 0.f;
        }
        __syncwarp();
        float pg = 0.f, pb = 0.f, pd = 0.f;
        for (int k = lane; k < NP; k += 32) {
            pg += sg[k] * sd[k];
            pb += sb[k] * sm[k];
            pd += sd[k] * sm[k];
        }
        const float gd = warp_sum(pg), mb = warp_sum(pb), md = warp_sum(pd);
        float eb[C::NODES], ed[C::NODES];
        exponent<N>(sb, s_he, s_lw, lane, true, eb);
        exponent<N>(sd, s_he, s_lw, lane, false, ed);
        float Lcur = S.Lcur[c];
        if (isnan(Lcur)) {  // first pass: objective at the start point
            float m = -INFINITY;
#pragma unroll
            for (int q = 0; q < C::NODES; ++q) m = fmaxf(m, eb[q]);
            const float mx0 = warp_max(m);
            float z = 0.f;
#pragma unroll
            for (int q = 0; q < C::NODES; ++q) z += __expf(eb[q] - mx0);
            Lcur = mx0 + logf(warp_sum(z)) - mb;
        }
        float alpha = 2.f, Lt = NAN, mx = 0.f, Z = 1.f;
        bool sat = false;
        for (int s = 0; !sat && s <= o.maxT; ++s) {
            alpha *= 0.5f;
            float m = -INFINITY;
#pragma unroll
            for (int q = 0; q < C::NODES; ++q) m = fmaxf(m, fmaf(alpha, ed[q], eb[q]));
            mx = warp_max(m);
            float z = 0.f;
#pragma unroll
            for (int q = 0; q < C::NODES; ++q) z += __expf(fmaf(alpha, ed[q], eb[q]) - mx);
            Z = warp_sum(z);
            Lt = mx + logf(Z) - (mb + alpha * md);
            const float LD = Lcur - Lt, gradD = -o.c_armijo * alpha * gd;
            sat = (LD - gradD) >= -(o.atol + o.rtol * fabsf(LD));
        }
        const float invZ = 1.f / Z;
        float *hi_row = S.sigma + (size_t)slot * Q, *lo_row = S.sig_lo + (size_t)slot * Q;
#pragma unroll
        for (int r = 0; r < C::R; ++r) {
            const int p = lane + 32 * r;
            if (p < C::P) {
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    const float v = __expf(fmaf(alpha, ed[r * N + i], eb[r * N + i]) - mx) * invZ;
                    const float hi = tc_round(v);
                    hi_row[i * C::P + p] = hi;
                    lo_row[i * C::P + p] = tc_round(v - hi);
                }
            }
        }
        for (int k = lane; k < NP; k += 32)
            if (k >= 1) bc[k] = sb[k] + alpha * sd[k];
        if (lane == 0) { S.Lcur[c] = Lt; S.alpha[c] = alpha; }
        __syncwarp();  // the warp's vectors are free for its next cell
    }
}

// C[M x N] = A[M x K] B[K x N], row-major, 64x64 tiles, 4x4 per thread.
__global__ void __launch_bounds__(256) k_sgemm(const float *__restrict__ A, const float *__restrict__ Bm,
                                               float *__restrict__ C, int M, int N, int K) {
    __shared__ float As[16][68];
    __shared__ float Bs[16][64];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int e = threadIdx.x + l * 256;
            const int r = e >> 4, cc = e & 15;
            As[cc][r] = (row0 + r < M && k0 + cc < K) ? A[(size_t)(row0 + r) * K + k0 + cc] : 0.f;
            const int rb = e >> 6, cb = e & 63;
            Bs[rb][cb] = (k0 + rb < K && col0 + cb < N) ? Bm[(size_t)(k0 + rb) * N + col0 + cb] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = row0 + ty * 4 + i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int cc = col0 + tx * 4 + j;
            if (cc < N) C[(size_t)r * N + cc] = acc[i][j];
        }
    }
}

// LDH (sumfact.cuh): leading dimension of the 34 x 34 Hessian in shared memory

// Warp per active cell: gradient, Hessian, modified Cholesky, Newton
// direction, decrement and the convergence test of Algorithm 1.
__global__ void __launch_bounds__(128) k_newton(const int *__restrict__ act, int nact, const float *__restrict__ M,
                                                float *__restrict__ beta, PlainState S, int *__restrict__ act_next,
                                                int *__restrict__ cnt_next, mem_solve_opts o,
                                                int32_t *status, int32_t *iters) {
    __shared__ float sA[4][NP1 * LDH];
    __shared__ float sv[4][3][NP];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = blockIdx.x * 4 + w;
    if (slot >= nact) return;
    const int c = act[slot];
    float *A = sA[w], *m = sv[w][0], *G = sv[w][1], *b = sv[w][2];
    const float *mom = S.mom + (size_t)slot * MEM_NCOL_SOLVE;
    const float *Mc = M + (size_t)c * NP;
    const float n = Mc[0];
    for (int k = lane; k < NP; k += 32) m[k] = mom[k];
    __syncwarp();
    for (int k = lane; k < NP; k += 32) {
        G[k] = k ? m[k] - Mc[k] / n : 0.f;
        S.G[(size_t)c * NP + k] = G[k];
    }
    int st = S.st[c];
    auto load_H = [&](float lam) {
        __syncwarp();
        for (int p = lane; p < NP1 * (NP1 + 1) / 2; p += 32) {
            int i = (int)((sqrtf(8.f * p + 1.f) - 1.f) * 0.5f);
            while (i * (i + 1) / 2 > p) --i;
            while ((i + 1) * (i + 2) / 2 <= p) ++i;
            const int j = p - i * (i + 1) / 2;
            float h = mom[NP + p] - m[i + 1] * m[j + 1];
            if (i == j) h += lam;
            A[i * LDH + j] = h;
        }
        __syncwarp();
    };
    load_H(0.f);
    bool ok = warp_cholesky(A, NP1, LDH, lane);
    float lam = o.lambda0;
    for (int t = 0; !ok && t < o.max_lambda; ++t) {
        st |= MEM_ST_LAMBDA;
        load_H(lam);
        ok = warp_cholesky(A, NP1, LDH, lane);
        lam *= o.lambda_mul;
    }
    const int it = S.it[c] + 1;
    bool done = false;
    float res = NAN;
    if (!ok) {
        st |= MEM_ST_LAMBDA_CAP | MEM_ST_NONFINITE;
        done = true;
    } else {
        for (int k = lane; k < NP1; k += 32) b[k] = -G[k + 1];
        warp_solve_lower(A, NP1, LDH, b, lane);
        warp_solve_upperT(A, NP1, LDH, b, lane);
        float part = 0.f;
        for (int k = lane; k < NP1; k += 32) part += b[k] * G[k + 1];
        res = 0.5f * fabsf(warp_sum(part));
        for (int k = lane; k < NP; k += 32) S.db[(size_t)c * NP + k] = k ? b[k - 1] : 0.f;
        if (!isfinite(res)) {
            st |= MEM_ST_NONFINITE;
            done = true;
        } else {
            const float alpha = S.alpha[c];
            const bool conv_res = res <= o.tol, conv_a = alpha <= o.alpha_min;
            if (conv_res) st |= MEM_ST_CONVERGED;
            if (conv_a) st |= MEM_ST_STAGNATED;
            if (conv_res || conv_a) done = true;
            else if (it > o.maxI) { st |= MEM_ST_MAXITER; done = true; }
            if (done && conv_res && o.final_step) {
                float *bc = beta + (size_t)c * NP;
                for (int k = lane + 1; k < NP; k += 32) bc[k] += b[k - 1];
            }
        }
    }
    if (lane == 0) {
        S.it[c] = it;
        S.st[c] = st;
        if (done) {
            if (status) status[c] = st;
            if (iters) iters[c] = it;
        } else {
            act_next[atomicAdd(cnt_next, 1)] = c;
        }
    }
}

// The Newton step of the mixed back-end: k_newton with the register-resident
// Cholesky of the fused back-end (reg_chol_solve34: lane j holds column j,
// pivot columns broadcast through shared memory, both triangular solves
// fused) in place of the shared-memory factorisation.  Same results up to
// rounding order, same lambda I retries and status bits.  Persistent: a grid
// of resident blocks whose warps loop over the active cells; the packed
// Hessian index of each entry comes from a per-block table.
__global__ void __launch_bounds__(128) k_newton_reg(const int *__restrict__ act, int nact, const float *__restrict__ M,
                                                    float *__restrict__ beta, PlainState S, int *__restrict__ act_next,
                                                    int *__restrict__ cnt_next, mem_solve_opts o, int32_t *status,
                                                    int32_t *iters) {
    __shared__ float sA[4][NP1 * LDH];
    __shared__ float sv[4][2][36];
    __shared__ __align__(16) float sbc[4][36];
    __shared__ int s_pij[NP1 * (NP1 + 1) / 2];  // packed entry p -> i | j << 8
    for (int p = threadIdx.x; p < NP1 * (NP1 + 1) / 2; p += blockDim.x) {
        int i = 0;
        while ((i + 1) * (i + 2) / 2 <= p) ++i;
        s_pij[p] = i | ((p - i * (i + 1) / 2) << 8);
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // persistent: each warp takes active cells gridDim.x * 4 apart
    for (int slot = blockIdx.x * 4 + w; slot < nact; slot += gridDim.x * 4) {
        const int c = act[slot];
        float *A = sA[w], *m = sv[w][0], *G = sv[w][1];
        const float *mom = S.mom + (size_t)slot * MEM_NCOL_SOLVE;
        const float *Mc = M + (size_t)c * NP;
        const float n = Mc[0];
        for (int k = lane; k < NP; k += 32) m[k] = mom[k];
        __syncwarp();
        for (int k = lane; k < NP; k += 32) {
            G[k] = k ? m[k] - Mc[k] / n : 0.f;
            S.G[(size_t)c * NP + k] = G[k];
        }
        for (int p = lane; p < NP1 * (NP1 + 1) / 2; p += 32) {
            const int ij = s_pij[p], i = ij & 255, j = ij >> 8;
            A[i * LDH + j] = mom[NP + p] - m[i + 1] * m[j + 1];
        }
        __syncwarp();
        int st = S.st[c];
        const float g_l = G[lane + 1], g32 = G[33], g33 = G[34];
        float x = 0.f, x32 = 0.f, x33 = 0.f, lam = 0.f;
        bool ok = false;
        for (int t = 0; t <= o.max_lambda; ++t) {
            ok = reg_chol_solve34<true>(A, lam, lane, -g_l, -g32, -g33, x, x32, x33, sbc[w]);
            if (ok) break;
            st |= MEM_ST_LAMBDA;
            lam = (t == 0) ? o.lambda0 : lam * o.lambda_mul;
        }
        const int it = S.it[c] + 1;
        bool done = false;
        if (!ok) {
            st |= MEM_ST_LAMBDA_CAP | MEM_ST_NONFINITE;
            done = true;
        } else {
            const float res = 0.5f * fabsf(warp_sum(x * g_l) + x32 * g32 + x33 * g33);
            float *db = S.db + (size_t)c * NP;
            db[lane + 1] = x;
            if (lane == 0) { db[0] = 0.f; db[33] = x32; db[34] = x33; }
            if (!isfinite(res)) {
                st |= MEM_ST_NONFINITE;
                done = true;
            } else {
                const float alpha = S.alpha[c];
                const bool conv_res = res <= o.tol, conv_a = alpha <= o.alpha_min;
                if (conv_res) st |= MEM_ST_CONVERGED;
                if (conv_a) st |= MEM_ST_STAGNATED;
                if (conv_res || conv_a) done = true;
                else if (it > o.maxI) { st |= MEM_ST_MAXITER; done = true; }
                if (done && conv_res && o.final_step) {
                    float *bc = beta + (size_t)c * NP;
                    bc[lane + 1] += x;
                    if (lane == 0) { bc[33] += x32; bc[34] += x33; }
                }
            }
        }
        if (lane == 0) {
            S.it[c] = it;
            S.st[c] = st;
            if (done) {
                if (status) status[c] = st;
                if (iters) iters[c] = it;
            } else {
                act_next[atomicAdd(cnt_next, 1)] = c;
            }
        }
        __syncwarp();  // the warp's buffers are free for its next cell
    }
}

// sigma_q of each cell at beta (flux path), one block per cell.
__global__ void __launch_bounds__(BLK) k_sigma(const float *__restrict__ beta, float *__restrict__ sigma,
                                               const float *__restrict__ phiT, const float *__restrict__ logw, int Q) {
    __shared__ float sb[NP], red[32];
    const int c = blockIdx.x, tid = threadIdx.x;
    if (tid < NP) sb[tid] = tid ? beta[(size_t)c * NP + tid] : 0.f;
    __syncthreads();
    float e[MAXJ];
    const int nj = (Q + BLK - 1) / BLK;
    float mx = -INFINITY;
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) {
        e[j] = -INFINITY;
        const int q = tid + j * BLK;
        if (j < nj && q < Q) {
            float s = logw[q];
            for (int k = 1; k < NP; ++k) s += sb[k] * phiT[(size_t)k * Q + q];
            e[j] = s;
            mx = fmaxf(mx, s);
        }
    }
    mx = block_reduce_max(mx, red);
    float z = 0.f;
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) z += (j < nj) ? __expf(e[j] - mx) : 0.f;
    z = block_reduce_sum(z, red);
    const float inv = 1.f / z;
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) {
        const int q = tid + j * BLK;
        if (j < nj && q < Q) sigma[(size_t)c * Q + q] = __expf(e[j] - mx) * inv;
    }
}

constexpr int LDF = 36;

// Warp per cell: F = n (w_x E phi + s_x E ubar_x phi) and the spectral radius
// of the pencil (E[ubar_x phi phi^T], E[phi phi^T]) mapped to u_x: Cholesky
// whitening C = L^{-1} X L^{-T}, Lanczos with full re-orthogonalisation, and
// Sturm multisection on the tridiagonal matrix for both extreme eigenvalues.
__global__ void __launch_bounds__(64) k_flux_speed(const float *__restrict__ mom, const float *__restrict__ M,
                                                   const float *__restrict__ gauge, float *__restrict__ F,
                                                   float *__restrict__ speed, int B, float xmax) {
    __shared__ float sL[2][NP * LDF], sY[2][NP * LDF], sC[2][NP * LDF], sab[2][2][NP + 1];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * 2 + w;
    if (c >= B) return;
    float *L = sL[w], *Y = sY[w], *C = sC[w], *al = sab[w][0], *bt = sab[w][1];
    const float *mr = mom + (size_t)c * MEM_NCOL_FLUX;
    const float n = M[(size_t)c * NP];
    const float wx = gauge[(size_t)c * 6], sx = gauge[(size_t)c * 6 + 3];
    if (F)
        for (int k = lane; k < NP; k += 32) F[(size_t)c * NP + k] = n * (wx * mr[k] + sx * mr[NP + k]);
    if (!speed) return;
    for (int p = lane; p < 630; p += 32) {
        int i = (int)((sqrtf(8.f * p + 1.f) - 1.f) * 0.5f);
        while (i * (i + 1) / 2 > p) --i;
        while ((i + 1) * (i + 2) / 2 <= p) ++i;
        const int j = p - i * (i + 1) / 2;
        L[i * LDF + j] = mr[70 + p];
        const float x = mr[700 + p];
        Y[i * LDF + j] = x;
        Y[j * LDF + i] = x;
    }
    __syncwarp();
    if (!warp_cholesky(L, NP, LDF, lane)) {
        if (lane == 0) speed[c] = fmaxf(fabsf(wx + sx * xmax), fabsf(wx - sx * xmax));
        return;
    }
    // Y <- L^{-1} Y (columns), then C = L^{-1} Y^T (columns of Y^T = rows of Y).
    for (int j = lane; j < NP; j += 32)
        for (int i = 0; i < NP; ++i) {
            float s = Y[i * LDF + j];
            for (int k = 0; k < i; ++k) s -= L[i * LDF + k] * Y[k * LDF + j];
            Y[i * LDF + j] = s / L[i * LDF + i];
        }
    __syncwarp();
    for (int j = lane; j < NP; j += 32)
        for (int i = 0; i < NP; ++i) {
            float s = Y[j * LDF + i];
            for (int k = 0; k < i; ++k) s -= L[i * LDF + k] * C[k * LDF + j];
            C[i * LDF + j] = s / L[i * LDF + i];
        }
    __syncwarp();
    for (int p = lane; p < NP * NP; p += 32) {
        const int i = p / NP, j = p % NP;
        if (j < i) {
            const float s = 0.5f * (C[i * LDF + j] + C[j * LDF + i]);
            C[i * LDF + j] = s;
            C[j * LDF + i] = s;
        }
    }
    __syncwarp();
    // Lanczos; the vectors live in Y (row k = v_k).
    float *V = Y;
    const float inv35 = rsqrtf((float)NP);
    for (int i = lane; i < NP; i += 32) V[i] = inv35;
    float cnorm = 0.f;
    for (int i = lane; i < NP; i += 32) cnorm = fmaxf(cnorm, fabsf(C[i * LDF + i]));
    for (int p = lane; p < NP * NP; p += 32) cnorm = fmaxf(cnorm, fabsf(C[(p / NP) * LDF + p % NP]));
    cnorm = warp_max(cnorm) + 1e-30f;
    __syncwarp();
    int m = 0;
    for (int k = 0; k < NP; ++k) {
        float wv[2] = {0.f, 0.f};
        for (int r = 0; r < 2; ++r) {
            const int i = lane + 32 * r;
            if (i < NP) {
                float s = 0.f;
                for (int j = 0; j < NP; ++j) s += C[i * LDF + j] * V[k * LDF + j];
                wv[r] = s;
            }
        }
        float part = 0.f;
        for (int r = 0; r < 2; ++r) { const int i = lane + 32 * r; if (i < NP) part += wv[r] * V[k * LDF + i]; }
        const float a = warp_sum(part);
        if (lane == 0) al[k] = a;
        // full re-orthogonalisation (two classical Gram-Schmidt passes)
        for (int pass = 0; pass < 2; ++pass)
            for (int j = 0; j <= k; ++j) {
                float pp = 0.f;
                for (int r = 0; r < 2; ++r) { const int i = lane + 32 * r; if (i < NP) pp += wv[r] * V[j * LDF + i]; }
                const float d = warp_sum(pp);
                for (int r = 0; r < 2; ++r) { const int i = lane + 32 * r; if (i < NP) wv[r] -= d * V[j * LDF + i]; }
            }
        float nn = 0.f;
        for (int r = 0; r < 2; ++r) { const int i = lane + 32 * r; if (i < NP) nn += wv[r] * wv[r]; }
        const float bk = sqrtf(warp_sum(nn));
        m = k + 1;
        if (k + 1 == NP || bk <= 1e-6f * cnorm) break;
        if (lane == 0) bt[k] = bk;
        for (int r = 0; r < 2; ++r) { const int i = lane + 32 * r; if (i < NP) V[(k + 1) * LDF + i] = wv[r] / bk; }
        __syncwarp();
    }
    __syncwarp();
    const float mu_hi = warp_tridiag_extreme(al, bt, m, true, lane);
    const float mu_lo = warp_tridiag_extreme(al, bt, m, false, lane);
    // the exact speed never exceeds the node bound (Rayleigh quotients of u_x);
    // a larger or non-finite FP32 estimate is replaced by it
    const float bound = fmaxf(fabsf(wx + sx * xmax), fabsf(wx - sx * xmax));
    const float sp = fmaxf(fabsf(wx + sx * mu_hi), fabsf(wx + sx * mu_lo));
    if (lane == 0) speed[c] = sp <= bound ? sp : bound;
}

// Relative moment residual ||E phi(beta) - M/n|| / ||M/n|| in FP64 (the
// sums over i >= 1; the norm of M/n includes M_0/n = 1), warp per cell,
// grid-stride; only cells with (status & mask) != 0 when mask != 0.
__global__ void __launch_bounds__(128) k_residual64(const float *__restrict__ M, const float *__restrict__ beta,
                                                    const int32_t *__restrict__ status, int32_t mask,
                                                    double *__restrict__ res, int32_t *status_out, double accept,
                                                    int64_t B, const double *__restrict__ phiT,
                                                    const double *__restrict__ logw, int Q) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * 4;
    for (int64_t c = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5); c < B; c += nw) {
        if (mask && !(status[c] & mask)) continue;
        double b[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) b[k] = k ? (double)beta[c * NP + k] : 0.0;
        double mx = -INFINITY;
        for (int q = lane; q < Q; q += 32) {
            double e = logw[q];
            for (int k = 1; k < NP; ++k) e += b[k] * phiT[(size_t)k * Q + q];
            mx = fmax(mx, e);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        double m[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) m[k] = 0.0;
        for (int q = lane; q < Q; q += 32) {
            double e = logw[q];
            for (int k = 1; k < NP; ++k) e += b[k] * phiT[(size_t)k * Q + q];
            const double w = exp(e - mx);
#pragma unroll
            for (int k = 0; k < NP; ++k) m[k] += w * phiT[(size_t)k * Q + q];
        }
        double num = 0.0, den = 0.0;
        const double n = (double)M[c * NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            double v = m[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            m[k] = v;
        }
        const double Z = m[0];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const double t = (double)M[c * NP + k] / n;
            den += t * t;
            if (k) num += (m[k] / Z - t) * (m[k] / Z - t);
        }
        const double r = sqrt(num / den);
        if (lane == 0) {
            res[c] = r;
            if (status_out && r <= accept) status_out[c] |= MEM_ST_FP64_OK;
        }
    }
}

void sgemm(const float *A, const float *Bm, float *C, int M, int N, int K, cudaStream_t st) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_sgemm<<<grid, 256, 0, st>>>(A, Bm, C, M, N, K);
}

}  // namespace

namespace mem_host {

// Resident blocks of the mixed back-end's persistent line-search kernel.
template <int N>
static int linesearch_sf_grid(mem_ctx *ctx) {
    static int grid = 0;
    if (!grid) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_linesearch_sf<N>, 128, 0);
        cudaGetLastError();
        grid = std::max(1, sms * std::max(1, per_sm));
    }
    return grid;
}

// Resident blocks of the mixed back-end's persistent Newton kernel.
static int newton_reg_grid(mem_ctx *ctx) {
    static int grid = 0;
    if (!grid) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_newton_reg, 128, 0);
        cudaGetLastError();
        grid = std::max(1, sms * std::max(1, per_sm));
    }
    return grid;
}

static size_t plain_need(int Q, size_t CH) {
    // sigma hi + lo (mixed: whole tiles of 128 cells), moments,
    // per-cell vectors and scalars, the FP64 residuals of failed cells
    const size_t sig = tc_sigma_floats(Q, (int64_t)CH);
    return sizeof(float) * (2 * sig + CH * ((size_t)MEM_NCOL_SOLVE + 2 * NP + 2)) + sizeof(int) * (CH * 4 + 4) +
           sizeof(double) * CH + 16 * 256;
}

size_t plain_scratch_bytes(int Q) { return plain_need(Q, CHUNK); }
size_t flux_scratch_bytes(int Q) { return sizeof(float) * (size_t)CHUNK * ((size_t)Q + MEM_NCOL_FLUX) + 1024; }

// The plain (FP32 SIMT contraction) and mixed (tensor-core contraction)
// back-ends: per chunk of cells, a host loop over Newton passes of
// line search -> contraction -> Newton step, compacting the active cells.
static int solve_dense(mem_ctx *ctx, const float *M, float *beta, int32_t *status, int32_t *iters, int64_t B,
                       const mem_solve_opts &o, cudaStream_t st, const unsigned char *active, bool mixed) {
    std::lock_guard<std::mutex> lock(ctx->mu);
    const int Q = ctx->Q;
    if (mixed && (!tc_available(ctx) || Q > MAXJ * BLK)) return MEM_EINVAL;
    const size_t CH = (size_t)std::min<int64_t>(B, CHUNK);
    int rc = scratch_begin(ctx, plain_need(Q, CH), st);
    if (rc) return rc;
    struct End {
        mem_ctx *c;
        cudaStream_t s;
        ~End() { scratch_end(c, s); }
    } end_{ctx, st};
    char *p = (char *)ctx->scratch;
    auto take = [&](size_t bytes) { char *r = p; p += (bytes + 255) & ~(size_t)255; return r; };
    PlainState S;
    const size_t sig = mixed ? tc_sigma_floats(Q, (int64_t)CH) : CH * Q;
    S.sigma = (float *)take(sizeof(float) * sig);
    S.sig_lo = mixed ? (float *)take(sizeof(float) * sig) : nullptr;
    S.mom = (float *)take(sizeof(float) * CH * MEM_NCOL_SOLVE);
    S.db = (float *)take(sizeof(float) * CH * NP);
    S.G = (float *)take(sizeof(float) * CH * NP);
    S.Lcur = (float *)take(sizeof(float) * CH);
    S.alpha = (float *)take(sizeof(float) * CH);
    S.it = (int *)take(sizeof(int) * CH);
    S.st = (int *)take(sizeof(int) * CH);
    S.act0 = (int *)take(sizeof(int) * CH);
    S.act1 = (int *)take(sizeof(int) * CH);
    S.cnt = (int *)take(sizeof(int) * 2);
    S.err = (int *)take(sizeof(int) * 2);
    double *res64 = (double *)take(sizeof(double) * CH);
    if ((size_t)(p - (char *)ctx->scratch) > ctx->scratch_bytes) return MEM_ENOMEM;
    if (mixed) MEM_CUDA_TRY(cudaMemsetAsync(S.err, 0, sizeof(int), st));
    for (int64_t c0 = 0; c0 < B; c0 += CH) {
        const int n = (int)std::min<int64_t>(CH, B - c0);
        const float *Mc = M + c0 * NP;
        float *bc = beta + c0 * NP;
        int32_t *stc = status ? status + c0 : nullptr, *itc = iters ? iters + c0 : nullptr;
        MEM_CUDA_TRY(cudaMemsetAsync(S.cnt, 0, 2 * sizeof(int), st));
        k_init<<<(n + 255) / 256, 256, 0, st>>>(Mc, bc, n, S, stc, itc, active ? active + c0 : nullptr);
        int hc[2] = {0, 0};  // active cells, tensor-core error flag
        MEM_CUDA_TRY(cudaMemcpyAsync(&hc[0], S.cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
        MEM_CUDA_TRY(cudaStreamSynchronize(st));
        int nact = hc[0];
        int *cur = S.act0, *nxt = S.act1;
        int cur_cnt = 0;
        for (int pass = 0; pass <= o.maxI + 1 && nact > 0; ++pass) {
            if (mixed) {
                if (ctx->n1d == 8)
                    k_linesearch_sf<8><<<std::min((nact + 3) / 4, linesearch_sf_grid<8>(ctx)), 128, 0, st>>>(cur, nact, Mc, bc, S, ctx->d_he1d,
                                                                      ctx->d_logw1d, o);
                else
                    k_linesearch_sf<12><<<std::min((nact + 3) / 4, linesearch_sf_grid<12>(ctx)), 128, 0, st>>>(cur, nact, Mc, bc, S, ctx->d_he1d,
                                                                       ctx->d_logw1d, o);
                rc = tc_contract(ctx, S.sigma, S.sig_lo, (int64_t)(sig / Q), S.mom, nact, S.err, st);
                if (rc) return rc;
            } else {
                k_linesearch<<<nact, BLK, 0, st>>>(cur, Mc, bc, S, ctx->d_phiT, ctx->d_logw, Q, o);
                sgemm(S.sigma, ctx->d_tab_solve, S.mom, nact, MEM_NCOL_SOLVE, Q, st);
            }
            const int nxt_cnt = 1 - cur_cnt;
            MEM_CUDA_TRY(cudaMemsetAsync(S.cnt + nxt_cnt, 0, sizeof(int), st));
            if (mixed)
                k_newton_reg<<<std::min((nact + 3) / 4, newton_reg_grid(ctx)), 128, 0, st>>>(cur, nact, Mc, bc, S, nxt,
                                                                                          S.cnt + nxt_cnt, o, stc, itc);
            else
                k_newton<<<(nact + 3) / 4, 128, 0, st>>>(cur, nact, Mc, bc, S, nxt, S.cnt + nxt_cnt, o, stc, itc);
            MEM_CUDA_TRY(cudaMemcpyAsync(&hc[0], S.cnt + nxt_cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
            if (mixed) MEM_CUDA_TRY(cudaMemcpyAsync(&hc[1], S.err, sizeof(int), cudaMemcpyDeviceToHost, st));
            MEM_CUDA_TRY(cudaStreamSynchronize(st));
            if (hc[1]) return MEM_ECUDA;  // the tensor cores did not signal completion in time
            nact = hc[0];
            std::swap(cur, nxt);
            cur_cnt = nxt_cnt;
        }
        // The safeguard of the mixed back-end: cells whose step failed get
        // their moment residual recomputed in FP64.
        if (mixed && stc) {
            rc = residual64(ctx, Mc, bc, stc, MEM_ST_MAXITER | MEM_ST_NONFINITE | MEM_ST_LAMBDA_CAP, res64, stc, 1e-5,
                            n, st);
            if (rc) return rc;
        }
    }
    MEM_CUDA_TRY(cudaGetLastError());
    return MEM_OK;
}

int solve_plain(mem_ctx *ctx, const float *M, float *beta, int32_t *status, int32_t *iters, int64_t B,
                const mem_solve_opts &o, cudaStream_t st, const unsigned char *active) {
    return solve_dense(ctx, M, beta, status, iters, B, o, st, active, false);
}

int solve_mixed(mem_ctx *ctx, const float *M, float *beta, int32_t *status, int32_t *iters, int64_t B,
                const mem_solve_opts &o, cudaStream_t st, const unsigned char *active) {
    return solve_dense(ctx, M, beta, status, iters, B, o, st, active, true);
}

// FP64 relative moment residual, warp per evaluated cell.
int residual64(mem_ctx *ctx, const float *M, const float *beta, const int32_t *status, int32_t mask, double *res,
               int32_t *status_out, double accept, int64_t B, cudaStream_t st) {
    if (!ctx->d_phiT64) return MEM_EINVAL;
    const int blocks = (int)std::min<int64_t>((B + 3) / 4, 65535);
    k_residual64<<<blocks, 128, 0, st>>>(M, beta, status, mask, res, status_out, accept, B, ctx->d_phiT64,
                                        ctx->d_logw64, ctx->Q);
    MEM_CUDA_TRY(cudaGetLastError());
    return MEM_OK;
}

int flux_bufs(mem_ctx *ctx, const float *M, const float *beta, const float *g, float *F, float *speed, int64_t B,
              float *sigma, float *mom, cudaStream_t st) {
    const int n = (int)B;
    k_sigma<<<n, BLK, 0, st>>>(beta, sigma, ctx->d_phiT, ctx->d_logw, ctx->Q);
    sgemm(sigma, ctx->d_tab_flux, mom, n, MEM_NCOL_FLUX, ctx->Q, st);
    k_flux_speed<<<(n + 1) / 2, 64, 0, st>>>(mom, M, g, F, speed, n, ctx->xmax);
    MEM_CUDA_TRY(cudaGetLastError());
    return MEM_OK;
}

int flux(mem_ctx *ctx, const float *M, const float *beta, const float *g, float *F, float *speed, int64_t B,
         cudaStream_t st) {
    std::lock_guard<std::mutex> lock(ctx->mu);
    const int Q = ctx->Q;
    const size_t CH = (size_t)std::min<int64_t>(B, CHUNK);
    int rc = scratch_begin(ctx, sizeof(float) * CH * ((size_t)Q + MEM_NCOL_FLUX) + 1024, st);
    if (rc) return rc;
    float *sigma = (float *)ctx->scratch;
    float *mom = sigma + ((CH * Q + 63) & ~(size_t)63);
    for (int64_t c0 = 0; c0 < B; c0 += CH) {
        const int64_t n = std::min<int64_t>(CH, B - c0);
        rc = flux_bufs(ctx, M + c0 * NP, beta + c0 * NP, g + c0 * 6, F ? F + c0 * NP : nullptr,
                       speed ? speed + c0 : nullptr, n, sigma, mom, st);
        if (rc) break;
    }
    scratch_end(ctx, st);
    return rc;
}

}  // namespace mem_host

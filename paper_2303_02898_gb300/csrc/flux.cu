// flux.cu -- fused flux and characteristic speed, one warp per cell, no
// scratch memory (Eq. "The ME equation" subeq. 3 and Eq. "The lax F").
//
//   sigma_q      from the sum-factorised exponent at beta (log-sum-exp);
//   mu_abc       the 220 Hermite-product moments of degree <= 9, by the three
//                axis stages over the tensor grid;
//   F_k          = n (w_x mu_k + s_x E[ubar_x phi_k]), with
//                  ubar_x he_a = sqrt(a+1) he_{a+1} + sqrt(a) he_{a-1};
//   E[phi phi^T], E[ubar_x phi phi^T] (35 x 35, phi_0 included) from mu by
//                the Hermite linearisation (per-lane term sequences);
//   speed        = max |w_x + s_x mu| over the generalised eigenvalues mu of
//                  (E[ubar_x phi phi^T], E[phi phi^T]): Cholesky whitening
//                  C = L^{-1} X L^{-T}, Lanczos (three-term recurrence, 35
//                  steps or until breakdown) and Sturm multisection for both
//                  extreme Ritz values.  Ritz values of a symmetric matrix lie
//                  inside its spectrum and the extremes converge first, so
//                  lost orthogonality (ghost copies) cannot move the spectral
//                  radius; if E[phi phi^T] is numerically singular the
//                  Rayleigh-quotient bound over the nodes is used.
#include "common.cuh"
#include "ctx.h"
#include "linalg.cuh"
#include "sumfact.cuh"

using namespace mem;

namespace {

constexpr int FWARPS = 2;
constexpr int LDF = 36;

// Per-warp work area: the stage buffers (unless the moments come in), then
// the matrices of the speed: 2 x 35 x 36 for the full pencil, 928 floats for
// the three parity blocks (offsets up to 848 + 5 x 16).  A smaller area keeps
// more warps resident.
template <int N, bool AXI = false, bool MU_IN = false>
struct FluxCfg {
    using C = FusedCfg<N>;
    static constexpr int S1 = 10 * C::P;  // stage x, a <= 9
    static constexpr int T2 = 55 * N;     // stage y, a + b <= 9
    static constexpr int STAGES = MU_IN ? 0 : S1 + T2;
    static constexpr int MAT = AXI ? 928 : 2 * NP * LDF;
    static constexpr int WORK = STAGES > MAT ? STAGES : MAT;
    static constexpr int WARP_FLOATS = 36 + 224 + 2 * 36 + 36 + 72 + WORK;  // beta, mu, alpha/beta, v, l0/inv, work
};

struct FluxArgs {
    const float *M, *beta, *gauge;
    float *F, *speed;
    int64_t B;
    const float *he1d, *logw1d;
    const int2 *slots;
    int n_slots;
    const int2 *aslots;
    int n_aslots;
    float xmax;
    const float *mu;  // moments rows [B][MEM_MU_STRIDE] (moments-in variant)
};

// Every generalised eigenvalue of (E[u_x phi phi^T], E[phi phi^T]) is a
// Rayleigh quotient, i.e. a weighted average of the nodes' u_x, so the exact
// speed never exceeds the node bound.  An FP32 estimate above it (or not
// finite) comes from a pencil too ill-conditioned for single precision and is
// replaced by the bound.
__device__ __forceinline__ float clamp_speed(float sp, float bound) { return sp <= bound ? sp : bound; }

// MU_IN: the moments of degree <= 9 come precomputed per cell (rows of
// A.mu, with the node range of u_x in slots 220, 221) instead of from the
// gauge-frame rule; everything after the moments is shared.
template <int N, bool AXI, bool MU_IN>
__global__ void __launch_bounds__(FWARPS * 32) k_fused_flux(FluxArgs A) {
    using C = FusedCfg<N>;
    using Cf = FluxCfg<N, AXI, MU_IN>;
    extern __shared__ float smem[];
    float *s_he = smem;
    float *s_lw = s_he + N * MEM_HE_STRIDE;
    int *s_abc = (int *)(s_lw + 16);  // [220] packed (a, b, c)
    int *s_ab = s_abc + 224;          // [55]  packed (a, b)
    int *s_pij = s_ab + 56;           // [595] packed (i, j), i >= j, 34 x 34
    int *s_pij35 = s_pij + 596;       // [630] packed (i, j), i >= j, 35 x 35
    float *wbase = (float *)(s_pij35 + 632);
    if (!MU_IN) {
        for (int t = threadIdx.x; t < N * MEM_HE_STRIDE; t += blockDim.x) s_he[t] = A.he1d[t];
        for (int t = threadIdx.x; t < N; t += blockDim.x) s_lw[t] = A.logw1d[t];
    }
    for (int t = threadIdx.x; t < 220; t += blockDim.x) s_abc[t] = exp_a(t) | (exp_b(t) << 8) | (exp_c(t) << 16);
    for (int t = threadIdx.x; t < NP * (NP + 1) / 2; t += blockDim.x) {
        int i = 0;
        while ((i + 1) * (i + 2) / 2 <= t) ++i;
        const int v = i | ((t - i * (i + 1) / 2) << 8);
        s_pij35[t] = v;
        if (t < NP1 * (NP1 + 1) / 2) s_pij[t] = v;
    }
    for (int t = threadIdx.x; t < 55; t += blockDim.x) {
        int d = 0;
        while ((d + 1) * (d + 2) / 2 <= t) ++d;
        const int b = t - d * (d + 1) / 2;
        s_ab[t] = (d - b) | (b << 8);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *W = wbase + warp * Cf::WARP_FLOATS;
    float *sb = W, *smu = W + 36, *al = smu + 224, *bt = al + 36, *sv = bt + 36, *sl0 = sv + 36, *sinv = sl0 + 36;
    float *work = sinv + 36;
    float *S1 = work, *T2 = work + Cf::S1;
    float *L = work, *Y = work + NP * LDF;  // alias the stage buffers (H in L, LDH rows)

    const int64_t nwarps = (int64_t)gridDim.x * FWARPS;
    for (int64_t cell = (int64_t)blockIdx.x * FWARPS + warp; cell < A.B; cell += nwarps) {
        const float n = A.M[cell * NP];
        const float wx = A.gauge[cell * 6], sx = A.gauge[cell * 6 + 3];
        // speed bound over the nodes, used when the pencil has no reliable spectrum
        float bound;
        if (MU_IN) {
            const float *row = A.mu + cell * MEM_MU_STRIDE;
            for (int t = lane; t < 220; t += 32) smu[t] = row[t];
            bound = fmaxf(fabsf(row[220]), fabsf(row[221]));
            __syncwarp();
        } else {
            bound = fmaxf(fabsf(wx + sx * A.xmax), fabsf(wx - sx * A.xmax));
        }
        if (!MU_IN) {
        if (lane < NP) sb[lane] = lane ? A.beta[cell * NP + lane] : 0.f;
        if (lane + 32 < NP) sb[lane + 32] = A.beta[cell * NP + lane + 32];
        __syncwarp();
        // ---- sigma
        float eb[C::NODES];
        exponent<N>(sb, s_he, s_lw, lane, true, eb);
        float mx = -INFINITY;
#pragma unroll
        for (int q = 0; q < C::NODES; ++q) mx = fmaxf(mx, eb[q]);
        mx = warp_max(mx);
        float z = 0.f;
#pragma unroll
        for (int q = 0; q < C::NODES; ++q) { eb[q] = __expf(eb[q] - mx); z += eb[q]; }
        const float invZ = 1.f / warp_sum(z);
        // ---- stage x: s_a(p) = sum_i sigma(i,p) he_a(x_i), a <= 9
        {
            float sa[C::R][10];
#pragma unroll
            for (int r = 0; r < C::R; ++r)
#pragma unroll
                for (int a = 0; a < 10; ++a) sa[r][a] = 0.f;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                float hx[10];
#pragma unroll
                for (int a = 0; a < 10; ++a) hx[a] = s_he[i * MEM_HE_STRIDE + a];
#pragma unroll
                for (int r = 0; r < C::R; ++r) {
                    const float sg = eb[r * N + i] * invZ;
#pragma unroll
                    for (int a = 0; a < 10; ++a) sa[r][a] += sg * hx[a];
                }
            }
#pragma unroll
            for (int r = 0; r < C::R; ++r) {
                const int p = lane + 32 * r;
                if (p < C::P) {
#pragma unroll
                    for (int a = 0; a < 10; ++a) S1[a * C::P + p] = sa[r][a];
                }
            }
        }
        __syncwarp();
        // ---- stage y: t_ab(k) = sum_j s_a(j,k) he_b(y_j), a + b <= 9
        for (int t = lane; t < Cf::T2; t += 32) {
            const int ab = t / N, k = t % N;
            const int abp = s_ab[ab], a = abp & 255, b = abp >> 8;
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < N; ++j) acc += S1[a * C::P + j * N + k] * s_he[j * MEM_HE_STRIDE + b];
            T2[ab * N + k] = acc;
        }
        __syncwarp();
        // ---- stage z: mu_abc = sum_k t_ab(k) he_c(z_k), a + b + c <= 9
        for (int t = lane; t < 220; t += 32) {
            const int abc = s_abc[t], a = abc & 255, b = (abc >> 8) & 255, c = abc >> 16;
            const int ab = (a + b) * (a + b + 1) / 2 + b;
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < N; ++k) acc += T2[ab * N + k] * s_he[k * MEM_HE_STRIDE + c];
            smu[t] = acc;
        }
        __syncwarp();
        }
        // ---- flux
        if (A.F) {
            for (int k = lane; k < NP; k += 32) {
                const int a = exp_a(k), b = exp_b(k), c = exp_c(k);
                float xk = sqrtf((float)(a + 1)) * smu[idx3(a + 1, b, c)];
                if (a > 0) xk += sqrtf((float)a) * smu[idx3(a - 1, b, c)];
                A.F[cell * NP + k] = n * (wx * smu[k] + sx * xk);
            }
        }
        if (!A.speed) continue;
        if (AXI) {
            // Axisymmetric cell: the pencil is block-diagonal over the parity
            // classes of (b, c); the spectral radius is the largest over the
            // blocks ee (14, phi_0 included), oe (8; eo has the same
            // spectrum) and oo (5).
            {
                float acc = 0.f;
#pragma unroll 4
                for (int t = 0; t < A.n_aslots; ++t) {
                    const int2 sl = __ldg(&A.aslots[t * 32 + lane]);
                    acc = fmaf(__int_as_float(sl.y), smu[sl.x & 255], acc);
                    if (sl.x < 0) {
                        work[(sl.x >> 8) & 0xffff] = acc;
                        acc = 0.f;
                    }
                }
            }
            __syncwarp();
            float mlo, mhi, lo, hi;
            bool ok = small_pencil_extremes(work, work + 256, 14, al, bt, sv, lane, mlo, mhi);
            if (ok) ok = small_pencil_extremes(work + 512, work + 640, 8, al, bt, sv, lane, lo, hi);
            if (ok) {
                mlo = fminf(mlo, lo);
                mhi = fmaxf(mhi, hi);
                ok = small_pencil_extremes(work + 768, work + 848, 5, al, bt, sv, lane, lo, hi);
            }
            if (ok) {
                mlo = fminf(mlo, lo);
                mhi = fmaxf(mhi, hi);
            }
            if (lane == 0)
                A.speed[cell] = clamp_speed(ok ? fmaxf(fabsf(wx + sx * mhi), fabsf(wx + sx * mlo)) : bound, bound);
            __syncwarp();
            continue;
        }
        // ---- E[phi phi^T] without its phi_0 border, and E[ubar_x phi phi^T]
        // (lower triangles), from the linearisation terms; every slot carries
        // the shared-memory offset of its entry.
        {
            float acc = 0.f;
#pragma unroll 4
            for (int t = 0; t < A.n_slots; ++t) {
                const int2 sl = __ldg(&A.slots[t * 32 + lane]);
                acc = fmaf(__int_as_float(sl.y), smu[sl.x & 255], acc);
                if (sl.x < 0) {
                    work[(sl.x >> 8) & 0xffff] = acc;
                    acc = 0.f;
                }
            }
        }
        __syncwarp();
        // H = S_1 - m m^T / S_00 (the border of phi_0 = 1 removed) and the
        // upper triangle of X mirrored from the lower.
        const float i00 = 1.f / smu[0];
        for (int p = lane; p < NP1 * (NP1 + 1) / 2; p += 32) {
            const int pij = s_pij[p], i = pij & 255, j = pij >> 8;
            L[i * LDH + j] -= smu[i + 1] * smu[j + 1] * i00;
        }
        for (int p = lane; p < NP * (NP + 1) / 2; p += 32) {
            const int pij = s_pij35[p], i = pij & 255, j = pij >> 8;
            Y[j * LDF + i] = Y[i * LDF + j];
        }
        __syncwarp();
        // Cholesky of S = E[phi phi^T] by bordering: phi_0 = 1 gives
        // chol(S) = [[sqrt S00, 0], [m / sqrt S00, chol(S_1 - m m^T / S00)]].
        if (!(smu[0] > 0.f) || !reg_cholesky34_store(L, lane, al)) {  // al: free until Lanczos
            if (lane == 0) A.speed[cell] = bound;
            continue;
        }
        // Column 0 of chol(S) and the inverse pivots, once.
        const float l00 = sqrtf(smu[0]);
        for (int i = lane; i < NP; i += 32) {
            sl0[i] = i == 0 ? l00 : smu[i] / l00;
            sinv[i] = 1.f / (i == 0 ? l00 : L[(i - 1) * LDH + (i - 1)]);
        }
        __syncwarp();
        // Right-looking column solves: Y <- Ls^{-1} Y, then C = Ls^{-1} Y^T
        // (C overwrites Y after an in-place transpose by pairwise swaps).
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1) {
                for (int p = lane; p < NP * (NP + 1) / 2; p += 32) {
                    const int pij = s_pij35[p], i = pij & 255, j = pij >> 8;
                    if (j < i) {
                        const float t = Y[i * LDF + j];
                        Y[i * LDF + j] = Y[j * LDF + i];
                        Y[j * LDF + i] = t;
                    }
                }
                __syncwarp();
            }
            for (int j = lane; j < NP; j += 32) {
                // k = 0: the bordered column
                const float y0 = Y[j] * sinv[0];
                Y[j] = y0;
                for (int i = 1; i < NP; ++i) Y[i * LDF + j] -= sl0[i] * y0;
                for (int k = 1; k < NP; ++k) {
                    const float yk = Y[k * LDF + j] * sinv[k];
                    Y[k * LDF + j] = yk;
                    const float *Lk = L + (k - 1);
                    for (int i = k + 1; i < NP; ++i) Y[i * LDF + j] -= Lk[(i - 1) * LDH] * yk;
                }
            }
            __syncwarp();
        }
        float *Cm = Y;
        for (int p = lane; p < NP * (NP + 1) / 2; p += 32) {
            const int pij = s_pij35[p], i = pij & 255, j = pij >> 8;
            if (j < i) {
                const float s = 0.5f * (Cm[i * LDF + j] + Cm[j * LDF + i]);
                Cm[i * LDF + j] = s;
                Cm[j * LDF + i] = s;
            }
        }
        __syncwarp();
        // ---- Lanczos on the (symmetrised) C; columns are read, conflict-free
        float cn = 0.f;
        for (int p = lane; p < NP * NP; p += 32) cn = fmaxf(cn, fabsf(Cm[(p / NP) * LDF + p % NP]));
        const float cnorm = warp_max(cn) + 1e-30f;
        const float inv35 = rsqrtf((float)NP);
        float v0 = lane < NP ? inv35 : 0.f, v1 = lane + 32 < NP ? inv35 : 0.f;  // v_k
        float p0 = 0.f, p1 = 0.f, bprev = 0.f;                                 // v_{k-1}
        int m = 0;
        for (int k = 0; k < NP; ++k) {
            sv[lane] = v0;
            if (lane + 32 < NP) sv[lane + 32] = v1;
            __syncwarp();
            float w0 = 0.f, w1 = 0.f;
            {
                float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    a0 += Cm[j * LDF + lane] * sv[j];
                    a1 += Cm[(j + 1) * LDF + lane] * sv[j + 1];
                    a2 += Cm[(j + 2) * LDF + lane] * sv[j + 2];
                    a3 += Cm[(j + 3) * LDF + lane] * sv[j + 3];
                }
                for (int j = 32; j < NP; ++j) a0 += Cm[j * LDF + lane] * sv[j];
                w0 = (a0 + a1) + (a2 + a3);
            }
            if (lane + 32 < NP) {
                const int i = lane + 32;
                for (int j = 0; j < NP; ++j) w1 += Cm[j * LDF + i] * sv[j];
            }
            __syncwarp();
            w0 -= bprev * p0;
            w1 -= bprev * p1;
            const float a = warp_sum(w0 * v0 + w1 * v1);
            w0 -= a * v0;
            w1 -= a * v1;
            if (lane == 0) al[k] = a;
            const float bk = sqrtf(warp_sum(w0 * w0 + w1 * w1));
            m = k + 1;
            if (k + 1 == NP || bk <= 1e-6f * cnorm) break;
            if (lane == 0) bt[k] = bk;
            p0 = v0; p1 = v1;
            v0 = w0 / bk; v1 = w1 / bk;
            bprev = bk;
        }
        __syncwarp();
        const float mu_hi = warp_tridiag_extreme(al, bt, m, true, lane);
        const float mu_lo = warp_tridiag_extreme(al, bt, m, false, lane);
        if (lane == 0) A.speed[cell] = clamp_speed(fmaxf(fabsf(wx + sx * mu_hi), fabsf(wx + sx * mu_lo)), bound);
        __syncwarp();
    }
}

template <int N, bool AXI, bool MU_IN = false>
int launch_flux(mem_ctx *ctx, const FluxArgs &a, cudaStream_t st) {
    using Cf = FluxCfg<N, AXI, MU_IN>;
    // per-warp areas and the Cholesky broadcast column (al = W + 260) are 16-byte aligned
    static_assert((N * MEM_HE_STRIDE + 16 + 224 + 56 + 596 + 632) % 4 == 0 && Cf::WARP_FLOATS % 4 == 0, "alignment");
    const size_t smem = sizeof(float) * (N * MEM_HE_STRIDE + 16 + 224 + 56 + 596 + 632) + sizeof(float) * FWARPS * Cf::WARP_FLOATS;
    static int configured = 0;
    if (!configured) {
        MEM_CUDA_TRY(cudaFuncSetAttribute(k_fused_flux<N, AXI, MU_IN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = 1;
    }
    int sms = 0, per_sm = 0;
    MEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    MEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_flux<N, AXI, MU_IN>, FWARPS * 32, smem));
    if (per_sm < 1) return MEM_ECUDA;
    const int64_t want = (a.B + FWARPS - 1) / FWARPS;
    const int grid = (int)std::min<int64_t>(want, (int64_t)sms * per_sm);
    k_fused_flux<N, AXI, MU_IN><<<grid, FWARPS * 32, smem, st>>>(a);
    MEM_CUDA_TRY(cudaGetLastError());
    return MEM_OK;
}

}  // namespace

namespace mem_host {

bool flux_fused_available(const mem_ctx *ctx) { return ctx->n1d == 8 || ctx->n1d == 12; }

int flux_fused(mem_ctx *ctx, const float *M, const float *beta, const float *g, float *F, float *speed, int64_t B,
               cudaStream_t st, bool axisym) {
    FluxArgs a;
    a.M = M; a.beta = beta; a.gauge = g; a.F = F; a.speed = speed; a.B = B;
    a.he1d = ctx->d_he1d; a.logw1d = ctx->d_logw1d; a.slots = ctx->d_flux_slots; a.n_slots = ctx->n_flux_slots;
    a.aslots = ctx->d_axi_slots; a.n_aslots = ctx->n_axi_slots;
    a.xmax = ctx->xmax;
    a.mu = nullptr;
    switch (ctx->n1d * 2 + (axisym ? 1 : 0)) {
        case 16: return launch_flux<8, false>(ctx, a, st);
        case 17: return launch_flux<8, true>(ctx, a, st);
        case 24: return launch_flux<12, false>(ctx, a, st);
        case 25: return launch_flux<12, true>(ctx, a, st);
        default: return MEM_EINVAL;
    }
}

}  // namespace mem_host

namespace mem_host {

// Flux and speed from precomputed moment rows (velocity-space contexts).
int flux_from_mu(mem_ctx *ctx, const float *mu, const float *M, const float *g, float *F, float *speed, int64_t B,
                 cudaStream_t st, bool axisym) {
    if (B == 0) return MEM_OK;
    FluxArgs a;
    a.M = M; a.beta = nullptr; a.gauge = g; a.F = F; a.speed = speed; a.B = B;
    a.he1d = nullptr; a.logw1d = nullptr;
    a.slots = ctx->d_flux_slots; a.n_slots = ctx->n_flux_slots;
    a.aslots = ctx->d_axi_slots; a.n_aslots = ctx->n_axi_slots;
    a.xmax = 0.f;
    a.mu = mu;
    return axisym ? launch_flux<8, true, true>(ctx, a, st) : launch_flux<8, false, true>(ctx, a, st);
}

}  // namespace mem_host

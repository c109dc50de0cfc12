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

template <int N>
struct FluxCfg {
    using C = FusedCfg<N>;
    static constexpr int S1 = 10 * C::P;  // stage x, a <= 9
    static constexpr int T2 = 55 * N;     // stage y, a + b <= 9
    static constexpr int MAT = 3 * NP * LDF;
    static constexpr int WORK = (S1 + T2) > MAT ? (S1 + T2) : MAT;
    static constexpr int WARP_FLOATS = 36 + 224 + 2 * 36 + 36 + WORK;  // beta, mu, alpha/beta, v, work
};

struct FluxArgs {
    const float *M, *beta, *gauge;
    float *F, *speed;
    int64_t B;
    const float *he1d, *logw1d;
    const int2 *slots;
    int n_slots;
    float xmax;
};

template <int N>
__global__ void __launch_bounds__(FWARPS * 32) k_fused_flux(FluxArgs A) {
    using C = FusedCfg<N>;
    using Cf = FluxCfg<N>;
    extern __shared__ float smem[];
    float *s_he = smem;
    float *s_lw = s_he + N * MEM_HE_STRIDE;
    int *s_abc = (int *)(s_lw + 16);  // [220] packed (a, b, c)
    int *s_ab = s_abc + 224;          // [55]  packed (a, b)
    float *wbase = (float *)(s_ab + 56);
    for (int t = threadIdx.x; t < N * MEM_HE_STRIDE; t += blockDim.x) s_he[t] = A.he1d[t];
    for (int t = threadIdx.x; t < N; t += blockDim.x) s_lw[t] = A.logw1d[t];
    for (int t = threadIdx.x; t < 220; t += blockDim.x) s_abc[t] = exp_a(t) | (exp_b(t) << 8) | (exp_c(t) << 16);
    for (int t = threadIdx.x; t < 55; t += blockDim.x) {
        int d = 0;
        while ((d + 1) * (d + 2) / 2 <= t) ++d;
        const int b = t - d * (d + 1) / 2;
        s_ab[t] = (d - b) | (b << 8);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *W = wbase + warp * Cf::WARP_FLOATS;
    float *sb = W, *smu = W + 36, *al = smu + 224, *bt = al + 36, *sv = bt + 36, *work = sv + 36;
    float *S1 = work, *T2 = work + Cf::S1;
    float *L = work, *Y = work + NP * LDF, *Cm = work + 2 * NP * LDF;  // alias the stage buffers

    const int64_t nwarps = (int64_t)gridDim.x * FWARPS;
    for (int64_t cell = (int64_t)blockIdx.x * FWARPS + warp; cell < A.B; cell += nwarps) {
        const float n = A.M[cell * NP];
        const float wx = A.gauge[cell * 6], sx = A.gauge[cell * 6 + 3];
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
        // ---- E[phi phi^T] (lower, into L) and E[ubar_x phi phi^T] (full, into Y)
        {
            float acc = 0.f;
#pragma unroll 4
            for (int t = 0; t < A.n_slots; ++t) {
                const int2 sl = __ldg(&A.slots[t * 32 + lane]);
                acc = fmaf(__int_as_float(sl.y), smu[sl.x & 255], acc);
                if (sl.x < 0) {
                    const int p = (sl.x >> 8) & 2047;
                    const int q = p < 630 ? p : p - 630;
                    int i = (int)((sqrtf(8.f * q + 1.f) - 1.f) * 0.5f);
                    while (i * (i + 1) / 2 > q) --i;
                    while ((i + 1) * (i + 2) / 2 <= q) ++i;
                    const int j = q - i * (i + 1) / 2;
                    if (p < 630) {
                        L[i * LDF + j] = acc;
                    } else {
                        Y[i * LDF + j] = acc;
                        Y[j * LDF + i] = acc;
                    }
                    acc = 0.f;
                }
            }
        }
        __syncwarp();
        if (!warp_cholesky(L, NP, LDF, lane)) {
            if (lane == 0) A.speed[cell] = fmaxf(fabsf(wx + sx * A.xmax), fabsf(wx - sx * A.xmax));
            continue;
        }
        // Y <- L^{-1} Y (columns), then C = L^{-1} Y^T (columns of Y^T = rows of Y)
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
                for (int k = 0; k < i; ++k) s -= L[i * LDF + k] * Cm[k * LDF + j];
                Cm[i * LDF + j] = s / L[i * LDF + i];
            }
        __syncwarp();
        for (int p = lane; p < NP * NP; p += 32) {
            const int i = p / NP, j = p % NP;
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
            for (int j = 0; j < NP; ++j) w0 += Cm[j * LDF + lane] * sv[j];
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
        if (lane == 0) A.speed[cell] = fmaxf(fabsf(wx + sx * mu_hi), fabsf(wx + sx * mu_lo));
        __syncwarp();
    }
}

template <int N>
int launch_flux(mem_ctx *ctx, const FluxArgs &a, cudaStream_t st) {
    using Cf = FluxCfg<N>;
    const size_t smem = sizeof(float) * (N * MEM_HE_STRIDE + 16 + 224 + 56) + sizeof(float) * FWARPS * Cf::WARP_FLOATS;
    static int configured = 0;
    if (!configured) {
        MEM_CUDA_TRY(cudaFuncSetAttribute(k_fused_flux<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = 1;
    }
    int sms = 0, per_sm = 0;
    MEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    MEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_flux<N>, FWARPS * 32, smem));
    if (per_sm < 1) return MEM_ECUDA;
    const int64_t want = (a.B + FWARPS - 1) / FWARPS;
    const int grid = (int)std::min<int64_t>(want, (int64_t)sms * per_sm);
    k_fused_flux<N><<<grid, FWARPS * 32, smem, st>>>(a);
    MEM_CUDA_TRY(cudaGetLastError());
    return MEM_OK;
}

}  // namespace

namespace mem_host {

bool flux_fused_available(const mem_ctx *ctx) { return ctx->n1d == 8 || ctx->n1d == 12; }

int flux_fused(mem_ctx *ctx, const float *M, const float *beta, const float *g, float *F, float *speed, int64_t B,
               cudaStream_t st) {
    FluxArgs a;
    a.M = M; a.beta = beta; a.gauge = g; a.F = F; a.speed = speed; a.B = B;
    a.he1d = ctx->d_he1d; a.logw1d = ctx->d_logw1d; a.slots = ctx->d_flux_slots; a.n_slots = ctx->n_flux_slots;
    a.xmax = ctx->xmax;
    switch (ctx->n1d) {
        case 8: return launch_flux<8>(ctx, a, st);
        case 12: return launch_flux<12>(ctx, a, st);
        default: return MEM_EINVAL;
    }
}

}  // namespace mem_host

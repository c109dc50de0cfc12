// fused.cu -- the tuned back-end of mem_solve: Algorithm 1 for one cell per
// warp, start to finish inside one kernel, FP32, no scratch memory.
//
// The quadrature nodes are a tensor grid (x_i, x_j, x_k) of the 1D
// Gauss-Hermite rule, fixed in the gauge frame, and every statistic is a
// product he_a(x) he_b(y) he_c(z).  Both contractions of the method therefore
// factor axis by axis:
//   exponent  e_q = log w_q + sum_{abc} beta_abc he_a(x) he_b(y) he_c(z)
//             = log w_q + sum_a he_a(x_i) u_a(j,k),
//             u_a(j,k) = sum_{b,c} beta_abc he_b(y_j) he_c(z_k);
//   moments   mu_abc = sum_q sigma_q he_a he_b he_c   (a+b+c <= 8)
//             s_a(j,k)   = sum_i sigma(i,j,k) he_a(x_i)       (stage x)
//             t_ab(k)    = sum_j s_a(j,k) he_b(y_j)           (stage y)
//             mu_abc     = sum_k t_ab(k) he_c(z_k)            (stage z).
// E[phi_i phi_j] follows exactly from the 165 moments mu of degree <= 8 by
// the linearisation he_a he_b = sum_k C(a,k) C(b,k) k! sqrt((a+b-2k)!/(a!b!))
// he_{a+b-2k}; the gradient is mu_i - M_i/n and the Hessian
// E[phi_i phi_j] - mu_i mu_j (Appendix C).  sigma never leaves registers.
//
// Lane l of the warp owns the node lines (j,k) = p with p = l + 32 r.
#include "common.cuh"
#include "ctx.h"
#include "linalg.cuh"
#include "sumfact.cuh"

#include <algorithm>

using namespace mem;

namespace {


struct FusedArgs {
    const float *M;
    float *beta;
    int32_t *status;
    int32_t *iters;
    int64_t B;
    const float *he1d;    // [N][16]
    const float *logw1d;  // [N]
    const int2 *rslots;   // Hessian linearisation terms in rounds of 32 entries
    const int *rounds;    // [n_rounds] terms per round
    const int *rent;      // [n_rounds][32] destination (i | j << 8) or -1
    int n_rounds;
    const unsigned char *active;  // optional per-cell mask: 0 = leave the cell untouched
    mem_solve_opts o;
};

// NW warps per block (the launch shape is chosen by the autotuner); the
// register budget per thread is the same for every NW.
template <int N, int NW>
__global__ void __launch_bounds__(NW * 32, (N <= 8 ? 16 : 8) / NW) k_fused_solve(FusedArgs A) {
    using C = FusedCfg<N>;
    extern __shared__ float smem[];
    float *s_he = smem;                        // [N][16]
    float *s_lw = s_he + N * MEM_HE_STRIDE;    // [N] (padded to 16)
    int *s_abc = (int *)(s_lw + 16);           // [165] packed (a, b, c)
    int *s_pij = s_abc + 168;                  // [595] packed (i, j) of Hessian entry p
    int *s_ab = s_pij + 596;                   // [45]  packed (a, b) of stage-y row
    float *wbase = (float *)(s_ab + 48);
    for (int t = threadIdx.x; t < N * MEM_HE_STRIDE; t += blockDim.x) s_he[t] = A.he1d[t];
    for (int t = threadIdx.x; t < N; t += blockDim.x) s_lw[t] = A.logw1d[t];
    for (int t = threadIdx.x; t < 165; t += blockDim.x) s_abc[t] = exp_a(t) | (exp_b(t) << 8) | (exp_c(t) << 16);
    for (int t = threadIdx.x; t < NP1 * (NP1 + 1) / 2; t += blockDim.x) {
        int i = 0;
        while ((i + 1) * (i + 2) / 2 <= t) ++i;
        s_pij[t] = i | ((t - i * (i + 1) / 2) << 8);
    }
    for (int t = threadIdx.x; t < 45; t += blockDim.x) {
        int d = 0;
        while ((d + 1) * (d + 2) / 2 <= t) ++d;
        const int b = t - d * (d + 1) / 2;
        s_ab[t] = (d - b) | (b << 8);
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *W = wbase + warp * C::WARP_FLOATS;
    float *sb = W, *sd = W + 36, *sm = W + 72, *sg = W + 108, *sbc = W + 144, *smu = W + 180;
    float *work = smu + 168;
    float *S1 = work, *T2 = work + C::S1, *H = work;  // H aliases the stage buffers
    const mem_solve_opts &o = A.o;

    const int64_t nwarps = (int64_t)gridDim.x * NW;
    for (int64_t cell = (int64_t)blockIdx.x * NW + warp; cell < A.B; cell += nwarps) {
        if (A.active && !A.active[cell]) continue;
        const float *Mc = A.M + cell * NP;
        float *bc = A.beta + cell * NP;
        // ---- load and validate
        float mval = lane < NP ? Mc[lane] : 0.f, m2 = lane + 32 < NP ? Mc[lane + 32] : 0.f;
        float bval = lane < NP ? bc[lane] : 0.f, b2 = lane + 32 < NP ? bc[lane + 32] : 0.f;
        const float n = __shfl_sync(0xffffffffu, mval, 0);
        bool bad = !isfinite(mval) || !isfinite(m2) || (lane > 0 && !isfinite(bval)) || !isfinite(b2);
        bad = __any_sync(0xffffffffu, bad) || !(n > 0.f) || !isfinite(n);
        if (bad) {
            if (lane == 0) {
                if (A.status) A.status[cell] = MEM_ST_BADINPUT;
                if (A.iters) A.iters[cell] = 0;
            }
            continue;
        }
        if (lane < NP) { sm[lane] = lane ? mval / n : 0.f; sb[lane] = lane ? bval : 0.f; sd[lane] = 0.f; sg[lane] = 0.f; }
        if (lane + 32 < NP) { sm[lane + 32] = m2 / n; sb[lane + 32] = b2; sd[lane + 32] = 0.f; sg[lane + 32] = 0.f; }
        __syncwarp();

        auto dot_m = [&](const float *v) {  // sum_{k>=1} v_k M_k / n
            float p = (lane >= 1 && lane < NP ? v[lane] * sm[lane] : 0.f) + (lane + 32 < NP ? v[lane + 32] * sm[lane + 32] : 0.f);
            return warp_sum(p);
        };
        float Lcur = 0.f;
        int st = 0, it = 0;
        float alpha = 1.f;
        bool done = false;
        while (!done) {
            // The exponent arrays live only until stage x: they are recomputed
            // from beta (and dbeta) at the start of every pass.
            float eb[C::NODES];
            exponent<N>(sb, s_he, s_lw, lane, true, eb);
            float mx, Z;
            if (it == 0) {
                // BackTrackingLineSearch with dbeta = 0: alpha = 1 is accepted.
                float m = -INFINITY;
#pragma unroll
                for (int q = 0; q < C::NODES; ++q) m = fmaxf(m, eb[q]);
                mx = warp_max(m);
                float z = 0.f;
#pragma unroll
                for (int q = 0; q < C::NODES; ++q) z += __expf(eb[q] - mx);
                Z = warp_sum(z);
                Lcur = mx + __logf(Z) - dot_m(sb);
            } else {
                // ---- BackTrackingLineSearch / ArmijoCondition (Algorithm 1):
                // trial exponents are e_beta + alpha e_dbeta.
                float ed[C::NODES];
                exponent<N>(sd, s_he, s_lw, lane, false, ed);
                float gp = (lane >= 1 && lane < NP ? sg[lane] * sd[lane] : 0.f) + (lane + 32 < NP ? sg[lane + 32] * sd[lane + 32] : 0.f);
                const float gd = warp_sum(gp), mb = dot_m(sb), md = dot_m(sd);
                alpha = 2.f;
                bool sat = false;
                float Lt = Lcur;
                mx = 0.f;
                Z = 1.f;
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
                    Lt = mx + __logf(Z) - (mb + alpha * md);
                    const float LD = Lcur - Lt, gradD = -o.c_armijo * alpha * gd;
                    sat = (LD - gradD) >= -(o.atol + o.rtol * fabsf(LD));
                }
                // accepted (or last) trial: beta += alpha dbeta; its exponents
                // give sigma for this pass
#pragma unroll
                for (int q = 0; q < C::NODES; ++q) eb[q] = fmaf(alpha, ed[q], eb[q]);
                Lcur = Lt;
                if (lane >= 1 && lane < NP) sb[lane] += alpha * sd[lane];
                if (lane + 32 < NP) sb[lane + 32] += alpha * sd[lane + 32];
                __syncwarp();
            }
            // ---- sigma and stage x: s_a(p) = sum_i sigma(i,p) he_a(x_i), a <= 8
            {
                const float invZ = 1.f / Z;
                float sa[C::R][9];
#pragma unroll
                for (int r = 0; r < C::R; ++r)
#pragma unroll
                    for (int a = 0; a < 9; ++a) sa[r][a] = 0.f;
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    float hx[9];
#pragma unroll
                    for (int a = 0; a < 9; ++a) hx[a] = s_he[i * MEM_HE_STRIDE + a];
#pragma unroll
                    for (int r = 0; r < C::R; ++r) {
                        const float sg_ = __expf(eb[r * N + i] - mx) * invZ;
#pragma unroll
                        for (int a = 0; a < 9; ++a) sa[r][a] += sg_ * hx[a];
                    }
                }
#pragma unroll
                for (int r = 0; r < C::R; ++r) {
                    const int p = lane + 32 * r;
                    if (p < C::P) {
#pragma unroll
                        for (int a = 0; a < 9; ++a) S1[a * C::P + p] = sa[r][a];
                    }
                }
            }
            __syncwarp();
            // ---- stage y: t_ab(k) = sum_j s_a(j,k) he_b(y_j), a + b <= 8
            for (int t = lane; t < C::T2; t += 32) {
                const int ab = t / N, k = t % N;
                const int abp = s_ab[ab], a = abp & 255, b = abp >> 8;
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < N; ++j) acc += S1[a * C::P + j * N + k] * s_he[j * MEM_HE_STRIDE + b];
                T2[ab * N + k] = acc;
            }
            __syncwarp();
            // ---- stage z: mu_abc = sum_k t_ab(k) he_c(z_k)
            for (int t = lane; t < 165; t += 32) {
                const int abc = s_abc[t], a = abc & 255, b = (abc >> 8) & 255, c = abc >> 16;
                const int ab = (a + b) * (a + b + 1) / 2 + b;
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < N; ++k) acc += T2[ab * N + k] * s_he[k * MEM_HE_STRIDE + c];
                smu[t] = acc;
            }
            __syncwarp();
            // ---- gradient and Hessian (Appendix C)
            if (lane >= 1 && lane < NP) sg[lane] = smu[lane] - sm[lane];
            if (lane + 32 < NP) sg[lane + 32] = smu[lane + 32] - sm[lane + 32];
            __syncwarp();
            // Hessian entries E[phi_i phi_j] - mu_i mu_j (packed lower, i >= j)
            // from the linearisation terms, in rounds of 32 entries (one per
            // lane, similar term counts): a branch-free term loop, whose loads
            // can be issued ahead since nothing is stored in between, then one
            // store per lane.
            {
                const int2 *sl = A.rslots;
                for (int r = 0; r < A.n_rounds; ++r) {
                    const int T = __ldg(&A.rounds[r]);
                    float a0 = 0.f, a1 = 0.f;
                    int t = 0;
                    for (; t + 1 < T; t += 2) {
                        const int2 s0 = __ldg(&sl[t * 32 + lane]), s1 = __ldg(&sl[(t + 1) * 32 + lane]);
                        a0 = fmaf(__int_as_float(s0.y), smu[s0.x], a0);
                        a1 = fmaf(__int_as_float(s1.y), smu[s1.x], a1);
                    }
                    if (t < T) {
                        const int2 s0 = __ldg(&sl[t * 32 + lane]);
                        a0 = fmaf(__int_as_float(s0.y), smu[s0.x], a0);
                    }
                    sl += T * 32;
                    const int e = __ldg(&A.rent[r * 32 + lane]);
                    if (e >= 0) {
                        const int i = e & 255, j = e >> 8;
                        H[i * LDH + j] = (a0 + a1) - smu[i + 1] * smu[j + 1];
                    }
                }
            }
            __syncwarp();
            // Cholesky of H, then of H + lambda I with lambda = lambda0 * mul^t
            // until it succeeds; the Newton direction solves H dbeta = -grad.
            const float g_l = lane < 32 ? sg[lane + 1] : 0.f, g32 = sg[33], g33 = sg[34];
            float x = 0.f, x32 = 0.f, x33 = 0.f;
            bool ok = false;
            float lam = 0.f;
            for (int t = 0; t <= o.max_lambda; ++t) {
                ok = reg_chol_solve34<true>(H, lam, lane, -g_l, -g32, -g33, x, x32, x33, sbc);
                if (ok) break;
                st |= MEM_ST_LAMBDA;
                lam = (t == 0) ? o.lambda0 : lam * o.lambda_mul;
            }
            ++it;
            if (!ok) {
                st |= MEM_ST_LAMBDA_CAP | MEM_ST_NONFINITE;
                break;
            }
            const float res = 0.5f * fabsf(warp_sum(x * g_l) + x32 * g32 + x33 * g33);
            sd[lane + 1] = x;
            if (lane == 0) { sd[33] = x32; sd[34] = x33; }
            __syncwarp();
            if (!isfinite(res)) { st |= MEM_ST_NONFINITE; break; }
            const bool conv_res = res <= o.tol, conv_a = alpha <= o.alpha_min;
            if (conv_res) st |= MEM_ST_CONVERGED;
            if (conv_a) st |= MEM_ST_STAGNATED;
            if (conv_res || conv_a) {
                if (conv_res && o.final_step) {
                    if (lane >= 1 && lane < NP) sb[lane] += sd[lane];
                    if (lane + 32 < NP) sb[lane + 32] += sd[lane + 32];
                    __syncwarp();
                }
                done = true;
            } else if (it > o.maxI) {
                st |= MEM_ST_MAXITER;
                done = true;
            }
        }
        __syncwarp();
        if (lane < NP) bc[lane] = lane ? sb[lane] : n;
        if (lane + 32 < NP) bc[lane + 32] = sb[lane + 32];
        if (lane == 0) {
            if (A.status) A.status[cell] = st;
            if (A.iters) A.iters[cell] = it;
        }
        __syncwarp();
    }
}

template <int N, int W>
int launch_fused(mem_ctx *ctx, const FusedArgs &a, cudaStream_t st, int bps_cap) {
    using C = FusedCfg<N>;
    // the per-warp areas (and the broadcast column at W + 144) are 16-byte aligned
    static_assert((N * MEM_HE_STRIDE + 16 + 168 + 596 + 48) % 4 == 0 && C::WARP_FLOATS % 4 == 0, "alignment");
    const size_t smem = sizeof(float) * (N * MEM_HE_STRIDE + 16 + 168 + 596 + 48) + sizeof(float) * W * C::WARP_FLOATS;
    static int configured = 0;
    if (!configured) {
        MEM_CUDA_TRY(cudaFuncSetAttribute(k_fused_solve<N, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = 1;
    }
    int sms = 0, per_sm = 0;
    MEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    MEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_solve<N, W>, W * 32, smem));
    if (per_sm < 1) return MEM_ECUDA;
    if (bps_cap > 0) per_sm = std::min(per_sm, bps_cap);
    const int64_t want = (a.B + W - 1) / W;
    const int grid = (int)std::min<int64_t>(want, (int64_t)sms * per_sm);
    k_fused_solve<N, W><<<grid, W * 32, smem, st>>>(a);
    MEM_CUDA_TRY(cudaGetLastError());
    return MEM_OK;
}

template <int N>
int launch_fused_cfg(mem_ctx *ctx, const FusedArgs &a, cudaStream_t st, const mem_launch_cfg &c) {
    switch (c.warps) {
        case 2: return launch_fused<N, 2>(ctx, a, st, c.blocks_per_sm);
        case 8: return launch_fused<N, 8>(ctx, a, st, c.blocks_per_sm);
        default: return launch_fused<N, 4>(ctx, a, st, c.blocks_per_sm);
    }
}

template <int N>
int occupancy_fused(int W, int *per_sm) {
    using C = FusedCfg<N>;
    const size_t smem = sizeof(float) * (N * MEM_HE_STRIDE + 16 + 168 + 596 + 48) + sizeof(float) * W * C::WARP_FLOATS;
    cudaError_t e;
    switch (W) {
        case 2:
            cudaFuncSetAttribute(k_fused_solve<N, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_fused_solve<N, 2>, 64, smem);
            break;
        case 8:
            cudaFuncSetAttribute(k_fused_solve<N, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_fused_solve<N, 8>, 256, smem);
            break;
        default:
            cudaFuncSetAttribute(k_fused_solve<N, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_fused_solve<N, 4>, 128, smem);
    }
    return e == cudaSuccess ? MEM_OK : MEM_ECUDA;
}

}  // namespace

namespace mem_host {

int solve_fused(mem_ctx *ctx, const float *M, float *beta, int32_t *status, int32_t *iters, int64_t B,
                const mem_solve_opts &o, cudaStream_t st, const unsigned char *active) {
    FusedArgs a;
    a.active = active;
    a.M = M; a.beta = beta; a.status = status; a.iters = iters; a.B = B;
    a.he1d = ctx->d_he1d; a.logw1d = ctx->d_logw1d; a.rslots = ctx->d_hr_slots; a.rounds = ctx->d_hr_rounds;
    a.rent = ctx->d_hr_ent; a.n_rounds = ctx->n_hess_rounds;
    a.o = o;
    switch (ctx->n1d) {
        case 8: return launch_fused_cfg<8>(ctx, a, st, ctx->cfg_fused);
        case 12: return launch_fused_cfg<12>(ctx, a, st, ctx->cfg_fused);
        default: return active ? MEM_EINVAL : solve_plain(ctx, M, beta, status, iters, B, o, st);
    }
}

// Blocks per SM that the fused solve can keep resident with W warps per block.
int fused_occupancy(mem_ctx *ctx, int W, int *per_sm) {
    switch (ctx->n1d) {
        case 8: return occupancy_fused<8>(W, per_sm);
        case 12: return occupancy_fused<12>(W, per_sm);
        default: return MEM_EINVAL;
    }
}

}  // namespace mem_host

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

using namespace mem;

namespace {

constexpr int WARPS = 4;
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

struct FusedArgs {
    const float *M;
    float *beta;
    int32_t *status;
    int32_t *iters;
    int64_t B;
    const float *he1d;    // [N][16]
    const float *logw1d;  // [N]
    const int *lin_off;   // [596]
    const int2 *lin_terms;
    mem_solve_opts o;
};

// Exponent contribution of a parameter vector v (slots 1..34) on the lane's
// nodes: out[r*N + i] = sum_a he_a(x_i) u_a(line r).  add_logw adds log w_q.
template <int N>
__device__ __forceinline__ void exponent(const float *v, const float *he, const float *lw, int lane, bool add_logw,
                                         float (&out)[FusedCfg<N>::NODES]) {
    using C = FusedCfg<N>;
#pragma unroll
    for (int r = 0; r < C::R; ++r) {
        const int p = lane + 32 * r;
        const bool live = p < C::P;
        const int j = live ? p / N : 0, k = live ? p % N : 0;
        const float *hy = he + j * MEM_HE_STRIDE, *hz = he + k * MEM_HE_STRIDE;
        float u[5];
#pragma unroll
        for (int a = 0; a <= 4; ++a) {
            float acc = 0.f;
#pragma unroll
            for (int b = 0; a + b <= 4; ++b) {
                float inner = 0.f;
#pragma unroll
                for (int c = 0; a + b + c <= 4; ++c)
                    if (a + b + c > 0) inner += v[idx3(a, b, c)] * hz[c];
                acc += inner * hy[b];
            }
            u[a] = acc;
        }
        const float lwjk = add_logw ? lw[j] + lw[k] : 0.f;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const float *hx = he + i * MEM_HE_STRIDE;
            float e = lwjk + (add_logw ? lw[i] : 0.f);
#pragma unroll
            for (int a = 0; a <= 4; ++a) e += u[a] * hx[a];
            out[r * N + i] = live ? e : (add_logw ? -INFINITY : 0.f);
        }
    }
}

template <int N>
__global__ void __launch_bounds__(WARPS * 32) k_fused_solve(FusedArgs A) {
    using C = FusedCfg<N>;
    extern __shared__ float smem[];
    float *s_he = smem;                        // [N][16]
    float *s_lw = s_he + N * MEM_HE_STRIDE;    // [N] (padded to 16)
    int *s_abc = (int *)(s_lw + 16);           // [165] packed (a, b, c)
    float *wbase = (float *)(s_abc + 168);
    for (int t = threadIdx.x; t < N * MEM_HE_STRIDE; t += blockDim.x) s_he[t] = A.he1d[t];
    for (int t = threadIdx.x; t < N; t += blockDim.x) s_lw[t] = A.logw1d[t];
    for (int t = threadIdx.x; t < 165; t += blockDim.x) s_abc[t] = exp_a(t) | (exp_b(t) << 8) | (exp_c(t) << 16);
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *W = wbase + warp * C::WARP_FLOATS;
    float *sb = W, *sd = W + 36, *sm = W + 72, *sg = W + 108, *srhs = W + 144, *smu = W + 180;
    float *work = smu + 168;
    float *S1 = work, *T2 = work + C::S1, *H = work;  // H aliases the stage buffers
    const mem_solve_opts &o = A.o;

    const int64_t nwarps = (int64_t)gridDim.x * WARPS;
    for (int64_t cell = (int64_t)blockIdx.x * WARPS + warp; cell < A.B; cell += nwarps) {
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

        float eb[C::NODES];
        exponent<N>(sb, s_he, s_lw, lane, true, eb);
        auto lse = [&](const float (&e)[C::NODES], float &mx) {
            float m = -INFINITY;
#pragma unroll
            for (int q = 0; q < C::NODES; ++q) m = fmaxf(m, e[q]);
            mx = warp_max(m);
            float z = 0.f;
#pragma unroll
            for (int q = 0; q < C::NODES; ++q) z += __expf(e[q] - mx);
            return warp_sum(z);
        };
        auto dot_m = [&](const float *v) {  // sum_{k>=1} v_k M_k / n
            float p = (lane >= 1 && lane < NP ? v[lane] * sm[lane] : 0.f) + (lane + 32 < NP ? v[lane + 32] * sm[lane + 32] : 0.f);
            return warp_sum(p);
        };
        float mx, Z = lse(eb, mx);
        float Lcur = mx + __logf(Z) - dot_m(sb);
        int st = 0, it = 0;
        float alpha = 1.f;
        bool done = false;
        while (!done) {
            // ---- BackTrackingLineSearch (no-op on the first pass: dbeta = 0)
            if (it > 0) {
                float ed[C::NODES];
                exponent<N>(sd, s_he, s_lw, lane, false, ed);
                float gp = (lane >= 1 && lane < NP ? sg[lane] * sd[lane] : 0.f) + (lane + 32 < NP ? sg[lane + 32] * sd[lane + 32] : 0.f);
                const float gd = warp_sum(gp), mb = dot_m(sb), md = dot_m(sd);
                alpha = 2.f;
                bool sat = false;
                for (int s = 0; !sat && s <= o.maxT; ++s) {
                    alpha *= 0.5f;
                    float m = -INFINITY;
#pragma unroll
                    for (int q = 0; q < C::NODES; ++q) m = fmaxf(m, eb[q] + alpha * ed[q]);
                    m = warp_max(m);
                    float z = 0.f;
#pragma unroll
                    for (int q = 0; q < C::NODES; ++q) z += __expf(eb[q] + alpha * ed[q] - m);
                    z = warp_sum(z);
                    const float Lt = m + __logf(z) - (mb + alpha * md);
                    const float LD = Lcur - Lt, gradD = -o.c_armijo * alpha * gd;
                    sat = (LD - gradD) >= -(o.atol + o.rtol * fabsf(LD));
                }
                if (lane >= 1 && lane < NP) sb[lane] += alpha * sd[lane];
                if (lane + 32 < NP) sb[lane + 32] += alpha * sd[lane + 32];
                __syncwarp();
                exponent<N>(sb, s_he, s_lw, lane, true, eb);
                Z = lse(eb, mx);
                Lcur = mx + __logf(Z) - dot_m(sb);
            }
            // ---- sigma and stage x: s_a(p) = sum_i sigma(i,p) he_a(x_i), a <= 8
            const float invZ = 1.f / Z;
#pragma unroll
            for (int r = 0; r < C::R; ++r) {
                const int p = lane + 32 * r;
                float sa[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    const float sg_ = __expf(eb[r * N + i] - mx) * invZ;
                    const float *hx = s_he + i * MEM_HE_STRIDE;
#pragma unroll
                    for (int a = 0; a < 9; ++a) sa[a] += sg_ * hx[a];
                }
                if (p < C::P) {
#pragma unroll
                    for (int a = 0; a < 9; ++a) S1[a * C::P + p] = sa[a];
                }
            }
            __syncwarp();
            // ---- stage y: t_ab(k) = sum_j s_a(j,k) he_b(y_j), a + b <= 8
            for (int t = lane; t < C::T2; t += 32) {
                const int ab = t / N, k = t % N;
                int d = 0;
                while ((d + 1) * (d + 2) / 2 <= ab) ++d;
                const int b = ab - d * (d + 1) / 2, a = d - b;
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
            auto build_H = [&](float lam) {
                for (int p = lane; p < NP1 * (NP1 + 1) / 2; p += 32) {
                    int i = (int)((sqrtf(8.f * p + 1.f) - 1.f) * 0.5f);
                    while (i * (i + 1) / 2 > p) --i;
                    while ((i + 1) * (i + 2) / 2 <= p) ++i;
                    const int j = p - i * (i + 1) / 2;
                    float acc = 0.f;
                    const int t1 = A.lin_off[p + 1];
                    for (int t = A.lin_off[p]; t < t1; ++t) {
                        const int2 tm = __ldg(&A.lin_terms[t]);
                        acc += __int_as_float(tm.y) * smu[tm.x];
                    }
                    acc -= smu[i + 1] * smu[j + 1];
                    if (i == j) acc += lam;
                    H[i * LDH + j] = acc;
                }
                __syncwarp();
            };
            build_H(0.f);
            bool ok = warp_cholesky(H, NP1, LDH, lane);
            float lam = o.lambda0;
            for (int t = 0; !ok && t < o.max_lambda; ++t) {
                st |= MEM_ST_LAMBDA;
                build_H(lam);
                ok = warp_cholesky(H, NP1, LDH, lane);
                lam *= o.lambda_mul;
            }
            ++it;
            if (!ok) {
                st |= MEM_ST_LAMBDA_CAP | MEM_ST_NONFINITE;
                break;
            }
            if (lane < NP1) srhs[lane] = -sg[lane + 1];
            if (lane + 32 < NP1) srhs[lane + 32] = -sg[lane + 33];
            warp_solve_lower(H, NP1, LDH, srhs, lane);
            warp_solve_upperT(H, NP1, LDH, srhs, lane);
            float part = (lane < NP1 ? srhs[lane] * sg[lane + 1] : 0.f) + (lane + 32 < NP1 ? srhs[lane + 32] * sg[lane + 33] : 0.f);
            const float res = 0.5f * fabsf(warp_sum(part));
            if (lane < NP1) sd[lane + 1] = srhs[lane];
            if (lane + 32 < NP1) sd[lane + 33] = srhs[lane + 32];
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

template <int N>
int launch_fused(mem_ctx *ctx, const FusedArgs &a, cudaStream_t st) {
    using C = FusedCfg<N>;
    const size_t smem = sizeof(float) * (N * MEM_HE_STRIDE + 16 + 168) + sizeof(float) * WARPS * C::WARP_FLOATS;
    static int configured = 0;
    if (!configured) {
        MEM_CUDA_TRY(cudaFuncSetAttribute(k_fused_solve<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = 1;
    }
    int sms = 0, per_sm = 0;
    MEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    MEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_solve<N>, WARPS * 32, smem));
    if (per_sm < 1) return MEM_ECUDA;
    const int64_t want = (a.B + WARPS - 1) / WARPS;
    const int grid = (int)std::min<int64_t>(want, (int64_t)sms * per_sm);
    k_fused_solve<N><<<grid, WARPS * 32, smem, st>>>(a);
    MEM_CUDA_TRY(cudaGetLastError());
    return MEM_OK;
}

}  // namespace

namespace mem_host {

int solve_fused(mem_ctx *ctx, const float *M, float *beta, int32_t *status, int32_t *iters, int64_t B,
                const mem_solve_opts &o, cudaStream_t st) {
    FusedArgs a;
    a.M = M; a.beta = beta; a.status = status; a.iters = iters; a.B = B;
    a.he1d = ctx->d_he1d; a.logw1d = ctx->d_logw1d; a.lin_off = ctx->d_lin_off; a.lin_terms = ctx->d_lin_terms;
    a.o = o;
    switch (ctx->n1d) {
        case 8: return launch_fused<8>(ctx, a, st);
        case 12: return launch_fused<12>(ctx, a, st);
        default: return solve_plain(ctx, M, beta, status, iters, B, o, st);
    }
}

}  // namespace mem_host

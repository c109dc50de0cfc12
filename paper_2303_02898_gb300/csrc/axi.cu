// axi.cu -- the paper's own system for axisymmetric flow (Appendix B, Eq.
// "Sufficient 35" and its orthonormal form) on the velocity-space rule: nine
// statistics psi_j of (u_x, u_r), Algorithm 1 over eight unknowns, the flux
// and the characteristic speed of the nine-moment system, one warp per cell.
//
// In the Hermite-product basis the nine statistics are orthonormal
// combinations psi_j = v_j . phi of the 35 (the axisymmetric subspace), and
// pointwise they are Hermite polynomials in ubar_x times Laguerre
// polynomials in s = ubar_r^2 / 2:
//   psi = 1, he1, he2, -L1, he3, he4, L2, -he1 L1, -he2 L1,
// orthonormal under the gauge's Gaussian exp(-ubar_x^2/2 - s).  For an
// axisymmetric cell the 35-statistic solve stays in that subspace (the
// gradient lies in it and the covariance maps it to itself), so this solve
// is the 35-statistic solve in exact arithmetic, with 8 unknowns instead of
// 34 and a 2D rule instead of the 3D one (every integrand depends on u_x and
// u_r only, so one azimuth integrates it exactly).
//
// Sum factorisation over the rule's product structure (x nodes i, radial
// nodes m; lane l owns the radial nodes m = l + 32 r):
//   exponent  e(i, m) = lw_x(i) + lw_r(m) + P0(m) + he1(x_i) P1(m)
//                      + he2(x_i) P2(m) + he3(x_i) a4 + he4(x_i) a5,
//             P0 = -a3 L1 + a6 L2, P1 = a1 - a7 L1, P2 = a2 - a8 L1;
//   x stage   T_c(m) = sum_i sigma(i, m) he_c(x_i), c <= 9 (in the sweep);
//   s stage   mu_ck = sum_m T_c(m) L_k(s_m), k <= 4 (50 moments).
// E[psi_p psi_q] and E[ubar_x psi_p psi_q] follow from mu through the
// Hermite and Laguerre linearisations (term lists built with the context),
// the gradient is E[psi] - M9 / n, the Hessian E[psi psi^T] - E[psi]E[psi]^T
// (Appendix C).  Node placement follows the 35-statistic kernel: u - w in
// FP64, ubar and ubar^2 / 2 in float-float, one rounding of the log weight.
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "ffloat.cuh"
#include "linalg.cuh"

using namespace mem;

namespace {

constexpr int NS = 9;  // statistics
constexpr int NMU = 50;  // mu_ck, c <= 9, k <= 4: index 5 c + k

// psi_j = sign_j he_{a_j} L_{m_j}; its 35-product coefficients v_j (up to
// three entries each)
__constant__ int c_pa[NS] = {0, 1, 2, 0, 3, 4, 0, 1, 2};
__constant__ int c_pm[NS] = {0, 0, 0, 1, 0, 0, 2, 1, 1};
__constant__ float c_psg[NS] = {1.f, 1.f, 1.f, -1.f, 1.f, 1.f, 1.f, -1.f, -1.f};
__constant__ int c_vk[NS][3];
__constant__ float c_vc[NS][3];
__constant__ int c_vn[NS];

struct AxiArgs {
    const float *M;
    float *beta;
    const float *gauge;
    int32_t *status, *iters;
    float *F, *speed, *cond;
    const int *pid;
    const float *dom;    // [domains][DOM_REC] domain records
    const unsigned char *active;
    const float2 *vt2;   // node offsets in block widths, float pairs
    const float *vtf;
    const int2 *terms;  // (mu index, coefficient bits)
    const int *toff;    // [91]: entries 0..44 E[psi_p psi_q], 45..89 E[ubar_x psi_p psi_q] (p >= q, packed)
    int64_t B;
    int nbx, nbr, K, nx, nr;
    int solve;
    mem_solve_opts o;
};

struct AxiLayout {
    int hx, lwx, Tt, Lt, mu, vec, H, HL, rhs, Sm, Xm, al, bt, sv, total;
};

__host__ __device__ inline AxiLayout axi_layout(int nx, int nrp) {
    AxiLayout L;
    int o = 0;
    L.hx = o; o += 12 * nx;  // per x node: he_0..he_9, log weight, pad (three 16-byte loads)
    L.lwx = L.hx;
    L.Tt = o; o += 10 * nrp;
    L.Lt = o; o += 5 * nrp;
    L.mu = o; o += 52;
    L.vec = o; o += 6 * 12;  // a | da | M9/n | grad | M35 staging (2 x 36 below)
    L.H = o; o += 64;
    L.HL = o; o += 64;
    L.rhs = o; o += 8;
    L.Sm = o; o += 144;
    L.Xm = o; o += 144;
    L.al = o; o += 16;
    L.bt = o; o += 16;
    L.sv = o; o += 32;
    o += 72;  // 35-vectors of the cell (M, beta)
    L.total = (o + 3) & ~3;
    return L;
}

// Coefficients of the exponent on the lane's radial nodes for the parameter
// vector a (uniform he3 / he4 coefficients a[4], a[5]).
template <int R>
__device__ __forceinline__ void axi_coeffs(const float *a, const float (&L1)[R], const float (&L2)[R],
                                           float (&c)[R][3]) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
        c[r][0] = fmaf(-a[3], L1[r], a[6] * L2[r]);
        c[r][1] = fmaf(-a[7], L1[r], a[1]);
        c[r][2] = fmaf(-a[8], L1[r], a[2]);
    }
}

// One evaluation of the partition function at coefficients (c, c3, c4):
// a sweep over the x nodes with a running per-lane maximum (warm-started at
// mx), the warp log-sum-exp, and the sigma-weighted x stage T_c(m), c <= 9,
// stored transposed for the s stage.  Returns log Z.
template <int R>
__device__ __forceinline__ float axi_sweep(const float (&c)[R][3], float c3, float c4, const float (&lwr)[R],
                                           const float *hx, const float *lwx, int nx, float *Tt, int nrp, int lane,
                                           float &mx) {
    float T[R][10], m, s, em;
    auto run = [&](float m0) {
        m = m0;
        s = 0.f;
        em = -INFINITY;
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int k = 0; k < 10; ++k) T[r][k] = 0.f;
        for (int i = 0; i < nx; ++i) {
            const float4 *hp = reinterpret_cast<const float4 *>(hx + 12 * i);
            const float4 q0 = hp[0], q1 = hp[1], q2 = hp[2];
            const float h[10] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y};
            const float lx = q2.z;
            const float cx = fmaf(h[3], c3, h[4] * c4);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float e = lx + lwr[r] + c[r][0] + fmaf(h[1], c[r][1], fmaf(h[2], c[r][2], cx));
                em = fmaxf(em, e);
                float w;
                if (e > m) {
                    const float sc = __expf(m - e);
                    s *= sc;
#pragma unroll
                    for (int rr = 0; rr < R; ++rr)
#pragma unroll
                        for (int k = 0; k < 10; ++k) T[rr][k] *= sc;
                    m = e;
                    w = 1.f;
                } else {
                    w = __expf(e - m);
                }
                s += w;
#pragma unroll
                for (int k = 0; k < 10; ++k) T[r][k] = fmaf(w, h[k], T[r][k]);
            }
        }
    };
    run(mx);
    // a maximum far below the warm start would underflow the top weights
    const float E = warp_max(em);
    if (E < mx - 40.f) run(E);
    mx = warp_max(m);
    const float Z = warp_sum(s * __expf(m - mx));
    const float f = __expf(m - mx) / Z;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int mm = lane + 32 * r;
#pragma unroll
        for (int k = 0; k < 10; ++k) Tt[k * nrp + mm] = T[r][k] * f;
    }
    return mx + __logf(Z);
}

// s stage: mu_ck = sum_m T_c(m) L_k(s_m); lane o < 50 (and o - 32 ... ) per output.
__device__ __forceinline__ void axi_s_stage(const float *Tt, const float *Lt, int nr, int nrp, float *mu, int lane) {
    __syncwarp();
    for (int o = lane; o < NMU; o += 32) {
        const float *t = Tt + (o / 5) * nrp, *l = Lt + (o % 5) * nrp;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        int m = 0;
        for (; m + 3 < nr; m += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fmaf(t[m + u], l[m + u], acc[u]);
        }
        for (; m < nr; ++m) acc[0] = fmaf(t[m], l[m], acc[0]);
        mu[o] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }
    __syncwarp();
}

// Entries e (packed lower, p >= q) of E[psi psi^T] (e < 45) and of
// E[ubar_x psi psi^T] (45 <= e < 90) from the term lists.
__device__ __forceinline__ float axi_entry(const AxiArgs &A, const float *mu, int e) {
    float acc = 0.f;
    for (int t = __ldg(&A.toff[e]); t < __ldg(&A.toff[e + 1]); ++t) {
        const int2 tm = __ldg(&A.terms[t]);
        acc = fmaf(__int_as_float(tm.y), mu[tm.x], acc);
    }
    return acc;
}

__device__ __forceinline__ void packed_pq(int e, int &p, int &q) {
    p = 0;
    while ((p + 1) * (p + 2) / 2 <= e) ++p;
    q = e - p * (p + 1) / 2;
}

// AW warps (cells) per block: the launch shape is chosen by the autotuner.
// With one radial node per lane (R = 1) the register budget is held to
// about 100 per thread (5 blocks of 4 warps per SM) except for 8-warp blocks.
template <int R, int AW>
__global__ void __launch_bounds__(AW * 32, (R == 1 && AW < 8) ? 20 / AW : 1) k_axi(AxiArgs A) {
    extern __shared__ float smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nx = A.nx, nr = A.nr, nrp = 32 * R;
    const AxiLayout Ly = axi_layout(nx, nrp);
    float *W = smem + (size_t)warp * Ly.total;
    float *hx = W + Ly.hx, *lwx = W + Ly.lwx, *Tt = W + Ly.Tt, *Lt = W + Ly.Lt, *mu = W + Ly.mu;
    float *va = W + Ly.vec, *vda = va + 12, *vm = vda + 12, *vg = vm + 12, *vx = vg + 12;
    float *H = W + Ly.H, *HL = W + Ly.HL, *rhs = W + Ly.rhs, *Sm = W + Ly.Sm, *Xm = W + Ly.Xm;
    float *al = W + Ly.al, *bt = W + Ly.bt, *sv = W + Ly.sv, *m35 = W + Ly.sv + 32, *b35 = m35 + 36;
    const mem_solve_opts &o = A.o;
    const int64_t nw = (int64_t)gridDim.x * AW;
    for (int64_t cell = (int64_t)blockIdx.x * AW + warp; cell < A.B; cell += nw) {
        const bool do_solve = A.solve && (!A.active || A.active[cell]);
        const bool want_flux = A.F || A.speed;
        if (!do_solve && !want_flux) continue;
        // ---- the rule as seen from this cell (gauge (w_x, 0, 0, s_x, s_r, s_r))
        const float *gc = A.gauge + cell * 6;
        const float wx = gc[0], sx = gc[3], sr = gc[4];
        const float *dr = A.dom + mem_host::DOM_REC * (A.pid ? A.pid[cell] : 0);
        const float axh = dr[0], axl = dr[1], hxh = dr[2], hxl = dr[3], hrh = dr[4], hrl = dr[5];
        const float lhx = __logf(0.5f * hxh), lhr2 = 2.f * __logf(hrh);
        float rxh, rxl, rrh, rrl;
        ff_recip(sx, rxh, rxl);
        ff_recip(sr, rrh, rrl);
        const float *lgx = A.vtf, *lrw = A.vtf + nx;
        __syncwarp();  // the previous cell is done with the tables
        for (int i = lane; i < nx; i += 32) {
            float dh, dl, uh, ul, hs, hl;
            ff_offset(axh, axl, hxh, hxl, A.vt2[i], wx, dh, dl);
            ff_ubar(dh, dl, rxh, rxl, uh, ul);
            ff_half_square(uh, ul, hs, hl);
            float h[10];
            hermite_vals<9>(uh, h);
#pragma unroll
            for (int k = 0; k < 10; ++k) hx[12 * i + k] = h[k];
            hx[12 * i + 10] = ((lhx + lgx[i]) - hs) - hl;
            hx[12 * i + 11] = 0.f;
        }
        float lwr[R], L1[R], L2[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int m = lane + 32 * r;
            float Lk[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            lwr[r] = -INFINITY;
            if (m < nr) {
                // the radial offset of node m is the y offset of its first azimuth
                float dh, dl, uh, ul, hs, hl;
                ff_offset(0.f, 0.f, hrh, hrl, A.vt2[nx + (size_t)m * A.K], 0.f, dh, dl);
                ff_ubar(dh, dl, rrh, rrl, uh, ul);
                ff_half_square(uh, ul, hs, hl);
                const float s = hs + hl;
                Lk[0] = 1.f;
                Lk[1] = 1.f - s;
#pragma unroll
                for (int k = 1; k < 4; ++k) Lk[k + 1] = ((2.f * k + 1.f - s) * Lk[k] - k * Lk[k - 1]) / (k + 1.f);
                lwr[r] = ((lhr2 + lrw[m]) - hs) - hl;
            }
            L1[r] = Lk[1];
            L2[r] = Lk[2];
#pragma unroll
            for (int k = 0; k < 5; ++k) Lt[k * nrp + m] = Lk[k];
        }
        // ---- the cell's moments and parameters, projected on the nine statistics
        const float *Mc = A.M + cell * NP;
        float *bc = A.beta + cell * NP;
        const float n = Mc[0];
        bool bad = false;
        for (int k = lane; k < NP; k += 32) {
            m35[k] = Mc[k];
            b35[k] = bc[k];
            bad |= !isfinite(m35[k]) || (k > 0 && !isfinite(b35[k]));
        }
        bad = __any_sync(0xffffffffu, bad) || !(n > 0.f) || !isfinite(n);
        __syncwarp();
        if (lane < NS) {
            float pm = 0.f, pb = 0.f;
            for (int t = 0; t < c_vn[lane]; ++t) {
                pm = fmaf(c_vc[lane][t], m35[c_vk[lane][t]], pm);
                pb = fmaf(c_vc[lane][t], b35[c_vk[lane][t]], pb);
            }
            va[lane] = lane ? pb : 0.f;
            vm[lane] = lane ? pm / n : 0.f;
            vda[lane] = 0.f;
            vg[lane] = 0.f;
        }
        if (lane < 4) vx[lane] = 0.f;
        __syncwarp();
        float cb[R][3];
        axi_coeffs<R>(va, L1, L2, cb);
        float mxc = -1e30f;
        bool mu_current = false;  // mu holds the moments of the current va
        if (do_solve && bad) {
            if (lane == 0) {
                if (A.status) A.status[cell] = MEM_ST_BADINPUT;
                if (A.iters) A.iters[cell] = 0;
            }
        } else if (do_solve) {
            // ---- Algorithm 1 on the eight unknowns a_1 .. a_8
            const float lz0 = axi_sweep<R>(cb, va[4], va[5], lwr, hx, lwx, nx, Tt, nrp, lane, mxc);
            float mb = 0.f;
#pragma unroll
            for (int j = 1; j < NS; ++j) mb = fmaf(va[j], vm[j], mb);
            float Lcur = lz0 - mb, alpha = 1.f, pmin = 0.f, pmax = 0.f;
            int st = 0, it = 0;
            while (true) {
                axi_s_stage(Tt, Lt, nr, nrp, mu, lane);
                // gradient and Hessian (Appendix C)
                if (lane >= 1 && lane < NS)
                    vg[lane] = c_psg[lane] * mu[5 * c_pa[lane] + c_pm[lane]] - vm[lane];
                for (int e = lane; e < 45; e += 32) {
                    int p, q;
                    packed_pq(e, p, q);
                    if (q >= 1) {
                        const float ep = c_psg[p] * mu[5 * c_pa[p] + c_pm[p]];
                        const float eq = c_psg[q] * mu[5 * c_pa[q] + c_pm[q]];
                        H[(p - 1) * 8 + (q - 1)] = axi_entry(A, mu, e) - ep * eq;
                    }
                }
                __syncwarp();
                // Cholesky of H, then of H + lambda I, lambda = lambda0 mul^t
                bool ok = false;
                float lam = 0.f;
                for (int t = 0; t <= o.max_lambda; ++t) {
                    for (int e = lane; e < 64; e += 32) {
                        const int p = e >> 3, q = e & 7;
                        if (q <= p) HL[e] = H[e] + (p == q ? lam : 0.f);
                    }
                    ok = warp_cholesky(HL, 8, 8, lane);
                    if (ok) break;
                    st |= MEM_ST_LAMBDA;
                    lam = (t == 0) ? o.lambda0 : lam * o.lambda_mul;
                }
                ++it;
                if (!ok) {
                    st |= MEM_ST_LAMBDA_CAP | MEM_ST_NONFINITE;
                    break;
                }
                {
                    const float d = lane < 8 ? HL[lane * 9] * HL[lane * 9] : 0.f;
                    pmax = warp_max(d);
                    pmin = -warp_max(lane < 8 ? -d : -INFINITY);
                }
                if (lane < 8) rhs[lane] = -vg[lane + 1];
                warp_solve_lower(HL, 8, 8, rhs, lane);
                warp_solve_upperT(HL, 8, 8, rhs, lane);
                const float x = lane < 8 ? rhs[lane] : 0.f;
                const float gd = warp_sum(lane < 8 ? x * vg[lane + 1] : 0.f);
                const float md = warp_sum(lane < 8 ? x * vm[lane + 1] : 0.f);
                if (lane < 8) vda[lane + 1] = x;
                __syncwarp();
                const float res = 0.5f * fabsf(gd);
                if (!isfinite(res)) {
                    st |= MEM_ST_NONFINITE;
                    break;
                }
                const bool conv_res = res <= o.tol, conv_a = alpha <= o.alpha_min;
                if (conv_res) st |= MEM_ST_CONVERGED;
                if (conv_a) st |= MEM_ST_STAGNATED;
                if (conv_res || conv_a) {
                    mu_current = true;
                    if (conv_res && o.final_step) {
                        if (lane >= 1 && lane < NS) va[lane] += vda[lane];
                        __syncwarp();
                        mu_current = false;
                    }
                    break;
                }
                if (it > o.maxI) {
                    st |= MEM_ST_MAXITER;
                    mu_current = true;
                    break;
                }
                // ---- BackTrackingLineSearch / ArmijoCondition (Algorithm 1)
                float cd[R][3], ca[R][3];
                axi_coeffs<R>(vda, L1, L2, cd);
                const float d4 = vda[4], d5 = vda[5], b4 = va[4], b5 = va[5];
                alpha = 2.f;
                bool sat = false;
                float Lt_ = Lcur;
                for (int s_ = 0; !sat && s_ <= o.maxT; ++s_) {
                    alpha *= 0.5f;
#pragma unroll
                    for (int r = 0; r < R; ++r)
#pragma unroll
                        for (int k = 0; k < 3; ++k) ca[r][k] = fmaf(alpha, cd[r][k], cb[r][k]);
                    const float lz = axi_sweep<R>(ca, fmaf(alpha, d4, b4), fmaf(alpha, d5, b5), lwr, hx, lwx, nx, Tt,
                                                  nrp, lane, mxc);
                    Lt_ = lz - (mb + alpha * md);
                    const float LD = Lcur - Lt_, gradD = -o.c_armijo * alpha * gd;
                    sat = (LD - gradD) >= -(o.atol + o.rtol * fabsf(LD));
                }
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int k = 0; k < 3; ++k) cb[r][k] = ca[r][k];
                Lcur = Lt_;
                mb += alpha * md;
                if (lane >= 1 && lane < NS) va[lane] += alpha * vda[lane];
                __syncwarp();
            }
            // beta = sum_j a_j v_j
            for (int k = lane; k < NP; k += 32) b35[k] = 0.f;
            __syncwarp();
            if (lane < NS && lane > 0)
                for (int t = 0; t < c_vn[lane]; ++t) b35[c_vk[lane][t]] = c_vc[lane][t] * va[lane];
            __syncwarp();
            for (int k = lane; k < NP; k += 32) bc[k] = k ? b35[k] : n;
            if (lane == 0) {
                if (A.status) A.status[cell] = st;
                if (A.iters) A.iters[cell] = it;
                if (A.cond) A.cond[cell] = pmin > 0.f ? pmax / pmin : 0.f;
            }
        }
        if (!want_flux) continue;
        // ---- flux and speed of the nine-moment system at the final parameters
        if (!mu_current) {
            axi_coeffs<R>(va, L1, L2, cb);
            axi_sweep<R>(cb, va[4], va[5], lwr, hx, lwx, nx, Tt, nrp, lane, mxc);
            axi_s_stage(Tt, Lt, nr, nrp, mu, lane);
        }
        const float nF = bad ? 0.f : n;
        if (A.F) {
            // F_j = n (w_x E[psi_j] + s_x E[ubar_x psi_j]), ubar_x he_a =
            // sqrt(a+1) he_{a+1} + sqrt(a) he_{a-1}; F (35) = sum_j F_j v_j
            if (lane < NS) {
                const int a = c_pa[lane], mm = c_pm[lane];
                float xm = sqrtf((float)(a + 1)) * mu[5 * (a + 1) + mm];
                if (a > 0) xm = fmaf(sqrtf((float)a), mu[5 * (a - 1) + mm], xm);
                sv[lane] = c_psg[lane] * nF * fmaf(wx, mu[5 * a + mm], sx * xm);
            }
            for (int k = lane; k < NP; k += 32) b35[k] = 0.f;
            __syncwarp();
            if (lane < NS)
                for (int t = 0; t < c_vn[lane]; ++t) b35[c_vk[lane][t]] = c_vc[lane][t] * sv[lane];
            __syncwarp();
            for (int k = lane; k < NP; k += 32) A.F[cell * NP + k] = b35[k];
            __syncwarp();
        }
        if (A.speed) {
            // the 9 x 9 pencil (E[ubar_x psi psi^T], E[psi psi^T]) of Eq. "The lax F"
            for (int e = lane; e < 90; e += 32) {
                int p, q;
                packed_pq(e < 45 ? e : e - 45, p, q);
                (e < 45 ? Sm : Xm)[p * 16 + q] = axi_entry(A, mu, e);
            }
            __syncwarp();
            float ulo, uhi, el;
            ff_offset(axh, axl, hxh, hxl, A.vt2[0], 0.f, ulo, el);
            ff_offset(axh, axl, hxh, hxl, A.vt2[nx - 1], 0.f, uhi, el);
            const float bound = fmaxf(fabsf(ulo), fabsf(uhi));
            float lo = 0.f, hi = 0.f;
            const bool ok = !bad && small_pencil_extremes(Sm, Xm, NS, al, bt, sv, lane, lo, hi);
            if (lane == 0) {
                const float sp = ok ? fmaxf(fabsf(wx + sx * hi), fabsf(wx + sx * lo)) : bound;
                A.speed[cell] = (sp <= bound) ? sp : bound;
            }
            __syncwarp();
        }
    }
}

template <int R, int AW>
int launch_axi(mem_ctx *ctx, const AxiArgs &a, cudaStream_t st, int bps_cap) {
    const size_t smem = sizeof(float) * (size_t)axi_layout(a.nx, 32 * R).total * AW;
    if (smem > 227 * 1024) return MEM_EINVAL;
    MEM_CUDA_TRY(cudaFuncSetAttribute(k_axi<R, AW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int sms = 0, per_sm = 0;
    MEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    MEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_axi<R, AW>, AW * 32, smem));
    if (per_sm < 1) return MEM_ECUDA;
    if (bps_cap > 0) per_sm = std::min(per_sm, bps_cap);
    const int grid = (int)std::min<int64_t>((a.B + AW - 1) / AW, (int64_t)sms * per_sm);
    k_axi<R, AW><<<grid, AW * 32, smem, st>>>(a);
    MEM_CUDA_TRY(cudaGetLastError());
    return MEM_OK;
}

template <int R>
int launch_axi_cfg(mem_ctx *ctx, const AxiArgs &a, cudaStream_t st, const mem_launch_cfg &c) {
    switch (c.warps) {
        case 2: return launch_axi<R, 2>(ctx, a, st, c.blocks_per_sm);
        case 8: return launch_axi<R, 8>(ctx, a, st, c.blocks_per_sm);
        default: return launch_axi<R, 4>(ctx, a, st, c.blocks_per_sm);
    }
}

template <int R, int AW>
int occ_axi(int nx, int *per_sm) {
    const size_t smem = sizeof(float) * (size_t)axi_layout(nx, 32 * R).total * AW;
    if (smem > 227 * 1024) { *per_sm = 0; return MEM_OK; }
    cudaFuncSetAttribute(k_axi<R, AW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_axi<R, AW>, AW * 32, smem) == cudaSuccess
               ? MEM_OK
               : MEM_ECUDA;
}

template <int R>
int occ_axi_w(int W, int nx, int *per_sm) {
    switch (W) {
        case 2: return occ_axi<R, 2>(nx, per_sm);
        case 8: return occ_axi<R, 8>(nx, per_sm);
        default: return occ_axi<R, 4>(nx, per_sm);
    }
}

// ---- host: linearisation terms of the nine statistics
double fact_h(int n) {
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= i;
    return r;
}
double binom_h(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}
// coefficient of he_c in he_a he_b (orthonormal Hermite)
double hlin(int a, int b, int c) {
    const int s = a + b - c;
    if (s < 0 || s % 2) return 0.0;
    const int k = s / 2;
    if (k > a || k > b) return 0.0;
    return binom_h(a, k) * binom_h(b, k) * fact_h(k) * sqrt(fact_h(a + b - 2 * k) / (fact_h(a) * fact_h(b)));
}
// Laguerre polynomial coefficients in powers of s: L_k = sum_j l[k][j] s^j
void laguerre_poly(int K, std::vector<std::vector<double>> &l) {
    l.assign(K + 1, std::vector<double>(K + 1, 0.0));
    for (int k = 0; k <= K; ++k)
        for (int j = 0; j <= k; ++j) l[k][j] = (j % 2 ? -1.0 : 1.0) * binom_h(k, j) / fact_h(j);
}
// coefficient of L_k in L_m L_n: int L_m L_n L_k e^{-s} ds, int s^j e^{-s} = j!
double llin(int m, int n, int k, const std::vector<std::vector<double>> &l) {
    double r = 0.0;
    for (int i = 0; i <= m; ++i)
        for (int j = 0; j <= n; ++j)
            for (int t = 0; t <= k; ++t) r += l[m][i] * l[n][j] * l[k][t] * fact_h(i + j + t);
    return r;
}

}  // namespace

namespace mem_host {

int build_axi_tables(mem_ctx *ctx) {
    static const int pa[NS] = {0, 1, 2, 0, 3, 4, 0, 1, 2}, pm[NS] = {0, 0, 0, 1, 0, 0, 2, 1, 1};
    static const double ps[NS] = {1, 1, 1, -1, 1, 1, 1, -1, -1};
    std::vector<std::vector<double>> l;
    laguerre_poly(8, l);
    std::vector<int2> terms;
    std::vector<int> off;
    for (int pass = 0; pass < 2; ++pass)  // E[psi psi^T], then E[ubar_x psi psi^T]
        for (int e = 0; e < 45; ++e) {
            int p = 0;
            while ((p + 1) * (p + 2) / 2 <= e) ++p;
            const int q = e - p * (p + 1) / 2;
            off.push_back((int)terms.size());
            std::vector<double> acc(NMU, 0.0);
            for (int c = 0; c <= 8; ++c) {
                const double hc = hlin(pa[p], pa[q], c);
                if (hc == 0.0) continue;
                for (int k = 0; k <= 4; ++k) {
                    const double lk = llin(pm[p], pm[q], k, l);
                    if (fabs(lk) < 1e-12) continue;
                    const double w = ps[p] * ps[q] * hc * lk;
                    if (pass == 0) acc[5 * c + k] += w;
                    else {
                        acc[5 * (c + 1) + k] += w * sqrt((double)(c + 1));
                        if (c > 0) acc[5 * (c - 1) + k] += w * sqrt((double)c);
                    }
                }
            }
            for (int i = 0; i < NMU; ++i)
                if (acc[i] != 0.0) {
                    const float f = (float)acc[i];
                    int bits;
                    memcpy(&bits, &f, 4);
                    terms.push_back(make_int2(i, bits));
                }
        }
    off.push_back((int)terms.size());
    // 35-product coefficients of the nine statistics
    int vk[NS][3] = {}, vn[NS] = {};
    float vc[NS][3] = {};
    auto put = [&](int j, int a, int b, int c, float w) {
        vk[j][vn[j]] = idx3(a, b, c);
        vc[j][vn[j]] = w;
        ++vn[j];
    };
    const float r2 = (float)sqrt(0.5), q = (float)(sqrt(24.0) / 8.0);
    put(0, 0, 0, 0, 1.f);
    put(1, 1, 0, 0, 1.f);
    put(2, 2, 0, 0, 1.f);
    put(3, 0, 2, 0, r2); put(3, 0, 0, 2, r2);
    put(4, 3, 0, 0, 1.f);
    put(5, 4, 0, 0, 1.f);
    put(6, 0, 4, 0, q); put(6, 0, 0, 4, q); put(6, 0, 2, 2, 0.5f);
    put(7, 1, 2, 0, r2); put(7, 1, 0, 2, r2);
    put(8, 2, 2, 0, r2); put(8, 2, 0, 2, r2);
    MEM_CUDA_TRY(cudaMemcpyToSymbol(c_vk, vk, sizeof(vk)));
    MEM_CUDA_TRY(cudaMemcpyToSymbol(c_vc, vc, sizeof(vc)));
    MEM_CUDA_TRY(cudaMemcpyToSymbol(c_vn, vn, sizeof(vn)));
    if (cudaMalloc((void **)&ctx->d_axi_terms, sizeof(int2) * terms.size()) != cudaSuccess ||
        cudaMalloc((void **)&ctx->d_axi_toff, sizeof(int) * off.size()) != cudaSuccess) {
        cudaGetLastError();
        return MEM_ENOMEM;
    }
    MEM_CUDA_TRY(cudaMemcpy(ctx->d_axi_terms, terms.data(), sizeof(int2) * terms.size(), cudaMemcpyHostToDevice));
    MEM_CUDA_TRY(cudaMemcpy(ctx->d_axi_toff, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
    return MEM_OK;
}

int axi_run(mem_ctx *ctx, const float *M, float *beta, const float *g, int32_t *status, int32_t *iters, float *F,
            float *speed, const int *pid, const float *dom, int64_t B, const mem_solve_opts &o, bool solve,
            cudaStream_t st, const unsigned char *active, float *cond) {
    if (!ctx->vel || !ctx->d_axi_terms) return MEM_EINVAL;
    if (B == 0) return MEM_OK;
    AxiArgs a;
    a.M = M; a.beta = beta; a.gauge = g; a.status = status; a.iters = iters; a.F = F; a.speed = speed;
    a.cond = cond; a.pid = pid; a.dom = dom ? dom : ctx->d_dom0; a.active = active;
    a.vt2 = ctx->d_vt2; a.vtf = ctx->d_vtf;
    a.terms = ctx->d_axi_terms; a.toff = ctx->d_axi_toff;
    a.B = B;
    a.nbx = ctx->nbx; a.nbr = ctx->nbr; a.K = ctx->K; a.nx = ctx->nx; a.nr = ctx->nbr * ctx->ng;
    a.solve = solve ? 1 : 0;
    a.o = o;
    const int R = (a.nr + 31) / 32;
    switch (R) {
        case 1: return launch_axi_cfg<1>(ctx, a, st, ctx->cfg_axi);
        case 2: return launch_axi_cfg<2>(ctx, a, st, ctx->cfg_axi);
        case 3: return launch_axi_cfg<3>(ctx, a, st, ctx->cfg_axi);
        case 4: return launch_axi_cfg<4>(ctx, a, st, ctx->cfg_axi);
        default: return MEM_EINVAL;
    }
}

int axi_occupancy(mem_ctx *ctx, int W, int *per_sm) {
    const int R = (ctx->nbr * ctx->ng + 31) / 32;
    switch (R) {
        case 1: return occ_axi_w<1>(W, ctx->nx, per_sm);
        case 2: return occ_axi_w<2>(W, ctx->nx, per_sm);
        case 3: return occ_axi_w<3>(W, ctx->nx, per_sm);
        case 4: return occ_axi_w<4>(W, ctx->nx, per_sm);
        default: return MEM_EINVAL;
    }
}

}  // namespace mem_host

// velocity.cu -- Algorithm 1 and the flux moments with a quadrature rule fixed
// in velocity space, as in the paper's shock computations (Section 3.1, Eq.
// "Numerical integration": fixed nodes u_q and weights w_q; Appendix D: the
// integration domain (u_x, u_r) in [a_x, b_x] x [0, b_r] is set by the
// Rankine-Hugoniot states).  One thread block per cell, FP32, no scratch.
//
// Rule.  u_x on [a_x, b_x] in nbx equal blocks of ng Gauss-Legendre points
// (i < nx = nbx ng); the transverse plane in polar form, u_r on [0, b_r] in
// nbr equal blocks of ng Gauss-Legendre points with the weight u_r, times K
// equispaced azimuths (p < npt = nbr ng K).  Nodes u = (x_i, y_p, z_p).  In a
// cell of gauge g, ubar = (u - w)/s and the log weight is
// log w_q - |ubar|^2/2, so that beta stays relative to the gauge's Gaussian
// (constant factors cancel in Z).  With a gauge-frame rule the nodes would
// not follow the cell; here a cold upstream beam stays resolved in every cell
// of a strong shock, which is what the paper's Mach-10 run needs.
//
// Both contractions factor over x and the plane, because every statistic is
// he_a(ubar_x) psi_bc(p) with psi_bc = he_b(ubar_y) he_c(ubar_z):
//   exponent  e(i,p) = lw_x(i) + lw_t(p) + sum_a he_a(x_i) P_a(p),
//             P_a(p) = sum_{b,c} beta_abc psi_bc(p)
//   moments   T_a(p) = sum_i sigma(i,p) he_a(x_i)            (x stage)
//             mu_abc = sum_p T_a(p) he_b(y_p) he_c(z_p)       (plane stage)
// Thread t owns the plane points p = t + VT r and sweeps all x_i; the
// partition function is a block log-sum-exp.  E[phi_i phi_j] follows from the
// moments of degree <= 8 by the Hermite linearisation (as in fused.cu); the
// Newton linear algebra (Hessian, register Cholesky with lambda I) runs on
// warp 0 while the other warps wait at the barrier.
#include "common.cuh"
#include "ctx.h"
#include "ffloat.cuh"
#include "linalg.cuh"
#include "sumfact.cuh"

using namespace mem;

namespace {

constexpr int VT = 128;
constexpr int VW = VT / 32;

struct VelArgs {
    const float *M;
    float *beta;
    const float *gauge;
    int32_t *status;
    int32_t *iters;
    float *mu;                    // [B][MEM_MU_STRIDE] moments of degree <= 9 at the final beta, or null
    float *cond;                  // [B] largest / smallest Cholesky pivot of the last Newton pass, or null
    const int *pid;               // per-cell domain index, or null (domain 0)
    const float *dom;             // [domains][DOM_REC] domain records (dom_record)
    const unsigned char *active;  // 0: no solve for this cell (its moments are still produced)
    const float2 *vt2;            // [nx] x | [npt] y | [npt] z offsets in block widths, float pairs
    const float *vtf;             // [nx] log w^GL of the x node | [nr] log(w^GL t_r / K) of the radial node
    const int2 *slots;            // Hessian linearisation terms over the block's 128 lanes
    int n_slots;
    int64_t B;
    int nbx, nbr, ng, K, nx, npt, PS;
    int solve;
    mem_solve_opts o;
};

struct VelLayout {
    int hx, lwx, hy, hz, T, lwp, pij, abc, vec, H, red, total;
};

__host__ __device__ inline int plane_stride(int npt) { return ((npt + 31) / 32) * 32 + 1; }

__host__ __device__ inline VelLayout vel_layout(int nx, int npt) {
    VelLayout L;
    const int PS = plane_stride(npt);
    int o = 0;
    L.hx = o; o += 10 * nx;
    L.lwx = o; o += nx;
    L.hy = o; o += 10 * PS;
    L.hz = o; o += 10 * PS;
    L.T = o; o += 10 * PS;
    L.lwp = o; o += PS;
    L.pij = o; o += 596;
    L.abc = o; o += 220;
    o = (o + 3) & ~3;  // 16-byte aligned: the Cholesky broadcast column lives at vec + 180
    L.vec = o; o += 6 * 36 + 224;  // beta, dbeta, M/n, grad, scalars (6 used) | broadcast column | mu
    L.H = o; o += NP1 * LDH;
    L.red = o; o += 2 * VW + 2;
    L.total = o;
    return L;
}

__device__ __forceinline__ float block_max(float v, float *red, int warp, int lane) {
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float r = red[0];
#pragma unroll
    for (int w = 1; w < VW; ++w) r = fmaxf(r, red[w]);
    return r;
}

__device__ __forceinline__ float block_sum(float v, float *red, int warp, int lane) {
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[VW + warp] = v;
    __syncthreads();
    float r = 0.f;
#pragma unroll
    for (int w = 0; w < VW; ++w) r += red[VW + w];
    return r;
}

// P_a(p) of a parameter vector v (slots 1..34, shared) on the thread's plane
// points; points beyond npt get zeros (their log weight is -inf).
template <int PPT>
__device__ __forceinline__ void plane_coeffs(const float *v, const float *hy, const float *hz, int PS, int npt,
                                             int tid, float (&c)[PPT][5]) {
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
        const int p = tid + VT * r;
        float y[5], z[5];
#pragma unroll
        for (int a = 0; a < 5; ++a) {
            y[a] = p < npt ? hy[a * PS + p] : 0.f;
            z[a] = p < npt ? hz[a * PS + p] : 0.f;
        }
#pragma unroll
        for (int a = 0; a <= 4; ++a) {
            float acc = 0.f;
#pragma unroll
            for (int b = 0; a + b <= 4; ++b) {
                float inner = 0.f;
#pragma unroll
                for (int cc = 0; a + b + cc <= 4; ++cc)
                    if (a + b + cc > 0) inner += v[idx3(a, b, cc)] * z[cc];
                acc += inner * y[b];
            }
            c[r][a] = acc;
        }
    }
}

// Plane stage mu_o = sum_p T_a(p) he_b(y_p) he_c(z_p), o = idx3(a, b, c) < NO,
// one output per thread; consecutive threads read different rows at the same
// p, which the odd row stride keeps in distinct banks.  Eight interleaved
// accumulators keep each FP32 chain short (a single 384-long chain costs
// ~1e-5 in the moments of the stiffest Mach-10 cells) and give the loads
// independent work.  Fixed order; the caller synchronises before reading out.
__device__ __forceinline__ void plane_stage(int NO, const float *sT, const float *hy, const float *hz, int PS,
                                            int npt, const int *abc, float *out, int warp, int lane) {
    const int tid = warp * 32 + lane;
    for (int o = tid; o < NO; o += VT) {
        const int e = abc[o];
        const float *Ta = sT + (e & 255) * PS, *Yb = hy + ((e >> 8) & 255) * PS, *Zc = hz + (e >> 16) * PS;
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int p = 0;
        for (; p + 7 < npt; p += 8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] = fmaf(Ta[p + u] * Yb[p + u], Zc[p + u], acc[u]);
        }
        for (; p < npt; ++p) acc[0] = fmaf(Ta[p] * Yb[p], Zc[p], acc[0]);
        out[o] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    }
}

// Log-sum-exp and x stage in one sweep: with a running per-thread maximum m,
// s = sum_q exp(e_q - m) and T_a(p) = sum_i exp(e - m) he_a(x_i), a < AM; a
// new maximum rescales both.  m starts at m0, the block maximum of the
// previous evaluation of the same cell (or -1e30), so rescaling, which
// diverges the warp, is rare; nodes more than ~87 below m0 underflow to zero
// weight, i.e. sigma < 1e-38.  The caller turns the per-thread results into
// sigma-weighted moments with one factor exp(m - M) / S from the block
// maximum M and sum S.
template <int PPT, int AM>
__device__ __forceinline__ void node_lse_moments(const float (&c)[PPT][5], const float (&lwp)[PPT], const float *hx,
                                                 const float *lwx, int nx, float m0, float &m, float &s,
                                                 float &emax, float (&T)[PPT][10]) {
    m = m0;
    emax = -INFINITY;
    s = 0.f;
#pragma unroll
    for (int r = 0; r < PPT; ++r)
#pragma unroll
        for (int a = 0; a < 10; ++a) T[r][a] = 0.f;
    for (int i = 0; i < nx; ++i) {
        float h[AM];
#pragma unroll
        for (int a = 0; a < AM; ++a) h[a] = hx[a * nx + i];
        const float lx = lwx[i];
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const float e = lx + lwp[r] + c[r][0] + h[1] * c[r][1] + h[2] * c[r][2] + h[3] * c[r][3] + h[4] * c[r][4];
            emax = fmaxf(emax, e);
            float w;
            if (e > m) {
                const float sc = __expf(m - e);
                s *= sc;
#pragma unroll
                for (int rr = 0; rr < PPT; ++rr)
#pragma unroll
                    for (int a = 0; a < AM; ++a) T[rr][a] *= sc;
                m = e;
                w = 1.f;
            } else {
                w = __expf(e - m);
            }
            s += w;
#pragma unroll
            for (int a = 0; a < AM; ++a) T[r][a] = fmaf(w, h[a], T[r][a]);
        }
    }
}

// One evaluation at the plane coefficients c: the fused sweep, the block
// log-sum-exp, and the sigma-weighted x stage T_a(p) stored to the shared
// table (rows a < AM).  Returns log Z; mx carries the block maximum from one
// evaluation of the cell to the next.  The table is only read by the plane
// stage, which runs after the accepted evaluation, so a rejected line-search
// trial just gets overwritten by the next one.
template <int PPT, int AM>
__device__ __forceinline__ float sweep_store(const float (&c)[PPT][5], const float (&lwp)[PPT], const float *hx,
                                             const float *lwx, int nx, float *sT, int PS, int npt, float *red,
                                             int tid, int warp, int lane, float &mx) {
    float T[PPT][10];
    float m, s, em;
    node_lse_moments<PPT, AM>(c, lwp, hx, lwx, nx, mx, m, s, em, T);
    // If the true maximum fell far below the warm start, weights near the
    // top would underflow: redo the sweep from the true maximum (uniform).
    const float E = block_max(em, red, warp, lane);
    if (E < mx - 40.f) node_lse_moments<PPT, AM>(c, lwp, hx, lwx, nx, E, m, s, em, T);
    mx = block_max(m, red, warp, lane);
    const float Z = block_sum(s * __expf(m - mx), red, warp, lane);
    const float f = __expf(m - mx) / Z;
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
        const int p = tid + VT * r;
        if (p < npt) {
#pragma unroll
            for (int a = 0; a < AM; ++a) sT[a * PS + p] = T[r][a] * f;
        }
    }
    return mx + __logf(Z);
}

template <int PPT>
__global__ void __launch_bounds__(VT, 3) k_vel(VelArgs A) {
    extern __shared__ float smem[];
    const VelLayout Ly = vel_layout(A.nx, A.npt);
    const int nx = A.nx, npt = A.npt, PS = A.PS;
    float *s_hx = smem + Ly.hx, *s_lwx = smem + Ly.lwx, *s_hy = smem + Ly.hy, *s_hz = smem + Ly.hz;
    float *s_T = smem + Ly.T, *s_lwp = smem + Ly.lwp, *H = smem + Ly.H, *red = smem + Ly.red;
    int *s_pij = (int *)(smem + Ly.pij), *s_abc = (int *)(smem + Ly.abc);
    float *sb = smem + Ly.vec, *sd = sb + 36, *smv = sd + 36, *sg = smv + 36, *sx = sg + 36, *smu = sx + 72;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const mem_solve_opts &o = A.o;
    for (int t = tid; t < NP1 * (NP1 + 1) / 2; t += VT) {
        int i = 0;
        while ((i + 1) * (i + 2) / 2 <= t) ++i;
        s_pij[t] = i | ((t - i * (i + 1) / 2) << 8);
    }
    for (int t = tid; t < 220; t += VT) s_abc[t] = exp_a(t) | (exp_b(t) << 8) | (exp_c(t) << 16);

    for (int64_t cell = blockIdx.x; cell < A.B; cell += gridDim.x) {
        const bool do_solve = A.solve && (!A.active || A.active[cell]);
        if (!do_solve && !A.mu) continue;
        // ---- the rule as seen from this cell
        const float *gc = A.gauge + cell * 6;
        const float wx = gc[0], wy = gc[1], wz = gc[2], sx_ = gc[3], sy = gc[4], sz = gc[5];
        // u - w cancels on a box tens of thermal widths wide, and the hot tail
        // of a mixed cell sits at |ubar| ~ 5-10, where plain FP32 rounding of
        // ubar and ubar^2 / 2 moves its weights by ~1e-5.  So u - w, ubar =
        // (u - w) / s and ubar^2 / 2 are formed in error-free float-float
        // arithmetic from the domain record and the offsets as float pairs,
        // and the log weight is rounded once.
        const float *dr = A.dom + mem_host::DOM_REC * (A.pid ? A.pid[cell] : 0);
        const float axh = dr[0], axl = dr[1], hxh = dr[2], hxl = dr[3], hrh = dr[4], hrl = dr[5];
        const float lhx = __logf(0.5f * hxh), lhr2 = 2.f * __logf(hrh);
        float rxh, rxl, ryh, ryl, rzh, rzl;
        ff_recip(sx_, rxh, rxl);
        ff_recip(sy, ryh, ryl);
        ff_recip(sz, rzh, rzl);
        const float2 *xt = A.vt2, *yt = A.vt2 + nx, *zt = yt + npt;
        const float *lgx = A.vtf, *lrw = A.vtf + nx;
        __syncthreads();  // the previous cell is done with every table
        for (int i = tid; i < nx; i += VT) {
            float dh, dl, uh, ul, hs, hl;
            ff_offset(axh, axl, hxh, hxl, xt[i], wx, dh, dl);
            ff_ubar(dh, dl, rxh, rxl, uh, ul);
            ff_half_square(uh, ul, hs, hl);
            float h[10];
            hermite_vals<9>(uh, h);
#pragma unroll
            for (int a = 0; a < 10; ++a) s_hx[a * nx + i] = h[a];
            s_lwx[i] = ((lhx + lgx[i]) - hs) - hl;
        }
        for (int p = tid; p < npt; p += VT) {
            float dh, dl, yh, yl, zh, zl, ys, yls, zs, zls;
            ff_offset(0.f, 0.f, hrh, hrl, yt[p], wy, dh, dl);
            ff_ubar(dh, dl, ryh, ryl, yh, yl);
            ff_offset(0.f, 0.f, hrh, hrl, zt[p], wz, dh, dl);
            ff_ubar(dh, dl, rzh, rzl, zh, zl);
            ff_half_square(yh, yl, ys, yls);
            ff_half_square(zh, zl, zs, zls);
            float h[10];
            hermite_vals<9>(yh, h);
#pragma unroll
            for (int a = 0; a < 10; ++a) s_hy[a * PS + p] = h[a];
            hermite_vals<9>(zh, h);
#pragma unroll
            for (int a = 0; a < 10; ++a) s_hz[a * PS + p] = h[a];
            s_lwp[p] = ((lhr2 + lrw[p / A.K]) - (ys + zs)) - (yls + zls);
        }
        // ---- load and validate
        const float *Mc = A.M + cell * NP;
        float *bc = A.beta + cell * NP;
        const float n = Mc[0];
        bool bad = false;
        if (tid < NP) {
            const float mv = Mc[tid], bv = bc[tid];
            bad = !isfinite(mv) || (tid > 0 && !isfinite(bv));
            sb[tid] = tid ? bv : 0.f;
            smv[tid] = tid ? mv / n : 0.f;
            if (tid == 6 || tid == 7) sx[tid] = 0.f;  // pivot range of the last factorisation
            sd[tid] = 0.f;
            sg[tid] = 0.f;
        }
        bad = __syncthreads_or(bad) || !(n > 0.f) || !isfinite(n);
        float lwp[PPT];
#pragma unroll
        for (int r = 0; r < PPT; ++r) lwp[r] = tid + VT * r < npt ? s_lwp[tid + VT * r] : -INFINITY;
        float cb[PPT][5], cd[PPT][5], ca[PPT][5];
        float mxc = -1e30f;  // block maximum of the exponent at the latest evaluation of this cell
        if (do_solve && bad) {
            if (tid == 0) {
                if (A.status) A.status[cell] = MEM_ST_BADINPUT;
                if (A.iters) A.iters[cell] = 0;
            }
        } else if (do_solve) {
            // ---- Algorithm 1.  Every evaluation of the partition function
            // also produces the x stage at the same beta (node_lse_moments):
            // the accepted line-search trial therefore already carries the
            // moments of the next pass.
            plane_coeffs<PPT>(sb, s_hy, s_hz, PS, npt, tid, cb);
            const float lz0 = sweep_store<PPT, 9>(cb, lwp, s_hx, s_lwx, nx, s_T, PS, npt, red, tid, warp, lane, mxc);
            if (warp == 0) {
                const float pb = (lane >= 1 && lane < NP ? sb[lane] * smv[lane] : 0.f) +
                                 (lane + 32 < NP ? sb[lane + 32] * smv[lane + 32] : 0.f);
                const float mb = warp_sum(pb);
                if (lane == 0) sx[4] = mb;
            }
            __syncthreads();
            float mb = sx[4];
            float Lcur = lz0 - mb, alpha = 1.f;
            int st = 0, it = 0;
            while (true) {
                // ---- plane stage on the x stage of the last accepted sweep:
                // mu_abc, a+b+c <= 8
                __syncthreads();
                plane_stage(165, s_T, s_hy, s_hz, PS, npt, s_abc, smu, warp, lane);
                __syncthreads();
                // ---- gradient and Hessian (Appendix C) by the whole block,
                // from the linearisation terms spread over 128 lanes
                if (tid >= 1 && tid < NP) sg[tid] = smu[tid] - smv[tid];
                {
                    float acc = 0.f;
#pragma unroll 4
                    for (int t = 0; t < A.n_slots; ++t) {
                        const int2 sl = __ldg(&A.slots[t * VT + tid]);
                        acc = fmaf(__int_as_float(sl.y), smu[sl.x & 255], acc);
                        if (sl.x < 0) {
                            const int pp = (sl.x >> 8) & 1023;
                            const int pij = s_pij[pp], i = pij & 255, j = pij >> 8;
                            H[i * LDH + j] = acc - smu[i + 1] * smu[j + 1];
                            acc = 0.f;
                        }
                    }
                }
                __syncthreads();
                // ---- warp 0: Cholesky with lambda I, Newton direction
                if (warp == 0) {
                    const float g_l = sg[lane + 1], g32 = sg[33], g33 = sg[34];
                    float x = 0.f, x32 = 0.f, x33 = 0.f, lam = 0.f;
                    bool ok = false, used = false;
                    for (int t = 0; t <= o.max_lambda; ++t) {
                        ok = reg_chol_solve34<false>(H, lam, lane, -g_l, -g32, -g33, x, x32, x33, sx + 36,
                                                     A.cond ? sx + 6 : nullptr);
                        if (ok) break;
                        used = true;
                        lam = (t == 0) ? o.lambda0 : lam * o.lambda_mul;
                    }
                    const float dg = warp_sum(x * g_l) + x32 * g32 + x33 * g33;
                    const float dm_ = warp_sum(x * smv[lane + 1]) + x32 * smv[33] + x33 * smv[34];
                    sd[lane + 1] = ok ? x : 0.f;
                    if (lane == 0) {
                        sd[33] = ok ? x32 : 0.f;
                        sd[34] = ok ? x33 : 0.f;
                        sx[0] = ok ? 1.f : 0.f;
                        sx[1] = used ? 1.f : 0.f;
                        sx[2] = 0.5f * fabsf(dg);
                        sx[3] = dg;
                        sx[5] = dm_;
                    }
                }
                __syncthreads();
                ++it;
                if (sx[1] != 0.f) st |= MEM_ST_LAMBDA;
                if (sx[0] == 0.f) {
                    st |= MEM_ST_LAMBDA_CAP | MEM_ST_NONFINITE;
                    break;
                }
                const float res = sx[2], gd = sx[3], md = sx[5];
                if (!isfinite(res)) {
                    st |= MEM_ST_NONFINITE;
                    break;
                }
                const bool conv_res = res <= o.tol, conv_a = alpha <= o.alpha_min;
                if (conv_res) st |= MEM_ST_CONVERGED;
                if (conv_a) st |= MEM_ST_STAGNATED;
                if (conv_res || conv_a) {
                    if (conv_res && o.final_step && tid >= 1 && tid < NP) sb[tid] += sd[tid];
                    break;
                }
                if (it > o.maxI) {
                    st |= MEM_ST_MAXITER;
                    break;
                }
                // ---- BackTrackingLineSearch / ArmijoCondition (Algorithm 1)
                // for the next pass; trial coefficients P + alpha D.
                plane_coeffs<PPT>(sd, s_hy, s_hz, PS, npt, tid, cd);
                alpha = 2.f;
                bool sat = false;
                float Lt = Lcur;
                for (int s_ = 0; !sat && s_ <= o.maxT; ++s_) {
                    alpha *= 0.5f;
#pragma unroll
                    for (int r = 0; r < PPT; ++r)
#pragma unroll
                        for (int a = 0; a < 5; ++a) ca[r][a] = fmaf(alpha, cd[r][a], cb[r][a]);
                    const float lz = sweep_store<PPT, 9>(ca, lwp, s_hx, s_lwx, nx, s_T, PS, npt, red, tid, warp, lane, mxc);
                    Lt = lz - (mb + alpha * md);
                    const float LD = Lcur - Lt, gradD = -o.c_armijo * alpha * gd;
                    sat = (LD - gradD) >= -(o.atol + o.rtol * fabsf(LD));
                }
#pragma unroll
                for (int r = 0; r < PPT; ++r)
#pragma unroll
                    for (int a = 0; a < 5; ++a) cb[r][a] = ca[r][a];
                Lcur = Lt;
                mb += alpha * md;
                if (tid >= 1 && tid < NP) sb[tid] += alpha * sd[tid];
                __syncthreads();
            }
            __syncthreads();
            if (tid < NP) bc[tid] = tid ? sb[tid] : n;
            if (tid == 0) {
                if (A.status) A.status[cell] = st;
                if (A.cond) A.cond[cell] = sx[6] > 0.f ? sx[7] / sx[6] : 0.f;
                if (A.iters) A.iters[cell] = it;
            }
        }
        // ---- moments of degree <= 9 at the final beta (flux and speed)
        if (A.mu) {
            __syncthreads();
            plane_coeffs<PPT>(sb, s_hy, s_hz, PS, npt, tid, cb);
            sweep_store<PPT, 10>(cb, lwp, s_hx, s_lwx, nx, s_T, PS, npt, red, tid, warp, lane, mxc);
            __syncthreads();
            float *out = A.mu + cell * MEM_MU_STRIDE;
            plane_stage(220, s_T, s_hy, s_hz, PS, npt, s_abc, out, warp, lane);
            if (tid == 0) {
                // u_x range of the nodes: the speed bound when the pencil has
                // no reliable spectrum
                float el;
                ff_offset(axh, axl, hxh, hxl, xt[0], 0.f, out[220], el);
                ff_offset(axh, axl, hxh, hxl, xt[nx - 1], 0.f, out[221], el);
            }
        }
    }
}

template <int PPT>
int launch_vel(mem_ctx *ctx, const VelArgs &a, cudaStream_t st) {
    const size_t smem = sizeof(float) * (size_t)vel_layout(a.nx, a.npt).total;
    if (smem > 227 * 1024) return MEM_EINVAL;
    MEM_CUDA_TRY(cudaFuncSetAttribute(k_vel<PPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int sms = 0, per_sm = 0;
    MEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    MEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_vel<PPT>, VT, smem));
    if (per_sm < 1) return MEM_ECUDA;
    const int grid = (int)std::min<int64_t>(a.B, (int64_t)sms * per_sm);
    k_vel<PPT><<<grid, VT, smem, st>>>(a);
    MEM_CUDA_TRY(cudaGetLastError());
    return MEM_OK;
}

}  // namespace

namespace mem_host {

void dom_record(double ax, double bx, double br, int nbx, int nbr, float *rec) {
    auto split = [](double v, float *hl) {
        hl[0] = (float)v;
        hl[1] = (float)(v - (double)hl[0]);
    };
    const double hx = (bx - ax) / nbx, hr = br / nbr;
    split(ax, rec);
    split(hx, rec + 2);
    split(hr, rec + 4);
    rec[6] = rec[7] = 0.f;
}

size_t vel_smem_bytes(int nx, int npt) { return sizeof(float) * (size_t)vel_layout(nx, npt).total; }

int vel_run(mem_ctx *ctx, const float *M, float *beta, const float *g, int32_t *status, int32_t *iters, float *mu,
            const int *pid, const float *dom, int64_t B, const mem_solve_opts &o, bool solve, cudaStream_t st,
            const unsigned char *active, float *cond) {
    if (!ctx->vel) return MEM_EINVAL;
    if (B == 0) return MEM_OK;
    VelArgs a;
    a.M = M; a.beta = beta; a.gauge = g; a.status = status; a.iters = iters; a.mu = mu; a.cond = cond;
    a.pid = pid; a.dom = dom ? dom : ctx->d_dom0; a.active = active;
    a.vt2 = ctx->d_vt2; a.vtf = ctx->d_vtf;
    a.slots = ctx->d_hess_slots128; a.n_slots = ctx->n_hess_slots128;
    a.B = B;
    a.nbx = ctx->nbx; a.nbr = ctx->nbr; a.ng = ctx->ng; a.K = ctx->K;
    a.nx = ctx->nx; a.npt = ctx->npt; a.PS = plane_stride(ctx->npt);
    a.solve = solve ? 1 : 0;
    a.o = o;
    const int ppt = (ctx->npt + VT - 1) / VT;
    if (ppt <= 2) return launch_vel<2>(ctx, a, st);
    if (ppt <= 3) return launch_vel<3>(ctx, a, st);
    if (ppt <= 4) return launch_vel<4>(ctx, a, st);
    if (ppt <= 8) return launch_vel<8>(ctx, a, st);
    return MEM_EINVAL;
}

}  // namespace mem_host

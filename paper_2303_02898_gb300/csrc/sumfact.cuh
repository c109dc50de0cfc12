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
    // per-warp floats: beta, dbeta, M/n, grad, Cholesky broadcast column,
    // mu(165) + work; a multiple of 4 so that every warp's area (and the
    // 16-byte vector accesses of the broadcast column) stays aligned
    static constexpr int WARP_FLOATS = ((5 * 36 + 168 + WORK + 3) / 4) * 4;
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

// Eight right-looking Cholesky steps k = K0 .. K0+7 on the register columns
// (see reg_chol_solve34).  Rows i <= K0 are finished before the block starts,
// so the row loop runs statically over K0+1 .. 33.  bc is a per-warp,
// 16-byte-aligned scratch of 36 floats for the pivot column.  No row or lane
// is masked:
// lanes j <= k multiply by a zero coefficient (fma(-a, 0, x) == x), and in
// the live columns j > k the rows i <= k hold entries that were consumed at
// step i and are never read again (the factor and both triangular solves
// read rows i >= j only), so one shuffle and one FMA per element suffice.
// PIV = true takes each lane's A_kj, the pivot and the pivot lane's
// forward-solve value from the published column (fewer instructions; A_kj is
// the pivot lane's copy of the entry, which differs from the lane's own copy
// by rounding).  PIV = false selects the lane's own A_kj from its registers
// and shuffles the pivot: the form for the stiffest systems, whose FP32
// solves sit at the rounding floor.
template <int K0, bool PIV>
__device__ __forceinline__ bool chol_block8(float (&col)[NP1], float &t00, float &t10, float &t11, float &bb,
                                            float &b32, float &b33, float &myinv, float &myw, int lane,
                                            float *bc) {
    constexpr int I0 = ((K0 + 1) / 4) * 4;  // first 16-byte group holding a live row
#pragma unroll 1
    for (int kk = 0; kk < 8; ++kk) {
        const int k = K0 + kk;
        // The pivot lane publishes its column (rows I0..33) with 16-byte
        // stores, and its forward-solve value in slot 34; every lane reads
        // the column back with broadcast loads (about a quarter of the
        // memory-pipe instructions of one shuffle per row).  By symmetry the
        // column also holds each lane's own A_kj in row j and the pivot in
        // row k.  Lanes below I0 read stale rows, but they are finished and
        // their coefficient is zero.
        float ck, d, wk0;
        if (!PIV) {
            float s1[4], s2[2];
#pragma unroll
            for (int m = 0; m < 4; ++m) s1[m] = (kk & 1) ? col[K0 + 2 * m + 1] : col[K0 + 2 * m];
#pragma unroll
            for (int m = 0; m < 2; ++m) s2[m] = (kk & 2) ? s1[2 * m + 1] : s1[2 * m];
            ck = (kk & 4) ? s2[1] : s2[0];  // this lane's own A_kj
            d = __shfl_sync(0xffffffffu, ck, k);
            wk0 = __shfl_sync(0xffffffffu, bb, k);
        }
        __syncwarp();  // the previous step's column has been read
        if (lane == k) {
#pragma unroll
            for (int i = I0; i < 32; i += 4)
                *reinterpret_cast<float4 *>(bc + i) = make_float4(col[i], col[i + 1], col[i + 2], col[i + 3]);
            *reinterpret_cast<float2 *>(bc + 32) = make_float2(col[32], col[33]);
            if (PIV) bc[34] = bb;
        }
        __syncwarp();
        if (PIV) {
            d = bc[k];
            ck = bc[lane];  // the pivot lane's copy of A_kj
            wk0 = bc[34];
        }
        if (!(d > 0.f) || !isfinite(d)) return false;
        const float inv = rsqrtf(d), inv2 = inv * inv;
        const float c = ck * inv2;
        const float wk = wk0 * inv;
        const bool upd = lane > k;
        const float cm = upd ? c : 0.f;
#pragma unroll
        for (int i = I0; i < 32; i += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(bc + i);
            if (i + 0 > K0) col[i + 0] = fmaf(-v.x, cm, col[i + 0]);
            if (i + 1 > K0) col[i + 1] = fmaf(-v.y, cm, col[i + 1]);
            if (i + 2 > K0) col[i + 2] = fmaf(-v.z, cm, col[i + 2]);
            if (i + 3 > K0) col[i + 3] = fmaf(-v.w, cm, col[i + 3]);
        }
        const float2 v2 = *reinterpret_cast<const float2 *>(bc + 32);
        const float r32 = v2.x, r33 = v2.y;
        col[32] = fmaf(-r32, cm, col[32]);
        col[33] = fmaf(-r33, cm, col[33]);
        if (upd) bb = fmaf(-ck * inv, wk, bb);
        b32 = fmaf(-r32 * inv, wk, b32);
        b33 = fmaf(-r33 * inv, wk, b33);
        t00 = fmaf(-r32 * r32, inv2, t00);
        t10 = fmaf(-r33 * r32, inv2, t10);
        t11 = fmaf(-r33 * r33, inv2, t11);
        if (lane == k) { myinv = inv; myw = wk; }
    }
    return true;
}

// Register-resident Cholesky H = L L^T of the 34 x 34 SPD matrix whose lower
// triangle is in shared memory (row-major, leading dimension LDH), written
// back as L (lower triangle).  Same column-per-lane scheme as the solver's
// factorisation (chol_block8); returns false, uniformly, on a pivot that is
// not positive and finite.
__device__ __forceinline__ bool reg_cholesky34_store(float *Hs, int lane, float *bc) {
    constexpr bool PIV = false;
    float col[NP1];
#pragma unroll
    for (int i = 0; i < NP1; ++i) {
        const int r = i > lane ? i : lane, c = i > lane ? lane : i;
        col[i] = Hs[r * LDH + c];
    }
    float t00 = Hs[32 * LDH + 32], t10 = Hs[33 * LDH + 32], t11 = Hs[33 * LDH + 33];
    float bb = 0.f, b32 = 0.f, b33 = 0.f, myinv = 1.f, myw = 0.f;
    if (!chol_block8<0, PIV>(col, t00, t10, t11, bb, b32, b33, myinv, myw, lane, bc)) return false;
    if (!chol_block8<8, PIV>(col, t00, t10, t11, bb, b32, b33, myinv, myw, lane, bc)) return false;
    if (!chol_block8<16, PIV>(col, t00, t10, t11, bb, b32, b33, myinv, myw, lane, bc)) return false;
    if (!chol_block8<24, PIV>(col, t00, t10, t11, bb, b32, b33, myinv, myw, lane, bc)) return false;
    if (!(t00 > 0.f) || !isfinite(t00)) return false;
    const float l32 = sqrtf(t00), l3332 = t10 / l32, d33 = t11 - l3332 * l3332;
    if (!(d33 > 0.f) || !isfinite(d33)) return false;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < NP1; ++i)
        if (i >= lane) Hs[i * LDH + lane] = (i == lane) ? 1.f / myinv : col[i] * myinv;
    if (lane == 0) {
        Hs[32 * LDH + 32] = l32;
        Hs[33 * LDH + 32] = l3332;
        Hs[33 * LDH + 33] = sqrtf(d33);
    }
    __syncwarp();
    return true;
}

// Solve (H + lam I) x = rhs by a register-resident Cholesky factorisation,
// H the 34 x 34 SPD matrix whose lower triangle is in shared memory
// (row-major, leading dimension LDH).  Lane j < 32 holds column j of the
// symmetric matrix (all 34 rows) in registers; rows/columns 32 and 33 (the
// trailing 2 x 2 block) and rhs/x entries 32, 33 are carried, identical, by
// every lane; entry i < 32 of rhs and x lives on lane i.
// Right-looking factorisation: in step k lane j takes its own A_kj (= A_jk,
// the matrix is kept symmetric), the pivot d = A_kk comes from lane k, and
// every lane j > k applies A_ij -= A_ik A_jk / A_kk for i > k with A_ik
// broadcast from lane k.  The forward solve L w = rhs rides along (lane i > k
// subtracts L_ik w_k, L_ik = A_ik / l_k being its own register), and the
// backward solve L^T x = w broadcasts one x_i per step.  Returns false,
// uniformly, when a pivot is not positive and finite (the "failed
// decomposition" of Algorithm 1).  bc: per-warp 16-byte-aligned scratch of
// 36 floats (the broadcast pivot column).  prange (optional, uniform across
// the warp): receives the smallest and largest pivot.
template <bool PIV>
__device__ __forceinline__ bool reg_chol_solve34(const float *Hs, float lam, int lane, float rhs, float rhs32,
                                                 float rhs33, float &x, float &x32, float &x33, float *bc,
                                                 float *prange = nullptr) {
    float col[NP1];
#pragma unroll
    for (int i = 0; i < NP1; ++i) {
        const int r = i > lane ? i : lane, c = i > lane ? lane : i;
        float v = Hs[r * LDH + c];
        if (i == lane) v += lam;
        col[i] = v;
    }
    float t00 = Hs[32 * LDH + 32] + lam, t10 = Hs[33 * LDH + 32], t11 = Hs[33 * LDH + 33] + lam;
    float bb = rhs, b32 = rhs32, b33 = rhs33;
    float myinv = 0.f, myw = 0.f;
    if (!chol_block8<0, PIV>(col, t00, t10, t11, bb, b32, b33, myinv, myw, lane, bc)) return false;
    if (!chol_block8<8, PIV>(col, t00, t10, t11, bb, b32, b33, myinv, myw, lane, bc)) return false;
    if (!chol_block8<16, PIV>(col, t00, t10, t11, bb, b32, b33, myinv, myw, lane, bc)) return false;
    if (!chol_block8<24, PIV>(col, t00, t10, t11, bb, b32, b33, myinv, myw, lane, bc)) return false;
    if (!(t00 > 0.f) || !isfinite(t00)) return false;
    const float inv32 = rsqrtf(t00), l3332 = t10 * inv32, d33 = t11 - l3332 * l3332;
    if (!(d33 > 0.f) || !isfinite(d33)) return false;
    const float inv33 = rsqrtf(d33);
    if (prange) {
        // smallest and largest Cholesky pivot d_k = L_kk^2 (k < 32 on lane k,
        // then t00 and d33): their ratio bounds cond(H + lam I) from below
        const float dk = 1.f / (myinv * myinv);
        const float pmn = fminf(warp_min(dk), fminf(t00, d33)), pmx = fmaxf(warp_max(dk), fmaxf(t00, d33));
        if (lane == 0) { prange[0] = pmn; prange[1] = pmx; }
    }
    const float w32 = b32 * inv32, w33 = (b33 - l3332 * w32) * inv33;
    x33 = w33 * inv33;
    x32 = (w32 - l3332 * x33) * inv32;
    // lane j: x_j = (w_j - inv_j sum_{i>j} A_ij x_i) inv_j, with A_ij its own column
    float acc = fmaf(col[32], x32, col[33] * x33);
#pragma unroll
    for (int i = 31; i >= 0; --i) {
        const float xi = __shfl_sync(0xffffffffu, (myw - myinv * acc) * myinv, i);
        if (lane == i) x = xi;
        if (lane < i) acc = fmaf(col[i], xi, acc);
    }
    return true;
}

}  // namespace mem

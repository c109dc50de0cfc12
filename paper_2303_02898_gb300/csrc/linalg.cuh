// linalg.cuh -- warp-cooperative dense linear algebra on small matrices held
// in shared memory (one warp per cell).  All loops are bounded; nothing waits
// on another warp.
#pragma once

#include "common.cuh"

namespace mem {

// In-place Cholesky A = L L^T of the n x n symmetric matrix in shared memory
// (row-major, leading dimension ld; only the lower triangle is read or
// written).  Right-looking; lane l owns rows i with (i - k - 1) % 32 == l in
// step k.  Returns false (uniformly across the warp) if a pivot is not
// positive and finite -- the "failed decomposition" of Algorithm 1.
__device__ __forceinline__ bool warp_cholesky(float *A, int n, int ld, int lane) {
    for (int k = 0; k < n; ++k) {
        __syncwarp();
        const float d = A[k * ld + k];
        if (!(d > 0.f) || !isfinite(d)) return false;
        const float l = sqrtf(d), inv = 1.f / l;
        __syncwarp();
        for (int i = k + 1 + lane; i < n; i += 32) A[i * ld + k] *= inv;
        if (lane == 0) A[k * ld + k] = l;
        __syncwarp();
        for (int i = k + 1 + lane; i < n; i += 32) {
            const float lik = A[i * ld + k];
            for (int j = k + 1; j <= i; ++j) A[i * ld + j] -= lik * A[j * ld + k];
        }
    }
    __syncwarp();
    return true;
}

// Solve L x = b (forward) in place on b (shared, length n).
__device__ __forceinline__ void warp_solve_lower(const float *L, int n, int ld, float *b, int lane) {
    for (int k = 0; k < n; ++k) {
        __syncwarp();
        const float xk = b[k] / L[k * ld + k];
        __syncwarp();
        if (lane == 0) b[k] = xk;
        for (int i = k + 1 + lane; i < n; i += 32) b[i] -= L[i * ld + k] * xk;
    }
    __syncwarp();
}

// Solve L^T x = b (backward) in place on b.
__device__ __forceinline__ void warp_solve_upperT(const float *L, int n, int ld, float *b, int lane) {
    for (int k = n - 1; k >= 0; --k) {
        __syncwarp();
        const float xk = b[k] / L[k * ld + k];
        __syncwarp();
        if (lane == 0) b[k] = xk;
        for (int i = lane; i < k; i += 32) b[i] -= L[k * ld + i] * xk;
    }
    __syncwarp();
}

// Number of eigenvalues below x of the symmetric tridiagonal matrix with
// diagonal a[0..m) and off-diagonal b[0..m-1) (Sturm sequence).
__device__ __forceinline__ int sturm_count(const float *a, const float *b, int m, float x) {
    int cnt = 0;
    float q = 1.f;
    for (int i = 0; i < m; ++i) {
        const float bb = i ? b[i - 1] * b[i - 1] : 0.f;
        q = a[i] - x - (i ? __fdividef(bb, q) : 0.f);
        if (fabsf(q) < 1e-20f) q = -1e-20f;
        cnt += q < 0.f;
    }
    return cnt;
}

// Smallest (want_max = false) or largest eigenvalue of the tridiagonal matrix
// by 32-way multisection over Gershgorin bounds (every lane evaluates one
// Sturm count per round).
__device__ __forceinline__ float warp_tridiag_extreme(const float *a, const float *b, int m, bool want_max, int lane) {
    float lo = a[0], hi = a[0];
    for (int i = 0; i < m; ++i) {
        const float r = (i ? fabsf(b[i - 1]) : 0.f) + (i + 1 < m ? fabsf(b[i]) : 0.f);
        lo = fminf(lo, a[i] - r);
        hi = fmaxf(hi, a[i] + r);
    }
    const float span = fmaxf(hi - lo, 1e-30f);
    lo -= 1e-6f * span;
    hi += 1e-6f * span;
    const int target = want_max ? m - 1 : 0;  // eigenvalue number (0-based)
    for (int round = 0; round < 8; ++round) {
        const float h = (hi - lo) / 32.f;
        const float x = lo + h * (float)(lane + 1);
        const int c = sturm_count(a, b, m, x);
        // first lane whose point has more than `target` eigenvalues below it
        const unsigned ball = __ballot_sync(0xffffffffu, c > target);
        const int first = ball ? __ffs(ball) - 1 : 31;
        const float nlo = lo + h * (float)first;
        hi = lo + h * (float)(first + 1);
        lo = nlo;
        if (hi - lo <= 1e-7f * fmaxf(fabsf(lo), fabsf(hi)) + 1e-30f) break;
    }
    return 0.5f * (lo + hi);
}

// Extreme generalised eigenvalues of one small symmetric-definite pencil
// (X, S), n <= 16, lower triangles in shared memory with leading dimension
// 16: Cholesky S = L L^T (in place), C = L^{-1} X L^{-T} by right-looking
// column solves (lane j < n owns column j) and a pairwise transpose, Lanczos
// without re-orthogonalisation and Sturm multisection.  Returns false if S
// is not numerically positive definite.  Not inlined: the axisymmetric speed
// calls it three times, and three inlined copies overflow the instruction
// cache once many warps are resident.
static __device__ __noinline__ bool small_pencil_extremes(float *S, float *X, int n, float *al, float *bt, float *sv,
                                                      int lane, float &lo, float &hi) {
    constexpr int LD = 16;
    // Lane j < n owns column j throughout (no index decoding): it mirrors,
    // transposes and symmetrises the pairs (i, j), i > j.
    if (lane < n)
        for (int i = lane + 1; i < n; ++i) X[lane * LD + i] = X[i * LD + lane];  // mirror X
    __syncwarp();
    if (!warp_cholesky(S, n, LD, lane)) return false;
    if (lane < n) sv[lane] = 1.f / S[lane * LD + lane];  // 1 / L_kk (sv is free until Lanczos)
    __syncwarp();
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            if (lane < n)
                for (int i = lane + 1; i < n; ++i) {
                    const float t = X[i * LD + lane];
                    X[i * LD + lane] = X[lane * LD + i];
                    X[lane * LD + i] = t;
                }
            __syncwarp();
        }
        if (lane < n) {
            for (int k = 0; k < n; ++k) {
                const float yk = X[k * LD + lane] * sv[k];
                X[k * LD + lane] = yk;
                for (int i = k + 1; i < n; ++i) X[i * LD + lane] -= S[i * LD + k] * yk;
            }
        }
        __syncwarp();
    }
    // symmetrise C (in X) and run Lanczos (lane i < n holds v_i)
    if (lane < n)
        for (int i = lane + 1; i < n; ++i) {
            const float sy = 0.5f * (X[i * LD + lane] + X[lane * LD + i]);
            X[i * LD + lane] = sy;
            X[lane * LD + i] = sy;
        }
    __syncwarp();
    float cn = 0.f;
    if (lane < n)
        for (int i = 0; i < n; ++i) cn = fmaxf(cn, fabsf(X[i * LD + lane]));
    const float cnorm = warp_max(cn) + 1e-30f;
    __syncwarp();
    float v = lane < n ? rsqrtf((float)n) : 0.f, vp = 0.f, bprev = 0.f;
    int m = 0;
    for (int k = 0; k < n; ++k) {
        sv[lane] = v;
        __syncwarp();
        float w = 0.f;
        if (lane < n)
            for (int j = 0; j < n; ++j) w += X[j * LD + lane] * sv[j];
        __syncwarp();
        w -= bprev * vp;
        const float a = warp_sum(w * v);
        w -= a * v;
        if (lane == 0) al[k] = a;
        const float bk = sqrtf(warp_sum(w * w));
        m = k + 1;
        if (k + 1 == n || bk <= 1e-6f * cnorm) break;
        if (lane == 0) bt[k] = bk;
        vp = v;
        v = w / bk;
        bprev = bk;
    }
    __syncwarp();
    hi = warp_tridiag_extreme(al, bt, m, true, lane);
    lo = warp_tridiag_extreme(al, bt, m, false, lane);
    __syncwarp();
    return true;
}

}  // namespace mem

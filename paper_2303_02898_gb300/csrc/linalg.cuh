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

}  // namespace mem

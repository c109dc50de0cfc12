// targets.cu -- synthetic solve targets (workload generator, not part of the
// paper's method).  Per cell: the density p(c) ~ exp(-|c|^2/2 + sum_k a_k c^k
// - sum_k b_k c^k), c = (u - v)/sqrt(T), n = 1; a Gauss-Hermite rule of
// gen_order^3 nodes is re-centred on the density in four passes (mean and
// standard deviation per axis), and the last pass gives the density's
// Hermite gauge and its 35 moments there.  One block per cell.
#include <vector>

#include "common.cuh"
#include "ctx.h"

using namespace mem;

namespace {

struct GenRule {
    int n;
    float x[32];
    float lw[32];
};

constexpr int TB = 256;

__device__ __forceinline__ float block_sum(float v, float *red) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = threadIdx.x < TB / 32 ? red[threadIdx.x] : 0.f;
    if (threadIdx.x < 32) r = warp_sum(r);
    if (threadIdx.x == 0) red[0] = r;
    __syncthreads();
    return red[0];
}
__device__ __forceinline__ float block_max(float v, float *red) {
    v = warp_max(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = threadIdx.x < TB / 32 ? red[threadIdx.x] : -INFINITY;
    if (threadIdx.x < 32) r = warp_max(r);
    if (threadIdx.x == 0) red[0] = r;
    __syncthreads();
    return red[0];
}

__device__ __forceinline__ float log_density(const float c[3], const float *a, const float *b) {
    const float x = c[0], y = c[1], z = c[2];
    // degree-3 monomials in statistic order (3,0,0) (2,1,0) (2,0,1) (1,2,0)
    // (1,1,1) (1,0,2) (0,3,0) (0,2,1) (0,1,2) (0,0,3)
    const float cub = a[0] * x * x * x + a[1] * x * x * y + a[2] * x * x * z + a[3] * x * y * y + a[4] * x * y * z +
                      a[5] * x * z * z + a[6] * y * y * y + a[7] * y * y * z + a[8] * y * z * z + a[9] * z * z * z;
    const float x2 = x * x, y2 = y * y, z2 = z * z;
    const float qua = b[0] * x2 * x2 + b[1] * y2 * y2 + b[2] * z2 * z2 + b[3] * x2 * y2 + b[4] * x2 * z2 + b[5] * y2 * z2;
    return -0.5f * (x2 + y2 + z2) + cub - qua;
}

__global__ void __launch_bounds__(TB) k_targets(GenRule R, const float *__restrict__ v, const float *__restrict__ T,
                                                const float *__restrict__ a, const float *__restrict__ b,
                                                float *__restrict__ M_out, float *__restrict__ g_out) {
    __shared__ float red[32], sa[10], sb[6], sacc[NP][TB / 32];
    const int64_t cell = blockIdx.x;
    const int tid = threadIdx.x;
    if (tid < 10) sa[tid] = a[cell * 10 + tid];
    if (tid < 6) sb[tid] = b[cell * 6 + tid];
    __syncthreads();
    const int n = R.n, Q = n * n * n;
    float mu[3] = {0.f, 0.f, 0.f}, sc[3] = {1.f, 1.f, 1.f};
    for (int pass = 0; pass < 4; ++pass) {
        float mx = -INFINITY;
        for (int q = tid; q < Q; q += TB) {
            const int i = q / (n * n), j = (q / n) % n, k = q % n;
            const float zz[3] = {R.x[i], R.x[j], R.x[k]};
            float c[3];
            for (int d = 0; d < 3; ++d) c[d] = mu[d] + sc[d] * zz[d];
            const float e = R.lw[i] + R.lw[j] + R.lw[k] + 0.5f * (zz[0] * zz[0] + zz[1] * zz[1] + zz[2] * zz[2]) + log_density(c, sa, sb);
            mx = fmaxf(mx, e);
        }
        mx = block_max(mx, red);
        float z0 = 0.f, m1[3] = {0.f, 0.f, 0.f}, m2[3] = {0.f, 0.f, 0.f};
        for (int q = tid; q < Q; q += TB) {
            const int i = q / (n * n), j = (q / n) % n, k = q % n;
            const float zz[3] = {R.x[i], R.x[j], R.x[k]};
            float c[3];
            for (int d = 0; d < 3; ++d) c[d] = mu[d] + sc[d] * zz[d];
            const float e = R.lw[i] + R.lw[j] + R.lw[k] + 0.5f * (zz[0] * zz[0] + zz[1] * zz[1] + zz[2] * zz[2]) + log_density(c, sa, sb);
            const float p = __expf(e - mx);
            z0 += p;
            for (int d = 0; d < 3; ++d) { m1[d] += p * zz[d]; m2[d] += p * zz[d] * zz[d]; }
        }
        const float Z = block_sum(z0, red);
        float mz[3], vz[3];
        for (int d = 0; d < 3; ++d) mz[d] = block_sum(m1[d], red) / Z;
        for (int d = 0; d < 3; ++d) vz[d] = block_sum(m2[d], red) / Z - mz[d] * mz[d];
        // mean and std of c in the current frame
        float mean_c[3], sd_c[3];
        for (int d = 0; d < 3; ++d) { mean_c[d] = mu[d] + sc[d] * mz[d]; sd_c[d] = sc[d] * sqrtf(fmaxf(vz[d], 1e-30f)); }
        if (pass == 3) {
            // Hermite gauge of u = v + sqrt(T) c and the moments there.
            const float sT = sqrtf(T[cell]);
            float gh[6];
            for (int d = 0; d < 3; ++d) { gh[d] = v[cell * 3 + d] + sT * mean_c[d]; gh[3 + d] = sT * sd_c[d]; }
            float acc[NP];
            for (int k = 0; k < NP; ++k) acc[k] = 0.f;
            for (int q = tid; q < Q; q += TB) {
                const int i = q / (n * n), j = (q / n) % n, k = q % n;
                const float zz[3] = {R.x[i], R.x[j], R.x[k]};
                float c[3], ub[3];
                for (int d = 0; d < 3; ++d) { c[d] = mu[d] + sc[d] * zz[d]; ub[d] = (c[d] - mean_c[d]) / sd_c[d]; }
                const float e = R.lw[i] + R.lw[j] + R.lw[k] + 0.5f * (zz[0] * zz[0] + zz[1] * zz[1] + zz[2] * zz[2]) + log_density(c, sa, sb);
                const float p = __expf(e - mx) / Z;
                float hx[5], hy[5], hz[5];
                hermite_vals<4>(ub[0], hx);
                hermite_vals<4>(ub[1], hy);
                hermite_vals<4>(ub[2], hz);
#pragma unroll
                for (int kk = 0; kk < NP; ++kk) acc[kk] += p * hx[exp_a(kk)] * hy[exp_b(kk)] * hz[exp_c(kk)];
            }
#pragma unroll
            for (int kk = 0; kk < NP; ++kk) {
                float s = warp_sum(acc[kk]);
                if ((tid & 31) == 0) sacc[kk][tid >> 5] = s;
            }
            __syncthreads();
            if (tid < NP) {
                float s = 0.f;
                for (int w = 0; w < TB / 32; ++w) s += sacc[tid][w];
                M_out[cell * NP + tid] = tid ? s : 1.f;
            }
            if (tid < 6) g_out[cell * 6 + tid] = gh[tid];
        }
        for (int d = 0; d < 3; ++d) { mu[d] = mean_c[d]; sc[d] = sd_c[d]; }
    }
}

}  // namespace

namespace mem_host {

int targets(mem_ctx *, int gen_order, const float *v, const float *T, const float *a, const float *b, float *M_out,
            float *g_out, int64_t B, cudaStream_t st) {
    std::vector<double> x, w;
    int rc = gh_rule(gen_order, x, w);
    if (rc) return rc;
    GenRule R;
    R.n = gen_order;
    for (int i = 0; i < gen_order; ++i) { R.x[i] = (float)x[i]; R.lw[i] = (float)log(w[i]); }
    for (int64_t c0 = 0; c0 < B; c0 += (1 << 30)) {
        const int64_t n = std::min<int64_t>(B - c0, 1 << 30);
        k_targets<<<(unsigned)n, TB, 0, st>>>(R, v + c0 * 3, T + c0, a + c0 * 10, b + c0 * 6, M_out + c0 * NP, g_out + c0 * 6);
    }
    MEM_CUDA_TRY(cudaGetLastError());
    return MEM_OK;
}

}  // namespace mem_host

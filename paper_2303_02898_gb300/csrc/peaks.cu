// peaks.cu -- micro-benchmarks of the GB300 pipes the method's kernels use
// (FP32 FMA, the MUFU exp2 unit, tcgen05 tensor-core MMAs in BF16 and TF32)
// and a self-test of the tcgen05 operand and accumulator layouts.
//
// The roofline fractions reported for the library's kernels divide by these
// measured rates.  Every loop is bounded; the only wait (an mbarrier that the
// tensor cores arrive on) gives up after a fixed number of polls and reports
// the failure through the return code.
#include <cuda_bf16.h>

#include "common.cuh"
#include "ctx.h"
#include "tc.cuh"
#include "tmap.h"

namespace {

using namespace mem;

constexpr uint32_t kMaxPolls = 1u << 22;

// 8 independent FMA chains per thread.
__global__ void __launch_bounds__(512) k_fma_peak(int iters, float *out) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 1.0f + 1e-3f * (threadIdx.x + j);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], 0.999999f, 1e-6f);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == 12345.f) out[blockIdx.x] = s;  // never true; keeps the chains live
}

// 8 independent ex2.approx chains per thread (the multiplication that keeps
// the argument in range runs on the FMA pipe).
__global__ void __launch_bounds__(512) k_mufu_peak(int iters, float *out) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = -0.4f - 1e-4f * (threadIdx.x + j);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float y;
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[j]));
                x[j] = -0.5f * y;
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == 12345.f) out[blockIdx.x] = s;
}

__device__ __forceinline__ float hash_val(uint32_t i) {
    i ^= i >> 16;
    i *= 0x7feb352dU;
    i ^= i >> 15;
    i *= 0x846ca68bU;
    i ^= i >> 16;
    return (float)(i & 0xFFFF) * (1.0f / 65536.0f) - 0.5f;
}

// One CTA per SM: A [128 x 128 bytes of K], B [256 x 128 bytes of K] in
// shared memory, D [128 x 256] FP32 in TMEM; the elected thread issues
// 4 iters MMAs of 128 x 256 x (32 bytes of K) back to back.
template <int AB>  // 1 = BF16, 2 = TF32
__global__ void __launch_bounds__(128, 1) k_tc_peak(int iters, float *out, int *err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar;
    constexpr int SZ = AB == 1 ? 2 : 4, KE = 128 / SZ;  // K elements per row
    uint8_t *A = smem, *B = smem + 128 * 128;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, 256);
        tc::tmem_relinquish();
    }
    if (tid == 0) tc::mbar_init(&s_bar, 1);
    for (int r = tid; r < 128 + 256; r += 128) {
        uint8_t *base = r < 128 ? A : B;
        const int rr = r < 128 ? r : r - 128;
        for (int k = 0; k < KE; ++k) {
            const float v = hash_val((uint32_t)(r * KE + k + 977 * blockIdx.x));
            const uint32_t off = tc::kmajor_off(rr, k, KE, SZ);
            if (AB == 1) *reinterpret_cast<__nv_bfloat16 *>(base + off) = __float2bfloat16(v);
            else *reinterpret_cast<float *>(base + off) = tc::to_tf32(v);
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    if (tid == 0) {
        const uint32_t sa = tc::smem_u32(A), sb = tc::smem_u32(B);
        constexpr uint32_t id = tc::idesc(128, 256, AB);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const uint64_t da = tc::sdesc(sa + 256 * s, 128, 128 * KE * SZ / 16);
                const uint64_t db = tc::sdesc(sb + 256 * s, 128, 128 * KE * SZ / 16);
                if (AB == 1) tc::mma_bf16(tmem, da, db, id, (it | s) != 0);
                else tc::mma_tf32(tmem, da, db, id, (it | s) != 0);
            }
        }
        tc::mma_commit(&s_bar);
    }
    __syncwarp();
    bool ok = tc::mbar_wait(&s_bar, 0, kMaxPolls);
    if (!ok) {
        // report, then give the MMAs in flight a second bounded window
        // before the accumulator's columns are released
        atomicExch(err, 1);
        tc::mbar_wait(&s_bar, 0, kMaxPolls);
    }
    ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
    tc::fence_after_sync();
    if (ok) {
        float v[8];
        tc::tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16), v);
        if (v[0] == 12345.f) out[blockIdx.x] = v[1];
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// D [128 x N] = A [128 x 64] . B [N x 64]^T through one CTA's tensor cores,
// operands converted to BF16 (AB = 1) or TF32 (AB = 2).
template <int AB>
__global__ void __launch_bounds__(128, 1) k_tc_selftest(const float *Ag, const float *Bg, float *Dg, int N,
                                                        int *err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar;
    constexpr int SZ = AB == 1 ? 2 : 4, K = 64;
    uint8_t *A = smem, *B = smem + 128 * K * SZ;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, 256);
        tc::tmem_relinquish();
    }
    if (tid == 0) tc::mbar_init(&s_bar, 1);
    for (int r = tid; r < 128 + N; r += 128) {
        const bool isA = r < 128;
        const int rr = isA ? r : r - 128;
        const float *src = isA ? Ag + (size_t)rr * K : Bg + (size_t)rr * K;
        uint8_t *base = isA ? A : B;
        for (int k = 0; k < K; ++k) {
            const uint32_t off = tc::kmajor_off(rr, k, K, SZ);
            if (AB == 1) *reinterpret_cast<__nv_bfloat16 *>(base + off) = __float2bfloat16(src[k]);
            else *reinterpret_cast<float *>(base + off) = tc::to_tf32(src[k]);
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    if (tid == 0) {
        const uint32_t sa = tc::smem_u32(A), sb = tc::smem_u32(B), id = tc::idesc(128, N, AB);
        for (int s = 0; s < K * SZ / 32; ++s) {
            const uint64_t da = tc::sdesc(sa + 256 * s, 128, 128 * K * SZ / 16);
            const uint64_t db = tc::sdesc(sb + 256 * s, 128, 128 * K * SZ / 16);
            if (AB == 1) tc::mma_bf16(tmem, da, db, id, s != 0);
            else tc::mma_tf32(tmem, da, db, id, s != 0);
        }
        tc::mma_commit(&s_bar);
    }
    __syncwarp();
    bool ok = tc::mbar_wait(&s_bar, 0, kMaxPolls);
    if (!ok) {
        // report, then give the MMAs in flight a second bounded window
        // before the accumulator's columns are released
        atomicExch(err, 1);
        tc::mbar_wait(&s_bar, 0, kMaxPolls);
    }
    ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
    tc::fence_after_sync();
    if (ok) {
        const int row = 32 * (warp & 3) + (tid & 31);
        for (int c = 0; c < N; c += 8) {
            float v[8];
            tc::tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int j = 0; j < 8; ++j) Dg[(size_t)row * N + c + j] = v[j];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// D [128 x N] = A [128 x 64] . B [N x 64]^T with TF32 operands brought in
// by TMA tensor loads (boxes of 32 columns, 128-byte swizzle) and read by
// the MMAs through swizzled descriptors: the layout of the mixed back-end's
// contraction.
__global__ void __launch_bounds__(128, 1) k_tc_selftest_tma(const __grid_constant__ CUtensorMap tA,
                                                            const __grid_constant__ CUtensorMap tB, float *Dg,
                                                            int N, int *err) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_load, s_bar;
    // the swizzled tiles start on a 1024-byte boundary
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5;
    uint8_t *A = smem, *B = smem + 2 * 16384;  // two K-chunks of 32 columns each
    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, 256);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&s_load, 1);
        tc::mbar_init(&s_bar, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t bbytes = (uint32_t)N * 128;
    if (tid == 0) {
        tc::mbar_expect_tx(&s_load, 2 * 16384 + 2 * bbytes);
        for (int kc = 0; kc < 2; ++kc) {
            tc::tma_load_2d(A + kc * 16384, &tA, 32 * kc, 0, &s_load);
            tc::tma_load_2d(B + kc * bbytes, &tB, 32 * kc, 0, &s_load);
        }
        bool ok = tc::mbar_wait(&s_load, 0, kMaxPolls);
        if (!ok) {
            atomicExch(err, 1);
            tc::mbar_wait(&s_load, 0, kMaxPolls);  // the copies land before the CTA may exit
        } else {
            const uint32_t sa = tc::smem_u32(A), sb = tc::smem_u32(B), id = tc::idesc(128, N, 2);
            for (int kc = 0; kc < 2; ++kc)
                for (int s = 0; s < 4; ++s)
                    tc::mma_tf32(tmem, tc::sdesc_sw128(sa + kc * 16384 + 32 * s, 1024),
                                 tc::sdesc_sw128(sb + kc * bbytes + 32 * s, 1024), id, (kc | s) != 0);
        }
        tc::mma_commit(&s_bar);
    }
    __syncwarp();
    bool ok = tc::mbar_wait(&s_bar, 0, kMaxPolls);
    if (!ok) {
        atomicExch(err, 1);
        tc::mbar_wait(&s_bar, 0, kMaxPolls);
    }
    ok = __all_sync(0xffffffffu, ok);
    tc::fence_after_sync();
    if (ok) {
        const int row = 32 * (warp & 3) + (tid & 31);
        for (int c = 0; c < N; c += 8) {
            float v[8];
            tc::tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int j = 0; j < 8; ++j) Dg[(size_t)row * N + c + j] = v[j];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

int sm_count(int dev) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

}  // namespace

extern "C" {

int mem_bench_peak(int kind, int64_t iters, double *seconds, double *work) {
    if (kind < 0 || kind > 3 || iters < 1 || iters > (1 << 24) || !seconds || !work) return MEM_EINVAL;
    int dev = 0;
    MEM_CUDA_TRY(cudaGetDevice(&dev));
    const int sms = sm_count(dev);
    if (sms < 1) return MEM_ECUDA;
    float *out = nullptr;
    int *err = nullptr;
    MEM_CUDA_TRY(cudaMalloc(&out, sizeof(float) * 4096));
    MEM_CUDA_TRY(cudaMalloc(&err, sizeof(int)));
    MEM_CUDA_TRY(cudaMemset(err, 0, sizeof(int)));
    cudaStream_t st;
    MEM_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    MEM_CUDA_TRY(cudaEventCreate(&e0));
    MEM_CUDA_TRY(cudaEventCreate(&e1));
    const size_t tc_smem = 200 * 1024;  // one CTA per SM
    if (kind >= 2) {
        MEM_CUDA_TRY(cudaFuncSetAttribute(k_tc_peak<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem));
        MEM_CUDA_TRY(cudaFuncSetAttribute(k_tc_peak<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem));
    }
    auto launch = [&](int n) {
        switch (kind) {
            case 0: k_fma_peak<<<sms * 4, 512, 0, st>>>(n, out); break;
            case 1: k_mufu_peak<<<sms * 4, 512, 0, st>>>(n, out); break;
            case 2: k_tc_peak<1><<<sms, 128, tc_smem, st>>>(n, out, err); break;
            default: k_tc_peak<2><<<sms, 128, tc_smem, st>>>(n, out, err); break;
        }
    };
    launch(1);  // warm-up
    MEM_CUDA_TRY(cudaEventRecord(e0, st));
    launch((int)iters);
    MEM_CUDA_TRY(cudaEventRecord(e1, st));
    MEM_CUDA_TRY(cudaEventSynchronize(e1));
    MEM_CUDA_TRY(cudaGetLastError());
    float ms = 0.f;
    MEM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    int herr = 0;
    MEM_CUDA_TRY(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(out);
    cudaFree(err);
    if (herr) return MEM_ECUDA;
    *seconds = ms * 1e-3;
    const double threads = (double)sms * 4 * 512;
    switch (kind) {
        case 0: *work = 2.0 * 8 * 16 * (double)iters * threads; break;        // flops
        case 1: *work = 8.0 * 8 * (double)iters * threads; break;             // exp2 evaluations
        case 2: *work = 2.0 * 128 * 256 * 16 * 4 * (double)iters * sms; break;  // flops, K = 16 per MMA
        default: *work = 2.0 * 128 * 256 * 8 * 4 * (double)iters * sms; break;  // flops, K = 8 per MMA
    }
    return MEM_OK;
}

int mem_tc_selftest(int kind, int N, const float *A_host, const float *B_host, float *D_host) {
    if (kind < 1 || kind > 3 || N < 16 || N > 256 || N % 16 || !A_host || !B_host || !D_host) return MEM_EINVAL;
    float *A = nullptr, *B = nullptr, *D = nullptr;
    int *err = nullptr;
    MEM_CUDA_TRY(cudaMalloc(&A, sizeof(float) * 128 * 64));
    MEM_CUDA_TRY(cudaMalloc(&B, sizeof(float) * N * 64));
    MEM_CUDA_TRY(cudaMalloc(&D, sizeof(float) * 128 * N));
    MEM_CUDA_TRY(cudaMalloc(&err, sizeof(int)));
    MEM_CUDA_TRY(cudaMemset(err, 0, sizeof(int)));
    MEM_CUDA_TRY(cudaMemcpy(A, A_host, sizeof(float) * 128 * 64, cudaMemcpyHostToDevice));
    MEM_CUDA_TRY(cudaMemcpy(B, B_host, sizeof(float) * N * 64, cudaMemcpyHostToDevice));
    const size_t smem = (size_t)(128 + 256) * 64 * 4;
    if (kind == 3) {
        CUtensorMap tA, tB;
        int rc = mem_host::encode_tmap_2d_f32(&tA, A, 64, 128, 32, 128);
        if (!rc) rc = mem_host::encode_tmap_2d_f32(&tB, B, 64, (uint64_t)N, 32, (uint32_t)N);
        if (rc) {
            cudaFree(A); cudaFree(B); cudaFree(D); cudaFree(err);
            return rc;
        }
        const size_t sm3 = 2 * 16384 + 2 * (size_t)N * 128 + 1024;
        MEM_CUDA_TRY(cudaFuncSetAttribute(k_tc_selftest_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
        k_tc_selftest_tma<<<1, 128, sm3>>>(tA, tB, D, N, err);
    } else if (kind == 1) {
        MEM_CUDA_TRY(cudaFuncSetAttribute(k_tc_selftest<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_tc_selftest<1><<<1, 128, smem>>>(A, B, D, N, err);
    } else {
        MEM_CUDA_TRY(cudaFuncSetAttribute(k_tc_selftest<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_tc_selftest<2><<<1, 128, smem>>>(A, B, D, N, err);
    }
    MEM_CUDA_TRY(cudaDeviceSynchronize());
    int herr = 0;
    MEM_CUDA_TRY(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    MEM_CUDA_TRY(cudaMemcpy(D_host, D, sizeof(float) * 128 * N, cudaMemcpyDeviceToHost));
    cudaFree(A);
    cudaFree(B);
    cudaFree(D);
    cudaFree(err);
    return herr ? MEM_ECUDA : MEM_OK;
}

}  // extern "C"

// mixed.cu -- the tensor-core contraction of the mixed-precision back-end:
// the moment and Hessian sums of Section 3.1 / Appendix C,
//     E[phi_k]          = sum_q sigma_q phi_k(ubar_q)          (35 columns)
//     E[phi_i phi_j]    = sum_q sigma_q phi_i phi_j (ubar_q)   (595 columns)
// as one GEMM [cells x Q] . [Q x 630] on tcgen05 tensor cores.  The moments
// feed the gradient, so they use split TF32 (sigma = hi + lo, phi = hi + lo;
// hi.hi + hi.lo + lo.hi, FP32 accumulation: about FP32 accuracy); the
// Hessian, which Newton's method only needs as a model, uses one TF32
// product.
//
// Layout (tc.cuh, K-major, no swizzle): the line-search kernel writes sigma
// for tile t of 128 cells and K-chunk kc of 32 nodes as one 16 KB block
// (hi and lo in two arrays); the constant statistics tables are stored the
// same way, ROWS_g rows (N) x 32 nodes (K) per block, in three column groups:
//   group 0 (96 rows):  0-47 phi_hi (35 used), 48-95 phi_lo;
//   group 1 (304 rows): Hessian entries 0-303;
//   group 2 (304 rows): Hessian entries 304-594 (rows 291-303 zero).
// One CTA (128 threads) computes one tile and one group: thread 0 issues the
// bulk copies (TMA engine, double-buffered, mbarrier transaction counts) and
// the MMAs (accumulators in TMEM); then all four warps read their 32 rows of
// TMEM and write the moments row of each cell.  Every wait is bounded.
//
// Accumulation: the tensor cores add the products of one MMA into the FP32
// accumulator with truncation, so a long chain of MMAs into one accumulator
// drifts by about (number of K steps) x 2^-24 of the running sum, which at
// 12^3 nodes reached 1e-5 in the moments.  The moment columns therefore
// start a fresh accumulator for every K-chunk of 32 nodes, and the reading
// warps add the chunk sums in FP32 registers with rounding to nearest.
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "tc.cuh"
#include "tmap.h"

#include <cudaTypedefs.h>

using namespace mem;

namespace {

constexpr int NGRP = 3;
constexpr int ROWS0 = 96, ROWS12 = 304;      // N rows per block of group 0 / groups 1, 2
constexpr int HSPLIT = 304;                 // Hessian entries of group 1
constexpr int KCH = 32;                     // nodes per K-chunk
constexpr uint32_t A_BYTES = 128 * KCH * 4;  // 16 KB
constexpr uint32_t SBO = KCH / 4 * 128;       // 1024: bytes between 8-row groups
constexpr uint32_t STAGE = 2 * A_BYTES + ROWS12 * KCH * 4;
constexpr uint32_t kMaxPolls = 1u << 22;

__host__ __device__ constexpr int grp_rows(int g) { return g == 0 ? ROWS0 : ROWS12; }
// first float of group g's blocks in the table (KC chunks per group)
__host__ __device__ constexpr size_t grp_base(int g, int KC) {
    return g == 0 ? 0 : (size_t)KC * KCH * (ROWS0 + (size_t)(g - 1) * ROWS12);
}

struct ContractArgs {
    const float *a_hi, *a_lo;  // [tiles][KC][128 x 32] tiled sigma
    const float *tab;          // [2][KC][352 x 32] tiled tables
    float *mom;                // [n][630]
    int n, KC;
    int *err;
};

// Warps 0-3 own the 128 accumulator lanes (cells); warp 4 issues the bulk
// copies and the MMAs.  Group 0 (the moments): each K-chunk's three split
// products go into a fresh accumulator buffer (NB buffers in rotation), which
// warps 0-3 add into FP32 registers as soon as the chunk completes, so no
// accumulator chain is longer than one chunk.  Groups 1, 2 (the Hessian):
// one accumulator chain over all chunks, read once at the end.
constexpr int NB = 8;  // moment accumulator buffers (48 columns each)

__global__ void __launch_bounds__(160, 1) k_tc_contract(ContractArgs A) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_full[2], s_empty[2], s_done, s_accf[NB], s_acce[NB];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x, grp = blockIdx.y;
    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&s_full[0], 1);
        tc::mbar_init(&s_full[1], 1);
        tc::mbar_init(&s_empty[0], 1);
        tc::mbar_init(&s_empty[1], 1);
        tc::mbar_init(&s_done, 1);
        for (int b = 0; b < NB; ++b) {
            tc::mbar_init(&s_accf[b], 1);  // the MMAs of a chunk are done
            tc::mbar_init(&s_acce[b], 4);  // the four reading warps are done with it
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const int KC = A.KC;
    if (warp == 4) {
        if (lane == 0) {
            bool failed = false;
            int loaded = 0;  // chunks whose copies were issued
            const uint32_t b_bytes = (uint32_t)grp_rows(grp) * KCH * 4;
            auto load = [&](int kc) {
                const int s = kc & 1;
                uint8_t *st = smem + s * STAGE;
                const size_t ablk = ((size_t)tile * KC + kc) * (A_BYTES / 4);
                const size_t bblk = grp_base(grp, KC) + (size_t)kc * (b_bytes / 4);
                const uint32_t bytes = (grp == 0 ? 2 * A_BYTES : A_BYTES) + b_bytes;
                tc::mbar_expect_tx(&s_full[s], bytes);
                tc::bulk_g2s(st, A.a_hi + ablk, A_BYTES, &s_full[s]);
                if (grp == 0) tc::bulk_g2s(st + A_BYTES, A.a_lo + ablk, A_BYTES, &s_full[s]);
                tc::bulk_g2s(st + 2 * A_BYTES, A.tab + bblk, b_bytes, &s_full[s]);
                loaded = kc + 1;
            };
            load(0);
            const uint32_t id48 = tc::idesc(128, 48, 2), id256 = tc::idesc(128, 256, 2);
            int kc = 0;
            for (; kc < KC; ++kc) {
                if (kc + 1 < KC) {
                    // stage (kc+1)&1 was last read by the MMAs of chunk kc-1
                    if (kc >= 1 && !tc::mbar_wait(&s_empty[(kc + 1) & 1], ((kc - 1) >> 1) & 1, kMaxPolls)) {
                        failed = true;
                        break;
                    }
                    load(kc + 1);
                }
                if (!tc::mbar_wait(&s_full[kc & 1], (kc >> 1) & 1, kMaxPolls)) {
                    failed = true;
                    break;
                }
                const int bf = kc % NB;
                if (grp == 0 && kc >= NB && !tc::mbar_wait(&s_acce[bf], ((kc / NB) - 1) & 1, kMaxPolls)) {
                    failed = true;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t base = tc::smem_u32(smem + (kc & 1) * STAGE);
                const uint32_t ahi = base, alo = base + A_BYTES, b = base + 2 * A_BYTES;
                const uint32_t dacc = tmem + (uint32_t)(48 * bf);
#pragma unroll
                for (int s = 0; s < KCH / 8; ++s) {
                    const uint64_t dh = tc::sdesc(ahi + 256 * s, 128, SBO);
                    if (grp == 0) {
                        const uint64_t dl = tc::sdesc(alo + 256 * s, 128, SBO);
                        const uint64_t bmh = tc::sdesc(b + 256 * s, 128, SBO);
                        const uint64_t bml = tc::sdesc(b + 6 * SBO + 256 * s, 128, SBO);
                        tc::mma_tf32(dacc, dl, bmh, id48, s != 0);  // lo . hi (a fresh chunk sum)
                        tc::mma_tf32(dacc, dh, bml, id48, 1);       // hi . lo
                        tc::mma_tf32(dacc, dh, bmh, id48, 1);       // hi . hi
                    } else {
                        const uint32_t acc = (kc | s) != 0;
                        const uint64_t b0 = tc::sdesc(b + 256 * s, 128, SBO);
                        const uint64_t b1 = tc::sdesc(b + 32 * SBO + 256 * s, 128, SBO);
                        tc::mma_tf32(tmem, dh, b0, id256, acc);
                        tc::mma_tf32(tmem + 256, dh, b1, id48, acc);
                    }
                }
                tc::mma_commit(&s_empty[kc & 1]);
                if (grp == 0) tc::mma_commit(&s_accf[bf]);
            }
            if (failed) {
                atomicExch(A.err, 1);
                // copies still in flight land in this CTA's shared memory:
                // wait for them (bounded) before the CTA can exit
                for (int j = kc; j < loaded; ++j) tc::mbar_wait(&s_full[j & 1], (j >> 1) & 1, kMaxPolls);
            }
            tc::mma_commit(&s_done);  // every MMA issued above
        }
        __syncwarp();
    } else {
        const int row = 32 * warp + lane;
        const int cell = tile * 128 + row;
        const bool live = cell < A.n;
        const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
        float *m = A.mom + (size_t)cell * MEM_NCOL_SOLVE;
        bool ok = true;
        if (grp == 0) {
            float sum[40];
#pragma unroll
            for (int c = 0; c < 40; ++c) sum[c] = 0.f;
            for (int kc = 0; kc < KC; ++kc) {
                const int bf = kc % NB;
                ok = tc::mbar_wait(&s_accf[bf], (kc / NB) & 1, kMaxPolls);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                tc::fence_after_sync();
#pragma unroll
                for (int c = 0; c < 40; c += 8) {
                    float v[8];
                    tc::tmem_ld8(tl + (uint32_t)(48 * bf + c), v);
#pragma unroll
                    for (int j = 0; j < 8; ++j) sum[c + j] += v[j];
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&s_acce[bf]))
                                            : "memory");
            }
            if (!ok) atomicExch(A.err, 1);
            if (ok && live) {
#pragma unroll
                for (int c = 0; c < NP; ++c) m[c] = sum[c];
            }
        }
        // every MMA of the CTA is complete before its accumulators are read
        // (groups 1, 2) or released
        bool done = tc::mbar_wait(&s_done, 0, kMaxPolls);
        if (!done) {
            atomicExch(A.err, 1);
            done = tc::mbar_wait(&s_done, 0, kMaxPolls);
        }
        done = __all_sync(0xffffffffu, done);
        tc::fence_after_sync();
        if (grp != 0 && done) {
            const int off = grp == 1 ? 0 : HSPLIT, cnt = grp == 1 ? HSPLIT : NP1 * NP / 2 - HSPLIT;
            for (int c = 0; c < 304; c += 8) {
                float v[8];
                tc::tmem_ld8(tl + (uint32_t)c, v);
                if (live) {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (c + j < cnt) m[NP + off + c + j] = v[j];
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// Host round to TF32 (nearest, ties away from zero: the rounding of
// cvt.rna.tf32.f32 on the device).
float tf32_host(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;
    u = (u + 0x1000u) & 0xffffe000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

}  // namespace

namespace mem_host {

int encode_tmap_2d_f32(CUtensorMap *out, const void *base, uint64_t cols, uint64_t rows, uint32_t box_cols,
                       uint32_t box_rows) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return MEM_ECUDA;
        }
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 4};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? MEM_OK : MEM_ECUDA;
}

bool tc_available(const mem_ctx *ctx) { return ctx->d_tc_tab != nullptr; }

// Tiled tables of the contraction for a Gauss-Hermite context (Q a multiple
// of 32): phi values and packed products phi_i phi_j, i >= j >= 1, at the
// nodes in the order of the dense tables (Section 3.1 statistics).
int build_tc_tables(mem_ctx *ctx, const std::vector<double> &phi /*[Q][35]*/) {
    const int Q = ctx->Q;
    if (Q % KCH) return MEM_OK;  // no tensor-core path for this order
    const int KC = Q / KCH;
    std::vector<float> tab(grp_base(NGRP, KC), 0.f);
    auto put = [&](int grp, int row, int q, float v) {
        const int kc = q / KCH, k = q % KCH;
        const size_t blk = grp_base(grp, KC) + (size_t)kc * grp_rows(grp) * KCH;
        const size_t off = (size_t)(row >> 3) * (SBO / 4) + (size_t)(k >> 2) * 32 + (row & 7) * 4 + (k & 3);
        tab[blk + off] = v;
    };
    for (int q = 0; q < Q; ++q) {
        const double *ph = &phi[(size_t)q * NP];
        for (int k = 0; k < NP; ++k) {
            const float f = (float)ph[k], hi = tf32_host(f), lo = tf32_host(f - hi);
            put(0, k, q, hi);
            put(0, 48 + k, q, lo);
        }
        for (int i = 1; i < NP; ++i)
            for (int j = 1; j <= i; ++j) {
                const int p = (i - 1) * i / 2 + (j - 1);
                const float v = tf32_host((float)(ph[i] * ph[j]));
                if (p < HSPLIT) put(1, p, q, v);
                else put(2, p - HSPLIT, q, v);
            }
    }
    if (cudaMalloc((void **)&ctx->d_tc_tab, sizeof(float) * tab.size()) != cudaSuccess) {
        cudaGetLastError();
        ctx->d_tc_tab = nullptr;
        return MEM_ENOMEM;
    }
    if (cudaMemcpy(ctx->d_tc_tab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return MEM_ECUDA;
    return MEM_OK;
}

size_t tc_sigma_floats(int Q, int64_t cells) { return (size_t)((cells + 127) / 128) * 128 * Q; }

int tc_contract(mem_ctx *ctx, const float *a_hi, const float *a_lo, float *mom, int n, int *err, cudaStream_t st) {
    if (!ctx->d_tc_tab) return MEM_EINVAL;
    static bool configured = false;
    const int smem = 2 * STAGE;
    if (!configured) {
        MEM_CUDA_TRY(cudaFuncSetAttribute(k_tc_contract, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        configured = true;
    }
    ContractArgs a{a_hi, a_lo, ctx->d_tc_tab, mom, n, ctx->Q / KCH, err};
    dim3 grid((n + 127) / 128, NGRP);
    k_tc_contract<<<grid, 160, smem, st>>>(a);
    MEM_CUDA_TRY(cudaGetLastError());
    return MEM_OK;
}

}  // namespace mem_host

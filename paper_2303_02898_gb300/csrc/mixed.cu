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
// Layout: sigma (hi and lo, one array each) is row-major [cells][Q], written
// coalesced by the line-search kernel; the constant statistics tables are
// row-major [704][Q]:
//   rows   0- 47: phi_hi (35 used),      rows  48- 95: phi_lo;
//   rows 96 + p:  Hessian entry p, p = 0 .. 594 (rows 691-703 zero).
// Tensor maps (TMA descriptors) cut them into boxes of 32 nodes (128 bytes:
// one swizzle span) x 128 cells, or 48, 208 or 192 table rows, which the TMA
// engine writes to shared memory with the 128-byte swizzle (tc.cuh,
// sdesc_sw128).  One CTA (160 threads) computes one tile of 128 cells and
// one column group (0: moments; 1, 2, 3: Hessian entries 0-207, 208-415,
// 416-594); the group index runs fastest in the grid, so the four CTAs of a
// tile run together and three of them read sigma from L2.  Warp 4 issues the
// tensor loads (two stages, mbarrier transaction counts) and the MMAs
// (accumulators in TMEM); warps 0-3 read their 32 TMEM lanes, stage the rows
// in shared memory and write each cell's row of the moments array with
// coalesced stores.  Every wait is bounded.
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

constexpr int NGRP = 4;
constexpr int TROWS = 704;                    // table rows
constexpr int HN = 208;                       // Hessian entries of groups 1 and 2 (group 3: 179 of 192)
constexpr int KCH = 32;                       // nodes per K-chunk (128 bytes of FP32)
constexpr int STAGES = 2;
constexpr uint32_t A_BYTES = 128 * KCH * 4;   // 16 KB: one box of sigma
constexpr uint32_t STAGE = 2 * A_BYTES + 96 * KCH * 4;  // 44 KB: sigma hi + lo + 96 table rows (moments)
constexpr uint32_t SMEM = STAGES * STAGE + 1024;  // + the 1024-byte alignment of the swizzled tiles
constexpr int EPC = 104;                      // columns per epilogue round
constexpr int EP = 108;                       // row pitch (floats) of the staged epilogue
constexpr uint32_t TMEM_COLS = 256;           // two CTAs share an SM's 512 TMEM columns
constexpr uint32_t kMaxPolls = 1u << 22;
static_assert(STAGE % 1024 == 0, "stages must keep the 1024-byte alignment of the swizzle atoms");
static_assert(A_BYTES + HN * KCH * 4 <= STAGE, "a Hessian group's operands fit a stage");
static_assert(128 * EP * 4 <= STAGES * STAGE, "the epilogue staging reuses the stage buffers");
static_assert(2 * (SMEM + 1024) <= 227 * 1024, "two CTAs per SM");

__host__ __device__ constexpr int hess_first(int g) { return (g - 1) * HN; }             // first entry of group g
__host__ __device__ constexpr int hess_cols(int g) { return g == 3 ? 192 : HN; }          // MMA N of group g
__host__ __device__ constexpr int hess_count(int g) { return g == 3 ? NP1 * NP / 2 - 2 * HN : HN; }

// Warps 0-3 own the 128 accumulator lanes (cells); warp 4 issues the tensor
// loads and the MMAs.  Group 0 (the moments): each K-chunk's three split
// products go into a fresh accumulator buffer (NB buffers in rotation), which
// warps 0-3 add into FP32 registers as soon as the chunk completes, so no
// accumulator chain is longer than one chunk.  Groups 1-3 (the Hessian):
// one accumulator chain over all chunks, read once at the end.  Each CTA
// holds 256 TMEM columns and 89 KB of shared memory, so two run on an SM
// and one's epilogue overlaps the other's loads and MMAs.
constexpr int NB = 5;  // moment accumulator buffers (48 columns each)

__global__ void __launch_bounds__(160, 2)
    k_tc_contract(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
                  const __grid_constant__ CUtensorMap tm_t48, const __grid_constant__ CUtensorMap tm_t208,
                  const __grid_constant__ CUtensorMap tm_t192,
                  float *__restrict__ mom, int n, int KC, int *err) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    __shared__ __align__(8) uint64_t s_full[STAGES], s_empty[STAGES], s_done, s_accf[NB], s_acce[NB];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = blockIdx.x, tile = blockIdx.y;
    if (warp == 0) {
        tc::tmem_alloc(&s_tmem, TMEM_COLS);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&s_full[s], 1);
            tc::mbar_init(&s_empty[s], 1);
        }
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
    float sum[40];  // group 0: the moment sums of this thread's cell
#pragma unroll
    for (int c = 0; c < 40; ++c) sum[c] = 0.f;
    if (warp == 4) {
        if (lane == 0) {
            bool failed = false;
            int loaded = 0, waited = 0;  // chunks whose loads were issued / have landed
            const int y = tile * 128;
            auto load = [&](int kc) {
                uint8_t *st = smem + (kc % STAGES) * STAGE;
                uint8_t *b = st + 2 * A_BYTES;
                uint64_t *bar = &s_full[kc % STAGES];
                const int x = kc * KCH;  // 128-byte multiple: the TMA alignment rule holds
                if (grp == 0) {
                    tc::mbar_expect_tx(bar, 2 * A_BYTES + 96 * 128);
                    tc::tma_load_2d(st, &tm_hi, x, y, bar);
                    tc::tma_load_2d(st + A_BYTES, &tm_lo, x, y, bar);
                    tc::tma_load_2d(b, &tm_t48, x, 0, bar);
                    tc::tma_load_2d(b + 48 * 128, &tm_t48, x, 48, bar);
                } else {
                    // the table rows follow sigma hi directly (16 KB: the 1024-byte alignment holds)
                    const int t0 = 96 + hess_first(grp);
                    tc::mbar_expect_tx(bar, A_BYTES + hess_cols(grp) * 128);
                    tc::tma_load_2d(st, &tm_hi, x, y, bar);
                    tc::tma_load_2d(st + A_BYTES, grp == 3 ? &tm_t192 : &tm_t208, x, t0, bar);
                }
                loaded = kc + 1;
            };
            for (int j = 0; j < STAGES - 1 && j < KC; ++j) load(j);
            const uint32_t id48 = tc::idesc(128, 48, 2), idh = tc::idesc(128, hess_cols(grp), 2);
            for (int kc = 0; kc < KC; ++kc) {
                const int s = kc % STAGES, bf = kc % NB;
                if (!tc::mbar_wait(&s_full[s], (kc / STAGES) & 1, kMaxPolls)) {
                    failed = true;
                    break;
                }
                waited = kc + 1;
                if (grp == 0 && kc >= NB && !tc::mbar_wait(&s_acce[bf], ((kc / NB) - 1) & 1, kMaxPolls)) {
                    failed = true;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t base = tc::smem_u32(smem + s * STAGE);
                const uint32_t ahi = base, alo = base + A_BYTES, b = base + 2 * A_BYTES;
                const uint32_t dacc = tmem + (uint32_t)(48 * bf);
#pragma unroll
                for (int k = 0; k < KCH / 8; ++k) {  // one MMA consumes 8 nodes (32 bytes)
                    const uint64_t dh = tc::sdesc_sw128(ahi + 32 * k, 1024);
                    if (grp == 0) {
                        const uint64_t dl = tc::sdesc_sw128(alo + 32 * k, 1024);
                        const uint64_t bmh = tc::sdesc_sw128(b + 32 * k, 1024);
                        const uint64_t bml = tc::sdesc_sw128(b + 48 * 128 + 32 * k, 1024);
                        tc::mma_tf32(dacc, dl, bmh, id48, k != 0);  // lo . hi (a fresh chunk sum)
                        tc::mma_tf32(dacc, dh, bml, id48, 1);       // hi . lo
                        tc::mma_tf32(dacc, dh, bmh, id48, 1);       // hi . hi
                    } else {
                        const uint32_t acc = (kc | k) != 0;
                        tc::mma_tf32(tmem, dh, tc::sdesc_sw128(ahi + A_BYTES + 32 * k, 1024), idh, acc);  // rows after sigma hi
                    }
                }
                tc::mma_commit(&s_empty[s]);
                if (grp == 0) tc::mma_commit(&s_accf[bf]);
                // refill the stage of chunk kc - 1 once its MMAs are done (the
                // MMAs of chunk kc are already queued behind them)
                const int nxt = kc + STAGES - 1;
                if (nxt < KC) {
                    if (kc >= 1 && !tc::mbar_wait(&s_empty[(kc - 1) % STAGES], ((kc - 1) / STAGES) & 1, kMaxPolls)) {
                        failed = true;
                        break;
                    }
                    load(nxt);
                }
            }
            if (failed) {
                atomicExch(err, 1);
                s_fail = 1;
                // copies still in flight land in this CTA's shared memory:
                // wait for them (bounded) before the CTA can exit
                for (int j = waited; j < loaded; ++j) tc::mbar_wait(&s_full[j % STAGES], (j / STAGES) & 1, kMaxPolls);
            }
            tc::mma_commit(&s_done);  // every MMA issued above
        }
        __syncwarp();
    } else if (grp == 0) {
        const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
        bool ok = true;
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
        if (!ok) {
            atomicExch(err, 1);
            s_fail = 1;
        }
    }
    __syncthreads();  // s_fail is final
    if (warp < 4) {
        // every MMA of the CTA is complete (and every tensor load has landed)
        // before the accumulators are read or the stage buffers reused
        bool done = tc::mbar_wait(&s_done, 0, kMaxPolls);
        if (!done) {
            atomicExch(err, 1);
            done = tc::mbar_wait(&s_done, 0, kMaxPolls);
        }
        done = __all_sync(0xffffffffu, done) && !s_fail;
        tc::fence_after_sync();
        if (done) {
            // stage this warp's 32 rows in shared memory, EPC columns at a
            // time, then write each row with the whole warp (consecutive
            // addresses)
            float *ep = reinterpret_cast<float *>(smem) + (size_t)32 * warp * EP;
            float *my = ep + (size_t)lane * EP;
            const int col0 = grp == 0 ? 0 : NP + hess_first(grp);
            const int cnt = grp == 0 ? NP : hess_count(grp);
            const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
            const int cell0 = tile * 128 + 32 * warp;
            for (int c0 = 0; c0 < cnt; c0 += EPC) {
                if (grp == 0) {
#pragma unroll
                    for (int c = 0; c < 36; c += 4)
                        *reinterpret_cast<float4 *>(my + c) = make_float4(sum[c], sum[c + 1], sum[c + 2], sum[c + 3]);
                } else {
                    for (int c = 0; c < EPC && c0 + c < hess_cols(grp); c += 8) {
                        float v[8];
                        tc::tmem_ld8(tl + (uint32_t)(c0 + c), v);
                        *reinterpret_cast<float4 *>(my + c) = make_float4(v[0], v[1], v[2], v[3]);
                        *reinterpret_cast<float4 *>(my + c + 4) = make_float4(v[4], v[5], v[6], v[7]);
                    }
                }
                __syncwarp();
                const int w = min(EPC, cnt - c0);
                for (int r = 0; r < 32 && cell0 + r < n; ++r) {
                    float *m = mom + (size_t)(cell0 + r) * MEM_NCOL_SOLVE + col0 + c0;
                    const float *e = ep + (size_t)r * EP;
                    for (int j = lane; j < w; j += 32) m[j] = e[j];
                }
                __syncwarp();  // the staging rows are free for the next round
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, TMEM_COLS);
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

// Tables of the contraction for a Gauss-Hermite context (Q a multiple of
// 32), row-major [704][Q]: phi values (TF32 hi and lo) and the products
// phi_i phi_j, i >= j >= 1, packed in the order of the dense tables, at the
// nodes (Section 3.1 statistics), with their tensor maps.  No tensor-core
// path (and MEM_OK) for other orders or when the driver offers no tensor-map
// encoder.
int build_tc_tables(mem_ctx *ctx, const std::vector<double> &phi /*[Q][35]*/) {
    const int Q = ctx->Q;
    if (Q % KCH) return MEM_OK;
    std::vector<float> tab((size_t)TROWS * Q, 0.f);
    auto put = [&](int row, int q, float v) { tab[(size_t)row * Q + q] = v; };
    for (int q = 0; q < Q; ++q) {
        const double *ph = &phi[(size_t)q * NP];
        for (int k = 0; k < NP; ++k) {
            const float f = (float)ph[k], hi = tf32_host(f), lo = tf32_host(f - hi);
            put(k, q, hi);
            put(48 + k, q, lo);
        }
        for (int i = 1; i < NP; ++i)
            for (int j = 1; j <= i; ++j) {
                const int p = (i - 1) * i / 2 + (j - 1);
                put(96 + p, q, tf32_host((float)(ph[i] * ph[j])));
            }
    }
    float *d = nullptr;
    if (cudaMalloc((void **)&d, sizeof(float) * tab.size()) != cudaSuccess) {
        cudaGetLastError();
        return MEM_ENOMEM;
    }
    if (cudaMemcpy(d, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return MEM_ECUDA;
    }
    if (encode_tmap_2d_f32(&ctx->tm_tab48, d, Q, TROWS, KCH, 48) ||
        encode_tmap_2d_f32(&ctx->tm_tab208, d, Q, TROWS, KCH, 208) ||
        encode_tmap_2d_f32(&ctx->tm_tab192, d, Q, TROWS, KCH, 192)) {
        cudaFree(d);
        return MEM_OK;  // no tensor maps: the mixed back-end is unavailable (MEM_EINVAL)
    }
    ctx->d_tc_tab = d;
    return MEM_OK;
}

size_t tc_sigma_floats(int Q, int64_t cells) { return (size_t)((cells + 127) / 128) * 128 * Q; }

// sigma hi / lo: row-major [rows][Q] (rows a multiple of 128); moment rows
// of the first n of them go to mom.
int tc_contract(mem_ctx *ctx, const float *a_hi, const float *a_lo, int64_t rows, float *mom, int n, int *err,
                cudaStream_t st) {
    if (!ctx->d_tc_tab || rows % 128 || n > rows) return MEM_EINVAL;
    if (n <= 0) return MEM_OK;
    static bool configured = false;
    if (!configured) {
        MEM_CUDA_TRY(cudaFuncSetAttribute(k_tc_contract, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM));
        configured = true;
    }
    CUtensorMap thi, tlo;
    if (encode_tmap_2d_f32(&thi, a_hi, ctx->Q, rows, KCH, 128) || encode_tmap_2d_f32(&tlo, a_lo, ctx->Q, rows, KCH, 128))
        return MEM_ECUDA;
    dim3 grid(NGRP, (n + 127) / 128);
    k_tc_contract<<<grid, 160, SMEM, st>>>(thi, tlo, ctx->tm_tab48, ctx->tm_tab208, ctx->tm_tab192, mom, n,
                                           ctx->Q / KCH, err);
    MEM_CUDA_TRY(cudaGetLastError());
    return MEM_OK;
}

}  // namespace mem_host

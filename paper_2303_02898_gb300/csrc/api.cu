// api.cu -- context, constant tables and the C-ABI entry points of the MEM
// library.  Every compute step runs in CUDA kernels; the host code here only
// builds constant tables (once per context), validates arguments and
// dispatches.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "ctx.h"

using namespace mem;

// Cells per chunk of the velocity-space flux (moment rows in context scratch).
static constexpr int64_t VEL_FLUX_CHUNK = (int64_t)1 << 16;

namespace mem_host {

// 1D Gauss-Hermite rule for the standard normal weight: the nodes are the
// roots of He_n, bracketed on a fine grid and refined by bisection in long
// double; the weights are w_i = n! / (n^2 He_{n-1}(x_i)^2), which sum to 1.
int gh_rule(int n, std::vector<double> &x, std::vector<double> &w) {
    if (n < 1 || n > 32) return MEM_EINVAL;
    auto he = [n](long double t, long double &hn, long double &hn1) {
        long double a = 1.0L, b = t;  // He_0, He_1
        if (n == 1) { hn = b; hn1 = a; return; }
        for (int k = 1; k < n; ++k) {
            long double c = t * b - (long double)k * a;
            a = b;
            b = c;
        }
        hn = b;
        hn1 = a;
    };
    x.clear();
    w.clear();
    const long double L = sqrtl(4.0L * n + 2.0L) + 2.0L;
    const int G = 20001;
    long double xp = -L, hp, dummy;
    he(xp, hp, dummy);
    for (int k = 1; k <= G; ++k) {
        long double xc = -L + 2.0L * L * k / G, hc;
        he(xc, hc, dummy);
        if ((hp < 0) != (hc < 0)) {
            long double lo = xp, hi = xc, flo = hp;
            for (int it = 0; it < 200; ++it) {
                long double mid = 0.5L * (lo + hi), fm;
                he(mid, fm, dummy);
                if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else hi = mid;
            }
            x.push_back((double)(0.5L * (lo + hi)));
        }
        xp = xc;
        hp = hc;
    }
    if ((int)x.size() != n) return MEM_EINVAL;
    long double fact = 1.0L;
    for (int k = 2; k <= n; ++k) fact *= k;
    long double sw = 0.0L;
    std::vector<long double> wl(n);
    for (int i = 0; i < n; ++i) {
        long double hn, hn1;
        he((long double)x[i], hn, hn1);
        wl[i] = fact / ((long double)n * n * hn1 * hn1);
        sw += wl[i];
    }
    for (int i = 0; i < n; ++i) w.push_back((double)(wl[i] / sw));
    return MEM_OK;
}

int reserve_scratch(mem_ctx *ctx, size_t bytes) {
    if (cudaMalloc(&ctx->scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        ctx->scratch = nullptr;
        return MEM_ENOMEM;
    }
    ctx->scratch_bytes = bytes;
    if (cudaEventCreateWithFlags(&ctx->scratch_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        ctx->scratch_ev = nullptr;
        return MEM_ECUDA;
    }
    return MEM_OK;
}

// Order this use of the context scratch after the previous one, which may
// have been enqueued on another stream.  Stream capture cannot wait on an
// event recorded outside it, so a capturing stream is not ordered here
// (none of the scratch paths is captured by the library itself).
int scratch_begin(mem_ctx *ctx, size_t bytes, cudaStream_t st) {
    if (bytes > ctx->scratch_bytes || !ctx->scratch) return MEM_ENOMEM;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MEM_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (ctx->scratch_ev_live && cs == cudaStreamCaptureStatusNone) MEM_CUDA_TRY(cudaStreamWaitEvent(st, ctx->scratch_ev, 0));
    return MEM_OK;
}

void scratch_end(mem_ctx *ctx, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    if (cudaEventRecord(ctx->scratch_ev, st) == cudaSuccess) ctx->scratch_ev_live = true;
    else cudaGetLastError();
}

// 1D Gauss-Legendre rule on [-1, 1]: the roots of P_n by Newton's method in
// long double from the estimates cos(pi (i + 3/4) / (n + 1/2)), weights
// 2 / ((1 - x^2) P_n'(x)^2); ascending nodes.
int gl_rule(int n, std::vector<double> &x, std::vector<double> &w) {
    if (n < 1 || n > 64) return MEM_EINVAL;
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < n; ++i) {
        long double t = cosl(pi * (i + 0.75L) / (n + 0.5L)), dp = 1.0L;
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1.0L, p1 = t;  // P_0, P_1
            for (int k = 2; k <= n; ++k) {
                const long double p2 = ((2.0L * k - 1.0L) * t * p1 - (k - 1.0L) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const long double pn = n == 1 ? t : p1, pn1 = n == 1 ? 1.0L : p0;
            dp = n * (t * pn - pn1) / (t * t - 1.0L);
            const long double step = pn / dp;
            t -= step;
            if (fabsl(step) < 1e-19L) break;
        }
        x[n - 1 - i] = (double)t;
        w[n - 1 - i] = (double)(2.0L / ((1.0L - t * t) * dp * dp));
    }
    return MEM_OK;
}

}  // namespace mem_host

// ---------------------------------------------------------------------------
// Host evaluation of the statistics (double) for the constant tables.
static void he_host(double x, int K, double *h) {
    double hm1 = 0.0, hc = 1.0, inv = 1.0;
    h[0] = 1.0;
    for (int k = 0; k < K; ++k) {
        double hp = x * hc - k * hm1;
        hm1 = hc;
        hc = hp;
        inv /= sqrt((double)(k + 1));
        h[k + 1] = hc * inv;
    }
}

static double binom_d(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}
static double fact_d(int n) {
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= i;
    return r;
}

// Linearisation of Hermite products: he_a he_b = sum_k L(a,b,k) he_{a+b-2k},
// L(a,b,k) = C(a,k) C(b,k) k! sqrt((a+b-2k)! / (a! b!)).
static double lin_coef(int a, int b, int k) {
    return binom_d(a, k) * binom_d(b, k) * fact_d(k) * sqrt(fact_d(a + b - 2 * k) / (fact_d(a) * fact_d(b)));
}

// Term lists that express E[phi_i phi_j] (i >= j >= j0) -- and with
// with_x, E[ubar_x phi_i phi_j] -- as sums of Hermite-product moments.
static void build_lin_terms(int j0, bool with_x, std::vector<int> &off, std::vector<int2> &terms) {
    off.clear();
    terms.clear();
    for (int i = j0; i < NP; ++i)
        for (int j = j0; j <= i; ++j) {
            off.push_back((int)terms.size());
            int a1 = exp_a(i), b1 = exp_b(i), c1 = exp_c(i), a2 = exp_a(j), b2 = exp_b(j), c2 = exp_c(j);
            // product of the two statistics, optionally times he_1(x)
            std::vector<std::pair<int, double>> xs;  // (x-degree, coefficient) of he_a1 he_a2 [he_1]
            for (int kx = 0; kx <= std::min(a1, a2); ++kx) {
                int dx = a1 + a2 - 2 * kx;
                double cx = lin_coef(a1, a2, kx);
                if (!with_x) {
                    xs.push_back({dx, cx});
                } else {
                    // he_1 he_d = sqrt(d+1) he_{d+1} + sqrt(d) he_{d-1}
                    xs.push_back({dx + 1, cx * sqrt((double)(dx + 1))});
                    if (dx > 0) xs.push_back({dx - 1, cx * sqrt((double)dx)});
                }
            }
            for (auto &px : xs)
                for (int ky = 0; ky <= std::min(b1, b2); ++ky)
                    for (int kz = 0; kz <= std::min(c1, c2); ++kz) {
                        int dy = b1 + b2 - 2 * ky, dz = c1 + c2 - 2 * kz;
                        double cf = px.second * lin_coef(b1, b2, ky) * lin_coef(c1, c2, kz);
                        float cff = (float)cf;
                        int2 t;
                        t.x = idx3(px.first, dy, dz);
                        memcpy(&t.y, &cff, 4);
                        terms.push_back(t);
                    }
        }
    off.push_back((int)terms.size());
}

// Per-lane term sequences for the fused kernel's Hessian assembly: lane l
// takes the packed entries p = l, l + 32, ...; slot t of lane l is stored at
// [t][l] as (mu index | p << 8 | last-term flag in the sign bit, coefficient).
// Sequences are padded with zero terms to a common length.
// Hessian terms in rounds: entries sorted by term count, L per round (one
// per lane), each round padded to its longest entry.  The kernel then runs a
// branch-free term loop per round (loads can be pipelined: no store in
// between) and stores all L entries at once.  slots[(base + t) * L + l] =
// (mu index, coefficient bits); rounds[r] = terms of round r; ent[r * L + l] =
// destination (i | j << 8) of lane l's entry, or -1.
static void build_hess_rounds(const std::vector<int> &off, const std::vector<int2> &terms, int L,
                              std::vector<int2> &slots, std::vector<int> &rounds, std::vector<int> &ent) {
    const int NE = (int)off.size() - 1;
    std::vector<int> order(NE);
    for (int e = 0; e < NE; ++e) order[e] = e;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
    slots.clear();
    rounds.clear();
    ent.clear();
    for (int r0 = 0; r0 < NE; r0 += L) {
        int T = 0;
        for (int l = 0; l < L && r0 + l < NE; ++l) T = std::max(T, off[order[r0 + l] + 1] - off[order[r0 + l]]);
        rounds.push_back(T);
        for (int t = 0; t < T; ++t)
            for (int l = 0; l < L; ++l) {
                int2 sl = {0, 0};
                if (r0 + l < NE) {
                    const int e = order[r0 + l];
                    if (off[e] + t < off[e + 1]) sl = terms[off[e] + t];
                }
                sl.x &= 255;
                slots.push_back(sl);
            }
        for (int l = 0; l < L; ++l) {
            if (r0 + l >= NE) { ent.push_back(-1); continue; }
            // packed entry p of the 34 x 34 lower triangle (rows/cols of phi_1..34)
            const int p = order[r0 + l];
            int i = 0;
            while ((i + 1) * (i + 2) / 2 <= p) ++i;
            ent.push_back(i | ((p - i * (i + 1) / 2) << 8));
        }
    }
}

static void build_hess_slots(const std::vector<int> &off, const std::vector<int2> &terms, std::vector<int2> &slots,
                             int &nslots, const std::vector<int> *off2 = nullptr, const std::vector<int2> *terms2 = nullptr,
                             int L = 32) {
    const int NE1 = (int)off.size() - 1, NE2 = off2 ? (int)off2->size() - 1 : 0;
    std::vector<std::vector<int2>> per(L);
    for (int p = 0; p < NE1 + NE2; ++p) {
        // L = 32: entry p on lane p % 32; wider tables put each entry on the
        // lane with the fewest terms so far (entries have 1 to 30 terms).
        int lane = p % 32;
        if (L != 32) {
            lane = 0;
            for (int l = 1; l < L; ++l)
                if (per[l].size() < per[lane].size()) lane = l;
        }
        auto &v = per[lane];
        const std::vector<int> &o = p < NE1 ? off : *off2;
        const std::vector<int2> &tm = p < NE1 ? terms : *terms2;
        const int q = p < NE1 ? p : p - NE1;
        for (int t = o[q]; t < o[q + 1]; ++t) {
            int2 s = tm[t];
            s.x = (s.x & 255) | (p << 8);
            if (t == o[q + 1] - 1) s.x |= (int)0x80000000;
            v.push_back(s);
        }
    }
    nslots = 0;
    for (auto &v : per) nslots = std::max(nslots, (int)v.size());
    slots.assign((size_t)nslots * L, int2{0, 0});
    for (int l = 0; l < L; ++l)
        for (int t = 0; t < (int)per[l].size(); ++t) slots[(size_t)t * L + l] = per[l][t];
}

// Axisymmetric cells (invariant under u_y -> -u_y and u_z -> -u_z, as every
// 1D-shock cell is) make E[phi phi^T] and E[ubar_x phi phi^T] block-diagonal
// over the parity classes of (b, c): even/even (14 statistics, phi_0
// included), odd/even (8), even/odd (8, the same spectrum by y <-> z) and
// odd/odd (5).  These slots assemble the blocks ee, oe and oo (lower
// triangles, leading dimension 16) at work offsets S: 0, 512, 768 and
// X: 256, 640, 848 of the flux kernel.
static void build_axi_slots(const std::vector<int> &soff, const std::vector<int2> &sterms, const std::vector<int> &xoff,
                            const std::vector<int2> &xterms, std::vector<int2> &slots, int &nslots) {
    const int cls_of_block[3] = {0, 1, 3}, oS[3] = {0, 512, 768}, oX[3] = {256, 640, 848};
    struct Entry { const std::vector<int2> *terms; int t0, t1, dst; };
    std::vector<Entry> ent;
    for (int blk = 0; blk < 3; ++blk) {
        std::vector<int> mem;
        for (int k = 0; k < NP; ++k)
            if (((exp_b(k) & 1) | ((exp_c(k) & 1) << 1)) == cls_of_block[blk]) mem.push_back(k);
        for (int a = 0; a < (int)mem.size(); ++a)
            for (int b = 0; b <= a; ++b) {
                const int i = mem[a], j = mem[b], P = i * (i + 1) / 2 + j;
                ent.push_back({&sterms, soff[P], soff[P + 1], oS[blk] + a * 16 + b});
                ent.push_back({&xterms, xoff[P], xoff[P + 1], oX[blk] + a * 16 + b});
            }
    }
    std::vector<std::vector<int2>> per(32);
    for (size_t e = 0; e < ent.size(); ++e) {
        auto &v = per[e % 32];
        for (int t = ent[e].t0; t < ent[e].t1; ++t) {
            int2 sl = (*ent[e].terms)[t];
            sl.x = (sl.x & 255) | (ent[e].dst << 8);
            if (t == ent[e].t1 - 1) sl.x |= (int)0x80000000;
            v.push_back(sl);
        }
    }
    nslots = 0;
    for (auto &v : per) nslots = std::max(nslots, (int)v.size());
    slots.assign((size_t)nslots * 32, int2{0, 0});
    for (int l = 0; l < 32; ++l)
        for (int t = 0; t < (int)per[l].size(); ++t) slots[(size_t)t * 32 + l] = per[l][t];
}

template <typename T>
static int upload(T **dst, const std::vector<T> &src) {
    if (cudaMalloc((void **)dst, sizeof(T) * std::max<size_t>(1, src.size())) != cudaSuccess) return MEM_ENOMEM;
    if (!src.empty() && cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return MEM_ECUDA;
    return MEM_OK;
}

extern "C" {

void mem_solve_opts_default(mem_solve_opts *o) {
    o->tol = 1e-8f;
    o->maxI = 500;
    o->lambda0 = 1e-3f;
    o->lambda_mul = 10.f;
    o->max_lambda = 20;
    o->c_armijo = 5e-4f;
    o->atol = 5e-6f;
    o->rtol = 5e-5f;
    o->maxT = 25;
    o->alpha_min = 1e-6f;
    o->final_step = 0;
    o->impl = MEM_IMPL_FUSED;
}

const char *mem_version(void) { return "mem-gb300 0.1 (sm_103a)"; }

// Linearisation tables shared by every kind of context: Hessian slots of the
// solver, flux and parity-block slots of the speed kernel, and the plain
// path's term lists.
static int build_slot_tables(mem_ctx *ctx) {
    int rc = MEM_OK;
    std::vector<int> off, xoff;
    std::vector<int2> terms, xterms;
    build_lin_terms(1, false, off, terms);
    build_lin_terms(0, true, xoff, xterms);
    std::vector<int2> slots, fslots;
    build_hess_slots(off, terms, slots, ctx->n_hess_slots);
    std::vector<int2> slots128;
    build_hess_slots(off, terms, slots128, ctx->n_hess_slots128, nullptr, nullptr, 128);
    std::vector<int2> rslots;
    std::vector<int> rrounds, rent;
    build_hess_rounds(off, terms, 32, rslots, rrounds, rent);
    ctx->n_hess_rounds = (int)rrounds.size();
    std::vector<int> soff;
    std::vector<int2> sterms;
    build_lin_terms(1, false, soff, sterms);  // E[phi_i phi_j], i >= j >= 1
    build_hess_slots(soff, sterms, fslots, ctx->n_flux_slots, &xoff, &xterms);
    std::vector<int> s0off;
    std::vector<int2> s0terms, aslots;
    build_lin_terms(0, false, s0off, s0terms);
    build_axi_slots(s0off, s0terms, xoff, xterms, aslots, ctx->n_axi_slots);
    // Flux slots carry their destination in the flux kernel's per-warp work
    // area instead of the entry number: entries 0..594 (E[phi_i phi_j],
    // i >= j >= 1) go to H[(i-1) * 35 + (j-1)]; entries 595..1224
    // (E[ubar_x phi_i phi_j], i >= j >= 0) go to 1260 + i * 36 + j.
    {
        std::vector<int> dst;
        for (int i = 1; i < NP; ++i)
            for (int j = 1; j <= i; ++j) dst.push_back((i - 1) * 35 + (j - 1));
        for (int i = 0; i < NP; ++i)
            for (int j = 0; j <= i; ++j) dst.push_back(1260 + i * 36 + j);
        for (auto &sl : fslots) {
            const bool last = sl.x < 0;
            const int p = (sl.x >> 8) & 4095, idx = sl.x & 255;
            if (sl.x == 0 && sl.y == 0) continue;  // padding
            sl.x = idx | (dst[p] << 8) | (last ? (int)0x80000000 : 0);
        }
    }
    if (!rc) rc = upload(&ctx->d_lin_off, off);
    if (!rc) rc = upload(&ctx->d_lin_terms, terms);
    if (!rc) rc = upload(&ctx->d_hess_slots, slots);
    if (!rc) rc = upload(&ctx->d_hess_slots128, slots128);
    if (!rc) rc = upload(&ctx->d_hr_slots, rslots);
    if (!rc) rc = upload(&ctx->d_hr_rounds, rrounds);
    if (!rc) rc = upload(&ctx->d_hr_ent, rent);
    if (!rc) rc = upload(&ctx->d_flux_slots, fslots);
    if (!rc) rc = upload(&ctx->d_axi_slots, aslots);
    if (!rc) rc = upload(&ctx->d_xlin_off, xoff);
    if (!rc) rc = upload(&ctx->d_xlin_terms, xterms);
    ctx->n_lin_terms = (int)terms.size();
    return rc;
}

int mem_init(int degree, int quad_order, mem_ctx **out) {
    if (!out || degree != 4 || quad_order < 4 || quad_order > 16) return MEM_EINVAL;
    *out = nullptr;
    mem_ctx *ctx = new mem_ctx();
    cudaGetDevice(&ctx->device);
    int rc = mem_host::gh_rule(quad_order, ctx->x1d, ctx->w1d);
    if (rc) { delete ctx; return rc; }
    const int n = quad_order, Q = n * n * n;
    ctx->n1d = n;
    ctx->Q = Q;
    ctx->xmax = (float)ctx->x1d[n - 1];
    std::vector<float> phiT((size_t)NP * Q), logw(Q), tabS((size_t)Q * MEM_NCOL_SOLVE), tabF((size_t)Q * MEM_NCOL_FLUX);
    std::vector<float> he1d((size_t)n * MEM_HE_STRIDE, 0.f), x1d(n), lw1d(n);
    std::vector<double> phi64((size_t)Q * NP), phiT64((size_t)NP * Q), logw64(Q);
    std::vector<double> hx(n * 10);
    for (int i = 0; i < n; ++i) {
        he_host(ctx->x1d[i], 9, &hx[i * 10]);
        for (int k = 0; k < 10; ++k) he1d[i * MEM_HE_STRIDE + k] = (float)hx[i * 10 + k];
        x1d[i] = (float)ctx->x1d[i];
        lw1d[i] = (float)log(ctx->w1d[i]);
    }
    for (int ix = 0; ix < n; ++ix)
        for (int iy = 0; iy < n; ++iy)
            for (int iz = 0; iz < n; ++iz) {
                const int q = (ix * n + iy) * n + iz;
                double ph[NP];
                for (int k = 0; k < NP; ++k) ph[k] = hx[ix * 10 + exp_a(k)] * hx[iy * 10 + exp_b(k)] * hx[iz * 10 + exp_c(k)];
                const double ux = ctx->x1d[ix];
                logw64[q] = log(ctx->w1d[ix]) + log(ctx->w1d[iy]) + log(ctx->w1d[iz]);
                logw[q] = (float)logw64[q];
                for (int k = 0; k < NP; ++k) phi64[(size_t)q * NP + k] = phiT64[(size_t)k * Q + q] = ph[k];
                for (int k = 0; k < NP; ++k) phiT[(size_t)k * Q + q] = (float)ph[k];
                float *rs = &tabS[(size_t)q * MEM_NCOL_SOLVE];
                for (int k = 0; k < NP; ++k) rs[k] = (float)ph[k];
                for (int i = 1; i < NP; ++i)
                    for (int j = 1; j <= i; ++j) rs[NP + (i - 1) * i / 2 + (j - 1)] = (float)(ph[i] * ph[j]);
                float *rf = &tabF[(size_t)q * MEM_NCOL_FLUX];
                for (int k = 0; k < NP; ++k) { rf[k] = (float)ph[k]; rf[NP + k] = (float)(ux * ph[k]); }
                for (int i = 0; i < NP; ++i)
                    for (int j = 0; j <= i; ++j) {
                        rf[70 + i * (i + 1) / 2 + j] = (float)(ph[i] * ph[j]);
                        rf[700 + i * (i + 1) / 2 + j] = (float)(ux * ph[i] * ph[j]);
                    }
            }
    rc = MEM_OK;
    if (!rc) rc = upload(&ctx->d_phiT, phiT);
    if (!rc) rc = upload(&ctx->d_logw, logw);
    if (!rc) rc = upload(&ctx->d_tab_solve, tabS);
    if (!rc) rc = upload(&ctx->d_tab_flux, tabF);
    if (!rc) rc = upload(&ctx->d_he1d, he1d);
    if (!rc) rc = upload(&ctx->d_x1d, x1d);
    if (!rc) rc = upload(&ctx->d_logw1d, lw1d);
    if (!rc) rc = build_slot_tables(ctx);
    if (!rc) rc = upload(&ctx->d_phiT64, phiT64);
    if (!rc) rc = upload(&ctx->d_logw64, logw64);
    if (!rc && (n == 8 || n == 12)) rc = mem_host::build_tc_tables(ctx, phi64);
    if (!rc)
        rc = mem_host::reserve_scratch(
            ctx, std::max(mem_host::plain_scratch_bytes(Q), mem_host::flux_scratch_bytes(Q)));
    if (rc) { mem_destroy(ctx); return rc; }
    if (cudaDeviceSynchronize() != cudaSuccess) { mem_destroy(ctx); return MEM_ECUDA; }
    if (const char *table = getenv("MEM_TUNE_TABLE")) mem_tune_load(ctx, table);  // a missing entry keeps the defaults
    *out = ctx;
    return MEM_OK;
}

int mem_init_velocity(int degree, int nbx, int nbr, int ng, int K, double ax, double bx, double br, mem_ctx **out) {
    if (!out) return MEM_EINVAL;
    *out = nullptr;
    if (degree != 4 || nbx < 1 || nbr < 1 || ng < 1 || ng > 16 || K < 1 || K > 64) return MEM_EINVAL;
    if (nbx * ng > 256 || nbr * ng * K > 1024 || !(bx > ax) || !(br > 0.0) || !isfinite(ax) || !isfinite(bx) ||
        !isfinite(br))
        return MEM_EINVAL;
    if (mem_host::vel_smem_bytes(nbx * ng, nbr * ng * K) > 227 * 1024) return MEM_EINVAL;
    mem_ctx *ctx = new mem_ctx();
    cudaGetDevice(&ctx->device);
    ctx->vel = 1;
    ctx->nbx = nbx; ctx->nbr = nbr; ctx->ng = ng; ctx->K = K;
    ctx->nx = nbx * ng;
    ctx->npt = nbr * ng * K;
    ctx->Q = ctx->nx * ctx->npt;
    ctx->dom[0] = ax; ctx->dom[1] = bx; ctx->dom[2] = br;
    std::vector<double> x, w;
    int rc = mem_host::gl_rule(ng, x, w);
    if (rc) { delete ctx; return rc; }
    std::vector<float> d0(mem_host::DOM_REC);
    mem_host::dom_record(ax, bx, br, nbx, nbr, d0.data());
    // Per-node constants of the rule: offsets in units of the block width
    // (x_i = a_x + h_x t_i; y_p = h_r t_m cos(2 pi k / K), z_p likewise with
    // sin, p = m K + k) and the log weights without the per-cell block widths.
    const int nx = nbx * ng, nr = nbr * ng;
    std::vector<double> vtd;
    std::vector<float> vtf;
    std::vector<float2> vt2;
    const double two_pi = 6.283185307179586476925286766559;
    std::vector<double> rt(nr);
    for (int m = 0; m < nr; ++m) rt[m] = (m / ng) + 0.5 * (x[m % ng] + 1.0);
    for (int i = 0; i < nx; ++i) vtd.push_back((i / ng) + 0.5 * (x[i % ng] + 1.0));
    for (int p = 0; p < nr * K; ++p) vtd.push_back(rt[p / K] * cos(two_pi * (p % K) / K));
    for (int p = 0; p < nr * K; ++p) vtd.push_back(rt[p / K] * sin(two_pi * (p % K) / K));
    for (int i = 0; i < nx; ++i) vtf.push_back((float)log(w[i % ng]));
    for (int m = 0; m < nr; ++m) vtf.push_back((float)log(w[m % ng] * rt[m] / K));
    for (double t : vtd) {
        const float hi = (float)t;
        vt2.push_back(make_float2(hi, (float)(t - (double)hi)));
    }
    if (!rc) rc = upload(&ctx->d_vt2, vt2);
    if (!rc) rc = upload(&ctx->d_vtf, vtf);
    if (!rc) rc = upload(&ctx->d_dom0, d0);
    if (!rc) rc = build_slot_tables(ctx);
    if (!rc) rc = mem_host::build_axi_tables(ctx);
    if (!rc) rc = mem_host::reserve_scratch(ctx, sizeof(float) * (size_t)VEL_FLUX_CHUNK * MEM_MU_STRIDE);
    if (rc) { mem_destroy(ctx); return rc; }
    if (cudaDeviceSynchronize() != cudaSuccess) { mem_destroy(ctx); return MEM_ECUDA; }
    if (const char *table = getenv("MEM_TUNE_TABLE")) mem_tune_load(ctx, table);  // a missing entry keeps the defaults
    *out = ctx;
    return MEM_OK;
}

int mem_velocity_rule(const mem_ctx *ctx, int32_t *shape, double *domain) {
    if (!ctx || !ctx->vel) return MEM_EINVAL;
    if (shape) { shape[0] = ctx->nbx; shape[1] = ctx->nbr; shape[2] = ctx->ng; shape[3] = ctx->K; }
    if (domain) { domain[0] = ctx->dom[0]; domain[1] = ctx->dom[1]; domain[2] = ctx->dom[2]; }
    return MEM_OK;
}

void mem_destroy(mem_ctx *ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    void *ptrs[] = {ctx->d_phiT, ctx->d_logw, ctx->d_tab_solve, ctx->d_tab_flux, ctx->d_he1d, ctx->d_x1d,
                    ctx->d_logw1d, ctx->d_lin_off, ctx->d_lin_terms, ctx->d_hess_slots, ctx->d_hess_slots128, ctx->d_hr_slots, ctx->d_hr_rounds, ctx->d_hr_ent, ctx->d_flux_slots, ctx->d_axi_slots, ctx->d_xlin_off, ctx->d_xlin_terms,
                    ctx->scratch, ctx->d_vt2, ctx->d_vtf, ctx->d_dom0, ctx->d_tc_tab, ctx->d_phiT64, ctx->d_logw64, ctx->d_axi_terms, ctx->d_axi_toff};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (ctx->scratch_ev) cudaEventDestroy(ctx->scratch_ev);
    delete ctx;
}

int mem_quad_order(const mem_ctx *ctx) { return ctx ? ctx->n1d : 0; }

int mem_solve(mem_ctx *ctx, const float *M, float *beta, int32_t *status, int32_t *iters, int64_t B,
              const mem_solve_opts *opts, void *stream) {
    if (!ctx || B < 0) return MEM_EINVAL;
    if (B == 0) return MEM_OK;
    if (!M || !beta) return MEM_EINVAL;
    mem_solve_opts o;
    mem_solve_opts_default(&o);
    if (opts) o = *opts;
    if (o.maxI < 0 || o.maxT < 0 || o.maxT > 60 || o.max_lambda < 0 || o.max_lambda > 60) return MEM_EINVAL;
    if (ctx->vel) return MEM_EINVAL;  // the rule follows the gauge: mem_solve_gauge
    cudaStream_t st = (cudaStream_t)stream;
    if (o.impl == MEM_IMPL_PLAIN) return mem_host::solve_plain(ctx, M, beta, status, iters, B, o, st);
    if (o.impl == MEM_IMPL_FUSED) return mem_host::solve_fused(ctx, M, beta, status, iters, B, o, st);
    if (o.impl == MEM_IMPL_MIXED) return mem_host::solve_mixed(ctx, M, beta, status, iters, B, o, st);
    return MEM_EINVAL;
}

int mem_solve_axi(mem_ctx *ctx, const float *M, float *beta, const float *gauge, int32_t *status, int32_t *iters,
                  float *F, float *speed, int64_t B, const mem_solve_opts *opts, void *stream) {
    if (!ctx || B < 0 || !ctx->vel) return MEM_EINVAL;
    if (B == 0) return MEM_OK;
    if (!M || !beta || !gauge) return MEM_EINVAL;
    mem_solve_opts o;
    mem_solve_opts_default(&o);
    if (opts) o = *opts;
    if (o.maxI < 0 || o.maxT < 0 || o.maxT > 60 || o.max_lambda < 0 || o.max_lambda > 60) return MEM_EINVAL;
    return mem_host::axi_run(ctx, M, beta, gauge, status, iters, F, speed, nullptr, nullptr, B, o, true,
                             (cudaStream_t)stream);
}

int mem_residual64(mem_ctx *ctx, const float *M, const float *beta, const int32_t *status, int32_t mask, double *res,
                   int32_t *status_out, double accept, int64_t B, void *stream) {
    if (!ctx || B < 0 || ctx->vel) return MEM_EINVAL;
    if (B == 0) return MEM_OK;
    if (!M || !beta || !res || (mask && !status)) return MEM_EINVAL;
    return mem_host::residual64(ctx, M, beta, status, mask, res, status_out, accept, B, (cudaStream_t)stream);
}

int mem_solve_gauge(mem_ctx *ctx, const float *M, float *beta, const float *gauge, int32_t *status, int32_t *iters,
                    int64_t B, const mem_solve_opts *opts, void *stream) {
    if (!ctx || B < 0) return MEM_EINVAL;
    if (!ctx->vel) return mem_solve(ctx, M, beta, status, iters, B, opts, stream);
    if (B == 0) return MEM_OK;
    if (!M || !beta || !gauge) return MEM_EINVAL;
    mem_solve_opts o;
    mem_solve_opts_default(&o);
    if (opts) o = *opts;
    if (o.maxI < 0 || o.maxT < 0 || o.maxT > 60 || o.max_lambda < 0 || o.max_lambda > 60) return MEM_EINVAL;
    return mem_host::vel_run(ctx, M, beta, gauge, status, iters, nullptr, nullptr, nullptr, B, o, true,
                             (cudaStream_t)stream);
}

// Flux and speed on a velocity-space context: moment rows into context
// scratch (chunked), then the shared flux/speed kernel.
static int vel_flux(mem_ctx *ctx, const float *M, const float *beta, const float *gauge, float *F, float *speed,
                    int64_t B, cudaStream_t st, bool axisym) {
    std::lock_guard<std::mutex> lock(ctx->mu);
    const int64_t CH = std::min<int64_t>(B, VEL_FLUX_CHUNK);
    int rc = mem_host::scratch_begin(ctx, sizeof(float) * (size_t)CH * MEM_MU_STRIDE, st);
    if (rc) return rc;
    float *mu = (float *)ctx->scratch;
    mem_solve_opts o;
    mem_solve_opts_default(&o);
    for (int64_t c0 = 0; c0 < B; c0 += CH) {
        const int64_t n = std::min<int64_t>(CH, B - c0);
        rc = mem_host::vel_run(ctx, M + c0 * NP, (float *)(beta + c0 * NP), gauge + c0 * 6, nullptr, nullptr, mu,
                               nullptr, nullptr, n, o, false, st);
        if (!rc)
            rc = mem_host::flux_from_mu(ctx, mu, M + c0 * NP, gauge + c0 * 6, F ? F + c0 * NP : nullptr,
                                        speed ? speed + c0 : nullptr, n, st, axisym);
        if (rc) break;
    }
    mem_host::scratch_end(ctx, st);
    return rc;
}

int mem_flux(mem_ctx *ctx, const float *M, const float *beta, const float *gauge, float *F, float *speed,
             int64_t B, void *stream) {
    if (!ctx || B < 0) return MEM_EINVAL;
    if (B == 0) return MEM_OK;
    if (!M || !beta || !gauge) return MEM_EINVAL;
    if (ctx->vel) return vel_flux(ctx, M, beta, gauge, F, speed, B, (cudaStream_t)stream, false);
    if (mem_host::flux_fused_available(ctx))
        return mem_host::flux_fused(ctx, M, beta, gauge, F, speed, B, (cudaStream_t)stream, false);
    return mem_host::flux(ctx, M, beta, gauge, F, speed, B, (cudaStream_t)stream);
}

int mem_flux_axisym(mem_ctx *ctx, const float *M, const float *beta, const float *gauge, float *F, float *speed,
                    int64_t B, void *stream) {
    if (!ctx || B < 0) return MEM_EINVAL;
    if (B == 0) return MEM_OK;
    if (!M || !beta || !gauge) return MEM_EINVAL;
    if (ctx->vel) return vel_flux(ctx, M, beta, gauge, F, speed, B, (cudaStream_t)stream, true);
    if (mem_host::flux_fused_available(ctx))
        return mem_host::flux_fused(ctx, M, beta, gauge, F, speed, B, (cudaStream_t)stream, true);
    return mem_host::flux(ctx, M, beta, gauge, F, speed, B, (cudaStream_t)stream);
}

int mem_gauge_hermite(mem_ctx *ctx, const float *M_in, const float *g_in, float *g_out, float *M_out,
                      float *beta_inout, int64_t B, int axisym, void *stream) {
    if (!ctx || B < 0) return MEM_EINVAL;
    if (B == 0) return MEM_OK;
    if (!M_in || !g_in || !g_out || !M_out) return MEM_EINVAL;
    return mem_host::gauge_hermite(ctx, M_in, g_in, g_out, M_out, beta_inout, B, axisym, (cudaStream_t)stream);
}

int mem_gauge_transform(mem_ctx *ctx, const float *g_to, const float *g_from, const float *M_in, float *M_out,
                        int64_t B, void *stream) {
    if (!ctx || B < 0) return MEM_EINVAL;
    if (B == 0) return MEM_OK;
    if (!g_to || !g_from || !M_in || !M_out) return MEM_EINVAL;
    return mem_host::gauge_transform(g_to, g_from, M_in, M_out, B, (cudaStream_t)stream);
}

int mem_targets(mem_ctx *ctx, int gen_order, const float *v, const float *T, const float *a, const float *b,
                float *M_out, float *g_out, int64_t B, void *stream) {
    if (!ctx || B < 0 || gen_order < 4 || gen_order > 32) return MEM_EINVAL;
    if (B == 0) return MEM_OK;
    if (!v || !T || !a || !b || !M_out || !g_out) return MEM_EINVAL;
    return mem_host::targets(ctx, gen_order, v, T, a, b, M_out, g_out, B, (cudaStream_t)stream);
}

}  // extern "C"

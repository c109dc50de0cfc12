// ffloat.cuh -- float-float (double-FP32) helpers for placing the nodes of a
// velocity-space rule in a cell's gauge without FP64 arithmetic: error-free
// products (FMA) and sums (Knuth's two-sum), renormalised once.
#pragma once

namespace mem {

// Float-float helpers (Dekker products with FMA; __fmul_rn keeps the
// products from being contracted).  1/s as rh + rl with one Newton correction.
__device__ __forceinline__ void ff_recip(float s, float &rh, float &rl) {
    rh = 1.f / s;
    rl = rh * fmaf(-s, rh, 1.f);
}
// d = a + h t - w in float-float arithmetic (a, h, t given as float pairs,
// w a float): an exact product and two exact sums (no rounding until the
// final renormalisation), d = dh + dl to about 2^-44 relative.  The _rn
// intrinsics keep the compiler from contracting or reordering the steps.
__device__ __forceinline__ void ff_offset(float ah, float al, float hh, float hl, float2 t, float w, float &dh,
                                          float &dl) {
    const float p = __fmul_rn(hh, t.x);
    const float pe = fmaf(hh, t.x, -p) + fmaf(hh, t.y, __fmul_rn(hl, t.x));
    const float s1 = __fadd_rn(ah, p), v1 = __fsub_rn(s1, ah);
    const float e1 = __fadd_rn(__fsub_rn(ah, __fsub_rn(s1, v1)), __fsub_rn(p, v1));
    const float s2 = __fsub_rn(s1, w), v2 = __fsub_rn(s2, s1);
    const float e2 = __fadd_rn(__fsub_rn(s1, __fsub_rn(s2, v2)), __fsub_rn(-w, v2));
    const float lo = __fadd_rn(__fadd_rn(e1, pe), __fadd_rn(al, e2));
    dh = __fadd_rn(s2, lo);
    dl = __fsub_rn(lo, __fsub_rn(dh, s2));
}
// ubar = d / s for d = dh + dl: ubar = uh + ul to about 2^-44 relative.
__device__ __forceinline__ void ff_ubar(float dh, float dl, float rh, float rl, float &uh, float &ul) {
    const float p = __fmul_rn(dh, rh);
    const float e = fmaf(dh, rh, -p);
    uh = p;
    ul = e + fmaf(dh, rl, dl * rh);
}
// ubar^2 / 2 = hs + hl.
__device__ __forceinline__ void ff_half_square(float uh, float ul, float &hs, float &hl) {
    const float q = __fmul_rn(uh, uh);
    const float qe = fmaf(uh, uh, -q);
    hs = 0.5f * q;
    hl = fmaf(uh, ul, 0.5f * qe);
}

}  // namespace mem

// ffmath.cuh -- float-float arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant
// bits.  Error-free transformations after Dekker (1971, the product through a
// fused multiply-add) and Knuth (TAOCP vol. 2, sec. 4.2.2, TwoSum); the
// "sloppy" addition, whose error is bounded relative to |a| + |b|, as for a
// FP64 accumulation.  Every rounding-sensitive step uses the explicit _rn
// intrinsics, so the compiler cannot contract or reorder it.
//
// ff2_sincos: Cody-Waite reduction by pi/2 (pi/2 split into three FP32
// parts, Cody & Waite 1980), then the Taylor series of sin and cos on
// |t| <= pi/4: the leading terms in float-float, the tail (below 3e-8 of the
// result) in FP32, and the quadrant from n mod 4.
#pragma once

#include <cuda_runtime.h>

struct ff {
    float hi, lo;
};

__host__ __device__ inline ff ff_make(double d) {
    const float h = (float)d;
    return ff{h, (float)(d - (double)h)};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return ff{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ ff ff_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return ff{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = ff_two_sum(a.hi, b.hi);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const ff p = ff_two_prod(a.hi, b.hi);
    return ff_fast_two_sum(p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo)));
}

__device__ __forceinline__ ff ff_fma(ff a, ff b, ff c) { return ff_add(ff_mul(a, b), c); }

__device__ __forceinline__ ff ff_sqrt(ff a) {  // a > 0
    const float s = __fsqrt_rn(a.hi);
    const ff p = ff_two_prod(s, s);
    const float d = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), a.lo);
    return ff_fast_two_sum(s, __fmul_rn(d, __fdiv_rn(0.5f, s)));
}

__device__ __forceinline__ ff ff_rcp(ff a) {  // a != 0
    const float y = __frcp_rn(a.hi);
    const ff p = ff_two_prod(a.hi, y);
    const float e = __fmaf_rn(-a.lo, y, __fsub_rn(__fsub_rn(1.f, p.hi), p.lo));
    return ff_fast_two_sum(y, __fmul_rn(y, e));
}

__device__ __forceinline__ ff ff_dot3(const ff *a, const ff *b) {
    return ff_add(ff_add(ff_mul(a[0], b[0]), ff_mul(a[1], b[1])), ff_mul(a[2], b[2]));
}

// ---- two float-float numbers packed into FP32x2 lanes -------------------
// The same algorithms on float2 pairs with the packed FP32x2 instructions
// (one instruction per step for both lanes); lane x and lane y are
// independent numbers (two wavenumbers, or the real and imaginary parts).
struct ff2 {
    float2 hi, lo;
};

__device__ __forceinline__ float2 f2_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2_dup(float a) { return make_float2(a, a); }
__device__ __forceinline__ ff2 ff2_make(ff x, ff y) {
    return ff2{make_float2(x.hi, y.hi), make_float2(x.lo, y.lo)};
}
__device__ __forceinline__ ff2 ff2_dup(ff a) { return ff2{f2_dup(a.hi), f2_dup(a.lo)}; }
__device__ __forceinline__ ff ff2_x(ff2 a) { return ff{a.hi.x, a.lo.x}; }
__device__ __forceinline__ ff ff2_y(ff2 a) { return ff{a.hi.y, a.lo.y}; }
__device__ __forceinline__ ff2 ff2_neg(ff2 a) { return ff2{f2_neg(a.hi), f2_neg(a.lo)}; }

__device__ __forceinline__ ff2 ff2_fast_two_sum(float2 a, float2 b) {
    const float2 s = __fadd2_rn(a, b);
    return ff2{s, __fadd2_rn(b, f2_neg(__fadd2_rn(s, f2_neg(a))))};
}

__device__ __forceinline__ ff2 ff2_two_sum(float2 a, float2 b) {
    const float2 s = __fadd2_rn(a, b);
    const float2 bb = __fadd2_rn(s, f2_neg(a));
    const float2 ea = __fadd2_rn(a, f2_neg(__fadd2_rn(s, f2_neg(bb))));
    return ff2{s, __fadd2_rn(ea, __fadd2_rn(b, f2_neg(bb)))};
}

__device__ __forceinline__ ff2 ff2_two_prod(float2 a, float2 b) {
    const float2 p = __fmul2_rn(a, b);
    return ff2{p, __ffma2_rn(a, b, f2_neg(p))};
}

__device__ __forceinline__ ff2 ff2_add(ff2 a, ff2 b) {
    const ff2 s = ff2_two_sum(a.hi, b.hi);
    return ff2_fast_two_sum(s.hi, __fadd2_rn(s.lo, __fadd2_rn(a.lo, b.lo)));
}

__device__ __forceinline__ ff2 ff2_sub(ff2 a, ff2 b) { return ff2_add(a, ff2_neg(b)); }

__device__ __forceinline__ ff2 ff2_mul(ff2 a, ff2 b) {
    const ff2 p = ff2_two_prod(a.hi, b.hi);
    return ff2_fast_two_sum(p.hi, __ffma2_rn(a.hi, b.lo, __ffma2_rn(a.lo, b.hi, p.lo)));
}

__device__ __forceinline__ ff2 ff2_fma(ff2 a, ff2 b, ff2 c) { return ff2_add(ff2_mul(a, b), c); }

// sin and cos of both lanes, x >= 0 (|x| < 2^22 pi/2)
__device__ __forceinline__ void ff2_sincos(ff2 x, ff2 &s, ff2 &c) {
    // pi/2 = P1 + P2 + P3 (each the FP32 rounding of what is left)
    const float P1 = 1.5707963705062866f, P2 = -4.371138828673793e-08f, P3 = -1.7151245100058819e-15f;
    const float2 xh = __fmul2_rn(x.hi, f2_dup(0.6366197466850281f));
    const float2 n = make_float2(rintf(xh.x), rintf(xh.y));
    ff2 t = ff2_sub(x, ff2_two_prod(n, f2_dup(P1)));
    t = ff2_sub(t, ff2_two_prod(n, f2_dup(P2)));
    t = ff2_add(t, ff2{__fmul2_rn(f2_neg(n), f2_dup(P3)), f2_dup(0.f)});
    const ff2 u = ff2_mul(t, t);
    const float2 uh = u.hi;
    auto K = [](float h, float l) { return ff2{f2_dup(h), f2_dup(l)}; };
    // sin t = t (1 - u/3! + u^2/5! - ... ), u = t^2; terms from u^5 in FP32
    float2 ts = __ffma2_rn(uh, f2_dup(2.8114573589663704e-15f), f2_dup(-7.647163609812713e-13f));
    ts = __ffma2_rn(uh, ts, f2_dup(1.6059044372074283e-10f));
    ts = __ffma2_rn(uh, ts, f2_dup(-2.5052107943679403e-08f));
    ff2 ps = ff2_fma(ff2{ts, f2_dup(0.f)}, u, K(2.7557318844628753e-06f, 3.793571224297229e-14f));
    ps = ff2_fma(ps, u, K(-0.00019841270113829523f, 2.725596874933456e-12f));
    ps = ff2_fma(ps, u, K(0.008333333767950535f, -4.34617203337595e-10f));
    ps = ff2_fma(ps, u, K(-0.1666666716337204f, 4.967053879312289e-09f));
    ps = ff2_fma(ps, u, K(1.f, 0.f));
    const ff2 st = ff2_mul(ps, t);
    // cos t = 1 - u/2! + u^2/4! - ... ; terms from u^6 in FP32
    float2 tc = __ffma2_rn(uh, f2_dup(4.7794772561329454e-14f), f2_dup(-1.147074536050896e-11f));
    tc = __ffma2_rn(uh, tc, f2_dup(2.0876755879584152e-09f));
    ff2 pc = ff2_fma(ff2{tc, f2_dup(0.f)}, u, K(-2.755731998149713e-07f, 7.575112209051195e-15f));
    pc = ff2_fma(pc, u, K(2.4801587642286904e-05f, -3.40699609366682e-13f));
    pc = ff2_fma(pc, u, K(-0.0013888889225199819f, 3.3631094437103215e-11f));
    pc = ff2_fma(pc, u, K(0.0416666679084301f, -1.2417634698280722e-09f));
    pc = ff2_fma(pc, u, K(-0.5f, 0.f));
    const ff2 ct = ff2_fma(pc, u, K(1.f, 0.f));
    // quadrant per lane
    ff sl[2], cl[2];
    const ff stl[2] = {ff2_x(st), ff2_y(st)}, ctl[2] = {ff2_x(ct), ff2_y(ct)};
    const int q[2] = {((int)n.x) & 3, ((int)n.y) & 3};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        if (q[i] == 0) { sl[i] = stl[i]; cl[i] = ctl[i]; }
        else if (q[i] == 1) { sl[i] = ctl[i]; cl[i] = ff_neg(stl[i]); }
        else if (q[i] == 2) { sl[i] = ff_neg(stl[i]); cl[i] = ff_neg(ctl[i]); }
        else { sl[i] = ff_neg(ctl[i]); cl[i] = stl[i]; }
    }
    s = ff2_make(sl[0], sl[1]);
    c = ff2_make(cl[0], cl[1]);
}

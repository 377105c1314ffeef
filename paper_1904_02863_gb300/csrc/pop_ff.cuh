// Float-float ("double-single") arithmetic on packed sample pairs.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2,
// about 48 significant bits; an ff2 holds two such values (the two samples of a pair)
// in packed f32x2 registers.  GB300 runs FP32 at 64 times its FP64 rate, so FP64-grade
// arithmetic costs several times less this way than on the FP64 pipe.
//
// The error-free transformations are the classic ones: two-sum (Knuth), fast-two-sum
// (Dekker; |a| >= |b|) and the FMA two-product.  The addition keeps one two-sum of the
// high parts (absolute error a few 2^-48 (|x| + |y|)), the products have relative error
// a few 2^-48.  Every product error term is an explicit fma.  A product whose rounded value
// takes part in an error term is itself an fma with a zero addend that the compiler cannot
// see (z, from a kernel parameter): the compiler contracts a packed mul.rn.f32x2 into a
// following add/sub.rn.f32x2 otherwise, with or without --fmad=false (measured: the
// fast-two-sum after a product then returned s - x y rounded once instead of its error).
//
// exp and expm1 follow Tang's table method (P. T. P. Tang, ACM TOMS 15 (1989) 144-157):
// x = (2048 m + j) ln2/2048 + r with |r| <= ln2/4096, the reduction in float-float (k ln2/2048
// from a two-product with the hi part of the constant and a product with its lo part),
// e^r - 1 = r + r^2 (1/2 + r/6) (the next term, r^4/24 < 4e-17), and 2^(j/2048) from a table
// of (hi, lo) FP32 pairs built on the host in extended precision.  Results under the FP32
// normal range (about e^-87) give 0; a caller can shift the range by a power of two.
#pragma once

#include "pop_f32x2.cuh"

namespace pop {

constexpr int FF_TABLE_BITS = 11;
constexpr int FF_TABLE_SIZE = 1 << FF_TABLE_BITS;  // 2048 (hi, lo) FP32 pairs

// Reduction constants: 2048/ln2, and ln2/2048 = l_hi + l_lo (l_hi the nearest float); zero is 0,
// passed at run time so that fma(a, b, zero) stays a product rounded on its own.
struct FFConsts {
    float inv_l, l_hi, l_lo, zero;
};

struct ff2 {
    f2 hi, lo;
};

// A per-lane constant in both halves.
__device__ __forceinline__ ff2 ff_const(double x)
{
    const float h = (float)x;
    const float l = (float)(x - (double)h);
    return ff2{bc(h), bc(l)};
}

// s + e == a + b exactly.
__device__ __forceinline__ ff2 two_sum2(f2 a, f2 b)
{
    const f2 s = add2(a, b);
    const f2 bb = sub2(s, a);
    return ff2{s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}

// s + e == a + b exactly when |a| >= |b| or a == 0.
__device__ __forceinline__ ff2 fast_two_sum2(f2 a, f2 b)
{
    const f2 s = add2(a, b);
    return ff2{s, sub2(b, sub2(s, a))};
}

__device__ __forceinline__ ff2 ff_add(ff2 x, ff2 y)
{
    const ff2 s = two_sum2(x.hi, y.hi);
    return fast_two_sum2(s.hi, add2(s.lo, add2(x.lo, y.lo)));
}

// fl(a b), never merged into a later addition (z is a run-time zero).
__device__ __forceinline__ f2 prod2(f2 a, f2 b, f2 z) { return fma2(a, b, z); }

// x y: p = fl(x.hi y.hi), e = x.hi y.hi - p exactly (fma), plus the cross terms.
__device__ __forceinline__ ff2 ff_mul(ff2 x, ff2 y, f2 z)
{
    const f2 p = prod2(x.hi, y.hi, z);
    f2 e = fma2(x.hi, y.hi, sub2(0ull, p));
    e = fma2(x.hi, y.lo, e);
    e = fma2(x.lo, y.hi, e);
    return fast_two_sum2(p, e);
}

// x c + y.
__device__ __forceinline__ ff2 ff_fma(ff2 x, ff2 c, ff2 y, f2 z) { return ff_add(ff_mul(x, c, z), y); }

__device__ __forceinline__ ff2 ff_neg(ff2 x) { return ff2{sub2(0ull, x.hi), sub2(0ull, x.lo)}; }

// A compensated sum of products and float-float terms (Ogita, Rump and Oishi's Dot2, SIAM J.
// Sci. Comput. 26 (2005) 1955-1988, with float-float inputs): s is the running FP32 sum of the
// terms' leading parts, kept by two-sums; c collects every rounding error and every lower-order
// part, in FP32.  ff() renormalises once at the end.  Error: a few 2^-48 of the sum of the
// terms' magnitudes, as a chain of float-float additions, with fewer operations.
struct FFAcc {
    f2 s, c;
};

__device__ __forceinline__ FFAcc acc_of(ff2 x) { return FFAcc{x.hi, x.lo}; }

// a + x
__device__ __forceinline__ FFAcc acc_add(FFAcc a, ff2 x)
{
    const ff2 t = two_sum2(a.s, x.hi);
    return FFAcc{t.hi, add2(a.c, add2(t.lo, x.lo))};
}

// a + x y: the product's leading part fl(x.hi y.hi) enters the two-sum, its exact error and the
// cross terms x.hi y.lo + x.lo y.hi go to c.
__device__ __forceinline__ FFAcc acc_add_prod(FFAcc a, ff2 x, ff2 y, f2 z)
{
    const f2 p = prod2(x.hi, y.hi, z);
    f2 e = fma2(x.hi, y.hi, sub2(0ull, p));
    e = fma2(x.hi, y.lo, e);
    e = fma2(x.lo, y.hi, e);
    const ff2 t = two_sum2(a.s, p);
    return FFAcc{t.hi, add2(a.c, add2(t.lo, e))};
}

__device__ __forceinline__ ff2 acc_ff(FFAcc a) { return fast_two_sum2(a.s, a.c); }

// 1/x for normal x of either sign: the hardware seed y0 and one Newton step in float-float,
// y = y0 + y0 (1 - x y0) (relative error about the square of the seed's, 2e-14, plus rounding).
__device__ __forceinline__ ff2 ff_rcp(ff2 x, f2 z)
{
    float xa, xb;
    upk(x.hi, xa, xb);
    const f2 y0 = pk(rcpf(xa), rcpf(xb));
    const f2 p = prod2(x.hi, y0, z);
    const f2 pe = fma2(x.hi, y0, sub2(0ull, p));                 // x.hi y0 - p exactly
    const f2 e = sub2(sub2(bc(1.0f), p), fma2(x.lo, y0, pe));    // 1 - x y0 (small)
    return fast_two_sum2(y0, prod2(y0, e, z));
}

// The reduction shared by exp and expm1: returns e^r - 1 as float-float and, per half, the
// table index j and the power m.
__device__ __forceinline__ ff2 ff_exp_reduce(ff2 x, const FFConsts& k, int& ja, int& jb, int& ma, int& mb)
{
    float xa, xb;
    upk(x.hi, xa, xb);
    const float ka = rintf(xa * k.inv_l), kb = rintf(xb * k.inv_l);
    const f2 kf = pk(ka, kb);
    const f2 z = bc(k.zero);
    const f2 q = prod2(kf, bc(-k.l_hi), z);                        // -fl(k l_hi)
    const f2 e = fma2(kf, bc(k.l_hi), q);                          // k l_hi - fl(k l_hi)
    const f2 rh = add2(x.hi, q);                                    // exact (Sterbenz) for k != 0
    const f2 rl = fma2(kf, bc(-k.l_lo), sub2(x.lo, e));
    const ff2 r = fast_two_sum2(rh, rl);
    const f2 rr = prod2(r.hi, r.hi, z);
    const f2 t = prod2(rr, fma2(r.hi, bc(1.0f / 6.0f), bc(0.5f)), z);  // r^2/2 + r^3/6
    ff2 p = fast_two_sum2(r.hi, t);
    p.lo = add2(p.lo, r.lo);
    const int ia = (int)ka, ib = (int)kb;
    ja = ia & (FF_TABLE_SIZE - 1);
    jb = ib & (FF_TABLE_SIZE - 1);
    ma = ia >> FF_TABLE_BITS;  // arithmetic shift: floor
    mb = ib >> FF_TABLE_BITS;
    return p;
}

__device__ __forceinline__ float pow2i(int m) { return __int_as_float((m + 127) << 23); }  // -126 <= m <= 127

// T (1 + p) with T = T_hi + T_lo from the table: T_hi + [T_hi p_hi]_exact + T_hi p_lo + T_lo (1 + p_hi).
__device__ __forceinline__ ff2 ff_table_times(f2 th, f2 tl, ff2 p, f2 z)
{
    const f2 nq = prod2(th, sub2(0ull, p.hi), z);                // -fl(T_hi p_hi)
    const f2 pe = fma2(th, p.hi, nq);                            // T_hi p_hi - fl(T_hi p_hi)
    const f2 s = sub2(th, nq);                                   // T_hi + fl(T_hi p_hi)
    const f2 se = sub2(sub2(th, s), nq);                         // its rounding error (|T_hi| >= |T_hi p_hi|)
    f2 lo = add2(se, pe);
    lo = add2(lo, tl);
    lo = fma2(tl, p.hi, lo);
    lo = fma2(th, p.lo, lo);
    return fast_two_sum2(s, lo);
}

// e^x 2^-sh: 0 where the result falls under the FP32 normal range, +inf above it (NaN gives 0).
// sh lets a caller keep a run of tiny or huge exponentials in range with an exact power-of-two
// scale of its own.
__device__ __forceinline__ ff2 ff_exp(ff2 x, const float2* __restrict__ tab, const FFConsts& k, int sh = 0)
{
    int ja, jb, ma, mb;
    float xa, xb;
    upk(x.hi, xa, xb);
    // The reduction needs |x| well inside the int range of k: larger arguments, and NaN, are
    // evaluated at 0 and replaced after.
    const bool fa = fabsf(xa) < 1.0e6f, fb = fabsf(xb) < 1.0e6f;
    ff2 xs = x;
    if (!(fa & fb)) {
        float la, lb;
        upk(x.lo, la, lb);
        xs = ff2{pk(fa ? xa : 0.0f, fb ? xb : 0.0f), pk(fa ? la : 0.0f, fb ? lb : 0.0f)};
    }
    const ff2 p = ff_exp_reduce(xs, k, ja, jb, ma, mb);
    ma -= sh;
    mb -= sh;
    const bool ua = fa ? ma < -126 : !(xa > 0.0f), ub = fb ? mb < -126 : !(xb > 0.0f);
    const bool oa = fa ? ma > 127 : xa > 0.0f, ob = fb ? mb > 127 : xb > 0.0f;
    const float2 Ta = tab[ja], Tb = tab[jb];
    const f2 z = bc(k.zero);
    ff2 r = ff_table_times(pk(Ta.x, Tb.x), pk(Ta.y, Tb.y), p, z);
    const f2 sc = pk(pow2i(min(max(ma, -126), 127)), pow2i(min(max(mb, -126), 127)));
    r.hi = prod2(r.hi, sc, z);
    r.lo = prod2(r.lo, sc, z);
    if (ua | oa | ub | ob) {
        float ha, hb, la, lb;
        upk(r.hi, ha, hb);
        upk(r.lo, la, lb);
        const float inf = __int_as_float(0x7f800000);
        ha = ua ? 0.0f : (oa ? inf : ha);
        la = (ua | oa) ? 0.0f : la;
        hb = ub ? 0.0f : (ob ? inf : hb);
        lb = (ub | ob) ? 0.0f : lb;
        r = ff2{pk(ha, hb), pk(la, lb)};
    }
    return r;
}

// e^u - 1 for -87 <= u <= 88 and |u| >= 1/16 (no cancellation worth a series):
// (2^m T_hi - 1) + 2^m (T (1 + p) - T_hi), the first part an exact two-sum.
__device__ __forceinline__ ff2 ff_expm1_far(ff2 u, const float2* __restrict__ tab, const FFConsts& k)
{
    int ja, jb, ma, mb;
    const ff2 p = ff_exp_reduce(u, k, ja, jb, ma, mb);
    const float2 Ta = tab[ja], Tb = tab[jb];
    const f2 th = pk(Ta.x, Tb.x);
    const f2 z = bc(k.zero);
    ff2 t = ff_table_times(th, pk(Ta.y, Tb.y), p, z);
    const f2 sc = pk(pow2i(ma), pow2i(mb));
    const f2 s = prod2(th, sc, z);                     // 2^m T_hi, exact
    const ff2 a = two_sum2(s, bc(-1.0f));               // 2^m T_hi - 1, exact
    // t - T_hi: t.hi and T_hi are within a factor 2 (Sterbenz), so the difference is exact.
    const ff2 b = ff2{prod2(sub2(t.hi, th), sc, z), prod2(t.lo, sc, z)};
    return ff_add(a, b);
}

// e^u - 1 for |u| < 1/16 by its Taylor series, u (1 + u/2 + u^2/6 + u^3/24 + u^4/120 + u^5 t(u)):
// the coefficients to 1/120 in float-float, t(u) = 1/720 + u/5040 + u^2/40320 + u^3/362880 in
// FP32 (relative to |u|: truncation u^8/9! < 1e-16, the FP32 tail's rounding u^4 t 2^-22 < 5e-15).
struct FFSeries {
    ff2 c6, c24, c120;
};

__device__ __forceinline__ FFSeries ff_series_consts()
{
    return FFSeries{ff_const(1.0 / 6.0), ff_const(1.0 / 24.0), ff_const(1.0 / 120.0)};
}

__device__ __forceinline__ ff2 ff_expm1_near(ff2 u, const FFSeries& c, f2 z)
{
    f2 t = fma2(u.hi, bc(1.0f / 362880.0f), bc(1.0f / 40320.0f));
    t = fma2(t, u.hi, bc(1.0f / 5040.0f));
    t = fma2(t, u.hi, bc(1.0f / 720.0f));
    ff2 P = ff_add(ff_mul(u, ff2{t, 0ull}, z), c.c120);  // 1/120 + u t
    P = ff_add(ff_mul(P, u, z), c.c24);                    // 1/24 + u (...)
    P = ff_add(ff_mul(P, u, z), c.c6);                     // 1/6 + u (...)
    P = ff_add(ff_mul(P, u, z), ff2{bc(0.5f), 0ull});      // 1/2 + u (...)
    P = ff_add(ff_mul(P, u, z), ff2{bc(1.0f), 0ull});      // 1 + u (...)
    return ff_mul(P, u, z);
}

}  // namespace pop

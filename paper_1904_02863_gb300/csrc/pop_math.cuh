// FP64 exponential, expm1, log1p near 0 and reciprocal for the FP64 kernels.
//
// GB300 runs FP64 at 2 FMA lanes per SM per clock (1/64 of FP32), so the
// weight kernel is bound by the number of FP64 instructions per pair; these
// versions use as few as the accuracy allows and push the rest (table lookup,
// exponent scaling, range tests) onto the integer and load pipes.
//
// exp / expm1: P. T. P. Tang, "Table-driven implementation of the exponential
// function in IEEE floating-point arithmetic", ACM TOMS 15 (1989) 144-157.
// x is written as (2048 m + j) ln2/2048 + r with |r| <= ln2/4096, so
// exp(x) = 2^m 2^(j/2048) e^r; 2^(j/2048) comes from a 2048-entry table held as
// hi + lo doubles (built on the host in extended precision), e^r - 1 from its
// Taylor series to r^3 for exp (truncation r^4/24 < 4e-17 of a result near 1)
// and to r^4 for expm1 (whose result can be as small as r).
//
// The index k = m 2048 + j, the integer nearest to x 2048/ln2, is found off the FP64
// pipe: an FP32 image of x (its top 24 significant bits, assembled from the bit
// pattern by integer operations), one FP32 fma with the 1.5 2^23 rounding shift, and
// kd = (double)k assembled from k's bits.  The FP32 rounding leaves k within one of
// the nearest integer: |x 2048/ln2 - k| <= 0.5 + |x| 5.3e-4 (the image's truncation,
// 2^-23, and fl32(2048/ln2), 2^-24, relative), so |r| <= 0.51 ln2/2048 for |x| <= 20
// and 0.88 ln2/2048 at the ends of the range.  The exp series' truncation r^4/24 stays
// below 5e-17 relative for |x| <= 20 (3.4e-17 with exact rounding) and 3.3e-16 at
// |x| = 709; expm1's, r^4/120 relative to the result, below 7e-17.  Only the
// reduction's fma and the series remain on the FP64 pipe.
//
// The reduction r = x - kd l takes one fma with l = fl(ln2/2048), not Tang's
// two-part constant.  l carries the relative error of fl(ln 2), 3.35e-17, so r
// is off by at most |kd| l 3.35e-17 ~ |x| 3.35e-17: the result gains |x| 3.35e-17
// relative error (0.31 |x| ulp) over the two-part form.  An argument that comes
// out of a rounded FP64 operation already carries up to |x| 1.1e-16, so the
// second fma of the two-part form buys accuracy below that floor, at the cost of
// one FP64 operation per exponential (the weight has four).  For expm1 the added
// error is also relative to the result: for |kd| >= 1 the result is at least
// about kd l / 2 in magnitude, and for kd = 0, r = u exactly.
//
// exp(x) for x < -707 (results below ~1e-307) is returned as 0, and above 709.7 as +inf.
#pragma once

#include <stdint.h>

namespace pop {

constexpr int EXP_TABLE_BITS = 11;
constexpr int EXP_TABLE_SIZE = 1 << EXP_TABLE_BITS;   // 2048 entries of (hi, lo)

// Reduction constants (computed once on the host from long double ln 2).
struct ExpConsts {
    float inv_l;    // 2048 / ln 2, rounded to FP32 (the index is formed in FP32)
    double l;       // ln 2 / 2048, rounded to nearest
};

// Arguments whose result (and 2^m scaling) stays a normal double.
constexpr double EXP_X_MIN = -707.0;
constexpr double EXP_X_MAX = 709.7;

__device__ __forceinline__ int64_t bits_of(double x) { return __double_as_longlong(x); }

// k within one of the integer nearest to x 2048/ln2, for |x| < 1024, with no FP64 instruction.
// The FP32 image of x: the bit pattern shifted left by 3 puts the low 9 exponent bits and the
// top 23 mantissa bits in the upper word; subtracting 384 from those 9 bits turns a double
// exponent e in [897, 1033] into the float exponent e - 896 (mod 512, with the float's sign bit
// left clear), and |x| below 2^-126 becomes 0.  Then k = rn(x' 2048/ln2 + 1.5 2^23) - 1.5 2^23,
// read off the sum's bit pattern (|x' 2048/ln2| < 2^22).
__device__ __forceinline__ int exp_index(double x, float inv_l)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned y = (__funnelshift_l(lo, hi, 3) - (384u << 23)) | (hi & 0x80000000u);
    const float xf = (hi & 0x7fffffffu) >= (897u << 20) ? __uint_as_float(y) : 0.0f;
    return __float_as_int(fmaf(xf, inv_l, 12582912.0f)) - 0x4B400000;
}

// (double)k, exact for |k| < 2^31, from k's bits: the leading one of |k| shifted to bit 31 and
// then to bit 20 of the high word, where it adds one to the biased exponent 1053 - clz(|k|).
__device__ __forceinline__ double dbl_of_int(int k)
{
    const unsigned a = (unsigned)abs(k);
    const int lz = __clz(a);
    const unsigned m = a << (lz & 31);
    const unsigned hi = (((unsigned)(1053 - lz) << 20) + (m >> 11)) | ((unsigned)k & 0x80000000u);
    return a ? __hiloint2double((int)hi, (int)(m << 21)) : 0.0;
}

// exp(x).  tab = [hi, lo] pairs in shared memory.
__device__ __forceinline__ double exp_tab(double x, const double2* __restrict__ tab, const ExpConsts& k)
{
    // Range tests on bit patterns (integer pipe): x < EXP_X_MIN or x > EXP_X_MAX (or -inf/+inf).
    const int64_t b = bits_of(x);
    const bool under = (uint64_t)b > (uint64_t)bits_of(EXP_X_MIN);  // negative and below the range
    const bool over = b > bits_of(EXP_X_MAX);                         // positive and above the range
    const double xs = (under | over) ? 0.0 : x;
    const int n = exp_index(xs, k.inv_l);
    const double r = fma(dbl_of_int(n), -k.l, xs);
    const double p = fma(fma(r, 1.0 / 6.0, 0.5), r * r, r);  // e^r - 1
    // 2^(j/2048) e^r in [0.99, 2.01): the correctly rounded T_hi alone keeps the result
    // within about one ulp (the lo part matters only for expm1's cancellation).
    const double th = tab[n & (EXP_TABLE_SIZE - 1)].x;
    const double res = fma(th, p, th);
    const int m = n >> EXP_TABLE_BITS;                       // arithmetic shift: floor
    const double scaled = __hiloint2double(__double2hiint(res) + (int)((unsigned)m << 20), __double2loint(res));
    return under ? 0.0 : (over ? __longlong_as_double(0x7ff0000000000000LL) : scaled);
}

// expm1(u) for EXP_X_MIN <= u <= EXP_X_MAX: (2^m T_hi - 1) + 2^m (T_hi p + T_lo).  When m = j = 0
// this is p itself, so tiny arguments keep full relative accuracy; 2^m T_hi - 1 is exact when
// 2^m T_hi is within a factor of two of 1.
__device__ __forceinline__ double expm1_tab(double u, const double2* __restrict__ tab, const ExpConsts& k)
{
    const int64_t b = bits_of(u);
    const bool under = (uint64_t)b > (uint64_t)bits_of(EXP_X_MIN);
    const bool over = b > bits_of(EXP_X_MAX);
    const double us = (under | over) ? 0.0 : u;
    const int n = exp_index(us, k.inv_l);
    const double r = fma(dbl_of_int(n), -k.l, us);
    // To r^4 here: near the first table steps the result is as small as ~1.7e-4, so the
    // truncation must be small relative to r, not to 1 (r^5/120 / r < 1e-17).
    const double p = fma(fma(fma(r, 1.0 / 24.0, 1.0 / 6.0), r, 0.5), r * r, r);
    const double2 tj = tab[n & (EXP_TABLE_SIZE - 1)];
    const int m = n >> EXP_TABLE_BITS;
    const double s = __hiloint2double(__double2hiint(tj.x) + (int)((unsigned)m << 20), __double2loint(tj.x));
    const double sc = __hiloint2double((m + 1023) << 20, 0);                                     // 2^m
    const double res = fma(fma(tj.x, p, tj.y), sc, s - 1.0);
    return under ? -1.0 : (over ? __longlong_as_double(0x7ff0000000000000LL) : res);
}

// |bits(m1) - bits(mmin)| below 2^46 means m1/mmin - 1 is below ~2^-6: there
// ln(mmin/m1) is taken as log1p((mmin - m1)/m1) by the series below, since the
// difference of the two logs would cancel.
constexpr long long NEAR_EDGE_BITS = 1LL << 46;

// log1p(t) for |t| < 2^-5 from its Taylor series to t^12 (truncation < 1e-19
// relative).
__device__ __forceinline__ double log1p_near0(double t)
{
    double p = -1.0 / 12;
    p = fma(p, t, 1.0 / 11);
    p = fma(p, t, -1.0 / 10);
    p = fma(p, t, 1.0 / 9);
    p = fma(p, t, -1.0 / 8);
    p = fma(p, t, 1.0 / 7);
    p = fma(p, t, -1.0 / 6);
    p = fma(p, t, 1.0 / 5);
    p = fma(p, t, -1.0 / 4);
    p = fma(p, t, 1.0 / 3);
    p = fma(p, t, -1.0 / 2);
    p = fma(p, t, 1.0);
    return p * t;
}

// 1/d for positive normal d: the hardware seed (rcp.approx.ftz.f64) refined by one cubic
// Newton step y = y0 (1 + e + e^2), e = 1 - d y0 (error e^3).
__device__ __forceinline__ double rcp_pos(double d)
{
    double y0;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(d));
    const double e = fma(-d, y0, 1.0);
    return fma(fma(e, e, e), y0, y0);
}

}  // namespace pop

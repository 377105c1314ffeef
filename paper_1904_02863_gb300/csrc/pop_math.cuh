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
// Taylor series.
//
// The index k = m 2048 + j, the integer nearest to x 2048/ln2, is found off the FP64
// pipe: an FP32 image of x (its top 24 significant bits, assembled from the bit
// pattern by integer operations), one FP32 fma with the 1.5 2^23 rounding shift, and
// kd = (double)k assembled from k's bits.  The FP32 rounding leaves k within one of
// the nearest integer: |x 2048/ln2 - k| <= 0.5 + |x| 5.3e-4 (the image's truncation,
// 2^-23, and fl32(2048/ln2), 2^-24, relative), so |r| <= 0.51 ln2/2048 for |x| <= 20
// and 0.88 ln2/2048 (3e-4) at the ends of the range.
//
// exp takes k near floor(x 2048/ln2) instead (r in [-0.44, 1.44] ln2/2048) and never forms
// e^r - 1 in FP64: the table value times 1 + c, c = e^r - 1 - r, lies in [1, 2), so T_hi + T_lo +
// T_hi c is T_hi's bit pattern plus an integer that FP32 arithmetic and integer operations
// give, and exp(x) = 2^m fma(T_hi, r, that): 2 FP64 operations, within one ulp (exp_t2).
//
// expm1 keeps the nearest k (so that k = 0 and the result is e^r - 1 itself for |u| below
// ln2/4096) and the series e^r - 1 = r + r^2 q, q = 1/2 + r/6 + r^2/24 + r^3/120 (truncation
// r^6/720): q lies within 5e-5 of 1/2, so its tail is formed in FP32 (an FP32 pair, since the
// result can be as small as r), turned into a fixed-point integer and added to the bit pattern
// of 1/2.  What stays on the FP64 pipe is the reduction's fma, r^2, the fma r + r^2 q and the
// reconstruction: 6 operations.
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

// The FP32 image of x for 2^-126 <= |x| < 1024: its top 24 significant bits (truncated), with
// no FP64 instruction; smaller |x| gives 0.  The bit pattern shifted left by 3 puts the low 9
// exponent bits and the top 23 mantissa bits in the upper word; subtracting 384 from those 9 bits
// turns a double exponent e in [897, 1033] into the float exponent e - 896 (mod 512, with the
// float's sign bit left clear).
__device__ __forceinline__ float f32_image(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned y = (__funnelshift_l(lo, hi, 3) - (384u << 23)) | (hi & 0x80000000u);
    return (hi & 0x7fffffffu) >= (897u << 20) ? __uint_as_float(y) : 0.0f;
}

// The rest of x after its image, x - f32_image(x), rounded to FP32: the low 29 mantissa bits
// scaled by 2^(e - 1075); 0 where that scale is below the FP32 normal range (|x| < 2^-74).
__device__ __forceinline__ float f32_image_rest(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned e = (hi >> 20) & 0x7ffu;
    const float v = __fmul_rn(__uint2float_rn(lo & 0x1fffffffu), __uint_as_float((e - 948u) << 23));
    return e >= 949u ? __uint_as_float(__float_as_uint(v) | (hi & 0x80000000u)) : 0.0f;
}

// k within one of the integer nearest to x 2048/ln2, for |x| < 1024, with no FP64 instruction:
// k = rn(x' 2048/ln2 + 1.5 2^23) - 1.5 2^23 with x' = f32_image(x), read off the sum's bit
// pattern (|x' 2048/ln2| < 2^22).
__device__ __forceinline__ int exp_index(double x, float inv_l)
{
    return __float_as_int(fmaf(f32_image(x), inv_l, 12582912.0f)) - 0x4B400000;
}

// The same for floor(x 2048/ln2): k = rn(v) with v = fl32(x' 2048/ln2 - 1/2).  With
// e = 5.3e-4 |x| + 1/16 (the image's and 2048/ln2's FP32 errors, and v's rounding for
// |v| < 2^21), x 2048/ln2 - k lies in [-e, 1 + e].
__device__ __forceinline__ int exp_index_floor(double x, float inv_l)
{
    const float v = fmaf(f32_image(x), inv_l, -0.5f);
    return __float_as_int(__fadd_rn(v, 12582912.0f)) - 0x4B400000;
}

// v 2^P rounded toward zero, for |v 2^P| < 2^62, from v's bits (integer operations); FP32
// subnormals give 0.
template <int P>
__device__ __forceinline__ long long fx(float v)
{
    const unsigned b = __float_as_uint(v);
    const int sh = (int)((b >> 23) & 0xffu) - 150 + P;  // |v| 2^P = m 2^sh
    const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
    const long long q = sh >= 0 ? m << (sh & 63) : (sh > -24 ? m >> ((-sh) & 31) : 0ll);
    return (b >> 31) ? -q : q;
}

// The double 1/2 + D 2^-53, exactly, for |D| < 2^50, from its bits: above 1/2 the ulp is 2^-53,
// below it 2^-54, so a negative D moves the pattern twice as far (and borrows the exponent).
__device__ __forceinline__ double half_plus(long long D)
{
    return __longlong_as_double((1022ll << 52) + (D >= 0 ? D : 2 * D));
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

// T2 = T_hi + T_lo + T_hi c with c = e^r - 1 - r, to within half a unit of 2^-52 plus 2^-8 of
// one, for T_hi in [1, 2^(2047/2048)] and |r| <= 1.5 ln2/2048.  T2 lies in [1, 2) (c < 1.3e-7),
// so it is T_hi's bit pattern plus round((T_lo + T_hi c) 2^52), and no FP64 instruction forms it:
// c = r^2 (1/2 + r/6 + r^2/24) (truncation r^5/120 < 3e-19) from r's two FP32 parts (r^2 as an
// FP32 pair with the square's exact error; r/6 + r^2/24 in FP32, whose error enters c at 2^-22 of
// r^2/6), then (T_lo + T_hi c) 2^60 as an FP32 pair from T_hi's two FP32 parts, each part turned
// into an integer and the sum rounded to units of 2^-52 (the pair's error is below 2^-37 of it,
// a few units of 2^-60).
__device__ __forceinline__ double exp_t2(double th, double tl, double r)
{
    const float rh = f32_image(r), rl = f32_image_rest(r);
    const float sh = __fmul_rn(rh, rh);
    const float sl = fmaf(2.0f * rh, rl, fmaf(rh, rh, -sh));                  // r^2 = sh + sl
    const float d = __fmul_rn(rh, fmaf(rh, 1.0f / 24.0f, 1.0f / 6.0f));       // r/6 + r^2/24
    const float ch = __fmul_rn(sh, 0x1p59f);                                   // c 2^60 = ch + cl
    const float cl = __fmul_rn(fmaf(sh, d, 0.5f * sl), 0x1p60f);
    const float tf = f32_image(th), tr = f32_image_rest(th);                   // T_hi = tf + tr
    const float ph = __fmul_rn(tf, ch);                                        // (T_lo + T_hi c) 2^60
    float pl = fmaf(tf, ch, -ph);                                              //   = ph + pl
    pl = fmaf(tr, ch, pl);
    pl = fmaf(tf, cl, pl);
    pl = fmaf(f32_image(tl), 0x1p60f, pl);
    const long long F = (fx<0>(ph) + fx<0>(pl) + 128) >> 8;
    return __longlong_as_double(__double_as_longlong(th) + F);
}

// exp(x).  tab = [hi, lo] pairs in shared memory.  k is taken near floor(x 2048/ln2), so that
// r = x - k ln2/2048 lies in [-e, 1 + e] ln2/2048 (exp_index_floor) and the result 2^m T e^r
// has T e^r in [1, 2.001) except when j = 0 and r < 0.  With T2 from exp_t2 the result is
// fma(T_hi, r, T2) 2^m: 2 FP64 operations with the reduction's fma.  Error: T2's half unit of
// 2^-52 and the fma's rounding, at most one ulp of a result in [1, 2) (1.5 in the rare j = 0,
// r < 0 case, whose result lies in [1 - 2e-4, 1)); the table's own rounding enters only through
// T_hi r, below 2^-64.
__device__ __forceinline__ double exp_tab(double x, const double2* __restrict__ tab, const ExpConsts& k)
{
    // Range tests on bit patterns (integer pipe): x < EXP_X_MIN or x > EXP_X_MAX (or -inf/+inf).
    const int64_t b = bits_of(x);
    const bool under = (uint64_t)b > (uint64_t)bits_of(EXP_X_MIN);  // negative and below the range
    const bool over = b > bits_of(EXP_X_MAX);                         // positive and above the range
    const double xs = (under | over) ? 0.0 : x;
    const int n = exp_index_floor(xs, k.inv_l);
    const double r = fma(dbl_of_int(n), -k.l, xs);
    const double2 T = tab[n & (EXP_TABLE_SIZE - 1)];
    const double res = fma(T.x, r, exp_t2(T.x, T.y, r));
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
    // e^r - 1 = r + r^2 q with q = 1/2 + r/6 + r^2/24 + r^3/120 (truncation r^6/720, below 1e-24
    // of the result).  The result can be as small as r, so q's error enters relative to it as
    // |r| times that error: q is wanted to about 3e-14.  r/6 is taken as an FP32 pair (r's two
    // FP32 parts times the two parts of 1/6, with the product's exact error), the rest
    // (< 4e-9) in FP32 from r's top part; q = 1/2 + their sum, assembled from bits (error below
    // 2^-52 + 1e-15 of the tail, i.e. under 1e-18 of the result relative).
    const float rh = f32_image(r), rl = f32_image_rest(r);
    const float a = __fmul_rn(rh, 0.16666667163372039795f);
    float t = fmaf(rh, 0.16666667163372039795f, -a);                // rh c6_hi - a, exact
    t = fmaf(rh, -4.9670538793e-9f, t);                                // + rh c6_lo
    t = fmaf(rl, 0.16666667163372039795f, t);                        // + rl c6_hi
    t = fmaf(__fmul_rn(rh, rh), fmaf(rh, 1.0f / 120.0f, 1.0f / 24.0f), t);
    const double q = half_plus(fx<53>(a) + fx<53>(t));
    const double p = fma(r * r, q, r);
    const double2 tj = tab[n & (EXP_TABLE_SIZE - 1)];
    const int m = n >> EXP_TABLE_BITS;
    const double s = __hiloint2double(__double2hiint(tj.x) + (int)((unsigned)m << 20), __double2loint(tj.x));
    const double sc = __hiloint2double((m + 1023) << 20, 0);                                     // 2^m
    const double res = fma(fma(tj.x, p, tj.y), sc, s - 1.0);
    return under ? -1.0 : (over ? __longlong_as_double(0x7ff0000000000000LL) : res);
}

// ln x for positive normal finite x, after P. T. P. Tang, "Table-driven implementation of the
// logarithm function in IEEE floating-point arithmetic", ACM TOMS 16 (1990) 378-400:
// x = 2^e m, m in [1, 2), F = 1 + j/128 the nearest such point (j = 0..128), f = m - F exact
// (|f| <= 2^-8), and ln x = e ln2 + ln F + log1p(z) with z = f (1/F) (|z| <= 2^-8; exact for
// j = 0 and 128).  ln2 and ln F are hi + lo pairs whose hi parts lie on the grid of 2^-43, so
// e L_hi + lnF_hi is exact for |e| < 1100.  log1p(z) = z - z^2 q, q = 1/2 - z/3 + z^2/4 - z^3/5 +
// z^4/6 - z^5/7 (truncation z^8/8, below 2^-59 of the result): q's error enters relative to the
// result as |z| times it, so q is wanted to about 2^-46 and, lying within 0.0013 of 1/2, is
// assembled from bits like expm1's coefficient: -z/3 and z^2/4 as FP32 pairs (z's two FP32
// parts, the products' exact errors and the two parts of 1/3), the rest in FP32.  8 FP64
// operations: f, z, z^2, the fma z - z^2 q, the two table fmas and two additions.  Error: within
// about one ulp (z's own rounding, 2^-52 of |z|, matters most where the result is a few times
// |z|, next to x = 1 +- 2^-8).
constexpr int LOG_TABLE_SIZE = 129;  // F_j = 1 + j/128, j = 0..128

struct LogEntry {
    double inv_f;  // 1/F_j, rounded
    double ln_hi;  // ln F_j on the grid of 2^-43
    double ln_lo;  // ln F_j - ln_hi, rounded
};

struct LogConsts {
    double l_hi, l_lo;  // ln 2 = l_hi + l_lo, l_hi on the grid of 2^-43
};

__device__ __forceinline__ double log_tab(double x, const LogEntry* __restrict__ tab, const LogConsts& k)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)(hi >> 20) - 1023;
    const unsigned j = ((((hi & 0x000fffffu) >> 12) + 1u) >> 1);  // round((m - 1) 128), 0..128
    const double m = __hiloint2double((int)((hi & 0x000fffffu) | 0x3ff00000u), (int)lo);
    const double f = m - __hiloint2double((int)(0x3ff00000u + (j << 13)), 0);
    const double z = f * __ldg(&tab[j].inv_f);
    const float zh = f32_image(z), zl = f32_image_rest(z);
    const float a = __fmul_rn(-zh, 0.3333333432674407959f);                  // -z/3 = a + t (pair)
    float t = fmaf(-zh, 0.3333333432674407959f, -a);
    t = fmaf(-zh, -9.9341077586e-9f, t);
    t = fmaf(-zl, 0.3333333432674407959f, t);
    const float sh = __fmul_rn(zh, zh);                                       // z^2 = sh + sl
    const float sl = fmaf(2.0f * zh, zl, fmaf(zh, zh, -sh));
    t = fmaf(0.25f, sl, t);
    t = fmaf(__fmul_rn(sh, zh), fmaf(fmaf(zh, -1.0f / 7.0f, 1.0f / 6.0f), zh, -0.2f), t);
    const double q = half_plus(fx<53>(a) + fx<53>(0.25f * sh) + fx<53>(t));
    const double l1p = fma(-(z * z), q, z);
    const double ed = dbl_of_int(e);
    const double A = fma(ed, k.l_hi, __ldg(&tab[j].ln_hi));
    const double B = fma(ed, k.l_lo, __ldg(&tab[j].ln_lo));
    return A + (l1p + B);
}

// ln x for any x: log_tab for positive normal finite x, the library's log otherwise (0, subnormal,
// infinite, negative or NaN arguments).
__device__ __forceinline__ double log_pos(double x, const LogEntry* __restrict__ tab, const LogConsts& k)
{
    const long long b = __double_as_longlong(x);
    return (b >= 0x0010000000000000LL && b < 0x7ff0000000000000LL) ? log_tab(x, tab, k) : log(x);
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

// FP64-grade sample weights in float-float arithmetic (POP_MODE_FF).
//
// The weight of the FP64 kernel, p(theta|Lambda)/pi of Eq. (poplike), with every quantity
// held as a float-float value (pop_ff.cuh: about 48 significant bits on the FP32 pipe,
// which GB300 runs at 64 times its FP64 rate).  The work decomposition is the FP32
// kernel's: one Lambda per thread with its constants in registers, a block stages a chunk's
// samples in pairs that every lane reads from the same shared-memory words, the two samples
// of a pair go through the arithmetic in packed f32x2 instructions, and the lower support
// edge is an index from a binary search on the (q m1, m1)-sorted samples.  The staging
// turns the FP64 features into (hi, lo) FP32 pairs once per block for its 128 Lambda.
//
// FP64 instructions remain where float-float cannot carry the value: the q normalisation
// of samples within 2^-6 of the lower mass edge, whose ln(mmin/m1) is log1p((mmin - m1)/m1)
// with the exact FP64 difference (as in the FP64 kernel).  Elsewhere ln(mmin/m1) is the
// float-float difference of the logs, and 1 - (mmin/m1)^(1+beta) comes from Tang's table
// expm1 for |(1+beta) ln(mmin/m1)| >= 1/16 and from the Taylor series below that.
//
// Accuracy: a weight is within a few 1e-14 relative (a few 2^-48 per operation, and the
// exponentials' arguments within ~2^-47 times the sum of their terms' magnitudes); the
// per-thread sums are float-float, the (Lambda, chunk) partial FP64.  Weights below e^-87
// (under the FP32 normal range) are 0.
#include <math.h>

#include <algorithm>

#include "pop_ff.cuh"
#include "pop_internal.h"

namespace pop {

namespace {

constexpr int FF_NT = 128;        // threads per block = Lambda per work item
constexpr int FF_SP = 64;         // sample pairs per staged sub-tile
// Resident blocks per SM the register budget is set for (65536 / (128 x this) per thread).
#ifndef POP_FF_MIN_BLOCKS
#define POP_FF_MIN_BLOCKS 4
#endif
constexpr int FF_MIN_BLOCKS = POP_FF_MIN_BLOCKS;

// Staged pair (8-byte words): word 2f = hi parts (sample a, sample b) and word 2f + 1 = lo
// parts of feature f = ln m1, m1, ln q, s_a, s_b, d_c, -ln pi (f = 0..6); words 14, 15 = the
// FP64 bit patterns of m1 (a, b); with redshift words 16, 17 = ln(1+z) hi, lo.
template <bool HAS_Z>
struct FFWords {
    static constexpr int W = HAS_Z ? 18 : 16;
};

struct FFLane {
    ff2 beta, ac, bc_, km1, cpl, nalpha, cg, nmu, nh, b1, lmmin, nht, ct, t0;
    f2 sgn;  // -sign(1+beta) (-1 with beta = -1): den = sgn (e^u - 1) > 0 inside the support
};

__device__ __forceinline__ FFLane ff_lane(const LamF64& L)
{
    FFLane c;
    c.beta = ff_const(L.beta);
    c.ac = ff_const(L.ac);
    c.bc_ = ff_const(L.bc);
    c.km1 = ff_const(L.km1);
    c.cpl = ff_const(L.cpl);
    c.nalpha = ff_const(L.nalpha);
    c.cg = ff_const(L.cg);
    c.nmu = ff_const(-L.mu);
    c.nh = ff_const(L.nh);
    c.b1 = ff_const(L.b1);
    c.lmmin = ff_const(L.lmmin);
    c.nht = ff_const(L.nht);
    c.ct = ff_const(L.ct);
    c.t0 = ff_const(L.t0);
    c.sgn = bc((L.beta_m1 || L.b1 > 0.0) ? -1.0f : 1.0f);
    return c;
}

struct FFPair {
    ff2 lm1, m1, lq, sa, sb, dc, nlpi, lz1;
    long long m1a, m1b;  // FP64 bit patterns of m1
};

template <bool HAS_Z>
__device__ __forceinline__ void load_ff_pair(const unsigned long long* __restrict__ buf, int p, FFPair& x)
{
    const ulonglong2* q = reinterpret_cast<const ulonglong2*>(buf + FFWords<HAS_Z>::W * p);
    ulonglong2 v;
    v = q[0]; x.lm1 = ff2{v.x, v.y};
    v = q[1]; x.m1 = ff2{v.x, v.y};
    v = q[2]; x.lq = ff2{v.x, v.y};
    v = q[3]; x.sa = ff2{v.x, v.y};
    v = q[4]; x.sb = ff2{v.x, v.y};
    v = q[5]; x.dc = ff2{v.x, v.y};
    v = q[6]; x.nlpi = ff2{v.x, v.y};
    v = q[7]; x.m1a = (long long)v.x; x.m1b = (long long)v.y;
    if (HAS_Z) {
        v = q[8];
        x.lz1 = ff2{v.x, v.y};
    }
}

__device__ __forceinline__ ff2 ff_sub(ff2 x, ff2 y) { return ff_add(x, ff_neg(y)); }

// Exponent arguments of both halves: A = aE + cpl - alpha ln m1 (power law), B = aE + cg -
// (m1 - mu)^2/(2 sig^2) (peak), T = ct + nht d_c (tilt), with aE = -ln pi + beta ln q +
// (alpha_chi - 1) s_a + (beta_chi - 1) s_b [+ (kappa - 1) ln(1+z)].
struct FFArgs {
    ff2 A, B, T;
};

template <bool HAS_Z>
__device__ __forceinline__ FFArgs ff_args(const FFPair& x, const FFLane& c, f2 z)
{
    // aE as one compensated sum, shared by A and B, each then closed with its own terms.
    FFAcc aE = acc_add_prod(acc_of(x.nlpi), x.lq, c.beta, z);
    aE = acc_add_prod(aE, x.sa, c.ac, z);
    aE = acc_add_prod(aE, x.sb, c.bc_, z);
    if (HAS_Z) aE = acc_add_prod(aE, x.lz1, c.km1, z);
    FFArgs a;
    a.A = acc_ff(acc_add_prod(acc_add(aE, c.cpl), x.lm1, c.nalpha, z));
    const ff2 d = ff_add(x.m1, c.nmu);
    a.B = acc_ff(acc_add_prod(acc_add(aE, c.cg), ff_mul(d, c.nh, z), d, z));
    a.T = acc_ff(acc_add_prod(acc_of(c.ct), x.dc, c.nht, z));
    return a;
}

// |1 - (mmin/m1)^(1+beta)| up to the sign sgn, from lr = ln(mmin/m1).  SLOW: the halves near the
// lower mass edge take lr from the exact FP64 gap, small |u| the series, beta = -1 the log.
template <bool SLOW>
__device__ __forceinline__ ff2 ff_qnorm(const FFPair& x, const FFLane& c, const LamF64& L, const FeatF64& F,
                                        int64_t start, int j, const float2* __restrict__ tab, const FFConsts& k,
                                        const FFSeries& ser, f2 z)
{
    ff2 lr = ff_sub(c.lmmin, x.lm1);
    if (!SLOW) return ff_expm1_far(ff_mul(lr, c.b1, z), tab, k);
    // Near the edge (bit patterns within 2^46: m1/mmin - 1 below ~2^-6) the FP64 gap is exact.
    const bool na = llabs(x.m1a - L.mmin_bits) < NEAR_EDGE_BITS, nb = llabs(x.m1b - L.mmin_bits) < NEAR_EDGE_BITS;
    if (na | nb) {
        float ha, hb, la, lb;
        upk(lr.hi, ha, hb);
        upk(lr.lo, la, lb);
        if (na) {
            const double m1 = __longlong_as_double(x.m1a);
            const double v = log1p_near0(__ldg(F.base + F_INVM1 * F.stride + start + j) * (L.mmin - m1));
            ha = (float)v;
            la = (float)(v - (double)ha);
        }
        if (nb) {
            const double m1 = __longlong_as_double(x.m1b);
            const double v = log1p_near0(__ldg(F.base + F_INVM1 * F.stride + start + j + 1) * (L.mmin - m1));
            hb = (float)v;
            lb = (float)(v - (double)hb);
        }
        lr = ff2{pk(ha, hb), pk(la, lb)};
    }
    const ff2 u = ff_mul(lr, c.b1, z);
    const ff2 far = ff_expm1_far(u, tab, k);
    const ff2 near = ff_expm1_near(u, ser, z);
    float ua, ub, fa, fb, ga, gb, qa, qb, ra, rb;
    upk(u.hi, ua, ub);
    upk(far.hi, fa, fb);
    upk(far.lo, ga, gb);
    upk(near.hi, qa, qb);
    upk(near.lo, ra, rb);
    const bool small_a = fabsf(ua) < 0.0625f, small_b = fabsf(ub) < 0.0625f;
    float da = small_a ? qa : fa, db = small_b ? qb : fb;
    float ea = small_a ? ra : ga, eb = small_b ? rb : gb;
    if (L.beta_m1) {  // normalisation ln(m1/mmin) = -lr (sgn = -1)
        upk(lr.hi, da, db);
        upk(lr.lo, ea, eb);
    }
    return ff2{pk(da, db), pk(ea, eb)};
}

// Per-lane power-of-two scales of the rerun pass: the weights are accumulated as
// w 2^-(mu + muT), with mu following the largest power-law/peak exponent seen and muT the
// largest tilt exponent (only with xi_t = 1, where the tilt factor has no isotropic floor).
struct FFScale {
    int mu, muT;
};

constexpr int FF_NO_MASS = -(1 << 20);  // scale before the first in-support sample

__device__ __forceinline__ void ff_rescale(ff2& v, int d)
{
    if (d < -120) {
        v = ff2{0ull, 0ull};
    } else {
        const f2 sc = bc(pow2i(d));
        v.hi = mul2(v.hi, sc);
        v.lo = mul2(v.lo, sc);
    }
}

// Adds the masked weights of pair p (first sample at chunk index j) to s (and w^2 to s2).
// SCALED: the running scales of FFScale keep every exponential inside the FP32 range.
template <bool SLOW, bool SCALED, bool INJ, bool HAS_Z>
__device__ __forceinline__ void ff_pair(const unsigned long long* __restrict__ buf, int p, int j, int j0,
                                        const FFLane& c, const LamF64& L, const FeatF64& F, int64_t start,
                                        const float2* __restrict__ tab, const FFConsts& k, const FFSeries& ser,
                                        ff2& s, ff2& s2, FFScale& sc)
{
    FFPair x;
    load_ff_pair<HAS_Z>(buf, p, x);
    const f2 z = bc(k.zero);
    const bool ia = j >= j0 && x.m1a <= L.mmax_bits;
    const bool ib = j + 1 >= j0 && x.m1b <= L.mmax_bits;
    const FFArgs a = ff_args<HAS_Z>(x, c, z);
    int sh = 0, shT = 0;
    if (SCALED) {
        float Aa, Ab, Ba, Bb, Ta, Tb;
        upk(a.A.hi, Aa, Ab);
        upk(a.B.hi, Ba, Bb);
        upk(a.T.hi, Ta, Tb);
        const float NEG = -3.0e38f;
        const float m = fmaxf(ia ? fmaxf(Aa, Ba) : NEG, ib ? fmaxf(Ab, Bb) : NEG);
        const float mt = fmaxf(ia ? Ta : NEG, ib ? Tb : NEG);
        const float LOG2E = 1.44269504f;
        const int cand = m > -1.0e30f ? (int)floorf(m * LOG2E) : FF_NO_MASS;
        const int candT = (L.t0 == 0.0 && mt > -1.0e30f) ? (int)floorf(mt * LOG2E) : sc.muT;
        if (cand > sc.mu || candT > sc.muT) {
            const int mu = max(cand, sc.mu), muT = L.t0 == 0.0 ? max(candT, sc.muT) : 0;
            const int d = (sc.mu - mu) + (sc.muT - muT);
            ff_rescale(s, d);
            if (INJ) ff_rescale(s2, 2 * d);
            sc.mu = mu;
            sc.muT = muT;
        }
        sh = sc.mu;
        shT = sc.muT;
    }
    const ff2 e12 = ff_add(ff_exp(a.A, tab, k, sh), ff_exp(a.B, tab, k, sh));
    const ff2 tt = ff_add(c.t0, ff_exp(a.T, tab, k, shT));
    const ff2 den = ff_qnorm<SLOW>(x, c, L, F, start, j, tab, k, ser, z);
    ff2 w = ff_mul(ff_mul(e12, tt, z), ff_rcp(den, z), z);
    w.hi = prod2(w.hi, c.sgn, z);
    w.lo = prod2(w.lo, c.sgn, z);
    float wa, wb, va, vb;
    upk(w.hi, wa, wb);
    upk(w.lo, va, vb);
    w = ff2{pk(ia ? wa : 0.0f, ib ? wb : 0.0f), pk(ia ? va : 0.0f, ib ? vb : 0.0f)};
    s = ff_add(s, w);
    if (INJ) s2 = ff_add(s2, ff_mul(w, w, z));
}

template <bool SLOW, bool SCALED, bool INJ, bool HAS_Z>
__device__ __forceinline__ void ff_run(const unsigned long long* __restrict__ buf, int p0, int p1, int jb, int j0,
                                       const FFLane& c, const LamF64& L, const FeatF64& F, int64_t start,
                                       const float2* __restrict__ tab, const FFConsts& k, const FFSeries& ser,
                                       ff2& s, ff2& s2, FFScale& sc)
{
#pragma unroll 1
    for (int p = p0; p < p1; ++p)
        ff_pair<SLOW, SCALED, INJ, HAS_Z>(buf, p, jb + 2 * p, j0, c, L, F, start, tab, k, ser, s, s2, sc);
}

// First chunk index whose (m2, m1) exceeds (mmin, mmin) lexicographically (the first sample
// with m1 > mmin and m2 >= mmin); len when there is none.
__device__ __forceinline__ int lower_edge64(const FeatF64& F, const Chunk& ch, double mmin)
{
    const double* m2 = F.base + F_M2 * F.stride + ch.start;
    const double* m1 = F.base + F_M1 * F.stride + ch.start;
    int lo = 0, hi = ch.len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const double a = __ldg(m2 + mid);
        if (a > mmin || (a == mmin && __ldg(m1 + mid) > mmin)) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ int first_m2_at_least64(const FeatF64& F, const Chunk& ch, double t)
{
    const double* m2 = F.base + F_M2 * F.stride + ch.start;
    int lo = 0, hi = ch.len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(m2 + mid) >= t) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ void split_ff(double x, float& h, float& l)
{
    h = (float)x;
    l = (float)(x - (double)h);
}

// Stage samples [2 FF_SP st, 2 FF_SP (st+1)) of the chunk, converted to (hi, lo) pairs;
// positions past the chunk's end get zeros and m1 = +inf (outside every support).
template <bool HAS_Z>
__device__ __forceinline__ void stage_ff(const FeatF64& F, const Chunk& ch, int st, unsigned long long* buf)
{
    constexpr int W = FFWords<HAS_Z>::W;
    for (int s = threadIdx.x; s < 2 * FF_SP; s += FF_NT) {
        const int j = 2 * FF_SP * st + s;
        float* dst = reinterpret_cast<float*>(buf + W * (s >> 1)) + (s & 1);
        long long* bits = reinterpret_cast<long long*>(buf + W * (s >> 1) + 14) + (s & 1);
        if (j < ch.len) {
            const double* src = F.base + ch.start + j;
#pragma unroll
            for (int f = 0; f < 7; ++f) {
                // staged features in the row order F_LM1, F_M1, F_LQ, F_SA, F_SB, F_DC, F_NLPI
                const double v = __ldg(src + f * F.stride);
                split_ff(v, dst[4 * f], dst[4 * f + 2]);
            }
            *bits = __double_as_longlong(__ldg(src + F_M1 * F.stride));
            if (HAS_Z) split_ff(__ldg(src + F_LZ1 * F.stride), dst[32], dst[34]);
        } else {
#pragma unroll
            for (int f = 0; f < 7; ++f) dst[4 * f] = dst[4 * f + 2] = 0.0f;
            *bits = 0x7ff0000000000000LL;
            if (HAS_Z) dst[32] = dst[34] = 0.0f;
        }
    }
}

// One pass of the block over the chunk's sub-tiles from `first` on; every thread of the block
// calls it (the staging is shared).  SCALED warps without a lane that asked for it skip the
// arithmetic.
template <bool SCALED, bool HAS_Z>
__device__ __forceinline__ void ff_pass(const FeatF64& F, const Chunk& ch, bool is_inj, int first, int n_sub, int wj0,
                                        int wjs, int j0, bool warp_on, const FFLane& c, const LamF64& L,
                                        const float2* __restrict__ tab, const FFConsts& k, const FFSeries& ser,
                                        unsigned long long* sbuf, ff2& s, ff2& s2, FFScale& sc)
{
    for (int st = first; st < n_sub; ++st) {
        __syncthreads();  // every warp is done with the previous sub-tile
        stage_ff<HAS_Z>(F, ch, st, sbuf);
        __syncthreads();
        if (!warp_on) continue;
        const int jb = 2 * FF_SP * st;
        const int p_end = min(FF_SP, (ch.len - jb + 1) >> 1);
        const int p_beg = min(p_end, max(0, (wj0 - jb) >> 1));
        const int p_slow = min(p_end, max(p_beg, (wjs - jb + 1) >> 1));
        const int64_t start = ch.start;
        if (is_inj) {
            ff_run<true, SCALED, true, HAS_Z>(sbuf, p_beg, p_slow, jb, j0, c, L, F, start, tab, k, ser, s, s2, sc);
            ff_run<false, SCALED, true, HAS_Z>(sbuf, p_slow, p_end, jb, j0, c, L, F, start, tab, k, ser, s, s2, sc);
        } else {
            ff_run<true, SCALED, false, HAS_Z>(sbuf, p_beg, p_slow, jb, j0, c, L, F, start, tab, k, ser, s, s2, sc);
            ff_run<false, SCALED, false, HAS_Z>(sbuf, p_slow, p_end, jb, j0, c, L, F, start, tab, k, ser, s, s2, sc);
        }
    }
}

__device__ __forceinline__ double ff_total(const ff2& s)
{
    float a, b, la, lb;
    upk(s.hi, a, b);
    upk(s.lo, la, lb);
    return ((double)a + (double)la) + ((double)b + (double)lb);
}

template <bool HAS_Z>
__global__ void __launch_bounds__(FF_NT, FF_MIN_BLOCKS)
weight_ff_kernel(FeatF64 ev, FeatF64 inj, WorkDesc wd, const LamF64* __restrict__ lam,
                 const int32_t* __restrict__ order, const int32_t* __restrict__ n_mc,
                  unsigned long long* __restrict__ queue, int64_t K_cap,
                 const int64_t* __restrict__ dK, double* __restrict__ part, double* __restrict__ part2,
                 const float2* __restrict__ fftab, FFConsts kc)
{
    static_assert(F_LM1 == 0 && F_M1 == 1 && F_LQ == 2 && F_SA == 3 && F_SB == 4 && F_DC == 5 && F_NLPI == 6,
                  "staging reads the first seven feature rows in order");
    constexpr int W = FFWords<HAS_Z>::W;
    __shared__ float2 tab[FF_TABLE_SIZE];
    __shared__ __align__(16) unsigned long long sbuf[FF_SP * W];
    for (int i = threadIdx.x; i < FF_TABLE_SIZE; i += FF_NT) tab[i] = fftab[i];
    const int64_t K = *dK;
    const int64_t K_inj = *n_mc;
    const int64_t tiles_ev = (K + FF_NT - 1) / FF_NT;
    const int64_t tiles_inj = (K_inj + FF_NT - 1) / FF_NT;
    const int n_inj_chunks = wd.n_chunks - wd.n_ev_chunks;
    const int64_t n_ev_items = (int64_t)wd.n_ev_chunks * tiles_ev;
    const int64_t n_items = n_ev_items + (int64_t)n_inj_chunks * tiles_inj;
    __shared__ int s_jmin;
    const int lane = threadIdx.x & 31;
    const FFSeries ser = ff_series_consts();

    // Items come from a queue (zeroed before the launch): their costs differ (event and injection
    // chunks, lower edges), and blocks that finish early take more.
    __shared__ unsigned long long s_item;
    for (;;) {
        __syncthreads();  // every thread has read the previous item
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1ull);
        __syncthreads();
        const int64_t item = (int64_t)s_item;
        if (item >= n_items) break;
        int c;
        int64_t tile;
        if (item < n_ev_items) {
            c = (int)(item / tiles_ev);
            tile = item - (int64_t)c * tiles_ev;
        } else {
            const int64_t i2 = item - n_ev_items;
            const int ci = (int)(i2 / tiles_inj);
            tile = i2 - (int64_t)ci * tiles_inj;
            c = wd.n_ev_chunks + ci;
        }
        const Chunk ch = wd.chunks[c];
        const bool is_inj = ch.inj != 0;
        const FeatF64 F = is_inj ? inj : ev;
        const int64_t slot = tile * FF_NT + threadIdx.x;
        const bool active = slot < (is_inj ? K_inj : K);
        const int k = active ? order[(is_inj ? K_cap : 0) + slot] : 0;
        const LamF64 L = lam[k];
        int j0 = ch.len, js = 0;
        if (active) {
            const double mmin = __longlong_as_double(L.mmin_bits);  // +inf for an invalid Lambda
            j0 = lower_edge64(F, ch, mmin);
            if (j0 < ch.len) {
                if (L.beta_m1) {
                    js = ch.len;
                } else {
                    // From m1 >= mmin max(e^(1/(16|1+beta|)), 1 + 2^-5) (2^-10 margin) on, neither the
                    // series nor the exact gap is needed, and m1 >= m2.
                    const double t = mmin * fmax(exp(0.0625 / fabs(L.b1)), 1.0 + 0x1p-5) * (1.0 + 0x1p-10);
                    js = first_m2_at_least64(F, ch, t);
                }
            }
        }
        const FFLane cl = ff_lane(L);
        const int wj0 = __reduce_min_sync(0xffffffffu, j0);
        const int wjs = __reduce_max_sync(0xffffffffu, js);
        __syncthreads();  // the previous item is done with s_jmin and the staging buffer
        if (threadIdx.x == 0) s_jmin = ch.len;
        __syncthreads();
        if (lane == 0 && wj0 < ch.len) atomicMin(&s_jmin, wj0);
        __syncthreads();
        const int n_sub = (ch.len + 2 * FF_SP - 1) / (2 * FF_SP);
        const int first = s_jmin < ch.len ? s_jmin / (2 * FF_SP) : n_sub;
        ff2 s{0ull, 0ull}, s2{0ull, 0ull};
        FFScale none{0, 0};
        ff_pass<false, HAS_Z>(F, ch, is_inj, first, n_sub, wj0, wjs, j0, true, cl, L, tab, kc, ser, sbuf, s, s2, none);
        double tot = ff_total(s), tot2 = is_inj ? ff_total(s2) : 0.0;
        // A sum under 2^-60 may have lost weights under the FP32 range (e^-87), and an infinite one
        // overflowed: such lanes rerun the chunk with running power-of-two scales.
        const bool rerun = active && j0 < ch.len && (!(tot >= 0x1p-60 && tot < INFINITY) || !(tot2 < INFINITY));
        if (__syncthreads_or(rerun)) {
            FFScale sc{FF_NO_MASS, L.t0 == 0.0 ? FF_NO_MASS : 0};
            ff2 r{0ull, 0ull}, r2{0ull, 0ull};
            const bool warp_on = __any_sync(0xffffffffu, rerun);
            ff_pass<true, HAS_Z>(F, ch, is_inj, first, n_sub, wj0, wjs, j0, warp_on, cl, L, tab, kc, ser, sbuf, r, r2,
                                 sc);
            if (rerun) {
                const int e = sc.mu == FF_NO_MASS ? 0 : sc.mu + sc.muT;
                tot = ldexp(ff_total(r), e);
                tot2 = is_inj ? ldexp(ff_total(r2), 2 * e) : 0.0;
            }
        }
        if (active) {
            part[(int64_t)k * wd.n_chunks + c] = tot;
            if (is_inj) part2[(int64_t)k * n_inj_chunks + (c - wd.n_ev_chunks)] = tot2;
        }
    }
}

__global__ void ff_math_kernel(int fn, int64_t n, const double* __restrict__ x, double* __restrict__ y,
                               const float2* __restrict__ fftab, FFConsts kc)
{
    __shared__ float2 tab[FF_TABLE_SIZE];
    for (int i = threadIdx.x; i < FF_TABLE_SIZE; i += blockDim.x) tab[i] = fftab[i];
    __syncthreads();
    const FFSeries ser = ff_series_consts();
    const f2 z = bc(kc.zero);
    for (int64_t i = 2 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); i < n;
         i += 2 * (int64_t)gridDim.x * blockDim.x) {
        const double xa = x[i], xb = i + 1 < n ? x[i + 1] : x[i];
        float ha, la, hb, lb;
        split_ff(xa, ha, la);
        split_ff(xb, hb, lb);
        const ff2 v{pk(ha, hb), pk(la, lb)};
        ff2 r;
        if (fn == 3) {
            r = ff_exp(v, tab, kc);
        } else if (fn == 4) {
            const ff2 far = ff_expm1_far(v, tab, kc), near = ff_expm1_near(v, ser, z);
            float fa, fb, ga, gb, qa, qb, sa, sb;
            upk(far.hi, fa, fb);
            upk(far.lo, ga, gb);
            upk(near.hi, qa, qb);
            upk(near.lo, sa, sb);
            const bool na = fabsf(ha) < 0.0625f, nb = fabsf(hb) < 0.0625f;
            r = ff2{pk(na ? qa : fa, nb ? qb : fb), pk(na ? sa : ga, nb ? sb : gb)};
        } else if (fn == 5) {
            r = ff_rcp(v, z);
        } else if (fn == 6) {
            r = ff_mul(v, v, z);
        } else {
            const f2 p = prod2(v.hi, v.hi, z);
            r = ff2{p, fma2(v.hi, v.hi, sub2(0ull, p))};
        }
        float a0, b0, a1, b1;
        upk(r.hi, a0, b0);
        upk(r.lo, a1, b1);
        y[i] = (double)a0 + (double)a1;
        if (i + 1 < n) y[i + 1] = (double)b0 + (double)b1;
    }
}

}  // namespace

cudaError_t launch_ff_math_check(int fn, int64_t n, const double* x, double* y, const float2* fftab, FFConsts kc,
                                 cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n / 2 + 256) / 256, 4096);
    ff_math_kernel<<<(unsigned)blocks, 256, 0, s>>>(fn, n, x, y, fftab, kc);
    return cudaGetLastError();
}

const void* weight_ff_fn(bool has_z)
{
    return has_z ? (const void*)weight_ff_kernel<true> : (const void*)weight_ff_kernel<false>;
}

int weight_ff_threads() { return FF_NT; }

cudaError_t launch_weight_ff(int grid, FeatF64 ev, FeatF64 inj, WorkDesc wd, const LamF64* lam, const int32_t* order,
                             const int32_t* n_mc, unsigned long long* queue, int64_t K_cap, const int64_t* dK,
                             double* part, double* part2, const float2* fftab, FFConsts kc, cudaStream_t s)
{
    const void* fn = weight_ff_fn(wd.has_z != 0);
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    void* args[] = {&ev, &inj, &wd, &lam, &order, &n_mc, &queue, &K_cap, &dK, &part, &part2, &fftab, &kc};
    return cudaLaunchKernel(fn, dim3(grid), dim3(FF_NT), args, 0, s);
}

// 2^(j/2048) as FP32 (hi, lo) pairs and the reduction constants, from long double.
void build_ff_table(float2* tab, FFConsts* kc)
{
    for (int j = 0; j < FF_TABLE_SIZE; ++j) {
        const long double v = exp2l((long double)j / FF_TABLE_SIZE);
        const float hi = (float)v;
        tab[j] = make_float2(hi, (float)(v - (long double)hi));
    }
    const long double ln2 = logl(2.0L);
    const long double L = ln2 / FF_TABLE_SIZE;
    kc->inv_l = (float)(FF_TABLE_SIZE / ln2);
    kc->l_hi = (float)L;
    kc->l_lo = (float)(L - (long double)kc->l_hi);
    kc->zero = 0.0f;
}

}  // namespace pop

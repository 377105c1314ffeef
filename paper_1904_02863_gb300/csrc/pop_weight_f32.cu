// FP32 sample-weight kernel: Lambda points in lanes, sample pairs in packed FP32.
//
// A work item is one chunk (a run of one event's samples, or of injections) against
// a tile of NT Lambda points, one per thread.  Each thread keeps its Lambda's
// constants in registers and sums its weights over the whole chunk, so there is no
// reduction across threads and the (Lambda, chunk) partial does not depend on which
// lane computed it.  The block stages the chunk's features in shared memory with the
// two samples of a pair interleaved, and all lanes read the same words (broadcast
// loads); the pair goes through the weight in packed f32x2 FMA / ADD / MUL
// instructions (one instruction for both samples, Blackwell's FFMA2 family), the
// exponentials and the reciprocal per sample on MUFU (ex2.approx, rcp.approx).
//
// Support.  Samples are stored in increasing (q m1, m1) order per event, so the lower
// edge (m1 > mmin and fl64(q m1) >= mmin; q m1 <= m1 because q <= 1) is a suffix of
// the chunk: each lane finds its first index j0 by a binary search in FP64 and the
// per-pair test is j >= j0 and rd32(m1) <= thr_hi = rd32(mmax) (both rounded toward
// -inf).  That float test keeps every sample with m1 <= mmax; it also keeps the samples
// with m1 in (mmax, next float above thr_hi), and upper_edge_fixup_kernel takes those
// (rarely any) back out after the main loop, so every support decision is the oracle's.
// lam_order_kernel orders the Lambda across the lanes by mmin, so the j0 of a warp are
// close and the warp starts at their minimum.
//
// The q normalisation 1 - 2^u (u = (1+beta) log2(mmin/m1), base-2 units) loses
// relative accuracy as u -> 0, where the Taylor series of e^x - 1 in x = u ln2 takes
// over (|u| < 1/8).  A lane can need it only below m2 = mmin 2^(1/(8|1+beta|)), found
// by a second binary search; each warp runs the variant with the series up to the
// largest such index of its lanes and the plain one after it.
//
// Per (thread, Lambda) the two halves of the pair accumulate separate Kahan sums
// (packed); the thread adds the four FP32 numbers in FP64 for the partial.  The
// per-Lambda constants come from the FP64 prologue; the per-event log and the
// cross-event sum are FP64 in the finalise kernel.
#include <math.h>

#include "pop_f32x2.cuh"
#include "pop_internal.h"

namespace pop {

namespace {

// Resident warps per SM the register budget is set for (65536 / (32 x this) registers per thread).
#ifndef POP_F32_WARPS_PER_SM
#define POP_F32_WARPS_PER_SM 24
#endif

// Sample pairs per staged sub-tile (up to 512 samples, 32 KB double-buffered) and the blocks
// per SM of the register budget.
template <int NT>
struct F32Cfg {
    static constexpr int SP = NT >= 128 ? 256 : 2 * NT;
    static constexpr int MIN_BLOCKS = (32 * POP_F32_WARPS_PER_SM) / NT > 0 ? (32 * POP_F32_WARPS_PER_SM) / NT : 1;
};

// One lane's Lambda, in the packed form of the pair arithmetic.
struct LaneConsts {
    f2 beta, ac, bc_, km1, nalpha, cpl, nmu, nh, cg, b1, lmmin, nb1, b1lo, nht, ct, t0, neg1;
    f2 zero;          // 0 that the compiler cannot see (see pair_weight)
    float thr_hi;     // largest float <= mmax
    int beta_m1;      // beta == -1: the q normalisation is -u
};

__device__ __forceinline__ LaneConsts lane_consts(const LamF32& L, float zero = 0.0f)
{
    LaneConsts c;
    c.beta = bc(L.beta);
    c.ac = bc(L.ac);
    c.bc_ = bc(L.bc);
    c.km1 = bc(L.km1);
    c.nalpha = bc(L.nalpha);
    c.cpl = bc(L.cpl);
    c.nmu = bc(-L.mu);
    c.nh = bc(L.nh);
    c.cg = bc(L.cg);
    c.b1 = bc(L.b1);
    c.lmmin = bc(L.lmmin);
    c.nb1 = bc(L.nb1);
    c.b1lo = bc(L.b1lmmin_lo);
    c.nht = bc(L.nht);
    c.ct = bc(L.ct);
    c.t0 = bc(L.t0);
    c.neg1 = bc(-1.0f);
    c.zero = bc(zero);
    c.thr_hi = L.thr_hi;
    c.beta_m1 = L.beta_m1;
    return c;
}

// Staged features of one pair: {lm1, m1}, {lq, sa}, {sb, dc}, {nlpi, lm1lo}, each
// feature a packed (sample a, sample b) value.
struct PairFeat {
    f2 lm1, m1, lq, sa, sb, dc, nlpi, lm1lo, lz1;
};

template <bool HAS_Z>
__device__ __forceinline__ void load_pair(const ulonglong2* __restrict__ buf, const f2* __restrict__ zb, int p,
                                          PairFeat& x)
{
    const ulonglong2 q0 = buf[4 * p + 0], q1 = buf[4 * p + 1], q2 = buf[4 * p + 2], q3 = buf[4 * p + 3];
    x.lm1 = q0.x;
    x.m1 = q0.y;
    x.lq = q1.x;
    x.sa = q1.y;
    x.sb = q2.x;
    x.dc = q2.y;
    x.nlpi = q3.x;
    x.lm1lo = q3.y;
    x.lz1 = HAS_Z ? zb[p] : 0ull;
}

// Weights of both samples of a pair (unmasked: the caller applies the support).
//   w = (2^(-alpha lm1 + aE + cpl) + 2^(-(m1-mu)^2/(2 sig^2) + aE + cg)) (t0 + 2^(nht dc + ct)) / |1 - 2^u|
// with aE = beta lq - log2 pi + ac sa + bc sb [+ (kappa-1) lz1] and
// u = b1 ((lmmin - lm1) + (lmmin_lo - lm1_lo)).  SLOW adds the series for |u| < 1/8 and the
// beta = -1 normalisation.
template <bool SLOW, bool HAS_Z>
__device__ __forceinline__ f2 pair_weight(const PairFeat& x, const LaneConsts& c)
{
    f2 aE = fma2(c.beta, x.lq, x.nlpi);
    aE = fma2(c.ac, x.sa, aE);
    aE = fma2(c.bc_, x.sb, aE);
    if (HAS_Z) aE = fma2(c.km1, x.lz1, aE);
    const f2 A = fma2(c.nalpha, x.lm1, add2(aE, c.cpl));
    const f2 d = add2(x.m1, c.nmu);
    const f2 B = fma2(mul2(c.nh, d), d, add2(aE, c.cg));
    const f2 e12 = add2(ex2_2(A), ex2_2(B));
    // The hi parts of (lmmin - lm1) cancel exactly near m1 = mmin; the lo parts carry the rest.
    const f2 u = fma2(c.b1, sub2(c.lmmin, x.lm1), fma2(c.nb1, x.lm1lo, c.b1lo));
    f2 den = add2(ex2_2(u), c.neg1);  // 2^u - 1
    if (SLOW) {
        // e^(u ln2) - 1 to fifth order in u ln2 (truncation below 1e-8 relative for |u| < 1/8).
        const f2 c1 = bc(0.693147180559945f), c2 = bc(0.240226506959101f), c3 = bc(0.0555041086648216f),
                 c4 = bc(0.00961812910762848f), c5 = bc(0.00133335581464284f);
        f2 p = fma2(c5, u, c4);
        p = fma2(p, u, c3);
        p = fma2(p, u, c2);
        p = fma2(p, u, c1);
        p = mul2(p, u);
        float ua, ub, pa, pb, da, db;
        upk(u, ua, ub);
        upk(p, pa, pb);
        upk(den, da, db);
        da = fabsf(ua) < 0.125f ? pa : da;
        db = fabsf(ub) < 0.125f ? pb : db;
        if (c.beta_m1) {  // normalisation ln(m1/mmin) = -u ln2 (u < 0 inside the support)
            da = ua;
            db = ub;
        }
        den = pk(da, db);
    }
    const f2 tt = add2(c.t0, ex2_2(fma2(c.nht, x.dc, c.ct)));
    float da, db;
    upk(den, da, db);
    // The last product as an fma with a zero addend that the compiler cannot see, so that it is
    // rounded on its own even where an add follows it directly (the compiler otherwise contracts
    // a packed multiply into a following packed add, and the sums would depend on which path
    // the caller took).
    return fma2(mul2(e12, tt), pk(rcpf(fabsf(da)), rcpf(fabsf(db))), c.zero);
}

__device__ __forceinline__ void kahan2(f2& s, f2& cs, f2 w)
{
    const f2 y = sub2(w, cs);
    const f2 t = add2(s, y);
    cs = sub2(sub2(t, s), y);
    s = t;
}

// Masked weights of pair p of the staged sub-tile (first sample at chunk index j).  CHECK_J
// applies the lower edge j >= j0; past the largest j0 of the warp only m1 <= mmax is tested
// (a lane without in-support samples has thr_hi = -inf).  CHECK_HI = false drops that test
// where the caller knows that every staged m1 passes it for every lane with support.
template <bool SLOW, bool CHECK_J, bool HAS_Z, bool CHECK_HI>
__device__ __forceinline__ f2 masked_pair(const ulonglong2* __restrict__ buf, const f2* __restrict__ zb, int p, int j,
                                          int j0, const LaneConsts& c)
{
    PairFeat x;
    load_pair<HAS_Z>(buf, zb, p, x);
    const f2 w = pair_weight<SLOW, HAS_Z>(x, c);
    float wa, wb, m1a, m1b;
    upk(w, wa, wb);
    upk(x.m1, m1a, m1b);
    const bool ia = (!CHECK_HI || m1a <= c.thr_hi) && (!CHECK_J || j >= j0);
    const bool ib = (!CHECK_HI || m1b <= c.thr_hi) && (!CHECK_J || j + 1 >= j0);
    return pk(ia ? wa : 0.0f, ib ? wb : 0.0f);
}

// Pairs [p0, p1) of the staged sub-tile whose first sample is chunk index jb + 2p.  Four pairs
// are added first (two roundings more per four pairs), then the packed Kahan sums take the
// result: a fifth of the compensated additions.  p0 is a multiple of 4, so the groups are the
// same for every lane whatever its warp.
template <bool SLOW, bool CHECK_J, bool INJ, bool HAS_Z, bool CHECK_HI>
__device__ __forceinline__ void run_pairs(const ulonglong2* __restrict__ buf, const f2* __restrict__ zb, int p0, int p1,
                                          int jb, int j0, const LaneConsts& c, f2& s, f2& cs, f2& s2, f2& cs2)
{
    int p = p0;
#pragma unroll 1
    for (; p + 3 < p1; p += 4) {
        const f2 w0 = masked_pair<SLOW, CHECK_J, HAS_Z, CHECK_HI>(buf, zb, p, jb + 2 * p, j0, c);
        const f2 w1 = masked_pair<SLOW, CHECK_J, HAS_Z, CHECK_HI>(buf, zb, p + 1, jb + 2 * p + 2, j0, c);
        const f2 w2 = masked_pair<SLOW, CHECK_J, HAS_Z, CHECK_HI>(buf, zb, p + 2, jb + 2 * p + 4, j0, c);
        const f2 w3 = masked_pair<SLOW, CHECK_J, HAS_Z, CHECK_HI>(buf, zb, p + 3, jb + 2 * p + 6, j0, c);
        kahan2(s, cs, add2(add2(w0, w1), add2(w2, w3)));
        if (INJ) kahan2(s2, cs2, fma2(w0, w0, fma2(w1, w1, fma2(w2, w2, mul2(w3, w3)))));
    }
#pragma unroll 1
    for (; p + 1 < p1; p += 2) {
        const f2 w0 = masked_pair<SLOW, CHECK_J, HAS_Z, CHECK_HI>(buf, zb, p, jb + 2 * p, j0, c);
        const f2 w1 = masked_pair<SLOW, CHECK_J, HAS_Z, CHECK_HI>(buf, zb, p + 1, jb + 2 * p + 2, j0, c);
        kahan2(s, cs, add2(w0, w1));
        if (INJ) kahan2(s2, cs2, fma2(w0, w0, mul2(w1, w1)));
    }
    if (p < p1) {
        const f2 w0 = masked_pair<SLOW, CHECK_J, HAS_Z, CHECK_HI>(buf, zb, p, jb + 2 * p, j0, c);
        kahan2(s, cs, w0);
        if (INJ) kahan2(s2, cs2, mul2(w0, w0));
    }
}

// The three regions of a sub-tile's pairs for one warp: with the series (and the lower-edge
// test), then without the series but with the test, then neither.
template <bool INJ, bool HAS_Z, bool CHECK_HI>
__device__ __forceinline__ void run_regions(const ulonglong2* __restrict__ buf, const f2* __restrict__ zb, int p_beg,
                                            int p_slow, int p_chk, int p_end, int jb, int j0, const LaneConsts& c,
                                            f2& s, f2& cs, f2& s2, f2& cs2)
{
    run_pairs<true, true, INJ, HAS_Z, CHECK_HI>(buf, zb, p_beg, p_slow, jb, j0, c, s, cs, s2, cs2);
    run_pairs<false, true, INJ, HAS_Z, CHECK_HI>(buf, zb, p_slow, p_chk, jb, j0, c, s, cs, s2, cs2);
    run_pairs<false, false, INJ, HAS_Z, CHECK_HI>(buf, zb, p_chk, p_end, jb, j0, c, s, cs, s2, cs2);
}

// The two searches of a work item's start, in lockstep so that their loads overlap (each is
// a lower bound over the chunk; the range halves the same way for both):
//   j0 = first chunk index whose (m2, m1) exceeds (mmin, mmin) lexicographically, i.e. the
//        first sample with m1 > mmin and m2 >= mmin (both in FP64);
//   js = first chunk index with m2 >= t.
// Each lower bound keeps its base on the last position known to fail its test (len >= 1).
__device__ __forceinline__ void item_searches(const FeatF32& F, const Chunk& ch, double mmin, double t, int& j0,
                                              int& js)
{
    const double* m2 = F.m2 + ch.start;
    const double* m1 = F.m1d + ch.start;
    auto before_edge = [&](int i) {
        const double a = __ldg(m2 + i);
        return !(a > mmin || (a == mmin && __ldg(m1 + i) > mmin));
    };
    int b0 = 0, b1 = 0, n = ch.len;
    while (n > 1) {
        const int half = n >> 1;
        const bool f0 = before_edge(b0 + half);
        const bool f1 = __ldg(m2 + b1 + half) < t;
        b0 = f0 ? b0 + half : b0;
        b1 = f1 ? b1 + half : b1;
        n -= half;
    }
    j0 = b0 + (before_edge(b0) ? 1 : 0);
    js = b1 + (__ldg(m2 + b1) < t ? 1 : 0);
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Stage samples [2 SP st, 2 SP (st+1)) of the chunk: sample s of the sub-tile goes to pair
// s/2, half s%2; positions past the chunk's end get a sample outside every support
// (m1 = +inf).  Lane l of a warp copies feature ((l/4 + i) mod 8) of sample 32 w + l in
// step i, so the 32 four-byte writes of a step land in 32 different banks.
template <int NT, bool HAS_Z>
__device__ __forceinline__ void stage(const FeatF32& F, const Chunk& ch, int st, float* __restrict__ buf,
                                      float* __restrict__ zb)
{
    constexpr int SP = F32Cfg<NT>::SP;
    const int lane = threadIdx.x & 31;
    for (int s = threadIdx.x; s < 2 * SP; s += NT) {
        const int j = 2 * SP * st + s;
        float* dst = buf + 16 * (s >> 1) + (s & 1);
        if (j < ch.len) {
            const float* src = F.base + ch.start + j;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int f = ((lane >> 2) + i) & 7;  // staged slot: lm1 m1 lq sa sb dc nlpi lm1lo
                cp_async4(dst + 2 * f, src + (f == 7 ? F32_LM1LO : f) * F.stride);
            }
            if (HAS_Z) cp_async4(zb + s, src + F_LZ1 * F.stride);
        } else {
#pragma unroll
            for (int f = 0; f < 8; ++f) dst[2 * f] = (f == 1) ? INFINITY : 0.0f;
            if (HAS_Z) zb[s] = 0.0f;
        }
    }
}

template <int NT, bool HAS_Z>
__global__ void __launch_bounds__(NT, F32Cfg<NT>::MIN_BLOCKS)
weight_f32_kernel(FeatF32 ev, FeatF32 inj, WorkDesc wd, const LamF32* __restrict__ lam,
                  const int32_t* __restrict__ order, const int32_t* __restrict__ n_mc,
                  unsigned long long* __restrict__ queue, int64_t K_cap,
                  const int64_t* __restrict__ dK, double* __restrict__ part, double* __restrict__ part2, float zero)
{
    constexpr int SP = F32Cfg<NT>::SP;
    __shared__ __align__(16) float sbuf[2][SP * 16];
    __shared__ __align__(16) float szb[HAS_Z ? 2 : 1][HAS_Z ? 2 * SP : 2];
    __shared__ int s_jmin;
    const int64_t K = *dK;
    const int64_t K_inj = *n_mc;  // Lambda whose xi needs the injections, first in the injection order
    const int64_t tiles_ev = (K + NT - 1) / NT;
    const int64_t tiles_inj = (K_inj + NT - 1) / NT;
    const int n_inj_chunks = wd.n_chunks - wd.n_ev_chunks;
    const int64_t n_ev_items = (int64_t)wd.n_ev_chunks * tiles_ev;
    const int64_t n_items = n_ev_items + (int64_t)n_inj_chunks * tiles_inj;
    const int lane = threadIdx.x & 31;

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
        const FeatF32 F = is_inj ? inj : ev;
        const int64_t slot = tile * NT + threadIdx.x;
        const bool active = slot < (is_inj ? K_inj : K);
        const int k = active ? order[(is_inj ? K_cap : 0) + slot] : 0;
        const LamF32 L = lam[k];
        int j0 = ch.len, js = 0;
        if (active) {
            const double mmin = __longlong_as_double(L.mmin_bits);  // +inf for an invalid Lambda
            // |u| >= 1/8 (with a 2^-10 margin) from m1 >= mmin 2^(1/(8|1+beta|)) on, and m1 >= m2.
            const double t = L.beta_m1 ? INFINITY : mmin * exp2(0.125 / fabs((double)L.b1)) * (1.0 + 0x1p-10);
            item_searches(F, ch, mmin, t, j0, js);
            if (j0 >= ch.len) js = 0;
            else if (L.beta_m1) js = ch.len;
        }
        LaneConsts cl = lane_consts(L, zero);
        // The smallest upper edge over the warp's lanes with in-support samples (positive floats
        // order like their bits; +inf when there is none).
        const float wthr =
            __uint_as_float(__reduce_min_sync(0xffffffffu, j0 < ch.len ? __float_as_uint(cl.thr_hi) : 0x7f800000u));
        if (j0 >= ch.len) cl.thr_hi = -INFINITY;  // no in-support sample: masked without the index test
        const int wj0 = __reduce_min_sync(0xffffffffu, j0);
        const int wj1 = __reduce_max_sync(0xffffffffu, j0 < ch.len ? j0 : 0);
        const int wjs = __reduce_max_sync(0xffffffffu, js);
        __syncthreads();  // the previous item is done with s_jmin
        if (threadIdx.x == 0) s_jmin = ch.len;
        __syncthreads();
        if (lane == 0 && wj0 < ch.len) atomicMin(&s_jmin, wj0);
        __syncthreads();
        const int n_sub = (ch.len + 2 * SP - 1) / (2 * SP);
        const int first = s_jmin < ch.len ? s_jmin / (2 * SP) : n_sub;
        f2 s = 0ull, cs = 0ull, s2 = 0ull, cs2 = 0ull;
        if (first < n_sub) {
            stage<NT, HAS_Z>(F, ch, first, sbuf[0], szb[0]);
            cp_async_commit();
            for (int st = first; st < n_sub; ++st) {
                const int b = (st - first) & 1;
                if (st + 1 < n_sub) stage<NT, HAS_Z>(F, ch, st + 1, sbuf[b ^ 1], szb[HAS_Z ? (b ^ 1) : 0]);
                cp_async_commit();
                cp_async_wait1();
                __syncthreads();
                const int jb = 2 * SP * st;
                // Region edges at pair indices that are multiples of 4 (SP is one, so they are in
                // the chunk too): the pre-summed groups of 4 pairs are the same for every warp,
                // and so is every lane's rounding.  Zero pairs ahead of a lane's j0 leave its sums
                // at 0.  Only p_end, the same for every warp, may fall between.
                const int p_end = min(SP, (ch.len - jb + 1) >> 1);
                const int p_beg = min(p_end, max(0, (wj0 - jb) >> 1)) & ~3;
                const int p_slow = min(p_end, max(p_beg, ((((wjs - jb + 1) >> 1) + 1) + 3) & ~3));
                const int p_chk = min(p_end, max(p_slow, ((((wj1 - jb + 1) >> 1) + 1) + 3) & ~3));
                const ulonglong2* bq = reinterpret_cast<const ulonglong2*>(sbuf[b]);
                const f2* bz = reinterpret_cast<const f2*>(szb[HAS_Z ? b : 0]);
                // A sub-tile without padding whose samples all lie at or below the warp's smallest
                // upper edge (from the per-block maxima of rd32(m1)) skips the upper-edge test.
                bool check_hi = true;
                if (jb + 2 * SP <= ch.len) {
                    const int64_t b0 = (ch.start + jb) / M1MAX_BLOCK, b1 = (ch.start + jb + 2 * SP - 1) / M1MAX_BLOCK;
                    static_assert(2 * SP / M1MAX_BLOCK + 1 <= 32, "a lane per block");
                    const unsigned mx = __reduce_max_sync(
                        0xffffffffu, b0 + lane <= b1 ? __float_as_uint(__ldg(F.m1max + b0 + lane)) : 0u);
                    check_hi = !(__uint_as_float(mx) <= wthr);
                }
                if (check_hi) {
                    if (is_inj)
                        run_regions<true, HAS_Z, true>(bq, bz, p_beg, p_slow, p_chk, p_end, jb, j0, cl, s, cs, s2, cs2);
                    else
                        run_regions<false, HAS_Z, true>(bq, bz, p_beg, p_slow, p_chk, p_end, jb, j0, cl, s, cs, s2, cs2);
                } else {
                    if (is_inj)
                        run_regions<true, HAS_Z, false>(bq, bz, p_beg, p_slow, p_chk, p_end, jb, j0, cl, s, cs, s2, cs2);
                    else
                        run_regions<false, HAS_Z, false>(bq, bz, p_beg, p_slow, p_chk, p_end, jb, j0, cl, s, cs, s2, cs2);
                }
                __syncthreads();  // buffer b is refilled two sub-tiles on
            }
        }
        if (j0 >= ch.len) s = cs = s2 = cs2 = 0ull;  // no in-support sample (the unchecked sub-tiles added to it)
        if (active) {
            float sa, sb, ca, cb;
            upk(s, sa, sb);
            upk(cs, ca, cb);
            part[(int64_t)k * wd.n_chunks + c] = ((double)sa - (double)ca) + ((double)sb - (double)cb);
            if (is_inj) {
                upk(s2, sa, sb);
                upk(cs2, ca, cb);
                part2[(int64_t)k * n_inj_chunks + (c - wd.n_ev_chunks)] =
                    ((double)sa - (double)ca) + ((double)sb - (double)cb);
            }
        }
    }
}

// ---------------------------------------------------------------- upper-edge fix-up
// Features of one sample in both halves of a pair, read from the feature rows.
template <bool HAS_Z>
__device__ __forceinline__ void load_single(const FeatF32& F, int64_t idx, PairFeat& x)
{
    const float* b = F.base + idx;
    x.lm1 = bc(__ldg(b + F_LM1 * F.stride));
    x.m1 = bc(__ldg(b + F_M1 * F.stride));
    x.lq = bc(__ldg(b + F_LQ * F.stride));
    x.sa = bc(__ldg(b + F_SA * F.stride));
    x.sb = bc(__ldg(b + F_SB * F.stride));
    x.dc = bc(__ldg(b + F_DC * F.stride));
    x.nlpi = bc(__ldg(b + F_NLPI * F.stride));
    x.lm1lo = bc(__ldg(b + F32_LM1LO * F.stride));
    x.lz1 = HAS_Z ? bc(__ldg(b + F_LZ1 * F.stride)) : 0ull;
}

// First entry of the set's m1-sorted table with m1 > x (n when there is none; n >= 1).
__device__ __forceinline__ int64_t first_m1_above(const FeatF32& F, double x)
{
    int64_t b = 0, n = F.n;
    while (n > 1) {
        const int64_t half = n >> 1;
        b = __ldg(F.m1sort + b + half) <= x ? b + half : b;
        n -= half;
    }
    return b + (__ldg(F.m1sort + b) <= x ? 1 : 0);
}

// One Lambda per thread.  The main loop kept every sample with j >= j0 and rd32(m1) <= thr_hi;
// the ones among them with m1 > mmax lie outside the support.  They are the entries of the
// m1-sorted table from the first m1 > mmax on, while rd32(m1) is still thr_hi (none, in
// practice, but one per Lambda costs nothing to check).  Each one that the lower edge keeps
// (m2 > mmin, or m2 == mmin and m1 > mmin) has its weight taken out of its chunk's partials.
// pair_weight<true> reproduces the main loop's weight bit for bit: the series branch changes
// the result only where |u| < 1/8 or beta = -1, and there the main loop runs it as well; so a
// chunk whose only kept sample is such a one comes back to exactly 0.
template <bool HAS_Z>
__global__ void __launch_bounds__(128)
upper_edge_fixup_kernel(FeatF32 ev, FeatF32 inj, WorkDesc wd, const LamF32* __restrict__ lam,
                        const uint8_t* __restrict__ need_mc, const int64_t* __restrict__ dK,
                        double* __restrict__ part, double* __restrict__ part2)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= *dK) return;
    const LamF32 L = lam[k];
    if (!L.valid) return;
    const double mmin = __longlong_as_double(L.mmin_bits), mmax = __longlong_as_double(L.mmax_bits);
    const LaneConsts c = lane_consts(L);
    const int n_inj_chunks = wd.n_chunks - wd.n_ev_chunks;
    const bool do_inj = n_inj_chunks > 0 && inj.n > 0 && (need_mc == nullptr || need_mc[k]);
    for (int set = 0; set < (do_inj ? 2 : 1); ++set) {
        const FeatF32& F = set ? inj : ev;
        if (F.n < 1) continue;
        for (int64_t i = first_m1_above(F, mmax); i < F.n; ++i) {
            const double m1 = __ldg(F.m1sort + i);
            if (__double2float_rd(m1) != L.thr_hi) break;
            const uint2 pc = F.m1pos[i];
            const double m2 = __ldg(F.m2 + pc.x);
            if (!(m2 > mmin || (m2 == mmin && m1 > mmin))) continue;
            PairFeat x;
            load_single<HAS_Z>(F, pc.x, x);
            float w, w_b;
            upk(pair_weight<true, HAS_Z>(x, c), w, w_b);
            if (set == 0) {
                part[k * wd.n_chunks + pc.y] -= (double)w;
            } else {
                part[k * wd.n_chunks + wd.n_ev_chunks + pc.y] -= (double)w;
                part2[k * n_inj_chunks + pc.y] -= (double)__fmul_rn(w, w);
            }
        }
    }
}

template <int NT>
const void* pick_f32(bool has_z)
{
    return has_z ? (const void*)weight_f32_kernel<NT, true> : (const void*)weight_f32_kernel<NT, false>;
}

// ---------------------------------------------------------------- Lambda order
constexpr int ORDER_THREADS = 1024;
constexpr int ORDER_BINS = 1024;

// Exclusive prefix sum of one value per thread over the block (ORDER_THREADS threads).
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_tot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();  // warp_tot is free
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    return (warp ? warp_tot[warp - 1] : 0) + x - v;
}

// order[0, K): the Lambda by increasing mmin (1024 bins, equal in the bit pattern of mmin, which
// orders positive doubles like their values, over the batch's range; invalid Lambda last).  The
// range and the bins use integer operations only (an FP64 min/max loop over the warps' partials
// on every thread took most of this kernel's time).  order[K_cap, K_cap + K): the same with the Lambda that need the
// Monte Carlo xi (need_mc[k] != 0) first; *n_mc = their number (K without need_mc).  The order
// within a bin is arbitrary: it only decides which lane evaluates which Lambda.
__global__ void __launch_bounds__(ORDER_THREADS)
lam_order_kernel(const LamF32* __restrict__ lam, const int64_t* __restrict__ dK, const uint8_t* __restrict__ need_mc,
                 int64_t K_cap, int32_t* __restrict__ order, int32_t* __restrict__ n_mc)
{
    __shared__ int h_ev[ORDER_BINS], h_inj[2 * ORDER_BINS], warp_tot[32];
    __shared__ long long s_lo[32], s_hi[32];
    constexpr long long INF_BITS = 0x7ff0000000000000LL;  // +inf: an invalid Lambda's mmin
    const int K = (int)*dK;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long lo = INF_BITS, hi = 0;
    int cnt = 0;
    for (int k = threadIdx.x; k < K; k += ORDER_THREADS) {
        const long long m = lam[k].mmin_bits;
        if (m < INF_BITS) {
            lo = min(lo, m);
            hi = max(hi, m);
        }
        cnt += (need_mc == nullptr || need_mc[k]) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0) {
        s_lo[warp] = lo;
        s_hi[warp] = hi;
        warp_tot[warp] = cnt;
    }
    for (int i = threadIdx.x; i < ORDER_BINS; i += ORDER_THREADS) h_ev[i] = 0;
    for (int i = threadIdx.x; i < 2 * ORDER_BINS; i += ORDER_THREADS) h_inj[i] = 0;
    __syncthreads();
    lo = s_lo[0];
    hi = s_hi[0];
    cnt = 0;
    for (int w = 0; w < ORDER_THREADS / 32; ++w) {
        lo = min(lo, s_lo[w]);
        hi = max(hi, s_hi[w]);
        cnt += warp_tot[w];
    }
    // bin = floor((m - lo) 1024 / (range + 1)) on the bit patterns, both shifted to 20 bits.
    const unsigned long long range = hi > lo ? (unsigned long long)(hi - lo) : 0ull;
    const int sh = (range >> 20) ? 44 - __clzll((long long)range) : 0;
    const unsigned den = (unsigned)(range >> sh) + 1u;
    auto bin = [&](int k) {
        const long long m = lam[k].mmin_bits;
        if (m >= INF_BITS) return ORDER_BINS - 1;
        return min(ORDER_BINS - 1, (int)(((unsigned)((unsigned long long)(m - lo) >> sh) * ORDER_BINS) / den));
    };
    for (int k = threadIdx.x; k < K; k += ORDER_THREADS) {
        const int b = bin(k);
        atomicAdd(&h_ev[b], 1);
        atomicAdd(&h_inj[(need_mc == nullptr || need_mc[k]) ? b : ORDER_BINS + b], 1);
    }
    __syncthreads();
    {
        const int i = threadIdx.x;  // ORDER_THREADS == ORDER_BINS
        const int e = block_exclusive_scan(h_ev[i], warp_tot);
        const int a = h_inj[2 * i], b = h_inj[2 * i + 1];
        const int f = block_exclusive_scan(a + b, warp_tot);
        __syncthreads();
        h_ev[i] = e;
        h_inj[2 * i] = f;
        h_inj[2 * i + 1] = f + a;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += ORDER_THREADS) {
        const int b = bin(k);
        order[atomicAdd(&h_ev[b], 1)] = k;
        order[K_cap + atomicAdd(&h_inj[(need_mc == nullptr || need_mc[k]) ? b : ORDER_BINS + b], 1)] = k;
    }
    if (threadIdx.x == 0) *n_mc = cnt;
}

}  // namespace

const void* weight_f32_fn(const Tiling& t, bool has_z)
{
    if (t.lambda_tile != t.block_threads) return nullptr;
    switch (t.block_threads) {
        case 32: return pick_f32<32>(has_z);
        case 64: return pick_f32<64>(has_z);
        case 128: return pick_f32<128>(has_z);
        case 256: return pick_f32<256>(has_z);
        default: return nullptr;
    }
}

cudaError_t launch_upper_edge_fixup(FeatF32 ev, FeatF32 inj, WorkDesc wd, const LamF32* lam, const uint8_t* need_mc,
                                    int64_t K_cap, const int64_t* dK, double* part, double* part2, cudaStream_t s)
{
    if (K_cap <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((K_cap + 127) / 128);
    if (wd.has_z) upper_edge_fixup_kernel<true><<<blocks, 128, 0, s>>>(ev, inj, wd, lam, need_mc, dK, part, part2);
    else upper_edge_fixup_kernel<false><<<blocks, 128, 0, s>>>(ev, inj, wd, lam, need_mc, dK, part, part2);
    return cudaGetLastError();
}

cudaError_t launch_lam_order(const LamF32* lam, const int64_t* dK, const uint8_t* need_mc, int64_t K_cap,
                             int32_t* order, int32_t* n_mc, cudaStream_t s)
{
    static_assert(ORDER_THREADS == ORDER_BINS, "one scan element per thread");
    lam_order_kernel<<<1, ORDER_THREADS, 0, s>>>(lam, dK, need_mc, K_cap, order, n_mc);
    return cudaGetLastError();
}

cudaError_t launch_weight_f32(const Tiling& t, int grid, FeatF32 ev, FeatF32 inj, WorkDesc wd, const LamF32* lam,
                              const int32_t* order, const int32_t* n_mc, unsigned long long* queue, int64_t K_cap,
                              const int64_t* dK, double* part, double* part2, cudaStream_t s)
{
    const void* fn = weight_f32_fn(t, wd.has_z != 0);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    float zero = 0.0f;  // passed at run time (pair_weight)
    void* args[] = {&ev, &inj, &wd, &lam, &order, &n_mc, &queue, &K_cap, &dK, &part, &part2, &zero};
    return cudaLaunchKernel(fn, dim3(grid), dim3(t.block_threads), args, 0, s);
}

}  // namespace pop

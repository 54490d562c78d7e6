// Exact SURE threshold of one subband without sorting it (Sec. 3, the
// unnumbered equation after Algorithm 1; alpha of line 7): the batched form
// of the threshold step.
//
// SURE(theta) = sum_{a <= theta} (a^2 - tau) + sum_{a > theta} (theta^2 + tau - tau theta / a)
// over the magnitudes a of the subband.  On each interval between consecutive
// sorted magnitudes it is the convex quadratic of sure_dev.cuh, and the exact
// minimiser is the best clamped vertex over all intervals.  Only the intervals
// near the minimum need the magnitudes in sorted order, so:
//   1. bucket the magnitudes by their IEEE-754 bit patterns (exactly ordered
//      buckets: 16 << lpo buckets over the 16 octaves below the maximum,
//      smaller ones in bucket 0; exact zeros apart, always "below");
//   2. per bucket j the count n_j and the sums of a^2 and of 1/a, as integer
//      sums of 16-bit quantised offsets inside the bucket's value range (order-
//      independent, hence deterministic; bucket 0 summed per thread in a fixed
//      order instead), prefix sums over buckets;
//   3. for theta in bucket j's range [lo_j, hi_j) every magnitude of the bucket
//      contributes at least lo_j^2 - tau (below theta: a^2 - tau; above:
//      theta^2 + tau (1 - theta / a) >= theta^2), the others exactly a convex
//      quadratic in theta, so
//        LB_j = C_<j - tau m_<j + n_j (lo_j^2 - tau) + min_[lo_j,hi_j] (K_>j (t^2 + tau) - tau t H_>j)
//      bounds SURE from below there; SURE just below lo_j (where the split is
//      known exactly) and at theta >= max a are attained values, UB their minimum;
//   4. only buckets with LB_j <= UB + 1e-5 (sum a^2 + N_b tau) can hold the
//      minimiser (the margin covers the FP32 rounding of the bounds): an
//      empty one is a single quadratic piece, evaluated at once; the keys of
//      the others (a few hundred of N_b) are gathered from the magnitudes,
//      which stay in shared memory from the first step (r_k is read once),
//      ranked within their bucket, and every interval piece inside these
//      buckets is evaluated as in the full search.
// A piece whose vertex lies beyond the bucket's upper edge is skipped: its
// minimum over the interval lies in a higher bucket, where it is either
// evaluated or bounded above UB.  Candidates are compared in FP32 (ties to
// the smaller theta, then the smaller m), the winner recomputed in FP64.
//
// Precision and cost: FP64 runs at a small fraction of the FP32 rate on this
// GPU, so no per-thread step uses it.  A prefix sum is carried as an FP64
// base per warp (formed by one warp's FP64 shuffle scan over the warp totals)
// plus an FP32 offset inside the warp; the FP32 comparisons use the base
// rounded once to FP32, and only the winning candidate forms base + offset in
// FP64.
//
// A CTA of PRUNE_THREADS threads takes one large subband, two medium ones (up
// to PRUNE_MED_BAND magnitudes, a group of PRUNE_MED threads each) or four
// small ones (up to PRUNE_SMALL_BAND magnitudes, PRUNE_GROUP threads each);
// a group has a named barrier of its own, so the groups' barrier-separated
// phases overlap and the fixed cost of a phase is shared.  A subband whose candidates exceed its
// tables (PruneLimits: non-empty candidate buckets, candidate magnitudes,
// magnitudes of one candidate bucket; heavy ties or degenerate data) is
// appended to a device list, and sure_fallback_kernel solves it with the
// one-CTA full sort and search.
#pragma once

#include "sure_dev.cuh"

namespace vdamp {

#define PRUNE_THREADS 1024       // threads of a CTA: one large subband, or four groups
#define PRUNE_WARPS (PRUNE_THREADS / 32)
#define PRUNE_GROUP 256          // threads of a group that takes one small subband
#define PRUNE_GROUPS (PRUNE_THREADS / PRUNE_GROUP)
#define PRUNE_SMALL_BAND (8 * PRUNE_GROUP)   // subbands up to 2048 magnitudes go to a group
#define PRUNE_MED 512            // threads of a group that takes one medium subband
#define PRUNE_MED_BAND (16 * PRUNE_MED)      // subbands up to 8192 magnitudes: two per CTA
#define PRUNE_BIG_BAND 32768     // the largest subband of the pruned search

// Limits per subband, for a whole CTA (NT = PRUNE_THREADS), a medium group and a
// small group: magnitudes held, log2 buckets per octave, candidate magnitudes,
// non-empty candidate buckets, magnitudes of one candidate bucket.
template <int NT> struct PruneLimits {
    static constexpr bool big = NT == PRUNE_THREADS, med = NT == PRUNE_MED;
    static constexpr int max_band = big ? PRUNE_BIG_BAND : (med ? PRUNE_MED_BAND : PRUNE_SMALL_BAND);
    static constexpr int max_lpo = big ? 8 : (med ? 7 : 6);   // 4096 / 2048 / 1024 buckets
    static constexpr int cap = big || med ? 2048 : 1024;
    static constexpr int table = big || med ? 256 : 128;
    static constexpr int bucket_max = big ? 1024 : (med ? 512 : 256);
    static constexpr int loads = NT >= PRUNE_MED ? 16 : 8;   // r_k loads in flight per thread
};

// log2 of the buckets per octave: about one bucket per magnitude, 16 .. 2^max_lpo.
__host__ __device__ inline int prune_lpo(int nb, int max_lpo) {
    int l = 4;
    while (l < max_lpo && (16 << l) < nb) ++l;
    return l;
}

// A sum carried as an FP64 base and an FP32 offset (base + off in FP64 only
// where the exact value is needed; basef = base rounded to FP32).
struct Split {
    double base;
    float basef, off;
    __device__ __forceinline__ float approx() const { return basef + off; }
    __device__ __forceinline__ double exact() const { return base + (double)off; }
    __device__ __forceinline__ Split plus(float x) const { return Split{base, basef, off + x}; }
};

struct PruneEntry {   // one non-empty candidate bucket
    Split c_lt;       // sum of a^2 over the magnitudes below the bucket
    Split h_gt;       // sum of 1/a over the magnitudes above the bucket
    float lo, hi;     // the bucket's value range [lo, hi)
    int m_lt;         // magnitudes below the bucket (exact zeros included)
    int n;            // magnitudes in the bucket
    int start;        // first slot in the candidate buffers
    int fill;         // gather counter
};

// Dynamic shared memory of one subband's search (a CTA's, or a group's share):
// the magnitudes, three per-bucket words (count, sum of quantised a^2
// offsets, sum of quantised 1/a offsets; later the packed local prefixes),
// the candidate-bucket bits, three candidate buffers (gathered keys, later
// their prefix sums of a^2; sorted keys; prefix sums of 1/a) and the table of
// candidate buckets.
template <int NT>
__host__ __device__ inline size_t prune_words() {
    using Lim = PruneLimits<NT>;
    constexpr size_t nbk = (size_t)16 << Lim::max_lpo;
    return (size_t)Lim::max_band + 3 * nbk + nbk / 32 + 3 * (size_t)Lim::cap +
           Lim::table * (sizeof(PruneEntry) / sizeof(unsigned));
}
// Dynamic shared memory of the pruned kernel: the largest of one CTA-wide
// search, two medium and four small group searches.
inline size_t prune_smem_bytes() {
    const size_t big = prune_words<PRUNE_THREADS>();
    const size_t med = (PRUNE_THREADS / PRUNE_MED) * prune_words<PRUNE_MED>();
    const size_t small = PRUNE_GROUPS * prune_words<PRUNE_GROUP>();
    const size_t m = big > med ? big : med;
    return (m > small ? m : small) * sizeof(unsigned);
}

// Barrier of the threads taking one subband: the whole CTA (barrier 0), or a
// group's named barrier (1 + its index in the CTA).
template <int NT>
__device__ __forceinline__ void psync(int bar) {
    if (NT == PRUNE_THREADS) __syncthreads();
    else asm volatile("bar.sync %0, %1;" :: "r"(bar), "r"(NT) : "memory");
}

// The best candidate a thread has seen, with what the FP64 recomputation needs.
struct PruneBest {
    float v, t;       // FP32 SURE value and theta
    int m;            // magnitudes at or below theta (nb: theta = max a, the flat top)
    Split c, h;       // sum of a^2 below and of 1/a above theta
    float lo, hi;     // the piece: theta in [lo, hi) (lo = hi = theta on the flat top)
};

__device__ __forceinline__ bool prune_better(float v, float t, int m, const PruneBest& b) {
    return v < b.v || (v == b.v && (t < b.t || (t == b.t && m < b.m)));
}

__device__ __forceinline__ void prune_take(PruneBest& b, float v, float t, int m, const Split& c,
                                           const Split& h, float lo, float hi) {
    if (prune_better(v, t, m, b)) {
        b.v = v;
        b.t = t;
        b.m = m;
        b.c = c;
        b.h = h;
        b.lo = lo;
        b.hi = hi;
    }
}

// One interval piece: m magnitudes at or below theta, the sums c (a^2 below)
// and h (1/a above), theta in [lo, hi): the clamped vertex, if inside (FP32).
__device__ __forceinline__ void prune_piece(PruneBest& best, int nb, float tf, int m,
                                            const Split& c, const Split& h, float lo, float hi) {
    const int K = nb - m;
    if (K <= 0) return;
    const float hf = h.approx(), cf = c.approx(), Kf = (float)K;
    float t = tf * hf * __frcp_rn(2.0f * Kf);
    t = fmaxf(t, lo);
    if (!(t < hi)) return;
    const float v = cf - (float)m * tf + Kf * t * t + Kf * tf - tf * t * hf;
    prune_take(best, v, t, m, c, h, lo, hi);
}

// Static shared state of one subband's search, declared by the kernel (one
// per group; a __shared__ variable inside the templated routine would exist
// once per instantiation).
struct PruneShared {
    double tau, s20, h0;          // tau; sums of a^2 and 1/a over bucket 0
    float s20f, h0f;
    unsigned max;
    int zero, bad, win;
    float flat, ub, delta;        // SURE for theta >= max a, the upper bound, the margin
    int wi[PRUNE_WARPS + 1];      // scan: per-warp exclusive bases (ints), total last
    double wc[PRUNE_WARPS], wh[PRUNE_WARPS];   // FP64 warp bases: prefix of c, suffix of h
    float wcf[PRUNE_WARPS], whf[PRUNE_WARPS];
    double tot_c;
    float tc[PRUNE_WARPS], th[PRUNE_WARPS];    // per-warp totals handed to warp 0
    float red_v[PRUNE_WARPS], red_t[PRUNE_WARPS];
    int red_m[PRUNE_WARPS], red_w[PRUNE_WARPS];
};

// Scan over the NT threads of a subband's search (gtid: index among them) of an int, an FP32 prefix and an
// FP32 suffix per thread: the int's exclusive prefix ei (exact), the
// exclusive prefix c of vc and the sum h of vh over the threads after this
// one, each as an FP64 warp base plus an FP32 offset inside the warp.  The
// FP64 bases come from one warp's shuffle scan over the warp totals.
template <int NT>
__device__ __forceinline__ void prune_scan(PruneShared& sh, int gtid, int bar, int vi, float vc,
                                           float vh, int& ei, Split& c, Split& h, int& tot_i) {
    constexpr int NW = NT / 32;
    const int lane = gtid & 31, warp = gtid >> 5;
    int ii = vi;
    float ic = vc, ih = vh;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {   // inclusive prefix (i, c), inclusive suffix (h)
        const int ti = __shfl_up_sync(0xffffffffu, ii, o);
        const float tc = __shfl_up_sync(0xffffffffu, ic, o);
        const float th = __shfl_down_sync(0xffffffffu, ih, o);
        if (lane >= o) {
            ii += ti;
            ic += tc;
        }
        if (lane + o < 32) ih += th;
    }
    if (lane == 31) {
        sh.wi[warp] = ii;
        sh.tc[warp] = ic;
    }
    if (lane == 0) sh.th[warp] = ih;
    psync<NT>(bar);
    if (warp == 0) {   // FP64 over the warps (lane = warp): exclusive prefix, exclusive suffix
        const bool live = lane < NW;
        int xi = live ? sh.wi[lane] : 0;
        double xc = live ? (double)sh.tc[lane] : 0.0, xh = live ? (double)sh.th[lane] : 0.0;
        int pi = xi;
        double pc = xc, sh_ = xh;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ti = __shfl_up_sync(0xffffffffu, pi, o);
            const double tc = __shfl_up_sync(0xffffffffu, pc, o);
            const double th = __shfl_down_sync(0xffffffffu, sh_, o);
            if (lane >= o) {
                pi += ti;
                pc += tc;
            }
            if (lane + o < 32) sh_ += th;
        }
        const int tot = __shfl_sync(0xffffffffu, pi, 31);
        const double totc = __shfl_sync(0xffffffffu, pc, 31);
        if (live) {
            sh.wi[lane] = pi - xi;
            sh.wc[lane] = pc - xc;
            sh.wh[lane] = sh_ - xh;
            sh.wcf[lane] = (float)(pc - xc);
            sh.whf[lane] = (float)(sh_ - xh);
        }
        if (lane == 0) {
            sh.wi[NW] = tot;
            sh.tot_c = totc;
        }
    }
    psync<NT>(bar);
    int xi = __shfl_up_sync(0xffffffffu, ii, 1);
    float xc = __shfl_up_sync(0xffffffffu, ic, 1);
    float xh = __shfl_down_sync(0xffffffffu, ih, 1);
    if (lane == 0) {
        xi = 0;
        xc = 0.f;
    }
    if (lane == 31) xh = 0.f;
    ei = sh.wi[warp] + xi;
    c = Split{sh.wc[warp], sh.wcf[warp], xc};
    h = Split{sh.wh[warp], sh.whf[warp], xh};
    tot_i = sh.wi[NW];
    psync<NT>(bar);   // the scratch is reused by the next scan
}

// Exclusive prefix (over the NT threads) of two ints (exact) and their totals.
template <int NT>
__device__ __forceinline__ void prune_scan_int2(PruneShared& sh, int gtid, int bar, int va, int vb,
                                                int& ea, int& eb, int& ta, int& tb) {
    constexpr int NW = NT / 32;
    const int lane = gtid & 31, warp = gtid >> 5;
    int ia = va, ib = vb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, ia, o);
        const int y = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += x;
            ib += y;
        }
    }
    if (lane == 31) {
        sh.wi[warp] = ia;
        sh.red_m[warp] = ib;
    }
    psync<NT>(bar);
    if (warp == 0) {
        const bool live = lane < NW;
        const int xa = live ? sh.wi[lane] : 0, xb = live ? sh.red_m[lane] : 0;
        int pa = xa, pb = xb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, pa, o);
            const int y = __shfl_up_sync(0xffffffffu, pb, o);
            if (lane >= o) {
                pa += x;
                pb += y;
            }
        }
        const int tpa = __shfl_sync(0xffffffffu, pa, 31), tpb = __shfl_sync(0xffffffffu, pb, 31);
        if (live) {
            sh.wi[lane] = pa - xa;
            sh.red_m[lane] = pb - xb;
        }
        if (lane == 0) {
            sh.wi[NW] = tpa;
            sh.red_w[0] = tpb;
        }
    }
    psync<NT>(bar);
    ea = sh.wi[warp] + ia - va;
    eb = sh.red_m[warp] + ib - vb;
    ta = sh.wi[NW];
    tb = sh.red_w[0];
    psync<NT>(bar);
}

// Minimum of a float over the NT threads, broadcast to each.
template <int NT>
__device__ __forceinline__ float prune_min(PruneShared& sh, int gtid, int bar, float v) {
    constexpr int NW = NT / 32;
    const int lane = gtid & 31, warp = gtid >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) sh.red_v[warp] = v;
    psync<NT>(bar);
    if (warp == 0) {
        float m = lane < NW ? sh.red_v[lane] : INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) sh.ub = m;
    }
    psync<NT>(bar);
    return sh.ub;
}

// Bucket edges: bucket q >= 1 holds the bit patterns [lo_bits + q 2^shift,
// lo_bits + (q + 1) 2^shift); bucket 0 everything nonzero below its upper edge.
__device__ __forceinline__ float prune_lo(unsigned lo_bits, int shift, int q) {
    return q == 0 ? 0.f : __uint_as_float(lo_bits + ((unsigned)q << shift));
}
__device__ __forceinline__ float prune_hi(unsigned lo_bits, int shift, int q) {
    return __uint_as_float(lo_bits + ((unsigned)(q + 1) << shift));
}

// Sums of a^2 and 1/a over bucket q >= 1 from its count n and the integer sums
// of the quantised offsets (midpoint reconstruction).
__device__ __forceinline__ void prune_bucket_sums(unsigned lo_bits, int shift, int q, int n,
                                                  unsigned q2, unsigned qh, float& s2,
                                                  float& hs) {
    const float lo = prune_lo(lo_bits, shift, q), hi = prune_hi(lo_bits, shift, q);
    const float fn = (float)n;
    s2 = fn * lo * lo + ((float)q2 + 0.5f * fn) * ((hi - lo) * (hi + lo)) * (1.f / 65536.f);
    hs = fn * __frcp_rn(hi) +
         ((float)qh + 0.5f * fn) * ((hi - lo) * __frcp_rn(lo * hi)) * (1.f / 65536.f);
}

// The exact SURE threshold of subband b of slice `slice`, its alpha and the
// line-8 constants (sure_finish), or, when its candidates do not fit the
// table, the subband appended to the fallback list a.fallback ([0] entries,
// [1] the fallback kernel's done counter, [2] a running total of the subbands
// ever appended, [3 ..] slice B + b).  Called by the NT threads that take
// the subband (gtid: index among them; bar: their barrier, see psync); N_b at
// most PruneLimits<NT>::max_band; dyn: prune_words<NT>() words of dynamic
// shared memory of their own.
template <int NT>
static __device__ void sure_prune_subband(const SureArgs& a, int b, int slice, unsigned* dyn,
                                          PruneShared& sh, int gtid, int bar) {
    using Lim = PruneLimits<NT>;
    constexpr int NW = NT / 32;
    const int tid = gtid, lane = tid & 31, warp = tid >> 5;
    const int off = a.off[b], nb = a.off[b + 1] - off;
    const float2* r = a.r + (size_t)slice * a.N + off;
    const int lpo = prune_lpo(nb, Lim::max_lpo), nbk = 16 << lpo, shift = 23 - lpo;
    float* mag = reinterpret_cast<float*>(dyn);   // the magnitudes, in packed order
    if (nb > Lim::max_band) {   // not a subband for this group size: the full sort takes it
        if (tid == 0) {
            const int idx = atomicAdd(&a.fallback[0], 1);
            a.fallback[3 + idx] = slice * a.B + b;
            atomicAdd(&a.fallback[2], 1);
        }
        return;
    }
    unsigned* X = dyn + Lim::max_band;   // count, then (local prefix of counts << 16 | count), then entry
    unsigned* Y = X + nbk;    // sum of quantised a^2 offsets, then local prefix of a^2 (FP32)
    unsigned* Z = Y + nbk;    // sum of quantised 1/a offsets, then local suffix of 1/a (FP32)
    unsigned* F = Z + nbk;    // candidate bits
    float* candA = reinterpret_cast<float*>(F + nbk / 32);   // gathered (bucket order)
    float* candB = candA + Lim::cap;                          // sorted
    float* candH = candB + Lim::cap;                          // prefix sums of 1/a in a bucket
    PruneEntry* tab = reinterpret_cast<PruneEntry*>(candH + Lim::cap);   // 8-byte aligned

    for (int i = tid; i < 3 * nbk + nbk / 32; i += NT) X[i] = 0u;
    if (tid == 0) {
        sh.max = 0u;
        sh.zero = 0;
        sh.bad = 0;
    }
    // tau: a fixed-order FP64 sum of the column blocks' partials; warp 0's first two
    // partials per lane go out before the magnitudes
    const double* tp = a.tau_part + (size_t)slice * a.nparts * a.B + b;
    double t0 = 0.0, t1 = 0.0;
    if (warp == 0) {
        if (lane < a.nparts) t0 = tp[(size_t)lane * a.B];
        if (lane + 32 < a.nparts) t1 = tp[(size_t)(lane + 32) * a.B];
    }
    // the magnitudes into shared memory (Lim::loads loads in flight per thread):
    // the largest (as bits) and the exact zeros
    unsigned mx = 0u;
    int nz = 0;
    for (int i0 = tid; i0 < nb; i0 += Lim::loads * NT) {
        float2 v[Lim::loads];
#pragma unroll
        for (int u = 0; u < Lim::loads; ++u) {
            const int i = i0 + u * NT;
            v[u] = i < nb ? r[i] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < Lim::loads; ++u) {
            const int i = i0 + u * NT;
            if (i < nb) {
                const float x = cabs_f(v[u]);
                mag[i] = x;
                const unsigned bits = __float_as_uint(x);
                mx = max(mx, bits);
                nz += bits == 0u;
            }
        }
    }
    if (warp == 0) {
        double t = t0;
        t += t1;
        for (int p = lane + 64; p < a.nparts; p += 32) t += tp[(size_t)p * a.B];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh.tau = t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        nz += __shfl_xor_sync(0xffffffffu, nz, o);
    }
    psync<NT>(bar);
    if (lane == 0) {
        atomicMax(&sh.max, mx);
        atomicAdd(&sh.zero, nz);
    }
    psync<NT>(bar);
    const double tau = sh.tau;
    const unsigned M = sh.max;
    const int z = sh.zero;
    if (!(tau > 0.0) || !isfinite(tau) || M >= 0x7f800000u || M == 0u) {
        // no effective noise; a numeric failure (tau or a magnitude not finite); or an
        // all-zero subband, where theta = max a = 0
        if (tid == 0) {
            const bool zero = tau > 0.0 && isfinite(tau) && M == 0u;
            sure_finish(a, a.k, b, slice, nb, tau, zero ? nb : -1, 0.0, 0.0,
                        zero ? -(double)nb * tau : 0.0);
        }
        return;
    }
    const float tf = (float)tau;
    const unsigned span = (unsigned)nbk << shift;
    const unsigned lo_bits = M + 1u > span ? M + 1u - span : 0u;

    // ---- counts and quantised sums per bucket (bucket 0 summed per thread)
    float s20 = 0.f, h0 = 0.f;
    for (int i = tid; i < nb; i += NT) {
        const float x = mag[i];
        const unsigned u = __float_as_uint(x);
        if (u == 0u) continue;   // exact zeros
        const int q = u < lo_bits ? 0 : (int)((u - lo_bits) >> shift);
        atomicAdd(&X[q], 1u);
        if (q == 0) {
            s20 += x * x;
            h0 += __frcp_rn(x);
            continue;
        }
        const float lo = prune_lo(lo_bits, shift, q), hi = prune_hi(lo_bits, shift, q);
        // the quantisation needs neither correct rounding nor more than ~1e-6
        const float w = __fdividef(1.f, hi - lo);
        const float r2 = (x - lo) * w * __fdividef(x + lo, hi + lo);   // (a^2 - lo^2) / (hi^2 - lo^2)
        const float rh = (hi - x) * w * __fdividef(lo, x);             // (1/a - 1/hi) / (1/lo - 1/hi)
        atomicAdd(&Y[q], min(__float2uint_rz(r2 * 65536.f), 65535u));
        atomicAdd(&Z[q], min(__float2uint_rz(rh * 65536.f), 65535u));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s20 += __shfl_xor_sync(0xffffffffu, s20, o);
        h0 += __shfl_xor_sync(0xffffffffu, h0, o);
    }
    if (lane == 0) {
        sh.red_v[warp] = s20;
        sh.red_t[warp] = h0;
    }
    psync<NT>(bar);
    if (warp == 0) {   // bucket 0: FP64 over the warps, in a fixed order
        double x2 = lane < NW ? (double)sh.red_v[lane] : 0.0;
        double xh = lane < NW ? (double)sh.red_t[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x2 += __shfl_xor_sync(0xffffffffu, x2, o);
            xh += __shfl_xor_sync(0xffffffffu, xh, o);
        }
        if (lane == 0) {
            sh.s20 = x2;
            sh.h0 = xh;
            sh.s20f = (float)x2;
            sh.h0f = (float)xh;
        }
    }
    psync<NT>(bar);

    // ---- prefix sums over buckets: each thread owns a run of consecutive buckets
    const int per = nbk >= NT ? nbk / NT : 1;
    const int j0 = min(tid * per, nbk), j1 = min(j0 + per, nbk);
    auto sums = [&](int j, int n, float& s2, float& hs) {
        if (j == 0) {
            s2 = sh.s20f;
            hs = sh.h0f;
        } else {
            prune_bucket_sums(lo_bits, shift, j, n, Y[j], Z[j], s2, hs);
        }
    };
    int tm = 0;
    float tc = 0.f, th = 0.f;
    for (int j = j0; j < j1; ++j) {   // the bucket's sums, kept in Y and Z from here on
        float s2, hs;
        const int n = (int)X[j];
        sums(j, n, s2, hs);
        Y[j] = __float_as_uint(s2);
        Z[j] = __float_as_uint(hs);
        tm += n;
        tc += s2;
        th += hs;
    }
    int em, tot_m;
    Split cS, hS;   // a^2 below this thread's buckets, 1/a above them
    prune_scan<NT>(sh, gtid, bar, tm, tc, th, em, cS, hS, tot_m);
    const double c_all = sh.tot_c;
    const int mb = z + em;          // magnitudes below this thread's buckets
    // local prefixes: X = (count below in the run << 16 | count), Y = a^2 below in the run
    {
        int lm = 0;
        float lc = 0.f;
        for (int j = j0; j < j1; ++j) {
            const int n = (int)X[j];
            const float s2 = __uint_as_float(Y[j]);
            X[j] = ((unsigned)lm << 16) | (unsigned)n;
            Y[j] = __float_as_uint(lc);
            lm += n;
            lc += s2;
        }
    }
    // local suffixes of 1/a (Z), and the attained SURE just below each bucket's lower edge
    float umin = INFINITY;
    if (tid == 0) {   // theta >= max a: constant; and the pruning margin
        const float flat = (float)(c_all - (double)nb * tau);
        umin = flat;
        sh.delta = 1e-5f * (float)(c_all + (double)nb * tau);
    }
    {
        float lh = 0.f;
        for (int j = j1 - 1; j >= j0; --j) {
            const unsigned xw = X[j];
            const int n = (int)(xw & 0xffffu), m_lt = mb + (int)(xw >> 16);
            const float hs = __uint_as_float(Z[j]);
            Z[j] = __float_as_uint(lh);
            const float c_lt = cS.basef + (cS.off + __uint_as_float(Y[j]));
            const float h_ge = hS.basef + (hS.off + lh + hs);
            const float t = j == 0 ? 0.f : __uint_as_float(lo_bits + ((unsigned)j << shift) - 1u);
            const float kge = (float)(nb - m_lt);
            umin = fminf(umin, c_lt - tf * (float)m_lt + kge * (t * t + tf) - tf * t * h_ge);
            lh += hs;
        }
    }
    const float ub = prune_min<NT>(sh, gtid, bar, umin);
    const float delta = sh.delta;

    // ---- lower bounds: empty candidate buckets are evaluated now, the others marked
    PruneBest best;
    best.v = INFINITY;
    best.t = INFINITY;
    best.m = 0x7fffffff;
    best.c = best.h = Split{0.0, 0.f, 0.f};
    best.lo = best.hi = 0.f;
    int my_e = 0, my_k = 0;
    for (int j = j0; j < j1; ++j) {
        const unsigned xw = X[j];
        const int n = (int)(xw & 0xffffu), m_lt = mb + (int)(xw >> 16);
        const Split c_lt = cS.plus(__uint_as_float(Y[j]));
        const Split h_gt = hS.plus(__uint_as_float(Z[j]));
        const float lo = prune_lo(lo_bits, shift, j), hi = prune_hi(lo_bits, shift, j);
        const int K = nb - m_lt - n;
        const float hf = h_gt.approx();
        float t = K > 0 ? tf * hf * __frcp_rn(2.f * (float)K) : lo;
        t = fminf(fmaxf(t, lo), hi);
        const float lb = c_lt.approx() - tf * (float)m_lt + (float)n * (lo * lo - tf) +
                         (float)K * (t * t + tf) - tf * t * hf;
        if (!(lb <= ub + delta)) continue;
        if (n == 0) {
            prune_piece(best, nb, tf, m_lt, c_lt, h_gt, lo, hi);
        } else {
            atomicOr(&F[j >> 5], 1u << (j & 31));
            ++my_e;
            my_k += n;
            if (n > Lim::bucket_max) sh.bad = 1;
        }
    }
    int e0, k0, tot_e, tot_k;
    prune_scan_int2<NT>(sh, gtid, bar, my_e, my_k, e0, k0, tot_e, tot_k);
    if (tot_e > Lim::table || tot_k > Lim::cap || sh.bad) {
        if (tid == 0) {
            const int idx = atomicAdd(&a.fallback[0], 1);
            a.fallback[3 + idx] = slice * a.B + b;
            atomicAdd(&a.fallback[2], 1);   // subbands left to the full sort, ever
        }
        return;
    }

    // ---- the table of non-empty candidate buckets; X[j] becomes j's entry (or none)
    {
        int e = e0, kpos = k0;
        for (int j = j0; j < j1; ++j) {
            const unsigned xw = X[j];
            const int n = (int)(xw & 0xffffu);
            if (n > 0 && ((F[j >> 5] >> (j & 31)) & 1u)) {
                PruneEntry& E = tab[e];
                E.c_lt = cS.plus(__uint_as_float(Y[j]));
                E.h_gt = hS.plus(__uint_as_float(Z[j]));
                E.lo = prune_lo(lo_bits, shift, j);
                E.hi = prune_hi(lo_bits, shift, j);
                E.m_lt = mb + (int)(xw >> 16);
                E.n = n;
                E.start = kpos;
                E.fill = 0;
                X[j] = (unsigned)e;
                ++e;
                kpos += n;
            } else {
                X[j] = 0xffffffffu;
            }
        }
    }
    psync<NT>(bar);
    // ---- gather the candidates' magnitudes, grouped by bucket
    for (int i = tid; i < nb; i += NT) {
        const float x = mag[i];
        const unsigned u = __float_as_uint(x);
        if (u == 0u) continue;
        const int q = u < lo_bits ? 0 : (int)((u - lo_bits) >> shift);
        const unsigned ent = X[q];
        if (ent < (unsigned)tot_e) {   // (an entry beyond the table is never written)
            const int slot = tab[ent].start + atomicAdd(&tab[ent].fill, 1);
            if (slot < tot_k) candA[slot] = x;
        }
    }
    psync<NT>(bar);
    auto entry_of = [&](int p) {   // the entry whose slots hold position p
        int l = 0, h = tot_e - 1;
        while (l < h) {
            const int mid = (l + h + 1) >> 1;
            if (tab[mid].start <= p) l = mid;
            else h = mid - 1;
        }
        return l;
    };
    // rank within the bucket (ties by gather slot): the sorted order, whatever the gather order
    for (int p = tid; p < tot_k; p += NT) {
        const PruneEntry& E = tab[entry_of(p)];
        const float x = candA[p];
        int rk = 0;
        for (int k = E.start; k < E.start + E.n; ++k) {
            const float y = candA[k];
            rk += (y < x) || (y == x && k < p);
        }
        candB[E.start + rk] = x;
    }
    psync<NT>(bar);
    // per candidate bucket, in sorted order: inclusive prefix sums of a^2 (candA, no
    // longer needed for the gathered keys) and of 1/a (candH), a warp per bucket
    // (chunks of 32 by shuffle scans)
    for (int e = warp; e < tot_e; e += NW) {
        const PruneEntry& E = tab[e];
        float cs = 0.f, hs = 0.f;   // the chunks before
        for (int i0 = E.start; i0 < E.start + E.n; i0 += 32) {
            const int i = i0 + lane;
            const bool in = i < E.start + E.n;
            const float y = in ? candB[i] : 1.f;
            float c2 = in ? y * y : 0.f, h = in ? __frcp_rn(y) : 0.f;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float tc2 = __shfl_up_sync(0xffffffffu, c2, o);
                const float th2 = __shfl_up_sync(0xffffffffu, h, o);
                if (lane >= o) {
                    c2 += tc2;
                    h += th2;
                }
            }
            if (in) {
                candA[i] = cs + c2;
                candH[i] = hs + h;
            }
            cs += __shfl_sync(0xffffffffu, c2, 31);
            hs += __shfl_sync(0xffffffffu, h, 31);
        }
    }
    psync<NT>(bar);
    // ---- every piece inside the candidate buckets: the interval after each magnitude ...
    for (int p = tid; p < tot_k; p += NT) {
        const PruneEntry& E = tab[entry_of(p)];
        const int k = p - E.start, last = E.start + E.n - 1;
        const float cs = candA[p];                  // a^2 up to and including k
        const float hs = candH[last] - candH[p];    // 1/a after k
        const float bk = candB[p];
        const int m = E.m_lt + k + 1;
        const Split c = E.c_lt.plus(cs);
        if (m == nb) {   // theta >= max a: SURE is constant, theta = max a
            prune_take(best, c.approx() - (float)nb * tf, bk, nb, c, Split{0.0, 0.f, 0.f}, bk, bk);
        } else {
            const float nxt = k + 1 < E.n ? candB[p + 1] : E.hi;
            prune_piece(best, nb, tf, m, c, E.h_gt.plus(hs), bk, nxt);
        }
    }
    // ... and the piece below each candidate bucket's first magnitude
    for (int e = tid; e < tot_e; e += NT) {
        const PruneEntry& E = tab[e];
        prune_piece(best, nb, tf, E.m_lt, E.c_lt, E.h_gt.plus(candH[E.start + E.n - 1]), E.lo,
                    candB[E.start]);
    }

    // ---- the best candidate of the CTA (ties: smaller theta, smaller m, lower thread)
    {
        float v = best.v, t = best.t;
        int m = best.m, w = tid;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
            const float t2 = __shfl_xor_sync(0xffffffffu, t, o);
            const int m2 = __shfl_xor_sync(0xffffffffu, m, o);
            const int w2 = __shfl_xor_sync(0xffffffffu, w, o);
            if (v2 < v || (v2 == v && (t2 < t || (t2 == t && (m2 < m || (m2 == m && w2 < w)))))) {
                v = v2;
                t = t2;
                m = m2;
                w = w2;
            }
        }
        if (lane == 0) {
            sh.red_v[warp] = v;
            sh.red_t[warp] = t;
            sh.red_m[warp] = m;
            sh.red_w[warp] = w;
        }
        psync<NT>(bar);
        if (warp == 0) {
            const bool live = lane < NW;
            v = live ? sh.red_v[lane] : INFINITY;
            t = live ? sh.red_t[lane] : INFINITY;
            m = live ? sh.red_m[lane] : 0x7fffffff;
            w = live ? sh.red_w[lane] : 0x7fffffff;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
                const float t2 = __shfl_xor_sync(0xffffffffu, t, o);
                const int m2 = __shfl_xor_sync(0xffffffffu, m, o);
                const int w2 = __shfl_xor_sync(0xffffffffu, w, o);
                if (v2 < v || (v2 == v && (t2 < t || (t2 == t && (m2 < m || (m2 == m && w2 < w)))))) {
                    v = v2;
                    t = t2;
                    m = m2;
                    w = w2;
                }
            }
            if (lane == 0) sh.win = w;
        }
        psync<NT>(bar);
    }
    // ---- the winner in FP64 (theta, alpha and the line-8 constants by sure_finish)
    if (tid == sh.win) {
        if (!(best.v < INFINITY)) {   // nothing found: recorded as a numeric failure
            sure_finish(a, a.k, b, slice, nb, tau, -1, 0.0, 0.0, 0.0);
        } else if (best.m == nb) {
            sure_finish(a, a.k, b, slice, nb, tau, nb, (double)best.t, 0.0,
                        best.c.exact() - (double)nb * tau);
        } else {
            const double K = (double)(nb - best.m), c = best.c.exact(), h = best.h.exact();
            double theta = fmax(pdiv(tau * h, 2.0 * K), (double)best.lo);
            theta = fmin(theta, (double)best.hi);
            const double val = c - best.m * tau + K * theta * theta + K * tau - tau * theta * h;
            sure_finish(a, a.k, b, slice, nb, tau, best.m, theta, h, val);
        }
    }
}

// Subbands of up to PRUNE_SMALL_BAND magnitudes (the coarse ones, b = 0 ..
// n_small - 1 in packed order) go four to a CTA, the next ones up to
// PRUNE_MED_BAND (b = n_small .. n_small + n_med - 1) two to a CTA, the
// larger ones one to a CTA: CTAs per slice.
__host__ __device__ inline int prune_n_small(const int* off, int B) {
    int n = 0;
    while (n < B && off[n + 1] - off[n] <= PRUNE_SMALL_BAND) ++n;
    return n;
}
__host__ __device__ inline int prune_n_med(const int* off, int B, int n_small) {
    int n = n_small;
    while (n < B && off[n + 1] - off[n] <= PRUNE_MED_BAND) ++n;
    return n - n_small;
}
__host__ __device__ inline int prune_ctas(const int* off, int B) {
    const int ns = prune_n_small(off, B), nm = prune_n_med(off, B, ns);
    constexpr int per_med = PRUNE_THREADS / PRUNE_MED;
    return (B - ns - nm) + (nm + per_med - 1) / per_med + (ns + PRUNE_GROUPS - 1) / PRUNE_GROUPS;
}

}  // namespace vdamp

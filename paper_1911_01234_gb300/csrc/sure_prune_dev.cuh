// Exact SURE threshold of one subband without sorting it (Sec. 3, the
// unnumbered equation after Algorithm 1; alpha of line 7): the batched form
// of the threshold step, one CTA of PRUNE_THREADS threads per subband.
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
//      order instead), prefix sums over buckets (FP32 within a thread's run of
//      buckets, FP64 across threads);
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
//      the others (a few hundred of N_b) are gathered in a second pass over
//      r_k, ranked within their bucket, and every interval piece inside these
//      buckets is evaluated as in the full search.
// A piece whose vertex lies beyond the bucket's upper edge is skipped: its
// minimum over the interval lies in a higher bucket, where it is either
// evaluated or bounded above UB.  Candidates are compared in FP32 (ties to
// the smaller theta, then the smaller m), the winner recomputed in FP64.
//
// A subband whose candidates exceed the table (PRUNE_TABLE non-empty
// buckets, PRUNE_CAP keys, PRUNE_BUCKET_MAX keys in one bucket; heavy ties
// or degenerate data) is appended to a device list, and sure_fallback_kernel
// solves it with the one-CTA full sort and search.
#pragma once

#include "sure_dev.cuh"

namespace vdamp {

#define PRUNE_THREADS 512
#define PRUNE_MAX_LPO 8          // at most 4096 buckets (256 per octave)
#define PRUNE_TABLE 128          // non-empty candidate buckets of one subband
#define PRUNE_CAP 1024           // candidate magnitudes of one subband
#define PRUNE_BUCKET_MAX 256     // magnitudes of one candidate bucket

// log2 of the buckets per octave: about two buckets per magnitude, 16 .. 256.
__host__ __device__ inline int prune_lpo(int nb) {
    int l = 4;
    while (l < PRUNE_MAX_LPO && (16 << l) < 2 * nb) ++l;
    return l;
}

// Dynamic shared memory: three per-bucket words (count, sum of quantised a^2
// offsets, sum of quantised 1/a offsets; later the packed local prefixes),
// the candidate-bucket bits, and two candidate key buffers.
inline size_t prune_smem_bytes(int max_band) {
    const size_t nbk = (size_t)16 << prune_lpo(max_band);
    return 3 * nbk * sizeof(unsigned) + (nbk / 32) * sizeof(unsigned) +
           2 * (size_t)PRUNE_CAP * sizeof(float);
}

struct PruneEntry {   // one non-empty candidate bucket
    double c_lt;      // sum of a^2 over the magnitudes below the bucket
    double h_gt;      // sum of 1/a over the magnitudes above the bucket
    float lo, hi;     // the bucket's value range [lo, hi)
    int m_lt;         // magnitudes below the bucket (exact zeros included)
    int n;            // magnitudes in the bucket
    int start;        // first slot in the candidate buffers
    int fill;         // gather counter
};

// The best candidate a thread has seen, with what the FP64 recomputation needs.
struct PruneBest {
    float v, t;       // FP32 SURE value and theta
    int m;            // magnitudes at or below theta (nb: theta = max a, the flat top)
    double c, h;      // FP64 sum of a^2 below and of 1/a above theta
    float lo, hi;     // the piece: theta in [lo, hi) (lo = hi = theta on the flat top)
};

__device__ __forceinline__ bool prune_better(float v, float t, int m, const PruneBest& b) {
    return v < b.v || (v == b.v && (t < b.t || (t == b.t && m < b.m)));
}

__device__ __forceinline__ void prune_take(PruneBest& b, float v, float t, int m, double c,
                                           double h, float lo, float hi) {
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
// and h (1/a above), theta in [lo, hi): the clamped vertex, if inside.
__device__ __forceinline__ void prune_piece(PruneBest& best, int nb, float tf, int m, double c,
                                            double h, float lo, float hi) {
    const int K = nb - m;
    if (K <= 0) return;
    const float hf = (float)h, cf = (float)c, Kf = (float)K;
    float t = tf * hf * __frcp_rn(2.0f * Kf);
    t = fmaxf(t, lo);
    if (!(t < hi)) return;
    const float v = cf - (float)m * tf + Kf * t * t + Kf * tf - tf * t * hf;
    prune_take(best, v, t, m, c, h, lo, hi);
}

// Block-wide (PRUNE_THREADS) exclusive scan of (int, float, float) per thread:
// FP32 within each warp, FP64 across warps.  Returns the exclusive prefixes
// and, through tot_*, the block totals.
__device__ __forceinline__ void prune_scan3(int vi, float vc, float vh, int& ei, double& ec,
                                            double& eh, int& tot_i, double& tot_c,
                                            double& tot_h) {
    constexpr int NW = PRUNE_THREADS / 32;
    __shared__ int s_i[NW + 1];
    __shared__ double s_c[NW + 1], s_h[NW + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int ii = vi;
    float ic = vc, ih = vh;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ti = __shfl_up_sync(0xffffffffu, ii, o);
        const float tc = __shfl_up_sync(0xffffffffu, ic, o);
        const float th = __shfl_up_sync(0xffffffffu, ih, o);
        if (lane >= o) {
            ii += ti;
            ic += tc;
            ih += th;
        }
    }
    if (lane == 31) {
        s_i[warp] = ii;
        s_c[warp] = ic;
        s_h[warp] = ih;
    }
    __syncthreads();
    if (threadIdx.x == 0) {   // FP64 over the warps, in warp order
        int ai = 0;
        double ac = 0.0, ah = 0.0;
        for (int w = 0; w < NW; ++w) {
            const int xi = s_i[w];
            const double xc = s_c[w], xh = s_h[w];
            s_i[w] = ai;
            s_c[w] = ac;
            s_h[w] = ah;
            ai += xi;
            ac += xc;
            ah += xh;
        }
        s_i[NW] = ai;
        s_c[NW] = ac;
        s_h[NW] = ah;
    }
    __syncthreads();
    int xi = __shfl_up_sync(0xffffffffu, ii, 1);
    float xc = __shfl_up_sync(0xffffffffu, ic, 1), xh = __shfl_up_sync(0xffffffffu, ih, 1);
    if (lane == 0) {
        xi = 0;
        xc = 0.f;
        xh = 0.f;
    }
    ei = s_i[warp] + xi;
    ec = s_c[warp] + (double)xc;
    eh = s_h[warp] + (double)xh;
    tot_i = s_i[NW];
    tot_c = s_c[NW];
    tot_h = s_h[NW];
    __syncthreads();   // the scratch is reused by the next scan
}

// Block-wide minimum of a float (PRUNE_THREADS threads).
__device__ __forceinline__ float prune_min(float v) {
    constexpr int NW = PRUNE_THREADS / 32;
    __shared__ float s_m[NW];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = v;
    __syncthreads();
    float m = s_m[0];
    for (int w = 1; w < NW; ++w) m = fminf(m, s_m[w]);
    __syncthreads();
    return m;
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
// ever appended, [3 ..] slice B + b).  Called by all
// PRUNE_THREADS threads of a CTA; dyn: prune_smem_bytes(largest subband).
static __device__ void sure_prune_subband(const SureArgs& a, int b, int slice, unsigned* dyn) {
    constexpr int NT = PRUNE_THREADS, NW = NT / 32;
    __shared__ double s_tau, s_s20, s_h0;
    __shared__ unsigned s_max;
    __shared__ int s_zero, s_bad, s_win;
    __shared__ float s_w2[NW], s_wh[NW], s_bv[NW], s_bt[NW];
    __shared__ int s_bm[NW], s_bw[NW];
    __shared__ PruneEntry s_tab[PRUNE_TABLE];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int off = a.off[b], nb = a.off[b + 1] - off;
    const float2* r = a.r + (size_t)slice * a.N + off;
    const int lpo = prune_lpo(nb), nbk = 16 << lpo, shift = 23 - lpo;
    unsigned* X = dyn;        // count, then (local prefix of counts << 16 | count), then entry
    unsigned* Y = X + nbk;    // sum of quantised a^2 offsets, then local prefix of a^2 (FP32)
    unsigned* Z = Y + nbk;    // sum of quantised 1/a offsets, then local suffix of 1/a (FP32)
    unsigned* F = Z + nbk;    // candidate bits
    float* candA = reinterpret_cast<float*>(F + nbk / 32);   // gathered (bucket order)
    float* candB = candA + PRUNE_CAP;                         // sorted

    if (warp == 0) {   // tau: fixed-order FP64 sum of the column partials
        double t = 0.0;
        for (int p = lane; p < a.nparts; p += 32)
            t += a.tau_part[((size_t)slice * a.nparts + p) * a.B + b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) s_tau = t;
    }
    for (int i = tid; i < 3 * nbk + nbk / 32; i += NT) X[i] = 0u;
    if (tid == 0) {
        s_max = 0u;
        s_zero = 0;
        s_bad = 0;
    }
    __syncthreads();
    const double tau = s_tau;
    if (!(tau > 0.0) || !isfinite(tau)) {   // no effective noise, or a numeric failure
        if (tid == 0) sure_finish(a, a.k, b, slice, nb, tau, -1, 0.0, 0.0, 0.0);
        return;
    }
    const float tf = (float)tau;

    // ---- pass 1 over r_k: the largest magnitude (as bits) and the exact zeros
    unsigned mx = 0u;
    int nz = 0;
    for (int i = tid; i < nb; i += NT) {
        const unsigned u = __float_as_uint(cabs_f(r[i]));
        mx = max(mx, u);
        nz += u == 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        nz += __shfl_xor_sync(0xffffffffu, nz, o);
    }
    if (lane == 0) {
        atomicMax(&s_max, mx);
        atomicAdd(&s_zero, nz);
    }
    __syncthreads();
    const unsigned M = s_max;
    const int z = s_zero;
    if (M >= 0x7f800000u || M == 0u) {
        // non-finite magnitudes (recorded as a numeric failure), or all zero: theta = max a = 0
        if (tid == 0)
            sure_finish(a, a.k, b, slice, nb, tau, M == 0u ? nb : -1, 0.0, 0.0,
                        -(double)nb * tau);
        return;
    }
    const unsigned span = (unsigned)nbk << shift;
    const unsigned lo_bits = M + 1u > span ? M + 1u - span : 0u;

    // ---- pass 2: counts and quantised sums per bucket (bucket 0 summed per thread)
    float s20 = 0.f, h0 = 0.f;
    for (int i = tid; i < nb; i += NT) {
        const float x = cabs_f(r[i]);
        const unsigned u = __float_as_uint(x);
        if (u == 0u) continue;
        const int q = u < lo_bits ? 0 : (int)((u - lo_bits) >> shift);
        atomicAdd(&X[q], 1u);
        if (q == 0) {
            s20 += x * x;
            h0 += __frcp_rn(x);
            continue;
        }
        const float lo = prune_lo(lo_bits, shift, q), hi = prune_hi(lo_bits, shift, q);
        const float w = __frcp_rn(hi - lo);
        const float r2 = (x - lo) * w * ((x + lo) * __frcp_rn(hi + lo));   // (a^2 - lo^2) / (hi^2 - lo^2)
        const float rh = (hi - x) * w * (lo * __frcp_rn(x));               // (1/a - 1/hi) / (1/lo - 1/hi)
        atomicAdd(&Y[q], min(__float2uint_rz(r2 * 65536.f), 65535u));
        atomicAdd(&Z[q], min(__float2uint_rz(rh * 65536.f), 65535u));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s20 += __shfl_xor_sync(0xffffffffu, s20, o);
        h0 += __shfl_xor_sync(0xffffffffu, h0, o);
    }
    if (lane == 0) {
        s_w2[warp] = s20;
        s_wh[warp] = h0;
    }
    __syncthreads();
    if (tid == 0) {
        double t2 = 0.0, th = 0.0;
        for (int w = 0; w < NW; ++w) {
            t2 += s_w2[w];
            th += s_wh[w];
        }
        s_s20 = t2;
        s_h0 = th;
    }
    __syncthreads();

    // ---- prefix sums over buckets: each thread owns a run of consecutive buckets
    const int per = nbk >= NT ? nbk / NT : 1;
    const int j0 = min(tid * per, nbk), j1 = min(j0 + per, nbk);
    auto sums = [&](int j, int n, float& s2, float& hs) {
        if (j == 0) {
            s2 = (float)s_s20;
            hs = (float)s_h0;
        } else {
            prune_bucket_sums(lo_bits, shift, j, n, Y[j], Z[j], s2, hs);
        }
    };
    int tm = 0;
    float tc = 0.f, th = 0.f;
    for (int j = j0; j < j1; ++j) {
        float s2, hs;
        const int n = (int)X[j];
        sums(j, n, s2, hs);
        tm += n;
        tc += s2;
        th += hs;
    }
    int em, tot_m;
    double ec, eh, c_all, tot_h;
    prune_scan3(tm, tc, th, em, ec, eh, tot_m, c_all, tot_h);
    const int mb = z + em;                       // magnitudes below this thread's buckets
    const double cb = ec;                        // their sum of a^2
    const double hb = tot_h - (eh + (double)th); // sum of 1/a above this thread's buckets
    // local prefixes: X = (count below in the run << 16 | count), Y = a^2 below in the run
    {
        int lm = 0;
        float lc = 0.f;
        for (int j = j0; j < j1; ++j) {
            float s2, hs;
            const int n = (int)X[j];
            sums(j, n, s2, hs);
            X[j] = ((unsigned)lm << 16) | (unsigned)n;
            Y[j] = __float_as_uint(lc);
            lm += n;
            lc += s2;
        }
    }
    // local suffixes of 1/a (Z), and the attained SURE just below each bucket's lower edge
    float umin = (float)(c_all - (double)nb * tau);   // theta >= max a
    {
        float lh = 0.f;
        for (int j = j1 - 1; j >= j0; --j) {
            const unsigned xw = X[j];
            const int n = (int)(xw & 0xffffu), m_lt = mb + (int)(xw >> 16);
            float hs = (float)s_h0;
            if (j > 0) {
                float s2_unused;
                prune_bucket_sums(lo_bits, shift, j, n, 0u, Z[j], s2_unused, hs);
            }
            Z[j] = __float_as_uint(lh);
            const float c_lt = (float)(cb + (double)__uint_as_float(Y[j]));
            const float h_ge = (float)(hb + (double)lh) + hs;
            const float t = j == 0 ? 0.f : __uint_as_float(lo_bits + ((unsigned)j << shift) - 1u);
            const float kge = (float)(nb - m_lt);
            umin = fminf(umin, c_lt - tf * (float)m_lt + kge * (t * t + tf) - tf * t * h_ge);
            lh += hs;
        }
    }
    const float ub = prune_min(umin);
    const float delta = 1e-5f * (float)(c_all + (double)nb * tau);

    // ---- lower bounds: empty candidate buckets are evaluated now, the others marked
    PruneBest best;
    best.v = INFINITY;
    best.t = INFINITY;
    best.m = 0x7fffffff;
    best.c = best.h = 0.0;
    best.lo = best.hi = 0.f;
    int my_e = 0, my_k = 0;
    for (int j = j0; j < j1; ++j) {
        const unsigned xw = X[j];
        const int n = (int)(xw & 0xffffu), m_lt = mb + (int)(xw >> 16);
        const double c_lt = cb + (double)__uint_as_float(Y[j]);
        const double h_gt = hb + (double)__uint_as_float(Z[j]);
        const float lo = prune_lo(lo_bits, shift, j), hi = prune_hi(lo_bits, shift, j);
        const int K = nb - m_lt - n;
        const float hf = (float)h_gt;
        float t = K > 0 ? tf * hf * __frcp_rn(2.f * (float)K) : lo;
        t = fminf(fmaxf(t, lo), hi);
        const float lb = (float)c_lt - tf * (float)m_lt + (float)n * (lo * lo - tf) +
                         (float)K * (t * t + tf) - tf * t * hf;
        if (!(lb <= ub + delta)) continue;
        if (n == 0) {
            prune_piece(best, nb, tf, m_lt, c_lt, h_gt, lo, hi);
        } else {
            atomicOr(&F[j >> 5], 1u << (j & 31));
            ++my_e;
            my_k += n;
            if (n > PRUNE_BUCKET_MAX) s_bad = 1;
        }
    }
    int e0, tot_e;
    double k0d, unused0, tot_kd, unused1;
    prune_scan3(my_e, (float)my_k, 0.f, e0, k0d, unused0, tot_e, tot_kd, unused1);
    const int tot_k = (int)tot_kd;
    if (tot_e > PRUNE_TABLE || tot_k > PRUNE_CAP || s_bad) {
        if (tid == 0) {
            const int idx = atomicAdd(&a.fallback[0], 1);
            a.fallback[3 + idx] = slice * a.B + b;
            atomicAdd(&a.fallback[2], 1);   // subbands left to the full sort, ever
        }
        return;
    }

    // ---- the table of non-empty candidate buckets; X[j] becomes j's entry (or none)
    {
        int e = e0, kpos = (int)k0d;
        for (int j = j0; j < j1; ++j) {
            const unsigned xw = X[j];
            const int n = (int)(xw & 0xffffu);
            if (n > 0 && ((F[j >> 5] >> (j & 31)) & 1u)) {
                PruneEntry& E = s_tab[e];
                E.c_lt = cb + (double)__uint_as_float(Y[j]);
                E.h_gt = hb + (double)__uint_as_float(Z[j]);
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
    __syncthreads();
    // ---- pass 3 over r_k: gather the candidates' magnitudes, grouped by bucket
    for (int i = tid; i < nb; i += NT) {
        const float x = cabs_f(r[i]);
        const unsigned u = __float_as_uint(x);
        if (u == 0u) continue;
        const int q = u < lo_bits ? 0 : (int)((u - lo_bits) >> shift);
        const unsigned e = X[q];
        if (e != 0xffffffffu) candA[s_tab[e].start + atomicAdd(&s_tab[e].fill, 1)] = x;
    }
    __syncthreads();
    auto entry_of = [&](int p) {   // the entry whose slots hold position p
        int l = 0, h = tot_e - 1;
        while (l < h) {
            const int mid = (l + h + 1) >> 1;
            if (s_tab[mid].start <= p) l = mid;
            else h = mid - 1;
        }
        return l;
    };
    // rank within the bucket (ties by gather slot): the sorted order, whatever the gather order
    for (int p = tid; p < tot_k; p += NT) {
        const PruneEntry& E = s_tab[entry_of(p)];
        const float x = candA[p];
        int rk = 0;
        for (int k = E.start; k < E.start + E.n; ++k) {
            const float y = candA[k];
            rk += (y < x) || (y == x && k < p);
        }
        candB[E.start + rk] = x;
    }
    __syncthreads();
    // ---- every piece inside the candidate buckets: the interval after each magnitude ...
    for (int p = tid; p < tot_k; p += NT) {
        const PruneEntry& E = s_tab[entry_of(p)];
        const int k = p - E.start;
        float cs = 0.f, hs = 0.f;   // a^2 up to and including k, 1/a after k (bucket order)
        for (int i = 0; i < E.n; ++i) {
            const float y = candB[E.start + i];
            if (i <= k) cs += y * y;
            else hs += __frcp_rn(y);
        }
        const float bk = candB[p];
        const int m = E.m_lt + k + 1;
        const double c = E.c_lt + (double)cs;
        if (m == nb) {   // theta >= max a: SURE is constant, theta = max a
            prune_take(best, (float)c - (float)nb * tf, bk, nb, c, 0.0, bk, bk);
        } else {
            const float nxt = k + 1 < E.n ? candB[p + 1] : E.hi;
            prune_piece(best, nb, tf, m, c, E.h_gt + (double)hs, bk, nxt);
        }
    }
    // ... and the piece below each candidate bucket's first magnitude
    for (int e = tid; e < tot_e; e += NT) {
        const PruneEntry& E = s_tab[e];
        float hs = 0.f;
        for (int i = 0; i < E.n; ++i) hs += __frcp_rn(candB[E.start + i]);
        prune_piece(best, nb, tf, E.m_lt, E.c_lt, E.h_gt + (double)hs, E.lo, candB[E.start]);
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
            s_bv[warp] = v;
            s_bt[warp] = t;
            s_bm[warp] = m;
            s_bw[warp] = w;
        }
        __syncthreads();
        if (tid == 0) {
            float bv = s_bv[0], bt = s_bt[0];
            int bm = s_bm[0], bw = s_bw[0];
            for (int q = 1; q < NW; ++q) {
                const float v2 = s_bv[q], t2 = s_bt[q];
                const int m2 = s_bm[q], w2 = s_bw[q];
                if (v2 < bv || (v2 == bv && (t2 < bt || (t2 == bt && (m2 < bm || (m2 == bm && w2 < bw)))))) {
                    bv = v2;
                    bt = t2;
                    bm = m2;
                    bw = w2;
                }
            }
            s_win = bw;
        }
        __syncthreads();
    }
    // ---- the winner in FP64 (theta, alpha and the line-8 constants by sure_finish)
    if (tid == s_win) {
        if (!(best.v < INFINITY)) {   // nothing found: recorded as a numeric failure
            sure_finish(a, a.k, b, slice, nb, tau, -1, 0.0, 0.0, 0.0);
        } else if (best.m == nb) {
            sure_finish(a, a.k, b, slice, nb, tau, nb, (double)best.t, 0.0,
                        best.c - (double)nb * tau);
        } else {
            const double K = (double)(nb - best.m);
            double theta = fmax(tau * best.h / (2.0 * K), (double)best.lo);
            theta = fmin(theta, (double)best.hi);
            const double val = best.c - best.m * tau + K * theta * theta + K * tau -
                               tau * theta * best.h;
            sure_finish(a, a.k, b, slice, nb, tau, best.m, theta, best.h, val);
        }
    }
}

}  // namespace vdamp

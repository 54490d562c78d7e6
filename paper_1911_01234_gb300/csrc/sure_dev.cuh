// Device code of the SURE-tuned complex soft threshold per subband (Sec. 3,
// the unnumbered equation after Algorithm 1), the subband-mean derivative
// alpha (Algorithm 1 line 7) and the final sum of tau (line 5).
//
// For magnitudes a sorted ascending, on the interval [a_(m), a_(m+1)) the
// complex colored SURE of soft(., theta) is the convex quadratic
//   C_m - m tau + K theta^2 + K tau - tau theta H_m,   K = N_b - m,
// C_m the sum of a^2 below, H_m the sum of 1/a above.  Its minimiser
// tau H_m / (2K) is clamped to the interval; a minimiser that lands on the
// right end is never the global one (SURE drops by tau there).  theta >= max a
// gives the constant C_N - N_b tau.  The global minimum over all intervals is
// the threshold; ties go to the smaller theta.  alpha = (K - theta H_m / 2) / N_b.
//
// Two steps, each run by one 1024-thread CTA per work item:
//   sure_sort_part   : part q of subband b sorts its share of the magnitudes
//                      and writes them to their final places in `sorted`;
//   sure_search_band : reads the sorted magnitudes of subband b and finds the
//                      exact minimiser.
// Sorting: for a >= 0 the IEEE-754 bit pattern is an increasing integer
// function of a, so buckets made of consecutive ranges of bit patterns
// ((bits - lo) >> SORT_SHIFT, 1024 buckets per octave over the 16 octaves below
// the maximum; smaller magnitudes share bucket 0) are exactly ordered.  Each
// bucket belongs to the part in which its first position falls, and is
// sorted in registers by a bitonic network (up to 32 keys) or in shared
// memory.  A bucket above SORT_MAX_BUCKET keys (ties, or a degenerate subband)
// sends the whole subband to a bitonic sort done by part 0.
//
// Precision: magnitudes, keys and per-thread partial sums are FP32; the
// cross-warp scans of C and H, tau, theta and alpha of the chosen interval
// are FP64.
#pragma once

#include <math.h>

#include "vdamp_internal.cuh"

namespace vdamp {

#define SORT_BUCKETS 16384
#define SORT_SHIFT 13
#define SORT_MAX_BUCKET 96
#define SORT_MAX_PER_THREAD 32            // largest subband = 32 x 1024 keys
#define SORT_HIST_WORDS (SORT_BUCKETS + SORT_BUCKETS / 32)
#define HIX(q) ((q) + ((q) >> 5))          // padding against bank conflicts in the scan
#define SURE_THREADS 1024
#define SURE_MAX_PARTS 8
#define SURE_KEYS_PER_PART 2048

__host__ __device__ inline int sure_parts(int nb) {
    int q = (nb + SURE_KEYS_PER_PART - 1) / SURE_KEYS_PER_PART;
    return q < 1 ? 1 : (q > SURE_MAX_PARTS ? SURE_MAX_PARTS : q);
}

// Shared memory for either step: keys padded to a power of two, then the
// bucket counters.
inline size_t sure_smem_bytes(int max_band) {
    int np = 2;
    while (np < max_band) np <<= 1;
    return (size_t)np * sizeof(float) + SORT_HIST_WORDS * sizeof(int);
}

__device__ __forceinline__ void record_numeric(int* status, int k) {
    atomicExch(&status[0], 4 /* VDAMP_ENUMERIC */);
    atomicMin(&status[1], k);
}

// Bitonic sorting network on N registers, ascending (fully unrolled).
template <int N>
__device__ __forceinline__ void sort_regs(float* v) {
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const float x = v[i], y = v[l];
                    const bool sw = up ? (x > y) : (x < y);
                    v[i] = sw ? y : x;
                    v[l] = sw ? x : y;
                }
            }
        }
    }
}

// Bitonic sort of keys[0, np) (np a power of two) by the whole CTA.
__device__ __forceinline__ void block_bitonic(float* keys, int np) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int k = 2; k <= np; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < (np >> 1); i += nthr) {
                const int lo = 2 * i - (i & (j - 1));
                const int hi = lo + j;
                const bool up = (lo & k) == 0;
                const float x = keys[lo], y = keys[hi];
                if ((x > y) == up) {
                    keys[lo] = y;
                    keys[hi] = x;
                }
            }
            __syncthreads();
        }
    }
}

// Part `part` of subband b of slice `slice`: sort and write its share of |r|.
// Called by all threads of a CTA of SURE_THREADS threads; `keys` is dynamic
// shared memory of sure_smem_bytes(max band) bytes.
template <int EMAX>
__device__ __forceinline__ void sure_sort_part_t(const SureArgs& a, const float2* rk, int part,
                                                 int b, int slice, float* keys) {
    __shared__ unsigned s_max_bits;
    __shared__ int s_big;
    __shared__ int wsum[32];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    const int off = a.off[b], nb = a.off[b + 1] - off;
    const int Q = sure_parts(nb);
    if (part >= Q) return;  // uniform over the CTA
    int np = 2;
    while (np < nb) np <<= 1;
    int* hist = reinterpret_cast<int*>(keys + np);
    float* out = a.sorted + (size_t)slice * a.N + off;

    if (tid == 0) {
        s_max_bits = 0u;
        s_big = 0;
    }
    const float2* r = rk + (size_t)slice * a.N + off;
    float kr[EMAX];
    unsigned mx = 0u;
#pragma unroll
    for (int e = 0; e < EMAX; ++e) {
        const int i = tid + e * nthr;
        kr[e] = i < nb ? cabs_f(r[i]) : 0.f;
        mx = max(mx, __float_as_uint(kr[e]));
    }
    for (int i = tid; i < SORT_HIST_WORDS; i += nthr) hist[i] = 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if (lane == 0) atomicMax(&s_max_bits, mx);
    __syncthreads();
    const unsigned span = (unsigned)SORT_BUCKETS << SORT_SHIFT;
    const unsigned lo_bits = s_max_bits + 1u > span ? s_max_bits + 1u - span : 0u;
    auto bucket = [&](float x) -> int {
        const unsigned u = __float_as_uint(x);
        return u < lo_bits ? 0 : (int)((u - lo_bits) >> SORT_SHIFT);
    };
#pragma unroll
    for (int e = 0; e < EMAX; ++e)
        if (tid + e * nthr < nb) atomicAdd(&hist[HIX(bucket(kr[e]))], 1);
    __syncthreads();
    {   // exclusive scan of the counts; each thread owns SORT_BUCKETS / nthr consecutive buckets
        const int per = SORT_BUCKETS / nthr;
        const int b0 = tid * per;
        int loc = 0, big = 0;
        for (int q = 0; q < per; ++q) {
            const int c = hist[HIX(b0 + q)];
            big = max(big, c);
            loc += c;
        }
        if (big > SORT_MAX_BUCKET) s_big = 1;
        int inc = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            int v = lane < nw ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += t;
            }
            wsum[lane] = v;
        }
        __syncthreads();
        int run = inc - loc + (warp > 0 ? wsum[warp - 1] : 0);
        for (int q = 0; q < per; ++q) {
            const int c = hist[HIX(b0 + q)];
            hist[HIX(b0 + q)] = run;
            run += c;
        }
    }
    __syncthreads();
    if (s_big) {
        // degenerate subband: part 0 sorts everything
        if (part != 0) return;
#pragma unroll
        for (int e = 0; e < EMAX; ++e)
            if (tid + e * nthr < nb) keys[tid + e * nthr] = kr[e];
        for (int i = nb + tid; i < np; i += nthr) keys[i] = INFINITY;
        __syncthreads();
        block_bitonic(keys, np);
        for (int i = tid; i < nb; i += nthr) out[i] = keys[i];
        return;
    }
#pragma unroll
    for (int e = 0; e < EMAX; ++e)
        if (tid + e * nthr < nb) keys[atomicAdd(&hist[HIX(bucket(kr[e]))], 1)] = kr[e];
    __syncthreads();
    // hist[q] now holds the end of bucket q; the bucket belongs to the part in
    // which its first position falls.
    for (int q = tid; q < SORT_BUCKETS; q += nthr) {
        const int s0 = q > 0 ? hist[HIX(q - 1)] : 0, s1 = hist[HIX(q)];
        const int n = s1 - s0;
        if (n <= 0 || (int)(((long long)s0 * Q) / nb) != part) continue;
        if (n <= 16) {
            float v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = i < n ? keys[s0 + i] : INFINITY;
            if (n > 1) sort_regs<16>(v);
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (i < n) out[s0 + i] = v[i];
        } else if (n <= 32) {
            float v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = i < n ? keys[s0 + i] : INFINITY;
            sort_regs<32>(v);
#pragma unroll
            for (int i = 0; i < 32; ++i)
                if (i < n) out[s0 + i] = v[i];
        } else {
            for (int i = s0 + 1; i < s1; ++i) {
                const float x = keys[i];
                int j = i - 1;
                while (j >= s0 && keys[j] > x) {
                    keys[j + 1] = keys[j];
                    --j;
                }
                keys[j + 1] = x;
            }
            for (int i = s0; i < s1; ++i) out[i] = keys[i];
        }
    }
}

static __device__ void sure_sort_part(const SureArgs& a, const float2* rk, int part, int b,
                                      int slice, float* keys) {
    const int nb = a.off[b + 1] - a.off[b];
    if (nb <= 16 * SURE_THREADS)
        sure_sort_part_t<16>(a, rk, part, b, slice, keys);
    else
        sure_sort_part_t<SORT_MAX_PER_THREAD>(a, rk, part, b, slice, keys);
}

// Subband b of slice `slice`: tau, the exact SURE minimiser theta and alpha.
static __device__ void sure_search_band(const SureArgs& a, int k, int b, int slice, float* keys) {
    __shared__ double s_tau;
    __shared__ float wc[32], wh[32];
    __shared__ double woc[33], woh[33];
    __shared__ float bq[32], bt[32];
    __shared__ int bm[32];
    __shared__ int s_win_m;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    const int off = a.off[b], nb = a.off[b + 1] - off;

    if (warp == 0) {   // tau: fixed-order sum of the column partials, lane by lane then a tree
        double t = 0.0;
        for (int p = lane; p < a.nparts; p += 32)
            t += a.tau_part[((size_t)slice * a.nparts + p) * a.B + b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) s_tau = t;
    }
    const float* srt = a.sorted + (size_t)slice * a.N + off;
    batched_for<16, float>(tid, nb, nthr, [&](int i) { return srt[i]; },
                           [&](int i, float v) { keys[i] = v; });
    __syncthreads();
    const double tau = s_tau;
    const size_t orow = ((size_t)slice * a.iters + k) * a.B + b;
    if (!(tau > 0.0) || !isfinite(tau)) {
        // No effective noise (p = 1 and sigma = 0): keep r, no Onsager term.
        if (tid == 0) {
            a.tau_out[orow] = tau;
            a.thr_out[orow] = 0.0;
            a.alpha_out[orow] = 0.0;
            a.coef[slice * a.B + b] = make_float4(0.f, 0.f, 1.f, 0.f);
            if (!isfinite(tau)) record_numeric(a.status, k);
        }
        return;
    }

    // ---- prefix sums of a^2 (from below) and suffix sums of 1/a (from above)
    const int E = (nb + nthr - 1) / nthr;
    const int m0 = min(tid * E, nb), m1 = min(m0 + E, nb);
    float cs = 0.f, hs = 0.f;
    for (int i = m0; i < m1; ++i) {
        const float x = keys[i];
        cs += x * x;
        hs += x > 0.f ? __frcp_rn(x) : 0.f;
    }
    float ic = cs, ih = hs;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float t = __shfl_up_sync(0xffffffffu, ic, o);
        if (lane >= o) ic += t;
        const float u = __shfl_down_sync(0xffffffffu, ih, o);
        if (lane + o < 32) ih += u;
    }
    float ec = __shfl_up_sync(0xffffffffu, ic, 1);
    float eh = __shfl_down_sync(0xffffffffu, ih, 1);
    if (lane == 0) ec = 0.f;
    if (lane == 31) eh = 0.f;
    if (lane == 31) wc[warp] = ic;
    if (lane == 0) wh[warp] = ih;
    __syncthreads();
    if (warp == 0) {   // FP64 scans of the warp totals: C from below, H from above
        double c = lane < nw ? (double)wc[lane] : 0.0;
        double h = lane < nw ? (double)wh[nw - 1 - lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double tc = __shfl_up_sync(0xffffffffu, c, o);
            const double th = __shfl_up_sync(0xffffffffu, h, o);
            if (lane >= o) {
                c += tc;
                h += th;
            }
        }
        // inclusive -> exclusive
        const double ce = __shfl_up_sync(0xffffffffu, c, 1);
        const double he = __shfl_up_sync(0xffffffffu, h, 1);
        if (lane < nw) {
            woc[lane] = lane ? ce : 0.0;
            woh[nw - 1 - lane] = lane ? he : 0.0;
        }
        if (lane == nw - 1) {
            woc[nw] = c;
            woh[nw] = h;
        }
    }
    __syncthreads();
    const double c_base = woc[warp] + (double)ec;   // sum of a^2 over indices < m0
    const double h_after = woh[warp] + (double)eh;  // sum of 1/a over indices >= m1
    const double c_total = woc[nw];

    // ---- best candidate of this thread's intervals (FP32)
    const float tf = (float)tau;
    const float cb = (float)c_base, ha = (float)h_after;
    float best_q = INFINITY, best_t = INFINITY;
    int best_m = -1;
    float csuf = 0.f, hsuf = 0.f;
    for (int m = m1 - 1; m >= m0; --m) {
        const float x = keys[m];
        csuf += x * x;
        hsuf += x > 0.f ? __frcp_rn(x) : 0.f;
        const float cm = cb + (cs - csuf);
        const float hm = ha + hsuf;
        const float K = (float)(nb - m);
        const float lo = m > 0 ? keys[m - 1] : 0.f;
        float th = tf * hm * __frcp_rn(2.0f * K);
        th = fmaxf(th, lo);
        if (th < x) {
            const float q = cm - (float)m * tf + K * th * th + K * tf - tf * th * hm;
            if (q < best_q || (q == best_q && th < best_t)) {
                best_q = q;
                best_t = th;
                best_m = m;
            }
        }
    }
    if (m1 == nb && m0 < m1) {  // theta >= max a: everything thresholded
        const float q = (float)(c_total - (double)nb * tau);
        const float th = keys[nb - 1];
        if (q < best_q || (q == best_q && th < best_t)) {
            best_q = q;
            best_t = th;
            best_m = nb;
        }
    }

    // ---- block argmin (q, then theta)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float q2 = __shfl_xor_sync(0xffffffffu, best_q, o);
        const float t2 = __shfl_xor_sync(0xffffffffu, best_t, o);
        const int m2 = __shfl_xor_sync(0xffffffffu, best_m, o);
        if (q2 < best_q || (q2 == best_q && (t2 < best_t || (t2 == best_t && m2 < best_m)))) {
            best_q = q2;
            best_t = t2;
            best_m = m2;
        }
    }
    if (lane == 0) {
        bq[warp] = best_q;
        bt[warp] = best_t;
        bm[warp] = best_m;
    }
    __syncthreads();
    if (tid == 0) {
        float q = bq[0], t = bt[0];
        int m = bm[0];
        for (int w = 1; w < nw; ++w) {
            if (bq[w] < q || (bq[w] == q && (bt[w] < t || (bt[w] == t && bm[w] < m)))) {
                q = bq[w];
                t = bt[w];
                m = bm[w];
            }
        }
        s_win_m = m;
    }
    __syncthreads();

    // ---- theta and alpha of the chosen interval, FP64, by the thread that owns it
    const int wm = s_win_m;
    const bool owner = (wm == nb) ? (m1 == nb && m0 < m1) : (wm >= m0 && wm < m1);
    if (owner) {
        double theta, alpha;
        if (wm == nb) {
            theta = (double)keys[nb - 1];
            alpha = 0.0;
        } else {
            float hl = 0.f;   // same FP32 reciprocals as the candidate pass
            for (int i = m1 - 1; i >= wm; --i) {
                const float x = keys[i];
                hl += x > 0.f ? __frcp_rn(x) : 0.f;
            }
            const double hm = h_after + (double)hl;
            const double K = (double)(nb - wm);
            const double lo = wm > 0 ? (double)keys[wm - 1] : 0.0;
            theta = fmax(tau * hm / (2.0 * K), lo);
            theta = fmin(theta, (double)keys[wm]);
            alpha = (K - 0.5 * theta * hm) / (double)nb;
        }
        a.tau_out[orow] = tau;
        a.thr_out[orow] = theta;
        a.alpha_out[orow] = alpha;
        const double inv = 1.0 / (1.0 - alpha);
        a.coef[slice * a.B + b] = make_float4((float)theta, (float)alpha, (float)inv, 0.f);
        if (!isfinite(alpha) || !isfinite(theta) || !isfinite(inv)) record_numeric(a.status, k);
    }
}

}  // namespace vdamp

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
// Two steps, each run by one 1024-thread CTA per work item (or, when every
// subband is a single part, both in one CTA with the sorted keys kept in
// shared memory between them):
//   sure_sort_part   : part q of subband b sorts its share of the magnitudes,
//                      writes them to their final places in `sorted` and
//                      publishes its position range with the sums of a^2 and
//                      1/a over it;
//   sure_search_part : part q takes the sums below and above its range from
//                      the other parts' records, finds the best interval
//                      starting in its range, and the last part of the
//                      subband to finish picks the global minimiser.
// Sorting: for a >= 0 the IEEE-754 bit pattern is an increasing integer
// function of a, so buckets made of consecutive ranges of bit patterns
// ((bits - lo) >> shift over the 16 octaves below the maximum, 16 to 1024
// buckets per octave growing with the subband size; smaller magnitudes share
// bucket 0) are exactly ordered.  Each
// bucket belongs to the part in which its first position falls, and is
// sorted in registers by a bitonic network of 2, 4, 8, 16 or 32 keys (the
// smallest that holds it) or, above 32 keys, in shared memory.  A bucket
// above SORT_MAX_BUCKET keys (ties, or a degenerate subband) sends the whole
// subband to a bitonic sort done by part 0.  Subbands above SURE_SMALL_BAND
// coefficients (512x512 images) do not fit one CTA's shared memory: their
// parts stream the magnitudes from global memory and keep only their own
// buckets (sure_sort_part_big).
//
// Precision: magnitudes, keys and per-thread partial sums are FP32; the
// cross-warp scans of C and H, tau, theta and alpha of the chosen interval
// are FP64.
#pragma once

#include <math.h>

#include "vdamp_internal.cuh"

namespace vdamp {

#define SORT_BUCKETS 16384                // most buckets (1024 per octave)
#define SORT_MAX_BUCKET 96
#define SORT_MAX_PER_THREAD 32            // largest subband = 32 x 1024 keys
#define SORT_HIST_WORDS (SORT_BUCKETS + SORT_BUCKETS / 32)
#define HIX(q) ((q) + ((q) >> 5))          // padding against bank conflicts in the scan
#define SURE_THREADS 1024
#define SURE_MAX_PARTS 8
#define SURE_KEYS_PER_PART 2048
#define SURE_SMALL_BAND (SORT_MAX_PER_THREAD * SURE_THREADS)   // subbands held whole in shared memory
#define SURE_PART_CAP 32768               // keys one part of a larger subband may hold
#define SURE_MIN_PARTS_BIG 4              // parts of a larger subband at least

// Buckets per octave: about nb / 16, between 16 and 1024 (a power of two).
__host__ __device__ inline int sort_log2_per_octave(int nb) {
    int l = 4;
    while (l < 10 && (16 << l) < nb) ++l;
    return l;
}

__host__ __device__ inline int sure_parts(int nb, int max_parts) {
    int q = (nb + SURE_KEYS_PER_PART - 1) / SURE_KEYS_PER_PART;
    return q < 1 ? 1 : (q > max_parts ? max_parts : q);
}


// Shared memory of the sort (and an upper bound for the search): keys padded
// to a power of two, four spare slots (the one-CTA sort + search keeps its
// keys one slot up), then the bucket counters.
inline size_t sure_smem_bytes(int max_band) {
    int np = 2;
    while (np < max_band) np <<= 1;
    return ((size_t)np + 4) * sizeof(float) + SORT_HIST_WORDS * sizeof(int);
}

// Shared memory of the split sort and search for subbands of up to max_band
// coefficients: whole subbands up to SURE_SMALL_BAND, else one part's keys.
inline size_t sure_split_smem_bytes(int max_band) {
    if (max_band <= SURE_SMALL_BAND) return sure_smem_bytes(max_band);
    return ((size_t)SURE_PART_CAP + 8) * sizeof(float) + SORT_HIST_WORDS * sizeof(int);
}
// Shared memory of the search: the keys of a part and the one below it.
inline size_t sure_split_search_smem_bytes(int max_band) {
    return ((size_t)(max_band <= SURE_SMALL_BAND ? max_band : SURE_PART_CAP) + 8) * sizeof(float);
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

// Sorts bucket keys[s0, s0 + n), 0 < n <= NR, in registers by a bitonic
// network of NR keys and writes it to out (adding each key's a^2 and 1/a, in
// sorted order, to ps2 and ph), or back in place (FUSED).  The network is
// the smallest power of two that holds the bucket: a bucket of a few keys
// costs a few compare-exchanges.
template <int NR, bool FUSED>
__device__ __forceinline__ void sort_bucket_regs(float* keys, float* out, int s0, int n,
                                                 float& ps2, float& ph) {
    if (FUSED && n == 1) return;
    float v[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) v[i] = i < n ? keys[s0 + i] : INFINITY;
    if (n > 1) sort_regs<NR>(v);
#pragma unroll
    for (int i = 0; i < NR; ++i)
        if (i < n) {
            if (FUSED) {
                keys[s0 + i] = v[i];
            } else {
                out[s0 + i] = v[i];
                ps2 += v[i] * v[i];
                ph += v[i] > 0.f ? __frcp_rn(v[i]) : 0.f;
            }
        }
}

// Publishes the position range [p0, p1) a part sorted and the FP64 sums of a^2
// and 1/a over it (fixed summation order: thread t takes positions p0 + t,
// p0 + t + nthr, ..., then a tree over lanes and an ordered sum over warps).
__device__ __forceinline__ void part_record_range(const SureArgs& a, int part, int b, int slice,
                                                  int p0, int p1, const float* out) {
    __shared__ double r_s2[32], r_h[32];
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    float s2 = 0.f, h = 0.f;
    for (int i = p0 + tid; i < p1; i += nthr) {
        const float x = out[i];
        s2 += x * x;
        h += x > 0.f ? __frcp_rn(x) : 0.f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        h += __shfl_xor_sync(0xffffffffu, h, o);
    }
    if (lane == 0) {
        r_s2[warp] = s2;
        r_h[warp] = h;
    }
    __syncthreads();
    if (tid == 0) {
        double ts = 0.0, th = 0.0;
        for (int w = 0; w < (nthr >> 5); ++w) {
            ts += r_s2[w];
            th += r_h[w];
        }
        a.partrec[((size_t)slice * a.B + b) * SURE_MAX_PARTS + part] =
            p1 > p0 ? make_double4_32a((double)p0, (double)p1, ts, th)
                    : make_double4_32a(-1.0, -1.0, 0.0, 0.0);
    }
}

// Publishes range [p0, p1) with per-thread partial sums s2, h already formed
// (each thread over the buckets it sorted, in a fixed order): a tree over
// lanes, then an FP64 sum over warps in warp order.
__device__ __forceinline__ void part_record_sums(const SureArgs& a, int part, int b, int slice,
                                                 int p0, int p1, float s2, float h) {
    __shared__ double r_s2[32], r_h[32];
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        h += __shfl_xor_sync(0xffffffffu, h, o);
    }
    if (lane == 0) {
        r_s2[warp] = s2;
        r_h[warp] = h;
    }
    __syncthreads();
    if (warp == 0) {
        double ts = lane < (nthr >> 5) ? r_s2[lane] : 0.0;
        double th = lane < (nthr >> 5) ? r_h[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ts += __shfl_xor_sync(0xffffffffu, ts, o);
            th += __shfl_xor_sync(0xffffffffu, th, o);
        }
        if (lane == 0)
            a.partrec[((size_t)slice * a.B + b) * SURE_MAX_PARTS + part] =
                p1 > p0 ? make_double4_32a((double)p0, (double)p1, ts, th)
                        : make_double4_32a(-1.0, -1.0, 0.0, 0.0);
    }
}

// Part `part` of subband b of slice `slice`: sort and write its share of |r|.
// Called by all threads of a CTA of SURE_THREADS threads; `keys` is dynamic
// shared memory of sure_smem_bytes(max band) bytes.
// FUSED (one part per subband, the search follows in the same CTA): the
// sorted subband stays in shared memory at keys[1 .. nb] (keys[0] is left
// for the search's predecessor entry), nothing is written to global memory
// and no part record is published.
template <int EMAX, bool FUSED>
__device__ __forceinline__ void sure_sort_part_t(const SureArgs& a, const float2* rk, int part,
                                                 int b, int slice, float* keys_base) {
    __shared__ unsigned s_max_bits;
    __shared__ int s_big;
    __shared__ int wsum[32];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    const int off = a.off[b], nb = a.off[b + 1] - off;
    const int Q = sure_parts(nb, a.max_parts);
    if (part >= Q) return;  // uniform over the CTA
    // bucket q (first position s0) belongs to part floor(s0 Q / nb), i.e. to the
    // part whose position bounds [ceil(part nb / Q), ceil((part + 1) nb / Q)) hold s0
    const int lo_pos = (int)(((long long)part * nb + Q - 1) / Q);
    const int hi_pos = (int)(((long long)(part + 1) * nb + Q - 1) / Q);
    __shared__ int s_qa, s_qb;
    int np = 2;
    while (np < nb) np <<= 1;
    float* keys = FUSED ? keys_base + 1 : keys_base;
    int* hist = reinterpret_cast<int*>(keys_base + np + (FUSED ? 4 : 0));
    float* out = a.sorted + (size_t)slice * a.N + off;

    if (tid == 0) {
        s_max_bits = 0u;
        s_big = 0;
        s_qa = 0;
        s_qb = 0;
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
    const int lpo = sort_log2_per_octave(nb);
    const int nbk = 16 << lpo;          // buckets
    const int shift = 23 - lpo;         // an octave spans 2^23 bit patterns
    for (int i = tid; i < nbk + (nbk >> 5); i += nthr) hist[i] = 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if (lane == 0) atomicMax(&s_max_bits, mx);
    __syncthreads();
    const unsigned span = (unsigned)nbk << shift;
    const unsigned lo_bits = s_max_bits + 1u > span ? s_max_bits + 1u - span : 0u;
    auto bucket = [&](float x) -> int {
        const unsigned u = __float_as_uint(x);
        return u < lo_bits ? 0 : (int)((u - lo_bits) >> shift);
    };
#pragma unroll
    for (int e = 0; e < EMAX; ++e)
        if (tid + e * nthr < nb) atomicAdd(&hist[HIX(bucket(kr[e]))], 1);
    __syncthreads();
    {   // exclusive scan of the counts; each thread owns `per` consecutive buckets
        const int per = nbk >= nthr ? nbk / nthr : 1;
        const int b0 = min(tid * per, nbk);
        const int nq = min(per, nbk - b0);   // 0 for threads past the last bucket
        int loc = 0, big = 0;
        for (int q = 0; q < nq; ++q) {
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
        int na = 0, nbq = 0;   // buckets starting below lo_pos / hi_pos
        for (int q = 0; q < nq; ++q) {
            const int c = hist[HIX(b0 + q)];
            hist[HIX(b0 + q)] = run;
            na += run < lo_pos;
            nbq += run < hi_pos;
            run += c;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            na += __shfl_xor_sync(0xffffffffu, na, o);
            nbq += __shfl_xor_sync(0xffffffffu, nbq, o);
        }
        if (lane == 0) {
            atomicAdd(&s_qa, na);
            atomicAdd(&s_qb, nbq);
        }
    }
    __syncthreads();
    if (s_big) {
        // degenerate subband: part 0 sorts everything, the other parts are empty
        if (part != 0) {   // never with FUSED (one part)
            if (tid == 0)
                a.partrec[((size_t)slice * a.B + b) * SURE_MAX_PARTS + part] =
                    make_double4_32a(-1.0, -1.0, 0.0, 0.0);
            return;
        }
#pragma unroll
        for (int e = 0; e < EMAX; ++e)
            if (tid + e * nthr < nb) keys[tid + e * nthr] = kr[e];
        for (int i = nb + tid; i < np; i += nthr) keys[i] = INFINITY;
        __syncthreads();
        block_bitonic(keys, np);
        if (FUSED) return;
        for (int i = tid; i < nb; i += nthr) out[i] = keys[i];
        __syncthreads();
        part_record_range(a, part, b, slice, 0, nb, out);
        return;
    }
#pragma unroll
    for (int e = 0; e < EMAX; ++e)
        if (tid + e * nthr < nb) keys[atomicAdd(&hist[HIX(bucket(kr[e]))], 1)] = kr[e];
    __syncthreads();
    // hist[q] now holds the end of bucket q; this part sorts buckets [qa, qb).
    const int qa = s_qa, qb = s_qb;
    float ps2 = 0.f, ph = 0.f;   // this thread's sums of a^2 and 1/a, in sorted order
    for (int q = qa + tid; q < qb; q += nthr) {
        const int s0 = q > 0 ? hist[HIX(q - 1)] : 0, s1 = hist[HIX(q)];
        const int n = s1 - s0;
        if (n <= 0) continue;
        if (n <= 2) {
            sort_bucket_regs<2, FUSED>(keys, out, s0, n, ps2, ph);
        } else if (n <= 4) {
            sort_bucket_regs<4, FUSED>(keys, out, s0, n, ps2, ph);
        } else if (n <= 8) {
            sort_bucket_regs<8, FUSED>(keys, out, s0, n, ps2, ph);
        } else if (n <= 16) {
            sort_bucket_regs<16, FUSED>(keys, out, s0, n, ps2, ph);
        } else if (n <= 32) {
            sort_bucket_regs<32, FUSED>(keys, out, s0, n, ps2, ph);
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
            if (FUSED) continue;
            for (int i = s0; i < s1; ++i) {
                const float x = keys[i];
                out[i] = x;
                ps2 += x * x;
                ph += x > 0.f ? __frcp_rn(x) : 0.f;
            }
        }
    }
    if (FUSED) return;
    const int p0 = qa > 0 ? hist[HIX(qa - 1)] : 0;
    const int p1 = qb > qa ? hist[HIX(qb - 1)] : p0;
    part_record_sums(a, part, b, slice, p0, p1, ps2, ph);
}

// Part `part` of a subband above SURE_SMALL_BAND coefficients (split search
// only).  The magnitudes are read from global memory three times (maximum,
// histogram, scatter) instead of being held in registers, and only the
// part's own buckets go to shared memory, at keys[position - base].  Exact
// zeros (a mostly or wholly zero subband) take the first positions without a
// bucket; part 0 writes them and publishes its range from the last of them
// on.  Buckets are sorted by the register networks or, above 32 keys, by
// insertion in shared memory.  A part whose buckets hold more than
// SURE_PART_CAP keys (magnitudes packed into a few buckets) records a numeric
// failure and publishes nothing.
static __device__ void sure_sort_part_big(const SureArgs& a, const float2* rk, int part, int b,
                                          int slice, float* keys) {
    __shared__ unsigned s_max_bits;
    __shared__ int wsum[32];
    __shared__ int s_qa, s_qb, s_zero, s_base, s_end;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    const int off = a.off[b], nb = a.off[b + 1] - off;
    const int Q = sure_parts(nb, a.max_parts);
    if (part >= Q) return;  // uniform over the CTA
    const int lo_pos = (int)(((long long)part * nb + Q - 1) / Q);
    const int hi_pos = (int)(((long long)(part + 1) * nb + Q - 1) / Q);
    int* hist = reinterpret_cast<int*>(keys + SURE_PART_CAP + 8);
    float* out = a.sorted + (size_t)slice * a.N + off;
    const float2* r = rk + (size_t)slice * a.N + off;
    const size_t rec = ((size_t)slice * a.B + b) * SURE_MAX_PARTS + part;

    if (tid == 0) {
        s_max_bits = 0u;
        s_qa = 0;
        s_qb = 0;
        s_zero = 0;
    }
    unsigned mx = 0u;
    for (int i = tid; i < nb; i += nthr) mx = max(mx, __float_as_uint(cabs_f(r[i])));
    const int lpo = sort_log2_per_octave(nb);
    const int nbk = 16 << lpo;
    const int shift = 23 - lpo;
    for (int i = tid; i < nbk + (nbk >> 5); i += nthr) hist[i] = 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if (lane == 0) atomicMax(&s_max_bits, mx);
    __syncthreads();
    const unsigned span = (unsigned)nbk << shift;
    const unsigned lo_bits = s_max_bits + 1u > span ? s_max_bits + 1u - span : 0u;
    auto bucket = [&](unsigned u) -> int {
        return u < lo_bits ? 0 : (int)((u - lo_bits) >> shift);
    };
    int nz = 0;
    for (int i = tid; i < nb; i += nthr) {
        const unsigned u = __float_as_uint(cabs_f(r[i]));
        if (u == 0u) ++nz;
        else atomicAdd(&hist[HIX(bucket(u))], 1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nz += __shfl_xor_sync(0xffffffffu, nz, o);
    if (lane == 0 && nz) atomicAdd(&s_zero, nz);
    __syncthreads();
    const int z = s_zero;
    {   // exclusive scan of the counts from position z on; each thread owns `per` buckets
        const int per = nbk >= nthr ? nbk / nthr : 1;
        const int b0 = min(tid * per, nbk);
        const int nq = min(per, nbk - b0);
        int loc = 0;
        for (int q = 0; q < nq; ++q) loc += hist[HIX(b0 + q)];
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
        int run = z + inc - loc + (warp > 0 ? wsum[warp - 1] : 0);
        int na = 0, nbq = 0;
        for (int q = 0; q < nq; ++q) {
            const int c = hist[HIX(b0 + q)];
            hist[HIX(b0 + q)] = run;
            na += run < lo_pos;
            nbq += run < hi_pos;
            run += c;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            na += __shfl_xor_sync(0xffffffffu, na, o);
            nbq += __shfl_xor_sync(0xffffffffu, nbq, o);
        }
        if (lane == 0) {
            atomicAdd(&s_qa, na);
            atomicAdd(&s_qb, nbq);
        }
    }
    __syncthreads();
    const int qa = s_qa, qb = s_qb;
    if (tid == 0) {   // the part's buckets occupy positions [base, end)
        s_base = qb > qa ? hist[HIX(qa)] : z;
        s_end = qb > qa ? (qb < nbk ? hist[HIX(qb)] : nb) : z;
    }
    __syncthreads();
    const int base = s_base, end = s_end;
    if (end - base > SURE_PART_CAP) {
        if (tid == 0) {
            record_numeric(a.status, a.k);
            a.partrec[rec] = make_double4_32a(-1.0, -1.0, 0.0, 0.0);
        }
        return;
    }
    if (part == 0)
        for (int i = tid; i < z; i += nthr) out[i] = 0.f;
    for (int i = tid; i < nb; i += nthr) {
        const float x = cabs_f(r[i]);
        const unsigned u = __float_as_uint(x);
        if (u == 0u) continue;
        const int q = bucket(u);
        if (q >= qa && q < qb) keys[atomicAdd(&hist[HIX(q)], 1) - base] = x;
    }
    __syncthreads();
    // hist[q] now holds the end of bucket q for the part's buckets
    float ps2 = 0.f, ph = 0.f;
    for (int q = qa + tid; q < qb; q += nthr) {
        const int s0 = q > qa ? hist[HIX(q - 1)] : base, s1 = hist[HIX(q)];
        const int n = s1 - s0;
        if (n <= 0) continue;
        float* kin = keys + (s0 - base);
        float* kout = out + s0;
        if (n <= 2) {
            sort_bucket_regs<2, false>(kin, kout, 0, n, ps2, ph);
        } else if (n <= 4) {
            sort_bucket_regs<4, false>(kin, kout, 0, n, ps2, ph);
        } else if (n <= 8) {
            sort_bucket_regs<8, false>(kin, kout, 0, n, ps2, ph);
        } else if (n <= 16) {
            sort_bucket_regs<16, false>(kin, kout, 0, n, ps2, ph);
        } else if (n <= 32) {
            sort_bucket_regs<32, false>(kin, kout, 0, n, ps2, ph);
        } else {
            for (int i = 1; i < n; ++i) {
                const float x = kin[i];
                int j = i - 1;
                while (j >= 0 && kin[j] > x) {
                    kin[j + 1] = kin[j];
                    --j;
                }
                kin[j + 1] = x;
            }
            for (int i = 0; i < n; ++i) {
                const float x = kin[i];
                kout[i] = x;
                ps2 += x * x;
                ph += x > 0.f ? __frcp_rn(x) : 0.f;
            }
        }
    }
    // part 0 starts at the last zero (the search needs one key to offer theta >= max a)
    const int p0 = part == 0 ? (z > 0 ? z - 1 : 0) : base;
    const int p1 = qb > qa ? end : (part == 0 ? z : p0);
    part_record_sums(a, part, b, slice, p0, p1, ps2, ph);
}

// The magnitudes a thread holds in registers.  One CTA per subband (FUSED):
// the smallest power of two that covers the subband (a 100-coefficient
// subband runs one unrolled step, not 16).  Split parts: 16 or 32, and
// subbands above SURE_SMALL_BAND stream from global memory (measured: the
// six register variants cost the split sort 3 % per 256x256 solve, and gain
// the one-CTA kernel 1 % at 256 x 320x320).
template <bool FUSED>
static __device__ void sure_sort_part_f(const SureArgs& a, const float2* rk, int part, int b,
                                        int slice, float* keys) {
    const int nb = a.off[b + 1] - a.off[b];
    if (!FUSED) {
        if (nb > SURE_SMALL_BAND)
            sure_sort_part_big(a, rk, part, b, slice, keys);
        else if (nb <= 16 * SURE_THREADS)
            sure_sort_part_t<16, FUSED>(a, rk, part, b, slice, keys);
        else
            sure_sort_part_t<SORT_MAX_PER_THREAD, FUSED>(a, rk, part, b, slice, keys);
        return;
    }
    if (nb <= SURE_THREADS)
        sure_sort_part_t<1, FUSED>(a, rk, part, b, slice, keys);
    else if (nb <= 2 * SURE_THREADS)
        sure_sort_part_t<2, FUSED>(a, rk, part, b, slice, keys);
    else if (nb <= 4 * SURE_THREADS)
        sure_sort_part_t<4, FUSED>(a, rk, part, b, slice, keys);
    else if (nb <= 8 * SURE_THREADS)
        sure_sort_part_t<8, FUSED>(a, rk, part, b, slice, keys);
    else if (nb <= 16 * SURE_THREADS)
        sure_sort_part_t<16, FUSED>(a, rk, part, b, slice, keys);
    else
        sure_sort_part_t<SORT_MAX_PER_THREAD, FUSED>(a, rk, part, b, slice, keys);
}

static __device__ void sure_sort_part(const SureArgs& a, const float2* rk, int part, int b,
                                      int slice, float* keys) {
    sure_sort_part_f<false>(a, rk, part, b, slice, keys);
}

// n / d in FP64 from an FP32 reciprocal and Newton steps (the FP64 divider is
// slow here): d and n / d within the FP32 range, d != 0.
__device__ __forceinline__ double pdiv(double n, double d) {
    double r = (double)__frcp_rn((float)d);
    r = r * (2.0 - d * r);
    r = r * (2.0 - d * r);
    const double q = n * r;
    return q + r * (n - d * q);
}

// Writes the results of subband b at iteration k (one thread): tau, theta and
// alpha of the chosen interval (bmi keys below theta, the sum bh of 1/a above
// it, SURE value bv; bmi = nb for theta >= max a, bmi < 0 when nothing was
// found), the minimum SURE, and the per-subband constants of line 8.
__device__ __forceinline__ void sure_finish(const SureArgs& a, int k, int b, int slice, int nb,
                                            double tau, int bmi, double btheta, double bh,
                                            double bv) {
    const size_t orow = ((size_t)slice * a.iters + k) * a.B + b;
    if (!(tau > 0.0) || !isfinite(tau)) {
        // No effective noise (p = 1 and sigma = 0): keep r, no Onsager term.
        a.tau_out[orow] = tau;
        a.thr_out[orow] = 0.0;
        a.alpha_out[orow] = 0.0;
        a.coef[slice * a.B + b] = make_float4(0.f, 0.f, 0.f, 0.f);   // r~ = r
        if (a.sure_out) a.sure_out[(size_t)slice * a.B + b] = 0.0;
        if (!isfinite(tau)) record_numeric(a.status, k);
        return;
    }
    double theta = 0.0, alpha = 0.0;
    if (bmi >= 0) {
        theta = btheta;
        alpha = (bmi == nb) ? 0.0 : pdiv((double)(nb - bmi) - 0.5 * theta * bh, (double)nb);
    }
    a.tau_out[orow] = tau;
    a.thr_out[orow] = theta;
    a.alpha_out[orow] = alpha;
    if (a.sure_out) a.sure_out[(size_t)slice * a.B + b] = bmi >= 0 ? bv : 0.0;
    // line 8 as r~ = r (1 - c1 / |r|) above theta and -c2 r below, c1 = theta / (1 - alpha),
    // c2 = alpha / (1 - alpha): no FP32 difference of nearly equal terms when alpha -> 1
    const double inv = pdiv(1.0, 1.0 - alpha);
    a.coef[slice * a.B + b] =
        make_float4((float)theta, (float)(theta * inv), (float)(alpha * inv), 0.f);
    if (bmi < 0 || !isfinite(alpha) || !isfinite(theta) || !isfinite(inv)) record_numeric(a.status, k);
}

// Search part `part` of subband b: the exact minimiser over the intervals whose
// lower end lies in the part's sorted range, combined across parts by the last
// part to finish (an atomic counter per subband, returned to zero by that part),
// which writes tau, theta and alpha.
// FUSED: the subband is one part whose sorted magnitudes sure_sort_part_t<.., true>
// left at keys[1 .. nb] of the same CTA.
template <bool FUSED>
static __device__ void sure_search_part_t(const SureArgs& a, int k, int part, int b, int slice,
                                          float* keys) {
    __shared__ double s_tau, s_cbase, s_hafter;
    __shared__ int s_p0, s_p1, s_last;
    __shared__ float wc[32], wh[32];
    __shared__ double woc[33], woh[33];
    __shared__ float bq[32], bt[32];
    __shared__ int bm[32];
    __shared__ int s_win_m;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    const int off = a.off[b], nb = a.off[b + 1] - off;
    const int Q = sure_parts(nb, a.max_parts);
    if (part >= Q) return;  // uniform over the CTA
    const size_t rec = ((size_t)slice * a.B + b) * SURE_MAX_PARTS;

    if (warp == 0) {   // tau: fixed-order sum of the column partials, lane by lane then a tree
        double t = 0.0;
        for (int p = lane; p < a.nparts; p += 32)
            t += a.tau_part[((size_t)slice * a.nparts + p) * a.B + b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) s_tau = t;
    }
    if (FUSED && warp == 1) {   // the whole subband, nothing below or above it
        if (lane == 0) {
            s_p0 = 0;
            s_p1 = nb;
            s_cbase = 0.0;
            s_hafter = 0.0;
        }
    } else if (warp == 1) {   // this part's range and the sums of the parts below and above it
        const double4_32a me = a.partrec[rec + part];
        const int p0 = (int)me.x, p1 = (int)me.y;
        double cb = 0.0, ha = 0.0;
        if (lane < Q && lane != part) {
            const double4_32a o = a.partrec[rec + lane];
            if (o.x >= 0.0) {
                if ((int)o.y <= p0) cb = o.z;
                if ((int)o.x >= p1) ha = o.w;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cb += __shfl_xor_sync(0xffffffffu, cb, o);
            ha += __shfl_xor_sync(0xffffffffu, ha, o);
        }
        if (lane == 0) {
            s_p0 = p0;
            s_p1 = p1;
            s_cbase = cb;
            s_hafter = ha;
        }
    }
    __syncthreads();
    const double tau = s_tau;
    const bool live = tau > 0.0 && isfinite(tau) && s_p1 > s_p0;
    const int p0 = live ? s_p0 : 0, len = live ? s_p1 - s_p0 : 0;
    // keys[0] = the magnitude just below the part (0 for the first), keys[1 + i] = a_(p0 + i)
    const float* srt = a.sorted + (size_t)slice * a.N + off;
    if (tid == 0) keys[0] = p0 > 0 ? srt[p0 - 1] : 0.f;
    if (!FUSED)
        batched_for<16, float>(tid, len, nthr, [&](int i) { return srt[p0 + i]; },
                               [&](int i, float v) { keys[1 + i] = v; });
    __syncthreads();

    // ---- prefix sums of a^2 (from below) and suffix sums of 1/a (from above), local
    const int E = (len + nthr - 1) / nthr;
    const int l0 = min(tid * E, len), l1 = min(l0 + E, len);
    float cs = 0.f, hs = 0.f;
    for (int i = l0; i < l1; ++i) {
        const float x = keys[1 + i];
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
    if (warp == 0) {   // FP64 scans of the warp totals, offset by the other parts' sums
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
        const double ce = __shfl_up_sync(0xffffffffu, c, 1);
        const double he = __shfl_up_sync(0xffffffffu, h, 1);
        if (lane < nw) {
            woc[lane] = s_cbase + (lane ? ce : 0.0);
            woh[nw - 1 - lane] = s_hafter + (lane ? he : 0.0);
        }
        if (lane == nw - 1) {
            woc[nw] = s_cbase + c;
            woh[nw] = s_hafter + h;
        }
    }
    __syncthreads();
    const double c_base = woc[warp] + (double)ec;   // sum of a^2 below position p0 + l0
    const double h_after = woh[warp] + (double)eh;  // sum of 1/a from position p0 + l1 on
    const double c_all = woc[nw];                    // sum of a^2 below p0 + len

    // ---- best candidate of this thread's intervals (FP32); m is the global position
    const float tf = (float)tau;
    const float cb = (float)c_base, ha = (float)h_after;
    float best_q = INFINITY, best_t = INFINITY;
    int best_m = -1;
    float csuf = 0.f, hsuf = 0.f;
    for (int l = l1 - 1; l >= l0; --l) {
        const float x = keys[1 + l];
        csuf += x * x;
        hsuf += x > 0.f ? __frcp_rn(x) : 0.f;
        const int m = p0 + l;
        const float cm = cb + (cs - csuf);
        const float hm = ha + hsuf;
        const float K = (float)(nb - m);
        const float lo = keys[l];  // a_(m-1), or 0 at m = 0
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
    const bool has_top = live && p0 + len == nb && l1 == len && l0 < l1;
    if (has_top) {  // theta >= max a: everything thresholded
        const float q = (float)(c_all - (double)nb * tau);
        const float th = keys[len];
        if (q < best_q || (q == best_q && th < best_t)) {
            best_q = q;
            best_t = th;
            best_m = nb;
        }
    }
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
    if (warp == 0) {
        float q = lane < nw ? bq[lane] : INFINITY, t = lane < nw ? bt[lane] : INFINITY;
        int m = lane < nw ? bm[lane] : -1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float q2 = __shfl_xor_sync(0xffffffffu, q, o);
            const float t2 = __shfl_xor_sync(0xffffffffu, t, o);
            const int m2 = __shfl_xor_sync(0xffffffffu, m, o);
            if (q2 < q || (q2 == q && (t2 < t || (t2 == t && m2 < m)))) {
                q = q2;
                t = t2;
                m = m2;
            }
        }
        if (lane == 0) {
            s_win_m = m;
            if (m < 0) a.bestrec[rec + part] = make_double4_32a(INFINITY, 0.0, 0.0, -1.0);
        }
    }
    __syncthreads();

    // ---- the part's best in FP64, by the thread that owns it
    const int wm = s_win_m;
    const bool owner = wm >= 0 && ((wm == nb) ? has_top : (wm >= p0 + l0 && wm < p0 + l1));
    if (owner) {
        double theta, hmd, val;
        if (wm == nb) {
            theta = (double)keys[len];
            hmd = 0.0;
            val = c_all - (double)nb * tau;
        } else {
            float hl = 0.f, cl = 0.f;  // same FP32 sums as the candidate pass
            for (int l = l1 - 1; l >= wm - p0; --l) {
                const float x = keys[1 + l];
                hl += x > 0.f ? __frcp_rn(x) : 0.f;
            }
            for (int l = l0; l < wm - p0; ++l) {
                const float x = keys[1 + l];
                cl += x * x;
            }
            hmd = h_after + (double)hl;
            const double cmd = c_base + (double)cl;
            const double K = (double)(nb - wm);
            const double lo = (double)keys[wm - p0];
            theta = fmax(tau * hmd / (2.0 * K), lo);
            theta = fmin(theta, (double)keys[1 + wm - p0]);
            val = cmd - wm * tau + K * theta * theta + K * tau - tau * theta * hmd;
        }
        a.bestrec[rec + part] = make_double4_32a(val, theta, hmd, (double)wm);
    }
    __syncthreads();

    // ---- the last part of the subband to finish combines the parts
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(&a.counter[(size_t)slice * a.B + b], 1u) == (unsigned)(Q - 1);
    }
    __syncthreads();
    if (!s_last || warp != 0) return;
    __threadfence();
    // lane q reads part q's best; ties go to the smaller theta, then the smaller m
    double bv = INFINITY, btheta = INFINITY, bh = 0.0;
    int bmi = -1;
    if (lane < Q) {
        const volatile double* br = reinterpret_cast<const volatile double*>(a.bestrec + rec + lane);
        const int m = (int)br[3];
        if (m >= 0) {
            bv = br[0];
            btheta = br[1];
            bh = br[2];
            bmi = m;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
        const double t2 = __shfl_xor_sync(0xffffffffu, btheta, o);
        const double h2 = __shfl_xor_sync(0xffffffffu, bh, o);
        const int m2 = __shfl_xor_sync(0xffffffffu, bmi, o);
        const bool take = m2 >= 0 && (bmi < 0 || v2 < bv ||
                                      (v2 == bv && (t2 < btheta || (t2 == btheta && m2 < bmi))));
        if (take) {
            bv = v2;
            btheta = t2;
            bh = h2;
            bmi = m2;
        }
    }
    if (lane != 0) return;
    a.counter[(size_t)slice * a.B + b] = 0u;
    sure_finish(a, k, b, slice, nb, tau, bmi, btheta, bh, bv);
}

static __device__ void sure_search_part(const SureArgs& a, int k, int part, int b, int slice,
                                        float* keys) {
    sure_search_part_t<false>(a, k, part, b, slice, keys);
}

}  // namespace vdamp

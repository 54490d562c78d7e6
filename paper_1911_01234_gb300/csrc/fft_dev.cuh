// Device code of the unitary 2D DFT (Phi = M_Omega F, Sec. 1) for the VDAMP
// iteration: shared-memory Stockham autosort transforms of mixed radix
// 2, 3, 4, 5, 8.  At a stage of radix R after sub-transforms of length Ns,
// butterfly j reads x[j + r n/R], multiplies by w_n^{r (j mod Ns) n/(Ns R)},
// takes a length-R DFT and writes to (j div Ns) Ns R + (j mod Ns) + r Ns.
//
// fft_rows_block transforms whole rows (contiguous).  col_pass_block owns
// whole columns and, between the forward and the inverse column transform,
// applies the k-space part of Algorithm 1:
//   z = m (y - U)                                  (line 3)
//   v = p^-1 ((p^-1 - 1)|z|^2 + sigma^2)           (line 5, per frequency)
//   tau partials  sum_k S_y(ky) S_x(kx) v           (line 5, S^H v)
//   p^-1 z feeds the inverse transform             (line 4, Phi^H P^-1 z)
// so one read and one write of the k-space grid serve lines 3-5.  Both are run
// by all threads of one CTA.
#pragma once

#include "vdamp_internal.cuh"

namespace vdamp {

// ---------------------------------------------------------- small DFTs ---
template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot90(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV>
struct Dft<4, INV> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        float2 t2 = cadd(v[1], v[3]), t3 = rot90<INV>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

template <bool INV>
struct Dft<8, INV> {
    __device__ __forceinline__ static void run(float2* v) {
        const float c = 0.70710678118654752440f;  // cos(pi/4)
        float2 e[4] = {v[0], v[2], v[4], v[6]};
        float2 o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, INV>::run(e);
        Dft<4, INV>::run(o);
        // o[q] *= w8^q, w8 = exp(-+ i pi/4)
        float2 o1 = INV ? make_float2(c * (o[1].x - o[1].y), c * (o[1].x + o[1].y))
                        : make_float2(c * (o[1].x + o[1].y), c * (o[1].y - o[1].x));
        float2 o2 = rot90<INV>(o[2]);
        float2 o3 = INV ? make_float2(-c * (o[3].x + o[3].y), c * (o[3].x - o[3].y))
                        : make_float2(c * (o[3].y - o[3].x), -c * (o[3].x + o[3].y));
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

template <bool INV>
struct Dft<3, INV> {
    __device__ __forceinline__ static void run(float2* v) {
        const float s3 = 0.86602540378443864676f;  // sin(2 pi / 3)
        float2 t = cadd(v[1], v[2]);
        float2 d = csub(v[1], v[2]);
        float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
        // forward: X1 = m - i s3 d, X2 = m + i s3 d
        float2 r = make_float2(s3 * d.y, -s3 * d.x);  // -i s3 d
        if (INV) r = make_float2(-r.x, -r.y);
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    }
};

template <bool INV>
struct Dft<5, INV> {
    __device__ __forceinline__ static void run(float2* v) {
        const float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
        const float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
        const float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
        const float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
        float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        float2 d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
        float2 a1 = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
        float2 a2 = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
        float2 b1 = make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);
        float2 b2 = make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
        // forward: X1 = a1 - i b1, X4 = a1 + i b1, X2 = a2 - i b2, X3 = a2 + i b2
        float2 ib1 = make_float2(-b1.y, b1.x), ib2 = make_float2(-b2.y, b2.x);
        if (INV) {
            ib1 = make_float2(-ib1.x, -ib1.y);
            ib2 = make_float2(-ib2.x, -ib2.y);
        }
        v[0] = make_float2(v[0].x + t1.x + t2.x, v[0].y + t1.y + t2.y);
        v[1] = csub(a1, ib1);
        v[4] = cadd(a1, ib1);
        v[2] = csub(a2, ib2);
        v[3] = cadd(a2, ib2);
    }
};

// Quotient and remainder of 0 <= n < 2^23 by d >= 1 from a float reciprocal
// inv ~ 1/d: the float quotient is off by at most one, fixed by the remainder.
__device__ __forceinline__ int fdivmod(int n, int d, float inv, int& rem) {
    int q = __float2int_rz(__int2float_rn(n) * inv);
    int r = n - q * d;
    if (r < 0) {
        --q;
        r += d;
    } else if (r >= d) {
        ++q;
        r -= d;
    }
    rem = r;
    return q;
}

// One Stockham butterfly of radix R.  Element e of transform t lives at
// buf[tbase + e * es].
template <int R, bool INV>
__device__ __forceinline__ void bfly(const float2* __restrict__ src, float2* __restrict__ dst,
                                     int tbase, int es, int nR, int j, int Ns, float inv_ns,
                                     int step, const float2* __restrict__ tw) {
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[tbase + (j + r * nR) * es];
    int k;
    fdivmod(j, Ns, inv_ns, k);
    if (k != 0) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
            float2 w = __ldg(&tw[r * k * step]);
            if (INV) w.y = -w.y;
            v[r] = cmul(v[r], w);
        }
    }
    Dft<R, INV>::run(v);
    const int d = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[tbase + (d + r * Ns) * es] = v[r];
}

// One stage of radix R over all transforms; then fft_stages, all stages for
// `ntrans` transforms.  ROWS: transform t at t*tstride with
// unit element stride, consecutive threads take consecutive butterflies.
// Otherwise (columns): CB transforms (a power of two), transform t at t with
// element stride CB, consecutive threads take consecutive transforms.
// Returns the buffer that holds the result.  Ends with a __syncthreads().
template <int R, bool INV, bool ROWS, int CB>
__device__ __forceinline__ void fft_stage(const float2* src, float2* dst, const FftAxis& ax,
                                          int ntrans, int tstride, int nb, int Ns, int step) {
    const int total = nb * ntrans;
    const float inv_nb = 1.0f / (float)nb;
    const float inv_ns = 1.0f / (float)Ns;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int t, j;
        if (ROWS) {
            t = fdivmod(idx, nb, inv_nb, j);
        } else {
            t = idx & (CB - 1);
            j = idx / CB;
        }
        bfly<R, INV>(src, dst, ROWS ? t * tstride : t, ROWS ? 1 : CB, nb, j, Ns, inv_ns, step,
                     ax.tw);
    }
}

template <bool INV, bool ROWS, int CB = 1>
static __device__ float2* fft_stages(float2* a, float2* b, const FftAxis& ax, int ntrans,
                                     int tstride) {
    const int n = ax.n;
    int Ns = 1;
    float2* src = a;
    float2* dst = b;
    if (!ROWS) ntrans = CB;
    for (int s = 0; s < ax.nstages; ++s) {
        const int R = ax.radix[s];
        const int nb = n / R;
        const int step = n / (Ns * R);
        // one dispatch per stage; the butterfly loop itself has no indirect branch
        switch (R) {
            case 2: fft_stage<2, INV, ROWS, CB>(src, dst, ax, ntrans, tstride, nb, Ns, step); break;
            case 3: fft_stage<3, INV, ROWS, CB>(src, dst, ax, ntrans, tstride, nb, Ns, step); break;
            case 4: fft_stage<4, INV, ROWS, CB>(src, dst, ax, ntrans, tstride, nb, Ns, step); break;
            case 5: fft_stage<5, INV, ROWS, CB>(src, dst, ax, ntrans, tstride, nb, Ns, step); break;
            default: fft_stage<8, INV, ROWS, CB>(src, dst, ax, ntrans, tstride, nb, Ns, step); break;
        }
        __syncthreads();
        float2* t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

// ------------------------------------------------- compile-time plans ---
// For the axis lengths of the workloads the radix plan is fixed at compile
// time, so that the stage loops, divisions and twiddle strides of fft_stage
// become constants.  radix_plan builds the same plans as the host (variant
// 0: radix 8 first; 1: radix 4 only; 2: the radices 3 and 5 first); a kernel
// uses a compiled plan only when the axis' plan is equal to it, and computes
// exactly what fft_stages computes with it.
struct RadixPlan {
    int ns;
    int r[VDAMP_MAX_STAGES];
};

constexpr RadixPlan radix_plan(int n, int variant) {
    RadixPlan p{0, {0, 0, 0, 0, 0, 0, 0, 0}};
    int m = n, a = 0;
    while (m % 2 == 0) {
        m /= 2;
        ++a;
    }
    int p2[VDAMP_MAX_STAGES] = {0, 0, 0, 0, 0, 0, 0, 0};
    int n2 = 0;
    if (variant == 1) {
        for (int i = 0; i < a / 2; ++i) p2[n2++] = 4;
        if (a & 1) p2[n2++] = 2;
    } else {
        int e8 = a / 3, rem = a % 3;
        if (rem == 1 && e8 > 0) {
            --e8;
            rem = 4;
        }
        for (int i = 0; i < e8; ++i) p2[n2++] = 8;
        if (rem == 4) {
            p2[n2++] = 4;
            p2[n2++] = 4;
        } else if (rem == 2) {
            p2[n2++] = 4;
        } else if (rem == 1) {
            p2[n2++] = 2;
        }
    }
    int odd[VDAMP_MAX_STAGES] = {0, 0, 0, 0, 0, 0, 0, 0};
    int no = 0;
    while (m % 3 == 0 && no < VDAMP_MAX_STAGES) {
        odd[no++] = 3;
        m /= 3;
    }
    while (m % 5 == 0 && no < VDAMP_MAX_STAGES) {
        odd[no++] = 5;
        m /= 5;
    }
    if (variant == 2)
        for (int i = 0; i < no; ++i) p.r[p.ns++] = odd[i];
    for (int i = 0; i < n2; ++i) p.r[p.ns++] = p2[i];
    if (variant != 2)
        for (int i = 0; i < no; ++i) p.r[p.ns++] = odd[i];
    return p;
}

constexpr int plan_prefix(RadixPlan p, int s) {
    int v = 1;
    for (int i = 0; i < s; ++i) v *= p.r[i];
    return v;
}

template <int N, int VAR>
__device__ __forceinline__ bool axis_has_plan(const FftAxis& ax) {
    constexpr RadixPlan P = radix_plan(N, VAR);
    if (ax.n != N || ax.nstages != P.ns) return false;
    bool same = true;
#pragma unroll
    for (int s = 0; s < P.ns; ++s) same &= ax.radix[s] == P.r[s];
    return same;
}

// fft_stage with the length N, the radix R and the sub-transform length NS
// known at compile time (same butterflies, same order of operations); SCALE:
// the outputs are multiplied by `scale` as they are stored.
template <int R, bool INV, bool ROWS, int CB, int N, int NS, bool SCALE = false>
__device__ __forceinline__ void fft_stage_ct(const float2* __restrict__ src, float2* __restrict__ dst,
                                             const float2* __restrict__ tw, int ntrans,
                                             float scale = 1.f) {
    constexpr int NB = N / R;
    constexpr int STEP = N / (NS * R);
    constexpr int ES = ROWS ? 1 : CB;
    const int total = NB * (ROWS ? ntrans : CB);
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int t, j;
        if (ROWS) {
            t = idx / NB;
            j = idx - t * NB;
        } else {
            t = idx & (CB - 1);
            j = idx / CB;
        }
        const int tbase = ROWS ? t * N : t;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[tbase + (j + r * NB) * ES];
        const int k = j % NS;
        if (NS > 1 && k != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = __ldg(&tw[r * k * STEP]);
                if (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        Dft<R, INV>::run(v);
        const int d = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[tbase + (d + r * NS) * ES] = SCALE ? cscale(v[r], scale) : v[r];
    }
}

// Whole rows with the compiled plan (N, VAR) from stage S on: stage 0 reads the
// rows from `src` (global memory), the stages between alternate between the
// shared buffers s0 and s1, and the last stage stores the scaled result to
// `gout` (global memory): two shared-memory passes fewer than loading,
// transforming and storing, with the same arithmetic.
template <int N, int VAR, int S, bool INV>
__device__ __forceinline__ void fft_rows_io(const float2* src, float2* gout, float2* s0, float2* s1,
                                            const float2* tw, int ntrans, float scale) {
    constexpr RadixPlan P = radix_plan(N, VAR);
    constexpr int R = P.r[S];
    constexpr int NS = plan_prefix(P, S);
    if constexpr (S + 1 == P.ns) {
        fft_stage_ct<R, INV, true, 1, N, NS, true>(src, gout, tw, ntrans, scale);
    } else {
        fft_stage_ct<R, INV, true, 1, N, NS>(src, s0, tw, ntrans);
        __syncthreads();
        fft_rows_io<N, VAR, S + 1, INV>(s0, gout, s1, s0, tw, ntrans, scale);
    }
}

// One stage of a compiled plan over the CB columns of a column block, with its
// own element strides on the source and the destination side (CB in shared
// memory, the image width in global memory): the first stage of the forward
// column transform reads the block from global memory, the last stage of the
// inverse one stores it there (scaled).  Same butterflies as fft_stage_ct.
template <int R, bool INV, int CB, int N, int NS, bool SCALE>
__device__ __forceinline__ void fft_stage_cols_io(const float2* __restrict__ src, int ses,
                                                  float2* __restrict__ dst, int des,
                                                  const float2* __restrict__ tw, float scale) {
    constexpr int NB = N / R;
    constexpr int STEP = N / (NS * R);
    for (int idx = threadIdx.x; idx < NB * CB; idx += blockDim.x) {
        const int t = idx & (CB - 1), j = idx / CB;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[t + (size_t)(j + r * NB) * ses];
        const int k = j % NS;
        if (NS > 1 && k != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = __ldg(&tw[r * k * STEP]);
                if (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        Dft<R, INV>::run(v);
        const int d = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r)
            dst[t + (size_t)(d + r * NS) * des] = SCALE ? cscale(v[r], scale) : v[r];
    }
}

// All stages of the compiled plan (N, VAR) from stage S on; returns the
// buffer holding the result.  Each stage ends with a __syncthreads().
template <int N, int VAR, int S, bool INV, bool ROWS, int CB>
__device__ __forceinline__ float2* fft_stages_ct(float2* src, float2* dst, const float2* tw,
                                                 int ntrans) {
    constexpr RadixPlan P = radix_plan(N, VAR);
    if constexpr (S >= P.ns) {
        return src;
    } else {
        constexpr int R = P.r[S];
        constexpr int NS = plan_prefix(P, S);
        fft_stage_ct<R, INV, ROWS, CB, N, NS>(src, dst, tw, ntrans);
        __syncthreads();
        return fft_stages_ct<N, VAR, S + 1, INV, ROWS, CB>(dst, src, tw, ntrans);
    }
}

// The forward column transform of a column block with the compiled plan (N,
// VAR): stage 0 from global memory (gsrc, row stride gstride) into s0, the
// others in shared memory; returns the buffer holding the result.
template <int N, int VAR, int CB>
__device__ __forceinline__ float2* col_fwd_io(const float2* gsrc, int gstride, float2* s0, float2* s1,
                                              const float2* tw) {
    constexpr RadixPlan P = radix_plan(N, VAR);
    fft_stage_cols_io<P.r[0], false, CB, N, 1, false>(gsrc, gstride, s0, CB, tw, 1.f);
    __syncthreads();
    return fft_stages_ct<N, VAR, 1, false, false, CB>(s0, s1, tw, CB);
}

// The inverse column transform from shared memory (src, with `other` the
// second buffer) whose last stage stores the scaled result to global memory
// (gdst, row stride gstride).
template <int N, int VAR, int S, int CB>
__device__ __forceinline__ void col_inv_io(float2* src, float2* other, float2* gdst, int gstride,
                                           const float2* tw, float scale) {
    constexpr RadixPlan P = radix_plan(N, VAR);
    constexpr int R = P.r[S];
    constexpr int NS = plan_prefix(P, S);
    if constexpr (S + 1 == P.ns) {
        fft_stage_cols_io<R, true, CB, N, NS, true>(src, CB, gdst, gstride, tw, scale);
    } else {
        fft_stage_ct<R, true, false, CB, N, NS>(src, other, tw, CB);
        __syncthreads();
        col_inv_io<N, VAR, S + 1, CB>(other, src, gdst, gstride, tw, scale);
    }
}

// Stages of an axis: the compiled plan (N > 0) or the axis' own plan.
template <int N, int VAR, bool INV, bool ROWS, int CB = 1>
__device__ __forceinline__ float2* axis_stages(float2* a, float2* b, const FftAxis& ax,
                                               int ntrans, int tstride) {
    if constexpr (N > 0) {
        return fft_stages_ct<N, VAR, 0, INV, ROWS, CB>(a, b, ax.tw, ntrans);
    } else {
        return fft_stages<INV, ROWS, CB>(a, b, ax, ntrans, tstride);
    }
}

// Rows [row0, row0 + rows) of slice `slice`: out = scale * (F or F^H along x) in.
template <bool INV, int N = 0, int VAR = 0>
static __device__ void fft_rows_block(const float2* in, float2* out, int ny, int nx_rt, const FftAxis& ax,
                               float scale, int row0, int rows, int slice, float2* sm) {
    const int nx = N > 0 ? N : nx_rt;
    float2* A = sm;
    float2* Bf = sm + rows * nx;
    const size_t base = (size_t)slice * ny * nx + (size_t)row0 * nx;
    const int cnt = rows * nx;
    if constexpr (N > 0) {   // compiled plans have at least two stages
        fft_rows_io<N, VAR, 0, INV>(in + base, out + base, A, Bf, ax.tw, rows, scale);
        return;
    }
    batched_for<8, float2>(threadIdx.x, cnt, blockDim.x, [&](int i) { return in[base + i]; },
                           [&](int i, float2 v) { A[i] = v; });
    __syncthreads();
    float2* res = axis_stages<N, VAR, INV, true>(A, Bf, ax, rows, nx);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) out[base + i] = cscale(res[i], scale);
}

// Rows with a compiled plan where the axis has one of the workloads' plans,
// else the axis' own plan.
template <bool INV, int N, int VAR>
__device__ __forceinline__ bool fft_rows_ct(const float2* in, float2* out, int ny, int nx,
                                            const FftAxis& ax, float scale, int row0, int rows,
                                            int slice, float2* sm) {
    if (nx != N || !axis_has_plan<N, VAR>(ax)) return false;
    fft_rows_block<INV, N, VAR>(in, out, ny, nx, ax, scale, row0, rows, slice, sm);
    return true;
}

template <bool INV>
__device__ __forceinline__ void fft_rows_dispatch(const float2* in, float2* out, int ny, int nx,
                                                  const FftAxis& ax, float scale, int row0,
                                                  int rows, int slice, float2* sm) {
    if (fft_rows_ct<INV, 256, 0>(in, out, ny, nx, ax, scale, row0, rows, slice, sm)) return;
    if (fft_rows_ct<INV, 256, 1>(in, out, ny, nx, ax, scale, row0, rows, slice, sm)) return;
    if (fft_rows_ct<INV, 320, 0>(in, out, ny, nx, ax, scale, row0, rows, slice, sm)) return;
    if (fft_rows_ct<INV, 320, 2>(in, out, ny, nx, ax, scale, row0, rows, slice, sm)) return;
    if (fft_rows_ct<INV, 128, 0>(in, out, ny, nx, ax, scale, row0, rows, slice, sm)) return;
    if (fft_rows_ct<INV, 128, 1>(in, out, ny, nx, ax, scale, row0, rows, slice, sm)) return;
    fft_rows_block<INV>(in, out, ny, nx, ax, scale, row0, rows, slice, sm);
}

// Shared memory of a column block: two ny x cb work buffers, the per-column
// tau sums (FP64), the y spectra and the per-warp column sums (up to 32 warps).
inline size_t col_pass_smem_bytes(int ny, int cb, int ntypes) {
    return 2 * (size_t)ny * cb * sizeof(float2) + (size_t)ntypes * cb * sizeof(double) +
           (size_t)ntypes * ny * sizeof(float) + (size_t)32 * ntypes * cb * sizeof(float);
}

// Column block cblk (columns [cblk CB, (cblk + 1) CB)) of slice `slice`; its
// tau partial sums go to tau_part[slice][cblk][B] (nparts blocks per slice).
// Element idx of the block is row idx / CB, column idx % CB; blockDim.x must
// be a multiple of 32 (and so of CB), so a thread keeps one column.
template <int CB, int N = 0, int VAR = 0>
__device__ __forceinline__ void col_pass_block_t(const ColArgs& a, int mode, int u_zero, int cblk,
                                                 int nparts, int slice, float2* sm) {
    const int ny = N > 0 ? N : a.ny, nx = a.nx;
    const int nt = a.ntypes;
    float2* A = sm;
    float2* Bf = sm + ny * CB;
    double* colq = reinterpret_cast<double*>(sm + 2 * ny * CB);  // [nt][CB]
    float* eys = reinterpret_cast<float*>(colq + nt * CB);        // [nt][ny]
    float* red = eys + nt * ny;                                    // [warp][nt][CB]
    const int c0 = cblk * CB;
    const size_t sbase = (size_t)slice * ny * nx + c0;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int cnt = ny * CB;
    auto gidx = [&](int idx) { return sbase + (size_t)(idx / CB) * nx + (idx & (CB - 1)); };

    // ---- forward column transform (or U = 0)
    float2* U = nullptr;
    bool fwd_done = false;
    if constexpr (N > 0) {   // compiled plan: the first stage reads the block from global memory
        if ((mode == COL_ITER || mode == COL_FINAL) && !u_zero) {
            U = col_fwd_io<N, VAR, CB>(a.in + sbase, nx, A, Bf, a.ax.tw);
            fwd_done = true;
        }
    }
    if (fwd_done || (mode != COL_INV && u_zero)) {
        // U is set (or zero)
    } else {
        batched_for<8, float2>(tid, cnt, nthr, [&](int idx) { return a.in[gidx(idx)]; },
                               [&](int idx, float2 v) { A[idx] = v; });
        __syncthreads();
        if (mode == COL_INV) {
            float2* res = axis_stages<N, VAR, true, false, CB>(A, Bf, a.ax, CB, 0);
            for (int idx = tid; idx < cnt; idx += nthr) a.out[gidx(idx)] = cscale(res[idx], a.scale_inv);
            return;
        }
        U = axis_stages<N, VAR, false, false, CB>(A, Bf, a.ax, CB, 0);
        if (mode == COL_FWD) {
            for (int idx = tid; idx < cnt; idx += nthr) a.out[gidx(idx)] = cscale(U[idx], a.scale_fwd);
            return;
        }
    }

    // ---- k-space step of Algorithm 1 (lines 3-5), written into X
    float2* X = (U == A) ? Bf : A;
    if (mode == COL_ITER) {
        batched_for<8, float>(tid, nt * ny, nthr, [&](int i) { return a.ey[i]; },
                              [&](int i, float v) { eys[i] = v; });
        __syncthreads();
    }
    const float sig = mode == COL_ITER ? a.sigma[slice] : 0.f;
    const float sig2 = sig * sig;
    float q[2 * VDAMP_MAX_LEVELS];  // this thread's column: sum over its rows of S_y,t(ky) v
#pragma unroll
    for (int t = 0; t < 2 * VDAMP_MAX_LEVELS; ++t) q[t] = 0.f;
    if (a.klist) {
        // compacted inputs: the unsampled entries are 0 (lines 3-4) or U (the return
        // line), then each thread takes the listed entries of its own column
        for (int idx = tid; idx < cnt; idx += nthr)
            X[idx] = (mode == COL_FINAL) ? cscale(U[idx], a.scale_fwd) : make_float2(0.f, 0.f);
        __syncthreads();
        const int c = tid & (CB - 1), lanes = nthr / CB;
        const size_t lb = ((size_t)slice * nparts + cblk) * CB + c;
        const KEntry* el = a.klist + lb * ny;
        const int ne = a.kcnt[lb];
        for (int e = tid / CB; e < ne; e += lanes) {
            const KEntry k = el[e];
            const int idx = k.row * CB + c;
            if (mode == COL_FINAL) {
                X[idx] = k.y;
                continue;
            }
            const float2 uu = U ? cscale(U[idx], a.scale_fwd) : make_float2(0.f, 0.f);
            const float2 z = csub(k.y, uu);
            const float w = k.w;   // P^-1 (1/p rounded once)
            const float z2 = z.x * z.x + z.y * z.y;
            const float v = w * ((w - 1.0f) * z2 + sig2);
#pragma unroll
            for (int t = 0; t < 2 * VDAMP_MAX_LEVELS; ++t)
                if (t < nt) q[t] += eys[t * ny + k.row] * v;
            X[idx] = cscale(z, w);
        }
    } else {   // dense inputs
        // chunks of 4 elements per thread: the mask, y and p loads of a chunk go out together
        for (int base = tid; base < cnt; base += 4 * nthr) {
            bool mv[4];
            float2 yv[4];
            float pv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = base + u * nthr;
                if (idx < cnt) {
                    const size_t g = gidx(idx);
                    mv[u] = a.mask[g] != 0;
                    yv[u] = a.y[g];
                    pv[u] = mode == COL_ITER ? a.density[g] : 1.f;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = base + u * nthr;
                if (idx >= cnt) continue;
                const int i = idx / CB;
                const float2 uu = U ? cscale(U[idx], a.scale_fwd) : make_float2(0.f, 0.f);
                const bool m = mv[u];
                if (mode == COL_FINAL) {
                    X[idx] = m ? yv[u] : uu;
                    continue;
                }
                const float2 z = m ? csub(yv[u], uu) : make_float2(0.f, 0.f);
                const float w = m ? __frcp_rn(pv[u]) : 0.f;  // P^-1 on Omega (1/p rounded once), 0 elsewhere
                const float z2 = z.x * z.x + z.y * z.y;
                const float v = w * ((w - 1.0f) * z2 + sig2);
#pragma unroll
                for (int t = 0; t < 2 * VDAMP_MAX_LEVELS; ++t)
                    if (t < nt) q[t] += eys[t * ny + i] * v;
                X[idx] = cscale(z, w);
            }
        }
    }

    if (mode == COL_ITER) {
        // Per-column sums: lanes of a warp that share a column (lane mod CB) are
        // combined by shuffles, then the warps by an FP64 sum in warp order;
        // the partial of band b is sum over the block's columns of S_x(kx) Q_ty(b)(kx).
        const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
#pragma unroll
        for (int t = 0; t < 2 * VDAMP_MAX_LEVELS; ++t) {
            if (t < nt) {
                float v = q[t];
#pragma unroll
                for (int o = 16; o >= CB; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane < CB) red[(warp * nt + t) * CB + lane] = v;
            }
        }
        __syncthreads();
        for (int e = tid; e < nt * CB; e += nthr) {
            const int t = e / CB, c = e & (CB - 1);
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += (double)red[(w * nt + t) * CB + c];
            colq[t * CB + c] = s;
        }
        __syncthreads();
        if (tid < a.B) {
            const int b = tid, t = a.ty[b];
            const float* exr = a.ex + (size_t)a.tx[b] * nx + c0;
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < CB; ++c) s += (double)exr[c] * colq[t * CB + c];
            a.tau_part[((size_t)slice * nparts + cblk) * a.B + b] = s;
        }
    } else {
        __syncthreads();
    }

    // ---- inverse column transform (line 4: F^H of P^-1 z, or the return line)
    float2* other = (X == A) ? Bf : A;
    if constexpr (N > 0) {   // compiled plan: the last stage stores to global memory
        col_inv_io<N, VAR, 0, CB>(X, other, a.out + sbase, nx, a.ax.tw, a.scale_inv);
        return;
    }
    float2* res = axis_stages<N, VAR, true, false, CB>(X, other, a.ax, CB, 0);
    for (int idx = tid; idx < cnt; idx += nthr) a.out[gidx(idx)] = cscale(res[idx], a.scale_inv);
}

// Column block with a compiled plan where the column axis has one of the
// workloads' plans, else with the axis' own plan.
template <int CB, int N, int VAR>
__device__ __forceinline__ bool col_pass_ct(const ColArgs& a, int mode, int u_zero, int cblk,
                                            int nparts, int slice, float2* sm) {
    if (a.ny != N || !axis_has_plan<N, VAR>(a.ax)) return false;
    col_pass_block_t<CB, N, VAR>(a, mode, u_zero, cblk, nparts, slice, sm);
    return true;
}

template <int CB>
__device__ __forceinline__ void col_pass_dispatch_cb(const ColArgs& a, int mode, int u_zero,
                                                     int cblk, int nparts, int slice, float2* sm) {
    if (col_pass_ct<CB, 256, 0>(a, mode, u_zero, cblk, nparts, slice, sm)) return;
    if (col_pass_ct<CB, 256, 1>(a, mode, u_zero, cblk, nparts, slice, sm)) return;
    if (col_pass_ct<CB, 320, 0>(a, mode, u_zero, cblk, nparts, slice, sm)) return;
    if (col_pass_ct<CB, 320, 2>(a, mode, u_zero, cblk, nparts, slice, sm)) return;
    if (col_pass_ct<CB, 384, 0>(a, mode, u_zero, cblk, nparts, slice, sm)) return;
    if (col_pass_ct<CB, 384, 2>(a, mode, u_zero, cblk, nparts, slice, sm)) return;
    if (col_pass_ct<CB, 128, 0>(a, mode, u_zero, cblk, nparts, slice, sm)) return;
    if (col_pass_ct<CB, 128, 1>(a, mode, u_zero, cblk, nparts, slice, sm)) return;
    col_pass_block_t<CB>(a, mode, u_zero, cblk, nparts, slice, sm);
}

// The column pass with compiled plans for the workloads' column lengths.
static __device__ void col_pass_dispatch(const ColArgs& a, int mode, int u_zero, int cblk,
                                         int nparts, int slice, float2* sm) {
    switch (a.cb) {
        case 2: col_pass_dispatch_cb<2>(a, mode, u_zero, cblk, nparts, slice, sm); break;
        case 4: col_pass_dispatch_cb<4>(a, mode, u_zero, cblk, nparts, slice, sm); break;
        case 8: col_pass_dispatch_cb<8>(a, mode, u_zero, cblk, nparts, slice, sm); break;
        case 16: col_pass_dispatch_cb<16>(a, mode, u_zero, cblk, nparts, slice, sm); break;
        default: col_pass_block_t<1>(a, mode, u_zero, cblk, nparts, slice, sm); break;
    }
}

static __device__ void col_pass_block(const ColArgs& a, int mode, int u_zero, int cblk, int nparts,
                                      int slice, float2* sm) {
    switch (a.cb) {
        case 1: col_pass_block_t<1>(a, mode, u_zero, cblk, nparts, slice, sm); break;
        case 2: col_pass_block_t<2>(a, mode, u_zero, cblk, nparts, slice, sm); break;
        case 4: col_pass_block_t<4>(a, mode, u_zero, cblk, nparts, slice, sm); break;
        case 8: col_pass_block_t<8>(a, mode, u_zero, cblk, nparts, slice, sm); break;
        default: col_pass_block_t<16>(a, mode, u_zero, cblk, nparts, slice, sm); break;
    }
}

}  // namespace vdamp

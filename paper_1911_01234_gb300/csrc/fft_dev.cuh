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

// All stages for `ntrans` transforms.  ROWS: transform t at t*tstride with
// unit element stride, consecutive threads take consecutive butterflies.
// Otherwise (columns): transform t at t with element stride `es`,
// consecutive threads take consecutive transforms.  Returns the buffer that
// holds the result.  Ends with a __syncthreads().
template <bool INV, bool ROWS>
static __device__ float2* fft_stages(float2* a, float2* b, const FftAxis& ax, int ntrans, int tstride,
                              int es) {
    const int n = ax.n;
    int Ns = 1;
    float2* src = a;
    float2* dst = b;
    const float inv_tr = 1.0f / (float)ntrans;
    for (int s = 0; s < ax.nstages; ++s) {
        const int R = ax.radix[s];
        const int nb = n / R;
        const int total = nb * ntrans;
        const int step = n / (Ns * R);
        const float inv_nb = 1.0f / (float)nb;
        const float inv_ns = 1.0f / (float)Ns;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            int t, j;
            if (ROWS)
                t = fdivmod(idx, nb, inv_nb, j);
            else
                j = fdivmod(idx, ntrans, inv_tr, t);
            const int tb = ROWS ? t * tstride : t;
            const int e = ROWS ? 1 : es;
            switch (R) {
                case 2: bfly<2, INV>(src, dst, tb, e, nb, j, Ns, inv_ns, step, ax.tw); break;
                case 3: bfly<3, INV>(src, dst, tb, e, nb, j, Ns, inv_ns, step, ax.tw); break;
                case 4: bfly<4, INV>(src, dst, tb, e, nb, j, Ns, inv_ns, step, ax.tw); break;
                case 5: bfly<5, INV>(src, dst, tb, e, nb, j, Ns, inv_ns, step, ax.tw); break;
                default: bfly<8, INV>(src, dst, tb, e, nb, j, Ns, inv_ns, step, ax.tw); break;
            }
        }
        __syncthreads();
        float2* t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

// Rows [row0, row0 + rows) of slice `slice`: out = scale * (F or F^H along x) in.
template <bool INV>
static __device__ void fft_rows_block(const float2* in, float2* out, int ny, int nx, const FftAxis& ax,
                               float scale, int row0, int rows, int slice, float2* sm) {
    float2* A = sm;
    float2* Bf = sm + rows * nx;
    const size_t base = (size_t)slice * ny * nx + (size_t)row0 * nx;
    const int cnt = rows * nx;
    batched_for<8, float2>(threadIdx.x, cnt, blockDim.x, [&](int i) { return in[base + i]; },
                           [&](int i, float2 v) { A[i] = v; });
    __syncthreads();
    float2* res = fft_stages<INV, true>(A, Bf, ax, rows, nx, 1);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) out[base + i] = cscale(res[i], scale);
}

inline size_t col_pass_smem_bytes(int ny, int cb, int ntypes) {
    return 2 * (size_t)ny * cb * sizeof(float2) + (size_t)ntypes * ny * sizeof(float);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Column block cblk (columns [cblk cb, (cblk + 1) cb)) of slice `slice`; its
// tau partial sums go to tau_part[slice][cblk][B] (nparts blocks per slice).
// blockDim.x must be a multiple of cb.
static __device__ void col_pass_block(const ColArgs& a, int mode, int u_zero, int cblk, int nparts,
                                      int slice, float2* sm) {
    const int ny = a.ny, nx = a.nx, cb = a.cb;
    float2* A = sm;
    float2* Bf = sm + ny * cb;
    float* eys = reinterpret_cast<float*>(sm + 2 * ny * cb);
    const int c0 = cblk * cb;
    const size_t sbase = (size_t)slice * ny * nx;
    const int tid = threadIdx.x;
    const int cnt = ny * cb;

    // ---- forward column transform (or U = 0)
    float2* U = nullptr;
    if (mode != COL_INV && u_zero) {
        U = nullptr;
    } else {
        batched_for<8, float2>(
            tid, cnt, blockDim.x,
            [&](int idx) {
                const int c = idx % cb, i = idx / cb;
                return a.in[sbase + (size_t)i * nx + c0 + c];
            },
            [&](int idx, float2 v) { A[idx] = v; });
        __syncthreads();
        if (mode == COL_INV) {
            float2* res = fft_stages<true, false>(A, Bf, a.ax, cb, 0, cb);
            for (int idx = tid; idx < cnt; idx += blockDim.x) {
                int c = idx % cb, i = idx / cb;
                a.out[sbase + (size_t)i * nx + c0 + c] = cscale(res[idx], a.scale_inv);
            }
            return;
        }
        U = fft_stages<false, false>(A, Bf, a.ax, cb, 0, cb);
        if (mode == COL_FWD) {
            for (int idx = tid; idx < cnt; idx += blockDim.x) {
                int c = idx % cb, i = idx / cb;
                a.out[sbase + (size_t)i * nx + c0 + c] = cscale(U[idx], a.scale_fwd);
            }
            return;
        }
    }

    // ---- k-space step of Algorithm 1 (lines 3-5), written into X
    float2* X = (U == A) ? Bf : A;
    if (mode == COL_ITER) {
        batched_for<8, float>(tid, a.ntypes * ny, blockDim.x, [&](int i) { return a.ey[i]; },
                              [&](int i, float v) { eys[i] = v; });
        __syncthreads();
    }
    const float sig = mode == COL_ITER ? a.sigma[slice] : 0.f;
    const float sig2 = sig * sig;
    float q[2 * VDAMP_MAX_LEVELS];
#pragma unroll
    for (int t = 0; t < 2 * VDAMP_MAX_LEVELS; ++t) q[t] = 0.f;
    // chunks of 4 elements per thread: the mask, y and p loads of a chunk go out together
    for (int base = tid; base < cnt; base += 4 * blockDim.x) {
        bool mv[4];
        float2 yv[4];
        float pv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int idx = base + u * blockDim.x;
            if (idx < cnt) {
                const int c = idx % cb, i = idx / cb;
                const size_t g = sbase + (size_t)i * nx + c0 + c;
                mv[u] = a.mask[g] != 0;
                yv[u] = a.y[g];
                pv[u] = mode == COL_ITER ? a.density[g] : 1.f;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int idx = base + u * blockDim.x;
            if (idx >= cnt) continue;
            const int i = idx / cb;
            const float2 uu = U ? cscale(U[idx], a.scale_fwd) : make_float2(0.f, 0.f);
            const bool m = mv[u];
            if (mode == COL_FINAL) {
                X[idx] = m ? yv[u] : uu;
                continue;
            }
            const float2 z = m ? csub(yv[u], uu) : make_float2(0.f, 0.f);
            const float w = m ? 1.0f / pv[u] : 0.f;  // P^-1 on Omega, 0 elsewhere
            const float z2 = z.x * z.x + z.y * z.y;
            const float v = w * ((w - 1.0f) * z2 + sig2);
#pragma unroll
            for (int t = 0; t < 2 * VDAMP_MAX_LEVELS; ++t)
                if (t < a.ntypes) q[t] += eys[t * ny + i] * v;
            X[idx] = cscale(z, w);
        }
    }
    __syncthreads();

    if (mode == COL_ITER) {
        // tau partials: column kx = c0 + tid % cb is fixed for this thread
        __shared__ float red[32][VDAMP_MAX_BANDS];
        const int kx = c0 + tid % cb;
        const int warp = tid >> 5, lane = tid & 31;
        for (int b = 0; b < a.B; ++b) {
            float val = 0.f;
            if (tid < cnt) {
#pragma unroll
                for (int t = 0; t < 2 * VDAMP_MAX_LEVELS; ++t)
                    if (t == a.ty[b]) val = a.ex[a.tx[b] * nx + kx] * q[t];
            }
            val = warp_sum(val);
            if (lane == 0) red[warp][b] = val;
        }
        __syncthreads();
        const int nw = (blockDim.x + 31) >> 5;
        if (tid < a.B) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += (double)red[w][tid];
            a.tau_part[((size_t)slice * nparts + cblk) * a.B + tid] = s;
        }
    }

    // ---- inverse column transform (line 4: F^H of P^-1 z, or the return line)
    float2* other = (X == A) ? Bf : A;
    float2* res = fft_stages<true, false>(X, other, a.ax, cb, 0, cb);
    for (int idx = tid; idx < cnt; idx += blockDim.x) {
        int c = idx % cb, i = idx / cb;
        a.out[sbase + (size_t)i * nx + c0 + c] = cscale(res[idx], a.scale_inv);
    }
}

}  // namespace vdamp

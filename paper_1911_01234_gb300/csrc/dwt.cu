// Orthonormal periodic 2D wavelet transform Psi and its adjoint Psi^H
// (Sec. 1, Eq. 5-6), one scale per launch, tiled in shared memory.
//
// Analysis of an H x W image into four (H/2 x W/2) bands:
//   rows:    lo[y][n] = sum_k h[k] X[y][(2n+k) mod W],  hi uses g
//   columns: LL = h*lo, V = g*lo, H = h*hi, D = g*hi along y, same indexing.
// Synthesis is the exact adjoint: X[y][x] += f[k] c[n] for y = (2n+k) mod L.
//
// The packed outputs of the analysis carry Algorithm 1 line 4's addition
// r_k = r~_k + Psi u' (r~_k formed on the fly by SrcSpec), and the packed
// inputs of the synthesis carry line 8 (r~ = (soft(r) - alpha r)/(1 - alpha))
// or line 6 (soft(r)), so that neither r~ nor w_hat is ever stored.
#include "vdamp_internal.cuh"

namespace vdamp {

#define DWT_TO 16   // analysis: output coefficients per tile side
#define IDWT_TO 32  // synthesis: output pixels per tile side

__device__ __forceinline__ int pmod(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

__global__ void __launch_bounds__(256) dwt_level_kernel(DwtArgs a) {
    extern __shared__ float2 sm[];
    const int L = a.f.L;
    const int IT = 2 * DWT_TO + L - 2;
    float2* X = sm;                  // IT x IT input tile
    float2* Lx = X + IT * IT;        // IT x TO
    float2* Hx = Lx + IT * DWT_TO;   // IT x TO
    const int slice = blockIdx.z;
    const int m0 = blockIdx.y * DWT_TO, n0 = blockIdx.x * DWT_TO;
    const int H = a.H, W = a.W;
    const float2* in = a.in + (size_t)slice * a.in_stride;
    const int tid = threadIdx.x;

    for (int idx = tid; idx < IT * IT; idx += blockDim.x) {
        const int r = idx / IT, c = idx - r * IT;
        X[idx] = in[(size_t)pmod(2 * m0 + r, H) * W + pmod(2 * n0 + c, W)];
    }
    __syncthreads();
    for (int idx = tid; idx < IT * DWT_TO; idx += blockDim.x) {
        const int r = idx / DWT_TO, n = idx - r * DWT_TO;
        const float2* xr = X + r * IT + 2 * n;
        float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
        for (int k = 0; k < L; ++k) {
            const float2 x = xr[k];
            lo.x += a.f.h[k] * x.x; lo.y += a.f.h[k] * x.y;
            hi.x += a.f.g[k] * x.x; hi.y += a.f.g[k] * x.y;
        }
        Lx[idx] = lo;
        Hx[idx] = hi;
    }
    __syncthreads();
    const int Ho = H >> 1, Wo = W >> 1;
    const size_t sN = (size_t)slice * a.N;
    for (int idx = tid; idx < DWT_TO * DWT_TO; idx += blockDim.x) {
        const int m = idx / DWT_TO, n = idx - m * DWT_TO;
        const int gm = m0 + m, gn = n0 + n;
        if (gm >= Ho || gn >= Wo) continue;
        float2 ll = make_float2(0.f, 0.f), v = ll, hh = ll, d = ll;
        for (int k = 0; k < L; ++k) {
            const float2 l = Lx[(2 * m + k) * DWT_TO + n];
            const float2 x = Hx[(2 * m + k) * DWT_TO + n];
            const float hk = a.f.h[k], gk = a.f.g[k];
            ll.x += hk * l.x; ll.y += hk * l.y;
            v.x += gk * l.x;  v.y += gk * l.y;
            hh.x += hk * x.x; hh.y += hk * x.y;
            d.x += gk * x.x;  d.y += gk * x.y;
        }
        const size_t pos = (size_t)gm * Wo + gn;
        const float2 outs[4] = {ll, hh, v, d};
#pragma unroll
        for (int q = 1; q < 4; ++q) {
            const size_t p = a.off[q] + pos;
            a.packed[sN + p] = cadd(outs[q], src_value(a.src, slice, a.N, p, a.band[q]));
        }
        if (a.last) {
            const size_t p = a.off[0] + pos;
            a.packed[sN + p] = cadd(ll, src_value(a.src, slice, a.N, p, a.band[0]));
        } else {
            a.ll_out[(size_t)slice * a.ll_stride + pos] = ll;
        }
    }
}

cudaError_t launch_dwt_level(const DwtArgs& a, int batch, cudaStream_t st) {
    const int Ho = a.H >> 1, Wo = a.W >> 1;
    dim3 grid((Wo + DWT_TO - 1) / DWT_TO, (Ho + DWT_TO - 1) / DWT_TO, batch);
    const int IT = 2 * DWT_TO + a.f.L - 2;
    size_t smem = ((size_t)IT * IT + 2 * (size_t)IT * DWT_TO) * sizeof(float2);
    dwt_level_kernel<<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) idwt_level_kernel(IdwtArgs a) {
    extern __shared__ float2 sm[];
    const int L = a.f.L, hL = L >> 1;
    const int CT = IDWT_TO / 2 + hL - 1;
    float2* C = sm;                       // 4 x CT x CT (LL, H, V, D)
    float2* TL = C + 4 * CT * CT;         // TO x CT, low along x
    float2* TH = TL + IDWT_TO * CT;       // TO x CT, high along x
    const int slice = blockIdx.z;
    const int y0 = blockIdx.y * IDWT_TO, x0 = blockIdx.x * IDWT_TO;
    const int h = a.h, w = a.w;
    const int ms = y0 / 2 - (hL - 1), ns = x0 / 2 - (hL - 1);
    const int tid = threadIdx.x;

    for (int idx = tid; idx < 4 * CT * CT; idx += blockDim.x) {
        const int q = idx / (CT * CT);
        const int rem = idx - q * CT * CT;
        const int r = rem / CT, c = rem - r * CT;
        const size_t pos = (size_t)pmod(ms + r, h) * w + pmod(ns + c, w);
        float2 val;
        if (q == 0 && !a.first)
            val = a.ll_in[(size_t)slice * a.ll_stride + pos];
        else
            val = src_value(a.src, slice, a.N, a.off[q] + pos, a.band[q]);
        C[idx] = val;
    }
    __syncthreads();
    const float2* LL = C;
    const float2* HB = C + CT * CT;
    const float2* VB = C + 2 * CT * CT;
    const float2* DB = C + 3 * CT * CT;
    for (int idx = tid; idx < IDWT_TO * CT; idx += blockDim.x) {
        const int t = idx / CT, c = idx - t * CT;
        float2 lo = make_float2(0.f, 0.f), hi = lo;
        for (int k = t & 1; k < L; k += 2) {
            const int r = (t - k) / 2 + hL - 1;
            const float hk = a.f.h[k], gk = a.f.g[k];
            const float2 ll = LL[r * CT + c], vv = VB[r * CT + c];
            const float2 hb = HB[r * CT + c], dd = DB[r * CT + c];
            lo.x += hk * ll.x + gk * vv.x; lo.y += hk * ll.y + gk * vv.y;
            hi.x += hk * hb.x + gk * dd.x; hi.y += hk * hb.y + gk * dd.y;
        }
        TL[idx] = lo;
        TH[idx] = hi;
    }
    __syncthreads();
    const int Ho = 2 * h, Wo = 2 * w;
    for (int idx = tid; idx < IDWT_TO * IDWT_TO; idx += blockDim.x) {
        const int t = idx / IDWT_TO, s = idx - t * IDWT_TO;
        const int gy = y0 + t, gx = x0 + s;
        if (gy >= Ho || gx >= Wo) continue;
        float2 o = make_float2(0.f, 0.f);
        for (int l = s & 1; l < L; l += 2) {
            const int c = (s - l) / 2 + hL - 1;
            const float2 lo = TL[t * CT + c], hi = TH[t * CT + c];
            o.x += a.f.h[l] * lo.x + a.f.g[l] * hi.x;
            o.y += a.f.h[l] * lo.y + a.f.g[l] * hi.y;
        }
        a.out[(size_t)slice * a.out_stride + (size_t)gy * Wo + gx] = o;
    }
}

cudaError_t launch_idwt_level(const IdwtArgs& a, int batch, cudaStream_t st) {
    const int Ho = 2 * a.h, Wo = 2 * a.w;
    dim3 grid((Wo + IDWT_TO - 1) / IDWT_TO, (Ho + IDWT_TO - 1) / IDWT_TO, batch);
    const int CT = IDWT_TO / 2 + a.f.L / 2 - 1;
    size_t smem = (4 * (size_t)CT * CT + 2 * (size_t)IDWT_TO * CT) * sizeof(float2);
    idwt_level_kernel<<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

// r~_{k+1} written out (line 8), for resume and the single-iteration call.
__global__ void line8_kernel(Line8Args a) {
    const int slice = blockIdx.y;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N;
         i += (size_t)gridDim.x * blockDim.x) {
        int b = 0;
        while (b + 1 < a.B && (size_t)a.off[b + 1] <= i) ++b;
        a.out[(size_t)slice * a.N + i] = src_value(a.src, slice, a.N, i, b);
    }
}

cudaError_t launch_line8(const Line8Args& a, int batch, cudaStream_t st) {
    int blocks = (int)((a.N + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    line8_kernel<<<dim3(blocks, batch), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace vdamp

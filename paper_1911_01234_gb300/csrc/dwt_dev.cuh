// Device code of one scale of the orthonormal periodic 2D wavelet transform
// Psi and of its adjoint Psi^H (Sec. 1, Eq. 5-6), tiled in shared memory.
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
//
// A tile is computed by all threads of one CTA (any block size).  Tile sides
// (a.to) are runtime values: analysis tiles are to x to output coefficients,
// synthesis tiles to x to output pixels (to even).
#pragma once

#include "vdamp_internal.cuh"

namespace vdamp {


// Shared memory of one tile.
inline size_t dwt_tile_smem(int to, int L) {
    const size_t IT = 2 * (size_t)to + L - 2;
    return (IT * IT + 2 * IT * to) * sizeof(float2);
}
inline size_t idwt_tile_smem(int to, int L) {
    const size_t CT = (size_t)to / 2 + L / 2 - 1;
    return (4 * CT * CT + 2 * (size_t)to * CT) * sizeof(float2);
}

// Periodic index: v mod n for v within a few periods of [0, n).
__device__ __forceinline__ int wrap(int v, int n) {
    while (v < 0) v += n;
    while (v >= n) v -= n;
    return v;
}

// Analysis tile (tile_x, tile_y) of slice `slice`; L taps, TO x TO outputs.
template <int L, int TO>
__device__ __forceinline__ void dwt_tile_t(const DwtArgs& a, const float2* in_base,
                                           float2* packed, const SrcSpec& src, int tile_x,
                                           int tile_y, int slice, float2* sm) {
    constexpr int IT = 2 * TO + L - 2;
    float2* X = sm;              // IT x IT input tile
    float2* Lx = X + IT * IT;    // IT x TO
    float2* Hx = Lx + IT * TO;   // IT x TO
    const int m0 = tile_y * TO, n0 = tile_x * TO;
    const int H = a.H, W = a.W;
    const float2* in = in_base + (size_t)slice * a.in_stride;
    const int tid = threadIdx.x;

    // a window row or column is wrapped once (a cheap test where the image is at
    // least a window wide)
    auto wr = [](int v, int n) { return n >= IT ? (v >= n ? v - n : v) : wrap(v, n); };
    batched_for<8, float2>(
        tid, IT * IT, blockDim.x,
        [&](int idx) {
            const int r = idx / IT, c = idx - r * IT;
            return in[(size_t)wr(2 * m0 + r, H) * W + wr(2 * n0 + c, W)];
        },
        [&](int idx, float2 v) { X[idx] = v; });
    __syncthreads();
    for (int idx = tid; idx < IT * TO; idx += blockDim.x) {
        const int r = idx / TO, n = idx - r * TO;
        const float2* xr = X + r * IT + 2 * n;
        float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
#pragma unroll
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
    const float4 kq[4] = {src_coef(src, slice, a.band[0]), src_coef(src, slice, a.band[1]),
                          src_coef(src, slice, a.band[2]), src_coef(src, slice, a.band[3])};
    const float2* rs = src.r + sN;
    for (int idx = tid; idx < TO * TO; idx += blockDim.x) {
        const int m = idx / TO, n = idx - m * TO;
        const int gm = m0 + m, gn = n0 + n;
        if (gm >= Ho || gn >= Wo) continue;
        float2 ll = make_float2(0.f, 0.f), v = ll, hh = ll, d = ll;
#pragma unroll
        for (int k = 0; k < L; ++k) {
            const float2 l = Lx[(2 * m + k) * TO + n];
            const float2 x = Hx[(2 * m + k) * TO + n];
            const float hk = a.f.h[k], gk = a.f.g[k];
            ll.x += hk * l.x; ll.y += hk * l.y;
            v.x += gk * l.x;  v.y += gk * l.y;
            hh.x += hk * x.x; hh.y += hk * x.y;
            d.x += gk * x.x;  d.y += gk * x.y;
        }
        const int pos = gm * Wo + gn;
        const float2 outs[4] = {ll, hh, v, d};
        float2 rv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)   // the r~ values of the four bands, loads issued together
            rv[q] = (src.mode == SRC_ZERO || (q == 0 && !a.last)) ? make_float2(0.f, 0.f)
                                                                  : rs[a.off[q] + pos];
#pragma unroll
        for (int q = 1; q < 4; ++q)
            packed[sN + a.off[q] + pos] = cadd(outs[q], src_apply(src.mode, rv[q], kq[q]));
        if (a.last) {
            packed[sN + a.off[0] + pos] = cadd(ll, src_apply(src.mode, rv[0], kq[0]));
        } else {
            a.ll_out[(size_t)slice * a.ll_stride + pos] = ll;
        }
    }
}

// Synthesis tile (tile_x, tile_y) of slice `slice`; L taps, TO x TO outputs.
// Polyphase form: output rows 2u and 2u + 1 read the same coefficient rows
// (u - kk + L/2 - 1 for tap pairs 2kk, 2kk + 1), and likewise along x, so a
// thread forms both phases from one set of shared-memory reads with the taps
// at compile-time positions.
template <int L, int TO>
__device__ __forceinline__ void idwt_tile_t(const IdwtArgs& a, float2* out, const SrcSpec& src,
                                            int tile_x, int tile_y, int slice, float2* sm) {
    constexpr int hL = L / 2;
    constexpr int CT = TO / 2 + hL - 1;
    constexpr int CTT = CT * CT;
    constexpr int TH2 = TO / 2;
    float2* C = sm;                  // 4 x CT x CT (LL, H, V, D)
    float2* TL = C + 4 * CTT;        // TO x CT, low along x
    float2* TH = TL + TO * CT;       // TO x CT, high along x
    const int y0 = tile_y * TO, x0 = tile_x * TO;
    const int h = a.h, w = a.w;
    const int ms = y0 / 2 - (hL - 1), ns = x0 / 2 - (hL - 1);
    const int tid = threadIdx.x, nthr = blockDim.x;
    // per-band packed offsets and denoiser parameters, selected without indexing
    const int o0 = a.off[0], o1 = a.off[1], o2 = a.off[2], o3 = a.off[3];
    const float4 k0 = src_coef(src, slice, a.band[0]), k1 = src_coef(src, slice, a.band[1]);
    const float4 k2 = src_coef(src, slice, a.band[2]), k3 = src_coef(src, slice, a.band[3]);
    const float2* rs = src.r + (size_t)slice * a.N;
    const float2* lls = a.ll_in + (size_t)slice * a.ll_stride;
    const bool ll_dense = !a.first;
    const int mode = src.mode;

    // the four bands' CT x CT windows: each thread takes window positions e and
    // e + nthr of every band, so eight loads go out together; a window row is
    // wrapped once (a cheap test where the band is at least a window wide)
    auto wr = [](int v, int n) { return n >= CT ? (v < 0 ? v + n : (v >= n ? v - n : v)) : wrap(v, n); };
    const float2* base[4] = {ll_dense ? lls : rs + o0, rs + o1, rs + o2, rs + o3};
    const float4 kq[4] = {k0, k1, k2, k3};
    for (int e0 = tid; e0 < CTT; e0 += 2 * nthr) {
        float2 v[2][4];
        int pos[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int e = e0 + j * nthr;
            const int r = e / CT, c = e - r * CT;
            pos[j] = wr(ms + r, h) * w + wr(ns + c, w);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool live = e < CTT && (mode != SRC_ZERO || (q == 0 && ll_dense));
                v[j][q] = live ? base[q][pos[j]] : make_float2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int e = e0 + j * nthr;
            if (e >= CTT) continue;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                C[q * CTT + e] = (q == 0 && ll_dense) ? v[j][q] : src_apply(mode, v[j][q], kq[q]);
        }
    }
    __syncthreads();
    const float2* LL = C;
    const float2* HB = C + CTT;
    const float2* VB = C + 2 * CTT;
    const float2* DB = C + 3 * CTT;
    // along y: rows 2u, 2u + 1 of TL (from LL, V) and TH (from H, D)
    for (int idx = tid; idx < TH2 * CT; idx += nthr) {
        const int u = idx / CT, c = idx - u * CT;
        float2 le = make_float2(0.f, 0.f), lo = le, he = le, ho = le;
#pragma unroll
        for (int kk = 0; kk < hL; ++kk) {
            const int r = u - kk + hL - 1;
            const float2 ll = LL[r * CT + c], vv = VB[r * CT + c];
            const float2 hb = HB[r * CT + c], dd = DB[r * CT + c];
            const float he0 = a.f.h[2 * kk], ge0 = a.f.g[2 * kk];
            const float he1 = a.f.h[2 * kk + 1], ge1 = a.f.g[2 * kk + 1];
            le.x += he0 * ll.x + ge0 * vv.x; le.y += he0 * ll.y + ge0 * vv.y;
            lo.x += he1 * ll.x + ge1 * vv.x; lo.y += he1 * ll.y + ge1 * vv.y;
            he.x += he0 * hb.x + ge0 * dd.x; he.y += he0 * hb.y + ge0 * dd.y;
            ho.x += he1 * hb.x + ge1 * dd.x; ho.y += he1 * hb.y + ge1 * dd.y;
        }
        TL[(2 * u) * CT + c] = le;
        TL[(2 * u + 1) * CT + c] = lo;
        TH[(2 * u) * CT + c] = he;
        TH[(2 * u + 1) * CT + c] = ho;
    }
    __syncthreads();
    // along x: pixels 2v, 2v + 1 of row t, stored as one 16-byte pair when the
    // slice's output starts on a 16-byte boundary (rows have an even length)
    const int Ho = 2 * h, Wo = 2 * w;
    float2* obase = out + (size_t)slice * a.out_stride;
    const bool al16 = (reinterpret_cast<uintptr_t>(obase) & 15) == 0;
    for (int idx = tid; idx < TO * TH2; idx += nthr) {
        const int t = idx / TH2, v = idx - t * TH2;
        const int gy = y0 + t, gx = x0 + 2 * v;
        if (gy >= Ho || gx >= Wo) continue;
        float2 oe = make_float2(0.f, 0.f), oo = oe;
#pragma unroll
        for (int l2 = 0; l2 < hL; ++l2) {
            const int c = v - l2 + hL - 1;
            const float2 lo = TL[t * CT + c], hi = TH[t * CT + c];
            const float h0 = a.f.h[2 * l2], g0 = a.f.g[2 * l2];
            const float h1 = a.f.h[2 * l2 + 1], g1 = a.f.g[2 * l2 + 1];
            oe.x += h0 * lo.x + g0 * hi.x; oe.y += h0 * lo.y + g0 * hi.y;
            oo.x += h1 * lo.x + g1 * hi.x; oo.y += h1 * lo.y + g1 * hi.y;
        }
        float2* o = obase + (size_t)gy * Wo + gx;
        if (al16) {
            *reinterpret_cast<float4*>(o) = make_float4(oe.x, oe.y, oo.x, oo.y);
        } else {
            o[0] = oe;
            o[1] = oo;
        }
    }
}

// Dispatch on (taps, tile side); the plans use L in {2, 8}, to in {16, 32, 64}.
static __device__ void dwt_tile(const DwtArgs& a, const float2* in, float2* packed,
                                const SrcSpec& src, int tile_x, int tile_y, int slice, float2* sm) {
    if (a.f.L == 2) {
        if (a.to == 16) dwt_tile_t<2, 16>(a, in, packed, src, tile_x, tile_y, slice, sm);
        else if (a.to == 32) dwt_tile_t<2, 32>(a, in, packed, src, tile_x, tile_y, slice, sm);
        else dwt_tile_t<2, 64>(a, in, packed, src, tile_x, tile_y, slice, sm);
    } else {
        if (a.to == 16) dwt_tile_t<8, 16>(a, in, packed, src, tile_x, tile_y, slice, sm);
        else if (a.to == 32) dwt_tile_t<8, 32>(a, in, packed, src, tile_x, tile_y, slice, sm);
        else dwt_tile_t<8, 64>(a, in, packed, src, tile_x, tile_y, slice, sm);
    }
}

static __device__ void idwt_tile(const IdwtArgs& a, float2* out, const SrcSpec& src, int tile_x,
                                 int tile_y, int slice, float2* sm) {
    if (a.f.L == 2) {
        if (a.to == 16) idwt_tile_t<2, 16>(a, out, src, tile_x, tile_y, slice, sm);
        else if (a.to == 32) idwt_tile_t<2, 32>(a, out, src, tile_x, tile_y, slice, sm);
        else idwt_tile_t<2, 64>(a, out, src, tile_x, tile_y, slice, sm);
    } else {
        if (a.to == 16) idwt_tile_t<8, 16>(a, out, src, tile_x, tile_y, slice, sm);
        else if (a.to == 32) idwt_tile_t<8, 32>(a, out, src, tile_x, tile_y, slice, sm);
        else idwt_tile_t<8, 64>(a, out, src, tile_x, tile_y, slice, sm);
    }
}

// r~ (line 8) for packed coefficients [i0, i1) of slice `slice`.
__device__ __forceinline__ void line8_range(const Line8Args& a, const SrcSpec& src, float2* out,
                                            int slice, size_t i0, size_t i1, size_t stride) {
    for (size_t i = i0; i < i1; i += stride) {
        int b = 0;
        while (b + 1 < a.B && (size_t)a.off[b + 1] <= i) ++b;
        out[(size_t)slice * a.N + i] = src_value(src, slice, a.N, i, b);
    }
}

}  // namespace vdamp

// Kernels of the learned per-subband denoiser (see cnn_dev.cuh): the 3x3
// convolution as an implicit GEMM on the tcgen05 tensor cores (128 pixels x
// COUT outputs x 9 CIN taps per tile, BF16 operands in shared memory, FP32
// accumulator in tensor memory), its weight gradient, and the elementwise
// steps around the network (input planes, residual output, Hutchinson probe,
// loss gradient, Adam).
#include <atomic>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "../../include/vdamp.h"
#include "cnn_dev.cuh"
#include "vdamp_internal.cuh"

namespace vdamp {

namespace {

constexpr uint32_t kWaitLimit = 1u << 24;
constexpr int CONV_STAGES = 4;   // halo buffers: the current tile and three in flight

// ---------------------------------------------------------------- conv ---
// Implicit GEMM without an im2col copy.  A tile is a block of the image
// (conv_block: R rows x Wb columns); its zero-padded halo of pitch P = Wb + 2
// lives in shared memory as CIN/8 chunk planes [chunk][position][8 channels]
// (16 bytes per position), so that for tap (dy, dx) the A operand of the MMA
// is the same buffer read from position P + 1 + m + dy P + dx: a descriptor
// whose start moves by 16 bytes per position, 8-row groups 128 bytes apart
// (SBO), and the two chunks of a K step one chunk plane apart (LBO).  The halo (and, for the masked
// modes, the mask rows) of the next tile arrive by cp.async (zero-filled
// outside the image) while the current tile's MMAs and epilogue run; weights
// and bias are staged once per band.
// Where a tile sits: its image (dense offset, size, band) and its block
// (pitch, width, rows, the image pixel of halo position (0, 0)).
struct ConvTile {
    int off, h, w, band, pitch, wb, rows, y0, x0;
};

constexpr int CONV_THREADS = 256;   // 128 output rows x 2 halves of the output channels

template <int CIN, int COUT>
__global__ void __launch_bounds__(CONV_THREADS) conv3x3_kernel(const __grid_constant__ ConvArgs a) {
    constexpr int K = 9 * CIN;
    constexpr int NCH = CIN / 8;
    constexpr int KPT = CIN / 16;   // K steps per tap
    constexpr int HC = COUT / 2;    // output channels per thread
    constexpr int B_BYTES = COUT * K * 2;
    constexpr int M_BYTES = 128 * COUT * 2;
    constexpr uint32_t SBO_B = (K / 8) * 128, LBO_B = 128;
    constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, COUT);
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t mbar[2];   // one per TMEM accumulator
    __shared__ uint32_t tbase;
    __shared__ float s_bias[2][COUT];   // bias of the current band and of the next one
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & 127, half = tid >> 7;   // output row m and channel half of this thread
    const int nq = a.nq;
    const uint32_t CS = (uint32_t)nq * 16;
    const uint32_t A_BYTES = NCH * CS;
    uint8_t* const sA0 = smem;                       // STAGES stages
    uint8_t* const sB = smem + CONV_STAGES * A_BYTES;
    uint8_t* const sM0 = sB + B_BYTES;               // STAGES stages (masked mode)
    const bool masked = a.mode == CONV_MASK;

    // a contiguous range of tiles per CTA: weight bands change rarely
    const int per = (a.total_tiles + gridDim.x - 1) / gridDim.x;
    const int t_begin = blockIdx.x * per;
    const int t_end = min(a.total_tiles, t_begin + per);
    if (t_begin >= t_end) return;   // uniform over the CTA

    cudaGridDependencySynchronize();
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
    }
    if (warp == 0) tc::tmem_alloc(&tbase, 64);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tbase;

    // Tiles come in increasing order: the image is found by stepping from the
    // last one (one binary search per CTA) and its block shape is recomputed
    // only when the image changes.
    int load_idx = find_conv_image(a.img, a.n_img, t_begin);
    CnnImage lim = a.img[load_idx];
    ConvBlock lcb = conv_block(lim.h, lim.w);
    auto locate = [&](int t) -> ConvTile {
        bool moved = false;
        while (load_idx + 1 < a.n_img && __ldg(&a.img[load_idx + 1].ctile0) <= t) {
            ++load_idx;
            moved = true;
        }
        if (moved) {
            lim = a.img[load_idx];
            lcb = conv_block(lim.h, lim.w);
        }
        const int ti = t - lim.ctile0, by = ti / lcb.nbx, bx = ti - by * lcb.nbx;
        return ConvTile{lim.off, lim.h, lim.w, lim.band, lcb.pitch, lcb.wb, lcb.rows,
                        by * lcb.rows - 1, bx * lcb.wb - 1};
    };
    // asynchronous loads of a tile's halo (and mask rows) into stage st (one commit group)
    auto issue_loads = [&](const ConvTile& ct, int st) {
        uint8_t* sA = sA0 + st * A_BYTES;
        const int P = ct.pitch, nqi = conv_halo(P);
        const __nv_bfloat16* base = a.in + (size_t)ct.off * CIN;
        for (int q = tid; q < nqi; q += CONV_THREADS) {
            const int i = q / P, j = q - i * P;
            const int y = ct.y0 + i, x = ct.x0 + j;
            const bool inb = y >= 0 && y < ct.h && x >= 0 && x < ct.w;
            const __nv_bfloat16* src = inb ? base + (size_t)(y * ct.w + x) * CIN : base;
#pragma unroll
            for (int c = 0; c < NCH; ++c)
                tc::cp_async16(sA + c * CS + (uint32_t)q * 16, src + 8 * c, inb ? 16u : 0u);
        }
        if (masked) {   // the mask row of output m: half of it per thread
            const int q = P + 1 + row, i = q / P, j = q - i * P;
            const int y = ct.y0 + i, x = ct.x0 + j;
            const bool ok = i <= ct.rows && j >= 1 && j <= ct.wb && y < ct.h && x < ct.w;
            const __nv_bfloat16* src =
                ok ? a.mask + ((size_t)ct.off + (size_t)y * ct.w + x) * COUT + half * HC : a.mask;
            uint8_t* dst = sM0 + st * M_BYTES + row * COUT * 2 + half * HC * 2;
#pragma unroll
            for (int c = 0; c < HC / 8; ++c) tc::cp_async16(dst + 16 * c, src + 8 * c, ok ? 16u : 0u);
        }
        tc::cp_async_commit();
    };
    auto load_band = [&](int band, int slot) {   // synchronous: no MMA may be in flight
        const uint4* src = reinterpret_cast<const uint4*>(a.wimg + (size_t)band * COUT * K);
        for (int i = tid; i < B_BYTES / 16; i += CONV_THREADS) reinterpret_cast<uint4*>(sB)[i] = src[i];
        if (tid < COUT) s_bias[slot][tid] = a.bias ? a.bias[(size_t)band * COUT + tid] : 0.f;
    };
    auto issue_mma = [&](const ConvTile& ct, int st, int acc) {   // one thread
        const int W2 = ct.pitch;
        const uint32_t abase = tc::smem_u32(sA0 + st * A_BYTES);
        const uint32_t bbase = tc::smem_u32(sB);
#pragma unroll
        for (int ks = 0; ks < 9 * KPT; ++ks) {
            const int tp = ks / KPT, j = ks - tp * KPT;
            int sh = tap_dy(tp) * W2 + tap_dx(tp);
            if (a.mirror) sh = -sh;
            const uint32_t aaddr = abase + (uint32_t)(W2 + 1 + sh) * 16 + (uint32_t)(2 * j) * CS;
            tc::mma_bf16(tmem + acc * 32, tc::make_desc(aaddr, CS, 128),
                         tc::make_desc(bbase + ks * 256, LBO_B, SBO_B), IDESC, ks > 0);
        }
        tc::mma_commit(&mbar[acc]);
    };

    constexpr int D = CONV_STAGES - 1;   // tiles in flight ahead of the current one
    uint32_t phase[2] = {0, 0};
    bool ok = true, pending[2] = {false, false};
    bool timed_out = false;   // this thread's MMA wait ran out (made uniform at the next barrier)
    // tiles t_begin .. t_begin + D - 1 into stages 0 .. D - 1; every iteration t
    // then refills the stage of tile t - 1 with tile t + D
    ConvTile cur = locate(t_begin);
    issue_loads(cur, 0);
    ConvTile ahead[D - 1];               // at iteration t: tiles t + 1 .. t + D - 1
#pragma unroll
    for (int d = 1; d < D; ++d) {
        ahead[d - 1] = cur;              // defined even past the range (then never used)
        if (t_begin + d < t_end) {
            ahead[d - 1] = locate(t_begin + d);
            issue_loads(ahead[d - 1], d);
        } else {
            tc::cp_async_commit();       // empty group: the group count stays aligned
        }
    }
    int band = cur.band, bslot = 0;
    load_band(band, 0);
    tc::cp_async_wait<D - 2>();          // tile t_begin has landed
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
        tc::fence_after_sync();
        issue_mma(cur, 0, 0);
    }
    pending[0] = true;
    // Iteration t: MMAs of tile t are in flight in accumulator t & 1.  Issue
    // the MMAs of tile t + 1 into the other accumulator (free since the
    // epilogue of tile t - 1), then wait for tile t and run its epilogue.
    for (int t = t_begin; t < t_end; ++t) {
        const int k = t - t_begin, ac = k & 1;
        const int st = k % CONV_STAGES;
        const bool more = t + 1 < t_end;
        const ConvTile nxt = ahead[0];
        // tile t + 1 has landed (t + 2 .. t + D - 1 may still fly; t + D is issued below)
        tc::cp_async_wait<D - 2>();
        const bool new_band = more && nxt.band != band;
        if (new_band) {
            // the weights change: the tensor cores must be done with tile t first
            ok = __syncthreads_and(tc::mbar_wait(&mbar[ac], phase[ac], a.wait_limit)) != 0;
            if (!ok) break;
            band = nxt.band;
            load_band(band, bslot ^ 1);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        // every thread is past the epilogue of tile t - 1; a wait that ran out stops all
        if (__syncthreads_or(timed_out)) {
            ok = false;
            break;
        }
        if (more) {
            if (tid == 0) {
                tc::fence_after_sync();
                issue_mma(nxt, (k + 1) % CONV_STAGES, ac ^ 1);
            }
            pending[ac ^ 1] = true;
        }
        // the stage of tile t - 1 is free (its MMAs and epilogue are done): refill it
        ConvTile fresh = cur;
        if (t + D < t_end) {
            fresh = locate(t + D);
            issue_loads(fresh, (k + D) % CONV_STAGES);
        } else {
            tc::cp_async_commit();
        }
#pragma unroll
        for (int d = 0; d + 2 < D; ++d) ahead[d] = ahead[d + 1];
        ahead[D - 2] = fresh;
        if (!new_band && !tc::mbar_wait(&mbar[ac], phase[ac], a.wait_limit)) {
            timed_out = true;   // each warp waits on its own; the outcome meets at the next barrier
            continue;
        }
        phase[ac] ^= 1;
        pending[ac] = false;
        tc::fence_after_sync();
        // epilogue: this thread's row m = row, channels [half HC, half HC + HC)
        float acc[HC];
        const uint32_t ta = tmem + ac * 32 + half * HC + ((uint32_t)((warp & 3) * 32) << 16);
        if (HC == 16) tc::tmem_ld16(ta, acc);
        else tc::tmem_ld8(ta, acc);
        const int q = cur.pitch + 1 + row, bi = q / cur.pitch, bj = q - bi * cur.pitch;
        const int oy = cur.y0 + bi, ox = cur.x0 + bj;
        if (bi <= cur.rows && bj >= 1 && bj <= cur.wb && oy < cur.h && ox < cur.w) {
            const size_t p = (size_t)cur.off + (size_t)oy * cur.w + ox;
            const float* bs = s_bias[bslot] + half * HC;
            if (a.mode == CONV_BIAS_RELU || masked) {
                uint32_t mk[HC / 2];
                if (masked) {
                    const uint4* ms = reinterpret_cast<const uint4*>(sM0 + st * M_BYTES +
                                                                     row * COUT * 2 + half * HC * 2);
#pragma unroll
                    for (int c = 0; c < HC / 8; ++c) {
                        const uint4 v = ms[c];
                        mk[4 * c] = v.x;
                        mk[4 * c + 1] = v.y;
                        mk[4 * c + 2] = v.z;
                        mk[4 * c + 3] = v.w;
                    }
                }
                uint32_t pk[HC / 2];
#pragma unroll
                for (int c = 0; c < HC / 2; ++c) {
                    float v0 = acc[2 * c], v1 = acc[2 * c + 1];
                    if (!masked) {
                        v0 = fmaxf(v0 + bs[2 * c], 0.f);
                        v1 = fmaxf(v1 + bs[2 * c + 1], 0.f);
                    } else {   // keep where the mask's bfloat16 is > 0 (sign bit clear, not zero)
                        const uint32_t m2 = mk[c];
                        const uint32_t lo = m2 & 0xFFFFu, hi = m2 >> 16;
                        v0 = (lo != 0u && !(lo & 0x8000u)) ? v0 : 0.f;
                        v1 = (hi != 0u && !(hi & 0x8000u)) ? v1 : 0.f;
                    }
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(v0, v1);
                    pk[c] = *reinterpret_cast<const uint32_t*>(&b2);
                }
                uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(a.out) +
                                                      p * COUT + half * HC);
#pragma unroll
                for (int c = 0; c < HC / 8; ++c)
                    dst[c] = make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
            } else {
                float* dst = reinterpret_cast<float*>(a.out) + p * a.cout_store;
#pragma unroll
                for (int c = 0; c < HC; ++c) {
                    const int ch = half * HC + c;
                    if (ch < a.cout_store)
                        dst[ch] = acc[c] + (a.mode == CONV_BIAS_F32 ? bs[c] : 0.f);
                }
            }
        }
        tc::fence_before_sync();   // the accumulator reads happen before the next barrier
        if (new_band) bslot ^= 1;
        cur = nxt;
    }
    if (ok && __syncthreads_or(timed_out)) ok = false;   // the last tile's wait
    if (!ok) {
        // a wait ran out: record it, give the MMAs in flight one more bounded
        // wait (always the full kWaitLimit, whatever the first wait's limit),
        // then free the tensor memory as on the normal path
        if (tid == 0) atomicExch(a.status, 1);
        for (int i = 0; i < 2; ++i)
            if (pending[i]) tc::mbar_wait(&mbar[i], phase[i], kWaitLimit);
    }
    tc::cp_async_wait_all();
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

// ------------------------------------------------------ weight packing ---
// w [bands][cout][9][cin] FP32 -> B images [bands][COUT x 9 CIN] BF16 in
// core-matrix order; transpose: the image of the transposed convolution
// (rows = cin, K = (tap, cout)), zero where a padded channel has no weight.
__global__ void pack_weights_kernel(const float* w, int bands, int cin, int cout, int CIN, int COUT,
                                    int transpose, __nv_bfloat16* img) {
    const int K = 9 * CIN;
    const size_t total = (size_t)bands * COUT * K;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / ((size_t)COUT * K));
        const int rem = (int)(i - (size_t)b * COUT * K);
        const int row = rem / K, k = rem - row * K;
        const int tp = k / CIN, c = k - tp * CIN;
        float v = 0.f;
        if (!transpose) {   // row = output channel, c = input channel
            if (row < cout && c < cin) v = w[(((size_t)b * cout + row) * 9 + tp) * cin + c];
        } else {            // row = forward input channel, c = forward output channel
            if (row < cin && c < cout) v = w[(((size_t)b * cout + c) * 9 + tp) * cin + row];
        }
        img[(size_t)b * COUT * K + tc::kmajor_offset(row, k, K) / 2] = __float2bfloat16_rn(v);
    }
}

// ------------------------------------------------------ weight gradient ---
// dw[band][co][tap][ci] += sum over the image pixels p of
//   x[p + offset(tap)][ci] dy[p][co]       (zero outside the image)
// db[band][co] += sum_p dy[p][co].  CTA i takes the WGRAD_CHUNK consecutive
// tiles of 128 pixels from i WGRAD_CHUNK on; thread j owns the (co, ci) pairs
// j, j + 256, ... for all nine taps and sums them in FP32 registers over the
// tiles of one band, then stores the sums as record i WGRAD_CHUNK + s of
// `part` (s counts the CTA's bands; pband names each record's band, -1 when
// unused).  wgrad_reduce_kernel adds the records of each band in record
// order: the gradient does not depend on the order in which CTAs finish.
#define WGRAD_CHUNK 2
#define WGRAD_MAX_BANDS 32
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) wgrad_kernel(const __nv_bfloat16* x, const __nv_bfloat16* dy,
                                                    int cin, int cout, const CnnImage* img, int n_img,
                                                    int total_tiles, float* part, int* pband) {
    constexpr int PPT = (COUT * CIN + 255) / 256;   // (co, ci) pairs per thread
    __shared__ float sx[128][CIN + 1];
    __shared__ float sd[128][COUT + 1];
    cudaGridDependencySynchronize();
    const int tid = threadIdx.x;
    const int pairs = cout * cin;
    float acc[9][PPT];
    float accb = 0.f;
    int band = -1, seg = 0;
    const size_t wtot = (size_t)cout * 9 * cin + cout;   // a record: weights, then biases
    auto flush = [&]() {
        if (band < 0) return;
        const size_t rec = (size_t)blockIdx.x * WGRAD_CHUNK + seg;
        float* dst = part + rec * wtot;
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            const int q = tid + j * 256;
            if (q >= pairs) continue;
            const int co = q / cin, ci = q - co * cin;
#pragma unroll
            for (int tp = 0; tp < 9; ++tp) dst[((size_t)co * 9 + tp) * cin + ci] = acc[tp][j];
        }
        if (tid < cout) dst[(size_t)cout * 9 * cin + tid] = accb;
        if (tid == 0) pband[rec] = band;
        ++seg;
    };
    const int t_begin = blockIdx.x * WGRAD_CHUNK;
    const int t_end = min(total_tiles, t_begin + WGRAD_CHUNK);
    for (int t = t_begin; t < t_end; ++t) {
        const CnnImage im = img[find_image(img, n_img, t)];
        if (im.band != band) {   // uniform over the CTA
            flush();
            band = im.band;
#pragma unroll
            for (int tp = 0; tp < 9; ++tp)
#pragma unroll
                for (int j = 0; j < PPT; ++j) acc[tp][j] = 0.f;
            accb = 0.f;
        }
        const int npx = im.h * im.w;
        for (int e = tid; e < 128 * COUT; e += 256) {
            const int c = e % COUT, m = e / COUT;
            const int pl = (t - im.tile0) * 128 + m;
            sd[m][c] = pl < npx ? __bfloat162float(dy[(size_t)(im.off + pl) * COUT + c]) : 0.f;
        }
        for (int tp = 0; tp < 9; ++tp) {
            for (int e = tid; e < 128 * CIN; e += 256) {
                const int c = e % CIN, m = e / CIN;
                const int pl = (t - im.tile0) * 128 + m;
                float v = 0.f;
                if (pl < npx) {
                    const int y = pl / im.w, xx = pl - y * im.w;
                    const int yy = y + tap_dy(tp), x2 = xx + tap_dx(tp);
                    if (yy >= 0 && yy < im.h && x2 >= 0 && x2 < im.w)
                        v = __bfloat162float(x[(size_t)(im.off + yy * im.w + x2) * CIN + c]);
                }
                sx[m][c] = v;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                const int q = tid + j * 256;
                if (q >= pairs) continue;
                const int co = q / cin, ci = q - co * cin;
                float s = 0.f;
#pragma unroll 8
                for (int m = 0; m < 128; ++m) s += sx[m][ci] * sd[m][co];
                acc[tp][j] += s;
            }
            if (tp == 0 && tid < cout)
                for (int m = 0; m < 128; ++m) accb += sd[m][tid];
            __syncthreads();
        }
    }
    flush();
    if (tid == 0)
        for (int s2 = seg; s2 < WGRAD_CHUNK; ++s2) pband[(size_t)blockIdx.x * WGRAD_CHUNK + s2] = -1;
}

// dw[b][w] += sum over the records r with pband[r] == b, in increasing r, of
// part[r][w] (w < cout 9 cin; the biases follow in part and go to db).
__global__ void __launch_bounds__(256) wgrad_reduce_kernel(const float* part, const int* pband,
                                                           int nrec, int cout, int cin, float* dw,
                                                           float* db) {
    __shared__ float sacc[WGRAD_MAX_BANDS][256];
    cudaGridDependencySynchronize();
    const int tid = threadIdx.x;
    const size_t nw = (size_t)cout * 9 * cin, wtot = nw + cout;
    const size_t w = (size_t)blockIdx.x * 256 + tid;
    for (int b = 0; b < WGRAD_MAX_BANDS; ++b) sacc[b][tid] = 0.f;
    unsigned touched = 0u;
    if (w < wtot) {
        for (int r = 0; r < nrec; ++r) {
            const int b = pband[r];
            if (b < 0 || b >= WGRAD_MAX_BANDS) continue;
            sacc[b][tid] += part[(size_t)r * wtot + w];
            touched |= 1u << b;
        }
        while (touched) {
            const int b = __ffs(touched) - 1;
            touched &= touched - 1;
            if (w < nw) dw[(size_t)b * nw + w] += sacc[b][tid];
            else db[(size_t)b * cout + (w - nw)] += sacc[b][tid];
        }
    }
}

// ------------------------------------------------------- input planes ---
// x[p] = (Re r / sqrt(tau), Im r / sqrt(tau), plane, 0, ...) for each pixel
// of each image, with plane = 0.1 ln(tau) (the noise level the network is
// told about); tau = tau[slice][band].
__global__ void cnn_input_kernel(const float2* r, const double* tau, int B, const CnnImage* img,
                                 int n_img, int total_tiles, __nv_bfloat16* x) {
    cudaGridDependencySynchronize();
    const int t = blockIdx.x;
    if (t >= total_tiles) return;
    const CnnImage im = img[find_image(img, n_img, t)];
    const int pl = (t - im.tile0) * 128 + threadIdx.x;
    if (pl >= im.h * im.w) return;
    const int y = pl / im.w, xx = pl - y * im.w;
    const float tv = (float)tau[(size_t)im.slice * B + im.band];   // per-image constants in FP32
    const float is = tv > 0.f ? 1.f / sqrtf(tv) : 0.f;
    const float plane = tv > 0.f ? 0.1f * logf(tv) : 0.f;
    const float2 v = r[(size_t)im.src_off + (size_t)y * im.src_pitch + xx];
    __align__(16) __nv_bfloat16 o[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16_rn(0.f);
    o[0] = __float2bfloat16_rn(v.x * is);
    o[1] = __float2bfloat16_rn(v.y * is);
    o[2] = __float2bfloat16_rn(plane);
    uint4* dst = reinterpret_cast<uint4*>(x + ((size_t)im.off + pl) * 16);
    dst[0] = reinterpret_cast<const uint4*>(o)[0];
    dst[1] = reinterpret_cast<const uint4*>(o)[1];
}

// Rademacher probe: component c (0 re, 1 im) of pixel p of image i is
// +-1 from bit 0 of splitmix64(seed + 2 (image pixel key) + c), the key
// being src_off + y src_pitch + x (the coefficient's packed index).
__device__ __forceinline__ float rademacher(uint64_t seed, uint64_t key, int c) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (2 * key + (uint64_t)c + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (z & 1) ? 1.f : -1.f;
}

__global__ void cnn_probe_kernel(uint64_t seed, const CnnImage* img, int n_img, int total_tiles,
                                 __nv_bfloat16* t0) {
    cudaGridDependencySynchronize();
    const int t = blockIdx.x;
    if (t >= total_tiles) return;
    const CnnImage im = img[find_image(img, n_img, t)];
    const int pl = (t - im.tile0) * 128 + threadIdx.x;
    if (pl >= im.h * im.w) return;
    const int y = pl / im.w, xx = pl - y * im.w;
    const uint64_t key = (uint64_t)im.src_off + (uint64_t)y * im.src_pitch + xx;
    __align__(16) __nv_bfloat16 o[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16_rn(0.f);
    o[0] = __float2bfloat16_rn(rademacher(seed, key, 0));
    o[1] = __float2bfloat16_rn(rademacher(seed, key, 1));
    uint4* dst = reinterpret_cast<uint4*>(t0 + ((size_t)im.off + pl) * 16);
    dst[0] = reinterpret_cast<const uint4*>(o)[0];
    dst[1] = reinterpret_cast<const uint4*>(o)[1];
}

// Per image: f = r - sqrt(tau) n written to the packed array, and the sums
//   rss   = sum |f - r|^2 = tau sum |n|^2,
//   probe = sum eta . (J_n eta)   (if jn != NULL: the network's JVP output)
// accumulated in FP64 per tile and added to sums[2 i], sums[2 i + 1].
__global__ void cnn_output_kernel(const float2* r, const double* tau, int B, const CnnImage* img,
                                  int n_img, int total_tiles, const float* n, const float* jn,
                                  uint64_t seed, float2* f, double* sums) {
    __shared__ double s_rss[4], s_pr[4];
    cudaGridDependencySynchronize();
    const int t = blockIdx.x;
    if (t >= total_tiles) return;
    const int ii = find_image(img, n_img, t);
    const CnnImage im = img[ii];
    const int pl = (t - im.tile0) * 128 + threadIdx.x;
    double rss = 0.0, pr = 0.0;
    if (pl < im.h * im.w) {
        const int y = pl / im.w, xx = pl - y * im.w;
        const float tv = (float)tau[(size_t)im.slice * B + im.band];
        const float st = tv > 0.f ? sqrtf(tv) : 0.f;
        const size_t q = (size_t)im.src_off + (size_t)y * im.src_pitch + xx;
        const size_t p = (size_t)im.off + pl;
        const float n0 = n[2 * p], n1 = n[2 * p + 1];
        const float2 v = r[q];
        const float2 fv = make_float2(v.x - st * n0, v.y - st * n1);
        if (f) f[q] = fv;
        const float e0 = fv.x - v.x, e1 = fv.y - v.y;
        rss = (double)(e0 * e0 + e1 * e1);
        if (jn) {
            const uint64_t key = (uint64_t)im.src_off + (uint64_t)y * im.src_pitch + xx;
            pr = (double)(rademacher(seed, key, 0) * jn[2 * p] +
                          rademacher(seed, key, 1) * jn[2 * p + 1]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rss += __shfl_xor_sync(0xffffffffu, rss, o);
        pr += __shfl_xor_sync(0xffffffffu, pr, o);
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_rss[warp] = rss;
        s_pr[warp] = pr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&sums[2 * ii], s_rss[0] + s_rss[1] + s_rss[2] + s_rss[3]);
        atomicAdd(&sums[2 * ii + 1], s_pr[0] + s_pr[1] + s_pr[2] + s_pr[3]);
    }
}

// Training loss L = sum over images and pixels of |f - w0|^2 / npix_total
// with f = r - sqrt(tau) n; dL/dn = -2 sqrt(tau) (f - w0) / npix_total,
// written as BF16 [pixel][16] (channels 0, 1); loss added to *loss (FP64).
__global__ void cnn_loss_kernel(const float2* r, const float2* w0, const double* tau, int B,
                                const CnnImage* img, int n_img, int total_tiles, const float* n,
                                float inv_count, __nv_bfloat16* dn, double* loss) {
    __shared__ double s_l[4];
    cudaGridDependencySynchronize();
    const int t = blockIdx.x;
    if (t >= total_tiles) return;
    const CnnImage im = img[find_image(img, n_img, t)];
    const int pl = (t - im.tile0) * 128 + threadIdx.x;
    double l = 0.0;
    if (pl < im.h * im.w) {
        const int y = pl / im.w, xx = pl - y * im.w;
        const float tv = (float)tau[(size_t)im.slice * B + im.band];
        const float st = tv > 0.f ? sqrtf(tv) : 0.f;
        const size_t q = (size_t)im.src_off + (size_t)y * im.src_pitch + xx;
        const size_t p = (size_t)im.off + pl;
        const float2 v = r[q], w = w0[q];
        const float e0 = v.x - st * n[2 * p] - w.x, e1 = v.y - st * n[2 * p + 1] - w.y;
        l = ((double)e0 * e0 + (double)e1 * e1) * inv_count;
        __align__(16) __nv_bfloat16 o[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16_rn(0.f);
        o[0] = __float2bfloat16_rn(-2.f * st * e0 * inv_count);
        o[1] = __float2bfloat16_rn(-2.f * st * e1 * inv_count);
        uint4* dst = reinterpret_cast<uint4*>(dn + p * 16);
        dst[0] = reinterpret_cast<const uint4*>(o)[0];
        dst[1] = reinterpret_cast<const uint4*>(o)[1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) s_l[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(loss, s_l[0] + s_l[1] + s_l[2] + s_l[3]);
}

// Adam step on FP32 parameters (bias-corrected, step number t >= 1).
__global__ void adam_kernel(float* p, const float* g, float* m, float* v, size_t n, float lr,
                            float b1, float b2, float eps, int t) {
    // bias corrections 1 / (1 - beta^t), with 1 - beta^t = -expm1(t log1p(beta - 1)):
    // beta - 1 is exact in FP32, and no difference of nearly equal numbers is formed
    // (1 - powf(0.999, 2) would lose four digits)
    const float c1 = -1.f / expm1f((float)t * log1pf(b1 - 1.f));
    const float c2 = -1.f / expm1f((float)t * log1pf(b2 - 1.f));
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}


// Per subband image: the SURE of the network's denoiser,
//   SURE_cnn = sum |f - r|^2 - N_b tau + tau div,  div = 2 N_b - probe
// (div estimated by one Hutchinson probe: probe = eta . J_n eta), against
// the soft threshold's minimum SURE; the smaller one gives w_hat (f, or
// soft(r, theta)) and alpha (div / (2 N_b), or the soft alpha), and
// r~ = (w_hat - alpha r) / (1 - alpha) (Algorithm 1 lines 6-8).
__global__ void cnn_onsager_kernel(const float2* r, const float2* f, const double* tau,
                                   const double* thr, const double* alpha_soft,
                                   const double* sure_soft, int B, const double* sums,
                                   const CnnImage* img, int n_img, int total_tiles, float2* rt,
                                   float2* w_hat, int* use_out, double* alpha_out) {
    __shared__ int s_use;
    __shared__ float s_fa, s_inv, s_th, s_c1, s_c2;
    cudaGridDependencySynchronize();
    const int t = blockIdx.x;
    if (t >= total_tiles) return;
    const int ii = find_image(img, n_img, t);
    const CnnImage im = img[ii];
    const int nb = im.h * im.w;
    const size_t sb = (size_t)im.slice * B + im.band;
    if (threadIdx.x == 0) {   // the per-subband decision, in FP64, once per block
        const double tv = tau[sb];
        const double div = 2.0 * nb - sums[2 * ii + 1];
        const double sure_cnn = sums[2 * ii] - nb * tv + tv * div;
        const double ac = div / (2.0 * nb);
        const bool use = f != nullptr && tv > 0.0 && sure_cnn < sure_soft[sb] && ac >= 0.0 &&
                         ac < 1.0;
        const double al = use ? ac : alpha_soft[sb];
        s_use = use ? 1 : 0;
        s_fa = (float)al;
        const double inv = 1.0 / (1.0 - al);
        s_inv = (float)inv;
        s_th = (float)thr[sb];
        s_c1 = (float)(thr[sb] * inv);   // the soft threshold's line 8 as the plain path
        s_c2 = (float)(al * inv);        // forms it: r (1 - c1 / |r|) above theta, -c2 r below
        if (t == im.tile0) {
            if (use_out) use_out[ii] = use ? 1 : 0;
            if (alpha_out) alpha_out[ii] = al;
        }
    }
    __syncthreads();
    const bool use = s_use != 0;
    const int pl = (t - im.tile0) * 128 + threadIdx.x;
    if (pl >= nb) return;
    const int y = pl / im.w, xx = pl - y * im.w;
    const size_t q = (size_t)im.src_off + (size_t)y * im.src_pitch + xx;
    const float2 v = r[q];
    float2 w;
    if (use) {
        w = f[q];
        rt[q] = make_float2((w.x - s_fa * v.x) * s_inv, (w.y - s_fa * v.y) * s_inv);
    } else {
        const float a = cabs_f(v);
        const float sc = a > s_th ? 1.f - s_th / a : 0.f;
        w = make_float2(__fmul_rn(v.x, sc), __fmul_rn(v.y, sc));
        const float g = a > s_th ? 1.f - s_c1 / a : -s_c2;
        rt[q] = make_float2(__fmul_rn(v.x, g), __fmul_rn(v.y, g));
    }
    if (w_hat) w_hat[q] = w;
}

template <int CIN, int COUT>
cudaError_t launch_conv(const ConvArgs& a, cudaStream_t st) {
    const size_t smem = CONV_STAGES * (size_t)(CIN / 8) * a.nq * 16 + (size_t)COUT * 9 * CIN * 2 +
                        (a.mode == CONV_MASK ? CONV_STAGES * (size_t)128 * COUT * 2 : 0);
    if (smem > 220 * 1024) return cudaErrorInvalidValue;
    static size_t raised = 48 * 1024;   // the attribute only ever grows (process-wide)
    if (smem > raised) {
        cudaError_t e = cudaFuncSetAttribute(conv3x3_kernel<CIN, COUT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        raised = smem;
    }
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::min(a.total_tiles, 2 * sms);
    if (grid < 1) return cudaSuccess;
    return launch_pdl(conv3x3_kernel<CIN, COUT>, dim3(grid), dim3(CONV_THREADS), smem, st, a);
}

}  // namespace
}  // namespace vdamp

using namespace vdamp;

// Device records of vdamp_cnn_wgrad, grown on demand and kept for the process
// (one set for all calls: calls that overlap on the GPU would share it).
static bool wgrad_workspace(size_t floats, size_t ints, float** part, int** pband) {
    static std::mutex mu;
    static float* p = nullptr;
    static int* q = nullptr;
    static size_t np = 0, nq = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (floats > np) {
        if (p) cudaFree(p);
        p = nullptr;
        np = 0;
        if (cudaMalloc(&p, floats * sizeof(float)) != cudaSuccess) return false;
        np = floats;
    }
    if (ints > nq) {
        if (q) cudaFree(q);
        q = nullptr;
        nq = 0;
        if (cudaMalloc(&q, ints * sizeof(int)) != cudaSuccess) return false;
        nq = ints;
    }
    *part = p;
    *pband = q;
    return true;
}

static vdamp_status cnn_fail(const char* msg) {
    vdamp::set_last_error(msg);
    return VDAMP_EINVAL;
}

// Polls of the first wait for a tile's tensor-core result (set per process).
static std::atomic<unsigned> g_wait_limit{kWaitLimit};

extern "C" vdamp_status vdamp_cnn_set_wait_limit(unsigned polls, unsigned* previous) {
    const unsigned old = g_wait_limit.exchange(polls);
    if (previous) *previous = old;
    return VDAMP_OK;
}

extern "C" unsigned vdamp_cnn_default_wait_limit(void) { return kWaitLimit; }

extern "C" vdamp_status vdamp_cnn_status(int* status, void* stream) {
    if (!status) return cnn_fail("vdamp_cnn_status: NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(&h, status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(status, 0, sizeof(int));
    if (e != cudaSuccess) {
        vdamp::set_last_error(cudaGetErrorString(e));
        return VDAMP_ECUDA;
    }
    if (h != 0) {
        vdamp::set_last_error("vdamp_cnn_status: a bounded wait for the tensor cores ran out");
        return VDAMP_ETIMEOUT;
    }
    return VDAMP_OK;
}

extern "C" vdamp_status vdamp_cnn_conv3x3(const void* in, int cin_pad, const void* wimg,
                                          int cout_pad, const float* bias, const void* mask,
                                          void* out, int mode, int mirror, int cout_store,
                                          const int* images, int n_img, int conv_tiles_total,
                                          int max_w, int* status, void* stream) {
    if (!in || !wimg || !out || !images || !status || n_img < 1 || conv_tiles_total < 0 ||
        max_w < 1)
        return cnn_fail("vdamp_cnn_conv3x3: invalid argument");
    if ((cin_pad != 16 && cin_pad != 32) || (cout_pad != 16 && cout_pad != 32))
        return cnn_fail("vdamp_cnn_conv3x3: channels must be 16 or 32");
    if (mode < 0 || mode > 3 || (mode == CONV_MASK && !mask) ||
        ((mode == CONV_BIAS_RELU || mode == CONV_BIAS_F32) && !bias) ||
        (mode >= CONV_BIAS_F32 && (cout_store < 1 || cout_store > cout_pad)))
        return cnn_fail("vdamp_cnn_conv3x3: invalid mode arguments");
    ConvArgs a;
    a.in = (const __nv_bfloat16*)in;
    a.wimg = (const __nv_bfloat16*)wimg;
    a.bias = bias;
    a.mask = (const __nv_bfloat16*)mask;
    a.out = out;
    a.cout_store = cout_store;
    a.img = (const CnnImage*)images;
    a.n_img = n_img;
    a.total_tiles = conv_tiles_total;
    a.nq = conv_halo(conv_block(1, max_w).pitch);
    a.mirror = mirror ? 1 : 0;
    a.mode = mode;
    a.status = status;
    a.wait_limit = g_wait_limit.load();
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (cin_pad == 16 && cout_pad == 32) e = launch_conv<16, 32>(a, st);
    else if (cin_pad == 32 && cout_pad == 32) e = launch_conv<32, 32>(a, st);
    else if (cin_pad == 32 && cout_pad == 16) e = launch_conv<32, 16>(a, st);
    else e = launch_conv<16, 16>(a, st);
    return e == cudaSuccess ? VDAMP_OK : cnn_fail(cudaGetErrorString(e));
}

extern "C" vdamp_status vdamp_cnn_pack_weights(const float* w, int bands, int cin, int cout,
                                               int cin_pad, int cout_pad, int transpose,
                                               void* img, void* stream) {
    if (!w || !img || bands < 1 || cin < 1 || cout < 1)
        return cnn_fail("vdamp_cnn_pack_weights: invalid argument");
    const int rows = transpose ? cin : cout, kc = transpose ? cout : cin;
    if (rows > cout_pad || kc > cin_pad || (cin_pad != 16 && cin_pad != 32) ||
        (cout_pad != 16 && cout_pad != 32))
        return cnn_fail("vdamp_cnn_pack_weights: channels exceed the padding");
    const size_t total = (size_t)bands * cout_pad * 9 * cin_pad;
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
    launch_pdl(pack_weights_kernel, dim3(blocks), dim3(256), 0, (cudaStream_t)stream, w, bands,
               cin, cout, cin_pad, cout_pad, transpose ? 1 : 0, (__nv_bfloat16*)img);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VDAMP_OK : cnn_fail(cudaGetErrorString(e));
}

extern "C" vdamp_status vdamp_cnn_wgrad(const void* x, int cin, int cin_pad, const void* dy,
                                        int cout, int cout_pad, const int* images, int n_img,
                                        int total_tiles, float* dw, float* db, void* stream) {
    if (!x || !dy || !images || !dw || !db || n_img < 1 || cin > cin_pad || cout > cout_pad)
        return cnn_fail("vdamp_cnn_wgrad: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    const CnnImage* im = (const CnnImage*)images;
    if (total_tiles < 1) return VDAMP_OK;
    const int grid = (total_tiles + WGRAD_CHUNK - 1) / WGRAD_CHUNK;
    const int nrec = grid * WGRAD_CHUNK;
    const size_t wtot = (size_t)cout * 9 * cin + cout;
    float* part = nullptr;
    int* pband = nullptr;
    if (!wgrad_workspace((size_t)nrec * wtot, (size_t)nrec, &part, &pband))
        return cnn_fail("vdamp_cnn_wgrad: cannot allocate the gradient records");
    const __nv_bfloat16* xb = (const __nv_bfloat16*)x;
    const __nv_bfloat16* db16 = (const __nv_bfloat16*)dy;
    if (cin_pad == 16 && cout_pad == 32)
        launch_pdl(wgrad_kernel<16, 32>, dim3(grid), dim3(256), 0, st, xb, db16, cin, cout, im,
                   n_img, total_tiles, part, pband);
    else if (cin_pad == 32 && cout_pad == 32)
        launch_pdl(wgrad_kernel<32, 32>, dim3(grid), dim3(256), 0, st, xb, db16, cin, cout, im,
                   n_img, total_tiles, part, pband);
    else if (cin_pad == 32 && cout_pad == 16)
        launch_pdl(wgrad_kernel<32, 16>, dim3(grid), dim3(256), 0, st, xb, db16, cin, cout, im,
                   n_img, total_tiles, part, pband);
    else
        return cnn_fail("vdamp_cnn_wgrad: unsupported channel padding");
    launch_pdl(wgrad_reduce_kernel, dim3((unsigned)((wtot + 255) / 256)), dim3(256), 0, st,
               (const float*)part, (const int*)pband, nrec, cout, cin, dw, db);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VDAMP_OK : cnn_fail(cudaGetErrorString(e));
}

extern "C" vdamp_status vdamp_cnn_input(const float* r, const double* tau, int B,
                                        const int* images, int n_img, int total_tiles, void* x,
                                        void* stream) {
    if (!r || !tau || !images || !x || n_img < 1) return cnn_fail("vdamp_cnn_input: invalid argument");
    if (total_tiles < 1) return VDAMP_OK;
    launch_pdl(cnn_input_kernel, dim3(total_tiles), dim3(128), 0, (cudaStream_t)stream,
               (const float2*)r, tau, B, (const CnnImage*)images, n_img, total_tiles,
               (__nv_bfloat16*)x);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VDAMP_OK : cnn_fail(cudaGetErrorString(e));
}

extern "C" vdamp_status vdamp_cnn_probe(unsigned long long seed, const int* images, int n_img,
                                        int total_tiles, void* t0, void* stream) {
    if (!images || !t0 || n_img < 1) return cnn_fail("vdamp_cnn_probe: invalid argument");
    if (total_tiles < 1) return VDAMP_OK;
    launch_pdl(cnn_probe_kernel, dim3(total_tiles), dim3(128), 0, (cudaStream_t)stream,
               (uint64_t)seed, (const CnnImage*)images, n_img, total_tiles, (__nv_bfloat16*)t0);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VDAMP_OK : cnn_fail(cudaGetErrorString(e));
}

extern "C" vdamp_status vdamp_cnn_output(const float* r, const double* tau, int B,
                                         const int* images, int n_img, int total_tiles,
                                         const float* n, const float* jn, unsigned long long seed,
                                         float* f, double* sums, void* stream) {
    if (!r || !tau || !images || !n || !sums || n_img < 1)
        return cnn_fail("vdamp_cnn_output: invalid argument");
    if (total_tiles < 1) return VDAMP_OK;
    launch_pdl(cnn_output_kernel, dim3(total_tiles), dim3(128), 0, (cudaStream_t)stream,
               (const float2*)r, tau, B, (const CnnImage*)images, n_img, total_tiles, n, jn,
               (uint64_t)seed, (float2*)f, sums);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VDAMP_OK : cnn_fail(cudaGetErrorString(e));
}

extern "C" vdamp_status vdamp_cnn_loss(const float* r, const float* w0, const double* tau, int B,
                                       const int* images, int n_img, int total_tiles,
                                       const float* n, float inv_count, void* dn, double* loss,
                                       void* stream) {
    if (!r || !w0 || !tau || !images || !n || !dn || !loss || n_img < 1)
        return cnn_fail("vdamp_cnn_loss: invalid argument");
    if (total_tiles < 1) return VDAMP_OK;
    launch_pdl(cnn_loss_kernel, dim3(total_tiles), dim3(128), 0, (cudaStream_t)stream,
               (const float2*)r, (const float2*)w0, tau, B, (const CnnImage*)images, n_img,
               total_tiles, n, inv_count, (__nv_bfloat16*)dn, loss);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VDAMP_OK : cnn_fail(cudaGetErrorString(e));
}

extern "C" vdamp_status vdamp_cnn_adam(float* p, const float* g, float* m, float* v, size_t n,
                                       float lr, float beta1, float beta2, float eps, int step,
                                       void* stream) {
    if (!p || !g || !m || !v || step < 1) return cnn_fail("vdamp_cnn_adam: invalid argument");
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 2048);
    if (blocks < 1) return VDAMP_OK;
    launch_pdl(adam_kernel, dim3(blocks), dim3(256), 0, (cudaStream_t)stream, p, g, m, v, n, lr,
               beta1, beta2, eps, step);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VDAMP_OK : cnn_fail(cudaGetErrorString(e));
}

extern "C" vdamp_status vdamp_cnn_onsager(const float* r, const float* f, const double* tau,
                                          const double* thr, const double* alpha_soft,
                                          const double* sure_soft, int B, const double* sums,
                                          const int* images, int n_img, int total_tiles,
                                          float* r_tilde, float* w_hat, int* use_out,
                                          double* alpha_out, void* stream) {
    if (!r || !tau || !thr || !alpha_soft || !sure_soft || !sums || !images || !r_tilde ||
        n_img < 1)
        return cnn_fail("vdamp_cnn_onsager: invalid argument");
    if (total_tiles < 1) return VDAMP_OK;
    launch_pdl(cnn_onsager_kernel, dim3(total_tiles), dim3(128), 0, (cudaStream_t)stream,
               (const float2*)r, (const float2*)f, tau, thr, alpha_soft, sure_soft, B, sums,
               (const CnnImage*)images, n_img, total_tiles, (float2*)r_tilde, (float2*)w_hat,
               use_out, alpha_out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VDAMP_OK : cnn_fail(cudaGetErrorString(e));
}

// Device code of the learned per-subband denoiser: a 5-layer 3x3
// convolutional network per subband index (32 channels, ReLU), applied to
// r_b / sqrt(tau_b) with a tau plane, in residual form
//     f(r) = r - sqrt(tau) n(r / sqrt(tau), tau plane),
// with BF16 weights and activations and FP32 accumulation on the tcgen05
// tensor cores.
//
// Images.  The network runs on a list of "images" (a subband of one slice,
// or a training patch cut from one): image i has h x w pixels stored densely
// in the activation arrays from pixel off on, row-major; its 128-pixel tiles
// (elementwise kernels) are tile0 .. tile0 + ceil(h w / 128) - 1 and its
// convolution tiles (blocks, see conv_block) ctile0 .. ctile0 + conv_tiles(h, w)
// - 1 of the launch.
// src_off and src_pitch locate the image in packed complex arrays (r, w0, f),
// band picks the weight set and slice the per-slice tau.
//
// Activations are BF16 [pixel][C], C = 16 (the input: Re, Im of
// r / sqrt(tau), the tau plane, zeros) or 32; the last layer has 2 output
// channels, computed as 16 (zero weights beyond 2).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "tc_dev.cuh"

namespace vdamp {

struct CnnImage {
    int off, h, w, tile0;
    int src_off, src_pitch, band, slice;
    int ctile0;   // first convolution tile (128 positions of the zero-padded image)
};

enum ConvMode {
    CONV_BIAS_RELU = 0,   // out = relu(acc + bias), BF16
    CONV_MASK = 1,        // out = acc * (mask > 0), BF16   (JVP, backward data)
    CONV_BIAS_F32 = 2,    // out = acc + bias, FP32, first cout_store channels (last layer)
    CONV_F32 = 3          // out = acc, FP32, first cout_store channels (last layer, JVP)
};

struct ConvArgs {
    const __nv_bfloat16* in;     // [npix][CIN]
    const __nv_bfloat16* wimg;   // [bands][COUT x 9 CIN] B operand images (core-matrix order)
    const float* bias;           // [bands][COUT]
    const __nv_bfloat16* mask;   // [npix][COUT] (CONV_MASK)
    void* out;                   // [npix][COUT] BF16, or [npix][cout_store] FP32
    int cout_store;
    const CnnImage* img;         // [n_img]
    int n_img;
    int total_tiles;             // convolution tiles of all images
    int nq;                      // halo positions per stage: conv_halo(largest pitch)
    int mirror;                  // 1: neighbour offsets negated (transposed convolution)
    int mode;
    int* status;                 // [0] set to 1 when a bounded wait ran out
    unsigned wait_limit;         // polls of a tensor-core wait before it gives up
};

// Neighbour offset (dy, dx) of tap t = 3 (dy + 1) + (dx + 1).
__device__ __forceinline__ int tap_dy(int t) { return t / 3 - 1; }
__device__ __forceinline__ int tap_dx(int t) { return t % 3 - 1; }

__device__ __forceinline__ int find_image(const CnnImage* img, int n, int tile) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (img[mid].tile0 <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_conv_image(const CnnImage* img, int n, int tile) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (img[mid].ctile0 <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Convolution tiles.  An h x w image is cut into blocks of R rows x Wb
// columns, Wb = min(w, 30), each computed from a zero-padded halo of pitch
// P = Wb + 2: MMA row m is the halo position P + 1 + m, so the 128 rows cover
// R = floor(128 / P) block rows (the pad columns and the rows past R are
// computed and dropped).  The halo holds positions 0 .. 2P + 129 (the reach
// of the nine taps from the 128 rows).
struct ConvBlock {
    int wb, pitch, rows, nbx;
};
__host__ __device__ inline ConvBlock conv_block(int h, int w) {
    ConvBlock b;
    b.wb = w < 30 ? w : 30;
    b.pitch = b.wb + 2;
    b.rows = 128 / b.pitch;
    b.nbx = (w + b.wb - 1) / b.wb;
    (void)h;
    return b;
}
__host__ __device__ inline int conv_tiles(int h, int w) {
    const ConvBlock b = conv_block(h, w);
    return b.nbx * ((h + b.rows - 1) / b.rows);
}
__host__ __device__ inline int conv_halo(int pitch) { return 2 * pitch + 130; }

}  // namespace vdamp

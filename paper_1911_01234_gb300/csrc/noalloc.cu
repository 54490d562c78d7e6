// vdamp_tau_estimate_noalloc: the colored noise estimate tau of the VDAMP
// iteration, computed from a k-space residual z without allocating any
// device memory.  The paper has no such entry point; it is a service of the
// library for callers that cannot allocate.
//
// Some callers cannot call cudaMalloc: code that runs inside a fixed device
// memory pool or budget, allocator-less embedded or real-time hosts, and
// tools that must not disturb a caching allocator they share with other
// code.  For them this file keeps all of the call's device scratch (the
// separable S tables and the per-CTA partial sums) in one file-scope
// __device__ array of fixed size.  Every GPU that loads the library holds
// that array until the process exits.
//
// The tables are filled on the device by a kernel whose only inputs are the
// wavelet's filter taps and the sizes, passed by value: the call reads no
// host buffer after it returns, and calls on one stream see their own tables
// in stream order.  The tau kernel is a variant of the tau stage of the
// column pass: the same per-frequency term p^-1 ((p^-1 - 1)|z|^2 + sigma^2)
// weighted by the subband spectra, FP32 per thread, FP64 across warps and
// CTAs.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/vdamp.h"
#include "vdamp_internal.cuh"

namespace {

constexpr int kMaxSide = VDAMP_NOALLOC_MAX_SIDE;
constexpr int kSpecFloats = 2 * 2 * VDAMP_MAX_LEVELS * kMaxSide;   // y and x tables
constexpr int kMaxParts = kMaxSide / 2;                              // columns per CTA >= 2
constexpr size_t kSpecBytes = (size_t)kSpecFloats * sizeof(float);
constexpr size_t kPartBytes = (size_t)kMaxParts * VDAMP_MAX_BANDS * sizeof(double);
constexpr size_t kScratchBytes = kSpecBytes + kPartBytes;

// The shared scratch: spectra tables first, then the partial sums.  In host
// code this name is only a stand-in; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

struct TauArgs {
    const float2* z;
    const uint8_t* mask;
    const float* density;
    float sigma;
    int ny, nx, cb, ntypes, B;
    int ty[VDAMP_MAX_BANDS];
    int tx[VDAMP_MAX_BANDS];
    const float* ey;   // [ntypes][ny] inside the scratch
    const float* ex;   // [ntypes][nx] inside the scratch
    double* part;      // [nx / cb][B] inside the scratch
};

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Filter taps of the wavelet, by value (a kernel parameter).
struct FilterTaps {
    double h[VDAMP_MAX_TAPS];
    int L;
};

// |sum_k f[k] e^{-i 2 pi k m / n}|^2 for integer frequency m (argument reduced
// exactly: the phase of tap k is ((k m) mod n) / n of a turn).
__device__ double resp2_dev(const double* f, int L, long long m, int n) {
    double re = 0.0, im = 0.0;
    for (int k = 0; k < L; ++k) {
        double s, c;
        sincospi(2.0 * (double)((k * m) % n) / (double)n, &s, &c);
        re += f[k] * c;
        im -= f[k] * s;
    }
    return re * re + im * im;
}

// The 1D factors of S along an axis of length n (the same quantity as the
// plan's host tables): entry (2 (j - 1) + t) n + k is |F_n psi|^2 at frequency
// k of the level-j scaling (t = 0) or wavelet (t = 1) atom.  The level-j atoms
// have DTFT prod_{l<j} H(2^l w) and G(2^{j-1} w) prod_{l<j-1} H(2^l w),
// sampled at w = 2 pi k / n (the unitary DFT of the periodised atom).
// Grid-stride over k; one thread per frequency.
__global__ void spectra_noalloc_kernel(FilterTaps ft, int levels, int n, float* out) {
    double g[VDAMP_MAX_TAPS];
    for (int k = 0; k < ft.L; ++k) g[k] = ((k & 1) ? -1.0 : 1.0) * ft.h[ft.L - 1 - k];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        double low = 1.0;   // prod over the coarser factors so far
        long long m = k;
        for (int j = 1; j <= levels; ++j) {
            out[(2 * (j - 1) + 1) * n + k] = (float)(low * resp2_dev(g, ft.L, m, n) / n);
            low *= resp2_dev(ft.h, ft.L, m, n);
            out[(2 * (j - 1)) * n + k] = (float)(low / n);
            m = (2 * m) % n;
        }
    }
}

__global__ void tau_part_noalloc_kernel(TauArgs a) {
    __shared__ float red[32][VDAMP_MAX_BANDS];
    const int cb = a.cb, ny = a.ny, nx = a.nx;
    const int c0 = blockIdx.x * cb;
    const int tid = threadIdx.x;
    const int cnt = ny * cb;
    const float sig2 = a.sigma * a.sigma;
    float q[2 * VDAMP_MAX_LEVELS];
#pragma unroll
    for (int t = 0; t < 2 * VDAMP_MAX_LEVELS; ++t) q[t] = 0.f;
    for (int idx = tid; idx < cnt; idx += blockDim.x) {
        const int c = idx % cb, i = idx / cb;
        const size_t g = (size_t)i * nx + c0 + c;
        const bool m = a.mask[g] != 0;
        const float2 z = m ? a.z[g] : make_float2(0.f, 0.f);
        const float w = m ? 1.0f / a.density[g] : 0.f;
        const float v = w * ((w - 1.0f) * (z.x * z.x + z.y * z.y) + sig2);
#pragma unroll
        for (int t = 0; t < 2 * VDAMP_MAX_LEVELS; ++t)
            if (t < a.ntypes) q[t] += a.ey[t * ny + i] * v;
    }
    const int kx = c0 + tid % cb;
    const int warp = tid >> 5, lane = tid & 31;
    for (int b = 0; b < a.B; ++b) {
        float val = 0.f;
        if (tid < cnt) {
#pragma unroll
            for (int t = 0; t < 2 * VDAMP_MAX_LEVELS; ++t)
                if (t == a.ty[b]) val = a.ex[a.tx[b] * nx + kx] * q[t];
        }
        val = warp_sum_f(val);
        if (lane == 0) red[warp][b] = val;
    }
    __syncthreads();
    if (tid < a.B) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += (double)red[w][tid];
        a.part[(size_t)blockIdx.x * a.B + tid] = s;
    }
}

__global__ void tau_reduce_noalloc_kernel(const double* part, int nparts, int B, double* tau) {
    const int b = threadIdx.x;
    if (b >= B) return;
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += part[(size_t)p * B + b];
    tau[b] = s;
}

vdamp_status bad(vdamp_status st, const char* msg) {
    char buf[256];
    snprintf(buf, sizeof(buf), "vdamp_tau_estimate_noalloc: %s", msg);
    vdamp::set_last_error(buf);
    return st;
}

vdamp_status bad_cuda(const char* what, cudaError_t e) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return bad(VDAMP_ECUDA, buf);
}

bool radix_ok(int n) {
    for (int f : {2, 3, 5})
        while (n % f == 0) n /= f;
    return n == 1;
}

}  // namespace

extern "C" vdamp_status vdamp_tau_estimate_noalloc(int ny, int nx, int wavelet, int levels,
                                                   const float* z, const uint8_t* mask,
                                                   const float* density, float sigma,
                                                   double* tau, void* stream) {
    if (wavelet != VDAMP_HAAR && wavelet != VDAMP_DB4) return bad(VDAMP_EINVAL, "bad wavelet");
    if (levels < 1 || levels > VDAMP_MAX_LEVELS) return bad(VDAMP_EINVAL, "levels outside [1, 6]");
    if (ny < 8 || nx < 8 || !radix_ok(ny) || !radix_ok(nx) || (ny % (1 << levels)) ||
        (nx % (1 << levels)))
        return bad(VDAMP_EINVAL, "ny, nx must be 2^a 3^b 5^c >= 8 and divisible by 2^levels");
    if (ny > kMaxSide || nx > kMaxSide)
        return bad(VDAMP_EINVAL, "ny or nx above the scratch limit VDAMP_NOALLOC_MAX_SIDE");
    if (!z || !mask || !density || !tau) return bad(VDAMP_EINVAL, "a pointer is NULL");
    if (!(sigma >= 0.f) || !std::isfinite(sigma)) return bad(VDAMP_EINVAL, "sigma must be >= 0");

    // An error left by earlier work (asynchronous, or sticky) is reported as
    // such, before anything is launched, and not cleared.
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return bad_cuda("an earlier CUDA error is pending", e);

    // Set-up, once per device with that device current: the device address of
    // the scratch array.
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return bad(VDAMP_ECUDA, "cudaGetDevice failed or device index too large");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) return bad_cuda("cudaGetSymbolAddress", e);
            g_scratch_addr[dev] = ptr;
        }
        base = g_scratch_addr[dev];
    }
    float* ey = (float*)base;
    float* ex = ey + 2 * VDAMP_MAX_LEVELS * kMaxSide;
    double* part = (double*)((unsigned char*)base + kSpecBytes);

    // S factors for this call, filled on the device over the previous call's
    // tables (calls on one stream are ordered; the taps travel by value).
    const int nt = 2 * levels;
    FilterTaps ft;
    if (vdamp_wavelet_filter(wavelet, ft.h, &ft.L) != VDAMP_OK) return bad(VDAMP_EINVAL, "filter");
    cudaStream_t st = (cudaStream_t)stream;
    spectra_noalloc_kernel<<<(ny + 127) / 128, 128, 0, st>>>(ft, levels, ny, ey);
    spectra_noalloc_kernel<<<(nx + 127) / 128, 128, 0, st>>>(ft, levels, nx, ex);
    if ((e = cudaGetLastError()) != cudaSuccess) return bad_cuda("table launch failed", e);

    TauArgs a;
    a.z = (const float2*)z;
    a.mask = mask;
    a.density = density;
    a.sigma = sigma;
    a.ny = ny;
    a.nx = nx;
    int cb = 8;
    while (nx % cb) cb >>= 1;
    a.cb = cb;
    a.ntypes = nt;
    a.B = 1 + 3 * levels;
    a.ty[0] = a.tx[0] = 2 * (levels - 1);
    int b = 1;
    for (int j = levels; j >= 1; --j) {
        const int lo = 2 * (j - 1), hi = lo + 1;
        const int tys[3] = {lo, hi, hi}, txs[3] = {hi, lo, hi};  // H, V, D
        for (int q = 0; q < 3; ++q, ++b) {
            a.ty[b] = tys[q];
            a.tx[b] = txs[q];
        }
    }
    a.ey = ey;
    a.ex = ex;
    a.part = part;
    const int nparts = nx / cb;
    int threads = ny * cb / 4;
    threads = threads < 64 ? 64 : (threads > 512 ? 512 : threads);
    threads = (threads + 31) / 32 * 32;
    tau_part_noalloc_kernel<<<nparts, threads, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return bad_cuda("partials launch failed", e);
    tau_reduce_noalloc_kernel<<<1, 32, 0, st>>>(part, nparts, a.B, tau);
    if ((e = cudaGetLastError()) != cudaSuccess) return bad_cuda("reduce launch failed", e);
    return VDAMP_OK;
}

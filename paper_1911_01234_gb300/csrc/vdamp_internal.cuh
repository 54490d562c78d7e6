// Internal declarations shared by the VDAMP CUDA translation units.
//
// Data layout (all per slice, slices contiguous):
//   image / k-space : float2 [ny][nx], k-space unshifted
//   packed wavelet  : float2 [ny*nx], subbands A_s, H_s, V_s, D_s, ..., D_1
//   coef            : float4 [B] per slice = (theta, theta/(1-alpha),
//                     alpha/(1-alpha), 0), from FP64: what the denoiser of
//                     the previous iteration chose
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#define VDAMP_MAX_LEVELS 6
#define VDAMP_MAX_BANDS (1 + 3 * VDAMP_MAX_LEVELS)
#define VDAMP_MAX_TAPS 8
#define VDAMP_MAX_STAGES 12

namespace vdamp {

// ---------------------------------------------------------------- complex ---
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// Product rounded on its own (never fused into a following add), so that a
// value formed here and one read back from memory are the same bits.
__device__ __forceinline__ float2 cscale_rn(float2 a, float s) {
    return make_float2(__fmul_rn(a.x, s), __fmul_rn(a.y, s));
}

// |v| as the SURE searches key it (correctly rounded square root).  The
// transforms' threshold tests (src_apply) compare squares instead: the maps
// they apply are continuous at |v| = theta, so the two may disagree on a
// coefficient only where the outcome differs by rounding.
__device__ __forceinline__ float cabs_f(float2 v) {
    return sqrtf(__fmaf_rn(v.x, v.x, __fmul_rn(v.y, v.y)));
}

// Strided loop over idx = start, start + step, ... < cnt in chunks of U:
// the U loads of a chunk are all issued before any of their stores, so a
// thread waits for one memory round trip per chunk instead of one per element.
template <int U, class T, class LoadF, class StoreF>
__device__ __forceinline__ void batched_for(int start, int cnt, int step, LoadF load,
                                            StoreF store) {
    for (int base = start; base < cnt; base += U * step) {
        T v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * step;
            if (idx < cnt) v[u] = load(idx);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * step;
            if (idx < cnt) store(idx, v[u]);
        }
    }
}

// ----------------------------------------------------------------- params ---
struct Filt {
    float h[VDAMP_MAX_TAPS];
    float g[VDAMP_MAX_TAPS];
    int L;
};

struct FftAxis {
    int n;
    int nstages;
    int radix[VDAMP_MAX_STAGES];
    const float2* tw;  // device, tw[k] = exp(-2 pi i k / n)
};

// SMs of the current device (read once per process).
inline int device_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
            sms = n;
        else
            return 1;
    }
    return sms;
}

inline int max_radix(const FftAxis& ax) {
    int r = 2;
    for (int s = 0; s < ax.nstages; ++s) r = ax.radix[s] > r ? ax.radix[s] : r;
    return r;
}

// How a transform forms the coefficient it reads from a packed array.
enum SrcMode {
    SRC_ZERO = 0,      // r~ = 0 (Algorithm 1 line 1)
    SRC_EXPLICIT = 1,  // r~ read as given
    SRC_LINE8 = 2,     // r~ = (soft(r, theta) - alpha r) / (1 - alpha) (line 8)
    SRC_SOFT = 3       // w_hat = soft(r, theta) (line 6, for the return line)
};

struct SrcSpec {
    int mode;
    const float2* r;     // packed base (slice 0)
    const float4* coef;  // [batch][B]
    int B;
};

// The coefficient a source forms from the stored value v of subband b, whose
// denoiser parameters are c = coef[slice][b].
// |r| > theta is tested on the squares and 1/|r| is one reciprocal square
// root (a few ulp): both maps are continuous at |r| = theta, so a rounding-level
// difference in the test moves the result only by rounding.
__device__ __forceinline__ float2 src_apply(int mode, float2 v, float4 c) {
    if (mode == SRC_ZERO) return make_float2(0.f, 0.f);
    if (mode == SRC_EXPLICIT) return v;
    const float a2 = __fmaf_rn(v.x, v.x, __fmul_rn(v.y, v.y));
    const bool above = a2 > c.x * c.x;   // theta >= 0
    const float inv = rsqrtf(a2);        // used only above theta, where a2 > 0
    if (mode == SRC_SOFT) return cscale_rn(v, above ? 1.f - c.x * inv : 0.f);
    // (soft(r) - alpha r) / (1 - alpha) = r (1 - c1 / |r|) above theta, -c2 r below
    return cscale_rn(v, above ? 1.f - c.y * inv : -c.z);
}

__device__ __forceinline__ float4 src_coef(const SrcSpec& s, int slice, int b) {
    return (s.mode == SRC_LINE8 || s.mode == SRC_SOFT) ? s.coef[slice * s.B + b]
                                                        : make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ float2 src_value(const SrcSpec& s, int slice, size_t N, size_t idx,
                                            int b) {
    if (s.mode == SRC_ZERO) return make_float2(0.f, 0.f);
    float2 v = s.r[(size_t)slice * N + idx];
    if (s.mode == SRC_EXPLICIT) return v;
    return src_apply(s.mode, v, s.coef[slice * s.B + b]);
}

// Column-pass modes of the fused k-space kernel.
enum ColMode {
    COL_FWD = 0,    // out = F-column of in, scaled (plain transform)
    COL_INV = 1,    // out = inverse F-column of in, scaled (plain transform)
    COL_ITER = 2,   // U = F u; z = m(y - U); tau partials; out = F^H-column (w z)
    COL_FINAL = 3   // U = F u; out = F^H-column (m y + (1-m) U)
};

// One sampled frequency of a column (the compacted k-space inputs of a solve):
// its row, P^-1 = 1/p rounded once, and the measurement y.
struct __align__(16) KEntry {
    int row;
    float w;
    float2 y;
};

struct ColArgs {
    const float2* in;    // row-transformed data [batch][ny][nx] (ignored if u_zero)
    float2* out;         // [batch][ny][nx]
    int ny, nx, cb;      // cb = columns per CTA
    int plan_batch;      // the plan's largest batch (sets the launch's threads; 0: the call's)
    FftAxis ax;          // along y
    int mode;
    int u_zero;          // 1: the image is zero, skip the forward transform
    float scale_fwd;     // applied after the forward column transform
    float scale_inv;     // applied after the inverse column transform
    const float2* y;
    const uint8_t* mask;
    const float* density;
    const float* sigma;  // device [batch]
    // tau (Algorithm 1 line 5): tau_b = sum_k Ey[ty_b][ky] Ex[tx_b][kx] v(k)
    const float* ey;     // [2 levels][ny]
    const float* ex;     // [2 levels][nx]
    int ntypes;          // 2 levels
    int B;
    int ty[VDAMP_MAX_BANDS];
    int tx[VDAMP_MAX_BANDS];
    double* tau_part;    // [batch][nx / cb][B]
    // the sampled entries, compacted once per solve (NULL: read y, mask, density densely):
    // klist[slice][cblk][c][ny] (column c of block cblk, rows ascending), kcnt[slice][cblk][c]
    const KEntry* klist;
    const int* kcnt;
};

struct DwtArgs {   // one analysis level: image (H x W) -> four (H/2 x W/2) bands
    const float2* in;
    size_t in_stride;
    int H, W;
    float2* ll_out;    // dense LL (when not last)
    size_t ll_stride;
    int last;          // 1: LL is A_s and goes to the packed array
    float2* packed;    // packed output base
    size_t N;
    int off[4];        // packed offsets of A (if last), H, V, D
    int band[4];       // subband indices of A, H, V, D
    SrcSpec src;       // r~ added to every packed output (ZERO for plain Psi)
    Filt f;
    int to;            // tile side (output coefficients)
};

struct IdwtArgs {  // one synthesis level: four (h x w) bands -> image (2h x 2w)
    const float2* ll_in;  // dense LL (when not first)
    size_t ll_stride;
    int h, w;
    int first;            // 1: LL is A_s, read from the packed source
    float2* out;
    size_t out_stride;
    size_t N;
    int off[4];
    int band[4];
    SrcSpec src;          // how packed coefficients are formed
    Filt f;
    int to;               // tile side (output pixels, even)
};

struct SureArgs {
    const float2* r;      // packed r_k
    float* sorted;        // [batch][N] scratch: |r_k| sorted within each subband
    size_t N;
    int B;
    int off[VDAMP_MAX_BANDS + 1];
    const double* tau_part;  // [batch][nparts][B]
    int nparts;
    int iters, k;         // output row
    double* tau_out;      // [batch][iters][B]
    double* thr_out;
    double* alpha_out;
    float4* coef;         // [batch][B]
    int* status;          // [0] code, [1] first bad iteration
    int max_parts;        // sort parts per subband at most (1 when slices fill the GPU)
    double4_32a* partrec; // [batch][B][SURE_MAX_PARTS] (first, end, sum a^2, sum 1/a) of a part
    double4_32a* bestrec; // [batch][B][SURE_MAX_PARTS] (SURE, theta, H, m) of a part's best
    unsigned* counter;    // [batch][B] search parts done (returns to 0 after each search)
    double* sure_out;     // [batch][B] minimum SURE of the last search
    int* fallback;        // [3 + batch B]: subbands the pruned search leaves to the full sort
    // the split search's subbands: b_top, b_top - 1, ..., b_top - nb_launch + 1; the
    // pruned search's CTAs of a slice: items item0 .. item0 + nb_launch - 1
    int b_top, nb_launch, item0;
};

struct Line8Args {
    SrcSpec src;
    float2* out;
    size_t N;
    int B;
    int off[VDAMP_MAX_BANDS + 1];
};

// Launch with programmatic dependent launch: the kernel may be scheduled while
// its predecessor on the stream drains; every kernel of this library calls
// cudaGridDependencySynchronize() before its first global memory access, so
// it still sees all of the predecessor's writes.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// --------------------------------------------------------------- launchers ---
// All return cudaGetLastError() after the launch.
cudaError_t launch_fft_rows(const float2* in, float2* out, int ny, int nx, int batch,
                            const FftAxis& ax, int inverse, float scale, int rows_per_cta,
                            int plan_batch, cudaStream_t st);
cudaError_t launch_col_pass(const ColArgs& a, int batch, cudaStream_t st);
// Compacts the sampled entries of every column block (a.mask, a.density, a.y) into
// a.klist / a.kcnt for the column passes of one solve.
cudaError_t launch_kspace_list(const ColArgs& a, int batch, cudaStream_t st);
size_t col_pass_smem(int ny, int cb, int ntypes);
cudaError_t launch_dwt_level(const DwtArgs& a, int batch, cudaStream_t st);
cudaError_t launch_idwt_level(const IdwtArgs& a, int batch, cudaStream_t st);
// fallback_ctas: grid of the fallback kernel that follows the pruned search
// (max_parts == 1); one wave of CTAs.
cudaError_t launch_sure(const SureArgs& a, int batch, int max_band, int fallback_ctas,
                        cudaStream_t st);
size_t sure_smem(int max_band);
cudaError_t launch_line8(const Line8Args& a, int batch, cudaStream_t st);
cudaError_t configure_col_pass(size_t smem_bytes);
cudaError_t configure_fft_rows(size_t smem_bytes);
cudaError_t configure_sure(size_t smem_bytes);
cudaError_t configure_dwt(size_t smem_bytes);

// Scales lo .. s of Psi^H (coarse to fine) or of Psi (fine to coarse) in one
// launch: one thread-block cluster of `cluster` CTAs per slice, the tiles of a
// scale spread over the cluster, a cluster barrier between scales.
struct WaveletArgs {
    IdwtArgs idwt[VDAMP_MAX_LEVELS];   // level j at [j - 1]
    DwtArgs dwt[VDAMP_MAX_LEVELS];
    int levels;                        // scales lo .. levels in this launch
    int lo;
};
cudaError_t configure_wavelet_cluster(int cluster, size_t smem, int* max_clusters);
cudaError_t launch_psi_h_cluster(const WaveletArgs& w, int batch, int cluster, size_t smem,
                                 cudaStream_t st);
cudaError_t launch_psi_cluster(const WaveletArgs& w, int batch, int cluster, size_t smem,
                               cudaStream_t st);
void set_last_error(const char* msg);  // text returned by vdamp_last_error()

}  // namespace vdamp

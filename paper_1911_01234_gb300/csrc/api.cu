// C ABI of the VDAMP library: plans, table setup and the launch sequence of
// Algorithm 1.  See include/vdamp.h for the contract of every entry point.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/vdamp.h"
#include "dwt_dev.cuh"
#include "fft_dev.cuh"
#include "fused.cuh"
#include "sure_prune_dev.cuh"   // (includes sure_dev.cuh)

using vdamp::FftAxis;
using vdamp::Filt;
using vdamp::SrcSpec;

// ------------------------------------------------------------- errors ---
static thread_local std::string g_last_error;

static vdamp_status fail(vdamp_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

#define CUDA_TRY(expr)                                                                    \
    do {                                                                                  \
        cudaError_t _e = (expr);                                                          \
        if (_e != cudaSuccess)                                                            \
            return fail(VDAMP_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

// ------------------------------------------- filters (Daubechies 1988) ---
using cd = std::complex<double>;

static std::vector<cd> conv(const std::vector<cd>& a, const std::vector<cd>& b) {
    std::vector<cd> o(a.size() + b.size() - 1, cd(0.0, 0.0));
    for (size_t i = 0; i < a.size(); ++i)
        for (size_t j = 0; j < b.size(); ++j) o[i + j] += a[i] * b[j];
    return o;
}

// Minimum-phase Daubechies low-pass filter with p vanishing moments (2p taps):
// |H(w)|^2 = 2 cos^{2p}(w/2) P(sin^2(w/2)), P(y) = sum_{k<p} C(p-1+k, k) y^k.
// The roots of P are found by Durand-Kerner iteration; each root y_r gives
// z^2 - (2 - 4 y_r) z + 1 = 0 whose root inside the unit circle is kept.
static void daubechies(int p, double* h) {
    std::vector<cd> poly{cd(1.0, 0.0)};
    for (int i = 0; i < p; ++i) poly = conv(poly, {cd(0.5, 0.0), cd(0.5, 0.0)});
    if (p > 1) {
        const int d = p - 1;
        std::vector<double> c(p);
        for (int k = 0; k < p; ++k) {
            double b = 1.0;  // C(p-1+k, k)
            for (int i = 1; i <= k; ++i) b = b * (p - 1 + i) / i;
            c[k] = b;
        }
        auto eval = [&](cd y) {
            cd acc(0.0, 0.0);
            for (int k = d; k >= 0; --k) acc = acc * y + c[k];
            return acc / c[d];
        };
        std::vector<cd> z(d);
        const cd seed(0.4, 0.9);
        cd pw(1.0, 0.0);
        for (int i = 0; i < d; ++i) {
            z[i] = pw;
            pw *= seed;
        }
        for (int it = 0; it < 1000; ++it) {
            double delta = 0.0;
            for (int i = 0; i < d; ++i) {
                cd den(1.0, 0.0);
                for (int j = 0; j < d; ++j)
                    if (j != i) den *= (z[i] - z[j]);
                cd step = eval(z[i]) / den;
                z[i] -= step;
                delta = std::max(delta, std::abs(step));
            }
            if (delta < 1e-16) break;
        }
        for (int i = 0; i < d; ++i) {
            cd b = 2.0 - 4.0 * z[i];
            cd disc = std::sqrt(b * b - 4.0);
            cd z1 = (b + disc) / 2.0, z2 = (b - disc) / 2.0;
            cd zr = std::abs(z1) < 1.0 ? z1 : z2;
            poly = conv(poly, {cd(1.0, 0.0), -zr});
            for (auto& q : poly) q /= (1.0 - zr);
        }
    }
    for (int k = 0; k < 2 * p; ++k) h[k] = std::sqrt(2.0) * poly[k].real();
}

static int wavelet_taps(int wavelet) {
    if (wavelet == VDAMP_HAAR) return 2;
    if (wavelet == VDAMP_DB4) return 8;
    return 0;
}

static double resp2(const double* f, int L, double w) {
    double re = 0.0, im = 0.0;
    for (int k = 0; k < L; ++k) {
        re += f[k] * std::cos(w * k);
        im -= f[k] * std::sin(w * k);
    }
    return re * re + im * im;
}

// 1D factors of S = |Phi Psi^H|^2 (Algorithm 1 line 1).  The level-j atoms
// have DTFT prod_{l<j} H(2^l w) (scaling) and G(2^{j-1} w) prod_{l<j-1} H(2^l w)
// (wavelet); the unitary DFT of the periodised atom samples it at 2 pi k / n.
static void spectra(const double* h, int L, int levels, int n, double* out) {
    double g[VDAMP_MAX_TAPS];
    for (int k = 0; k < L; ++k) g[k] = ((k & 1) ? -1.0 : 1.0) * h[L - 1 - k];
    const double two_pi = 2.0 * 3.14159265358979323846;
    for (int k = 0; k < n; ++k) {
        double low = 1.0;  // prod_{l < j-1} |H(2^l w)|^2
        long long m = k;
        for (int j = 1; j <= levels; ++j) {
            const double w = two_pi * (double)(m % n) / n;
            out[(2 * (j - 1) + 1) * n + k] = low * resp2(g, L, w) / n;
            low *= resp2(h, L, w);
            out[(2 * (j - 1)) * n + k] = low / n;
            m = (2 * m) % n;
        }
    }
}

// ----------------------------------------------------------- fft plan ---
// Radix plan of an n-point transform (n = 2^a 3^b 5^c).  Variant 0: radix 8
// first (then 4, 4 / 4 / 2), then 3s and 5s; variant 1: radix 4 (one 2 for an
// odd power of two), then 3s and 5s; variant 2: variant 0 with the odd radices
// first.
static bool fft_radices(int n, int* radix, int* nst, int variant = 0) {
    int m = n, a = 0;
    while (m % 2 == 0) { m /= 2; ++a; }
    int p2[VDAMP_MAX_STAGES], n2 = 0;
    if (variant == 1) {
        for (int i = 0; i < a / 2; ++i) p2[n2++] = 4;
        if (a & 1) p2[n2++] = 2;
    } else {
        int e8 = a / 3, rem = a % 3;
        if (rem == 1 && e8 > 0) { --e8; rem = 4; }
        for (int i = 0; i < e8; ++i) p2[n2++] = 8;
        if (rem == 4) { p2[n2++] = 4; p2[n2++] = 4; }
        else if (rem == 2) p2[n2++] = 4;
        else if (rem == 1) p2[n2++] = 2;
    }
    int odd[VDAMP_MAX_STAGES], no = 0;
    while (m % 3 == 0) { odd[no++] = 3; m /= 3; }
    while (m % 5 == 0) { odd[no++] = 5; m /= 5; }
    if (m != 1 || n2 + no > VDAMP_MAX_STAGES) return false;
    int s = 0;
    if (variant == 2)
        for (int i = 0; i < no; ++i) radix[s++] = odd[i];
    for (int i = 0; i < n2; ++i) radix[s++] = p2[i];
    if (variant != 2)
        for (int i = 0; i < no; ++i) radix[s++] = odd[i];
    *nst = s;
    return true;
}

// -------------------------------------------------------------- plan ---
namespace {
struct GraphKey {
    int kind, batch, iters;
    const void* p[12];
    bool operator==(const GraphKey& o) const {
        if (kind != o.kind || batch != o.batch || iters != o.iters) return false;
        for (int i = 0; i < 12; ++i)
            if (p[i] != o.p[i]) return false;
        return true;
    }
};
struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec;
    int launches;
};
struct SigmaBlock {
    int n;
    float v[512];
};
__global__ void set_sigma_kernel(float* dst, SigmaBlock b) {
    cudaGridDependencySynchronize();
    if ((int)threadIdx.x < b.n) dst[threadIdx.x] = b.v[threadIdx.x];
}
}  // namespace

struct vdamp_plan {
    int ny, nx, levels, wavelet, B, max_batch, max_iters;
    int last_k0 = 0;                   // k0 of the last solve (added to reported iterations)
    size_t N;
    Filt filt;
    FftAxis axy, axx;
    int off[VDAMP_MAX_BANDS + 1];
    int ty[VDAMP_MAX_BANDS], tx[VDAMP_MAX_BANDS];
    int cb, nparts, rpc;
    int idwt_to = 32, dwt_to = 16;     // wavelet tile sides
    size_t smem_col = 0, smem_rows = 0, smem_dwt = 0;  // attributes raised for the tuner's choices
    int radix_var[2] = {0, 0};         // radix plan variant along y, x
    int wcluster = 0;                  // CTAs of the one-launch wavelet cluster (0: unavailable)
    int use_wcluster = 0;              // tuning: coarse scales in one cluster launch (1: small
                                       // batches, scales s..2; 2: any batch, scales s..coarse_lo)
    int sure_parts = 0;                // tuning: SURE parts per subband (0: by batch size)
    int num_sms = 152;
    float* ey = nullptr;
    float* ex = nullptr;
    float2* tw_y = nullptr;
    float2* tw_x = nullptr;
    float2* u = nullptr;
    float2* kbuf = nullptr;
    float2* ll0 = nullptr;
    float2* ll1 = nullptr;
    float2* rA = nullptr;
    float2* rB = nullptr;
    double* tau_part = nullptr;
    float* sorted = nullptr;
    double* sure_val = nullptr;       // [max_batch][B] minimum SURE of the last search
    double4_32a* partrec = nullptr;
    double4_32a* bestrec = nullptr;
    unsigned* counter = nullptr;
    int* fallback = nullptr;           // [3 + max_batch B] subbands left to the full SURE sort
    int* fallback2 = nullptr;          // the same for the search on the side stream
    vdamp::KEntry* klist = nullptr;    // [max_batch][nx][ny] sampled entries of a solve, per column
    int* kcnt = nullptr;               // [max_batch][nx] their counts
    float4* coef = nullptr;
    float* sigma_d = nullptr;
    int* status = nullptr;
    // staging for the host-buffer entry point
    float2* st_y = nullptr;
    uint8_t* st_mask = nullptr;
    float* st_p = nullptr;
    float2* st_x = nullptr;
    float2* st_r0 = nullptr;
    double* st_out = nullptr;
    size_t st_out_cap = 0;
    size_t ws_bytes = 0;
    int use_graph = 1;
    int timing = 0;
    int use_fused = 0;
    int overlap = 1;       // the finest subbands' threshold search on a side stream (split path)
    // side stream j (j = 1 .. levels - 1) searches the subbands of scale j, with its
    // fork and join events (scales >= 2: split path only)
    cudaStream_t side[VDAMP_MAX_LEVELS] = {};
    cudaEvent_t ev_fork[VDAMP_MAX_LEVELS] = {}, ev_join[VDAMP_MAX_LEVELS] = {};
    int fused_ok = 0;      // the device can hold the cluster
    int fused_C = 0, fused_cb = 0, fused_rpc = 0, fused_idwt_to = 0, fused_dwt_to = 0;
    size_t fused_smem = 0;
    int last_launches = 0;
    std::vector<cudaEvent_t> ev_pool;       // timing events, reused
    std::vector<std::pair<int, int>> ev_used;  // (kind, index of start event)
    int ev_next = 0;
    cudaStream_t cap = nullptr;
    std::vector<GraphEntry> graphs;
};

static void purge_group_graphs(const vdamp_plan* p);

static void plan_free(vdamp_plan* p) {
    if (!p) return;
    purge_group_graphs(p);
    for (auto& g : p->graphs) cudaGraphExecDestroy(g.exec);
    for (auto& e : p->ev_pool) cudaEventDestroy(e);
    void* bufs[] = {p->ey,       p->ex,      p->tw_y,    p->tw_x,    p->u,      p->kbuf,
                    p->ll0,      p->ll1,     p->rA,      p->rB,      p->tau_part, p->sorted,
                    p->partrec,  p->bestrec, p->counter, p->coef,    p->sigma_d, p->status,
                    p->sure_val, p->fallback, p->fallback2, p->klist, p->kcnt,
                    p->st_y,     p->st_mask, p->st_p,    p->st_x,    p->st_r0,  p->st_out};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (p->cap) cudaStreamDestroy(p->cap);
    for (int j = 0; j < VDAMP_MAX_LEVELS; ++j) {
        if (p->side[j]) cudaStreamDestroy(p->side[j]);
        if (p->ev_fork[j]) cudaEventDestroy(p->ev_fork[j]);
        if (p->ev_join[j]) cudaEventDestroy(p->ev_join[j]);
    }
    delete p;
}

static bool fft_size_ok(int n) {
    if (n < 8 || n > 1024) return false;
    int m = n;
    for (int f : {2, 3, 5})
        while (m % f == 0) m /= f;
    return m == 1;
}

extern "C" const char* vdamp_last_error(void) { return g_last_error.c_str(); }

namespace vdamp {
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace vdamp

extern "C" vdamp_status vdamp_wavelet_filter(int wavelet, double* h, int* len) {
    const int L = wavelet_taps(wavelet);
    if (!L || !h || !len) return fail(VDAMP_EINVAL, "vdamp_wavelet_filter: bad wavelet or NULL");
    daubechies(L / 2, h);
    *len = L;
    return VDAMP_OK;
}

extern "C" vdamp_status vdamp_subband_spectra(int wavelet, int levels, int n, double* out) {
    const int L = wavelet_taps(wavelet);
    if (!L || levels < 1 || levels > VDAMP_MAX_LEVELS || n < 2 || !out)
        return fail(VDAMP_EINVAL, "vdamp_subband_spectra: bad argument");
    double h[VDAMP_MAX_TAPS];
    daubechies(L / 2, h);
    spectra(h, L, levels, n, out);
    return VDAMP_OK;
}

template <class T>
static cudaError_t dalloc(T** p, size_t count, size_t* acc) {
    *acc += count * sizeof(T);
    return cudaMalloc((void**)p, count * sizeof(T));
}

extern "C" vdamp_status vdamp_plan_create(vdamp_plan** out, int ny, int nx, int wavelet,
                                          int levels, int max_iters, int max_batch) {
    if (!out) return fail(VDAMP_EINVAL, "vdamp_plan_create: out is NULL");
    *out = nullptr;
    const int L = wavelet_taps(wavelet);
    if (!L) return fail(VDAMP_EINVAL, "vdamp_plan_create: wavelet must be VDAMP_HAAR or VDAMP_DB4");
    if (levels < 1 || levels > VDAMP_MAX_LEVELS)
        return fail(VDAMP_EINVAL, "vdamp_plan_create: levels must be in [1, 6]");
    if (!fft_size_ok(ny) || !fft_size_ok(nx))
        return fail(VDAMP_EINVAL, "vdamp_plan_create: ny, nx must be 2^a 3^b 5^c in [8, 1024]");
    if ((ny % (1 << levels)) || (nx % (1 << levels)))
        return fail(VDAMP_EINVAL, "vdamp_plan_create: ny and nx must be divisible by 2^levels");
    if (max_batch < 1) return fail(VDAMP_EINVAL, "vdamp_plan_create: max_batch must be >= 1");
    if (max_iters < 1 || max_iters > 100000)
        return fail(VDAMP_EINVAL, "vdamp_plan_create: max_iters must be in [1, 100000]");
    const size_t N = (size_t)ny * nx;
    const int max_band = (int)(N / 4);
    if (vdamp::sure_smem(max_band) > 227 * 1024)
        return fail(VDAMP_EINVAL, "vdamp_plan_create: the SURE search does not fit shared memory");

    vdamp_plan* p = new vdamp_plan();
    p->ny = ny;
    p->nx = nx;
    p->levels = levels;
    p->wavelet = wavelet;
    p->B = 1 + 3 * levels;
    p->max_batch = max_batch;
    p->max_iters = max_iters;
    p->N = N;

    double h[VDAMP_MAX_TAPS];
    daubechies(L / 2, h);
    p->filt.L = L;
    for (int k = 0; k < VDAMP_MAX_TAPS; ++k) {
        p->filt.h[k] = k < L ? (float)h[k] : 0.f;
        p->filt.g[k] = k < L ? (float)(((k & 1) ? -1.0 : 1.0) * h[L - 1 - k]) : 0.f;
    }
    // packed subband offsets and the spectra each subband takes along y and x
    p->off[0] = 0;
    p->ty[0] = p->tx[0] = 2 * (levels - 1);
    int o = (ny >> levels) * (nx >> levels);
    int b = 1;
    for (int j = levels; j >= 1; --j) {
        const int sz = (ny >> j) * (nx >> j);
        const int lo = 2 * (j - 1), hi = 2 * (j - 1) + 1;
        const int tys[3] = {lo, hi, hi}, txs[3] = {hi, lo, hi};  // H, V, D
        for (int q = 0; q < 3; ++q) {
            p->off[b] = o;
            p->ty[b] = tys[q];
            p->tx[b] = txs[q];
            o += sz;
            ++b;
        }
    }
    p->off[p->B] = o;

    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    // columns per CTA of the column pass: 8, fewer while a full batch would
    // leave SMs without a column block (never below 2: each block stages the
    // y spectra once for all its columns)
    int cb = 8;
    while (nx % cb) cb >>= 1;
    while (cb > 2 && (size_t)max_batch * (nx / cb) < (size_t)std::max(p->num_sms, 1)) cb >>= 1;
    p->cb = cb;
    p->nparts = nx / cb;
    p->rpc = std::max(1, 512 / nx);

    // persistent cluster solve: work-item sizes and shared memory
    {
        const int C = 16;
        int fcb = 16;
        while (nx % fcb || vdamp::col_pass_smem_bytes(ny, fcb, 2 * levels) > 128 * 1024) fcb >>= 1;
        int frpc = (ny + C - 1) / C;
        const int cap = std::max(1, (96 * 1024) / (int)(2 * nx * sizeof(float2)));
        if (frpc > cap) frpc = cap;
        p->fused_cb = std::max(fcb, 1);
        p->fused_rpc = frpc;
        p->fused_idwt_to = 64;
        p->fused_dwt_to = 32;
        size_t sm = vdamp::sure_smem_bytes(max_band);
        sm = std::max(sm, vdamp::idwt_tile_smem(p->fused_idwt_to, L));
        sm = std::max(sm, vdamp::dwt_tile_smem(p->fused_dwt_to, L));
        sm = std::max(sm, 2 * (size_t)frpc * nx * sizeof(float2));
        sm = std::max(sm, vdamp::col_pass_smem_bytes(ny, p->fused_cb, 2 * levels));
        p->fused_smem = sm;
    }
    const int nparts_alloc = std::max(nx / 2, nx / p->fused_cb);  // any column block >= 2 columns

    p->axy.n = ny;
    p->axx.n = nx;
    if (!fft_radices(ny, p->axy.radix, &p->axy.nstages) ||
        !fft_radices(nx, p->axx.radix, &p->axx.nstages)) {
        plan_free(p);
        return fail(VDAMP_EINVAL, "vdamp_plan_create: no radix plan");
    }

    size_t acc = 0;
    cudaError_t e = cudaSuccess;
    const size_t MB = (size_t)max_batch;
    const int nt = 2 * levels;
    auto A = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    A(dalloc(&p->ey, (size_t)nt * ny, &acc));
    A(dalloc(&p->ex, (size_t)nt * nx, &acc));
    A(dalloc(&p->tw_y, (size_t)ny, &acc));
    A(dalloc(&p->tw_x, (size_t)nx, &acc));
    A(dalloc(&p->u, MB * N, &acc));
    A(dalloc(&p->kbuf, MB * N, &acc));
    A(dalloc(&p->ll0, MB * N / 4, &acc));
    A(dalloc(&p->ll1, MB * N / 4, &acc));
    A(dalloc(&p->rA, MB * N, &acc));
    A(dalloc(&p->rB, MB * N, &acc));
    A(dalloc(&p->tau_part, MB * nparts_alloc * p->B, &acc));
    A(dalloc(&p->sorted, MB * N, &acc));
    A(dalloc(&p->partrec, MB * p->B * SURE_MAX_PARTS, &acc));
    A(dalloc(&p->bestrec, MB * p->B * SURE_MAX_PARTS, &acc));
    A(dalloc(&p->counter, MB * p->B, &acc));
    A(dalloc(&p->sure_val, MB * p->B, &acc));
    A(dalloc(&p->fallback, 3 + MB * p->B, &acc));
    A(dalloc(&p->fallback2, 3 + MB * p->B, &acc));
    A(dalloc(&p->klist, MB * N, &acc));
    A(dalloc(&p->kcnt, MB * (size_t)nx, &acc));
    A(dalloc(&p->coef, MB * p->B, &acc));
    A(dalloc(&p->sigma_d, MB, &acc));
    A(dalloc(&p->status, (size_t)2, &acc));
    // output staging of the host-buffer and descriptor entry points (tau, thr, alpha)
    p->st_out_cap = 3 * MB * (size_t)max_iters * p->B;
    A(dalloc(&p->st_out, p->st_out_cap, &acc));
    if (e != cudaSuccess) {
        plan_free(p);
        return fail(e == cudaErrorMemoryAllocation ? VDAMP_ENOMEM : VDAMP_ECUDA,
                    std::string("vdamp_plan_create: ") + cudaGetErrorString(e));
    }
    p->ws_bytes = acc;

    // tables
    std::vector<double> sy((size_t)nt * ny), sx((size_t)nt * nx);
    spectra(h, L, levels, ny, sy.data());
    spectra(h, L, levels, nx, sx.data());
    std::vector<float> fy(sy.begin(), sy.end()), fx(sx.begin(), sx.end());
    std::vector<float2> twy(ny), twx(nx);
    const double two_pi = 2.0 * 3.14159265358979323846;
    for (int k = 0; k < ny; ++k)
        twy[k] = make_float2((float)std::cos(two_pi * k / ny), (float)-std::sin(two_pi * k / ny));
    for (int k = 0; k < nx; ++k)
        twx[k] = make_float2((float)std::cos(two_pi * k / nx), (float)-std::sin(two_pi * k / nx));
    A(cudaMemcpy(p->ey, fy.data(), fy.size() * sizeof(float), cudaMemcpyHostToDevice));
    A(cudaMemcpy(p->ex, fx.data(), fx.size() * sizeof(float), cudaMemcpyHostToDevice));
    A(cudaMemcpy(p->tw_y, twy.data(), ny * sizeof(float2), cudaMemcpyHostToDevice));
    A(cudaMemcpy(p->tw_x, twx.data(), nx * sizeof(float2), cudaMemcpyHostToDevice));
    A(cudaMemset(p->status, 0, 2 * sizeof(int)));
    A(cudaMemset(p->counter, 0, MB * p->B * sizeof(unsigned)));  // each search returns it to 0
    A(cudaMemset(p->fallback, 0, 3 * sizeof(int)));
    A(cudaMemset(p->fallback2, 0, 3 * sizeof(int)));               // each fallback launch empties it
    A(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
    for (int j = 1; j < levels; ++j) {
        A(cudaStreamCreateWithFlags(&p->side[j], cudaStreamNonBlocking));
        A(cudaEventCreateWithFlags(&p->ev_fork[j], cudaEventDisableTiming));
        A(cudaEventCreateWithFlags(&p->ev_join[j], cudaEventDisableTiming));
    }
    // shared-memory attributes large enough for every tile choice the tuner may make
    p->smem_col = vdamp::col_pass_smem(ny, cb, nt);
    for (int c2 = 2; c2 <= 16; c2 *= 2) {
        const size_t sm = vdamp::col_pass_smem(ny, c2, nt);
        if (nx % c2 == 0 && sm <= 200 * 1024) p->smem_col = std::max(p->smem_col, sm);
    }
    p->smem_rows = 2 * (size_t)p->rpc * nx * sizeof(float2);
    for (int r2 = 1; r2 <= 8; r2 *= 2) {
        const size_t sm = 2 * (size_t)r2 * nx * sizeof(float2);
        if (sm <= 128 * 1024) p->smem_rows = std::max(p->smem_rows, sm);
    }
    p->smem_dwt = std::max(vdamp::idwt_tile_smem(64, L), vdamp::dwt_tile_smem(32, L));
    A(vdamp::configure_col_pass(p->smem_col));
    A(vdamp::configure_fft_rows(p->smem_rows));
    A(vdamp::configure_dwt(p->smem_dwt));
    A(vdamp::configure_sure(vdamp::sure_smem(max_band)));
    if (e != cudaSuccess) {
        plan_free(p);
        return fail(VDAMP_ECUDA, std::string("vdamp_plan_create: ") + cudaGetErrorString(e));
    }
    p->axy.tw = p->tw_y;
    p->axx.tw = p->tw_x;
    // Can the device hold one cluster of 16 (else 8) such CTAs?
    if (p->fused_smem <= 227 * 1024) {
        for (int C : {16, 8}) {
            int nclus = 0;
            cudaError_t fe = vdamp::fused_configure(C, p->fused_smem, &nclus);
            if (fe == cudaSuccess && nclus >= 1) {
                p->fused_ok = 1;
                p->fused_C = C;
                break;
            }
            cudaGetLastError();  // clear a refusal before trying the smaller cluster
        }
    }
    // one cluster per slice for all wavelet scales (16 CTAs, else 8)
    for (int C : {16, 8}) {
        int nclus = 0;
        if (vdamp::configure_wavelet_cluster(C, p->smem_dwt, &nclus) == cudaSuccess && nclus > 0) {
            p->wcluster = C;
            break;
        }
        cudaGetLastError();
    }
    *out = p;
    return VDAMP_OK;
}

extern "C" vdamp_status vdamp_plan_destroy(vdamp_plan* p) {
    if (!p) return fail(VDAMP_EINVAL, "vdamp_plan_destroy: NULL plan");
    cudaDeviceSynchronize();
    plan_free(p);
    return VDAMP_OK;
}

extern "C" int vdamp_num_subbands(const vdamp_plan* p) { return p ? p->B : -1; }
extern "C" size_t vdamp_workspace_bytes(const vdamp_plan* p) { return p ? p->ws_bytes : 0; }
extern "C" int vdamp_last_launch_count(const vdamp_plan* p) { return p ? p->last_launches : -1; }

extern "C" vdamp_status vdamp_plan_set_option(vdamp_plan* p, int option, int value) {
    if (!p) return fail(VDAMP_EINVAL, "vdamp_plan_set_option: NULL plan");
    if (option == VDAMP_OPT_GRAPH) {
        p->use_graph = value ? 1 : 0;
        return VDAMP_OK;
    }
    if (option == VDAMP_OPT_KERNEL_TIMING) {
        p->timing = value ? 1 : 0;
        return VDAMP_OK;
    }
    if (option == VDAMP_OPT_FUSED) {
        p->use_fused = value ? 1 : 0;
        return VDAMP_OK;
    }
    if (option == VDAMP_OPT_OVERLAP) {
        p->overlap = value ? 1 : 0;
        for (auto& g : p->graphs) cudaGraphExecDestroy(g.exec);  // they hold the old structure
        p->graphs.clear();
        purge_group_graphs(p);
        return VDAMP_OK;
    }
    return fail(VDAMP_EINVAL, "vdamp_plan_set_option: unknown option");
}

// ------------------------------------------------------ launch helpers ---
namespace {

struct Ctx {
    vdamp_plan* p;
    int batch;
    cudaStream_t st;
    int launches = 0;
    cudaError_t err = cudaSuccess;
    bool timed = false;
    int ev_start = -1;
    // the compacted k-space inputs of this solve (NULL: the column passes read y, mask, p)
    const vdamp::KEntry* klist = nullptr;
    const int* kcnt = nullptr;
    cudaEvent_t ev(int i) {
        while ((int)p->ev_pool.size() <= i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            p->ev_pool.push_back(e);
        }
        return p->ev_pool[i];
    }
    // call before a launch
    void pre() {
        if (!timed) return;
        ev_start = p->ev_next;
        p->ev_next += 2;
        cudaEvent_t e = ev(ev_start);
        if (e) cudaEventRecord(e, st);
    }
    // call after `n` launches of one kind with their status
    void chk(cudaError_t e, int kind, int n = 1) {
        launches += n;
        if (err == cudaSuccess) err = e;
        if (timed && ev_start >= 0) {
            cudaEvent_t f = ev(ev_start + 1);
            if (f) {
                cudaEventRecord(f, st);
                p->ev_used.push_back({kind, ev_start});
            }
            ev_start = -1;
        }
    }
};

SrcSpec make_src(const vdamp_plan* p, int mode, const float2* r) {
    SrcSpec s;
    s.mode = mode;
    s.r = r;
    s.coef = p->coef;
    s.B = p->B;
    return s;
}

// The first scale of the many-slice cluster path: the smallest j >= 2 whose
// synthesis output is at most 128 x 128 (levels + 1: none).
int coarse_lo(const vdamp_plan* p) {
    for (int j = 2; j <= p->levels; ++j)
        if ((p->ny >> (j - 1)) <= 128 && (p->nx >> (j - 1)) <= 128) return j;
    return p->levels + 1;
}

// The cluster path for the coarse scales (the finer ones keep their own wide
// launches): tuning 1, while one cluster of wcluster CTAs per slice leaves SMs
// free: scales s .. 2; tuning 2, any batch: clusters of up to 4 CTAs per slice
// for the scales s .. coarse_lo.  Returns the cluster size (0: per-scale
// launches) and sets *lo.
int wavelet_cluster(const Ctx& c, int* lo) {
    const vdamp_plan* p = c.p;
    if (p->wcluster <= 0 || p->levels < 2) return 0;
    if (p->use_wcluster == 1 && c.batch * p->wcluster <= p->num_sms) {
        *lo = 2;
        return p->wcluster;
    }
    if (p->use_wcluster == 2 && coarse_lo(p) <= p->levels) {
        *lo = coarse_lo(p);
        return std::min(4, p->wcluster);
    }
    return 0;
}

// x = Psi^H (src), levels s .. 1; before_scale(j) (if set) runs before a scale j
// launched on its own is enqueued (it reads the subbands of scale j)
void enq_psi_h(Ctx& c, const SrcSpec& src, float2* img,
               const std::function<void(int)>& before_scale = nullptr) {
    vdamp_plan* p = c.p;
    const int s = p->levels;
    const float2* ll_in = nullptr;
    int lo = 2;
    const int C = wavelet_cluster(c, &lo);
    const bool cl = C > 0;
    vdamp::WaveletArgs w;
    if (cl) {
        memset(&w, 0, sizeof(w));
        w.levels = s;
        w.lo = lo;
    }
    for (int j = s; j >= 1; --j) {
        vdamp::IdwtArgs a;
        a.ll_in = ll_in;
        a.ll_stride = p->N / 4;
        a.h = p->ny >> j;
        a.w = p->nx >> j;
        a.first = (j == s);
        a.out = (j == 1) ? img : (((s - j) & 1) ? p->ll1 : p->ll0);
        a.out_stride = (j == 1) ? p->N : p->N / 4;
        a.N = p->N;
        const int bh = 1 + 3 * (s - j);
        a.off[0] = p->off[0];
        a.off[1] = p->off[bh];
        a.off[2] = p->off[bh + 1];
        a.off[3] = p->off[bh + 2];
        a.band[0] = 0;
        a.band[1] = bh;
        a.band[2] = bh + 1;
        a.band[3] = bh + 2;
        a.src = src;
        a.f = p->filt;
        a.to = p->idwt_to;
        ll_in = a.out;
        if (cl && j >= lo) {
            a.to = 32;   // one tile pass per CTA and scale up to 128x128 outputs (16 CTAs)
            w.idwt[j - 1] = a;
            if (j == lo) {   // the coarse scales in one cluster launch
                c.pre();
                c.chk(vdamp::launch_psi_h_cluster(w, c.batch, C, p->smem_dwt, c.st),
                      VDAMP_KERNEL_IDWT);
            }
            continue;
        }
        if (before_scale) before_scale(j);
        c.pre();
        c.chk(vdamp::launch_idwt_level(a, c.batch, c.st), VDAMP_KERNEL_IDWT);
    }
}

// packed = Psi img + src (levels 1 .. s); after_scale(j) (if set) runs once a
// scale j launched on its own (it writes the subbands of scale j) is enqueued
void enq_psi(Ctx& c, const float2* img, float2* packed, const SrcSpec& src,
             const std::function<void(int)>& after_scale = nullptr) {
    vdamp_plan* p = c.p;
    const int s = p->levels;
    const float2* in = img;
    size_t in_stride = p->N;
    int lo = 2;
    const int C = wavelet_cluster(c, &lo);
    const bool cl = C > 0;
    vdamp::WaveletArgs w;
    if (cl) {
        memset(&w, 0, sizeof(w));
        w.levels = s;
        w.lo = lo;
    }
    for (int j = 1; j <= s; ++j) {
        vdamp::DwtArgs a;
        a.in = in;
        a.in_stride = in_stride;
        a.H = p->ny >> (j - 1);
        a.W = p->nx >> (j - 1);
        a.last = (j == s);
        a.ll_out = (j & 1) ? p->ll0 : p->ll1;
        a.ll_stride = p->N / 4;
        a.packed = packed;
        a.N = p->N;
        const int bh = 1 + 3 * (s - j);
        a.off[0] = p->off[0];
        a.off[1] = p->off[bh];
        a.off[2] = p->off[bh + 1];
        a.off[3] = p->off[bh + 2];
        a.band[0] = 0;
        a.band[1] = bh;
        a.band[2] = bh + 1;
        a.band[3] = bh + 2;
        a.src = src;
        a.f = p->filt;
        a.to = p->dwt_to;
        in = a.ll_out;
        in_stride = p->N / 4;
        if (cl && j >= lo) {
            w.dwt[j - 1] = a;
            continue;
        }
        c.pre();
        c.chk(vdamp::launch_dwt_level(a, c.batch, c.st), VDAMP_KERNEL_DWT);
        if (after_scale) after_scale(j);
    }
    if (cl) {   // the coarse scales in one cluster launch
        c.pre();
        c.chk(vdamp::launch_psi_cluster(w, c.batch, C, p->smem_dwt, c.st),
              VDAMP_KERNEL_DWT);
    }
}

vdamp::ColArgs col_args(const vdamp_plan* p, int mode, const float2* in, float2* out,
                        const float2* y, const uint8_t* mask, const float* density) {
    vdamp::ColArgs a;
    memset(&a, 0, sizeof(a));
    a.in = in;
    a.out = out;
    a.ny = p->ny;
    a.nx = p->nx;
    a.cb = p->cb;
    a.plan_batch = p->max_batch;
    a.ax = p->axy;
    a.mode = mode;
    a.u_zero = 0;
    const float isn = (float)(1.0 / std::sqrt((double)p->N));
    a.scale_fwd = isn;
    a.scale_inv = 1.0f;
    a.y = y;
    a.mask = mask;
    a.density = density;
    a.sigma = p->sigma_d;
    a.ey = p->ey;
    a.ex = p->ex;
    a.ntypes = 2 * p->levels;
    a.B = p->B;
    for (int b = 0; b < p->B; ++b) {
        a.ty[b] = p->ty[b];
        a.tx[b] = p->tx[b];
    }
    a.tau_part = p->tau_part;
    return a;
}

float inv_sqrt_n(const vdamp_plan* p) { return (float)(1.0 / std::sqrt((double)p->N)); }

// The sampled entries of y, 1/p (and the mask) compacted per column, once per solve;
// later column passes on this Ctx read the list instead of the dense inputs.
void enq_kspace_list(Ctx& c, const float2* y, const uint8_t* mask, const float* density) {
    vdamp_plan* p = c.p;
    vdamp::ColArgs a = col_args(p, vdamp::COL_ITER, p->kbuf, p->kbuf, y, mask, density);
    a.klist = p->klist;
    a.kcnt = p->kcnt;
    c.pre();
    c.chk(vdamp::launch_kspace_list(a, c.batch, c.st), VDAMP_KERNEL_OTHER);
    c.klist = p->klist;
    c.kcnt = p->kcnt;
}

// k-space part of one iteration: from the image u (or zero) to u' = F^H P^-1 z
void enq_kspace_iter(Ctx& c, bool u_zero, const float2* y, const uint8_t* mask,
                     const float* density) {
    vdamp_plan* p = c.p;
    if (!u_zero) {   // r~ = 0 (cold start): U = 0, the column pass needs no row transform
        c.pre();
        c.chk(vdamp::launch_fft_rows(p->u, p->kbuf, p->ny, p->nx, c.batch, p->axx, 0, 1.0f,
                                     p->rpc, p->max_batch, c.st), VDAMP_KERNEL_FFT_ROWS);
    }
    vdamp::ColArgs a = col_args(p, vdamp::COL_ITER, p->kbuf, p->kbuf, y, mask, density);
    a.u_zero = u_zero ? 1 : 0;
    a.klist = c.klist;
    a.kcnt = c.kcnt;
    c.pre();
    c.chk(vdamp::launch_col_pass(a, c.batch, c.st), VDAMP_KERNEL_COL_PASS);
    c.pre();
    c.chk(vdamp::launch_fft_rows(p->kbuf, p->u, p->ny, p->nx, c.batch, p->axx, 1, inv_sqrt_n(p),
                                 p->rpc, p->max_batch, c.st), VDAMP_KERNEL_FFT_ROWS);
}

// return line: x = u + F^H M^T (y - M F u) with u = Psi^H (src)
void enq_final(Ctx& c, const SrcSpec& src, const float2* y, const uint8_t* mask, float2* x) {
    vdamp_plan* p = c.p;
    enq_psi_h(c, src, p->u);
    c.pre();
    c.chk(vdamp::launch_fft_rows(p->u, p->kbuf, p->ny, p->nx, c.batch, p->axx, 0, 1.0f, p->rpc, p->max_batch,
                                 c.st), VDAMP_KERNEL_FFT_ROWS);
    vdamp::ColArgs a = col_args(p, vdamp::COL_FINAL, p->kbuf, p->kbuf, y, mask, nullptr);
    a.klist = c.klist;
    a.kcnt = c.kcnt;
    c.pre();
    c.chk(vdamp::launch_col_pass(a, c.batch, c.st), VDAMP_KERNEL_COL_PASS);
    c.pre();
    c.chk(vdamp::launch_fft_rows(p->kbuf, x, p->ny, p->nx, c.batch, p->axx, 1, inv_sqrt_n(p),
                                 p->rpc, p->max_batch, c.st), VDAMP_KERNEL_FFT_ROWS);
}

// CTAs per subband of the threshold search (1: the pruned search)
int sure_max_parts(const Ctx& c) {
    const vdamp_plan* p = c.p;
    // Split big subbands over several CTAs only while the split grid fits in one wave
    // (each part rereads its whole subband: past one wave one CTA per subband is
    // faster), unless the tuning fixes the number of parts.
    int split = 0;
    for (int b = 0; b < p->B; ++b)
        split += vdamp::sure_parts(p->off[b + 1] - p->off[b], SURE_MAX_PARTS);
    int mp = p->sure_parts ? p->sure_parts : ((c.batch * split > p->num_sms) ? 1 : SURE_MAX_PARTS);
    // a finest subband above what one CTA holds is always split (SURE_MIN_PARTS_BIG or more)
    if ((int)(p->N / 4) > SURE_SMALL_BAND && mp < SURE_MIN_PARTS_BIG) mp = SURE_MAX_PARTS;
    return mp;
}

// Large subbands of the pruned search (one CTA each; the finest ones).
int prune_big(const vdamp_plan* p) {
    const int ns = vdamp::prune_n_small(p->off, p->B);
    return p->B - ns - vdamp::prune_n_med(p->off, p->B, ns);
}

// Lines 5-7 for the subbands b_top, b_top - 1, ..., b_top - nb + 1 (default: all).
// On the pruned path a subset is either the large subbands (b_top = B - 1,
// nb = prune_big) or all the others.  fallback: the pruned search's list (NULL:
// the plan's first one).
void enq_sure(Ctx& c, const float2* r, int iters, int k, double* tau, double* thr,
              double* alpha, int b_top = -1, int nb = -1, int* fallback = nullptr) {
    vdamp_plan* p = c.p;
    vdamp::SureArgs a;
    a.r = r;
    a.sorted = p->sorted;
    a.N = p->N;
    a.B = p->B;
    for (int b = 0; b <= p->B; ++b) a.off[b] = p->off[b];
    a.tau_part = p->tau_part;
    a.nparts = p->nparts;
    a.iters = iters;
    a.k = k;
    a.tau_out = tau;
    a.thr_out = thr;
    a.alpha_out = alpha;
    a.coef = p->coef;
    a.status = p->status;
    a.partrec = p->partrec;
    a.bestrec = p->bestrec;
    a.counter = p->counter;
    a.sure_out = p->sure_val;
    a.fallback = fallback ? fallback : p->fallback;
    a.max_parts = sure_max_parts(c);
    a.b_top = b_top < 0 ? p->B - 1 : b_top;
    a.nb_launch = nb < 0 ? p->B : nb;
    a.item0 = 0;
    if (a.max_parts == 1) {   // the pruned search: a range of work items
        const int ctas = vdamp::prune_ctas(p->off, p->B), big = prune_big(p);
        if (nb < 0) {
            a.nb_launch = ctas;
        } else if (a.b_top == p->B - 1) {
            a.nb_launch = big;
        } else {
            a.item0 = big;
            a.nb_launch = ctas - big;
        }
    }
    c.pre();
    // the pruned search and its fallback when every subband is one part, else sort and search
    c.chk(vdamp::launch_sure(a, c.batch, (int)(p->N / 4), std::max(p->num_sms, 1), c.st),
          VDAMP_KERNEL_SURE, 2);
}

void enq_line8(Ctx& c, const float2* r, float2* out) {
    vdamp_plan* p = c.p;
    vdamp::Line8Args a;
    a.src = make_src(p, vdamp::SRC_LINE8, r);
    a.out = out;
    a.N = p->N;
    a.B = p->B;
    for (int b = 0; b <= p->B; ++b) a.off[b] = p->off[b];
    c.pre();
    c.chk(vdamp::launch_line8(a, c.batch, c.st), VDAMP_KERNEL_OTHER);
}

struct SolveArgs {
    const float2* y;
    const uint8_t* mask;
    const float* density;
    int iters;
    const float2* r_tilde0;
    float2* x_hat;
    double *tau, *thr, *alpha;
    float2* r_tilde_out;
    float2* x_hat_iters;
    bool reset_status = true;   // clear the plan's error record first (false: keep earlier ones)
};

void enq_fused(Ctx& c, const SolveArgs& s);

// Algorithm 1, lines 1-10.
void enq_solve(Ctx& c, const SolveArgs& s) {
    vdamp_plan* p = c.p;
    if (p->fused_ok && p->use_fused) {
        enq_fused(c, s);
        return;
    }
    if (s.reset_status && c.err == cudaSuccess)
        c.err = cudaMemsetAsync(p->status, 0, sizeof(int), c.st);
    if (s.reset_status && c.err == cudaSuccess)
        c.err = cudaMemsetAsync(p->status + 1, 0x7f, sizeof(int), c.st);
    enq_kspace_list(c, s.y, s.mask, s.density);   // the column passes of this solve read only these
    // The finest subbands' threshold search (lines 5-7 for the three subbands of
    // scale 1, the costliest; on the pruned path when they are its large subbands)
    // runs on a side stream from the moment scale 1 of Psi has produced them, beside
    // the coarser scales of Psi, their search and the coarser scales of the next
    // Psi^H; the next scale 1 of Psi^H (which reads the finest subbands) waits for
    // it.  Same kernels and arguments (the side's pruned search has a fallback list
    // of its own), so the same results.
    const bool ov = p->overlap && !c.timed && p->levels >= 2 && p->B > 3 &&
                    (sure_max_parts(c) > 1 || prune_big(p) == 3);
    // On the split path the subbands of every scale j < s launched on its own do the
    // same on side stream j (from scale j of Psi to scale j of the next Psi^H); the
    // coarsest scale and the approximation band stay in line.
    int clo = p->levels + 1;
    const int ccl = wavelet_cluster(c, &clo);
    const bool split = sure_max_parts(c) > 1;
    bool forks[VDAMP_MAX_LEVELS] = {};   // scale j's search goes to side stream j
    int side_bands = 0;                  // subbands searched on side streams
    for (int j = 1; ov && j < p->levels; ++j) {
        if (j >= 2 && (!split || (ccl > 0 && j >= clo))) break;
        forks[j] = true;
        side_bands += 3;
    }
    bool pending[VDAMP_MAX_LEVELS] = {};   // scale j's search in flight on side stream j
    auto join_scale = [&](int j) {
        if (j < 1 || j >= VDAMP_MAX_LEVELS || !pending[j]) return;
        if (c.err == cudaSuccess) c.err = cudaStreamWaitEvent(c.st, p->ev_join[j], 0);
        pending[j] = false;
    };
    auto join = [&]() {
        for (int j = 1; j < VDAMP_MAX_LEVELS; ++j) join_scale(j);
    };
    float2* prev = p->rA;  // r_{k-1}
    float2* cur = p->rB;   // r_k
    for (int k = 0; k < s.iters; ++k) {
        SrcSpec src;
        bool zero = false;
        if (k == 0) {
            zero = (s.r_tilde0 == nullptr);
            src = make_src(p, zero ? vdamp::SRC_ZERO : vdamp::SRC_EXPLICIT, s.r_tilde0);
        } else {
            src = make_src(p, vdamp::SRC_LINE8, prev);
        }
        if (!zero) enq_psi_h(c, src, p->u, join_scale);  // Psi^H r~_k        (line 3)
        join();
        enq_kspace_iter(c, zero, s.y, s.mask, s.density);  // z, tau parts, F^H P^-1 z (3-5)
        if (ov) {
            auto fork = [&](int j) {   // the subbands of scale j of r_k are written
                if (j < 1 || j >= VDAMP_MAX_LEVELS || !forks[j]) return;
                if (c.err == cudaSuccess) c.err = cudaEventRecord(p->ev_fork[j], c.st);
                if (c.err == cudaSuccess) c.err = cudaStreamWaitEvent(p->side[j], p->ev_fork[j], 0);
                Ctx side{p, c.batch, p->side[j]};
                enq_sure(side, cur, s.iters, k, s.tau, s.thr, s.alpha, p->B - 1 - 3 * (j - 1), 3,
                         j == 1 ? p->fallback2 : nullptr);
                c.launches += side.launches;
                if (c.err == cudaSuccess) c.err = side.err;
                if (c.err == cudaSuccess) c.err = cudaEventRecord(p->ev_join[j], p->side[j]);
                pending[j] = true;
            };
            enq_psi(c, p->u, cur, src, fork);            // r_k = r~_k + Psi u' (line 4)
            enq_sure(c, cur, s.iters, k, s.tau, s.thr, s.alpha, p->B - 1 - side_bands,
                     p->B - side_bands);                 // the other subbands in line
        } else {
            enq_psi(c, p->u, cur, src);                  // r_k = r~_k + Psi u' (line 4)
            enq_sure(c, cur, s.iters, k, s.tau, s.thr, s.alpha);  // tau, theta, alpha (5-7)
        }
        if (s.x_hat_iters) {
            join();
            enq_final(c, make_src(p, vdamp::SRC_SOFT, cur), s.y, s.mask,
                      s.x_hat_iters + (size_t)k * c.batch * p->N);
        }
        float2* t = prev;
        prev = cur;
        cur = t;
    }
    join();
    enq_final(c, make_src(p, vdamp::SRC_SOFT, prev), s.y, s.mask, s.x_hat);  // return line
    if (s.r_tilde_out) enq_line8(c, prev, s.r_tilde_out);                      // line 8
}

// Algorithm 1, lines 1-10, as one persistent cluster launch.
void enq_fused(Ctx& c, const SolveArgs& s) {
    vdamp_plan* p = c.p;
    if (s.reset_status && c.err == cudaSuccess)
        c.err = cudaMemsetAsync(p->status, 0, sizeof(int), c.st);
    if (s.reset_status && c.err == cudaSuccess)
        c.err = cudaMemsetAsync(p->status + 1, 0x7f, sizeof(int), c.st);
    const int lv = p->levels;
    const size_t N = p->N;
    vdamp::FusedArgs f;
    memset(&f, 0, sizeof(f));
    f.levels = lv;
    f.B = p->B;
    f.iters = s.iters;
    f.N = N;
    f.ny = p->ny;
    f.nx = p->nx;
    f.rpc = p->fused_rpc;
    f.nrowblk = (p->ny + p->fused_rpc - 1) / p->fused_rpc;
    f.nparts = p->nx / p->fused_cb;
    f.inv_sqrt_n = inv_sqrt_n(p);
    f.axx = p->axx;
    for (int j = 1; j <= lv; ++j) {
        const int bh = 1 + 3 * (lv - j);
        vdamp::IdwtArgs& a = f.idwt[j - 1];
        a.ll_in = (j == lv) ? nullptr : (((lv - (j + 1)) & 1) ? p->ll1 : p->ll0);
        a.ll_stride = N / 4;
        a.h = p->ny >> j;
        a.w = p->nx >> j;
        a.first = (j == lv);
        a.out = (j == 1) ? nullptr : (((lv - j) & 1) ? p->ll1 : p->ll0);
        a.out_stride = (j == 1) ? N : N / 4;
        a.N = N;
        a.f = p->filt;
        a.to = p->fused_idwt_to;
        vdamp::DwtArgs& d = f.dwt[j - 1];
        d.in = (j == 1) ? nullptr : (((j - 1) & 1) ? p->ll0 : p->ll1);
        d.in_stride = (j == 1) ? N : N / 4;
        d.H = p->ny >> (j - 1);
        d.W = p->nx >> (j - 1);
        d.last = (j == lv);
        d.ll_out = (j & 1) ? p->ll0 : p->ll1;
        d.ll_stride = N / 4;
        d.N = N;
        d.f = p->filt;
        d.to = p->fused_dwt_to;
        const int offs[4] = {p->off[0], p->off[bh], p->off[bh + 1], p->off[bh + 2]};
        const int bands[4] = {0, bh, bh + 1, bh + 2};
        for (int q = 0; q < 4; ++q) {
            a.off[q] = d.off[q] = offs[q];
            a.band[q] = d.band[q] = bands[q];
        }
    }
    f.col = col_args(p, vdamp::COL_ITER, p->kbuf, p->kbuf, s.y, s.mask, s.density);
    f.col.cb = p->fused_cb;
    vdamp::SureArgs& u = f.sure;
    u.r = nullptr;
    u.sorted = p->sorted;
    u.N = N;
    u.B = p->B;
    for (int b = 0; b <= p->B; ++b) u.off[b] = p->off[b];
    u.tau_part = p->tau_part;
    u.nparts = f.nparts;
    u.iters = s.iters;
    u.k = 0;
    u.tau_out = s.tau;
    u.thr_out = s.thr;
    u.alpha_out = s.alpha;
    u.coef = p->coef;
    u.status = p->status;
    u.partrec = p->partrec;
    u.bestrec = p->bestrec;
    u.counter = p->counter;
    u.sure_out = p->sure_val;
    u.fallback = p->fallback;
    u.b_top = p->B - 1;
    u.nb_launch = p->B;
    u.item0 = 0;
    u.max_parts = SURE_MAX_PARTS;
    f.l8.src = make_src(p, vdamp::SRC_LINE8, nullptr);
    f.l8.N = N;
    f.l8.B = p->B;
    for (int b = 0; b <= p->B; ++b) f.l8.off[b] = p->off[b];
    f.r_tilde0 = s.r_tilde0;
    f.x_hat = s.x_hat;
    f.r_tilde_out = s.r_tilde_out;
    f.x_hat_iters = s.x_hat_iters;
    f.u = p->u;
    f.kbuf = p->kbuf;
    f.rA = p->rA;
    f.rB = p->rB;
    f.coef = p->coef;
    f.C = p->fused_C;
    c.pre();
    c.chk(vdamp::launch_fused(f, c.batch, p->fused_smem, c.st), VDAMP_KERNEL_FUSED);
}

vdamp_status set_sigma(vdamp_plan* p, const float* sigma, int batch, cudaStream_t st,
                       int* launches) {
    for (int b0 = 0; b0 < batch; b0 += 512) {
        SigmaBlock blk;
        blk.n = std::min(512, batch - b0);
        for (int i = 0; i < blk.n; ++i) blk.v[i] = sigma[b0 + i];
        CUDA_TRY(vdamp::launch_pdl(set_sigma_kernel, dim3(1), dim3(512), 0, st, p->sigma_d + b0,
                                   blk));
        ++*launches;
    }
    return VDAMP_OK;
}

vdamp_status check_common(vdamp_plan* p, int batch, const char* who) {
    if (!p) return fail(VDAMP_EINVAL, std::string(who) + ": NULL plan");
    if (batch < 1 || batch > p->max_batch)
        return fail(VDAMP_EINVAL, std::string(who) + ": batch outside [1, max_batch]");
    return VDAMP_OK;
}

vdamp_status check_sigma(const float* sigma, int batch, const char* who) {
    if (!sigma) return fail(VDAMP_EINVAL, std::string(who) + ": sigma is NULL");
    for (int i = 0; i < batch; ++i)
        if (!(sigma[i] >= 0.f) || !std::isfinite(sigma[i]))
            return fail(VDAMP_EINVAL, std::string(who) + ": sigma must be finite and >= 0");
    return VDAMP_OK;
}

}  // namespace

static vdamp_status solve_impl(vdamp_plan* p, int batch, const float* y, const uint8_t* mask,
                               const float* density, const float* sigma, int iters,
                               const float* r_tilde0, int k0, float* x_hat, double* tau,
                               double* thr, double* alpha, float* r_tilde_out,
                               float* x_hat_iters, void* stream, bool reset_status) {
    vdamp_status st = check_common(p, batch, "vdamp_solve");
    if (st != VDAMP_OK) return st;
    if (!y || !mask || !density || !x_hat || !tau || !thr || !alpha)
        return fail(VDAMP_EINVAL, "vdamp_solve: a required pointer is NULL");
    if (iters < 1 || iters > p->max_iters)
        return fail(VDAMP_EINVAL, "vdamp_solve: iters must be in [1, max_iters]");
    if (k0 < 0 || (!r_tilde0 && k0 != 0))
        return fail(VDAMP_EINVAL, "vdamp_solve: k0 must be >= 0, and 0 for a cold start");
    if ((st = check_sigma(sigma, batch, "vdamp_solve")) != VDAMP_OK) return st;
    cudaStream_t us = (cudaStream_t)stream;
    int launches = 0;
    if ((st = set_sigma(p, sigma, batch, us, &launches)) != VDAMP_OK) return st;

    SolveArgs s;
    s.y = (const float2*)y;
    s.mask = mask;
    s.density = density;
    s.iters = iters;
    s.r_tilde0 = (const float2*)r_tilde0;
    s.x_hat = (float2*)x_hat;
    s.tau = tau;
    s.thr = thr;
    s.alpha = alpha;
    s.r_tilde_out = (float2*)r_tilde_out;
    s.x_hat_iters = (float2*)x_hat_iters;
    s.reset_status = reset_status;

    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CUDA_TRY(cudaStreamIsCapturing(us, &cs));
    if (p->use_graph && !p->timing && cs == cudaStreamCaptureStatusNone) {
        GraphKey key;
        memset(&key, 0, sizeof(key));
        key.kind = reset_status ? 1 : 3;
        key.batch = batch;
        key.iters = iters;
        const void* ptrs[] = {y, mask, density, r_tilde0, x_hat, tau, thr, alpha, r_tilde_out,
                              x_hat_iters};
        for (int i = 0; i < 10; ++i) key.p[i] = ptrs[i];
        GraphEntry* hit = nullptr;
        for (auto& g : p->graphs)
            if (g.key == key) hit = &g;
        if (!hit) {
            Ctx c{p, batch, p->cap};
            CUDA_TRY(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
            enq_solve(c, s);
            cudaGraph_t graph = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(p->cap, &graph);
            if (c.err != cudaSuccess || e2 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return fail(VDAMP_ECUDA, std::string("vdamp_solve capture: ") +
                                             cudaGetErrorString(c.err != cudaSuccess ? c.err : e2));
            }
            cudaGraphExec_t exec = nullptr;
            cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e3 != cudaSuccess)
                return fail(VDAMP_ECUDA, std::string("vdamp_solve instantiate: ") +
                                             cudaGetErrorString(e3));
            if (p->graphs.size() >= 16) {
                cudaGraphExecDestroy(p->graphs.front().exec);
                p->graphs.erase(p->graphs.begin());
            }
            p->graphs.push_back(GraphEntry{key, exec, c.launches});
            hit = &p->graphs.back();
        }
        CUDA_TRY(cudaGraphLaunch(hit->exec, us));
        p->last_launches = launches + hit->launches;
        p->last_k0 = k0;
        return VDAMP_OK;
    }
    Ctx c{p, batch, us};
    c.timed = p->timing != 0;
    enq_solve(c, s);
    p->last_launches = launches + c.launches;
    p->last_k0 = k0;
    if (c.err != cudaSuccess)
        return fail(VDAMP_ECUDA, std::string("vdamp_solve: ") + cudaGetErrorString(c.err));
    return VDAMP_OK;
}

extern "C" vdamp_status vdamp_solve(vdamp_plan* p, int batch, const float* y, const uint8_t* mask,
                                    const float* density, const float* sigma, int iters,
                                    const float* r_tilde0, int k0, float* x_hat, double* tau,
                                    double* thr, double* alpha, float* r_tilde_out,
                                    float* x_hat_iters, void* stream) {
    return solve_impl(p, batch, y, mask, density, sigma, iters, r_tilde0, k0, x_hat, tau, thr,
                      alpha, r_tilde_out, x_hat_iters, stream, true);
}

// Device staging of one batch of inputs and image outputs for the host-buffer
// and descriptor entry points (allocated on first use, kept by the plan).
static vdamp_status ensure_staging(vdamp_plan* p, const char* who) {
    if (p->st_y) return VDAMP_OK;
    const size_t MB = (size_t)p->max_batch, N = p->N;
    cudaError_t e = cudaSuccess;
    size_t acc = 0;
    auto A = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    A(dalloc(&p->st_y, MB * N, &acc));
    A(dalloc(&p->st_mask, MB * N, &acc));
    A(dalloc(&p->st_p, MB * N, &acc));
    A(dalloc(&p->st_x, MB * N, &acc));
    A(dalloc(&p->st_r0, MB * N, &acc));
    if (e != cudaSuccess)
        return fail(VDAMP_ENOMEM, std::string(who) + ": staging: " + cudaGetErrorString(e));
    p->ws_bytes += acc;
    return VDAMP_OK;
}

extern "C" vdamp_status vdamp_solve_host(vdamp_plan* p, int batch, const float* y,
                                         const uint8_t* mask, const float* density,
                                         const float* sigma, int iters, const float* r_tilde0,
                                         int k0, float* x_hat, double* tau, double* thr,
                                         double* alpha, void* stream) {
    vdamp_status st = check_common(p, batch, "vdamp_solve_host");
    if (st != VDAMP_OK) return st;
    if (!y || !mask || !density || !x_hat || !tau || !thr || !alpha)
        return fail(VDAMP_EINVAL, "vdamp_solve_host: a required pointer is NULL");
    if (iters < 1 || iters > p->max_iters)
        return fail(VDAMP_EINVAL, "vdamp_solve_host: iters must be in [1, max_iters]");
    if ((st = check_sigma(sigma, batch, "vdamp_solve_host")) != VDAMP_OK) return st;
    if ((st = ensure_staging(p, "vdamp_solve_host")) != VDAMP_OK) return st;
    const size_t N = p->N;
    const size_t nout = (size_t)batch * iters * p->B;   // <= a third of st_out_cap
    cudaStream_t us = (cudaStream_t)stream;
    const size_t n = (size_t)batch * N;
    CUDA_TRY(cudaMemcpyAsync(p->st_y, y, n * sizeof(float2), cudaMemcpyHostToDevice, us));
    CUDA_TRY(cudaMemcpyAsync(p->st_mask, mask, n, cudaMemcpyHostToDevice, us));
    CUDA_TRY(cudaMemcpyAsync(p->st_p, density, n * sizeof(float), cudaMemcpyHostToDevice, us));
    if (r_tilde0)
        CUDA_TRY(cudaMemcpyAsync(p->st_r0, r_tilde0, n * sizeof(float2), cudaMemcpyHostToDevice,
                                 us));
    st = vdamp_solve(p, batch, (const float*)p->st_y, p->st_mask, p->st_p, sigma, iters,
                     r_tilde0 ? (const float*)p->st_r0 : nullptr, k0, (float*)p->st_x, p->st_out,
                     p->st_out + nout, p->st_out + 2 * nout, nullptr, nullptr, stream);
    if (st != VDAMP_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(x_hat, p->st_x, n * sizeof(float2), cudaMemcpyDeviceToHost, us));
    CUDA_TRY(cudaMemcpyAsync(tau, p->st_out, nout * sizeof(double), cudaMemcpyDeviceToHost, us));
    CUDA_TRY(cudaMemcpyAsync(thr, p->st_out + nout, nout * sizeof(double), cudaMemcpyDeviceToHost,
                             us));
    CUDA_TRY(cudaMemcpyAsync(alpha, p->st_out + 2 * nout, nout * sizeof(double),
                             cudaMemcpyDeviceToHost, us));
    int it = 0;
    return vdamp_device_status(p, &it, stream);
}

// ------------------------------------------- solve from slice descriptors ---
namespace {

constexpr int kDescChunk = 32;   // slices per gather / scatter launch

struct GatherChunk {
    int n;
    const float2* y[kDescChunk];
    const uint8_t* mask[kDescChunk];
    const float* density[kDescChunk];
    const float2* r0[kDescChunk];   // NULL: zeros
};

// staging[base + s] <- slice s of the chunk (blockIdx.y = s), grid-stride over N
__global__ void gather_slices_kernel(GatherChunk g, size_t N, int base, float2* sy, uint8_t* sm,
                                     float* sp, float2* sr0) {
    const int s = blockIdx.y;
    if (s >= g.n) return;
    const size_t o = (size_t)(base + s) * N;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (size_t)gridDim.x * blockDim.x) {
        sy[o + i] = g.y[s][i];
        sm[o + i] = g.mask[s][i];
        sp[o + i] = g.density[s][i];
        if (sr0) sr0[o + i] = g.r0[s] ? g.r0[s][i] : make_float2(0.f, 0.f);
    }
}

struct ScatterChunk {
    int n;
    float2* x[kDescChunk];
    double* tau[kDescChunk];
    double* thr[kDescChunk];
    double* alpha[kDescChunk];
};

// slice s of the chunk <- staging[base + s]: x_hat (N values) and the three
// [iters][B] records, which the staging holds as [batch][iters][B] each.
__global__ void scatter_slices_kernel(ScatterChunk g, size_t N, int base, size_t nrec,
                                      const float2* sx, const double* sout, size_t nout) {
    const int s = blockIdx.y;
    if (s >= g.n) return;
    const size_t o = (size_t)(base + s) * N, r = (size_t)(base + s) * nrec;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (size_t)gridDim.x * blockDim.x) {
        g.x[s][i] = sx[o + i];
        if (i < nrec) {
            g.tau[s][i] = sout[r + i];
            g.thr[s][i] = sout[nout + r + i];
            g.alpha[s][i] = sout[2 * nout + r + i];
        }
    }
}

}  // namespace

extern "C" vdamp_status vdamp_solve_batched(vdamp_plan* p, const vdamp_slice_desc* slices,
                                            int count, void* stream) {
    if (!p) return fail(VDAMP_EINVAL, "vdamp_solve_batched: NULL plan");
    if (!slices || count < 1) return fail(VDAMP_EINVAL, "vdamp_solve_batched: no slices");
    for (int i = 0; i < count; ++i) {
        const vdamp_slice_desc& d = slices[i];
        if (!d.y || !d.mask || !d.density || !d.x_hat || !d.tau || !d.thr || !d.alpha)
            return fail(VDAMP_EINVAL, "vdamp_solve_batched: a required pointer is NULL");
        if (d.iters < 1 || d.iters > p->max_iters)
            return fail(VDAMP_EINVAL, "vdamp_solve_batched: iters must be in [1, max_iters]");
        if (d.k0 < 0 || (!d.r_tilde0 && d.k0 != 0))
            return fail(VDAMP_EINVAL, "vdamp_solve_batched: k0 must be >= 0, 0 for a cold start");
        if (!(d.sigma >= 0.f) || !std::isfinite(d.sigma))
            return fail(VDAMP_EINVAL, "vdamp_solve_batched: sigma must be finite and >= 0");
    }
    vdamp_status st = ensure_staging(p, "vdamp_solve_batched");
    if (st != VDAMP_OK) return st;
    cudaStream_t us = (cudaStream_t)stream;
    const size_t N = p->N;
    const int gx = (int)std::min<size_t>((N + 255) / 256, 64);
    // slices that share (iters, k0, cold start) are solved together, up to max_batch at a time
    std::vector<char> done(count, 0);
    int launches = 0;
    const int first = 0;
    for (int i0 = 0; i0 < count; ++i0) {
        if (done[i0]) continue;
        const vdamp_slice_desc& k = slices[i0];
        std::vector<int> grp;
        for (int i = i0; i < count && (int)grp.size() < p->max_batch; ++i)
            if (!done[i] && slices[i].iters == k.iters && slices[i].k0 == k.k0 &&
                (slices[i].r_tilde0 == nullptr) == (k.r_tilde0 == nullptr)) {
                grp.push_back(i);
                done[i] = 1;
            }
        const int nb = (int)grp.size();
        const bool cold = k.r_tilde0 == nullptr;
        std::vector<float> sig(nb);
        for (int c0 = 0; c0 < nb; c0 += kDescChunk) {
            GatherChunk g;
            memset(&g, 0, sizeof(g));
            g.n = std::min(kDescChunk, nb - c0);
            for (int j = 0; j < g.n; ++j) {
                const vdamp_slice_desc& d = slices[grp[c0 + j]];
                g.y[j] = (const float2*)d.y;
                g.mask[j] = d.mask;
                g.density[j] = d.density;
                g.r0[j] = (const float2*)d.r_tilde0;
            }
            gather_slices_kernel<<<dim3(gx, g.n), 256, 0, us>>>(g, N, c0, p->st_y, p->st_mask,
                                                                p->st_p, cold ? nullptr : p->st_r0);
            CUDA_TRY(cudaGetLastError());
            ++launches;
        }
        for (int j = 0; j < nb; ++j) sig[j] = slices[grp[j]].sigma;
        const size_t nout = (size_t)nb * k.iters * p->B;
        // the first group clears the error record, later ones keep what earlier ones found
        st = solve_impl(p, nb, (const float*)p->st_y, p->st_mask, p->st_p, sig.data(), k.iters,
                        cold ? nullptr : (const float*)p->st_r0, k.k0, (float*)p->st_x,
                        p->st_out, p->st_out + nout, p->st_out + 2 * nout, nullptr, nullptr,
                        stream, i0 == first);
        if (st != VDAMP_OK) return st;
        launches += p->last_launches;
        for (int c0 = 0; c0 < nb; c0 += kDescChunk) {
            ScatterChunk g;
            memset(&g, 0, sizeof(g));
            g.n = std::min(kDescChunk, nb - c0);
            for (int j = 0; j < g.n; ++j) {
                const vdamp_slice_desc& d = slices[grp[c0 + j]];
                g.x[j] = (float2*)d.x_hat;
                g.tau[j] = d.tau;
                g.thr[j] = d.thr;
                g.alpha[j] = d.alpha;
            }
            scatter_slices_kernel<<<dim3(gx, g.n), 256, 0, us>>>(
                g, N, c0, (size_t)k.iters * p->B, p->st_x, p->st_out, nout);
            CUDA_TRY(cudaGetLastError());
            ++launches;
        }
    }
    p->last_launches = launches;
    return VDAMP_OK;
}

extern "C" vdamp_status vdamp_iterate(vdamp_plan* p, int batch, const float* r_tilde,
                                      const float* y, const uint8_t* mask, const float* density,
                                      const float* sigma, float* r, double* tau, double* thr,
                                      double* alpha, float* r_tilde_next, void* stream) {
    vdamp_status st = check_common(p, batch, "vdamp_iterate");
    if (st != VDAMP_OK) return st;
    if (!r_tilde || !y || !mask || !density || !r || !tau || !thr || !alpha || !r_tilde_next)
        return fail(VDAMP_EINVAL, "vdamp_iterate: a pointer is NULL");
    if (r == r_tilde) return fail(VDAMP_EINVAL, "vdamp_iterate: r must not alias r_tilde");
    if ((st = check_sigma(sigma, batch, "vdamp_iterate")) != VDAMP_OK) return st;
    cudaStream_t us = (cudaStream_t)stream;
    int launches = 0;
    if ((st = set_sigma(p, sigma, batch, us, &launches)) != VDAMP_OK) return st;
    Ctx c{p, batch, us};
    c.timed = p->timing != 0;
    if (cudaMemsetAsync(p->status, 0, sizeof(int), us) != cudaSuccess ||
        cudaMemsetAsync(p->status + 1, 0x7f, sizeof(int), us) != cudaSuccess)
        return fail(VDAMP_ECUDA, "vdamp_iterate: memset");
    SrcSpec src = make_src(p, vdamp::SRC_EXPLICIT, (const float2*)r_tilde);
    enq_psi_h(c, src, p->u);
    enq_kspace_iter(c, false, (const float2*)y, mask, density);
    enq_psi(c, p->u, (float2*)r, src);
    enq_sure(c, (const float2*)r, 1, 0, tau, thr, alpha);
    enq_line8(c, (const float2*)r, (float2*)r_tilde_next);
    p->last_launches = launches + c.launches;
    p->last_k0 = 0;
    if (c.err != cudaSuccess)
        return fail(VDAMP_ECUDA, std::string("vdamp_iterate: ") + cudaGetErrorString(c.err));
    return VDAMP_OK;
}

extern "C" vdamp_status vdamp_final_estimate(vdamp_plan* p, int batch, const float* w,
                                             const float* y, const uint8_t* mask, float* x_hat,
                                             void* stream) {
    vdamp_status st = check_common(p, batch, "vdamp_final_estimate");
    if (st != VDAMP_OK) return st;
    if (!w || !y || !mask || !x_hat) return fail(VDAMP_EINVAL, "vdamp_final_estimate: NULL");
    Ctx c{p, batch, (cudaStream_t)stream};
    c.timed = p->timing != 0;
    enq_final(c, make_src(p, vdamp::SRC_EXPLICIT, (const float2*)w), (const float2*)y, mask,
              (float2*)x_hat);
    p->last_launches = c.launches;
    if (c.err != cudaSuccess)
        return fail(VDAMP_ECUDA, std::string("vdamp_final_estimate: ") + cudaGetErrorString(c.err));
    return VDAMP_OK;
}

extern "C" vdamp_status vdamp_psi(vdamp_plan* p, int batch, const float* x, float* w,
                                  void* stream) {
    vdamp_status st = check_common(p, batch, "vdamp_psi");
    if (st != VDAMP_OK) return st;
    if (!x || !w) return fail(VDAMP_EINVAL, "vdamp_psi: NULL");
    Ctx c{p, batch, (cudaStream_t)stream};
    c.timed = p->timing != 0;
    enq_psi(c, (const float2*)x, (float2*)w, make_src(p, vdamp::SRC_ZERO, nullptr));
    p->last_launches = c.launches;
    if (c.err != cudaSuccess)
        return fail(VDAMP_ECUDA, std::string("vdamp_psi: ") + cudaGetErrorString(c.err));
    return VDAMP_OK;
}

extern "C" vdamp_status vdamp_psi_h(vdamp_plan* p, int batch, const float* w, float* x,
                                    void* stream) {
    vdamp_status st = check_common(p, batch, "vdamp_psi_h");
    if (st != VDAMP_OK) return st;
    if (!x || !w) return fail(VDAMP_EINVAL, "vdamp_psi_h: NULL");
    Ctx c{p, batch, (cudaStream_t)stream};
    c.timed = p->timing != 0;
    enq_psi_h(c, make_src(p, vdamp::SRC_EXPLICIT, (const float2*)w), (float2*)x);
    p->last_launches = c.launches;
    if (c.err != cudaSuccess)
        return fail(VDAMP_ECUDA, std::string("vdamp_psi_h: ") + cudaGetErrorString(c.err));
    return VDAMP_OK;
}

extern "C" vdamp_status vdamp_fft2(vdamp_plan* p, int batch, const float* in, float* out,
                                   int inverse, void* stream) {
    vdamp_status st = check_common(p, batch, "vdamp_fft2");
    if (st != VDAMP_OK) return st;
    if (!in || !out || in == out) return fail(VDAMP_EINVAL, "vdamp_fft2: NULL or aliased");
    Ctx c{p, batch, (cudaStream_t)stream};
    c.timed = p->timing != 0;
    c.pre();
    c.chk(vdamp::launch_fft_rows((const float2*)in, (float2*)out, p->ny, p->nx, batch, p->axx,
                                 inverse ? 1 : 0, 1.0f, p->rpc, p->max_batch, c.st), VDAMP_KERNEL_FFT_ROWS);
    vdamp::ColArgs a = col_args(p, inverse ? vdamp::COL_INV : vdamp::COL_FWD, (float2*)out,
                                (float2*)out, nullptr, nullptr, nullptr);
    a.scale_inv = inv_sqrt_n(p);
    c.pre();
    c.chk(vdamp::launch_col_pass(a, batch, c.st), VDAMP_KERNEL_COL_PASS);
    p->last_launches = c.launches;
    if (c.err != cudaSuccess)
        return fail(VDAMP_ECUDA, std::string("vdamp_fft2: ") + cudaGetErrorString(c.err));
    return VDAMP_OK;
}

extern "C" vdamp_status vdamp_device_status(vdamp_plan* p, int* iter, void* stream) {
    if (!p) return fail(VDAMP_EINVAL, "vdamp_device_status: NULL plan");
    cudaStream_t us = (cudaStream_t)stream;
    CUDA_TRY(cudaStreamSynchronize(us));
    int h[2] = {0, 0};
    CUDA_TRY(cudaMemcpy(h, p->status, sizeof(h), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(p->status, 0, sizeof(int)));
    if (h[0] == VDAMP_ENUMERIC) {
        const int k = h[1] + p->last_k0;
        if (iter) *iter = k;
        return fail(VDAMP_ENUMERIC, "non-finite tau or alpha at iteration " + std::to_string(k));
    }
    if (iter) *iter = -1;
    return VDAMP_OK;
}

extern "C" vdamp_status vdamp_kernel_times(vdamp_plan* p, double* ms, int* counts) {
    if (!p || !ms || !counts) return fail(VDAMP_EINVAL, "vdamp_kernel_times: NULL");
    for (int k = 0; k < VDAMP_KERNEL_KINDS; ++k) {
        ms[k] = 0.0;
        counts[k] = 0;
    }
    for (auto& u : p->ev_used) {
        cudaEvent_t a = p->ev_pool[u.second], b = p->ev_pool[u.second + 1];
        CUDA_TRY(cudaEventSynchronize(b));
        float t = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&t, a, b));
        ms[u.first] += t;
        counts[u.first] += 1;
    }
    p->ev_used.clear();
    p->ev_next = 0;
    return VDAMP_OK;
}

// ------------------------------------------------------------- tuning ---
namespace {

bool tuning_valid(const vdamp_plan* p, const int* t) {
    const int cb = t[0], rpc = t[1], ito = t[2], dto = t[3];
    if (cb < 2 || cb > 16 || (cb & (cb - 1)) || p->nx % cb) return false;
    if (vdamp::col_pass_smem(p->ny, cb, 2 * p->levels) > p->smem_col) return false;
    if (rpc < 1 || rpc > 8 || 2 * (size_t)rpc * p->nx * sizeof(float2) > p->smem_rows) return false;
    if (ito != 16 && ito != 32 && ito != 64) return false;
    if (dto != 16 && dto != 32) return false;
    if (t[6] != 0 && t[6] != 1 && t[6] != 2) return false;
    if (t[6] == 2 && coarse_lo(p) > p->levels) return false;
    if (t[7] != 0 && t[7] != 1 && t[7] != 2 && t[7] != 4 && t[7] != SURE_MAX_PARTS) return false;
    if ((int)(p->N / 4) > SURE_SMALL_BAND && t[7] != 0 && t[7] < SURE_MIN_PARTS_BIG) return false;
    if (vdamp::idwt_tile_smem(ito, p->filt.L) > p->smem_dwt ||
        vdamp::dwt_tile_smem(dto, p->filt.L) > p->smem_dwt)
        return false;
    int r[VDAMP_MAX_STAGES], ns = 0;
    for (int ax = 0; ax < 2; ++ax)
        if (t[4 + ax] < 0 || t[4 + ax] > 2 || !fft_radices(ax ? p->nx : p->ny, r, &ns, t[4 + ax]))
            return false;
    return true;
}

void get_tuning(const vdamp_plan* p, int* t) {
    t[0] = p->cb;
    t[1] = p->rpc;
    t[2] = p->idwt_to;
    t[3] = p->dwt_to;
    t[4] = p->radix_var[0];
    t[5] = p->radix_var[1];
    t[6] = p->use_wcluster;
    t[7] = p->sure_parts;
}

void apply_tuning(vdamp_plan* p, const int* t) {
    p->cb = t[0];
    p->nparts = p->nx / p->cb;
    p->rpc = t[1];
    p->idwt_to = t[2];
    p->dwt_to = t[3];
    p->radix_var[0] = t[4];
    p->radix_var[1] = t[5];
    p->use_wcluster = t[6];
    p->sure_parts = t[7];
    fft_radices(p->ny, p->axy.radix, &p->axy.nstages, t[4]);
    fft_radices(p->nx, p->axx.radix, &p->axx.nstages, t[5]);
    for (auto& g : p->graphs) cudaGraphExecDestroy(g.exec);  // they hold the old launch shapes
    p->graphs.clear();
    purge_group_graphs(p);
}

// Synthetic problem for timing trials: pseudo-random measurements on a
// 30% mask with p = 0.3 and a pseudo-random r~ (a hash of the index).
__global__ void tune_fill_kernel(float2* y, uint8_t* m, float* d, float2* rt, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 2654435761u ^ (uint32_t)(i >> 32) * 40503u;
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        const float u0 = (float)(h & 0xffff) / 65536.f, u1 = (float)(h >> 16) / 65536.f;
        m[i] = u0 < 0.3f;
        d[i] = 0.3f;
        y[i] = make_float2(u0 - 0.5f, u1 - 0.5f);
        rt[i] = make_float2(0.1f * (u1 - 0.5f), 0.1f * (u0 - 0.5f));
    }
}

}  // namespace

extern "C" vdamp_status vdamp_plan_get_tuning(const vdamp_plan* p, int* tuning) {
    if (!p || !tuning) return fail(VDAMP_EINVAL, "vdamp_plan_get_tuning: NULL");
    get_tuning(p, tuning);
    return VDAMP_OK;
}

extern "C" vdamp_status vdamp_plan_set_tuning(vdamp_plan* p, const int* tuning) {
    if (!p || !tuning) return fail(VDAMP_EINVAL, "vdamp_plan_set_tuning: NULL");
    if (!tuning_valid(p, tuning)) return fail(VDAMP_EINVAL, "vdamp_plan_set_tuning: invalid tuning");
    apply_tuning(p, tuning);
    return VDAMP_OK;
}

extern "C" vdamp_status vdamp_plan_autotune(vdamp_plan* p, int batch, int trials, int* tuning,
                                            void* stream) {
    vdamp_status st = check_common(p, batch, "vdamp_plan_autotune");
    if (st != VDAMP_OK) return st;
    if (trials < 1 || trials > 1000) return fail(VDAMP_EINVAL, "vdamp_plan_autotune: trials");
    cudaStream_t us = (cudaStream_t)stream;
    const size_t n = (size_t)batch * p->N, nb = (size_t)batch * p->B;
    float2 *y = nullptr, *rt = nullptr, *r = nullptr, *rn = nullptr;
    uint8_t* m = nullptr;
    float* d = nullptr;
    double* outs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    A(cudaMalloc(&y, n * sizeof(float2)));
    A(cudaMalloc(&rt, n * sizeof(float2)));
    A(cudaMalloc(&r, n * sizeof(float2)));
    A(cudaMalloc(&rn, n * sizeof(float2)));
    A(cudaMalloc(&m, n));
    A(cudaMalloc(&d, n * sizeof(float)));
    const int iters = std::max(trials, 2);
    A(cudaMalloc(&outs, 3 * nb * (size_t)iters * sizeof(double)));
    A(cudaEventCreate(&e0));
    A(cudaEventCreate(&e1));
    auto cleanup = [&]() {
        cudaFree(y); cudaFree(rt); cudaFree(r); cudaFree(rn); cudaFree(m); cudaFree(d);
        cudaFree(outs);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (e != cudaSuccess) {
        cleanup();
        return fail(VDAMP_ENOMEM, std::string("vdamp_plan_autotune: ") + cudaGetErrorString(e));
    }
    tune_fill_kernel<<<std::min<size_t>((n + 255) / 256, 4096), 256, 0, us>>>(y, m, d, rt, n);
    std::vector<float> sig(batch, 0.01f);
    int launches = 0;
    if ((st = set_sigma(p, sig.data(), batch, us, &launches)) != VDAMP_OK) {
        cleanup();
        return st;
    }
    // One timing trial: a solve of max(trials, 2) iterations from the synthetic r~,
    // captured in one CUDA graph as vdamp_solve captures it (programmatic dependent
    // launches, the threshold searches of the finer scales on their side streams), so
    // that a shape is judged by what a solve costs with it; the faster of two timed
    // launches after a warm-up launch.
    auto trial = [&](const int* t, float* ms) -> cudaError_t {
        apply_tuning(p, t);
        Ctx c{p, batch, p->cap};
        SolveArgs sa;
        sa.y = y;
        sa.mask = m;
        sa.density = d;
        sa.iters = iters;
        sa.r_tilde0 = rt;
        sa.x_hat = rn;
        sa.tau = outs;
        sa.thr = outs + nb * iters;
        sa.alpha = outs + 2 * nb * iters;
        sa.r_tilde_out = nullptr;
        sa.x_hat_iters = nullptr;
        cudaError_t x = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
        if (x != cudaSuccess) return x;
        enq_solve(c, sa);
        cudaGraph_t graph = nullptr;
        x = cudaStreamEndCapture(p->cap, &graph);
        if (c.err != cudaSuccess || x != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return c.err != cudaSuccess ? c.err : x;
        }
        cudaGraphExec_t exec = nullptr;
        x = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (x != cudaSuccess) return x;
        float best = 0.f;
        x = cudaGraphLaunch(exec, us);
        for (int rep = 0; rep < 2 && x == cudaSuccess; ++rep) {
            float one = 0.f;
            x = cudaEventRecord(e0, us);
            if (x == cudaSuccess) x = cudaGraphLaunch(exec, us);
            if (x == cudaSuccess) x = cudaEventRecord(e1, us);
            if (x == cudaSuccess) x = cudaEventSynchronize(e1);
            if (x == cudaSuccess) x = cudaEventElapsedTime(&one, e0, e1);
            if (x == cudaSuccess && (rep == 0 || one < best)) best = one;
        }
        cudaGraphExecDestroy(exec);
        *ms = best;
        return x;
    };
    // coordinate descent over (cb, rpc, idwt tile, dwt tile, radix plan y, radix plan x,
    // wavelet cluster, SURE parts)
    static const int choices[VDAMP_TUNING_LEN][4] = {{2, 4, 8, 16}, {1, 2, 4, 8}, {16, 32, 64, 0},
                                                     {16, 32, 0, 0}, {0, 1, 2, -1}, {0, 1, 2, -1},
                                                     {0, 1, 2, -1}, {0, 1, 2, 4}};
    int best[VDAMP_TUNING_LEN];
    get_tuning(p, best);
    float best_ms = 0.f;
    A(trial(best, &best_ms));
    for (int q = 0; q < VDAMP_TUNING_LEN && e == cudaSuccess; ++q) {
        for (int c = 0; c < 4 && e == cudaSuccess; ++c) {
            int cand[VDAMP_TUNING_LEN];
            std::memcpy(cand, best, sizeof(cand));
            cand[q] = choices[q][c];
            if (cand[q] == best[q] || !tuning_valid(p, cand)) continue;
            float ms = 0.f;
            A(trial(cand, &ms));
            if (e == cudaSuccess && ms < best_ms) {
                best_ms = ms;
                std::memcpy(best, cand, sizeof(best));
            }
        }
    }
    apply_tuning(p, best);
    cleanup();
    if (e != cudaSuccess)
        return fail(VDAMP_ECUDA, std::string("vdamp_plan_autotune: ") + cudaGetErrorString(e));
    if (tuning) get_tuning(p, tuning);
    return VDAMP_OK;
}

// ------------------------------------------------------- grouped solve ---
namespace {

struct GroupGraph {
    std::vector<vdamp_group> key;
    cudaGraphExec_t exec;
    std::vector<int> launches;
};
std::mutex g_group_mu;
std::vector<GroupGraph> g_group_graphs;

bool same_group(const vdamp_group& a, const vdamp_group& b) {
    return a.plan == b.plan && a.batch == b.batch && a.iters == b.iters && a.y == b.y &&
           a.mask == b.mask && a.density == b.density && a.x_hat == b.x_hat && a.tau == b.tau &&
           a.thr == b.thr && a.alpha == b.alpha;
}

SolveArgs group_args(const vdamp_group& g) {
    SolveArgs s;
    s.y = (const float2*)g.y;
    s.mask = g.mask;
    s.density = g.density;
    s.iters = g.iters;
    s.r_tilde0 = nullptr;
    s.x_hat = (float2*)g.x_hat;
    s.tau = g.tau;
    s.thr = g.thr;
    s.alpha = g.alpha;
    s.r_tilde_out = nullptr;
    s.x_hat_iters = nullptr;
    return s;
}

}  // namespace

static void purge_group_graphs(const vdamp_plan* p) {
    std::lock_guard<std::mutex> lk(g_group_mu);
    for (size_t i = 0; i < g_group_graphs.size();) {
        bool uses = false;
        for (auto& g : g_group_graphs[i].key) uses = uses || g.plan == p;
        if (uses) {
            cudaGraphExecDestroy(g_group_graphs[i].exec);
            g_group_graphs.erase(g_group_graphs.begin() + i);
        } else {
            ++i;
        }
    }
}

extern "C" vdamp_status vdamp_solve_groups(const vdamp_group* groups, int count, void* stream) {
    if (!groups || count < 1 || count > 64)
        return fail(VDAMP_EINVAL, "vdamp_solve_groups: count outside [1, 64]");
    for (int i = 0; i < count; ++i) {
        const vdamp_group& g = groups[i];
        vdamp_status st = check_common(g.plan, g.batch, "vdamp_solve_groups");
        if (st != VDAMP_OK) return st;
        if (!g.y || !g.mask || !g.density || !g.x_hat || !g.tau || !g.thr || !g.alpha)
            return fail(VDAMP_EINVAL, "vdamp_solve_groups: a required pointer is NULL");
        if (g.iters < 1 || g.iters > g.plan->max_iters)
            return fail(VDAMP_EINVAL, "vdamp_solve_groups: iters must be in [1, max_iters]");
        if ((st = check_sigma(g.sigma, g.batch, "vdamp_solve_groups")) != VDAMP_OK) return st;
        for (int j = 0; j < i; ++j)
            if (groups[j].plan == g.plan)
                return fail(VDAMP_EINVAL, "vdamp_solve_groups: a plan appears in two groups");
    }
    cudaStream_t us = (cudaStream_t)stream;
    std::vector<int> launches(count, 0);
    for (int i = 0; i < count; ++i) {
        vdamp_status st = set_sigma(groups[i].plan, groups[i].sigma, groups[i].batch, us,
                                    &launches[i]);
        if (st != VDAMP_OK) return st;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CUDA_TRY(cudaStreamIsCapturing(us, &cs));
    vdamp_plan* p0 = groups[0].plan;
    bool direct = !p0->use_graph || cs != cudaStreamCaptureStatusNone;
    for (int i = 0; i < count; ++i) direct = direct || groups[i].plan->timing || groups[i].plan->use_fused;
    if (direct) {   // one group after another on the caller's stream
        for (int i = 0; i < count; ++i) {
            Ctx c{groups[i].plan, groups[i].batch, us};
            c.timed = groups[i].plan->timing != 0;
            enq_solve(c, group_args(groups[i]));
            groups[i].plan->last_launches = launches[i] + c.launches;
            groups[i].plan->last_k0 = 0;
            if (c.err != cudaSuccess)
                return fail(VDAMP_ECUDA, std::string("vdamp_solve_groups: ") +
                                             cudaGetErrorString(c.err));
        }
        return VDAMP_OK;
    }
    std::lock_guard<std::mutex> lk(g_group_mu);
    GroupGraph* hit = nullptr;
    for (auto& gg : g_group_graphs) {
        if ((int)gg.key.size() != count) continue;
        bool same = true;
        for (int i = 0; i < count && same; ++i) same = same_group(gg.key[i], groups[i]);
        if (same) hit = &gg;
    }
    if (!hit) {
        // One graph: a fork from the first plan's capture stream into every
        // group's own stream, each group's solve there, and a join back.
        std::vector<cudaEvent_t> ev(count + 1, nullptr);
        cudaError_t e = cudaSuccess;
        for (auto& x : ev)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
        std::vector<int> lc(count, 0);
        cudaGraph_t graph = nullptr;
        if (e == cudaSuccess) e = cudaStreamBeginCapture(p0->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t ce = cudaEventRecord(ev[count], p0->cap);
            for (int i = 1; i < count && ce == cudaSuccess; ++i)
                ce = cudaStreamWaitEvent(groups[i].plan->cap, ev[count], 0);
            for (int i = 0; i < count && ce == cudaSuccess; ++i) {
                Ctx c{groups[i].plan, groups[i].batch, groups[i].plan->cap};
                enq_solve(c, group_args(groups[i]));
                lc[i] = c.launches;
                ce = c.err;
                if (ce == cudaSuccess && i > 0) ce = cudaEventRecord(ev[i], groups[i].plan->cap);
            }
            for (int i = 1; i < count && ce == cudaSuccess; ++i)
                ce = cudaStreamWaitEvent(p0->cap, ev[i], 0);
            cudaError_t ee = cudaStreamEndCapture(p0->cap, &graph);
            e = ce != cudaSuccess ? ce : ee;
        }
        for (auto& x : ev)
            if (x) cudaEventDestroy(x);
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess)
            return fail(VDAMP_ECUDA, std::string("vdamp_solve_groups capture: ") +
                                         cudaGetErrorString(e));
        if (g_group_graphs.size() >= 16) {
            cudaGraphExecDestroy(g_group_graphs.front().exec);
            g_group_graphs.erase(g_group_graphs.begin());
        }
        GroupGraph gg;
        gg.key.assign(groups, groups + count);
        gg.exec = exec;
        gg.launches = lc;
        g_group_graphs.push_back(gg);
        hit = &g_group_graphs.back();
    }
    CUDA_TRY(cudaGraphLaunch(hit->exec, us));
    for (int i = 0; i < count; ++i) {
        groups[i].plan->last_launches = launches[i] + hit->launches[i];
        groups[i].plan->last_k0 = 0;
    }
    return VDAMP_OK;
}

extern "C" vdamp_status vdamp_sure_fallback_count(vdamp_plan* p, int* count, void* stream) {
    if (!p || !count) return fail(VDAMP_EINVAL, "vdamp_sure_fallback_count: NULL");
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    int n[2] = {0, 0};
    CUDA_TRY(cudaMemcpy(&n[0], p->fallback + 2, sizeof(int), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(&n[1], p->fallback2 + 2, sizeof(int), cudaMemcpyDeviceToHost));
    *count = n[0] + n[1];
    return VDAMP_OK;
}

extern "C" vdamp_status vdamp_last_sure(vdamp_plan* p, int batch, double* out, void* stream) {
    vdamp_status st = check_common(p, batch, "vdamp_last_sure");
    if (st != VDAMP_OK) return st;
    if (!out) return fail(VDAMP_EINVAL, "vdamp_last_sure: NULL");
    CUDA_TRY(cudaMemcpyAsync(out, p->sure_val, (size_t)batch * p->B * sizeof(double),
                             cudaMemcpyDefault, (cudaStream_t)stream));
    return VDAMP_OK;
}

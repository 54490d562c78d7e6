// SURE-tuned complex soft threshold per subband (Sec. 3, the unnumbered
// equation after Algorithm 1) and the subband-mean derivative alpha
// (Algorithm 1 line 7), plus the final sum of tau (line 5).
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
// Precision: magnitudes, sort keys and per-thread partial sums are FP32; the
// cross-warp scans of C and H, tau, theta and alpha of the chosen interval
// are FP64.
#include <math.h>
#include "vdamp_internal.cuh"

namespace vdamp {

__device__ __forceinline__ void record_numeric(int* status, int k) {
    atomicExch(&status[0], 4 /* VDAMP_ENUMERIC */);
    atomicMin(&status[1], k);
}

size_t sure_smem(int max_band) {
    int np = 2;
    while (np < max_band) np <<= 1;
    return (size_t)np * sizeof(float);
}

__global__ void __launch_bounds__(1024) sure_kernel(SureArgs a) {
    extern __shared__ float keys[];
    __shared__ double s_tau;
    __shared__ float wc[32], wh[32];
    __shared__ double woc[33], woh[33];
    __shared__ float bq[32], bt[32];
    __shared__ int bm[32];
    __shared__ int s_win_m;
    const int b = blockIdx.x, slice = blockIdx.y;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    const int off = a.off[b], nb = a.off[b + 1] - off;
    int np = 2;
    while (np < nb) np <<= 1;

    if (tid == 0) {
        double t = 0.0;
        for (int p = 0; p < a.nparts; ++p) t += a.tau_part[((size_t)slice * a.nparts + p) * a.B + b];
        s_tau = t;
    }
    const float2* r = a.r + (size_t)slice * a.N + off;
    for (int i = tid; i < np; i += nthr) keys[i] = i < nb ? cabs_f(r[i]) : INFINITY;
    __syncthreads();
    const double tau = s_tau;
    const size_t orow = ((size_t)slice * a.iters + a.k) * a.B + b;
    if (!(tau > 0.0) || !isfinite(tau)) {
        // No effective noise (p = 1 and sigma = 0): keep r, no Onsager term.
        if (tid == 0) {
            a.tau_out[orow] = tau;
            a.thr_out[orow] = 0.0;
            a.alpha_out[orow] = 0.0;
            a.coef[slice * a.B + b] = make_float4(0.f, 0.f, 1.f, 0.f);
            if (!isfinite(tau)) record_numeric(a.status, a.k);
        }
        return;
    }

    // ---- bitonic sort, ascending
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

    // ---- prefix sums of a^2 (from below) and suffix sums of 1/a (from above)
    const int E = (nb + nthr - 1) / nthr;
    const int m0 = min(tid * E, nb), m1 = min(m0 + E, nb);
    float cs = 0.f, hs = 0.f;
    for (int i = m0; i < m1; ++i) {
        const float x = keys[i];
        cs += x * x;
        hs += x > 0.f ? 1.0f / x : 0.f;
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
    if (tid == 0) {
        double acc = 0.0;
        for (int w = 0; w < nw; ++w) { woc[w] = acc; acc += (double)wc[w]; }
        woc[nw] = acc;
        acc = 0.0;
        for (int w = nw - 1; w >= 0; --w) { woh[w] = acc; acc += (double)wh[w]; }
        woh[nw] = acc;
    }
    __syncthreads();
    const double c_base = woc[warp] + (double)ec;   // sum of a^2 over indices < m0
    const double h_after = woh[warp] + (double)eh;  // sum of 1/a over indices >= m1
    const double c_total = woc[nw];

    // ---- best candidate of this thread's intervals (FP32)
    const float tf = (float)tau;
    const float cb = (float)c_base, ha = (float)h_after;
    float best_q = INFINITY, best_t = INFINITY;
    int best_m = -1;
    float csuf = 0.f, hsuf = 0.f;
    for (int m = m1 - 1; m >= m0; --m) {
        const float x = keys[m];
        csuf += x * x;
        hsuf += x > 0.f ? 1.0f / x : 0.f;
        const float cm = cb + (cs - csuf);
        const float hm = ha + hsuf;
        const float K = (float)(nb - m);
        const float lo = m > 0 ? keys[m - 1] : 0.f;
        float th = tf * hm / (2.0f * K);
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
    if (m1 == nb && m0 < m1) {  // theta >= max a: everything thresholded
        const float q = (float)(c_total - (double)nb * tau);
        const float th = keys[nb - 1];
        if (q < best_q || (q == best_q && th < best_t)) {
            best_q = q;
            best_t = th;
            best_m = nb;
        }
    }

    // ---- block argmin (q, then theta)
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
    if (tid == 0) {
        float q = bq[0], t = bt[0];
        int m = bm[0];
        for (int w = 1; w < nw; ++w) {
            if (bq[w] < q || (bq[w] == q && (bt[w] < t || (bt[w] == t && bm[w] < m)))) {
                q = bq[w];
                t = bt[w];
                m = bm[w];
            }
        }
        s_win_m = m;
    }
    __syncthreads();

    // ---- theta and alpha of the chosen interval, FP64, by the thread that owns it
    const int wm = s_win_m;
    const bool owner = (wm == nb) ? (m1 == nb && m0 < m1) : (wm >= m0 && wm < m1);
    if (owner) {
        double theta, alpha;
        if (wm == nb) {
            theta = (double)keys[nb - 1];
            alpha = 0.0;
        } else {
            double hm = h_after;
            for (int i = wm; i < m1; ++i) {
                const double x = (double)keys[i];
                hm += x > 0.0 ? 1.0 / x : 0.0;
            }
            const double K = (double)(nb - wm);
            const double lo = wm > 0 ? (double)keys[wm - 1] : 0.0;
            theta = fmax(tau * hm / (2.0 * K), lo);
            theta = fmin(theta, (double)keys[wm]);
            alpha = (K - 0.5 * theta * hm) / (double)nb;
        }
        a.tau_out[orow] = tau;
        a.thr_out[orow] = theta;
        a.alpha_out[orow] = alpha;
        const double inv = 1.0 / (1.0 - alpha);
        a.coef[slice * a.B + b] = make_float4((float)theta, (float)alpha, (float)inv, 0.f);
        if (!isfinite(alpha) || !isfinite(theta) || !isfinite(inv)) record_numeric(a.status, a.k);
    }
}

cudaError_t launch_sure(const SureArgs& a, int batch, int max_band, cudaStream_t st) {
    dim3 grid(a.B, batch);
    sure_kernel<<<grid, 1024, sure_smem(max_band), st>>>(a);
    return cudaGetLastError();
}

cudaError_t configure_sure(size_t smem_bytes) {
    // the attribute is per kernel and process-wide: only ever raise it
    static size_t raised = 48 * 1024;
    if (smem_bytes <= raised) return cudaSuccess;
    raised = smem_bytes;
    return cudaFuncSetAttribute(sure_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes);
}

}  // namespace vdamp

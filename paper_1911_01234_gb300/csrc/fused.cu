// Persistent cluster solve: Algorithm 1 (lines 1-10) for one slice per
// thread-block cluster, all iterations in a single launch.
//
// A slice's working set (a few MB) stays in L2 for the whole solve.  The C
// CTAs of a cluster (one per SM, 1024 threads each) split every step of the
// iteration into independent work items -- wavelet tiles of one scale, row
// blocks of the FFT, column blocks of the fused k-space pass, sort parts and
// subbands of the SURE search -- distributed round-robin over the cluster,
// with a cluster barrier (barrier.cluster arrive.release / wait.acquire)
// wherever a step needs all of the previous one: between wavelet scales,
// between the row and column passes of the FFT, and around the SURE search.
// All CTAs execute the same sequence of barriers: the control flow depends
// only on the iteration count and on launch-wide arguments.
#include <cooperative_groups.h>

#include "dwt_dev.cuh"
#include "fft_dev.cuh"
#include "fused.cuh"
#include "sure_dev.cuh"

namespace cg = cooperative_groups;

namespace vdamp {

namespace {

struct Ctx {
    const FusedArgs& f;   // refers to the __grid_constant__ kernel parameter: nothing is copied
    cg::cluster_group cl;
    int rank, C, slice, batch;
    float2* sm;
};

// x = Psi^H (src), scales s .. 1 (Algorithm 1 lines 3 and 10)
__device__ void phase_psi_h(Ctx& c, const SrcSpec& src, float2* img) {
    const FusedArgs& f = c.f;
    for (int j = f.levels; j >= 1; --j) {
        const IdwtArgs& a = f.idwt[j - 1];
        float2* out = (j == 1) ? img : a.out;
        const int ntx = (2 * a.w + a.to - 1) / a.to, nty = (2 * a.h + a.to - 1) / a.to;
        for (int t = c.rank; t < ntx * nty; t += c.C) {
            idwt_tile(a, out, src, t % ntx, t / ntx, c.slice, c.sm);
            __syncthreads();
        }
        c.cl.sync();
    }
}

// packed = Psi img + src, scales 1 .. s (Algorithm 1 line 4)
__device__ void phase_psi(Ctx& c, const float2* img, float2* packed, const SrcSpec& src) {
    const FusedArgs& f = c.f;
    for (int j = 1; j <= f.levels; ++j) {
        const DwtArgs& a = f.dwt[j - 1];
        const float2* in = (j == 1) ? img : a.in;
        const int Ho = a.H >> 1, Wo = a.W >> 1;
        const int ntx = (Wo + a.to - 1) / a.to, nty = (Ho + a.to - 1) / a.to;
        for (int t = c.rank; t < ntx * nty; t += c.C) {
            dwt_tile(a, in, packed, src, t % ntx, t / ntx, c.slice, c.sm);
            __syncthreads();
        }
        c.cl.sync();
    }
}

template <bool INV>
__device__ void phase_rows(Ctx& c, const float2* in, float2* out, float scale) {
    const FusedArgs& f = c.f;
    for (int t = c.rank; t < f.nrowblk; t += c.C) {
        const int row0 = t * f.rpc;
        fft_rows_block<INV>(in, out, f.ny, f.nx, f.axx, scale, row0, min(f.rpc, f.ny - row0),
                            c.slice, c.sm);
        __syncthreads();
    }
    c.cl.sync();
}

__device__ void phase_cols(Ctx& c, int mode, int u_zero) {
    const FusedArgs& f = c.f;
    for (int t = c.rank; t < f.nparts; t += c.C) {
        col_pass_block(f.col, mode, u_zero, t, f.nparts, c.slice, c.sm);
        __syncthreads();
    }
    c.cl.sync();
}

// Lines 5-7: sort parts, then search parts (the last part of a subband to
// finish writes its theta and alpha).
__device__ void phase_sure(Ctx& c, const float2* r, int k) {
    const FusedArgs& f = c.f;
    const SureArgs& a = f.sure;
    int total = 0;
    for (int b = 0; b < f.B; ++b) total += sure_parts(a.off[b + 1] - a.off[b], a.max_parts);
    for (int t = c.rank; t < total; t += c.C) {
        int b = 0, acc = 0;
        while (acc + sure_parts(a.off[b + 1] - a.off[b], a.max_parts) <= t) {
            acc += sure_parts(a.off[b + 1] - a.off[b], a.max_parts);
            ++b;
        }
        sure_sort_part(a, r, t - acc, b, c.slice, reinterpret_cast<float*>(c.sm));
        __syncthreads();
    }
    c.cl.sync();
    for (int t = c.rank; t < total; t += c.C) {
        int b = 0, acc = 0;
        while (acc + sure_parts(a.off[b + 1] - a.off[b], a.max_parts) <= t) {
            acc += sure_parts(a.off[b + 1] - a.off[b], a.max_parts);
            ++b;
        }
        sure_search_part(a, k, t - acc, b, c.slice, reinterpret_cast<float*>(c.sm));
        __syncthreads();
    }
    c.cl.sync();
}

// return line: x = Psi^H w + F^H M^T (y - M F Psi^H w), w = src
__device__ void phase_final(Ctx& c, const SrcSpec& src, float2* x) {
    const FusedArgs& f = c.f;
    phase_psi_h(c, src, f.u);
    phase_rows<false>(c, f.u, f.kbuf, 1.0f);
    phase_cols(c, COL_FINAL, 0);
    phase_rows<true>(c, f.kbuf, x, f.inv_sqrt_n);
}

}  // namespace

__global__ void __launch_bounds__(1024, 1) fused_solve_kernel(const __grid_constant__ FusedArgs f) {
    extern __shared__ float2 sm[];
    cudaGridDependencySynchronize();
    Ctx c{f, cg::this_cluster(), 0, 0, (int)blockIdx.y, (int)gridDim.y, sm};
    c.rank = (int)c.cl.block_rank();
    c.C = (int)c.cl.num_blocks();
    float2* prev = f.rA;  // r_{k-1}
    float2* cur = f.rB;   // r_k
    for (int k = 0; k < f.iters; ++k) {
        SrcSpec src;
        src.coef = f.coef;
        src.B = f.B;
        bool zero = false;
        if (k == 0) {
            zero = (f.r_tilde0 == nullptr);
            src.mode = zero ? SRC_ZERO : SRC_EXPLICIT;
            src.r = f.r_tilde0;
        } else {
            src.mode = SRC_LINE8;
            src.r = prev;
        }
        if (!zero) {
            phase_psi_h(c, src, f.u);                       // Psi^H r~_k      (line 3)
            phase_rows<false>(c, f.u, f.kbuf, 1.0f);
        }
        phase_cols(c, COL_ITER, zero ? 1 : 0);              // z, tau parts, F^H P^-1 z
        phase_rows<true>(c, f.kbuf, f.u, f.inv_sqrt_n);
        phase_psi(c, f.u, cur, src);                         // r_k = r~_k + Psi u' (line 4)
        phase_sure(c, cur, k);                               // tau, theta, alpha (lines 5-7)
        if (f.x_hat_iters) {
            SrcSpec w;
            w.mode = SRC_SOFT;
            w.r = cur;
            w.coef = f.coef;
            w.B = f.B;
            phase_final(c, w, f.x_hat_iters + (size_t)k * c.batch * f.N);
        }
        float2* t = prev;
        prev = cur;
        cur = t;
    }
    SrcSpec w;
    w.mode = SRC_SOFT;
    w.r = prev;
    w.coef = f.coef;
    w.B = f.B;
    phase_final(c, w, f.x_hat);                              // return line
    if (f.r_tilde_out) {                                     // line 8, state to resume from
        SrcSpec l8;
        l8.mode = SRC_LINE8;
        l8.r = prev;
        l8.coef = f.coef;
        l8.B = f.B;
        line8_range(f.l8, l8, f.r_tilde_out, c.slice, (size_t)c.rank * blockDim.x + threadIdx.x,
                    f.N, (size_t)c.C * blockDim.x);
    }
}

cudaError_t fused_configure(int cluster, size_t smem, int* max_clusters) {
    cudaError_t e = cudaFuncSetAttribute(fused_solve_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (cluster > 8) {
        e = cudaFuncSetAttribute(fused_solve_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster, 1, 1);
    cfg.blockDim = dim3(1024, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(max_clusters, fused_solve_kernel, &cfg);
}

cudaError_t launch_fused(const FusedArgs& f, int batch, size_t smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(f.C, batch, 1);
    cfg.blockDim = dim3(1024, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = f.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    cudaError_t e = cudaLaunchKernelEx(&cfg, fused_solve_kernel, f);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace vdamp

// Orthonormal periodic 2D wavelet transform Psi and its adjoint Psi^H
// (Sec. 1, Eq. 5-6), one scale per launch; the tile code is in dwt_dev.cuh.
#include <cooperative_groups.h>

#include "dwt_dev.cuh"

namespace cg = cooperative_groups;

namespace vdamp {

#define DWT_TO 16   // analysis: default output coefficients per tile side
#define IDWT_TO 32  // synthesis: default output pixels per tile side

__global__ void __launch_bounds__(256) dwt_level_kernel(const __grid_constant__ DwtArgs a) {
    extern __shared__ float2 sm[];
    cudaGridDependencySynchronize();
    dwt_tile(a, a.in, a.packed, a.src, blockIdx.x, blockIdx.y, blockIdx.z, sm);
}

cudaError_t launch_dwt_level(const DwtArgs& a_in, int batch, cudaStream_t st) {
    DwtArgs a = a_in;
    if (a.to != 16 && a.to != 32 && a.to != 64) a.to = DWT_TO;
    const int Ho = a.H >> 1, Wo = a.W >> 1;
    dim3 grid((Wo + a.to - 1) / a.to, (Ho + a.to - 1) / a.to, batch);
    return launch_pdl(dwt_level_kernel, grid, dim3(256), dwt_tile_smem(a.to, a.f.L), st, a);
}

__global__ void __launch_bounds__(256) idwt_level_kernel(const __grid_constant__ IdwtArgs a) {
    extern __shared__ float2 sm[];
    cudaGridDependencySynchronize();
    idwt_tile(a, a.out, a.src, blockIdx.x, blockIdx.y, blockIdx.z, sm);
}

cudaError_t launch_idwt_level(const IdwtArgs& a_in, int batch, cudaStream_t st) {
    IdwtArgs a = a_in;
    if (a.to != 16 && a.to != 32 && a.to != 64) a.to = IDWT_TO;
    const int Ho = 2 * a.h, Wo = 2 * a.w;
    dim3 grid((Wo + a.to - 1) / a.to, (Ho + a.to - 1) / a.to, batch);
    return launch_pdl(idwt_level_kernel, grid, dim3(256), idwt_tile_smem(a.to, a.f.L), st, a);
}

// r~_{k+1} written out (line 8), for resume and the single-iteration call.
__global__ void line8_kernel(const __grid_constant__ Line8Args a) {
    cudaGridDependencySynchronize();
    line8_range(a, a.src, a.out, blockIdx.y, (size_t)blockIdx.x * blockDim.x + threadIdx.x, a.N,
                (size_t)gridDim.x * blockDim.x);
}

cudaError_t launch_line8(const Line8Args& a, int batch, cudaStream_t st) {
    int blocks = (int)((a.N + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    return launch_pdl(line8_kernel, dim3(blocks, batch), dim3(256), 0, st, a);
}

// ------------------------------------------------ one launch for all scales ---
// Every CTA of a cluster runs the same scale loop and the same number of
// cluster barriers (the control flow depends only on launch arguments).
__global__ void __launch_bounds__(256) psi_h_cluster_kernel(const __grid_constant__ WaveletArgs w) {
    extern __shared__ float2 sm[];
    cudaGridDependencySynchronize();
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), C = (int)cl.num_blocks(), slice = blockIdx.y;
    for (int j = w.levels; j >= w.lo; --j) {
        const IdwtArgs& a = w.idwt[j - 1];
        const int ntx = (2 * a.w + a.to - 1) / a.to, nty = (2 * a.h + a.to - 1) / a.to;
        for (int t = rank; t < ntx * nty; t += C) {
            idwt_tile(a, a.out, a.src, t % ntx, t / ntx, slice, sm);
            __syncthreads();
        }
        if (j > w.lo) cl.sync();   // the next scale reads this scale's LL image
    }
}

__global__ void __launch_bounds__(256) psi_cluster_kernel(const __grid_constant__ WaveletArgs w) {
    extern __shared__ float2 sm[];
    cudaGridDependencySynchronize();
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), C = (int)cl.num_blocks(), slice = blockIdx.y;
    for (int j = w.lo; j <= w.levels; ++j) {
        const DwtArgs& a = w.dwt[j - 1];
        const int Ho = a.H >> 1, Wo = a.W >> 1;
        const int ntx = (Wo + a.to - 1) / a.to, nty = (Ho + a.to - 1) / a.to;
        for (int t = rank; t < ntx * nty; t += C) {
            dwt_tile(a, a.in, a.packed, a.src, t % ntx, t / ntx, slice, sm);
            __syncthreads();
        }
        if (j < w.levels) cl.sync();   // the next scale reads this scale's LL image
    }
}

template <typename K>
static cudaError_t launch_cluster(K kern, const WaveletArgs& w, int batch, int cluster,
                                  size_t smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster, batch, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, w);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_psi_h_cluster(const WaveletArgs& w, int batch, int cluster, size_t smem,
                                 cudaStream_t st) {
    return launch_cluster(psi_h_cluster_kernel, w, batch, cluster, smem, st);
}

cudaError_t launch_psi_cluster(const WaveletArgs& w, int batch, int cluster, size_t smem,
                               cudaStream_t st) {
    return launch_cluster(psi_cluster_kernel, w, batch, cluster, smem, st);
}

cudaError_t configure_wavelet_cluster(int cluster, size_t smem, int* max_clusters) {
    for (auto k : {psi_h_cluster_kernel, psi_cluster_kernel}) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        if (cluster > 8) {
            e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(max_clusters, psi_h_cluster_kernel, &cfg);
}

cudaError_t configure_dwt(size_t smem_bytes) {
    // the attribute is per kernel and process-wide: only ever raise it
    static size_t raised = 48 * 1024;
    if (smem_bytes <= raised) return cudaSuccess;
    raised = smem_bytes;
    cudaError_t e = cudaFuncSetAttribute(dwt_level_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(idwt_level_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes);
}

}  // namespace vdamp

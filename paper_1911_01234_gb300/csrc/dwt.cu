// Orthonormal periodic 2D wavelet transform Psi and its adjoint Psi^H
// (Sec. 1, Eq. 5-6), one scale per launch; the tile code is in dwt_dev.cuh.
#include "dwt_dev.cuh"

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

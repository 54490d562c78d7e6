// SURE threshold step of the VDAMP iteration (Algorithm 1 lines 5-7) as two
// kernels: the parallel sort of the subband magnitudes, then the parallel
// exact minimiser search, both split into parts per subband; or, with one
// part per subband (many slices), as one kernel doing both in the same CTA.  The arithmetic is in sure_dev.cuh.
#include "sure_dev.cuh"

namespace vdamp {

__global__ void __launch_bounds__(SURE_THREADS) sure_sort_kernel(const __grid_constant__ SureArgs a) {
    extern __shared__ float sm_keys[];
    cudaGridDependencySynchronize();
    // the finest (largest) subbands first: the long CTAs start in the first wave
    sure_sort_part(a, a.r, blockIdx.x, a.B - 1 - (int)blockIdx.y, blockIdx.z, sm_keys);
}

__global__ void __launch_bounds__(SURE_THREADS) sure_search_kernel(const __grid_constant__ SureArgs a) {
    extern __shared__ float sm_keys[];
    cudaGridDependencySynchronize();
    sure_search_part(a, a.k, blockIdx.x, a.B - 1 - (int)blockIdx.y, blockIdx.z, sm_keys);
}

// One CTA per subband (max_parts == 1): sort, then search the keys the sort
// left in shared memory.
__global__ void __launch_bounds__(SURE_THREADS) sure_one_cta_kernel(const __grid_constant__ SureArgs a) {
    extern __shared__ float sm_keys[];
    cudaGridDependencySynchronize();
    const int b = a.B - 1 - (int)blockIdx.y;
    sure_sort_part_f<true>(a, a.r, 0, b, blockIdx.z, sm_keys);
    __syncthreads();
    sure_search_part_t<true>(a, a.k, 0, b, blockIdx.z, sm_keys);
}

// Shared memory the SURE kernels are configured for: subbands held whole (up
// to SURE_SMALL_BAND coefficients) or one part of a larger subband.
size_t sure_smem(int max_band) { return sure_split_smem_bytes(max_band); }

cudaError_t launch_sure(const SureArgs& a, int batch, int max_band, cudaStream_t st) {
    if (a.max_parts == 1)
        return launch_pdl(sure_one_cta_kernel, dim3(1, a.B, batch), dim3(SURE_THREADS),
                          sure_smem_bytes(max_band), st, a);
    cudaError_t e = launch_pdl(sure_sort_kernel, dim3(a.max_parts, a.B, batch),
                               dim3(SURE_THREADS), sure_split_smem_bytes(max_band), st, a);
    if (e != cudaSuccess) return e;
    return launch_pdl(sure_search_kernel, dim3(a.max_parts, a.B, batch), dim3(SURE_THREADS),
                      sure_split_search_smem_bytes(max_band), st, a);
}

cudaError_t configure_sure(size_t smem_bytes) {
    // the attribute is per kernel and process-wide: only ever raise it
    static size_t raised = 48 * 1024;
    if (smem_bytes <= raised) return cudaSuccess;
    raised = smem_bytes;
    cudaError_t e = cudaFuncSetAttribute(sure_sort_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sure_one_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sure_search_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes);
}

}  // namespace vdamp

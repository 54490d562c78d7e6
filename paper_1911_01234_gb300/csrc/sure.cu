// SURE threshold step of the VDAMP iteration (Algorithm 1 lines 5-7) as two
// kernels: the parallel sort of the subband magnitudes, then the parallel
// exact minimiser search, both split into parts per subband; or, with one
// part per subband (many slices), the pruned exact search of one CTA per
// subband and a one-wave kernel for the subbands it leaves to the full sort.
// The arithmetic is in sure_dev.cuh and sure_prune_dev.cuh.
#include <algorithm>

#include "sure_prune_dev.cuh"

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

// One CTA per subband (max_parts == 1, many slices): the pruned exact search
// (sure_prune_dev.cuh); subbands it cannot take go to the fallback list.
__global__ void __launch_bounds__(PRUNE_THREADS) sure_prune_kernel(const __grid_constant__ SureArgs a) {
    extern __shared__ unsigned sm_words[];
    cudaGridDependencySynchronize();
    sure_prune_subband(a, a.B - 1 - (int)blockIdx.y, blockIdx.z, sm_words);
}

// The subbands on the fallback list, one after another per CTA (a fixed grid,
// one wave): the full bucket sort in shared memory, then the search on it.
// The last CTA to finish empties the list for the next launch.
__global__ void __launch_bounds__(SURE_THREADS) sure_fallback_kernel(const __grid_constant__ SureArgs a) {
    extern __shared__ float sm_keys[];
    __shared__ int s_n;
    cudaGridDependencySynchronize();
    if (threadIdx.x == 0) s_n = *reinterpret_cast<volatile int*>(&a.fallback[0]);
    __syncthreads();
    const int n = s_n;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int id = a.fallback[3 + i];
        const int slice = id / a.B, b = id - slice * a.B;
        sure_sort_part_f<true>(a, a.r, 0, b, slice, sm_keys);
        __syncthreads();
        sure_search_part_t<true>(a, a.k, 0, b, slice, sm_keys);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&a.fallback[1], 1) == (int)gridDim.x - 1) {   // every CTA has read n
            a.fallback[0] = 0;
            a.fallback[1] = 0;
        }
    }
}

// Shared memory the SURE kernels are configured for: subbands held whole (up
// to SURE_SMALL_BAND coefficients) or one part of a larger subband.
size_t sure_smem(int max_band) { return sure_split_smem_bytes(max_band); }

cudaError_t launch_sure(const SureArgs& a, int batch, int max_band, int fallback_ctas,
                        cudaStream_t st) {
    if (a.max_parts == 1) {
        cudaError_t e = launch_pdl(sure_prune_kernel, dim3(1, a.B, batch), dim3(PRUNE_THREADS),
                                   prune_smem_bytes(max_band), st, a);
        if (e != cudaSuccess) return e;
        return launch_pdl(sure_fallback_kernel, dim3(fallback_ctas), dim3(SURE_THREADS),
                          sure_smem_bytes(max_band), st, a);
    }
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
    e = cudaFuncSetAttribute(sure_fallback_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sure_prune_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)std::min(smem_bytes, (size_t)(227 * 1024)));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sure_search_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes);
}

}  // namespace vdamp

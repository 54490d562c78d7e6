// SURE threshold step of the VDAMP iteration (Algorithm 1 lines 5-7) as two
// kernels: the parallel sort of the subband magnitudes, then the parallel
// exact minimiser search, both split into parts per subband; or, with one
// part per subband (many slices), the pruned exact search of one CTA per
// subband and a one-wave kernel for the subbands it leaves to the full sort.
// The arithmetic is in sure_dev.cuh and sure_prune_dev.cuh.
#include "sure_prune_dev.cuh"

namespace vdamp {

__global__ void __launch_bounds__(SURE_THREADS) sure_sort_kernel(const __grid_constant__ SureArgs a) {
    extern __shared__ float sm_keys[];
    cudaGridDependencySynchronize();
    // the finest (largest) subbands first: the long CTAs start in the first wave
    sure_sort_part(a, a.r, blockIdx.x, a.b_top - (int)blockIdx.y, blockIdx.z, sm_keys);
}

__global__ void __launch_bounds__(SURE_THREADS) sure_search_kernel(const __grid_constant__ SureArgs a) {
    extern __shared__ float sm_keys[];
    cudaGridDependencySynchronize();
    sure_search_part(a, a.k, blockIdx.x, a.b_top - (int)blockIdx.y, blockIdx.z, sm_keys);
}

// Many slices (max_parts == 1): the pruned exact search (sure_prune_dev.cuh),
// one large subband, two medium or four small ones per CTA; subbands it cannot
// take go to the fallback list.  Grid: (work items of a slice, batch), the finest
// first; a launch may take a range of the items (from item0).
__global__ void __launch_bounds__(PRUNE_THREADS, 1) sure_prune_kernel(const __grid_constant__ SureArgs a) {
    extern __shared__ unsigned sm_words[];
    __shared__ PruneShared sh[PRUNE_GROUPS];
    cudaGridDependencySynchronize();
    const int slice = blockIdx.y, item = blockIdx.x + a.item0;
    const int ns = prune_n_small(a.off, a.B), nm = prune_n_med(a.off, a.B, ns);
    const int nbig = a.B - ns - nm;
    constexpr int per_med = PRUNE_THREADS / PRUNE_MED;
    const int cmed = (nm + per_med - 1) / per_med;
    if (item < nbig) {   // a large subband
        sure_prune_subband<PRUNE_THREADS>(a, a.B - 1 - item, slice, sm_words, sh[0], threadIdx.x, 0);
        return;
    }
    if (item < nbig + cmed) {   // two medium subbands
        const int g = threadIdx.x / PRUNE_MED;
        const int b = ns + (item - nbig) * per_med + g;
        if (b < ns + nm)
            sure_prune_subband<PRUNE_MED>(a, b, slice, sm_words + g * prune_words<PRUNE_MED>(), sh[g],
                                          threadIdx.x % PRUNE_MED, 1 + g);
        return;
    }
    const int g = threadIdx.x / PRUNE_GROUP;   // four small subbands
    const int b = (item - nbig - cmed) * PRUNE_GROUPS + g;
    if (b < ns)
        sure_prune_subband<PRUNE_GROUP>(a, b, slice, sm_words + g * prune_words<PRUNE_GROUP>(), sh[g],
                                        threadIdx.x % PRUNE_GROUP, 1 + g);
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
        cudaError_t e = launch_pdl(sure_prune_kernel, dim3(a.nb_launch, batch),
                                   dim3(PRUNE_THREADS), prune_smem_bytes(), st, a);
        if (e != cudaSuccess) return e;
        return launch_pdl(sure_fallback_kernel, dim3(fallback_ctas), dim3(SURE_THREADS),
                          sure_smem_bytes(max_band), st, a);
    }
    // subbands b_top, b_top - 1, ..., b_top - nb_launch + 1 (the finest first)
    cudaError_t e = launch_pdl(sure_sort_kernel, dim3(a.max_parts, a.nb_launch, batch),
                               dim3(SURE_THREADS), sure_split_smem_bytes(max_band), st, a);
    if (e != cudaSuccess) return e;
    return launch_pdl(sure_search_kernel, dim3(a.max_parts, a.nb_launch, batch), dim3(SURE_THREADS),
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
    // the pruned search always takes its largest layout (one CTA-wide subband)
    e = cudaFuncSetAttribute(sure_prune_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)prune_smem_bytes());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sure_search_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes);
}

}  // namespace vdamp

// The fused column pass of the VDAMP iteration (Algorithm 1 lines 3-5 between
// the forward and the inverse column transform of the unitary 2D DFT, Sec. 1):
// kernel, launch and configuration; the device code is in fft_dev.cuh.
#include "fft_dev.cuh"

namespace vdamp {

size_t col_pass_smem(int ny, int cb, int ntypes) { return col_pass_smem_bytes(ny, cb, ntypes); }

__global__ void __launch_bounds__(512, 2) col_pass_kernel(const __grid_constant__ ColArgs a) {
    extern __shared__ float2 sm[];
    cudaGridDependencySynchronize();
    col_pass_dispatch(a, a.mode, a.u_zero, blockIdx.x, gridDim.x, blockIdx.y, sm);
}

cudaError_t launch_col_pass(const ColArgs& a, int batch, cudaStream_t st) {
    dim3 grid(a.nx / a.cb, batch);
    int threads = a.ny * a.cb / 4;
    threads = threads < 64 ? 64 : (threads > 512 ? 512 : threads);
    threads = (threads + 31) / 32 * 32;
    // every thread keeps one column: blockDim must be a multiple of cb
    while (threads % a.cb) threads += 32;
    size_t smem = col_pass_smem(a.ny, a.cb, a.ntypes);
    return launch_pdl(col_pass_kernel, grid, dim3(threads), smem, st, a);
}

cudaError_t configure_col_pass(size_t smem_bytes) {
    // the attribute is per kernel and process-wide: only ever raise it
    static size_t raised = 48 * 1024;
    if (smem_bytes <= raised) return cudaSuccess;
    raised = smem_bytes;
    return cudaFuncSetAttribute(col_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes);
}

}  // namespace vdamp

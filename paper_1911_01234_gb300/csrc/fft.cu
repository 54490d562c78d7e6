// Unitary 2D DFT (Phi = M_Omega F, Sec. 1) for the VDAMP iteration: the row
// kernel (the fused column pass is in fft_col.cu); the device code is in
// fft_dev.cuh.
#include "fft_dev.cuh"

namespace vdamp {

template <bool INV>
__global__ void fft_rows_kernel(const float2* in, float2* out, int ny, int nx,
                                const __grid_constant__ FftAxis ax, float scale, int rpc) {
    extern __shared__ float2 sm[];
    cudaGridDependencySynchronize();
    const int row0 = blockIdx.x * rpc;
    fft_rows_dispatch<INV>(in, out, ny, nx, ax, scale, row0, min(rpc, ny - row0), blockIdx.y, sm);
}

cudaError_t launch_fft_rows(const float2* in, float2* out, int ny, int nx, int batch,
                            const FftAxis& ax, int inverse, float scale, int rpc,
                            int plan_batch, cudaStream_t st) {
    dim3 grid((ny + rpc - 1) / rpc, batch);
    // a plan whose largest batch fills the GPU: one thread per butterfly of the
    // axis plan's largest radix, so that its stages keep every lane busy (a
    // smaller radix loops over the butterflies); a plan for few slices (latency-
    // bound): more threads.  Decided by the plan, not by the call's batch, so
    // that a slice gives the same bits in any batch.
    const bool full = (long long)grid.x * plan_batch >= device_sms();
    int threads = rpc * nx / (full ? max_radix(ax) : 4);
    threads = threads < 32 ? 32 : (threads > 512 ? 512 : threads);
    threads = (threads + 31) / 32 * 32;
    size_t smem = 2 * (size_t)rpc * nx * sizeof(float2);
    if (inverse)
        return launch_pdl(fft_rows_kernel<true>, grid, dim3(threads), smem, st, in, out, ny, nx,
                          ax, scale, rpc);
    return launch_pdl(fft_rows_kernel<false>, grid, dim3(threads), smem, st, in, out, ny, nx, ax,
                      scale, rpc);
}

cudaError_t configure_fft_rows(size_t smem_bytes) {
    // the attribute is per kernel and process-wide: only ever raise it
    static size_t raised = 48 * 1024;
    if (smem_bytes <= raised) return cudaSuccess;
    raised = smem_bytes;
    cudaError_t e = cudaFuncSetAttribute(fft_rows_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fft_rows_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes);
}

}  // namespace vdamp

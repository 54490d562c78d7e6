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
    // threads per butterfly as in launch_fft_rows
    const bool full = (long long)grid.x * (a.plan_batch > 0 ? a.plan_batch : batch) >= device_sms();
    int threads = a.ny * a.cb / (full ? max_radix(a.ax) : 4);
    threads = threads < 64 ? 64 : (threads > 512 ? 512 : threads);
    threads = (threads + 31) / 32 * 32;
    // every thread keeps one column: blockDim must be a multiple of cb
    while (threads % a.cb) threads += 32;
    size_t smem = col_pass_smem(a.ny, a.cb, a.ntypes);
    return launch_pdl(col_pass_kernel, grid, dim3(threads), smem, st, a);
}

// Sampled entries of one column block (grid: column blocks x slices, 32 threads
// per row group): lane l of a warp takes column l % cb of rows r0 + l / cb, so a
// warp reads 32 / cb consecutive rows of the block's cb columns; a ballot ranks
// the sampled entries of each column in row order.
__global__ void kspace_list_kernel(const __grid_constant__ ColArgs a) {
    cudaGridDependencySynchronize();
    const int cb = a.cb, ny = a.ny, nx = a.nx, cblk = blockIdx.x, slice = blockIdx.y;
    const int nparts = nx / cb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int c = lane % cb, rpw = 32 / cb;     // rows per warp step
    // this warp's share of the rows: [r_begin, r_end), in steps of rpw
    const int steps = (ny + rpw - 1) / rpw;
    const int per = (steps + nw - 1) / nw * rpw;
    const int r_begin = min(warp * per, ny), r_end = min(r_begin + per, ny);
    const size_t g0 = (size_t)slice * ny * nx + (size_t)cblk * cb + c;
    unsigned colmask = 0u;   // the lanes of this lane's column
    for (int l = c; l < 32; l += cb) colmask |= 1u << l;
    const unsigned below = (1u << lane) - 1u;
    // pass 1: counts of this warp's rows, per column
    int mine = 0;
    for (int r0 = r_begin; r0 < r_end; r0 += rpw) {
        const int row = r0 + lane / cb;
        const bool m = row < r_end && a.mask[g0 + (size_t)row * nx] != 0;
        mine += __popc(__ballot_sync(0xffffffffu, m) & colmask);
    }
    __shared__ int s_cnt[16][32];   // [warp][column]
    if (lane < cb) s_cnt[warp][lane] = mine;   // mine is the same on every lane of column c
    __syncthreads();
    int cursor = 0;   // entries of column c in the warps before this one
    for (int w = 0; w < warp; ++w) cursor += s_cnt[w][c];
    const size_t lb = ((size_t)slice * nparts + cblk) * cb + c;
    KEntry* el = const_cast<KEntry*>(a.klist) + lb * ny;
    // pass 2: the entries, in row order
    for (int r0 = r_begin; r0 < r_end; r0 += rpw) {
        const int row = r0 + lane / cb;
        const size_t g = g0 + (size_t)row * nx;
        const bool m = row < r_end && a.mask[g] != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, m) & colmask;
        if (m) {
            KEntry k;
            k.row = row;
            k.w = __frcp_rn(a.density[g]);
            k.y = a.y[g];
            el[cursor + __popc(bal & below)] = k;
        }
        cursor += __popc(bal);
    }
    if (warp == nw - 1 && lane < cb) const_cast<int*>(a.kcnt)[lb] = cursor;
}

cudaError_t launch_kspace_list(const ColArgs& a, int batch, cudaStream_t st) {
    // up to 16 warps, each a run of rows of the block (32 / cb rows per step)
    int nw = (a.ny * a.cb + 31) / 32;
    nw = nw < 1 ? 1 : (nw > 16 ? 16 : nw);
    return launch_pdl(kspace_list_kernel, dim3(a.nx / a.cb, batch), dim3(32 * nw), 0, st, a);
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

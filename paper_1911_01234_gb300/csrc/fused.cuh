// Arguments and launchers of the persistent cluster solve (fused.cu).
#pragma once

#include "vdamp_internal.cuh"

namespace vdamp {

struct FusedArgs {
    int C;                   // CTAs per cluster (one cluster per slice)
    int levels, B, iters;
    size_t N;
    int ny, nx;
    int rpc, nrowblk;        // FFT rows per work item, number of row work items
    int nparts;              // column work items (= tau partial sums per slice)
    float inv_sqrt_n;
    FftAxis axx;
    IdwtArgs idwt[VDAMP_MAX_LEVELS];  // scale j at [j - 1]; src and the level-1 output set in-kernel
    DwtArgs dwt[VDAMP_MAX_LEVELS];    // scale j at [j - 1]; src, packed and the level-1 input set in-kernel
    ColArgs col;                      // mode and u_zero set in-kernel
    SureArgs sure;                    // r and k set in-kernel
    Line8Args l8;
    const float2* r_tilde0;
    float2* x_hat;
    float2* r_tilde_out;
    float2* x_hat_iters;
    float2* u;
    float2* kbuf;
    float2* rA;
    float2* rB;
    const float4* coef;
};

// Sets the kernel's attributes and reports how many clusters of `cluster`
// CTAs (1024 threads, `smem` bytes each) can be resident at once.
cudaError_t fused_configure(int cluster, size_t smem, int* max_clusters);
// Grid (cluster, batch), cluster dims (cluster, 1, 1), 1024 threads.
cudaError_t launch_fused(const FusedArgs& f, int batch, size_t smem, cudaStream_t st);

}  // namespace vdamp

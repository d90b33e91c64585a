// vi_fifo_col.cu -- the FIFO column sweep as a standalone kernel (the body and its
// derivation are in vi_fifo_col.cuh).
#include <cuda_runtime.h>

#include <algorithm>

#include "vi_fifo_col.cuh"

namespace vib {

template <int DP, int LT1>
__global__ void __launch_bounds__(kColWarps * 32)
sweep_fifo_col_kernel(KernelParams kp, int mode, const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int lpr) {
    __shared__ __align__(16) ColSmem sm;
    // the next sweep may launch while this one runs; values and the solve state are
    // read only after the grids this launch depends on have completed
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    fifo_col_body<DP, 0, LT1>(kp, blockIdx.x, gridDim.x, mode, vin_arg, vout_arg, pol_arg, sm);
}

// one product, float-pair values, FIFO, a stock slot in the rest besides the arriving
// order's (m >= 2 with a pipeline, m >= 3 with lead time one), 2 <= Q+1 <= 32 and
// dmax <= 62
bool fifo_col_supported(const KernelParams &kp, int vk, int kahan) {
    const ProdParams &P = kp.p[0];
    return kp.n_products == 1 && vk == VK_PAIR && !kahan && kp.issuing == 0 && P.G >= 2 && P.G <= 32 &&
           P.dmax <= 62 && !kp.pc && ((P.L >= 2 && P.m >= 2) || (P.L == 1 && P.m >= 3)) && P.n_rest_slots >= 1;
}

template <int DP>
static cudaError_t describe_fifo_col_t(const KernelParams &kp, LaunchDesc &d) {
    const ProdParams &P = kp.p[0];
    const uint32_t ncol = P.nS / (uint32_t)P.G / (uint32_t)P.G;
    d.fn = (P.L == 1) ? (const void *)sweep_fifo_col_kernel<DP, 1> : (const void *)sweep_fifo_col_kernel<DP, 0>;
    d.grid = dim3((ncol + kColWarps - 1) / kColWarps);
    d.block = dim3(kColWarps * 32);
    d.smem = 0;
    d.lpr = 1;
    d.pdl = 1;
    d.n_pre = 0;
    return cudaSuccess;
}

cudaError_t describe_fifo_col(const KernelParams &kp, LaunchDesc &d) {
    switch (fifo_col_dp(kp.p[0].dmax)) {
        case 16: return describe_fifo_col_t<16>(kp, d);
        case 32: return describe_fifo_col_t<32>(kp, d);
        case 48: return describe_fifo_col_t<48>(kp, d);
        default: return describe_fifo_col_t<64>(kp, d);
    }
}

}  // namespace vib

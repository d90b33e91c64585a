// vi_batch.cu -- the solve server's batched sweep: one launch covers every
// admitted instance of a lane-width class.
#include "vi_group.cuh"

namespace vib {

// ---------------------------------------------------------------------------
// batched sweep for the solve server: one launch covers every active instance.
// Block b belongs to the slot s with block_start[s] <= b < block_start[s+1];
// each slot has its own tables, value buffers and SolveState.
// ---------------------------------------------------------------------------
template <int XW>
__global__ void __launch_bounds__(kGroupThreads)
sweep_batch_kernel(const KernelParams *kps, const int *modes, const int *lprs, const uint32_t *block_start,
                   int n_slots) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ KernelParams s_kp;
    __shared__ int s_slot;
    const uint32_t b = blockIdx.x;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_slots - 1;   // last slot with block_start <= b
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (block_start[mid] <= b) lo = mid; else hi = mid - 1;
        }
        s_slot = lo;
        s_kp = kps[lo];
    }
    __syncthreads();
    const int s = s_slot;
    const unsigned nb = block_start[s + 1] - block_start[s];
    const uint32_t local = b - block_start[s];
    const bool pipe = s_kp.p[0].L >= 2;
    if (s_kp.issuing) {
        if (pipe)
            group_body<XW, 1, VK_PAIR, 1>(s_kp, local, nb, modes[s], nullptr, nullptr, nullptr, lprs[s], smem_raw);
        else
            group_body<XW, 1, VK_PAIR, 0>(s_kp, local, nb, modes[s], nullptr, nullptr, nullptr, lprs[s], smem_raw);
    } else {
        if (pipe)
            group_body<XW, 0, VK_PAIR, 1>(s_kp, local, nb, modes[s], nullptr, nullptr, nullptr, lprs[s], smem_raw);
        else
            group_body<XW, 0, VK_PAIR, 0>(s_kp, local, nb, modes[s], nullptr, nullptr, nullptr, lprs[s], smem_raw);
    }
}

// lane-width class of the batched server kernel for an instance: one lane per
// rest with the smallest instantiated width >= Q+1 (two lanes above 24)
int batch_width(int G) {
    if (G <= 8) return 8;
    if (G <= 12) return 12;
    if (G <= 16) return 16;
    if (G <= 21) return 21;
    return 24;
}

// blocks and shared memory the batched kernel needs for one slot
void batch_geometry(const KernelParams &kp, int *lpr, uint32_t *blocks, size_t *smem) {
    const int G = kp.p[0].G;
    const int xw = batch_width(G);
    const int l = (G + xw - 1) / xw;
    const int rb = kGroupThreads / l;
    *lpr = l;
    *blocks = (kp.p[0].nS / (uint32_t)G + rb - 1) / rb;
    *smem = group_smem(kp, rb, VK_PAIR);
}

template <int XW>
static cudaError_t launch_batch_t(const KernelParams *kps, const int *modes, const int *lprs,
                                  const uint32_t *block_start, int n_slots, uint32_t total_blocks, size_t smem,
                                  cudaStream_t stream) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(sweep_batch_kernel<XW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    sweep_batch_kernel<XW><<<total_blocks, kGroupThreads, smem, stream>>>(kps, modes, lprs, block_start, n_slots);
    return cudaGetLastError();
}

cudaError_t launch_sweep_batch(int xw, const KernelParams *kps, const int *modes, const int *lprs,
                               const uint32_t *block_start, int n_slots, uint32_t total_blocks, size_t smem,
                               cudaStream_t stream) {
    switch (xw) {
        case 8: return launch_batch_t<8>(kps, modes, lprs, block_start, n_slots, total_blocks, smem, stream);
        case 12: return launch_batch_t<12>(kps, modes, lprs, block_start, n_slots, total_blocks, smem, stream);
        case 16: return launch_batch_t<16>(kps, modes, lprs, block_start, n_slots, total_blocks, smem, stream);
        case 21: return launch_batch_t<21>(kps, modes, lprs, block_start, n_slots, total_blocks, smem, stream);
        case 24: return launch_batch_t<24>(kps, modes, lprs, block_start, n_slots, total_blocks, smem, stream);
        default: return cudaErrorInvalidValue;
    }
}


}  // namespace vib

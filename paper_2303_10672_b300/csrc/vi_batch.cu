// vi_batch.cu -- the solve server's batched sweep: one launch covers every
// admitted instance of a lane-width class.
#include "vi_group.cuh"

namespace vib {

// ---------------------------------------------------------------------------
// batched sweep for the solve server: one launch covers every active instance.
// Block b belongs to the slot s with block_start[s] <= b < block_start[s+1];
// each slot has its own tables, value buffers and SolveState.
// ---------------------------------------------------------------------------
template <int XW, int LIFO, int LPIPE>
__global__ void __launch_bounds__(kGroupThreads, group_min_blocks(XW, LIFO))
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
    group_body<XW, LIFO, VK_PAIR, LPIPE>(s_kp, local, nb, modes[s], nullptr, nullptr, nullptr, lprs[s], smem_raw);
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

template <int XW, int LIFO, int LPIPE>
static cudaError_t prepare_batch_t() {
    return cudaFuncSetAttribute(sweep_batch_kernel<XW, LIFO, LPIPE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024);
}

template <int XW>
static cudaError_t prepare_batch_w() {
    cudaError_t e;
    if ((e = prepare_batch_t<XW, 0, 0>()) != cudaSuccess || (e = prepare_batch_t<XW, 0, 1>()) != cudaSuccess ||
        (e = prepare_batch_t<XW, 1, 0>()) != cudaSuccess || (e = prepare_batch_t<XW, 1, 1>()) != cudaSuccess)
        return e;
    return cudaSuccess;
}

// set the shared-memory attribute of every batched variant; this also loads them,
// so that no first launch pays for loading its code (the server calls it at creation)
cudaError_t prepare_sweep_batch() {
    cudaError_t e;
    if ((e = prepare_batch_w<8>()) != cudaSuccess || (e = prepare_batch_w<12>()) != cudaSuccess ||
        (e = prepare_batch_w<16>()) != cudaSuccess || (e = prepare_batch_w<21>()) != cudaSuccess ||
        (e = prepare_batch_w<24>()) != cudaSuccess)
        return e;
    return cudaSuccess;
}

template <int XW, int LIFO, int LPIPE>
static cudaError_t launch_batch_t(const KernelParams *kps, const int *modes, const int *lprs,
                                  const uint32_t *block_start, int n_slots, uint32_t total_blocks, size_t smem,
                                  cudaStream_t stream) {
    sweep_batch_kernel<XW, LIFO, LPIPE><<<total_blocks, kGroupThreads, smem, stream>>>(kps, modes, lprs, block_start,
                                                                                       n_slots);
    return cudaGetLastError();
}

template <int XW>
static cudaError_t launch_batch_w(int variant, const KernelParams *kps, const int *modes, const int *lprs,
                                  const uint32_t *block_start, int n_slots, uint32_t total_blocks, size_t smem,
                                  cudaStream_t stream) {
    switch (variant) {
        case 0: return launch_batch_t<XW, 0, 0>(kps, modes, lprs, block_start, n_slots, total_blocks, smem, stream);
        case 1: return launch_batch_t<XW, 0, 1>(kps, modes, lprs, block_start, n_slots, total_blocks, smem, stream);
        case 2: return launch_batch_t<XW, 1, 0>(kps, modes, lprs, block_start, n_slots, total_blocks, smem, stream);
        case 3: return launch_batch_t<XW, 1, 1>(kps, modes, lprs, block_start, n_slots, total_blocks, smem, stream);
        default: return cudaErrorInvalidValue;
    }
}

int batch_variant(const KernelParams &kp) { return (kp.issuing ? 2 : 0) + (kp.p[0].L >= 2 ? 1 : 0); }

cudaError_t launch_sweep_batch(int xw, int variant, const KernelParams *kps, const int *modes, const int *lprs,
                               const uint32_t *block_start, int n_slots, uint32_t total_blocks, size_t smem,
                               cudaStream_t stream) {
    switch (xw) {
        case 8: return launch_batch_w<8>(variant, kps, modes, lprs, block_start, n_slots, total_blocks, smem, stream);
        case 12: return launch_batch_w<12>(variant, kps, modes, lprs, block_start, n_slots, total_blocks, smem, stream);
        case 16: return launch_batch_w<16>(variant, kps, modes, lprs, block_start, n_slots, total_blocks, smem, stream);
        case 21: return launch_batch_w<21>(variant, kps, modes, lprs, block_start, n_slots, total_blocks, smem, stream);
        case 24: return launch_batch_w<24>(variant, kps, modes, lprs, block_start, n_slots, total_blocks, smem, stream);
        default: return cudaErrorInvalidValue;
    }
}


}  // namespace vib

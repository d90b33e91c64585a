// vi_batch.cu -- the solve server's persistent sweep kernel: one launch advances
// every admitted instance, each at its own pace.
#include "vi_fifo_col.cuh"
#include "vi_group.cuh"

namespace vib {

// ---------------------------------------------------------------------------
// persistent server kernel.  Every block loops: claim one block of some instance's
// current sweep (atomic add on the instance's ticket), run the factorised body on
// it, count it done; the block that finishes the sweep's last block re-opens the
// ticket for the next sweep, or for the extraction sweep once the stopping test
// (decided by the sweep's own last block, block_reduce_and_finalize) has passed,
// or closes the instance after its extraction.  No block ever waits for another:
// a block that finds nothing to claim sleeps briefly and polls again, until the
// budget of device time is spent, every listed instance has finished, or (with
// finish_exit_ns > 0) one has and the launch has run that long, and at most
// kServeMaxPolls times.  A sweep left
// partly claimed at exit continues in the next launch (its state is in memory).
//
// Memory ordering: the finishing block writes its values, fences, counts itself
// done; the last one fences again (acquire) before reading the sweep's outcome and
// fences before publishing the ticket (release).  A claiming block fences after its
// claim (acquire), so the values it gathers -- written by other blocks of this
// launch -- come through plain loads (group_body's COH = 1), not the read-only path.
// ---------------------------------------------------------------------------
constexpr unsigned kServeMaxPolls = 1u << 22;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int XW, int LIFO, int LPIPE>
__device__ __forceinline__ void serve_block(const KernelParams &kp, uint32_t b, unsigned nb, int mode, int lpr,
                                            unsigned char *smem) {
    group_body<XW, LIFO, VK_PAIR, LPIPE, 1>(kp, b, nb, mode, nullptr, nullptr, nullptr, lpr, smem);
}

template <int XW>
__device__ __forceinline__ void serve_variant(int variant, const KernelParams &kp, uint32_t b, unsigned nb, int mode,
                                              int lpr, unsigned char *smem) {
    switch (variant) {
        case 0: serve_block<XW, 0, 0>(kp, b, nb, mode, lpr, smem); break;
        case 1: serve_block<XW, 0, 1>(kp, b, nb, mode, lpr, smem); break;
        case 2: serve_block<XW, 1, 0>(kp, b, nb, mode, lpr, smem); break;
        default: serve_block<XW, 1, 1>(kp, b, nb, mode, lpr, smem); break;
    }
}

__global__ void __launch_bounds__(kGroupThreads, group_min_blocks(21, 0))
serve_kernel(const KernelParams *kps, SrvSlot *slots, const int *act, int n_act, unsigned long long budget_ns,
             unsigned long long finish_exit_ns, unsigned *finished) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ KernelParams s_kp;
    __shared__ int s_slot, s_stop, s_mode;
    __shared__ unsigned s_b, s_nb;
    const unsigned long long t_start = global_ns();
    const unsigned long long deadline = t_start + budget_ns;
    const int lane = threadIdx.x & 31;
    for (unsigned poll = 0; poll < kServeMaxPolls; ++poll) {
        if (threadIdx.x < 32) {
            // warp 0 looks at 32 instances per round of loads and claims from the first
            // one with an unclaimed block.  Every block scans in the same order (the host
            // lists the instances largest first), so the device works through one large
            // instance's sweep at a time: its value buffers then share L2 with few others
            int claimed = -1;
            unsigned claimed_b = 0, claimed_nb = 0;
            bool any_open = false;
            // decided by lane 0 and broadcast: the ballots below need the whole warp
            int late0 = 0;
            if (lane == 0) {
                const unsigned long long now = global_ns();
                late0 = now > deadline || (finish_exit_ns > 0ull && now > t_start + finish_exit_ns &&
                                           *(volatile unsigned *)finished > 0u);
            }
            const bool late = __shfl_sync(0xffffffffu, late0, 0) != 0;
            for (int base = 0; !late && base < n_act && claimed < 0; base += 32) {
                const int k = base + lane;
                int i = -1;
                bool open = false, cand = false;
                unsigned nb = 0;
                if (k < n_act) {
                    i = act[k];
                    const SrvSlot &S = slots[i];
                    open = *(volatile const int *)&S.phase != 2;
                    nb = S.nblocks;
                    cand = open && (unsigned)*(volatile const unsigned long long *)&S.ticket < nb;
                }
                any_open |= (__ballot_sync(0xffffffffu, open) != 0u);
                unsigned m = __ballot_sync(0xffffffffu, cand);
                while (m && claimed < 0) {
                    const int leader = __ffs(m) - 1;
                    unsigned t = 0;
                    if (lane == leader) t = (unsigned)atomicAdd(&slots[i].ticket, 1ull);
                    t = __shfl_sync(0xffffffffu, t, leader);
                    const unsigned lnb = __shfl_sync(0xffffffffu, nb, leader);
                    const int li = __shfl_sync(0xffffffffu, i, leader);
                    if (t < lnb) {
                        claimed = li;
                        claimed_b = t;
                        claimed_nb = lnb;
                    }
                    m &= ~(1u << leader);
                }
            }
            if (lane == 0) {
                s_slot = claimed;
                s_stop = (claimed < 0 && !any_open) ? 1 : 0;
                if (late) s_stop = 1;
                if (claimed >= 0) {
                    __threadfence();   // acquire: the previous sweep's values and outcome
                    s_b = claimed_b;
                    s_nb = claimed_nb;
                    s_mode = *(volatile const int *)&slots[claimed].mode;
                }
            }
        }
        __syncthreads();
        if (s_stop) break;
        const int i = s_slot;
        if (i < 0) {
            if (threadIdx.x == 0) __nanosleep(200);
            __syncthreads();
            continue;
        }
        {
            // the instance's parameters, copied by the whole block
            const uint32_t *src = (const uint32_t *)(kps + i);
            uint32_t *dst = (uint32_t *)&s_kp;
            for (int w = threadIdx.x; w < (int)(sizeof(KernelParams) / 4); w += blockDim.x) dst[w] = __ldg(src + w);
        }
        __syncthreads();
        const SrvSlot &S = slots[i];
        if (S.variant == kSrvColVariant) {
            // FIFO with dmax <= 46 where the column sweep applies: its body (the same arithmetic
            // as the standalone sweep)
            ColSmem &sm = *(ColSmem *)smem_raw;
            const int dp = fifo_col_dp(s_kp.p[0].dmax);
            if (s_kp.p[0].L == 1) {
                switch (dp) {
                    case 16: fifo_col_body<16, 1, 1>(s_kp, s_b, s_nb, s_mode, nullptr, nullptr, nullptr, sm); break;
                    case 32: fifo_col_body<32, 1, 1>(s_kp, s_b, s_nb, s_mode, nullptr, nullptr, nullptr, sm); break;
                    default: fifo_col_body<48, 1, 1>(s_kp, s_b, s_nb, s_mode, nullptr, nullptr, nullptr, sm); break;
                }
            } else {
                switch (dp) {
                    case 16: fifo_col_body<16, 1, 0>(s_kp, s_b, s_nb, s_mode, nullptr, nullptr, nullptr, sm); break;
                    case 32: fifo_col_body<32, 1, 0>(s_kp, s_b, s_nb, s_mode, nullptr, nullptr, nullptr, sm); break;
                    default: fifo_col_body<48, 1, 0>(s_kp, s_b, s_nb, s_mode, nullptr, nullptr, nullptr, sm); break;
                }
            }
        } else {
            switch (S.xw) {
                case 8: serve_variant<8>(S.variant, s_kp, s_b, s_nb, s_mode, S.lpr, smem_raw); break;
                case 12: serve_variant<12>(S.variant, s_kp, s_b, s_nb, s_mode, S.lpr, smem_raw); break;
                case 16: serve_variant<16>(S.variant, s_kp, s_b, s_nb, s_mode, S.lpr, smem_raw); break;
                default: serve_variant<21>(S.variant, s_kp, s_b, s_nb, s_mode, S.lpr, smem_raw); break;
            }
        }
        __syncthreads();   // every thread's stores of this block are issued
        if (threadIdx.x == 0) {
            SrvSlot &W = slots[i];
            __threadfence();   // release: this block's values before its count
            if (atomicAdd(&W.done, 1u) == s_nb - 1u) {
                __threadfence();   // acquire: every block of the sweep, and its finalize
                atomicExch(&W.done, 0u);
                unsigned long long next = ((atomicAdd(&W.ticket, 0ull) >> 32) + 1ull) << 32;
                if (s_mode == MODE_EXTRACT) {
                    W.phase = 2;
                    next |= kSrvClosed;
                } else if (!*(volatile const int *)&s_kp.st->keep_going) {
                    W.mode = MODE_EXTRACT;
                    W.phase = 1;
                }
                __threadfence();   // release: the new mode and phase before the ticket
                atomicExch(&W.ticket, next);
                if (s_mode == MODE_EXTRACT) atomicAdd(finished, 1u);
            }
        }
        __syncthreads();   // s_kp and the claim are reused by the next round
    }
}

// lane-width class of an instance in the server: one lane per rest with the smallest
// width >= Q+1 among those the server kernel carries (two lanes of 12 above 21)
int batch_width(int G) {
    if (G <= 8) return 8;
    if (G <= 12) return 12;
    if (G <= 16) return 16;
    if (G <= 21) return 21;
    return 12;
}

// blocks per sweep and shared memory of one instance in the server kernel
void batch_geometry(const KernelParams &kp, int *lpr, uint32_t *blocks, size_t *smem) {
    const int G = kp.p[0].G;
    if (batch_variant(kp) == kSrvColVariant) {
        const uint32_t ncol = kp.p[0].nS / (uint32_t)G / (uint32_t)G;
        *lpr = 1;
        *blocks = (ncol + kColWarps - 1) / kColWarps;
        *smem = sizeof(ColSmem);
        return;
    }
    const int xw = batch_width(G);
    const int l = (G + xw - 1) / xw;
    const int rb = kGroupThreads / l;
    *lpr = l;
    *blocks = (kp.p[0].nS / (uint32_t)G + rb - 1) / rb;
    *smem = group_smem(kp, rb, VK_PAIR);
}

int batch_variant(const KernelParams &kp) {
    // the server carries the column body up to the 48-entry pmf capacity (dmax <= 46), so
    // that the largest instantiations' registers do not weigh on the persistent kernel
    if (fifo_col_supported(kp, VK_PAIR, 0) && fifo_col_dp(kp.p[0].dmax) <= 48) return kSrvColVariant;
    return (kp.issuing ? 2 : 0) + (kp.p[0].L >= 2 ? 1 : 0);
}

// loads the kernel and lets it use up to 200 KiB of dynamic shared memory, so that no
// first launch pays for loading its code (the server calls it at creation)
cudaError_t prepare_sweep_batch() {
    return cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_serve(const KernelParams *kps, SrvSlot *slots, const int *act, int n_act, size_t smem,
                         unsigned long long budget_ns, unsigned long long finish_exit_ns, unsigned *finished,
                         cudaStream_t stream) {
    static thread_local size_t last_smem = (size_t)-1;
    static thread_local int last_grid = 0;
    if (smem != last_smem) {
        int dev = 0, nsm = 0, per_sm = 0;
        cudaError_t e;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
            (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_kernel, kGroupThreads, smem)) !=
                cudaSuccess)
            return e;
        last_grid = std::max(1, nsm * std::max(per_sm, 1));
        last_smem = smem;
    }
    serve_kernel<<<last_grid, kGroupThreads, smem, stream>>>(kps, slots, act, n_act, budget_ns, finish_exit_ns,
                                                            finished);
    return cudaGetLastError();
}

}  // namespace vib

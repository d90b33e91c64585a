// vi_kernels.h -- launchers of the sm_103a kernels (host side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vi_common.cuh"

namespace vib {

// launch modes of the sweep kernels
enum {
    MODE_SWEEP = 0,     // solve sweep: buffers and normalisation from SolveState, span stats, stop test
    MODE_EXTRACT = 1,   // extraction sweep: policy from V_iters, V_iters copied into the caller's buffer
    MODE_PLAIN = 2      // one backup between explicit buffers, no normalisation, change stats only
};

// how values are stored and combined (see vi_kernels.cu)
enum { VK_SINGLE = 0, VK_PAIR = 1, VK_DOUBLE = 2 };

constexpr int kGroupThreads = 128;   // rests per block of the factorised kernel
constexpr int kGenericThreads = 128;
constexpr int kMaxGroupG = 64;       // largest Q+1 run by the factorised kernel (lane width <= 24)
constexpr int kMaxRollDmax = 255;

struct RollParams {
    int n_rollouts, horizon, warmup;
    unsigned long long seed;
    double cost[2][5];
    unsigned long long thr[2][kMaxRollDmax + 1];   // floor(2^32 CDF(d)), thr[dmax] = 2^32
};

// modified base-stock search: slot bounds of the plain stock vectors, and the
// grid of order-up-to pairs (pair = (S_1 - s_lo[0]) * n2 + (S_2 - s_lo[1]))
constexpr int kMbsMaxM = 8;   // m <= 8
constexpr int kMbsMaxL = 4;   // L <= 4
struct MbsParams {
    int s_lo[2];
    int n2, n_pairs;
    int mu[2];
    int cap;
};

bool group_supported(const KernelParams &kp, int vk, int kahan);
cudaError_t launch_next_states(const KernelParams &kp, const uint32_t *states, int n, uint32_t *out,
                               cudaStream_t stream);
cudaError_t launch_policy_eval(const KernelParams &kp, const uint8_t *policy, const double *vin,
                               double *vout, cudaStream_t stream);
cudaError_t launch_to_fp64(const void *v, int vk, double offset, double *out, uint32_t n, cudaStream_t stream);
// max and min of a - b into st->dmax_abs / st->dmin_abs
cudaError_t launch_diff_range(const double *a, const double *b, uint32_t n, SolveState *st,
                              cudaStream_t stream);
cudaError_t launch_solve_init(SolveState *st, uint32_t n, cudaStream_t stream);

// what a graph kernel node needs (the dynamic shared-memory attribute is set)
struct LaunchDesc {
    const void *fn;
    dim3 grid, block;
    size_t smem;
    int lpr;    // lanes per rest of the factorised kernel (0 for the generic kernel)
    // kernels that run before fn in every sweep and extraction, with the same arguments
    int n_pre = 0;
    const void *pre_fn[2] = {nullptr, nullptr};
    dim3 pre_grid[2], pre_block[2];
    // 1: fn lets its dependents launch early and waits for the grids it depends on
    // (griddepcontrol) before it reads any value or solve state, so it may be launched
    // as a programmatic dependent of the previous sweep (its set-up overlaps that
    // sweep's last blocks)
    int pdl = 0;
};
// use_group = 0: generic kernel; kTcWidth: tensor-core FIFO kernel; otherwise the
// factorised kernel with that lane width XW
cudaError_t describe_sweep(const KernelParams &kp, int vk, int kahan, int use_group, LaunchDesc &d);
bool group_width_supported(int xw);
// lane-width token that selects the tensor-core FIFO sweep (vi_tc.cu)
constexpr int kTcWidth = 100;
// lane-width token of the factorised two-product sweep
constexpr int kTwoWidth = 200;
// lane-width token of the persistent LIFO sweep for lead time one (vi_lifo1.cuh)
constexpr int kLifo1Width = 300;
bool lifo1_supported(const KernelParams &kp, int vk, int kahan);
cudaError_t describe_lifo1(const KernelParams &kp, LaunchDesc &d);
// lane-width token of the FIFO sweep by columns of rests (vi_fifo_col.cu)
constexpr int kFifoColWidth = 400;
bool fifo_col_supported(const KernelParams &kp, int vk, int kahan);
cudaError_t describe_fifo_col(const KernelParams &kp, LaunchDesc &d);
bool two_supported(const KernelParams &kp, int vk, int kahan);
size_t two_table_floats(const KernelParams &kp, size_t *mix_floats);
// rows of the substitution mixture table: product-1 stock T1 = 0..min(dmax1, m1 Q1)
int two_mix_rows(const ProdParams &P1);
bool tc_supported(const KernelParams &kp, int vk, int kahan);
cudaError_t describe_tc(const KernelParams &kp, LaunchDesc &d);
int batch_width(int G);
void batch_geometry(const KernelParams &kp, int *lpr, uint32_t *blocks, size_t *smem);
// loads the persistent server kernel and sets its shared-memory limit (before the first launch)
cudaError_t prepare_sweep_batch();
// loads the server's helper kernels (status gather, FP64 conversion, solve init)
cudaError_t prepare_server_helpers();
// body an instance runs in the server: the factorised body's variant 2 * LIFO + (L >= 2),
// or kSrvColVariant for the FIFO column body (where fifo_col_supported, dmax <= 46)
constexpr int kSrvColVariant = 4;
int batch_variant(const KernelParams &kp);

// One admitted instance of the solve server, as the persistent server kernel sees it.
// Blocks of the kernel claim the blocks of an instance's current sweep from `ticket`
// (next block index in the low 32 bits); the block that completes a sweep's last
// block publishes the next sweep (or the extraction, once the stopping test passed)
// by resetting the ticket, so every instance advances at its own pace.
constexpr unsigned kSrvClosed = 0xFFFFFFFFu;   // low ticket word of an instance with nothing to claim
struct SrvSlot {
    unsigned long long ticket;   // (sweeps published << 32) | next unclaimed block of the current sweep
    unsigned done;               // blocks of the current sweep that have finished
    int mode;                    // MODE_SWEEP or MODE_EXTRACT for the current sweep
    int phase;                   // 0 sweeping, 1 extracting, 2 finished (extraction written)
    unsigned nblocks;            // blocks per sweep
    int xw, variant, lpr;        // body of the instance: lane width, variant, lanes per rest
    int pad;
};
// the persistent server kernel: blocks claim work over the instances listed in act[0..n_act)
// until every one has finished, budget_ns of device time have passed, or (finish_exit_ns
// > 0) one has finished after the launch ran finish_exit_ns (a bounded number of polls in
// any case)
cudaError_t launch_serve(const KernelParams *kps, SrvSlot *slots, const int *act, int n_act, size_t smem,
                         unsigned long long budget_ns, unsigned long long finish_exit_ns, unsigned *finished,
                         cudaStream_t stream);
struct SlotStatus {
    int iter, keep_going, converged, pad;
    double crit;
};
cudaError_t launch_gather_status(SolveState *const *sts, int n, SlotStatus *out, cudaStream_t stream);
int group_width_candidates(int G, int *out, int max_out);
cudaError_t describe_solve_init(uint32_t n, LaunchDesc &d);
cudaError_t launch_basestock(const KernelParams &kp, const RollParams &rp, int s_lo, int n_S, double *returns,
                             cudaStream_t stream);
cudaError_t launch_rollouts(const KernelParams &kp, const RollParams &rp, const uint8_t *policy,
                            double *returns, double *kpis, double *kpis_prod, int32_t *traj, cudaStream_t stream);
cudaError_t launch_mbs(const KernelParams &kp, const RollParams &rp, const MbsParams &mp, double *returns,
                       double *kpis_prod, cudaStream_t stream);
// periodic problems (vi_pc.cu)
struct PcRollParams {
    int n_rollouts, horizon, warmup;
    unsigned long long seed;
    const unsigned long long *thr_d;   // device, 7 x (dmax+1): floor(2^32 CDF(d)) of each weekday
    const unsigned long long *thr_y;   // device, (Q+1) x m: floor(2^32 (p_1(a) + .. + p_k(a)))
};
cudaError_t describe_pc(const KernelParams &kp, LaunchDesc &d);
cudaError_t launch_pc_rollouts(const KernelParams &kp, const PcRollParams &rp, const uint8_t *policy,
                               double *returns, double *kpis, int32_t *traj, cudaStream_t stream);

}  // namespace vib

// vi_pc.cu -- the paper's Scenario C on sm_103a: weekday-periodic demand and
// uncertain useful life on arrival (Scenario C appendix), in FP64.
//
// State s = tau G^(m-1) + sum_j X_j G^(j-1), G = A_max + 1: weekday tau and the
// units X_1..X_{m-1} with j days of life left.  An order a arrives at once as
// y_1..y_m units with k days left (multinomial, log(p_k / p_1) = c0_k + c1_k a);
// an age class keeps at most A_max units (Z_j = min(X_j + y_j, A_max), Z_m =
// y_m).  Demand of weekday tau is issued oldest first.
//
// The expectation splits at the delivery: with the post-decision value
//   W(tau, Z) = sum_d P(d | tau) [r(Z, d) + gamma V(tau + 1, X'(Z, d))]
// (holding, shortage and waste costs in r), one sweep is
//   V'(s) = max_a [ -C_f 1{a > 0} + sum_y P(y | a) W(tau, Z(X, y)) ].
// pc_post_kernel builds W for all 7 G^m post-decision states; pc_sweep_kernel
// takes the max over orders, one thread per state, the profiles y of each order
// (with their probabilities, built on the host in FP64) read uniformly by the
// whole warp.  The periodic stopping test (Su and Deininger, Scenario C
// appendix) keeps the last seven weighted differences gamma^-(i-1) (V_i - V_{i-1})
// per state in a ring and reduces their sum.
#include <math.h>

#include "vi_device.cuh"

namespace vib {

__global__ void __launch_bounds__(kGenericThreads)
pc_post_kernel(KernelParams kp, int mode, const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int) {
    SolveState *st = kp.st;
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    const ProdParams &P = kp.p[0];
    const uint32_t G = (uint32_t)P.G;
    const int m = kp.pc_m;
    const uint32_t Gm = P.nS * G;   // G^m post-decision stock vectors per weekday
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 7ull * Gm) return;
    const uint32_t tau = (uint32_t)(t / Gm);
    uint32_t rem = (uint32_t)(t - (uint64_t)tau * Gm);
    int Z[kPcMaxM];
    int T = 0;
#pragma unroll
    for (int j = 0; j < kPcMaxM; ++j) {
        Z[j] = 0;
        if (j < m) {
            const uint32_t q = rem / G;
            Z[j] = (int)(rem - q * G);
            rem = q;
            T += Z[j];
        }
    }
    const double *V = (const double *)B.vin;
    const double *pd = kp.pc_pmf + (size_t)tau * (P.dmax + 1);
    const uint32_t base = ((tau + 1) % 7) * P.nS;
    const double gam = kp.gamma;
    double w = 0.0;
    for (int d = 0; d <= P.dmax; ++d) {
        // oldest first: X'_j = [Z_{j+1} - [d - sum_{k<=j} Z_k]^+]^+
        uint32_t idx = 0, wgt = 1;
        int cum = 0;
#pragma unroll
        for (int j = 0; j < kPcMaxM - 1; ++j) {
            if (j < m - 1) {
                cum += Z[j];
                const int reach = max(d - cum, 0);
                idx += (uint32_t)max(Z[j + 1] - reach, 0) * wgt;
                wgt *= G;
            }
        }
        double r = 0.0;
        r = __dsub_rn(r, __dmul_rn(kp.pc_cost[1], (double)max(T - d, 0)));
        r = __dsub_rn(r, __dmul_rn(kp.pc_cost[2], (double)max(d - T, 0)));
        r = __dsub_rn(r, __dmul_rn(kp.pc_cost[3], (double)max(Z[0] - d, 0)));
        w = __fma_rn(pd[d], __fma_rn(gam, V[base + idx], r), w);
    }
    kp.pc_W[t] = w;
}

__global__ void __launch_bounds__(kGenericThreads)
pc_sweep_kernel(KernelParams kp, int mode, const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int) {
    SolveState *st = kp.st;
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    const ProdParams &P = kp.p[0];
    const uint32_t G = (uint32_t)P.G;
    const int m = kp.pc_m;
    const int Q = P.Q;
    double mx = -INFINITY, mn = INFINITY;
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < kp.nS) {
        const uint32_t tau = s / P.nS;
        uint32_t rem = s - tau * P.nS;
        int X[kPcMaxM];
#pragma unroll
        for (int j = 0; j < kPcMaxM; ++j) {
            X[j] = 0;
            if (j < m - 1) {
                const uint32_t q = rem / G;
                X[j] = (int)(rem - q * G);
                rem = q;
            }
        }
        const double *W = kp.pc_W + (size_t)tau * P.nS * G;
        double best = -INFINITY;
        int arg = 0;
        for (int a = 0; a <= Q; ++a) {
            double q = 0.0;
            const int c1 = kp.pc_off[a + 1];
            for (int c = kp.pc_off[a]; c < c1; ++c) {
                const unsigned long long prof = kp.pc_prof[c];
                uint32_t idx = 0, wgt = 1;
#pragma unroll
                for (int j = 0; j < kPcMaxM - 1; ++j) {
                    if (j < m - 1) {
                        const int y = (int)((prof >> (6 * j)) & 63ull);
                        idx += (uint32_t)min(X[j] + y, Q) * wgt;
                        wgt *= G;
                    }
                }
                idx += (uint32_t)((prof >> (6 * (m - 1))) & 63ull) * wgt;
                q = __fma_rn(kp.pc_prob[c], W[idx], q);
            }
            if (a > 0) q = __dsub_rn(q, kp.pc_cost[0]);
            if (q > best) {
                best = q;
                arg = a;
            }
        }
        const double vold = ((const double *)B.vin)[s];
        if (mode == MODE_EXTRACT) {
            if (B.vout) ((double *)B.vout)[s] = vold;
        } else {
            ((double *)B.vout)[s] = best;
            const double dlt = best - vold;
            if (mode == MODE_SWEEP && st->stop_rule == kStopPeriodic) {
                // slot (i-1) mod 7 held gamma^-(i-8) (V_{i-7} - V_{i-8}); the seven
                // slots now hold the terms of Delta_i
                const int it = st->iter;   // sweeps completed before this one: i - 1
                const size_t n = kp.nS;
                kp.pc_ring[(size_t)(it % 7) * n + s] = dlt / pow(kp.gamma, (double)it);
                double D = 0.0;
                for (int k = 0; k < 7; ++k) D += kp.pc_ring[(size_t)k * n + s];
                mx = mn = D;
            } else {
                mx = mn = dlt;
            }
        }
        if (B.pol) B.pol[s] = (uint8_t)arg;
    }
    if (mode != MODE_EXTRACT) block_reduce_and_finalize<double>(mx, mn, st, mode, gridDim.x);
}

// Few states (the paper's m = 3 settings: 3,087): one warp per state, the
// orders spread over the lanes (lane l takes a = l, l + 32, ..), then the first
// maximum over the warp by shuffles.  One thread per state would give the
// device a few blocks only.
__global__ void __launch_bounds__(kGenericThreads)
pc_sweep_warp_kernel(KernelParams kp, int mode, const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int) {
    SolveState *st = kp.st;
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    const ProdParams &P = kp.p[0];
    const uint32_t G = (uint32_t)P.G;
    const int m = kp.pc_m;
    const int Q = P.Q;
    const int lane = threadIdx.x & 31;
    double mx = -INFINITY, mn = INFINITY;
    const uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s < kp.nS) {
        const uint32_t tau = s / P.nS;
        uint32_t rem = s - tau * P.nS;
        int X[kPcMaxM];
#pragma unroll
        for (int j = 0; j < kPcMaxM; ++j) {
            X[j] = 0;
            if (j < m - 1) {
                const uint32_t q = rem / G;
                X[j] = (int)(rem - q * G);
                rem = q;
            }
        }
        const double *W = kp.pc_W + (size_t)tau * P.nS * G;
        double best = -INFINITY;
        int arg = 0x7fffffff;
        for (int a = lane; a <= Q; a += 32) {
            double q = 0.0;
            const int c1 = kp.pc_off[a + 1];
            for (int c = kp.pc_off[a]; c < c1; ++c) {
                const unsigned long long prof = kp.pc_prof[c];
                uint32_t idx = 0, wgt = 1;
#pragma unroll
                for (int j = 0; j < kPcMaxM - 1; ++j) {
                    if (j < m - 1) {
                        const int y = (int)((prof >> (6 * j)) & 63ull);
                        idx += (uint32_t)min(X[j] + y, Q) * wgt;
                        wgt *= G;
                    }
                }
                idx += (uint32_t)((prof >> (6 * (m - 1))) & 63ull) * wgt;
                q = __fma_rn(kp.pc_prob[c], W[idx], q);
            }
            if (a > 0) q = __dsub_rn(q, kp.pc_cost[0]);
            if (q > best) {
                best = q;
                arg = a;
            }
        }
        // first maximum over the lanes: larger value, or equal value and smaller order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
            if (ob > best || (ob == best && oa < arg)) {
                best = ob;
                arg = oa;
            }
        }
        if (lane == 0) {
            const double vold = ((const double *)B.vin)[s];
            if (mode == MODE_EXTRACT) {
                if (B.vout) ((double *)B.vout)[s] = vold;
            } else {
                ((double *)B.vout)[s] = best;
                const double dlt = best - vold;
                if (mode == MODE_SWEEP && st->stop_rule == kStopPeriodic) {
                    const int it = st->iter;
                    const size_t n = kp.nS;
                    kp.pc_ring[(size_t)(it % 7) * n + s] = dlt / pow(kp.gamma, (double)it);
                    double D = 0.0;
                    for (int k = 0; k < 7; ++k) D += kp.pc_ring[(size_t)k * n + s];
                    mx = mn = D;
                } else {
                    mx = mn = dlt;
                }
            }
            if (B.pol) B.pol[s] = (uint8_t)arg;
        }
    }
    if (mode != MODE_EXTRACT) block_reduce_and_finalize<double>(mx, mn, st, mode, gridDim.x);
}

// states below which a sweep takes one warp per state
constexpr uint32_t kPcWarpStates = 1u << 16;

cudaError_t describe_pc(const KernelParams &kp, LaunchDesc &d) {
    const uint64_t n_post = 7ull * kp.p[0].nS * (uint32_t)kp.p[0].G;
    const bool warp = kp.nS <= kPcWarpStates;
    d.fn = warp ? (const void *)pc_sweep_warp_kernel : (const void *)pc_sweep_kernel;
    d.grid = warp ? dim3((unsigned)(((uint64_t)kp.nS * 32 + kGenericThreads - 1) / kGenericThreads))
                  : dim3((kp.nS + kGenericThreads - 1) / kGenericThreads);
    d.block = dim3(kGenericThreads);
    d.smem = 0;
    d.lpr = 0;
    d.n_pre = 1;
    d.pre_fn[0] = (const void *)pc_post_kernel;
    d.pre_grid[0] = dim3((unsigned)((n_post + kGenericThreads - 1) / kGenericThreads));
    d.pre_block[0] = dim3(kGenericThreads);
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// rollouts of a Scenario C policy: thread = rollout, serial over periods.
// Period t of rollout r: demand from word 0 of Philox4x32-10(ctr (t, r, 0, 0))
// by the weekday's thresholds; unit u of the order takes its age class from
// word u % 4 of Philox4x32-10(ctr (t, r, 1 + u / 4, 0)).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pc_draw(uint32_t w, const unsigned long long *thr, int n) {
    int i = 0;
    while (i < n - 1 && (unsigned long long)w >= thr[i]) ++i;
    return i;
}

__global__ void pc_rollout_kernel(KernelParams kp, PcRollParams rp, const uint8_t *policy, double *returns,
                                  double *kpis, int32_t *traj) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rp.n_rollouts) return;
    const ProdParams &P = kp.p[0];
    const uint32_t G = (uint32_t)P.G;
    const int m = kp.pc_m;
    const int Q = P.Q;
    const int nd = P.dmax + 1;
    const uint32_t k0 = (uint32_t)(rp.seed & 0xffffffffull), k1 = (uint32_t)(rp.seed >> 32);
    uint32_t s = 0;
    double ret = 0.0, disc = 1.0;
    // unit counts summed as integers: exactly the FP64 running sums of the same counts
    long long dem = 0, iss = 0, was = 0, acc = 0, held = 0;
    for (int t = 0; t < rp.warmup + rp.horizon; ++t) {
        uint32_t w[4];
        philox4x32_10((uint32_t)t, (uint32_t)r, 0u, 0u, k0, k1, w);
        const uint32_t tau = s / P.nS;
        const int d = pc_draw(w[0], rp.thr_d + (size_t)tau * nd, nd);
        const int a = min((int)policy[s], Q);   // entries above A_max are read as A_max
        int y[kPcMaxM];
#pragma unroll
        for (int k = 0; k < kPcMaxM; ++k) y[k] = 0;
        const unsigned long long *ty = rp.thr_y + (size_t)a * m;
        uint32_t wu[4];
        for (int u = 0; u < a; ++u) {
            if ((u & 3) == 0) philox4x32_10((uint32_t)t, (uint32_t)r, (uint32_t)(1 + u / 4), 0u, k0, k1, wu);
            const int k = pc_draw(wu[u & 3], ty, m);
#pragma unroll
            for (int j = 0; j < kPcMaxM; ++j) y[j] += (j == k) ? 1 : 0;
        }
        // delivery with the age capacity, then demand oldest first
        uint32_t rem = s - tau * P.nS;
        int Z[kPcMaxM];
        int accepted = 0, T = 0;
#pragma unroll
        for (int j = 0; j < kPcMaxM; ++j) {
            Z[j] = 0;
            if (j < m - 1) {
                const uint32_t q = rem / G;
                const int x = (int)(rem - q * G);
                rem = q;
                Z[j] = min(x + y[j], Q);
                accepted += Z[j] - x;
            } else if (j == m - 1) {
                Z[j] = y[j];
                accepted += y[j];
            }
            T += Z[j];
        }
        uint32_t idx = 0, wgt = 1;
        int cum = 0;
#pragma unroll
        for (int j = 0; j < kPcMaxM - 1; ++j) {
            if (j < m - 1) {
                cum += Z[j];
                const int reach = max(d - cum, 0);
                idx += (uint32_t)max(Z[j + 1] - reach, 0) * wgt;
                wgt *= G;
            }
        }
        const int left = max(T - d, 0), shortage = max(d - T, 0), wasted = max(Z[0] - d, 0);
        double rew = 0.0;
        if (a > 0) rew = __dsub_rn(rew, kp.pc_cost[0]);
        rew = __dsub_rn(rew, __dmul_rn(kp.pc_cost[1], (double)left));
        rew = __dsub_rn(rew, __dmul_rn(kp.pc_cost[2], (double)shortage));
        rew = __dsub_rn(rew, __dmul_rn(kp.pc_cost[3], (double)wasted));
        if (t >= rp.warmup) {
            if (traj) traj[(size_t)r * rp.horizon + (t - rp.warmup)] = (int32_t)s;
            ret = __dadd_rn(ret, __dmul_rn(disc, rew));
            disc = __dmul_rn(disc, kp.gamma);
            dem += d;
            iss += min(d, T);
            was += wasted;
            acc += accepted;
            held += left;
        }
        s = ((tau + 1) % 7) * P.nS + idx;
    }
    returns[r] = ret;
    if (kpis) {
        const double fd = (double)dem, fi = (double)iss, fw = (double)was, fa = (double)acc;
        kpis[3 * r + 0] = fd > 0.0 ? __ddiv_rn(__dmul_rn(100.0, fi), fd) : 100.0;
        kpis[3 * r + 1] = fa > 0.0 ? __ddiv_rn(__dmul_rn(100.0, fw), fa) : 0.0;
        kpis[3 * r + 2] = rp.horizon > 0 ? __ddiv_rn((double)held, (double)rp.horizon) : 0.0;
    }
}

cudaError_t launch_pc_rollouts(const KernelParams &kp, const PcRollParams &rp, const uint8_t *policy,
                               double *returns, double *kpis, int32_t *traj, cudaStream_t stream) {
    const int threads = 128;
    const int blocks = (rp.n_rollouts + threads - 1) / threads;
    pc_rollout_kernel<<<blocks, threads, 0, stream>>>(kp, rp, policy, returns, kpis, traj);
    return cudaGetLastError();
}

}  // namespace vib

// vi_kernels.cu -- sm_103a kernels of the value-iteration hot path.
//
//   sweep_group_kernel    factorised Bellman backup: one thread per rest index r,
//                         the G = Q+1 values of the expiring slot in registers
//   sweep_generic_kernel  one thread per state; one or two products
//   next_states_kernel    dump of T(s, a, omega) indices (bit-exact checks)
//   policy_eval_kernel    FP64 fixed-policy sweep
//   rollout_kernel        Philox4x32-10 policy rollouts with FP64 returns
//
// Bellman backup (Eq. valueiterationdetupdate):
//   V'(s) = max_a [ rbar(s,a) + gamma * sum_omega P(omega) V(s'(s,a,omega)) ]
// The expected one-step reward rbar comes from FP64-built tables: the reward of
// Eq. demoor:reward is affine in issued / short / wasted / carried units, so its
// expectation only needs E[(y - D)^+].
//
// Value kinds:
//   VK_SINGLE  float per state relative to an FP64 offset b (V_abs = b + v); each
//              sweep subtracts a constant so that v stays near zero.
//   VK_PAIR    an unevaluated float pair per state (V_abs = hi + lo).  All FP32
//              arithmetic works on differences V(s') - V(ref) between states
//              (unchanged when V shifts uniformly, so rounding does not add noise
//              to V_i - V_{i-1}); only the final absolute value is formed with
//              error-free TwoSum / TwoProd steps.
//   VK_DOUBLE  FP64 per state.
#include <math.h>

#include <type_traits>

#include "vi_device.cuh"
#include "vi_group_dispatch.h"

namespace vib {

// ===========================================================================
// per-state expectation helpers (generic kernels, policy evaluation)
// ===========================================================================
template <typename T, int KAHAN>
struct Acc {
    T s, c;
    __device__ __forceinline__ void init() {
        s = (T)0;
        c = (T)0;
    }
    __device__ __forceinline__ void add(T w, T v) {
        if (KAHAN) {
            const T y = w * v - c;
            const T t = s + y;
            c = (t - s) - y;
            s = t;
        } else {
            s = s + w * v;
        }
    }
};

// value accessors: plain load, or pair relative to a reference state
template <typename T>
struct GetPlain {
    const T *V;
    __device__ __forceinline__ T operator()(uint32_t i) const { return V[i]; }
};
struct GetRel {
    const float2 *V;
    float2 ref;
    __device__ __forceinline__ float operator()(uint32_t i) const { return pair_diff(V[i], ref); }
};

// expectation of g over the rest-demand e of one product:
//   FIFO: e = clamp(d - y1, 0, R); LIFO: e = min(d, R); g(e) = get(base + mult * s'(e))
// w-tables over d: pw point mass, cw cumulative, tw tail; entries at or beyond n
// (the support length) carry no mass and are skipped.
template <typename T, int KAHAN, class Get>
__device__ __forceinline__ void expect_rest(Acc<T, KAHAN> &acc, const Get &get, uint32_t base, uint32_t mult,
                                            Walker wk, int cb, int lifo, uint32_t G, int y1, int R, const T *pw,
                                            const T *cw, const T *tw, int n, T scale) {
    if (!lifo) {
        if (R == 0) {
            acc.add(scale * tw[0], get(base + mult * wk.idx));
            return;
        }
        const int y = y1 < n - 1 ? y1 : n - 1;
        acc.add(scale * cw[y], get(base + mult * wk.idx));
        int e = 1;
        for (; e < R; ++e) {
            if (y1 + e >= n) break;
            walker_step(wk, cb, 0, G);
            acc.add(scale * pw[y1 + e], get(base + mult * wk.idx));
        }
        if (y1 + R < n) {
            for (; e <= R; ++e) walker_step(wk, cb, 0, G);
            acc.add(scale * tw[y1 + R], get(base + mult * wk.idx));
        }
    } else {
        int d = 0;
        for (; d < R && d < n; ++d) {
            acc.add(scale * pw[d], get(base + mult * wk.idx));
            walker_step(wk, cb, 1, G);
        }
        if (R < n) acc.add(scale * tw[R], get(base + mult * wk.idx));
    }
}

// the state decomposition of one product: s_k = x + G r
struct ProdState {
    int x;
    uint32_t r;
    RestInfo ri;
};

template <class Div = PlainDiv>
__device__ __forceinline__ ProdState prod_state(const ProdParams &P, uint32_t sk) {
    ProdState ps;
    if (P.K >= 1) {
        ps.r = Div::q(sk, (uint32_t)P.G, &P);
        ps.x = (int)(sk - ps.r * (uint32_t)P.G);
    } else {
        ps.r = 0;
        ps.x = 0;
    }
    ps.ri = decode_rest<Div>(ps.r, P);
    return ps;
}

// per-action quantities of one product
struct ProdAction {
    Walker wk;
    int y1;   // units in the expiring slot Y_1
    int R;    // units in the other slots
    int T;    // all units available
};

__device__ __forceinline__ ProdAction prod_action(const ProdParams &P, const ProdState &ps, int a, int lifo) {
    ProdAction pa;
    unsigned long long packed;
    int R;
    slots_for_action(P, ps.ri, a, packed, R);
    pa.y1 = (P.K >= 1) ? ps.x : a;    // m = L = 1: the order itself is the only slot
    pa.R = R;
    pa.T = pa.y1 + R;
    const uint32_t idx0 = (P.K >= 1) ? ps.r + (uint32_t)a * P.w_top : 0u;
    walker_init(pa.wk, idx0, packed, P.m - 1, P.cb, lifo, P.w_zt);
    return pa;
}

// ---- single product ----------------------------------------------------------
// plain kinds: Q(s, a) as one number
template <typename T, int KAHAN>
__device__ __forceinline__ T q_single(const KernelParams &kp, const T *s_tab, const T *V, const ProdState &ps,
                                      int a) {
    const ProdParams &P = kp.p[0];
    const int lifo = kp.issuing;
    const ProdAction pa = prod_action(P, ps, a, lifo);
    Acc<T, KAHAN> acc;
    acc.init();
    GetPlain<T> get{V};
    expect_rest<T, KAHAN>(acc, get, 0u, 1u, pa.wk, P.cb, lifo, (uint32_t)P.G, pa.y1, pa.R, s_tab + P.off_p,
                          s_tab + P.off_F, s_tab + P.off_tail, P.dmax + 1, (T)1);
    const T rb = -(T)P.c_o * (T)a + s_tab[P.off_RT + pa.R * P.G + pa.y1];
    return rb + (T)kp.gamma * acc.s;
}

// pair kind: Q(s, a) - gamma R0 as a pair (qh, ql); R0 = V(s'_0 of action 0)
template <int KAHAN>
__device__ __forceinline__ void q_single_pair(const KernelParams &kp, const float *s_tab, const float2 *V,
                                              const ProdState &ps, int a, float2 R0, float &qh, float &ql) {
    const ProdParams &P = kp.p[0];
    const int lifo = kp.issuing;
    const ProdAction pa = prod_action(P, ps, a, lifo);
    const float2 ref = V[pa.wk.idx];
    Acc<float, KAHAN> acc;
    acc.init();
    GetRel get{V, ref};
    expect_rest<float, KAHAN>(acc, get, 0u, 1u, pa.wk, P.cb, lifo, (uint32_t)P.G, pa.y1, pa.R, s_tab + P.off_p,
                              s_tab + P.off_F, s_tab + P.off_tail, P.dmax + 1, 1.f);
    const float gam = (float)kp.gamma;
    action_base(gam, ref, R0, __fmul_rn(-(float)P.c_o, (float)a), qh, ql);
    const int ti = pa.R * P.G + pa.y1;
    pair_add(qh, ql, s_tab[P.off_RT + ti], s_tab[P.off_RTlo + ti]);
    ql = __fmaf_rn(gam, acc.s, ql);
}

// ---- two products (product-1 shortfall may take product 2) ----------------------
// expectation over (d1, z): d1 below product-1 stock with product-2 own demand,
// then the rows of M for d1 at or above the stock (substitution mixture)
template <typename T, int KAHAN, class Get>
__device__ __forceinline__ void expect_two(Acc<T, KAHAN> &acc, const Get &get, const KernelParams &kp,
                                           const T *s_tab, const ProdAction &A1, const ProdAction &A2) {
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    const int lifo = kp.issuing;
    const uint32_t S1 = P1.nS;
    Walker w1 = A1.wk;
    int e1c = 0;
    const int top1 = A1.T < P1.dmax + 1 ? A1.T : P1.dmax + 1;   // d1 in [0, top1)
    for (int d1 = 0; d1 < top1; ++d1) {
        const int e1 = lifo ? min(d1, A1.R) : max(d1 - A1.y1, 0);
        for (; e1c < e1; ++e1c) walker_step(w1, P1.cb, lifo, (uint32_t)P1.G);
        const T p1 = s_tab[P1.off_p + d1];
        expect_rest<T, KAHAN>(acc, get, w1.idx, S1, A2.wk, P2.cb, lifo, (uint32_t)P2.G, A2.y1, A2.R,
                              s_tab + P2.off_p, s_tab + P2.off_F, s_tab + P2.off_tail, P2.dmax + 1, p1);
    }
    if (A1.T <= P1.dmax) {
        for (; e1c < A1.R; ++e1c) walker_step(w1, P1.cb, lifo, (uint32_t)P1.G);
        const int row = A1.T * kp.zlen;
        expect_rest<T, KAHAN>(acc, get, w1.idx, S1, A2.wk, P2.cb, lifo, (uint32_t)P2.G, A2.y1, A2.R,
                              s_tab + kp.off_M + row, s_tab + kp.off_Mc + row, s_tab + kp.off_Mt + row, kp.zlen,
                              (T)1);
    }
}

__device__ __forceinline__ int h1_index(const KernelParams &kp, const ProdAction &A1) {
    const int ys1 = kp.issuing ? A1.R : A1.y1;
    return ys1 * (kp.p[0].tmax + 1) + A1.T;
}
__device__ __forceinline__ int h2_index(const KernelParams &kp, const ProdAction &A1, const ProdAction &A2) {
    const ProdParams &P2 = kp.p[1];
    const int ys2 = kp.issuing ? A2.R : A2.y1;
    const int ny2 = kp.issuing ? (P2.tmax + 1) : P2.G;
    return (A1.T * ny2 + ys2) * (P2.tmax + 1) + A2.T;
}

template <typename T, int KAHAN>
__device__ __forceinline__ T q_two(const KernelParams &kp, const T *s_tab, const T *g_tab, const T *V,
                                   const ProdState &p1s, const ProdState &p2s, int a) {
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    const int a1 = a / P2.G, a2 = a - a1 * P2.G;
    const ProdAction A1 = prod_action(P1, p1s, a1, kp.issuing);
    const ProdAction A2 = prod_action(P2, p2s, a2, kp.issuing);
    Acc<T, KAHAN> acc;
    acc.init();
    GetPlain<T> get{V};
    expect_two<T, KAHAN>(acc, get, kp, s_tab, A1, A2);
    const T rb = -(T)P1.c_o * (T)a1 - (T)P2.c_o * (T)a2 + g_tab[kp.off_H1 + h1_index(kp, A1)] +
                 g_tab[kp.off_H2 + h2_index(kp, A1, A2)];
    return rb + (T)kp.gamma * acc.s;
}

// next state of both products before any demand, for action a
__device__ __forceinline__ uint32_t two_base_state(const KernelParams &kp, const ProdState &p1s,
                                                   const ProdState &p2s, int a) {
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    const int a1 = a / P2.G, a2 = a - a1 * P2.G;
    const uint32_t i1 = (P1.K >= 1) ? p1s.r + (uint32_t)a1 * P1.w_top : 0u;
    const uint32_t i2 = (P2.K >= 1) ? p2s.r + (uint32_t)a2 * P2.w_top : 0u;
    return i1 + P1.nS * i2;
}

template <int KAHAN>
__device__ __forceinline__ void q_two_pair(const KernelParams &kp, const float *s_tab, const float *g_tab,
                                           const float2 *V, const ProdState &p1s, const ProdState &p2s, int a,
                                           float2 R0, float &qh, float &ql) {
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    const int a1 = a / P2.G, a2 = a - a1 * P2.G;
    const ProdAction A1 = prod_action(P1, p1s, a1, kp.issuing);
    const ProdAction A2 = prod_action(P2, p2s, a2, kp.issuing);
    const float2 ref = V[A1.wk.idx + P1.nS * A2.wk.idx];
    Acc<float, KAHAN> acc;
    acc.init();
    GetRel get{V, ref};
    expect_two<float, KAHAN>(acc, get, kp, s_tab, A1, A2);
    const float gam = (float)kp.gamma;
    const float ca = __fadd_rn(__fmul_rn(-(float)P1.c_o, (float)a1), __fmul_rn(-(float)P2.c_o, (float)a2));
    action_base(gam, ref, R0, ca, qh, ql);
    const int i1 = h1_index(kp, A1), i2 = h2_index(kp, A1, A2);
    pair_add(qh, ql, g_tab[kp.off_H1 + i1], g_tab[kp.off_H1lo + i1]);
    pair_add(qh, ql, g_tab[kp.off_H2 + i2], g_tab[kp.off_H2lo + i2]);
    ql = __fmaf_rn(gam, acc.s, ql);
}

// ===========================================================================
// generic sweep: thread = state
// ===========================================================================
template <int VK, int KAHAN>
__global__ void __launch_bounds__(kGenericThreads)
sweep_generic_kernel(KernelParams kp, int mode, const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int) {
    using T = typename std::conditional<VK == VK_DOUBLE, double, float>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SolveState *st = kp.st;
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    const T *g_tab = (const T *)kp.tables;
    const T *s_tab = g_tab;
    if (kp.tab_in_smem) {   // H tables of two products stay in global memory
        T *st_ = (T *)smem_raw;
        load_tables<T>(st_, g_tab, (kp.n_products == 2) ? kp.off_H1 : kp.n_tables);
        s_tab = st_;
    }

    T mx = (T)-INFINITY, mn = (T)INFINITY;
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < kp.nS) {
        int arg = 0;
        ProdState p1s, p2s;
        if (kp.n_products == 1) {
            p1s = prod_state(kp.p[0], s);
        } else {
            const uint32_t S1 = kp.p[0].nS;
            const uint32_t s2 = s / S1;
            p1s = prod_state(kp.p[0], s - s2 * S1);
            p2s = prod_state(kp.p[1], s2);
        }
        if (VK == VK_PAIR) {
            const float2 *V2 = (const float2 *)B.vin;
            const uint32_t i0 =
                (kp.n_products == 1) ? ((kp.p[0].K >= 1) ? p1s.r : 0u) : two_base_state(kp, p1s, p2s, 0);
            const float2 R0 = V2[i0];
            float bh = -INFINITY, bl = 0.f;
            for (int a = 0; a < kp.nA; ++a) {
                float qh, ql;
                if (kp.n_products == 1)
                    q_single_pair<KAHAN>(kp, (const float *)s_tab, V2, p1s, a, R0, qh, ql);
                else
                    q_two_pair<KAHAN>(kp, (const float *)s_tab, (const float *)g_tab, V2, p1s, p2s, a, R0, qh, ql);
                const float diff = __fadd_rn(__fsub_rn(qh, bh), __fsub_rn(ql, bl));
                if (diff > 0.f) {
                    bh = qh;
                    bl = ql;
                    arg = a;
                }
            }
            const float2 vold = V2[s];
            if (mode == MODE_EXTRACT) {
                if (B.vout) ((float2 *)B.vout)[s] = vold;
            } else {
                const float2 vnew = pair_finish((float)kp.gamma, R0, bh, bl);
                ((float2 *)B.vout)[s] = vnew;
                const float dlt = pair_diff(vnew, vold);
                mx = mn = (T)dlt;
            }
        } else {
            const T *V = (const T *)B.vin;
            T best = (T)-INFINITY;
            for (int a = 0; a < kp.nA; ++a) {
                const T q = (kp.n_products == 1) ? q_single<T, KAHAN>(kp, s_tab, V, p1s, a)
                                                 : q_two<T, KAHAN>(kp, s_tab, g_tab, V, p1s, p2s, a);
                if (q > best) {
                    best = q;
                    arg = a;
                }
            }
            if (VK == VK_SINGLE && s == 0 && mode == MODE_SWEEP) st->c_next = (float)best;
            if (mode == MODE_EXTRACT) {
                if (B.vout) ((T *)B.vout)[s] = V[s];
            } else {
                const T vnew = best - (T)B.cnorm;
                const T vold = V[s];
                ((T *)B.vout)[s] = vnew;
                mx = mn = vnew - vold;
            }
        }
        if (B.pol) B.pol[s] = (uint8_t)arg;
    }
    if (mode != MODE_EXTRACT) block_reduce_and_finalize<T>(mx, mn, st, mode, gridDim.x);
}

// ===========================================================================
// next-state dump with the sweep kernels' index arithmetic
// ===========================================================================
__global__ void next_states_kernel(KernelParams kp, const uint32_t *states, int n, uint32_t *out) {
    const int i = blockIdx.x;
    const int a = threadIdx.x + blockIdx.y * blockDim.x;
    if (i >= n || a >= kp.nA) return;
    const uint32_t s = states[i];
    const int lifo = kp.issuing;
    if (kp.n_products == 1) {
        const ProdParams &P = kp.p[0];
        const ProdState ps = prod_state(P, s);
        const ProdAction pa = prod_action(P, ps, a, lifo);
        uint32_t *o = out + ((size_t)i * kp.nA + a) * (size_t)(P.dmax + 1);
        Walker wk = pa.wk;
        int e_cur = 0;
        for (int d = 0; d <= P.dmax; ++d) {
            const int e = lifo ? min(d, pa.R) : min(max(d - pa.y1, 0), pa.R);
            for (; e_cur < e; ++e_cur) walker_step(wk, P.cb, lifo, (uint32_t)P.G);
            o[d] = wk.idx;
        }
        return;
    }
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    const uint32_t S1 = P1.nS;
    const uint32_t s2 = s / S1;
    const ProdState p1s = prod_state(P1, s - s2 * S1);
    const ProdState p2s = prod_state(P2, s2);
    const int a1 = a / P2.G, a2 = a - a1 * P2.G;
    const ProdAction A1 = prod_action(P1, p1s, a1, lifo);
    const ProdAction A2 = prod_action(P2, p2s, a2, lifo);
    const int zl = P1.dmax + P2.dmax + 1;
    uint32_t *o = out + ((size_t)i * kp.nA + a) * (size_t)(P1.dmax + 1) * (size_t)zl;
    Walker w1 = A1.wk;
    int e1c = 0;
    for (int d1 = 0; d1 <= P1.dmax; ++d1) {
        const int e1 = lifo ? min(d1, A1.R) : min(max(d1 - A1.y1, 0), A1.R);
        for (; e1c < e1; ++e1c) walker_step(w1, P1.cb, lifo, (uint32_t)P1.G);
        Walker w2 = A2.wk;
        int e2c = 0;
        for (int z = 0; z < zl; ++z) {
            const int e2 = lifo ? min(z, A2.R) : min(max(z - A2.y1, 0), A2.R);
            for (; e2c < e2; ++e2c) walker_step(w2, P2.cb, lifo, (uint32_t)P2.G);
            o[(size_t)d1 * zl + z] = w1.idx + S1 * w2.idx;
        }
    }
}

// ===========================================================================
// FP64 fixed-policy sweep: V_new(s) = Q(s, pi(s)) with double tables
// ===========================================================================
__global__ void __launch_bounds__(kGenericThreads)
policy_eval_kernel(KernelParams kp, const uint8_t *policy, const double *vin, double *vout) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const double *g_tab = (const double *)kp.tables;
    const double *s_tab = g_tab;
    if (kp.tab_in_smem) {
        double *st_ = (double *)smem_raw;
        load_tables<double>(st_, g_tab, (kp.n_products == 2) ? kp.off_H1 : kp.n_tables);
        s_tab = st_;
    }
    double mx = -INFINITY, mn = INFINITY;
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < kp.nS) {
        const int a = policy[s];
        double q;
        if (kp.n_products == 1) {
            const ProdState ps = prod_state(kp.p[0], s);
            q = q_single<double, 0>(kp, s_tab, vin, ps, a);
        } else {
            const uint32_t S1 = kp.p[0].nS;
            const uint32_t s2 = s / S1;
            const ProdState p1s = prod_state(kp.p[0], s - s2 * S1);
            const ProdState p2s = prod_state(kp.p[1], s2);
            q = q_two<double, 0>(kp, s_tab, g_tab, vin, p1s, p2s, a);
        }
        vout[s] = q;
        mx = mn = q - vin[s];
    }
    block_reduce_and_finalize<double>(mx, mn, kp.st, MODE_PLAIN, gridDim.x);
}

// V_abs in FP64 from any value kind
__global__ void to_fp64_kernel(const void *v, int vk, double offset, double *out, uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (vk == VK_SINGLE) {
        out[i] = offset + (double)((const float *)v)[i];
    } else if (vk == VK_PAIR) {
        const float2 p = ((const float2 *)v)[i];
        out[i] = (double)p.x + (double)p.y;
    } else {
        out[i] = ((const double *)v)[i];
    }
}

// max_s |a(s) - b(s)| into the state's plain accumulators
// max and min of a - b over the n entries, into st->dmax_abs / st->dmin_abs
__global__ void diff_range_kernel(const double *a, const double *b, uint32_t n, SolveState *st) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    double mx = -INFINITY, mn = INFINITY;
    if (i < n) mx = mn = a[i] - b[i];
    block_reduce_and_finalize<double>(mx, mn, st, MODE_PLAIN, gridDim.x);
}

// ===========================================================================
// solve bookkeeping
// ===========================================================================
__global__ void solve_init_kernel(SolveState *st, uint32_t n) {
    // zero V_0 unless warm-starting, reset the running state
    const int warm = st->warm;
    const int value_bytes = st->value_bytes;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (!warm && i < n) {
        if (value_bytes == 4)
            ((float *)st->buf[0])[i] = 0.f;
        else
            ((double *)st->buf[0])[i] = 0.0;   // also a (0, 0) float pair
    }
    if (i == 0) {
        st->key_max = 0ull;
        st->key_min = ~0ull;
        st->blocks_done = 0u;
        st->fault = 0;
        st->iter = 0;
        st->converged = 0;
        st->crit = INFINITY;
        st->dmax_abs = 0.0;
        st->dmin_abs = 0.0;
        st->c_cur = 0.f;
        st->c_next = 0.f;
        if (!warm) st->offset = 0.0;
        const int go = st->max_iters > 0;
        st->keep_going = go;
        if (st->use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)st->cond, go ? 1u : 0u);
    }
}

// ===========================================================================
// rollouts: one period of one product, the KPI sums, the cost table
// ===========================================================================
struct RollOut {
    uint32_t s_next;
    int issued, wasted, carried, shortage, arrived, total;
};

// one product, one period, with the sweep kernels' walker for the next state
// (Div: how indices are divided by G, see DivG)
template <class Div = PlainDiv>
__device__ __forceinline__ RollOut roll_product(const ProdParams &P, int lifo, uint32_t sk, int a, int z) {
    const ProdState ps = prod_state<Div>(P, sk);
    const ProdAction pa = prod_action(P, ps, a, lifo);
    RollOut o;
    const int e = lifo ? min(z, pa.R) : min(max(z - pa.y1, 0), pa.R);
    Walker wk = pa.wk;
    for (int k = 0; k < e; ++k) walker_step<Div>(wk, P.cb, lifo, (uint32_t)P.G, &P);
    o.s_next = wk.idx;
    o.total = pa.T;
    o.issued = min(z, pa.T);
    // the expiring slot is issued first (FIFO) or last (LIFO)
    o.wasted = lifo ? (pa.y1 - min(pa.y1, max(z - pa.R, 0))) : max(pa.y1 - z, 0);
    o.carried = pa.T - o.issued - o.wasted;
    o.shortage = max(z - pa.T, 0);
    // the arrival: P_1 when L >= 2 (digit m-1 of the state), else the order
    if (P.L >= 2) {
        if (P.m == 1) {
            o.arrived = ps.x;
        } else {
            uint32_t q = ps.r;
            for (int j = 0; j < P.m - 2; ++j) q = Div::q(q, (uint32_t)P.G, &P);
            o.arrived = (int)(q % (uint32_t)P.G);
        }
    } else {
        o.arrived = a;
    }
    return o;
}

// accepted substitutions among n short units: popcount of the low n bits of the
// 64-bit word (w3, w2); a shortfall above 64 uses all 64 bits
__device__ __forceinline__ int substitutes(uint32_t w2, uint32_t w3, int n) {
    const int lo = min(n, 32);
    const int hi = min(max(n - 32, 0), 32);
    const uint32_t mlo = (lo >= 32) ? 0xffffffffu : ((1u << lo) - 1u);
    const uint32_t mhi = (hi >= 32) ? 0xffffffffu : ((1u << hi) - 1u);
    return __popc(w2 & mlo) + __popc(w3 & mhi);
}

// smallest d with w < thr[d], thr[d] = floor(2^32 CDF(d)) (thr[dmax] = 2^32)
__device__ __forceinline__ int draw_demand(uint32_t w, const unsigned long long *thr, int dmax) {
    int d = 0;
    while (d < dmax && (unsigned long long)w >= thr[d]) ++d;
    return d;
}

// The cost terms c n of a period's reward, n a unit count: the products
// __dmul_rn(c, n) for n < kCostTab read from a table in shared memory (the same
// doubles, without an FP64 multiply and conversion per term), computed above it
constexpr int kCostTab = 256;
struct CostTab {
    const double *t;          // [product][cost][n], in shared memory
    const RollParams *rp;
    int len;                  // kCostTab, or 0: always multiply
    __device__ __forceinline__ double operator()(int j, int k, int n) const {
        return (unsigned)n < (unsigned)len ? t[(j * 5 + k) * kCostTab + n] : __dmul_rn(rp->cost[j][k], (double)n);
    }
};

__device__ __forceinline__ void fill_cost_tab(double *t, const RollParams &rp, int n_products) {
    for (int i = threadIdx.x; i < n_products * 5 * kCostTab; i += blockDim.x) {
        const int jk = i / kCostTab;
        t[i] = __dmul_rn(rp.cost[jk / 5][jk % 5], (double)(i - jk * kCostTab));
    }
}

// one period of a single product: reward (FP64, unfused, in the oracle's order) and outcome
template <class Div = PlainDiv>
__device__ __forceinline__ double single_period(const ProdParams &P1, int lifo, const CostTab &ct, uint32_t s, int a,
                                                int d1, RollOut &o) {
    o = roll_product<Div>(P1, lifo, s, a, d1);
    double rew = 0.0;
    rew = __dsub_rn(rew, ct(0, 0, a));
    rew = __dsub_rn(rew, ct(0, 1, o.carried));
    rew = __dsub_rn(rew, ct(0, 2, o.shortage));
    rew = __dsub_rn(rew, ct(0, 3, o.wasted));
    rew = __dadd_rn(rew, ct(0, 4, o.issued));
    return rew;
}

// per-product KPI sums of one rollout; unit counts summed as integers: exactly the FP64 running sums of the same counts
// (every partial sum is an integer below 2^53), without an FP64 add per period
struct KpiSums {
    long long dem[2], served[2], was[2], arr[2], car[2];
    __device__ __forceinline__ void init() {
        for (int j = 0; j < 2; ++j) dem[j] = served[j] = was[j] = arr[j] = car[j] = 0;
    }
    // service % (product 1 counts its shortfall met by substitution as served),
    // wastage % of the units received, mean units carried
    __device__ __forceinline__ void finish(int horizon, double *out6) const {
        for (int j = 0; j < 2; ++j) {
            const double d = (double)dem[j], sv = (double)served[j], w = (double)was[j], a = (double)arr[j];
            out6[3 * j + 0] = d > 0.0 ? __ddiv_rn(__dmul_rn(100.0, sv), d) : 100.0;
            out6[3 * j + 1] = a > 0.0 ? __ddiv_rn(__dmul_rn(100.0, w), a) : 0.0;
            out6[3 * j + 2] = horizon > 0 ? __ddiv_rn((double)car[j], (double)horizon) : 0.0;
        }
    }
};

// ---------------------------------------------------------------------------
// Rollouts: a group of LPR = 32 / RPW lanes per rollout, RPW rollouts per warp.  The
// state is all that one period hands to the next, so a group takes LPR periods at a
// time in three steps:
//   A. lane j of the group draws the random words and the demands of period t0 + j
//      (Philox counters (t, r): they do not depend on the state);
//   B. the group walks the state chain s_t -> a_t = pi(s_t) -> s_{t+1} through the LPR
//      periods, its lanes in step, each lane keeping (s_t, a_t) of its own period;
//   C. lane j evaluates its period: outcome, reward and counts.
// The return is folded in period order with the FP64 operations of a serial loop and
// the KPI counts are integer sums, so the results are those of one thread walking
// the whole rollout, bit for bit.  Only step B is serial, and its indices are
// divided by G with DivG's multiply-high.  The fold is the same in every lane of a
// group, so RPW rollouts share each FP64 instruction of it.
// ---------------------------------------------------------------------------
constexpr int kRollWarps = 4;   // warps per block
// rollouts per warp: measured on B300 (config 4, 4096 x 365): 1 0.51 ms, 2 0.41, 4 0.41, 8 0.45
constexpr int kRollRPW = 4;
constexpr int kRollLPR = 32 / kRollRPW;    // lanes (and periods per step) per rollout
using RollDiv = DivG;

// two products, one period: both outcomes, the substitution u from the words (w2, w3)
struct TwoOut {
    RollOut o1, o2;
    int own2, short1, short2;
    uint32_t s_next;
};
template <class Div>
__device__ __forceinline__ TwoOut two_period(const KernelParams &kp, int lifo, uint32_t s, int a, int d1, int d2,
                                             uint32_t w2, uint32_t w3) {
    const ProdParams &P1 = kp.p[0], &P2 = kp.p[1];
    const uint32_t S1 = P1.nS;
    const uint32_t s2 = s / S1, s1 = s - s2 * S1;
    const int a1 = a / P2.G, a2 = a - a1 * P2.G;
    TwoOut t;
    t.o1 = roll_product<Div>(P1, lifo, s1, a1, d1);
    const int u = substitutes(w2, w3, t.o1.shortage);
    t.o2 = roll_product<Div>(P2, lifo, s2, a2, d2 + u);
    t.own2 = min(d2, t.o2.total);
    t.short1 = t.o1.shortage - (t.o2.issued - t.own2);
    t.short2 = max(d2 - t.o2.total, 0);
    t.s_next = t.o1.s_next + S1 * t.o2.s_next;
    return t;
}

__global__ void __launch_bounds__(32 * kRollWarps)
rollout_kernel(KernelParams kp, RollParams rp, const uint8_t *policy, double *returns, double *kpis,
               double *kpis_prod, int32_t *traj) {
    __shared__ unsigned long long s_thr[2][kMaxRollDmax + 1];
    __shared__ double s_ct[2 * 5 * kCostTab];
    for (int i = threadIdx.x; i <= kMaxRollDmax; i += blockDim.x) {
        s_thr[0][i] = rp.thr[0][i];
        s_thr[1][i] = rp.thr[1][i];
    }
    fill_cost_tab(s_ct, rp, kp.n_products);
    __syncthreads();
    const CostTab ct{s_ct, &rp, kCostTab};
    constexpr int LPR = kRollLPR;
    const int lane = threadIdx.x & 31;
    const int sl = lane % LPR;   // lane within the rollout's group
    const int r = (blockIdx.x * kRollWarps + (int)(threadIdx.x >> 5)) * kRollRPW + lane / LPR;
    // a group past the last rollout runs along (its lanes take part in the shuffles) but
    // writes nothing; a warp with no rollout leaves at once
    if ((blockIdx.x * kRollWarps + (int)(threadIdx.x >> 5)) * kRollRPW >= rp.n_rollouts) return;
    const bool real = r < rp.n_rollouts;
    const int lifo = kp.issuing;
    const bool two = kp.n_products == 2;
    const uint32_t k0 = (uint32_t)(rp.seed & 0xffffffffull), k1 = (uint32_t)(rp.seed >> 32);
    const int T = rp.warmup + rp.horizon;
    const ProdParams &P1 = kp.p[0];
    uint32_t s = 0;
    double ret = 0.0, disc = 1.0;
    long long dem = 0, iss = 0, was = 0, arr = 0, car = 0;
    KpiSums ks;
    ks.init();
    for (int t0 = 0; t0 < T; t0 += LPR) {
        const int t = t0 + sl;
        const int nj = min(LPR, T - t0);   // the same for the whole warp
        // A. this lane's period: random words and demands
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        int d1 = 0, d2 = 0;
        if (t < T) {
            philox4x32_10((uint32_t)t, (uint32_t)r, 0u, 0u, k0, k1, w);
            d1 = draw_demand(w[0], s_thr[0], P1.dmax);
            if (two) d2 = draw_demand(w[1], s_thr[1], kp.p[1].dmax);
        }
        // B. the state chain of the group's periods
        uint32_t my_s = 0u;
        int my_a = 0;
        for (int j = 0; j < nj; ++j) {
            const int a = __ldg(policy + s);
            const int dj = __shfl_sync(0xffffffffu, d1, j, LPR);
            if (sl == j) {
                my_s = s;
                my_a = a;
            }
            if (!two) {
                s = roll_product<RollDiv>(P1, lifo, s, a, dj).s_next;
            } else {
                const int dj2 = __shfl_sync(0xffffffffu, d2, j, LPR);
                const uint32_t wj2 = __shfl_sync(0xffffffffu, w[2], j, LPR);
                const uint32_t wj3 = __shfl_sync(0xffffffffu, w[3], j, LPR);
                s = two_period<RollDiv>(kp, lifo, s, a, dj, dj2, wj2, wj3).s_next;
            }
        }
        // C. this lane's period: outcome, reward (FP64, unfused, in the oracle's order), counts
        double rew = 0.0;
        if (t < T) {
            int t_dem, t_iss, t_was, t_arr, t_car;
            int p_dem[2] = {0, 0}, p_srv[2] = {0, 0}, p_was[2] = {0, 0}, p_arr[2] = {0, 0}, p_car[2] = {0, 0};
            if (!two) {
                RollOut o;
                rew = single_period<RollDiv>(P1, lifo, ct, my_s, my_a, d1, o);
                t_dem = d1;
                t_iss = o.issued;
                t_was = o.wasted;
                t_arr = o.arrived;
                t_car = o.carried;
                p_dem[0] = d1;
                p_srv[0] = o.issued;
                p_was[0] = o.wasted;
                p_arr[0] = o.arrived;
                p_car[0] = o.carried;
            } else {
                const TwoOut q = two_period<RollDiv>(kp, lifo, my_s, my_a, d1, d2, w[2], w[3]);
                const int a1 = my_a / kp.p[1].G, a2 = my_a - a1 * kp.p[1].G;
                rew = __dsub_rn(rew, ct(0, 0, a1));
                rew = __dsub_rn(rew, ct(0, 1, q.o1.carried));
                rew = __dsub_rn(rew, ct(0, 2, q.short1));
                rew = __dsub_rn(rew, ct(0, 3, q.o1.wasted));
                rew = __dadd_rn(rew, ct(0, 4, q.o1.issued));
                rew = __dsub_rn(rew, ct(1, 0, a2));
                rew = __dsub_rn(rew, ct(1, 1, q.o2.carried));
                rew = __dsub_rn(rew, ct(1, 2, q.short2));
                rew = __dsub_rn(rew, ct(1, 3, q.o2.wasted));
                rew = __dadd_rn(rew, ct(1, 4, q.o2.issued));
                t_dem = d1 + d2;
                t_iss = q.o1.issued + q.o2.issued;
                t_was = q.o1.wasted + q.o2.wasted;
                t_arr = q.o1.arrived + q.o2.arrived;
                t_car = q.o1.carried + q.o2.carried;
                const int sub = q.o2.issued - q.own2;
                p_dem[0] = d1;
                p_dem[1] = d2;
                p_srv[0] = q.o1.issued + sub;
                p_srv[1] = q.own2;
                p_was[0] = q.o1.wasted;
                p_was[1] = q.o2.wasted;
                p_arr[0] = q.o1.arrived;
                p_arr[1] = q.o2.arrived;
                p_car[0] = q.o1.carried;
                p_car[1] = q.o2.carried;
            }
            if (t >= rp.warmup && real) {
                if (traj) traj[(size_t)r * rp.horizon + (t - rp.warmup)] = (int32_t)my_s;
                dem += t_dem;
                iss += t_iss;
                was += t_was;
                arr += t_arr;
                car += t_car;
                for (int j = 0; j < 2; ++j) {
                    ks.dem[j] += p_dem[j];
                    ks.served[j] += p_srv[j];
                    ks.was[j] += p_was[j];
                    ks.arr[j] += p_arr[j];
                    ks.car[j] += p_car[j];
                }
            }
        }
        // the discounted return, period by period
        for (int j = 0; j < nj; ++j) {
            const double rj = __shfl_sync(0xffffffffu, rew, j, LPR);
            if (t0 + j >= rp.warmup) {
                ret = __dadd_rn(ret, __dmul_rn(disc, rj));
                disc = __dmul_rn(disc, kp.gamma);
            }
        }
    }
    // the group's sums of the counts (integers: any order gives the same sums)
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) {
        dem += __shfl_xor_sync(0xffffffffu, dem, o);
        iss += __shfl_xor_sync(0xffffffffu, iss, o);
        was += __shfl_xor_sync(0xffffffffu, was, o);
        arr += __shfl_xor_sync(0xffffffffu, arr, o);
        car += __shfl_xor_sync(0xffffffffu, car, o);
        for (int j = 0; j < 2; ++j) {
            ks.dem[j] += __shfl_xor_sync(0xffffffffu, ks.dem[j], o);
            ks.served[j] += __shfl_xor_sync(0xffffffffu, ks.served[j], o);
            ks.was[j] += __shfl_xor_sync(0xffffffffu, ks.was[j], o);
            ks.arr[j] += __shfl_xor_sync(0xffffffffu, ks.arr[j], o);
            ks.car[j] += __shfl_xor_sync(0xffffffffu, ks.car[j], o);
        }
    }
    if (sl != 0 || !real) return;
    returns[r] = ret;
    if (kpis) {
        const double fd = (double)dem, fi = (double)iss, fw = (double)was, fa = (double)arr;
        kpis[3 * r + 0] = fd > 0.0 ? __ddiv_rn(__dmul_rn(100.0, fi), fd) : 100.0;
        kpis[3 * r + 1] = fa > 0.0 ? __ddiv_rn(__dmul_rn(100.0, fw), fa) : 0.0;
        kpis[3 * r + 2] = rp.horizon > 0 ? __ddiv_rn((double)car, (double)rp.horizon) : 0.0;
    }
    if (kpis_prod) ks.finish(rp.horizon, kpis_prod + 6 * (size_t)r);
}

// ===========================================================================
// base-stock policy search (Methods, Scenario A heuristic): thread = (S, rollout);
// A = min([S - I]^+, Q) with I the units on hand and in transit (the sum of the
// state's digits).  Every S sees the same demands (Philox counters (t, r)).
// ===========================================================================
__global__ void basestock_kernel(KernelParams kp, RollParams rp, int s_lo, int n_S, double *returns) {
    __shared__ unsigned long long s_thr[kMaxRollDmax + 1];
    for (int i = threadIdx.x; i <= kMaxRollDmax; i += blockDim.x) s_thr[i] = rp.thr[0][i];
    __syncthreads();
    // thousands of threads per SM: FP64 multiplies are not the bound here and the
    // table measured slower (1.4%), so the costs are multiplied
    const CostTab ct{nullptr, &rp, 0};
    const long long t_id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t_id >= (long long)n_S * rp.n_rollouts) return;
    const int S = s_lo + (int)(t_id / rp.n_rollouts);
    const int r = (int)(t_id % rp.n_rollouts);
    const ProdParams &P1 = kp.p[0];
    const int lifo = kp.issuing;
    const uint32_t k0 = (uint32_t)(rp.seed & 0xffffffffull), k1 = (uint32_t)(rp.seed >> 32);
    uint32_t s = 0;
    double ret = 0.0, disc = 1.0;
    for (int t = 0; t < rp.warmup + rp.horizon; ++t) {
        uint32_t w[4];
        philox4x32_10((uint32_t)t, (uint32_t)r, 0u, 0u, k0, k1, w);
        int stock = 0;
        uint32_t rem = s;
        for (int k = 0; k < P1.K; ++k) {
            const uint32_t q = DivG::q(rem, (uint32_t)P1.G, &P1);
            stock += (int)(rem - q * (uint32_t)P1.G);
            rem = q;
        }
        const int a = min(max(S - stock, 0), P1.Q);
        const int d1 = draw_demand(w[0], s_thr, P1.dmax);
        RollOut o;
        const double rew = single_period<DivG>(P1, lifo, ct, s, a, d1, o);
        if (t >= rp.warmup) {
            ret = __dadd_rn(ret, __dmul_rn(disc, rew));
            disc = __dmul_rn(disc, kp.gamma);
        }
        s = o.s_next;
    }
    returns[t_id] = ret;
}

cudaError_t launch_basestock(const KernelParams &kp, const RollParams &rp, int s_lo, int n_S, double *returns,
                             cudaStream_t stream) {
    const long long n = (long long)n_S * rp.n_rollouts;
    const int threads = 128;
    basestock_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, stream>>>(kp, rp, s_lo, n_S, returns);
    return cudaGetLastError();
}

// ===========================================================================
// modified base-stock search (Scenario B heuristic): thread = ((S_1, S_2), rollout).
// Product k orders [S_k - I_k + [X_{1,k} - mu_k]^+]^+ from its own stock (I_k:
// units on hand, X_1..X_{m-1} and the arrival P_1 when L >= 2), optionally
// capped at Q_k.  The stock is kept as plain slot counts, not as a state index,
// so an uncapped order may exceed Q_k.  Same random numbers as the rollouts.
// ===========================================================================
struct StockVec {
    int X[kMbsMaxM];       // X_1..X_{m-1}
    int P[kMbsMaxL];       // P_1..P_{L-1}
};

struct VecOut {
    int issued, wasted, carried, shortage, arrived, total;
};

__device__ __forceinline__ void vec_period(const ProdParams &P, int lifo, StockVec &v, int order, int z, VecOut &o) {
    int Y[kMbsMaxM];
#pragma unroll
    for (int j = 0; j < kMbsMaxM; ++j) Y[j] = (j < P.m - 1) ? v.X[j] : 0;
    const int arrival = (P.L >= 2) ? v.P[0] : order;
#pragma unroll
    for (int j = 0; j < kMbsMaxM; ++j)
        if (j == P.m - 1) Y[j] = arrival;
    int T = 0;
#pragma unroll
    for (int j = 0; j < kMbsMaxM; ++j) T += (j < P.m) ? Y[j] : 0;
    int left = z;
    if (!lifo) {
#pragma unroll
        for (int j = 0; j < kMbsMaxM; ++j) {
            if (j < P.m) {
                const int take = min(Y[j], left);
                Y[j] -= take;
                left -= take;
            }
        }
    } else {
#pragma unroll
        for (int j = kMbsMaxM - 1; j >= 0; --j) {
            if (j < P.m) {
                const int take = min(Y[j], left);
                Y[j] -= take;
                left -= take;
            }
        }
    }
    o.total = T;
    o.issued = min(z, T);
    o.wasted = Y[0];
    o.shortage = max(z - T, 0);
    o.arrived = arrival;
    int car = 0;
#pragma unroll
    for (int j = 0; j < kMbsMaxM - 1; ++j) {
        const int nx = (j < P.m - 1) ? Y[j + 1] : 0;
        v.X[j] = nx;
        car += nx;
    }
    o.carried = car;
#pragma unroll
    for (int j = 0; j < kMbsMaxL - 1; ++j)
        if (j < P.L - 2) v.P[j] = v.P[j + 1];
#pragma unroll
    for (int j = 0; j < kMbsMaxL; ++j)
        if (j == P.L - 2) v.P[j] = order;
}

__device__ __forceinline__ int mbs_order(const ProdParams &P, const StockVec &v, int S, int mu, int cap) {
    int onhand = 0;
#pragma unroll
    for (int j = 0; j < kMbsMaxM; ++j) onhand += (j < P.m - 1) ? v.X[j] : 0;
    if (P.L >= 2) onhand += v.P[0];
    const int expiring = (P.m >= 2) ? v.X[0] : ((P.L >= 2) ? v.P[0] : 0);
    int q = max(S - onhand + max(expiring - mu, 0), 0);
    if (cap) q = min(q, P.Q);
    return q;
}

__global__ void mbs_kernel(KernelParams kp, RollParams rp, MbsParams mp, double *returns, double *kpis_prod) {
    __shared__ unsigned long long s_thr[2][kMaxRollDmax + 1];
    __shared__ double s_ct[2 * 5 * kCostTab];
    for (int i = threadIdx.x; i <= kMaxRollDmax; i += blockDim.x) {
        s_thr[0][i] = rp.thr[0][i];
        s_thr[1][i] = rp.thr[1][i];
    }
    fill_cost_tab(s_ct, rp, 2);
    __syncthreads();
    const CostTab ct{s_ct, &rp, kCostTab};
    const long long t_id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t_id >= (long long)mp.n_pairs * rp.n_rollouts) return;
    const int pair = (int)(t_id / rp.n_rollouts);
    const int r = (int)(t_id % rp.n_rollouts);
    const int S1 = mp.s_lo[0] + pair / mp.n2, S2 = mp.s_lo[1] + pair % mp.n2;
    const int np = kp.n_products;
    const int lifo = kp.issuing;
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    const uint32_t k0 = (uint32_t)(rp.seed & 0xffffffffull), k1 = (uint32_t)(rp.seed >> 32);
    StockVec v1, v2;
#pragma unroll
    for (int j = 0; j < kMbsMaxM; ++j) v1.X[j] = v2.X[j] = 0;
#pragma unroll
    for (int j = 0; j < kMbsMaxL; ++j) v1.P[j] = v2.P[j] = 0;
    double ret = 0.0, disc = 1.0;
    KpiSums ks;
    ks.init();
    for (int t = 0; t < rp.warmup + rp.horizon; ++t) {
        uint32_t w[4];
        philox4x32_10((uint32_t)t, (uint32_t)r, 0u, 0u, k0, k1, w);
        const int q1 = mbs_order(P1, v1, S1, mp.mu[0], mp.cap);
        const int q2 = (np == 2) ? mbs_order(P2, v2, S2, mp.mu[1], mp.cap) : 0;
        const int d1 = draw_demand(w[0], s_thr[0], P1.dmax);
        const int d2 = (np == 2) ? draw_demand(w[1], s_thr[1], P2.dmax) : 0;
        VecOut o1, o2;
        vec_period(P1, lifo, v1, q1, d1, o1);
        int sub = 0, short1 = o1.shortage, short2 = 0;
        if (np == 2) {
            const int u = substitutes(w[2], w[3], o1.shortage);
            vec_period(P2, lifo, v2, q2, d2 + u, o2);
            const int own2 = min(d2, o2.total);
            sub = o2.issued - own2;
            short1 = o1.shortage - sub;
            short2 = max(d2 - o2.total, 0);
        }
        double rew = 0.0;
        rew = __dsub_rn(rew, ct(0, 0, q1));
        rew = __dsub_rn(rew, ct(0, 1, o1.carried));
        rew = __dsub_rn(rew, ct(0, 2, short1));
        rew = __dsub_rn(rew, ct(0, 3, o1.wasted));
        rew = __dadd_rn(rew, ct(0, 4, o1.issued));
        if (np == 2) {
            rew = __dsub_rn(rew, ct(1, 0, q2));
            rew = __dsub_rn(rew, ct(1, 1, o2.carried));
            rew = __dsub_rn(rew, ct(1, 2, short2));
            rew = __dsub_rn(rew, ct(1, 3, o2.wasted));
            rew = __dadd_rn(rew, ct(1, 4, o2.issued));
        }
        if (t >= rp.warmup) {
            ret = __dadd_rn(ret, __dmul_rn(disc, rew));
            disc = __dmul_rn(disc, kp.gamma);
            ks.dem[0] += d1;
            ks.served[0] += o1.issued + sub;
            ks.was[0] += o1.wasted;
            ks.arr[0] += o1.arrived;
            ks.car[0] += o1.carried;
            if (np == 2) {
                ks.dem[1] += d2;
                ks.served[1] += o2.issued - sub;
                ks.was[1] += o2.wasted;
                ks.arr[1] += o2.arrived;
                ks.car[1] += o2.carried;
            }
        }
    }
    returns[t_id] = ret;
    if (kpis_prod) ks.finish(rp.horizon, kpis_prod + 6 * t_id);
}

cudaError_t launch_mbs(const KernelParams &kp, const RollParams &rp, const MbsParams &mp, double *returns,
                       double *kpis_prod, cudaStream_t stream) {
    const long long n = (long long)mp.n_pairs * rp.n_rollouts;
    const int threads = 128;
    mbs_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, stream>>>(kp, rp, mp, returns, kpis_prod);
    return cudaGetLastError();
}

// ===========================================================================
// launch descriptors and launchers
// ===========================================================================
bool group_width_supported(int xw) {
    switch (xw) {
        case 1: case 2: case 3: case 4: case 5: case 6: case 7: case 8: case 9: case 10: case 11: case 12:
        case 16: case 21: case 24: return true;
        default: return false;
    }
}

template <int VK, int KAHAN>
static cudaError_t describe_generic_t(const KernelParams &kp, LaunchDesc &d) {
    using T = typename std::conditional<VK == VK_DOUBLE, double, float>::type;
    d.fn = (const void *)sweep_generic_kernel<VK, KAHAN>;
    d.grid = dim3((kp.nS + kGenericThreads - 1) / kGenericThreads);
    d.block = dim3(kGenericThreads);
    const int n_smem_tab = (kp.n_products == 2) ? kp.off_H1 : kp.n_tables;
    d.smem = kp.tab_in_smem ? (size_t)n_smem_tab * sizeof(T) : 0;
    return cudaFuncSetAttribute(sweep_generic_kernel<VK, KAHAN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)d.smem);
}

bool group_supported(const KernelParams &kp, int vk, int kahan) {
    const ProdParams &P = kp.p[0];
    return kp.n_products == 1 && (vk == VK_PAIR || vk == VK_SINGLE) && !kahan && P.K >= 1 && P.G >= 2 &&
           P.G <= kMaxGroupG;
}

// lane widths worth trying for an instance: G itself and G split over 2..4 lanes,
// rounded up to an instantiated width, plus a few small widths
int group_width_candidates(int G, int *out, int max_out) {
    const int base[] = {G, (G + 1) / 2, (G + 2) / 3, (G + 3) / 4, 8, 6, 4};
    int n = 0;
    for (int w : base) {
        while (w <= 24 && !group_width_supported(w)) ++w;
        if (w > 24 || w < 1 || w > G) continue;
        if ((G + w - 1) / w > kGroupThreads) continue;
        bool seen = false;
        for (int i = 0; i < n; ++i) seen |= (out[i] == w);
        if (!seen && n < max_out) out[n++] = w;
    }
    return n;
}

// ===========================================================================
// factorised two-product sweep.  Product 1's next state depends on (s1, a1, d1)
// only and product 2's on (s2, a2, z), z = d2 (d1 below product-1 stock) or the
// substitution mixture of d1 >= T1, which leaves product 1 empty (index 0 with
// L = 1).  So, with ref the no-demand next state of (s, a) and i2_0 that of
// product 2,
//   E[V(s') - ref] = sum_{d1 < T1} p1(d1) [E2(i1(d1), s2, a2) + V(i1(d1), i2_0) - ref]
//                  + Mix(s2, a2, T1) + tail1(T1) [V(0, i2_0) - ref],
// with E2 and Mix product-2 expectations measured from V(i1, i2_0), built once
// per sweep by two small kernels ahead of the sweep.
// ===========================================================================
template <int KAHAN>
__global__ void __launch_bounds__(kGenericThreads)
two_e2_kernel(KernelParams kp, int mode, const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int) {
    SolveState *st = kp.st;
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    const uint32_t S1 = P1.nS;
    const uint64_t n = (uint64_t)S1 * P2.nS * (uint32_t)P2.G;
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint32_t i1 = (uint32_t)(t % S1);
    const uint32_t rest = (uint32_t)(t / S1);
    const int a2 = (int)(rest % (uint32_t)P2.G);
    const uint32_t s2 = rest / (uint32_t)P2.G;
    const float *tab = (const float *)kp.tables;
    const ProdState p2s = prod_state(P2, s2);
    const ProdAction A2 = prod_action(P2, p2s, a2, kp.issuing);
    const float2 *V2 = (const float2 *)B.vin;
    Acc<float, KAHAN> acc;
    acc.init();
    GetRel get{V2, V2[i1 + S1 * A2.wk.idx]};
    expect_rest<float, KAHAN>(acc, get, i1, S1, A2.wk, P2.cb, kp.issuing, (uint32_t)P2.G, A2.y1, A2.R,
                              tab + P2.off_p, tab + P2.off_F, tab + P2.off_tail, P2.dmax + 1, 1.f);
    kp.two_e2[t] = acc.s;
}

template <int KAHAN>
__global__ void __launch_bounds__(kGenericThreads)
two_mix_kernel(KernelParams kp, int mode, const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int) {
    SolveState *st = kp.st;
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    const uint32_t S1 = P1.nS;
    const uint32_t nt = (uint32_t)kp.two_nt1;
    const uint32_t n = P2.nS * (uint32_t)P2.G * nt;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int T1 = (int)(t % nt);
    const uint32_t rest = t / nt;
    const int a2 = (int)(rest % (uint32_t)P2.G);
    const uint32_t s2 = rest / (uint32_t)P2.G;
    const float *tab = (const float *)kp.tables;
    const ProdState p2s = prod_state(P2, s2);
    const ProdAction A2 = prod_action(P2, p2s, a2, kp.issuing);
    const float2 *V2 = (const float2 *)B.vin;
    Acc<float, KAHAN> acc;
    acc.init();
    GetRel get{V2, V2[S1 * A2.wk.idx]};
    const int row = T1 * kp.zlen;
    expect_rest<float, KAHAN>(acc, get, 0u, S1, A2.wk, P2.cb, kp.issuing, (uint32_t)P2.G, A2.y1, A2.R,
                              tab + kp.off_M + row, tab + kp.off_Mc + row, tab + kp.off_Mt + row, kp.zlen, 1.f);
    kp.two_mix[t] = acc.s;
}

// KAHAN = 1: the sum over d1 is compensated like the E2 and mixture sums.  Sixteen
// lanes share a state, lane j taking the product-1 orders a1 = j, j + 16, ..: each
// keeps the first argmax of its orders, and the lanes' bests are combined pairwise
// (the better one wins, an exact tie goes to the smaller joint order), so the first
// argmax over all orders comes out.  (Lanes over the product-2 orders instead, which
// run equal d1 loops, measured 6% slower.)
constexpr int kTwoLanes = 16;
template <int KAHAN>
__global__ void __launch_bounds__(kGenericThreads)
sweep_two_kernel(KernelParams kp, int mode, const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int) {
    SolveState *st = kp.st;
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    const uint32_t S1 = P1.nS;
    const float *tab = (const float *)kp.tables;
    const float2 *V2 = (const float2 *)B.vin;
    const float gam = (float)kp.gamma;
    const int lifo = kp.issuing;
    float mx = -INFINITY, mn = INFINITY;
    const uint32_t s = blockIdx.x * (uint32_t)(kGenericThreads / kTwoLanes) + (threadIdx.x / kTwoLanes);
    const int j = (int)(threadIdx.x % kTwoLanes);
    float bh = -INFINITY, bl = 0.f;
    int arg = 0;
    float2 R0 = make_float2(0.f, 0.f);
    if (s < kp.nS) {
        const uint32_t s2 = s / S1;
        const ProdState p1s = prod_state(P1, s - s2 * S1);
        const ProdState p2s = prod_state(P2, s2);
        R0 = V2[two_base_state(kp, p1s, p2s, 0)];
        for (int a1 = j; a1 < P1.G; a1 += kTwoLanes) {
            const ProdAction A1 = prod_action(P1, p1s, a1, lifo);
            const int top1 = min(A1.T, P1.dmax + 1);   // d1 in [0, top1)
            for (int a2 = 0; a2 < P2.G; ++a2) {
                const ProdAction A2 = prod_action(P2, p2s, a2, lifo);
                const uint32_t i20 = S1 * A2.wk.idx;
                const float2 ref = V2[A1.wk.idx + i20];
                const float *e2 = kp.two_e2 + ((uint64_t)s2 * P2.G + a2) * S1;
                float acc = 0.f;
                Acc<float, 1> kacc;   // KAHAN = 1 only
                kacc.init();
                Walker w1 = A1.wk;
                int e1c = 0;
                for (int d1 = 0; d1 < top1; ++d1) {
                    const int e1 = lifo ? min(d1, A1.R) : max(d1 - A1.y1, 0);
                    for (; e1c < e1; ++e1c) walker_step(w1, P1.cb, lifo, (uint32_t)P1.G);
                    const float t = e2[w1.idx] + pair_diff(V2[w1.idx + i20], ref);
                    if (KAHAN) kacc.add(tab[P1.off_p + d1], t);
                    else acc = fmaf(tab[P1.off_p + d1], t, acc);
                }
                if (A1.T <= P1.dmax) {
                    const float t = kp.two_mix[((uint32_t)s2 * P2.G + a2) * kp.two_nt1 + A1.T];
                    if (KAHAN) {
                        kacc.add(1.f, t);
                        kacc.add(tab[P1.off_tail + A1.T], pair_diff(V2[i20], ref));
                    } else {
                        acc += t + tab[P1.off_tail + A1.T] * pair_diff(V2[i20], ref);
                    }
                }
                if (KAHAN) acc = kacc.s;
                float qh, ql;
                const float ca =
                    __fadd_rn(__fmul_rn(-(float)P1.c_o, (float)a1), __fmul_rn(-(float)P2.c_o, (float)a2));
                action_base(gam, ref, R0, ca, qh, ql);
                const int i1 = h1_index(kp, A1), i2 = h2_index(kp, A1, A2);
                pair_add(qh, ql, tab[kp.off_H1 + i1], tab[kp.off_H1lo + i1]);
                pair_add(qh, ql, tab[kp.off_H2 + i2], tab[kp.off_H2lo + i2]);
                ql = __fmaf_rn(gam, acc, ql);
                const float diff = __fadd_rn(__fsub_rn(qh, bh), __fsub_rn(ql, bl));
                const bool up = diff > 0.f;
                bh = up ? qh : bh;
                bl = up ? ql : bl;
                arg = up ? a1 * P2.G + a2 : arg;
            }
        }
    }
    // the state's lanes: lower lanes hold the lower product-1 orders
#pragma unroll
    for (int off = 1; off < kTwoLanes; off <<= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, bh, off);
        const float ol = __shfl_xor_sync(0xffffffffu, bl, off);
        const int oa = __shfl_xor_sync(0xffffffffu, arg, off);
        const bool lower = (j & off) == 0;
        const float Lh = lower ? bh : oh, Ll = lower ? bl : ol, Uh = lower ? oh : bh, Ul = lower ? ol : bl;
        const int La = lower ? arg : oa, Ua = lower ? oa : arg;
        const float diff = __fadd_rn(__fsub_rn(Uh, Lh), __fsub_rn(Ul, Ll));
        const bool up = diff > 0.f || (diff == 0.f && Ua < La);
        bh = up ? Uh : Lh;
        bl = up ? Ul : Ll;
        arg = up ? Ua : La;
    }
    if (s < kp.nS && j == 0) {
        const float2 vold = V2[s];
        if (mode == MODE_EXTRACT) {
            if (B.vout) ((float2 *)B.vout)[s] = vold;
        } else {
            const float2 vnew = pair_finish(gam, R0, bh, bl);
            ((float2 *)B.vout)[s] = vnew;
            const float dlt = pair_diff(vnew, vold);
            mx = mn = dlt;
        }
        if (B.pol) B.pol[s] = (uint8_t)arg;
    }
    if (mode != MODE_EXTRACT) block_reduce_and_finalize<float>(mx, mn, st, mode, gridDim.x);
}

// ===========================================================================
// factorised two-product sweep with lead times >= 2 (the paper's Scenario B:
// an order arrives before the next period, so this library's state holds it in
// the arrival slot P_1).  The order of this period then only fills the top
// pipeline digit: issuing, the expected reward and the next stock slots do not
// depend on the action, and V(s') is read at s'(no order) + a1 w1 + S1 a2 w2.
// Per sweep, with c(s2, a2) = V(0, i2_0 + a2 w2) the reference of a row,
//   E2(i1, s2, a2)  = sum_d2 p2(d2) [V(i1, i2(s2, d2) + a2 w2) - c]
//   Mix(s2, a2, pipe1, T1) = sum_z M(T1, z) [V(pipe1 W1, i2(s2, z) + a2 w2) - c]
// (M = the product-2 demand z = d2 + substitutes when d1 >= T1), and the sweep
//   Q(s, a) = H(s) - c_o a + gamma [c + sum_{d1 < T1} p1(d1) E2(i1(d1) + a1 w1, s2, a2)
//                                      + Mix(s2, a2, pipe1(a1), T1)].
// States sharing the rest r1 of product 1 (all X_1 = x) share every gathered
// E2 value: FIFO takes k = d1 - x units from the rest, LIFO min(d1, R1), so one
// thread computes all x of a rest as a correlation over k.  The E2 and Mix
// kernels use the same correlation over product 2's expiring slot.
// ===========================================================================

// pmf-like coefficients of a correlation row: point mass, cumulative, tail,
// with the values a table of length n takes beyond its end
struct CoefRow {
    const float *p, *c, *t;
    int n;
    __device__ __forceinline__ float pm(int i) const { return i < n ? p[i] : 0.f; }
    __device__ __forceinline__ float cum(int i) const { return i < n ? c[i] : c[n - 1]; }
    __device__ __forceinline__ float tl(int i) const { return i < n ? t[i] : 0.f; }
};

// expectation over product 2's issuing for every expiring-slot value x2 < XW of
// the rest r2: out[x2] = sum_e w(x2, e) g(e), g(e) = value after e units taken
// from the rest (FIFO: e = clamp(z - x2, 0, R2); LIFO: e = min(z, R2))
template <int XW, class Gather>
__device__ __forceinline__ void corr_product2(float (&out)[XW], const Gather &g, Walker wk, const ProdParams &P,
                                              int lifo, int R, const CoefRow &w) {
    if (!lifo) {
        const float g0 = g(wk.idx);
        if (R == 0) {
#pragma unroll
            for (int x = 0; x < XW; ++x) out[x] = w.cum(w.n - 1) * g0;
            return;
        }
#pragma unroll
        for (int x = 0; x < XW; ++x) out[x] = w.cum(x) * g0;
        int e = 1;
        for (; e < R && e < w.n; ++e) {
            walker_step(wk, P.cb, 0, (uint32_t)P.G);
            const float ge = g(wk.idx);
#pragma unroll
            for (int x = 0; x < XW; ++x) out[x] = fmaf(w.pm(x + e), ge, out[x]);
        }
        if (R < w.n) {
            for (; e <= R; ++e) walker_step(wk, P.cb, 0, (uint32_t)P.G);
            const float gR = g(wk.idx);
#pragma unroll
            for (int x = 0; x < XW; ++x) out[x] = fmaf(w.tl(x + R), gR, out[x]);
        }
    } else {
        float acc = 0.f;
        int e = 0;
        for (; e < R && e < w.n; ++e) {
            acc = fmaf(w.pm(e), g(wk.idx), acc);
            walker_step(wk, P.cb, 1, (uint32_t)P.G);
        }
        if (R < w.n) acc = fmaf(w.tl(R), g(wk.idx), acc);
#pragma unroll
        for (int x = 0; x < XW; ++x) out[x] = acc;
    }
}

struct GetRow {
    const float2 *V;
    uint32_t base, mult;
    float2 ref;
    __device__ __forceinline__ float operator()(uint32_t i2) const { return pair_diff(V[base + mult * i2], ref); }
};

// thread = (i1, r2, a2), i1 fastest: writes E2 for every x2 of the rest r2
template <int XW>
__global__ void __launch_bounds__(kGenericThreads)
twop_e2_kernel(KernelParams kp, int mode, const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int) {
    SolveState *st = kp.st;
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    const uint32_t S1 = P1.nS;
    const uint32_t G2 = (uint32_t)P2.G;
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (uint64_t)S1 * P2.nS) return;
    const uint32_t i1 = (uint32_t)(t % S1);
    const uint32_t rest = (uint32_t)(t / S1);
    const int a2 = (int)(rest % G2);
    const uint32_t r2 = rest / G2;
    const ProdState ps = prod_state(P2, r2 * G2);
    const ProdAction A = prod_action(P2, ps, a2, kp.issuing);
    const float2 *V2 = (const float2 *)B.vin;
    const float *tab = (const float *)kp.tables;
    const GetRow g{V2, i1, S1, V2[(uint64_t)S1 * A.wk.idx]};
    const CoefRow w{tab + P2.off_p, tab + P2.off_F, tab + P2.off_tail, P2.pn};
    float out[XW];
    corr_product2<XW>(out, g, A.wk, P2, kp.issuing, A.R, w);
#pragma unroll
    for (int x = 0; x < XW; ++x)
        if (x < P2.G) kp.two_e2[((uint64_t)(r2 * G2 + (uint32_t)x) * G2 + (uint32_t)a2) * S1 + i1] = out[x];
}

// thread = (pipe1, T1, a2, r2): the substitution mixture for every x2 of r2
template <int XW>
__global__ void __launch_bounds__(kGenericThreads)
twop_mix_kernel(KernelParams kp, int mode, const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int) {
    SolveState *st = kp.st;
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    const uint32_t S1 = P1.nS;
    const uint32_t G2 = (uint32_t)P2.G;
    const uint32_t np1 = (uint32_t)kp.two_npipe1, nt = (uint32_t)kp.two_nt1;
    const uint64_t n = (uint64_t)np1 * nt * P2.nS;
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint32_t pipe1 = (uint32_t)(t % np1);
    uint64_t rest = t / np1;
    const int T1 = (int)(rest % nt);
    rest /= nt;
    const int a2 = (int)(rest % G2);
    const uint32_t r2 = (uint32_t)(rest / G2);
    const ProdState ps = prod_state(P2, r2 * G2);
    const ProdAction A = prod_action(P2, ps, a2, kp.issuing);
    const float2 *V2 = (const float2 *)B.vin;
    const float *tab = (const float *)kp.tables;
    const uint32_t w1s = P1.nS / (uint32_t)np1;   // G1^(m1-1): weight of the first pipeline digit
    const GetRow g{V2, pipe1 * w1s, S1, V2[(uint64_t)S1 * A.wk.idx]};
    const int row = T1 * kp.zlen;
    const CoefRow w{tab + kp.off_M + row, tab + kp.off_Mc + row, tab + kp.off_Mt + row, kp.zlen};
    float out[XW];
    corr_product2<XW>(out, g, A.wk, P2, kp.issuing, A.R, w);
#pragma unroll
    for (int x = 0; x < XW; ++x)
        if (x < P2.G)
            kp.two_mix[(((uint64_t)(r2 * G2 + (uint32_t)x) * G2 + (uint32_t)a2) * np1 + pipe1) * nt + (uint32_t)T1] =
                out[x];
}

// shared-memory layout of the pipeline sweep: four copies of p1 shifted by
// 0..3 (so that the window p1[e..e+XW) is an aligned float4 run of copy e & 3),
// F1[x] and F1[x-1] for x < 32, then the per-thread column of rest-path indices
__host__ __device__ inline int twop_pn4(const ProdParams &P1) { return ((P1.dmax + 36) + 3) & ~3; }
__host__ __device__ inline size_t twop_smem(const ProdParams &P1, int threads) {
    return (size_t)(4 * twop_pn4(P1) + 64) * sizeof(float) + (size_t)(P1.dmax + 2) * threads * sizeof(uint32_t);
}

// orders handled together (their gathers share one probability-window load) and
// resident blocks per SM: split lanes trade order blocking for occupancy
template <int XW, int LPR>
struct TwopBlock {
    static constexpr int AB = (XW <= 8) ? (LPR == 1 ? 4 : 2) : ((XW <= 16) ? 2 : 1);
    static constexpr int MINB = (XW <= 8) ? (LPR == 1 ? 4 : 5) : ((XW <= 16) ? 4 : 3);
};

// thread = (part, rank, s2), part fastest; rank -> r1 through a permutation that
// orders the rests of product 1 by their unit total R1, so that the lanes of a
// warp walk rest paths of one length.  The LPR lanes of a rest split the G1
// states x + G1 r1 of product 1 with product-2 state s2 (lane `part` owns x =
// part XW .. part XW + XW - 1) and gather the same values, which the warp
// serves once; splitting keeps fewer accumulators per lane and more warps per
// SM.  A lane covers every joint order, keeps a float key of Q - gamma R0 - H
// per state and forms the exact float pair of the best order once at the end.
template <int XW, int LPR>
__global__ void __launch_bounds__(kGenericThreads, TwopBlock<XW, LPR>::MINB)
twop_sweep_kernel(KernelParams kp, int mode, const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int) {
    constexpr int AB = TwopBlock<XW, LPR>::AB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SolveState *st = kp.st;
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    const float *tab = (const float *)kp.tables;
    const int pn4 = twop_pn4(P1);
    float *s_pc = (float *)smem_raw;
    float *s_F0 = s_pc + 4 * pn4;
    float *s_Fm = s_F0 + 32;
    uint32_t *s_col = (uint32_t *)(s_Fm + 32);
    for (int i = threadIdx.x; i < 4 * pn4; i += blockDim.x) {
        const int j = i / pn4, k = i - j * pn4 + j;
        s_pc[i] = (k < P1.pn) ? tab[P1.off_p + k] : 0.f;
    }
    for (int i = threadIdx.x; i < 32; i += blockDim.x) {
        s_F0[i] = tab[P1.off_F + i];                      // pn > 32 always
        s_Fm[i] = (i == 0) ? 0.f : tab[P1.off_F + i - 1];
    }
    __syncthreads();
    const uint32_t S1 = P1.nS;
    const uint32_t G1 = (uint32_t)P1.G, G2 = (uint32_t)P2.G;
    const uint32_t NR1 = S1 / G1;
    const int lifo = kp.issuing;
    const int dmax1 = P1.dmax;
    const float gam = (float)kp.gamma;
    const float2 *V2 = (const float2 *)B.vin;
    const uint32_t bd = blockDim.x, tid = threadIdx.x;
    float mx = -INFINITY, mn = INFINITY;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t u = t / (uint32_t)LPR;
    const int x0 = (int)(t - u * (uint32_t)LPR) * XW;   // first expiring-slot value of this lane
    if (u < NR1 * P2.nS) {
        const uint32_t r1 = kp.two_rperm[u % NR1];
        const uint32_t s2 = u / NR1;
        const ProdState ps1 = prod_state(P1, r1 * G1);
        const ProdAction A1 = prod_action(P1, ps1, 0, lifo);
        const int R1 = A1.R;
        // rest path of product 1: s'(e) with no order, e = 0..E1
        const int E1 = lifo ? min(R1, dmax1 + 1) : min(max(R1 - 1, 0), dmax1);
        {
            Walker wk = A1.wk;
            s_col[tid] = wk.idx;
            for (int e = 1; e <= E1; ++e) {
                walker_step(wk, P1.cb, lifo, G1);
                s_col[e * bd + tid] = wk.idx;
            }
        }
        const ProdState ps2 = prod_state(P2, s2);
        const ProdAction A2 = prod_action(P2, ps2, 0, lifo);
        const float2 R0 = V2[r1 + S1 * A2.wk.idx];
        const uint32_t np1 = (uint32_t)kp.two_npipe1, nt = (uint32_t)kp.two_nt1;
        const uint32_t w1s = S1 / np1;
        const uint32_t pipe_base = r1 / w1s;                        // P_2..P_{L-1} of product 1
        const uint32_t pipe_step = np1 / G1;                        // G1^(L1-2): weight of the order
        const float *cf0 = ((R1 >= 1) ? s_F0 : s_Fm) + x0;          // weight of the rest-free path
        float key[XW];
        int arg[XW];
#pragma unroll
        for (int x = 0; x < XW; ++x) {
            key[x] = -INFINITY;
            arg[x] = 0;
        }
        for (int a2 = 0; a2 < P2.G; ++a2) {
            const uint32_t i2n = A2.wk.idx + (uint32_t)a2 * P2.w_top;
            const float2 c = V2[(uint64_t)S1 * i2n];
            const float *row = kp.two_e2 + ((uint64_t)s2 * G2 + (uint32_t)a2) * S1;
            const float *mixb = kp.two_mix + ((uint64_t)s2 * G2 + (uint32_t)a2) * np1 * nt;
            for (int a1b = 0; a1b < P1.G; a1b += AB) {
                uint32_t off[AB];
#pragma unroll
                for (int j = 0; j < AB; ++j) off[j] = (uint32_t)min(a1b + j, P1.G - 1) * P1.w_top;
                // accumulators in pairs of x; with 8 x per lane the correlation runs on
                // packed two-lane FP32 instructions, each lane rounded as the scalar one
                // (measured on B300: 2.5% faster at 8, 6-12% slower at 16, whose
                // registers are all taken)
                constexpr bool PK = XW <= 8;
                float2 acc2[AB][XW / 2];
                auto acc = [&](int j, int x) -> float & { return (x & 1) ? acc2[j][x >> 1].y : acc2[j][x >> 1].x; };
                if (!lifo) {
                    const uint32_t i0 = s_col[tid];
#pragma unroll
                    for (int j = 0; j < AB; ++j) {
                        const float g = row[i0 + off[j]];
#pragma unroll
                        for (int q = 0; q < XW / 4; ++q) {
                            const float4 f = ((const float4 *)cf0)[q];
                            if constexpr (PK) {
                                const float2 g2 = make_float2(g, g);
                                acc2[j][2 * q] = __fmul2_rn(make_float2(f.x, f.y), g2);
                                acc2[j][2 * q + 1] = __fmul2_rn(make_float2(f.z, f.w), g2);
                            } else {
                                acc(j, 4 * q + 0) = __fmul_rn(f.x, g);
                                acc(j, 4 * q + 1) = __fmul_rn(f.y, g);
                                acc(j, 4 * q + 2) = __fmul_rn(f.z, g);
                                acc(j, 4 * q + 3) = __fmul_rn(f.w, g);
                            }
                        }
                    }
                    for (int e = 1; e <= E1; ++e) {
                        const uint32_t ie = s_col[e * bd + tid];
                        float g[AB];
#pragma unroll
                        for (int j = 0; j < AB; ++j) g[j] = row[ie + off[j]];
                        const float4 *pw = (const float4 *)(s_pc + (e & 3) * pn4 + (e & ~3) + x0);
#pragma unroll
                        for (int q = 0; q < XW / 4; ++q) {
                            const float4 f = pw[q];
#pragma unroll
                            for (int j = 0; j < AB; ++j) {
                                if constexpr (PK) {
                                    const float2 g2 = make_float2(g[j], g[j]);
                                    acc2[j][2 * q] = __ffma2_rn(make_float2(f.x, f.y), g2, acc2[j][2 * q]);
                                    acc2[j][2 * q + 1] = __ffma2_rn(make_float2(f.z, f.w), g2, acc2[j][2 * q + 1]);
                                } else {
                                    acc(j, 4 * q + 0) = __fmaf_rn(f.x, g[j], acc(j, 4 * q + 0));
                                    acc(j, 4 * q + 1) = __fmaf_rn(f.y, g[j], acc(j, 4 * q + 1));
                                    acc(j, 4 * q + 2) = __fmaf_rn(f.z, g[j], acc(j, 4 * q + 2));
                                    acc(j, 4 * q + 3) = __fmaf_rn(f.w, g[j], acc(j, 4 * q + 3));
                                }
                            }
                        }
                    }
                } else {
                    const int ne = min(R1, dmax1 + 1);
#pragma unroll
                    for (int j = 0; j < AB; ++j) {
                        float sum = 0.f;
                        for (int e = 0; e < ne; ++e) sum = __fmaf_rn(s_pc[e], row[s_col[e * bd + tid] + off[j]], sum);
                        if (R1 <= dmax1) {
                            // d1 in [R1, T1): all of the rest taken, the expiring slot partly
                            const float gR = row[s_col[R1 * bd + tid] + off[j]];
                            float cw = 0.f;
                            for (int y = 0; y < x0; ++y) cw = __fadd_rn(cw, s_pc[R1 + y]);
#pragma unroll
                            for (int x = 0; x < XW; ++x) {
                                acc(j, x) = __fmaf_rn(cw, gR, sum);
                                cw = __fadd_rn(cw, s_pc[R1 + x0 + x]);
                            }
                        } else {
#pragma unroll
                            for (int x = 0; x < XW; ++x) acc(j, x) = sum;
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < AB; ++j) {
                    const int a1 = a1b + j;
                    if (a1 < P1.G) {
                        const float *mixr = mixb + (pipe_base + (uint32_t)a1 * pipe_step) * nt;
                        float qh, ql;
                        const float ca =
                            __fadd_rn(__fmul_rn(-(float)P1.c_o, (float)a1), __fmul_rn(-(float)P2.c_o, (float)a2));
                        action_base(gam, c, R0, ca, qh, ql);
                        const float base = __fadd_rn(qh, ql);
                        const int code = a1 * P2.G + a2;
#pragma unroll
                        for (int x = 0; x < XW; ++x) {
                            const int T1 = x0 + x + R1;   // mixture rows exist for T1 <= min(dmax1, m1 Q1)
                            const float ax = (T1 < (int)nt) ? __fadd_rn(acc(j, x), mixr[T1]) : acc(j, x);
                            const float k = __fmaf_rn(gam, ax, base);
                            const bool up = k > key[x];
                            key[x] = up ? k : key[x];
                            arg[x] = up ? code : arg[x];
                        }
                    }
                }
            }
        }
        // exact float pair of the chosen order; the expected reward depends on
        // the state only and is added after the max
        const int ys2 = lifo ? A2.R : A2.y1;
        const int ny2 = lifo ? (P2.tmax + 1) : P2.G;
#pragma unroll
        for (int xl = 0; xl < XW; ++xl) {
            const int x = x0 + xl;
            if (x < P1.G) {
                const int a1 = arg[xl] / P2.G, a2 = arg[xl] - a1 * P2.G;
                const uint32_t i2n = A2.wk.idx + (uint32_t)a2 * P2.w_top;
                const float2 c = V2[(uint64_t)S1 * i2n];
                const float *row = kp.two_e2 + ((uint64_t)s2 * G2 + (uint32_t)a2) * S1;
                const uint32_t off = (uint32_t)a1 * P1.w_top;
                float ax;
                if (!lifo) {
                    ax = __fmul_rn(cf0[xl], row[s_col[tid] + off]);
                    for (int e = 1; e <= E1; ++e) ax = __fmaf_rn(s_pc[x + e], row[s_col[e * bd + tid] + off], ax);
                } else {
                    float sum = 0.f;
                    const int ne = min(R1, dmax1 + 1);
                    for (int e = 0; e < ne; ++e) sum = __fmaf_rn(s_pc[e], row[s_col[e * bd + tid] + off], sum);
                    if (R1 <= dmax1) {
                        float cw = 0.f;
                        for (int y = 0; y < x; ++y) cw = __fadd_rn(cw, s_pc[R1 + y]);
                        ax = __fmaf_rn(cw, row[s_col[R1 * bd + tid] + off], sum);
                    } else {
                        ax = sum;
                    }
                }
                const int T1 = x + R1;
                if (T1 < (int)nt) {
                    const float *mixr = kp.two_mix + (((uint64_t)s2 * G2 + (uint32_t)a2) * np1 + pipe_base +
                                                      (uint32_t)a1 * pipe_step) * nt;
                    ax = __fadd_rn(ax, mixr[T1]);
                }
                float h, l;
                const float ca =
                    __fadd_rn(__fmul_rn(-(float)P1.c_o, (float)a1), __fmul_rn(-(float)P2.c_o, (float)a2));
                action_base(gam, c, R0, ca, h, l);
                l = __fmaf_rn(gam, ax, l);
                const uint32_t s = (uint32_t)x + G1 * r1 + S1 * s2;
                const int i1 = (lifo ? R1 : x) * (P1.tmax + 1) + T1;
                const int i2 = (T1 * ny2 + ys2) * (P2.tmax + 1) + A2.T;
                pair_add(h, l, tab[kp.off_H1 + i1], tab[kp.off_H1lo + i1]);
                pair_add(h, l, tab[kp.off_H2 + i2], tab[kp.off_H2lo + i2]);
                const float2 vold = V2[s];
                if (mode == MODE_EXTRACT) {
                    if (B.vout) ((float2 *)B.vout)[s] = vold;
                } else {
                    const float2 vnew = pair_finish(gam, R0, h, l);
                    ((float2 *)B.vout)[s] = vnew;
                    const float dlt = pair_diff(vnew, vold);
                    mx = fmaxf(mx, dlt);
                    mn = fminf(mn, dlt);
                }
                if (B.pol) B.pol[s] = (uint8_t)arg[xl];
            }
        }
    }
    if (mode != MODE_EXTRACT) block_reduce_and_finalize<float>(mx, mn, st, mode, gridDim.x);
}

static int twop_width(int G) { return G <= 8 ? 8 : (G <= 16 ? 16 : 32); }
// Lanes per rest of the sweep: one lane per rest while that gives the device
// about four waves of threads (measured best at 10-17M states); below, lanes of
// 8 values, which doubled the threads of the 15K-38K-state settings and cut
// their sweep by about a fifth.
static int twop_lanes(const ProdParams &P1, const ProdParams &P2) {
    const uint64_t threads = (uint64_t)(P1.nS / (uint32_t)P1.G) * P2.nS;
    if (P1.G <= 8 || threads >= 4ull * 148 * 512) return 1;
    return P1.G <= 16 ? 2 : 4;
}

static cudaError_t describe_twop(const KernelParams &kp, LaunchDesc &d) {
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    const int w1 = twop_width(P1.G), w2 = twop_width(P2.G);
    const uint64_t n_e2 = (uint64_t)P1.nS * P2.nS;
    const uint64_t n_mix = (uint64_t)kp.two_npipe1 * (uint32_t)kp.two_nt1 * P2.nS;
    const int lp = twop_lanes(P1, P2);
    const uint64_t n_sw = (uint64_t)(P1.nS / (uint32_t)P1.G) * P2.nS * (uint64_t)lp;
    if (lp == 1)
        d.fn = (w1 == 8) ? (const void *)twop_sweep_kernel<8, 1>
                         : (w1 == 16) ? (const void *)twop_sweep_kernel<16, 1> : (const void *)twop_sweep_kernel<32, 1>;
    else
        d.fn = (lp == 2) ? (const void *)twop_sweep_kernel<8, 2> : (const void *)twop_sweep_kernel<8, 4>;
    d.grid = dim3((unsigned)((n_sw + kGenericThreads - 1) / kGenericThreads));
    d.block = dim3(kGenericThreads);
    d.smem = twop_smem(P1, kGenericThreads);
    d.lpr = 0;
    d.n_pre = 2;
    d.pre_fn[0] = (w2 == 8) ? (const void *)twop_e2_kernel<8>
                            : (w2 == 16) ? (const void *)twop_e2_kernel<16> : (const void *)twop_e2_kernel<32>;
    d.pre_grid[0] = dim3((unsigned)((n_e2 + kGenericThreads - 1) / kGenericThreads));
    d.pre_block[0] = dim3(kGenericThreads);
    d.pre_fn[1] = (w2 == 8) ? (const void *)twop_mix_kernel<8>
                            : (w2 == 16) ? (const void *)twop_mix_kernel<16> : (const void *)twop_mix_kernel<32>;
    d.pre_grid[1] = dim3((unsigned)((n_mix + kGenericThreads - 1) / kGenericThreads));
    d.pre_block[1] = dim3(kGenericThreads);
    return cudaSuccess;
}

// pipeline classes of product 1's emptied next state: G1^(L1-1) (1 with L1 = 1)
static size_t two_npipe1(const ProdParams &P1) {
    size_t n = 1;
    for (int k = 1; k < P1.L; ++k) n *= (size_t)P1.G;
    return n;
}

bool two_supported(const KernelParams &kp, int vk, int kahan) {
    if (kp.n_products != 2 || vk != VK_PAIR) return false;
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    size_t mix = 0;
    const size_t e2 = two_table_floats(kp, &mix);
    if (P1.L == 1 && P2.L == 1) return e2 <= ((size_t)1 << 27) && mix <= ((size_t)1 << 27);
    // lead times >= 2 on both products: the pipeline form; the correlation keeps
    // up to 32 expiring-slot values per thread and the rest path in shared memory.
    // Its sums are not compensated: VI_PREC_FP32_KAHAN runs the generic kernel instead.
    if (kahan || P1.L < 2 || P2.L < 2 || P1.m < 2 || P2.m < 2) return false;
    if (P1.G > 32 || P2.G > 32) return false;
    if (twop_smem(P1, kGenericThreads) > 48 * 1024) return false;
    return e2 <= ((size_t)1 << 30) && mix <= ((size_t)1 << 30);
}

int two_mix_rows(const ProdParams &P1) { return (P1.dmax < P1.tmax ? P1.dmax : P1.tmax) + 1; }

size_t two_table_floats(const KernelParams &kp, size_t *mix_floats) {
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    if (mix_floats) *mix_floats = (size_t)P2.nS * P2.G * two_npipe1(P1) * (size_t)two_mix_rows(P1);
    return (size_t)P1.nS * P2.nS * (size_t)P2.G;
}

static cudaError_t describe_two(const KernelParams &kp, int kahan, LaunchDesc &d) {
    const uint64_t n_e2 = (uint64_t)kp.p[0].nS * kp.p[1].nS * (uint32_t)kp.p[1].G;
    const uint64_t n_mix = (uint64_t)kp.p[1].nS * (uint32_t)kp.p[1].G * (uint32_t)kp.two_nt1;
    d.fn = kahan ? (const void *)sweep_two_kernel<1> : (const void *)sweep_two_kernel<0>;
    constexpr uint32_t per_block = kGenericThreads / kTwoLanes;   // states per block
    d.grid = dim3((unsigned)(((uint64_t)kp.nS + per_block - 1) / per_block));
    d.block = dim3(kGenericThreads);
    d.smem = 0;
    d.lpr = 0;
    d.n_pre = 2;
    d.pre_fn[0] = kahan ? (const void *)two_e2_kernel<1> : (const void *)two_e2_kernel<0>;
    d.pre_grid[0] = dim3((unsigned)((n_e2 + kGenericThreads - 1) / kGenericThreads));
    d.pre_block[0] = dim3(kGenericThreads);
    d.pre_fn[1] = kahan ? (const void *)two_mix_kernel<1> : (const void *)two_mix_kernel<0>;
    d.pre_grid[1] = dim3((unsigned)((n_mix + kGenericThreads - 1) / kGenericThreads));
    d.pre_block[1] = dim3(kGenericThreads);
    return cudaSuccess;
}

cudaError_t describe_sweep(const KernelParams &kp, int vk, int kahan, int use_group, LaunchDesc &d) {
    d.lpr = 0;
    d.n_pre = 0;
    if (kp.pc) return describe_pc(kp, d);
    if (use_group == kTcWidth) return describe_tc(kp, d);
    if (use_group == kLifo1Width) return describe_lifo1(kp, d);
    if (use_group == kFifoColWidth) return describe_fifo_col(kp, d);
    if (use_group == kTwoWidth) return (kp.p[0].L >= 2) ? describe_twop(kp, d) : describe_two(kp, kahan, d);
    if (use_group) {
        const int xw = use_group;   // lane width of the factorised kernel
        const bool pipe = kp.p[0].L >= 2;
        if (vk == VK_PAIR) {
            if (kp.issuing) return pipe ? describe_group_lifo_pipe(kp, xw, d) : describe_group_lifo(kp, xw, d);
            return pipe ? describe_group_fifo_pipe(kp, xw, d) : describe_group_fifo(kp, xw, d);
        }
        return kp.issuing ? describe_group_lifo_single(kp, xw, d) : describe_group_fifo_single(kp, xw, d);
    }
    if (vk == VK_DOUBLE) return describe_generic_t<VK_DOUBLE, 0>(kp, d);
    if (vk == VK_PAIR) return kahan ? describe_generic_t<VK_PAIR, 1>(kp, d) : describe_generic_t<VK_PAIR, 0>(kp, d);
    return kahan ? describe_generic_t<VK_SINGLE, 1>(kp, d) : describe_generic_t<VK_SINGLE, 0>(kp, d);
}

// compact per-slot status for the server's host loop
__global__ void gather_status_kernel(SolveState *const *sts, int n, SlotStatus *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const SolveState *st = sts[i];
    out[i].iter = st->iter;
    out[i].keep_going = st->keep_going;
    out[i].converged = st->converged;
    out[i].crit = st->crit;
}

cudaError_t prepare_server_helpers() {
    cudaFuncAttributes fa;
    cudaError_t e;
    if ((e = cudaFuncGetAttributes(&fa, gather_status_kernel)) != cudaSuccess ||
        (e = cudaFuncGetAttributes(&fa, to_fp64_kernel)) != cudaSuccess ||
        (e = cudaFuncGetAttributes(&fa, solve_init_kernel)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

cudaError_t launch_gather_status(SolveState *const *sts, int n, SlotStatus *out, cudaStream_t stream) {
    gather_status_kernel<<<(n + 63) / 64, 64, 0, stream>>>(sts, n, out);
    return cudaGetLastError();
}

cudaError_t launch_solve_init(SolveState *st, uint32_t n, cudaStream_t stream) {
    solve_init_kernel<<<(n + 255) / 256, 256, 0, stream>>>(st, n);
    return cudaGetLastError();
}

cudaError_t describe_solve_init(uint32_t n, LaunchDesc &d) {
    d.fn = (const void *)solve_init_kernel;
    d.grid = dim3((n + 255) / 256);
    d.block = dim3(256);
    d.smem = 0;
    return cudaSuccess;
}

cudaError_t launch_next_states(const KernelParams &kp, const uint32_t *states, int n, uint32_t *out,
                               cudaStream_t stream) {
    const dim3 block(64), grid(n, (kp.nA + 63) / 64);
    next_states_kernel<<<grid, block, 0, stream>>>(kp, states, n, out);
    return cudaGetLastError();
}

cudaError_t launch_policy_eval(const KernelParams &kp, const uint8_t *policy, const double *vin, double *vout,
                               cudaStream_t stream) {
    const uint32_t blocks = (kp.nS + kGenericThreads - 1) / kGenericThreads;
    const int n_smem_tab = (kp.n_products == 2) ? kp.off_H1 : kp.n_tables;
    const size_t smem = kp.tab_in_smem ? (size_t)n_smem_tab * sizeof(double) : 0;
    const cudaError_t e =
        cudaFuncSetAttribute(policy_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    policy_eval_kernel<<<blocks, kGenericThreads, smem, stream>>>(kp, policy, vin, vout);
    return cudaGetLastError();
}

cudaError_t launch_to_fp64(const void *v, int vk, double offset, double *out, uint32_t n, cudaStream_t stream) {
    to_fp64_kernel<<<(n + 255) / 256, 256, 0, stream>>>(v, vk, offset, out, n);
    return cudaGetLastError();
}

cudaError_t launch_diff_range(const double *a, const double *b, uint32_t n, SolveState *st, cudaStream_t stream) {
    diff_range_kernel<<<(n + 255) / 256, 256, 0, stream>>>(a, b, n, st);
    return cudaGetLastError();
}

cudaError_t launch_rollouts(const KernelParams &kp, const RollParams &rp, const uint8_t *policy, double *returns,
                            double *kpis, double *kpis_prod, int32_t *traj, cudaStream_t stream) {
    const int per_block = kRollWarps * kRollRPW;
    const int blocks = (rp.n_rollouts + per_block - 1) / per_block;
    rollout_kernel<<<blocks, 32 * kRollWarps, 0, stream>>>(kp, rp, policy, returns, kpis, kpis_prod, traj);
    return cudaGetLastError();
}

}  // namespace vib

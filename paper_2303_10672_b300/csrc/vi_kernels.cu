// vi_kernels.cu -- sm_103a kernels of the value-iteration hot path.
//
//   sweep_group_kernel    factorised Bellman backup (one thread per rest index r,
//                         all G = Q+1 values of the expiring slot in registers)
//   sweep_generic_kernel  one thread per state, float / double / Kahan, one or
//                         two products
//   next_states_kernel    dump of T(s, a, omega) indices (bit-exact checks)
//   policy_eval_kernel    FP64 fixed-policy sweep
//   rollout_kernel        Philox4x32-10 policy rollouts with FP64 returns
//
// Bellman backup (Eq. valueiterationdetupdate):
//   V'(s) = max_a [ rbar(s,a) + gamma * sum_omega P(omega) V(s'(s,a,omega)) ]
// with the expected one-step reward rbar taken from FP64-built expectation tables
// (the reward of Eq. demoor:reward is affine in issued / short / wasted / carried
// units, so its expectation only needs E[(y - D)^+] tables).
#include <math.h>

#include "vi_common.cuh"
#include "vi_kernels.h"

namespace vib {

// ---------------------------------------------------------------------------
// block reductions of the per-sweep change statistics
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_minmax(double &mx, double &mn) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
}

// All threads of the block call this.  Folds (mx, mn) of the block into the
// global accumulators; the last block of the grid then runs finalize().
__device__ void block_reduce_and_finalize(double mx, double mn, SolveState *st, int mode) {
    __shared__ double s_mx[32], s_mn[32];
    __shared__ int s_last;
    warp_minmax(mx, mn);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_mx[wid] = mx;
        s_mn[wid] = mn;
    }
    __syncthreads();
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        mx = lane < nw ? s_mx[lane] : -INFINITY;
        mn = lane < nw ? s_mn[lane] : INFINITY;
        warp_minmax(mx, mn);
        if (lane == 0) {
            atomicMax(&st->key_max, dkey(mx));
            atomicMin(&st->key_min, dkey(mn));
            __threadfence();
            unsigned prev = atomicAdd(&st->blocks_done, 1u);
            s_last = (prev == gridDim.x - 1);
        }
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    double vmax = dkey_inv(atomicAdd(&st->key_max, 0ull));
    double vmin = dkey_inv(atomicAdd(&st->key_min, 0ull));
    if (mode == MODE_SWEEP) {
        double b_old = st->offset;
        double b_new = st->normalise ? (st->gamma * b_old + (double)st->c_cur) : 0.0;
        double db = b_new - b_old;
        st->offset = b_new;
        st->dmax_abs = db + vmax;
        st->dmin_abs = db + vmin;
        double crit = (st->stop_rule == 0) ? (vmax - vmin)
                                           : fmax(fabs(st->dmax_abs), fabs(st->dmin_abs));
        st->crit = crit;
        st->iter += 1;
        int conv = crit < st->tol;
        st->converged = conv;
        int go = (!conv) && (st->iter < st->max_iters);
        st->keep_going = go;
        if (st->normalise) st->c_cur = st->c_next;
        if (st->use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)st->cond, go ? 1u : 0u);
    } else {
        st->dmax_abs = vmax;
        st->dmin_abs = vmin;
        st->crit = vmax - vmin;
    }
    st->key_max = 0ull;
    st->key_min = ~0ull;
    __threadfence();
    st->blocks_done = 0u;
}

// resolve the buffers of a launch
template <typename T>
struct Bufs {
    const T *vin;
    T *vout;        // may be null (extraction without copy)
    uint8_t *pol;   // may be null
    T cnorm;
};

template <typename T>
__device__ __forceinline__ bool resolve_bufs(const SolveState *st, int mode, const T *vin_arg, T *vout_arg,
                                             uint8_t *pol_arg, Bufs<T> &b) {
    if (mode == MODE_SWEEP) {
        if (!st->keep_going) return false;
        int it = st->iter;
        b.vin = (const T *)st->buf[it & 1];
        b.vout = (T *)st->buf[(it + 1) & 1];
        b.pol = nullptr;
        b.cnorm = st->normalise ? (T)st->c_cur : (T)0;
    } else if (mode == MODE_EXTRACT) {
        int it = st->iter;
        b.vin = (const T *)st->buf[it & 1];
        b.vout = (it & 1) ? (T *)st->buf[0] : nullptr;   // result must end in the caller's buffer
        b.pol = st->policy;
        b.cnorm = (T)0;
    } else {
        b.vin = vin_arg;
        b.vout = vout_arg;
        b.pol = pol_arg;
        b.cnorm = (T)0;
    }
    return true;
}

template <typename T>
__device__ __forceinline__ void load_tables(T *s_tab, const T *g_tab, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) s_tab[i] = g_tab[i];
    __syncthreads();
}

// packed rest-slot counts and their sum for action a (the order joins the
// slots as Z_{m-1} when L == 1 and m >= 2)
__device__ __forceinline__ void slots_for_action(const ProdParams &P, const RestInfo &ri, int a,
                                                 unsigned long long &packed, int &R) {
    packed = ri.packed;
    R = ri.R;
    if (P.L == 1 && P.m >= 2) {
        packed |= (unsigned long long)a << (P.cb * (P.m - 2));
        R += a;
    }
}

// ===========================================================================
// factorised single-product sweep (FP32): thread = rest index r, registers hold
// the G values of the expiring slot x = X_1 (or P_1 when m == 1).
//   FIFO: C(x) = sum_d p_d g(clamp(d - x, 0, R))   (x is issued first)
//   LIFO: C    = sum_d p_d g(min(d, R))            (x is issued last)
// where g(e) = V[s'(r, a, e)] follows the walker.  The FIFO correlation is
// evaluated in chunks of G demands with a register window of gathered values.
// ===========================================================================
template <int G, int LIFO>
__global__ void __launch_bounds__(kGroupThreads)
sweep_group_kernel(KernelParams kp, int mode, const float *vin_arg, float *vout_arg, uint8_t *pol_arg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SolveState *st = kp.st;
    Bufs<float> B;
    if (!resolve_bufs<float>(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    const ProdParams &P = kp.p[0];
    float *s_tab = (float *)smem_raw;
    float *s_out = s_tab + ((kp.n_tables + 3) & ~3);
    uint8_t *s_pol = (uint8_t *)(s_out + kGroupThreads * G);
    load_tables<float>(s_tab, (const float *)kp.tables, kp.n_tables);
    const float *s_p = s_tab + P.off_p;
    const float *s_TA = s_tab + P.off_TA;
    const float *s_TB = s_tab + P.off_TB;

    const uint32_t nR = P.nS / (uint32_t)G;
    const uint32_t r0 = blockIdx.x * (uint32_t)kGroupThreads;
    const uint32_t r = r0 + threadIdx.x;
    const float gam = (float)kp.gamma;
    const float c_o = (float)P.c_o;
    const int dmax = P.dmax;
    const int nch = (dmax + G) / G;      // chunks of G demands covering 0..dmax

    float best[G];
    int arg[G];
#pragma unroll
    for (int x = 0; x < G; ++x) {
        best[x] = -INFINITY;
        arg[x] = 0;
    }
    if (r < nR) {
        RestInfo ri = decode_rest(r, P);
        const float *V = B.vin;
        for (int a = 0; a < G; ++a) {
            unsigned long long packed;
            int R;
            slots_for_action(P, ri, a, packed, R);
            Walker wk;
            walker_init(wk, r + (uint32_t)a * P.w_top, packed, P.m - 1, P.cb, LIFO, P.w_zt);
            float acc[G];
            if (!LIFO) {
                float gprev[G];
                float g0 = __ldg(V + wk.idx);
#pragma unroll
                for (int x = 0; x < G; ++x) {
                    acc[x] = 0.f;
                    gprev[x] = g0;
                }
                float glast = g0;
                for (int c = 0; c < nch; ++c) {
                    const int d0 = c * G;
                    float gcur[G];
#pragma unroll
                    for (int j = 0; j < G; ++j) {
                        int e = d0 + j;
                        if (e >= 1 && e <= R) {
                            walker_step(wk, P.cb, 0, (uint32_t)G);
                            glast = __ldg(V + wk.idx);
                        }
                        gcur[j] = glast;
                    }
#pragma unroll
                    for (int j = 0; j < G; ++j) {
                        const float pd = s_p[d0 + j];
#pragma unroll
                        for (int x = 0; x < G; ++x) {
                            const int e = j - x;
                            const float gv = (e >= 0) ? gcur[e] : gprev[G + e];
                            acc[x] = fmaf(pd, gv, acc[x]);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < G; ++j) gprev[j] = gcur[j];
                }
            } else {
                float c = 0.f;
                float g = __ldg(V + wk.idx);
                for (int d = 0; d <= dmax; ++d) {
                    if (d >= 1 && d <= R) {
                        walker_step(wk, P.cb, 1, (uint32_t)G);
                        g = __ldg(V + wk.idx);
                    }
                    c = fmaf(s_p[d], g, c);
                }
#pragma unroll
                for (int x = 0; x < G; ++x) acc[x] = c;
            }
            const float base = -c_o * (float)a;
#pragma unroll
            for (int x = 0; x < G; ++x) {
                const float rb = base + s_TA[x + R] + s_TB[LIFO ? R : x];
                const float q = fmaf(gam, acc[x], rb);
                if (q > best[x]) {
                    best[x] = q;
                    arg[x] = a;
                }
            }
        }
        if (r == 0 && mode == MODE_SWEEP) st->c_next = best[0];
    }
    // stage the block's G*kGroupThreads contiguous states through shared memory
#pragma unroll
    for (int x = 0; x < G; ++x) {
        s_out[threadIdx.x * G + x] = best[x];
        s_pol[threadIdx.x * G + x] = (uint8_t)arg[x];
    }
    __syncthreads();
    const uint32_t s0 = r0 * (uint32_t)G;
    const uint32_t nblk = kGroupThreads * G;
    double mx = -INFINITY, mn = INFINITY;
    for (uint32_t i = threadIdx.x; i < nblk; i += kGroupThreads) {
        const uint32_t s = s0 + i;
        if (s >= P.nS) break;
        if (mode == MODE_EXTRACT) {
            if (B.vout) B.vout[s] = B.vin[s];
        } else {
            const float vnew = s_out[i] - B.cnorm;
            const float vold = B.vin[s];
            B.vout[s] = vnew;
            const double dlt = (double)vnew - (double)vold;
            mx = fmax(mx, dlt);
            mn = fmin(mn, dlt);
        }
        if (B.pol) B.pol[s] = s_pol[i];
    }
    if (mode != MODE_EXTRACT) block_reduce_and_finalize(mx, mn, st, mode);
}

// ===========================================================================
// per-state expectation helpers (generic kernels, policy evaluation)
// ===========================================================================
template <typename T, int KAHAN>
struct Acc {
    T s, c;
    __device__ __forceinline__ void init() { s = (T)0; c = (T)0; }
    __device__ __forceinline__ void add(T w, T v) {
        if (KAHAN) {
            T y = w * v - c;
            T t = s + y;
            c = (t - s) - y;
            s = t;
        } else {
            s = s + w * v;
        }
    }
};

// expectation of g over the rest-demand e for one product:
//   FIFO: e = clamp(d - y1, 0, R); LIFO: e = min(d, R); g(e) = V[base + mult * s'(e)]
// w-tables (pw = point mass, cw = cumulative, tw = tail) over d; entries at or beyond
// n (the support length) are zero mass and are skipped
template <typename T, int KAHAN>
__device__ __forceinline__ void expect_rest(Acc<T, KAHAN> &acc, const T *V, uint32_t base, uint32_t mult,
                                            Walker wk, int cb, int lifo, uint32_t G, int y1, int R,
                                            const T *pw, const T *cw, const T *tw, int n, T scale) {
    // the index arithmetic only ever steps while e <= R
    if (!lifo) {
        if (R == 0) {
            acc.add(scale * tw[0], V[base + mult * wk.idx]);
            return;
        }
        int y = y1 < n - 1 ? y1 : n - 1;
        acc.add(scale * cw[y], V[base + mult * wk.idx]);
        int e = 1;
        for (; e < R; ++e) {
            if (y1 + e >= n) break;
            walker_step(wk, cb, 0, G);
            acc.add(scale * pw[y1 + e], V[base + mult * wk.idx]);
        }
        if (y1 + R < n) {
            for (; e <= R; ++e) walker_step(wk, cb, 0, G);
            acc.add(scale * tw[y1 + R], V[base + mult * wk.idx]);
        }
    } else {
        int d = 0;
        for (; d < R && d < n; ++d) {
            acc.add(scale * pw[d], V[base + mult * wk.idx]);
            walker_step(wk, cb, 1, G);
        }
        if (R < n) acc.add(scale * tw[R], V[base + mult * wk.idx]);
    }
}

// the state decomposition of one product: s_k = x + G r
struct ProdState {
    int x;
    uint32_t r;
    RestInfo ri;
};

__device__ __forceinline__ ProdState prod_state(const ProdParams &P, uint32_t sk) {
    ProdState ps;
    if (P.K >= 1) {
        ps.r = sk / (uint32_t)P.G;
        ps.x = (int)(sk - ps.r * (uint32_t)P.G);
    } else {
        ps.r = 0;
        ps.x = 0;
    }
    ps.ri = decode_rest(ps.r, P);
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
    uint32_t idx0 = (P.K >= 1) ? ps.r + (uint32_t)a * P.w_top : 0u;
    walker_init(pa.wk, idx0, packed, P.m - 1, P.cb, lifo, P.w_zt);
    return pa;
}

// Q(s, a) of a single-product state
template <typename T, int KAHAN>
__device__ __forceinline__ T q_single(const KernelParams &kp, const T *s_tab, const T *V, const ProdState &ps,
                                      int a) {
    const ProdParams &P = kp.p[0];
    const int lifo = kp.issuing;
    ProdAction pa = prod_action(P, ps, a, lifo);
    Acc<T, KAHAN> acc;
    acc.init();
    expect_rest<T, KAHAN>(acc, V, 0u, 1u, pa.wk, P.cb, lifo, (uint32_t)P.G, pa.y1, pa.R, s_tab + P.off_p,
                          s_tab + P.off_F, s_tab + P.off_tail, P.dmax + 1, (T)1);
    const T rb = -(T)P.c_o * (T)a + s_tab[P.off_TA + pa.T] + s_tab[P.off_TB + (lifo ? pa.R : pa.y1)];
    return rb + (T)kp.gamma * acc.s;
}

// Q(s, a) of a two-product state (product-1 shortfall may take product 2)
template <typename T, int KAHAN>
__device__ __forceinline__ T q_two(const KernelParams &kp, const T *s_tab, const T *g_tab, const T *V,
                                   const ProdState &p1s, const ProdState &p2s, int a) {
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    const int lifo = kp.issuing;
    const int a1 = a / P2.G, a2 = a - a1 * P2.G;
    ProdAction A1 = prod_action(P1, p1s, a1, lifo);
    ProdAction A2 = prod_action(P2, p2s, a2, lifo);
    const uint32_t S1 = P1.nS;
    Acc<T, KAHAN> acc;
    acc.init();
    // product-1 demand below its stock: product 2 sees its own demand only
    Walker w1 = A1.wk;
    int e1c = 0;
    const int top1 = A1.T < P1.dmax + 1 ? A1.T : P1.dmax + 1;   // d1 in [0, top1)
    for (int d1 = 0; d1 < top1; ++d1) {
        const int e1 = lifo ? min(d1, A1.R) : max(d1 - A1.y1, 0);   // < R1 or == R1 (LIFO)
        for (; e1c < e1; ++e1c) walker_step(w1, P1.cb, lifo, (uint32_t)P1.G);
        const T p1 = s_tab[P1.off_p + d1];
        expect_rest<T, KAHAN>(acc, V, w1.idx, S1, A2.wk, P2.cb, lifo, (uint32_t)P2.G, A2.y1, A2.R,
                              s_tab + P2.off_p, s_tab + P2.off_F, s_tab + P2.off_tail, P2.dmax + 1, p1);
    }
    // product-1 demand at or above its stock: rows of M give product 2's demand
    if (A1.T <= P1.dmax) {
        // walker 1 must sit at e = R1 (all rest units issued)
        for (; e1c < A1.R; ++e1c) walker_step(w1, P1.cb, lifo, (uint32_t)P1.G);
        const int row = A1.T * kp.zlen;
        expect_rest<T, KAHAN>(acc, V, w1.idx, S1, A2.wk, P2.cb, lifo, (uint32_t)P2.G, A2.y1, A2.R,
                              s_tab + kp.off_M + row, s_tab + kp.off_Mc + row, s_tab + kp.off_Mt + row,
                              kp.zlen, (T)1);
    }
    const int ys1 = lifo ? A1.R : A1.y1;
    const int ys2 = lifo ? A2.R : A2.y1;
    const int ny2 = lifo ? (P2.tmax + 1) : P2.G;
    const T h1 = g_tab[kp.off_H1 + ys1 * (P1.tmax + 1) + A1.T];
    const T h2 = g_tab[kp.off_H2 + (A1.T * ny2 + ys2) * (P2.tmax + 1) + A2.T];
    const T rb = -(T)P1.c_o * (T)a1 - (T)P2.c_o * (T)a2 + h1 + h2;
    return rb + (T)kp.gamma * acc.s;
}

// ===========================================================================
// generic sweep: thread = state
// ===========================================================================
template <typename T, int KAHAN>
__global__ void __launch_bounds__(kGenericThreads)
sweep_generic_kernel(KernelParams kp, int mode, const T *vin_arg, T *vout_arg, uint8_t *pol_arg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SolveState *st = kp.st;
    Bufs<T> B;
    if (!resolve_bufs<T>(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    T *s_tab = (T *)smem_raw;
    const int n_smem_tab = (kp.n_products == 2) ? kp.off_H1 : kp.n_tables;   // H tables stay global
    load_tables<T>(s_tab, (const T *)kp.tables, n_smem_tab);
    const T *g_tab = (const T *)kp.tables;

    double mx = -INFINITY, mn = INFINITY;
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < kp.nS) {
        T best = (T)-INFINITY;
        int arg = 0;
        if (kp.n_products == 1) {
            ProdState ps = prod_state(kp.p[0], s);
            for (int a = 0; a < kp.nA; ++a) {
                T q = q_single<T, KAHAN>(kp, s_tab, B.vin, ps, a);
                if (q > best) {
                    best = q;
                    arg = a;
                }
            }
        } else {
            const uint32_t S1 = kp.p[0].nS;
            const uint32_t s2 = s / S1;
            ProdState p1s = prod_state(kp.p[0], s - s2 * S1);
            ProdState p2s = prod_state(kp.p[1], s2);
            for (int a = 0; a < kp.nA; ++a) {
                T q = q_two<T, KAHAN>(kp, s_tab, g_tab, B.vin, p1s, p2s, a);
                if (q > best) {
                    best = q;
                    arg = a;
                }
            }
        }
        if (s == 0 && mode == MODE_SWEEP) st->c_next = (float)best;
        if (mode == MODE_EXTRACT) {
            if (B.vout) B.vout[s] = B.vin[s];
        } else {
            const T vnew = best - B.cnorm;
            const T vold = B.vin[s];
            B.vout[s] = vnew;
            const double dlt = (double)vnew - (double)vold;
            mx = dlt;
            mn = dlt;
        }
        if (B.pol) B.pol[s] = (uint8_t)arg;
    }
    if (mode != MODE_EXTRACT) block_reduce_and_finalize(mx, mn, st, mode);
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
        ProdState ps = prod_state(P, s);
        ProdAction pa = prod_action(P, ps, a, lifo);
        uint32_t *o = out + ((size_t)i * kp.nA + a) * (size_t)(P.dmax + 1);
        Walker wk = pa.wk;
        int e_cur = 0;
        for (int d = 0; d <= P.dmax; ++d) {
            int e = lifo ? min(d, pa.R) : min(max(d - pa.y1, 0), pa.R);
            for (; e_cur < e; ++e_cur) walker_step(wk, P.cb, lifo, (uint32_t)P.G);
            o[d] = wk.idx;
        }
        return;
    }
    const ProdParams &P1 = kp.p[0];
    const ProdParams &P2 = kp.p[1];
    const uint32_t S1 = P1.nS;
    const uint32_t s2 = s / S1;
    ProdState p1s = prod_state(P1, s - s2 * S1);
    ProdState p2s = prod_state(P2, s2);
    const int a1 = a / P2.G, a2 = a - a1 * P2.G;
    ProdAction A1 = prod_action(P1, p1s, a1, lifo);
    ProdAction A2 = prod_action(P2, p2s, a2, lifo);
    const int zl = P1.dmax + P2.dmax + 1;
    uint32_t *o = out + ((size_t)i * kp.nA + a) * (size_t)(P1.dmax + 1) * (size_t)zl;
    Walker w1 = A1.wk;
    int e1c = 0;
    for (int d1 = 0; d1 <= P1.dmax; ++d1) {
        int e1 = lifo ? min(d1, A1.R) : min(max(d1 - A1.y1, 0), A1.R);
        for (; e1c < e1; ++e1c) walker_step(w1, P1.cb, lifo, (uint32_t)P1.G);
        Walker w2 = A2.wk;
        int e2c = 0;
        for (int z = 0; z < zl; ++z) {
            int e2 = lifo ? min(z, A2.R) : min(max(z - A2.y1, 0), A2.R);
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
    double *s_tab = (double *)smem_raw;
    const int n_smem_tab = (kp.n_products == 2) ? kp.off_H1 : kp.n_tables;
    load_tables<double>(s_tab, (const double *)kp.tables, n_smem_tab);
    const double *g_tab = (const double *)kp.tables;
    double mx = -INFINITY, mn = INFINITY;
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < kp.nS) {
        const int a = policy[s];
        double q;
        if (kp.n_products == 1) {
            ProdState ps = prod_state(kp.p[0], s);
            q = q_single<double, 0>(kp, s_tab, vin, ps, a);
        } else {
            const uint32_t S1 = kp.p[0].nS;
            const uint32_t s2 = s / S1;
            ProdState p1s = prod_state(kp.p[0], s - s2 * S1);
            ProdState p2s = prod_state(kp.p[1], s2);
            q = q_two<double, 0>(kp, s_tab, g_tab, vin, p1s, p2s, a);
        }
        vout[s] = q;
        mx = mn = q - vin[s];
    }
    block_reduce_and_finalize(mx, mn, kp.st, MODE_PLAIN);
}

// V_abs = offset + v in FP64
__global__ void to_fp64_kernel(const float *v, double offset, double *out, uint32_t n) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = offset + (double)v[i];
}

// max_s |a(s) - b(s)| into the state's PLAIN accumulators
__global__ void absdiff_kernel(const double *a, const double *b, uint32_t n, SolveState *st) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    double d = 0.0;
    if (i < n) d = fabs(a[i] - b[i]);
    block_reduce_and_finalize(d, d, st, MODE_PLAIN);
}

// ===========================================================================
// solve bookkeeping kernels
// ===========================================================================
__global__ void solve_init_kernel(SolveState *st, uint32_t n) {
    // zero V_0 unless warm-starting, reset the running state
    const int warm = st->warm;
    const int value_bytes = st->value_bytes;
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (!warm) {
        if (value_bytes == 4) {
            if (i < n) ((float *)st->buf[0])[i] = 0.f;
        } else {
            if (i < n) ((double *)st->buf[0])[i] = 0.0;
        }
    }
    if (i == 0) {
        st->key_max = 0ull;
        st->key_min = ~0ull;
        st->blocks_done = 0u;
        st->iter = 0;
        st->converged = 0;
        st->crit = INFINITY;
        st->dmax_abs = 0.0;
        st->dmin_abs = 0.0;
        st->c_cur = 0.f;
        st->c_next = 0.f;
        if (!warm) st->offset = 0.0;
        int go = st->max_iters > 0;
        st->keep_going = go;
        if (st->use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)st->cond, go ? 1u : 0u);
    }
}

__global__ void state_reset_kernel(SolveState *st) {
    st->key_max = 0ull;
    st->key_min = ~0ull;
    st->blocks_done = 0u;
}

// ===========================================================================
// rollouts: thread = rollout
// ===========================================================================
struct RollOut {
    uint32_t s_next;
    int issued, wasted, carried, shortage, arrived, total;
};

// one product, one period, with the sweep kernels' walker for the next state
__device__ __forceinline__ RollOut roll_product(const ProdParams &P, int lifo, uint32_t sk, int a, int z) {
    ProdState ps = prod_state(P, sk);
    ProdAction pa = prod_action(P, ps, a, lifo);
    RollOut o;
    int e = lifo ? min(z, pa.R) : min(max(z - pa.y1, 0), pa.R);
    Walker wk = pa.wk;
    for (int k = 0; k < e; ++k) walker_step(wk, P.cb, lifo, (uint32_t)P.G);
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
            for (int j = 0; j < P.m - 2; ++j) q /= (uint32_t)P.G;
            o.arrived = (int)(q % (uint32_t)P.G);
        }
    } else {
        o.arrived = a;
    }
    return o;
}

// smallest d with w < thr[d], thr[d] = floor(2^32 CDF(d)) (thr[dmax] = 2^32)
__device__ __forceinline__ int draw_demand(uint32_t w, const unsigned long long *thr, int dmax) {
    int d = 0;
    while (d < dmax && (unsigned long long)w >= thr[d]) ++d;
    return d;
}

__global__ void rollout_kernel(KernelParams kp, RollParams rp, const uint8_t *policy, double *returns,
                               double *kpis, int32_t *traj) {
    __shared__ unsigned long long s_thr[2][kMaxRollDmax + 1];
    for (int i = threadIdx.x; i <= kMaxRollDmax; i += blockDim.x) {
        s_thr[0][i] = rp.thr[0][i];
        s_thr[1][i] = rp.thr[1][i];
    }
    __syncthreads();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rp.n_rollouts) return;
    const int lifo = kp.issuing;
    const uint32_t k0 = (uint32_t)(rp.seed & 0xffffffffull), k1 = (uint32_t)(rp.seed >> 32);
    uint32_t s = 0;
    double ret = 0.0, disc = 1.0;
    double dem = 0.0, iss = 0.0, was = 0.0, arr = 0.0, car = 0.0;
    const ProdParams &P1 = kp.p[0];
    for (int t = 0; t < rp.warmup + rp.horizon; ++t) {
        uint32_t w[4];
        philox4x32_10((uint32_t)t, (uint32_t)r, 0u, 0u, k0, k1, w);
        const int a = policy[s];
        double rew = 0.0;
        double t_dem, t_iss, t_was, t_arr, t_car;
        uint32_t s_next;
        if (kp.n_products == 1) {
            const int d1 = draw_demand(w[0], s_thr[0], P1.dmax);
            RollOut o = roll_product(P1, lifo, s, a, d1);
            rew = __dsub_rn(rew, __dmul_rn(rp.cost[0][0], (double)a));
            rew = __dsub_rn(rew, __dmul_rn(rp.cost[0][1], (double)o.carried));
            rew = __dsub_rn(rew, __dmul_rn(rp.cost[0][2], (double)o.shortage));
            rew = __dsub_rn(rew, __dmul_rn(rp.cost[0][3], (double)o.wasted));
            rew = __dadd_rn(rew, __dmul_rn(rp.cost[0][4], (double)o.issued));
            s_next = o.s_next;
            t_dem = d1;
            t_iss = o.issued;
            t_was = o.wasted;
            t_arr = o.arrived;
            t_car = o.carried;
        } else {
            const ProdParams &P2 = kp.p[1];
            const int d1 = draw_demand(w[0], s_thr[0], P1.dmax);
            const int d2 = draw_demand(w[1], s_thr[1], P2.dmax);
            const uint32_t S1 = P1.nS;
            const uint32_t s2 = s / S1, s1 = s - s2 * S1;
            const int a1 = a / P2.G, a2 = a - a1 * P2.G;
            RollOut o1 = roll_product(P1, lifo, s1, a1, d1);
            const int n = o1.shortage;
            const uint32_t mask = (n >= 32) ? 0xffffffffu : ((1u << n) - 1u);
            const int u = __popc(w[2] & mask);
            RollOut o2 = roll_product(P2, lifo, s2, a2, d2 + u);
            const int own2 = min(d2, o2.total);
            const int short1 = n - (o2.issued - own2);
            const int short2 = max(d2 - o2.total, 0);
            rew = __dsub_rn(rew, __dmul_rn(rp.cost[0][0], (double)a1));
            rew = __dsub_rn(rew, __dmul_rn(rp.cost[0][1], (double)o1.carried));
            rew = __dsub_rn(rew, __dmul_rn(rp.cost[0][2], (double)short1));
            rew = __dsub_rn(rew, __dmul_rn(rp.cost[0][3], (double)o1.wasted));
            rew = __dadd_rn(rew, __dmul_rn(rp.cost[0][4], (double)o1.issued));
            rew = __dsub_rn(rew, __dmul_rn(rp.cost[1][0], (double)a2));
            rew = __dsub_rn(rew, __dmul_rn(rp.cost[1][1], (double)o2.carried));
            rew = __dsub_rn(rew, __dmul_rn(rp.cost[1][2], (double)short2));
            rew = __dsub_rn(rew, __dmul_rn(rp.cost[1][3], (double)o2.wasted));
            rew = __dadd_rn(rew, __dmul_rn(rp.cost[1][4], (double)o2.issued));
            s_next = o1.s_next + S1 * o2.s_next;
            t_dem = d1 + d2;
            t_iss = o1.issued + o2.issued;
            t_was = o1.wasted + o2.wasted;
            t_arr = o1.arrived + o2.arrived;
            t_car = o1.carried + o2.carried;
        }
        if (t >= rp.warmup) {
            if (traj) traj[(size_t)r * rp.horizon + (t - rp.warmup)] = (int32_t)s;
            ret = __dadd_rn(ret, __dmul_rn(disc, rew));
            disc = __dmul_rn(disc, kp.gamma);
            dem = __dadd_rn(dem, t_dem);
            iss = __dadd_rn(iss, t_iss);
            was = __dadd_rn(was, t_was);
            arr = __dadd_rn(arr, t_arr);
            car = __dadd_rn(car, t_car);
        }
        s = s_next;
    }
    returns[r] = ret;
    if (kpis) {
        kpis[3 * r + 0] = dem > 0.0 ? __ddiv_rn(__dmul_rn(100.0, iss), dem) : 100.0;
        kpis[3 * r + 1] = arr > 0.0 ? __ddiv_rn(__dmul_rn(100.0, was), arr) : 0.0;
        kpis[3 * r + 2] = rp.horizon > 0 ? __ddiv_rn(car, (double)rp.horizon) : 0.0;
    }
}

// ===========================================================================
// launchers
// ===========================================================================
static size_t group_smem(const KernelParams &kp, int G) {
    return (size_t)((kp.n_tables + 3) & ~3) * 4 + (size_t)kGroupThreads * G * 5;
}

template <int G, int LIFO>
static cudaError_t launch_group_t(const KernelParams &kp, int mode, const float *vin, float *vout,
                                  uint8_t *pol, cudaStream_t stream) {
    const uint32_t nR = kp.p[0].nS / (uint32_t)G;
    const uint32_t blocks = (nR + kGroupThreads - 1) / kGroupThreads;
    size_t smem = group_smem(kp, G);
    auto fn = sweep_group_kernel<G, LIFO>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<blocks, kGroupThreads, smem, stream>>>(kp, mode, vin, vout, pol);
    return cudaGetLastError();
}

template <int LIFO>
static cudaError_t launch_group_l(const KernelParams &kp, int G, int mode, const float *vin, float *vout,
                                  uint8_t *pol, cudaStream_t stream) {
    switch (G) {
#define VIB_G(g) \
    case g: return launch_group_t<g, LIFO>(kp, mode, vin, vout, pol, stream);
        VIB_G(2) VIB_G(3) VIB_G(4) VIB_G(5) VIB_G(6) VIB_G(7) VIB_G(8) VIB_G(9) VIB_G(10) VIB_G(11)
        VIB_G(12) VIB_G(13) VIB_G(14) VIB_G(15) VIB_G(16) VIB_G(17) VIB_G(18) VIB_G(19) VIB_G(20)
        VIB_G(21) VIB_G(22) VIB_G(23) VIB_G(24)
#undef VIB_G
        default: return cudaErrorInvalidValue;
    }
}

bool group_supported(const KernelParams &kp) {
    const ProdParams &P = kp.p[0];
    return kp.n_products == 1 && P.K >= 1 && P.G >= 2 && P.G <= kMaxGroupG;
}

cudaError_t launch_sweep_group(const KernelParams &kp, int mode, const float *vin, float *vout,
                               uint8_t *pol, cudaStream_t stream) {
    if (kp.issuing) return launch_group_l<1>(kp, kp.p[0].G, mode, vin, vout, pol, stream);
    return launch_group_l<0>(kp, kp.p[0].G, mode, vin, vout, pol, stream);
}

template <typename T, int KAHAN>
static cudaError_t launch_generic_t(const KernelParams &kp, int mode, const void *vin, void *vout,
                                    uint8_t *pol, cudaStream_t stream) {
    const uint32_t blocks = (kp.nS + kGenericThreads - 1) / kGenericThreads;
    const int n_smem_tab = (kp.n_products == 2) ? kp.off_H1 : kp.n_tables;
    size_t smem = (size_t)n_smem_tab * sizeof(T);
    auto fn = sweep_generic_kernel<T, KAHAN>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<blocks, kGenericThreads, smem, stream>>>(kp, mode, (const T *)vin, (T *)vout, pol);
    return cudaGetLastError();
}

cudaError_t launch_sweep_generic(const KernelParams &kp, int precision, int mode, const void *vin, void *vout,
                                 uint8_t *pol, cudaStream_t stream) {
    if (precision == 2) return launch_generic_t<double, 0>(kp, mode, vin, vout, pol, stream);
    if (precision == 1) return launch_generic_t<float, 1>(kp, mode, vin, vout, pol, stream);
    return launch_generic_t<float, 0>(kp, mode, vin, vout, pol, stream);
}

cudaError_t launch_next_states(const KernelParams &kp, const uint32_t *states, int n, uint32_t *out,
                               cudaStream_t stream) {
    dim3 block(64), grid(n, (kp.nA + 63) / 64);
    next_states_kernel<<<grid, block, 0, stream>>>(kp, states, n, out);
    return cudaGetLastError();
}

cudaError_t launch_policy_eval(const KernelParams &kp, const uint8_t *policy, const double *vin, double *vout,
                               cudaStream_t stream) {
    const uint32_t blocks = (kp.nS + kGenericThreads - 1) / kGenericThreads;
    const int n_smem_tab = (kp.n_products == 2) ? kp.off_H1 : kp.n_tables;
    size_t smem = (size_t)n_smem_tab * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(policy_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    policy_eval_kernel<<<blocks, kGenericThreads, smem, stream>>>(kp, policy, vin, vout);
    return cudaGetLastError();
}

cudaError_t launch_to_fp64(const float *v, double offset, double *out, uint32_t n, cudaStream_t stream) {
    to_fp64_kernel<<<(n + 255) / 256, 256, 0, stream>>>(v, offset, out, n);
    return cudaGetLastError();
}

cudaError_t launch_absdiff(const double *a, const double *b, uint32_t n, SolveState *st, cudaStream_t stream) {
    absdiff_kernel<<<(n + 255) / 256, 256, 0, stream>>>(a, b, n, st);
    return cudaGetLastError();
}

cudaError_t launch_solve_init(SolveState *st, uint32_t n, cudaStream_t stream) {
    solve_init_kernel<<<(n + 255) / 256, 256, 0, stream>>>(st, n);
    return cudaGetLastError();
}

cudaError_t launch_state_reset(SolveState *st, cudaStream_t stream) {
    state_reset_kernel<<<1, 1, 0, stream>>>(st);
    return cudaGetLastError();
}

cudaError_t launch_rollouts(const KernelParams &kp, const RollParams &rp, const uint8_t *policy, double *returns,
                            double *kpis, int32_t *traj, cudaStream_t stream) {
    const int threads = 128;
    const int blocks = (rp.n_rollouts + threads - 1) / threads;
    rollout_kernel<<<blocks, threads, 0, stream>>>(kp, rp, policy, returns, kpis, traj);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// kernel descriptors for CUDA-graph construction
// ---------------------------------------------------------------------------
template <int G, int LIFO>
static cudaError_t describe_group_t(const KernelParams &kp, LaunchDesc &d) {
    const uint32_t nR = kp.p[0].nS / (uint32_t)G;
    d.fn = (const void *)sweep_group_kernel<G, LIFO>;
    d.grid = dim3((nR + kGroupThreads - 1) / kGroupThreads);
    d.block = dim3(kGroupThreads);
    d.smem = group_smem(kp, G);
    return cudaFuncSetAttribute(sweep_group_kernel<G, LIFO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)d.smem);
}

template <int LIFO>
static cudaError_t describe_group_l(const KernelParams &kp, LaunchDesc &d) {
    switch (kp.p[0].G) {
#define VIB_G(g) \
    case g: return describe_group_t<g, LIFO>(kp, d);
        VIB_G(2) VIB_G(3) VIB_G(4) VIB_G(5) VIB_G(6) VIB_G(7) VIB_G(8) VIB_G(9) VIB_G(10) VIB_G(11)
        VIB_G(12) VIB_G(13) VIB_G(14) VIB_G(15) VIB_G(16) VIB_G(17) VIB_G(18) VIB_G(19) VIB_G(20)
        VIB_G(21) VIB_G(22) VIB_G(23) VIB_G(24)
#undef VIB_G
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int KAHAN>
static cudaError_t describe_generic_t(const KernelParams &kp, LaunchDesc &d) {
    d.fn = (const void *)sweep_generic_kernel<T, KAHAN>;
    d.grid = dim3((kp.nS + kGenericThreads - 1) / kGenericThreads);
    d.block = dim3(kGenericThreads);
    const int n_smem_tab = (kp.n_products == 2) ? kp.off_H1 : kp.n_tables;
    d.smem = (size_t)n_smem_tab * sizeof(T);
    return cudaFuncSetAttribute(sweep_generic_kernel<T, KAHAN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)d.smem);
}

cudaError_t describe_sweep(const KernelParams &kp, int precision, int use_group, LaunchDesc &d) {
    if (use_group) {
        if (kp.issuing) return describe_group_l<1>(kp, d);
        return describe_group_l<0>(kp, d);
    }
    if (precision == 2) return describe_generic_t<double, 0>(kp, d);
    if (precision == 1) return describe_generic_t<float, 1>(kp, d);
    return describe_generic_t<float, 0>(kp, d);
}

cudaError_t describe_solve_init(uint32_t n, LaunchDesc &d) {
    d.fn = (const void *)solve_init_kernel;
    d.grid = dim3((n + 255) / 256);
    d.block = dim3(256);
    d.smem = 0;
    return cudaSuccess;
}

}  // namespace vib

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

#include "vi_common.cuh"
#include "vi_kernels.h"

namespace vib {

// ---------------------------------------------------------------------------
// error-free float transformations (never contracted into FMAs)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {   // |a| >= |b|
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
// difference of two float pairs as an FP32 number (correctly rounded when the
// high parts are within a factor of two of each other)
__device__ __forceinline__ float pair_diff(float2 g, float2 ref) {
    return __fadd_rn(__fsub_rn(g.x, ref.x), __fsub_rn(g.y, ref.y));
}

// ---------------------------------------------------------------------------
// block reductions of the per-sweep change statistics
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void warp_minmax(T &mx, T &mn) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
}

// All threads of the block call this.  Folds (mx, mn) of the block into the
// global accumulators; the last block of the grid then finalises the sweep.
template <typename T>
__device__ void block_reduce_and_finalize(T mx, T mn, SolveState *st, int mode, unsigned n_blocks) {
    __shared__ T s_mx[32], s_mn[32];
    __shared__ int s_last;
    warp_minmax<T>(mx, mn);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_mx[wid] = mx;
        s_mn[wid] = mn;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        mx = lane < nw ? s_mx[lane] : (T)-INFINITY;
        mn = lane < nw ? s_mn[lane] : (T)INFINITY;
        warp_minmax<T>(mx, mn);
        if (lane == 0) {
            atomicMax(&st->key_max, dkey((double)mx));
            atomicMin(&st->key_min, dkey((double)mn));
            __threadfence();
            const unsigned prev = atomicAdd(&st->blocks_done, 1u);
            s_last = (prev == n_blocks - 1);
        }
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    const double vmax = dkey_inv(atomicAdd(&st->key_max, 0ull));
    const double vmin = dkey_inv(atomicAdd(&st->key_min, 0ull));
    if (mode == MODE_SWEEP) {
        const double b_old = st->offset;
        const double b_new = st->normalise ? (st->gamma * b_old + (double)st->c_cur) : 0.0;
        const double db = b_new - b_old;
        st->offset = b_new;
        st->dmax_abs = db + vmax;
        st->dmin_abs = db + vmin;
        const double crit = (st->stop_rule == 0) ? (vmax - vmin) : fmax(fabs(st->dmax_abs), fabs(st->dmin_abs));
        st->crit = crit;
        st->iter += 1;
        const int conv = crit < st->tol;
        st->converged = conv;
        const int go = (!conv) && (st->iter < st->max_iters);
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

// buffers of one launch
struct Bufs {
    const void *vin;
    void *vout;      // may be null (extraction without copy)
    uint8_t *pol;    // may be null
    float cnorm;     // VK_SINGLE normalisation constant
};

__device__ __forceinline__ bool resolve_bufs(const SolveState *st, int mode, const void *vin_arg, void *vout_arg,
                                             uint8_t *pol_arg, Bufs &b) {
    if (mode == MODE_SWEEP) {
        if (!st->keep_going) return false;
        const int it = st->iter;
        b.vin = st->buf[it & 1];
        b.vout = st->buf[(it + 1) & 1];
        b.pol = nullptr;
        b.cnorm = st->normalise ? st->c_cur : 0.f;
    } else if (mode == MODE_EXTRACT) {
        const int it = st->iter;
        b.vin = st->buf[it & 1];
        b.vout = (it & 1) ? st->buf[0] : nullptr;   // the result must end in the caller's buffer
        b.pol = st->policy;
        b.cnorm = 0.f;
    } else {
        b.vin = vin_arg;
        b.vout = vout_arg;
        b.pol = pol_arg;
        b.cnorm = 0.f;
    }
    return true;
}

template <typename T>
__device__ __forceinline__ void load_tables(T *s_tab, const T *g_tab, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) s_tab[i] = g_tab[i];
    __syncthreads();
}

// packed rest-slot counts and their sum for action a (the order joins the slots
// as Z_{m-1} when L == 1 and m >= 2)
__device__ __forceinline__ void slots_for_action(const ProdParams &P, const RestInfo &ri, int a,
                                                 unsigned long long &packed, int &R) {
    packed = ri.packed;
    R = ri.R;
    if (P.L == 1 && P.m >= 2) {
        packed |= (unsigned long long)a << (P.cb * (P.m - 2));
        R += a;
    }
}

// a pair (hi, lo) += (xh, xl), high parts added error-free
__device__ __forceinline__ void pair_add(float &h, float &l, float xh, float xl) {
    float s, e;
    two_sum(h, xh, s, e);
    h = s;
    l = __fadd_rn(e, __fadd_rn(l, xl));
}

// gamma * (ref - R0) - c_o a as a pair
__device__ __forceinline__ void action_base(float gam, float2 ref, float2 R0, float ca, float &bh, float &bl) {
    float dh, de;
    two_sum(ref.x, -R0.x, dh, de);
    const float dl = __fadd_rn(de, __fsub_rn(ref.y, R0.y));
    float ph, pe;
    two_prod(gam, dh, ph, pe);
    const float pl = __fmaf_rn(gam, dl, pe);
    float s, e;
    two_sum(ca, ph, s, e);
    bh = s;
    bl = __fadd_rn(e, pl);
}

// gamma * R0 + (bh, bl), normalised pair
__device__ __forceinline__ float2 pair_finish(float gam, float2 R0, float bh, float bl) {
    float ph, pe;
    two_prod(gam, R0.x, ph, pe);
    const float pl = __fmaf_rn(gam, R0.y, pe);
    float sh, se;
    two_sum(ph, bh, sh, se);
    const float lo = __fadd_rn(se, __fadd_rn(pl, bl));
    float vh, vl;
    fast_two_sum(sh, lo, vh, vl);
    return make_float2(vh, vl);
}

// ===========================================================================
// factorised single-product sweep.  A rest index r (digits 1..K-1 of s) is
// handled by `lpr` consecutive lanes; lane `part` owns the XW values
// x = part*XW .. part*XW+XW-1 of the expiring slot (digit 0 of s), kept in
// registers.  For a given order a the next states only depend on r, a and the
// demand e that reaches the other slots, g(e) = V[s'(r, a, e)]:
//   FIFO: C(x) = sum_d p_d g(clamp(d - x, 0, R))   (x is issued first)
//   LIFO: C    = sum_d p_d g(min(d, R))            (x is issued last)
// The FIFO correlation runs in chunks of XW demands over a register window of
// gathered values; each chunk first walks the next-state indices, then issues
// all of its loads, then consumes them, so the loads overlap.
// ===========================================================================
template <int XW, int LIFO, int VK>
__device__ __forceinline__ void group_body(const KernelParams &kp, uint32_t bid, unsigned n_blocks, int mode,
                                           const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int lpr,
                                           unsigned char *smem_raw) {
    constexpr bool PAIR = (VK == VK_PAIR);
    constexpr int LCH = 8;   // LIFO load batch
    SolveState *st = kp.st;
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    const ProdParams &P = kp.p[0];
    const int G = P.G;
    const int RB = kGroupThreads / lpr;                    // rests per block
    float *s_tab = (float *)smem_raw;
    float *s_out = s_tab + ((kp.n_tables + 3) & ~3);       // PAIR: float2 per state
    uint8_t *s_pol = (uint8_t *)(s_out + RB * G * (PAIR ? 2 : 1));
    load_tables<float>(s_tab, (const float *)kp.tables, kp.n_tables);
    const float *s_p = s_tab + P.off_p;
    const float *s_RT = s_tab + P.off_RT;
    const float *s_RTlo = s_tab + P.off_RTlo;

    const uint32_t nR = P.nS / (uint32_t)G;
    const int rl = threadIdx.x / lpr;
    const int part = threadIdx.x - rl * lpr;
    const uint32_t r = bid * (uint32_t)RB + (uint32_t)rl;
    const bool active = (rl < RB) && (r < nR);
    const int x0 = part * XW;
    const int nx = min(XW, G - x0);                        // >= 1 because lpr = ceil(G / XW)
    const float gam = (float)kp.gamma;
    const float c_o = (float)P.c_o;
    const int dmax = P.dmax;
    const bool shared_lifo = LIFO && lifo_shared_ok(P);
    const bool shared_fifo = !LIFO && fifo_shared_ok(P);
    // per-thread columns (stride kGroupThreads) of the shared LIFO sequences / FIFO path
    float *colT = (float *)(((uintptr_t)(s_pol + RB * G) + 15) & ~(uintptr_t)15) + threadIdx.x;
    float *colH = colT + G * kGroupThreads;
    uint32_t *colP = (uint32_t *)colT;
    int Rrest = 0;   // units in the rest slots (without the order when L = 1)

    float bh[XW], bl[XW];
    int arg[XW];
#pragma unroll
    for (int xi = 0; xi < XW; ++xi) {
        bh[xi] = -INFINITY;
        bl[xi] = 0.f;
        arg[xi] = 0;
    }
    float2 R0 = make_float2(0.f, 0.f);
    if (active) {
        const RestInfo ri = decode_rest(r, P);
        Rrest = ri.R;
        const float *V1 = (const float *)B.vin;
        const float2 *V2 = (const float2 *)B.vin;
        if (PAIR) R0 = __ldg(V2 + r);   // s'_0 of action 0
        if (shared_fifo) {
            // FIFO: the demand reaching the rest slots empties them oldest first; that path
            // (relative to the rest index r) is the same for every order
            Walker wp;
            walker_init(wp, r, ri.packed, P.n_rest_slots, P.cb, 0, 1u);
            const int nP = min(ri.R, dmax) + 1;
            uint32_t *cp = colP;
            cp[0] = r;
            for (int e = 1; e < nP; ++e) {
                walker_step(wp, P.cb, 0, (uint32_t)G);
                cp[e * kGroupThreads] = wp.idx;
            }
        }
        if (shared_lifo) {
            // LIFO with L = 1 issues the new order first, so every action's next states
            // come from two shared sequences: T[j] = V[r + j G^(K-1)] (part of the order
            // left) and H[k] = V[state r after k units issued LIFO from X_{m-1}..X_2]
            const int nH = min(ri.R, dmax) + 1;
            auto value = [&](uint32_t i) -> float {
                if (PAIR) return pair_diff(__ldg(V2 + i), R0);
                return __ldg(V1 + i);
            };
            for (int j0 = 0; j0 < G; j0 += LCH) {
                float v[LCH];
#pragma unroll
                for (int j = 0; j < LCH; ++j) v[j] = (j0 + j < G) ? value(r + (uint32_t)(j0 + j) * P.w_top) : 0.f;
#pragma unroll
                for (int j = 0; j < LCH; ++j)
                    if (j0 + j < G) colT[(j0 + j) * kGroupThreads] = v[j];
            }
            Walker wh;
            walker_init(wh, r, ri.packed, P.m - 2, P.cb, 1, P.m >= 3 ? P.w_zt / (uint32_t)G : 1u);
            int kc = 0;
            for (int k0 = 0; k0 < nH; k0 += LCH) {
                uint32_t idx[LCH];
#pragma unroll
                for (int j = 0; j < LCH; ++j) {
                    const int kk = min(k0 + j, nH - 1);
                    for (; kc < kk; ++kc) walker_step(wh, P.cb, 1, (uint32_t)G);
                    idx[j] = wh.idx;
                }
                float v[LCH];
#pragma unroll
                for (int j = 0; j < LCH; ++j) v[j] = value(idx[j]);
#pragma unroll
                for (int j = 0; j < LCH; ++j)
                    if (k0 + j < nH) colH[(k0 + j) * kGroupThreads] = v[j];
            }
        }
        for (int a = 0; a < G; ++a) {
            unsigned long long packed;
            int R;
            slots_for_action(P, ri, a, packed, R);
            Walker wk;
            const uint32_t idx0 = r + (uint32_t)a * P.w_top;
            walker_init(wk, idx0, packed, P.m - 1, P.cb, LIFO, P.w_zt);
            float2 ref = make_float2(0.f, 0.f);
            float g0 = 0.f;
            if (shared_lifo)
                ref = R0;   // all shared values are measured from R0
            else if (PAIR)
                ref = __ldg(V2 + idx0);
            else
                g0 = __ldg(V1 + idx0);
            float acc[XW];
            if (!LIFO) {
                // lane-local demand axis dd = d - x0: C(x0+xi) = sum_dd p[dd+x0] g(clamp(dd-xi, 0, R))
                float gprev[XW];
#pragma unroll
                for (int xi = 0; xi < XW; ++xi) {
                    acc[xi] = 0.f;
                    gprev[xi] = g0;
                }
                int ecur = 0;
                const int nch = (dmax + XW) / XW;
                // one chunk of XW demands; in the first chunk of a float-pair sweep the window
                // before it holds g(0) - ref = 0 exactly, so those products are skipped
                const uint32_t atop = (uint32_t)a * P.w_top;
                auto chunk = [&](int c, auto first) {
                    constexpr bool FIRST = decltype(first)::value;
                    const int d0 = c * XW - x0;
                    uint32_t idx[XW];
                    if (shared_fifo) {
                        // rest path shared by all orders; with L = 1 the order is issued last
                        // demands beyond dmax carry no mass: clamping e there keeps every index inside
                        // the column (0..min(Rrest, dmax)) and inside the value array
                        const int ecap = min(R, dmax);
#pragma unroll
                        for (int j = 0; j < XW; ++j) {
                            const int e = min(max(d0 + j, 0), ecap);
                            idx[j] = (e <= Rrest) ? colP[e * kGroupThreads] + atop
                                                  : (uint32_t)(a - (e - Rrest)) * P.w_top;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < XW; ++j) {
                            const int e = min(max(d0 + j, 0), R);
                            for (; ecur < e; ++ecur) walker_step(wk, P.cb, 0, (uint32_t)G);
                            idx[j] = wk.idx;
                        }
                    }
                    float gcur[XW];
                    if (PAIR) {
                        float2 raw[XW];
#pragma unroll
                        for (int j = 0; j < XW; ++j) raw[j] = __ldg(V2 + idx[j]);
#pragma unroll
                        for (int j = 0; j < XW; ++j) gcur[j] = pair_diff(raw[j], ref);
                    } else {
#pragma unroll
                        for (int j = 0; j < XW; ++j) gcur[j] = __ldg(V1 + idx[j]);
                    }
#pragma unroll
                    for (int j = 0; j < XW; ++j) {
                        const float pd = s_p[d0 + x0 + j];
#pragma unroll
                        for (int xi = 0; xi < XW; ++xi) {
                            const int kk = j - xi;
                            if (PAIR && FIRST && kk < 0) continue;
                            const float gv = (kk >= 0) ? gcur[kk] : gprev[XW + kk];
                            acc[xi] = fmaf(pd, gv, acc[xi]);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < XW; ++j) gprev[j] = gcur[j];
                };
                chunk(0, std::true_type{});
                for (int c = 1; c < nch; ++c) chunk(c, std::false_type{});
            } else if (shared_lifo) {
                // C_a = sum_d p_d g_a(min(d, R)), g_a(e) = T[a-e] (e <= a) or H[e-a] (e > a)
                float c = 0.f;
                for (int d = 0; d <= dmax; ++d) {
                    const int e = min(d, R);
                    const float v = (e <= a) ? colT[(a - e) * kGroupThreads] : colH[(e - a) * kGroupThreads];
                    c = fmaf(s_p[d], v, c);
                }
#pragma unroll
                for (int xi = 0; xi < XW; ++xi) acc[xi] = c;
            } else {
                float c = 0.f;
                int ecur = 0;
                for (int d0 = 0; d0 <= dmax; d0 += LCH) {
                    uint32_t idx[LCH];
#pragma unroll
                    for (int j = 0; j < LCH; ++j) {
                        const int e = min(d0 + j, R);
                        for (; ecur < e; ++ecur) walker_step(wk, P.cb, 1, (uint32_t)G);
                        idx[j] = wk.idx;
                    }
                    float gv[LCH];
                    if (PAIR) {
                        float2 raw[LCH];
#pragma unroll
                        for (int j = 0; j < LCH; ++j) raw[j] = __ldg(V2 + idx[j]);
#pragma unroll
                        for (int j = 0; j < LCH; ++j) gv[j] = pair_diff(raw[j], ref);
                    } else {
#pragma unroll
                        for (int j = 0; j < LCH; ++j) gv[j] = __ldg(V1 + idx[j]);
                    }
#pragma unroll
                    for (int j = 0; j < LCH; ++j) c = fmaf(s_p[d0 + j], gv[j], c);   // zero mass beyond dmax
                }
#pragma unroll
                for (int xi = 0; xi < XW; ++xi) acc[xi] = c;
            }
            const float *rt = s_RT + R * G + x0;
            if (PAIR) {
                float Bh, Bl;
                action_base(gam, ref, R0, __fmul_rn(-c_o, (float)a), Bh, Bl);
                const float *rtl = s_RTlo + R * G + x0;
#pragma unroll
                for (int xi = 0; xi < XW; ++xi) {
                    if (xi < nx) {
                        float qh = Bh, ql = Bl;
                        pair_add(qh, ql, rt[xi], rtl[xi]);
                        ql = __fmaf_rn(gam, acc[xi], ql);
                        const float diff = __fadd_rn(__fsub_rn(qh, bh[xi]), __fsub_rn(ql, bl[xi]));
                        if (diff > 0.f) {
                            bh[xi] = qh;
                            bl[xi] = ql;
                            arg[xi] = a;
                        }
                    }
                }
            } else {
                const float base = -c_o * (float)a;
#pragma unroll
                for (int xi = 0; xi < XW; ++xi) {
                    if (xi < nx) {
                        const float q = fmaf(gam, acc[xi], base + rt[xi]);
                        if (q > bh[xi]) {
                            bh[xi] = q;
                            arg[xi] = a;
                        }
                    }
                }
            }
        }
        if (!PAIR && r == 0 && part == 0 && mode == MODE_SWEEP) st->c_next = bh[0];
    }
    // stage the block's G * RB contiguous states through shared memory
    if (rl < RB) {
#pragma unroll
        for (int xi = 0; xi < XW; ++xi) {
            if (xi < nx) {
                const int o = rl * G + x0 + xi;
                if (PAIR)
                    ((float2 *)s_out)[o] = active ? pair_finish(gam, R0, bh[xi], bl[xi]) : make_float2(0.f, 0.f);
                else
                    s_out[o] = bh[xi];
                s_pol[o] = (uint8_t)arg[xi];
            }
        }
    }
    __syncthreads();
    const uint32_t s0 = bid * (uint32_t)(RB * G);
    const uint32_t nblk = (uint32_t)(RB * G);
    float mx = -INFINITY, mn = INFINITY;
    for (uint32_t i = threadIdx.x; i < nblk; i += kGroupThreads) {
        const uint32_t s = s0 + i;
        if (s >= P.nS) break;
        if (PAIR) {
            const float2 *vin2 = (const float2 *)B.vin;
            float2 *vout2 = (float2 *)B.vout;
            if (mode == MODE_EXTRACT) {
                if (vout2) vout2[s] = vin2[s];
            } else {
                const float2 vnew = ((const float2 *)s_out)[i];
                const float2 vold = vin2[s];
                vout2[s] = vnew;
                const float dlt = pair_diff(vnew, vold);
                mx = fmaxf(mx, dlt);
                mn = fminf(mn, dlt);
            }
        } else {
            const float *vin1 = (const float *)B.vin;
            float *vout1 = (float *)B.vout;
            if (mode == MODE_EXTRACT) {
                if (vout1) vout1[s] = vin1[s];
            } else {
                const float vnew = s_out[i] - B.cnorm;
                const float vold = vin1[s];
                vout1[s] = vnew;
                const float dlt = vnew - vold;
                mx = fmaxf(mx, dlt);
                mn = fminf(mn, dlt);
            }
        }
        if (B.pol) B.pol[s] = s_pol[i];
    }
    if (mode != MODE_EXTRACT) block_reduce_and_finalize<float>(mx, mn, st, mode, n_blocks);
}

template <int XW, int LIFO, int VK>
__global__ void __launch_bounds__(kGroupThreads)
sweep_group_kernel(KernelParams kp, int mode, const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int lpr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    group_body<XW, LIFO, VK>(kp, blockIdx.x, gridDim.x, mode, vin_arg, vout_arg, pol_arg, lpr, smem_raw);
}

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
    if (s_kp.issuing)
        group_body<XW, 1, VK_PAIR>(s_kp, local, nb, modes[s], nullptr, nullptr, nullptr, lprs[s], smem_raw);
    else
        group_body<XW, 0, VK_PAIR>(s_kp, local, nb, modes[s], nullptr, nullptr, nullptr, lprs[s], smem_raw);
}

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
__global__ void absdiff_kernel(const double *a, const double *b, uint32_t n, SolveState *st) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    double d = 0.0;
    if (i < n) d = fabs(a[i] - b[i]);
    block_reduce_and_finalize<double>(d, d, st, MODE_PLAIN, gridDim.x);
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
// rollouts: thread = rollout
// ===========================================================================
struct RollOut {
    uint32_t s_next;
    int issued, wasted, carried, shortage, arrived, total;
};

// one product, one period, with the sweep kernels' walker for the next state
__device__ __forceinline__ RollOut roll_product(const ProdParams &P, int lifo, uint32_t sk, int a, int z) {
    const ProdState ps = prod_state(P, sk);
    const ProdAction pa = prod_action(P, ps, a, lifo);
    RollOut o;
    const int e = lifo ? min(z, pa.R) : min(max(z - pa.y1, 0), pa.R);
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

__global__ void rollout_kernel(KernelParams kp, RollParams rp, const uint8_t *policy, double *returns, double *kpis,
                               int32_t *traj) {
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
            const RollOut o = roll_product(P1, lifo, s, a, d1);
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
            const RollOut o1 = roll_product(P1, lifo, s1, a1, d1);
            const int n = o1.shortage;
            const uint32_t mask = (n >= 32) ? 0xffffffffu : ((1u << n) - 1u);
            const int u = __popc(w[2] & mask);
            const RollOut o2 = roll_product(P2, lifo, s2, a2, d2 + u);
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
// launch descriptors and launchers
// ===========================================================================
static size_t group_smem(const KernelParams &kp, int rb, int vk) {
    const ProdParams &P = kp.p[0];
    const size_t vb = (vk == VK_PAIR) ? 8 : 4;
    size_t bytes = (size_t)((kp.n_tables + 3) & ~3) * 4 + (size_t)rb * P.G * (vb + 1) + 16;
    if (kp.issuing && lifo_shared_ok(P)) bytes += (size_t)(P.G + P.dmax + 1) * kGroupThreads * 4;
    if (!kp.issuing && fifo_shared_ok(P)) bytes += (size_t)(P.dmax + 1) * kGroupThreads * 4;
    return bytes;
}

template <int XW, int LIFO, int VK>
static cudaError_t describe_group_t(const KernelParams &kp, LaunchDesc &d) {
    const int G = kp.p[0].G;
    const int lpr = (G + XW - 1) / XW;
    const int rb = kGroupThreads / lpr;
    const uint32_t nR = kp.p[0].nS / (uint32_t)G;
    d.fn = (const void *)sweep_group_kernel<XW, LIFO, VK>;
    d.grid = dim3((nR + rb - 1) / rb);
    d.block = dim3(kGroupThreads);
    d.smem = group_smem(kp, rb, VK);
    d.lpr = lpr;
    return cudaFuncSetAttribute(sweep_group_kernel<XW, LIFO, VK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)d.smem);
}

template <int LIFO, int VK>
static cudaError_t describe_group_l(const KernelParams &kp, int xw, LaunchDesc &d) {
    switch (xw) {
#define VIB_XW(w) \
    case w: return describe_group_t<w, LIFO, VK>(kp, d);
        VIB_XW(1) VIB_XW(2) VIB_XW(3) VIB_XW(4) VIB_XW(5) VIB_XW(6) VIB_XW(7) VIB_XW(8) VIB_XW(9) VIB_XW(10)
        VIB_XW(11) VIB_XW(12) VIB_XW(16) VIB_XW(21) VIB_XW(24)
#undef VIB_XW
        default: return cudaErrorInvalidValue;
    }
}

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

cudaError_t describe_sweep(const KernelParams &kp, int vk, int kahan, int use_group, LaunchDesc &d) {
    d.lpr = 0;
    if (use_group) {
        const int xw = use_group;   // lane width of the factorised kernel
        if (vk == VK_PAIR)
            return kp.issuing ? describe_group_l<1, VK_PAIR>(kp, xw, d) : describe_group_l<0, VK_PAIR>(kp, xw, d);
        return kp.issuing ? describe_group_l<1, VK_SINGLE>(kp, xw, d) : describe_group_l<0, VK_SINGLE>(kp, xw, d);
    }
    if (vk == VK_DOUBLE) return describe_generic_t<VK_DOUBLE, 0>(kp, d);
    if (vk == VK_PAIR) return kahan ? describe_generic_t<VK_PAIR, 1>(kp, d) : describe_generic_t<VK_PAIR, 0>(kp, d);
    return kahan ? describe_generic_t<VK_SINGLE, 1>(kp, d) : describe_generic_t<VK_SINGLE, 0>(kp, d);
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

cudaError_t launch_absdiff(const double *a, const double *b, uint32_t n, SolveState *st, cudaStream_t stream) {
    absdiff_kernel<<<(n + 255) / 256, 256, 0, stream>>>(a, b, n, st);
    return cudaGetLastError();
}

cudaError_t launch_rollouts(const KernelParams &kp, const RollParams &rp, const uint8_t *policy, double *returns,
                            double *kpis, int32_t *traj, cudaStream_t stream) {
    const int threads = 128;
    const int blocks = (rp.n_rollouts + threads - 1) / threads;
    rollout_kernel<<<blocks, threads, 0, stream>>>(kp, rp, policy, returns, kpis, traj);
    return cudaGetLastError();
}

}  // namespace vib

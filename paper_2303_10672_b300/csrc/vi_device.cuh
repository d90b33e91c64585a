// vi_device.cuh -- device helpers shared by the sweep kernels: error-free float
// transformations, block reductions with the last-block finalize of a sweep,
// buffer resolution and the float-pair combinations.
#pragma once

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
        double crit;
        int conv;
        st->iter += 1;
        if (st->stop_rule == kStopPeriodic) {
            // periodic test on Delta_i (Scenario C appendix), from the seventh sweep on
            const double lo = fmin(fabs(vmax), fabs(vmin));
            crit = (vmax - vmin) / lo;
            conv = (st->iter >= 7) && (vmax - vmin <= 2.0 * st->tol * lo);
        } else {
            crit = (st->stop_rule == 0) ? (vmax - vmin) : fmax(fabs(st->dmax_abs), fabs(st->dmin_abs));
            conv = crit < st->tol;
        }
        st->crit = crit;
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
        // the result must end in the caller's buffer: pinned host memory written over
        // the bus while the sweep runs, else buf[0] if the last sweep wrote the scratch
        b.vout = st->vhost ? st->vhost : ((it & 1) ? st->buf[0] : nullptr);
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

// Stage a table blob in shared memory: 16-byte loads, eight in flight per thread
// before any is stored (a plain element loop waits one L2 round trip per element
// at the start of every block), then the elements past the last full 16 bytes.
template <typename T>
__device__ __forceinline__ void load_tables(T *s_tab, const T *g_tab, int n) {
    const int nb = n * (int)sizeof(T);
    int done = 0;   // elements copied by the vector part
    if ((((uintptr_t)g_tab | (uintptr_t)s_tab) & 15) == 0) {
        constexpr int U = 8;
        const int n16 = nb >> 4;
        const uint4 *src = (const uint4 *)g_tab;
        uint4 *dst = (uint4 *)s_tab;
        const int step = (int)blockDim.x;
        int i = (int)threadIdx.x;
        for (; i + (U - 1) * step < n16; i += U * step) {
            uint4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = __ldg(src + i + u * step);
#pragma unroll
            for (int u = 0; u < U; ++u) dst[i + u * step] = v[u];
        }
        for (; i < n16; i += step) dst[i] = __ldg(src + i);
        done = (n16 << 4) / (int)sizeof(T);
    }
    for (int i = done + (int)threadIdx.x; i < n; i += (int)blockDim.x) s_tab[i] = g_tab[i];
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


}  // namespace vib

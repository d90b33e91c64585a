// vi_group.cuh -- the factorised single-product sweep (template), included by
// the per-variant translation units vi_group_*.cu and by vi_batch.cu.
#pragma once

#include <algorithm>

#include "vi_device.cuh"

namespace vib {

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
// Value loads of the body.  A sweep launch reads values that no block of the same
// launch writes, through the read-only path (COH = 0).  The server's persistent
// launch runs many sweeps: a block reads values that other blocks of the same
// launch wrote in the previous sweep, after an acquire fence, so it uses ordinary
// (ld.global.ca, coherent after the fence) loads (COH = 1), written as the load
// intrinsic so that the gathers of a batch are still issued together.
template <int COH, typename T>
__device__ __forceinline__ T vload(const T *p) {
    if constexpr (COH) return __ldca(p);
    else return __ldg(p);
}

template <int XW, int LIFO, int VK, int LPIPE, int COH = 0>
__device__ __forceinline__ void group_body(const KernelParams &kp, uint32_t bid, unsigned n_blocks, int mode,
                                           const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int lpr,
                                           unsigned char *smem_raw) {
    constexpr bool PAIR = (VK == VK_PAIR);
    constexpr int LCH = 8;   // LIFO load batch
    constexpr int LCS = 8;   // load batch of the shared LIFO sequences
    SolveState *st = kp.st;
    // a standalone sweep lets the next sweep launch at its start and stages its tables
    // before it waits for the grids it depends on (a programmatic dependent launch:
    // the set-up overlaps the previous sweep's last blocks; the wait returns at once
    // for an ordinary launch).  Values and the solve state are read after the wait.
    if constexpr (COH == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const ProdParams &P = kp.p[0];
    const int G = P.G;
    const int RB = kGroupThreads / lpr;                    // rests per block
    float *s_tab = (float *)smem_raw;
    // LIFO, L = 1, shared sequences: per-thread column of gamma * C_a, one float per order
    const bool key_lifo = PAIR && LIFO && !LPIPE && lifo_key_ok(P) && lifo_shared_ok(P);
    // FIFO: four copies of the pmf shifted by 0..3, so that every probability window
    // starts on a 16-byte boundary in one of them
    const int pn4 = (P.pn + 3) & ~3;
    float *s_pc = s_tab + ((kp.n_tables + 3) & ~3);
    float *s_kc = s_pc + (LIFO ? 0 : 4 * pn4) + threadIdx.x;
    float *s_out = s_pc + (LIFO ? 0 : 4 * pn4) + (key_lifo ? G * kGroupThreads : 0);   // PAIR: float2 per state
    uint8_t *s_pol = (uint8_t *)(s_out + RB * G * (PAIR ? 2 : 1));
    load_tables<float>(s_tab, (const float *)kp.tables, kp.n_tables);
    const float *s_p = s_tab + P.off_p;
    if (!LIFO) {
        for (int i = threadIdx.x; i < 4 * pn4; i += kGroupThreads) {
            const int o = i / pn4, j = i - o * pn4;
            s_pc[i] = (j + o < P.pn) ? s_p[j + o] : 0.f;
        }
        __syncthreads();
    }
    if constexpr (COH == 0) asm volatile("griddepcontrol.wait;" ::: "memory");
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
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
    const bool shared_lifo = LIFO && !LPIPE && lifo_shared_ok(P);
    const bool shared_fifo = !LIFO && fifo_shared_ok(P);
    constexpr bool rt_common = LPIPE;   // L >= 2: the remaining stock R does not depend on the order
    // per-thread columns (stride kGroupThreads) of the shared LIFO sequences / FIFO path;
    // they share their space with the output staging, which is written after a barrier
    float *colT = s_out + threadIdx.x;
    float *colH = colT + G * kGroupThreads;
    uint32_t *colP = (uint32_t *)colT;
    int Rrest = 0;   // units in the rest slots (without the order when L = 1)
    uint32_t tail_rel = 0;   // L >= 2, shared FIFO path: next-state index after all R units (without the order)

    // best (hi, lo) per x, in pairs of x like the accumulators (packed arithmetic)
    float2 bh2[(XW + 1) / 2], bl2[(XW + 1) / 2];
    auto bhr = [&](int xi) -> float & { return (xi & 1) ? bh2[xi >> 1].y : bh2[xi >> 1].x; };
    auto blr = [&](int xi) -> float & { return (xi & 1) ? bl2[xi >> 1].y : bl2[xi >> 1].x; };
    uint32_t argp[(XW + 3) / 4];   // best order per x, one byte each (G <= 256)
#pragma unroll
    for (int i = 0; i < (XW + 1) / 2; ++i) {
        bh2[i] = make_float2(-INFINITY, -INFINITY);
        bl2[i] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < (XW + 3) / 4; ++i) argp[i] = 0u;
    // keep (h, l, a) as the best of x if `up`: selects, no branch.  Byte xi & 3 of
    // argp[xi >> 2] holds the order.
    auto take = [&](int xi, bool up, float h, float l, int a) {
        constexpr unsigned sel[4] = {0x3214u, 0x3240u, 0x3410u, 0x4210u};
        bhr(xi) = up ? h : bhr(xi);
        if (PAIR) blr(xi) = up ? l : blr(xi);
        const unsigned na = __byte_perm(argp[xi >> 2], (unsigned)a, sel[xi & 3]);
        argp[xi >> 2] = up ? na : argp[xi >> 2];
    };
    float2 R0 = make_float2(0.f, 0.f);
    if (active) {
        const RestInfo ri = decode_rest(r, P);
        Rrest = ri.R;
        const float *V1 = (const float *)B.vin;
        const float2 *V2 = (const float2 *)B.vin;
        if (PAIR) R0 = vload<COH>(V2 + r);   // s'_0 of action 0
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
            if (PAIR && LPIPE) {
                // R does not depend on the order, so neither does the k range of this lane: past
                // its last k the column points at the no-demand state, whose difference is
                // exactly zero, and the chunk loop needs no clamp or mask
                const int kend0 = min(ri.R - 1, dmax - x0);
                if (ri.R <= dmax) tail_rel = cp[ri.R * kGroupThreads];
                for (int k = max(kend0, 0) + 1; k <= max(kend0, 0) + 8; ++k) cp[k * kGroupThreads] = r;
            }
        }
        if (shared_lifo) {
            // LIFO with L = 1 issues the new order first, so every action's next states
            // come from two shared sequences: T[j] = V[r + j G^(K-1)] (part of the order
            // left) and H[k] = V[state r after k units issued LIFO from X_{m-1}..X_2]
            const int nH = min(ri.R, dmax) + 1;
            auto value = [&](uint32_t i) -> float {
                if (PAIR) return pair_diff(vload<COH>(V2 + i), R0);
                return vload<COH>(V1 + i);
            };
            for (int j0 = 0; j0 < G; j0 += LCS) {
                float v[LCS];
#pragma unroll
                for (int j = 0; j < LCS; ++j) v[j] = (j0 + j < G) ? value(r + (uint32_t)(j0 + j) * P.w_top) : 0.f;
#pragma unroll
                for (int j = 0; j < LCS; ++j)
                    if (j0 + j < G) colT[(j0 + j) * kGroupThreads] = v[j];
            }
            Walker wh;
            walker_init(wh, r, ri.packed, P.m - 2, P.cb, 1, P.m >= 3 ? P.w_zt / (uint32_t)G : 1u);
            int kc = 0;
            for (int k0 = 0; k0 < nH; k0 += LCS) {
                uint32_t idx[LCS];
#pragma unroll
                for (int j = 0; j < LCS; ++j) {
                    const int kk = min(k0 + j, nH - 1);
                    for (; kc < kk; ++kc) walker_step(wh, P.cb, 1, (uint32_t)G);
                    idx[j] = wh.idx;
                }
                float v[LCS];
#pragma unroll
                for (int j = 0; j < LCS; ++j) v[j] = value(idx[j]);
#pragma unroll
                for (int j = 0; j < LCS; ++j)
                    if (k0 + j < nH) colH[(k0 + j) * kGroupThreads] = v[j];
            }
        }
        // LIFO, L = 1, shared sequences, one lane covering every x: the expectations of
        // all orders at once, C[a] = sum_{d<=a} p_d T[a-d] + sum_{e>=1} p_{a+e} H[e]
        // + tail[R] g_a(R), summed per order in the same order as the scalar loop
        // below (terms past dmax carry zero mass), so the two agree bit for bit
        const bool vec_lifo = key_lifo && lpr == 1 && Rrest >= 1;
        if (vec_lifo) {
            float T[XW], C[XW];
#pragma unroll
            for (int j = 0; j < XW; ++j) {
                T[j] = (j < G) ? colT[j * kGroupThreads] : 0.f;
                C[j] = 0.f;
            }
#pragma unroll
            for (int d = 0; d < XW; ++d) {
                const float pd = s_p[d];
#pragma unroll
                for (int a = d; a < XW; ++a) C[a] = fmaf(pd, T[a - d], C[a]);
            }
            const int elast = min(Rrest - 1, dmax);
            for (int e = 1; e <= elast; ++e) {
                const float h = colH[e * kGroupThreads];
#pragma unroll
                for (int a = 0; a < XW; ++a) C[a] = fmaf(s_p[a + e], h, C[a]);
            }
            const float hR = (Rrest <= dmax) ? colH[Rrest * kGroupThreads] : 0.f;
            const float *s_tail = s_tab + P.off_tail + Rrest;
#pragma unroll
            for (int a = 0; a < XW; ++a)
                if (Rrest + a <= dmax) C[a] = fmaf(s_tail[a], hR, C[a]);
#pragma unroll
            for (int a = 0; a < XW; ++a) {
                if (a < G) {
                    const float Bh = __fmul_rn(-c_o, (float)a);
                    const float Bl = __fmaf_rn(gam, C[a], 0.f);
                    s_kc[a * kGroupThreads] = Bl;
                    const float ks = __fadd_rn(Bh, Bl);
                    const float *rt = s_RT + (Rrest + a) * G;
#pragma unroll
                    for (int xi = 0; xi < XW; ++xi) {
                        const float key = __fadd_rn(ks, rt[xi]);
                        take(xi, key > bhr(xi), key, 0.f, a);
                    }
                }
            }
        }
        for (int a = 0; a < (vec_lifo ? 0 : G); ++a) {
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
                ref = vload<COH>(V2 + idx0);
            else
                g0 = vload<COH>(V1 + idx0);
            // accumulators in pairs of x, so that the widest FIFO correlations run on
            // packed two-lane FMAs (each lane rounds exactly as fmaf)
            float2 acc2[(XW + 1) / 2];
            auto acc = [&](int xi) -> float & { return (xi & 1) ? acc2[xi >> 1].y : acc2[xi >> 1].x; };
#pragma unroll
            for (int i = 0; i < (XW + 1) / 2; ++i) acc2[i] = make_float2(0.f, 0.f);
            if (!LIFO) {
                // demand k = d - x reaching the other slots; d <= x leaves them untouched:
                //   C(x) = F(x) g(0) + sum_{k=1}^{R-1} p[x+k] g(k) + tail[x+R] g(R)      (R >= 1)
                // A float-pair sweep measures g from ref = g(0), so the first term vanishes.
                // k runs in chunks of KW over a register window of gathered values; the
                // probabilities p[x+k] come from shared memory, and groups of x whose whole
                // chunk lies beyond dmax (zero mass) are skipped.
                constexpr int KW = 8;
                // skip groups of x: more groups skip more zero-mass terms, fewer give the
                // packed loop more independent accumulator pairs per probability (two
                // measured best at 21 x per lane, 0.4% faster than three)
                constexpr int NG = XW >= 16 ? 2 : (XW >= 12 ? 3 : (XW >= 6 ? 2 : 1));
                constexpr int GS = (XW + NG - 1) / NG;
                // 16 or more x per lane: packed FMAs over pairs of x (measured on B300: 1% faster
                // at 21; the narrower lanes have too few independent pairs per skip group and
                // lose).  Pairs per skip group are even, so that each group's probability
                // window starts on a 16-byte boundary (2 q GP floats past the chunk's start).
                constexpr bool PACKED = XW >= 16;
                constexpr int XP = (XW + 1) / 2;
                constexpr int GP = (((XP + NG - 1) / NG) + 1) & ~1;
                constexpr int NGE = (XP + GP - 1) / GP;     // non-empty groups
                constexpr int WQ = (GP + KW / 2) / 2;       // float4 loads per group window
                static_assert(GP % 2 == 0 && 2 * WQ >= GP + KW / 2 - 1, "window layout");
                if (!PAIR) {
                    const float *s_F = s_tab + P.off_F + x0;
#pragma unroll
                    for (int xi = 0; xi < XW; ++xi) acc(xi) = (R == 0) ? g0 : s_F[xi] * g0;
                }
                const uint32_t atop = (uint32_t)a * P.w_top;
                // L >= 2 with the shared path: the tail value's index is known now, so its
                // load is issued before the chunks and is consumed after them (measured on
                // B300: 2% faster at 11 x per lane, 0.5% at 21)
                constexpr bool early_tail = PAIR && LPIPE;
                float2 rawR = make_float2(0.f, 0.f);
                if constexpr (early_tail) {
                    if (shared_fifo && R >= 1 && x0 + R <= dmax) rawR = vload<COH>(V2 + tail_rel + atop);
                }
                int ecur = 0;
                // index of g(e); e never decreases between calls (the walker moves forward)
                auto index_of = [&](int e) -> uint32_t {
                    if (shared_fifo) {
                        // the rest path is shared by all orders; with L = 1 the order is issued last
                        if (LPIPE || e <= Rrest) return colP[e * kGroupThreads] + atop;
                        return (uint32_t)(a - (e - Rrest)) * P.w_top;
                    }
                    for (; ecur < e; ++ecur) walker_step(wk, P.cb, 0, (uint32_t)G);
                    return wk.idx;
                };
                auto value_of = [&](uint32_t i) -> float {
                    if (PAIR) return pair_diff(vload<COH>(V2 + i), ref);
                    return vload<COH>(V1 + i);
                };
                const int kend = min(R - 1, dmax - x0);   // last k carrying mass for some x of this lane
                // window of chunk k0 (k0 = 1 mod 4): p[x0 + k0 + i] = copy_o[x0 + k0 - o + i]
                const int po = (x0 + 1) & 3;
                const float *s_px = s_pc + po * pn4 + (x0 + 1 - po);   // + (k0 - 1) is a multiple of 4
                const int po1 = (x0 + 2) & 3;                          // the window shifted by one
                const float *s_px1 = s_pc + po1 * pn4 + (x0 + 2 - po1);
                constexpr bool preclamped = PAIR && LPIPE;   // with shared_fifo: see the column set-up
                for (int k0 = 1; k0 <= kend; k0 += KW) {
                    uint32_t idx[KW];
                    if (preclamped && shared_fifo) {
#pragma unroll
                        for (int j = 0; j < KW; ++j) idx[j] = colP[(k0 + j) * kGroupThreads] + atop;
                    } else {
#pragma unroll
                        for (int j = 0; j < KW; ++j) idx[j] = index_of(min(k0 + j, kend));
                    }
                    float g[KW];
                    if (PAIR) {
                        float2 raw[KW];
#pragma unroll
                        for (int j = 0; j < KW; ++j) raw[j] = vload<COH>(V2 + idx[j]);
                        if (PACKED && preclamped && shared_fifo) {
                            // (raw - ref) per half as one packed fma(ref, -1, raw), then the
                            // halves added: the same rounding as pair_diff
                            const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
                            for (int j = 0; j < KW; ++j) {
                                const float2 d = __ffma2_rn(ref, m1, raw[j]);
                                g[j] = __fadd_rn(d.x, d.y);
                            }
                        } else if (preclamped && shared_fifo) {
#pragma unroll
                            for (int j = 0; j < KW; ++j) g[j] = pair_diff(raw[j], ref);
                        } else {
#pragma unroll
                            for (int j = 0; j < KW; ++j) g[j] = (k0 + j <= kend) ? pair_diff(raw[j], ref) : 0.f;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < KW; ++j) g[j] = (k0 + j <= kend) ? vload<COH>(V1 + idx[j]) : 0.f;
                    }
                    if constexpr (PACKED) {
#pragma unroll
                        for (int q = 0; q < NGE; ++q) {
                            if (q == 0 || x0 + 2 * q * GP + k0 <= dmax) {
                                // this group's probability pairs (p[x+k0+2t], p[x+k0+2t+1]) and
                                // the same shifted by one (x = x0 + 2 q GP), so that every
                                // (x pair, k) coefficient is one aligned register pair
                                float2 pe[2 * WQ], pod[2 * WQ];
                                const float4 *we = (const float4 *)(s_px + (k0 - 1) + 2 * q * GP);
                                const float4 *wo = (const float4 *)(s_px1 + (k0 - 1) + 2 * q * GP);
#pragma unroll
                                for (int t = 0; t < WQ; ++t) {
                                    const float4 v = we[t], u = wo[t];
                                    pe[2 * t] = make_float2(v.x, v.y);
                                    pe[2 * t + 1] = make_float2(v.z, v.w);
                                    pod[2 * t] = make_float2(u.x, u.y);
                                    pod[2 * t + 1] = make_float2(u.z, u.w);
                                }
#pragma unroll
                                for (int j = 0; j < KW; ++j) {
                                    const float2 gj = make_float2(g[j], g[j]);
#pragma unroll
                                    for (int i = q * GP; i < min(XP, (q + 1) * GP); ++i) {
                                        const int t = i - q * GP + (j >> 1);
                                        acc2[i] = __ffma2_rn((j & 1) ? pod[t] : pe[t], gj, acc2[i]);
                                    }
                                }
                            }
                        }
                    } else {
                        constexpr int NW4 = (XW + KW - 1 + 3) / 4;
                        float pw[4 * NW4];
                        const float4 *pw4 = (const float4 *)(s_px + (k0 - 1));
#pragma unroll
                        for (int t = 0; t < NW4; ++t) {
                            const float4 v = pw4[t];
                            pw[4 * t] = v.x;
                            pw[4 * t + 1] = v.y;
                            pw[4 * t + 2] = v.z;
                            pw[4 * t + 3] = v.w;
                        }
#pragma unroll
                        for (int q = 0; q < NG; ++q) {
                            if (q == 0 || x0 + q * GS + k0 <= dmax) {
#pragma unroll
                                for (int j = 0; j < KW; ++j)
#pragma unroll
                                    for (int xi = q * GS; xi < min(XW, (q + 1) * GS); ++xi)
                                        acc(xi) = fmaf(pw[xi + j], g[j], acc(xi));
                            }
                        }
                    }
                }
                if (R >= 1 && x0 + R <= dmax) {
                    float gR;
                    if constexpr (early_tail)
                        gR = shared_fifo ? pair_diff(rawR, ref) : value_of(index_of(R));
                    else
                        gR = value_of((preclamped && shared_fifo) ? tail_rel + atop : index_of(R));
                    const float *s_tx = s_tab + P.off_tail + x0 + R;
#pragma unroll
                    for (int xi = 0; xi < XW; ++xi) acc(xi) = fmaf(s_tx[xi], gR, acc(xi));
                }
            } else if (shared_lifo) {
                // C_a = sum_{d < R} p_d g_a(d) + tail[R] g_a(R), g_a(e) = T[a-e] while the
                // demand stays within the order (e <= a), H[e-a] beyond it
                float c = 0.f;
                const int dlast = min(R - 1, dmax);
                const int d1 = min(a, dlast);
                const float *pT = colT + a * kGroupThreads;
                for (int d = 0; d <= d1; ++d) c = fmaf(s_p[d], pT[-d * kGroupThreads], c);
                const float *pH = colH - a * kGroupThreads;
                for (int d = a + 1; d <= dlast; ++d) c = fmaf(s_p[d], pH[d * kGroupThreads], c);
                if (R <= dmax) {
                    const float *pR = (R <= a) ? colT + (a - R) * kGroupThreads : colH + (R - a) * kGroupThreads;
                    c = fmaf(s_tab[P.off_tail + R], *pR, c);
                }
#pragma unroll
                for (int xi = 0; xi < XW; ++xi) acc(xi) = c;
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
                        for (int j = 0; j < LCH; ++j) raw[j] = vload<COH>(V2 + idx[j]);
#pragma unroll
                        for (int j = 0; j < LCH; ++j) gv[j] = pair_diff(raw[j], ref);
                    } else {
#pragma unroll
                        for (int j = 0; j < LCH; ++j) gv[j] = vload<COH>(V1 + idx[j]);
                    }
#pragma unroll
                    for (int j = 0; j < LCH; ++j) c = fmaf(s_p[d0 + j], gv[j], c);   // zero mass beyond dmax
                }
#pragma unroll
                for (int xi = 0; xi < XW; ++xi) acc(xi) = c;
            }
            // lanes past the last x (x0 + xi >= G) compute values that are never stored;
            // their table reads stay inside the shared memory that follows the tables
            const float *rt = s_RT + R * G + x0;
            if (PAIR && rt_common && LIFO) {
                // L >= 2 and LIFO: neither the reward (added after the max) nor the
                // expectation depends on x, so one comparison serves every x
                float Bh, Bl;
                action_base(gam, ref, R0, __fmul_rn(-c_o, (float)a), Bh, Bl);
                const float ql = __fmaf_rn(gam, acc(0), Bl);
                const float diff = __fadd_rn(__fsub_rn(Bh, bhr(0)), __fsub_rn(ql, blr(0)));
                take(0, diff > 0.f, Bh, ql, a);
            } else if (PAIR && rt_common) {
                // L >= 2: R does not depend on the order, so RT(x, R) is common to all
                // orders and is added once per x after the max
                float Bh, Bl;
                action_base(gam, ref, R0, __fmul_rn(-c_o, (float)a), Bh, Bl);
                if constexpr (XW >= 16) {
                    // two x per packed instruction; a - b as fma(b, -1, a), rounded as the
                    // subtraction
                    const float2 g2 = make_float2(gam, gam), Bh2 = make_float2(Bh, Bh), Bl2 = make_float2(Bl, Bl);
                    const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
                    for (int i = 0; i < (XW + 1) / 2; ++i) {
                        const float2 ql = __ffma2_rn(g2, acc2[i], Bl2);
                        const float2 diff =
                            __fadd2_rn(__ffma2_rn(bh2[i], m1, Bh2), __ffma2_rn(bl2[i], m1, ql));
                        take(2 * i, diff.x > 0.f, Bh, ql.x, a);
                        if (2 * i + 1 < XW) take(2 * i + 1, diff.y > 0.f, Bh, ql.y, a);
                    }
                } else {
#pragma unroll
                    for (int xi = 0; xi < XW; ++xi) {
                        const float ql = __fmaf_rn(gam, acc(xi), Bl);
                        const float diff = __fadd_rn(__fsub_rn(Bh, bhr(xi)), __fsub_rn(ql, blr(xi)));
                        take(xi, diff > 0.f, Bh, ql, a);
                    }
                }
            } else if (PAIR && LIFO && key_lifo) {
                // L = 1, LIFO, values measured from R0: the base of order a is exactly
                // (-c_o a, gamma C_a).  Compare the single float -c_o a + gamma C_a + RT(x, R);
                // the exact pair of the chosen order is rebuilt after the last order.
                const float Bh = __fmul_rn(-c_o, (float)a);
                const float Bl = __fmaf_rn(gam, acc(0), 0.f);
                s_kc[a * kGroupThreads] = Bl;
                const float ks = __fadd_rn(Bh, Bl);
#pragma unroll
                for (int xi = 0; xi < XW; ++xi) {
                    const float key = __fadd_rn(ks, rt[xi]);
                    take(xi, key > bhr(xi), key, 0.f, a);
                }
            } else if (PAIR) {
                float Bh, Bl;
                action_base(gam, ref, R0, __fmul_rn(-c_o, (float)a), Bh, Bl);
                if (LIFO) Bl = __fmaf_rn(gam, acc(0), Bl);   // the expectation does not depend on x
                const float *rtl = s_RTlo + R * G + x0;
#pragma unroll
                for (int xi = 0; xi < XW; ++xi) {
                    float qh = Bh, ql = Bl;
                    pair_add(qh, ql, rt[xi], rtl[xi]);
                    if (!LIFO) ql = __fmaf_rn(gam, acc(xi), ql);
                    const float diff = __fadd_rn(__fsub_rn(qh, bhr(xi)), __fsub_rn(ql, blr(xi)));
                    take(xi, diff > 0.f, qh, ql, a);
                }
            } else {
                const float base = -c_o * (float)a;
#pragma unroll
                for (int xi = 0; xi < XW; ++xi) {
                    const float q = fmaf(gam, acc(xi), base + rt[xi]);
                    take(xi, q > bhr(xi), q, 0.f, a);
                }
            }
        }
        if (!PAIR && r == 0 && part == 0 && mode == MODE_SWEEP) st->c_next = bhr(0);
    }
    if (PAIR && rt_common && LIFO && active) {
#pragma unroll
        for (int xi = 1; xi < XW; ++xi) {
            bhr(xi) = bhr(0);
            blr(xi) = blr(0);
        }
#pragma unroll
        for (int i = 0; i < (XW + 3) / 4; ++i) argp[i] = (argp[0] & 0xFFu) * 0x01010101u;
    }
    if (key_lifo && active) {
        // the exact pair of each x's chosen order: its base plus RT(x, Rrest + a)
#pragma unroll
        for (int xi = 0; xi < XW; ++xi) {
            const int a = (int)((argp[xi >> 2] >> (8 * (xi & 3))) & 0xFFu);
            float qh = __fmul_rn(-c_o, (float)a), ql = s_kc[a * kGroupThreads];
            const int R = Rrest + a;
            pair_add(qh, ql, s_RT[R * G + x0 + xi], s_RTlo[R * G + x0 + xi]);
            bhr(xi) = qh;
            blr(xi) = ql;
        }
    }
    if (PAIR && rt_common && active) {
        const float *rt = s_RT + Rrest * G + x0;
        const float *rtl = s_RTlo + Rrest * G + x0;
#pragma unroll
        for (int xi = 0; xi < XW; ++xi)
            if (xi < nx) pair_add(bhr(xi), blr(xi), rt[xi], rtl[xi]);
    }
    // stage the block's G * RB contiguous states through shared memory
    if (shared_fifo || shared_lifo) __syncthreads();   // every column is consumed
    if (rl < RB) {
#pragma unroll
        for (int xi = 0; xi < XW; ++xi) {
            if (xi < nx) {
                const int o = rl * G + x0 + xi;
                if (PAIR)
                    ((float2 *)s_out)[o] = active ? pair_finish(gam, R0, bhr(xi), blr(xi)) : make_float2(0.f, 0.f);
                else
                    s_out[o] = bhr(xi);
                s_pol[o] = (uint8_t)(argp[xi >> 2] >> (8 * (xi & 3)));
            }
        }
    }
    __syncthreads();
    const uint32_t s0 = bid * (uint32_t)(RB * G);
    const uint32_t nblk = (uint32_t)(RB * G);
    float mx = -INFINITY, mn = INFINITY;
    if (PAIR && mode != MODE_EXTRACT) {
        // the previous values of WB states are loaded together, so that one load
        // latency serves WB states instead of one
        constexpr int WB = 4;
        const float2 *vin2 = (const float2 *)B.vin;
        float2 *vout2 = (float2 *)B.vout;
        for (uint32_t i0 = threadIdx.x; i0 < nblk; i0 += WB * kGroupThreads) {
            float2 vold[WB];
#pragma unroll
            for (int u = 0; u < WB; ++u) {
                const uint32_t i = i0 + (uint32_t)u * kGroupThreads;
                vold[u] = (i < nblk && s0 + i < P.nS) ? vin2[s0 + i] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < WB; ++u) {
                const uint32_t i = i0 + (uint32_t)u * kGroupThreads;
                if (i < nblk && s0 + i < P.nS) {
                    const float2 vnew = ((const float2 *)s_out)[i];
                    vout2[s0 + i] = vnew;
                    const float dlt = pair_diff(vnew, vold[u]);
                    mx = fmaxf(mx, dlt);
                    mn = fminf(mn, dlt);
                    if (B.pol) B.pol[s0 + i] = s_pol[i];
                }
            }
        }
    }
    for (uint32_t i = threadIdx.x; i < ((PAIR && mode != MODE_EXTRACT) ? 0u : nblk); i += kGroupThreads) {
        const uint32_t s = s0 + i;
        if (s >= P.nS) break;
        if (PAIR) {
            const float2 *vin2 = (const float2 *)B.vin;
            float2 *vout2 = (float2 *)B.vout;
            if (vout2) vout2[s] = vin2[s];   // extraction: only when the result must move
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

// Resident blocks per SM that the register allocation aims for: the register
// estimate grows with the lane width (accumulators, best pair and order per x).
// Measured on B300 for the 21-wide FIFO (L >= 2) and 11-wide LIFO (L = 1)
// kernels: 4 and 8 blocks beat both the compiler's own choice and one block.
__host__ __device__ constexpr int group_min_blocks(int xw, int lifo) {
    const int regs = lifo ? 3 * xw + 31 : 4 * xw + 44;
    const int b = 512 / regs;
    return b < 1 ? 1 : (b > 8 ? 8 : b);
}

template <int XW, int LIFO, int VK, int LPIPE>
__global__ void __launch_bounds__(kGroupThreads, group_min_blocks(XW, LIFO))
sweep_group_kernel(KernelParams kp, int mode, const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int lpr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // blocks start in the order of grp_order (most demand-reaching units first), so
    // that the last wave is made of the lightest blocks
    const uint32_t bid = kp.grp_order ? kp.grp_order[blockIdx.x] : blockIdx.x;
    group_body<XW, LIFO, VK, LPIPE>(kp, bid, gridDim.x, mode, vin_arg, vout_arg, pol_arg, lpr, smem_raw);
}


inline size_t group_smem(const KernelParams &kp, int rb, int vk) {
    const ProdParams &P = kp.p[0];
    const size_t vb = (vk == VK_PAIR) ? 8 : 4;
    size_t work = (size_t)rb * P.G * (vb + 1);   // output staging, shared with the columns
    const size_t keyc =
        (vk == VK_PAIR && kp.issuing && lifo_key_ok(P) && lifo_shared_ok(P)) ? (size_t)P.G * kGroupThreads * 4 : 0;
    if (kp.issuing && lifo_shared_ok(P)) work = std::max(work, (size_t)(P.G + P.dmax + 1) * kGroupThreads * 4);
    if (!kp.issuing && fifo_shared_ok(P)) work = std::max(work, (size_t)(P.dmax + 9) * kGroupThreads * 4);
    const size_t pcopies = kp.issuing ? 0 : (size_t)4 * ((P.pn + 3) & ~3) * 4;
    return (size_t)((kp.n_tables + 3) & ~3) * 4 + pcopies + keyc + work + 16;
}

template <int XW, int LIFO, int VK, int LPIPE>
cudaError_t describe_group_t(const KernelParams &kp, LaunchDesc &d) {
    const int G = kp.p[0].G;
    const int lpr = (G + XW - 1) / XW;
    const int rb = kGroupThreads / lpr;
    const uint32_t nR = kp.p[0].nS / (uint32_t)G;
    d.fn = (const void *)sweep_group_kernel<XW, LIFO, VK, LPIPE>;
    d.grid = dim3((nR + rb - 1) / rb);
    d.block = dim3(kGroupThreads);
    d.smem = group_smem(kp, rb, VK);
    d.lpr = lpr;
    d.pdl = 1;
    return cudaFuncSetAttribute(sweep_group_kernel<XW, LIFO, VK, LPIPE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)d.smem);
}

template <int LIFO, int VK, int LPIPE>
cudaError_t describe_group_l(const KernelParams &kp, int xw, LaunchDesc &d) {
    switch (xw) {
#define VIB_XW(w) \
    case w: return describe_group_t<w, LIFO, VK, LPIPE>(kp, d);
        VIB_XW(1) VIB_XW(2) VIB_XW(3) VIB_XW(4) VIB_XW(5) VIB_XW(6) VIB_XW(7) VIB_XW(8) VIB_XW(9) VIB_XW(10)
        VIB_XW(11) VIB_XW(12) VIB_XW(16) VIB_XW(21) VIB_XW(24)
#undef VIB_XW
        default: return cudaErrorInvalidValue;
    }
}


}  // namespace vib

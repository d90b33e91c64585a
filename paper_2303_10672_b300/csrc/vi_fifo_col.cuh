// vi_fifo_col.cuh -- FIFO sweep, one column of rests at a time (the body, included
// by vi_fifo_col.cu and, for lead times of two or more, by the server kernel in
// vi_batch.cu).
//
// Under FIFO (Eq. demoor:fifo) the expiring slot x is issued first and the oldest
// rest slot Z_1 (the lowest digit of the rest r) next.  With lead time L >= 2 the
// order only sets the top digit of the next state, so the next state after e units
// reached the rest is n_r(e) + a G^(K-1), where n_r is the rest's FIFO path, which
// stops moving at e = R (all R units of the rest gone).  Measured from the
// no-demand next state ref(r, a) = V[r + a G^(K-1)], the expectation of order a at
// x is
//   C(x, r, a) = sum_d p_d (V[n_r(min((d - x)^+, R)) + a G^(K-1)] - ref(r, a)).
// One unit more in Z_1 is the first unit to go, so n_{r+1}(e + 1) = n_r(e), and
//   C(x, r + 1, a) = C(x + 1, r, a) - P(D > x) (ref(r + 1, a) - ref(r, a)).
// The rests r0 + z (z = 0..Q) that differ only in Z_1 form a column: their
// expectations follow from those of r0 (Z_1 = 0) at x' = 0..2Q by one multiply-add
// per (x, z, a), in place of a sum over the demand.  At r0,
//   C(x', r0, a) = sum_{k >= 1} p[x' + k] g(min(k, R0)),
// g(k) the value after k units measured from ref(r0, a) (the tail mass beyond the
// rest is the pmf's own terms past R0), and C vanishes from x' = dmax on.
// With lead time one the order a arrives as the freshest stock slot, the last one
// issued: its digit of weight G^(K-1) holds what is left of it, the path runs on
// through those a units (R0 + a in place of R0), and the recurrence is unchanged
// because Z_1 is still the first slot after x; the reward-table row is R + a.
//
// One warp per column.  Lane a holds order a's C(., z, a) in registers (x'
// unrolled; the pmf and -P(D > x) come from the parameter constant bank), forms
// the order's float key gamma C + (gamma (ref - R0) - c_o a) for each x and writes
// the keys and C to shared memory.  Lane x then takes the first argmax over the
// orders of its x and rebuilds the chosen order's value exactly in float pairs:
// the base pair gamma (ref - R0) - c_o a, plus gamma C, plus the reward-table pair
// RT(R, x), plus gamma R0 (the operations of the factorised sweep).  With lead time
// one the key also holds RT(R + a, x), which then differs between orders.
#pragma once

#include <cuda_runtime.h>

#include "vi_device.cuh"

namespace vib {

constexpr int kColWarps = 4;    // columns per block (one per warp)
constexpr int kColRow = 36;     // floats per order row of the transposition buffers: 16-byte rows whose
                                // 128-bit stores from eight consecutive lanes fall in distinct banks

// pmf capacity of the instantiation serving dmax (dmax <= DP - 2, so C(DP - 2) = 0)
__host__ __device__ constexpr int fifo_col_dp(int dmax) {
    return dmax <= 14 ? 16 : (dmax <= 30 ? 32 : (dmax <= 46 ? 48 : 64));
}

// shared memory of one block of the body
struct ColSmem {
    float key[kColWarps][32 * kColRow];   // [order][x] keys of one rest
    float cv[kColWarps][32 * kColRow];    // [order][x] expectations C
    float2 base[kColWarps][32];           // base pair of each order
};

// Value loads.  A standalone sweep reads values that no block of the same launch
// writes, through the read-only path (COH = 0); the server's persistent launch reads
// values other blocks of the launch wrote in the previous sweep, after an acquire
// fence, through ordinary loads (COH = 1).
template <int COH>
__device__ __forceinline__ float2 col_load(const float2 *p) {
    if constexpr (COH) return __ldca(p);
    else return __ldg(p);
}

// Block `bid` of a sweep of n_blocks blocks (kColWarps columns, one per warp; all
// threads of the block call it).  kp may live in shared memory (the server).
// LT1 = 1: lead time one.  The order then arrives as the freshest stock slot, issued
// after the rest's units (its next-state digit, of weight G^(K-1), counts the units
// left of it), so each order's path continues past the rest's units into its own, and
// the reward table's R counts the order: RT(R + a, x) enters each order's key.
template <int DP, int COH, int LT1>
__device__ __forceinline__ void fifo_col_body(const KernelParams &kp, uint32_t bid, unsigned n_blocks, int mode,
                                              const void *vin_arg, void *vout_arg, uint8_t *pol_arg, ColSmem &sm) {
    constexpr int XE = DP - 1;   // C(x') kept for x' = 0..DP-2; zero from dmax on
    SolveState *st = kp.st;
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    const ProdParams &P = kp.p[0];
    const int G = P.G;
    const int dmax = P.dmax;
    const uint32_t nR = P.nS / (uint32_t)G;
    const uint32_t ncol = nR / (uint32_t)G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t col = bid * (uint32_t)kColWarps + (uint32_t)warp;
    float mx = -INFINITY, mn = INFINITY;
    if (col < ncol) {   // uniform across the warp
        const float gam = (float)kp.gamma;
        const float c_o = (float)P.c_o;
        const float2 *V2 = (const float2 *)B.vin;
        const float *tab = (const float *)kp.tables;
        const uint32_t r0 = col * (uint32_t)G;   // the column's rest with Z_1 = 0
        const int nz = P.n_rest_slots;            // stock slots of the rest: Z_1 .. Z_{m-1} (m-2 if LT1)
        // units of the column in Z_2 .. Z_{nz}
        int Rc = 0;
        {
            uint32_t q = col;
            for (int j = 1; j < nz; ++j) {
                const uint32_t q2 = DivG::q(q, (uint32_t)G, &P);
                Rc += (int)(q - q2 * (uint32_t)G);
                q = q2;
            }
        }
        // n_{r0}(k): k units taken oldest first from Z_2 (weight G) upward; past the
        // column's units it stays at the emptied rest
        auto path_at = [&](int k) -> uint32_t {
            uint32_t idx = r0, w = (uint32_t)G, q = col;
            int rem = k;
            for (int j = 1; j < nz && rem > 0; ++j) {
                const uint32_t q2 = DivG::q(q, (uint32_t)G, &P);
                const int t = min(rem, (int)(q - q2 * (uint32_t)G));
                idx -= (uint32_t)t * w;
                rem -= t;
                w *= (uint32_t)G;
                q = q2;
            }
            return idx;
        };
        const uint32_t pa = path_at(lane);                      // k = lane
        const uint32_t pb = (DP > 32) ? path_at(lane + 32) : 0u;  // k = lane + 32
        const int a = lane < G ? lane : 0;   // lanes past the last order repeat order 0 (never read)
        const float2 *Va = V2 + (size_t)a * P.w_top;
        const float2 ref0 = col_load<COH>(Va + r0);
        // units of the order left after k units reached the rest: all of them with a
        // pipeline (the order is not stock yet), else what the rest's Rc units left over
        auto order_left = [&](int k) -> uint32_t { return LT1 ? (uint32_t)max(a - max(k - Rc, 0), 0) : (uint32_t)a; };

        // -- C(x', r0, a) for x' = 0..DP-2, terms in increasing k (zero mass past dmax)
        float C[XE];
#pragma unroll
        for (int i = 0; i < XE; ++i) C[i] = 0.f;
#pragma unroll
        for (int k0 = 1; k0 < DP; k0 += 8) {
            if (k0 <= dmax) {   // uniform
                float2 raw[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int k = k0 + j;
                    if (k < DP) {
                        const uint32_t idx =
                            (k < 32) ? __shfl_sync(0xffffffffu, pa, k) : __shfl_sync(0xffffffffu, pb, k - 32);
                        raw[j] = col_load<COH>(V2 + (idx + order_left(k) * P.w_top));
                    }
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int k = k0 + j;
                    if (k < DP && k <= dmax) {
                        const float g = pair_diff(raw[j], ref0);
#pragma unroll
                        for (int x = 0; x < XE; ++x)   // constant trip count: every index of C is a constant
                            if (x + k < DP && (x & ~7) + k <= dmax)
                                C[x] = __fmaf_rn(kp.pmf32[min(x + k, DP - 1)], g, C[x]);
                    }
                }
            }
        }

        // -- the column's rests r0 + z, z = 0..Q
        float *krow = sm.key[warp] + lane * kColRow;
        float *crow = sm.cv[warp] + lane * kColRow;
        const int x = lane;   // the first argmax and the rebuild: one expiring-slot value per lane
        float2 *vout2 = (float2 *)B.vout;
        float2 refp = ref0, refz = ref0;          // ref(r0 + z - 1, a), ref(r0 + z, a)
        float2 R0z = col_load<COH>(V2 + r0);              // ref(r0 + z, 0)
        for (int z = 0; z < G; ++z) {
            // the next rest's references, one level ahead
            float2 refn = refz, R0n = R0z;
            if (z + 1 < G) {
                refn = col_load<COH>(Va + r0 + (uint32_t)(z + 1));
                R0n = col_load<COH>(V2 + r0 + (uint32_t)(z + 1));
            }
            // this lane's state, its previous value and its reward-table pair
            const uint32_t s = (r0 + (uint32_t)z) * (uint32_t)G + (uint32_t)x;
            float2 vold = make_float2(0.f, 0.f);
            float rth = 0.f, rtl = 0.f;
            if (x < G) {
                vold = col_load<COH>(V2 + s);
                if (!LT1) {   // with a pipeline the reward row does not depend on the order
                    const int ti = (Rc + z) * G + x;
                    rth = __ldg(tab + P.off_RT + ti);
                    rtl = __ldg(tab + P.off_RTlo + ti);
                }
            }
            if (z > 0) {
                // C(x, r0 + z) = C(x + 1, r0 + z - 1) - P(D > x) (ref(r0 + z) - ref(r0 + z - 1)),
                // for the x' still needed by this rest and the ones after it (x' <= 2Q - z)
                const float dl = pair_diff(refz, refp);
                const int xlim = min(dmax - 1, 2 * (G - 1) - z);
#pragma unroll
                for (int xx = 0; xx + 1 < XE; ++xx)
                    if ((xx & ~7) <= xlim) C[xx] = __fmaf_rn(kp.nsurv32[xx], dl, C[xx + 1]);
            }
            // the order's base pair gamma (ref - R0) - c_o a and its keys per x
            float Bh, Bl;
            action_base(gam, refz, R0z, __fmul_rn(-c_o, (float)a), Bh, Bl);
            const float kb = __fadd_rn(Bh, Bl);
            const float *rtk = tab + P.off_RT + (Rc + z + a) * G;   // LT1: this order's reward row
#pragma unroll
            for (int x4 = 0; x4 < 32; x4 += 4) {
                if (x4 < G) {   // uniform
                    float cv[4], kv[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        cv[i] = (x4 + i < XE) ? C[x4 + i] : 0.f;
                        kv[i] = __fmaf_rn(gam, cv[i], kb);
                        if (LT1) kv[i] = __fadd_rn(kv[i], (x4 + i < G) ? __ldg(rtk + x4 + i) : 0.f);
                    }
                    *(float4 *)(krow + x4) = make_float4(kv[0], kv[1], kv[2], kv[3]);
                    *(float4 *)(crow + x4) = make_float4(cv[0], cv[1], cv[2], cv[3]);
                }
            }
            sm.base[warp][lane] = make_float2(Bh, Bl);
            __syncwarp();
            if (x < G) {
                // first argmax over the orders of this x: even and odd orders in two
                // independent compare-select chains (each keeps its first maximum), then
                // the larger key, the smaller order on a tie (measured on B300: config 2
                // 0.129 -> 0.120 ms per sweep against one chain, results bit-identical)
                const float *kc = sm.key[warp] + x;
                float b0 = kc[0], b1 = -INFINITY;
                int a0 = 0, a1 = 1;
#pragma unroll 4
                for (int a2 = 1; a2 < G; a2 += 2) {
                    const float k1 = kc[a2 * kColRow];
                    const bool u1 = k1 > b1;
                    b1 = u1 ? k1 : b1;
                    a1 = u1 ? a2 : a1;
                    if (a2 + 1 < G) {
                        const float k0 = kc[(a2 + 1) * kColRow];
                        const bool u0 = k0 > b0;
                        b0 = u0 ? k0 : b0;
                        a0 = u0 ? a2 + 1 : a0;
                    }
                }
                const int ab = (b1 > b0 || (b1 == b0 && a1 < a0)) ? a1 : a0;
                // the chosen order's exact pair
                const float cbest = sm.cv[warp][ab * kColRow + x];
                const float2 bb = sm.base[warp][ab];
                if (LT1) {
                    const int ti = (Rc + z + ab) * G + x;
                    rth = __ldg(tab + P.off_RT + ti);
                    rtl = __ldg(tab + P.off_RTlo + ti);
                }
                float bh = bb.x, bl = __fmaf_rn(gam, cbest, bb.y);
                pair_add(bh, bl, rth, rtl);
                const float2 vnew = pair_finish(gam, R0z, bh, bl);
                if (mode != MODE_EXTRACT) {
                    vout2[s] = vnew;
                    const float dlt = pair_diff(vnew, vold);
                    mx = fmaxf(mx, dlt);
                    mn = fminf(mn, dlt);
                } else if (vout2) {
                    vout2[s] = vold;   // extraction: the values move unchanged
                }
                if (B.pol) B.pol[s] = (uint8_t)ab;
            }
            __syncwarp();   // the buffers are read before the next rest overwrites them
            refp = refz;
            refz = refn;
            R0z = R0n;
        }
    }
    if (mode != MODE_EXTRACT) block_reduce_and_finalize<float>(mx, mn, st, mode, n_blocks);
}

}  // namespace vib

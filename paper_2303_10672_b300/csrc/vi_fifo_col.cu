// vi_fifo_col.cu -- FIFO sweep for lead times of two or more, one column of rests
// at a time.
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
//
// One warp per column.  Lane a holds order a's C(., z, a) in registers (x'
// unrolled; the pmf and -P(D > x) come from the parameter constant bank), forms
// the order's float key gamma C + (gamma (ref - R0) - c_o a) for each x and writes
// the keys and C to shared memory.  Lane x then takes the first argmax over the
// orders of its x and rebuilds the chosen order's value exactly in float pairs:
// the base pair gamma (ref - R0) - c_o a, plus gamma C, plus the reward-table pair
// RT(R, x), plus gamma R0 (the operations of the factorised sweep).
#include <cuda_runtime.h>

#include <algorithm>

#include "vi_device.cuh"

namespace vib {

constexpr int kColWarps = 4;    // columns per block (one per warp)
constexpr int kColRow = 36;     // floats per order row of the transposition buffers: 16-byte rows whose
                                // 128-bit stores from eight consecutive lanes fall in distinct banks

// pmf capacity of the instantiation serving dmax (dmax <= DP - 2, so C(DP - 2) = 0)
__host__ __device__ constexpr int fifo_col_dp(int dmax) {
    return dmax <= 14 ? 16 : (dmax <= 30 ? 32 : (dmax <= 46 ? 48 : 64));
}

template <int DP>
__global__ void __launch_bounds__(kColWarps * 32)
sweep_fifo_col_kernel(KernelParams kp, int mode, const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int lpr) {
    constexpr int XE = DP - 1;   // C(x') kept for x' = 0..DP-2; zero from dmax on
    __shared__ __align__(16) float s_key[kColWarps][32 * kColRow];   // [order][x] keys of one level
    __shared__ __align__(16) float s_cv[kColWarps][32 * kColRow];    // [order][x] expectations C
    __shared__ float2 s_base[kColWarps][32];                         // base pair of each order
    // the next sweep may launch while this one runs; values and the solve state are
    // read only after the grids this launch depends on have completed
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    SolveState *st = kp.st;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    const ProdParams &P = kp.p[0];
    const int G = P.G;
    const int dmax = P.dmax;
    const uint32_t nR = P.nS / (uint32_t)G;
    const uint32_t ncol = nR / (uint32_t)G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t col = blockIdx.x * (uint32_t)kColWarps + (uint32_t)warp;
    float mx = -INFINITY, mn = INFINITY;
    if (col < ncol) {   // uniform across the warp
        const float gam = (float)kp.gamma;
        const float c_o = (float)P.c_o;
        const float2 *V2 = (const float2 *)B.vin;
        const float *tab = (const float *)kp.tables;
        const uint32_t r0 = col * (uint32_t)G;   // the column's rest with Z_1 = 0
        const int nz = P.n_rest_slots;            // stock slots of the rest: Z_1 .. Z_{m-1}
        // units of the column in Z_2 .. Z_{m-1}
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
        const float2 ref0 = __ldg(Va + r0);

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
                        raw[j] = __ldg(Va + idx);
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
        float *krow = s_key[warp] + lane * kColRow;
        float *crow = s_cv[warp] + lane * kColRow;
        const int x = lane;   // the first argmax and the rebuild: one expiring-slot value per lane
        float2 *vout2 = (float2 *)B.vout;
        float2 refp = ref0, refz = ref0;          // ref(r0 + z - 1, a), ref(r0 + z, a)
        float2 R0z = __ldg(V2 + r0);              // ref(r0 + z, 0)
        for (int z = 0; z < G; ++z) {
            // the next rest's references, one level ahead
            float2 refn = refz, R0n = R0z;
            if (z + 1 < G) {
                refn = __ldg(Va + r0 + (uint32_t)(z + 1));
                R0n = __ldg(V2 + r0 + (uint32_t)(z + 1));
            }
            // this lane's state, its previous value and its reward-table pair
            const uint32_t s = (r0 + (uint32_t)z) * (uint32_t)G + (uint32_t)x;
            float2 vold = make_float2(0.f, 0.f);
            float rth = 0.f, rtl = 0.f;
            if (x < G) {
                const int ti = (Rc + z) * G + x;
                vold = __ldg(V2 + s);
                rth = __ldg(tab + P.off_RT + ti);
                rtl = __ldg(tab + P.off_RTlo + ti);
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
#pragma unroll
            for (int x4 = 0; x4 < 32; x4 += 4) {
                if (x4 < G) {   // uniform
                    float cv[4], kv[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        cv[i] = (x4 + i < XE) ? C[x4 + i] : 0.f;
                        kv[i] = __fmaf_rn(gam, cv[i], kb);
                    }
                    *(float4 *)(krow + x4) = make_float4(kv[0], kv[1], kv[2], kv[3]);
                    *(float4 *)(crow + x4) = make_float4(cv[0], cv[1], cv[2], cv[3]);
                }
            }
            s_base[warp][lane] = make_float2(Bh, Bl);
            __syncwarp();
            if (x < G) {
                // first argmax over the orders of this x
                const float *kc = s_key[warp] + x;
                float best = kc[0];
                int ab = 0;
#pragma unroll 4
                for (int a2 = 1; a2 < G; ++a2) {
                    const float kk = kc[a2 * kColRow];
                    const bool up = kk > best;
                    best = up ? kk : best;
                    ab = up ? a2 : ab;
                }
                // the chosen order's exact pair
                const float cbest = s_cv[warp][ab * kColRow + x];
                const float2 bb = s_base[warp][ab];
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
    if (mode != MODE_EXTRACT) block_reduce_and_finalize<float>(mx, mn, st, mode, gridDim.x);
}

// one product, float-pair values, FIFO, lead time two or more, a stock slot in the
// rest (m >= 2), 2 <= Q+1 <= 32 and dmax <= 62
bool fifo_col_supported(const KernelParams &kp, int vk, int kahan) {
    const ProdParams &P = kp.p[0];
    return kp.n_products == 1 && vk == VK_PAIR && !kahan && kp.issuing == 0 && P.L >= 2 && P.m >= 2 && P.G >= 2 &&
           P.G <= 32 && P.dmax <= 62 && !kp.pc && P.n_rest_slots >= 1;
}

template <int DP>
static cudaError_t describe_fifo_col_t(const KernelParams &kp, LaunchDesc &d) {
    const ProdParams &P = kp.p[0];
    const uint32_t ncol = P.nS / (uint32_t)P.G / (uint32_t)P.G;
    d.fn = (const void *)sweep_fifo_col_kernel<DP>;
    d.grid = dim3((ncol + kColWarps - 1) / kColWarps);
    d.block = dim3(kColWarps * 32);
    d.smem = 0;
    d.lpr = 1;
    d.pdl = 1;
    d.n_pre = 0;
    return cudaSuccess;
}

cudaError_t describe_fifo_col(const KernelParams &kp, LaunchDesc &d) {
    switch (fifo_col_dp(kp.p[0].dmax)) {
        case 16: return describe_fifo_col_t<16>(kp, d);
        case 32: return describe_fifo_col_t<32>(kp, d);
        case 48: return describe_fifo_col_t<48>(kp, d);
        default: return describe_fifo_col_t<64>(kp, d);
    }
}

}  // namespace vib

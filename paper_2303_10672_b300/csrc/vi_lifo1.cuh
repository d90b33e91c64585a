// vi_lifo1.cuh -- persistent factorised sweep for LIFO issuing with lead time one
// (template), included by vi_lifo1_d16.cu and vi_lifo1_d32.cu.
//
// With L = 1 the order a arrives as the freshest slot and, under LIFO
// (Eq. demoor:lifo), is issued first; the expiring slot x = X_1 is issued last
// and never survives into the next state.  For a rest r = (X_2, .., X_{m-1})
// every next state therefore lies on one of two sequences shared by all orders
// and all x:
//   T[j] = V[r + j G^(m-2)]          the order not yet used up (j units left),
//   H[k] = V[r after k units issued]  the order used up, k units taken from
//                                     X_{m-1} down to X_2 (freshest first),
// and with the float-pair frame (values measured from R0 = V[r] = T[0] = H[0]):
//   C_a = sum_d p_d g_a(min(d, a + R)),  g_a(e) = T[a-e] (e <= a), H[e-a] (e > a)
//       = sum_{d<a} p_d T[a-d] + sum_{k>=1} p_{a+k} H~[k],   H~[k] = H[min(k, R)],
// R = units of the rest.  (The d = a term is p_a T[0] = 0; p is zero past dmax.)
// Then Q(s, a) = gamma R0 + (-c_o a + gamma C_a + RT(R + a, x)) (Eq.
// valueiterationdetupdate with the expected-reward table RT), and the first
// argmax over orders is taken per x.
//
// G = Q+1 and the pmf capacity DP (> dmax) are compile-time, so the gathers, the
// convolution and the max over (x, a) are fully unrolled without per-thread
// bounds.  One thread owns one rest (its G states); a block holds kL1Threads
// rests and walks the grid's tiles (persistent blocks, one expected-reward table
// staged per block).  The block's G kL1Threads new values go out through
// shared memory in 16-byte pieces, together with the change statistics.
#pragma once

#include <algorithm>

#include "vi_device.cuh"

namespace vib {

constexpr int kL1Threads = 128;

// bits per packed slot count for a radix G (ceil(log2 G))
__host__ __device__ constexpr int l1_bits(int G) { return G <= 2 ? 1 : (G <= 4 ? 2 : (G <= 8 ? 3 : (G <= 16 ? 4 : 5))); }

// shared memory of one block, in bytes
__host__ __device__ inline size_t lifo1_smem(int G, int DP, int rt_rows) {
    const int GP = (G + 3) & ~3;
    return (size_t)4 * (2 * rt_rows * GP + DP + G * kL1Threads) + (size_t)8 * G * kL1Threads +
           (size_t)G * kL1Threads + 16;
}

// resident blocks per SM the register allocation aims for: four (128 registers)
// with a 16-entry pmf, two with a 32-entry one (its gathered columns double)
__host__ __device__ constexpr int lifo1_min_blocks(int DP) { return DP <= 16 ? 4 : 2; }

template <int G, int DP>
__global__ void __launch_bounds__(kL1Threads, lifo1_min_blocks(DP))
sweep_lifo1_kernel(KernelParams kp, int mode, const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int lpr) {
    constexpr int GP = (G + 3) & ~3;   // RT rows padded to whole float4s
    constexpr int CB = l1_bits(G);
    constexpr int NT = kL1Threads;
    static_assert(G >= 2 && G <= 16 && DP >= G && DP % 4 == 0, "lifo1 geometry");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SolveState *st = kp.st;
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    const ProdParams &P = kp.p[0];
    const int rows = P.rt_rows;
    float *s_RTh = (float *)smem_raw;               // RT(R, x), row R padded to GP
    float *s_RTl = s_RTh + rows * GP;               // its low half
    float *s_p = s_RTl + rows * GP;                 // pmf, zero past dmax (DP entries)
    float *s_kc = s_p + DP;                         // per-thread columns: gamma C_a
    float2 *s_out = (float2 *)(s_kc + G * NT);      // new values of the tile's states
    uint8_t *s_pol = (uint8_t *)(s_out + G * NT);   // and their first argmax
    {
        const float *tab = (const float *)kp.tables;
        for (int i = threadIdx.x; i < rows * GP; i += NT) {
            const int R = i / GP, x = i - R * GP;
            s_RTh[i] = (x < G) ? tab[P.off_RT + R * G + x] : 0.f;
            s_RTl[i] = (x < G) ? tab[P.off_RTlo + R * G + x] : 0.f;
        }
        for (int i = threadIdx.x; i < DP; i += NT) s_p[i] = (i <= P.dmax) ? tab[P.off_p + i] : 0.f;
    }
    __syncthreads();
    float p[DP];
#pragma unroll
    for (int d = 0; d < DP; ++d) p[d] = s_p[d];

    const uint32_t nR = P.nS / (uint32_t)G;
    const uint32_t ntiles = (nR + NT - 1) / NT;
    const int nrs = P.n_rest_slots;                  // m - 2 rest slots: X_2 .. X_{m-1}
    const uint32_t w_top = P.w_top;                  // G^(m-2): weight of the order's next-state slot
    const int dmax = P.dmax;
    const float gam = (float)kp.gamma;
    const float c_o = (float)P.c_o;
    const float2 *V2 = (const float2 *)B.vin;
    float mx = -INFINITY, mn = INFINITY;
    const int tid = threadIdx.x;
    float *kc_col = s_kc + tid;

    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t r = tile * NT + (uint32_t)tid;
        if (r < nR) {
            // -- decode the rest: digit j of r is X_{j+2}
            unsigned long long packed = 0ull;
            int Rrest = 0;
            {
                uint32_t rem = r;
                for (int j = 0; j < nrs; ++j) {
                    const uint32_t q = rem / (uint32_t)G;
                    const int dg = (int)(rem - q * (uint32_t)G);
                    rem = q;
                    packed |= (unsigned long long)dg << (CB * j);
                    Rrest += dg;
                }
            }
            // -- next-state indices of the used-up-order sequence: LIFO from X_{m-1} down
            const int hcount = min(Rrest, dmax);
            uint32_t hidx[DP];
            {
                int slot = nrs - 1;
                uint32_t w = (nrs > 0) ? w_top / (uint32_t)G : 0u;
                int left = (nrs > 0) ? (int)((packed >> (CB * slot)) & ((1ull << CB) - 1ull)) : 0;
                uint32_t idx = r;
                hidx[0] = r;
#pragma unroll
                for (int k = 1; k < DP; ++k) {
                    if (k <= hcount) {
                        // k <= R: a non-empty slot remains below; the bound only guards the loop
                        while (left == 0 && slot > 0) {
                            --slot;
                            w /= (uint32_t)G;
                            left = (int)((packed >> (CB * slot)) & ((1ull << CB) - 1ull));
                        }
                        idx -= w;
                        --left;
                    }
                    hidx[k] = idx;
                }
            }
            // -- gathers: every load of the rest is issued before any is used
            const float2 R0 = __ldg(V2 + r);
            float2 traw[G];
            traw[0] = R0;
#pragma unroll
            for (int j = 1; j < G; ++j) traw[j] = __ldg(V2 + r + (uint32_t)j * w_top);
            float2 hraw[DP];
            hraw[0] = R0;
#pragma unroll
            for (int k = 1; k < DP; ++k) hraw[k] = (k <= hcount) ? __ldg(V2 + hidx[k]) : make_float2(0.f, 0.f);
            float T[G], H[DP];
            T[0] = 0.f;
            H[0] = 0.f;
#pragma unroll
            for (int j = 1; j < G; ++j) T[j] = pair_diff(traw[j], R0);
#pragma unroll
            for (int k = 1; k < DP; ++k) H[k] = (k <= hcount) ? pair_diff(hraw[k], R0) : H[k - 1];

            // -- expectations of every order: C_a = sum_{d<a} p_d T[a-d] + sum_{k>=1} p_{a+k} H~[k]
            float C[G];
#pragma unroll
            for (int a = 0; a < G; ++a) {
                float c = 0.f;
#pragma unroll
                for (int d = 0; d < a; ++d) c = fmaf(p[d], T[a - d], c);
#pragma unroll
                for (int k = 1; a + k < DP; ++k) c = fmaf(p[a + k], H[k], c);
                C[a] = c;
            }
            // -- first argmax over orders per x on the float key -c_o a + gamma C_a + RT(R + a, x)
            float best[G];
            int arg[G];
#pragma unroll
            for (int a = 0; a < G; ++a) {
                const float bl = __fmul_rn(gam, C[a]);
                kc_col[a * NT] = bl;
                const float ks = __fadd_rn(__fmul_rn(-c_o, (float)a), bl);
                const float4 *row = (const float4 *)(s_RTh + (Rrest + a) * GP);
                float rt[GP];
#pragma unroll
                for (int q = 0; q < GP / 4; ++q) {
                    const float4 v = row[q];
                    rt[4 * q] = v.x;
                    rt[4 * q + 1] = v.y;
                    rt[4 * q + 2] = v.z;
                    rt[4 * q + 3] = v.w;
                }
#pragma unroll
                for (int x = 0; x < G; ++x) {
                    const float key = __fadd_rn(ks, rt[x]);
                    if (a == 0) {
                        best[x] = key;
                        arg[x] = 0;
                    } else {
                        const bool up = key > best[x];
                        best[x] = up ? key : best[x];
                        arg[x] = up ? a : arg[x];
                    }
                }
            }
            // -- the exact pair of each x's chosen order: gamma R0 + (-c_o a) + gamma C_a + RT
            float ph, pe;
            two_prod(gam, R0.x, ph, pe);
            const float pl = __fmaf_rn(gam, R0.y, pe);
            float2 *o = s_out + tid * G;
            uint8_t *op = s_pol + tid * G;
#pragma unroll
            for (int x = 0; x < G; ++x) {
                const int a = arg[x];
                const int R = Rrest + a;
                float qh = __fmul_rn(-c_o, (float)a), ql = kc_col[a * NT];
                pair_add(qh, ql, s_RTh[R * GP + x], s_RTl[R * GP + x]);
                float sh, se;
                two_sum(ph, qh, sh, se);
                const float lo = __fadd_rn(se, __fadd_rn(pl, ql));
                float vh, vl;
                fast_two_sum(sh, lo, vh, vl);
                o[x] = make_float2(vh, vl);
                op[x] = (uint8_t)a;
            }
        }
        __syncthreads();
        // -- the tile's states leave in 16-byte pieces (two states), with the change statistics
        const uint32_t s0 = tile * (uint32_t)(NT * G);
        const uint32_t nblk = min((uint32_t)(NT * G), P.nS - s0);
        const float4 *vin4 = (const float4 *)((const float2 *)B.vin + s0);   // s0 is even: 16-byte aligned
        const float4 *out4 = (const float4 *)s_out;
        const uint32_t n2 = nblk >> 1;
        if (mode != MODE_EXTRACT) {
            float4 *vout4 = (float4 *)((float2 *)B.vout + s0);
            constexpr int WB = 3;   // loads of the previous values in flight per thread
            for (uint32_t i0 = tid; i0 < n2; i0 += WB * NT) {
                float4 vold[WB];
#pragma unroll
                for (int u = 0; u < WB; ++u) {
                    const uint32_t i = i0 + (uint32_t)u * NT;
                    vold[u] = (i < n2) ? vin4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < WB; ++u) {
                    const uint32_t i = i0 + (uint32_t)u * NT;
                    if (i < n2) {
                        const float4 vn = out4[i];
                        vout4[i] = vn;
                        const float d0 = pair_diff(make_float2(vn.x, vn.y), make_float2(vold[u].x, vold[u].y));
                        const float d1 = pair_diff(make_float2(vn.z, vn.w), make_float2(vold[u].z, vold[u].w));
                        mx = fmaxf(mx, fmaxf(d0, d1));
                        mn = fminf(mn, fminf(d0, d1));
                    }
                }
            }
            if ((nblk & 1u) && tid == 0) {
                const uint32_t i = nblk - 1;
                const float2 vn = s_out[i];
                const float2 vo = ((const float2 *)B.vin)[s0 + i];
                ((float2 *)B.vout)[s0 + i] = vn;
                const float dl = pair_diff(vn, vo);
                mx = fmaxf(mx, dl);
                mn = fminf(mn, dl);
            }
        } else if (B.vout) {
            // extraction: the values of V_iters move to the caller's buffer unchanged
            float4 *vout4 = (float4 *)((float2 *)B.vout + s0);
            for (uint32_t i = tid; i < n2; i += NT) vout4[i] = vin4[i];
            if ((nblk & 1u) && tid == 0) ((float2 *)B.vout)[s0 + nblk - 1] = ((const float2 *)B.vin)[s0 + nblk - 1];
        }
        if (B.pol)
            for (uint32_t i = tid; i < nblk; i += NT) B.pol[s0 + i] = s_pol[i];
        __syncthreads();   // s_out and s_pol are rewritten by the next tile
    }
    if (mode != MODE_EXTRACT) block_reduce_and_finalize<float>(mx, mn, st, mode, gridDim.x);
}

template <int G, int DP>
cudaError_t describe_lifo1_t(const KernelParams &kp, LaunchDesc &d) {
    const ProdParams &P = kp.p[0];
    const size_t smem = lifo1_smem(G, DP, P.rt_rows);
    cudaError_t e = cudaFuncSetAttribute(sweep_lifo1_kernel<G, DP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_lifo1_kernel<G, DP>, kL1Threads, smem)) !=
        cudaSuccess)
        return e;
    const uint32_t nR = P.nS / (uint32_t)G;
    const uint32_t ntiles = (nR + kL1Threads - 1) / kL1Threads;
    const uint32_t resident = (uint32_t)std::max(1, nsm * std::max(per_sm, 1));
    d.fn = (const void *)sweep_lifo1_kernel<G, DP>;
    d.grid = dim3(std::min(ntiles, resident));
    d.block = dim3(kL1Threads);
    d.smem = smem;
    d.lpr = 1;
    return cudaSuccess;
}

}  // namespace vib

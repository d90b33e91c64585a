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
// argmax over orders is taken per x.  Under LIFO the table splits as
// RT(R, x) = LF(x + R) + LH(R), so the float key of (x, a) is
// (-c_o a + gamma C_a + LH(R + a)) + LF(x + R + a): one window of 2G - 1 LF
// values per rest serves all G^2 keys; the exact value of the chosen order is
// rebuilt from the (hi, lo) pair of RT.
//
// Columns of rests.  X_{m-1}, the freshest rest slot, is the first one issued
// after the order, so a rest r' with one unit more there has H_{r'}[k] = H_r[k-1]
// (k >= 1), and the H part of each order's expectation,
// HP(a) = sum_{k>=1} p_{a+k} H~[k] measured from R0, follows from the previous
// rest's:  HP'(a) = HP(a + 1) - P(D > a) (V[r'] - V[r]).  The G rests that differ
// only in X_{m-1} form a column; its first rest gathers H and sums HP, each
// further rest gathers only T and takes HP by that recurrence.
//
// G = Q+1 and the pmf capacity DP (> dmax) are compile-time, so the convolution
// and the max over (x, a) are fully unrolled without per-thread bounds.  One
// thread owns one rest (its G states); each warp walks column tiles of 32 side by
// side on its own, rest by rest (persistent blocks, tables staged once per block,
// no block-wide barrier in the loop), so the warps of an SM drift apart and
// overlap each other's phases.  A warp takes floor(column tiles / warps) whole
// columns; the leftover columns' rests are then dealt out one at a time over all
// warps and computed afresh, so that the warps get nearly equal work.  The gathers
// of the warp's next tile and the previous values of its current one are copied
// into shared memory by cp.async while it computes; the new values replace the
// previous ones there (their change feeds the stopping test) and leave in 16-byte
// pieces where the tile starts on an even state.  HP waits for the next rest of a
// column in the lane's own H rows of that staging, which such a rest does not
// gather into.  The exact rebuild of the chosen orders runs on pairs of x in packed
// FP32 arithmetic, lane-wise the scalar operations.
#pragma once

#include <algorithm>

#include "vi_device.cuh"

namespace vib {

constexpr int kL1Threads = 128;

// two independent lanes of FP32 arithmetic in one instruction, each lane rounded as
// the scalar operation (a - b is a + (-b) exactly), so packed and scalar code agree
// bit for bit
__device__ __forceinline__ float2 l1_add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 l1_sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// bits per packed slot count for a radix G (ceil(log2 G))
__host__ __device__ constexpr int l1_bits(int G) { return G <= 2 ? 1 : (G <= 4 ? 2 : (G <= 8 ? 3 : (G <= 16 ? 4 : 5))); }

// asynchronous global -> shared copies (cp.async): the gathers of the next tile
// and the previous values of the current one land in shared memory while the
// block computes, without holding registers
__device__ __forceinline__ uint32_t l1_smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void l1_cp8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(l1_smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void l1_cp16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(l1_smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void l1_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void l1_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// shared memory of one block, in bytes: gathered columns (G + DP - 1 float pairs per
// rest), the tiles' previous / new values, the (hi, lo) pairs of RT at an odd row
// stride, the LIFO split LF / LH of RT, the gamma C_a columns and the policy bytes
// (the per-rest parts split into one region per warp)
__host__ __device__ inline size_t lifo1_smem(int G, int DP, int rt_rows, int tmax) {
    return (size_t)8 * (G + DP - 1) * kL1Threads + (size_t)8 * G * kL1Threads + (size_t)8 * rt_rows * (G | 1) +
           (size_t)4 * (tmax + 1 + rt_rows) + (size_t)4 * G * kL1Threads + (size_t)G * kL1Threads + 32;
}

// resident blocks per SM the register allocation aims for: four (128 registers)
// with a 16-entry pmf, two with a 32-entry one (five, with the table reads moved to
// L1 to make room, measured no faster on B300: their address arithmetic cost what
// the extra warps gained)
__host__ __device__ constexpr int lifo1_min_blocks(int DP) { return DP <= 16 ? 4 : 2; }

template <int G, int DP>
__global__ void __launch_bounds__(kL1Threads, lifo1_min_blocks(DP))
sweep_lifo1_kernel(KernelParams kp, int mode, const void *vin_arg, void *vout_arg, uint8_t *pol_arg, int lpr) {
    constexpr int GO = G | 1;          // odd row stride of the RT pairs: rows of different lanes hit other banks
    constexpr int CB = l1_bits(G);
    constexpr int NT = kL1Threads;
    constexpr int NTH = G + DP - 1;    // gathered per rest: T[0..G-1], H[1..DP-1]
    constexpr int XB = 2;              // x searched together in the first argmax
    static_assert(G >= 2 && G <= 16 && DP >= G && DP % 4 == 0 && DP <= 32, "lifo1 geometry");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // a sweep launched as a programmatic dependent of this one may start its set-up
    // (the tables below) while this one's last blocks run; values and the solve state
    // are read only after the wait, which returns once the grids this launch depends
    // on have completed (at once for an ordinary launch)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    SolveState *st = kp.st;
    const ProdParams &P = kp.p[0];
    const int rows = P.rt_rows;
    const int nF = P.tmax + 1;
    constexpr int WPB = NT / 32;       // warps per block; each warp walks tiles of 32 rests on its own
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // per-warp regions: gathered columns, the tile's states, gamma C_a columns, policy bytes
    float2 *s_TH = (float2 *)smem_raw + warp * (NTH * 32);                   // column j of a lane at [j * 32 + lane]
    float2 *s_VO = (float2 *)smem_raw + WPB * (NTH * 32) + warp * (G * 32);  // previous values, then new ones
    float2 *s_RTp = (float2 *)smem_raw + WPB * (NTH + G) * 32;               // (hi, lo) of RT(R, x) at [R * GO + x]
    float *s_LF = (float *)(s_RTp + rows * GO);      // LF(T), T = 0..tmax
    float *s_LH = s_LF + nF;                         // LH(R), R = 0..rows-1
    float *s_kc = s_LH + rows + warp * (G * 32);     // gamma C_a of a lane at [a * 32 + lane]
    uint8_t *s_pol = (uint8_t *)(s_LH + rows + WPB * (G * 32)) + warp * (G * 32);   // the tile's first argmax
    {
        const float *tab = (const float *)kp.tables;
        for (int i = threadIdx.x; i < rows * GO; i += NT) {
            const int R = i / GO, x = i - R * GO;
            s_RTp[i] = (x < G) ? make_float2(tab[P.off_RT + R * G + x], tab[P.off_RTlo + R * G + x])
                               : make_float2(0.f, 0.f);
        }
        for (int i = threadIdx.x; i < nF; i += NT) s_LF[i] = tab[P.off_LF + i];
        for (int i = threadIdx.x; i < rows; i += NT) s_LH[i] = tab[P.off_LH + i];
    }
    __syncthreads();   // the tables are shared by the block's warps; nothing else is
    asm volatile("griddepcontrol.wait;" ::: "memory");
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;

    const uint32_t nS = P.nS;
    const uint32_t nR = nS / (uint32_t)G;
    const int nrs = P.n_rest_slots;                  // m - 2 rest slots: X_2 .. X_{m-1}
    // columns: the G rests that differ only in X_{m-1}, the first rest slot issued after
    // the order (weight w7 in the rest index); a column tile is 32 columns side by side
    const uint32_t colLen = (nrs >= 2) ? (uint32_t)G : 1u;
    const uint32_t w7 = (nrs >= 2) ? P.w_top / (uint32_t)G : 0u;   // G^(m-3)
    const uint32_t nbase = nR / colLen;              // rests with X_{m-1} = 0 (every rest without columns)
    const uint32_t ncolt = (nbase + 31u) / 32u;      // column tiles
    const uint32_t w_top = P.w_top;                  // G^(m-2): weight of the order's next-state slot
    const int dmax = P.dmax;
    const float gam = (float)kp.gamma;
    const float c_o = (float)P.c_o;
    const float2 *V2 = (const float2 *)B.vin;
    // 16-byte pieces need 16-byte aligned value buffers and a tile that starts on an even state
    const bool al16 = ((((uintptr_t)B.vin) | ((uintptr_t)B.vout)) & 15u) == 0;
    float *kc_col = s_kc + lane;
    float mx = -INFINITY, mn = INFINITY;

    // the gathers of rest z of column tile c into this lane's column: T[j] = V[r + j G^(m-2)],
    // then (a fresh rest only) H[k] = V[r after k units issued freshest first] for
    // k <= min(R, dmax); returns R (Rprev + 1 for the next rest of the same column)
    auto prefetch_gathers = [&](uint32_t c, uint32_t z, bool fresh, int Rprev) -> int {
        const uint32_t rb = c * 32u + (uint32_t)lane;
        if (rb >= nbase) return 0;
        const uint32_t r = rb + z * w7;
        if (!fresh) {
#pragma unroll
            for (int j = 0; j < G; ++j) l1_cp8(s_TH + j * 32 + lane, V2 + r + (uint32_t)j * w_top);
            return Rprev + 1;
        }
        unsigned long long packed = 0ull;
        int Rr = 0;
        uint32_t rem = r;
        for (int j = 0; j < nrs; ++j) {
            const uint32_t q = rem / (uint32_t)G;
            const int dg = (int)(rem - q * (uint32_t)G);
            rem = q;
            packed |= (unsigned long long)dg << (CB * j);
            Rr += dg;
        }
#pragma unroll
        for (int j = 0; j < G; ++j) l1_cp8(s_TH + j * 32 + lane, V2 + r + (uint32_t)j * w_top);
        // slot by slot from X_{m-1} down: each unit issued subtracts the slot's weight
        const int hcount = min(Rr, dmax);
        uint32_t w = (nrs > 0) ? w_top / (uint32_t)G : 0u;
        uint32_t idx = r;
        float2 *col = s_TH + G * 32 + lane;   // H[1] of this lane
        int k = 0;
        for (int slot = nrs - 1; slot >= 0 && k < hcount; --slot) {
            const int units = min((int)((packed >> (CB * slot)) & ((1ull << CB) - 1ull)), hcount - k);
            for (int u = 0; u < units; ++u) {
                idx -= w;
                l1_cp8(col + k * 32, V2 + idx);
                ++k;
            }
            w /= (uint32_t)G;
        }
        return Rr;
    };
    // the previous values of a tile's states, in 16-byte pieces where aligned (a tile of
    // rests z w7 .. z w7 + 31 starts on an odd state when z w7 G is odd)
    auto tile_s0 = [&](uint32_t c, uint32_t z) -> uint32_t { return (c * 32u + z * w7) * (uint32_t)G; };
    auto tile_nblk = [&](uint32_t c) -> uint32_t { return min(32u, nbase - c * 32u) * (uint32_t)G; };
    auto prefetch_old = [&](uint32_t c, uint32_t z) {
        const uint32_t s0 = tile_s0(c, z);
        const uint32_t nblk = tile_nblk(c);
        const float2 *src = V2 + s0;
        if (al16 && !(s0 & 1u)) {
            for (uint32_t i = lane; i < (nblk >> 1); i += 32) l1_cp16(s_VO + 2 * i, src + 2 * i);
            if ((nblk & 1u) && lane == 0) l1_cp8(s_VO + nblk - 1, src + nblk - 1);
        } else {
            for (uint32_t i = lane; i < nblk; i += 32) l1_cp8(s_VO + i, src + i);
        }
    };

    // The warp's items (column tile, rest z of the column): first F whole columns
    // wid + k W rest by rest, the H part of each rest after the first following from the
    // previous one; then the leftover columns' rests dealt out one at a time over all
    // warps, each computed afresh, so that every warp gets nearly the same number of rests
    const uint32_t W = gridDim.x * (uint32_t)WPB;
    const uint32_t wid = blockIdx.x * (uint32_t)WPB + (uint32_t)warp;
    const uint32_t F = ncolt / W;
    const uint32_t NL = (ncolt - F * W) * colLen;
    auto item_at = [&](int ph, uint32_t k, uint32_t z, uint32_t j, uint32_t &ct, uint32_t &zt, bool &fr) -> bool {
        if (ph == 0) {
            ct = wid + k * W;
            zt = z;
            fr = (z == 0);
            return true;
        }
        const uint32_t jj = wid + j * W;
        if (jj >= NL) return false;
        const uint32_t q = jj / colLen;
        ct = F * W + q;
        zt = jj - q * colLen;
        fr = true;
        return true;
    };
    auto advance = [&](int &ph, uint32_t &k, uint32_t &z, uint32_t &j) {
        if (ph == 0) {
            if (z + 1 < colLen) {
                ++z;
                return;
            }
            z = 0;
            if (++k < F) return;
            ph = 1;
            j = 0;
            return;
        }
        ++j;
    };
    int ph = (F > 0) ? 0 : 1;
    uint32_t ik = 0, iz = 0, ij = 0;
    uint32_t ct = 0, zt = 0;
    bool fresh = true;
    bool have = item_at(ph, ik, iz, ij, ct, zt, fresh);
    int Rnext = 0;
    if (have) Rnext = prefetch_gathers(ct, zt, fresh, 0);
    l1_commit();
    if (have) prefetch_old(ct, zt);
    l1_commit();
    float2 R0prev = make_float2(0.f, 0.f);
    // H part of each order's expectation, HP(a) = sum_{k>=1} p_{a+k} H~[k] for a = 0..DP-2
    // (zero from dmax on).  It is carried from rest to rest along a column in the lane's
    // own H rows of the staging, two values per row: a rest that continues a column gathers
    // no H, and a fresh rest's H gathers land there only after the previous rest has taken
    // its values into registers
    constexpr int NHP = DP - 1;
    constexpr int NHR = (NHP + 1) / 2;
    float2 *hpcol = s_TH + G * 32 + lane;
    while (have) {
        int ph2 = ph;
        uint32_t k2 = ik, z2 = iz, j2 = ij, cn = 0, zn = 0;
        bool fn = true;
        advance(ph2, k2, z2, j2);
        const bool have_next = item_at(ph2, k2, z2, j2, cn, zn, fn);
        const bool active = ct * 32u + (uint32_t)lane < nbase;
        const int Rrest = Rnext;
        l1_wait<1>();   // this lane's gathers of the tile have landed (its previous values may not)
        float2 R0 = make_float2(0.f, 0.f);
        if (active) R0 = s_TH[lane];
        // pair_diff(g, R0) = (g.hi - R0.hi) + (g.lo - R0.lo), both differences in one packed add
        const float2 nR0 = make_float2(-R0.x, -R0.y);
        float hp[NHP];
        if (fresh) {
            // the H part from the rest's own sequence, read and summed before T is read (fewer
            // registers live at once)
            float H[DP];
            H[0] = 0.f;
            if (active) {
                const int hcount = min(Rrest, dmax);
#pragma unroll
                for (int k = 1; k < DP; ++k) {
                    const float2 d = l1_add2(s_TH[(G - 1 + k) * 32 + lane], nR0);
                    H[k] = (k <= hcount) ? __fadd_rn(d.x, d.y) : H[k - 1];
                }
            }
#pragma unroll
            for (int a = 0; a < NHP; ++a) {
                float h = 0.f;
                if (active) {
#pragma unroll
                    for (int k = 1; a + k < DP; ++k) h = fmaf(kp.pmf32[a + k], H[k], h);
                }
                hp[a] = h;
            }
        } else {
            // one unit more in X_{m-1}, the first rest unit issued after the order, shifts H by
            // one: H'[k] = H[k-1], so measured from R0' = V[r'],
            //   HP'(a) = HP(a + 1) - P(D > a) (V[r'] - V[r])
            const float dl = active ? pair_diff(R0, R0prev) : 0.f;
            float old[2 * NHR];
#pragma unroll
            for (int i = 0; i < NHR; ++i) {
                const float2 v = hpcol[i * 32];
                old[2 * i] = v.x;
                old[2 * i + 1] = v.y;
            }
#pragma unroll
            for (int a = 0; a < NHP; ++a) hp[a] = __fmaf_rn(kp.nsurv32[a], dl, (a + 1 < NHP) ? old[a + 1] : 0.f);
        }
        if (have_next && !fn) {
            // the next rest continues this column: keep the H part for it
#pragma unroll
            for (int i = 0; i < NHR; ++i) hpcol[i * 32] = make_float2(hp[2 * i], (2 * i + 1 < NHP) ? hp[2 * i + 1] : 0.f);
        }
        R0prev = R0;
        float T[G];
        T[0] = 0.f;
        if (active) {
#pragma unroll
            for (int j = 1; j < G; ++j) {
                const float2 d = l1_add2(s_TH[j * 32 + lane], nR0);
                T[j] = __fadd_rn(d.x, d.y);
            }
        }
        __syncwarp();   // the column is read (each lane reads and refills only its own)
        if (have_next) Rnext = prefetch_gathers(cn, zn, fn, Rrest);
        l1_commit();

        int arg[G];
        {
            // -- expectations of every order: C_a = sum_{d<a} p_d T[a-d] + sum_{k>=1} p_{a+k} H~[k]
            // (a lane past the last rest takes zeros: it only joins the warp's bounds below)
            float C[G];
#pragma unroll
            for (int a = 0; a < G; ++a) {
                float c = 0.f;
                if (active) {
#pragma unroll
                    for (int d = 0; d < a; ++d) c = fmaf(kp.pmf32[d], T[a - d], c);
                }
                C[a] = __fadd_rn(c, (a < NHP) ? hp[a] : 0.f);
            }
            // -- first argmax over orders per x on the float key ks_a + LF(x + R + a), with
            // ks_a = -c_o a + gamma C_a + LH(R + a): the rest's LF window covers every key
            float Fw[2 * G + XB];
#pragma unroll
            for (int i = 0; i < 2 * G - 1; ++i) Fw[i] = s_LF[Rrest + i];
#pragma unroll
            for (int i = 2 * G - 1; i < 2 * G + XB; ++i) Fw[i] = 0.f;
            float ks[G];
#pragma unroll
            for (int a = 0; a < G; ++a) {
                const float bl = __fmul_rn(gam, C[a]);
                kc_col[a * 32] = bl;
                ks[a] = __fadd_rn(__fadd_rn(__fmul_rn(-c_o, (float)a), bl), s_LH[Rrest + a]);
            }
            // LF is concave (its -E[(T - D)^+] term is), so the key has decreasing
            // differences in (x, a) and the first argmax does not increase with x: the orders
            // past the largest one the warp chose for the x before are not searched.  (Where
            // rounding of the float keys breaks the monotonicity, the orders it would have
            // preferred tie within that rounding.)  The x go in pairs under the bound of the
            // pair before, two independent compare-select chains in flight; once the bound is
            // order 0, every later x takes order 0 with no search.
            int lim = G - 1;
#pragma unroll
            for (int x = 0; x < G; x += XB) {
                if (x > 0 && lim == 0) {   // uniform across the warp
#pragma unroll
                    for (int i = 0; i < XB; ++i)
                        if (x + i < G) arg[x + i] = 0;
                    continue;
                }
                float b[XB];
                int ab[XB];
#pragma unroll
                for (int i = 0; i < XB; ++i) {
                    b[i] = __fadd_rn(ks[0], Fw[x + i]);   // x + i >= G reads the zero pad: unused
                    ab[i] = 0;
                }
#pragma unroll
                for (int a = 1; a < G; ++a) {
                    if (a > lim) break;   // uniform across the warp
#pragma unroll
                    for (int i = 0; i < XB; ++i) {
                        const float key = __fadd_rn(ks[a], Fw[x + i + a]);
                        const bool up = key > b[i];
                        b[i] = up ? key : b[i];
                        ab[i] = up ? a : ab[i];
                    }
                }
                int last = ab[0];
#pragma unroll
                for (int i = 0; i < XB; ++i)
                    if (x + i < G) {
                        arg[x + i] = ab[i];
                        last = ab[i];
                    }
                lim = __reduce_max_sync(0xffffffffu, active ? last : 0);
            }
        }
        l1_wait<1>();   // this lane's pieces of the previous values have landed
        __syncwarp();   // ... and every lane's: a lane's states were copied by other lanes
        if (active) {
            // -- the exact pair of each x's chosen order: gamma R0 + (-c_o a) + gamma C_a + RT,
            // its change from the previous value, and the new value in place of the old
            float ph, pe;
            two_prod(gam, R0.x, ph, pe);
            const float pl = __fmaf_rn(gam, R0.y, pe);
            float2 *o = s_VO + lane * G;
            uint8_t *op = s_pol + lane * G;
            // every shared-memory operand of the rebuild is loaded before its arithmetic; the
            // rebuild runs on pairs of x (x, x+1) in packed arithmetic, lane by lane the same
            // operations as pair_add, two_sum, fast_two_sum and pair_diff
            float kq[G], rh[G], rl[G], oh[G], ol[G];
#pragma unroll
            for (int x = 0; x < G; ++x) {
                const int a = arg[x];
                kq[x] = kc_col[a * 32];
                const float *rpx = (const float *)(s_RTp + (Rrest + a) * GO + x);
                rh[x] = rpx[0];
                rl[x] = rpx[1];
                if (mode != MODE_EXTRACT) {
                    oh[x] = ((const float *)(o + x))[0];
                    ol[x] = ((const float *)(o + x))[1];
                }
            }
            const float2 ph2 = make_float2(ph, ph), pl2 = make_float2(pl, pl), nco2 = make_float2(-c_o, -c_o);
#pragma unroll
            for (int x = 0; x < G; x += 2) {
                if (x + 1 < G) {
                    const int a0 = arg[x], a1 = arg[x + 1];
                    float2 qh = __fmul2_rn(nco2, make_float2((float)a0, (float)a1));
                    float2 ql = make_float2(kq[x], kq[x + 1]);
                    const float2 r_h = make_float2(rh[x], rh[x + 1]), r_l = make_float2(rl[x], rl[x + 1]);
                    // pair_add(qh, ql, r_h, r_l)
                    {
                        const float2 sm = l1_add2(qh, r_h);
                        const float2 bb = l1_sub2(sm, qh);
                        const float2 e = l1_add2(l1_sub2(qh, l1_sub2(sm, bb)), l1_sub2(r_h, bb));
                        qh = sm;
                        ql = l1_add2(e, l1_add2(ql, r_l));
                    }
                    // two_sum(ph, qh), then fast_two_sum(sh, se + (pl + ql))
                    const float2 sh = l1_add2(ph2, qh);
                    const float2 bb = l1_sub2(sh, ph2);
                    const float2 se = l1_add2(l1_sub2(ph2, l1_sub2(sh, bb)), l1_sub2(qh, bb));
                    const float2 lo = l1_add2(se, l1_add2(pl2, ql));
                    const float2 vh = l1_add2(sh, lo);
                    const float2 vl = l1_sub2(lo, l1_sub2(vh, sh));
                    if (mode != MODE_EXTRACT) {
                        const float2 dl = l1_add2(l1_sub2(vh, make_float2(oh[x], oh[x + 1])),
                                                  l1_sub2(vl, make_float2(ol[x], ol[x + 1])));
                        mx = fmaxf(mx, fmaxf(dl.x, dl.y));
                        mn = fminf(mn, fminf(dl.x, dl.y));
                        o[x] = make_float2(vh.x, vl.x);
                        o[x + 1] = make_float2(vh.y, vl.y);
                    }
                    if (B.pol) {
                        op[x] = (uint8_t)a0;
                        op[x + 1] = (uint8_t)a1;
                    }
                } else {
                    const int a = arg[x];
                    float qh = __fmul_rn(-c_o, (float)a), ql = kq[x];
                    pair_add(qh, ql, rh[x], rl[x]);
                    float sh, se;
                    two_sum(ph, qh, sh, se);
                    const float lo = __fadd_rn(se, __fadd_rn(pl, ql));
                    float vh, vl;
                    fast_two_sum(sh, lo, vh, vl);
                    if (mode != MODE_EXTRACT) {
                        const float dl = pair_diff(make_float2(vh, vl), make_float2(oh[x], ol[x]));
                        mx = fmaxf(mx, dl);
                        mn = fminf(mn, dl);
                        o[x] = make_float2(vh, vl);
                    }
                    if (B.pol) op[x] = (uint8_t)a;
                }
            }
        }
        __syncwarp();   // the tile's new values and policy bytes are in place
        // -- the tile's states leave in 16-byte pieces (two states) where aligned; an
        // extraction moves the previous values unchanged (only when a buffer is given).
        // The stores are marked streaming (evict first): this sweep never reads them, so
        // L2 keeps the values it still gathers instead
        const uint32_t s0 = tile_s0(ct, zt);
        const uint32_t nblk = tile_nblk(ct);
        if (B.vout) {
            float2 *dst = (float2 *)B.vout + s0;
            if (al16 && !(s0 & 1u)) {
                for (uint32_t i = lane; i < (nblk >> 1); i += 32) __stcs((float4 *)dst + i, ((const float4 *)s_VO)[i]);
                if ((nblk & 1u) && lane == 0) __stcs(dst + nblk - 1, s_VO[nblk - 1]);
            } else {
                for (uint32_t i = lane; i < nblk; i += 32) __stcs(dst + i, s_VO[i]);
            }
        }
        if (B.pol)
            for (uint32_t i = lane; i < nblk; i += 32) B.pol[s0 + i] = s_pol[i];
        __syncwarp();   // the value staging is free for the next tile's previous values
        if (have_next) prefetch_old(cn, zn);
        l1_commit();
        ph = ph2;
        ik = k2;
        iz = z2;
        ij = j2;
        ct = cn;
        zt = zn;
        fresh = fn;
        have = have_next;
    }
    l1_wait<0>();
    if (mode != MODE_EXTRACT) block_reduce_and_finalize<float>(mx, mn, st, mode, gridDim.x);
}

template <int G, int DP>
cudaError_t describe_lifo1_t(const KernelParams &kp, LaunchDesc &d) {
    const ProdParams &P = kp.p[0];
    const size_t smem = lifo1_smem(G, DP, P.rt_rows, P.tmax);
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
    d.pdl = 1;
    return cudaSuccess;
}

}  // namespace vib

// vi_common.cuh -- shared definitions of the B300 value-iteration kernels.
//
// State layout (mixed radix, G = Q+1): digit k has weight G^k; digits 0..m-2 are
// the on-hand stock X_1..X_{m-1} by remaining life, digits m-1..K-1 the orders in
// transit P_1..P_{L-1}.  Write s = x + G*r with x = digit 0.  Digit 0 is always
// the oldest unit slot Y_1 (X_1, or the arriving order P_1 when m = 1), and it
// never survives into the next state: whatever is left of it expires.  The next
// state only depends on the "rest" r, the action a and the demand reaching the
// other slots.  With Z_1..Z_{m-1} = (X_2, ..., X_{m-1}, u) (u = arriving units),
// the next state before any demand is s'_0 = r + a * G^(K-1), and every unit of
// demand that reaches the rest removes one unit from one Z slot, i.e. subtracts
// that slot's weight from the index: oldest slot first under FIFO, freshest slot
// first under LIFO (Eq. demoor:fifo, Eq. demoor:lifo).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vib {

constexpr int kMaxDigits = 31;      // (Q+1)^K < 2^32 with Q >= 1
constexpr int kMaxDmax = 4095;

// ---------------------------------------------------------------------------
// per-product parameters (plain data; passed by value inside KernelParams)
// ---------------------------------------------------------------------------
struct ProdParams {
    int m, L, Q, G;       // life, lead time, order cap, radix G = Q+1
    int K;                // number of state digits (m-1)+(L-1)
    int dmax;             // demand support 0..dmax
    int tmax;             // largest stock available in a period, m*Q
    int cb;               // bits per packed slot count = ceil(log2(G))
    uint32_t nS;          // G^K
    uint32_t w_top;       // G^(K-1) (0 if K == 0)
    int n_rest_slots;     // slots of r that are stock Z digits: m-2 (L=1) or m-1 (L>=2), >= 0
    uint32_t w_zt;        // G^(m-2): weight of the freshest stock slot Z_{m-1} (1 if m < 2)
    // offsets (in elements) of this product's tables inside the table blob
    int off_p;            // p[k]     = P(D = k), zero beyond dmax        (len pn)
    int off_F;            // F[k]     = P(D <= k), one beyond dmax         (len pn)
    int off_tail;         // tail[k]  = P(D >= k), zero beyond dmax        (len pn)
    int off_RT;           // RT[R * G + y1]: expected reward without the order cost, given
                          // y1 units in the expiring slot and R in the others (FP64-built)
    int off_RTlo;         // FP32 blobs: RT - fl32(RT), the low half of the pair (zero in FP64 blobs)
    int rt_rows;          // R ranges over 0..rt_rows-1 = (m-1)Q
    int off_LF, off_LH;   // LIFO: RT(R, y1) = LF[y1 + R] + LH[R] (LF over 0..tmax, LH over 0..rt_rows-1;
                          // 0 when absent), with y1 issued last the period's sums depend on y1 + R only
                          // except for the units of the other slots left unsold
    int pn;               // length of p / F / tail
    double c_o;           // order cost per unit
    uint32_t g_mag;       // x / G as a multiply-high and two shifts (DivG below)
    int g_sh1, g_sh2;
};

struct SolveState;  // device-resident solve bookkeeping (below)

struct KernelParams {
    ProdParams p[2];
    int n_products;
    int issuing;          // 0 FIFO, 1 LIFO
    uint32_t nS;          // total states
    int nA;               // total actions
    double gamma;
    const void *tables;   // device table blob (float or double, see precision)
    int n_tables;         // elements in the blob
    int tab_in_smem;      // generic kernels stage the (per-block) tables in shared memory
    // two-product extras (offsets into the blob)
    int off_M;            // M[T1][z]: mass of (d1 >= T1, product-2 demand z), row length zlen
    int off_Mc;           // cumulative of M rows
    int off_Mt;           // tail of M rows
    int off_H1;           // H1[y1][T1]  expected product-1 reward terms, row length (tmax1+1)
    int off_H2;           // H2[T1][y2][T2] expected product-2 + substitution terms
    int off_H1lo, off_H2lo;   // low halves of H1 / H2 (float blobs)
    int zlen;             // dmax1 + dmax2 + 1
    SolveState *st;       // solve bookkeeping
    int tc_stall;         // test hook: the tensor-core kernel withholds its MMAs, so its bounded wait runs out
    // factorised two-product sweep: per-sweep tables of product-2 expectations
    float *two_e2;        // [s2][a2][i1]  sum_z w(z) (V(i1, s2'(z)) - V(i1, s2'(0)))
    float *two_mix;       // [s2][a2][T1]  the substitution mixture of d1 >= T1, same frame with i1 = 0
                          // (lead times >= 2: [s2][a2][pipe1][T1], pipe1 = product-1 pipeline of s')
    int two_nt1;          // T1 values kept: 0..min(dmax1, m1 Q1)
    int two_npipe1;       // product-1 pipeline classes of an emptied next state: G1^(L1-1)
    const uint32_t *two_rperm;   // lead times >= 2: product-1 rests ordered by their unit total
    const uint32_t *grp_order;   // factorised sweep: block order, heaviest rests first (null: natural order)
    float pmf32[64];             // product 0's pmf in FP32, zero past dmax (kept here so that sweeps with
                                 // compile-time demand loops read it from the parameter constant bank)
    float nsurv32[64];           // -P(D > x) of product 0 in FP32, zero from dmax on (the FIFO column sweep)
    // Scenario C (periodic demand, life on arrival; vi_pc.cu): p[0] holds m, Q = A_max,
    // G, dmax, nS = G^(m-1) states per weekday
    int pc;                      // 1 for a periodic problem
    int pc_m;                    // maximum useful life on arrival
    const double *pc_pmf;        // 7 x (dmax+1): demand pmf of weekday tau in row tau
    const unsigned long long *pc_prof;   // arrival profiles y_1..y_m, 6 bits each (y_1 lowest), by order
    const double *pc_prob;       // P(y | a) of each profile
    const int *pc_off;           // the profiles of order a are [pc_off[a], pc_off[a+1])
    double *pc_W;                // 7 G^m post-decision values
    double *pc_ring;             // 7 |S| weighted differences of the periodic stopping test
    double pc_cost[4];           // C_f per order placed, C_h, C_s, C_w per unit
};

constexpr int kPcMaxM = 8;       // periodic problems: m <= 8
constexpr int kStopPeriodic = 2; // the periodic stopping test (VI_STOP_PERIODIC)

// ---------------------------------------------------------------------------
// device solve bookkeeping.  The sweep kernel reads its input/output buffers and
// the normalisation constant from here; the last block of every sweep folds the
// block reductions, updates the FP64 offset and decides whether to continue.
// ---------------------------------------------------------------------------
struct SolveState {
    // configuration (written by the host before a solve)
    void *buf[2];                 // buf[0] = caller's V, buf[1] = scratch
    uint8_t *policy;              // caller's policy or null
    void *vhost;                  // extraction writes V here (device view of pinned host memory) or null
    double tol;
    double gamma;
    int max_iters;
    int stop_rule;
    int normalise;                // FP32 paths subtract c each sweep
    int use_cond;                 // set the graph conditional from the last block
    int warm;                     // keep V and the offset given by the caller
    int value_bytes;              // 4 (float) or 8 (double or float pair)
    unsigned long long cond;      // cudaGraphConditionalHandle
    // running state
    unsigned long long key_max;   // order-preserving encoding of max(v_i - v_{i-1})
    unsigned long long key_min;
    unsigned int blocks_done;
    int iter;                     // sweeps done
    int keep_going;               // 1 while the sweep loop should run
    int converged;
    float c_cur;                  // constant subtracted in the current sweep
    float c_next;                 // unnormalised value of state 0 in the current sweep
    double offset;                // b: V_abs = b + v
    double crit, dmax_abs, dmin_abs;
    int fault;                    // set by a kernel whose bounded wait on the tensor cores gave up
};

// length of the p / F / tail tables: zero (p, tail) or one (F) beyond dmax, long
// enough for every index a sweep kernel forms (x + k + chunk padding, x + R)
__host__ __device__ inline int p_table_len(int dmax, int tmax, int G) { return dmax + 1 + tmax + 2 * G + 34; }

// LIFO with L = 1 (m >= 2): the factorised kernel gathers the two shared
// sequences of an action-independent layout once per rest, if their per-thread
// columns fit in 64 KiB of shared memory for a block of 128 threads
__host__ __device__ inline bool lifo_shared_ok(const ProdParams &P) {
    return P.L == 1 && P.m >= 2 && (P.G + P.dmax + 1) * 128 * 4 <= 64 * 1024;
}

// LIFO with L = 1 and the shared sequences: the running max compares one float
// per (x, order) and keeps each order's expectation term in a per-thread column
// of G floats
__host__ __device__ inline bool lifo_key_ok(const ProdParams &P) { return P.L == 1 && P.G <= 32; }

// FIFO: the rest path is kept per thread if a column of dmax+1 indices fits in
// 64 KiB of shared memory for a block of 128 threads
__host__ __device__ inline bool fifo_shared_ok(const ProdParams &P) {
    return P.m >= 2 && (P.dmax + 9) * 128 * 4 <= 64 * 1024;   // + 8 entries past the last k of a chunk
}

// order-preserving map double -> uint64 so that unsigned max/min give double max/min
__device__ __forceinline__ unsigned long long dkey(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

// Division of a 32-bit index by the radix G: the quotient operator (PlainDiv), or an
// exact multiply-high with the constants of Granlund and Montgomery, "Division by
// invariant integers using multiplication" (PLDI 1994; the round-up method for
// every 32-bit dividend), which the host sets per product: l = ceil(log2 G),
// g_mag = floor(2^32 (2^l - G) / G) + 1, g_sh1 = min(l, 1), g_sh2 = max(l - 1, 0).
struct PlainDiv {
    __device__ __forceinline__ static uint32_t q(uint32_t x, uint32_t G, const ProdParams *) { return x / G; }
};
struct DivG {
    __device__ __forceinline__ static uint32_t q(uint32_t x, uint32_t, const ProdParams *P) {
        const uint32_t t = __umulhi(x, P->g_mag);
        return (t + ((x - t) >> P->g_sh1)) >> P->g_sh2;
    }
};

// ---------------------------------------------------------------------------
// The next-state walker: index of s'(e) after e units of demand reached the rest
// slots.  Slot counts are packed `cb` bits each in consumption order.
// ---------------------------------------------------------------------------
struct Walker {
    uint32_t idx;        // current next-state index
    uint32_t w;          // weight of the slot being consumed
    unsigned long long packed;   // counts of Z_1..Z_{m-1}, Z_1 in the low bits
    int slot;            // 0-based slot being consumed (weight G^slot)
    int left;            // units left in it
};

// FIFO: consume Z_1 first (weight 1) upward.  LIFO: consume Z_{m-1} first.
__device__ __forceinline__ void walker_init(Walker &wk, uint32_t idx0, unsigned long long packed,
                                            int nslots, int cb, int lifo, uint32_t G_pow_top) {
    wk.idx = idx0;
    wk.packed = packed;
    unsigned long long mask = (1ull << cb) - 1ull;
    if (!lifo) {
        wk.slot = 0;
        wk.w = 1u;
        wk.left = (nslots > 0) ? (int)(packed & mask) : 0;
    } else {
        wk.slot = nslots - 1;
        wk.w = G_pow_top;   // G^(nslots-1)
        wk.left = (nslots > 0) ? (int)((packed >> (cb * (nslots - 1))) & mask) : 0;
    }
}

// consume one unit; callers only step while units remain in the slots (e <= R).
// The slot search is bounded so that a violated precondition cannot spin.
// (LIFO moves down a slot by dividing the slot weight by G: Div chooses how, with P
// holding DivG's constants.)
template <class Div = PlainDiv>
__device__ __forceinline__ void walker_step(Walker &wk, int cb, int lifo, uint32_t G, const ProdParams *P = nullptr) {
    unsigned long long mask = (1ull << cb) - 1ull;
    for (int guard = 0; wk.left == 0; ++guard) {
        if (guard >= kMaxDigits) return;
        if (!lifo) {
            wk.slot += 1;
            wk.w *= G;
        } else {
            wk.slot -= 1;
            wk.w = Div::q(wk.w, G, P);
        }
        wk.left = (int)((wk.packed >> (cb * wk.slot)) & mask);
    }
    wk.idx -= wk.w;
    wk.left -= 1;
}

// ---------------------------------------------------------------------------
// decode of the rest index r (digits 1..K-1 of s): stock slots + pipeline
// ---------------------------------------------------------------------------
struct RestInfo {
    unsigned long long packed;   // counts of the rest stock slots (without the arrival if L = 1)
    int R;                       // their sum
};

template <class Div = PlainDiv>
__device__ __forceinline__ RestInfo decode_rest(uint32_t r, const ProdParams &P) {
    RestInfo ri;
    ri.packed = 0ull;
    ri.R = 0;
    uint32_t rem = r;
    for (int j = 0; j < P.n_rest_slots; ++j) {
        uint32_t q = Div::q(rem, (uint32_t)P.G, &P);
        int dgt = (int)(rem - q * (uint32_t)P.G);
        rem = q;
        ri.packed |= (unsigned long long)dgt << (P.cb * j);
        ri.R += dgt;
    }
    return ri;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): rounds multiply words 0 and 2 by
// 0xD2511F53 / 0xCD9E8D57; key bumped by 0x9E3779B9 / 0xBB67AE85 between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t out[4]) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

}  // namespace vib

// vi_tc.cu -- the FIFO expectation of the factorised sweep on the tensor cores.
//
// For a rest r (digits 1..K-1 of the state) and an order a, the FIFO expectation
// of every expiring-slot count x is a correlation of the pmf with the values
// gathered along the rest's demand path (Eq. demoor:fifo, Algorithm 1):
//   C_a(x) = sum_{k>=1} p[x+k] (g_a(min(k, R)) - g_a(0)),
// k being the demand that reaches the slots after x.  With W[x][k] = p[x+k]
// fixed for the whole sweep, the expectations of a tile of rests are one dense
// product  C[(rest, order), x] = G[(rest, order), k] . W^T[k, x].
//
// Both operands are split exactly into three bf16 parts (bit truncation: the
// parts of an FP32 number v satisfy v = v1 + v2 + v3 exactly), and the six
// products whose magnitude is at least 2^-16 of the leading one are accumulated
// in FP32 in tensor memory, which keeps FP32 accuracy.  A tile is 128 rows
// (rests x orders) by 32 columns (x) by 16k K; one thread issues the
// tcgen05.mma instructions, the block reads the accumulator back with
// tcgen05.ld, and the running first-argmax over orders and the span statistics
// follow as in the CUDA-core kernel.
#include <algorithm>

#include "vi_device.cuh"
#include "vi_kernels.h"

namespace vib {

constexpr int kTcThreads = 128;   // one thread per accumulator row (tensor-memory lane)
constexpr int kTcCols = 32;       // accumulator columns: x = 0..31
constexpr int kTcRows = 128;      // MMA M
constexpr int kTcAG = 4;          // orders per staging item
constexpr long kTcMaxPolls = 1L << 22;   // bound on the wait for one tile's MMAs

// ---------------------------------------------------------------------------
// tcgen05 / mbarrier helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, K-major without swizzle: 8-row x 16-byte core
// matrices, `lbo` bytes between core matrices adjacent in K, `sbo` bytes between
// groups of 8 rows
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version
    return d;
}

// kind::f16 instruction descriptor: bf16 A and B (K-major), FP32 accumulator, M x N
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// exact split v = v1 + v2 + v3 into bf16 values (top 16 bits of each part)
__device__ __forceinline__ void split3(float v, uint32_t &b1, uint32_t &b2, uint32_t &b3) {
    const uint32_t u1 = __float_as_uint(v) & 0xFFFF0000u;
    const float r1 = __fsub_rn(v, __uint_as_float(u1));
    const uint32_t u2 = __float_as_uint(r1) & 0xFFFF0000u;
    const float r2 = __fsub_rn(r1, __uint_as_float(u2));
    b1 = u1;
    b2 = u2;
    b3 = __float_as_uint(r2);   // at most 8 significant bits: its low half is zero
}

// byte offset of element (row, col) in a K-major no-swizzle operand whose rows
// hold `nkc` 16-byte chunks
__device__ __forceinline__ uint32_t umma_off(int row, int col, int nkc) {
    return (uint32_t)((row >> 3) * (nkc * 128) + (col >> 3) * 128 + (row & 7) * 16 + (col & 7) * 2);
}

struct TcLayout {
    int kpad, nkc, rpt, rows, pn_pad;
    uint32_t planeA, planeB;
    int nag, nkd, n_items;
    uint32_t offB, offP, offPath, offQ, offBh, offRef, offR0, offR, offDig, offItems, offMbar, offTmem, total;
};

__host__ __device__ inline TcLayout tc_layout(const ProdParams &P) {
    TcLayout L;
    L.kpad = (P.dmax + 15) & ~15;
    L.nkc = L.kpad / 8;
    L.rpt = kTcRows / P.G;
    L.rows = L.rpt * P.G;
    L.pn_pad = (P.pn + 3) & ~3;
    L.planeA = (uint32_t)kTcRows * L.kpad * 2;
    L.planeB = (uint32_t)kTcCols * L.kpad * 2;
    uint32_t o = 3 * L.planeA;
    L.offB = o;
    o += 3 * L.planeB;
    L.offP = o;
    o += (uint32_t)L.pn_pad * 4;
    L.offPath = o;
    o += (uint32_t)L.rpt * (P.dmax + 1) * 4;
    L.offQ = o;
    o += (uint32_t)L.rows * P.G * 4;
    L.offBh = o;
    o += (uint32_t)L.rows * 4;
    o = (o + 7) & ~7u;
    L.offRef = o;
    o += (uint32_t)L.rows * 8;
    L.offR0 = o;
    o += (uint32_t)L.rpt * 8;
    L.offR = o;
    o += (uint32_t)L.rpt * 4;
    L.offDig = o;
    o += (uint32_t)L.rpt * kMaxDigits * 4;
    L.nag = (P.G + kTcAG - 1) / kTcAG;
    L.nkd = (P.dmax + 7) / 8;
    L.n_items = L.rpt * L.nag * L.nkd;
    L.offItems = o;
    o += (uint32_t)L.n_items * 4;
    o = (o + 7) & ~7u;
    L.offMbar = o;
    o += 8;
    L.offTmem = o;
    o += 8;
    L.total = o;
    return L;
}

__global__ void __launch_bounds__(kTcThreads) sweep_tc_kernel(KernelParams kp, int mode, const void *vin_arg,
                                                             void *vout_arg, uint8_t *pol_arg, int unused) {
    extern __shared__ __align__(16) unsigned char smem[];
    (void)unused;
    SolveState *st = kp.st;
    Bufs B;
    if (!resolve_bufs(st, mode, vin_arg, vout_arg, pol_arg, B)) return;
    const ProdParams &P = kp.p[0];
    const TcLayout Lo = tc_layout(P);
    const int G = P.G, dmax = P.dmax, rpt = Lo.rpt, rows = Lo.rows, nkc = Lo.nkc;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t nR = P.nS / (uint32_t)G;
    const uint32_t n_tiles = (nR + rpt - 1) / rpt;
    unsigned char *sA = smem;
    unsigned char *sB = smem + Lo.offB;
    float *s_p = (float *)(smem + Lo.offP);
    uint32_t *s_path = (uint32_t *)(smem + Lo.offPath);
    float *s_q = (float *)(smem + Lo.offQ);
    float *s_bh = (float *)(smem + Lo.offBh);
    float2 *s_ref = (float2 *)(smem + Lo.offRef);
    float2 *s_r0 = (float2 *)(smem + Lo.offR0);
    int *s_R = (int *)(smem + Lo.offR);
    int *s_dig = (int *)(smem + Lo.offDig);
    uint64_t *s_mbar = (uint64_t *)(smem + Lo.offMbar);
    uint32_t *s_tmem = (uint32_t *)(smem + Lo.offTmem);
    const float *tab = (const float *)kp.tables;
    const float2 *V2 = (const float2 *)B.vin;
    const float gam = (float)kp.gamma;
    const float c_o = (float)P.c_o;
    const int plen = dmax + 1;

    // ---- set-up: pmf, W = p[x + k] split into three bf16 planes, tensor memory
    for (int i = tid; i < Lo.pn_pad; i += kTcThreads) s_p[i] = (i < P.pn) ? tab[P.off_p + i] : 0.f;
    __syncthreads();
    for (int i = tid; i < kTcCols * Lo.kpad; i += kTcThreads) {
        const int x = i / Lo.kpad, c = i - x * Lo.kpad;   // column c holds k = c + 1
        const int pi = x + c + 1;
        const float w = (x < G && pi <= dmax) ? s_p[pi] : 0.f;
        uint32_t b1, b2, b3;
        split3(w, b1, b2, b3);
        const uint32_t off = umma_off(x, c, nkc);
        *(unsigned short *)(sB + off) = (unsigned short)(b1 >> 16);
        *(unsigned short *)(sB + Lo.planeB + off) = (unsigned short)(b2 >> 16);
        *(unsigned short *)(sB + 2 * Lo.planeB + off) = (unsigned short)(b3 >> 16);
    }
    // rows past rpt * G and columns past k = dmax never hold data: zero them once
    for (int i = tid; i < kTcRows * Lo.kpad; i += kTcThreads) {
        const int row = i / Lo.kpad, c = i - row * Lo.kpad;
        if (row < rows && c < dmax) continue;
        const uint32_t off = umma_off(row, c, nkc);
#pragma unroll
        for (int pl = 0; pl < 3; ++pl) *(unsigned short *)(sA + pl * Lo.planeA + off) = 0;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(s_mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    const uint32_t idesc = umma_idesc_bf16(kTcRows, kTcCols);
    const uint32_t sbo = (uint32_t)nkc * 128u;

    // staging work items (rest, group of kTcAG orders, chunk of 8 demands), packed once
    uint32_t *s_items = (uint32_t *)(smem + Lo.offItems);
    for (int it = tid; it < Lo.n_items; it += kTcThreads) {
        const int jj = it % rpt, rest = it / rpt;
        const int ag = rest % Lo.nag, kc = rest / Lo.nag;
        const int a0 = ag * kTcAG, a1 = min(G, a0 + kTcAG);
        s_items[it] = (uint32_t)jj | ((uint32_t)a0 << 8) | ((uint32_t)a1 << 16) | ((uint32_t)kc << 24);
    }
    __syncthreads();
    // fixed roles of this thread: accumulator row (order ra, rest rj) and output state (rest oj, slot ox)
    const int ra = tid / rpt, rj = tid - ra * rpt;
    const int oj = tid / G, ox = tid - oj * G;
    const bool row_ok = tid < rows;

    float mx = -INFINITY, mn = INFINITY;
    uint32_t parity = 0;
    bool fault = false;
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint32_t r0 = tile * (uint32_t)rpt;
        // ---- rest digits and stock (-1: past the last rest)
        if (tid < rpt) {
            const uint32_t r = r0 + tid;
            int R = 0;
            uint32_t rem = r;
            for (int i = 0; i < P.n_rest_slots; ++i) {
                const uint32_t q = rem / (uint32_t)G;
                const int dg = (int)(rem - q * (uint32_t)G);
                rem = q;
                s_dig[tid * kMaxDigits + i] = dg;
                R += dg;
            }
            s_R[tid] = (r < nR) ? R : -1;
        }
        __syncthreads();
        // ---- FIFO demand path of each rest: next-state index after e units (the order on top
        // excluded); a rest past the end gets index 0 so that its (unused) row reads valid memory
        for (int j = 0; j < rpt; ++j) {
            const int R = s_R[j];
            const int ecap = min(max(R, 0), dmax);
            for (int e = tid; e <= ecap; e += kTcThreads) {
                uint32_t idx = (R < 0) ? 0u : r0 + (uint32_t)j, w = 1u;
                int left = (R < 0) ? 0 : e;
                for (int sl = 0; sl < P.n_rest_slots && left > 0; ++sl) {
                    const int c = min(left, s_dig[j * kMaxDigits + sl]);
                    idx -= (uint32_t)c * w;
                    left -= c;
                    w *= (uint32_t)G;
                }
                s_path[j * plen + e] = idx;
            }
        }
        __syncthreads();
        // ---- staging: differences g_a(min(k, R)) - g_a(0), split into three bf16 planes.
        // Columns past dmax meet zero probabilities: any finite value will do there.
        for (int it = tid; it < Lo.n_items; it += kTcThreads) {
            const uint32_t code = s_items[it];
            const int jj = (int)(code & 0xFFu), a0 = (int)((code >> 8) & 0xFFu), a1 = (int)((code >> 16) & 0xFFu);
            const int kc = (int)(code >> 24);
            const int ecap = min(max(s_R[jj], 0), dmax);
            const uint32_t *path = s_path + jj * plen;
            uint32_t idx[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) idx[i] = path[min(kc * 8 + i + 1, ecap)];
            const bool on = s_R[jj] >= 0;
            // every gather of the item first (kTcAG orders x 8 demands and the references),
            // so that their latencies overlap; orders past a1 repeat the last one
            float2 ref[kTcAG], raw[kTcAG][8];
#pragma unroll
            for (int u = 0; u < kTcAG; ++u) {
                const int aa = min(a0 + u, a1 - 1);
                const float2 *Va = V2 + (size_t)aa * P.w_top;
                ref[u] = on ? __ldg(Va + path[0]) : make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < 8; ++i) raw[u][i] = __ldg(Va + idx[i]);
            }
#pragma unroll
            for (int u = 0; u < kTcAG; ++u) {
                const int aa = a0 + u;
                if (aa >= a1) break;
                const int row = aa * rpt + jj;
                if (kc == 0) {
                    s_ref[row] = ref[u];
                    if (aa == 0) s_r0[jj] = ref[u];
                }
                uint32_t p1[4], p2[4], p3[4];
#pragma unroll
                for (int i = 0; i < 8; i += 2) {
                    uint32_t a1b, a2b, a3b, b1b, b2b, b3b;
                    split3(pair_diff(raw[u][i], ref[u]), a1b, a2b, a3b);
                    split3(pair_diff(raw[u][i + 1], ref[u]), b1b, b2b, b3b);
                    p1[i / 2] = __byte_perm(a1b, b1b, 0x7632);
                    p2[i / 2] = __byte_perm(a2b, b2b, 0x7632);
                    p3[i / 2] = __byte_perm(a3b, b3b, 0x7632);
                }
                const uint32_t off = umma_off(row, kc * 8, nkc);
                *(uint4 *)(sA + off) = make_uint4(p1[0], p1[1], p1[2], p1[3]);
                *(uint4 *)(sA + Lo.planeA + off) = make_uint4(p2[0], p2[1], p2[2], p2[3]);
                *(uint4 *)(sA + 2 * Lo.planeA + off) = make_uint4(p3[0], p3[1], p3[2], p3[3]);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- six split products, smallest first, K in steps of 16
        if (tid == 0 && !kp.tc_stall) {
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
            const int pa[6] = {2, 1, 0, 1, 0, 0};
            const int pb[6] = {0, 1, 2, 0, 1, 0};
            uint32_t acc = 0;
#pragma unroll
            for (int pr = 0; pr < 6; ++pr) {
                for (int ks = 0; ks < Lo.kpad / 16; ++ks) {
                    const uint64_t da = umma_desc(a0 + pa[pr] * Lo.planeA + ks * 256, 128, sbo);
                    const uint64_t db = umma_desc(b0 + pb[pr] * Lo.planeB + ks * 256, 128, sbo);
                    umma_bf16(tmem, da, db, idesc, acc);
                    acc = 1;
                }
            }
            umma_commit(smem_u32(s_mbar));
        }
        bool done = false;
        const long polls = kp.tc_stall ? 4096 : kTcMaxPolls;
        for (long it = 0; it < polls && !done; ++it) done = mbar_try_wait(smem_u32(s_mbar), parity);
        parity ^= 1u;
        if (__syncthreads_or(!done)) {
            fault = true;
            break;
        }
        tc_fence_after();
        // ---- accumulator row (ra, rj) -> gamma * C + base, transposed into (rest, x, order)
        float c[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), c);
        if (row_ok && s_R[rj] >= 0) {
            float Bh, Bl;
            action_base(gam, s_ref[tid], s_r0[rj], __fmul_rn(-c_o, (float)ra), Bh, Bl);
            s_bh[rj * G + ra] = Bh;
            float *q = s_q + (rj * G) * G + ra;
#pragma unroll
            for (int x = 0; x < kTcCols; ++x)
                if (x < G) q[x * G] = __fmaf_rn(gam, c[x], Bl);
        }
        tc_fence_before();
        __syncthreads();
        // ---- first argmax over orders per state (oj, ox); the reward does not depend on the order (L >= 2)
        if (row_ok) {
            const int R = s_R[oj];
            if (R >= 0) {
                const float *q = s_q + (oj * G + ox) * G;
                const float *bhv = s_bh + oj * G;
                float bh = -INFINITY, bl = 0.f;
                int arg = 0;
                for (int aa = 0; aa < G; ++aa) {
                    const float h = bhv[aa], l = q[aa];
                    const float diff = __fadd_rn(__fsub_rn(h, bh), __fsub_rn(l, bl));
                    const bool up = diff > 0.f;
                    bh = up ? h : bh;
                    bl = up ? l : bl;
                    arg = up ? aa : arg;
                }
                pair_add(bh, bl, __ldg(tab + P.off_RT + R * G + ox), __ldg(tab + P.off_RTlo + R * G + ox));
                const uint32_t s = (r0 + (uint32_t)oj) * (uint32_t)G + (uint32_t)ox;
                const float2 *vin2 = (const float2 *)B.vin;
                float2 *vout2 = (float2 *)B.vout;
                if (mode == MODE_EXTRACT) {
                    if (vout2) vout2[s] = vin2[s];
                } else {
                    const float2 vnew = pair_finish(gam, s_r0[oj], bh, bl);
                    const float2 vold = vin2[s];
                    vout2[s] = vnew;
                    const float dlt = pair_diff(vnew, vold);
                    mx = fmaxf(mx, dlt);
                    mn = fminf(mn, dlt);
                }
                if (B.pol) B.pol[s] = (uint8_t)arg;
            }
        }
        __syncthreads();   // paths, transposed values and operand planes are rewritten by the next tile
    }
    if (fault && tid == 0) atomicExch(&st->fault, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
    if (mode != MODE_EXTRACT) block_reduce_and_finalize<float>(mx, mn, st, mode, gridDim.x);
}

bool tc_supported(const KernelParams &kp, int vk, int kahan) {
    const ProdParams &P = kp.p[0];
    if (kp.n_products != 1 || vk != VK_PAIR || kahan || kp.issuing != 0) return false;
    if (P.L < 2 || P.m < 2 || P.G < 2 || P.G > kTcCols || P.K < 2 || P.n_rest_slots < 1) return false;
    if (P.dmax < 1 || P.dmax > 127 || P.n_rest_slots > kMaxDigits) return false;
    return tc_layout(P).total <= 200 * 1024;
}

cudaError_t describe_tc(const KernelParams &kp, LaunchDesc &d) {
    const TcLayout Lo = tc_layout(kp.p[0]);
    d.fn = (const void *)sweep_tc_kernel;
    d.block = dim3(kTcThreads);
    d.smem = Lo.total;
    d.lpr = 0;
    cudaError_t e = cudaFuncSetAttribute(sweep_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int dev = 0, n_sm = 0, smem_sm = 0, smem_rsv = 0, regs_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess)
        return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, sweep_tc_kernel)) != cudaSuccess) return e;
    // resident blocks per SM from shared memory and registers (each block holds 32 tensor-memory columns)
    const int by_smem = smem_sm / (int)(d.smem + smem_rsv);
    const int by_regs = regs_sm / std::max(1, fa.numRegs * kTcThreads);
    const int per_sm = std::min(std::min(by_smem, by_regs), 512 / kTcCols);
    const uint32_t nR = kp.p[0].nS / (uint32_t)kp.p[0].G;
    const uint32_t n_tiles = (nR + Lo.rpt - 1) / Lo.rpt;
    const uint32_t resident = (uint32_t)std::max(1, n_sm * std::max(1, per_sm));
    d.grid = dim3(std::min(n_tiles, resident));
    return cudaSuccess;
}

}  // namespace vib

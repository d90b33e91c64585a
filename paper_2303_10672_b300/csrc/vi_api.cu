// vi_api.cu -- host side of the C ABI declared in include/vi.h.
//
// A handle owns: the FP64-built expectation tables (uploaded as float and as
// double blobs), the device SolveState, the scratch half of the value ping-pong,
// and a CUDA graph of the solve loop: init -> while(keep_going) { sweep } ->
// extraction.  The sweep kernel's last block evaluates the stopping test on the
// device and sets the while-node's condition, so a solve costs one graph launch
// and one small read-back.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/vi.h"
#include "vi_api_internal.h"
#include "vi_pool.h"
#include "vi_common.cuh"
#include "vi_kernels.h"

using namespace vib;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

vi_status vi_fail(vi_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

#define CUDA_TRY(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return vi_fail(e_ == cudaErrorMemoryAllocation ? VI_ENOMEM : VI_ECUDA, "%s: %s (%s:%d)", \
                           #call, cudaGetErrorString(e_), __FILE__, __LINE__);                  \
    } while (0)

extern "C" const char *vi_status_string(vi_status s) {
    switch (s) {
        case VI_OK: return "ok";
        case VI_EINVAL: return "invalid argument";
        case VI_ENOMEM: return "out of memory";
        case VI_ENOTCONVERGED: return "not converged within max_iters";
        case VI_ETIMEOUT: return "device wait timed out";
        case VI_EBUSY: return "busy / over memory budget";
        case VI_ECUDA: return "CUDA error";
        case VI_ECANCELLED: return "cancelled";
    }
    return "unknown status";
}

extern "C" const char *vi_last_error(void) { return g_err; }

// ---------------------------------------------------------------------------
// table construction (FP64 on the host)
// ---------------------------------------------------------------------------
static int ceil_log2(int g) {
    int b = 0;
    while ((1 << b) < g) ++b;
    return b;
}

struct HostTables {
    std::vector<double> blob;
};

// expected leftover E[(y - D)^+]
static std::vector<double> expected_leftover(const std::vector<double> &pmf, int ymax) {
    std::vector<double> g(ymax + 1, 0.0);
    for (int y = 0; y <= ymax; ++y) {
        double s = 0.0;
        for (int d = 0; d < (int)pmf.size() && d < y; ++d) s += pmf[d] * (double)(y - d);
        g[y] = s;
    }
    return g;
}

static void fill_product_tables(ProdParams &P, const std::vector<double> &pmf, int issuing, const double *cost,
                                bool with_reward, std::vector<double> &blob) {
    const int dmax = P.dmax;
    P.pn = p_table_len(dmax, P.tmax, P.G);
    P.off_p = (int)blob.size();
    for (int k = 0; k < P.pn; ++k) blob.push_back(k <= dmax ? pmf[k] : 0.0);
    P.off_F = (int)blob.size();
    double c = 0.0;
    for (int k = 0; k < P.pn; ++k) {
        if (k <= dmax) c += pmf[k];
        blob.push_back(c);
    }
    P.off_tail = (int)blob.size();
    std::vector<double> tail(P.pn, 0.0);
    double t = 0.0;
    for (int k = dmax; k >= 0; --k) {
        t += pmf[k];
        tail[k] = t;
    }
    for (int k = 0; k < P.pn; ++k) blob.push_back(tail[k]);
    P.off_RT = P.off_RTlo = 0;
    P.rt_rows = (P.m - 1) * P.Q + 1;
    if (!with_reward) return;
    // RT[R][y1]: expected one-step reward without the order cost, given y1 units in
    // the expiring slot and R units in the other slots (T = y1 + R available):
    //   (c_s + c_r) T - c_s E[D] - (c_h + c_s + c_r) E[(T-D)^+] + (c_h - c_w) E[W]
    // with E[W] = E[(y1-D)^+] (FIFO) or E[(T-D)^+] - E[(R-D)^+] (LIFO).
    const double c_h = cost[1], c_s = cost[2], c_w = cost[3], c_r = cost[4];
    double mu = 0.0;
    for (int d = 0; d <= dmax; ++d) mu += (double)d * pmf[d];
    std::vector<double> G = expected_leftover(pmf, P.tmax);
    std::vector<double> rt((size_t)P.rt_rows * P.G);
    for (int R = 0; R < P.rt_rows; ++R)
        for (int y1 = 0; y1 < P.G; ++y1) rt[(size_t)R * P.G + y1] = expected_period_reward(y1, R, G.data(), mu, cost, issuing);
    P.off_RT = (int)blob.size();
    blob.insert(blob.end(), rt.begin(), rt.end());
    P.off_RTlo = (int)blob.size();
    for (double v : rt) blob.push_back(v - (double)(float)v);
    P.off_LF = P.off_LH = 0;
    if (issuing == VI_LIFO) {
        // the same expected reward split as LF(T) + LH(R), T = y1 + R:
        //   LF(T) = (c_s + c_r) T - c_s E[D] - (c_s + c_r + c_w) E[(T-D)^+],  LH(R) = (c_w - c_h) E[(R-D)^+]
        P.off_LF = (int)blob.size();
        for (int T = 0; T <= P.tmax; ++T) blob.push_back((c_s + c_r) * T - c_s * mu - (c_s + c_r + c_w) * G[T]);
        P.off_LH = (int)blob.size();
        for (int R = 0; R < P.rt_rows; ++R) blob.push_back((c_w - c_h) * G[R]);
    }
}

static double binom(int n, int k, double rho) {
    double c = 1.0;
    for (int i = 1; i <= k; ++i) c = c * (double)(n - k + i) / (double)i;
    return c * pow(rho, (double)k) * pow(1.0 - rho, (double)(n - k));
}

// two-product extras: substitution mixture rows M and the expected-reward tables H1, H2
static void fill_two_product_tables(KernelParams &kp, const vi_problem_desc &d, const std::vector<double> &pm1,
                                    const std::vector<double> &pm2, std::vector<double> &blob) {
    ProdParams &P1 = kp.p[0], &P2 = kp.p[1];
    const int D1 = P1.dmax, D2 = P2.dmax;
    const int zl = D1 + D2 + 1;
    kp.zlen = zl;
    const double rho = d.subst_rate;
    // conv[n][z] = P(d2 + Bin(n, rho) = z)
    std::vector<double> conv((size_t)(D1 + 1) * zl, 0.0);
    for (int n = 0; n <= D1; ++n)
        for (int u = 0; u <= n; ++u) {
            double b = binom(n, u, rho);
            for (int d2 = 0; d2 <= D2; ++d2) conv[(size_t)n * zl + d2 + u] += pm2[d2] * b;
        }
    const int nT1 = P1.tmax + 1;
    std::vector<double> M((size_t)nT1 * zl, 0.0);
    for (int T1 = 0; T1 < nT1; ++T1)
        for (int d1 = T1; d1 <= D1; ++d1)
            for (int z = 0; z < zl; ++z) M[(size_t)T1 * zl + z] += pm1[d1] * conv[(size_t)(d1 - T1) * zl + z];
    kp.off_M = (int)blob.size();
    blob.insert(blob.end(), M.begin(), M.end());
    kp.off_Mc = (int)blob.size();
    for (int T1 = 0; T1 < nT1; ++T1) {
        double c = 0.0;
        for (int z = 0; z < zl; ++z) {
            c += M[(size_t)T1 * zl + z];
            blob.push_back(c);
        }
    }
    kp.off_Mt = (int)blob.size();
    for (int T1 = 0; T1 < nT1; ++T1) {
        std::vector<double> t(zl, 0.0);
        double c = 0.0;
        for (int z = zl - 1; z >= 0; --z) {
            c += M[(size_t)T1 * zl + z];
            t[z] = c;
        }
        blob.insert(blob.end(), t.begin(), t.end());
    }
    const double *c1 = d.cost[0], *c2 = d.cost[1];
    const int lifo = d.issuing == VI_LIFO;
    // H1[ys1][T1]: product-1 holding, waste and revenue (ys1 = Y_1 for FIFO, R for LIFO)
    kp.off_H1 = (int)blob.size();
    for (int ys = 0; ys < nT1; ++ys)
        for (int T1 = 0; T1 < nT1; ++T1) {
            double h = 0.0;
            int y1 = lifo ? T1 - ys : ys;
            if (y1 >= 0 && y1 <= T1) {
                int R = T1 - y1;
                for (int d1 = 0; d1 <= D1; ++d1) {
                    int iss = std::min(d1, T1);
                    int W = lifo ? y1 - std::min(y1, std::max(d1 - R, 0)) : std::max(y1 - d1, 0);
                    int car = T1 - iss - W;
                    h += pm1[d1] * (-c1[1] * car - c1[3] * W + c1[4] * iss);
                }
            }
            blob.push_back(h);
        }
    // H2[T1][ys2][T2]: product-2 terms with substitution + product-1 shortage
    const size_t h1_begin = (size_t)kp.off_H1, h1_len = blob.size() - h1_begin;
    kp.off_H2 = (int)blob.size();
    const int nT2 = P2.tmax + 1;
    const int ny2 = lifo ? nT2 : P2.G;
    std::vector<double> Pz((size_t)nT1 * zl, 0.0);
    std::vector<double> En1(nT1, 0.0);
    for (int T1 = 0; T1 < nT1; ++T1) {
        double below = 0.0;
        for (int d1 = 0; d1 <= D1 && d1 < T1; ++d1) below += pm1[d1];
        for (int z = 0; z < zl; ++z) {
            double own = (z <= D2) ? pm2[z] : 0.0;
            Pz[(size_t)T1 * zl + z] = below * own + M[(size_t)T1 * zl + z];
        }
        for (int d1 = T1; d1 <= D1; ++d1) En1[T1] += pm1[d1] * (double)(d1 - T1);
    }
    for (int T1 = 0; T1 < nT1; ++T1)
        for (int ys = 0; ys < ny2; ++ys)
            for (int T2 = 0; T2 < nT2; ++T2) {
                int y2 = lifo ? T2 - ys : ys;
                double h = 0.0;
                if (y2 >= 0 && y2 <= T2) {
                    int R2 = T2 - y2;
                    double eshort2 = 0.0, emin2 = 0.0;
                    for (int d2 = 0; d2 <= D2; ++d2) {
                        eshort2 += pm2[d2] * (double)std::max(d2 - T2, 0);
                        emin2 += pm2[d2] * (double)std::min(d2, T2);
                    }
                    for (int z = 0; z < zl; ++z) {
                        double pz = Pz[(size_t)T1 * zl + z];
                        if (pz == 0.0) continue;
                        int iss = std::min(z, T2);
                        int W = lifo ? y2 - std::min(y2, std::max(z - R2, 0)) : std::max(y2 - z, 0);
                        int car = T2 - iss - W;
                        h += pz * (-c2[1] * car - c2[3] * W + (c2[4] + c1[2]) * iss);
                    }
                    h += -c2[2] * eshort2 - c1[2] * (En1[T1] + emin2);   // short1 = n1 - iss2 + own2
                }
                blob.push_back(h);
            }
    // low halves for the float-pair kernels
    const size_t h2_begin = (size_t)kp.off_H2, h2_len = blob.size() - h2_begin;
    kp.off_H1lo = (int)blob.size();
    for (size_t i = 0; i < h1_len; ++i) {
        const double v = blob[h1_begin + i];
        blob.push_back(v - (double)(float)v);
    }
    kp.off_H2lo = (int)blob.size();
    for (size_t i = 0; i < h2_len; ++i) {
        const double v = blob[h2_begin + i];
        blob.push_back(v - (double)(float)v);
    }
}

// ---------------------------------------------------------------------------
// problem creation
// ---------------------------------------------------------------------------
static vi_status validate_product(int m, int L, int Q, const double *cost, const double *pmf, int dmax) {
    if (m < 1 || L < 1 || Q < 0) return vi_fail(VI_EINVAL, "need m >= 1, L >= 1, Q >= 0 (got %d, %d, %d)", m, L, Q);
    if (Q + 1 > 256) return vi_fail(VI_EINVAL, "Q+1 = %d actions exceeds the uint8 policy", Q + 1);
    if (dmax < 0 || dmax > kMaxDmax) return vi_fail(VI_EINVAL, "dmax %d outside 0..%d", dmax, kMaxDmax);
    if (!cost || !pmf) return vi_fail(VI_EINVAL, "null cost or pmf");
    for (int j = 0; j < 5; ++j)
        if (!(cost[j] >= 0.0) || !isfinite(cost[j])) return vi_fail(VI_EINVAL, "cost[%d] must be finite and >= 0", j);
    double s = 0.0;
    for (int d = 0; d <= dmax; ++d) {
        if (!(pmf[d] >= 0.0) || !isfinite(pmf[d])) return vi_fail(VI_EINVAL, "pmf[%d] must be >= 0", d);
        s += pmf[d];
    }
    if (fabs(s - 1.0) > 1e-12) return vi_fail(VI_EINVAL, "pmf sums to %.17g, not 1", s);
    int K = (m - 1) + (L - 1);
    double ns = pow((double)(Q + 1), (double)K);
    if (ns >= 4294967296.0 || K > kMaxDigits) return vi_fail(VI_EINVAL, "|S| = (Q+1)^%d does not fit 32 bits", K);
    return VI_OK;
}

// product 0's pmf and -P(D > x) in FP32 for the sweeps that read them from the
// parameter constant bank (zero past dmax; P(D > x) summed from the top in FP64)
static void fill_pmf_consts(KernelParams &kp, const double *pmf, int dmax) {
    constexpr int n = (int)(sizeof(kp.pmf32) / sizeof(kp.pmf32[0]));
    for (int i = 0; i < n; ++i) kp.pmf32[i] = (i <= dmax) ? (float)pmf[i] : 0.f;
    for (int x = 0; x < n; ++x) kp.nsurv32[x] = 0.f;
    double t = 0.0;
    for (int x = dmax - 1; x >= 0; --x) {
        t += pmf[x + 1];
        if (x < n) kp.nsurv32[x] = -(float)t;
    }
}

void fill_prod_params(ProdParams &P, int m, int L, int Q, int dmax, double c_o) {
    memset(&P, 0, sizeof(P));
    P.m = m;
    P.L = L;
    P.Q = Q;
    P.G = Q + 1;
    P.K = (m - 1) + (L - 1);
    P.dmax = dmax;
    P.tmax = m * Q;
    P.cb = ceil_log2(P.G);
    uint64_t n = 1;
    for (int k = 0; k < P.K; ++k) n *= (uint64_t)P.G;
    P.nS = (uint32_t)n;
    uint64_t wt = 1;
    for (int k = 0; k + 1 < P.K; ++k) wt *= (uint64_t)P.G;
    P.w_top = P.K >= 1 ? (uint32_t)wt : 0u;
    P.n_rest_slots = (L >= 2) ? (m - 1) : std::max(m - 2, 0);
    uint64_t wz = 1;
    for (int k = 0; k + 2 <= m - 1; ++k) wz *= (uint64_t)P.G;   // G^(m-2)
    P.w_zt = (uint32_t)wz;
    P.c_o = c_o;
    // exact division by G (Granlund and Montgomery's round-up constants, see DivG)
    const int l = ceil_log2(P.G);
    P.g_mag = (uint32_t)((((uint64_t)1 << 32) * (((uint64_t)1 << l) - (uint64_t)P.G)) / (uint64_t)P.G + 1u);
    P.g_sh1 = l < 1 ? l : 1;
    P.g_sh2 = l > 1 ? l - 1 : 0;
}

vi_status build_single_product(const vi_problem_desc &d, KernelParams &kp, std::vector<float> &ftab,
                               int &n_outcomes) {
    vi_status s = validate_product(d.m[0], d.L[0], d.Q[0], d.cost[0], d.pmf[0], d.dmax[0]);
    if (s != VI_OK) return s;
    if (!(d.gamma > 0.0 && d.gamma <= 1.0)) return vi_fail(VI_EINVAL, "gamma must be in (0, 1]");
    if (d.issuing != VI_FIFO && d.issuing != VI_LIFO) return vi_fail(VI_EINVAL, "issuing must be FIFO or LIFO");
    memset(&kp, 0, sizeof(kp));
    kp.n_products = 1;
    kp.issuing = d.issuing;
    kp.gamma = d.gamma;
    std::vector<double> pm(d.pmf[0], d.pmf[0] + d.dmax[0] + 1);
    std::vector<double> blob;
    fill_prod_params(kp.p[0], d.m[0], d.L[0], d.Q[0], d.dmax[0], d.cost[0][0]);
    fill_product_tables(kp.p[0], pm, d.issuing, d.cost[0], true, blob);
    fill_pmf_consts(kp, pm.data(), d.dmax[0]);
    kp.nS = kp.p[0].nS;
    kp.nA = kp.p[0].G;
    kp.n_tables = (int)blob.size();
    kp.tab_in_smem = ((size_t)kp.n_tables * 8 <= 160 * 1024) ? 1 : 0;
    n_outcomes = d.dmax[0] + 1;
    ftab.resize(blob.size());
    for (size_t i = 0; i < blob.size(); ++i) ftab[i] = (float)blob[i];
    return VI_OK;
}

static void destroy_internal(vi_problem *h);

extern "C" vi_status vi_problem_create_desc(const vi_problem_desc *desc, vi_handle *out) {
    if (!desc || !out) return vi_fail(VI_EINVAL, "null desc or out");
    *out = nullptr;
    const vi_problem_desc &d = *desc;
    if (d.n_products != 1 && d.n_products != 2) return vi_fail(VI_EINVAL, "n_products must be 1 or 2");
    for (int k = 0; k < d.n_products; ++k) {
        vi_status s = validate_product(d.m[k], d.L[k], d.Q[k], d.cost[k], d.pmf[k], d.dmax[k]);
        if (s != VI_OK) return s;
    }
    if (!(d.gamma > 0.0 && d.gamma <= 1.0)) return vi_fail(VI_EINVAL, "gamma must be in (0, 1]");
    if (d.issuing != VI_FIFO && d.issuing != VI_LIFO) return vi_fail(VI_EINVAL, "issuing must be FIFO or LIFO");
    if (d.precision < VI_PREC_FP32 || d.precision > VI_PREC_FP32_SINGLE) return vi_fail(VI_EINVAL, "bad precision");
    if (d.stop_rule != VI_STOP_SPAN && d.stop_rule != VI_STOP_SUPNORM) return vi_fail(VI_EINVAL, "bad stop_rule");
    if (d.n_products == 2) {
        if ((d.Q[0] + 1) * (d.Q[1] + 1) > 256) return vi_fail(VI_EINVAL, "joint actions exceed 256");
        if (!(d.subst_rate >= 0.0 && d.subst_rate <= 1.0)) return vi_fail(VI_EINVAL, "subst_rate in [0,1]");
        double ns = 1.0;
        for (int k = 0; k < 2; ++k) ns *= pow((double)(d.Q[k] + 1), (double)(d.m[k] - 1));
        if (ns >= 4294967296.0) return vi_fail(VI_EINVAL, "|S| does not fit 32 bits");
        if (d.dmax[0] > 255 || d.dmax[1] > 255) return vi_fail(VI_EINVAL, "two products need dmax <= 255");
    }

    vi_problem *h = new (std::nothrow) vi_problem();
    if (!h) return vi_fail(VI_ENOMEM, "host allocation failed");
    h->desc = d;
    for (int k = 0; k < d.n_products; ++k) {
        h->pmf[k].assign(d.pmf[k], d.pmf[k] + d.dmax[k] + 1);
        h->desc.pmf[k] = h->pmf[k].data();
    }
    KernelParams &kp = h->kp;
    memset(&kp, 0, sizeof(kp));
    kp.n_products = d.n_products;
    kp.issuing = d.issuing;
    kp.gamma = d.gamma;
    std::vector<double> blob;
    for (int k = 0; k < d.n_products; ++k) {
        fill_prod_params(kp.p[k], d.m[k], d.L[k], d.Q[k], d.dmax[k], d.cost[k][0]);
        fill_product_tables(kp.p[k], h->pmf[k], d.issuing, d.cost[k], d.n_products == 1, blob);
    }
    fill_pmf_consts(kp, h->pmf[0].data(), d.dmax[0]);
    if (d.n_products == 1) {
        kp.nS = kp.p[0].nS;
        kp.nA = kp.p[0].G;
        h->n_outcomes = d.dmax[0] + 1;
    } else {
        fill_two_product_tables(kp, d, h->pmf[0], h->pmf[1], blob);
        kp.nS = kp.p[0].nS * kp.p[1].nS;
        kp.nA = kp.p[0].G * kp.p[1].G;
        h->n_outcomes = (d.dmax[0] + 1) * (d.dmax[1] + 1);
    }
    kp.n_tables = (int)blob.size();
    // generic kernels stage the tables in shared memory when they fit (FP64 size)
    const int n_smem = (d.n_products == 2) ? kp.off_H1 : kp.n_tables;
    kp.tab_in_smem = ((size_t)n_smem * 8 <= 160 * 1024) ? 1 : 0;
    h->vk = (d.precision == VI_PREC_FP64) ? VK_DOUBLE : (d.precision == VI_PREC_FP32_SINGLE) ? VK_SINGLE : VK_PAIR;
    h->kahan = (d.precision == VI_PREC_FP32_KAHAN) ? 1 : 0;
    h->value_bytes = (h->vk == VK_SINGLE) ? 4 : 8;
    h->group_ok = group_supported(kp, h->vk, h->kahan);
    h->two_ok = two_supported(kp, h->vk, h->kahan);
    h->group_xw = 0;   // chosen by the autotuner on the first solve (or set explicitly)
    std::vector<float> fblob(blob.size());
    for (size_t i = 0; i < blob.size(); ++i) fblob[i] = (float)blob[i];

    cudaError_t e;
    if ((e = vip::dev_alloc_t(&h->d_tab_f, fblob.size() * sizeof(float))) != cudaSuccess ||
        (e = vip::dev_alloc_t(&h->d_tab_d, blob.size() * sizeof(double))) != cudaSuccess ||
        (e = vip::dev_alloc_t(&h->d_state, sizeof(SolveState))) != cudaSuccess ||
        (e = vip::host_alloc((void **)&h->h_state, sizeof(SolveState))) != cudaSuccess ||
        (e = cudaMemcpy(h->d_tab_f, fblob.data(), fblob.size() * sizeof(float), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(h->d_tab_d, blob.data(), blob.size() * sizeof(double), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaEventCreate(&h->ev0)) != cudaSuccess || (e = cudaEventCreate(&h->ev1)) != cudaSuccess) {
        destroy_internal(h);
        return vi_fail(e == cudaErrorMemoryAllocation ? VI_ENOMEM : VI_ECUDA, "problem setup: %s",
                       cudaGetErrorString(e));
    }
    memset(h->h_state, 0, sizeof(SolveState));
    h->h_state->key_min = ~0ull;
    if ((e = cudaMemcpy(h->d_state, h->h_state, sizeof(SolveState), cudaMemcpyHostToDevice)) != cudaSuccess) {
        destroy_internal(h);
        return vi_fail(VI_ECUDA, "state upload: %s", cudaGetErrorString(e));
    }
    if (h->two_ok) {
        size_t n_mix = 0;
        const size_t n_e2 = two_table_floats(kp, &n_mix);
        if ((e = vip::dev_alloc_t(&h->d_two_e2, n_e2 * sizeof(float))) != cudaSuccess ||
            (e = vip::dev_alloc_t(&h->d_two_mix, n_mix * sizeof(float))) != cudaSuccess) {
            destroy_internal(h);
            return vi_fail(e == cudaErrorMemoryAllocation ? VI_ENOMEM : VI_ECUDA, "two-product tables: %s",
                           cudaGetErrorString(e));
        }
        kp.two_e2 = h->d_two_e2;
        kp.two_mix = h->d_two_mix;
        if (kp.p[0].L >= 2) {
            // rests r1 of product 1 ordered by the units they hold (digits of the
            // n_rest_slots stock slots), so that a warp's lanes share one path length
            const ProdParams &P1 = kp.p[0];
            const uint32_t nr = P1.nS / (uint32_t)P1.G;
            std::vector<uint32_t> perm(nr), tot(nr);
            for (uint32_t r = 0; r < nr; ++r) {
                uint32_t rem = r, sum = 0;
                for (int j = 0; j < P1.n_rest_slots; ++j) {
                    sum += rem % (uint32_t)P1.G;
                    rem /= (uint32_t)P1.G;
                }
                tot[r] = sum;
                perm[r] = r;
            }
            std::stable_sort(perm.begin(), perm.end(), [&](uint32_t a, uint32_t b) { return tot[a] < tot[b]; });
            if ((e = vip::dev_alloc_t(&h->d_two_rperm, nr * sizeof(uint32_t))) != cudaSuccess ||
                (e = cudaMemcpy(h->d_two_rperm, perm.data(), nr * sizeof(uint32_t), cudaMemcpyHostToDevice)) !=
                    cudaSuccess) {
                destroy_internal(h);
                return vi_fail(e == cudaErrorMemoryAllocation ? VI_ENOMEM : VI_ECUDA, "two-product tables: %s",
                               cudaGetErrorString(e));
            }
            kp.two_rperm = h->d_two_rperm;
        }
        kp.two_nt1 = two_mix_rows(kp.p[0]);
        kp.two_npipe1 = 1;
        for (int k = 1; k < kp.p[0].L; ++k) kp.two_npipe1 *= kp.p[0].G;
    }
    kp.st = h->d_state;
    kp.tables = (h->vk == VK_DOUBLE) ? (const void *)h->d_tab_d : (const void *)h->d_tab_f;
    *out = h;
    return VI_OK;
}

// ---------------------------------------------------------------------------
// periodic problems (Scenario C)
// ---------------------------------------------------------------------------
// floor(2^32 CDF) thresholds of a pmf summed in ascending order, last one 2^32
static void pc_thresholds(const double *pmf, int n, unsigned long long *thr) {
    double cdf = 0.0;
    for (int i = 0; i < n; ++i) {
        cdf += pmf[i];
        double t = floor(cdf * 4294967296.0);
        t = t > 4294967296.0 ? 4294967296.0 : (t < 0.0 ? 0.0 : t);
        thr[i] = (unsigned long long)t;
    }
    thr[n - 1] = 4294967296ull;
}

// p_1(a)..p_m(a) of the multinomial life on arrival: log(p_k / p_1) = c0_k + c1_k a
static void pc_arrival_params(const vi_periodic_desc &d, int a, double *p) {
    double e[kPcMaxM + 1];
    double z = 1.0;
    e[1] = 1.0;
    for (int k = 2; k <= d.m; ++k) {
        e[k] = exp(d.c0[k] + d.c1[k] * (double)a);
        z += e[k];
    }
    for (int k = 1; k <= d.m; ++k) p[k] = e[k] / z;
}

extern "C" vi_status vi_problem_create_periodic(const vi_periodic_desc *desc, vi_handle *out) {
    if (!desc || !out) return vi_fail(VI_EINVAL, "null desc or out");
    *out = nullptr;
    const vi_periodic_desc &d = *desc;
    if (d.m < 2 || d.m > kPcMaxM) return vi_fail(VI_EINVAL, "m must be in 2..%d", kPcMaxM);
    if (d.Q < 0 || d.Q > 63) return vi_fail(VI_EINVAL, "A_max must be in 0..63");
    if (d.dmax < 0 || d.dmax > 4095 || !d.pmf) return vi_fail(VI_EINVAL, "bad demand pmf");
    if (!(d.gamma > 0.0 && d.gamma < 1.0)) return vi_fail(VI_EINVAL, "gamma must be in (0, 1)");
    if (d.stop_rule != VI_STOP_SPAN && d.stop_rule != VI_STOP_SUPNORM && d.stop_rule != VI_STOP_PERIODIC)
        return vi_fail(VI_EINVAL, "bad stop_rule");
    for (int j = 0; j < 4; ++j)
        if (!(d.cost[j] >= 0.0)) return vi_fail(VI_EINVAL, "costs must be >= 0");
    for (int t = 0; t < 7; ++t) {
        double sum = 0.0;
        for (int i = 0; i <= d.dmax; ++i) {
            const double v = d.pmf[(size_t)t * (d.dmax + 1) + i];
            if (!(v >= 0.0)) return vi_fail(VI_EINVAL, "negative demand probability");
            sum += v;
        }
        if (fabs(sum - 1.0) > 1e-12) return vi_fail(VI_EINVAL, "weekday %d pmf sums to %.17g", t, sum);
    }
    const int G = d.Q + 1;
    double n_post = 7.0;
    for (int j = 0; j < d.m; ++j) n_post *= G;
    if (n_post / G >= 4294967296.0 || n_post > 2147483648.0)
        return vi_fail(VI_EINVAL, "7 (A_max+1)^m must stay below 2^31");

    vi_problem *h = new (std::nothrow) vi_problem();
    if (!h) return vi_fail(VI_ENOMEM, "host allocation failed");
    h->periodic = true;
    memset(&h->desc, 0, sizeof(h->desc));
    h->desc.n_products = 1;
    h->desc.gamma = d.gamma;
    h->desc.stop_rule = d.stop_rule;
    h->desc.precision = VI_PREC_FP64;
    KernelParams &kp = h->kp;
    memset(&kp, 0, sizeof(kp));
    fill_prod_params(kp.p[0], d.m, 1, d.Q, d.dmax, 0.0);   // m-1 digits: the stock slots
    kp.n_products = 1;
    kp.gamma = d.gamma;
    kp.nS = 7u * kp.p[0].nS;
    kp.nA = G;
    kp.pc = 1;
    kp.pc_m = d.m;
    for (int j = 0; j < 4; ++j) kp.pc_cost[j] = d.cost[j];
    h->vk = VK_DOUBLE;
    h->value_bytes = 8;
    h->group_ok = false;
    h->two_ok = false;

    // arrival profiles by order size (all compositions of a into m classes), their
    // probabilities, and the rollout thresholds
    std::vector<unsigned long long> prof;
    std::vector<double> prob;
    std::vector<int> off(G + 1, 0);
    std::vector<unsigned long long> thr_y((size_t)G * d.m);
    for (int a = 0; a <= d.Q; ++a) {
        off[a] = (int)prof.size();
        double p[kPcMaxM + 1];
        pc_arrival_params(d, a, p);
        pc_thresholds(p + 1, d.m, thr_y.data() + (size_t)a * d.m);
        int y[kPcMaxM + 1] = {0};
        y[1] = a;
        while (true) {
            double coef = 1.0;
            int left = a;
            for (int k = 1; k <= d.m; ++k) {
                double c = 1.0;
                for (int i = 1; i <= y[k]; ++i) c = c * (double)(left - y[k] + i) / (double)i;
                coef *= c;
                left -= y[k];
            }
            double pr = coef;
            for (int k = 1; k <= d.m; ++k) pr *= pow(p[k], (double)y[k]);
            unsigned long long packed = 0;
            for (int k = 1; k <= d.m; ++k) packed |= (unsigned long long)y[k] << (6 * (k - 1));
            prof.push_back(packed);
            prob.push_back(pr);
            // next composition: raise the lowest class k >= 2 with room, reset the ones below
            int k = 2;
            for (; k <= d.m; ++k) {
                int upper = 0;
                for (int j = k; j <= d.m; ++j) upper += y[j];
                if (upper < a) break;
            }
            if (k > d.m) break;
            y[k] += 1;
            for (int j = 2; j < k; ++j) y[j] = 0;
            int rest = 0;
            for (int j = 2; j <= d.m; ++j) rest += y[j];
            y[1] = a - rest;
        }
    }
    off[G] = (int)prof.size();
    std::vector<unsigned long long> thr_d((size_t)7 * (d.dmax + 1));
    for (int t = 0; t < 7; ++t)
        pc_thresholds(d.pmf + (size_t)t * (d.dmax + 1), d.dmax + 1, thr_d.data() + (size_t)t * (d.dmax + 1));
    // the paper's |Omega|: demands x profiles with sum y <= A_max
    h->n_outcomes = (d.dmax + 1) * (int)prof.size();

    const size_t n_pmf = (size_t)7 * (d.dmax + 1);
    cudaError_t e;
    if ((e = vip::dev_alloc_t(&h->d_pc_pmf, n_pmf * sizeof(double))) != cudaSuccess ||
        (e = vip::dev_alloc_t(&h->d_pc_prof, prof.size() * sizeof(unsigned long long))) != cudaSuccess ||
        (e = vip::dev_alloc_t(&h->d_pc_prob, prob.size() * sizeof(double))) != cudaSuccess ||
        (e = vip::dev_alloc_t(&h->d_pc_off, off.size() * sizeof(int))) != cudaSuccess ||
        (e = vip::dev_alloc_t(&h->d_pc_W, (size_t)n_post * sizeof(double))) != cudaSuccess ||
        (e = vip::dev_alloc_t(&h->d_pc_ring, (size_t)7 * kp.nS * sizeof(double))) != cudaSuccess ||
        (e = vip::dev_alloc_t(&h->d_pc_thr_d, thr_d.size() * sizeof(unsigned long long))) != cudaSuccess ||
        (e = vip::dev_alloc_t(&h->d_pc_thr_y, thr_y.size() * sizeof(unsigned long long))) != cudaSuccess ||
        (e = vip::dev_alloc_t(&h->d_state, sizeof(SolveState))) != cudaSuccess ||
        (e = vip::host_alloc((void **)&h->h_state, sizeof(SolveState))) != cudaSuccess ||
        (e = cudaMemcpy(h->d_pc_pmf, d.pmf, n_pmf * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(h->d_pc_prof, prof.data(), prof.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(h->d_pc_prob, prob.data(), prob.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(h->d_pc_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(h->d_pc_thr_d, thr_d.data(), thr_d.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(h->d_pc_thr_y, thr_y.data(), thr_y.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(h->d_pc_ring, 0, (size_t)7 * kp.nS * sizeof(double))) != cudaSuccess ||
        (e = cudaEventCreate(&h->ev0)) != cudaSuccess || (e = cudaEventCreate(&h->ev1)) != cudaSuccess) {
        destroy_internal(h);
        return vi_fail(e == cudaErrorMemoryAllocation ? VI_ENOMEM : VI_ECUDA, "periodic problem setup: %s",
                       cudaGetErrorString(e));
    }
    kp.pc_pmf = h->d_pc_pmf;
    kp.pc_prof = h->d_pc_prof;
    kp.pc_prob = h->d_pc_prob;
    kp.pc_off = h->d_pc_off;
    kp.pc_W = h->d_pc_W;
    kp.pc_ring = h->d_pc_ring;
    memset(h->h_state, 0, sizeof(SolveState));
    h->h_state->key_min = ~0ull;
    if ((e = cudaMemcpy(h->d_state, h->h_state, sizeof(SolveState), cudaMemcpyHostToDevice)) != cudaSuccess) {
        destroy_internal(h);
        return vi_fail(VI_ECUDA, "state upload: %s", cudaGetErrorString(e));
    }
    kp.st = h->d_state;
    *out = h;
    return VI_OK;
}

extern "C" vi_status vi_problem_create(int m, int L, int Q, const double cost[5], const double *pmf, int dmax,
                                       double gamma, int issuing, vi_handle *out) {
    vi_problem_desc d;
    memset(&d, 0, sizeof(d));
    d.n_products = 1;
    d.m[0] = m;
    d.L[0] = L;
    d.Q[0] = Q;
    if (!cost) return vi_fail(VI_EINVAL, "null cost");
    for (int j = 0; j < 5; ++j) d.cost[0][j] = cost[j];
    d.pmf[0] = pmf;
    d.dmax[0] = dmax;
    d.gamma = gamma;
    d.issuing = issuing;
    d.precision = VI_PREC_FP32;
    d.stop_rule = VI_STOP_SPAN;
    return vi_problem_create_desc(&d, out);
}

static void destroy_internal(vi_problem *h) {
    if (!h) return;
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->d_tab_f) vip::release(h->d_tab_f);
    if (h->d_tab_d) vip::release(h->d_tab_d);
    if (h->d_state) vip::release(h->d_state);
    if (h->h_state) vip::release(h->h_state);
    if (h->d_scratch) vip::release(h->d_scratch);
    if (h->d_two_e2) vip::release(h->d_two_e2);
    if (h->d_two_mix) vip::release(h->d_two_mix);
    if (h->d_two_rperm) vip::release(h->d_two_rperm);
    if (h->d_grp_order) vip::release(h->d_grp_order);
    void *pc_bufs[] = {h->d_pc_pmf, h->d_pc_prof, h->d_pc_prob, h->d_pc_off, h->d_pc_W, h->d_pc_ring,
                       h->d_pc_thr_d, h->d_pc_thr_y};
    for (void *b : pc_bufs)
        if (b) vip::release(b);
    if (h->d_pe[0]) vip::release(h->d_pe[0]);
    if (h->d_pe[1]) vip::release(h->d_pe[1]);
    if (h->d_stage_v) vip::release(h->d_stage_v);
    if (h->d_stage_p) vip::release(h->d_stage_p);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->own_stream) vip::stream_put(h->own_stream);
    delete h;
}

extern "C" vi_status vi_problem_destroy(vi_handle h) {
    if (!h) return VI_OK;
    cudaDeviceSynchronize();
    destroy_internal(h);
    return VI_OK;
}

extern "C" vi_status vi_problem_sizes(vi_handle h, uint64_t *n_states, int *n_actions, int *n_outcomes,
                                      int *value_bytes) {
    if (!h) return vi_fail(VI_EINVAL, "null handle");
    if (n_states) *n_states = h->kp.nS;
    if (n_actions) *n_actions = h->kp.nA;
    if (n_outcomes) *n_outcomes = h->n_outcomes;
    if (value_bytes) *value_bytes = h->value_bytes;
    return VI_OK;
}

extern "C" vi_status vi_problem_set_option(vi_handle h, int option, int value) {
    if (!h) return vi_fail(VI_EINVAL, "null handle");
    if (option == VI_OPT_KERNEL) {
        if (value == VI_KERNEL_AUTO) {
            h->kernel_choice = VI_KERNEL_AUTO;
        } else if (value == VI_KERNEL_GENERIC) {
            h->kernel_choice = VI_KERNEL_GENERIC;
        } else if (value == VI_KERNEL_GROUP) {
            if (!h->group_ok)
                return vi_fail(VI_EINVAL,
                               "the factorised kernel needs one product, FP32 or FP32_SINGLE precision and "
                               "2 <= Q+1 <= %d", kMaxGroupG);
            h->kernel_choice = VI_KERNEL_GROUP;
        } else if (value == VI_KERNEL_TENSOR) {
            if (!h->group_ok || !tc_supported(h->kp, h->vk, h->kahan))
                return vi_fail(VI_EINVAL,
                               "the tensor-core kernel needs one product, FIFO, FP32 precision, L >= 2, "
                               "2 <= Q+1 <= 32 and Dmax <= 127");
            h->kernel_choice = VI_KERNEL_TENSOR;
        } else if (value == VI_KERNEL_LIFO_L1) {
            if (!h->group_ok || !lifo1_supported(h->kp, h->vk, h->kahan))
                return vi_fail(VI_EINVAL,
                               "the lead-time-one LIFO kernel needs one product, LIFO, FP32 precision, L = 1, "
                               "m >= 2, 2 <= Q+1 <= 16 and Dmax <= 31");
            h->kernel_choice = VI_KERNEL_LIFO_L1;
        } else if (value == VI_KERNEL_FIFO_COL) {
            if (!h->group_ok || !fifo_col_supported(h->kp, h->vk, h->kahan))
                return vi_fail(VI_EINVAL,
                               "the FIFO column kernel needs one product, FIFO, FP32 precision, m >= 2 "
                               "(m >= 3 if L = 1), 2 <= Q+1 <= 32 and Dmax <= 62");
            h->kernel_choice = VI_KERNEL_FIFO_COL;
        } else {
            return vi_fail(VI_EINVAL, "bad kernel choice %d", value);
        }
        h->group_xw = (value == VI_KERNEL_TENSOR)     ? kTcWidth
                      : (value == VI_KERNEL_LIFO_L1)  ? kLifo1Width
                      : (value == VI_KERNEL_FIFO_COL) ? kFifoColWidth
                                                      : 0;
        if (h->graph_exec) {
            cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
        }
        if (h->graph) {
            cudaGraphDestroy(h->graph);
            h->graph = nullptr;
        }
        return VI_OK;
    }
    if (option == VI_OPT_GROUP_WIDTH) {
        if (!h->group_ok || !group_width_supported(value) || value > h->kp.p[0].G)
            return vi_fail(VI_EINVAL, "lane width %d not available for this instance", value);
        h->kernel_choice = VI_KERNEL_GROUP;
        h->group_xw = value;
        if (h->graph_exec) {
            cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
        }
        if (h->graph) {
            cudaGraphDestroy(h->graph);
            h->graph = nullptr;
        }
        return VI_OK;
    }
    if (option == VI_OPT_TEST_STALL) {
        if (value != 0 && value != 1) return vi_fail(VI_EINVAL, "test stall must be 0 or 1");
        h->kp.tc_stall = value;
        if (h->graph_exec) {   // the graph holds a copy of the kernel parameters
            cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
        }
        if (h->graph) {
            cudaGraphDestroy(h->graph);
            h->graph = nullptr;
        }
        return VI_OK;
    }
    if (option == VI_OPT_PE_MAX_ITERS) {
        if (value < 0) return vi_fail(VI_EINVAL, "pe max iters must be >= 0");
        h->pe_max_iters = value;
        return VI_OK;
    }
    return vi_fail(VI_EINVAL, "unknown option %d", option);
}

// ---------------------------------------------------------------------------
// kernel choice and autotuning of the factorised kernel's lane width
// ---------------------------------------------------------------------------
struct TuneKey {
    int vk, issuing, m, L, Q, dmax, extra;   // extra: which dedicated kernels competed (bit 0 LIFO L=1, bit 1 FIFO column)
    bool operator<(const TuneKey &o) const {
        return std::tie(vk, issuing, m, L, Q, dmax, extra) < std::tie(o.vk, o.issuing, o.m, o.L, o.Q, o.dmax, o.extra);
    }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, int> g_tune_cache;

int heuristic_width(int G, int lifo) {
    // keep the per-lane register arrays small: at most 8 (FIFO) / 12 (LIFO) values per lane
    const int cap = lifo ? 12 : 8;
    int lanes = (G + cap - 1) / cap;
    int w = (G + lanes - 1) / lanes;
    while (!group_width_supported(w)) ++w;
    return w;
}

static vi_status launch_desc(const LaunchDesc &ld, void **args, cudaStream_t s);

// time one plain sweep per candidate width on scratch buffers, keep the fastest
static vi_status autotune(vi_problem *h, cudaStream_t s) {
    const ProdParams &P = h->kp.p[0];
    // the lead-time-one LIFO kernel competes when the caller left the choice open; the
    // tensor-core FIFO kernel (slower than the CUDA-core sweep as measured on B300)
    // runs only when asked for
    const int l1 = (h->kernel_choice == VI_KERNEL_AUTO && lifo1_supported(h->kp, h->vk, h->kahan)) ? 1 : 0;
    const int fc = (h->kernel_choice == VI_KERNEL_AUTO && fifo_col_supported(h->kp, h->vk, h->kahan)) ? 1 : 0;
    const TuneKey key{h->vk, h->kp.issuing, P.m, P.L, P.Q, P.dmax, l1 | (fc << 1)};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            h->group_xw = it->second;
            return VI_OK;
        }
    }
    const char *env = getenv("VI_AUTOTUNE");
    if (env && env[0] == '0') {
        h->group_xw = l1 ? kLifo1Width : fc ? kFifoColWidth : heuristic_width(P.G, h->kp.issuing);
        return VI_OK;
    }
    int cand[18];
    int nc = group_width_candidates(P.G, cand, 16);
    if (l1) cand[nc++] = kLifo1Width;
    if (fc) cand[nc++] = kFifoColWidth;
    const size_t nb = (size_t)h->kp.nS * h->value_bytes;
    void *a = nullptr, *b = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best_ms = INFINITY;
    int best = heuristic_width(P.G, h->kp.issuing);
    KernelParams kp = h->kp;
    kp.grp_order = nullptr;   // the block order belongs to one lane width
    int mode = MODE_PLAIN;
    uint8_t *np = nullptr;
    // every failure below falls through to the release of the scratch and events
    cudaError_t ce = cudaMallocAsync(&a, nb, s);
    if (ce == cudaSuccess) ce = cudaMallocAsync(&b, nb, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(a, 0, nb, s);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    for (int i = 0; i < nc && ce == cudaSuccess; ++i) {
        LaunchDesc ld;
        if (describe_sweep(kp, h->vk, h->kahan, cand[i], ld) != cudaSuccess) continue;
        int lpr = ld.lpr;
        void *args[] = {&kp, &mode, &a, &b, &np, &lpr};
        float ms_min = INFINITY;
        for (int rep = 0; rep < 3 && ce == cudaSuccess; ++rep) {
            float ms = 0.f;
            ce = cudaEventRecord(e0, s);
            if (ce == cudaSuccess) ce = cudaLaunchKernel(ld.fn, ld.grid, ld.block, args, ld.smem, s);
            if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
            if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
            if (ce == cudaSuccess && rep > 0) ms_min = std::min(ms_min, ms);   // first launch warms caches and code
        }
        if (ce == cudaSuccess && ms_min < best_ms) {
            best_ms = ms_min;
            best = cand[i];
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (a) cudaFreeAsync(a, s);
    if (b) cudaFreeAsync(b, s);
    cudaError_t se = cudaStreamSynchronize(s);
    if (ce == cudaSuccess) ce = se;
    if (ce != cudaSuccess)
        return vi_fail(ce == cudaErrorMemoryAllocation ? VI_ENOMEM : VI_ECUDA, "autotune: %s", cudaGetErrorString(ce));
    h->group_xw = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
    return VI_OK;
}

// Block order of the factorised sweep with lane width xw: blocks sorted by the
// demand they reach, sum over their rests of min(R, Dmax) + 1 (R = units in the
// slots the demand consumes after the expiring one), heaviest first.  Blocks are
// dispatched roughly in index order, so the last wave holds the lightest ones.
// orders computed so far, by (G, K, rest slots, Dmax, lane width)
static std::mutex g_order_mu;
static std::map<std::tuple<int, int, int, int, int>, std::vector<uint32_t>> g_order_cache;

static vi_status ensure_group_order(vi_problem *h, int xw) {
    if (h->order_xw == xw && h->d_grp_order) {
        h->kp.grp_order = h->d_grp_order;
        return VI_OK;
    }
    const ProdParams &P = h->kp.p[0];
    const uint32_t G = (uint32_t)P.G;
    const int lpr = (P.G + xw - 1) / xw;
    const uint32_t rb = (uint32_t)(kGroupThreads / lpr);
    const uint32_t nR = P.nS / G;
    const uint32_t nb = (nR + rb - 1) / rb;
    const auto key = std::make_tuple(P.G, P.K, P.n_rest_slots, P.dmax, xw);
    std::vector<uint32_t> order;
    {
        std::lock_guard<std::mutex> lk(g_order_mu);
        auto it = g_order_cache.find(key);
        if (it != g_order_cache.end()) order = it->second;
    }
    if (order.empty()) {
        std::vector<double> w(nb, 0.0);
        // the rests in index order: an odometer over their digits keeps the total
        // of the first n_rest_slots digits without divisions
        std::vector<uint32_t> dig((size_t)std::max(P.K - 1, 1), 0u);
        uint32_t R = 0;
        for (uint32_t r = 0; r < nR; ++r) {
            w[r / rb] += (double)std::min<uint32_t>(R, (uint32_t)P.dmax) + 1.0;
            for (int j = 0; j < P.K - 1; ++j) {
                if (++dig[j] < G) {
                    if (j < P.n_rest_slots) ++R;
                    break;
                }
                if (j < P.n_rest_slots) R -= G - 1;
                dig[j] = 0;
            }
        }
        order.resize(nb);
        for (uint32_t b = 0; b < nb; ++b) order[b] = b;
        std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return w[a] > w[b]; });
        std::lock_guard<std::mutex> lk(g_order_mu);
        g_order_cache[key] = order;
    }
    if (h->d_grp_order) {
        cudaDeviceSynchronize();   // queued sweeps may still read the old order
        vip::release(h->d_grp_order);
        h->d_grp_order = nullptr;
    }
    CUDA_TRY(vip::dev_alloc_t(&h->d_grp_order, (size_t)nb * sizeof(uint32_t)));
    CUDA_TRY(cudaMemcpy(h->d_grp_order, order.data(), (size_t)nb * sizeof(uint32_t), cudaMemcpyHostToDevice));
    h->order_xw = xw;
    h->kp.grp_order = h->d_grp_order;
    return VI_OK;
}

// resolve which sweep kernel runs: 0 = generic, > 0 = factorised with that lane width
static vi_status choose_kernel(vi_problem *h, cudaStream_t s) {
    if (h->two_ok && h->kernel_choice != VI_KERNEL_GENERIC) {
        h->sweep_xw = kTwoWidth;
        return VI_OK;
    }
    if (h->kernel_choice == VI_KERNEL_GENERIC || !h->group_ok) {
        h->sweep_xw = 0;
        return VI_OK;
    }
    if (h->group_xw == 0) {
        vi_status st = autotune(h, s);
        if (st != VI_OK) return st;
    }
    h->sweep_xw = h->group_xw;
    // measured on B300: 2.4% faster for the FIFO 4.08M-state sweep, none for LIFO
    if (h->sweep_xw == kTcWidth || h->sweep_xw == kLifo1Width || h->sweep_xw == kFifoColWidth ||
        h->kp.issuing != VI_FIFO) {
        h->kp.grp_order = nullptr;
        return VI_OK;
    }
    return ensure_group_order(h, h->sweep_xw);
}

extern "C" vi_status vi_problem_kernel(vi_handle h, int *kernel, int *width) {
    if (!h) return vi_fail(VI_EINVAL, "null handle");
    vi_status st = choose_kernel(h, nullptr);
    if (st != VI_OK) return st;
    const int xw = h->sweep_xw;
    if (kernel)
        *kernel = (xw == 0) ? VI_KERNEL_GENERIC
                  : (xw == kTcWidth) ? VI_KERNEL_TENSOR
                  : (xw == kLifo1Width) ? VI_KERNEL_LIFO_L1
                  : (xw == kFifoColWidth) ? VI_KERNEL_FIFO_COL : VI_KERNEL_GROUP;
    if (width)
        *width = (xw == 0 || xw == kTcWidth || xw == kTwoWidth || xw == kLifo1Width || xw == kFifoColWidth) ? 0 : xw;
    return VI_OK;
}

// ---------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------
static vi_status ensure_scratch(vi_problem *h) {
    if (h->d_scratch) return VI_OK;
    CUDA_TRY(vip::dev_alloc_t(&h->d_scratch, (size_t)h->kp.nS * h->value_bytes));
    return VI_OK;
}

static vi_status launch_desc(const LaunchDesc &ld, void **args, cudaStream_t s) {
    for (int i = 0; i < ld.n_pre; ++i) CUDA_TRY(cudaLaunchKernel(ld.pre_fn[i], ld.pre_grid[i], ld.pre_block[i], args, 0, s));
    if (!ld.pdl || ld.n_pre) {
        CUDA_TRY(cudaLaunchKernel(ld.fn, ld.grid, ld.block, args, ld.smem, s));
        return VI_OK;
    }
    // the kernel waits for the grids before it in the stream itself (griddepcontrol),
    // so it may start while the previous kernel's last blocks run
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = ld.grid;
    cfg.blockDim = ld.block;
    cfg.dynamicSmemBytes = ld.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CUDA_TRY(cudaLaunchKernelExC(&cfg, ld.fn, args));
    return VI_OK;
}

// kernel nodes of one sweep (pre-kernels, then the sweep) after `dep`; returns the last
// node.  programmatic: `dep` is the previous sweep of the same kernel, which lets this
// one start its set-up early (LaunchDesc::pdl)
static vi_status add_sweep_nodes(cudaGraph_t g, const LaunchDesc &ld, void **args, cudaGraphNode_t dep,
                                 cudaGraphNode_t *last, bool programmatic = false) {
    cudaKernelNodeParams kn;
    cudaGraphNode_t prev = dep;
    for (int i = 0; i <= ld.n_pre; ++i) {
        memset(&kn, 0, sizeof(kn));
        const bool pre = i < ld.n_pre;
        kn.func = (void *)(pre ? ld.pre_fn[i] : ld.fn);
        kn.gridDim = pre ? ld.pre_grid[i] : ld.grid;
        kn.blockDim = pre ? ld.pre_block[i] : ld.block;
        kn.sharedMemBytes = pre ? 0u : (unsigned)ld.smem;
        kn.kernelParams = args;
        cudaGraphNode_t node;
        if (programmatic && ld.pdl && !ld.n_pre && prev) {
            CUDA_TRY(cudaGraphAddKernelNode(&node, g, nullptr, 0, &kn));
            cudaGraphEdgeData ed;
            memset(&ed, 0, sizeof(ed));
            ed.from_port = cudaGraphKernelNodePortProgrammatic;
            ed.to_port = 0;
            ed.type = cudaGraphDependencyTypeProgrammatic;
            CUDA_TRY(cudaGraphAddDependencies(g, &prev, &node, &ed, 1));
        } else {
            CUDA_TRY(cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &kn));
        }
        prev = node;
    }
    *last = prev;
    return VI_OK;
}

constexpr int kSweepsPerPass = 4;

// programmatic edges between the sweeps of a loop pass; cleared (for the process) if a
// graph with them cannot be built or instantiated, and the graph is built without
static std::atomic<bool> g_graph_pdl{true};

static vi_status build_graph_once(vi_problem *h, bool pdl);

static vi_status build_graph(vi_problem *h) {
    if (h->graph_exec && h->graph_xw == h->sweep_xw) return VI_OK;
    if (g_graph_pdl.load()) {
        const vi_status st = build_graph_once(h, true);
        if (st == VI_OK) return VI_OK;
        cudaGetLastError();
        g_graph_pdl.store(false);
    }
    return build_graph_once(h, false);
}

static vi_status build_graph_once(vi_problem *h, bool pdl) {
    if (h->graph_exec && h->graph_xw == h->sweep_xw) return VI_OK;
    if (h->graph_exec) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
    }
    if (h->graph) {
        cudaGraphDestroy(h->graph);
        h->graph = nullptr;
    }
    h->graph_xw = h->sweep_xw;
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaGraphCreate(&g, 0));
    h->graph = g;
    cudaGraphConditionalHandle cond;
    CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
    h->cond = (unsigned long long)cond;

    LaunchDesc ld_init, ld_sweep;
    CUDA_TRY(describe_solve_init(h->kp.nS, ld_init));
    CUDA_TRY(describe_sweep(h->kp, h->vk, h->kahan, h->sweep_xw, ld_sweep));
    h->args_kp = h->kp;
    h->args_nS = h->kp.nS;
    h->args_mode_sweep = MODE_SWEEP;
    h->args_mode_extract = MODE_EXTRACT;
    h->args_null_v = nullptr;
    h->args_null_p = nullptr;
    h->args_lpr = ld_sweep.lpr;

    cudaKernelNodeParams kn;
    memset(&kn, 0, sizeof(kn));
    void *init_args[] = {&h->kp.st, &h->args_nS};
    kn.func = (void *)ld_init.fn;
    kn.gridDim = ld_init.grid;
    kn.blockDim = ld_init.block;
    kn.sharedMemBytes = 0;
    kn.kernelParams = init_args;
    cudaGraphNode_t n_init;
    CUDA_TRY(cudaGraphAddKernelNode(&n_init, g, nullptr, 0, &kn));

    // the union inside cudaGraphNodeParams has no default constructor: build it in zeroed storage
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    memset(cp_raw, 0, sizeof(cp_raw));
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t n_loop;
    CUDA_TRY(cudaGraphAddNode(&n_loop, g, &n_init, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];

    void *sweep_args[] = {&h->args_kp, &h->args_mode_sweep, &h->args_null_v, &h->args_null_v, &h->args_null_p,
                          &h->args_lpr};
    // kSweepsPerPass sweeps per pass of the loop body: the loop's per-pass cost is
    // paid once per pass; a sweep that finds the stop flag set returns at once
    cudaGraphNode_t n_sweep = nullptr;
    vi_status vs = VI_OK;
    for (int k = 0; k < kSweepsPerPass; ++k) {
        cudaGraphNode_t n_next;
        vs = add_sweep_nodes(body, ld_sweep, sweep_args, n_sweep, &n_next, pdl && k > 0);
        if (vs != VI_OK) return vs;
        n_sweep = n_next;
    }

    void *extract_args[] = {&h->args_kp, &h->args_mode_extract, &h->args_null_v, &h->args_null_v,
                            &h->args_null_p, &h->args_lpr};
    cudaGraphNode_t n_extract;
    vs = add_sweep_nodes(g, ld_sweep, extract_args, n_loop, &n_extract);
    if (vs != VI_OK) return vs;

    CUDA_TRY(cudaGraphInstantiate(&h->graph_exec, g, 0));
    return VI_OK;
}

// host-driven loop (VI_FLAG_NO_GRAPH): launches sweeps in batches and polls the flag
static vi_status run_host_loop(vi_problem *h, cudaStream_t s) {
    LaunchDesc ld_init, ld_sweep;
    CUDA_TRY(describe_solve_init(h->kp.nS, ld_init));
    CUDA_TRY(describe_sweep(h->kp, h->vk, h->kahan, h->sweep_xw, ld_sweep));
    KernelParams kp = h->kp;
    uint32_t nS = kp.nS;
    int mode_sweep = MODE_SWEEP, mode_extract = MODE_EXTRACT;
    void *nv = nullptr;
    uint8_t *np = nullptr;
    void *init_args[] = {&kp.st, &nS};
    vi_status st = launch_desc(ld_init, init_args, s);
    if (st != VI_OK) return st;
    int lpr = ld_sweep.lpr;
    void *sweep_args[] = {&kp, &mode_sweep, &nv, &nv, &np, &lpr};
    const int batch = 4;
    int launched = 0;
    while (launched < h->h_state->max_iters) {
        for (int k = 0; k < batch && launched < h->h_state->max_iters; ++k, ++launched) {
            st = launch_desc(ld_sweep, sweep_args, s);
            if (st != VI_OK) return st;
        }
        CUDA_TRY(cudaMemcpyAsync(h->h_state, h->d_state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        if (!h->h_state->keep_going) break;
    }
    void *extract_args[] = {&kp, &mode_extract, &nv, &nv, &np, &lpr};
    return launch_desc(ld_sweep, extract_args, s);
}

static vi_status policy_eval_impl(vi_problem *h, const uint8_t *policy, double *V, double tol, int max_iters,
                                  cudaStream_t s, int *iters_out, double *delta_out);

static vi_status solve_impl(vi_problem *h, double tol, int max_iters, void *V, uint8_t *policy, void *stream,
                            int flags, vi_solve_info *info, void *vhost);

extern "C" vi_status vi_solve(vi_handle h, double tol, int max_iters, void *V, uint8_t *policy, void *stream,
                              int flags, vi_solve_info *info) {
    return solve_impl(h, tol, max_iters, V, policy, stream, flags, info, nullptr);
}

// vhost: device view of pinned host memory that the extraction sweep fills with
// the final V (V itself then need not hold it), or null
static vi_status solve_impl(vi_problem *h, double tol, int max_iters, void *V, uint8_t *policy, void *stream,
                            int flags, vi_solve_info *info, void *vhost) {
    if (!h) return vi_fail(VI_EINVAL, "null handle");
    if (!V) return vi_fail(VI_EINVAL, "null V");
    if (((uintptr_t)V) % (uintptr_t)h->value_bytes != 0)
        return vi_fail(VI_EINVAL, "V must be aligned to its %d-byte values", h->value_bytes);
    if (!(tol >= 0.0) || max_iters < 0) return vi_fail(VI_EINVAL, "need tol >= 0 and max_iters >= 0");
    if ((flags & VI_FLAG_WARM_START) && !info) return vi_fail(VI_EINVAL, "warm start needs info->offset");
    if (h->periodic && (flags & VI_FLAG_POLICY_EVAL))
        return vi_fail(VI_EINVAL, "VI_FLAG_POLICY_EVAL is not available for periodic problems");
    cudaStream_t s = (cudaStream_t)stream;
    vi_status st = ensure_scratch(h);
    if (st != VI_OK) return st;
    st = choose_kernel(h, s);
    if (st != VI_OK) return st;

    const bool use_graph = !(flags & VI_FLAG_NO_GRAPH);
    if (use_graph) {
        st = build_graph(h);
        if (st != VI_OK) return st;
    }
    SolveState *hs = h->h_state;
    memset(hs, 0, sizeof(SolveState));
    hs->buf[0] = V;
    hs->buf[1] = h->d_scratch;
    hs->policy = policy;
    hs->vhost = vhost;
    hs->tol = tol;
    hs->gamma = h->desc.gamma;
    hs->max_iters = max_iters;
    hs->stop_rule = h->desc.stop_rule;
    hs->normalise = (h->vk == VK_SINGLE) ? 1 : 0;
    hs->use_cond = use_graph ? 1 : 0;
    hs->cond = h->cond;
    hs->warm = (flags & VI_FLAG_WARM_START) ? 1 : 0;
    hs->value_bytes = h->value_bytes;
    hs->key_min = ~0ull;
    hs->offset = (flags & VI_FLAG_WARM_START) ? info->offset : 0.0;
    CUDA_TRY(cudaMemcpyAsync(h->d_state, hs, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    if (h->periodic && hs->stop_rule == VI_STOP_PERIODIC)   // the periodic test restarts with every solve
        CUDA_TRY(cudaMemsetAsync(h->d_pc_ring, 0, (size_t)7 * h->kp.nS * sizeof(double), s));
    CUDA_TRY(cudaEventRecord(h->ev0, s));
    if (use_graph) {
        CUDA_TRY(cudaGraphLaunch(h->graph_exec, s));
    } else {
        st = run_host_loop(h, s);
        if (st != VI_OK) return st;
    }
    CUDA_TRY(cudaEventRecord(h->ev1, s));
    CUDA_TRY(cudaMemcpyAsync(hs, h->d_state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    if (hs->fault) return vi_fail(VI_ECUDA, "a sweep's bounded wait on the tensor cores gave up; V is not valid");
    vi_status result = hs->converged ? VI_OK : VI_ENOTCONVERGED;
    if (info) {
        memset(info, 0, sizeof(*info));
        info->iters = hs->iter;
        info->status = result;
        info->crit = hs->crit;
        info->dmax = hs->dmax_abs;
        info->dmin = hs->dmin_abs;
        info->offset = hs->normalise ? hs->offset : 0.0;
        info->wall_ms = ms;
        double nominal = (double)h->kp.nS * (double)h->kp.nA * (double)h->n_outcomes * (double)hs->iter;
        info->updates_per_s = ms > 0.f ? nominal / (ms * 1e-3) : 0.0;
    }
    if ((flags & VI_FLAG_POLICY_EVAL) && policy && info) {
        const uint32_t n = h->kp.nS;
        if (!h->d_pe[0]) {
            CUDA_TRY(vip::dev_alloc_t(&h->d_pe[0], (size_t)n * sizeof(double)));
            CUDA_TRY(vip::dev_alloc_t(&h->d_pe[1], (size_t)n * sizeof(double)));
        }
        // start from V_abs of the solve, evaluate the extracted policy in FP64
        CUDA_TRY(launch_to_fp64(V, h->vk, info->offset, h->d_pe[0], n, s));
        CUDA_TRY(cudaMemcpyAsync(h->d_pe[1], h->d_pe[0], (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
        int it = 0;
        double delta = 0.0;
        double scale = std::max(fabs(info->offset), 1.0);
        vi_status ps = policy_eval_impl(h, policy, h->d_pe[0], 1e-9 * scale, h->pe_max_iters, s, &it, &delta);
        if (ps != VI_OK && ps != VI_ENOTCONVERGED) return ps;
        CUDA_TRY(launch_diff_range(h->d_pe[0], h->d_pe[1], n, h->d_state, s));
        CUDA_TRY(cudaMemcpyAsync(hs, h->d_state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        info->pe_iters = it;
        info->pe_delta = delta;
        info->pe_gap = std::max(fabs(hs->dmax_abs), fabs(hs->dmin_abs));
        info->pe_span = hs->dmax_abs - hs->dmin_abs;
    }
    return result;
}

// the device view of page-locked host memory (cudaMallocHost / cudaHostAlloc /
// cudaHostRegister), or false for pageable memory
static bool pinned_view(void *p, void **dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
    *dev = a.devicePointer;
    return true;
}

extern "C" vi_status vi_solve_host(vi_handle h, double tol, int max_iters, void *V_host, uint8_t *policy_host,
                                   int flags, vi_solve_info *info) {
    if (!h) return vi_fail(VI_EINVAL, "null handle");
    if (!V_host) return vi_fail(VI_EINVAL, "null V_host");
    if (!h->own_stream) CUDA_TRY(vip::stream_get(&h->own_stream));
    const size_t nb = (size_t)h->kp.nS * h->value_bytes;
    if (!h->d_stage_v) CUDA_TRY(vip::dev_alloc_t(&h->d_stage_v, nb));
    if (policy_host && !h->d_stage_p) CUDA_TRY(vip::dev_alloc_t(&h->d_stage_p, h->kp.nS));
    cudaStream_t s = h->own_stream;
    if (flags & VI_FLAG_WARM_START) CUDA_TRY(cudaMemcpyAsync(h->d_stage_v, V_host, nb, cudaMemcpyHostToDevice, s));
    // pinned host buffers: the extraction sweep writes V and the policy straight into
    // them, so the transfer overlaps the sweep instead of following it (not with the
    // FP64 policy evaluation, which reads both on the device afterwards)
    void *dv = nullptr, *dp = nullptr;
    const bool direct = !(flags & VI_FLAG_POLICY_EVAL) && ((uintptr_t)V_host) % (uintptr_t)h->value_bytes == 0 &&
                        pinned_view(V_host, &dv) &&
                        (!policy_host || pinned_view(policy_host, &dp));
    vi_status st;
    if (direct) {
        st = solve_impl(h, tol, max_iters, h->d_stage_v, (uint8_t *)dp, s, flags, info, dv);
        return st;   // solve_impl synchronised the stream after the extraction sweep
    }
    st = vi_solve(h, tol, max_iters, h->d_stage_v, policy_host ? h->d_stage_p : nullptr, s, flags, info);
    if (st != VI_OK && st != VI_ENOTCONVERGED) return st;
    CUDA_TRY(cudaMemcpyAsync(V_host, h->d_stage_v, nb, cudaMemcpyDeviceToHost, s));
    if (policy_host) CUDA_TRY(cudaMemcpyAsync(policy_host, h->d_stage_p, h->kp.nS, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return st;
}

// ---------------------------------------------------------------------------
// single backup, next states, policy evaluation, rollouts
// ---------------------------------------------------------------------------
extern "C" vi_status vi_backup(vi_handle h, const void *V_in, void *V_out, uint8_t *policy, void *stream,
                               double *dstats) {
    if (!h) return vi_fail(VI_EINVAL, "null handle");
    if (!V_in || !V_out || V_in == V_out) return vi_fail(VI_EINVAL, "V_in and V_out must be distinct buffers");
    if ((((uintptr_t)V_in) | ((uintptr_t)V_out)) % (uintptr_t)h->value_bytes != 0)
        return vi_fail(VI_EINVAL, "V_in and V_out must be aligned to their %d-byte values", h->value_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    vi_status cs = choose_kernel(h, s);
    if (cs != VI_OK) return cs;
    LaunchDesc ld;
    CUDA_TRY(describe_sweep(h->kp, h->vk, h->kahan, h->sweep_xw, ld));
    KernelParams kp = h->kp;
    int mode = MODE_PLAIN;
    const void *vin = V_in;
    void *vout = V_out;
    int lpr = ld.lpr;
    void *args[] = {&kp, &mode, &vin, &vout, &policy, &lpr};
    vi_status st = launch_desc(ld, args, s);
    if (st != VI_OK) return st;
    if (dstats) {
        CUDA_TRY(cudaMemcpyAsync(h->h_state, h->d_state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        dstats[0] = h->h_state->dmax_abs;
        dstats[1] = h->h_state->dmin_abs;
        if (h->h_state->fault) {
            cudaMemsetAsync(&h->d_state->fault, 0, sizeof(int), s);   // reported once
            return vi_fail(VI_ECUDA, "the sweep's bounded wait on the tensor cores gave up");
        }
    }
    return VI_OK;
}

extern "C" vi_status vi_next_states(vi_handle h, const uint32_t *states, int n, uint32_t *out, void *stream) {
    if (!h) return vi_fail(VI_EINVAL, "null handle");
    if (h->periodic) return vi_fail(VI_EINVAL, "vi_next_states takes problems with demand outcomes only");
    if (n < 0 || (n > 0 && (!states || !out))) return vi_fail(VI_EINVAL, "bad states / out");
    if (n == 0) return VI_OK;
    if (n > 65535) return vi_fail(VI_EINVAL, "at most 65535 states per call");
    CUDA_TRY(launch_next_states(h->kp, states, n, out, (cudaStream_t)stream));
    return VI_OK;
}

static vi_status policy_eval_impl(vi_problem *h, const uint8_t *policy, double *V, double tol, int max_iters,
                                  cudaStream_t s, int *iters_out, double *delta_out) {
    const uint32_t n = h->kp.nS;
    double *tmp = nullptr;
    CUDA_TRY(cudaMallocAsync((void **)&tmp, (size_t)n * sizeof(double), s));
    KernelParams kp = h->kp;
    kp.tables = h->d_tab_d;
    double *cur = V, *nxt = tmp;
    int it = 0;
    double delta = INFINITY;
    vi_status result = VI_ENOTCONVERGED;
    while (it < max_iters) {
        cudaError_t e = launch_policy_eval(kp, policy, cur, nxt, s);
        if (e != cudaSuccess) {
            cudaFreeAsync(tmp, s);
            return vi_fail(VI_ECUDA, "policy eval launch: %s", cudaGetErrorString(e));
        }
        std::swap(cur, nxt);
        ++it;
        if (it % 8 == 0 || it == max_iters) {
            CUDA_TRY(cudaMemcpyAsync(h->h_state, h->d_state, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            delta = std::max(fabs(h->h_state->dmax_abs), fabs(h->h_state->dmin_abs));
            if (delta < tol) {
                result = VI_OK;
                break;
            }
        }
    }
    if (cur != V) CUDA_TRY(cudaMemcpyAsync(V, cur, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaFreeAsync(tmp, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (iters_out) *iters_out = it;
    if (delta_out) *delta_out = delta;
    return result;
}

extern "C" vi_status vi_policy_eval(vi_handle h, const uint8_t *policy, double *V, double tol, int max_iters,
                                    void *stream, int *iters, double *delta) {
    if (h && h->periodic) return vi_fail(VI_EINVAL, "vi_policy_eval is not available for periodic problems");
    if (!h) return vi_fail(VI_EINVAL, "null handle");
    if (!policy || !V || !(tol >= 0.0) || max_iters < 0) return vi_fail(VI_EINVAL, "bad policy-eval arguments");
    if (((uintptr_t)V) % sizeof(double) != 0) return vi_fail(VI_EINVAL, "V must be 8-byte aligned");
    return policy_eval_impl(h, policy, V, tol, max_iters, (cudaStream_t)stream, iters, delta);
}

static void make_thresholds(const std::vector<double> &pmf, unsigned long long *thr) {
    // floor(2^32 * CDF(d)), CDF summed in ascending order; the last entry is 2^32
    const int dmax = (int)pmf.size() - 1;
    double c = 0.0;
    for (int d = 0; d <= dmax; ++d) {
        c += pmf[d];
        double t = floor(c * 4294967296.0);
        if (t > 4294967296.0) t = 4294967296.0;
        if (t < 0.0) t = 0.0;
        thr[d] = (unsigned long long)t;
    }
    thr[dmax] = 4294967296ull;
}

// the rollout parameters shared by vi_simulate_ex and vi_mbs_search
static vi_status roll_params(const vi_problem *h, int n_rollouts, int horizon, int warmup, uint64_t seed,
                             RollParams &rp) {
    const vi_problem_desc &d = h->desc;
    for (int k = 0; k < d.n_products; ++k)
        if (d.dmax[k] > kMaxRollDmax) return vi_fail(VI_EINVAL, "rollouts need dmax <= %d", kMaxRollDmax);
    if (d.n_products == 2 && d.subst_rate != 0.5)
        return vi_fail(VI_EINVAL, "two-product rollouts draw substitutions as fair bits (subst_rate 1/2)");
    memset(&rp, 0, sizeof(rp));
    rp.n_rollouts = n_rollouts;
    rp.horizon = horizon;
    rp.warmup = warmup;
    rp.seed = seed;
    for (int k = 0; k < d.n_products; ++k) {
        for (int j = 0; j < 5; ++j) rp.cost[k][j] = d.cost[k][j];
        make_thresholds(h->pmf[k], rp.thr[k]);
    }
    return VI_OK;
}

extern "C" vi_status vi_simulate_ex(vi_handle h, const uint8_t *policy, int n_rollouts, int horizon, int warmup,
                                    uint64_t seed, double *returns, double *kpis, double *kpis_prod, int32_t *traj,
                                    void *stream) {
    if (!h) return vi_fail(VI_EINVAL, "null handle");
    if (!policy || !returns || n_rollouts < 0 || horizon < 0 || warmup < 0)
        return vi_fail(VI_EINVAL, "bad rollout arguments");
    if (n_rollouts == 0) return VI_OK;
    if (h->periodic) {
        if (kpis_prod) return vi_fail(VI_EINVAL, "periodic problems have one product (kpis_prod must be NULL)");
        PcRollParams pp;
        pp.n_rollouts = n_rollouts;
        pp.horizon = horizon;
        pp.warmup = warmup;
        pp.seed = seed;
        pp.thr_d = h->d_pc_thr_d;
        pp.thr_y = h->d_pc_thr_y;
        CUDA_TRY(launch_pc_rollouts(h->kp, pp, policy, returns, kpis, traj, (cudaStream_t)stream));
        return VI_OK;
    }
    RollParams rp;
    vi_status st = roll_params(h, n_rollouts, horizon, warmup, seed, rp);
    if (st != VI_OK) return st;
    CUDA_TRY(launch_rollouts(h->kp, rp, policy, returns, kpis, kpis_prod, traj, (cudaStream_t)stream));
    return VI_OK;
}

extern "C" vi_status vi_simulate(vi_handle h, const uint8_t *policy, int n_rollouts, int horizon, int warmup,
                                 uint64_t seed, double *returns, double *kpis, int32_t *traj, void *stream) {
    return vi_simulate_ex(h, policy, n_rollouts, horizon, warmup, seed, returns, kpis, nullptr, traj, stream);
}

extern "C" vi_status vi_mbs_search(vi_handle h, const int S_lo[2], const int S_hi[2], const int mu[2], int cap,
                                   int n_rollouts, int horizon, int warmup, uint64_t seed, double *returns,
                                   double *kpis_prod, double *mean_returns, int best_S[2], void *stream) {
    if (!h) return vi_fail(VI_EINVAL, "null handle");
    if (h->periodic) return vi_fail(VI_EINVAL, "the modified base-stock search takes Scenario A/B problems");
    const vi_problem_desc &d = h->desc;
    const int np = d.n_products;
    if (!S_lo || !S_hi || !mu || !returns || n_rollouts < 1 || horizon < 0 || warmup < 0)
        return vi_fail(VI_EINVAL, "bad search arguments");
    for (int k = 0; k < np; ++k) {
        if (S_lo[k] < 0 || S_hi[k] < S_lo[k] || mu[k] < 0) return vi_fail(VI_EINVAL, "bad order-up-to range");
        if (d.m[k] > kMbsMaxM || d.L[k] > kMbsMaxL)
            return vi_fail(VI_EINVAL, "the heuristic keeps m <= %d and L <= %d slots", kMbsMaxM, kMbsMaxL);
    }
    MbsParams mp;
    memset(&mp, 0, sizeof(mp));
    mp.s_lo[0] = S_lo[0];
    mp.s_lo[1] = (np == 2) ? S_lo[1] : 0;
    const int n1 = S_hi[0] - S_lo[0] + 1;
    mp.n2 = (np == 2) ? S_hi[1] - S_lo[1] + 1 : 1;
    mp.n_pairs = n1 * mp.n2;
    mp.mu[0] = mu[0];
    mp.mu[1] = (np == 2) ? mu[1] : 0;
    mp.cap = cap ? 1 : 0;
    if ((long long)mp.n_pairs * n_rollouts > (1ll << 31)) return vi_fail(VI_EINVAL, "too many (pair, rollout) runs");
    RollParams rp;
    vi_status st = roll_params(h, n_rollouts, horizon, warmup, seed, rp);
    if (st != VI_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(launch_mbs(h->kp, rp, mp, returns, kpis_prod, s));
    if (!mean_returns && !best_S) return VI_OK;
    std::vector<double> host((size_t)mp.n_pairs * n_rollouts);
    CUDA_TRY(cudaMemcpyAsync(host.data(), returns, host.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    int best = 0;
    double best_mean = -INFINITY;
    for (int i = 0; i < mp.n_pairs; ++i) {
        double sum = 0.0;   // rollout order, FP64
        for (int r = 0; r < n_rollouts; ++r) sum += host[(size_t)i * n_rollouts + r];
        const double mean = sum / (double)n_rollouts;
        if (mean_returns) mean_returns[i] = mean;
        if (mean > best_mean) {
            best_mean = mean;
            best = i;
        }
    }
    if (best_S) {
        best_S[0] = mp.s_lo[0] + best / mp.n2;
        best_S[1] = mp.s_lo[1] + best % mp.n2;
    }
    return VI_OK;
}

extern "C" vi_status vi_basestock_search(vi_handle h, int s_lo, int s_hi, int n_rollouts, int horizon, int warmup,
                                         uint64_t seed, double *returns, double *mean_returns, int *best_S,
                                         void *stream) {
    if (!h) return vi_fail(VI_EINVAL, "null handle");
    if (h->periodic) return vi_fail(VI_EINVAL, "the base-stock search takes Scenario A problems");
    const vi_problem_desc &d = h->desc;
    if (d.n_products != 1) return vi_fail(VI_EINVAL, "the base-stock search takes single-product instances");
    if (!returns || s_lo < 0 || s_hi < s_lo || n_rollouts < 1 || horizon < 0 || warmup < 0)
        return vi_fail(VI_EINVAL, "bad search arguments");
    if (d.dmax[0] > kMaxRollDmax) return vi_fail(VI_EINVAL, "rollouts need dmax <= %d", kMaxRollDmax);
    const int n_S = s_hi - s_lo + 1;
    if ((long long)n_S * n_rollouts > (1ll << 31)) return vi_fail(VI_EINVAL, "too many (S, rollout) pairs");
    RollParams rp;
    memset(&rp, 0, sizeof(rp));
    rp.n_rollouts = n_rollouts;
    rp.horizon = horizon;
    rp.warmup = warmup;
    rp.seed = seed;
    for (int j = 0; j < 5; ++j) rp.cost[0][j] = d.cost[0][j];
    make_thresholds(h->pmf[0], rp.thr[0]);
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(launch_basestock(h->kp, rp, s_lo, n_S, returns, s));
    if (!mean_returns && !best_S) return VI_OK;
    std::vector<double> host((size_t)n_S * n_rollouts);
    CUDA_TRY(cudaMemcpyAsync(host.data(), returns, host.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    int best = s_lo;
    double best_mean = -INFINITY;
    for (int i = 0; i < n_S; ++i) {
        double sum = 0.0;   // rollout order, FP64
        for (int r = 0; r < n_rollouts; ++r) sum += host[(size_t)i * n_rollouts + r];
        const double mean = sum / (double)n_rollouts;
        if (mean_returns) mean_returns[i] = mean;
        if (mean > best_mean) {
            best_mean = mean;
            best = s_lo + i;
        }
    }
    if (best_S) *best_S = best;
    return VI_OK;
}

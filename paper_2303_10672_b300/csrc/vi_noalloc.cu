// vi_noalloc.cu -- one Bellman sweep that allocates no memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where they
// need a sweep: code running under an allocator that must not be re-entered,
// callers whose memory is accounted by someone else, or code that has already
// reserved every byte it may use.  vi_backup_noalloc serves them: the caller
// passes the value and policy buffers, and the scratch the sweep kernel needs --
// the expectation tables and the reduction slots that vi_problem_create would
// otherwise allocate -- lives in a fixed array in device memory that belongs to
// this library.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "../../include/vi.h"
#include "vi_api_internal.h"
#include "vi_common.cuh"
#include "vi_kernels.h"

using namespace vib;

namespace {
constexpr int kTabFloats = VI_NOALLOC_MAX_TABLE_FLOATS;   // expectation tables
constexpr size_t kTabBytes = (size_t)kTabFloats * sizeof(float);
constexpr size_t kStateBytes = 1024;                       // reduction slots (SolveState)
constexpr int kMaxDevices = 64;
static_assert(sizeof(SolveState) <= kStateBytes, "reduction slots do not fit");
static_assert(kTabBytes % 256 == 0, "state region must stay 256-byte aligned");
}  // namespace

// Scratch shared by every call on a device; kept until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kTabBytes + kStateBytes];

static std::mutex g_noalloc_mu;                    // guards the host staging buffers and the address cache
static void *g_noalloc_addr[kMaxDevices];          // device address of g_noalloc_scratch, per device
static double g_tab_d[kTabFloats];                 // tables built in FP64 ...
static float g_tab_f[kTabFloats];                  // ... and staged as floats
static double g_leftover[kTabFloats];              // E[(y - D)^+], y = 0..m Q

// the same tables vi_problem_create builds for one product, into static storage
static int build_tables_static(ProdParams &P, const double *pmf, int issuing, const double *cost) {
    const int dmax = P.dmax;
    P.pn = p_table_len(dmax, P.tmax, P.G);
    P.rt_rows = (P.m - 1) * P.Q + 1;
    const long need = 3L * P.pn + 2L * P.G * P.rt_rows;
    if (need > kTabFloats || P.tmax + 1 > kTabFloats) return -1;
    int n = 0;
    P.off_p = n;
    for (int k = 0; k < P.pn; ++k) g_tab_d[n++] = k <= dmax ? pmf[k] : 0.0;
    P.off_F = n;
    double c = 0.0;
    for (int k = 0; k < P.pn; ++k) {
        if (k <= dmax) c += pmf[k];
        g_tab_d[n++] = c;
    }
    P.off_tail = n;
    for (int k = 0; k < P.pn; ++k) g_tab_d[n + k] = 0.0;
    double t = 0.0;
    for (int k = dmax; k >= 0; --k) {
        t += pmf[k];
        g_tab_d[n + k] = t;
    }
    n += P.pn;
    double mu = 0.0;
    for (int d = 0; d <= dmax; ++d) mu += (double)d * pmf[d];
    for (int y = 0; y <= P.tmax; ++y) {
        double s = 0.0;
        for (int d = 0; d <= dmax && d < y; ++d) s += pmf[d] * (double)(y - d);
        g_leftover[y] = s;
    }
    const double *G = g_leftover;
    P.off_RT = n;
    for (int R = 0; R < P.rt_rows; ++R)
        for (int y1 = 0; y1 < P.G; ++y1) g_tab_d[n++] = expected_period_reward(y1, R, G, mu, cost, issuing);
    P.off_RTlo = n;
    for (int i = 0; i < P.G * P.rt_rows; ++i) {
        const double v = g_tab_d[P.off_RT + i];
        g_tab_d[n++] = v - (double)(float)v;
    }
    return n;
}

extern "C" vi_status vi_backup_noalloc(int m, int L, int Q, const double cost[5], const double *pmf, int dmax,
                                       double gamma, int issuing, const void *V_in, void *V_out, uint8_t *policy,
                                       double *dstats, void *stream) {
    // argument checks (the rules of vi_problem_create)
    if (m < 1 || L < 1 || Q < 0 || Q + 1 > 256) return vi_fail(VI_EINVAL, "need m >= 1, L >= 1, 0 <= Q <= 255");
    if (!cost || !pmf || dmax < 0 || dmax > kMaxDmax) return vi_fail(VI_EINVAL, "bad cost / pmf / dmax");
    if (!V_in || !V_out || V_in == V_out) return vi_fail(VI_EINVAL, "V_in and V_out must be distinct buffers");
    if (!(gamma > 0.0 && gamma <= 1.0)) return vi_fail(VI_EINVAL, "gamma must be in (0, 1]");
    if (issuing != VI_FIFO && issuing != VI_LIFO) return vi_fail(VI_EINVAL, "issuing must be FIFO or LIFO");
    for (int j = 0; j < 5; ++j)
        if (!(cost[j] >= 0.0) || !isfinite(cost[j])) return vi_fail(VI_EINVAL, "costs must be finite and >= 0");
    double sum = 0.0;
    for (int d = 0; d <= dmax; ++d) {
        if (!(pmf[d] >= 0.0)) return vi_fail(VI_EINVAL, "pmf entries must be >= 0");
        sum += pmf[d];
    }
    if (fabs(sum - 1.0) > 1e-12) return vi_fail(VI_EINVAL, "pmf does not sum to 1");
    const int K = (m - 1) + (L - 1);
    double ns = 1.0;
    for (int k = 0; k < K; ++k) ns *= (double)(Q + 1);
    if (ns >= 4294967296.0 || K > kMaxDigits) return vi_fail(VI_EINVAL, "|S| does not fit 32 bits");

    cudaStream_t s = (cudaStream_t)stream;
    // the table upload reads a host staging buffer that the next call overwrites, and the
    // statistics read-back synchronises the stream: neither belongs in a captured graph
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &cs);
    if (ce != cudaSuccess) return vi_fail(VI_ECUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(ce));
    if (cs != cudaStreamCaptureStatusNone)
        return vi_fail(VI_EINVAL, "vi_backup_noalloc is refused on a stream that is being captured");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    KernelParams kp;
    memset(&kp, 0, sizeof(kp));
    fill_prod_params(kp.p[0], m, L, Q, dmax, cost[0]);
    const int n_tab = build_tables_static(kp.p[0], pmf, issuing, cost);
    if (n_tab < 0)
        return vi_fail(VI_EINVAL,
                       "tables for this instance need %ld floats; vi_backup_noalloc holds at most %d "
                       "(use vi_problem_create + vi_backup)",
                       3L * kp.p[0].pn + 2L * kp.p[0].G * kp.p[0].rt_rows, kTabFloats);

    // one-time set-up per device: the device address of the scratch array
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return vi_fail(VI_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return vi_fail(VI_EINVAL, "device %d beyond %d", dev, kMaxDevices);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return vi_fail(VI_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    unsigned char *base = (unsigned char *)g_noalloc_addr[dev];
    SolveState *st = (SolveState *)(base + kTabBytes);

    for (int i = 0; i < n_tab; ++i) g_tab_f[i] = (float)g_tab_d[i];
    // pageable source: the call returns once the staging buffer may be reused
    e = cudaMemcpyAsync(base, g_tab_f, (size_t)n_tab * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return vi_fail(VI_ECUDA, "table upload: %s", cudaGetErrorString(e));
    // the reduction slots keep the previous call's contents: reset them (max key 0, min key all ones)
    e = cudaMemsetAsync(st, 0, sizeof(SolveState), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&st->key_min, 0xff, sizeof(st->key_min), s);
    if (e != cudaSuccess) return vi_fail(VI_ECUDA, "scratch reset: %s", cudaGetErrorString(e));

    kp.n_products = 1;
    kp.issuing = issuing;
    kp.gamma = gamma;
    kp.nS = kp.p[0].nS;
    kp.nA = kp.p[0].G;
    kp.tables = base;
    kp.n_tables = n_tab;
    kp.tab_in_smem = 1;
    kp.st = st;
    const int xw = group_supported(kp, VK_PAIR, 0) ? heuristic_width(kp.p[0].G, issuing) : 0;
    LaunchDesc ld;
    e = describe_sweep(kp, VK_PAIR, 0, xw, ld);
    if (e != cudaSuccess) return vi_fail(VI_ECUDA, "kernel set-up: %s", cudaGetErrorString(e));
    int mode = MODE_PLAIN;
    int lpr = ld.lpr;
    const void *vin = V_in;
    void *vout = V_out;
    void *args[] = {&kp, &mode, &vin, &vout, &policy, &lpr};
    e = cudaLaunchKernel(ld.fn, ld.grid, ld.block, args, ld.smem, s);
    if (e != cudaSuccess) return vi_fail(VI_ECUDA, "sweep launch: %s", cudaGetErrorString(e));
    if (dstats) {
        double out[2];
        e = cudaMemcpyAsync(out, &st->dmax_abs, sizeof(out), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return vi_fail(VI_ECUDA, "change statistics: %s", cudaGetErrorString(e));
        dstats[0] = out[0];
        dstats[1] = out[1];
    }
    return VI_OK;
}

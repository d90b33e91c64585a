// vi_server.cu -- continuous-batching solve server.
//
// A host worker thread owns one CUDA stream.  Requests wait in a FIFO queue and
// are admitted, in order, while a slot is free and their device memory (value
// ping-pong and policy) fits the budget.  Each iteration of the worker runs a few
// batched sweeps over all admitted instances -- one launch per lane-width class
// and sweep, each block finding its instance from a prefix sum of block counts --
// so instances of different sizes advance together, then reads every slot's
// status once.  An instance whose stopping test passed gets an extraction sweep
// in the next iteration; its values are converted to FP64 on the device and a
// retirement thread copies them (and the policy) to pinned host memory on a
// second stream and releases the buffers, while the worker carries on.  The
// pinned result buffers come from a free list of the server's (power-of-two
// sizes) and go back to it when the caller polls the result: fresh pageable
// memory would cost a zero-fill and a page fault per page of every result.
//
// Slots own their expectation tables, solve state and pinned upload staging for
// the server's lifetime; value and policy buffers come from the stream-ordered
// allocator, so admitting and retiring a request never synchronises the device.
// Tables are built on the submitting thread.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <math.h>
#include <stdio.h>
#include <string.h>

#include "../../include/vi.h"
#include "vi_api_internal.h"
#include "vi_common.cuh"
#include "vi_kernels.h"

using namespace vib;

namespace {

constexpr int kSlotTabFloats = 16384;   // expectation-table capacity of a slot (64 KiB)
constexpr int kSweepsPerCheck = 4;      // batched sweeps between two status reads (small batches)
// Above this many active states a batched sweep outlasts the status round trip,
// and further sweeps would only delay the extraction of instances that stopped.
constexpr double kOneSweepStates = 1 << 20;
// retirement threads: results written straight into the callers' (pageable) buffers
// are mostly page faults and copies on the host, which several threads overlap
constexpr int kRetireThreads = 2;

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t id = 0;
    vi_problem_desc desc;
    KernelParams kp;               // built at submission (device pointers set at admission)
    std::vector<float> ftab;       // FP32 expectation tables
    int n_outcomes = 0;
    double tol = 1e-4;
    int max_iters = 0;
    size_t bytes = 0;              // device memory while admitted
    uint64_t n_states = 0;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    // result
    bool done = false;
    vi_status status = VI_OK;
    int iters = 0;
    double crit = 0.0;
    double *V = nullptr;           // pinned result buffers (from the server's free list)
    uint8_t *policy = nullptr;
    size_t V_cap = 0, policy_cap = 0;
    double *dst_V = nullptr;       // vi_server_submit_to: the caller's host buffers, written at retirement
    uint8_t *dst_policy = nullptr;
};

struct Slot {
    std::shared_ptr<Request> req;
    KernelParams kp;
    void *V = nullptr;             // float pairs
    void *scratch = nullptr;       // ping-pong partner, then the FP64 result
    uint8_t *policy = nullptr;
    int mode = MODE_SWEEP;
    int xw = 0, variant = 0, lpr = 0;
    uint32_t blocks = 0;
    size_t smem = 0;
    // owned for the server's lifetime
    SolveState *d_state = nullptr;
    SolveState *h_state = nullptr;   // pinned
    float *d_tab = nullptr;
    float *h_tab = nullptr;          // pinned
};

struct RetireJob {
    std::shared_ptr<Request> req;
    void *V = nullptr, *scratch = nullptr;
    uint8_t *policy = nullptr;
    cudaEvent_t ready = nullptr;
    uint32_t n = 0;
    SlotStatus ss;
};

}  // namespace

struct vi_server_s {
    size_t budget = 0, used = 0;
    int max_slots = 0;
    cudaStream_t stream = nullptr;    // batched sweeps
    cudaStream_t rstream[kRetireThreads] = {};   // retirement copies, one stream per retirement thread
    cudaMemPool_t pool = nullptr;     // value and policy buffers; keeps up to the budget between requests
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> all;
    std::vector<Slot> slots;
    std::thread worker, retirer[kRetireThreads];
    std::deque<RetireJob> retire_q;
    std::condition_variable retire_cv;
    bool stop = false, retire_stop = false;
    uint64_t next_id = 1;
    std::multimap<size_t, void *> pinned_free;   // pinned result buffers by capacity (guarded by mu)
    std::deque<uint64_t> completed;               // finished, not yet reported by vi_server_wait
    std::condition_variable done_cv;
    vi_status fatal = VI_OK;
    char fatal_msg[256] = "";
    // batch descriptors (device) and their pinned host mirrors
    KernelParams *d_kps = nullptr, *h_kps = nullptr;
    int *d_modes = nullptr, *h_modes = nullptr;
    int *d_modes_sweep = nullptr;     // MODE_SWEEP for every slot: the later sweeps of an iteration
    int *d_lprs = nullptr, *h_lprs = nullptr;
    uint32_t *d_bstart = nullptr, *h_bstart = nullptr;
    SolveState **d_sts = nullptr, **h_sts = nullptr;
    SlotStatus *d_status = nullptr, *h_status = nullptr;
};

static size_t request_bytes(uint64_t n) { return (size_t)n * (8 + 8 + 1) + (1 << 16); }

// a pinned host buffer of at least `bytes` (power-of-two capacity, 64 KiB or more)
static void *pinned_get(vi_server_s *srv, size_t bytes, size_t *cap) {
    size_t c = (size_t)1 << 16;
    while (c < bytes) c <<= 1;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->pinned_free.find(c);
        if (it != srv->pinned_free.end()) {
            void *p = it->second;
            srv->pinned_free.erase(it);
            *cap = c;
            return p;
        }
    }
    void *p = nullptr;
    if (cudaMallocHost(&p, c) != cudaSuccess) return nullptr;
    *cap = c;
    return p;
}

// caller holds srv->mu
static void pinned_put_locked(vi_server_s *srv, void *p, size_t cap) {
    if (p) srv->pinned_free.emplace(cap, p);
}

static bool server_shape_ok(const vi_problem_desc &d) {
    if (d.n_products != 1) return false;
    const int K = (d.m[0] - 1) + (d.L[0] - 1);
    return K >= 1 && d.Q[0] + 1 >= 2 && d.Q[0] + 1 <= 24;
}

static void set_fatal(vi_server_s *srv, const char *what, cudaError_t e) {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->fatal == VI_OK) {
        srv->fatal = VI_ECUDA;
        snprintf(srv->fatal_msg, sizeof(srv->fatal_msg), "%s: %s", what, cudaGetErrorString(e));
    }
    srv->stop = true;
    srv->cv.notify_all();
}

// admit a request into a free slot (worker thread; nothing here waits for the device)
static vi_status slot_open(vi_server_s *srv, Slot &sl, std::shared_ptr<Request> req) {
    sl.req = req;
    sl.kp = req->kp;
    const uint32_t n = sl.kp.nS;
    memcpy(sl.h_tab, req->ftab.data(), req->ftab.size() * sizeof(float));
    sl.kp.tables = sl.d_tab;
    sl.kp.st = sl.d_state;
    cudaError_t e;
    if ((e = cudaMallocFromPoolAsync(&sl.V, (size_t)n * 8, srv->pool, srv->stream)) != cudaSuccess ||
        (e = cudaMallocFromPoolAsync(&sl.scratch, (size_t)n * 8, srv->pool, srv->stream)) != cudaSuccess ||
        (e = cudaMallocFromPoolAsync((void **)&sl.policy, n, srv->pool, srv->stream)) != cudaSuccess)
        return vi_fail(VI_ENOMEM, "server slot allocation: %s", cudaGetErrorString(e));
    SolveState *hs = sl.h_state;
    memset(hs, 0, sizeof(SolveState));
    hs->buf[0] = sl.V;
    hs->buf[1] = sl.scratch;
    hs->policy = sl.policy;
    hs->tol = req->tol;
    hs->gamma = req->desc.gamma;
    hs->max_iters = req->max_iters;
    hs->stop_rule = VI_STOP_SPAN;
    hs->value_bytes = 8;
    hs->key_min = ~0ull;
    if ((e = cudaMemcpyAsync(sl.d_tab, sl.h_tab, req->ftab.size() * sizeof(float), cudaMemcpyHostToDevice,
                             srv->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(sl.d_state, hs, sizeof(SolveState), cudaMemcpyHostToDevice, srv->stream)) !=
            cudaSuccess ||
        (e = launch_solve_init(sl.d_state, n, srv->stream)) != cudaSuccess)
        return vi_fail(VI_ECUDA, "server slot init: %s", cudaGetErrorString(e));
    sl.mode = req->max_iters > 0 ? MODE_SWEEP : MODE_EXTRACT;
    sl.xw = batch_width(sl.kp.p[0].G);
    sl.variant = batch_variant(sl.kp);
    batch_geometry(sl.kp, &sl.lpr, &sl.blocks, &sl.smem);
    return VI_OK;
}

// give the slot's buffers back (stream ordered) and free the slot
static void slot_release(vi_server_s *srv, Slot &sl) {
    if (sl.V) cudaFreeAsync(sl.V, srv->stream);
    if (sl.scratch) cudaFreeAsync(sl.scratch, srv->stream);
    if (sl.policy) cudaFreeAsync(sl.policy, srv->stream);
    sl.V = sl.scratch = nullptr;
    sl.policy = nullptr;
    sl.req.reset();
}

static void finish(vi_server_s *srv, Request &rq, vi_status st) {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (st != VI_OK) rq.status = st;
    rq.done = true;
    rq.t_done = now_s();
    srv->used -= rq.bytes;
    srv->completed.push_back(rq.id);
    srv->cv.notify_all();
    srv->done_cv.notify_all();
}

// retirement thread: wait for a finished instance's FP64 conversion, copy the
// values and the policy to host memory (the caller's buffers given at submission,
// else pinned buffers of the server's), release the device buffers
static void retire_loop(vi_server_s *srv, int k) {
    cudaStream_t rs = srv->rstream[k];
    while (true) {
        RetireJob job;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            srv->retire_cv.wait(lk, [srv] { return srv->retire_stop || !srv->retire_q.empty(); });
            if (srv->retire_q.empty()) break;   // stop requested and nothing left
            job = srv->retire_q.front();
            srv->retire_q.pop_front();
        }
        Request &rq = *job.req;
        vi_status st = VI_OK;
        // device -> pinned staging (a pageable destination would make the copy
        // synchronous and hold up the worker's launches), then, for
        // vi_server_submit_to, a host copy into the caller's buffers on this thread
        rq.V = (double *)pinned_get(srv, (size_t)job.n * 8, &rq.V_cap);
        rq.policy = (uint8_t *)pinned_get(srv, job.n, &rq.policy_cap);
        cudaError_t e;
        if (!rq.V || !rq.policy) {
            st = vi_fail(VI_ENOMEM, "server retire: no pinned host memory for the result");
        } else if ((e = cudaStreamWaitEvent(rs, job.ready, 0)) != cudaSuccess ||
                   (e = cudaMemcpyAsync(rq.V, job.scratch, (size_t)job.n * 8, cudaMemcpyDeviceToHost, rs)) !=
                       cudaSuccess ||
                   (e = cudaMemcpyAsync(rq.policy, job.policy, job.n, cudaMemcpyDeviceToHost, rs)) != cudaSuccess ||
                   (e = cudaStreamSynchronize(rs)) != cudaSuccess) {
            st = vi_fail(VI_ECUDA, "server retire: %s", cudaGetErrorString(e));
        }
        cudaFreeAsync(job.V, rs);
        cudaFreeAsync(job.scratch, rs);
        cudaFreeAsync(job.policy, rs);
        if (st == VI_OK && (rq.dst_V || rq.dst_policy)) {
            if (rq.dst_V) memcpy(rq.dst_V, rq.V, (size_t)job.n * 8);
            if (rq.dst_policy) memcpy(rq.dst_policy, rq.policy, job.n);
            std::lock_guard<std::mutex> lk(srv->mu);
            if (rq.dst_V) {
                pinned_put_locked(srv, rq.V, rq.V_cap);
                rq.V = nullptr;
            }
            if (rq.dst_policy) {
                pinned_put_locked(srv, rq.policy, rq.policy_cap);
                rq.policy = nullptr;
            }
        }
        cudaEventDestroy(job.ready);
        rq.iters = job.ss.iter;
        rq.crit = job.ss.crit;
        rq.status = job.ss.converged ? VI_OK : VI_ENOTCONVERGED;
        finish(srv, rq, st);
    }
}

// one launch per (lane width, variant) class over the active slots; modes from the
// slots (first sweep of an iteration) or MODE_SWEEP for all (the later ones)
static cudaError_t launch_round(vi_server_s *srv, const std::vector<int> &act, bool first) {
    int koff = 0, boff = 0;
    for (int cls = 0; cls < 5 * 4; ++cls) {
        static const int widths[5] = {8, 12, 16, 21, 24};
        const int xw = widths[cls / 4], variant = cls % 4;
        const int kbase = koff, bbase = boff;
        uint32_t total = 0;
        size_t smem = 0;
        for (int i : act) {
            Slot &sl = srv->slots[i];
            if (sl.xw != xw || sl.variant != variant) continue;
            if (first) {
                srv->h_kps[koff] = sl.kp;
                srv->h_modes[koff] = sl.mode;
                srv->h_lprs[koff] = sl.lpr;
                srv->h_bstart[boff] = total;
            }
            ++boff;
            total += sl.blocks;
            smem = std::max(smem, sl.smem);
            ++koff;
        }
        const int n_cls = koff - kbase;
        if (n_cls == 0) continue;
        if (first) srv->h_bstart[boff] = total;
        ++boff;
        cudaError_t e;
        if (first) {
            if ((e = cudaMemcpyAsync(srv->d_kps + kbase, srv->h_kps + kbase, sizeof(KernelParams) * n_cls,
                                     cudaMemcpyHostToDevice, srv->stream)) != cudaSuccess ||
                (e = cudaMemcpyAsync(srv->d_modes + kbase, srv->h_modes + kbase, sizeof(int) * n_cls,
                                     cudaMemcpyHostToDevice, srv->stream)) != cudaSuccess ||
                (e = cudaMemcpyAsync(srv->d_lprs + kbase, srv->h_lprs + kbase, sizeof(int) * n_cls,
                                     cudaMemcpyHostToDevice, srv->stream)) != cudaSuccess ||
                (e = cudaMemcpyAsync(srv->d_bstart + bbase, srv->h_bstart + bbase, sizeof(uint32_t) * (n_cls + 1),
                                     cudaMemcpyHostToDevice, srv->stream)) != cudaSuccess)
                return e;
        }
        e = launch_sweep_batch(xw, variant, srv->d_kps + kbase, (first ? srv->d_modes : srv->d_modes_sweep) + kbase,
                               srv->d_lprs + kbase, srv->d_bstart + bbase, n_cls, total, smem, srv->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static void worker_loop(vi_server_s *srv) {
    const int cap = srv->max_slots;
    while (true) {
        std::vector<std::shared_ptr<Request>> admit;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            if (srv->stop) break;
            int active = 0;
            for (auto &s : srv->slots) active += (s.req != nullptr);
            while (!srv->queue.empty() && active + (int)admit.size() < cap) {
                auto &q = srv->queue.front();
                if (srv->used + q->bytes > srv->budget) break;   // admission in arrival order
                srv->used += q->bytes;
                q->t_admit = now_s();
                admit.push_back(q);
                srv->queue.pop_front();
            }
            if (active == 0 && admit.empty()) {
                srv->cv.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        for (auto &rq : admit) {
            auto it = std::find_if(srv->slots.begin(), srv->slots.end(), [](const Slot &s) { return !s.req; });
            vi_status st = slot_open(srv, *it, rq);
            if (st != VI_OK) {
                slot_release(srv, *it);
                finish(srv, *rq, st);
            }
        }
        std::vector<int> act;
        bool sweeping = false;
        double states = 0.0;
        for (int i = 0; i < cap; ++i)
            if (srv->slots[i].req) {
                act.push_back(i);
                sweeping |= (srv->slots[i].mode == MODE_SWEEP);
                states += (double)srv->slots[i].kp.nS;
            }
        if (act.empty()) continue;
        // a few sweeps back to back while the batch is small: an instance that stopped
        // turns the later ones into no-ops
        const int rounds = (sweeping && states < kOneSweepStates) ? kSweepsPerCheck : 1;
        cudaError_t e = cudaSuccess;
        for (int rd = 0; rd < rounds && e == cudaSuccess; ++rd) e = launch_round(srv, act, rd == 0);
        if (e != cudaSuccess) {
            set_fatal(srv, "batched sweep", e);
            break;
        }
        for (size_t j = 0; j < act.size(); ++j) srv->h_sts[j] = srv->slots[act[j]].d_state;
        if ((e = cudaMemcpyAsync(srv->d_sts, srv->h_sts, sizeof(SolveState *) * act.size(), cudaMemcpyHostToDevice,
                                 srv->stream)) != cudaSuccess ||
            (e = launch_gather_status(srv->d_sts, (int)act.size(), srv->d_status, srv->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(srv->h_status, srv->d_status, sizeof(SlotStatus) * act.size(),
                                 cudaMemcpyDeviceToHost, srv->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(srv->stream)) != cudaSuccess) {
            set_fatal(srv, "server stream", e);
            break;
        }
        for (size_t j = 0; j < act.size(); ++j) {
            Slot &sl = srv->slots[act[j]];
            const SlotStatus ss = srv->h_status[j];
            if (sl.mode == MODE_EXTRACT) {
                // extraction done: FP64 values into the scratch buffer, then hand over
                RetireJob job;
                job.req = sl.req;
                job.V = sl.V;
                job.scratch = sl.scratch;
                job.policy = sl.policy;
                job.n = sl.kp.nS;
                job.ss = ss;
                if ((e = launch_to_fp64(sl.V, VK_PAIR, 0.0, (double *)sl.scratch, job.n, srv->stream)) !=
                        cudaSuccess ||
                    (e = cudaEventCreateWithFlags(&job.ready, cudaEventDisableTiming)) != cudaSuccess ||
                    (e = cudaEventRecord(job.ready, srv->stream)) != cudaSuccess) {
                    set_fatal(srv, "server retire", e);
                    break;
                }
                sl.V = sl.scratch = nullptr;
                sl.policy = nullptr;
                sl.req.reset();
                std::lock_guard<std::mutex> lk(srv->mu);
                srv->retire_q.push_back(job);
                srv->retire_cv.notify_one();
            } else if (!ss.keep_going) {
                sl.mode = MODE_EXTRACT;
            }
        }
        if (e != cudaSuccess) break;
    }
    // cancel whatever is left
    for (auto &sl : srv->slots)
        if (sl.req) {
            auto rq = sl.req;
            slot_release(srv, sl);
            finish(srv, *rq, VI_ECANCELLED);
        }
    std::lock_guard<std::mutex> lk(srv->mu);
    for (auto &rq : srv->queue) {
        rq->status = VI_ECANCELLED;
        rq->done = true;
        rq->t_done = now_s();
    }
    srv->queue.clear();
    srv->cv.notify_all();
}

extern "C" vi_status vi_server_create(size_t mem_budget_bytes, int max_slots, void *stream, vi_server *out) {
    if (!out) return vi_fail(VI_EINVAL, "null out");
    *out = nullptr;
    if (max_slots < 1 || max_slots > 1024) return vi_fail(VI_EINVAL, "max_slots must be in 1..1024");
    if (mem_budget_bytes < (1u << 20)) return vi_fail(VI_EINVAL, "memory budget below 1 MiB");
    vi_server_s *srv = new (std::nothrow) vi_server_s();
    if (!srv) return vi_fail(VI_ENOMEM, "host allocation failed");
    srv->budget = mem_budget_bytes;
    srv->max_slots = max_slots;
    srv->slots.resize(max_slots);
    const int n = max_slots + 24;   // one extra block_start entry per (width, variant) class
    int dev = 0;
    cudaGetDevice(&dev);
    cudaError_t e;
    {
        // a pool of its own whose freed memory stays reserved up to the budget: the default
        // pool would hand it back at every synchronisation and the next admission would
        // map fresh memory
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        uint64_t keep = (uint64_t)mem_budget_bytes;
        if ((e = cudaMemPoolCreate(&srv->pool, &props)) != cudaSuccess ||
            (e = cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            vi_server_destroy(srv);
            return vi_fail(VI_ECUDA, "server memory pool: %s", cudaGetErrorString(e));
        }
        // map part of the budget now, so that the first large admissions do not pay for it
        void *warm = nullptr;
        const size_t warm_bytes = std::min(mem_budget_bytes, (size_t)1 << 30);
        if (cudaMallocFromPoolAsync(&warm, warm_bytes, srv->pool, nullptr) == cudaSuccess) {
            cudaFreeAsync(warm, nullptr);
            cudaStreamSynchronize(nullptr);
        } else {
            cudaGetLastError();   // not enough free memory to reserve now: grow on demand instead
        }
    }
    if ((e = cudaStreamCreateWithFlags(&srv->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&srv->rstream[0], cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&srv->rstream[1], cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaMalloc(&srv->d_kps, sizeof(KernelParams) * n)) != cudaSuccess ||
        (e = cudaMallocHost(&srv->h_kps, sizeof(KernelParams) * n)) != cudaSuccess ||
        (e = cudaMalloc(&srv->d_modes, sizeof(int) * n)) != cudaSuccess ||
        (e = cudaMalloc(&srv->d_modes_sweep, sizeof(int) * n)) != cudaSuccess ||
        (e = cudaMallocHost(&srv->h_modes, sizeof(int) * n)) != cudaSuccess ||
        (e = cudaMalloc(&srv->d_lprs, sizeof(int) * n)) != cudaSuccess ||
        (e = cudaMallocHost(&srv->h_lprs, sizeof(int) * n)) != cudaSuccess ||
        (e = cudaMalloc(&srv->d_bstart, sizeof(uint32_t) * n)) != cudaSuccess ||
        (e = cudaMallocHost(&srv->h_bstart, sizeof(uint32_t) * n)) != cudaSuccess ||
        (e = cudaMalloc(&srv->d_sts, sizeof(SolveState *) * n)) != cudaSuccess ||
        (e = cudaMallocHost(&srv->h_sts, sizeof(SolveState *) * n)) != cudaSuccess ||
        (e = cudaMalloc(&srv->d_status, sizeof(SlotStatus) * n)) != cudaSuccess ||
        (e = cudaMallocHost(&srv->h_status, sizeof(SlotStatus) * n)) != cudaSuccess) {
        vi_server_destroy(srv);
        return vi_fail(e == cudaErrorMemoryAllocation ? VI_ENOMEM : VI_ECUDA, "server setup: %s",
                       cudaGetErrorString(e));
    }
    for (auto &sl : srv->slots)
        if ((e = cudaMalloc(&sl.d_state, sizeof(SolveState))) != cudaSuccess ||
            (e = cudaMallocHost(&sl.h_state, sizeof(SolveState))) != cudaSuccess ||
            (e = cudaMalloc(&sl.d_tab, sizeof(float) * kSlotTabFloats)) != cudaSuccess ||
            (e = cudaMallocHost(&sl.h_tab, sizeof(float) * kSlotTabFloats)) != cudaSuccess) {
            vi_server_destroy(srv);
            return vi_fail(e == cudaErrorMemoryAllocation ? VI_ENOMEM : VI_ECUDA, "server slots: %s",
                           cudaGetErrorString(e));
        }
    if ((e = prepare_sweep_batch()) != cudaSuccess || (e = prepare_server_helpers()) != cudaSuccess) {
        vi_server_destroy(srv);
        return vi_fail(VI_ECUDA, "server kernels: %s", cudaGetErrorString(e));
    }
    {
        std::vector<int> sweep(n, MODE_SWEEP);
        if ((e = cudaMemcpy(srv->d_modes_sweep, sweep.data(), sizeof(int) * n, cudaMemcpyHostToDevice)) !=
            cudaSuccess) {
            vi_server_destroy(srv);
            return vi_fail(VI_ECUDA, "server setup: %s", cudaGetErrorString(e));
        }
    }
    (void)stream;   // the server keeps its own streams so that its host loops never block the caller's
    srv->worker = std::thread([srv, dev]() {
        cudaSetDevice(dev);
        worker_loop(srv);
    });
    for (int k = 0; k < kRetireThreads; ++k)
        srv->retirer[k] = std::thread([srv, dev, k]() {
            cudaSetDevice(dev);
            retire_loop(srv, k);
        });
    *out = srv;
    return VI_OK;
}

extern "C" vi_status vi_server_submit(vi_server srv, const vi_problem_desc *desc, double tol, int max_iters,
                                      uint64_t *request_id) {
    return vi_server_submit_to(srv, desc, tol, max_iters, nullptr, nullptr, request_id);
}

extern "C" vi_status vi_server_submit_to(vi_server srv, const vi_problem_desc *desc, double tol, int max_iters,
                                         double *V_host, uint8_t *policy_host, uint64_t *request_id) {
    if (!srv || !desc || !request_id) return vi_fail(VI_EINVAL, "null argument");
    if (!server_shape_ok(*desc))
        return vi_fail(VI_EINVAL, "the server takes single-product instances with at least one state digit "
                                  "and 2 <= Q+1 <= 24");
    if (!(tol >= 0.0) || max_iters < 0) return vi_fail(VI_EINVAL, "need tol >= 0 and max_iters >= 0");
    auto rq = std::make_shared<Request>();
    rq->desc = *desc;
    rq->desc.precision = VI_PREC_FP32;
    rq->desc.stop_rule = VI_STOP_SPAN;
    vi_status st = build_single_product(rq->desc, rq->kp, rq->ftab, rq->n_outcomes);
    if (st != VI_OK) return st;
    if ((int)rq->ftab.size() > kSlotTabFloats)
        return vi_fail(VI_EINVAL, "expectation tables of %zu entries exceed a slot's %d", rq->ftab.size(),
                       kSlotTabFloats);
    rq->desc.pmf[0] = nullptr;   // the caller's pmf is not kept
    rq->dst_V = V_host;
    rq->dst_policy = policy_host;
    rq->tol = tol;
    rq->max_iters = max_iters;
    rq->n_states = rq->kp.nS;
    rq->bytes = request_bytes(rq->n_states);
    rq->t_submit = now_s();
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->fatal != VI_OK) return vi_fail(srv->fatal, "server stopped: %s", srv->fatal_msg);
    if (rq->bytes > srv->budget) return vi_fail(VI_EBUSY, "request needs %zu bytes, budget %zu", rq->bytes, srv->budget);
    rq->id = srv->next_id++;
    srv->all[rq->id] = rq;
    srv->queue.push_back(rq);
    *request_id = rq->id;
    srv->cv.notify_all();
    return VI_OK;
}

extern "C" vi_status vi_server_poll(vi_server srv, uint64_t request_id, int *done, double *V_host,
                                    uint8_t *policy_host, vi_solve_info *info) {
    if (!srv || !done) return vi_fail(VI_EINVAL, "null argument");
    std::shared_ptr<Request> rq;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->all.find(request_id);
        if (it == srv->all.end()) return vi_fail(VI_EINVAL, "unknown request id %llu", (unsigned long long)request_id);
        rq = it->second;
        *done = rq->done ? 1 : 0;
        if (!rq->done) return VI_OK;
        srv->all.erase(it);
    }
    if (V_host && rq->V) memcpy(V_host, rq->V, (size_t)rq->n_states * sizeof(double));
    if (policy_host && rq->policy) memcpy(policy_host, rq->policy, (size_t)rq->n_states);
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        pinned_put_locked(srv, rq->V, rq->V_cap);
        pinned_put_locked(srv, rq->policy, rq->policy_cap);
        rq->V = nullptr;
        rq->policy = nullptr;
    }
    if (info) {
        memset(info, 0, sizeof(*info));
        info->iters = rq->iters;
        info->status = rq->status;
        info->crit = rq->crit;
        info->wall_ms = 1e3 * (rq->t_done - rq->t_submit);
        const double nominal = (double)rq->n_states * (double)(rq->desc.Q[0] + 1) * (double)(rq->desc.dmax[0] + 1);
        const double run = rq->t_done - rq->t_admit;
        info->updates_per_s = run > 0 ? nominal * rq->iters / run : 0.0;
    }
    return rq->status;
}

extern "C" vi_status vi_server_wait(vi_server srv, int timeout_ms, uint64_t *ids, int max_ids, int *n_out) {
    if (!srv || !n_out || max_ids < 0 || (max_ids > 0 && !ids)) return vi_fail(VI_EINVAL, "bad arguments");
    *n_out = 0;
    std::unique_lock<std::mutex> lk(srv->mu);
    if (srv->completed.empty() && timeout_ms > 0)
        srv->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                              [srv] { return !srv->completed.empty() || srv->stop; });
    int n = 0;
    while (n < max_ids && !srv->completed.empty()) {
        ids[n++] = srv->completed.front();
        srv->completed.pop_front();
    }
    *n_out = n;
    return VI_OK;
}

extern "C" vi_status vi_server_destroy(vi_server srv) {
    if (!srv) return VI_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->cv.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->retire_stop = true;
        srv->retire_cv.notify_all();
    }
    for (auto &t : srv->retirer)
        if (t.joinable()) t.join();
    if (srv->stream) cudaStreamSynchronize(srv->stream);
    for (auto rs : srv->rstream)
        if (rs) cudaStreamSynchronize(rs);
    for (auto &sl : srv->slots) {
        if (sl.d_state) cudaFree(sl.d_state);
        if (sl.h_state) cudaFreeHost(sl.h_state);
        if (sl.d_tab) cudaFree(sl.d_tab);
        if (sl.h_tab) cudaFreeHost(sl.h_tab);
    }
    cudaFree(srv->d_kps);
    cudaFreeHost(srv->h_kps);
    cudaFree(srv->d_modes);
    cudaFree(srv->d_modes_sweep);
    cudaFreeHost(srv->h_modes);
    cudaFree(srv->d_lprs);
    cudaFreeHost(srv->h_lprs);
    cudaFree(srv->d_bstart);
    cudaFreeHost(srv->h_bstart);
    cudaFree(srv->d_sts);
    cudaFreeHost(srv->h_sts);
    cudaFree(srv->d_status);
    cudaFreeHost(srv->h_status);
    for (auto &kv : srv->all) {   // results that were never polled
        if (kv.second->V) cudaFreeHost(kv.second->V);
        if (kv.second->policy) cudaFreeHost(kv.second->policy);
    }
    for (auto &kv : srv->pinned_free) cudaFreeHost(kv.second);
    if (srv->stream) cudaStreamDestroy(srv->stream);
    for (auto rs : srv->rstream)
        if (rs) cudaStreamDestroy(rs);
    if (srv->pool) cudaMemPoolDestroy(srv->pool);
    delete srv;
    return VI_OK;
}

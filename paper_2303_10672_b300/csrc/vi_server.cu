// vi_server.cu -- continuous-batching solve server.
//
// A host worker thread owns one CUDA stream.  Requests wait in a FIFO queue and
// are admitted, in order, while a slot is free and their device memory (value
// ping-pong and policy) fits the budget.  Each pass of the worker is one launch
// of the persistent server kernel (vi_batch.cu) over every admitted instance:
// its blocks claim blocks of the instances' current sweeps, largest instances
// first, and each instance's next sweep -- or its extraction sweep, once its
// stopping test has passed -- opens as soon as its previous one has finished, so
// instances of every size and lane width advance together, each at its own
// pace, with no host round trip between sweeps.  A launch runs until its budget
// of device time is spent, every instance has finished, or -- while requests
// wait for a slot -- one has finished.  The worker enqueues the next pass before
// it reads the outcome of the previous one, so the device does not wait for the
// host.  A finished instance's values are converted to FP64 on the device and a
// retirement thread copies them and the policy to host memory, through two
// pinned staging chunks of its own, on a stream of its own, and releases the
// device buffers.  No host buffer is pinned per request: pinning (and the driver
// lock it holds) had stalled the worker's own calls.
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
// device time one launch of the server kernel may run before the worker looks at
// the queue again; while requests wait for a slot, a launch also ends once an
// instance has finished and it has run kPassMinNs (ending at every finish would
// leave the device mostly waiting for the launches' slowest blocks)
constexpr unsigned long long kPassBudgetNs = 1000000ull;
constexpr unsigned long long kPassMinNs = 200000ull;
// retirement threads: results written into the callers' (pageable) buffers are
// mostly page faults and copies on the host, which several threads overlap
constexpr int kRetireThreads = 4;
constexpr size_t kRetireStageBytes = (size_t)4 << 20;   // one of a thread's two pinned staging chunks

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
    double *V = nullptr;           // host result buffers (malloc) held until the poll, unless delivered
    uint8_t *policy = nullptr;
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
    uint64_t gen = 0;              // occupant count: a pass's status names the occupant it was read for
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
    void *rstage[kRetireThreads] = {};           // pinned staging of each retirement thread: two chunks
    cudaEvent_t rstage_ev[kRetireThreads][2] = {};
    std::deque<uint64_t> completed;               // finished, not yet reported by vi_server_wait
    std::condition_variable done_cv;
    vi_status fatal = VI_OK;
    char fatal_msg[256] = "";
    // per slot: kernel parameters and the server kernel's descriptor (device), with
    // pinned staging written at admission; the pass lists (active slots, their
    // state pointers, status, descriptors read back) have two pinned halves of
    // n_desc entries, one per pass in flight
    int n_desc = 0;
    KernelParams *d_kps = nullptr, *h_kps = nullptr;
    SrvSlot *d_srv = nullptr, *h_srv = nullptr;
    SrvSlot *h_srv_back = nullptr;    // descriptors read back after a pass (two halves)
    int *d_act = nullptr, *h_act = nullptr;
    unsigned *d_finished = nullptr;   // instances finished during the current launch
    SolveState **d_sts = nullptr, **h_sts = nullptr;
    SlotStatus *d_status = nullptr, *h_status = nullptr;
};

static size_t request_bytes(uint64_t n) { return (size_t)n * (8 + 8 + 1) + (1 << 16); }

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
    sl.gen += 1;
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
    // the instance's parameters and its descriptor for the server kernel
    const int idx = (int)(&sl - srv->slots.data());
    srv->h_kps[idx] = sl.kp;
    SrvSlot &d = srv->h_srv[idx];
    memset(&d, 0, sizeof(d));
    d.ticket = 0ull;
    d.done = 0u;
    d.mode = sl.mode;
    d.phase = (sl.mode == MODE_EXTRACT) ? 1 : 0;
    d.nblocks = sl.blocks;
    d.xw = sl.xw;
    d.variant = sl.variant;
    d.lpr = sl.lpr;
    if ((e = cudaMemcpyAsync(srv->d_kps + idx, srv->h_kps + idx, sizeof(KernelParams), cudaMemcpyHostToDevice,
                             srv->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(srv->d_srv + idx, &d, sizeof(SrvSlot), cudaMemcpyHostToDevice, srv->stream)) !=
            cudaSuccess)
        return vi_fail(VI_ECUDA, "server slot init: %s", cudaGetErrorString(e));
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

// device -> host copy of n bytes through the thread's two pinned staging chunks: the
// copy of one chunk runs while the previous one is copied on into dst on the host
// (a direct copy into pageable memory would be synchronous in the driver)
static cudaError_t copy_out(vi_server_s *srv, int k, void *dst, const void *src, size_t n) {
    cudaStream_t rs = srv->rstream[k];
    char *stage[2] = {(char *)srv->rstage[k], (char *)srv->rstage[k] + kRetireStageBytes};
    const size_t nc = (n + kRetireStageBytes - 1) / kRetireStageBytes;
    cudaError_t e = cudaSuccess;
    auto issue = [&](size_t c) {
        const size_t off = c * kRetireStageBytes, len = std::min(kRetireStageBytes, n - off);
        cudaError_t r = cudaMemcpyAsync(stage[c & 1], (const char *)src + off, len, cudaMemcpyDeviceToHost, rs);
        if (r == cudaSuccess) r = cudaEventRecord(srv->rstage_ev[k][c & 1], rs);
        return r;
    };
    if (nc > 0) e = issue(0);
    for (size_t c = 0; c < nc && e == cudaSuccess; ++c) {
        if (c + 1 < nc) e = issue(c + 1);
        if (e == cudaSuccess) e = cudaEventSynchronize(srv->rstage_ev[k][c & 1]);
        if (e == cudaSuccess) {
            const size_t off = c * kRetireStageBytes, len = std::min(kRetireStageBytes, n - off);
            memcpy((char *)dst + off, stage[c & 1], len);
        }
    }
    return e;
}

// retirement thread: copy a finished instance's FP64 values and policy to host
// memory -- the caller's buffers given at submission, else host buffers the server
// keeps until the poll -- and release its device buffers
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
        double *dV = rq.dst_V;
        uint8_t *dP = rq.dst_policy;
        if (!dV) dV = rq.V = (double *)malloc((size_t)job.n * 8);
        if (!dP) dP = rq.policy = (uint8_t *)malloc(job.n);
        cudaError_t e = cudaSuccess;
        if (!dV || !dP) {
            st = vi_fail(VI_ENOMEM, "server retire: no host memory for the result");
        } else if ((e = cudaStreamWaitEvent(rs, job.ready, 0)) != cudaSuccess ||
                   (e = copy_out(srv, k, dV, job.scratch, (size_t)job.n * 8)) != cudaSuccess ||
                   (e = copy_out(srv, k, dP, job.policy, job.n)) != cudaSuccess) {
            st = vi_fail(VI_ECUDA, "server retire: %s", cudaGetErrorString(e));
        }
        cudaFreeAsync(job.V, rs);
        cudaFreeAsync(job.scratch, rs);
        cudaFreeAsync(job.policy, rs);
        cudaEventDestroy(job.ready);
        rq.iters = job.ss.iter;
        rq.crit = job.ss.crit;
        rq.status = job.ss.converged ? VI_OK : VI_ENOTCONVERGED;
        finish(srv, rq, st);
    }
}

// a pass of batched sweeps whose status has not been read yet
struct Pass {
    bool valid = false;
    int buf = 0;                   // half of the pinned staging it used
    std::vector<int> slot;         // active slots, in the order of the status array
    std::vector<uint64_t> gen;     // their occupants when the pass was enqueued
};

// hand a slot whose extraction has run to a retirement thread
static cudaError_t retire_slot(vi_server_s *srv, Slot &sl, const SlotStatus &ss) {
    RetireJob job;
    job.req = sl.req;
    job.V = sl.V;
    job.scratch = sl.scratch;
    job.policy = sl.policy;
    job.n = sl.kp.nS;
    job.ss = ss;
    cudaError_t e;
    // FP64 values into the scratch buffer, after every sweep enqueued so far
    if ((e = launch_to_fp64(sl.V, VK_PAIR, 0.0, (double *)sl.scratch, job.n, srv->stream)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&job.ready, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventRecord(job.ready, srv->stream)) != cudaSuccess)
        return e;
    sl.V = sl.scratch = nullptr;
    sl.policy = nullptr;
    sl.req.reset();
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->retire_q.push_back(job);
    srv->retire_cv.notify_one();
    return cudaSuccess;
}

static void worker_loop(vi_server_s *srv) {
    const int cap = srv->max_slots;
    cudaEvent_t pass_done[2] = {nullptr, nullptr};
    for (auto &ev : pass_done)
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            set_fatal(srv, "server events", cudaGetLastError());
            return;
        }
    Pass prev;
    int buf = 0;
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
            if (active == 0 && admit.empty() && !prev.valid) {
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
        // -- enqueue this pass: one launch of the server kernel over every admitted
        // instance, then the status and the descriptors read back
        Pass cur;
        size_t smem = 0;
        for (int i = 0; i < cap; ++i)
            if (srv->slots[i].req) {
                cur.slot.push_back(i);
                smem = std::max(smem, srv->slots[i].smem);
            }
        // largest instances first: the kernel claims work in this order, so the device
        // works through one large sweep at a time and the small instances advance in the
        // gaps while a large sweep's last blocks finish
        std::stable_sort(cur.slot.begin(), cur.slot.end(),
                         [srv](int a, int b) { return srv->slots[a].kp.nS > srv->slots[b].kp.nS; });
        for (int i : cur.slot) cur.gen.push_back(srv->slots[i].gen);
        cudaError_t e = cudaSuccess;
        if (!cur.slot.empty()) {
            cur.valid = true;
            cur.buf = buf;
            const int na = (int)cur.slot.size();
            int *h_act = srv->h_act + buf * srv->n_desc;
            SolveState **h_sts = srv->h_sts + buf * srv->n_desc;
            for (int j = 0; j < na; ++j) {
                h_act[j] = cur.slot[j];
                h_sts[j] = srv->slots[cur.slot[j]].d_state;
            }
            bool queued;
            {
                std::lock_guard<std::mutex> lk(srv->mu);
                queued = !srv->queue.empty();
            }
            if ((e = cudaMemcpyAsync(srv->d_act, h_act, sizeof(int) * na, cudaMemcpyHostToDevice, srv->stream)) !=
                    cudaSuccess ||
                (e = cudaMemsetAsync(srv->d_finished, 0, sizeof(unsigned), srv->stream)) != cudaSuccess ||
                (e = launch_serve(srv->d_kps, srv->d_srv, srv->d_act, na, smem, kPassBudgetNs,
                                  queued ? kPassMinNs : 0ull, srv->d_finished, srv->stream)) != cudaSuccess) {
                set_fatal(srv, "server kernel", e);
                break;
            }
            if ((e = cudaMemcpyAsync(srv->d_sts, h_sts, sizeof(SolveState *) * na, cudaMemcpyHostToDevice,
                                     srv->stream)) != cudaSuccess ||
                (e = launch_gather_status(srv->d_sts, na, srv->d_status, srv->stream)) != cudaSuccess ||
                (e = cudaMemcpyAsync(srv->h_status + buf * srv->n_desc, srv->d_status, sizeof(SlotStatus) * na,
                                     cudaMemcpyDeviceToHost, srv->stream)) != cudaSuccess ||
                (e = cudaMemcpyAsync(srv->h_srv_back + buf * srv->n_desc, srv->d_srv, sizeof(SrvSlot) * cap,
                                     cudaMemcpyDeviceToHost, srv->stream)) != cudaSuccess ||
                (e = cudaEventRecord(pass_done[buf], srv->stream)) != cudaSuccess) {
                set_fatal(srv, "server stream", e);
                break;
            }
        }
        // -- the previous pass's outcome, read while this pass runs: an instance whose
        // extraction has been written is handed to a retirement thread
        if (prev.valid) {
            if ((e = cudaEventSynchronize(pass_done[prev.buf])) != cudaSuccess) {
                set_fatal(srv, "server stream", e);
                break;
            }
            const SlotStatus *hs = srv->h_status + prev.buf * srv->n_desc;
            const SrvSlot *hb = srv->h_srv_back + prev.buf * srv->n_desc;
            for (size_t j = 0; j < prev.slot.size() && e == cudaSuccess; ++j) {
                const int i = prev.slot[j];
                Slot &sl = srv->slots[i];
                if (!sl.req || sl.gen != prev.gen[j]) continue;   // retired since
                if (hb[i].phase == 2) {
                    e = retire_slot(srv, sl, hs[j]);
                    if (e != cudaSuccess) set_fatal(srv, "server retire", e);
                }
            }
            if (e != cudaSuccess) break;
        }
        prev = std::move(cur);
        buf ^= 1;
    }
    // cancel whatever is left once the last pass has finished
    if (srv->stream) cudaStreamSynchronize(srv->stream);
    for (auto &sl : srv->slots)
        if (sl.req) {
            auto rq = sl.req;
            slot_release(srv, sl);
            finish(srv, *rq, VI_ECANCELLED);
        }
    for (auto &ev : pass_done)
        if (ev) cudaEventDestroy(ev);
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
    const int n = max_slots;
    srv->n_desc = n;
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
    for (int k = 0; k < kRetireThreads; ++k)
        if ((e = cudaStreamCreateWithFlags(&srv->rstream[k], cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaMallocHost(&srv->rstage[k], 2 * kRetireStageBytes)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&srv->rstage_ev[k][0], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&srv->rstage_ev[k][1], cudaEventDisableTiming)) != cudaSuccess) {
            vi_server_destroy(srv);
            return vi_fail(e == cudaErrorMemoryAllocation ? VI_ENOMEM : VI_ECUDA, "server retirement set-up: %s",
                           cudaGetErrorString(e));
        }
    if ((e = cudaStreamCreateWithFlags(&srv->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaMalloc(&srv->d_kps, sizeof(KernelParams) * max_slots)) != cudaSuccess ||
        (e = cudaMallocHost(&srv->h_kps, sizeof(KernelParams) * max_slots)) != cudaSuccess ||
        (e = cudaMalloc(&srv->d_srv, sizeof(SrvSlot) * max_slots)) != cudaSuccess ||
        (e = cudaMallocHost(&srv->h_srv, sizeof(SrvSlot) * max_slots)) != cudaSuccess ||
        (e = cudaMallocHost(&srv->h_srv_back, sizeof(SrvSlot) * 2 * n)) != cudaSuccess ||
        (e = cudaMalloc(&srv->d_act, sizeof(int) * n)) != cudaSuccess ||
        (e = cudaMallocHost(&srv->h_act, sizeof(int) * 2 * n)) != cudaSuccess ||
        (e = cudaMalloc(&srv->d_finished, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMalloc(&srv->d_sts, sizeof(SolveState *) * n)) != cudaSuccess ||
        (e = cudaMallocHost(&srv->h_sts, sizeof(SolveState *) * 2 * n)) != cudaSuccess ||
        (e = cudaMalloc(&srv->d_status, sizeof(SlotStatus) * n)) != cudaSuccess ||
        (e = cudaMallocHost(&srv->h_status, sizeof(SlotStatus) * 2 * n)) != cudaSuccess) {
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
    free(rq->V);
    free(rq->policy);
    rq->V = nullptr;
    rq->policy = nullptr;
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
    cudaFree(srv->d_srv);
    cudaFreeHost(srv->h_srv);
    cudaFreeHost(srv->h_srv_back);
    cudaFree(srv->d_act);
    cudaFreeHost(srv->h_act);
    cudaFree(srv->d_finished);
    cudaFree(srv->d_sts);
    cudaFreeHost(srv->h_sts);
    cudaFree(srv->d_status);
    cudaFreeHost(srv->h_status);
    for (auto &kv : srv->all) {   // results that were never polled
        free(kv.second->V);
        free(kv.second->policy);
    }
    for (int k = 0; k < kRetireThreads; ++k) {
        if (srv->rstage[k]) cudaFreeHost(srv->rstage[k]);
        for (auto ev : srv->rstage_ev[k])
            if (ev) cudaEventDestroy(ev);
    }
    if (srv->stream) cudaStreamDestroy(srv->stream);
    for (auto rs : srv->rstream)
        if (rs) cudaStreamDestroy(rs);
    if (srv->pool) cudaMemPoolDestroy(srv->pool);
    delete srv;
    return VI_OK;
}

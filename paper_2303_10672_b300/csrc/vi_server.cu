// vi_server.cu -- continuous-batching solve server.
//
// A host worker thread owns one CUDA stream.  Requests wait in a FIFO queue and
// are admitted, in order, while a slot is free and their device memory (value
// ping-pong, policy, tables) fits the budget.  Every iteration of the worker runs
// one batched sweep over all admitted instances -- one launch per lane-width
// class, each block finding its instance from a prefix sum of block counts -- so
// instances of different sizes advance together.  An instance whose stopping
// test passed gets an extraction sweep in the next launch and is then retired:
// its values (FP64) and policy are copied to host memory, its device memory is
// released and queued requests can take its place.
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

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t id = 0;
    vi_problem_desc desc;
    std::vector<double> pmf;
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
    std::vector<double> V;
    std::vector<uint8_t> policy;
};

struct Slot {
    std::shared_ptr<Request> req;
    vi_handle h = nullptr;
    void *V = nullptr;             // float pairs
    uint8_t *policy = nullptr;
    int mode = MODE_SWEEP;
    int xw = 0, lpr = 0;
    uint32_t blocks = 0;
    size_t smem = 0;
    double updates = 0.0;          // nominal updates per sweep
};

}  // namespace

struct vi_server_s {
    size_t budget = 0, used = 0;
    int max_slots = 0;
    cudaStream_t stream = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> all;
    std::vector<Slot> slots;
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    vi_status fatal = VI_OK;
    char fatal_msg[256] = "";
    // batch descriptors (device) and their pinned host mirrors
    KernelParams *d_kps = nullptr, *h_kps = nullptr;
    int *d_modes = nullptr, *h_modes = nullptr;
    int *d_lprs = nullptr, *h_lprs = nullptr;
    uint32_t *d_bstart = nullptr, *h_bstart = nullptr;
    SolveState **d_sts = nullptr, **h_sts = nullptr;
    SlotStatus *d_status = nullptr, *h_status = nullptr;
};

static size_t request_bytes(uint64_t n) { return (size_t)n * (8 + 8 + 1) + (1 << 16); }

static bool server_shape_ok(const vi_problem_desc &d) {
    if (d.n_products != 1) return false;
    const int K = (d.m[0] - 1) + (d.L[0] - 1);
    return K >= 1 && d.Q[0] + 1 >= 2 && d.Q[0] + 1 <= 24;
}

// create the slot's problem, buffers and initial solve state (worker thread)
static vi_status slot_open(vi_server_s *srv, Slot &sl, std::shared_ptr<Request> req) {
    sl.req = req;
    vi_problem_desc d = req->desc;
    d.pmf[0] = req->pmf.data();
    d.precision = VI_PREC_FP32;
    d.stop_rule = VI_STOP_SPAN;
    vi_status st = vi_problem_create_desc(&d, &sl.h);
    if (st != VI_OK) return st;
    const uint32_t n = sl.h->kp.nS;
    cudaError_t e;
    if ((e = cudaMallocAsync(&sl.V, (size_t)n * 8, srv->stream)) != cudaSuccess ||
        (e = cudaMallocAsync(&sl.h->d_scratch, (size_t)n * 8, srv->stream)) != cudaSuccess ||
        (e = cudaMallocAsync((void **)&sl.policy, n, srv->stream)) != cudaSuccess)
        return vi_fail(VI_ENOMEM, "server slot allocation: %s", cudaGetErrorString(e));
    SolveState *hs = sl.h->h_state;
    memset(hs, 0, sizeof(SolveState));
    hs->buf[0] = sl.V;
    hs->buf[1] = sl.h->d_scratch;
    hs->policy = sl.policy;
    hs->tol = req->tol;
    hs->gamma = d.gamma;
    hs->max_iters = req->max_iters;
    hs->stop_rule = VI_STOP_SPAN;
    hs->value_bytes = 8;
    hs->key_min = ~0ull;
    if ((e = cudaMemcpyAsync(sl.h->d_state, hs, sizeof(SolveState), cudaMemcpyHostToDevice, srv->stream)) !=
        cudaSuccess)
        return vi_fail(VI_ECUDA, "server slot state: %s", cudaGetErrorString(e));
    if ((e = launch_solve_init(sl.h->d_state, n, srv->stream)) != cudaSuccess)
        return vi_fail(VI_ECUDA, "server slot init: %s", cudaGetErrorString(e));
    // pinned host mirror is reused for the next state upload; wait until the copy is done
    if ((e = cudaStreamSynchronize(srv->stream)) != cudaSuccess)
        return vi_fail(VI_ECUDA, "server slot init: %s", cudaGetErrorString(e));
    sl.mode = req->max_iters > 0 ? MODE_SWEEP : MODE_EXTRACT;
    sl.xw = batch_width(sl.h->kp.p[0].G);
    batch_geometry(sl.h->kp, &sl.lpr, &sl.blocks, &sl.smem);
    sl.updates = (double)n * (double)sl.h->kp.nA * (double)sl.h->n_outcomes;
    return VI_OK;
}

static void slot_close(vi_server_s *srv, Slot &sl) {
    if (sl.V) cudaFreeAsync(sl.V, srv->stream);
    if (sl.policy) cudaFreeAsync(sl.policy, srv->stream);
    if (sl.h) {
        if (sl.h->d_scratch) {
            cudaFreeAsync(sl.h->d_scratch, srv->stream);
            sl.h->d_scratch = nullptr;
        }
        cudaStreamSynchronize(srv->stream);
        vi_problem_destroy(sl.h);
    }
    sl = Slot();
}

// copy the finished instance to host memory (FP64 values in the scratch buffer)
static vi_status slot_retire(vi_server_s *srv, Slot &sl, const SlotStatus &ss) {
    Request &rq = *sl.req;
    const uint32_t n = sl.h->kp.nS;
    rq.V.resize(n);
    rq.policy.resize(n);
    cudaError_t e;
    if ((e = launch_to_fp64(sl.V, VK_PAIR, 0.0, (double *)sl.h->d_scratch, n, srv->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(rq.V.data(), sl.h->d_scratch, (size_t)n * 8, cudaMemcpyDeviceToHost, srv->stream)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(rq.policy.data(), sl.policy, n, cudaMemcpyDeviceToHost, srv->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(srv->stream)) != cudaSuccess)
        return vi_fail(VI_ECUDA, "server retire: %s", cudaGetErrorString(e));
    rq.iters = ss.iter;
    rq.crit = ss.crit;
    rq.status = ss.converged ? VI_OK : VI_ENOTCONVERGED;
    return VI_OK;
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
                std::lock_guard<std::mutex> lk(srv->mu);
                rq->status = st;
                rq->done = true;
                rq->t_done = now_s();
                srv->used -= rq->bytes;
                slot_close(srv, *it);
                srv->cv.notify_all();
            }
        }
        // one batched sweep (or extraction) for every active slot, per width class
        std::vector<int> act;
        for (int i = 0; i < cap; ++i)
            if (srv->slots[i].req) act.push_back(i);
        if (act.empty()) continue;
        int koff = 0, boff = 0;
        bool failed = false;
        for (int xw : {8, 12, 16, 21, 24}) {
            const int kbase = koff, bbase = boff;
            uint32_t total = 0;
            size_t smem = 0;
            for (int i : act) {
                Slot &sl = srv->slots[i];
                if (sl.xw != xw) continue;
                srv->h_kps[koff] = sl.h->kp;
                srv->h_modes[koff] = sl.mode;
                srv->h_lprs[koff] = sl.lpr;
                srv->h_bstart[boff++] = total;
                total += sl.blocks;
                smem = std::max(smem, sl.smem);
                ++koff;
            }
            const int n_cls = koff - kbase;
            if (n_cls == 0) continue;
            srv->h_bstart[boff++] = total;
            cudaMemcpyAsync(srv->d_kps + kbase, srv->h_kps + kbase, sizeof(KernelParams) * n_cls,
                            cudaMemcpyHostToDevice, srv->stream);
            cudaMemcpyAsync(srv->d_modes + kbase, srv->h_modes + kbase, sizeof(int) * n_cls,
                            cudaMemcpyHostToDevice, srv->stream);
            cudaMemcpyAsync(srv->d_lprs + kbase, srv->h_lprs + kbase, sizeof(int) * n_cls, cudaMemcpyHostToDevice,
                            srv->stream);
            cudaMemcpyAsync(srv->d_bstart + bbase, srv->h_bstart + bbase, sizeof(uint32_t) * (n_cls + 1),
                            cudaMemcpyHostToDevice, srv->stream);
            cudaError_t e = launch_sweep_batch(xw, srv->d_kps + kbase, srv->d_modes + kbase, srv->d_lprs + kbase,
                                               srv->d_bstart + bbase, n_cls, total, smem, srv->stream);
            if (e != cudaSuccess) {
                std::lock_guard<std::mutex> lk(srv->mu);
                srv->fatal = VI_ECUDA;
                snprintf(srv->fatal_msg, sizeof(srv->fatal_msg), "batched sweep: %s", cudaGetErrorString(e));
                srv->stop = true;
                failed = true;
                break;
            }
        }
        if (failed) break;
        // statuses of every active slot
        for (size_t j = 0; j < act.size(); ++j) srv->h_sts[j] = srv->slots[act[j]].h->d_state;
        cudaMemcpyAsync(srv->d_sts, srv->h_sts, sizeof(SolveState *) * act.size(), cudaMemcpyHostToDevice,
                        srv->stream);
        launch_gather_status(srv->d_sts, (int)act.size(), srv->d_status, srv->stream);
        cudaMemcpyAsync(srv->h_status, srv->d_status, sizeof(SlotStatus) * act.size(), cudaMemcpyDeviceToHost,
                        srv->stream);
        cudaError_t e = cudaStreamSynchronize(srv->stream);
        if (e != cudaSuccess) {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->fatal = VI_ECUDA;
            snprintf(srv->fatal_msg, sizeof(srv->fatal_msg), "server stream: %s", cudaGetErrorString(e));
            srv->stop = true;
            srv->cv.notify_all();
            break;
        }
        for (size_t j = 0; j < act.size(); ++j) {
            Slot &sl = srv->slots[act[j]];
            const SlotStatus ss = srv->h_status[j];
            if (sl.mode == MODE_EXTRACT) {
                vi_status st = slot_retire(srv, sl, ss);
                auto rq = sl.req;
                slot_close(srv, sl);
                std::lock_guard<std::mutex> lk(srv->mu);
                if (st != VI_OK) rq->status = st;
                rq->done = true;
                rq->t_done = now_s();
                srv->used -= rq->bytes;
                srv->cv.notify_all();
            } else if (!ss.keep_going) {
                sl.mode = MODE_EXTRACT;
            }
        }
    }
    // cancel whatever is left
    std::lock_guard<std::mutex> lk(srv->mu);
    for (auto &sl : srv->slots)
        if (sl.req) {
            sl.req->status = VI_ECANCELLED;
            sl.req->done = true;
            slot_close(srv, sl);
        }
    for (auto &q : srv->queue) {
        q->status = VI_ECANCELLED;
        q->done = true;
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
    const int n = max_slots + 8;   // one extra block_start entry per width class
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&srv->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaMalloc(&srv->d_kps, sizeof(KernelParams) * n)) != cudaSuccess ||
        (e = cudaMallocHost(&srv->h_kps, sizeof(KernelParams) * n)) != cudaSuccess ||
        (e = cudaMalloc(&srv->d_modes, sizeof(int) * n)) != cudaSuccess ||
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
    (void)stream;   // the server keeps its own stream so that its host loop never blocks the caller's
    int dev = 0;
    cudaGetDevice(&dev);
    srv->worker = std::thread([srv, dev]() {
        cudaSetDevice(dev);
        worker_loop(srv);
    });
    *out = srv;
    return VI_OK;
}

extern "C" vi_status vi_server_submit(vi_server srv, const vi_problem_desc *desc, double tol, int max_iters,
                                      uint64_t *request_id) {
    if (!srv || !desc || !request_id) return vi_fail(VI_EINVAL, "null argument");
    if (!server_shape_ok(*desc))
        return vi_fail(VI_EINVAL, "the server takes single-product instances with at least one state digit "
                                  "and 2 <= Q+1 <= 24");
    if (!(tol >= 0.0) || max_iters < 0) return vi_fail(VI_EINVAL, "need tol >= 0 and max_iters >= 0");
    // validate everything vi_problem_create_desc would check, on the host, now
    vi_problem_desc d = *desc;
    d.precision = VI_PREC_FP32;
    d.stop_rule = VI_STOP_SPAN;
    {
        const int K = (d.m[0] - 1) + (d.L[0] - 1);
        double ns = 1.0;
        for (int k = 0; k < K; ++k) ns *= (double)(d.Q[0] + 1);
        if (ns >= 4294967296.0) return vi_fail(VI_EINVAL, "|S| does not fit 32 bits");
        if (!d.pmf[0] || d.dmax[0] < 0 || d.dmax[0] > kMaxDmax) return vi_fail(VI_EINVAL, "bad pmf");
        double s = 0.0;
        for (int i = 0; i <= d.dmax[0]; ++i) {
            if (!(d.pmf[0][i] >= 0.0)) return vi_fail(VI_EINVAL, "pmf entries must be >= 0");
            s += d.pmf[0][i];
        }
        if (fabs(s - 1.0) > 1e-9) return vi_fail(VI_EINVAL, "pmf does not sum to 1");
        for (int j = 0; j < 5; ++j)
            if (!(d.cost[0][j] >= 0.0)) return vi_fail(VI_EINVAL, "costs must be >= 0");
        if (!(d.gamma > 0.0 && d.gamma <= 1.0)) return vi_fail(VI_EINVAL, "gamma must be in (0, 1]");
        if (d.issuing != VI_FIFO && d.issuing != VI_LIFO) return vi_fail(VI_EINVAL, "bad issuing rule");
        auto rq = std::make_shared<Request>();
        rq->desc = d;
        rq->pmf.assign(d.pmf[0], d.pmf[0] + d.dmax[0] + 1);
        rq->tol = tol;
        rq->max_iters = max_iters;
        rq->n_states = (uint64_t)ns;
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
    }
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
    if (V_host && !rq->V.empty()) memcpy(V_host, rq->V.data(), rq->V.size() * sizeof(double));
    if (policy_host && !rq->policy.empty()) memcpy(policy_host, rq->policy.data(), rq->policy.size());
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

extern "C" vi_status vi_server_destroy(vi_server srv) {
    if (!srv) return VI_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->cv.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    if (srv->stream) cudaStreamSynchronize(srv->stream);
    cudaFree(srv->d_kps);
    cudaFreeHost(srv->h_kps);
    cudaFree(srv->d_modes);
    cudaFreeHost(srv->h_modes);
    cudaFree(srv->d_lprs);
    cudaFreeHost(srv->h_lprs);
    cudaFree(srv->d_bstart);
    cudaFreeHost(srv->h_bstart);
    cudaFree(srv->d_sts);
    cudaFreeHost(srv->h_sts);
    cudaFree(srv->d_status);
    cudaFreeHost(srv->h_status);
    if (srv->stream) cudaStreamDestroy(srv->stream);
    delete srv;
    return VI_OK;
}

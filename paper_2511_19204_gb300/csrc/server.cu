// Serving loop: continuous batching of controller requests on one GPU.
//
// A worker thread owns `max_inflight` launch slots (stream, event, pinned image, device
// launch block). The slots' device blocks and pinned images are allocated once, when the
// server is created, at a fixed capacity, and that reservation is charged to the memory
// budget for the server's lifetime; no slot ever grows, so the worker never calls
// cudaMalloc / cudaFree (which can synchronise the device) while launches run.
//
// Whenever a slot is free the worker admits pending requests in arrival order, skipping
// requests whose context is still in flight, while the device bytes of the admitted
// contexts fit in the budget left after the reservation and the batch's launch block fits
// in the slot, and launches them as one persistent batched kernel on the slot's stream
// (batch_impl.cuh). Requests that arrive while other launches run are admitted as soon as
// a slot and memory free up; their launch overlaps the running ones on the device (its
// blocks take SMs as the earlier launch drains). With a deadline set, a request still
// waiting for admission longer than the deadline is shed: it completes with
// MPPI_ERR_DEADLINE without running, so the queue (and the latency of what runs) stays
// bounded past capacity. Completion is observed by polling the slots' events.
//
// The lock guards the queues, tickets and counters only: batch images are built and
// launched, and results unpacked, outside it, so mppi_submit and mppi_poll never wait
// behind a launch.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <utility>
#include <vector>

#include "batch.h"
#include "capi_internal.h"
#include "nvtx.h"

namespace mppi {

constexpr int SERVER_MAX_BATCH = 512;
constexpr size_t SLOT_BYTES_MAX = (size_t)4 << 20;   // device launch block per slot
constexpr size_t SLOT_BYTES_MIN = (size_t)16 << 10;

static int64_t mono_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (int64_t)ts.tv_sec * 1000000000ll + ts.tv_nsec;
}

struct Request {
    uint64_t ticket = 0;
    mppi_ctx* ctx = nullptr;
    std::vector<double> state;
    std::vector<float> warm;
    bool has_warm = false;
    int64_t submit_ns = 0, done_ns = 0;
    bool done = false;
    mppi_status status = MPPI_PENDING;
    std::vector<float> mean, best;
    mppi_result info;
};

struct Slot {
    cudaStream_t stream = nullptr;
    BatchStreams aux;  // the groups' kernels fork onto these
    cudaEvent_t ev = nullptr;
    unsigned char* h_img = nullptr;   // [slot_bytes] pinned
    unsigned char* h_out = nullptr;   // [slot_bytes] pinned
    unsigned char* d_block = nullptr; // [slot_bytes] device
    bool busy = false;                // launched (or being launched) and not yet retired
    size_t bytes = 0;                 // context bytes charged to the budget
    std::vector<Request*> reqs;
    BatchLayout L;
    std::vector<size_t> in_off, out_off;
};

}  // namespace mppi

struct mppi_server {
    int device = 0;
    size_t budget = 0;
    size_t slot_bytes = 0;     // capacity of each slot's device block and pinned images
    size_t reserved = 0;       // max_inflight * slot_bytes, charged to the budget
    int max_inflight = 1;
    int64_t deadline_ns = 0;   // 0: no shedding
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<mppi::Request*> pending;
    std::unordered_map<uint64_t, mppi::Request*> tickets;
    std::deque<uint64_t> completed;
    std::vector<mppi::Slot> slots;
    std::unordered_set<mppi_ctx*> busy_ctx;
    std::thread worker;
    bool stop = false;
    size_t inflight_bytes = 0;
    uint64_t next_ticket = 1;
    int64_t n_submitted = 0, n_completed = 0, n_launches = 0, peak_bytes = 0, n_waited = 0, n_shed = 0;
    // the worker's longest pass of its loop and its longest launch and unpack calls (ns):
    // where a request's latency went when the device was not the reason
    int64_t max_pass_ns = 0, max_launch_ns = 0, max_unpack_ns = 0;
    size_t smem = 0;
    int capacity = 1;
};

namespace mppi {

// Completes a request (lock held): records it for mppi_next_completed.
static void complete(mppi_server* S, Request* r, mppi_status st, int64_t now) {
    r->status = st;
    r->done = true;
    r->done_ns = now;
    S->completed.push_back(r->ticket);
    S->n_completed++;
}

// Pending requests waiting longer than the deadline complete with MPPI_ERR_DEADLINE
// without running (lock held).
static void shed_expired(mppi_server* S, int64_t now) {
    if (S->deadline_ns <= 0) return;
    for (auto it = S->pending.begin(); it != S->pending.end();) {
        Request* r = *it;
        if (now - r->submit_ns > S->deadline_ns) {
            complete(S, r, MPPI_ERR_DEADLINE, now);
            S->n_shed++;
            it = S->pending.erase(it);
        } else {
            ++it;
        }
    }
}

// Pending requests for one free slot, in arrival order (lock held): a request waits while
// its context is in flight (it keeps its place), and admission stops at the first request
// whose context bytes exceed the budget left or whose launch block would overflow the slot.
static std::vector<Request*> take_requests(mppi_server* S, size_t* bytes_out) {
    std::vector<Request*> take;
    size_t bytes = 0, block = batch_fixed_bound();
    std::unordered_set<mppi_ctx*> in_batch;
    const size_t ctx_budget = S->budget - S->reserved;
    for (auto it = S->pending.begin(); it != S->pending.end() && (int)take.size() < SERVER_MAX_BATCH;) {
        Request* r = *it;
        if (S->busy_ctx.count(r->ctx) || in_batch.count(r->ctx)) {
            ++it;
            continue;
        }
        const size_t b = r->ctx->dev_bytes;
        const size_t lb = batch_instance_bound(r->ctx);
        if (S->inflight_bytes + bytes + b > ctx_budget) {
            S->n_waited++;
            break;  // arrival order: later requests wait behind it
        }
        if (block + lb > S->slot_bytes) break;  // the next slot takes it
        take.push_back(r);
        in_batch.insert(r->ctx);
        bytes += b;
        block += lb;
        it = S->pending.erase(it);
    }
    *bytes_out = bytes;
    return take;
}

// Builds and enqueues one slot's launch (no lock: the slot and its requests belong to the
// worker until they are published).
static cudaError_t launch_slot(mppi_server* S, Slot& s) {
    MPPI_NVTX("mppi_server_launch");
    std::vector<mppi_ctx*> ctxs;
    std::vector<const double*> states;
    std::vector<const float*> warms;
    for (Request* r : s.reqs) {
        ctxs.push_back(r->ctx);
        states.push_back(r->state.data());
        warms.push_back(r->has_warm ? r->warm.data() : nullptr);
    }
    s.L = layout_batch(ctxs.data(), (int)ctxs.size());
    if (s.L.dev_bytes > S->slot_bytes) return cudaErrorInvalidValue;  // excluded by take_requests
    fill_batch_image(ctxs.data(), s.L, states.data(), warms.data(), s.h_img, &s.in_off, &s.out_off);
    // grid: one block per prefilled tile, at most the resident capacity, so small
    // launches leave SMs to the launches running beside them
    const int grid = (int)std::max<long>(1, std::min<long>(S->capacity, s.L.nprefill));
    cudaError_t e = enqueue_batch(s.L, s.h_img, s.d_block, s.h_out, grid, S->smem, s.stream, s.aux);
    if (e == cudaSuccess) e = cudaEventRecord(s.ev, s.stream);
    return e;
}

// Results of a finished slot into its request records (no lock).
static mppi_status unpack_slot(Slot& s, cudaError_t q, std::vector<mppi_result>& infos) {
    MPPI_NVTX("mppi_server_retire");
    std::vector<mppi_ctx*> ctxs;
    std::vector<float*> means, bests;
    infos.assign(s.reqs.size(), mppi_result{});
    for (Request* r : s.reqs) {
        ctxs.push_back(r->ctx);
        r->mean.resize(r->ctx->E);
        r->best.resize(r->ctx->E);
        means.push_back(r->mean.data());
        bests.push_back(r->best.data());
    }
    if (q != cudaSuccess) return MPPI_ERR_CUDA;
    return unpack_batch(ctxs.data(), s.L, s.out_off, s.h_out, means.data(), bests.data(), infos.data());
}

static void worker_loop(mppi_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    int64_t pass_start = mono_ns();
    while (!S->stop) {
        {
            const int64_t now = mono_ns();
            S->max_pass_ns = std::max(S->max_pass_ns, now - pass_start);
            pass_start = now;
        }
        // 1. under the lock: finished slots, shedding, admission decisions
        std::vector<std::pair<Slot*, cudaError_t>> finished;
        for (Slot& s : S->slots) {
            if (!s.busy) continue;
            const cudaError_t q = cudaEventQuery(s.ev);
            if (q != cudaErrorNotReady) finished.push_back({&s, q});
        }
        const int64_t now = mono_ns();
        shed_expired(S, now);
        std::vector<Slot*> to_launch;
        for (Slot& s : S->slots) {
            if (s.busy || S->pending.empty()) continue;
            size_t bytes = 0;
            std::vector<Request*> take = take_requests(S, &bytes);
            if (take.empty()) break;
            for (Request* r : take) S->busy_ctx.insert(r->ctx);
            s.reqs = std::move(take);
            s.bytes = bytes;
            s.busy = true;
            S->inflight_bytes += bytes;
            S->peak_bytes = std::max<int64_t>(S->peak_bytes, (int64_t)(S->reserved + S->inflight_bytes));
            to_launch.push_back(&s);
        }
        if (finished.empty() && to_launch.empty()) {
            bool busy = false;
            for (Slot& s : S->slots) busy |= s.busy;
            if (busy) {
                // poll the launches in flight at ~20 us granularity
                S->cv_work.wait_for(lk, std::chrono::microseconds(20));
            } else {
                S->cv_work.wait_for(lk, std::chrono::milliseconds(S->deadline_ns > 0 ? 1 : 5),
                                    [&] { return S->stop || !S->pending.empty(); });
            }
            continue;
        }
        lk.unlock();
        // 2. without the lock: launches and result unpacking
        std::vector<cudaError_t> launch_err(to_launch.size(), cudaSuccess);
        int64_t t_launch = 0, t_unpack = 0;
        for (size_t k = 0; k < to_launch.size(); ++k) {
            const int64_t t0 = mono_ns();
            launch_err[k] = launch_slot(S, *to_launch[k]);
            t_launch = std::max(t_launch, mono_ns() - t0);
        }
        std::vector<std::vector<mppi_result>> infos(finished.size());
        std::vector<mppi_status> fin_st(finished.size());
        for (size_t k = 0; k < finished.size(); ++k) {
            const int64_t t0 = mono_ns();
            fin_st[k] = unpack_slot(*finished[k].first, finished[k].second, infos[k]);
            t_unpack = std::max(t_unpack, mono_ns() - t0);
        }
        lk.lock();
        S->max_launch_ns = std::max(S->max_launch_ns, t_launch);
        S->max_unpack_ns = std::max(S->max_unpack_ns, t_unpack);
        // 3. under the lock: publish
        const int64_t t_done = mono_ns();
        for (size_t k = 0; k < to_launch.size(); ++k) {
            Slot& s = *to_launch[k];
            if (launch_err[k] == cudaSuccess) {
                S->n_launches++;
                continue;
            }
            cuda_fail(nullptr, launch_err[k], "server launch");
            // nothing of a failed launch is in flight on the slot's stream that could still
            // write its buffers once the stream drains: wait for it, then release the slot
            lk.unlock();
            cudaStreamSynchronize(s.stream);
            lk.lock();
            for (Request* r : s.reqs) {
                S->busy_ctx.erase(r->ctx);
                complete(S, r, MPPI_ERR_CUDA, t_done);
            }
            S->inflight_bytes -= s.bytes;
            s.bytes = 0;
            s.reqs.clear();
            s.busy = false;
        }
        for (size_t k = 0; k < finished.size(); ++k) {
            Slot& s = *finished[k].first;
            const mppi_status st = fin_st[k];
            for (size_t i = 0; i < s.reqs.size(); ++i) {
                Request* r = s.reqs[i];
                r->info = infos[k][i];
                S->busy_ctx.erase(r->ctx);
                complete(S, r, (st == MPPI_ERR_TIMEOUT || st == MPPI_ERR_CUDA) ? st : infos[k][i].status, t_done);
            }
            S->inflight_bytes -= s.bytes;
            s.bytes = 0;
            s.reqs.clear();
            s.busy = false;
        }
        S->cv_done.notify_all();
    }
}

}  // namespace mppi

using namespace mppi;

extern "C" {

mppi_status mppi_server_create(int32_t device, size_t mem_budget_bytes, int32_t max_inflight, mppi_server** out) {
    if (!out || max_inflight < 1 || max_inflight > 64 || mem_budget_bytes == 0) return MPPI_ERR_INVALID_ARG;
    *out = nullptr;
    // each slot's launch block: up to 4 MiB, at most a quarter of the budget over all slots
    size_t slot = std::min(SLOT_BYTES_MAX, (mem_budget_bytes / (4 * (size_t)max_inflight)) & ~(size_t)255);
    if (slot < SLOT_BYTES_MIN) {
        set_error(nullptr, "the memory budget cannot hold the launch slots (16 KiB each at least, a quarter of the budget)");
        return MPPI_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
    mppi_server* S = new (std::nothrow) mppi_server();
    if (!S) return MPPI_ERR_OUT_OF_MEMORY;
    S->device = device;
    S->budget = mem_budget_bytes;
    S->max_inflight = max_inflight;
    S->slot_bytes = slot;
    S->reserved = slot * (size_t)max_inflight;
    int per_sm = 0, sms = 0;
    e = prepare_batch_kernel(992, &S->smem, &per_sm);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    S->capacity = std::max(1, per_sm) * std::max(1, sms);
    S->slots.resize(max_inflight);
    for (Slot& s : S->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = s.aux.ensure(BATCH_VARIANTS - 1);
        if (e == cudaSuccess) e = cudaMalloc(&s.d_block, slot);
        if (e == cudaSuccess) e = cudaMallocHost(&s.h_img, slot);
        if (e == cudaSuccess) e = cudaMallocHost(&s.h_out, slot);
        if (e == cudaSuccess) memset(s.h_img, 0, slot);
    }
    if (e != cudaSuccess) {
        mppi_status st = e == cudaErrorMemoryAllocation ? MPPI_ERR_OUT_OF_MEMORY : cuda_fail(nullptr, e, "server creation");
        mppi_server_destroy(S);
        return st;
    }
    S->peak_bytes = (int64_t)S->reserved;
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return MPPI_OK;
}

void mppi_server_destroy(mppi_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (Slot& s : S->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.ev) cudaEventDestroy(s.ev);
        if (s.stream) cudaStreamDestroy(s.stream);
        s.aux.release();
        if (s.h_img) cudaFreeHost(s.h_img);
        if (s.h_out) cudaFreeHost(s.h_out);
        if (s.d_block) cudaFree(s.d_block);
    }
    for (auto& kv : S->tickets) delete kv.second;
    delete S;
}

mppi_status mppi_server_set_deadline(mppi_server* S, int64_t deadline_us) {
    if (!S || deadline_us < 0) return MPPI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    S->deadline_ns = deadline_us * 1000;
    return MPPI_OK;
}

mppi_status mppi_submit(mppi_server* S, mppi_ctx* c, const double* h_state, const float* h_warm, uint64_t* ticket) {
    if (!S || !c || !h_state || !ticket) return MPPI_ERR_INVALID_ARG;
    mppi_status st = check_batchable(c, S->device);
    if (st != MPPI_OK) return st;
    for (int k = 0; k < c->nx; ++k)
        if (!isfinite(h_state[k])) {
            set_error(c, "state is not finite");
            return MPPI_ERR_NONFINITE_STATE;
        }
    if (c->dev_bytes > S->budget - S->reserved) {
        set_error(c, "the request alone exceeds the server's memory budget (after the launch slots' reservation)");
        return MPPI_ERR_ADMISSION;
    }
    if (batch_fixed_bound() + batch_instance_bound(c) > S->slot_bytes) {
        set_error(c, "the request's launch block alone exceeds a launch slot of the server");
        return MPPI_ERR_ADMISSION;
    }
    Request* r = new (std::nothrow) Request();
    if (!r) return MPPI_ERR_OUT_OF_MEMORY;
    r->ctx = c;
    r->state.assign(h_state, h_state + c->nx);
    if (h_warm) {
        r->warm.assign(h_warm, h_warm + c->E);
        r->has_warm = true;
    }
    r->submit_ns = mono_ns();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->ticket = S->next_ticket++;
        S->tickets[r->ticket] = r;
        S->pending.push_back(r);
        S->n_submitted++;
    }
    S->cv_work.notify_one();
    *ticket = r->ticket;
    return MPPI_OK;
}

mppi_status mppi_poll(mppi_server* S, uint64_t ticket, float* h_out_mean, float* h_out_best, mppi_result* h_info,
                      int64_t timeout_us) {
    if (!S) return MPPI_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return MPPI_ERR_NOT_FOUND;
    Request* r = it->second;
    if (!r->done && timeout_us != 0) {
        auto pred = [&] { return r->done; };
        if (timeout_us < 0) S->cv_done.wait(lk, pred);
        else S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred);
    }
    if (!r->done) return MPPI_PENDING;
    if (h_out_mean && !r->mean.empty()) memcpy(h_out_mean, r->mean.data(), sizeof(float) * r->mean.size());
    if (h_out_best && !r->best.empty()) memcpy(h_out_best, r->best.data(), sizeof(float) * r->best.size());
    if (h_info) *h_info = r->info;
    const mppi_status st = r->status;
    S->tickets.erase(it);
    delete r;
    return st;
}

mppi_status mppi_next_completed(mppi_server* S, int64_t timeout_us, uint64_t* ticket, int64_t* times_ns) {
    if (!S || !ticket) return MPPI_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->completed.empty() && timeout_us != 0) {
        auto pred = [&] { return !S->completed.empty(); };
        if (timeout_us < 0) S->cv_done.wait(lk, pred);
        else S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred);
    }
    if (S->completed.empty()) return MPPI_PENDING;
    *ticket = S->completed.front();
    S->completed.pop_front();
    if (times_ns) {
        auto it = S->tickets.find(*ticket);
        times_ns[0] = it != S->tickets.end() ? it->second->submit_ns : 0;
        times_ns[1] = it != S->tickets.end() ? it->second->done_ns : 0;
    }
    return MPPI_OK;
}

mppi_status mppi_server_stats_ex(mppi_server* S, int64_t* o, int32_t n) {
    if (!S || !o || n < 0) return MPPI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    const int64_t v[11] = {S->n_submitted,   S->n_completed, S->n_launches,       S->peak_bytes,
                           S->n_waited,      S->n_shed,      (int64_t)S->reserved, (int64_t)S->slot_bytes,
                           S->max_pass_ns,   S->max_launch_ns, S->max_unpack_ns};
    for (int k = 0; k < n && k < 11; ++k) o[k] = v[k];
    return MPPI_OK;
}

mppi_status mppi_server_stats(mppi_server* S, int64_t* o) { return mppi_server_stats_ex(S, o, 5); }

mppi_status mppi_server_reset_timing(mppi_server* S) {
    if (!S) return MPPI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    S->max_pass_ns = S->max_launch_ns = S->max_unpack_ns = 0;
    return MPPI_OK;
}

}  // extern "C"

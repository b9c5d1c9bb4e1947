// Serving loop: continuous batching of controller requests on one GPU.
//
// A worker thread owns `max_inflight` launch slots (stream, event, pinned image,
// device block). Whenever a slot is free it admits pending requests in arrival order,
// skipping requests whose context is still in flight, while the device bytes of the
// admitted contexts stay within the memory budget, and launches them as one persistent
// batched kernel on the slot's stream (batch.cu). Requests that arrive while other
// launches run are admitted as soon as a slot and memory free up; their launch overlaps
// the running ones on the device (its blocks take SMs as the earlier launch drains).
// Completion is observed by polling the slots' events; results are copied into the
// request records and the tickets queued for retrieval.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>
#include <time.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "batch.h"
#include "capi_internal.h"

namespace mppi {

constexpr int SERVER_MAX_BATCH = 512;

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
    unsigned char* h_img = nullptr;
    unsigned char* h_out = nullptr;
    unsigned char* d_block = nullptr;
    size_t cap_img = 0, cap_out = 0, cap_dev = 0;
    bool busy = false;
    size_t bytes = 0;
    std::vector<Request*> reqs;
    BatchLayout L;
    std::vector<size_t> in_off, out_off;
};

}  // namespace mppi

struct mppi_server {
    int device = 0;
    size_t budget = 0;
    int max_inflight = 1;
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
    int64_t n_submitted = 0, n_completed = 0, n_launches = 0, peak_bytes = 0, n_waited = 0;
    size_t smem = 0;
    int capacity = 1;
    mppi_status worker_error = MPPI_OK;
};

namespace mppi {

static cudaError_t grow(Slot& s, const BatchLayout& L) {
    cudaError_t e = cudaSuccess;
    if (L.image_bytes > s.cap_img) {
        if (s.h_img) cudaFreeHost(s.h_img);
        s.h_img = nullptr;
        e = cudaMallocHost(&s.h_img, L.image_bytes * 2);
        s.cap_img = e == cudaSuccess ? L.image_bytes * 2 : 0;
    }
    if (e == cudaSuccess && L.out_bytes > s.cap_out) {
        if (s.h_out) cudaFreeHost(s.h_out);
        s.h_out = nullptr;
        e = cudaMallocHost(&s.h_out, L.out_bytes * 2);
        s.cap_out = e == cudaSuccess ? L.out_bytes * 2 : 0;
    }
    if (e == cudaSuccess && L.dev_bytes > s.cap_dev) {
        if (s.d_block) cudaFree(s.d_block);
        s.d_block = nullptr;
        e = cudaMalloc(&s.d_block, L.dev_bytes * 2);
        s.cap_dev = e == cudaSuccess ? L.dev_bytes * 2 : 0;
    }
    return e;
}

// Completed slots -> request records (lock held).
static void retire(mppi_server* S) {
    for (Slot& s : S->slots) {
        if (!s.busy) continue;
        const cudaError_t q = cudaEventQuery(s.ev);
        if (q == cudaErrorNotReady) continue;
        const int64_t now = mono_ns();
        std::vector<mppi_ctx*> ctxs;
        std::vector<float*> means, bests;
        std::vector<mppi_result> infos(s.reqs.size());
        for (Request* r : s.reqs) {
            ctxs.push_back(r->ctx);
            r->mean.resize(r->ctx->E);
            r->best.resize(r->ctx->E);
            means.push_back(r->mean.data());
            bests.push_back(r->best.data());
        }
        mppi_status st = MPPI_ERR_CUDA;
        if (q == cudaSuccess)
            st = unpack_batch(ctxs.data(), s.L, s.out_off, s.h_out, means.data(), bests.data(), infos.data());
        for (size_t i = 0; i < s.reqs.size(); ++i) {
            Request* r = s.reqs[i];
            r->info = infos[i];
            r->status = (st == MPPI_ERR_TIMEOUT || st == MPPI_ERR_CUDA) ? st : infos[i].status;
            r->done = true;
            r->done_ns = now;
            S->busy_ctx.erase(r->ctx);
            S->completed.push_back(r->ticket);
            S->n_completed++;
        }
        S->inflight_bytes -= s.bytes;
        s.bytes = 0;
        s.reqs.clear();
        s.busy = false;
        S->cv_done.notify_all();
    }
}

// Admit pending requests into free slots (lock held). Returns true if it launched.
static bool admit(mppi_server* S) {
    bool launched = false;
    for (Slot& s : S->slots) {
        if (s.busy || S->pending.empty()) continue;
        std::vector<Request*> take;
        size_t bytes = 0;
        std::unordered_set<mppi_ctx*> in_batch;
        for (auto it = S->pending.begin(); it != S->pending.end() && (int)take.size() < SERVER_MAX_BATCH;) {
            Request* r = *it;
            const size_t b = r->ctx->dev_bytes;
            if (S->busy_ctx.count(r->ctx) || in_batch.count(r->ctx)) {
                ++it;  // its context is busy: it keeps its place in the queue
                continue;
            }
            if (S->inflight_bytes + bytes + b > S->budget) {
                S->n_waited++;
                break;  // arrival order: later requests wait behind it
            }
            take.push_back(r);
            in_batch.insert(r->ctx);
            bytes += b;
            it = S->pending.erase(it);
        }
        if (take.empty()) break;
        std::vector<mppi_ctx*> ctxs;
        std::vector<const double*> states;
        std::vector<const float*> warms;
        for (Request* r : take) {
            ctxs.push_back(r->ctx);
            states.push_back(r->state.data());
            warms.push_back(r->has_warm ? r->warm.data() : nullptr);
        }
        s.L = layout_batch(ctxs.data(), (int)ctxs.size());
        cudaError_t e = grow(s, s.L);
        if (e == cudaSuccess) {
            fill_batch_image(ctxs.data(), s.L, states.data(), warms.data(), s.h_img, &s.in_off, &s.out_off);
            // grid: one block per prefilled tile, at most the resident capacity, so small
            // launches leave SMs to the launches running beside them
            const int grid = (int)std::max<long>(1, std::min<long>(S->capacity, s.L.nprefill));
            e = enqueue_batch(s.L, s.h_img, s.d_block, s.h_out, grid, S->smem, s.stream, s.aux);
        }
        if (e == cudaSuccess) e = cudaEventRecord(s.ev, s.stream);
        if (e != cudaSuccess) {
            cuda_fail(nullptr, e, "server launch");
            for (Request* r : take) {
                r->status = MPPI_ERR_CUDA;
                r->done = true;
                r->done_ns = mono_ns();
                S->completed.push_back(r->ticket);
                S->n_completed++;
            }
            S->cv_done.notify_all();
            continue;
        }
        for (Request* r : take) S->busy_ctx.insert(r->ctx);
        s.reqs = take;
        s.bytes = bytes;
        s.busy = true;
        S->inflight_bytes += bytes;
        S->peak_bytes = std::max<int64_t>(S->peak_bytes, (int64_t)S->inflight_bytes);
        S->n_launches++;
        launched = true;
    }
    return launched;
}

static void worker_loop(mppi_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        retire(S);
        admit(S);
        bool busy = false;
        for (Slot& s : S->slots) busy |= s.busy;
        if (busy) {
            // poll the launches in flight at ~20 us granularity
            S->cv_work.wait_for(lk, std::chrono::microseconds(20));
        } else {
            S->cv_work.wait_for(lk, std::chrono::milliseconds(5), [&] { return S->stop || !S->pending.empty(); });
        }
    }
}

}  // namespace mppi

using namespace mppi;

extern "C" {

mppi_status mppi_server_create(int32_t device, size_t mem_budget_bytes, int32_t max_inflight, mppi_server** out) {
    if (!out || max_inflight < 1 || max_inflight > 64 || mem_budget_bytes == 0) return MPPI_ERR_INVALID_ARG;
    *out = nullptr;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
    mppi_server* S = new (std::nothrow) mppi_server();
    if (!S) return MPPI_ERR_OUT_OF_MEMORY;
    S->device = device;
    S->budget = mem_budget_bytes;
    S->max_inflight = max_inflight;
    int per_sm = 0, sms = 0;
    e = prepare_batch_kernel(992, &S->smem, &per_sm);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    S->capacity = std::max(1, per_sm) * std::max(1, sms);
    S->slots.resize(max_inflight);
    for (Slot& s : S->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        mppi_status st = cuda_fail(nullptr, e, "server creation");
        mppi_server_destroy(S);
        return st;
    }
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

mppi_status mppi_submit(mppi_server* S, mppi_ctx* c, const double* h_state, const float* h_warm, uint64_t* ticket) {
    if (!S || !c || !h_state || !ticket) return MPPI_ERR_INVALID_ARG;
    mppi_status st = check_batchable(c, S->device);
    if (st != MPPI_OK) return st;
    for (int k = 0; k < c->nx; ++k)
        if (!isfinite(h_state[k])) {
            set_error(c, "state is not finite");
            return MPPI_ERR_NONFINITE_STATE;
        }
    if (c->dev_bytes > S->budget) {
        set_error(c, "the request alone exceeds the server's memory budget");
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

mppi_status mppi_server_stats(mppi_server* S, int64_t* o) {
    if (!S || !o) return MPPI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    o[0] = S->n_submitted;
    o[1] = S->n_completed;
    o[2] = S->n_launches;
    o[3] = S->peak_bytes;
    o[4] = S->n_waited;
    return MPPI_OK;
}

}  // extern "C"

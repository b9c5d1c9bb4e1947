// Rollout-mapping autotuner: for one context, time every supported (mapping, block size)
// on the context's own buffers (knots drawn around the resident nominal) and keep the
// fastest. Results are cached per (device, model contents, K, H, knots) for the life of
// the process, so later contexts of the same shape reuse the choice without timing.
#include <cuda_runtime.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>

#include "capi_internal.h"

namespace mppi {

namespace {

struct TuneKey {
    int device;
    uint64_t model_hash;
    int N, H, nk;
    bool operator<(const TuneKey& o) const {
        return std::tie(device, model_hash, N, H, nk) < std::tie(o.device, o.model_hash, o.N, o.H, o.nk);
    }
};

struct TuneVal {
    int mapping, block;
    float ms[16];
};

std::mutex g_mu;
std::map<TuneKey, TuneVal> g_cache;

uint64_t fnv1a(const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

constexpr int kMappings[4] = {MPPI_MAP_WARP, MPPI_MAP_HALFWARP, MPPI_MAP_CHAIN, MPPI_MAP_THREAD};
constexpr int kBlocks[4] = {32, 64, 128, 256};

}  // namespace

mppi_status autotune_ctx(mppi_ctx* c, int reps, TuneVal* out) {
    // fill the context's knot buffer once: iteration-0 noise around the resident nominal
    SampleArgs sa;
    sa.nominal = c->d_nominal;
    sa.sigma_row = c->d_sigma;
    sa.model = (const DevModel<float>*)c->model->d_f;
    sa.knots = c->d_knots;
    sa.solve = nullptr;
    sa.iter_offset = 0;
    sa.iter_counter_override = 0x7fffffffu;
    sa.inst = c->instance_id;
    sa.seed_lo = (uint32_t)(c->seed & 0xffffffffu);
    sa.seed_hi = (uint32_t)(c->seed >> 32);
    sa.N = c->N;
    sa.nk = c->nk;
    sa.nj = c->nj;
    sa.has_limits = c->model->host_f.has_limits;
    sa.scale_q = (float)c->scale_q;
    sa.scale_v = (float)c->scale_v;
    sa.dtk = (float)c->dtk;
    sa.spline = c->spline;
    cudaError_t e = launch_sample_knots(sa, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "autotune: sample knots");
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_fail(c, e, "autotune: event");
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(c, e, "autotune: event");
    }
    const int saved_m = c->mapping, saved_b = c->block;
    float best = 1e30f;
    int bm = saved_m, bb = saved_b;
    for (int k = 0; k < 16; ++k) out->ms[k] = -1.f;
    // two rounds over every candidate, keeping each one's faster round: the first round
    // also absorbs the clock ramp of a GPU that was idle before the call
    for (int round = 0; round < 2; ++round) {
        for (int mi = 0; mi < 4; ++mi) {
            for (int bi = 0; bi < 4; ++bi) {
                const int m = kMappings[mi], b = kBlocks[bi];
                if (!mapping_valid(c->model, m, b)) continue;
                c->mapping = m;
                c->block = b;
                // one untimed launch, then reps timed ones
                e = enqueue_rollout(c, c->d_x0, c->d_knots, c->N, c->d_costs, nullptr, c->stream);
                if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
                for (int r = 0; r < reps && e == cudaSuccess; ++r)
                    e = enqueue_rollout(c, c->d_x0, c->d_knots, c->N, c->d_costs, nullptr, c->stream);
                if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    c->mapping = saved_m;
                    c->block = saved_b;
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return cuda_fail(c, e, "autotune: timed rollout");
                }
                ms /= (float)reps;
                float& slot = out->ms[mi * 4 + bi];
                if (slot < 0.f || ms < slot) slot = ms;
                if (ms < best) {
                    best = ms;
                    bm = m;
                    bb = b;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->mapping = bm;
    c->block = bb;
    out->mapping = bm;
    out->block = bb;
    return MPPI_OK;
}

}  // namespace mppi

using namespace mppi;

extern "C" mppi_status mppi_autotune(mppi_ctx* c, int32_t* mapping, int32_t* block, float* h_ms) {
    if (!c) return MPPI_ERR_INVALID_ARG;
    // the timed rollouts start from the context's last state if a solve ran, else from
    // the model's rest pose half a metre above the ground
    TuneKey key{c->device, fnv1a(&c->model->host_f, sizeof(DevModel<float>)), c->N, c->H, c->nk};
    TuneVal v;
    bool hit = false;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            v = it->second;
            hit = true;
        }
    }
    if (!hit) {
        if (!c->has_state) {
            std::vector<double> x(c->nx, 0.0);
            x[2] = 0.5;
            x[3] = 1.0;
            for (int j = 0; j < c->nj; ++j) x[7 + j] = c->model->q_init[j];
            cudaError_t e =
                cudaMemcpyAsync(c->d_x0, x.data(), sizeof(double) * c->nx, cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "autotune: state");
        }
        mppi_status st = autotune_ctx(c, 3, &v);
        if (st != MPPI_OK) return st;
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key] = v;
    } else {
        c->mapping = v.mapping;
        c->block = v.block;
    }
    invalidate_graph(c);
    if (mapping) *mapping = v.mapping;
    if (block) *block = v.block;
    if (h_ms) memcpy(h_ms, v.ms, sizeof v.ms);
    return MPPI_OK;
}

// Rollout-mapping autotuner: for one context, time every supported (mapping, block size)
// on the context's own buffers (knots drawn around the resident nominal) and keep the
// fastest. Results are cached per (device type, model contents, K, H, knots) for the life
// of the process, and, once a cache file is named (mppi_autotune_cache_file), in that JSON
// file too, so later processes on the same kind of GPU reuse the choice without timing.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "capi_internal.h"
#include "nvtx.h"

namespace mppi {

namespace {

struct TuneKey {
    std::string device;  // "<name>|<SM count>|<compute capability>"
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
std::string g_cache_path;  // empty: the process cache only

std::string device_id(int dev) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "device" + std::to_string(dev);
    std::string name(p.name);
    for (char& ch : name)
        if (ch == '"' || ch == '|' || ch == '\\') ch = '_';
    return name + "|" + std::to_string(p.multiProcessorCount) + "|" + std::to_string(p.major) + "." +
           std::to_string(p.minor);
}

// ---- the JSON cache file: an array with one object per line, written and read here ----
// {"device": "<id>", "model": "<16 hex digits>", "K": n, "H": n, "knots": n, "mapping": n,
//  "block": n, "ms": [16 numbers]}

std::string entry_json(const TuneKey& k, const TuneVal& v) {
    char head[512];
    snprintf(head, sizeof head,
             "{\"device\": \"%s\", \"model\": \"%016llx\", \"K\": %d, \"H\": %d, \"knots\": %d, "
             "\"mapping\": %d, \"block\": %d, \"ms\": [",
             k.device.c_str(), (unsigned long long)k.model_hash, k.N, k.H, k.nk, v.mapping, v.block);
    std::string out(head);
    for (int i = 0; i < 16; ++i) {
        char num[32];
        snprintf(num, sizeof num, "%s%.6g", i ? ", " : "", (double)v.ms[i]);
        out += num;
    }
    return out + "]}";
}

// the value text after "<key>": in one line (nullptr if absent)
const char* field(const std::string& line, const char* key) {
    const std::string pat = std::string("\"") + key + "\":";
    const size_t at = line.find(pat);
    if (at == std::string::npos) return nullptr;
    const char* p = line.c_str() + at + pat.size();
    while (*p == ' ') ++p;
    return p;
}

bool parse_entry(const std::string& line, TuneKey& k, TuneVal& v) {
    const char* d = field(line, "device");
    const char* m = field(line, "model");
    const char* ms = field(line, "ms");
    if (!d || !m || !ms || *d != '"' || *m != '"' || *ms != '[') return false;
    const char* de = strchr(d + 1, '"');
    if (!de) return false;
    k.device.assign(d + 1, de);
    unsigned long long h = 0;
    if (sscanf(m + 1, "%16llx", &h) != 1) return false;
    k.model_hash = h;
    const char* fK = field(line, "K");
    const char* fH = field(line, "H");
    const char* fk = field(line, "knots");
    const char* fm = field(line, "mapping");
    const char* fb = field(line, "block");
    if (!fK || !fH || !fk || !fm || !fb) return false;
    if (sscanf(fK, "%d", &k.N) != 1 || sscanf(fH, "%d", &k.H) != 1 || sscanf(fk, "%d", &k.nk) != 1 ||
        sscanf(fm, "%d", &v.mapping) != 1 || sscanf(fb, "%d", &v.block) != 1)
        return false;
    const char* p = ms + 1;
    for (int i = 0; i < 16; ++i) {
        char* end = nullptr;
        v.ms[i] = strtof(p, &end);
        if (end == p) return false;
        p = end;
        while (*p == ' ' || *p == ',') ++p;
    }
    return *p == ']';
}

// caller holds g_mu
bool load_cache_file(const std::string& path) {
    FILE* f = fopen(path.c_str(), "r");
    if (!f) return true;  // no file yet: it is created by the first tuning
    std::map<TuneKey, TuneVal> got;
    char buf[4096];
    bool ok = true;
    while (fgets(buf, sizeof buf, f)) {
        std::string line(buf);
        if (line.find('{') == std::string::npos) continue;  // the array's brackets
        TuneKey k;
        TuneVal v;
        if (!parse_entry(line, k, v)) {
            ok = false;
            break;
        }
        got[k] = v;
    }
    fclose(f);
    if (!ok) return false;
    for (auto& kv : got) g_cache[kv.first] = kv.second;
    return true;
}

// caller holds g_mu; written to a temporary file, then renamed over the old one
bool save_cache_file(const std::string& path) {
    const std::string tmp = path + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    fputs("[\n", f);
    size_t i = 0;
    for (auto& kv : g_cache) {
        fputs(entry_json(kv.first, kv.second).c_str(), f);
        fputs(++i < g_cache.size() ? ",\n" : "\n", f);
    }
    fputs("]\n", f);
    const bool ok = fclose(f) == 0;
    return ok && rename(tmp.c_str(), path.c_str()) == 0;
}

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
    MPPI_NVTX("mppi_autotune");
    if (!c) return MPPI_ERR_INVALID_ARG;
    // the timed rollouts start from the context's last state if a solve ran, else from
    // the model's rest pose half a metre above the ground
    TuneKey key{device_id(c->device), fnv1a(&c->model->host_f, sizeof(DevModel<float>)), c->N, c->H, c->nk};
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
        if (!g_cache_path.empty() && !save_cache_file(g_cache_path)) {
            set_error(c, "mppi_autotune: the cache file could not be written");
            // the choice stands for this process; only the file is missing the entry
        }
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

extern "C" mppi_status mppi_autotune_cache_file(const char* path) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!path || !*path) {
        g_cache_path.clear();
        return MPPI_OK;
    }
    if (!load_cache_file(path)) {
        set_error(nullptr, std::string("mppi_autotune_cache_file: cannot parse ") + path);
        return MPPI_ERR_INVALID_ARG;
    }
    g_cache_path = path;
    return MPPI_OK;
}

// Batched solves: many independent MPC instances (uneven model, K, H, knots, lambda,
// iterations) in one persistent kernel that walks a device work queue.
//
// Items are ROLLOUT(instance, tile) and REDUCE(instance, chunk). A ROLLOUT block draws
// its tile's knots (Alg. 1 sampling) and rolls them out with the instance's mapping; the
// last tile of an instance publishes its REDUCE items (weights and FP64 partial knot sums
// per chunk of AVG_CHUNK samples); the last REDUCE item runs the iteration's finalize and
// publishes the next iteration's ROLLOUT tiles. Every step calls the same device
// functions as the per-instance kernels, so each instance's result is bit-identical to
// its mppi_solve result.
//
// The instances of a batch are grouped by rollout variant (mapping, axis plan, modular
// cost on or off) and each group walks its own queue in its own instantiation of the
// persistent kernel, the groups' kernels running side by side on a share of the SMs in
// proportion to their estimated work. A kernel that can call several rollout functions
// gets fewer registers for each (ptxas spilled 450-950 bytes per rollout function when
// all variants shared one kernel, none with one variant per kernel; a quadruped-only batch
// ran 18 % faster).
//
// Progress needs no co-residency: a block waits only for an item of its own queue whose
// producer is a block that has already taken and finished its own item and publishes
// without waiting. Every wait is bounded by the global timer and sets an error word when
// it gives up.
#pragma once
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <list>
#include <mutex>
#include <new>
#include <vector>

#include "batch.h"
#include "nvtx.h"
#include "capi_internal.h"
#include "noise.cuh"
#include "reduce.cuh"
#include "chain_f32.cuh"

namespace mppi {

constexpr int ITEM_ROLLOUT = 1;
constexpr int ITEM_REDUCE = 2;

struct BatchInst {
    const DevModel<float>* model;
    const double* x0;
    float* knots;
    float* costs;
    double* zq;
    double* partial;
    double* gpartial;
    double* gzq;
    uint32_t* gcount;
    float* nominal;
    float* mean;
    float* best;
    const float* sigma;
    DevIterInfo* info;
    DevSolve* solve;
    mppi_result* result;
    double lambda;
    int N, H, nk, nj, E, iters, mapping, tile, ntiles, nchunks, ngroups, normalize, warm_from, has_limits, spline;
    float dt, dtk, scale_q, scale_v;
    uint32_t inst, seed_lo, seed_hi;
    // packed host <-> device exchange
    int in_off;    // offset (bytes) of this instance's input record in the packed input
    int out_off;   // offset (bytes) of this instance's output record in the packed output
};

struct InstCounters {
    int it, done_roll, pad0, pad1;
};

struct QueueItem {
    int type, inst, idx;
    volatile int ready;
};

struct BatchQueue {
    int head, append, total, nprefill;
    uint32_t error;
    int count;   // instances of the batch (bounds of the items' instance index)
    uint32_t pad1, pad2;
};

// Where a group's queue, items and prefill list sit in the device block (byte offsets).
struct GroupDev {
    long long q, items, pre;
};

// Rollout variants of batched instances: one persistent kernel instantiation each.
constexpr int BV_XYY = 0, BV_XYY_P = 1, BV_QUAD = 2, BV_QUAD_P = 3, BV_HUMG = 4, BV_HUMG_P = 5, BV_SPLIT = 6,
              BV_SPLIT_P = 7, BV_HALF = 8, BV_WARP = 9, BV_COUNT = 10;
static_assert(BV_COUNT == BATCH_VARIANTS, "one persistent kernel per rollout variant");

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bulk copy into shared memory with a persistent mbarrier (phase parity flips each use).
__device__ __forceinline__ bool bulk_load_phase(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* mbar,
                                                uint32_t phase) {
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(mbar);
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(smem_dst);
    __syncthreads();  // everyone is done with the previous contents
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
            "l"(gsrc), "r"(bytes), "r"(bar)
            : "memory");
    }
    auto wait = [&](int limit) {
        bool done = false;
        for (int i = 0; i < limit && !done; ++i) {
            uint32_t ok;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(ok)
                : "r"(bar), "r"(phase)
                : "memory");
            done = ok != 0;
        }
        return done;
    };
    if (__syncthreads_and(wait(1 << 22) ? 1 : 0)) return true;
    wait(1 << 22);
    __syncthreads();
    return false;
}

// Publish `count` items of one type for instance `inst` (whole block).
__device__ __forceinline__ void publish(QueueItem* items, BatchQueue* q, int type, int inst, int count) {
    __shared__ int s_base;
    if (threadIdx.x == 0) s_base = atomicAdd(&q->append, count);
    __syncthreads();
    const int base = s_base;
    for (int k = threadIdx.x; k < count; k += blockDim.x) {
        if (base + k >= q->total) continue;  // cannot happen with a consistent plan
        items[base + k].type = type;
        items[base + k].inst = inst;
        items[base + k].idx = k;
    }
    __threadfence();
    __syncthreads();
    for (int k = threadIdx.x; k < count; k += blockDim.x)
        if (base + k < q->total) items[base + k].ready = 1;
    __threadfence();
    __syncthreads();
}

__device__ __forceinline__ FinalizeArgs finalize_args(const BatchInst& I, int it) {
    FinalizeArgs f;
    f.partial = I.partial;
    f.zq = I.zq;
    f.gpartial = I.gpartial;
    f.gzq = I.gzq;
    f.gcount = I.gcount;
    f.nchunks = I.nchunks;
    f.ngroups = I.ngroups;
    f.E = I.E;
    f.iter = it;
    f.iters = I.iters;
    f.warm_from = I.warm_from;
    f.knots = I.knots;
    f.costs = I.costs;
    f.info = I.info;
    f.solve = I.solve;
    f.nominal = I.nominal;
    f.mean_out = I.mean;
    f.best_out = I.best;
    f.result = I.result;
    return f;
}

// One tile's rollouts in variant V (the instance's mapping, axis plan and cost).
template <int V>
__device__ __forceinline__ void rollout_tile(const DevModel<float>& M, const BatchInst& I, int n0, int last_n,
                                             float* work) {
    if constexpr (V == BV_SPLIT || V == BV_SPLIT_P) {
        // two-warp split: 4 pairs of 16 samples; `work` is free again after the noise pass
        static_assert(4 * SPLIT_PAIR_FLOATS <= 27 * BATCH_THREADS, "split exchange area exceeds work");
        static_assert(BATCH_THREADS / 4 == 4 * SPLIT_SPP, "tile = 4 warp pairs");
        __syncthreads();
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, pair = warp >> 1;
        const int n = n0 + pair * SPLIT_SPP + (lane >> 1);
        const int ne = min(n, last_n);
        const float* kn = I.knots + (size_t)ne * I.E;
        float* rec = work + pair * SPLIT_PAIR_FLOATS;
        const float c =
            split_rollout<V == BV_SPLIT_P>(M, warp & 1, lane, rec, 1 + pair, I.x0, kn, I.H, I.nk, I.dt, I.dtk, nullptr);
        if (n <= last_n && (warp & 1) == 0 && (lane & 1) == 0) I.costs[n] = c;
    } else if constexpr (V <= BV_HUMG_P) {
        const int g = threadIdx.x & 3;
        const int n = n0 + (threadIdx.x >> 2);
        const int ne = min(n, last_n);
        const float* kn = I.knots + (size_t)ne * I.E;
        constexpr bool paper = V == BV_XYY_P || V == BV_QUAD_P || V == BV_HUMG_P;
        float c;
        if constexpr (V == BV_XYY || V == BV_XYY_P)
            c = lanes_rollout<3, false, paper, AXP_XYY>(M, g, I.x0, kn, I.H, I.nk, I.dt, I.dtk, nullptr);
        else if constexpr (V == BV_QUAD || V == BV_QUAD_P)
            c = lanes_rollout<3, false, paper, AXP_GENERIC>(M, g, I.x0, kn, I.H, I.nk, I.dt, I.dtk, nullptr);
        else
            c = lanes_rollout<6, true, paper, AXP_GENERIC>(M, g, I.x0, kn, I.H, I.nk, I.dt, I.dtk, nullptr);
        if (n <= last_n && g == 0) I.costs[n] = c;
    } else {
        constexpr int G = V == BV_HALF ? 16 : 32;
        const int gl = threadIdx.x & (G - 1);
        const int n = n0 + (threadIdx.x / G);
        const int ne = min(n, last_n);
        LaneConst<float> L;
        load_lane_const(M, gl, L);
        const float c = warp_rollout<float, G, double>(M, L, gl, I.x0, I.knots + (size_t)ne * I.E, I.H, I.H, I.nk,
                                                       I.dt, I.dtk, work, nullptr);
        if (n <= last_n && gl == 0) I.costs[n] = c;
    }
}

template <int V>
__global__ void __launch_bounds__(BATCH_THREADS, 1)
    persistent_kernel(const BatchInst* __restrict__ insts, InstCounters* ctr, QueueItem* items, BatchQueue* q,
                      uint64_t budget_ns) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t mbar;
    __shared__ int s_type, s_inst, s_item, s_last;
    __shared__ const void* s_loaded;
    DevModel<float>* M = reinterpret_cast<DevModel<float>*>(smem);
    float* work = reinterpret_cast<float*>(smem + sizeof(DevModel<float>));
    const uint64_t t0 = globaltimer_ns();
    uint32_t phase = 0;
    if (threadIdx.x == 0) {
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&mbar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_loaded = nullptr;
    }
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {
            const int idx = atomicAdd(&q->head, 1);
            int type = 0;
            if (idx < q->total) {
                // wait (bounded) until the item is published
                while (items[idx].ready == 0) {
                    if (globaltimer_ns() - t0 > budget_ns) {
                        atomicOr(&q->error, DEV_ERR_QUEUE_TIMEOUT);
                        type = -1;
                        break;
                    }
                    __nanosleep(200);
                }
                __threadfence();
                if (type == 0) {
                    const volatile QueueItem* vi = items + idx;
                    type = vi->type;
                    s_inst = vi->inst;
                    s_item = vi->idx;
                }
            }
            s_type = type;
        }
        __syncthreads();
        const int type = s_type;
        if (type != ITEM_ROLLOUT && type != ITEM_REDUCE) {
            if (type > 0 && threadIdx.x == 0) atomicOr(&q->error, DEV_ERR_BAD_ITEM);
            break;
        }
        const int ii = s_inst;
        if (!MPPI_CHECK_OK(ii >= 0 && ii < q->count, CHECK_QUEUE)) {
            if (threadIdx.x == 0) atomicOr(&q->error, DEV_ERR_BAD_ITEM);
            break;
        }
        const BatchInst& I = insts[ii];
        if (!MPPI_CHECK_OK(s_item >= 0 && s_item < (type == ITEM_ROLLOUT ? I.ntiles : I.nchunks), CHECK_QUEUE)) {
            if (threadIdx.x == 0) atomicOr(&q->error, DEV_ERR_BAD_ITEM);
            break;
        }
        const int it = *reinterpret_cast<volatile int*>(&ctr[ii].it);
        if (type == ITEM_ROLLOUT) {
            if (s_loaded != (const void*)I.model) {
                const bool ok = bulk_load_phase(M, I.model, (uint32_t)sizeof(DevModel<float>), &mbar, phase);
                phase ^= 1u;
                if (!ok) {
                    if (threadIdx.x == 0) atomicOr(&q->error, DEV_ERR_TMA_TIMEOUT);
                    break;
                }
                if (threadIdx.x == 0) s_loaded = I.model;
                __syncthreads();
            }
            const int n0 = s_item * I.tile;
            const int cnt = min(I.tile, I.N - n0);
            // knots of this tile (Alg. 1 sampling), NOISE_SPB samples at a time
            NoiseParams np;
            np.nominal = I.nominal;
            np.sigma_row = I.sigma + (size_t)it * I.nk;
            np.model = M;
            np.knots = I.knots;
            np.it = *reinterpret_cast<volatile uint32_t*>(&I.solve->iter_counter) + (uint32_t)it;
            np.inst = I.inst;
            np.seed_lo = I.seed_lo;
            np.seed_hi = I.seed_hi;
            np.N = I.N;
            np.nk = I.nk;
            np.nj = I.nj;
            np.has_limits = I.has_limits;
            np.scale_q = I.scale_q;
            np.scale_v = I.scale_v;
            np.dtk = I.dtk;
            np.spline = I.spline;
            for (int s0 = 0; s0 < cnt; s0 += NOISE_SPB) block_sample_knots(np, n0 + s0, min(NOISE_SPB, cnt - s0), work);
            // rollouts of the tile with the instance's mapping
            rollout_tile<V>(*M, I, n0, n0 + cnt - 1, work);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) s_last = atomicAdd(&ctr[ii].done_roll, 1) == I.ntiles - 1;
            __syncthreads();
            if (s_last) {
                __threadfence();
                if (threadIdx.x == 0) ctr[ii].done_roll = 0;
                publish(items, q, ITEM_REDUCE, ii, I.nchunks);
            }
        } else {
            // the chunk's weights and partial sums; the last chunk of its group sums the
            // group, the last group runs the finalize (the same function as single solves)
            if (reduce_chunk(finalize_args(I, it), I.N, I.lambda, I.normalize, s_item)) {
                __threadfence();
                __syncthreads();
                if (it + 1 < I.iters) {
                    if (threadIdx.x == 0) ctr[ii].it = it + 1;
                    __threadfence();
                    __syncthreads();
                    publish(items, q, ITEM_ROLLOUT, ii, I.ntiles);
                }
            }
        }
        __syncthreads();
    }
}

// Reset of a batch before the persistent launches: each group's queue counters and its
// prefilled iteration-0 ROLLOUT items, per-instance counters and solve state (as
// solve_begin), and the inputs scattered from the packed host record: state [nx] doubles,
// then (if flagged) the warm start [E] floats into the nominal.
__global__ void batch_reset_kernel(const BatchInst* __restrict__ insts, int count, InstCounters* ctr,
                                   const GroupDev* __restrict__ groups, int ngroups, unsigned char* base,
                                   const unsigned char* __restrict__ packed_in) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    for (int g = 0; g < ngroups; ++g) {
        BatchQueue* q = reinterpret_cast<BatchQueue*>(base + groups[g].q);
        QueueItem* items = reinterpret_cast<QueueItem*>(base + groups[g].items);
        const int* prefill = reinterpret_cast<const int*>(base + groups[g].pre);
        const int total = q->total, npre = q->nprefill;
        for (int k = tid; k < total; k += nth) {
            if (k < npre) {
                items[k].type = ITEM_ROLLOUT;
                items[k].inst = prefill[2 * k];
                items[k].idx = prefill[2 * k + 1];
                items[k].ready = 1;
            } else {
                items[k].type = 0;
                items[k].ready = 0;
            }
        }
    }
    for (int i = blockIdx.x; i < count; i += gridDim.x) {
        const BatchInst& I = insts[i];
        const unsigned char* rec = packed_in + I.in_off;
        const int nx = 13 + 2 * I.nj;
        const double* st = reinterpret_cast<const double*>(rec);
        const int has_warm = *reinterpret_cast<const int*>(rec + 8 * nx);
        const float* warm = reinterpret_cast<const float*>(rec + 8 * nx + 16);
        for (int k = threadIdx.x; k < nx; k += blockDim.x) const_cast<double*>(I.x0)[k] = st[k];
        for (int e = threadIdx.x; e < I.E; e += blockDim.x) {
            const float v = has_warm ? warm[e] : I.nominal[e];
            I.nominal[e] = v;
            I.best[e] = v;
        }
        for (int g = threadIdx.x; g < I.ngroups; g += blockDim.x) I.gcount[g] = 0;
        if (threadIdx.x == 0) {
            ctr[i].it = 0;
            ctr[i].done_roll = 0;
            I.solve->best_cost = INFINITY;
            I.solve->best_index = -1;
            I.solve->best_iter = -1;
            I.solve->status = MPPI_OK;
            I.solve->blocks_done = 0;
        }
    }
    // head, append and error are read by no thread of this kernel (total and nprefill,
    // which are, stay as the image set them)
    if (tid < ngroups) {
        BatchQueue* q = reinterpret_cast<BatchQueue*>(base + groups[tid].q);
        q->head = 0;
        q->append = q->nprefill;
        q->error = 0;
    }
}

// Outputs of every instance into one packed record per instance: result, mean [E],
// best [E]; and the groups' error words (or-ed) at offset 0.
__global__ void batch_gather_kernel(const BatchInst* __restrict__ insts, int count, const GroupDev* __restrict__ groups,
                                    int ngroups, const unsigned char* base, unsigned char* __restrict__ packed_out) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        uint32_t err = 0;
        for (int g = 0; g < ngroups; ++g) err |= reinterpret_cast<const BatchQueue*>(base + groups[g].q)->error;
        *reinterpret_cast<uint32_t*>(packed_out) = err;
    }
    for (int i = blockIdx.x; i < count; i += gridDim.x) {
        const BatchInst& I = insts[i];
        unsigned char* rec = packed_out + I.out_off;
        if (threadIdx.x == 0) *reinterpret_cast<mppi_result*>(rec) = *I.result;
        float* mean = reinterpret_cast<float*>(rec + sizeof(mppi_result));
        float* best = mean + I.E;
        for (int e = threadIdx.x; e < I.E; e += blockDim.x) {
            mean[e] = I.mean[e];
            best[e] = I.best[e];
        }
    }
}

// ------------------------------------------------------------------------------------
// Host side. A batch image is one contiguous block, identical in pinned host memory and
// on the device: [queue header][descriptors][prefilled items][packed inputs], followed
// on the device by the counters, the item array and the packed outputs. One H2D copy of
// the image, the reset/scatter kernel, the persistent kernel, the gather kernel and one
// D2H copy of the outputs make a launch.
// ------------------------------------------------------------------------------------
static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

int batch_variant(const mppi_ctx* c) {
    const DevModel<float>& M = c->model->host_f;
    const bool paper = M.paper_cost != 0;
    if (c->mapping == MPPI_MAP_CHAIN) {
        if (M.axis_plan == AXP_HUM) return paper ? BV_SPLIT_P : BV_SPLIT;
        if (M.topology == TOPO_QUADRUPED) {
            if (M.axis_plan == AXP_XYY) return paper ? BV_XYY_P : BV_XYY;
            return paper ? BV_QUAD_P : BV_QUAD;
        }
        return paper ? BV_HUMG_P : BV_HUMG;
    }
    return c->mapping == MPPI_MAP_HALFWARP ? BV_HALF : BV_WARP;
}

// Estimated duration (us) of one of an instance's tiles: H steps of its variant's step
// time in the persistent kernel (one 256-thread block per SM), measured on GB300 for the
// specialised chain variants (quadruped 3.2 us, +10 % with the modular cost) and scaled
// from the per-instance kernels' ratios for the others. Orders the prefill (longest
// first) and shares the SMs between groups, so only the ratios matter. The humanoid
// split's weight comes from the two groups' kernel times in the 256-instance mix (each
// alone on its share of the SMs under ncu: the quadruped group 6.58 ms on 73 SMs, the
// split group 5.17 ms on 79 with a weight of 7.5, i.e. a true ratio of 1.84 to the
// quadruped's) and a sweep of it (7.5, 6.5, 5.9, 5.3: 7.85, 7.43, 7.22, 7.53 ms per batch).
static double step_us(const mppi_ctx* c) {
    switch (batch_variant(c)) {
        case BV_XYY: return 3.2;
        case BV_XYY_P: return 3.5;
        case BV_QUAD: return 6.5;
        case BV_QUAD_P: return 7.2;
        case BV_SPLIT: return 5.9;
        case BV_SPLIT_P: return 6.5;
        case BV_HUMG: return 15.0;
        case BV_HUMG_P: return 16.5;
        case BV_HALF: return 0.8 * c->model->nb;
        default: return 1.0 * c->model->nb;
    }
}
static double tile_cost(const mppi_ctx* c) { return c->H * step_us(c); }

BatchLayout layout_batch(mppi_ctx* const* ctxs, int count) {
    BatchLayout L;
    L.count = count;
    long total = 0, nprefill = 0;
    size_t in_bytes = 0, out_bytes = 16;
    int max_E = 0;
    int gidx[BV_COUNT];
    for (int v = 0; v < BV_COUNT; ++v) gidx[v] = -1;
    for (int i = 0; i < count; ++i) {
        mppi_ctx* c = ctxs[i];
        const int tile = batch_tile(c->mapping);
        const int ntiles = (c->N + tile - 1) / tile;
        const long items = (long)c->iters * (ntiles + num_chunks(c->N));
        const int v = batch_variant(c);
        if (gidx[v] < 0) {
            gidx[v] = (int)L.groups.size();
            BatchGroup g;
            g.variant = v;
            L.groups.push_back(g);
        }
        BatchGroup& g = L.groups[gidx[v]];
        g.total += items;
        g.nprefill += ntiles;
        g.work += (double)c->iters * ntiles * tile_cost(c);
        total += items;
        nprefill += ntiles;
        in_bytes += ((size_t)8 * c->nx + 16 + 4 * (size_t)c->E + 15) & ~(size_t)15;
        out_bytes += (sizeof(mppi_result) + 8 * (size_t)c->E + 15) & ~(size_t)15;
        max_E = std::max(max_E, c->E);
    }
    L.total = total;
    L.nprefill = nprefill;
    L.max_E = max_E;
    L.in_bytes = in_bytes;
    L.out_bytes = out_bytes;
    const int ng = (int)L.groups.size();
    size_t off = 0;
    L.o_groups = off;
    off += al256(sizeof(GroupDev) * ng);
    L.o_q = off;
    off += al256(sizeof(BatchQueue) * ng);
    L.o_insts = off;
    off += al256(sizeof(BatchInst) * count);
    L.o_pre = off;
    off += al256(sizeof(int) * 2 * nprefill);
    L.o_in = off;
    off += al256(in_bytes);
    L.image_bytes = off;
    L.o_ctr = off;
    off += al256(sizeof(InstCounters) * count);
    L.o_items = off;
    off += al256(sizeof(QueueItem) * total);
    L.o_out = off;
    off += al256(out_bytes);
    L.dev_bytes = off;
    long pre = 0, it = 0;
    for (int k = 0; k < ng; ++k) {
        BatchGroup& g = L.groups[k];
        g.o_q = L.o_q + sizeof(BatchQueue) * k;
        g.o_pre = L.o_pre + sizeof(int) * 2 * pre;
        g.o_items = L.o_items + sizeof(QueueItem) * it;
        pre += g.nprefill;
        it += g.total;
    }
    return L;
}

// Upper bound of a launch block's bytes (layout_batch's dev_bytes): the fixed part (every
// group's queue header and descriptor, the output header, the 256-byte rounding of each
// section) plus each instance's share (descriptor, prefill entries, counters, queue items
// of all its iterations, packed input and output records).
size_t batch_fixed_bound() { return al256(sizeof(GroupDev) * BV_COUNT) + al256(sizeof(BatchQueue) * BV_COUNT) + 6 * 256 + 16; }

size_t batch_instance_bound(const mppi_ctx* c) {
    const size_t tile = (size_t)batch_tile(c->mapping);
    const size_t ntiles = ((size_t)c->N + tile - 1) / tile;
    const size_t items = (size_t)c->iters * (ntiles + (size_t)num_chunks(c->N));
    const size_t in_rec = ((size_t)8 * c->nx + 16 + 4 * (size_t)c->E + 15) & ~(size_t)15;
    const size_t out_rec = (sizeof(mppi_result) + 8 * (size_t)c->E + 15) & ~(size_t)15;
    return sizeof(BatchInst) + sizeof(int) * 2 * ntiles + sizeof(InstCounters) + sizeof(QueueItem) * items + in_rec +
           out_rec;
}

int batch_tile(int mapping) {
    return mapping == MPPI_MAP_CHAIN ? BATCH_THREADS / 4 : mapping == MPPI_MAP_HALFWARP ? BATCH_THREADS / 16
                                                                                         : BATCH_THREADS / 32;
}

// Writes the image (queue header, descriptors pointing at each context's buffers, the
// prefill list with the longest tiles first, and the packed inputs) into `img`.
void fill_batch_image(mppi_ctx* const* ctxs, const BatchLayout& L, const double* const* states,
                      const float* const* warm, unsigned char* img, std::vector<size_t>* in_off,
                      std::vector<size_t>* out_off) {
    const int ng = (int)L.groups.size();
    GroupDev* gd = reinterpret_cast<GroupDev*>(img + L.o_groups);
    for (int k = 0; k < ng; ++k) {
        const BatchGroup& g = L.groups[k];
        BatchQueue* q = reinterpret_cast<BatchQueue*>(img + g.o_q);
        memset(q, 0, sizeof *q);
        q->total = (int)g.total;
        q->nprefill = (int)g.nprefill;
        q->count = L.count;
        gd[k].q = (long long)g.o_q;
        gd[k].items = (long long)g.o_items;
        gd[k].pre = (long long)g.o_pre;
    }
    BatchInst* hi = reinterpret_cast<BatchInst*>(img + L.o_insts);
    size_t ioff = 0, ooff = 16;
    if (in_off) in_off->clear();
    if (out_off) out_off->clear();
    std::vector<int> order(L.count);
    for (int i = 0; i < L.count; ++i) {
        mppi_ctx* c = ctxs[i];
        BatchInst& I = hi[i];
        I.model = (const DevModel<float>*)c->model->d_f;
        I.x0 = c->d_x0;
        I.knots = c->d_knots;
        I.costs = c->d_costs;
        I.zq = c->d_zq;
        I.partial = c->d_partial;
        I.gpartial = c->d_gpartial;
        I.gzq = c->d_gzq;
        I.gcount = c->d_gcount;
        I.nominal = c->d_nominal;
        I.mean = c->d_mean;
        I.best = c->d_best;
        I.sigma = c->d_sigma;
        I.info = c->d_info;
        I.solve = c->d_solve;
        I.result = c->d_result;
        I.lambda = c->lambda;
        I.N = c->N;
        I.H = c->H;
        I.nk = c->nk;
        I.nj = c->nj;
        I.E = c->E;
        I.iters = c->iters;
        I.mapping = c->mapping;
        I.tile = batch_tile(c->mapping);
        I.ntiles = (c->N + I.tile - 1) / I.tile;
        I.nchunks = num_chunks(c->N);
        I.ngroups = num_groups(c->N);
        I.normalize = c->normalize;
        I.warm_from = c->warm_from;
        I.has_limits = c->model->host_f.has_limits;
        I.spline = c->spline;
        I.dt = (float)c->dt;
        I.dtk = (float)c->dtk;
        I.scale_q = (float)c->scale_q;
        I.scale_v = (float)c->scale_v;
        I.inst = c->instance_id;
        I.seed_lo = (uint32_t)(c->seed & 0xffffffffu);
        I.seed_hi = (uint32_t)(c->seed >> 32);
        I.in_off = (int)ioff;
        I.out_off = (int)ooff;
        if (in_off) in_off->push_back(ioff);
        if (out_off) out_off->push_back(ooff);
        if (states) {
            unsigned char* rec = img + L.o_in + ioff;
            memcpy(rec, states[i], sizeof(double) * c->nx);
            const int has = (warm && warm[i]) ? 1 : 0;
            memcpy(rec + 8 * c->nx, &has, sizeof has);
            if (has) memcpy(rec + 8 * c->nx + 16, warm[i], sizeof(float) * c->E);
        }
        ioff += ((size_t)8 * c->nx + 16 + 4 * (size_t)c->E + 15) & ~(size_t)15;
        ooff += (sizeof(mppi_result) + 8 * (size_t)c->E + 15) & ~(size_t)15;
        order[i] = i;
    }
    // per group: longest tiles first, then the largest instances: the long rollouts start
    // early and the queue ends on short tiles, which keeps the tail of the launch short
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const double ta = tile_cost(ctxs[a]), tb = tile_cost(ctxs[b]);
        if (ta != tb) return ta > tb;
        return (long)hi[a].N * hi[a].H > (long)hi[b].N * hi[b].H;
    });
    for (int k = 0; k < ng; ++k) {
        const BatchGroup& g = L.groups[k];
        int* pre = reinterpret_cast<int*>(img + g.o_pre);
        long n = 0;
        for (int i : order) {
            if (batch_variant(ctxs[i]) != g.variant) continue;
            for (int t = 0; t < hi[i].ntiles; ++t) {
                pre[2 * n] = i;
                pre[2 * n + 1] = t;
                ++n;
            }
        }
    }
}

// Packed inputs of instance i only (states / warm starts change between launches).
void fill_batch_inputs(mppi_ctx* const* ctxs, const BatchLayout& L, const std::vector<size_t>& in_off,
                       const double* const* states, const float* const* warm, unsigned char* img) {
    for (int i = 0; i < L.count; ++i) {
        mppi_ctx* c = ctxs[i];
        unsigned char* rec = img + L.o_in + in_off[i];
        memcpy(rec, states[i], sizeof(double) * c->nx);
        const int has = (warm && warm[i]) ? 1 : 0;
        memcpy(rec + 8 * c->nx, &has, sizeof has);
        if (has) memcpy(rec + 8 * c->nx + 16, warm[i], sizeof(float) * c->E);
    }
}

using PersistentFn = void (*)(const BatchInst*, InstCounters*, QueueItem*, BatchQueue*, uint64_t);
static const PersistentFn kPersistent[BV_COUNT] = {
    persistent_kernel<0>, persistent_kernel<1>, persistent_kernel<2>, persistent_kernel<3>, persistent_kernel<4>,
    persistent_kernel<5>, persistent_kernel<6>, persistent_kernel<7>, persistent_kernel<8>, persistent_kernel<9>};

cudaError_t prepare_batch_kernel(int max_E, size_t* smem, int* per_sm) {
    *smem = batch_smem_bytes(max_E);
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < BV_COUNT && e == cudaSuccess; ++v)
        e = cudaFuncSetAttribute(kPersistent[v], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem_bytes(992));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kPersistent[BV_XYY], BATCH_THREADS, *smem);
    return e;
}

cudaError_t BatchStreams::ensure(int n) {
    cudaError_t e = cudaSuccess;
    if (!fork && (e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming)) != cudaSuccess) return e;
    while ((int)aux.size() < n) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
            cudaStreamDestroy(st);
            return e;
        }
        aux.push_back(st);
        join.push_back(ev);
    }
    return e;
}

void BatchStreams::release() {
    for (cudaStream_t st : aux) cudaStreamDestroy(st);
    for (cudaEvent_t ev : join) cudaEventDestroy(ev);
    if (fork) cudaEventDestroy(fork);
    aux.clear();
    join.clear();
    fork = nullptr;
}

// Blocks per group, in proportion to the groups' estimated work, at least one each and
// `grid` in all where there are no more groups than that.
static std::vector<int> group_grids(const BatchLayout& L, int grid) {
    const int ng = (int)L.groups.size();
    std::vector<int> out(ng, 1);
    double W = 0.0;
    for (const BatchGroup& g : L.groups) W += g.work;
    if (ng == 0 || grid <= ng || W <= 0.0) return out;
    int used = 0;
    for (int k = 0; k < ng; ++k) {
        out[k] = std::max(1, (int)(grid * L.groups[k].work / W));
        used += out[k];
    }
    // hand the blocks lost to rounding down to the groups with the most work per block
    while (used < grid) {
        int best = 0;
        for (int k = 1; k < ng; ++k)
            if (L.groups[k].work / out[k] > L.groups[best].work / out[best]) best = k;
        ++out[best];
        ++used;
    }
    for (int k = 0; k < ng; ++k) out[k] = (int)std::min<long>(out[k], std::max<long>(1, L.groups[k].nprefill));
    return out;
}

// H2D image, reset/scatter, the groups' persistent kernels side by side (forked onto the
// auxiliary streams and joined back), gather, D2H outputs (host image and device block
// share the layout `L`).
cudaError_t enqueue_batch(const BatchLayout& L, const unsigned char* h_img, unsigned char* d_block,
                          unsigned char* h_out, int grid, size_t smem, cudaStream_t s, BatchStreams& bs) {
    const int ng = (int)L.groups.size();
    cudaError_t e = bs.ensure(std::max(0, ng - 1));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_block, h_img, L.image_bytes, cudaMemcpyHostToDevice, s);
    const BatchInst* insts = reinterpret_cast<const BatchInst*>(d_block + L.o_insts);
    InstCounters* ctr = reinterpret_cast<InstCounters*>(d_block + L.o_ctr);
    const GroupDev* gd = reinterpret_cast<const GroupDev*>(d_block + L.o_groups);
    if (e == cudaSuccess) {
        batch_reset_kernel<<<std::min(L.count, 1024), 256, 0, s>>>(insts, L.count, ctr, gd, ng, d_block,
                                                                  d_block + L.o_in);
        e = cudaGetLastError();
    }
    const std::vector<int> grids = group_grids(L, grid);
    if (e == cudaSuccess && ng > 1) e = cudaEventRecord(bs.fork, s);
    for (int k = 0; k < ng && e == cudaSuccess; ++k) {
        cudaStream_t st = k == 0 ? s : bs.aux[k - 1];
        if (k > 0) e = cudaStreamWaitEvent(st, bs.fork, 0);
        if (e != cudaSuccess) break;
        const BatchGroup& g = L.groups[k];
        const uint64_t budget_ns = 20ull * 1000 * 1000 * 1000;  // 20 s
        kPersistent[g.variant]<<<grids[k], BATCH_THREADS, smem, st>>>(
            insts, ctr, reinterpret_cast<QueueItem*>(d_block + g.o_items), reinterpret_cast<BatchQueue*>(d_block + g.o_q),
            budget_ns);
        e = cudaGetLastError();
        if (e == cudaSuccess && k > 0) e = cudaEventRecord(bs.join[k - 1], st);
    }
    for (int k = 1; k < ng && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(s, bs.join[k - 1], 0);
    if (e == cudaSuccess) {
        batch_gather_kernel<<<std::min(L.count, 1024), 128, 0, s>>>(insts, L.count, gd, ng, d_block, d_block + L.o_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, d_block + L.o_out, L.out_bytes, cudaMemcpyDeviceToHost, s);
    return e;
}

// Unpack outputs; returns the first non-OK instance status or TIMEOUT.
mppi_status unpack_batch(mppi_ctx* const* ctxs, const BatchLayout& L, const std::vector<size_t>& out_off,
                         const unsigned char* h_out, float* const* out_mean, float* const* out_best,
                         mppi_result* info) {
    uint32_t err;
    memcpy(&err, h_out, sizeof err);
    mppi_status st = MPPI_OK;
    for (int i = 0; i < L.count; ++i) {
        const int E = ctxs[i]->E;
        const unsigned char* rec = h_out + out_off[i];
        mppi_result r;
        memcpy(&r, rec, sizeof r);
        const float* mean = reinterpret_cast<const float*>(rec + sizeof(mppi_result));
        if (out_mean && out_mean[i]) memcpy(out_mean[i], mean, sizeof(float) * E);
        if (out_best && out_best[i]) memcpy(out_best[i], mean + E, sizeof(float) * E);
        if (info) info[i] = r;
        if (r.status != MPPI_OK && st == MPPI_OK) st = r.status;
        ctxs[i]->has_state = true;
    }
    if (err) {
        set_error(nullptr, "a bounded device wait of the batched kernel gave up");
        return MPPI_ERR_TIMEOUT;
    }
    return st;
}

// Cached plans for mppi_solve_batch: per batch composition (contexts by unique id) one
// image, device block and captured graph; LRU of 4.
struct BatchPlan {
    std::vector<uint64_t> uids;
    BatchLayout L;
    std::vector<size_t> in_off, out_off;
    unsigned char* h_img = nullptr;
    unsigned char* h_out = nullptr;
    unsigned char* d_block = nullptr;
    cudaStream_t stream = nullptr;
    BatchStreams streams;
    cudaGraphExec_t graph = nullptr;
    ~BatchPlan() {
        if (graph) cudaGraphExecDestroy(graph);
        if (stream) cudaStreamDestroy(stream);
        streams.release();
        if (d_block) cudaFree(d_block);
        if (h_img) cudaFreeHost(h_img);
        if (h_out) cudaFreeHost(h_out);
    }
};

static std::mutex g_plan_mu;
static std::list<BatchPlan*> g_plans;

size_t batch_smem_bytes(int max_E) {
    const size_t contrib = (size_t)27 * BATCH_THREADS * sizeof(float);
    const size_t eps = (size_t)NOISE_SPB * max_E * sizeof(float);
    return sizeof(DevModel<float>) + std::max(contrib, eps);
}

static mppi_status build_plan(mppi_ctx* const* ctxs, int count, BatchPlan* P) {
    int dev;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    P->L = layout_batch(ctxs, count);
    e = cudaMalloc(&P->d_block, P->L.dev_bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&P->h_img, P->L.image_bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&P->h_out, P->L.out_bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch plan allocation");
    memset(P->h_img, 0, P->L.image_bytes);
    fill_batch_image(ctxs, P->L, nullptr, nullptr, P->h_img, &P->in_off, &P->out_off);
    size_t smem = 0;
    int per_sm = 0, sms = 0;
    e = prepare_batch_kernel(P->L.max_E, &smem, &per_sm);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch occupancy");
    const int grid = (int)std::min<long>((long)std::max(1, per_sm) * sms, P->L.total);
    // the launch sequence, captured once
    cudaGraph_t g = nullptr;
    e = P->streams.ensure((int)P->L.groups.size() - 1);  // before the capture
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch streams");
    e = cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch capture");
    cudaError_t ce = enqueue_batch(P->L, P->h_img, P->d_block, P->h_out, grid, smem, P->stream, P->streams);
    e = cudaStreamEndCapture(P->stream, &g);
    if (ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(nullptr, ce, "batch launch capture");
    }
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch end capture");
    e = cudaGraphInstantiate(&P->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch graph instantiate");
    return MPPI_OK;
}

BatchPlan* get_plan(mppi_ctx* const* ctxs, int count, mppi_status* st) {
    std::vector<uint64_t> uids(count);
    for (int i = 0; i < count; ++i) uids[i] = ctxs[i]->uid;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (auto it = g_plans.begin(); it != g_plans.end(); ++it)
        if ((*it)->uids == uids) {
            BatchPlan* p = *it;
            g_plans.erase(it);
            g_plans.push_front(p);
            *st = MPPI_OK;
            return p;
        }
    BatchPlan* p = new (std::nothrow) BatchPlan();
    if (!p) {
        *st = MPPI_ERR_OUT_OF_MEMORY;
        return nullptr;
    }
    p->uids = uids;
    *st = build_plan(ctxs, count, p);
    if (*st != MPPI_OK) {
        delete p;
        return nullptr;
    }
    g_plans.push_front(p);
    while (g_plans.size() > 4) {
        BatchPlan* old = g_plans.back();
        g_plans.pop_back();
        cudaStreamSynchronize(old->stream);
        delete old;
    }
    return p;
}

mppi_status run_plan(BatchPlan* P, mppi_ctx* const* ctxs, const double* const* states, const float* const* warm,
                     float* const* out_mean, float* const* out_best, mppi_result* info) {
    fill_batch_inputs(ctxs, P->L, P->in_off, states, warm, P->h_img);
    cudaError_t e = cudaGraphLaunch(P->graph, P->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch launch");
    return unpack_batch(ctxs, P->L, P->out_off, P->h_out, out_mean, out_best, info);
}

}  // namespace mppi

using namespace mppi;

namespace mppi {
mppi_status check_batchable(const mppi_ctx* c, int dev) {
    if (c->device != dev) {
        set_error(nullptr, "batched contexts must live on the current device");
        return MPPI_ERR_UNSUPPORTED;
    }
    if (c->mapping != MPPI_MAP_WARP && c->mapping != MPPI_MAP_HALFWARP && c->mapping != MPPI_MAP_CHAIN) {
        set_error(nullptr, "batched contexts need the warp, half-warp or chain mapping");
        return MPPI_ERR_UNSUPPORTED;
    }
    return MPPI_OK;
}
}  // namespace mppi

extern "C" mppi_status mppi_solve_batch(mppi_ctx* const* ctxs, int32_t count, const double* const* h_states,
                                        const float* const* h_warm, float* const* h_out_mean,
                                        float* const* h_out_best, mppi_result* h_info) {
    MPPI_NVTX("mppi_solve_batch");
    if (!ctxs || count < 1 || !h_states || !h_out_mean) return MPPI_ERR_INVALID_ARG;
    int dev;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    for (int i = 0; i < count; ++i) {
        mppi_ctx* c = ctxs[i];
        if (!c || !h_states[i] || !h_out_mean[i]) return MPPI_ERR_INVALID_ARG;
        mppi_status st = check_batchable(c, dev);
        if (st != MPPI_OK) return st;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) {
                set_error(nullptr, "a context appears twice in one batch");
                return MPPI_ERR_INVALID_ARG;
            }
        for (int k = 0; k < c->nx; ++k)
            if (!isfinite(h_states[i][k])) {
                set_error(nullptr, "state is not finite");
                return MPPI_ERR_NONFINITE_STATE;
            }
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "context stream");
    }
    mppi_status st;
    BatchPlan* P = get_plan(ctxs, count, &st);
    if (!P) return st;
    return run_plan(P, ctxs, h_states, h_warm, h_out_mean, h_out_best, h_info);
}

namespace mppi {
// Self-test of the persistent kernel's bounded wait: a queue of one item that is never
// published. The block that takes it must give up after budget_us and set the error word.
mppi_status queue_timeout_selftest(int64_t budget_us, int32_t* observed) {
    unsigned char* d = nullptr;
    const size_t bytes = 256 + 256;
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "selftest allocation");
    BatchQueue hq;
    memset(&hq, 0, sizeof hq);
    hq.total = 1;
    hq.nprefill = 0;
    QueueItem hi;
    memset(&hi, 0, sizeof hi);
    e = cudaMemcpy(d, &hq, sizeof hq, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + 256, &hi, sizeof hi, cudaMemcpyHostToDevice);
    size_t smem = 0;
    int per_sm = 0;
    if (e == cudaSuccess) e = prepare_batch_kernel(8, &smem, &per_sm);
    if (e == cudaSuccess) {
        persistent_kernel<BV_XYY><<<1, BATCH_THREADS, smem>>>(nullptr, nullptr, reinterpret_cast<QueueItem*>(d + 256),
                                                    reinterpret_cast<BatchQueue*>(d), (uint64_t)budget_us * 1000ull);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    uint32_t err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, d + offsetof(BatchQueue, error), sizeof err, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "selftest launch");
    if (observed) *observed = (int32_t)err;
    if (err & DEV_ERR_QUEUE_TIMEOUT) {
        set_error(nullptr, "the persistent kernel's queue wait gave up as designed");
        return MPPI_ERR_TIMEOUT;
    }
    return MPPI_OK;
}
}  // namespace mppi

extern "C" mppi_status mppi_selftest_queue_timeout(int64_t budget_us, int32_t* h_error_bits) {
    if (budget_us < 1 || budget_us > 10000000) return MPPI_ERR_INVALID_ARG;
    return mppi::queue_timeout_selftest(budget_us, h_error_bits);
}

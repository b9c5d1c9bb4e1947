// Cost -> weight reduction (Sec. III-C Eqs. omega-weights / softmax_minmax) and the
// FP64 knot average (Eq. update-nominal), shared by the per-iteration kernels and the
// persistent batched kernel so both produce identical bits.
//
// Layout of the work: samples are cut into chunks of AVG_CHUNK. For chunk c a block
//   1. scans all N FP32 costs for S_min, S_max, the argmin (ties -> lowest index) and the
//      number of finite costs (cheap; every block does it redundantly),
//   2. forms the unnormalised weights e_n = exp(-S_hat_n / lambda) of its own samples in
//      FP64 (every e_n <= 1 and the argmin's e is exactly 1, so nothing overflows),
//   3. writes P_c[e] = sum_{n in c} e_n theta_{n,e} (FP64) and, from the first element
//      tile, z_c = sum e_n and q_c = sum e_n^2.
// The iteration's finalize then forms z = sum_c z_c, lse = log z, ESS = z^2 / sum q_c and
// the mean sum_c P_c[e] / z. Each sum runs in a fixed order (interleaved accumulators and
// balanced trees, since a long chain of dependent FP64 operations is slow on this part),
// so results depend only on AVG_CHUNK, never on the block size, the grid or scheduling.
#pragma once
#include "internal.h"

namespace mppi {

struct MinMax {
    float smin, smax;
    int best, nfinite;
};

// Block-wide scan of N costs; every thread receives the result. Any block size that is a
// multiple of 32 and at most 1024.
__device__ __forceinline__ MinMax block_minmax(const float* __restrict__ costs, int N) {
    __shared__ float s_min[32], s_max[32];
    __shared__ int s_arg[32], s_cnt[32];
    __shared__ MinMax s_res;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    float mn = INFINITY, mx = -INFINITY;
    int arg = 0x7fffffff, cnt = 0;
    auto take = [&](float c, int n) {
        if (isfinite(c)) {
            ++cnt;
            if (c < mn) {
                mn = c;
                arg = n;
            }
            mx = fmaxf(mx, c);
        }
    };
    // 16-byte loads, unrolled so a thread's loads (from L2) are in flight together. The
    // result does not depend on how indices are spread over threads: min and max are
    // exact and ties go to the lowest index.
    int head = 0;
    if ((reinterpret_cast<uintptr_t>(costs) & 15) == 0) {
        const float4* c4 = reinterpret_cast<const float4*>(costs);
        const int n4 = N >> 2;
#pragma unroll 4
        for (int i = t; i < n4; i += blockDim.x) {
            const float4 v = c4[i];
            take(v.x, 4 * i);
            take(v.y, 4 * i + 1);
            take(v.z, 4 * i + 2);
            take(v.w, 4 * i + 3);
        }
        head = n4 << 2;
    }
#pragma unroll 4
    for (int n = head + t; n < N; n += blockDim.x) take(costs[n], n);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float omn = __shfl_xor_sync(0xffffffffu, mn, off);
        const int oarg = __shfl_xor_sync(0xffffffffu, arg, off);
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
        if (omn < mn || (omn == mn && oarg < arg)) {
            mn = omn;
            arg = oarg;
        }
    }
    __syncthreads();
    if (lane == 0) {
        s_min[wid] = mn;
        s_max[wid] = mx;
        s_arg[wid] = arg;
        s_cnt[wid] = cnt;
    }
    __syncthreads();
    if (t == 0) {
        MinMax r{INFINITY, -INFINITY, 0x7fffffff, 0};
        for (int i = 0; i < nw; ++i) {
            if (s_min[i] < r.smin || (s_min[i] == r.smin && s_arg[i] < r.best)) {
                r.smin = s_min[i];
                r.best = s_arg[i];
            }
            r.smax = fmaxf(r.smax, s_max[i]);
            r.nfinite += s_cnt[i];
        }
        if (r.nfinite == 0) r.best = -1;
        s_res = r;
    }
    __syncthreads();
    return s_res;
}

// Unnormalised weight of one cost given the scan (0 for non-finite costs).
__device__ __forceinline__ double unnorm_weight(float c, const MinMax& mm, double lambda, int normalize) {
    if (!isfinite(c)) return 0.0;
    const double range = (double)mm.smax - (double)mm.smin;
    const double scale = normalize == MPPI_NORM_MINMAX ? (range > 0.0 ? 1.0 / range : 0.0) : 1.0;
    return exp(-(((double)c - (double)mm.smin) * scale) / lambda);
}

// One (chunk, element tile) block: weights of the chunk and its partial knot sums.
// e_out (nullable) [N], zq [nchunks][2], partial [nchunks][E]. Element tile ey covers
// elements [ey * blockDim.x, (ey + 1) * blockDim.x).
__device__ __noinline__ void chunk_weights_average(const float* __restrict__ costs, const float* __restrict__ knots,
                                                      int N, int E, double lambda, int normalize, int c, int ey,
                                                      double* __restrict__ e_out, double* __restrict__ zq,
                                                      double* __restrict__ partial, DevIterInfo* __restrict__ info) {
    __shared__ double s_e[AVG_CHUNK];
    const MinMax mm = block_minmax(costs, N);
    const int n0 = c * AVG_CHUNK;
    const int cn = min(AVG_CHUNK, N - n0);
    for (int i = threadIdx.x; i < AVG_CHUNK; i += blockDim.x) {
        const double e = (i < cn && mm.nfinite > 0) ? unnorm_weight(costs[n0 + i], mm, lambda, normalize) : 0.0;
        s_e[i] = e;  // zero past the chunk's end
        if (e_out && ey == 0 && i < cn) e_out[n0 + i] = e;
    }
    __syncthreads();
    // FP64 latency is long on this part, so no sum is one long dependent chain: the knot
    // partials use 8 accumulators (sample i into i mod 8, increasing i) combined as a
    // balanced tree, and z, q a fixed pairwise tree over the 64 weights
    const int el = ey * blockDim.x + threadIdx.x;
    if (el < E) {
        // all AVG_CHUNK loads are independent and issued together; past the chunk's end
        // (the last, ragged chunk) the index is clamped and the weight is 0, so the term
        // adds nothing
        const float* kp = knots + (size_t)n0 * E + el;
        double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int i0 = 0; i0 < AVG_CHUNK; i0 += 8) {
            float kv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) kv[u] = kp[(size_t)min(i0 + u, cn - 1) * E];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = fma(s_e[i0 + u], (double)kv[u], a[u]);
        }
        partial[(size_t)c * E + el] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    }
    if (ey == 0 && threadIdx.x < 32) {
        const int t = threadIdx.x;
        const double e0 = s_e[t], e1 = s_e[t + 32];
        double z = e0 + e1, q = fma(e0, e0, e1 * e1);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            z += __shfl_down_sync(0xffffffffu, z, off);
            q += __shfl_down_sync(0xffffffffu, q, off);
        }
        if (t == 0) {
            zq[2 * c] = z;
            zq[2 * c + 1] = q;
            if (c == 0) {
                info->smin = mm.nfinite ? (double)mm.smin : NAN;
                info->smax = mm.nfinite ? (double)mm.smax : NAN;
                info->best = mm.best;
                info->nfinite = mm.nfinite;
                info->status = mm.nfinite ? MPPI_OK : MPPI_ERR_ALL_COSTS_NONFINITE;
            }
        }
    }
    __syncthreads();
}

constexpr int FIN_SPLIT = 16;  // interleaved sub-sums per element total in the finalize
constexpr int FIN_TILE = 128;   // elements per finalize tile

// sum of 16 values in a fixed balanced tree
__device__ __forceinline__ double tree16(const double* v, int stride) {
    double l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) l[i] = v[(2 * i) * stride] + v[(2 * i + 1) * stride];
    return ((l[0] + l[1]) + (l[2] + l[3])) + ((l[4] + l[5]) + (l[6] + l[7]));
}

// Block-wide: z = sum_c z_c and q = sum_c q_c. One warp per total: lane l sums chunks
// c = l, l + 32, ... in increasing order, then a fixed shuffle tree. Every thread receives
// the totals. Needs blockDim.x >= 64.
__device__ __forceinline__ void block_total_zq(const double* __restrict__ zq, int nchunks, double* z, double* q) {
    __shared__ double s_tot[2];
    const int t = threadIdx.x;
    if (t < 64) {
        const int lane = t & 31, which = t >> 5;
        double acc = 0.0;
#pragma unroll 4
        for (int c = lane; c < nchunks; c += 32) acc += zq[2 * c + which];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
        if (lane == 0) s_tot[which] = acc;
    }
    __syncthreads();
    *z = s_tot[0];
    *q = s_tot[1];
}

// Sum of the partials of element e over chunks in increasing order.
__device__ __forceinline__ double chunk_total(const double* __restrict__ partial, int nchunks, int E, int e) {
    double acc = 0.0;
    for (int c = 0; c < nchunks; ++c) acc += partial[(size_t)c * E + e];
    return acc;
}

// End of one iteration (one block, any size): lse and ESS, mean = sum_c P_c / z,
// best-trajectory tracking over the solve (Sec. III-D), next nominal, and at the last
// iteration the outputs, the resident warm start and the noise counter.
__device__ __noinline__ void finalize_iteration(const FinalizeArgs& a) {
    __shared__ int s_update;
    const int t = threadIdx.x;
    DevIterInfo inf = *a.info;
    const bool ok = inf.status == MPPI_OK;
    double z = 0.0, q = 0.0;
    block_total_zq(a.zq, a.nchunks, &z, &q);
    // the mean multiplies by 1 / z; lse and ESS are formed at the end, off the element path
    const double inv_z = 1.0 / z;
    if (t == 0) {
        int upd = 0;
        if (ok) {
            const double cb = (double)a.costs[inf.best];
            if (cb < a.solve->best_cost) {
                upd = 1;
                a.solve->best_cost = cb;
                a.solve->best_index = inf.best;
                a.solve->best_iter = a.iter;
            }
        } else {
            a.solve->status = inf.status;
        }
        s_update = upd;
    }
    __syncthreads();
    const bool last = a.iter == a.iters - 1;
    // chunk totals: FIN_SPLIT interleaved sub-sums per element (chunks c = s, s + FIN_SPLIT,
    // ... in increasing order) spread over the block, then combined by a balanced tree
    __shared__ double s_sub[FIN_SPLIT * FIN_TILE];
    for (int e0 = 0; e0 < a.E; e0 += FIN_TILE) {
        if (ok)
            for (int task = t; task < FIN_SPLIT * FIN_TILE; task += blockDim.x) {
                const int sidx = task / FIN_TILE, el = task - sidx * FIN_TILE, e = e0 + el;
                double acc = 0.0;
                if (e < a.E) {
#pragma unroll 8
                    for (int c = sidx; c < a.nchunks; c += FIN_SPLIT) acc += a.partial[(size_t)c * a.E + e];
                }
                s_sub[task] = acc;
            }
        __syncthreads();
        for (int el = t; el < FIN_TILE && e0 + el < a.E; el += blockDim.x) {
            const int e = e0 + el;
            float m = a.nominal[e];
            if (ok) m = (float)(tree16(s_sub + el, FIN_TILE) * inv_z);
            if (s_update) a.best_out[e] = a.knots[(size_t)inf.best * a.E + e];
            if (last) a.mean_out[e] = m;
            a.nominal[e] = m;
        }
        __syncthreads();
    }
    if (t == 0) {
        inf.lse = ok ? log(z) : NAN;
        inf.ess = ok ? z * z / q : 0.0;
        a.info->lse = inf.lse;
        a.info->ess = inf.ess;
    }
    if (last) {
        if (a.warm_from == MPPI_WARM_BEST && a.solve->best_index >= 0)
            for (int e = t; e < a.E; e += blockDim.x) a.nominal[e] = a.best_out[e];
        if (t == 0) {
            mppi_result r;
            r.cost_min = inf.smin;
            r.cost_max = inf.smax;
            r.best_cost = a.solve->best_cost;
            r.ess = inf.ess;
            r.lse = inf.lse;
            r.best_index = a.solve->best_index;
            r.best_iter = a.solve->best_iter;
            r.n_finite = inf.nfinite;
            r.status = a.solve->status;
            *a.result = r;
            a.solve->iter_counter += (uint32_t)a.iters;
        }
    }
    __syncthreads();
}

}  // namespace mppi

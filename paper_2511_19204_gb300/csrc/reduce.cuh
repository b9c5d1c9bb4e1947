// Cost -> weight reduction (Sec. III-C Eqs. omega-weights / softmax_minmax) and the
// FP64 knot average (Eq. update-nominal), shared by the per-iteration kernels and the
// persistent batched kernel so both produce identical bits.
//
// Layout of the work: samples are cut into chunks of AVG_CHUNK, chunks into groups of
// AVG_GROUP. For chunk c a block
//   1. scans all N FP32 costs for S_min, S_max, the argmin (ties -> lowest index) and the
//      number of finite costs (cheap; every block does it redundantly),
//   2. forms the unnormalised weights e_n = exp(-S_hat_n / lambda) of its own samples in
//      FP64 (every e_n <= 1 and the argmin's e is exactly 1, so nothing overflows),
//   3. writes P_c[e] = sum_{n in c} e_n theta_{n,e} (FP64), z_c = sum e_n and
//      q_c = sum e_n^2.
// The last chunk of a group to finish sums the group's partials (G_g), and the last group
// to finish runs the finalize: z = sum_g z_g, lse = log z, ESS = z^2 / sum q, the mean
// sum_g G_g[e] / z. Each sum runs in a fixed order (interleaved accumulators and balanced
// trees, since a long chain of dependent FP64 operations is slow on this part), so results
// depend only on AVG_CHUNK and AVG_GROUP, never on the block size, the grid or scheduling.
#pragma once
#include "internal.h"

namespace mppi {

// Acquire-release fence at GPU scope. The arrival counters of the reduction use it instead
// of __threadfence() (a sequentially consistent fence, about a microsecond on this
// two-die part): every thread fences its own stores (release) before the block's barrier
// and the counting atomic; the block that finds itself last fences again (acquire) before
// reading the others' results through L2.
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

struct MinMax {
    float smin, smax;
    int best, nfinite;
    double k;   // weight scale: 1 / ((S_max - S_min) lambda) (min-max normalised) or 1 / lambda (raw)
};

__device__ __forceinline__ void minmax_merge(float& mn, int& arg, float& mx, int& cnt, float omn, int oarg, float omx,
                                             int ocnt) {
    if (omn < mn || (omn == mn && oarg < arg)) {
        mn = omn;
        arg = oarg;
    }
    mx = fmaxf(mx, omx);
    cnt += ocnt;
}

// Block-wide scan of N costs; every thread receives the result, including the weight
// scale k (computed once, by one thread: FP64 division is slow on this part). Any block
// size that is a multiple of 32 and at most 1024.
__device__ __forceinline__ MinMax block_minmax(const float* __restrict__ costs, int N, double lambda, int normalize) {
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
    for (int off = 16; off > 0; off >>= 1)
        minmax_merge(mn, arg, mx, cnt, __shfl_xor_sync(0xffffffffu, mn, off), __shfl_xor_sync(0xffffffffu, arg, off),
                     __shfl_xor_sync(0xffffffffu, mx, off), __shfl_xor_sync(0xffffffffu, cnt, off));
    __syncthreads();
    if (lane == 0) {
        s_min[wid] = mn;
        s_max[wid] = mx;
        s_arg[wid] = arg;
        s_cnt[wid] = cnt;
    }
    __syncthreads();
    if (wid == 0) {
        // warp 0 merges the warps' results by the same shuffle tree
        mn = lane < nw ? s_min[lane] : INFINITY;
        mx = lane < nw ? s_max[lane] : -INFINITY;
        arg = lane < nw ? s_arg[lane] : 0x7fffffff;
        cnt = lane < nw ? s_cnt[lane] : 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            minmax_merge(mn, arg, mx, cnt, __shfl_xor_sync(0xffffffffu, mn, off),
                         __shfl_xor_sync(0xffffffffu, arg, off), __shfl_xor_sync(0xffffffffu, mx, off),
                         __shfl_xor_sync(0xffffffffu, cnt, off));
        if (lane == 0) {
            MinMax r{mn, mx, cnt ? arg : -1, cnt, 0.0};
            if (cnt) {
                // one division: a dependent FP64 division takes ~400 cycles on this part
                const double range = (double)mx - (double)mn;
                r.k = normalize == MPPI_NORM_MINMAX ? (range > 0.0 ? 1.0 / (range * lambda) : 0.0) : 1.0 / lambda;
            }
            s_res = r;
        }
    }
    __syncthreads();
    return s_res;
}

// Unnormalised weight of one cost given the scan: exp(-(S - S_min) k), 0 for non-finite
// costs. S - S_min of two FP32 values is exact in FP64.
__device__ __forceinline__ double unnorm_weight(float c, const MinMax& mm) {
    if (!isfinite(c)) return 0.0;
    return exp(-(((double)c - (double)mm.smin) * mm.k));
}

// Exact FP32 -> FP64 widening by integer operations only (IEEE 754 binary32 ->
// binary64), so that converting every knot does not occupy the FP64 pipe, which is narrow
// on this part (about two lanes per SM per clock, shared by FP64 arithmetic and
// conversions). Normal numbers: the sign kept, the exponent rebiased by 1023 - 127 = 896,
// the significand shifted left by 29 bits. Zeros: the sign alone. Subnormals m 2^-149
// (m < 2^23): normalised by the position p of m's leading one, exponent p - 149 + 1023,
// fraction m shifted left by 52 - p with the leading one dropped. Infinities and NaNs: the
// all-ones exponent with the significand shifted as for normals, NaNs quieted. Every
// branch is a select: nothing here issues an FP64 instruction.
__device__ __forceinline__ double widen(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t sign = b & 0x80000000u;
    const uint32_t ex = (b >> 23) & 0xffu;
    const uint32_t m = b & 0x7fffffu;
    // normal (and, with the exponent field replaced, infinity / NaN)
    uint32_t hi = sign | ((ex + 896u) << 20) | (m >> 3);
    uint32_t lo = m << 29;
    // subnormal: p = 31 - clz(m) in 0..22, fraction (m << (52 - p)) without bit 52
    const int p = 31 - __clz((int)(m | 1u));
    const uint64_t frac = ((uint64_t)m << (52 - p)) & 0x000fffffffffffffull;
    const uint32_t hi_sub = sign | ((uint32_t)(p + 874) << 20) | (uint32_t)(frac >> 32);
    const uint32_t lo_sub = (uint32_t)frac;
    const bool sub = ex == 0u && m != 0u, zero = ex == 0u && m == 0u, special = ex == 0xffu;
    const uint32_t m_nan = m != 0u ? (m | 0x400000u) : 0u;  // quiet NaN, infinity unchanged
    hi = special ? (sign | 0x7ff00000u | (m_nan >> 3)) : hi;
    lo = special ? (m_nan << 29) : lo;
    hi = sub ? hi_sub : (zero ? sign : hi);
    lo = sub ? lo_sub : (zero ? 0u : lo);
    return __hiloint2double((int)hi, (int)lo);
}

// Sum of the first n <= 16 of v[0..15] in the fixed balanced tree of 16 leaves with the
// missing leaves zero: (((v0 + v1) + (v2 + v3)) + ((v4 + v5) + (v6 + v7))) + (...). A node
// whose right subtree is all zeros passes its left value up unchanged, so those additions
// (exact: x + 0 = x) are skipped; n is the same for every thread that calls it.
__device__ __forceinline__ double tree16n(double* v, int n) {
#pragma unroll
    for (int w = 1; w < 16; w *= 2) {
        // level: nodes i of width 2w; node value = left (v[2 w i]) + right (v[2 w i + w])
#pragma unroll
        for (int i = 0; i < 16; i += 2 * w)
            if (i + w < n) v[i] = v[i] + v[i + w];
    }
    return v[0];
}

// Sum of n values src[0], src[stride], ... (written by other blocks of the launch) in a
// fixed order: blocks of 16 consecutive values, each summed by tree16n, added in
// increasing order.
__device__ __forceinline__ double ordered_total(const double* src, int n, size_t stride) {
    double acc = 0.0;
    for (int b0 = 0; b0 < n; b0 += 16) {
        const int m = min(16, n - b0);
        double v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = k < m ? __ldcg(src + (size_t)(b0 + k) * stride) : 0.0;
        acc = b0 == 0 ? tree16n(v, m) : acc + tree16n(v, m);
    }
    return acc;
}

constexpr int SUB_SPLIT = 8;    // interleaved sub-sums per element of a chunk (sample i -> i mod 8)
constexpr int SUB_TILE = 256;   // elements per tile of the chunk sums
constexpr int SUB_TERMS = AVG_CHUNK / SUB_SPLIT;

// The SUB_TERMS knots of task k of a tile of ne elements starting at e0 (sub-sum u = k / ne,
// element e0 + k mod ne) of the chunk at n0 (cn samples; a clamped index past the ragged
// end meets a zero weight).
__device__ __forceinline__ void load_task(const float* __restrict__ knots, int n0, int cn, int E, int e0, int ne,
                                          int k, float* kv) {
    const int u = k / ne, el = k - u * ne;
    const float* kp = knots + (size_t)n0 * E + e0 + el;
#pragma unroll
    for (int j = 0; j < SUB_TERMS; ++j) kv[j] = kp[(size_t)min(u + SUB_SPLIT * j, cn - 1) * E];
}

// One chunk of AVG_CHUNK samples (block-wide, any block size that is a multiple of 32 and
// at least 64): its unnormalised weights (written to e_out when non-null), z_c and q_c,
// and (E > 0) its FP64 partial knot sums P_c[e] = sum_i e_i theta_{n0+i, e}. Each partial
// is formed as SUB_SPLIT interleaved sub-sums (sample i into sub-sum i mod 8, increasing
// i, fused multiply-adds from 0) combined as a balanced tree; the (sub-sum, element) tasks
// are spread evenly over the whole block, two at a time per thread with their chains
// interleaved (a dependent FP64 multiply-add takes ~65 cycles on this part), so the
// result never depends on the block size. Every sum runs in a fixed order: no sum is one
// long dependent chain, and the same bits come out of every launch shape. The knots of a
// thread's first two tasks are loaded while the weights are formed.
__device__ __noinline__ void chunk_partial(const float* __restrict__ costs, const float* __restrict__ knots, int N,
                                           int E, double lambda, int normalize, int c, double* __restrict__ e_out,
                                           double* __restrict__ zq, double* __restrict__ partial,
                                           DevIterInfo* __restrict__ info) {
    __shared__ double s_e[AVG_CHUNK];
    __shared__ double s_sub[SUB_SPLIT][SUB_TILE];
    const int t = threadIdx.x, B = blockDim.x;
    const int n0 = c * AVG_CHUNK;
    const int cn = min(AVG_CHUNK, N - n0);
    if (!MPPI_CHECK_OK(n0 < N && n0 >= 0, CHECK_CHUNK)) return;
    const MinMax mm = block_minmax(costs, N, lambda, normalize);
    // the first pair of tasks of the first tile: loads in flight while the weights form
    const int ne0 = min(SUB_TILE, E), nt0 = SUB_SPLIT * ne0;
    float ka[SUB_TERMS], kb[SUB_TERMS];
    if (t < nt0) load_task(knots, n0, cn, E, 0, ne0, t, ka);
    if (t + B < nt0) load_task(knots, n0, cn, E, 0, ne0, t + B, kb);
    for (int i = t; i < AVG_CHUNK; i += B) {
        const double e = (i < cn && mm.nfinite > 0) ? unnorm_weight(costs[n0 + i], mm) : 0.0;
        s_e[i] = e;  // zero past the chunk's end: a clamped index then adds nothing
        if (e_out && i < cn) e_out[n0 + i] = e;
    }
    if (c == 0 && t == 0) {
        info->smin = mm.nfinite ? (double)mm.smin : NAN;
        info->smax = mm.nfinite ? (double)mm.smax : NAN;
        info->best = mm.best;
        info->nfinite = mm.nfinite;
        info->status = mm.nfinite ? MPPI_OK : MPPI_ERR_ALL_COSTS_NONFINITE;
    }
    __syncthreads();
    if (t >= B - 32) {
        // the last warp forms z_c = sum e and q_c = sum e^2 (fixed shuffle tree) before its
        // knot tasks (it has the fewest of them)
        const int l = t - (B - 32);
        const double e0v = s_e[l], e1v = s_e[l + 32];
        double z = e0v + e1v, q = fma(e0v, e0v, e1v * e1v);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            z += __shfl_down_sync(0xffffffffu, z, off);
            q += __shfl_down_sync(0xffffffffu, q, off);
        }
        if (l == 0) {
            zq[2 * c] = z;
            zq[2 * c + 1] = q;
        }
    }
    for (int e0 = 0; e0 < E; e0 += SUB_TILE) {
        const int ne = min(SUB_TILE, E - e0), nt = SUB_SPLIT * ne;
        for (int k = t; k < nt; k += 2 * B) {
            const bool two = k + B < nt;
            if (e0 > 0 || k > t) {
                load_task(knots, n0, cn, E, e0, ne, k, ka);
                if (two) load_task(knots, n0, cn, E, e0, ne, k + B, kb);
            }
            const int ua = k / ne, ub = (k + B) / ne;
            double acc_a = 0.0, acc_b = 0.0;
#pragma unroll
            for (int j = 0; j < SUB_TERMS; ++j) {
                acc_a = fma(s_e[ua + SUB_SPLIT * j], widen(ka[j]), acc_a);
                if (two) acc_b = fma(s_e[ub + SUB_SPLIT * j], widen(kb[j]), acc_b);
            }
            s_sub[ua][k - ua * ne] = acc_a;
            if (two) s_sub[ub][k + B - ub * ne] = acc_b;
        }
        __syncthreads();
        for (int el = t; el < ne; el += B)
            partial[(size_t)c * E + e0 + el] = ((s_sub[0][el] + s_sub[1][el]) + (s_sub[2][el] + s_sub[3][el])) +
                                               ((s_sub[4][el] + s_sub[5][el]) + (s_sub[6][el] + s_sub[7][el]));
        __syncthreads();
    }
}

// Group g's totals (block-wide): G_g[e] = tree16n of the partials of chunks 16 g ..
// 16 g + 15 (the last group may have fewer), and the same for (z_c, q_c).
__device__ __forceinline__ void group_total(const double* __restrict__ partial, const double* __restrict__ zq,
                                            int nchunks, int E, int g, double* __restrict__ gpartial,
                                            double* __restrict__ gzq) {
    const int c0 = g * AVG_GROUP, cn = min(AVG_GROUP, nchunks - c0);
    for (int e = threadIdx.x; e < E + 2; e += blockDim.x) {
        const double* src = e < E ? partial + (size_t)c0 * E + e : zq + 2 * c0 + (e - E);
        const size_t stride = e < E ? (size_t)E : 2;
        double v[AVG_GROUP];
#pragma unroll
        for (int k = 0; k < AVG_GROUP; ++k) v[k] = k < cn ? __ldcg(src + k * stride) : 0.0;
        const double tot = tree16n(v, cn);
        if (e < E) gpartial[(size_t)g * E + e] = tot;
        else gzq[2 * g + (e - E)] = tot;
    }
}

constexpr int FIN_BARRIER = 15;   // named barrier of the finalize (the rollouts use 1..4)

// End of one iteration (one block of at least 64 threads): z = sum_g z_g, q = sum_g q_g,
// lse and ESS, the mean sum_g G_g / z, best-trajectory tracking over the solve
// (Sec. III-D), the next nominal, and at the last iteration the outputs, the resident warm
// start and the noise counter. Dependent FP64 operations are slow on this part (an add
// ~65 cycles, a division ~400, a logarithm ~2000) and so is a load of what another SM
// wrote (it may sit in the other die's L2), so the work is laid out to keep one round
// trip and few dependent FP64 operations on the path to the stores:
//   - the last warp is the scalar warp: its lane 0 issues every load it needs at once (the
//     iteration's info, the solve's best so far, the group (z_g, q_g)), forms z and 1 / z
//     and the best tracking (the iteration's best cost is S_min, stored by chunk 0, so no
//     load waits on the best index), publishes them in shared memory and arrives at a
//     named barrier; it then forms log z and the ESS and the result while
//   - the other warps, after loading and summing the group totals of their elements,
//     wait at that barrier only for 1 / z and the best index, and store the elements.
__device__ __noinline__ void finalize_iteration(const FinalizeArgs& a) {
    __shared__ double s_inv_z;
    __shared__ int s_update, s_ok, s_best, s_best_final;
    const int t = threadIdx.x, B = blockDim.x;
    const int ts = B - 32;   // first lane of the scalar warp
    const bool last = a.iter == a.iters - 1;
    if (t >= ts) {
        DevIterInfo inf;
        double z = 0.0, q = 0.0, best_cost = 0.0;
        int best_index = -1, best_iter = -1, status = MPPI_OK;
        uint32_t ctr = 0;
        bool ok = false, upd = false;
        if (t == ts) {
            const int ng = a.ngroups;
            // every load first: one round trip
            inf = *a.info;
            const double prev = a.solve->best_cost;
            const int prev_index = a.solve->best_index;
            const int prev_iter = a.solve->best_iter;
            const int prev_status = a.solve->status;
            ctr = a.solve->iter_counter;
            z = ordered_total(a.gzq, ng, 2);
            q = ordered_total(a.gzq + 1, ng, 2);
            ok = inf.status == MPPI_OK;
            upd = ok && inf.smin < prev;   // S_min is the best sample's cost (ties -> lowest index)
            best_cost = upd ? inf.smin : prev;
            best_index = upd ? inf.best : prev_index;
            best_iter = upd ? a.iter : prev_iter;
            status = ok ? prev_status : inf.status;
            s_inv_z = 1.0 / z;
            s_update = upd;
            s_ok = ok;
            s_best = inf.best;
            s_best_final = best_index;
            __threadfence_block();
        }
        __syncwarp();
        asm volatile("bar.arrive %0, %1;" ::"r"(FIN_BARRIER), "r"(B) : "memory");
        if (t == ts) {
            if (upd) {
                a.solve->best_cost = best_cost;
                a.solve->best_index = best_index;
                a.solve->best_iter = best_iter;
            }
            if (!ok) a.solve->status = status;
            const double lse = ok ? log(z) : NAN;
            const double ess = ok ? z * z / q : 0.0;
            a.info->lse = lse;
            a.info->ess = ess;
            if (last) {
                mppi_result r;
                r.cost_min = inf.smin;
                r.cost_max = inf.smax;
                r.best_cost = best_cost;
                r.ess = ess;
                r.lse = lse;
                r.best_index = best_index;
                r.best_iter = best_iter;
                r.n_finite = inf.nfinite;
                r.status = status;
                *a.result = r;
                a.solve->iter_counter = ctr + (uint32_t)a.iters;
            }
        }
    } else {
        // element warps: totals of this thread's elements (independent of the scalar lane)
        constexpr int PER = 8;   // elements per thread held across the barrier: E <= PER (B - 32)
        static_assert(PER * (160 - 32) >= MAXK * 2 * (MAXB - 1), "finalize blocks need >= 160 threads");
        double tot[PER];
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = t + r * ts;
            tot[r] = e < a.E ? ordered_total(a.gpartial + e, a.ngroups, (size_t)a.E) : 0.0;
        }
        asm volatile("bar.sync %0, %1;" ::"r"(FIN_BARRIER), "r"(B) : "memory");
        const double inv_z = s_inv_z;
        const bool ok = s_ok;
        const int best = s_best;
        // (the check build skips the copy of an out-of-range best sample; no early return,
        // the block's last barrier is still ahead)
        const bool upd = s_update && MPPI_CHECK_OK(best >= 0 && best < a.nchunks * AVG_CHUNK, CHECK_BEST);
        const bool keep_best = last && a.warm_from == MPPI_WARM_BEST && s_best_final >= 0;
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = t + r * ts;
            if (e >= a.E) break;
            const float m = ok ? (float)(tot[r] * inv_z) : a.nominal[e];
            float bv = 0.f;
            if (upd) {
                bv = a.knots[(size_t)best * a.E + e];
                a.best_out[e] = bv;
            } else if (keep_best) {
                bv = a.best_out[e];
            }
            if (last) a.mean_out[e] = m;
            a.nominal[e] = keep_best ? bv : m;
        }
    }
    __syncthreads();
}

// The weights and average of one chunk, then whatever finishing the chunk's arrival
// completes (block-wide): the last chunk of a group to finish sums the group's partials,
// and the last group to finish runs the iteration's finalize. Each block fences its
// writes before counting itself; the last block of a group resets the group's counter and
// the finalizing block resets DevSolve::blocks_done. The sums and their order depend only
// on AVG_CHUNK and AVG_GROUP, so a single solve and a batched instance give the same
// bits. Returns true in the block that ran the finalize.
__device__ __noinline__ bool reduce_chunk(const FinalizeArgs& f, int N, double lambda, int normalize, int c) {
    __shared__ int s_last;
    chunk_partial(f.costs, f.knots, N, f.E, lambda, normalize, c, nullptr, f.zq, f.partial, f.info);
    const int g = c / AVG_GROUP;
    const int members = min(AVG_GROUP, f.nchunks - g * AVG_GROUP);
    fence_acq_rel_gpu();
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool last = atomicAdd(&f.gcount[g], 1u) == (unsigned)(members - 1);
        if (last) fence_acq_rel_gpu();
        s_last = last;
    }
    __syncthreads();
    if (!s_last) return false;
    if (threadIdx.x == 0) f.gcount[g] = 0;
    group_total(f.partial, f.zq, f.nchunks, f.E, g, f.gpartial, f.gzq);
    fence_acq_rel_gpu();
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool last = atomicAdd(&f.solve->blocks_done, 1u) == (unsigned)(f.ngroups - 1);
        if (last) fence_acq_rel_gpu();
        s_last = last;
    }
    __syncthreads();
    if (!s_last) return false;
    finalize_iteration(f);
    if (threadIdx.x == 0) f.solve->blocks_done = 0;
    return true;
}

// ------------------------------------------------------------------------------------
// Single-level finish for launches whose chunks all fit on the device at once (a
// cooperative launch, one chunk per block): after its chunk, every block waits at a
// device-wide barrier and then reduces a slice of the elements over all chunks itself,
// forming the same group totals G_g (tree16n over 16 chunks) and the same total over the
// groups as the two-level path, so the results are bit-identical to it (and to batched
// instances). This replaces two hand-offs through global memory (a fence, an atomic and a
// round of loads each, 1-3 us on this two-die part) by one.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

constexpr uint64_t GRID_WAIT_NS = 2000000000ull;   // 2 s: far beyond any legitimate wait

// Device-wide barrier of a cooperative launch: each block adds one to `counter` (which
// only grows within a solve: the solve's first kernel resets it) and waits until it reaches
// `target`. The wait is bounded by the global timer; when it gives up it sets
// DEV_ERR_GRID_TIMEOUT in *err and returns false.
__device__ __forceinline__ bool grid_wait(uint32_t* counter, uint32_t target, uint32_t* err) {
    __shared__ int s_ok;
    fence_acq_rel_gpu();
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(counter, 1u);
        const uint64_t t0 = global_ns();
        bool ok = true;
        while (ld_acquire_gpu(counter) < target) {
            if (global_ns() - t0 > GRID_WAIT_NS) {
                atomicOr(err, DEV_ERR_GRID_TIMEOUT);
                ok = false;
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Block-wide, blockDim.x >= 64, one chunk per block, gridDim.x == nchunks <= 16 AVG_GROUP
// (at most 16 groups), the solve's blocks_done counter reset by the solve's first kernel.
__device__ __forceinline__ void reduce_chunk_grid(const FinalizeArgs& f, int N, double lambda, int normalize) {
    __shared__ double s_G[1024];       // [element slot][group] group totals of this block's elements
    __shared__ double s_zq[2 * 16 * AVG_GROUP];   // every chunk's (z_c, q_c), loaded coalesced
    __shared__ double s_zg[2 * 16];    // [z | q][group]
    __shared__ double s_inv_z;
    __shared__ int s_ok, s_upd, s_best, s_best_final;
    const int t = threadIdx.x, B = blockDim.x, ts = B - 32;
    const int G = gridDim.x, c = blockIdx.x;
    const bool last = f.iter == f.iters - 1;
    // the solve's best so far, read before the barrier: block 0 updates it after
    double prev = 0.0;
    int prev_index = -1, prev_iter = -1, prev_status = MPPI_OK;
    uint32_t ctr = 0;
    if (t == ts) {
        prev = f.solve->best_cost;
        prev_index = f.solve->best_index;
        prev_iter = f.solve->best_iter;
        prev_status = f.solve->status;
        ctr = f.solve->iter_counter;
    }
    chunk_partial(f.costs, f.knots, N, f.E, lambda, normalize, c, nullptr, f.zq, f.partial, f.info);
    if (!grid_wait(&f.solve->blocks_done, (uint32_t)(f.iter + 1) * (uint32_t)G, &f.solve->dev_error)) return;
    const int ng = f.ngroups;
    const int epb = (f.E + G - 1) / G;            // elements per block
    const int e_lo = c * epb;
    const int ne = max(0, min(epb, f.E - e_lo));
    // group totals of this block's elements (threads below ts) and of (z, q) (scalar warp)
    DevIterInfo inf;
    if (t < ts) {
        for (int k = t; k < ne * ng; k += ts) {
            const int sl = k / ng, g = k - sl * ng;
            const int c0 = g * AVG_GROUP, cn = min(AVG_GROUP, f.nchunks - c0);
            const double* src = f.partial + (size_t)c0 * f.E + e_lo + sl;
            double v[AVG_GROUP];
#pragma unroll
            for (int j = 0; j < AVG_GROUP; ++j) v[j] = j < cn ? __ldcg(src + (size_t)j * f.E) : 0.0;
            s_G[k] = tree16n(v, cn);
        }
    } else {
        // the scalar warp: every chunk's (z_c, q_c) in coalesced loads (each block reads all
        // of them, so scattered per-lane loads would queue on their few L2 lines), then
        // the group trees from shared memory
        const int l = t - ts;
        if (l == 0) inf = *f.info;
        for (int i = l; i < 2 * f.nchunks; i += 32) s_zq[i] = __ldcg(f.zq + i);
        __syncwarp();
        if (l < 2 * ng) {
            const int which = l / ng, g = l - which * ng;
            const int c0 = g * AVG_GROUP, cn = min(AVG_GROUP, f.nchunks - c0);
            double v[AVG_GROUP];
#pragma unroll
            for (int j = 0; j < AVG_GROUP; ++j) v[j] = j < cn ? s_zq[2 * (c0 + j) + which] : 0.0;
            s_zg[which * 16 + g] = tree16n(v, cn);
        }
    }
    __syncthreads();
    double z = 0.0, q = 0.0;
    if (t == ts) {
        double vz[16], vq[16];
#pragma unroll
        for (int g = 0; g < 16; ++g) {
            vz[g] = g < ng ? s_zg[g] : 0.0;
            vq[g] = g < ng ? s_zg[16 + g] : 0.0;
        }
        z = tree16n(vz, ng);
        q = tree16n(vq, ng);
        const bool ok = inf.status == MPPI_OK;
        const bool upd = ok && inf.smin < prev;   // S_min is the best sample's cost (ties -> lowest index)
        s_inv_z = 1.0 / z;
        s_ok = ok;
        s_upd = upd;
        s_best = inf.best;
        s_best_final = upd ? inf.best : prev_index;
    }
    __syncthreads();
    if (t < ne) {
        const int e = e_lo + t;
        double v[16];
#pragma unroll
        for (int g = 0; g < 16; ++g) v[g] = g < ng ? s_G[t * ng + g] : 0.0;
        const double tot = tree16n(v, ng);
        const bool ok = s_ok;
        const bool upd = s_upd && MPPI_CHECK_OK(s_best >= 0 && s_best < N, CHECK_BEST);
        const bool keep_best = last && f.warm_from == MPPI_WARM_BEST && s_best_final >= 0;
        const float m = ok ? (float)(tot * s_inv_z) : f.nominal[e];
        float bv = 0.f;
        if (upd) {
            bv = f.knots[(size_t)s_best * f.E + e];
            f.best_out[e] = bv;
        } else if (keep_best) {
            bv = f.best_out[e];
        }
        if (last) f.mean_out[e] = m;
        f.nominal[e] = keep_best ? bv : m;
    }
    if (c == 0 && t == ts) {
        const bool ok = inf.status == MPPI_OK;
        const bool upd = ok && inf.smin < prev;
        const double best_cost = upd ? inf.smin : prev;
        const int best_index = upd ? inf.best : prev_index;
        const int best_iter = upd ? f.iter : prev_iter;
        const int status = ok ? prev_status : inf.status;
        if (upd) {
            f.solve->best_cost = best_cost;
            f.solve->best_index = best_index;
            f.solve->best_iter = best_iter;
        }
        if (!ok) f.solve->status = status;
        const double lse = ok ? log(z) : NAN;
        const double ess = ok ? z * z / q : 0.0;
        f.info->lse = lse;
        f.info->ess = ess;
        if (last) {
            mppi_result r;
            r.cost_min = inf.smin;
            r.cost_max = inf.smax;
            r.best_cost = best_cost;
            r.ess = ess;
            r.lse = lse;
            r.best_index = best_index;
            r.best_iter = best_iter;
            r.n_finite = inf.nfinite;
            r.status = status;
            *f.result = r;
            f.solve->iter_counter = ctr + (uint32_t)f.iters;
        }
    }
}

// Sum over chunks of the standalone average's partials (increasing chunk order).
__device__ __forceinline__ double chunk_total(const double* __restrict__ partial, int nchunks, int E, int e) {
    double acc = 0.0;
    for (int c = 0; c < nchunks; ++c) acc += partial[(size_t)c * E + e];
    return acc;
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

}  // namespace mppi

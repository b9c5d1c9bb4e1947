// Per-iteration kernels around the rollout: knot noise (Alg. 1 sampling + Eq. vel-clamp),
// chunked weights with FP64 partial knot sums and group totals (Eqs. omega-weights /
// softmax_minmax, Eq. update-nominal) and the iteration's finalize (log-sum-exp, mean,
// best tracking of Sec. III-D).
#pragma once
#include <utility>

#include "internal.h"
#include "noise.cuh"
#include "reduce.cuh"

namespace mppi {

// ------------------------------------------------------------------------------------
// K1: knot noise, NOISE_SPB samples per block (block_sample_knots: one Philox block of 4
// words -> 2 Box-Muller pairs per thread into shared memory, then theta = nominal +
// sigma_k * scale * eps per (knot, joint), clamped, consecutive joints on consecutive
// threads).
// ------------------------------------------------------------------------------------
constexpr int SAMPLE_THREADS = 256;

__global__ void __launch_bounds__(SAMPLE_THREADS) sample_knots_kernel(SampleArgs a) {
    extern __shared__ float eps[];  // [NOISE_SPB][E]
    pdl_trigger();  // the solve's rollout may launch now; it waits for these knots
    pdl_wait();     // the nominal from the previous iteration's finalize
    NoiseParams p;
    p.nominal = a.nominal;
    p.sigma_row = a.sigma_row;
    p.model = a.model;
    p.knots = a.knots;
    p.it = (a.solve ? a.solve->iter_counter : a.iter_counter_override) + a.iter_offset;
    p.inst = a.inst;
    p.seed_lo = a.seed_lo;
    p.seed_hi = a.seed_hi;
    p.N = a.N;
    p.nk = a.nk;
    p.nj = a.nj;
    p.has_limits = a.has_limits;
    p.scale_q = a.scale_q;
    p.scale_v = a.scale_v;
    p.dtk = a.dtk;
    p.spline = a.spline;
    block_sample_knots(p, blockIdx.x * NOISE_SPB, NOISE_SPB, eps);
}

// The same knots without the shared-memory stage and its barrier, for joint counts that
// are multiples of 4 under the Hermite parameterisation (the x, y, y quadruped's 12):
// thread (n, k, m) draws the two Philox blocks that hold knot k's positions and
// velocities of joints 4m .. 4m + 3 (each block's 4 words start on a knot's position or
// velocity half, since 2 k nj and nj are multiples of 4), and writes both halves clamped,
// 16 bytes each. Same counters, Box-Muller pairs and arithmetic as block_sample_knots,
// so the knots are identical bit for bit to the batched path's.
__global__ void __launch_bounds__(SAMPLE_THREADS) sample_knots_j4_kernel(SampleArgs a) {
    pdl_trigger();  // the solve's rollout may launch now; it waits for these knots
    pdl_wait();     // the nominal from the previous iteration's finalize
    const int nj = a.nj, nk = a.nk, E = nk * 2 * nj, G = nj / 4;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)a.N * nk * G) return;
    const int n = (int)(t / (nk * G));
    const int r = (int)(t - (long)n * nk * G);
    const int k = r / G, m = r - k * G;
    const uint32_t it = (a.solve ? a.solve->iter_counter : a.iter_counter_override) + a.iter_offset;
    const int eq = 2 * k * nj + 4 * m, ev = eq + nj;
    if (!MPPI_CHECK_OK(ev + 3 < E, CHECK_NOISE)) return;
    float e_q[4] = {0.f, 0.f, 0.f, 0.f}, e_v[4] = {0.f, 0.f, 0.f, 0.f};
    if (n > 0) {
        const U4 wq = philox4x32_10(U4{(uint32_t)(eq / 4), (uint32_t)n, it, a.inst}, a.seed_lo, a.seed_hi);
        const U4 wv = philox4x32_10(U4{(uint32_t)(ev / 4), (uint32_t)n, it, a.inst}, a.seed_lo, a.seed_hi);
        box_muller<float>(wq.x, wq.y, &e_q[0], &e_q[1]);
        box_muller<float>(wq.z, wq.w, &e_q[2], &e_q[3]);
        box_muller<float>(wv.x, wv.y, &e_v[0], &e_v[1]);
        box_muller<float>(wv.z, wv.w, &e_v[2], &e_v[3]);
    }
    const float sg = a.sigma_row[k];
    const float sq = __fmul_rn(sg, a.scale_q), sv = __fmul_rn(sg, a.scale_v);
    float q[4], v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        q[i] = __fmaf_rn(sq, e_q[i], a.nominal[eq + i]);
        v[i] = __fmaf_rn(sv, e_v[i], a.nominal[ev + i]);
        if (a.has_limits) {
            const int j = 4 * m + i;
            const float lo = a.model->q_min[j + 1], hi = a.model->q_max[j + 1];
            if (isfinite(lo) || isfinite(hi)) {
                q[i] = fminf(fmaxf(q[i], lo), hi);
                const float room = fminf(hi - q[i], q[i] - lo);
                const float vmax = room / (a.dtk * 0.5f);
                v[i] = fminf(fmaxf(v[i], -vmax), vmax);
            }
        }
    }
    float* kn = a.knots + (size_t)n * E;
    *reinterpret_cast<float4*>(kn + eq) = make_float4(q[0], q[1], q[2], q[3]);
    *reinterpret_cast<float4*>(kn + ev) = make_float4(v[0], v[1], v[2], v[3]);
}

// The same knots for any joint count when the model has no joint limits (nothing couples a
// knot's velocity to its clamped position): thread (n, b) draws Philox block b of sample n
// and writes its 4 values, each with its own knot's sigma and its own position or velocity
// scale; again the counters, pairs and arithmetic of block_sample_knots.
__global__ void __launch_bounds__(SAMPLE_THREADS) sample_knots_flat_kernel(SampleArgs a) {
    pdl_trigger();  // the solve's rollout may launch now; it waits for these knots
    pdl_wait();     // the nominal from the previous iteration's finalize
    const int nj = a.nj, E = a.nk * 2 * nj, B4 = (E + 3) / 4;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)a.N * B4) return;
    const int n = (int)(t / B4), b = (int)(t - (long)n * B4);
    const uint32_t it = (a.solve ? a.solve->iter_counter : a.iter_counter_override) + a.iter_offset;
    float e4[4] = {0.f, 0.f, 0.f, 0.f};
    if (n > 0) {
        const U4 w = philox4x32_10(U4{(uint32_t)b, (uint32_t)n, it, a.inst}, a.seed_lo, a.seed_hi);
        box_muller<float>(w.x, w.y, &e4[0], &e4[1]);
        box_muller<float>(w.z, w.w, &e4[2], &e4[3]);
    }
    float v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int e = 4 * b + i;
        const int ec = e < E ? e : E - 1;
        const int k = ec / (2 * nj);
        const bool vel = ec - 2 * nj * k >= nj;
        v[i] = __fmaf_rn(__fmul_rn(a.sigma_row[k], vel ? a.scale_v : a.scale_q), e4[i], a.nominal[ec]);
    }
    float* kn = a.knots + (size_t)n * E;
    if ((E & 3) == 0) {
        *reinterpret_cast<float4*>(kn + 4 * b) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (4 * b + i < E) kn[4 * b + i] = v[i];
    }
}

// One launch through cudaLaunchKernelEx, optionally cooperative and/or as a programmatic
// dependent of the kernel before it in the stream.
template <typename... P, typename... A>
static cudaError_t launch_ex(void (*kernel)(P...), int grid, int block, size_t smem, cudaStream_t s, bool pdl,
                             bool cooperative, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    int n = 0;
    if (cooperative) {
        attr[n].id = cudaLaunchAttributeCooperative;
        attr[n].val.cooperative = 1;
        ++n;
    }
    if (pdl) {
        attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[n].val.programmaticStreamSerializationAllowed = 1;
        ++n;
    }
    cfg.attrs = attr;
    cfg.numAttrs = n;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

cudaError_t launch_sample_knots(const SampleArgs& a, cudaStream_t s, bool pdl) {
    const int E = a.nk * 2 * a.nj;
    if (a.nj % 4 == 0 && a.spline == MPPI_SPLINE_HERMITE && (reinterpret_cast<uintptr_t>(a.knots) & 15) == 0) {
        const long threads = (long)a.N * a.nk * (a.nj / 4);
        if (threads == 0) return cudaSuccess;
        return launch_ex(sample_knots_j4_kernel, (int)((threads + SAMPLE_THREADS - 1) / SAMPLE_THREADS),
                         SAMPLE_THREADS, 0, s, pdl, false, a);
    }
    if (!a.has_limits && a.spline == MPPI_SPLINE_HERMITE && (reinterpret_cast<uintptr_t>(a.knots) & 15) == 0) {
        const long threads = (long)a.N * ((E + 3) / 4);
        if (threads == 0) return cudaSuccess;
        return launch_ex(sample_knots_flat_kernel, (int)((threads + SAMPLE_THREADS - 1) / SAMPLE_THREADS),
                         SAMPLE_THREADS, 0, s, pdl, false, a);
    }
    const int grid = (a.N + NOISE_SPB - 1) / NOISE_SPB;
    if (grid == 0) return cudaSuccess;
    const size_t sm = (size_t)NOISE_SPB * E * sizeof(float);
    return launch_ex(sample_knots_kernel, grid, SAMPLE_THREADS, sm, s, pdl, false, a);
}

// ------------------------------------------------------------------------------------
// K3 (standalone weights entry point): weights and (z_c, q_c) per chunk (grid = chunks).
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(AVG_THREADS) weights_average_kernel(const float* __restrict__ costs,
                                                                      const float* __restrict__ knots, int N, int E,
                                                                      double lambda, int normalize, double* e_out,
                                                                      double* zq, double* partial, DevIterInfo* info) {
    chunk_partial(costs, knots, N, E, lambda, normalize, blockIdx.x, e_out, zq, partial, info);
}

cudaError_t launch_weights_average(const float* costs, const float* knots, int N, int E, double lambda, int normalize,
                                   double* e_out, double* zq, double* partial, DevIterInfo* info, cudaStream_t s) {
    const int grid = num_chunks(N);
    if (grid == 0) return cudaSuccess;
    weights_average_kernel<<<grid, AVG_THREADS, 0, s>>>(costs, knots, N, E, lambda, normalize, e_out, zq, partial, info);
    return cudaGetLastError();
}

__global__ void normalize_weights_kernel(const double* __restrict__ e, const double* __restrict__ zq, int N,
                                         double* __restrict__ w, DevIterInfo* info) {
    __shared__ double s_z;
    double zt = 0.0, qt = 0.0;
    block_total_zq(zq, num_chunks(N), &zt, &qt);
    if (threadIdx.x == 0) {
        const double z = zt, q = qt;
        s_z = z;
        const bool ok = info->status == MPPI_OK;
        info->lse = ok ? log(z) : NAN;
        info->ess = ok ? z * z / q : 0.0;
    }
    __syncthreads();
    const double z = s_z;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x)
        w[n] = z > 0.0 ? e[n] / z : 0.0;
}

cudaError_t launch_normalize_weights(const double* e, const double* zq, int N, double* w, DevIterInfo* info,
                                     cudaStream_t s) {
    normalize_weights_kernel<<<1, 256, 0, s>>>(e, zq, N, w, info);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// K4 (standalone): FP64 average with given weights, in two deterministic stages:
// per-chunk partial sums over 64 samples, then chunk totals in increasing order.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(AVG_THREADS) average_partial_kernel(const float* __restrict__ knots,
                                                                      const double* __restrict__ w, int N, int E,
                                                                      double* __restrict__ partial) {
    const int c = blockIdx.x;
    const int e = blockIdx.y * AVG_THREADS + threadIdx.x;
    if (e >= E) return;
    const int n0 = c * AVG_CHUNK, n1 = min(N, n0 + AVG_CHUNK);
    double acc = 0.0;
    for (int n = n0; n < n1; ++n) acc = fma(w[n], (double)knots[(size_t)n * E + e], acc);
    partial[(size_t)c * E + e] = acc;
}

cudaError_t launch_average_partial(const float* knots, const double* w, int N, int E, double* partial,
                                   cudaStream_t s) {
    const dim3 grid(num_chunks(N), (E + AVG_THREADS - 1) / AVG_THREADS);
    if (grid.x == 0) return cudaSuccess;
    average_partial_kernel<<<grid, AVG_THREADS, 0, s>>>(knots, w, N, E, partial);
    return cudaGetLastError();
}

__global__ void average_reduce_kernel(const double* __restrict__ partial, int nchunks, int E, double* out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x)
        out[e] = chunk_total(partial, nchunks, E, e);
}

cudaError_t launch_average_reduce(const double* partial, int nchunks, int E, double* out, cudaStream_t s) {
    average_reduce_kernel<<<(E + 255) / 256, 256, 0, s>>>(partial, nchunks, E, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Iteration bookkeeping.
// ------------------------------------------------------------------------------------
// Weights, chunk partial sums, group totals and the iteration's finalize in one launch per
// iteration: one block per chunk; the last chunk of each group sums the group, the last
// group runs the finalize (reduce_chunk). 1024 threads: a chunk's 8 x 128 first-tile
// (sub-sum, element) tasks take one thread each, and the FP64 work of a chunk is spread
// over all four schedulers of its SM.
constexpr int WF_THREADS = 1024;

__global__ void __launch_bounds__(WF_THREADS) weights_finalize_kernel(FinalizeArgs f, int N, double lambda,
                                                                       int normalize) {
    pdl_wait();  // the rollout's costs
    reduce_chunk(f, N, lambda, normalize, blockIdx.x);
}

// The single-level finish (reduce_chunk_grid) in a cooperative launch, one chunk per block.
__global__ void __launch_bounds__(WF_THREADS) weights_grid_kernel(FinalizeArgs f, int N, double lambda,
                                                                   int normalize) {
    pdl_wait();  // the rollout's costs
    reduce_chunk_grid(f, N, lambda, normalize);
}

// Blocks of weights_grid_kernel that can be resident at once on each device (0 where
// cooperative launches are not supported); filled by prepare_weights_kernels.
static int g_grid_capacity[64] = {0};

cudaError_t prepare_weights_kernels() {
    int dev = 0, coop = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, weights_grid_kernel, WF_THREADS, 0);
    if (e == cudaSuccess && dev >= 0 && dev < 64) g_grid_capacity[dev] = coop ? per_sm * sms : 0;
    return e;
}

// One launch per iteration. When all chunks fit on the device at once (and in at most 16
// groups) the cooperative single-level finish runs, else the two-level one; both give the
// same bits.
cudaError_t launch_weights_finalize(const FinalizeArgs& a, int N, double lambda, int normalize, cudaStream_t s,
                                    bool pdl) {
    const int grid = num_chunks(N);
    if (grid == 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int cap = dev >= 0 && dev < 64 ? g_grid_capacity[dev] : 0;
    if (grid <= cap && grid <= 16 * AVG_GROUP)
        return launch_ex(weights_grid_kernel, grid, WF_THREADS, 0, s, pdl, true, a, N, lambda, normalize);
    return launch_ex(weights_finalize_kernel, grid, WF_THREADS, 0, s, pdl, false, a, N, lambda, normalize);
}

// Start of a solve: best tracking reset, the best knots start as the nominal, and the
// reduction's counters are cleared (they are zero after every completed iteration; a
// launch that gave up part-way could have left them set).
__global__ void solve_begin_kernel(DevSolve* solve, uint32_t* gcount, int ngroups, const float* nominal,
                                   float* best_out, int E) {
    if (threadIdx.x == 0) {
        solve->best_cost = INFINITY;
        solve->best_index = -1;
        solve->best_iter = -1;
        solve->status = MPPI_OK;
        solve->blocks_done = 0;
    }
    for (int g = threadIdx.x; g < ngroups; g += blockDim.x) gcount[g] = 0;
    for (int e = threadIdx.x; e < E; e += blockDim.x) best_out[e] = nominal[e];
}

cudaError_t launch_solve_begin(DevSolve* solve, uint32_t* gcount, int ngroups, const float* nominal, float* best_out,
                               int E, cudaStream_t s) {
    solve_begin_kernel<<<1, 256, 0, s>>>(solve, gcount, ngroups, nominal, best_out, E);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Shift of the warm start (Sec. III-E). The knots define a spline over the horizon
// T = H dt with knot j at t_j = j T / (nk - 1). Shifting the action sequence by `steps`
// control steps makes the new knot j the old spline's value and time derivative at
// t_j + steps dt; beyond T the spline's end point (the last knot) is repeated. In the
// rollout's integer time units r = t (nk - 1) / dt the read time is
// r_j = min(j H + steps (nk - 1), H (nk - 1)), its segment k = min(floor(r_j / H), nk - 2)
// and s = (r_j - k H) / H. Evaluated in FP64 from the FP32 knots, rounded once.
// One block; in place through shared memory.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) shift_knots_kernel(float* knots, int nj, int nk, int H, int steps, double dtk) {
    __shared__ float old[MAXK * 2 * (MAXB - 1)];
    const int E = nk * 2 * nj;
    for (int e = threadIdx.x; e < E; e += blockDim.x) old[e] = knots[e];
    __syncthreads();
    const long long rmax = (long long)H * (nk - 1);
    for (int e = threadIdx.x; e < nk * nj; e += blockDim.x) {
        const int j = e / nj, i = e - (e / nj) * nj;
        long long r = (long long)j * H + (long long)steps * (nk - 1);
        if (r > rmax) r = rmax;
        int k = (int)(r / H);
        if (k > nk - 2) k = nk - 2;
        const double s = (double)(r - (long long)k * H) / (double)H;
        const double p0 = old[(2 * k) * nj + i], m0 = old[(2 * k + 1) * nj + i];
        const double p1 = old[(2 * k + 2) * nj + i], m1 = old[(2 * k + 3) * nj + i];
        const double s2 = s * s, s3 = s2 * s;
        // cubic Hermite basis and its derivative in s (Eq. hermite_segment)
        const double q = (2.0 * s3 - 3.0 * s2 + 1.0) * p0 + (s3 - 2.0 * s2 + s) * dtk * m0 +
                         (3.0 * s2 - 2.0 * s3) * p1 + (s3 - s2) * dtk * m1;
        const double v = ((6.0 * s2 - 6.0 * s) * (p0 - p1)) / dtk + (3.0 * s2 - 4.0 * s + 1.0) * m0 +
                         (3.0 * s2 - 2.0 * s) * m1;
        knots[(2 * j) * nj + i] = (float)q;
        knots[(2 * j + 1) * nj + i] = (float)v;
    }
}

cudaError_t launch_shift_knots(float* knots, int nj, int nk, int H, int steps, double dtk, cudaStream_t s) {
    if (nj < 1 || nk < 2 || nk > MAXK || nj > MAXB - 1 || H < 1 || steps < 0) return cudaErrorInvalidValue;
    shift_knots_kernel<<<1, 256, 0, s>>>(knots, nj, nk, H, steps, dtk);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// The rollout's FP32 sine/cosine (fast_sincos) and tilt arctangent (fast_atan2_pos) on a
// list of arguments, for accuracy checks: out[i] = (sin x, cos x, atan2(y, x)).
// ------------------------------------------------------------------------------------
__global__ void fast_math_kernel(int n, const float* __restrict__ x, const float* __restrict__ y,
                                 float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s, c;
    fast_sincos(x[i], &s, &c);
    out[3 * i] = s;
    out[3 * i + 1] = c;
    out[3 * i + 2] = fast_atan2_pos(y[i], x[i]);
}

cudaError_t launch_fast_math(int n, const float* x, const float* y, float* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    fast_math_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, x, y, out);
    return cudaGetLastError();
}

// The reduction's integer FP32 -> FP64 widening on a list of values (exactness checks).
__global__ void widen_kernel(int n, const float* __restrict__ x, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = widen(x[i]);
}

cudaError_t launch_widen(int n, const float* x, double* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    widen_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, x, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Philox words for a list of counters (bit-exactness checks).
// ------------------------------------------------------------------------------------
__global__ void philox_words_kernel(int n, const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1,
                                    uint32_t* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const U4 w = philox4x32_10(U4{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]}, k0, k1);
    out[4 * i] = w.x;
    out[4 * i + 1] = w.y;
    out[4 * i + 2] = w.z;
    out[4 * i + 3] = w.w;
}

cudaError_t launch_philox_words(int n, const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    philox_words_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, ctr, k0, k1, out);
    return cudaGetLastError();
}

}  // namespace mppi

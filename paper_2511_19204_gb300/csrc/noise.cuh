// Knot noise (Alg. 1 sampling step with the per-knot standard deviations of
// Eq. overall-noise-kernel, then the clamp of Eq. vel-clamp) as a block-cooperative
// device function, shared by the noise kernel and the persistent batched kernel so both
// write identical knots. Counter = (e / 4, n, iteration counter, instance),
// key = (seed lo, seed hi); sample 0 is the unperturbed nominal.
#pragma once
#include "internal.h"

namespace mppi {

constexpr int NOISE_SPB = 8;  // samples per shared-memory tile

struct NoiseParams {
    const float* nominal;    // [E]
    const float* sigma_row;  // [nk]
    const DevModel<float>* model;  // q_min / q_max (may point to shared memory)
    float* knots;            // [N][E]
    uint32_t it, inst, seed_lo, seed_hi;
    int N, nk, nj, has_limits;
    float scale_q, scale_v, dtk;
};

// Samples [n0, n0 + cnt) (cnt <= NOISE_SPB) by the whole block; eps: shared [NOISE_SPB][E].
__device__ __noinline__ void block_sample_knots(const NoiseParams& a, int n0, int cnt, float* eps) {
    const int E = a.nk * 2 * a.nj;
    const int B4 = (E + 3) / 4;
    for (int idx = threadIdx.x; idx < cnt * B4; idx += blockDim.x) {
        const int nl = idx / B4, b = idx - nl * B4;
        const int n = n0 + nl;
        if (n >= a.N) continue;
        float e4[4] = {0.f, 0.f, 0.f, 0.f};
        if (n > 0) {
            const U4 w = philox4x32_10(U4{(uint32_t)b, (uint32_t)n, a.it, a.inst}, a.seed_lo, a.seed_hi);
            box_muller<float>(w.x, w.y, &e4[0], &e4[1]);
            box_muller<float>(w.z, w.w, &e4[2], &e4[3]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (4 * b + i < E) eps[nl * E + 4 * b + i] = e4[i];
    }
    __syncthreads();
    const int KJ = a.nk * a.nj;
    for (int idx = threadIdx.x; idx < cnt * KJ; idx += blockDim.x) {
        const int nl = idx / KJ, rem = idx - nl * KJ;
        const int n = n0 + nl;
        if (n >= a.N) continue;
        const int k = rem / a.nj, j = rem - k * a.nj;
        const int eq = (2 * k) * a.nj + j, ev = eq + a.nj;
        const float sg = a.sigma_row[k];
        float q = __fmaf_rn(__fmul_rn(sg, a.scale_q), eps[nl * E + eq], a.nominal[eq]);
        float v = __fmaf_rn(__fmul_rn(sg, a.scale_v), eps[nl * E + ev], a.nominal[ev]);
        if (a.has_limits) {
            const float lo = a.model->q_min[j + 1], hi = a.model->q_max[j + 1];
            if (isfinite(lo) || isfinite(hi)) {
                q = fminf(fmaxf(q, lo), hi);
                const float room = fminf(hi - q, q - lo);
                const float vmax = room / (a.dtk * 0.5f);
                v = fminf(fmaxf(v, -vmax), vmax);
            }
        }
        a.knots[(size_t)n * E + eq] = q;
        a.knots[(size_t)n * E + ev] = v;
    }
    __syncthreads();
}

}  // namespace mppi

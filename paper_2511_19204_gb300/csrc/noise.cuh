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
    int spline = 0;          // MPPI_SPLINE_*
};

// Node derivatives of the position-only spline variants of the ablation (Sec. IV-D):
// MPPI_SPLINE_CUBIC, the natural cubic spline through the nodes (second derivative zero
// at both ends); MPPI_SPLINE_QUADRATIC, the C1 piecewise-quadratic spline through the
// nodes starting from rest (d_0 = 0, d_{k+1} = 2 (q_{k+1} - q_k) / h - d_k). Each segment
// of either spline is a polynomial of degree <= 3 fixed by its end values and end slopes,
// so it is exactly the cubic Hermite segment (Eq. hermite_segment) with these node
// slopes: the rollout evaluates every variant unchanged. q, d: nk values with stride st.
__device__ __forceinline__ void spline_slopes(int spline, int nk, float h, const float* q, int st, float* d) {
    if (spline == MPPI_SPLINE_QUADRATIC) {
        float dk = 0.f;
        d[0] = 0.f;
        for (int k = 0; k + 1 < nk; ++k) {
            dk = 2.f * (q[(k + 1) * st] - q[k * st]) / h - dk;
            d[(k + 1) * st] = dk;
        }
        return;
    }
    // natural cubic: M_{k-1} + 4 M_k + M_{k+1} = 6 (q_{k+1} - 2 q_k + q_{k-1}) / h^2 for
    // k = 1..nk-2, M_0 = M_{nk-1} = 0, by the Thomas algorithm
    float cp[MAXK], rp[MAXK], M[MAXK];
    const float s6 = 6.f / (h * h);
    M[0] = 0.f;
    M[nk - 1] = 0.f;
    for (int k = 1; k + 1 < nk; ++k) {
        const float r = s6 * (q[(k + 1) * st] - 2.f * q[k * st] + q[(k - 1) * st]);
        const float den = (k == 1) ? 4.f : 4.f - cp[k - 1];
        cp[k] = 1.f / den;
        rp[k] = (k == 1) ? r / den : (r - rp[k - 1]) / den;
    }
    for (int k = nk - 2; k >= 1; --k) M[k] = (k == nk - 2) ? rp[k] : rp[k] - cp[k] * M[k + 1];
    for (int k = 0; k + 1 < nk; ++k)
        d[k * st] = (q[(k + 1) * st] - q[k * st]) / h - h * (2.f * M[k] + M[k + 1]) / 6.f;
    d[(nk - 1) * st] = (q[(nk - 1) * st] - q[(nk - 2) * st]) / h + h * (M[nk - 2] + 2.f * M[nk - 1]) / 6.f;
}

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
        if (!MPPI_CHECK_OK(nl < NOISE_SPB && ev < E, CHECK_NOISE)) continue;
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
    if (a.spline != MPPI_SPLINE_HERMITE) {
        // position-only variants: the velocity knots become the spline's node slopes
        for (int idx = threadIdx.x; idx < cnt * a.nj; idx += blockDim.x) {
            const int nl = idx / a.nj, j = idx - nl * a.nj;
            const int n = n0 + nl;
            if (n >= a.N) continue;
            float* kn = a.knots + (size_t)n * E;
            spline_slopes(a.spline, a.nk, a.dtk, kn + j, 2 * a.nj, kn + a.nj + j);
        }
        __syncthreads();
    }
}

}  // namespace mppi

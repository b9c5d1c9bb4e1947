// Host implementation of the C ABI declared in include/mppi.h: model upload, contexts
// with their device buffers, the CUDA-graph-captured solve (one graph launch per MPPI
// update: solve_begin + iters x [noise, rollout, chunk weights + partial sums, finalize]),
// and the kernel-level entry points.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "capi_internal.h"
#include "nvtx.h"

namespace mppi {

static thread_local std::string g_last_error;

void set_error(mppi_ctx* ctx, const std::string& msg) {
    g_last_error = msg;
    if (ctx) ctx->last_error = msg;
}

mppi_status cuda_fail(mppi_ctx* ctx, cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
    set_error(ctx, buf);
    if (e == cudaErrorMemoryAllocation) return MPPI_ERR_OUT_OF_MEMORY;
    return MPPI_ERR_CUDA;
}

#define CK(ctx, call)                                            \
    do {                                                         \
        cudaError_t e__ = (call);                                \
        if (e__ != cudaSuccess) return cuda_fail(ctx, e__, #call); \
    } while (0)

// ------------------------------------------------------------------------------------
// Models
// ------------------------------------------------------------------------------------
// Tree shapes with a lanes-per-chain kernel, and their lane plans. Bodies must be
// numbered chain by chain: a chain is a run of bodies each the child of the previous.
struct LanePlan {
    int topology = TOPO_GENERIC;
    int b0[4] = {0, 0, 0, 0}, len[4] = {0, 0, 0, 0};
    int branch = 0;
    int axis_plan = AXP_GENERIC;
};

static bool axis_is(const mppi_model_desc& d, int b, int k) {
    for (int i = 0; i < 3; ++i)
        if (d.axis[3 * b + i] != (i == k ? 1.0 : 0.0)) return false;
    return true;
}

// the joint offset of body b lies on coordinate axis k (its other components are zero)
static bool offset_along(const mppi_model_desc& d, int b, int k) {
    for (int i = 0; i < 3; ++i)
        if (i != k && d.jpos[3 * b + i] != 0.0) return false;
    return true;
}

// every contact point sits on one of the bodies leaf[0..n)
static bool contacts_on(const mppi_model_desc& d, const int* leaf, int n) {
    for (int i = 0; i < d.nc; ++i) {
        bool on = false;
        for (int k = 0; k < n; ++k) on = on || d.contact_body[i] == leaf[k];
        if (!on) return false;
    }
    return true;
}

static bool offset_zero(const mppi_model_desc& d, int b) {
    return d.jpos[3 * b] == 0.0 && d.jpos[3 * b + 1] == 0.0 && d.jpos[3 * b + 2] == 0.0;
}

static bool is_chain(const mppi_model_desc& d, int first, int len, int parent) {
    if (len < 1 || first + len > d.nb || d.parent[first] != parent) return false;
    for (int j = 1; j < len; ++j)
        if (d.parent[first + j] != first + j - 1) return false;
    return true;
}

static LanePlan detect_topology(const mppi_model_desc& d) {
    LanePlan P;
    if (d.fixed_base) return P;
    // base + 4 chains of L <= 3
    if ((d.nb - 1) % 4 == 0) {
        const int L = (d.nb - 1) / 4;
        bool ok = L >= 1 && L <= 3;
        for (int l = 0; l < 4 && ok; ++l) ok = is_chain(d, 1 + l * L, L, 0);
        if (ok) {
            P.topology = TOPO_QUADRUPED;
            bool xyy = L == 3;
            for (int l = 0; l < 4; ++l) {
                P.b0[l] = 1 + l * L;
                P.len[l] = L;
                if (xyy)
                    xyy = axis_is(d, P.b0[l], 0) && axis_is(d, P.b0[l] + 1, 1) && axis_is(d, P.b0[l] + 2, 1) &&
                          d.jpos[3 * P.b0[l] + 2] == 0.0 && offset_along(d, P.b0[l] + 1, 1) &&
                          offset_along(d, P.b0[l] + 2, 2);
            }
            const int calves[4] = {P.b0[0] + 2, P.b0[1] + 2, P.b0[2] + 2, P.b0[3] + 2};
            if (xyy && contacts_on(d, calves, 4)) P.axis_plan = AXP_XYY;
            return P;
        }
    }
    // base + 2 chains of A <= 6, a branch body on the base, 2 chains of C <= 6 on it
    for (int A = 1; A <= 6; ++A) {
        const int rest = d.nb - 1 - 2 * A - 1;
        if (rest < 2 || rest % 2) continue;
        const int C = rest / 2, br = 1 + 2 * A;
        if (C > 6) continue;
        if (is_chain(d, 1, A, 0) && is_chain(d, 1 + A, A, 0) && d.parent[br] == 0 && is_chain(d, br + 1, C, br) &&
            is_chain(d, br + 1 + C, C, br)) {
            P.topology = TOPO_HUMANOID;
            P.b0[0] = 1;
            P.len[0] = A;
            P.b0[1] = 1 + A;
            P.len[1] = A;
            P.b0[2] = br + 1;
            P.len[2] = C;
            P.b0[3] = br + 1 + C;
            P.len[3] = C;
            P.branch = br;
            // the usual humanoid layout (AXP_HUM): legs z, x, y, y, y, x with offsets in the
            // yz-plane, on z, zero, on z, on z, zero; waist z on z; arms y, x, z, y with
            // offsets in the yz-plane, on y, zero, on z
            bool hum = A == 6 && C == 4 && axis_is(d, br, 2) && offset_along(d, br, 2);
            for (int l = 0; l < 2 && hum; ++l) {
                const int b = P.b0[l];
                hum = axis_is(d, b, 2) && axis_is(d, b + 1, 0) && axis_is(d, b + 2, 1) && axis_is(d, b + 3, 1) &&
                      axis_is(d, b + 4, 1) && axis_is(d, b + 5, 0) && d.jpos[3 * b] == 0.0 &&
                      offset_along(d, b + 1, 2) && offset_zero(d, b + 2) && offset_along(d, b + 3, 2) &&
                      offset_along(d, b + 4, 2) && offset_zero(d, b + 5);
            }
            for (int l = 2; l < 4 && hum; ++l) {
                const int b = P.b0[l];
                hum = axis_is(d, b, 1) && axis_is(d, b + 1, 0) && axis_is(d, b + 2, 2) && axis_is(d, b + 3, 1) &&
                      d.jpos[3 * b] == 0.0 && offset_along(d, b + 1, 1) && offset_zero(d, b + 2) &&
                      offset_along(d, b + 3, 2);
            }
            const int feet[2] = {P.b0[0] + 5, P.b0[1] + 5};
            const bool cost_off_legs = d.cost_body < P.b0[0] || d.cost_body >= P.b0[1] + 6;
            if (hum && contacts_on(d, feet, 2) && cost_off_legs) P.axis_plan = AXP_HUM;
            return P;
        }
    }
    return P;
}

template <typename T>
static void fill_model(const mppi_model_desc& d, const std::vector<int>& level, int nlevels,
                       const std::vector<std::vector<int>>& children, const std::vector<int>& corder,
                       const LanePlan& plan, DevModel<T>& M) {
    memset(&M, 0, sizeof(M));
    const int nb = d.nb;
    for (int b = 0; b < nb; ++b) {
        for (int k = 0; k < 3; ++k) {
            M.axis[k][b] = (T)d.axis[3 * b + k];
            M.jpos[k][b] = (T)d.jpos[3 * b + k];
            M.mc[k][b] = (T)(d.mass[b] * d.com[3 * b + k]);
        }
        const double m = d.mass[b];
        const double* c = &d.com[3 * b];
        const double* I = &d.inertia[6 * b];
        M.Ao[0][b] = (T)(I[0] + m * (c[1] * c[1] + c[2] * c[2]));
        M.Ao[1][b] = (T)(I[1] + m * (c[0] * c[0] + c[2] * c[2]));
        M.Ao[2][b] = (T)(I[2] + m * (c[0] * c[0] + c[1] * c[1]));
        M.Ao[3][b] = (T)(I[3] - m * c[0] * c[1]);
        M.Ao[4][b] = (T)(I[4] - m * c[0] * c[2]);
        M.Ao[5][b] = (T)(I[5] - m * c[1] * c[2]);
        M.mass[b] = (T)m;
        M.armature[b] = (T)d.armature[b];
        M.parent[b] = d.parent[b];
        M.level[b] = level[b];
        M.nchild[b] = (int)children[b].size();
        for (size_t k = 0; k < children[b].size(); ++k) M.child[k][b] = children[b][k];
        if (b > 0) {
            M.kp[b] = (T)d.kp[b - 1];
            M.kd[b] = (T)d.kd[b - 1];
            M.tau_max[b] = (T)d.tau_max[b - 1];
            M.q_min[b] = (T)d.q_min[b - 1];
            M.q_max[b] = (T)d.q_max[b - 1];
            M.q_init[b] = d.q_init ? (T)d.q_init[b - 1] : T(0);
        }
    }
    for (int b = 0; b < nb; ++b) M.ccount[b] = 0;
    for (int i = 0; i < d.nc; ++i) {
        const int ci = corder[i];
        for (int k = 0; k < 3; ++k) M.cpos[k][i] = (T)d.contact_pos[3 * ci + k];
        const int b = d.contact_body[ci];
        if (M.ccount[b] == 0) M.cfirst[b] = i;
        M.ccount[b]++;
    }
    M.nb = nb;
    M.nc = d.nc;
    M.nlevels = nlevels;
    M.fixed_base = d.fixed_base ? 1 : 0;
    M.cost_body = d.cost_body;
    int lim = 0;
    for (int j = 0; j < nb - 1; ++j)
        if (isfinite(d.q_min[j]) || isfinite(d.q_max[j])) lim = 1;
    M.has_limits = lim;
    M.topology = plan.topology;
    M.axis_plan = plan.axis_plan;
    for (int l = 0; l < 4; ++l) {
        M.lane_b0[l] = plan.b0[l];
        M.lane_len[l] = plan.len[l];
    }
    M.branch_body = plan.branch;
    M.contact_k = (T)d.contact_k;
    M.contact_c = (T)d.contact_c;
    M.mu = (T)d.mu;
    M.eps_f = (T)d.eps_f;
    M.gravity = (T)d.gravity;
    M.z_des = (T)d.z_des;
    M.vx_des = (T)d.vx_des;
    M.w_z = (T)d.w_z;
    M.w_vx = (T)d.w_vx;
    M.w_tilt = (T)d.w_tilt;
    M.w_tau = (T)d.w_tau;
    M.w_h = (T)d.w_h;
    M.w_orient = (T)d.w_orient;
    M.w_q = (T)d.w_q;
    M.w_cvel = (T)d.w_cvel;
    M.w_cforce = (T)d.w_cforce;
    M.w_term = (T)d.w_term;
    M.cf_off = (T)(d.w_cforce * (fabs(d.f0[0]) + fabs(d.f0[1]) + fabs(d.f0[2])));
    for (int k = 0; k < 3; ++k) {
        M.f0[k] = (T)d.f0[k];
        M.pdot_des[k] = (T)d.pdot_des[k];
    }
    // R_des from the normalised quaternion (all zeros = identity)
    double qw = d.quat_des[0], qx = d.quat_des[1], qy = d.quat_des[2], qz = d.quat_des[3];
    const double qn = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
    if (qn > 0) {
        qw /= qn;
        qx /= qn;
        qy /= qn;
        qz /= qn;
    } else {
        qw = 1;
        qx = qy = qz = 0;
    }
    const double R[9] = {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz),     2 * (qx * qz + qw * qy),
                         2 * (qx * qy + qw * qz),     1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx),
                         2 * (qx * qz - qw * qy),     2 * (qy * qz + qw * qx),     1 - 2 * (qx * qx + qy * qy)};
    for (int k = 0; k < 9; ++k) M.Rdes[k] = (T)R[k];
    M.paper_cost = (d.w_h != 0 || d.w_orient != 0 || d.w_q != 0 || d.w_cvel != 0 || d.w_cforce != 0 ||
                    d.w_term != 0)
                       ? 1
                       : 0;
}

}  // namespace mppi

using namespace mppi;

extern "C" {

const char* mppi_status_str(mppi_status s) {
    switch (s) {
        case MPPI_OK: return "ok";
        case MPPI_PENDING: return "pending";
        case MPPI_ERR_INVALID_ARG: return "invalid argument";
        case MPPI_ERR_NONFINITE_STATE: return "state is not finite";
        case MPPI_ERR_ALL_COSTS_NONFINITE: return "no finite cost in an iteration";
        case MPPI_ERR_OUT_OF_MEMORY: return "out of device memory";
        case MPPI_ERR_ADMISSION: return "request exceeds the memory budget";
        case MPPI_ERR_TIMEOUT: return "device wait timed out";
        case MPPI_ERR_CUDA: return "CUDA error";
        case MPPI_ERR_UNSUPPORTED: return "unsupported";
        case MPPI_ERR_NOT_FOUND: return "unknown ticket";
        case MPPI_ERR_DEADLINE: return "shed: waited past the server's deadline";
        default: return "unknown status";
    }
}

const char* mppi_last_error(const mppi_ctx* ctx) {
    return ctx ? ctx->last_error.c_str() : g_last_error.c_str();
}

mppi_status mppi_model_create(const mppi_model_desc* d, mppi_model** out) {
    MPPI_NVTX("mppi_model_create");
    if (!d || !out) return MPPI_ERR_INVALID_ARG;
    *out = nullptr;
    auto bad = [&](const char* why) {
        set_error(nullptr, why);
        return MPPI_ERR_INVALID_ARG;
    };
    if (d->nb < 1 || d->nb > MAXB) return bad("nb out of range");
    if (d->nc < 0 || d->nc > MAXC) return bad("nc out of range");
    if (!d->parent || !d->axis || !d->jpos || !d->mass || !d->com || !d->inertia || !d->armature)
        return bad("null body array");
    if (d->nb > 1 && (!d->q_min || !d->q_max || !d->kp || !d->kd || !d->tau_max)) return bad("null joint array");
    if (d->nc > 0 && (!d->contact_body || !d->contact_pos)) return bad("null contact array");
    if (d->parent[0] != -1) return bad("parent[0] must be -1");
    if (d->cost_body < 0 || d->cost_body >= d->nb) return bad("cost_body out of range");
    {
        const double w[10] = {d->w_z, d->w_vx, d->w_tilt, d->w_tau, d->w_h, d->w_orient, d->w_q, d->w_cvel,
                              d->w_cforce, d->w_term};
        for (double v : w)
            if (!(v >= 0) || !isfinite(v)) return bad("cost weights must be finite and >= 0");
        for (int k = 0; k < 4; ++k)
            if (!isfinite(d->quat_des[k])) return bad("quat_des must be finite");
        for (int k = 0; k < 3; ++k)
            if (!isfinite(d->f0[k]) || !isfinite(d->pdot_des[k])) return bad("f0 and pdot_des must be finite");
    }
    std::vector<int> level(d->nb, 0);
    std::vector<std::vector<int>> children(d->nb);
    int nlevels = 1;
    for (int i = 1; i < d->nb; ++i) {
        const int p = d->parent[i];
        if (p < 0 || p >= i) return bad("parent[i] must be in [0, i)");
        level[i] = level[p] + 1;
        nlevels = std::max(nlevels, level[i] + 1);
        children[p].push_back(i);
        if ((int)children[p].size() > MAXCH) return bad("too many children on one body");
        const double* a = &d->axis[3 * i];
        const double n = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        if (!(fabs(n - 1.0) < 1e-6)) return bad("joint axis must be a unit vector");
        if (!(d->tau_max[i - 1] >= 0)) return bad("tau_max must be >= 0");
        if (d->q_min[i - 1] > d->q_max[i - 1]) return bad("q_min > q_max");
    }
    for (int b = 0; b < d->nb; ++b) {
        if (!(d->mass[b] > 0) || !isfinite(d->mass[b])) return bad("masses must be positive");
        if (b > 0 && !(d->armature[b] >= 0)) return bad("armature must be >= 0");
    }
    std::vector<int> corder(d->nc);
    for (int i = 0; i < d->nc; ++i) {
        if (d->contact_body[i] < 0 || d->contact_body[i] >= d->nb) return bad("contact_body out of range");
        corder[i] = i;
    }
    std::stable_sort(corder.begin(), corder.end(),
                     [&](int a, int b) { return d->contact_body[a] < d->contact_body[b]; });
    mppi_model* m = new (std::nothrow) mppi_model();
    if (!m) return MPPI_ERR_OUT_OF_MEMORY;
    m->nb = d->nb;
    m->nj = d->nb - 1;
    m->nc = d->nc;
    m->fixed_base = d->fixed_base != 0;
    const LanePlan plan = detect_topology(*d);
    m->topology = plan.topology;
    fill_model(*d, level, nlevels, children, corder, plan, m->host_f);
    fill_model(*d, level, nlevels, children, corder, plan, m->host_d);
    m->q_init.assign(m->nj, 0.f);
    if (d->q_init)
        for (int j = 0; j < m->nj; ++j) m->q_init[j] = (float)d->q_init[j];
    cudaError_t e = cudaGetDevice(&m->device);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_f, sizeof(DevModel<float>));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_d, sizeof(DevModel<double>));
    if (e == cudaSuccess) e = cudaMemcpy(m->d_f, &m->host_f, sizeof(DevModel<float>), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_d, &m->host_d, sizeof(DevModel<double>), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        mppi_status st = cuda_fail(nullptr, e, "model upload");
        mppi_model_destroy(m);
        return st;
    }
    *out = m;
    return MPPI_OK;
}

void mppi_model_destroy(mppi_model* m) {
    if (!m) return;
    if (m->d_f) cudaFree(m->d_f);
    if (m->d_d) cudaFree(m->d_d);
    delete m;
}

}  // extern "C"

namespace mppi {

// ------------------------------------------------------------------------------------
// Context buffers: one device allocation carved into 256-byte aligned pieces.
// ------------------------------------------------------------------------------------
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t ctx_layout(mppi_ctx* c, bool assign) {
    const size_t N = c->N, E = c->E, nx = c->nx;
    size_t off = 0;
    auto take = [&](size_t bytes, void** slot) {
        if (assign) *slot = (char*)c->dev_block + off;
        off += align256(bytes);
    };
    take(sizeof(double) * nx, (void**)&c->d_x0);
    take(sizeof(float) * N * E, (void**)&c->d_knots);
    take(sizeof(float) * N, (void**)&c->d_costs);
    take(sizeof(double) * N, (void**)&c->d_w);
    take(sizeof(double) * num_chunks((int)N) * E, (void**)&c->d_partial);
    take(sizeof(double) * num_chunks((int)N) * 2, (void**)&c->d_zq);
    take(sizeof(double) * num_groups((int)N) * E, (void**)&c->d_gpartial);
    take(sizeof(double) * num_groups((int)N) * 2, (void**)&c->d_gzq);
    take(sizeof(uint32_t) * num_groups((int)N), (void**)&c->d_gcount);
    take(sizeof(float) * E, (void**)&c->d_nominal);
    take(sizeof(float) * E, (void**)&c->d_mean);
    take(sizeof(float) * E, (void**)&c->d_best);
    take(sizeof(float) * c->iters * c->nk, (void**)&c->d_sigma);
    take(sizeof(DevIterInfo), (void**)&c->d_info);
    take(sizeof(DevSolve), (void**)&c->d_solve);
    take(sizeof(mppi_result), (void**)&c->d_result);
    return off;
}

cudaError_t enqueue_rollout(mppi_ctx* c, const double* d_x0, const float* d_knots, int N, float* d_costs,
                            double* d_finals, cudaStream_t s, bool after_noise) {
    RolloutArgs<float> a;
    a.model = (const DevModel<float>*)c->model->d_f;
    a.x0 = d_x0;
    a.knots = d_knots;
    a.costs = d_costs;
    a.finals = d_finals;
    a.status = &c->d_solve->dev_error;
    a.N = N;
    a.H = c->H;
    a.nk = c->nk;
    a.dt = (float)c->dt;
    a.dtk = (float)c->dtk;
    switch (c->mapping) {
        case MPPI_MAP_WARP: return launch_rollout_warp_f32(a, 32, c->block, s);
        case MPPI_MAP_HALFWARP: return launch_rollout_warp_f32(a, 16, c->block, s);
        case MPPI_MAP_CHAIN:
            // no programmatic launch behind the profiling events (they sit between the kernels)
            return launch_rollout_chain_f32(a, c->model->topology, c->model->host_f.paper_cost != 0,
                                            c->model->host_f.axis_plan, c->block, s, after_noise && !c->profile);
        default: return cudaErrorInvalidValue;
    }
}

// One iteration's kernels (noise, rollout, weights, partial average, finalize).
cudaError_t enqueue_iteration(mppi_ctx* c, int it, cudaStream_t s) {
    SampleArgs sa;
    sa.nominal = c->d_nominal;
    sa.sigma_row = c->d_sigma + (size_t)it * c->nk;
    sa.model = (const DevModel<float>*)c->model->d_f;
    sa.knots = c->d_knots;
    sa.solve = c->d_solve;
    sa.iter_offset = (uint32_t)it;
    sa.iter_counter_override = 0;
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
    // the kernels of a solve after its first follow each other as programmatic dependents
    // (not behind the profiling events, which sit between them)
    cudaError_t e = launch_sample_knots(sa, s, it > 0 && !c->profile);
    if (e == cudaSuccess && c->profile) e = cudaEventRecordWithFlags(c->ev[2 * it], s, cudaEventRecordExternal);
    if (e == cudaSuccess) e = enqueue_rollout(c, c->d_x0, c->d_knots, c->N, c->d_costs, nullptr, s, true);
    if (e == cudaSuccess && c->profile) e = cudaEventRecordWithFlags(c->ev[2 * it + 1], s, cudaEventRecordExternal);
    if (e == cudaSuccess) {
        FinalizeArgs f;
        f.partial = c->d_partial;
        f.zq = c->d_zq;
        f.gpartial = c->d_gpartial;
        f.gzq = c->d_gzq;
        f.gcount = c->d_gcount;
        f.nchunks = num_chunks(c->N);
        f.ngroups = num_groups(c->N);
        f.E = c->E;
        f.iter = it;
        f.iters = c->iters;
        f.warm_from = c->warm_from;
        f.knots = c->d_knots;
        f.costs = c->d_costs;
        f.info = c->d_info;
        f.solve = c->d_solve;
        f.nominal = c->d_nominal;
        f.mean_out = c->d_mean;
        f.best_out = c->d_best;
        f.result = c->d_result;
        e = launch_weights_finalize(f, c->N, c->lambda, c->normalize, s, !c->profile);
    }
    return e;
}

cudaError_t enqueue_solve_kernels(mppi_ctx* c, cudaStream_t s) {
    cudaError_t e = launch_solve_begin(c->d_solve, c->d_gcount, num_groups(c->N), c->d_nominal, c->d_best, c->E, s);
    for (int it = 0; it < c->iters && e == cudaSuccess; ++it) e = enqueue_iteration(c, it, s);
    return e;
}

static mppi_status build_graph(mppi_ctx* c) {
    if (c->graph_exec) return MPPI_OK;
    cudaGraph_t g = nullptr;
    CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_solve_kernels(c, c->stream);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, e, "capture solve");
    }
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph_exec = nullptr;
        return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    return MPPI_OK;
}

void invalidate_graph(mppi_ctx* c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
}

mppi_status launch_solve(mppi_ctx* c) {
    mppi_status st = build_graph(c);
    if (st != MPPI_OK) return st;
    CK(c, cudaGraphLaunch(c->graph_exec, c->stream));
    return MPPI_OK;
}

int default_mapping(const mppi_model* m, int N) {
    (void)N;
    if (chain_mapping_supported(m->topology)) return MPPI_MAP_CHAIN;
    return m->nb <= 16 ? MPPI_MAP_HALFWARP : MPPI_MAP_WARP;
}

cudaError_t prepare_kernels() {
    cudaError_t e = prepare_weights_kernels();
    if (e == cudaSuccess) e = prepare_warp_f32();
    if (e == cudaSuccess) e = prepare_warp_f64();
    return e;
}

int default_block(int mapping) { return mapping == MPPI_MAP_WARP || mapping == MPPI_MAP_HALFWARP ? 64 : 128; }

bool mapping_valid(const mppi_model* m, int mapping, int block) {
    switch (mapping) {
        case MPPI_MAP_WARP: return block == 0 || (block % 32 == 0 && block >= 32 && block <= 256);
        case MPPI_MAP_HALFWARP:
            return m->nb <= 16 && (block == 0 || (block % 32 == 0 && block >= 32 && block <= 256));
        case MPPI_MAP_CHAIN:
            if (m->host_f.axis_plan == AXP_HUM)  // warp pairs
                return block == 0 || (block % 64 == 0 && block >= 64 && block <= 256);
            return chain_mapping_supported(m->topology) && (block == 0 || (block % 32 == 0 && block >= 32 && block <= 256));
        case MPPI_MAP_THREAD:   // reserved: no kernel
            return false;
        default: return false;
    }
}

}  // namespace mppi

extern "C" {

mppi_status mppi_create(const mppi_model* model, int32_t K, int32_t H, int32_t knots, double lambda,
                        const float* h_sigma, int32_t iters, const mppi_params* p, mppi_ctx** out) {
    MPPI_NVTX("mppi_create");
    if (!out) return MPPI_ERR_INVALID_ARG;
    *out = nullptr;
    auto bad = [&](const char* why) {
        set_error(nullptr, why);
        return MPPI_ERR_INVALID_ARG;
    };
    if (!model || !p || !h_sigma) return bad("null argument");
    if (model->nj < 1) return bad("the model has no joints to parameterise");
    if (K < 1 || H < 1 || knots < 2 || knots > MAXK || iters < 1) return bad("K, H, knots or iters out of range");
    if (!(lambda > 0) || !isfinite(lambda)) return bad("lambda must be positive");
    if (!(p->dt > 0) || !isfinite(p->dt)) return bad("dt must be positive");
    if (p->normalize != MPPI_NORM_MINMAX && p->normalize != MPPI_NORM_RAW) return bad("normalize");
    if (p->warm_from != MPPI_WARM_BEST && p->warm_from != MPPI_WARM_MEAN) return bad("warm_from");
    if (p->spline != MPPI_SPLINE_HERMITE && p->spline != MPPI_SPLINE_CUBIC && p->spline != MPPI_SPLINE_QUADRATIC)
        return bad("spline");
    if ((int64_t)H * (knots - 1) > 0x7fffffff) return bad("H too large");
    for (int i = 0; i < iters * knots; ++i)
        if (!(h_sigma[i] >= 0) || !isfinite(h_sigma[i])) return bad("sigma must be finite and >= 0");
    int mapping = p->mapping == MPPI_MAP_AUTO ? default_mapping(model, K) : p->mapping;
    if (!mapping_valid(model, mapping, p->block_size)) return bad("unsupported mapping / block size");
    int dev;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    if (dev != model->device) return bad("model lives on another device");
    mppi_ctx* c = new (std::nothrow) mppi_ctx();
    if (!c) return MPPI_ERR_OUT_OF_MEMORY;
    static std::atomic<uint64_t> next_uid{1};
    c->model = model;
    c->uid = next_uid++;
    c->device = dev;
    c->N = K;
    c->H = H;
    c->nk = knots;
    c->iters = iters;
    c->nj = model->nj;
    c->E = knots * 2 * model->nj;
    c->nx = 13 + 2 * model->nj;
    c->lambda = lambda;
    c->dt = p->dt;
    c->dtk = (double)H * p->dt / (double)(knots - 1);
    c->scale_q = p->scale_q;
    c->scale_v = p->scale_v > 0 ? p->scale_v : 1.0 / c->dtk;
    c->normalize = p->normalize;
    c->warm_from = p->warm_from;
    c->spline = p->spline;
    c->seed = p->seed;
    c->instance_id = p->instance_id;
    c->mapping = mapping;
    c->block = p->block_size > 0 ? p->block_size : default_block(mapping);
    c->auto_mapping = p->mapping == MPPI_MAP_AUTO;
    if (p->stream) {
        c->stream = (cudaStream_t)p->stream;
        c->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return cuda_fail(nullptr, e, "cudaStreamCreate");
        }
        c->own_stream = true;
    }
    c->dev_bytes = ctx_layout(c, false);
    e = cudaMalloc(&c->dev_block, c->dev_bytes);
    if (e == cudaSuccess) {
        ctx_layout(c, true);
        e = cudaMallocHost(&c->host_block, sizeof(double) * c->nx + sizeof(float) * 3 * c->E + sizeof(mppi_result) + 64);
    }
    if (e != cudaSuccess) {
        mppi_status st = cuda_fail(nullptr, e, "context allocation");
        mppi_destroy(c);
        return st;
    }
    c->h_x0 = (double*)c->host_block;
    c->h_mean = (float*)(c->h_x0 + c->nx);
    c->h_best = c->h_mean + c->E;
    c->h_warm = c->h_best + c->E;
    c->h_result = (mppi_result*)(((uintptr_t)(c->h_warm + c->E) + 15) & ~(uintptr_t)15);
    std::vector<float> nom(c->E, 0.f);
    for (int k = 0; k < knots; ++k)
        for (int j = 0; j < c->nj; ++j) nom[(size_t)(2 * k) * c->nj + j] = model->q_init[j];
    DevSolve ds;
    memset(&ds, 0, sizeof ds);
    e = cudaMemcpy(c->d_sigma, h_sigma, sizeof(float) * iters * knots, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_nominal, nom.data(), sizeof(float) * c->E, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_solve, &ds, sizeof ds, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->d_gcount, 0, sizeof(uint32_t) * num_groups(c->N));
    if (e == cudaSuccess) e = prepare_kernels();
    if (e != cudaSuccess) {
        mppi_status st = cuda_fail(nullptr, e, "context initialisation");
        mppi_destroy(c);
        return st;
    }
    *out = c;
    return MPPI_OK;
}

void mppi_destroy(mppi_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    invalidate_graph(c);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    if (c->dev_block) cudaFree(c->dev_block);
    if (c->host_block) cudaFreeHost(c->host_block);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

mppi_status mppi_solve(mppi_ctx* c, const double* h_state, const float* h_warm, float* h_out_mean,
                       float* h_out_best, mppi_result* h_info) {
    MPPI_NVTX("mppi_solve");
    if (!c || !h_state || !h_out_mean) return MPPI_ERR_INVALID_ARG;
    for (int i = 0; i < c->nx; ++i)
        if (!isfinite(h_state[i])) {
            set_error(c, "state is not finite");
            return MPPI_ERR_NONFINITE_STATE;
        }
    memcpy(c->h_x0, h_state, sizeof(double) * c->nx);
    CK(c, cudaMemcpyAsync(c->d_x0, c->h_x0, sizeof(double) * c->nx, cudaMemcpyHostToDevice, c->stream));
    c->has_state = true;
    if (h_warm) {
        memcpy(c->h_warm, h_warm, sizeof(float) * c->E);
        CK(c, cudaMemcpyAsync(c->d_nominal, c->h_warm, sizeof(float) * c->E, cudaMemcpyHostToDevice, c->stream));
    }
    mppi_status st = launch_solve(c);
    if (st != MPPI_OK) return st;
    CK(c, cudaMemcpyAsync(c->h_mean, c->d_mean, sizeof(float) * c->E, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(c->h_best, c->d_best, sizeof(float) * c->E, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(c->h_result, c->d_result, sizeof(mppi_result), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    memcpy(h_out_mean, c->h_mean, sizeof(float) * c->E);
    if (h_out_best) memcpy(h_out_best, c->h_best, sizeof(float) * c->E);
    if (h_info) *h_info = *c->h_result;
    return c->h_result->status;
}

mppi_status mppi_solve_device(mppi_ctx* c, const double* d_state, const float* d_warm, float* d_out_mean,
                              float* d_out_best, mppi_result* d_info) {
    MPPI_NVTX("mppi_solve_device");
    if (!c || !d_state || !d_out_mean) return MPPI_ERR_INVALID_ARG;
    CK(c, cudaMemcpyAsync(c->d_x0, d_state, sizeof(double) * c->nx, cudaMemcpyDeviceToDevice, c->stream));
    c->has_state = true;
    if (d_warm)
        CK(c, cudaMemcpyAsync(c->d_nominal, d_warm, sizeof(float) * c->E, cudaMemcpyDeviceToDevice, c->stream));
    mppi_status st = launch_solve(c);
    if (st != MPPI_OK) return st;
    CK(c, cudaMemcpyAsync(d_out_mean, c->d_mean, sizeof(float) * c->E, cudaMemcpyDeviceToDevice, c->stream));
    if (d_out_best)
        CK(c, cudaMemcpyAsync(d_out_best, c->d_best, sizeof(float) * c->E, cudaMemcpyDeviceToDevice, c->stream));
    if (d_info)
        CK(c, cudaMemcpyAsync(d_info, c->d_result, sizeof(mppi_result), cudaMemcpyDeviceToDevice, c->stream));
    return MPPI_OK;
}

mppi_status mppi_sync(mppi_ctx* c) {
    if (!c) return MPPI_ERR_INVALID_ARG;
    CK(c, cudaStreamSynchronize(c->stream));
    uint32_t err = 0;
    CK(c, cudaMemcpy(&err, &c->d_solve->dev_error, sizeof err, cudaMemcpyDeviceToHost));
    if (err) {
        set_error(c, "a bounded device wait gave up");
        return MPPI_ERR_TIMEOUT;
    }
    return MPPI_OK;
}

mppi_status mppi_rollout_explicit(mppi_ctx* c, const double* h_state, const float* h_knots, double* h_costs,
                                  double* h_finals) {
    MPPI_NVTX("mppi_rollout_explicit");
    if (!c || !h_state || !h_knots || !h_costs) return MPPI_ERR_INVALID_ARG;
    const int N = c->N, E = c->E, nx = c->nx;
    double* d_x = nullptr;
    float* d_k = nullptr;
    void* d_c = nullptr;
    double* d_f = nullptr;
    uint32_t* d_err = nullptr;
    const size_t csz = c->fp64_check ? sizeof(double) : sizeof(float);
    cudaError_t e = cudaMalloc(&d_x, sizeof(double) * nx);
    if (e == cudaSuccess) e = cudaMalloc(&d_k, sizeof(float) * (size_t)N * E);
    if (e == cudaSuccess) e = cudaMalloc(&d_c, csz * N);
    if (e == cudaSuccess && h_finals) e = cudaMalloc(&d_f, sizeof(double) * (size_t)N * nx);
    if (e == cudaSuccess) e = cudaMalloc(&d_err, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(uint32_t), c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_x, h_state, sizeof(double) * nx, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_k, h_knots, sizeof(float) * (size_t)N * E, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        if (c->fp64_check) {
            RolloutArgs<double> a;
            a.model = (const DevModel<double>*)c->model->d_d;
            a.x0 = d_x;
            a.knots = d_k;
            a.costs = (double*)d_c;
            a.finals = d_f;
            a.status = d_err;
            a.N = N;
            a.H = c->H;
            a.nk = c->nk;
            a.dt = c->dt;
            a.dtk = c->dtk;
            if (c->mapping == MPPI_MAP_CHAIN)  // the product's chain kernels, in double
                e = launch_rollout_chain_f64(a, c->model->topology, c->model->host_f.paper_cost != 0,
                                             c->model->host_f.axis_plan, c->stream);
            else
                e = launch_rollout_warp_f64(a, c->mapping == MPPI_MAP_HALFWARP ? 16 : 32,
                                            c->mapping == MPPI_MAP_WARP || c->mapping == MPPI_MAP_HALFWARP ? c->block
                                                                                                          : 64,
                                            c->stream);
        } else {
            RolloutArgs<float> a;
            e = enqueue_rollout(c, d_x, d_k, N, (float*)d_c, d_f, c->stream);
            (void)a;
        }
    }
    std::vector<float> cf;
    if (e == cudaSuccess) {
        if (c->fp64_check) {
            e = cudaMemcpyAsync(h_costs, d_c, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream);
        } else {
            cf.resize(N);
            e = cudaMemcpyAsync(cf.data(), d_c, sizeof(float) * N, cudaMemcpyDeviceToHost, c->stream);
        }
    }
    if (e == cudaSuccess && h_finals)
        e = cudaMemcpyAsync(h_finals, d_f, sizeof(double) * (size_t)N * nx, cudaMemcpyDeviceToHost, c->stream);
    uint32_t err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, d_err, sizeof err, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (d_x) cudaFree(d_x);
    if (d_k) cudaFree(d_k);
    if (d_c) cudaFree(d_c);
    if (d_f) cudaFree(d_f);
    if (d_err) cudaFree(d_err);
    if (e != cudaSuccess) return cuda_fail(c, e, "rollout_explicit");
    if (!c->fp64_check)
        for (int n = 0; n < N; ++n) h_costs[n] = cf[n];
    if (err) {
        set_error(c, "a bounded device wait gave up");
        return MPPI_ERR_TIMEOUT;
    }
    return MPPI_OK;
}

mppi_status mppi_sample_knots(mppi_ctx* c, int32_t iter, uint32_t iter_counter, const float* h_nominal,
                              float* h_out) {
    MPPI_NVTX("mppi_sample_knots");
    if (!c || !h_nominal || !h_out || iter < 0 || iter >= c->iters) return MPPI_ERR_INVALID_ARG;
    float *d_nom = nullptr, *d_out = nullptr;
    const size_t NE = (size_t)c->N * c->E;
    cudaError_t e = cudaMalloc(&d_nom, sizeof(float) * c->E);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(float) * NE);
    if (e == cudaSuccess) e = cudaMemcpy(d_nom, h_nominal, sizeof(float) * c->E, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        SampleArgs sa;
        sa.nominal = d_nom;
        sa.sigma_row = c->d_sigma + (size_t)iter * c->nk;
        sa.model = (const DevModel<float>*)c->model->d_f;
        sa.knots = d_out;
        sa.solve = nullptr;
        sa.iter_offset = 0;
        sa.iter_counter_override = iter_counter;
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
        e = launch_sample_knots(sa, c->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, d_out, sizeof(float) * NE, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (d_nom) cudaFree(d_nom);
    if (d_out) cudaFree(d_out);
    if (e != cudaSuccess) return cuda_fail(c, e, "sample_knots");
    return MPPI_OK;
}

mppi_status mppi_get_iter_counter(const mppi_ctx* c, uint32_t* out) {
    if (!c || !out) return MPPI_ERR_INVALID_ARG;
    mppi_ctx* cc = const_cast<mppi_ctx*>(c);
    CK(cc, cudaStreamSynchronize(c->stream));
    CK(cc, cudaMemcpy(out, &c->d_solve->iter_counter, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    return MPPI_OK;
}

mppi_status mppi_set_iter_counter(mppi_ctx* c, uint32_t value) {
    if (!c) return MPPI_ERR_INVALID_ARG;
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, cudaMemcpy(&c->d_solve->iter_counter, &value, sizeof(uint32_t), cudaMemcpyHostToDevice));
    return MPPI_OK;
}

// State blob: magic, E, nj, nk, iter counter, then E floats of the resident nominal.
mppi_status mppi_export_state(const mppi_ctx* c, void* buf, size_t* len) {
    if (!c || !len) return MPPI_ERR_INVALID_ARG;
    const size_t need = 5 * sizeof(uint32_t) + sizeof(float) * c->E;
    if (!buf) {
        *len = need;
        return MPPI_OK;
    }
    if (*len < need) return MPPI_ERR_INVALID_ARG;
    mppi_ctx* cc = const_cast<mppi_ctx*>(c);
    uint32_t hdr[5] = {0x4D505049u, (uint32_t)c->E, (uint32_t)c->nj, (uint32_t)c->nk, 0};
    CK(cc, cudaStreamSynchronize(c->stream));
    CK(cc, cudaMemcpy(&hdr[4], &c->d_solve->iter_counter, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    memcpy(buf, hdr, sizeof hdr);
    CK(cc, cudaMemcpy((char*)buf + sizeof hdr, c->d_nominal, sizeof(float) * c->E, cudaMemcpyDeviceToHost));
    *len = need;
    return MPPI_OK;
}

mppi_status mppi_import_state(mppi_ctx* c, const void* buf, size_t len) {
    if (!c || !buf) return MPPI_ERR_INVALID_ARG;
    uint32_t hdr[5];
    if (len < sizeof hdr) return MPPI_ERR_INVALID_ARG;
    memcpy(hdr, buf, sizeof hdr);
    if (hdr[0] != 0x4D505049u || hdr[1] != (uint32_t)c->E || hdr[2] != (uint32_t)c->nj || hdr[3] != (uint32_t)c->nk ||
        len < sizeof hdr + sizeof(float) * c->E)
        return MPPI_ERR_INVALID_ARG;
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, cudaMemcpy(&c->d_solve->iter_counter, &hdr[4], sizeof(uint32_t), cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->d_nominal, (const char*)buf + sizeof hdr, sizeof(float) * c->E, cudaMemcpyHostToDevice));
    return MPPI_OK;
}

// ------------------------------------------------------------------------------------
// Receding horizon (Sec. III-E): state prediction over the compute delay and the shift
// of the resident warm start. Both run on the context's stream, after any solve already
// enqueued there.
// ------------------------------------------------------------------------------------
static mppi_status enqueue_predict(mppi_ctx* c, const double* d_state, int32_t steps, double* d_out) {
    cudaError_t e = cudaSuccess;
    if (steps == 0) {
        if (d_out != d_state)
            e = cudaMemcpyAsync(d_out, d_state, sizeof(double) * c->nx, cudaMemcpyDeviceToDevice, c->stream);
    } else if (c->fp64_check) {
        e = launch_predict_f64((const DevModel<double>*)c->model->d_d, d_state, c->d_nominal, c->H, steps, c->nk,
                               c->dt, c->dtk, d_out, &c->d_solve->dev_error, c->stream);
    } else {
        e = launch_predict_f32((const DevModel<float>*)c->model->d_f, d_state, c->d_nominal, c->H, steps, c->nk,
                               (float)c->dt, (float)c->dtk, d_out, &c->d_solve->dev_error, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "predict_state");
    return MPPI_OK;
}

mppi_status mppi_predict_state_device(mppi_ctx* c, const double* d_state, int32_t steps, double* d_out) {
    MPPI_NVTX("mppi_predict_state_device");
    if (!c) return MPPI_ERR_INVALID_ARG;
    if (!d_state || !d_out || steps < 0 || steps > c->H) {
        set_error(c, "mppi_predict_state_device: needs device state and output and 0 <= steps <= H");
        return MPPI_ERR_INVALID_ARG;
    }
    return enqueue_predict(c, d_state, steps, d_out);
}

mppi_status mppi_predict_state(mppi_ctx* c, const double* h_state, int32_t steps, double* h_out) {
    MPPI_NVTX("mppi_predict_state");
    if (!c) return MPPI_ERR_INVALID_ARG;
    if (!h_state || !h_out || steps < 0 || steps > c->H) {
        set_error(c, "mppi_predict_state: needs state and output and 0 <= steps <= H");
        return MPPI_ERR_INVALID_ARG;
    }
    for (int i = 0; i < c->nx; ++i)
        if (!isfinite(h_state[i])) {
            set_error(c, "mppi_predict_state: state is not finite");
            return MPPI_ERR_NONFINITE_STATE;
        }
    double* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double) * 2 * c->nx);
    if (e != cudaSuccess) return cuda_fail(c, e, "predict_state: cudaMalloc");
    e = cudaMemcpyAsync(d, h_state, sizeof(double) * c->nx, cudaMemcpyHostToDevice, c->stream);
    mppi_status st = e == cudaSuccess ? enqueue_predict(c, d, steps, d + c->nx) : cuda_fail(c, e, "predict_state");
    if (st == MPPI_OK) {
        e = cudaMemcpyAsync(h_out, d + c->nx, sizeof(double) * c->nx, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = cuda_fail(c, e, "predict_state");
    }
    cudaFree(d);
    if (st == MPPI_OK) st = mppi_sync(c);
    return st;
}

mppi_status mppi_shift_warm_start(mppi_ctx* c, int32_t steps) {
    MPPI_NVTX("mppi_shift_warm_start");
    if (!c) return MPPI_ERR_INVALID_ARG;
    if (steps < 0) {
        set_error(c, "mppi_shift_warm_start: steps must be >= 0");
        return MPPI_ERR_INVALID_ARG;
    }
    if (steps == 0) return MPPI_OK;
    cudaError_t e = launch_shift_knots(c->d_nominal, c->nj, c->nk, c->H, steps > c->H ? c->H : steps, c->dtk, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "shift_warm_start");
    return MPPI_OK;
}

mppi_status mppi_get_warm_start(const mppi_ctx* c, float* h_out) {
    if (!c || !h_out) return MPPI_ERR_INVALID_ARG;
    mppi_ctx* cc = const_cast<mppi_ctx*>(c);
    CK(cc, cudaStreamSynchronize(c->stream));
    CK(cc, cudaMemcpy(h_out, c->d_nominal, sizeof(float) * c->E, cudaMemcpyDeviceToHost));
    return MPPI_OK;
}

mppi_status mppi_selftest_math(int32_t n, const float* h_x, const float* h_y, float* h_out) {
    if (n < 0 || (n > 0 && (!h_x || !h_y || !h_out))) return MPPI_ERR_INVALID_ARG;
    if (n == 0) return MPPI_OK;
    float *d_x = nullptr, *d_y = nullptr, *d_o = nullptr;
    cudaError_t e = cudaMalloc(&d_x, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_y, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_o, sizeof(float) * 3 * n);
    if (e == cudaSuccess) e = cudaMemcpy(d_x, h_x, sizeof(float) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_y, h_y, sizeof(float) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_fast_math(n, d_x, d_y, d_o, 0);
    if (e == cudaSuccess) e = cudaMemcpy(h_out, d_o, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost);
    if (d_x) cudaFree(d_x);
    if (d_y) cudaFree(d_y);
    if (d_o) cudaFree(d_o);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "selftest_math");
    return MPPI_OK;
}

mppi_status mppi_selftest_widen(int32_t n, const float* h_x, double* h_out) {
    if (n < 0 || (n > 0 && (!h_x || !h_out))) return MPPI_ERR_INVALID_ARG;
    if (n == 0) return MPPI_OK;
    float* d_x = nullptr;
    double* d_o = nullptr;
    cudaError_t e = cudaMalloc(&d_x, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_o, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMemcpy(d_x, h_x, sizeof(float) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_widen(n, d_x, d_o, 0);
    if (e == cudaSuccess) e = cudaMemcpy(h_out, d_o, sizeof(double) * n, cudaMemcpyDeviceToHost);
    if (d_x) cudaFree(d_x);
    if (d_o) cudaFree(d_o);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "selftest_widen");
    return MPPI_OK;
}

mppi_status mppi_philox_words(int32_t n, const uint32_t* h_ctr, const uint32_t* h_key, uint32_t* h_out) {
    if (n < 0 || (n > 0 && (!h_ctr || !h_key || !h_out))) return MPPI_ERR_INVALID_ARG;
    if (n == 0) return MPPI_OK;
    uint32_t *d_c = nullptr, *d_o = nullptr;
    cudaError_t e = cudaMalloc(&d_c, sizeof(uint32_t) * 4 * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_o, sizeof(uint32_t) * 4 * n);
    if (e == cudaSuccess) e = cudaMemcpy(d_c, h_ctr, sizeof(uint32_t) * 4 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_philox_words(n, d_c, h_key[0], h_key[1], d_o, 0);
    if (e == cudaSuccess) e = cudaMemcpy(h_out, d_o, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost);
    if (d_c) cudaFree(d_c);
    if (d_o) cudaFree(d_o);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "philox_words");
    return MPPI_OK;
}

mppi_status mppi_weights(int32_t K, const float* h_costs, double lambda, int32_t normalize, double* h_w,
                         mppi_result* h_info) {
    MPPI_NVTX("mppi_weights");
    if (K < 1 || !h_costs || !h_w || !(lambda > 0)) return MPPI_ERR_INVALID_ARG;
    if (normalize != MPPI_NORM_MINMAX && normalize != MPPI_NORM_RAW) return MPPI_ERR_INVALID_ARG;
    float *d_c = nullptr, *d_k = nullptr;
    double *d_e = nullptr, *d_w = nullptr, *d_zq = nullptr, *d_p = nullptr;
    DevIterInfo* d_i = nullptr;
    DevIterInfo inf;
    const int nch = num_chunks(K);
    cudaError_t e = cudaMalloc(&d_c, sizeof(float) * K);
    if (e == cudaSuccess) e = cudaMalloc(&d_k, sizeof(float) * K);
    if (e == cudaSuccess) e = cudaMalloc(&d_e, sizeof(double) * K);
    if (e == cudaSuccess) e = cudaMalloc(&d_w, sizeof(double) * K);
    if (e == cudaSuccess) e = cudaMalloc(&d_zq, sizeof(double) * 2 * nch);
    if (e == cudaSuccess) e = cudaMalloc(&d_p, sizeof(double) * nch);
    if (e == cudaSuccess) e = cudaMalloc(&d_i, sizeof(DevIterInfo));
    if (e == cudaSuccess) e = cudaMemcpy(d_c, h_costs, sizeof(float) * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d_k, 0, sizeof(float) * K);
    // one knot element of zeros: the chunk kernel's partial sums are not needed here
    if (e == cudaSuccess) e = launch_weights_average(d_c, d_k, K, 1, lambda, normalize, d_e, d_zq, d_p, d_i, 0);
    if (e == cudaSuccess) e = launch_normalize_weights(d_e, d_zq, K, d_w, d_i, 0);
    if (e == cudaSuccess) e = cudaMemcpy(h_w, d_w, sizeof(double) * K, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&inf, d_i, sizeof inf, cudaMemcpyDeviceToHost);
    for (void* ptr : {(void*)d_c, (void*)d_k, (void*)d_e, (void*)d_w, (void*)d_zq, (void*)d_p, (void*)d_i})
        if (ptr) cudaFree(ptr);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "weights");
    if (h_info) {
        h_info->cost_min = inf.smin;
        h_info->cost_max = inf.smax;
        h_info->best_cost = inf.best >= 0 ? (double)h_costs[inf.best] : NAN;
        h_info->ess = inf.ess;
        h_info->lse = inf.lse;
        h_info->best_index = inf.best;
        h_info->best_iter = 0;
        h_info->n_finite = inf.nfinite;
        h_info->status = inf.status;
    }
    return inf.status;
}

mppi_status mppi_average(int32_t K, int32_t E, const float* h_knots, const double* h_w, double* h_out) {
    MPPI_NVTX("mppi_average");
    if (K < 1 || E < 1 || !h_knots || !h_w || !h_out) return MPPI_ERR_INVALID_ARG;
    float* d_k = nullptr;
    double *d_w = nullptr, *d_p = nullptr, *d_o = nullptr;
    const int nch = num_chunks(K);
    cudaError_t e = cudaMalloc(&d_k, sizeof(float) * (size_t)K * E);
    if (e == cudaSuccess) e = cudaMalloc(&d_w, sizeof(double) * K);
    if (e == cudaSuccess) e = cudaMalloc(&d_p, sizeof(double) * (size_t)nch * E);
    if (e == cudaSuccess) e = cudaMalloc(&d_o, sizeof(double) * E);
    if (e == cudaSuccess) e = cudaMemcpy(d_k, h_knots, sizeof(float) * (size_t)K * E, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_w, h_w, sizeof(double) * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_average_partial(d_k, d_w, K, E, d_p, 0);
    if (e == cudaSuccess) e = launch_average_reduce(d_p, nch, E, d_o, 0);
    if (e == cudaSuccess) e = cudaMemcpy(h_out, d_o, sizeof(double) * E, cudaMemcpyDeviceToHost);
    if (d_k) cudaFree(d_k);
    if (d_w) cudaFree(d_w);
    if (d_p) cudaFree(d_p);
    if (d_o) cudaFree(d_o);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "average");
    return MPPI_OK;
}

mppi_status mppi_forward_dynamics(const mppi_model* m, int32_t n, const double* h_x, const double* h_tau,
                                  double* h_acc) {
    return mppi_forward_dynamics_ex(m, n, h_x, h_tau, h_acc, 0);
}

mppi_status mppi_forward_dynamics_ex(const mppi_model* m, int32_t n, const double* h_x, const double* h_tau,
                                     double* h_acc, int32_t fp64) {
    MPPI_NVTX("mppi_forward_dynamics");
    if (!m || n < 0 || (n > 0 && (!h_x || !h_acc || (m->nj > 0 && !h_tau)))) return MPPI_ERR_INVALID_ARG;
    if (n == 0) return MPPI_OK;
    const int nx = 13 + 2 * m->nj, nv = 6 + m->nj;
    double *d_x = nullptr, *d_t = nullptr, *d_a = nullptr;
    cudaError_t e = cudaMalloc(&d_x, sizeof(double) * (size_t)n * nx);
    if (e == cudaSuccess) e = cudaMalloc(&d_t, sizeof(double) * (size_t)n * std::max(m->nj, 1));
    if (e == cudaSuccess) e = cudaMalloc(&d_a, sizeof(double) * (size_t)n * nv);
    if (e == cudaSuccess) e = cudaMemcpy(d_x, h_x, sizeof(double) * (size_t)n * nx, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && m->nj > 0)
        e = cudaMemcpy(d_t, h_tau, sizeof(double) * (size_t)n * m->nj, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d_a, 0, sizeof(double) * (size_t)n * nv);
    if (e == cudaSuccess) e = prepare_kernels();
    if (e == cudaSuccess) {
        if (fp64) e = launch_dynamics_f64((const DevModel<double>*)m->d_d, n, d_x, d_t, d_a, 0);
        else e = launch_dynamics_f32((const DevModel<float>*)m->d_f, n, d_x, d_t, d_a, 0);
    }
    if (e == cudaSuccess) e = cudaMemcpy(h_acc, d_a, sizeof(double) * (size_t)n * nv, cudaMemcpyDeviceToHost);
    if (d_x) cudaFree(d_x);
    if (d_t) cudaFree(d_t);
    if (d_a) cudaFree(d_a);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "forward_dynamics");
    return MPPI_OK;
}

mppi_status mppi_ctx_info(const mppi_ctx* c, int32_t* o) {
    if (!c || !o) return MPPI_ERR_INVALID_ARG;
    o[0] = c->N;
    o[1] = c->H;
    o[2] = c->nk;
    o[3] = c->iters;
    o[4] = c->nj;
    o[5] = c->nx;
    o[6] = c->mapping;
    o[7] = c->block;
    return MPPI_OK;
}

mppi_status mppi_ctx_io_bytes(const mppi_ctx* c, int64_t* o) {
    if (!c || !o) return MPPI_ERR_INVALID_ARG;
    o[0] = (int64_t)(sizeof(double) * c->nx);
    o[1] = (int64_t)(sizeof(float) * 2 * c->E + sizeof(mppi_result));
    return MPPI_OK;
}

mppi_status mppi_model_info(const mppi_model* m, int32_t* o) {
    if (!m || !o) return MPPI_ERR_INVALID_ARG;
    o[0] = m->topology;
    o[1] = m->host_f.axis_plan;
    o[2] = m->host_f.paper_cost;
    o[3] = m->nb;
    return MPPI_OK;
}

size_t mppi_ctx_device_bytes(const mppi_ctx* c) { return c ? c->dev_bytes : 0; }

int32_t mppi_ctx_kernels_per_solve(const mppi_ctx* c) { return c ? 1 + 3 * c->iters : 0; }

mppi_status mppi_ctx_set_fp64_check(mppi_ctx* c, int32_t on) {
    if (!c) return MPPI_ERR_INVALID_ARG;
    c->fp64_check = on != 0;
    return MPPI_OK;
}

mppi_status mppi_ctx_set_mapping(mppi_ctx* c, int32_t mapping, int32_t block) {
    if (!c) return MPPI_ERR_INVALID_ARG;
    if (!mapping_valid(c->model, mapping, block)) return MPPI_ERR_INVALID_ARG;
    c->mapping = mapping;
    c->block = block > 0 ? block : default_block(mapping);
    invalidate_graph(c);
    return MPPI_OK;
}

mppi_status mppi_ctx_profile(mppi_ctx* c, int32_t on) {
    if (!c) return MPPI_ERR_INVALID_ARG;
    if (on && c->ev.empty()) {
        c->ev.resize(2 * c->iters);
        for (auto& e : c->ev) CK(c, cudaEventCreate(&e));
    }
    c->profile = on != 0;
    invalidate_graph(c);
    return MPPI_OK;
}

mppi_status mppi_ctx_rollout_ms(mppi_ctx* c, float* h_ms) {
    if (!c || !h_ms || !c->profile) return MPPI_ERR_INVALID_ARG;
    CK(c, cudaStreamSynchronize(c->stream));
    for (int it = 0; it < c->iters; ++it) CK(c, cudaEventElapsedTime(&h_ms[it], c->ev[2 * it], c->ev[2 * it + 1]));
    return MPPI_OK;
}

mppi_status mppi_noise_schedule(int32_t iters, int32_t knots, double beta1, double beta2, double scale,
                                float* h_sigma) {
    if (iters < 1 || knots < 1 || !h_sigma || !(beta1 > 0) || !(beta2 > 0) || !(scale >= 0) || !isfinite(scale))
        return MPPI_ERR_INVALID_ARG;
    for (int it = 0; it < iters; ++it) {
        const int i = iters - it;  // iterations run i = I..1
        for (int k = 0; k < knots; ++k)
            h_sigma[it * knots + k] =
                (float)(scale * exp(-(double)(iters - i) / (beta1 * iters) - (double)(knots - k) / (beta2 * knots)));
    }
    return MPPI_OK;
}

}  // extern "C"

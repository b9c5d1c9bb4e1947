// Warp-per-sample rollout: one sample per group of G lanes (G = 32: a warp, G = 16: a
// half warp), lane b of the group owns body b. The floating-base articulated-body
// algorithm runs level by level across lanes:
//   pass 1 (root -> leaves): world pose and spatial velocity of each body from its
//          parent's (warp shuffles), contact forces, bias forces;
//   pass 2 (leaves -> root): articulated inertia and bias of each body, handed to the
//          parent through shared memory (27 values per body);
//   root:  6x6 Cholesky solve for the base acceleration;
//   pass 3 (root -> leaves): joint accelerations.
// Joint lanes evaluate their own Hermite setpoint and PD torque (Sec. III-A
// Eq. hermite_segment, Sec. III-C Eq. pd-controller); the root lane integrates the base
// and accumulates the running cost with Kahan compensation.
#pragma once
#include "common.cuh"

namespace mppi {

template <typename T, int G>
__device__ __forceinline__ T gshfl(T v, int src) {
    return __shfl_sync(0xffffffffu, v, src, G);
}

template <typename T>
struct LaneConst {
    V3<T> a, r;          // joint axis (child frame), joint position (parent frame)
    T Ao[6];             // rotational inertia about the body origin
    V3<T> mc;            // mass * com
    T m, arm, kp, kd, tmax;
    int par, lvl, cfirst, ccount, nchild;
    bool body, joint;
};

// Pins a loop-invariant value to a register (an opaque empty asm), so the compiler keeps
// it across the step loop instead of reloading or recomputing it each step.
__device__ __forceinline__ void pin_r(float& x) { asm volatile("" : "+f"(x)); }
__device__ __forceinline__ void pin_r(double& x) { asm volatile("" : "+d"(x)); }
template <typename T>
__device__ __forceinline__ void pin_lane_const(LaneConst<T>& L) {
    pin_r(L.a.x);
    pin_r(L.a.y);
    pin_r(L.a.z);
    pin_r(L.r.x);
    pin_r(L.r.y);
    pin_r(L.r.z);
#pragma unroll
    for (int k = 0; k < 6; ++k) pin_r(L.Ao[k]);
    pin_r(L.mc.x);
    pin_r(L.mc.y);
    pin_r(L.mc.z);
    pin_r(L.m);
    pin_r(L.arm);
    pin_r(L.kp);
    pin_r(L.kd);
    pin_r(L.tmax);
}

template <typename T>
__device__ __forceinline__ void load_lane_const(const DevModel<T>& M, int b, LaneConst<T>& L) {
    L.body = b < M.nb;
    L.joint = L.body && b > 0;
    const int bb = L.body ? b : 0;
    L.a = v3(M.axis[0][bb], M.axis[1][bb], M.axis[2][bb]);
    L.r = v3(M.jpos[0][bb], M.jpos[1][bb], M.jpos[2][bb]);
#pragma unroll
    for (int k = 0; k < 6; ++k) L.Ao[k] = M.Ao[k][bb];
    L.mc = v3(M.mc[0][bb], M.mc[1][bb], M.mc[2][bb]);
    L.m = M.mass[bb];
    L.arm = M.armature[bb];
    L.kp = M.kp[bb];
    L.kd = M.kd[bb];
    L.tmax = M.tau_max[bb];
    L.par = L.joint ? M.parent[bb] : 0;
    L.lvl = L.body ? M.level[bb] : -1;
    L.cfirst = M.cfirst[bb];
    L.ccount = L.body ? M.ccount[bb] : 0;
    L.nchild = L.body ? M.nchild[bb] : 0;
}

// Per-lane state: the root lane uses p, quat, w, vl; joint lanes use q, qd.
template <typename T>
struct LaneState {
    V3<T> p;
    T qw, qx, qy, qz;
    V3<T> w, vl;
    T q, qd;
};

// Outputs of one dynamics evaluation.
template <typename T>
struct StepOut {
    T qdd;            // joint lanes
    V3<T> aw, av;     // root lane: true base spatial acceleration (body coordinates)
    M3<T> R0;         // root lane: base rotation (pre-step)
    T cost_z, cost_tilt;  // cost-body terms (valid on every lane after the broadcast)
    T cost_paper;         // modular running-cost terms of Sec. IV-A (every lane; 0 when off)
};

// One evaluation of the forward dynamics for the group's sample under joint torque tau
// (joint lanes). contrib: shared memory [27][blockDim.x]. gl: lane within group.
template <typename T, int G>
__device__ __forceinline__ void warp_dynamics(const DevModel<T>& M, const LaneConst<T>& L, const LaneState<T>& S,
                                              T tau, T* __restrict__ contrib, int gl, StepOut<T>& out) {
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    // ---- pass 1: poses and velocities ----
    M3<T> Rj;
    {
        T sq, cq;
        sc_sincos_r(L.joint ? S.q : T(0), &sq, &cq);
        Rj = axis_rotation(L.a, sq, cq);
    }
    M3<T> R;
    V3<T> p, w, vl;
    if (gl == 0) {
        R = quat_to_R(S.qw, S.qx, S.qy, S.qz);
        p = S.p;
        if (M.fixed_base) {
            w = v3(T(0), T(0), T(0));
            vl = w;
        } else {
            w = S.w;
            vl = S.vl;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) R.m[k] = T(0);
        p = v3(T(0), T(0), T(0));
        w = p;
        vl = p;
    }
    const int nlev = M.nlevels;
    for (int l = 1; l < nlev; ++l) {
        M3<T> Rp;
#pragma unroll
        for (int k = 0; k < 9; ++k) Rp.m[k] = gshfl<T, G>(R.m[k], L.par);
        const V3<T> pp = v3(gshfl<T, G>(p.x, L.par), gshfl<T, G>(p.y, L.par), gshfl<T, G>(p.z, L.par));
        const V3<T> wp = v3(gshfl<T, G>(w.x, L.par), gshfl<T, G>(w.y, L.par), gshfl<T, G>(w.z, L.par));
        const V3<T> vp = v3(gshfl<T, G>(vl.x, L.par), gshfl<T, G>(vl.y, L.par), gshfl<T, G>(vl.z, L.par));
        if (L.lvl == l) {
            R = mul(Rp, Rj);
            p = pp + mul(Rp, L.r);
            w = mulT(Rj, wp) + S.qd * L.a;
            vl = mulT(Rj, vp - cross(L.r, wp));
        }
    }
    // velocity product c = v x (S qd) = (w x s, vl x s)
    V3<T> cw = v3(T(0), T(0), T(0)), cv = cw;
    if (L.joint) {
        const V3<T> s = S.qd * L.a;
        cw = cross(w, s);
        cv = cross(vl, s);
    }
    // ---- contact forces (ground plane z = 0), external spatial force in body frame ----
    V3<T> fe_n = v3(T(0), T(0), T(0)), fe_f = fe_n;
    const bool paper = M.paper_cost != 0;
    T pcost = T(0);  // this lane's share of the modular running cost
    for (int c = 0; c < L.ccount; ++c) {
        const int ci = L.cfirst + c;
        const V3<T> rc = v3(M.cpos[0][ci], M.cpos[1][ci], M.cpos[2][ci]);
        const V3<T> pc = p + mul(R, rc);
        const T depth = -pc.z;
        if (depth > T(0)) {
            const V3<T> vw = mul(R, vl + cross(w, rc));
            const T fn = sc_max(M.contact_k * depth - M.contact_c * vw.z, T(0));
            const T sc = -M.mu * fn * sc_rsqrt(vw.x * vw.x + vw.y * vw.y + M.eps_f * M.eps_f);
            const V3<T> F = v3(sc * vw.x, sc * vw.y, fn);
            const V3<T> fb = mulT(R, F);
            fe_f = fe_f + fb;
            fe_n = fe_n + cross(rc, fb);
            if (paper) pcost += contact_cost(M, vw, F);
        } else if (paper) {
            pcost += M.cf_off;
        }
    }
    if (paper) {
        if (L.joint) {
            const T dq = S.q - M.q_init[gl];
            pcost += M.w_q * dq * dq;
        }
        if (gl == 0) pcost += base_cost(M, R, p);
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) pcost += __shfl_xor_sync(0xffffffffu, pcost, off, G);
    }
    out.cost_paper = pcost;
    // ---- bias pA = v x* (I v) - f_ext ; articulated inertia starts at the body's ----
    // h = I v = (Ao w + mc x vl, m vl - mc x w); v x* h = (w x hn + vl x hf, w x hf) with
    // vl x hf = -vl x (mc x w) exactly (vl x vl = 0), written so FP32 does not leave a
    // rounding residue of m |vl|^2 that a small rotational inertia would amplify.
    const V3<T> mcw = cross(L.mc, w);
    const V3<T> hn = sym_mul(L.Ao, w) + cross(L.mc, vl);
    const V3<T> hf = L.m * vl - mcw;
    V3<T> pAn = cross(w, hn) - cross(vl, mcw) - fe_n;
    V3<T> pAf = cross(w, hf) - fe_f;
    Art<T> IA;
#pragma unroll
    for (int k = 0; k < 6; ++k) IA.A[k] = L.Ao[k];
    IA.B[0] = T(0);
    IA.B[1] = -L.mc.z;
    IA.B[2] = L.mc.y;
    IA.B[3] = L.mc.z;
    IA.B[4] = T(0);
    IA.B[5] = -L.mc.x;
    IA.B[6] = -L.mc.y;
    IA.B[7] = L.mc.x;
    IA.B[8] = T(0);
    IA.C[0] = IA.C[1] = IA.C[2] = L.m;
    IA.C[3] = IA.C[4] = IA.C[5] = T(0);
    // ---- cost-body terms (pre-step pose), broadcast from the cost body's lane ----
    {
        T tz = T(0), tt = T(0);
        if (gl == M.cost_body) {
            const T dz = p.z - M.z_des;
            const T tilt = sc_atan2_pos(sc_sqrt(R.m[2] * R.m[2] + R.m[5] * R.m[5]), R.m[8]);
            tz = M.w_z * dz * dz;
            tt = M.w_tilt * tilt * tilt;
        }
        out.cost_z = gshfl<T, G>(tz, M.cost_body);
        out.cost_tilt = gshfl<T, G>(tt, M.cost_body);
    }
    // ---- pass 2: articulated inertias, leaves -> root ----
    V3<T> Ua = v3(T(0), T(0), T(0)), Ul = Ua;
    T invD = T(0), uu = T(0);
    const int gbase = tid - gl;
    for (int l = nlev - 1; l >= 1; --l) {
        if (L.lvl == l) {
            Ua = sym_mul(IA.A, L.a);
            Ul = v3(IA.B[0] * L.a.x + IA.B[3] * L.a.y + IA.B[6] * L.a.z,
                    IA.B[1] * L.a.x + IA.B[4] * L.a.y + IA.B[7] * L.a.z,
                    IA.B[2] * L.a.x + IA.B[5] * L.a.y + IA.B[8] * L.a.z);
            const T D = dot(L.a, Ua) + L.arm;
            invD = sc_rcp(D);
            uu = tau - dot(L.a, pAn);
            Art<T> Ia;
            const T U[6] = {Ua.x, Ua.y, Ua.z, Ul.x, Ul.y, Ul.z};
            Ia.A[0] = IA.A[0] - U[0] * U[0] * invD;
            Ia.A[1] = IA.A[1] - U[1] * U[1] * invD;
            Ia.A[2] = IA.A[2] - U[2] * U[2] * invD;
            Ia.A[3] = IA.A[3] - U[0] * U[1] * invD;
            Ia.A[4] = IA.A[4] - U[0] * U[2] * invD;
            Ia.A[5] = IA.A[5] - U[1] * U[2] * invD;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) Ia.B[3 * i + j] = IA.B[3 * i + j] - U[i] * U[3 + j] * invD;
            Ia.C[0] = IA.C[0] - U[3] * U[3] * invD;
            Ia.C[1] = IA.C[1] - U[4] * U[4] * invD;
            Ia.C[2] = IA.C[2] - U[5] * U[5] * invD;
            Ia.C[3] = IA.C[3] - U[3] * U[4] * invD;
            Ia.C[4] = IA.C[4] - U[3] * U[5] * invD;
            Ia.C[5] = IA.C[5] - U[4] * U[5] * invD;
            // pa = pA + Ia c + U u / D
            const T ud = uu * invD;
            const V3<T> Icn = sym_mul(Ia.A, cw) + mul(*reinterpret_cast<const M3<T>*>(Ia.B), cv);
            const V3<T> Icf = mulT(*reinterpret_cast<const M3<T>*>(Ia.B), cw) + sym_mul(Ia.C, cv);
            const V3<T> pan = pAn + Icn + ud * Ua;
            const V3<T> paf = pAf + Icf + ud * Ul;
            Art<T> Ip;
            art_to_parent(Ia, Rj, L.r, Ip);
            const V3<T> fpf = mul(Rj, paf);
            const V3<T> fpn = mul(Rj, pan) + cross(L.r, fpf);
#pragma unroll
            for (int k = 0; k < 6; ++k) contrib[k * nthr + tid] = Ip.A[k];
#pragma unroll
            for (int k = 0; k < 9; ++k) contrib[(6 + k) * nthr + tid] = Ip.B[k];
#pragma unroll
            for (int k = 0; k < 6; ++k) contrib[(15 + k) * nthr + tid] = Ip.C[k];
            contrib[21 * nthr + tid] = fpn.x;
            contrib[22 * nthr + tid] = fpn.y;
            contrib[23 * nthr + tid] = fpn.z;
            contrib[24 * nthr + tid] = fpf.x;
            contrib[25 * nthr + tid] = fpf.y;
            contrib[26 * nthr + tid] = fpf.z;
        }
        __syncwarp();
        if (L.lvl == l - 1) {
            for (int ch = 0; ch < L.nchild; ++ch) {
                const int src = gbase + M.child[ch][gl];
#pragma unroll
                for (int k = 0; k < 6; ++k) IA.A[k] += contrib[k * nthr + src];
#pragma unroll
                for (int k = 0; k < 9; ++k) IA.B[k] += contrib[(6 + k) * nthr + src];
#pragma unroll
                for (int k = 0; k < 6; ++k) IA.C[k] += contrib[(15 + k) * nthr + src];
                pAn = pAn + v3(contrib[21 * nthr + src], contrib[22 * nthr + src], contrib[23 * nthr + src]);
                pAf = pAf + v3(contrib[24 * nthr + src], contrib[25 * nthr + src], contrib[26 * nthr + src]);
            }
        }
        __syncwarp();
    }
    // ---- root: a0' = -IA0^-1 pA0 (gravity as a base offset a' = a - a_g) ----
    V3<T> aw = v3(T(0), T(0), T(0)), av = aw;
    if (gl == 0) {
        const V3<T> g_b = v3(-M.gravity * R.m[6], -M.gravity * R.m[7], -M.gravity * R.m[8]);  // R0^T g
        if (M.fixed_base) {
            av = v3(-g_b.x, -g_b.y, -g_b.z);
        } else {
            const T rhs[6] = {-pAn.x, -pAn.y, -pAn.z, -pAf.x, -pAf.y, -pAf.z};
            T x[6];
            art_solve(IA, rhs, x);
            aw = v3(x[0], x[1], x[2]);
            av = v3(x[3], x[4], x[5]);
        }
        out.R0 = R;
        out.aw = M.fixed_base ? v3(T(0), T(0), T(0)) : aw;
        out.av = M.fixed_base ? v3(T(0), T(0), T(0)) : av + g_b;
    }
    // ---- pass 3: accelerations, root -> leaves ----
    T qdd = T(0);
    for (int l = 1; l < nlev; ++l) {
        const V3<T> awp = v3(gshfl<T, G>(aw.x, L.par), gshfl<T, G>(aw.y, L.par), gshfl<T, G>(aw.z, L.par));
        const V3<T> avp = v3(gshfl<T, G>(av.x, L.par), gshfl<T, G>(av.y, L.par), gshfl<T, G>(av.z, L.par));
        if (L.lvl == l) {
            const V3<T> a1w = mulT(Rj, awp) + cw;
            const V3<T> a1v = mulT(Rj, avp - cross(L.r, awp)) + cv;
            qdd = (uu - dot(Ua, a1w) - dot(Ul, a1v)) * invD;
            aw = a1w + qdd * L.a;
            av = a1v;
        }
    }
    out.qdd = qdd;
}

// Semi-implicit Euler: velocities first, then positions with the new velocities; the
// base orientation by the quaternion exponential of the new body angular velocity.
template <typename T>
__device__ __forceinline__ void integrate_lane(const DevModel<T>& M, const LaneConst<T>& L, int gl,
                                               const StepOut<T>& o, T dt, LaneState<T>& S) {
    if (L.joint) {
        S.qd += dt * o.qdd;
        S.q += dt * S.qd;
    } else if (gl == 0 && !M.fixed_base) {
        S.w = S.w + dt * o.aw;
        S.vl = S.vl + dt * o.av;
        S.p = S.p + dt * mul(o.R0, S.vl);
        const T wn = sc_sqrt(dot(S.w, S.w));
        T dq0, dqs;
        if (wn * dt < T(1e-12)) {
            dq0 = T(1);
            dqs = T(0.5) * dt;
        } else {
            T sh, ch;
            sc_sincos_r(T(0.5) * wn * dt, &sh, &ch);
            dq0 = ch;
            dqs = sh / wn;
        }
        const T dx = dqs * S.w.x, dy = dqs * S.w.y, dz = dqs * S.w.z;
        const T nw = S.qw * dq0 - S.qx * dx - S.qy * dy - S.qz * dz;
        const T nx = S.qw * dx + S.qx * dq0 + S.qy * dz - S.qz * dy;
        const T ny = S.qw * dy - S.qx * dz + S.qy * dq0 + S.qz * dx;
        const T nz = S.qw * dz + S.qx * dy - S.qy * dx + S.qz * dq0;
        const T inv = sc_rsqrt(nw * nw + nx * nx + ny * ny + nz * nz);
        S.qw = nw * inv;
        S.qx = nx * inv;
        S.qy = ny * inv;
        S.qz = nz * inv;
    }
}

template <typename T, typename XT>
__device__ __forceinline__ void load_lane_state(const DevModel<T>& M, const LaneConst<T>& L, int gl,
                                                const XT* __restrict__ x, LaneState<T>& S) {
    const int nj = M.nb - 1, nq = 7 + nj;
    S.p = v3((T)x[0], (T)x[1], (T)x[2]);
    S.qw = (T)x[3];
    S.qx = (T)x[4];
    S.qy = (T)x[5];
    S.qz = (T)x[6];
    S.vl = v3((T)x[nq], (T)x[nq + 1], (T)x[nq + 2]);
    S.w = v3((T)x[nq + 3], (T)x[nq + 4], (T)x[nq + 5]);
    S.q = L.joint ? (T)x[7 + gl - 1] : T(0);
    S.qd = L.joint ? (T)x[nq + 6 + gl - 1] : T(0);
}

template <typename T, typename XT>
__device__ __forceinline__ void store_lane_state(const DevModel<T>& M, const LaneConst<T>& L, int gl,
                                                 const LaneState<T>& S, XT* __restrict__ x) {
    const int nj = M.nb - 1, nq = 7 + nj;
    if (gl == 0) {
        x[0] = (XT)S.p.x;
        x[1] = (XT)S.p.y;
        x[2] = (XT)S.p.z;
        x[3] = (XT)S.qw;
        x[4] = (XT)S.qx;
        x[5] = (XT)S.qy;
        x[6] = (XT)S.qz;
        x[nq] = (XT)S.vl.x;
        x[nq + 1] = (XT)S.vl.y;
        x[nq + 2] = (XT)S.vl.z;
        x[nq + 3] = (XT)S.w.x;
        x[nq + 4] = (XT)S.w.y;
        x[nq + 5] = (XT)S.w.z;
    } else if (L.joint) {
        x[7 + gl - 1] = (XT)S.q;
        x[nq + 6 + gl - 1] = (XT)S.qd;
    }
}

// Rollout of one sample by its group: the first nsteps (<= H) of the H steps tracking the
// Hermite setpoints of knots [nk][2][nj] (global), returning the Kahan-compensated cost
// sum on every lane. x0: initial state [nx] (global, FP32 or FP64). xf: optional state
// after the last step simulated.
template <typename T, int G, typename XT>
__device__ __noinline__ T warp_rollout(const DevModel<T>& M, const LaneConst<T>& Lin, int gl,
                                          const XT* __restrict__ x0, const float* __restrict__ knots, int H,
                                          int nsteps, int nk, T dt, T dtk, T* __restrict__ contrib,
                                          XT* __restrict__ xf) {
    const int nj = M.nb - 1;
    LaneConst<T> L = Lin;
    pin_lane_const(L);
    LaneState<T> S;
    load_lane_state(M, L, gl, x0, S);
    const V3<T> p_start = S.p;
    const T inv_dtk = T(1) / dtk;
    T sum = T(0), comp = T(0);
    int kcur = -1;
    T q0 = T(0), v0 = T(0), q1 = T(0), v1 = T(0);
    const int j = gl - 1;
    for (int h = 0; h < nsteps; ++h) {
        // segment by integer arithmetic: r = h (nk-1), k = floor(r / H), s = (r - k H) / H
        const int r = h * (nk - 1);
        int k = r / H;
        if (k > nk - 2) k = nk - 2;
        const T s = (T)(r - k * H) / (T)H;
        if (k != kcur) {
            kcur = k;
            if (L.joint) {
                q0 = (T)knots[(k * 2 + 0) * nj + j];
                v0 = (T)knots[(k * 2 + 1) * nj + j];
                q1 = (T)knots[((k + 1) * 2 + 0) * nj + j];
                v1 = (T)knots[((k + 1) * 2 + 1) * nj + j];
            }
        }
        T tau = T(0);
        if (L.joint) {
            const T s2 = s * s, s3 = s2 * s;
            const T h00 = T(2) * s3 - T(3) * s2 + T(1), h10 = s3 - T(2) * s2 + s;
            const T h01 = T(-2) * s3 + T(3) * s2, h11 = s3 - s2;
            const T d00 = T(6) * s2 - T(6) * s, d10 = T(3) * s2 - T(4) * s + T(1);
            const T d01 = T(-6) * s2 + T(6) * s, d11 = T(3) * s2 - T(2) * s;
            const T qref = h00 * q0 + h10 * dtk * v0 + h01 * q1 + h11 * dtk * v1;
            const T vref = (d00 * q0 + d01 * q1) * inv_dtk + d10 * v0 + d11 * v1;
            tau = sc_clamp(L.kp * (qref - S.q) + L.kd * (vref - S.qd), -L.tmax, L.tmax);
        }
        StepOut<T> o;
        warp_dynamics<T, G>(M, L, S, tau, contrib, gl, o);
        // running cost on the pre-step state: |tau|^2 reduced across the group
        T tt = tau * tau;
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) tt += __shfl_xor_sync(0xffffffffu, tt, off, G);
        if (gl == 0) {
            const T vx = M.fixed_base ? T(0) : (o.R0.m[0] * S.vl.x + o.R0.m[1] * S.vl.y + o.R0.m[2] * S.vl.z);
            const T dv = vx - M.vx_des;
            const T c = o.cost_z + M.w_vx * dv * dv + o.cost_tilt + M.w_tau * tt + o.cost_paper;
            const T y = c - comp;
            const T t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
        integrate_lane(M, L, gl, o, dt, S);
    }
    if (M.paper_cost && nsteps == H && gl == 0) {  // terminal cost of a full rollout
        const T y = terminal_cost(M, S.p, p_start, H, dt) - comp;
        const T t = sum + y;
        comp = (t - sum) - y;
        sum = t;
    }
    if (xf) store_lane_state(M, L, gl, S, xf);
    return gshfl<T, G>(sum, 0);
}

}  // namespace mppi

namespace mppi {

// ------------------------------------------------------------------------------------
// Kernels. Shared memory: the model (one bulk copy) followed by the per-lane
// child->parent exchange area [27][blockDim.x].
// ------------------------------------------------------------------------------------
template <typename T>
__host__ __device__ constexpr size_t warp_smem_bytes(int block) {
    return sizeof(DevModel<T>) + (size_t)27 * block * sizeof(T);
}

template <typename T, int G>
__global__ void __launch_bounds__(256) rollout_warp_kernel(RolloutArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t mbar;
    DevModel<T>* M = reinterpret_cast<DevModel<T>*>(smem);
    T* contrib = reinterpret_cast<T*>(smem + sizeof(DevModel<T>));
    if (!bulk_load_to_smem(M, a.model, (uint32_t)sizeof(DevModel<T>), &mbar)) {
        if (threadIdx.x == 0 && a.status) atomicOr(a.status, DEV_ERR_TMA_TIMEOUT);
        return;
    }
    const int gl = threadIdx.x % G;
    const int spb = blockDim.x / G;
    const int n = blockIdx.x * spb + threadIdx.x / G;
    const bool active = n < a.N;
    const int ne = active ? n : a.N - 1;
    LaneConst<T> L;
    load_lane_const(*M, gl, L);
    const int nj = M->nb - 1;
    const int nx = 13 + 2 * nj;
    const int E = a.nk * 2 * nj;
    double* xf = (active && a.finals) ? a.finals + (size_t)n * nx : nullptr;
    const T c = warp_rollout<T, G, double>(*M, L, gl, a.x0, a.knots + (size_t)ne * E, a.H, a.H, a.nk, a.dt,
                                           a.dtk, contrib, xf);
    if (active && gl == 0) a.costs[n] = c;
}

template <typename T>
__global__ void __launch_bounds__(256) dynamics_kernel(const DevModel<T>* gm, int n, const double* __restrict__ x,
                                                       const double* __restrict__ tau, double* __restrict__ acc) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t mbar;
    DevModel<T>* M = reinterpret_cast<DevModel<T>*>(smem);
    T* contrib = reinterpret_cast<T*>(smem + sizeof(DevModel<T>));
    if (!bulk_load_to_smem(M, gm, (uint32_t)sizeof(DevModel<T>), &mbar)) return;
    const int gl = threadIdx.x & 31;
    const int s = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const bool active = s < n;
    const int se = active ? s : n - 1;
    const int nj = M->nb - 1, nx = 13 + 2 * nj, nv = 6 + nj;
    LaneConst<T> L;
    load_lane_const(*M, gl, L);
    LaneState<T> S;
    load_lane_state(*M, L, gl, x + (size_t)se * nx, S);
    const T t = L.joint ? (T)tau[(size_t)se * nj + gl - 1] : T(0);
    StepOut<T> o;
    warp_dynamics<T, 32>(*M, L, S, t, contrib, gl, o);
    if (!active) return;
    if (gl == 0) {
        double* out = acc + (size_t)s * nv;
        out[0] = o.aw.x;
        out[1] = o.aw.y;
        out[2] = o.aw.z;
        out[3] = o.av.x;
        out[4] = o.av.y;
        out[5] = o.av.z;
    } else if (L.joint) {
        acc[(size_t)s * nv + 6 + gl - 1] = o.qdd;
    }
}

// State prediction (Sec. III-E): one warp simulates the first nsteps steps of the
// spline of knots [nk][2][nj] over a horizon of H steps from x0 and writes the state
// reached to out [nx].
template <typename T>
__global__ void __launch_bounds__(32) predict_kernel(const DevModel<T>* gm, const double* __restrict__ x0,
                                                     const float* __restrict__ knots, int H, int nsteps, int nk, T dt,
                                                     T dtk, double* __restrict__ out, uint32_t* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t mbar;
    DevModel<T>* M = reinterpret_cast<DevModel<T>*>(smem);
    T* contrib = reinterpret_cast<T*>(smem + sizeof(DevModel<T>));
    if (!bulk_load_to_smem(M, gm, (uint32_t)sizeof(DevModel<T>), &mbar)) {
        if (threadIdx.x == 0 && status) atomicOr(status, DEV_ERR_TMA_TIMEOUT);
        return;
    }
    const int gl = threadIdx.x;
    LaneConst<T> L;
    load_lane_const(*M, gl, L);
    (void)warp_rollout<T, 32, double>(*M, L, gl, x0, knots, H, nsteps, nk, dt, dtk, contrib, out);
}

template <typename T>
cudaError_t launch_predict_t(const DevModel<T>* m, const double* x0, const float* knots, int H, int nsteps, int nk,
                             T dt, T dtk, double* out, uint32_t* status, cudaStream_t s) {
    if (nsteps < 0 || nsteps > H) return cudaErrorInvalidValue;
    predict_kernel<T><<<1, 32, warp_smem_bytes<T>(32), s>>>(m, x0, knots, H, nsteps, nk, dt, dtk, out, status);
    return cudaGetLastError();
}

template <typename T, int G>
cudaError_t launch_rollout_warp_t(const RolloutArgs<T>& a, int block, cudaStream_t s) {
    if (block <= 0) block = 128;
    if (block % G != 0 || block > 256) return cudaErrorInvalidValue;
    const size_t sm = warp_smem_bytes<T>(block);
    const int spb = block / G;
    const int grid = (a.N + spb - 1) / spb;
    if (grid == 0) return cudaSuccess;
    rollout_warp_kernel<T, G><<<grid, block, sm, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dynamics_t(const DevModel<T>* m, int n, const double* x, const double* tau, double* acc,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int block = 128;
    const size_t sm = warp_smem_bytes<T>(block);
    const int grid = (n + block / 32 - 1) / (block / 32);
    dynamics_kernel<T><<<grid, block, sm, s>>>(m, n, x, tau, acc);
    return cudaGetLastError();
}

// Raise the dynamic shared-memory limit of every instantiation (outside any stream
// capture; once per device is enough, repeating is harmless).
template <typename T>
cudaError_t prepare_warp_kernels() {
    const int sm = (int)warp_smem_bytes<T>(256);
    cudaError_t e = cudaFuncSetAttribute(rollout_warp_kernel<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(rollout_warp_kernel<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(dynamics_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(predict_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)warp_smem_bytes<T>(32));
    return e;
}

}  // namespace mppi

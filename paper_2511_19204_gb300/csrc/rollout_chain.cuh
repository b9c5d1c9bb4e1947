// Lanes-per-chain rollout (device function) for trees made of a floating base and NLEG equal chains of
// LLEN bodies hanging from it (the quadruped: 4 legs x hip/thigh/calf). NLEG lanes share
// one sample; lane g runs leg g's three articulated-body passes serially in registers,
// and every lane of the group carries an identical copy of the base: the legs' articulated
// inertias reach the base through a log2(NLEG)-step butterfly whose sums are bitwise the
// same on every lane, so the replicated base solve and integration never diverge.
// Equations as in the warp-per-sample kernel (Featherstone's articulated-body algorithm,
// Sec. III-A Hermite setpoints, Sec. III-C PD tracking, semi-implicit Euler, Kahan cost).
#pragma once
#include "internal.h"
#include "rollout_warp.cuh"

namespace mppi {

template <int NLEG>
__device__ __forceinline__ float gsum(float v) {
#pragma unroll
    for (int off = NLEG / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off, NLEG);
    return v;
}

template <int NLEG, int LLEN>
__device__ __noinline__ float chain_rollout(const DevModel<float>& M, int g, const double* __restrict__ x0,
                                               const float* __restrict__ knots, int H, int nk, float dt, float dtk,
                                               double* __restrict__ xf) {
    const int nj = M.nb - 1, nq = 7 + nj;
    const int b0 = 1 + g * LLEN;  // first body of this lane's leg
    // base state (replicated on every lane of the group)
    V3<float> p = v3((float)x0[0], (float)x0[1], (float)x0[2]);
    float qw = (float)x0[3], qx = (float)x0[4], qy = (float)x0[5], qz = (float)x0[6];
    V3<float> vl = v3((float)x0[nq], (float)x0[nq + 1], (float)x0[nq + 2]);
    V3<float> w = v3((float)x0[nq + 3], (float)x0[nq + 4], (float)x0[nq + 5]);
    float q[LLEN], qd[LLEN];
#pragma unroll
    for (int j = 0; j < LLEN; ++j) {
        q[j] = (float)x0[7 + b0 - 1 + j];
        qd[j] = (float)x0[nq + 6 + b0 - 1 + j];
    }
    const float inv_dtk = 1.0f / dtk;
    float sum = 0.f, comp = 0.f;
    int kcur = -1;
    float kq0[LLEN], kv0[LLEN], kq1[LLEN], kv1[LLEN];
    const int cb = M.cost_body;
    const int cleg = cb > 0 ? (cb - 1) / LLEN : -1, cj = cb > 0 ? (cb - 1) % LLEN : -1;
    for (int h = 0; h < H; ++h) {
        const int r = h * (nk - 1);
        int k = r / H;
        if (k > nk - 2) k = nk - 2;
        const float s = (float)(r - k * H) / (float)H;
        if (k != kcur) {
            kcur = k;
#pragma unroll
            for (int j = 0; j < LLEN; ++j) {
                const int jj = b0 - 1 + j;
                kq0[j] = knots[(k * 2 + 0) * nj + jj];
                kv0[j] = knots[(k * 2 + 1) * nj + jj];
                kq1[j] = knots[((k + 1) * 2 + 0) * nj + jj];
                kv1[j] = knots[((k + 1) * 2 + 1) * nj + jj];
            }
        }
        // ---- Hermite setpoints and PD torques of this leg's joints ----
        float tau[LLEN];
        {
            const float s2 = s * s, s3 = s2 * s;
            const float h00 = 2.f * s3 - 3.f * s2 + 1.f, h10 = s3 - 2.f * s2 + s;
            const float h01 = -2.f * s3 + 3.f * s2, h11 = s3 - s2;
            const float d00 = 6.f * s2 - 6.f * s, d10 = 3.f * s2 - 4.f * s + 1.f;
            const float d01 = -6.f * s2 + 6.f * s, d11 = 3.f * s2 - 2.f * s;
#pragma unroll
            for (int j = 0; j < LLEN; ++j) {
                const int b = b0 + j;
                const float qref = h00 * kq0[j] + h10 * dtk * kv0[j] + h01 * kq1[j] + h11 * dtk * kv1[j];
                const float vref = (d00 * kq0[j] + d01 * kq1[j]) * inv_dtk + d10 * kv0[j] + d11 * kv1[j];
                tau[j] = sc_clamp(M.kp[b] * (qref - q[j]) + M.kd[b] * (vref - qd[j]), -M.tau_max[b], M.tau_max[b]);
            }
        }
        // ---- base: pose, velocity, bias (replicated) ----
        const M3<float> R0 = quat_to_R(qw, qx, qy, qz);
        const V3<float> w0 = M.fixed_base ? v3(0.f, 0.f, 0.f) : w;
        const V3<float> v0 = M.fixed_base ? v3(0.f, 0.f, 0.f) : vl;
        V3<float> fe0n = v3(0.f, 0.f, 0.f), fe0f = fe0n;
        auto contacts = [&](int b, const M3<float>& R, V3<float> pb, V3<float> wb, V3<float> vb, V3<float>& fen,
                            V3<float>& fef) {
            const int c0 = M.cfirst[b], cn = M.ccount[b];
            for (int c = 0; c < cn; ++c) {
                const int ci = c0 + c;
                const V3<float> rc = v3(M.cpos[0][ci], M.cpos[1][ci], M.cpos[2][ci]);
                const V3<float> pc = pb + mul(R, rc);
                const float depth = -pc.z;
                if (depth > 0.f) {
                    const V3<float> vw = mul(R, vb + cross(wb, rc));
                    const float fn = fmaxf(M.contact_k * depth - M.contact_c * vw.z, 0.f);
                    const float sc = -M.mu * fn / sqrtf(vw.x * vw.x + vw.y * vw.y + M.eps_f * M.eps_f);
                    const V3<float> F = v3(sc * vw.x, sc * vw.y, fn);
                    const V3<float> fb = mulT(R, F);
                    fef = fef + fb;
                    fen = fen + cross(rc, fb);
                }
            }
        };
        contacts(0, R0, p, w0, v0, fe0n, fe0f);
        auto bias = [&](int b, V3<float> wb, V3<float> vb, V3<float> fen, V3<float> fef, V3<float>& pn,
                        V3<float>& pf) {
            const float Ao[6] = {M.Ao[0][b], M.Ao[1][b], M.Ao[2][b], M.Ao[3][b], M.Ao[4][b], M.Ao[5][b]};
            const V3<float> mc = v3(M.mc[0][b], M.mc[1][b], M.mc[2][b]);
            const V3<float> mcw = cross(mc, wb);
            const V3<float> hn = sym_mul(Ao, wb) + cross(mc, vb);
            const V3<float> hf = M.mass[b] * vb - mcw;
            pn = cross(wb, hn) - cross(vb, mcw) - fen;
            pf = cross(wb, hf) - fef;
        };
        V3<float> pA0n, pA0f;
        bias(0, w0, v0, fe0n, fe0f, pA0n, pA0f);
        float tz = 0.f, tt = 0.f;
        if (cb == 0) {
            const float dz = p.z - M.z_des;
            const float tilt = atan2f(sqrtf(R0.m[2] * R0.m[2] + R0.m[5] * R0.m[5]), R0.m[8]);
            tz = M.w_z * dz * dz;
            tt = M.w_tilt * tilt * tilt;
        }
        // ---- leg pass 1: rotations, poses, velocities, velocity products, biases ----
        M3<float> Rj[LLEN];
        V3<float> cw[LLEN], cv[LLEN], pn[LLEN], pf[LLEN];
        {
            M3<float> Rp = R0;
            V3<float> pp = p, wp = w0, vp = v0;
#pragma unroll
            for (int j = 0; j < LLEN; ++j) {
                const int b = b0 + j;
                const V3<float> a = v3(M.axis[0][b], M.axis[1][b], M.axis[2][b]);
                const V3<float> rj = v3(M.jpos[0][b], M.jpos[1][b], M.jpos[2][b]);
                float sq, cq;
                sincosf(q[j], &sq, &cq);
                Rj[j] = axis_rotation(a, sq, cq);
                const M3<float> R = mul(Rp, Rj[j]);
                const V3<float> pb = pp + mul(Rp, rj);
                const V3<float> wb = mulT(Rj[j], wp) + qd[j] * a;
                const V3<float> vb = mulT(Rj[j], vp - cross(rj, wp));
                const V3<float> sa = qd[j] * a;
                cw[j] = cross(wb, sa);
                cv[j] = cross(vb, sa);
                V3<float> fen = v3(0.f, 0.f, 0.f), fef = fen;
                contacts(b, R, pb, wb, vb, fen, fef);
                bias(b, wb, vb, fen, fef, pn[j], pf[j]);
                if (g == cleg && j == cj) {
                    const float dz = pb.z - M.z_des;
                    const float tilt = atan2f(sqrtf(R.m[2] * R.m[2] + R.m[5] * R.m[5]), R.m[8]);
                    tz = M.w_z * dz * dz;
                    tt = M.w_tilt * tilt * tilt;
                }
                Rp = R;
                pp = pb;
                wp = wb;
                vp = vb;
            }
        }
        if (cb > 0) {
            const int src = cleg;  // lane within the group that owns the cost body
            tz = __shfl_sync(0xffffffffu, tz, src, NLEG);
            tt = __shfl_sync(0xffffffffu, tt, src, NLEG);
        }
        // ---- leg pass 2: articulated inertias, calf -> hip -> base contribution ----
        V3<float> Ua[LLEN], Ul[LLEN];
        float uu[LLEN];
        Art<float> carry;
        V3<float> cpn = v3(0.f, 0.f, 0.f), cpf = cpn;
#pragma unroll
        for (int j = LLEN - 1; j >= 0; --j) {
            const int b = b0 + j;
            const V3<float> a = v3(M.axis[0][b], M.axis[1][b], M.axis[2][b]);
            const V3<float> rj = v3(M.jpos[0][b], M.jpos[1][b], M.jpos[2][b]);
            Art<float> IA;
            const float mb = M.mass[b];
            const V3<float> mc = v3(M.mc[0][b], M.mc[1][b], M.mc[2][b]);
#pragma unroll
            for (int t = 0; t < 6; ++t) IA.A[t] = M.Ao[t][b];
            IA.B[0] = 0.f;
            IA.B[1] = -mc.z;
            IA.B[2] = mc.y;
            IA.B[3] = mc.z;
            IA.B[4] = 0.f;
            IA.B[5] = -mc.x;
            IA.B[6] = -mc.y;
            IA.B[7] = mc.x;
            IA.B[8] = 0.f;
            IA.C[0] = IA.C[1] = IA.C[2] = mb;
            IA.C[3] = IA.C[4] = IA.C[5] = 0.f;
            V3<float> pAn = pn[j], pAf = pf[j];
            if (j < LLEN - 1) {
#pragma unroll
                for (int t = 0; t < 6; ++t) IA.A[t] += carry.A[t];
#pragma unroll
                for (int t = 0; t < 9; ++t) IA.B[t] += carry.B[t];
#pragma unroll
                for (int t = 0; t < 6; ++t) IA.C[t] += carry.C[t];
                pAn = pAn + cpn;
                pAf = pAf + cpf;
            }
            const V3<float> ua = sym_mul(IA.A, a);
            const V3<float> ul = v3(IA.B[0] * a.x + IA.B[3] * a.y + IA.B[6] * a.z,
                                    IA.B[1] * a.x + IA.B[4] * a.y + IA.B[7] * a.z,
                                    IA.B[2] * a.x + IA.B[5] * a.y + IA.B[8] * a.z);
            const float invD = 1.f / (dot(a, ua) + M.armature[b]);
            const float u = tau[j] - dot(a, pAn);
            const float U[6] = {ua.x, ua.y, ua.z, ul.x, ul.y, ul.z};
            Art<float> Ia;
            Ia.A[0] = IA.A[0] - U[0] * U[0] * invD;
            Ia.A[1] = IA.A[1] - U[1] * U[1] * invD;
            Ia.A[2] = IA.A[2] - U[2] * U[2] * invD;
            Ia.A[3] = IA.A[3] - U[0] * U[1] * invD;
            Ia.A[4] = IA.A[4] - U[0] * U[2] * invD;
            Ia.A[5] = IA.A[5] - U[1] * U[2] * invD;
#pragma unroll
            for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
                for (int j2 = 0; j2 < 3; ++j2) Ia.B[3 * i2 + j2] = IA.B[3 * i2 + j2] - U[i2] * U[3 + j2] * invD;
            Ia.C[0] = IA.C[0] - U[3] * U[3] * invD;
            Ia.C[1] = IA.C[1] - U[4] * U[4] * invD;
            Ia.C[2] = IA.C[2] - U[5] * U[5] * invD;
            Ia.C[3] = IA.C[3] - U[3] * U[4] * invD;
            Ia.C[4] = IA.C[4] - U[3] * U[5] * invD;
            Ia.C[5] = IA.C[5] - U[4] * U[5] * invD;
            const float ud = u * invD;
            const M3<float>& Bm = *reinterpret_cast<const M3<float>*>(Ia.B);
            const V3<float> pan = pAn + sym_mul(Ia.A, cw[j]) + mul(Bm, cv[j]) + ud * ua;
            const V3<float> paf = pAf + mulT(Bm, cw[j]) + sym_mul(Ia.C, cv[j]) + ud * ul;
            art_to_parent(Ia, Rj[j], rj, carry);
            cpf = mul(Rj[j], paf);
            cpn = mul(Rj[j], pan) + cross(rj, cpf);
            // stored for pass 3, pre-scaled by 1/D
            Ua[j] = invD * ua;
            Ul[j] = invD * ul;
            uu[j] = ud;
        }
        // ---- base: sum the legs' contributions (butterfly), solve ----
        Art<float> IA0;
        {
            const float m0 = M.mass[0];
            const V3<float> mc = v3(M.mc[0][0], M.mc[1][0], M.mc[2][0]);
#pragma unroll
            for (int t = 0; t < 6; ++t) IA0.A[t] = M.Ao[t][0] + gsum<NLEG>(carry.A[t]);
            const float Bb[9] = {0.f, -mc.z, mc.y, mc.z, 0.f, -mc.x, -mc.y, mc.x, 0.f};
#pragma unroll
            for (int t = 0; t < 9; ++t) IA0.B[t] = Bb[t] + gsum<NLEG>(carry.B[t]);
#pragma unroll
            for (int t = 0; t < 3; ++t) IA0.C[t] = m0 + gsum<NLEG>(carry.C[t]);
#pragma unroll
            for (int t = 3; t < 6; ++t) IA0.C[t] = gsum<NLEG>(carry.C[t]);
            pA0n = pA0n + v3(gsum<NLEG>(cpn.x), gsum<NLEG>(cpn.y), gsum<NLEG>(cpn.z));
            pA0f = pA0f + v3(gsum<NLEG>(cpf.x), gsum<NLEG>(cpf.y), gsum<NLEG>(cpf.z));
        }
        const V3<float> g_b = v3(-M.gravity * R0.m[6], -M.gravity * R0.m[7], -M.gravity * R0.m[8]);
        V3<float> aw, av;
        if (M.fixed_base) {
            aw = v3(0.f, 0.f, 0.f);
            av = v3(-g_b.x, -g_b.y, -g_b.z);
        } else {
            const float rhs[6] = {-pA0n.x, -pA0n.y, -pA0n.z, -pA0f.x, -pA0f.y, -pA0f.z};
            float x[6];
            art_solve(IA0, rhs, x);
            aw = v3(x[0], x[1], x[2]);
            av = v3(x[3], x[4], x[5]);
        }
        // ---- leg pass 3: joint accelerations ----
        float qdd[LLEN];
        {
            V3<float> apw = aw, apv = av;
#pragma unroll
            for (int j = 0; j < LLEN; ++j) {
                const int b = b0 + j;
                const V3<float> a = v3(M.axis[0][b], M.axis[1][b], M.axis[2][b]);
                const V3<float> rj = v3(M.jpos[0][b], M.jpos[1][b], M.jpos[2][b]);
                const V3<float> a1w = mulT(Rj[j], apw) + cw[j];
                const V3<float> a1v = mulT(Rj[j], apv - cross(rj, apw)) + cv[j];
                qdd[j] = uu[j] - dot(Ua[j], a1w) - dot(Ul[j], a1v);
                apw = a1w + qdd[j] * a;
                apv = a1v;
            }
        }
        // ---- running cost on the pre-step state ----
        float te = 0.f;
#pragma unroll
        for (int j = 0; j < LLEN; ++j) te += tau[j] * tau[j];
        te = gsum<NLEG>(te);
        {
            const float vx = M.fixed_base ? 0.f : (R0.m[0] * vl.x + R0.m[1] * vl.y + R0.m[2] * vl.z);
            const float dv = vx - M.vx_des;
            const float c = tz + M.w_vx * dv * dv + tt + M.w_tau * te;
            const float y = c - comp;
            const float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
        // ---- semi-implicit Euler ----
#pragma unroll
        for (int j = 0; j < LLEN; ++j) {
            qd[j] += dt * qdd[j];
            q[j] += dt * qd[j];
        }
        if (!M.fixed_base) {
            w = w + dt * aw;
            vl = vl + dt * (av + g_b);
            p = p + dt * mul(R0, vl);
            const float wn = sqrtf(dot(w, w));
            float dq0, dqs;
            if (wn * dt < 1e-12f) {
                dq0 = 1.f;
                dqs = 0.5f * dt;
            } else {
                float sh, ch;
                sincosf(0.5f * wn * dt, &sh, &ch);
                dq0 = ch;
                dqs = sh / wn;
            }
            const float dx = dqs * w.x, dy = dqs * w.y, dz = dqs * w.z;
            const float nw = qw * dq0 - qx * dx - qy * dy - qz * dz;
            const float nx = qw * dx + qx * dq0 + qy * dz - qz * dy;
            const float ny = qw * dy - qx * dz + qy * dq0 + qz * dx;
            const float nz = qw * dz + qx * dy - qy * dx + qz * dq0;
            const float inv = 1.f / sqrtf(nw * nw + nx * nx + ny * ny + nz * nz);
            qw = nw * inv;
            qx = nx * inv;
            qy = ny * inv;
            qz = nz * inv;
        }
    }
    if (xf) {
        if (g == 0) {
            xf[0] = p.x;
            xf[1] = p.y;
            xf[2] = p.z;
            xf[3] = qw;
            xf[4] = qx;
            xf[5] = qy;
            xf[6] = qz;
            xf[nq] = vl.x;
            xf[nq + 1] = vl.y;
            xf[nq + 2] = vl.z;
            xf[nq + 3] = w.x;
            xf[nq + 4] = w.y;
            xf[nq + 5] = w.z;
        }
#pragma unroll
        for (int j = 0; j < LLEN; ++j) {
            xf[7 + b0 - 1 + j] = q[j];
            xf[nq + 6 + b0 - 1 + j] = qd[j];
        }
    }
    return sum;
}

}  // namespace mppi

/*
 * FP64 CPU oracle of the Hermite-spline MPPI hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load this file's library. The product (the CUDA library) shares no
 * code with it and never calls it.
 *
 * Plain, slow, obviously correct: every quantity in real precision, 6x6 spatial
 * matrices written out densely, no blocking or fusion beyond what the method states.
 * Sections follow the paper ("Reference-Free Sampling-Based Model Predictive
 * Control", arXiv 2511.19204):
 *
 *   noise      Sec. III-B Eq. (overall-noise-kernel) as a per-knot std-dev table and
 *              Alg. 1 sampling step: theta_n = theta + sigma_k * scale * eps, n >= 1;
 *              sample 0 is the unperturbed nominal. eps from Philox4x32-10 (Salmon et
 *              al., SC'11) and the Box-Muller transform (Box & Muller 1958).
 *   clamp      Sec. III-A Eq. (vel-clamp).
 *   spline     Sec. III-A Eq. (hermite_segment) and the Hermite basis; the velocity
 *              setpoint is the analytic time derivative of the position spline.
 *   PD         Sec. III-C Eq. (pd-controller), torques clipped to actuator limits.
 *   dynamics   floating-base articulated-body algorithm (Featherstone, Rigid Body
 *              Dynamics Algorithms, 2008, ch. 7 and 9) with soft spring-damper ground
 *              contact and smooth Coulomb friction, semi-implicit Euler; these stand in
 *              for the paper's simulator (Sec. III-C, Sec. IV-A).
 *              CRBA + RNEA (ibid. ch. 5-6) are here only as an independent check.
 *   cost       Sec. IV-A cost sum S = sum_{h<H} c(x_h, u_h) + c_T(x_H): the quadratic
 *              running terms of the synthetic workloads plus the paper's modular
 *              running and terminal cost (zero weights disable a term).
 *   weights    Sec. III-C Eq. (omega-weights) and the min-max normalised
 *              Eq. (softmax_minmax), evaluated as a log-sum-exp.
 *   average    Sec. III-C Eq. (update-nominal) on the knots.
 *   solve      Alg. 1 iterations with best-trajectory tracking (Sec. III-D).
 *
 * Parity of the whole solve against the paper is unpinned (the paper's simulator and
 * robots are not available); each part above is pinned by the tests separately.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXB 64
#define ORC_MAXNV (6 + ORC_MAXB)

/* The scalar of all arithmetic: double. The operation-counting build (count.cc, test
 * infrastructure for the work per rollout step) compiles this file as C++ with `real` a
 * double-sized type that counts the operations it performs, and ORC_PHASE naming the
 * algorithm's phase they belong to; here ORC_PHASE does nothing. */
#ifndef ORC_COUNTING
typedef double real;
#define ORC_PHASE(p) ((void)0)
#endif
enum { PH_SPLINE, PH_PD, PH_PASS1, PH_CONTACT, PH_BIAS, PH_PASS2, PH_SOLVE, PH_PASS3, PH_COST, PH_INTEGRATE,
       PH_OTHER, PH_COUNT };

typedef struct {
    int32_t nb, nc, fixed_base, cost_body;
    const int32_t* parent;     /* [nb] */
    const real* axis;        /* [nb][3] */
    const real* jpos;        /* [nb][3] */
    const real* mass;        /* [nb] */
    const real* com;         /* [nb][3] */
    const real* inertia;     /* [nb][6] Ixx Iyy Izz Ixy Ixz Iyz about the com */
    const real* armature;    /* [nb] */
    const real* q_min;       /* [nb-1] */
    const real* q_max;       /* [nb-1] */
    const real* kp;          /* [nb-1] */
    const real* kd;          /* [nb-1] */
    const real* tau_max;     /* [nb-1] */
    const int32_t* contact_body; /* [nc] */
    const real* contact_pos;   /* [nc][3] */
    real contact_k, contact_c, mu, eps_f, gravity;
    real z_des, vx_des, w_z, w_vx, w_tilt, w_tau;
    /* modular cost of Sec. IV-A */
    real w_h, w_orient, w_q, w_cvel, w_cforce, w_term;
    real quat_des[4];        /* (w, x, y, z), unit */
    real f0[3];
    real pdot_des[3];
    const real* q0;          /* [nb-1] or NULL (zeros) */
} orc_model;

/* ------------------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).           */
/* ------------------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Sec. III-B Eq. (overall-noise-kernel): the isotropic per-knot factor
 * exp(-(I - i)/(beta1 I) - (K - k)/(beta2 K)) for iterations i = I..1 and knots
 * k = 0..K-1, used as the standard-deviation factor sigma[it][k] with it = I - i (so the
 * first iteration, i = I, is row 0), times `scale`. out [iters][knots]. */
void orc_noise_schedule(int iters, int knots, real beta1, real beta2, real scale, real* out) {
    for (int it = 0; it < iters; ++it) {
        int i = iters - it;
        for (int k = 0; k < knots; ++k)
            out[it * knots + k] =
                scale * exp(-(real)(iters - i) / (beta1 * iters) - (real)(knots - k) / (beta2 * knots));
    }
}

/* Box-Muller on two 32-bit words: u1 in (0,1], u2 in [0,1). */
static void box_muller(uint32_t wa, uint32_t wb, real* ea, real* eb) {
    const real two_m24 = 1.0 / 16777216.0;
    real u1 = ((real)(wa >> 8) + 1.0) * two_m24;
    real u2 = (real)(wb >> 8) * two_m24;
    real r = sqrt(-2.0 * log(u1));
    real ang = 2.0 * M_PI * u2;
    *ea = r * cos(ang);
    *eb = r * sin(ang);
}

/* Standard normal eps for one element e of sample n (n >= 1):
 * counter = (e/4, n, iteration counter, instance), key = (seed lo, seed hi);
 * element pairs (2m, 2m+1) share one Box-Muller draw from words (e%4 & ~1, +1). */
real orc_normal(uint64_t seed, uint32_t iter_ctr, uint32_t inst, uint32_t n, uint32_t e) {
    uint32_t ctr[4] = {e / 4u, n, iter_ctr, inst};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox(ctr, key, w);
    uint32_t j = (e % 4u) & ~1u;
    real ea, eb;
    box_muller(w[j], w[j + 1], &ea, &eb);
    return (e & 1u) ? eb : ea;
}

/* Knot spacing of nk uniform knots over H steps of dt, both endpoints included. */
static real knot_dt(int nk, int H, real dt) { return (real)H * dt / (real)(nk - 1); }

/* Sec. III-A Eq. (vel-clamp): clip theta^q into the limits, then bound |theta^v| by the
 * distance to the nearest limit over half a knot interval. Only joints with a finite
 * limit are clamped. knots: [nk][2][nu]. */
void orc_clamp(int nu, int nk, real dtk, const real* qmin, const real* qmax, real* kn) {
    for (int k = 0; k < nk; ++k)
        for (int j = 0; j < nu; ++j) {
            real lo = qmin[j], hi = qmax[j];
            if (!isfinite(lo) && !isfinite(hi)) continue;
            real* q = &kn[(k * 2 + 0) * nu + j];
            real* v = &kn[(k * 2 + 1) * nu + j];
            if (*q < lo) *q = lo;
            if (*q > hi) *q = hi;
            real room = fmin(hi - *q, *q - lo);
            real vmax = room / (dtk / 2.0);
            if (*v > vmax) *v = vmax;
            if (*v < -vmax) *v = -vmax;
        }
}

/* Alg. 1 sampling: theta_{n,k} ~ N(theta_k, sigma_k * scale) for n in [1, N), sample 0
 * is the nominal itself; then the clamp (when the model has finite limits).
 * nominal [E], sigma_row [nk], out [N][E], E = nk*2*nu.
 * scale_v <= 0 selects the default 1/knot-spacing. */
void orc_sample_knots(int nu, int nk, int N, int H, real dt, const real* nominal,
                      const real* sigma_row, real scale_q, real scale_v, uint64_t seed,
                      uint32_t iter_ctr, uint32_t inst, const real* qmin, const real* qmax,
                      real* out) {
    const int E = nk * 2 * nu;
    const real dtk = knot_dt(nk, H, dt);
    if (scale_v <= 0.0) scale_v = 1.0 / dtk;
    for (int n = 0; n < N; ++n) {
        real* kn = out + (size_t)n * E;
        for (int e = 0; e < E; ++e) {
            int k = e / (2 * nu);
            int p = (e / nu) % 2;
            real eps = (n == 0) ? 0.0 : orc_normal(seed, iter_ctr, inst, (uint32_t)n, (uint32_t)e);
            kn[e] = nominal[e] + sigma_row[k] * (p == 0 ? scale_q : scale_v) * eps;
        }
        if (qmin && qmax) orc_clamp(nu, nk, dtk, qmin, qmax, kn);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Cubic Hermite spline (Sec. III-A Eq. hermite_segment).                               */
/* ------------------------------------------------------------------------------------ */
/* Segment and local time for step h: r = h*(nk-1); k = floor(r/H) (<= nk-2);
 * s = (r - k*H)/H = (t_h - t_k)/knot spacing, t_h = h*dt. */
void orc_segment(int h, int H, int nk, int* k_out, real* s_out) {
    long r = (long)h * (long)(nk - 1);
    long k = r / H;
    if (k > nk - 2) k = nk - 2;
    *k_out = (int)k;
    *s_out = (real)(r - k * (long)H) / (real)H;
}

/* q(s) and dq/dt on one segment with knot spacing dtk. */
void orc_hermite(real s, real dtk, real q0, real v0, real q1, real v1,
                 real* q, real* qdot) {
    real s2 = s * s, s3 = s2 * s;
    real h00 = 2 * s3 - 3 * s2 + 1, h10 = s3 - 2 * s2 + s;
    real h01 = -2 * s3 + 3 * s2, h11 = s3 - s2;
    real d00 = 6 * s2 - 6 * s, d10 = 3 * s2 - 4 * s + 1;
    real d01 = -6 * s2 + 6 * s, d11 = 3 * s2 - 2 * s;
    *q = h00 * q0 + h10 * dtk * v0 + h01 * q1 + h11 * dtk * v1;
    *qdot = (d00 * q0 + d01 * q1) / dtk + d10 * v0 + d11 * v1;
}

/* ------------------------------------------------------------------------------------ */
/* Small dense linear algebra                                                            */
/* ------------------------------------------------------------------------------------ */
typedef real m3[3][3];
typedef real m6[6][6];

static void m3_mul(const m3 a, const m3 b, m3 c) {
    m3 t;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            t[i][j] = 0;
            for (int k = 0; k < 3; ++k) t[i][j] += a[i][k] * b[k][j];
        }
    memcpy(c, t, sizeof(m3));
}
static void m3_vec(const m3 a, const real* x, real* y) {
    real t[3];
    for (int i = 0; i < 3; ++i) t[i] = a[i][0] * x[0] + a[i][1] * x[1] + a[i][2] * x[2];
    memcpy(y, t, sizeof t);
}
static void m3_tvec(const m3 a, const real* x, real* y) {
    real t[3];
    for (int i = 0; i < 3; ++i) t[i] = a[0][i] * x[0] + a[1][i] * x[1] + a[2][i] * x[2];
    memcpy(y, t, sizeof t);
}
static void cross3(const real* a, const real* b, real* c) {
    real t[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    memcpy(c, t, sizeof t);
}
static void skew(const real* a, m3 s) {
    s[0][0] = 0; s[0][1] = -a[2]; s[0][2] = a[1];
    s[1][0] = a[2]; s[1][1] = 0; s[1][2] = -a[0];
    s[2][0] = -a[1]; s[2][1] = a[0]; s[2][2] = 0;
}
/* Rodrigues: rotation about unit axis a by angle t (child -> parent coordinates). */
static void axis_angle(const real* a, real t, m3 R) {
    m3 K, K2;
    skew(a, K);
    m3_mul(K, K, K2);
    real s = sin(t), c = cos(t);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[i][j] = (i == j ? 1.0 : 0.0) + s * K[i][j] + (1 - c) * K2[i][j];
}
static void quat_to_R(const real* q, m3 R) {
    real w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}
static void m6_zero(m6 a) { memset(a, 0, sizeof(m6)); }
static void m6_mul(const m6 a, const m6 b, m6 c) {
    m6 t;
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            real s = 0;
            for (int k = 0; k < 6; ++k) s += a[i][k] * b[k][j];
            t[i][j] = s;
        }
    memcpy(c, t, sizeof(m6));
}
static void m6_tmul(const m6 a, const m6 b, m6 c) { /* c = a^T b */
    m6 t;
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            real s = 0;
            for (int k = 0; k < 6; ++k) s += a[k][i] * b[k][j];
            t[i][j] = s;
        }
    memcpy(c, t, sizeof(m6));
}
static void m6_vec(const m6 a, const real* x, real* y) {
    real t[6];
    for (int i = 0; i < 6; ++i) {
        real s = 0;
        for (int k = 0; k < 6; ++k) s += a[i][k] * x[k];
        t[i] = s;
    }
    memcpy(y, t, sizeof t);
}
static void m6_tvec(const m6 a, const real* x, real* y) {
    real t[6];
    for (int i = 0; i < 6; ++i) {
        real s = 0;
        for (int k = 0; k < 6; ++k) s += a[k][i] * x[k];
        t[i] = s;
    }
    memcpy(y, t, sizeof t);
}
/* Solve A x = b for a symmetric positive definite n x n matrix (Cholesky). */
static int spd_solve(int n, const real* A, const real* b, real* x) {
    real L[ORC_MAXNV * ORC_MAXNV];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            real s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            if (i == j) {
                if (!(s > 0)) return -1;
                L[i * n + i] = sqrt(s);
            } else {
                L[i * n + j] = s / L[j * n + j];
            }
        }
    real y[ORC_MAXNV];
    for (int i = 0; i < n; ++i) {
        real s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
        y[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        real s = y[i];
        for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
        x[i] = s / L[i * n + i];
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Spatial algebra (Featherstone): motion (w, v), force (n, f), body coordinates.       */
/* ------------------------------------------------------------------------------------ */
/* Plucker transform parent -> child: X = [E 0; -E [r]x  E], E = rotation parent->child
 * coordinates, r = child origin in parent coordinates. */
static void plucker(const m3 E, const real* r, m6 X) {
    m3 S, ES;
    skew(r, S);
    m3_mul(E, S, ES);
    m6_zero(X);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            X[i][j] = E[i][j];
            X[3 + i][3 + j] = E[i][j];
            X[3 + i][j] = -ES[i][j];
        }
}
/* Rigid-body spatial inertia about the body origin. */
static void body_inertia(const orc_model* m, int b, m6 I) {
    const real* c = &m->com[3 * b];
    const real* ic = &m->inertia[6 * b];
    real mass = m->mass[b];
    m3 Ic = {{ic[0], ic[3], ic[4]}, {ic[3], ic[1], ic[5]}, {ic[4], ic[5], ic[2]}};
    m3 C, CCt;
    skew(c, C);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            real s = 0;
            for (int k = 0; k < 3; ++k) s += C[i][k] * C[j][k]; /* C C^T */
            CCt[i][j] = s;
        }
    m6_zero(I);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            I[i][j] = Ic[i][j] + mass * CCt[i][j];
            I[i][3 + j] = mass * C[i][j];
            I[3 + i][j] = mass * C[j][i];
            I[3 + i][3 + j] = (i == j) ? mass : 0.0;
        }
}
static void crm(const real* a, const real* b, real* c) { /* motion x motion */
    real t[6], u[3];
    cross3(a, b, t);
    cross3(a, b + 3, t + 3);
    cross3(a + 3, b, u);
    t[3] += u[0]; t[4] += u[1]; t[5] += u[2];
    memcpy(c, t, sizeof t);
}
static void crf(const real* a, const real* f, real* c) { /* motion x* force */
    real t[6], u[3];
    cross3(a, f, t);
    cross3(a + 3, f + 3, u);
    t[0] += u[0]; t[1] += u[1]; t[2] += u[2];
    cross3(a, f + 3, t + 3);
    memcpy(c, t, sizeof t);
}

/* ------------------------------------------------------------------------------------ */
/* Kinematics, contact forces                                                            */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    m6 X[ORC_MAXB];          /* parent -> body transform */
    m3 R[ORC_MAXB];          /* body -> world rotation */
    real p[ORC_MAXB][3];   /* body origin, world */
    real v[ORC_MAXB][6];   /* spatial velocity, body coordinates */
    real fext[ORC_MAXB][6];/* external spatial force, body coordinates */
} orc_kin;

static void kinematics(const orc_model* m, const real* x, orc_kin* K) {
    const int nb = m->nb, nj = nb - 1, nq = 7 + nj;
    const real* q = x + 7;
    const real* vb = x + nq;       /* v_lin(3), omega(3), body frame */
    const real* qd = x + nq + 6;
    ORC_PHASE(PH_PASS1);
    quat_to_R(x + 3, K->R[0]);
    memcpy(K->p[0], x, 3 * sizeof(real));
    K->v[0][0] = vb[3]; K->v[0][1] = vb[4]; K->v[0][2] = vb[5];
    K->v[0][3] = vb[0]; K->v[0][4] = vb[1]; K->v[0][5] = vb[2];
    if (m->fixed_base) memset(K->v[0], 0, 6 * sizeof(real));
    for (int i = 1; i < nb; ++i) {
        int l = m->parent[i];
        m3 Rj, E;
        axis_angle(&m->axis[3 * i], q[i - 1], Rj);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) E[a][b] = Rj[b][a];
        plucker(E, &m->jpos[3 * i], K->X[i]);
        m3_mul(K->R[l], Rj, K->R[i]);
        real t[3];
        m3_vec(K->R[l], &m->jpos[3 * i], t);
        for (int a = 0; a < 3; ++a) K->p[i][a] = K->p[l][a] + t[a];
        m6_vec(K->X[i], K->v[l], K->v[i]);
        for (int a = 0; a < 3; ++a) K->v[i][a] += m->axis[3 * i + a] * qd[i - 1];
    }
    for (int i = 0; i < nb; ++i) memset(K->fext[i], 0, 6 * sizeof(real));
    ORC_PHASE(PH_CONTACT);
    /* soft ground contact on the plane z = 0 */
    for (int c = 0; c < m->nc; ++c) {
        int b = m->contact_body[c];
        const real* rc = &m->contact_pos[3 * c];
        real pw[3], vloc[3], vw[3], t[3];
        m3_vec(K->R[b], rc, t);
        for (int a = 0; a < 3; ++a) pw[a] = K->p[b][a] + t[a];
        cross3(K->v[b], rc, vloc); /* w x r */
        for (int a = 0; a < 3; ++a) vloc[a] += K->v[b][3 + a];
        m3_vec(K->R[b], vloc, vw);
        real depth = -pw[2];
        if (depth <= 0) continue;
        real fn = m->contact_k * depth - m->contact_c * vw[2];
        if (fn < 0) fn = 0;
        real vt2 = vw[0] * vw[0] + vw[1] * vw[1];
        real scale = -m->mu * fn / sqrt(vt2 + m->eps_f * m->eps_f);
        real F[3] = {scale * vw[0], scale * vw[1], fn};
        real fb[3], nb3[3];
        m3_tvec(K->R[b], F, fb);
        cross3(rc, fb, nb3);
        for (int a = 0; a < 3; ++a) {
            K->fext[b][a] += nb3[a];
            K->fext[b][3 + a] += fb[a];
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Articulated-body algorithm (floating or fixed base, gravity as a base offset).       */
/* acc[nv] = (base spatial acceleration (w_dot, v_dot) in body coordinates, qdd).       */
/* For a fixed base the base part is zero.                                               */
/* ------------------------------------------------------------------------------------ */
static int aba(const orc_model* m, const real* x, const real* tau, orc_kin* K, real* acc) {
    const int nb = m->nb, nj = nb - 1, nq = 7 + nj;
    const real* qd = x + nq + 6;
    static __thread m6 IA[ORC_MAXB];
    real pA[ORC_MAXB][6], c[ORC_MAXB][6], U[ORC_MAXB][6], D[ORC_MAXB], u[ORC_MAXB];
    real a[ORC_MAXB][6];
    kinematics(m, x, K);
    ORC_PHASE(PH_BIAS);
    for (int i = 0; i < nb; ++i) {
        m6 I;
        real Iv[6];
        body_inertia(m, i, I);
        memcpy(IA[i], I, sizeof(m6));
        m6_vec(I, K->v[i], Iv);
        crf(K->v[i], Iv, pA[i]);
        for (int k = 0; k < 6; ++k) pA[i][k] -= K->fext[i][k];
        memset(c[i], 0, sizeof c[i]);
        if (i > 0) {
            real Sq[6] = {0};
            for (int k = 0; k < 3; ++k) Sq[k] = m->axis[3 * i + k] * qd[i - 1];
            crm(K->v[i], Sq, c[i]);
        }
    }
    ORC_PHASE(PH_PASS2);
    for (int i = nb - 1; i >= 1; --i) {
        const real* S = &m->axis[3 * i]; /* S = (axis, 0) */
        for (int k = 0; k < 6; ++k) U[i][k] = IA[i][k][0] * S[0] + IA[i][k][1] * S[1] + IA[i][k][2] * S[2];
        D[i] = S[0] * U[i][0] + S[1] * U[i][1] + S[2] * U[i][2] + m->armature[i];
        u[i] = tau[i - 1] - (S[0] * pA[i][0] + S[1] * pA[i][1] + S[2] * pA[i][2]);
        m6 Ia, tmp, XtIaX;
        real pa[6], Iac[6], Xtpa[6];
        for (int r = 0; r < 6; ++r)
            for (int s = 0; s < 6; ++s) Ia[r][s] = IA[i][r][s] - U[i][r] * U[i][s] / D[i];
        m6_vec(Ia, c[i], Iac);
        for (int k = 0; k < 6; ++k) pa[k] = pA[i][k] + Iac[k] + U[i][k] * u[i] / D[i];
        m6_mul(Ia, K->X[i], tmp);
        m6_tmul(K->X[i], tmp, XtIaX);
        m6_tvec(K->X[i], pa, Xtpa);
        int l = m->parent[i];
        for (int r = 0; r < 6; ++r) {
            for (int s = 0; s < 6; ++s) IA[l][r][s] += XtIaX[r][s];
            pA[l][r] += Xtpa[r];
        }
    }
    ORC_PHASE(PH_SOLVE);
    /* gravity offset: a' = a - a_g, a_g = (0, R0^T g) */
    real g_w[3] = {0, 0, -m->gravity}, g_b[3];
    m3_tvec(K->R[0], g_w, g_b);
    if (m->fixed_base) {
        a[0][0] = a[0][1] = a[0][2] = 0;
        a[0][3] = -g_b[0]; a[0][4] = -g_b[1]; a[0][5] = -g_b[2];
    } else {
        real rhs[6];
        for (int k = 0; k < 6; ++k) rhs[k] = -pA[0][k];
        if (spd_solve(6, &IA[0][0][0], rhs, a[0]) != 0) return -1;
    }
    ORC_PHASE(PH_PASS3);
    for (int i = 1; i < nb; ++i) {
        const real* S = &m->axis[3 * i];
        int l = m->parent[i];
        real ap[6];
        m6_vec(K->X[i], a[l], ap);
        for (int k = 0; k < 6; ++k) ap[k] += c[i][k];
        real qdd = (u[i] - (U[i][0] * ap[0] + U[i][1] * ap[1] + U[i][2] * ap[2] + U[i][3] * ap[3] +
                              U[i][4] * ap[4] + U[i][5] * ap[5])) / D[i];
        for (int k = 0; k < 6; ++k) a[i][k] = ap[k];
        for (int k = 0; k < 3; ++k) a[i][k] += S[k] * qdd;
        acc[6 + i - 1] = qdd;
    }
    if (m->fixed_base) {
        for (int k = 0; k < 6; ++k) acc[k] = 0;
    } else {
        for (int k = 0; k < 3; ++k) acc[k] = a[0][k];
        for (int k = 0; k < 3; ++k) acc[3 + k] = a[0][3 + k] + g_b[k];
    }
    return 0;
}

/* Joint-space mass matrix by the composite-rigid-body algorithm (check only).
 * Generalised velocity = (base (w, v) body coordinates [floating only], qdot). */
int orc_crba(const orc_model* mdl, const real* x, real* M) {
    const int nb = mdl->nb, nj = nb - 1;
    const int off = mdl->fixed_base ? 0 : 6;
    const int n = off + nj;
    static __thread orc_kin K;
    m6 Ic[ORC_MAXB];
    kinematics(mdl, x, &K);
    for (int i = 0; i < nb; ++i) body_inertia(mdl, i, Ic[i]);
    for (int i = nb - 1; i >= 1; --i) {
        m6 t, XtIX;
        m6_mul(Ic[i], K.X[i], t);
        m6_tmul(K.X[i], t, XtIX);
        int l = mdl->parent[i];
        for (int r = 0; r < 6; ++r)
            for (int s = 0; s < 6; ++s) Ic[l][r][s] += XtIX[r][s];
    }
    memset(M, 0, sizeof(real) * n * n);
    if (!mdl->fixed_base)
        for (int r = 0; r < 6; ++r)
            for (int s = 0; s < 6; ++s) M[r * n + s] = Ic[0][r][s];
    for (int i = 1; i < nb; ++i) {
        const real* S = &mdl->axis[3 * i];
        real F[6];
        for (int k = 0; k < 6; ++k) F[k] = Ic[i][k][0] * S[0] + Ic[i][k][1] * S[1] + Ic[i][k][2] * S[2];
        int di = off + i - 1;
        M[di * n + di] = S[0] * F[0] + S[1] * F[1] + S[2] * F[2] + mdl->armature[i];
        int j = i;
        while (mdl->parent[j] > 0) {
            real t[6];
            m6_tvec(K.X[j], F, t);
            memcpy(F, t, sizeof t);
            j = mdl->parent[j];
            const real* Sj = &mdl->axis[3 * j];
            int dj = off + j - 1;
            real val = Sj[0] * F[0] + Sj[1] * F[1] + Sj[2] * F[2];
            M[di * n + dj] = val;
            M[dj * n + di] = val;
        }
        if (!mdl->fixed_base) {
            real t[6];
            m6_tvec(K.X[j], F, t); /* j's parent is the base */
            for (int k = 0; k < 6; ++k) {
                M[di * n + k] = t[k];
                M[k * n + di] = t[k];
            }
        }
    }
    return n;
}

/* Bias forces h(q, v) (Coriolis, gravity, minus contact forces) by the recursive
 * Newton-Euler algorithm with zero generalised acceleration (check only). */
int orc_rnea_bias(const orc_model* mdl, const real* x, real* h) {
    const int nb = mdl->nb;
    const int off = mdl->fixed_base ? 0 : 6;
    static __thread orc_kin K;
    real a[ORC_MAXB][6], f[ORC_MAXB][6];
    const int nj = nb - 1, nq = 7 + nj;
    const real* qd = x + nq + 6;
    kinematics(mdl, x, &K);
    real g_w[3] = {0, 0, -mdl->gravity}, g_b[3];
    m3_tvec(K.R[0], g_w, g_b);
    a[0][0] = a[0][1] = a[0][2] = 0;
    a[0][3] = -g_b[0]; a[0][4] = -g_b[1]; a[0][5] = -g_b[2];
    for (int i = 0; i < nb; ++i) {
        if (i > 0) {
            int l = mdl->parent[i];
            real Sq[6] = {0}, cc[6];
            for (int k = 0; k < 3; ++k) Sq[k] = mdl->axis[3 * i + k] * qd[i - 1];
            crm(K.v[i], Sq, cc);
            m6_vec(K.X[i], a[l], a[i]);
            for (int k = 0; k < 6; ++k) a[i][k] += cc[k];
        }
        m6 I;
        real Ia[6], Iv[6], vxIv[6];
        body_inertia(mdl, i, I);
        m6_vec(I, a[i], Ia);
        m6_vec(I, K.v[i], Iv);
        crf(K.v[i], Iv, vxIv);
        for (int k = 0; k < 6; ++k) f[i][k] = Ia[k] + vxIv[k] - K.fext[i][k];
    }
    for (int i = nb - 1; i >= 1; --i) {
        const real* S = &mdl->axis[3 * i];
        h[off + i - 1] = S[0] * f[i][0] + S[1] * f[i][1] + S[2] * f[i][2];
        real t[6];
        m6_tvec(K.X[i], f[i], t);
        int l = mdl->parent[i];
        for (int k = 0; k < 6; ++k) f[l][k] += t[k];
    }
    if (!mdl->fixed_base)
        for (int k = 0; k < 6; ++k) h[k] = f[0][k];
    return off + nj;
}

/* Generalised accelerations from ABA. acc[nv]: base (w_dot, v_dot) then qdd. */
int orc_forward_dynamics(const orc_model* m, const real* x, const real* tau, real* acc) {
    static __thread orc_kin K;
    return aba(m, x, tau, &K, acc);
}

/* Contact forces in the world frame for every contact point: out [nc][3]. */
void orc_contact_forces(const orc_model* m, const real* x, real* out) {
    static __thread orc_kin K;
    kinematics(m, x, &K);
    for (int c = 0; c < m->nc; ++c) {
        int b = m->contact_body[c];
        const real* rc = &m->contact_pos[3 * c];
        real pw[3], vloc[3], vw[3], t[3];
        m3_vec(K.R[b], rc, t);
        for (int a = 0; a < 3; ++a) pw[a] = K.p[b][a] + t[a];
        cross3(K.v[b], rc, vloc);
        for (int a = 0; a < 3; ++a) vloc[a] += K.v[b][3 + a];
        m3_vec(K.R[b], vloc, vw);
        real depth = -pw[2];
        out[3 * c] = out[3 * c + 1] = out[3 * c + 2] = 0;
        if (depth <= 0) continue;
        real fn = m->contact_k * depth - m->contact_c * vw[2];
        if (fn < 0) fn = 0;
        real vt2 = vw[0] * vw[0] + vw[1] * vw[1];
        real scale = -m->mu * fn / sqrt(vt2 + m->eps_f * m->eps_f);
        out[3 * c] = scale * vw[0];
        out[3 * c + 1] = scale * vw[1];
        out[3 * c + 2] = fn;
    }
}

/* World position of every body origin and contact point: bodies [nb][3], contacts [nc][3]. */
void orc_positions(const orc_model* m, const real* x, real* bodies, real* contacts) {
    static __thread orc_kin K;
    kinematics(m, x, &K);
    for (int b = 0; b < m->nb; ++b)
        for (int a = 0; a < 3; ++a) bodies[3 * b + a] = K.p[b][a];
    for (int c = 0; c < m->nc; ++c) {
        int b = m->contact_body[c];
        real t[3];
        m3_vec(K.R[b], &m->contact_pos[3 * c], t);
        for (int a = 0; a < 3; ++a) contacts[3 * c + a] = K.p[b][a] + t[a];
    }
}

/* Kinetic + gravitational potential energy (check only). */
real orc_energy(const orc_model* m, const real* x) {
    static __thread orc_kin K;
    kinematics(m, x, &K);
    real e = 0;
    for (int i = 0; i < m->nb; ++i) {
        m6 I;
        real Iv[6];
        body_inertia(m, i, I);
        m6_vec(I, K.v[i], Iv);
        for (int k = 0; k < 6; ++k) e += 0.5 * K.v[i][k] * Iv[k];
        real cw[3];
        m3_vec(K.R[i], &m->com[3 * i], cw);
        e += m->mass[i] * m->gravity * (K.p[i][2] + cw[2]);
    }
    for (int i = 1; i < m->nb; ++i) {
        real qd = x[7 + m->nb - 1 + 6 + i - 1];
        e += 0.5 * m->armature[i] * qd * qd;
    }
    return e;
}

/* ------------------------------------------------------------------------------------ */
/* PD tracking, running cost, semi-implicit Euler                                       */
/* ------------------------------------------------------------------------------------ */
/* Sec. III-C Eq. (pd-controller), clipped to +-tau_max. */
static void pd_torque(const orc_model* m, const real* x, const real* qref, const real* vref,
                      real* tau) {
    const int nj = m->nb - 1, nq = 7 + nj;
    for (int j = 0; j < nj; ++j) {
        real t = m->kp[j] * (qref[j] - x[7 + j]) + m->kd[j] * (vref[j] - x[nq + 6 + j]);
        if (t > m->tau_max[j]) t = m->tau_max[j];
        if (t < -m->tau_max[j]) t = -m->tau_max[j];
        tau[j] = t;
    }
}

/* Running cost c(x_h, u_h): w_z (z - z_des)^2 + w_vx (vx - vx_des)^2 + w_tilt tilt^2 +
 * w_tau |tau|^2, z and tilt of the cost body, vx = world x-velocity of the base origin,
 * tilt = angle between the cost body's z axis and the world z axis. */
static real running_cost(const orc_model* m, const real* x, const orc_kin* K, const real* tau) {
    const int nj = m->nb - 1, nq = 7 + nj;
    int b = m->cost_body;
    real z = K->p[b][2];
    real tilt = atan2(sqrt(K->R[b][0][2] * K->R[b][0][2] + K->R[b][1][2] * K->R[b][1][2]), K->R[b][2][2]);
    real vw[3];
    m3_vec(K->R[0], x + nq, vw);
    real vx = m->fixed_base ? 0.0 : vw[0];
    real tt = 0;
    for (int j = 0; j < nj; ++j) tt += tau[j] * tau[j];
    return m->w_z * (z - m->z_des) * (z - m->z_des) + m->w_vx * (vx - m->vx_des) * (vx - m->vx_des) +
           m->w_tilt * tilt * tilt + m->w_tau * tt;
}

/* Modular running cost of Sec. IV-A (Eq. running cost), on the pre-step state:
 *   w_h |p_base,z - z_des| + w_orient ||log3(R_base^T R_des)||^2 + w_q ||q - q0||^2
 *   + w_cvel sum_{c in contact} ||v_c||_1 + w_cforce sum_c ||f_c - f0||_1.
 * ||log3(R_base^T R_des)|| is the rotation angle of the relative quaternion
 * conj(q_base) * q_des: 2 atan2(|vector part|, |scalar part|). A contact point is in
 * contact when it penetrates the ground (depth > 0); v_c is its world velocity and f_c
 * its world contact force (zero when not in contact). */
static real modular_cost(const orc_model* m, const real* x, const orc_kin* K) {
    const int nj = m->nb - 1;
    real S = 0;
    S += m->w_h * fabs(x[2] - m->z_des);
    const real* qb = x + 3;
    const real* qd = m->quat_des;
    /* conj(qb) * qd */
    real rw = qb[0] * qd[0] + qb[1] * qd[1] + qb[2] * qd[2] + qb[3] * qd[3];
    real rx = qb[0] * qd[1] - qb[1] * qd[0] - qb[2] * qd[3] + qb[3] * qd[2];
    real ry = qb[0] * qd[2] + qb[1] * qd[3] - qb[2] * qd[0] - qb[3] * qd[1];
    real rz = qb[0] * qd[3] - qb[1] * qd[2] + qb[2] * qd[1] - qb[3] * qd[0];
    real th = 2.0 * atan2(sqrt(rx * rx + ry * ry + rz * rz), fabs(rw));
    S += m->w_orient * th * th;
    for (int j = 0; j < nj; ++j) {
        real d = x[7 + j] - (m->q0 ? m->q0[j] : 0.0);
        S += m->w_q * d * d;
    }
    for (int c = 0; c < m->nc; ++c) {
        int b = m->contact_body[c];
        const real* rc = &m->contact_pos[3 * c];
        real pw[3], vloc[3], vw[3], t[3], F[3] = {0, 0, 0};
        m3_vec(K->R[b], rc, t);
        for (int a = 0; a < 3; ++a) pw[a] = K->p[b][a] + t[a];
        cross3(K->v[b], rc, vloc);
        for (int a = 0; a < 3; ++a) vloc[a] += K->v[b][3 + a];
        m3_vec(K->R[b], vloc, vw);
        if (-pw[2] > 0) {
            real fn = m->contact_k * (-pw[2]) - m->contact_c * vw[2];
            if (fn < 0) fn = 0;
            real sc = -m->mu * fn / sqrt(vw[0] * vw[0] + vw[1] * vw[1] + m->eps_f * m->eps_f);
            F[0] = sc * vw[0];
            F[1] = sc * vw[1];
            F[2] = fn;
            S += m->w_cvel * (fabs(vw[0]) + fabs(vw[1]) + fabs(vw[2]));
        }
        S += m->w_cforce * (fabs(F[0] - m->f0[0]) + fabs(F[1] - m->f0[1]) + fabs(F[2] - m->f0[2]));
    }
    return S;
}

/* Terminal cost of Sec. IV-A (Eq. terminal cost): w_term ||p_base(x_H) - p_target||_1,
 * p_target = p_base(x_0) + pdot_des H dt. */
static real terminal_cost(const orc_model* m, const real* x0, const real* xH, int H, real dt) {
    real S = 0;
    for (int a = 0; a < 3; ++a) S += fabs(xH[a] - (x0[a] + m->pdot_des[a] * H * dt));
    return m->w_term * S;
}

/* Semi-implicit Euler: velocities first, then positions with the new velocities; base
 * orientation by the quaternion exponential of the new body angular velocity. */
static void integrate(const orc_model* m, real* x, const real* acc, real dt) {
    const int nj = m->nb - 1, nq = 7 + nj;
    real* vb = x + nq;
    real* qd = x + nq + 6;
    for (int j = 0; j < nj; ++j) {
        qd[j] += dt * acc[6 + j];
        x[7 + j] += dt * qd[j];
    }
    if (m->fixed_base) return;
    /* acc = (w_dot, v_dot); state velocity = (v_lin, omega) */
    for (int k = 0; k < 3; ++k) {
        vb[k] += dt * acc[3 + k];
        vb[3 + k] += dt * acc[k];
    }
    m3 R;
    quat_to_R(x + 3, R);
    real dp[3];
    m3_vec(R, vb, dp);
    for (int k = 0; k < 3; ++k) x[k] += dt * dp[k];
    const real* w = vb + 3;
    real wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    real th = wn * dt;
    real dq[4];
    if (th < 1e-12) {
        dq[0] = 1; dq[1] = 0.5 * dt * w[0]; dq[2] = 0.5 * dt * w[1]; dq[3] = 0.5 * dt * w[2];
    } else {
        real s = sin(0.5 * th) / wn;
        dq[0] = cos(0.5 * th); dq[1] = s * w[0]; dq[2] = s * w[1]; dq[3] = s * w[2];
    }
    real* q = x + 3;
    real r[4] = {q[0] * dq[0] - q[1] * dq[1] - q[2] * dq[2] - q[3] * dq[3],
                   q[0] * dq[1] + q[1] * dq[0] + q[2] * dq[3] - q[3] * dq[2],
                   q[0] * dq[2] - q[1] * dq[3] + q[2] * dq[0] + q[3] * dq[1],
                   q[0] * dq[3] + q[1] * dq[2] - q[2] * dq[1] + q[3] * dq[0]};
    real nrm = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
    for (int k = 0; k < 4; ++k) q[k] = r[k] / nrm;
}

/* One step under a given torque: x <- step(x, tau). Returns 0 or -1 (singular). */
int orc_step(const orc_model* m, real* x, const real* tau, real dt) {
    real acc[ORC_MAXNV];
    static __thread orc_kin K;
    if (aba(m, x, tau, &K, acc) != 0) return -1;
    integrate(m, x, acc, dt);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Position-only spline variants of the ablation (Sec. IV-D, Tab. III)                    */
/* ------------------------------------------------------------------------------------ */
#define ORC_SPLINE_HERMITE 0
#define ORC_SPLINE_CUBIC 1     /* natural cubic spline through the position nodes */
#define ORC_SPLINE_QUADRATIC 2 /* C1 quadratic spline through the nodes, zero initial slope */

/* Natural cubic spline on nodes y[0..K-1] with spacing h: the second derivatives M solve
 * the full K x K system (rows 0 and K-1: M = 0; row k: M_{k-1} + 4 M_k + M_{k+1} =
 * 6 (y_{k+1} - 2 y_k + y_{k-1}) / h^2), by dense Gaussian elimination with partial
 * pivoting. */
static void natural_cubic_moments(int K, real h, const real* y, real* M) {
    real A[32][33];
    for (int r = 0; r < K; ++r) {
        for (int c = 0; c <= K; ++c) A[r][c] = 0;
        if (r == 0 || r == K - 1) {
            A[r][r] = 1;
        } else {
            A[r][r - 1] = 1;
            A[r][r] = 4;
            A[r][r + 1] = 1;
            A[r][K] = 6.0 * (y[r + 1] - 2.0 * y[r] + y[r - 1]) / (h * h);
        }
    }
    for (int c = 0; c < K; ++c) {
        int piv = c;
        for (int r = c + 1; r < K; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (piv != c)
            for (int k = 0; k <= K; ++k) {
                real t = A[c][k];
                A[c][k] = A[piv][k];
                A[piv][k] = t;
            }
        for (int r = c + 1; r < K; ++r) {
            real f = A[r][c] / A[c][c];
            for (int k = c; k <= K; ++k) A[r][k] -= f * A[c][k];
        }
    }
    for (int r = K - 1; r >= 0; --r) {
        real acc = A[r][K];
        for (int k = r + 1; k < K; ++k) acc -= A[r][k] * M[k];
        M[r] = acc / A[r][r];
    }
}

/* C1 quadratic spline through y with zero slope at the first node: on segment k,
 * q(s) = y_k + d_k h s + (y_{k+1} - y_k - d_k h) s^2, so d_{k+1} = q'(end) = 2 (y_{k+1} -
 * y_k) / h - d_k. */
static void quadratic_slopes(int K, real h, const real* y, real* d) {
    d[0] = 0;
    for (int k = 0; k + 1 < K; ++k) d[k + 1] = 2.0 * (y[k + 1] - y[k]) / h - d[k];
}

/* Value and time derivative of joint j's variant spline at segment k, local time s. */
static void variant_eval(int spline, real h, const real* y, const real* aux, int k, real s,
                         real* q, real* qd) {
    if (spline == ORC_SPLINE_QUADRATIC) {
        real a2 = y[k + 1] - y[k] - aux[k] * h;
        *q = y[k] + aux[k] * h * s + a2 * s * s;
        *qd = aux[k] + 2.0 * a2 * s / h;
    } else { /* natural cubic in moment form */
        real u = 1.0 - s;
        *q = u * y[k] + s * y[k + 1] + h * h / 6.0 * ((u * u * u - u) * aux[k] + (s * s * s - s) * aux[k + 1]);
        *qd = (y[k + 1] - y[k]) / h + h / 6.0 * (-(3.0 * u * u - 1.0) * aux[k] + (3.0 * s * s - 1.0) * aux[k + 1]);
    }
}

/* The node derivatives of the variant spline of every joint's position knots, written
 * into the velocity knots: knots [nk][2][nu], spacing dtk. */
void orc_spline_slopes(int spline, int nu, int nk, real dtk, real* knots) {
    if (spline == ORC_SPLINE_HERMITE) return;
    real y[32], aux[32];
    for (int j = 0; j < nu; ++j) {
        for (int k = 0; k < nk; ++k) y[k] = knots[(k * 2 + 0) * nu + j];
        if (spline == ORC_SPLINE_QUADRATIC) {
            quadratic_slopes(nk, dtk, y, aux);
            for (int k = 0; k < nk; ++k) knots[(k * 2 + 1) * nu + j] = aux[k];
        } else {
            natural_cubic_moments(nk, dtk, y, aux);
            for (int k = 0; k < nk; ++k) {
                real q, qd;
                if (k + 1 < nk) variant_eval(spline, dtk, y, aux, k, 0.0, &q, &qd);
                else variant_eval(spline, dtk, y, aux, nk - 2, 1.0, &q, &qd);
                knots[(k * 2 + 1) * nu + j] = qd;
            }
        }
    }
}

/* Per-joint data of the position-only variants: node positions ys [nj][nk] and the
 * moments (cubic) or node slopes (quadratic) aux [nj][nk]. */
static void variant_prepare(int spline, int nj, int nk, real dtk, const real* knots, real* ys,
                            real* aux) {
    for (int j = 0; j < nj; ++j) {
        for (int k = 0; k < nk; ++k) ys[j * nk + k] = knots[(k * 2 + 0) * nj + j];
        if (spline == ORC_SPLINE_QUADRATIC) quadratic_slopes(nk, dtk, ys + j * nk, aux + j * nk);
        else natural_cubic_moments(nk, dtk, ys + j * nk, aux + j * nk);
    }
}

/* Setpoints (q_ref, v_ref) of step h for every joint: the spline at t_h = h dt. */
static void step_setpoints(int spline, int nj, int nk, int H, real dtk, const real* knots,
                           const real* ys, const real* aux, int h, real* qref, real* vref) {
    int k;
    real s;
    orc_segment(h, H, nk, &k, &s);
    for (int j = 0; j < nj; ++j) {
        if (spline == ORC_SPLINE_HERMITE)
            orc_hermite(s, dtk, knots[(k * 2 + 0) * nj + j], knots[(k * 2 + 1) * nj + j],
                        knots[((k + 1) * 2 + 0) * nj + j], knots[((k + 1) * 2 + 1) * nj + j], &qref[j],
                        &vref[j]);
        else
            variant_eval(spline, dtk, ys + j * nk, aux + j * nk, k, s, &qref[j], &vref[j]);
    }
}

/* The setpoints a rollout tracks: qref, vref [H][nu] for knots [nk][2][nu]. */
void orc_setpoints(int spline, int nu, int nk, int H, real dt, const real* knots, real* qref,
                   real* vref) {
    const real dtk = knot_dt(nk, H, dt);
    real* ys = (real*)malloc(sizeof(real) * (size_t)(nu > 0 ? nu : 1) * nk);
    real* aux = (real*)malloc(sizeof(real) * (size_t)(nu > 0 ? nu : 1) * nk);
    if (spline != ORC_SPLINE_HERMITE) variant_prepare(spline, nu, nk, dtk, knots, ys, aux);
    for (int h = 0; h < H; ++h)
        step_setpoints(spline, nu, nk, H, dtk, knots, ys, aux, h, qref + (size_t)h * nu, vref + (size_t)h * nu);
    free(ys);
    free(aux);
}

/* Rollout of one sample (Alg. 1 "simulate"): H steps from x0 tracking the Hermite
 * setpoints of knots [nk][2][nu]; returns S = sum_h c(x_h, u_h) + c_T(x_H) (Sec. IV-A).
 * x_final [nx] and traj [(H+1)][nx] are optional. */
real orc_rollout_ex(const orc_model* m, const real* x0, const real* knots, int nk, int H,
                      real dt, int spline, real* x_final, real* traj) {
    const int nj = m->nb - 1, nq = 7 + nj, nx = nq + 6 + nj;
    real x[7 + ORC_MAXB + 6 + ORC_MAXB];
    real qref[ORC_MAXB], vref[ORC_MAXB], tau[ORC_MAXB], acc[ORC_MAXNV];
    orc_kin* K = (orc_kin*)malloc(sizeof(orc_kin));
    memcpy(x, x0, sizeof(real) * nx);
    const real dtk = knot_dt(nk, H, dt);
    /* position-only variants: per-joint node positions and their spline data */
    real* ys = (real*)malloc(sizeof(real) * (size_t)(nj > 0 ? nj : 1) * nk);
    real* aux = (real*)malloc(sizeof(real) * (size_t)(nj > 0 ? nj : 1) * nk);
    if (spline != ORC_SPLINE_HERMITE) variant_prepare(spline, nj, nk, dtk, knots, ys, aux);
    real S = 0;
    if (traj) memcpy(traj, x, sizeof(real) * nx);
    for (int h = 0; h < H; ++h) {
        ORC_PHASE(PH_SPLINE);
        step_setpoints(spline, nj, nk, H, dtk, knots, ys, aux, h, qref, vref);
        ORC_PHASE(PH_PD);
        pd_torque(m, x, qref, vref, tau);
        if (aba(m, x, tau, K, acc) != 0) {
            S = NAN;
            break;
        }
        ORC_PHASE(PH_COST);
        S += running_cost(m, x, K, tau) + modular_cost(m, x, K);
        ORC_PHASE(PH_INTEGRATE);
        integrate(m, x, acc, dt);
        ORC_PHASE(PH_OTHER);
        if (traj) memcpy(traj + (size_t)(h + 1) * nx, x, sizeof(real) * nx);
    }
    if (H > 0 && isfinite(S)) S += terminal_cost(m, x0, x, H, dt);
    if (x_final) memcpy(x_final, x, sizeof(real) * nx);
    free(K);
    free(ys);
    free(aux);
    return S;
}

real orc_rollout(const orc_model* m, const real* x0, const real* knots, int nk, int H,
                   real dt, real* x_final, real* traj) {
    return orc_rollout_ex(m, x0, knots, nk, H, dt, ORC_SPLINE_HERMITE, x_final, traj);
}

/* Sec. III-E state prediction: simulate the first `nsteps` steps of the spline defined by
 * knots over a horizon of H steps (knot times as in the rollout) from x0; x_out [nx]. */
int orc_predict_state(const orc_model* m, const real* x0, const real* knots, int nk, int H, int nsteps,
                      real dt, real* x_out) {
    const int nj = m->nb - 1, nq = 7 + nj, nx = nq + 6 + nj;
    real* tr = (real*)malloc(sizeof(real) * (size_t)(H + 1) * nx);
    real S = orc_rollout(m, x0, knots, nk, H, dt, NULL, tr);
    (void)S;
    if (nsteps > H) nsteps = H;
    memcpy(x_out, tr + (size_t)nsteps * nx, sizeof(real) * nx);
    free(tr);
    return 0;
}

/* Sec. III-E shift of tau_best by `steps` actions with the tail held: the new knot j is
 * the old spline (value and time derivative) at time t_j + steps dt, capped at the
 * horizon end T = H dt. In the rollout's integer units r = t / dt * (nk - 1):
 * r_j = min(j H + steps (nk - 1), H (nk - 1)), segment k = min(floor(r_j / H), nk - 2),
 * s = (r_j - k H) / H. knots in/out [nk][2][nu] (may not alias). */
void orc_shift_knots(int nu, int nk, int H, int steps, real dt, const real* in, real* out) {
    const real dtk = knot_dt(nk, H, dt);
    for (int j = 0; j < nk; ++j) {
        long r = (long)j * H + (long)steps * (nk - 1);
        if (r > (long)H * (nk - 1)) r = (long)H * (nk - 1);
        long k = r / H;
        if (k > nk - 2) k = nk - 2;
        real s = (real)(r - k * (long)H) / (real)H;
        for (int i = 0; i < nu; ++i) {
            real q, qd;
            orc_hermite(s, dtk, in[(k * 2 + 0) * nu + i], in[(k * 2 + 1) * nu + i], in[((k + 1) * 2 + 0) * nu + i],
                        in[((k + 1) * 2 + 1) * nu + i], &q, &qd);
            out[(j * 2 + 0) * nu + i] = q;
            out[(j * 2 + 1) * nu + i] = qd;
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Weights and average (Sec. III-C)                                                      */
/* ------------------------------------------------------------------------------------ */
/* info[0..5] = S_min, S_max, argmin (ties -> lowest index), ESS = 1/sum w^2, n_finite,
 * log-sum-exp. normalize 0: min-max Eq. (softmax_minmax); 1: raw Eq. (omega-weights).
 * Non-finite costs get weight 0. Returns 0, or -3 when no cost is finite (w = 0). */
int orc_weights(int N, const real* S, real lambda, int normalize, real* w, real* info) {
    real smin = INFINITY, smax = -INFINITY;
    int best = -1, nf = 0;
    for (int n = 0; n < N; ++n) {
        if (!isfinite(S[n])) continue;
        ++nf;
        if (S[n] < smin) { smin = S[n]; best = n; }
        if (S[n] > smax) smax = S[n];
    }
    for (int n = 0; n < N; ++n) w[n] = 0;
    if (nf == 0) {
        info[0] = NAN; info[1] = NAN; info[2] = -1; info[3] = 0; info[4] = 0; info[5] = NAN;
        return -3;
    }
    real range = smax - smin;
    real z = 0;
    for (int n = 0; n < N; ++n) {
        if (!isfinite(S[n])) continue;
        real sh;
        if (normalize == 0) sh = range > 0 ? (S[n] - smin) / range : 0.0;
        else sh = S[n] - smin;
        z += exp(-sh / lambda);
    }
    real lse = log(z);
    real ess_den = 0;
    for (int n = 0; n < N; ++n) {
        if (!isfinite(S[n])) continue;
        real sh;
        if (normalize == 0) sh = range > 0 ? (S[n] - smin) / range : 0.0;
        else sh = S[n] - smin;
        w[n] = exp(-sh / lambda - lse);
        ess_den += w[n] * w[n];
    }
    info[0] = smin; info[1] = smax; info[2] = best; info[3] = 1.0 / ess_den; info[4] = nf; info[5] = lse;
    return 0;
}

/* Eq. (update-nominal) on the knots: out[e] = sum_n w_n theta_{n,e}. */
void orc_average(int N, int E, const real* knots, const real* w, real* out) {
    for (int e = 0; e < E; ++e) {
        real s = 0;
        for (int n = 0; n < N; ++n) s += w[n] * knots[(size_t)n * E + e];
        out[e] = s;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Parallel rollouts over samples (std pthreads; each sample is independent)            */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    const orc_model* m;
    const real* x0;
    const real* knots;
    int N, nk, H, E, nx, tid, nthreads, spline;
    real dt;
    real* costs;
    real* finals;
} rollout_job;

static void* rollout_worker(void* arg) {
    rollout_job* j = (rollout_job*)arg;
    for (int n = j->tid; n < j->N; n += j->nthreads)
        j->costs[n] = orc_rollout_ex(j->m, j->x0, j->knots + (size_t)n * j->E, j->nk, j->H, j->dt, j->spline,
                                     j->finals ? j->finals + (size_t)n * j->nx : NULL, NULL);
    return NULL;
}

/* costs[N] (and finals[N][nx] if non-null) for knots [N][nk][2][nu]. */
void orc_rollout_batch_ex(const orc_model* m, int N, const real* x0, const real* knots, int nk,
                          int H, real dt, int spline, real* costs, real* finals, int nthreads) {
    const int nj = m->nb - 1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    rollout_job jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (rollout_job){m, x0, knots, N, nk, H, nk * 2 * nj, 7 + nj + 6 + nj, t, nthreads, spline,
                                dt, costs, finals};
        if (nthreads > 1) pthread_create(&th[t], NULL, rollout_worker, &jobs[t]);
    }
    if (nthreads == 1) rollout_worker(&jobs[0]);
    else
        for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

void orc_rollout_batch(const orc_model* m, int N, const real* x0, const real* knots, int nk,
                       int H, real dt, real* costs, real* finals, int nthreads) {
    orc_rollout_batch_ex(m, N, x0, knots, nk, H, dt, ORC_SPLINE_HERMITE, costs, finals, nthreads);
}

/* ------------------------------------------------------------------------------------ */
/* Alg. 1: one MPPI solve of `iters` iterations from state x0 and nominal knots.         */
/* ------------------------------------------------------------------------------------ */
/* sigma [iters][nk]; mean_out, best_out [E]; knots_out (optional) [iters][N][E]
 * costs_out (optional) [iters][N].
 * info[0..7] = S_min, S_max (last iteration), best cost over the solve, best sample
 * index, iteration of the best, ESS (last iteration), n_finite (last), status.
 * Iteration i draws noise with counter iter_base + i. spline: ORC_SPLINE_* (the position-
 * only variants track their own spline of the sampled position knots).
 * Returns status (0 or -3). */
int orc_solve(const orc_model* m, int N, int nk, int H, int iters, real dt, real lambda,
              int normalize, const real* sigma, real scale_q, real scale_v, uint64_t seed,
              uint32_t iter_base, uint32_t inst, const real* x0, const real* nominal_in,
              real* mean_out, real* best_out, real* info, int nthreads, real* knots_out,
              real* costs_out, int spline) {
    const int nj = m->nb - 1, E = nk * 2 * nj;
    real* knots = (real*)malloc(sizeof(real) * (size_t)N * E);
    real* costs = (real*)malloc(sizeof(real) * N);
    real* w = (real*)malloc(sizeof(real) * N);
    real* nominal = (real*)malloc(sizeof(real) * (size_t)E);
    memcpy(nominal, nominal_in, sizeof(real) * E);
    int has_limits = 0;
    for (int j = 0; j < nj; ++j)
        if (isfinite(m->q_min[j]) || isfinite(m->q_max[j])) has_limits = 1;
    real best_cost = INFINITY;
    int best_idx = -1, best_it = -1, status = 0;
    real winfo[6] = {0};
    memcpy(best_out, nominal, sizeof(real) * E);
    for (int it = 0; it < iters; ++it) {
        orc_sample_knots(nj, nk, N, H, dt, nominal, sigma + (size_t)it * nk, scale_q, scale_v, seed,
                         iter_base + (uint32_t)it, inst, has_limits ? m->q_min : NULL,
                         has_limits ? m->q_max : NULL, knots);
        /* position-only variants: the velocity knots carry the variant spline's node slopes */
        for (int n = 0; n < N && spline != ORC_SPLINE_HERMITE; ++n)
            orc_spline_slopes(spline, nj, nk, knot_dt(nk, H, dt), knots + (size_t)n * E);
        orc_rollout_batch_ex(m, N, x0, knots, nk, H, dt, spline, costs, NULL, nthreads);
        if (knots_out) memcpy(knots_out + (size_t)it * N * E, knots, sizeof(real) * (size_t)N * E);
        if (costs_out) memcpy(costs_out + (size_t)it * N, costs, sizeof(real) * N);
        int st = orc_weights(N, costs, lambda, normalize, w, winfo);
        if (st != 0) {
            status = st;
            continue;
        }
        orc_average(N, E, knots, w, nominal);
        int b = (int)winfo[2];
        if (costs[b] < best_cost) {
            best_cost = costs[b];
            best_idx = b;
            best_it = it;
            memcpy(best_out, knots + (size_t)b * E, sizeof(real) * E);
        }
    }
    memcpy(mean_out, nominal, sizeof(real) * E);
    info[0] = winfo[0]; info[1] = winfo[1]; info[2] = best_cost; info[3] = best_idx;
    info[4] = best_it; info[5] = winfo[3]; info[6] = winfo[4]; info[7] = status;
    free(knots);
    free(costs);
    free(w);
    free(nominal);
    return status;
}

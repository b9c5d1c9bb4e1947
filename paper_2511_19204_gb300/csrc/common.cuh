// Device-side building blocks of the GB300 MPPI path: model constants, Philox4x32-10,
// Box-Muller, small spatial-algebra helpers. Everything is templated on the scalar
// type T (float for the product, double for the FP64 check build).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mppi.h"

namespace mppi {

constexpr int MAXB = MPPI_MAX_BODIES;
constexpr int MAXC = MPPI_MAX_CONTACTS;
constexpr int MAXCH = MPPI_MAX_CHILDREN;
constexpr int MAXK = MPPI_MAX_KNOTS;

// ------------------------------------------------------------------------------------
// Scalar helpers (overloads keep the templated code free of f/non-f spellings)
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void sc_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sc_sincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ void sc_sincospi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sc_sincospi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ float sc_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double sc_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float sc_log(float x) { return logf(x); }
__device__ __forceinline__ double sc_log(double x) { return log(x); }
__device__ __forceinline__ float sc_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double sc_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float sc_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double sc_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float sc_abs(float a) { return fabsf(a); }
__device__ __forceinline__ double sc_abs(double a) { return fabs(a); }
__device__ __forceinline__ float sc_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double sc_min(double a, double b) { return fmin(a, b); }
template <typename T>
__device__ __forceinline__ T sc_clamp(T x, T lo, T hi) { return sc_min(sc_max(x, lo), hi); }
// Reciprocal and reciprocal square root: FP32 takes the hardware approximations (within
// a couple of ulp, no slow path), FP64 (the check build) the correctly rounded forms.
__device__ __forceinline__ float sc_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double sc_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float sc_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double sc_rsqrt(double x) { return 1.0 / sqrt(x); }

// atan2(y, x) for y >= 0 (an angle in [0, pi]) in FP32 without a division slow path:
// t = min / max in [0, 1]; above tan(pi/8) the identity atan t = pi/4 + atan((t-1)/(t+1))
// brings the argument into [-tan(pi/8), tan(pi/8)], where the Taylor series of atan to
// u^17 has truncation error < 3e-9; then atan y/x = pi/2 - atan x/y for y > |x| and
// pi - that for x < 0.
__device__ __forceinline__ float fast_atan2_pos(float y, float x) {
    const float ax = fabsf(x);
    const float mx = fmaxf(y, ax), mn = fminf(y, ax);
    const bool zero = !(mx > 0.f);  // y = x = 0: atan2(0, +-0) = 0 or pi, selected at the end
    const float t = zero ? 0.f : __fdividef(mn, mx);
    const bool red = t > 0.414213562373095f;
    const float u = red ? __fdividef(t - 1.f, t + 1.f) : t;
    const float u2 = u * u;
    float p = fmaf(u2, 1.f / 17.f, -1.f / 15.f);
    p = fmaf(u2, p, 1.f / 13.f);
    p = fmaf(u2, p, -1.f / 11.f);
    p = fmaf(u2, p, 1.f / 9.f);
    p = fmaf(u2, p, -1.f / 7.f);
    p = fmaf(u2, p, 1.f / 5.f);
    p = fmaf(u2, p, -1.f / 3.f);
    float a = fmaf(u * u2, p, u);
    if (red) a += 0.785398163397448f;           // pi / 4
    if (y > ax) a = 1.57079632679490f - a;      // pi / 2
    const float r = x < 0.f ? 3.14159265358979f - a : a;
    return zero ? (signbit(x) ? 3.14159265358979f : 0.f) : r;
}

// sin and cos of an FP32 angle of moderate size (joint angles, |x| up to ~1e4): Cody and
// Waite's reduction by pi/2 with the constant split in two floats, then the Taylor
// polynomials of sin (to x^9) and cos (to x^10) on [-pi/4, pi/4], whose truncation errors
// (< 2e-9 and < 2e-10) lie below half an FP32 ulp of the results; the quadrant picks and
// signs the pair.
__device__ __forceinline__ void fast_sincos(float x, float* s, float* c) {
    const float k = rintf(x * 0.636619772367581343f);       // x / (pi / 2), rounded
    float r = fmaf(-k, 1.57079637050628662109375f, x);      // float(pi / 2)
    r = fmaf(-k, -4.37113900018624283e-8f, r);              // pi / 2 - float(pi / 2)
    const float r2 = r * r;
    float ps = fmaf(r2, 2.75573192e-6f, -1.98412698e-4f);  // 1/9!, -1/7!
    ps = fmaf(r2, ps, 8.33333333e-3f);                      // 1/5!
    ps = fmaf(r2, ps, -1.66666667e-1f);                     // -1/3!
    const float sn = fmaf(r * r2, ps, r);
    float pc = fmaf(r2, -2.75573192e-7f, 2.48015873e-5f);  // -1/10!, 1/8!
    pc = fmaf(r2, pc, -1.38888889e-3f);                     // -1/6!
    pc = fmaf(r2, pc, 4.16666667e-2f);                      // 1/4!
    pc = fmaf(r2, pc, -0.5f);
    const float cs = fmaf(r2, pc, 1.0f);
    const int q = (int)k & 3;
    const float a = (q & 1) ? cs : sn;   // sin: sn, cs, -sn, -cs
    const float b = (q & 1) ? sn : cs;   // cos: cs, -sn, -cs, sn
    *s = (q & 2) ? -a : a;
    *c = ((q + 1) & 2) ? -b : b;
}

// The rollout's elementary functions per precision: the FP32 path uses the own versions
// above and the hardware approximations, the FP64 check build the library's exact ones.
__device__ __forceinline__ void sc_sincos_r(float x, float* s, float* c) { fast_sincos(x, s, c); }
__device__ __forceinline__ void sc_sincos_r(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ float sc_atan2_pos(float y, float x) { return fast_atan2_pos(y, x); }
__device__ __forceinline__ double sc_atan2_pos(double y, double x) { return atan2(y, x); }

// ------------------------------------------------------------------------------------
// Model constants. Per-body arrays are structure-of-arrays over MAXB so that lane b of
// a warp reads entry b without bank conflicts. Joint j lives on body j + 1; per-joint
// arrays are indexed by body. The struct is copied into shared memory by one bulk
// (TMA) copy per block, so its size is a multiple of 16 bytes.
// ------------------------------------------------------------------------------------
template <typename T>
struct alignas(16) DevModel {
    T axis[3][MAXB];
    T jpos[3][MAXB];
    T mass[MAXB];
    T mc[3][MAXB];        // mass * centre of mass (body frame)
    T Ao[6][MAXB];        // rotational inertia about the body origin: xx yy zz xy xz yz
    T armature[MAXB];
    T kp[MAXB];
    T kd[MAXB];
    T tau_max[MAXB];
    T q_min[MAXB];
    T q_max[MAXB];
    T q_init[MAXB];
    T cpos[3][MAXC];      // contact points, sorted by body (stable)
    int32_t parent[MAXB];
    int32_t level[MAXB];
    int32_t nchild[MAXB];
    int32_t child[MAXCH][MAXB];
    int32_t cfirst[MAXB];
    int32_t ccount[MAXB];
    int32_t lane_b0[4];   // lanes-per-chain plan: first body of each lane's chain
    int32_t lane_len[4];  // and its length
    int32_t nb, nc, nlevels, fixed_base;
    int32_t cost_body, has_limits, topology, branch_body;
    T contact_k, contact_c, mu, eps_f;
    T gravity, z_des, vx_des, w_z;
    T w_vx, w_tilt, w_tau, pad1;
    // modular cost of Sec. IV-A; paper_cost = 0 when every one of its weights is zero
    T w_h, w_orient, w_q, w_cvel;
    T w_cforce, w_term, cf_off, pad2;   // cf_off = w_cforce ||f0||_1 (a point off contact)
    T f0[4];
    T pdot_des[4];
    T Rdes[12];                         // R_des row-major (9 used)
    int32_t paper_cost;
    int32_t axis_plan;                  // lanes-per-chain axis plan (AXP_*)
    int32_t pad3[2];
};

// Tree shapes with a lanes-per-chain kernel.
constexpr int TOPO_GENERIC = 0;
constexpr int TOPO_QUADRUPED = 1;   // 4 chains of <= 3 bodies off the base
constexpr int TOPO_HUMANOID = 2;    // 2 chains of <= 6 off the base + a branch body with 2 chains of <= 6

// Axis plans of the lanes-per-chain quadruped: AXP_GENERIC, any unit axes; AXP_XYY, the
// usual leg layout: every chain's joints turn about +x, +y, +y (hip abduction, hip and
// knee flexion), the hip sits in the base's xy-plane, the thigh joint along y from the
// hip and the knee along z from the thigh, and contact points only on the calves, which
// the passes exploit at compile time. AXP_HUM, the usual humanoid layout (6-joint legs off
// the base turning about z, x, y, y, y, x; a waist joint about z carrying 4-joint arms that
// turn about y, x, z, y; every joint offset on one axis, in the yz-plane or zero; contact
// points only on the feet; the cost body not on a leg), runs the two-warp split kernel.
constexpr int AXP_GENERIC = 0;
constexpr int AXP_XYY = 1;
constexpr int AXP_HUM = 2;

// ------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64-bit
// multiplies, Weyl key schedule.
// ------------------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        U4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
    }
    return c;
}

// Box-Muller (Box & Muller 1958) on two words: u1 = ((wa >> 8) + 1) 2^-24 in (0, 1],
// u2 = (wb >> 8) 2^-24 in [0, 1); eps_a = r cos(2 pi u2), eps_b = r sin(2 pi u2).
// u1 and 2*u2 are exact in FP32; sincospi avoids rounding 2*pi.
template <typename T>
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, T* ea, T* eb) {
    const T two_m24 = T(1.0 / 16777216.0);
    const T u1 = (T)((wa >> 8) + 1u) * two_m24;
    const T u2x2 = (T)(wb >> 8) * (T(2) * two_m24);
    const T r = sc_sqrt(T(-2) * sc_log(u1));
    T s, c;
    sc_sincospi(u2x2, &s, &c);
    *ea = r * c;
    *eb = r * s;
}

// ------------------------------------------------------------------------------------
// 3-vector / 3x3 helpers
// ------------------------------------------------------------------------------------
template <typename T>
struct V3 {
    T x, y, z;
};
template <typename T>
__device__ __forceinline__ V3<T> v3(T x, T y, T z) { return V3<T>{x, y, z}; }
template <typename T>
__device__ __forceinline__ V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename T>
__device__ __forceinline__ V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename T>
__device__ __forceinline__ V3<T> operator*(T s, V3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename T>
__device__ __forceinline__ T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T>
__device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Row-major 3x3.
template <typename T>
struct M3 {
    T m[9];
};
template <typename T>
__device__ __forceinline__ V3<T> mul(const M3<T>& R, V3<T> v) {
    return {R.m[0] * v.x + R.m[1] * v.y + R.m[2] * v.z, R.m[3] * v.x + R.m[4] * v.y + R.m[5] * v.z,
            R.m[6] * v.x + R.m[7] * v.y + R.m[8] * v.z};
}
template <typename T>
__device__ __forceinline__ V3<T> mulT(const M3<T>& R, V3<T> v) {
    return {R.m[0] * v.x + R.m[3] * v.y + R.m[6] * v.z, R.m[1] * v.x + R.m[4] * v.y + R.m[7] * v.z,
            R.m[2] * v.x + R.m[5] * v.y + R.m[8] * v.z};
}
template <typename T>
__device__ __forceinline__ M3<T> mul(const M3<T>& A, const M3<T>& B) {
    M3<T> C;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            C.m[3 * i + j] = A.m[3 * i] * B.m[j] + A.m[3 * i + 1] * B.m[3 + j] + A.m[3 * i + 2] * B.m[6 + j];
    return C;
}
// Rotation about unit axis a by angle (child -> parent): c I + s [a]x + (1 - c) a a^T.
template <typename T>
__device__ __forceinline__ M3<T> axis_rotation(V3<T> a, T s, T c) {
    const T t = T(1) - c;
    M3<T> R;
    R.m[0] = c + t * a.x * a.x;
    R.m[1] = t * a.x * a.y - s * a.z;
    R.m[2] = t * a.x * a.z + s * a.y;
    R.m[3] = t * a.y * a.x + s * a.z;
    R.m[4] = c + t * a.y * a.y;
    R.m[5] = t * a.y * a.z - s * a.x;
    R.m[6] = t * a.z * a.x - s * a.y;
    R.m[7] = t * a.z * a.y + s * a.x;
    R.m[8] = c + t * a.z * a.z;
    return R;
}
template <typename T>
__device__ __forceinline__ M3<T> quat_to_R(T w, T x, T y, T z) {
    M3<T> R;
    R.m[0] = T(1) - T(2) * (y * y + z * z);
    R.m[1] = T(2) * (x * y - w * z);
    R.m[2] = T(2) * (x * z + w * y);
    R.m[3] = T(2) * (x * y + w * z);
    R.m[4] = T(1) - T(2) * (x * x + z * z);
    R.m[5] = T(2) * (y * z - w * x);
    R.m[6] = T(2) * (x * z - w * y);
    R.m[7] = T(2) * (y * z + w * x);
    R.m[8] = T(1) - T(2) * (x * x + y * y);
    return R;
}

// ------------------------------------------------------------------------------------
// Modular cost of Sec. IV-A (Eq. running cost, Eq. terminal cost), the parts shared by
// the rollout mappings.
// ------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T abs1(V3<T> a) {
    return sc_abs(a.x) + sc_abs(a.y) + sc_abs(a.z);
}

// One contact point in contact (depth > 0), world velocity vw and force F:
// w_cvel ||v_c||_1 + w_cforce ||f_c - f0||_1. Off contact the point adds M.cf_off.
template <typename T>
__device__ __forceinline__ T contact_cost(const DevModel<T>& M, V3<T> vw, V3<T> F) {
    return M.w_cvel * abs1(vw) + M.w_cforce * abs1(F - v3(M.f0[0], M.f0[1], M.f0[2]));
}

// Base terms of the running cost: w_h |p_z - z_des| + w_orient theta^2 with theta the
// rotation angle of Q = R^T R_des (||log3 Q|| = theta): cos theta = (tr Q - 1) / 2,
// sin theta = |(Q21 - Q12, Q02 - Q20, Q10 - Q01)| / 2.
template <typename T>
__device__ __forceinline__ T base_cost(const DevModel<T>& M, const M3<T>& R, V3<T> p) {
    T Q[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            Q[3 * a + b] = R.m[a] * M.Rdes[b] + R.m[3 + a] * M.Rdes[3 + b] + R.m[6 + a] * M.Rdes[6 + b];
    const T vx = Q[7] - Q[5], vy = Q[2] - Q[6], vz = Q[3] - Q[1];
    const T th = sc_atan2_pos(sc_sqrt(vx * vx + vy * vy + vz * vz), Q[0] + Q[4] + Q[8] - T(1));
    return M.w_h * sc_abs(p.z - M.z_des) + M.w_orient * th * th;
}

// Terminal cost: w_term ||p_H - (p_0 + pdot_des H dt)||_1.
template <typename T>
__device__ __forceinline__ T terminal_cost(const DevModel<T>& M, V3<T> pH, V3<T> p0, int H, T dt) {
    const T hd = (T)H * dt;
    const V3<T> tgt = p0 + hd * v3(M.pdot_des[0], M.pdot_des[1], M.pdot_des[2]);
    return M.w_term * abs1(pH - tgt);
}

// ------------------------------------------------------------------------------------
// Symmetric 6x6 articulated inertia [[A, B], [B^T, C]], A and C symmetric (xx yy zz xy
// xz yz), B full row-major. Acts on motion (w, v) and yields force (n, f).
// ------------------------------------------------------------------------------------
template <typename T>
struct Art {
    T A[6];
    T B[9];
    T C[6];
};

template <typename T>
__device__ __forceinline__ V3<T> sym_mul(const T* S, V3<T> v) {
    return {S[0] * v.x + S[3] * v.y + S[4] * v.z, S[3] * v.x + S[1] * v.y + S[5] * v.z,
            S[4] * v.x + S[5] * v.y + S[2] * v.z};
}

// R S R^T for symmetric S.
template <typename T>
__device__ __forceinline__ void sym_rotate(const M3<T>& R, const T* S, T* out) {
    // N = S R^T  (N[i][j] = sum_k S[i][k] R[j][k])
    const T s[3][3] = {{S[0], S[3], S[4]}, {S[3], S[1], S[5]}, {S[4], S[5], S[2]}};
    T N[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) N[i][j] = s[i][0] * R.m[3 * j] + s[i][1] * R.m[3 * j + 1] + s[i][2] * R.m[3 * j + 2];
    auto e = [&](int i, int j) { return R.m[3 * i] * N[0][j] + R.m[3 * i + 1] * N[1][j] + R.m[3 * i + 2] * N[2][j]; };
    out[0] = e(0, 0);
    out[1] = e(1, 1);
    out[2] = e(2, 2);
    out[3] = e(0, 1);
    out[4] = e(0, 2);
    out[5] = e(1, 2);
}
// R B R^T for full B.
template <typename T>
__device__ __forceinline__ void full_rotate(const M3<T>& R, const T* B, T* out) {
    T N[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            N[i][j] = B[3 * i] * R.m[3 * j] + B[3 * i + 1] * R.m[3 * j + 1] + B[3 * i + 2] * R.m[3 * j + 2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            out[3 * i + j] = R.m[3 * i] * N[0][j] + R.m[3 * i + 1] * N[1][j] + R.m[3 * i + 2] * N[2][j];
}

// Congruence X^T Ia X for the parent->child Plucker transform X = [E 0; -E r^ E] with
// E = Rj^T (Rj = joint rotation child->parent) and r = joint position in the parent:
// rotate (Rj M Rj^T), then shift the reference point by r:
//   C' unchanged, B' += r^ C', A' += r^ B'^T - B'' r^  (B'' the shifted B).
// The reference-point shift of the congruence for already rotated blocks A, B, C.
template <typename T>
__device__ __forceinline__ void art_shift(const T* A, const T* B, const T* C, V3<T> r, Art<T>& out) {
    // B2 = B + r^ C : column j of r^ C = r x C[:, j]
    const V3<T> c0 = v3(C[0], C[3], C[4]), c1 = v3(C[3], C[1], C[5]), c2 = v3(C[4], C[5], C[2]);
    const V3<T> x0 = cross(r, c0), x1 = cross(r, c1), x2 = cross(r, c2);
    T B2[9] = {B[0] + x0.x, B[1] + x1.x, B[2] + x2.x, B[3] + x0.y, B[4] + x1.y,
               B[5] + x2.y, B[6] + x0.z, B[7] + x1.z, B[8] + x2.z};
    // D = r^ B^T : column j = r x (row j of B)
    const V3<T> d0 = cross(r, v3(B[0], B[1], B[2]));
    const V3<T> d1 = cross(r, v3(B[3], B[4], B[5]));
    const V3<T> d2 = cross(r, v3(B[6], B[7], B[8]));
    // F = B2 r^ : row i = (row i of B2) x r
    const V3<T> f0 = cross(v3(B2[0], B2[1], B2[2]), r);
    const V3<T> f1 = cross(v3(B2[3], B2[4], B2[5]), r);
    const V3<T> f2 = cross(v3(B2[6], B2[7], B2[8]), r);
    // A + D - F (symmetric in exact arithmetic; D[i][j] = d_j.i)
    out.A[0] = A[0] + d0.x - f0.x;
    out.A[1] = A[1] + d1.y - f1.y;
    out.A[2] = A[2] + d2.z - f2.z;
    out.A[3] = A[3] + d1.x - f0.y;
    out.A[4] = A[4] + d2.x - f0.z;
    out.A[5] = A[5] + d2.y - f1.z;
#pragma unroll
    for (int k = 0; k < 9; ++k) out.B[k] = B2[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) out.C[k] = C[k];
}

template <typename T>
__device__ __forceinline__ void art_to_parent(const Art<T>& Ia, const M3<T>& Rj, V3<T> r, Art<T>& out) {
    T A[6], B[9], C[6];
    sym_rotate(Rj, Ia.A, A);
    full_rotate(Rj, Ia.B, B);
    sym_rotate(Rj, Ia.C, C);
    art_shift(A, B, C, r, out);
}

// Solve the 6x6 SPD system [[A, B], [B^T, C]] x = b by Cholesky (in registers).
template <typename T>
__device__ __forceinline__ void art_solve(const Art<T>& I, const T* b, T* x) {
    T M[6][6];
    M[0][0] = I.A[0]; M[1][1] = I.A[1]; M[2][2] = I.A[2];
    M[0][1] = M[1][0] = I.A[3]; M[0][2] = M[2][0] = I.A[4]; M[1][2] = M[2][1] = I.A[5];
    M[3][3] = I.C[0]; M[4][4] = I.C[1]; M[5][5] = I.C[2];
    M[3][4] = M[4][3] = I.C[3]; M[3][5] = M[5][3] = I.C[4]; M[4][5] = M[5][4] = I.C[5];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[i][3 + j] = M[3 + j][i] = I.B[3 * i + j];
    T L[6][6];
    T inv[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            T s = M[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                inv[i] = sc_rsqrt(s);  // 1 / L[i][i]
            } else {
                L[i][j] = s * inv[j];
            }
        }
    }
    T y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        T s = b[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
        y[i] = s * inv[i];
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        T s = y[i];
#pragma unroll
        for (int k = i + 1; k < 6; ++k) s -= L[k][i] * x[k];
        x[i] = s * inv[i];
    }
}

// Programmatic dependent launch: a kernel launched as the programmatic dependent of the
// one before it in the stream may start while that one runs; pdl_wait() blocks until it
// has completed and its memory is visible (it returns at once in a kernel launched
// without the dependency), and pdl_trigger() in the primary lets the dependent launch
// as soon as every primary block has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ------------------------------------------------------------------------------------
// Bounded TMA bulk copy of a global block into shared memory (cp.async.bulk +
// mbarrier). Thread 0 issues; every thread waits with an iteration limit. Returns false
// when the wait gave up (the caller reports MPPI_ERR_TIMEOUT and skips its work).
// ------------------------------------------------------------------------------------
__device__ __forceinline__ bool bulk_load_to_smem(void* smem_dst, const void* gmem_src, uint32_t bytes,
                                                  uint64_t* mbar) {
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(mbar);
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(smem_dst);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
            "l"(gmem_src), "r"(bytes), "r"(bar)
            : "memory");
    }
    __syncthreads();
    auto wait = [&](int limit) {
        bool done = false;
        for (int it = 0; it < limit && !done; ++it) {
            uint32_t ok;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(ok)
                : "r"(bar)
                : "memory");
            done = ok != 0;
        }
        return done;
    };
    // every thread of the block takes the same decision
    if (__syncthreads_and(wait(1 << 22) ? 1 : 0)) return true;
    // gave up: wait once more (bounded) for the copy in flight before the caller exits
    wait(1 << 22);
    __syncthreads();
    return false;
}

// Bounds checks of the check build (compiled with -DMPPI_CHECK, in place of a memory
// checker): MPPI_CHECK_OK(cond, bit) is cond, and when cond fails it also
// sets `bit` in the translation unit's check word (mppi_check_word reads the word of the
// unit that holds every FP32 kernel); the caller then skips or clamps the access, so a
// failed check never traps. In the product build it is the constant true and the
// compiler removes the check.
#ifdef MPPI_CHECK
static __device__ uint32_t g_check_word;
#define MPPI_CHECK_OK(cond, bit) ((cond) ? true : (atomicOr(&::mppi::g_check_word, (uint32_t)(bit)), false))
#else
#define MPPI_CHECK_OK(cond, bit) true
#endif
constexpr uint32_t CHECK_NOISE = 1u;    // noise: a sample or element outside the knots
constexpr uint32_t CHECK_KNOT = 2u;     // rollout: a segment past the last knot pair
constexpr uint32_t CHECK_QUEUE = 4u;    // persistent kernel: an item outside its instance
constexpr uint32_t CHECK_CHUNK = 8u;    // reduction: a chunk or element outside the sums
constexpr uint32_t CHECK_SPLIT = 16u;   // split rollout: a record outside the pair's area
constexpr uint32_t CHECK_BEST = 32u;    // finalize: a best sample outside the knots

// Status word written by kernels whose bounded waits gave up.
constexpr uint32_t DEV_ERR_TMA_TIMEOUT = 1u;
constexpr uint32_t DEV_ERR_QUEUE_TIMEOUT = 2u;
constexpr uint32_t DEV_ERR_BAD_ITEM = 4u;
constexpr uint32_t DEV_ERR_GRID_TIMEOUT = 8u;

}  // namespace mppi

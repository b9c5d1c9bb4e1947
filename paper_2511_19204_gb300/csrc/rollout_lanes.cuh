// Lanes-per-chain rollout (device function): 4 lanes share one sample of a tree made of a
// floating base, chains hanging from it, and optionally one branch body that carries two
// of the chains (the quadruped: 4 leg chains of 3 bodies; the humanoid: 2 leg chains of 6
// from the pelvis, and the torso carrying 2 arm chains of 4).
//
// Lane g runs its chain's three articulated-body passes serially in registers. The base
// is replicated on the 4 lanes and the branch body on the two lanes whose chains hang
// from it; the arm chains' articulated inertias meet at the branch by a pair shuffle, and
// everything meets at the base by a 2-step butterfly. Those sums are commutative
// exchanges, so every replica sees bitwise the same numbers and the replicated base and
// branch never diverge. Equations as in the warp-per-sample kernel: Featherstone's
// articulated-body algorithm, Sec. III-A Hermite setpoints, Sec. III-C PD tracking,
// semi-implicit Euler, Kahan-summed running cost.
//
// This file is a body included by chain_f32.cuh (FP32 product, namespace mppi) and by the
// FP64 check build's translation unit (namespace mppi::f64), with the scalar type R_T and
// its literals and elementary functions (R_C, R_FMA, R_SINCOS, ...) from scalar_macros.h.
R_NS_BEGIN

constexpr int LANES = 4;

// Axis code and offset code of chain position J under an axis plan (AXP_* in common.cuh).
template <int AXP, int J>
__host__ __device__ constexpr int chain_axis() {
    return AXP == AXP_XYY ? (J == 0 ? 0 : 1) : -1;
}
template <int AXP, int J>
__host__ __device__ constexpr int chain_offset() {
    return AXP == AXP_XYY ? (J == 0 ? 3 : (J == 1 ? 1 : 2)) : -1;  // 3: the hip offset lies in the xy-plane
}

// f(std::integral_constant<int, J>) for J = B .. E - 1, unrolled at compile time.
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

__device__ __forceinline__ R_T lsum(R_T v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1, LANES);
    v += __shfl_xor_sync(0xffffffffu, v, 2, LANES);
    return v;
}

// What a body keeps between passes. x0/x1 hold the bias (n, f) after pass 1 and the
// scaled U_ang / D, U_lin / D after pass 2; uu = u / D. The joint rotation is kept
// whole (R) for short chains, else as its sine and cosine and rebuilt when needed (the
// same expression either way, so the numbers are identical).
struct BodyMem {
    R_T s, c;
    M3<R_T> R;
    V3<R_T> cw, cv;
    V3<R_T> x0, x1;
    R_T uu;
};

// ------------------------------------------------------------------------------------
// Joint rotations Rj (child -> parent). AX = 0, 1, 2: about the coordinate axis x, y, z
// (+1 direction), kept as (sin, cos), so applying one touches two components and costs 4
// multiplies instead of 9. AX = -1: any unit axis, the full matrix. The axis-vector
// operations below are written out per AX (a select, not a multiply by 0 or 1, which
// IEEE arithmetic would not fold away).
// ------------------------------------------------------------------------------------
template <int AX>
struct JRot {
    R_T s, c;
};
template <>
struct JRot<-1> {
    M3<R_T> R;
};

template <int AX>
__device__ __forceinline__ V3<R_T> jrot(const JRot<AX>& J, V3<R_T> v) {  // Rj v
    if constexpr (AX == 0) return v3(v.x, J.c * v.y - J.s * v.z, J.s * v.y + J.c * v.z);
    else if constexpr (AX == 1) return v3(J.c * v.x + J.s * v.z, v.y, J.c * v.z - J.s * v.x);
    else if constexpr (AX == 2) return v3(J.c * v.x - J.s * v.y, J.s * v.x + J.c * v.y, v.z);
    else return mul(J.R, v);
}
template <int AX>
__device__ __forceinline__ V3<R_T> jrotT(const JRot<AX>& J, V3<R_T> v) {  // Rj^T v
    if constexpr (AX == 0) return v3(v.x, J.c * v.y + J.s * v.z, J.c * v.z - J.s * v.y);
    else if constexpr (AX == 1) return v3(J.c * v.x - J.s * v.z, v.y, J.s * v.x + J.c * v.z);
    else if constexpr (AX == 2) return v3(J.c * v.x + J.s * v.y, J.c * v.y - J.s * v.x, v.z);
    else return mulT(J.R, v);
}
// R Rj: row i of the product is Rj^T applied to row i of R
template <int AX>
__device__ __forceinline__ M3<R_T> jcompose(const M3<R_T>& R, const JRot<AX>& J) {
    if constexpr (AX < 0) {
        return mul(R, J.R);
    } else {
        M3<R_T> o;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const V3<R_T> w = jrotT(J, v3(R.m[3 * i], R.m[3 * i + 1], R.m[3 * i + 2]));
            o.m[3 * i] = w.x;
            o.m[3 * i + 1] = w.y;
            o.m[3 * i + 2] = w.z;
        }
        return o;
    }
}
// Rj S Rj^T: N = S Rj^T has rows Rj (row i of S); the result has columns Rj (column j of N)
template <int AX>
__device__ __forceinline__ void jsym_rotate(const JRot<AX>& J, const R_T* S, R_T* out) {
    if constexpr (AX < 0) {
        sym_rotate(J.R, S, out);
    } else {
        const V3<R_T> r0 = jrot(J, v3(S[0], S[3], S[4])), r1 = jrot(J, v3(S[3], S[1], S[5])),
                        r2 = jrot(J, v3(S[4], S[5], S[2]));
        const V3<R_T> c0 = jrot(J, v3(r0.x, r1.x, r2.x)), c1 = jrot(J, v3(r0.y, r1.y, r2.y)),
                        c2 = jrot(J, v3(r0.z, r1.z, r2.z));
        out[0] = c0.x;
        out[1] = c1.y;
        out[2] = c2.z;
        out[3] = c1.x;
        out[4] = c2.x;
        out[5] = c2.y;
    }
}
template <int AX>
__device__ __forceinline__ void jfull_rotate(const JRot<AX>& J, const R_T* B, R_T* out) {
    if constexpr (AX < 0) {
        full_rotate(J.R, B, out);
    } else {
        const V3<R_T> r0 = jrot(J, v3(B[0], B[1], B[2])), r1 = jrot(J, v3(B[3], B[4], B[5])),
                        r2 = jrot(J, v3(B[6], B[7], B[8]));
        const V3<R_T> c0 = jrot(J, v3(r0.x, r1.x, r2.x)), c1 = jrot(J, v3(r0.y, r1.y, r2.y)),
                        c2 = jrot(J, v3(r0.z, r1.z, r2.z));
        out[0] = c0.x;
        out[1] = c1.x;
        out[2] = c2.x;
        out[3] = c0.y;
        out[4] = c1.y;
        out[5] = c2.y;
        out[6] = c0.z;
        out[7] = c1.z;
        out[8] = c2.z;
    }
}
// ------------------------------------------------------------------------------------
// Joint offsets r along one coordinate axis (OF = 0, 1, 2: r = rho e_OF), in the xy-plane
// (OF = 3: r.z = 0) or the yz-plane (OF = 4: r.x = 0), zero (OF = 5), or any r (OF = -1).
// (e_k x u)_i = eps_{i k p} u_p with p the third index: xk_src gives p (or -1 for i = k)
// and xk_sgn the sign, so the products by zero components are never formed.
// ------------------------------------------------------------------------------------
__host__ __device__ constexpr int xk_src(int k, int i) { return i == k ? -1 : 3 - i - k; }
__host__ __device__ constexpr R_T xk_sgn(int k, int i) {
    return i == k ? R_C(0.) : (((i - k + 3) % 3) == 2 ? R_C(1.) : -R_C(1.));
}
__device__ __forceinline__ R_T comp(V3<R_T> v, int i) { return i == 0 ? v.x : (i == 1 ? v.y : v.z); }

template <int OF>
__device__ __forceinline__ R_T rlen(V3<R_T> r) {
    return OF == 0 ? r.x : (OF == 1 ? r.y : r.z);
}
// r x u for r in the xy-plane (OF == 3: r.z == 0), the products with r.z left out
__device__ __forceinline__ V3<R_T> cross_rxy(V3<R_T> r, V3<R_T> u) {
    return v3(r.y * u.z, -(r.x * u.z), r.x * u.y - r.y * u.x);
}
// r x u for r in the yz-plane (OF == 4: r.x == 0), the products with r.x left out
__device__ __forceinline__ V3<R_T> cross_ryz(V3<R_T> r, V3<R_T> u) {
    return v3(r.y * u.z - r.z * u.y, r.z * u.x, -(r.y * u.x));
}
template <int OF>
__device__ __forceinline__ V3<R_T> cross_rp(V3<R_T> r, V3<R_T> u) {
    if constexpr (OF == 3) return cross_rxy(r, u);
    else return cross_ryz(r, u);
}
// v + s (r x u), s = +1 or -1
template <int OF>
__device__ __forceinline__ V3<R_T> add_rcross(V3<R_T> v, V3<R_T> r, V3<R_T> u, R_T sgn) {
    if constexpr (OF < 0) {
        return sgn > R_C(0.) ? v + cross(r, u) : v - cross(r, u);
    } else if constexpr (OF == 3 || OF == 4) {
        return sgn > R_C(0.) ? v + cross_rp<OF>(r, u) : v - cross_rp<OF>(r, u);
    } else if constexpr (OF == 5) {
        return v;
    } else {
        const R_T rho = sgn * rlen<OF>(r);
        R_T o[3] = {v.x, v.y, v.z};
#pragma unroll
        for (int i = 0; i < 3; ++i)
            if (i != OF) o[i] += (xk_sgn(OF, i) * rho) * comp(u, xk_src(OF, i));
        return v3(o[0], o[1], o[2]);
    }
}
// R r
template <int OF>
__device__ __forceinline__ V3<R_T> rot_r(const M3<R_T>& R, V3<R_T> r) {
    if constexpr (OF < 0) {
        return mul(R, r);
    } else if constexpr (OF == 3) {
        return v3(R.m[0] * r.x + R.m[1] * r.y, R.m[3] * r.x + R.m[4] * r.y, R.m[6] * r.x + R.m[7] * r.y);
    } else if constexpr (OF == 4) {
        return v3(R.m[1] * r.y + R.m[2] * r.z, R.m[4] * r.y + R.m[5] * r.z, R.m[7] * r.y + R.m[8] * r.z);
    } else if constexpr (OF == 5) {
        return v3(R_C(0.), R_C(0.), R_C(0.));
    } else {
        const R_T rho = rlen<OF>(r);
        return v3(R.m[OF] * rho, R.m[3 + OF] * rho, R.m[6 + OF] * rho);
    }
}
// The reference-point shift of the congruence (art_shift) for r = rho e_OF:
// B2 = B + r^ C, A' = A + r^ B^T - B2 r^, written per component.
template <int OF>
__device__ __forceinline__ void art_shift_r(const R_T* A, const R_T* B, const R_T* C, V3<R_T> r,
                                            Art<R_T>& out) {
    if constexpr (OF < 0) {
        art_shift(A, B, C, r, out);
    } else if constexpr (OF == 5) {
#pragma unroll
        for (int k = 0; k < 6; ++k) out.A[k] = A[k];
#pragma unroll
        for (int k = 0; k < 9; ++k) out.B[k] = B[k];
#pragma unroll
        for (int k = 0; k < 6; ++k) out.C[k] = C[k];
    } else if constexpr (OF == 3 || OF == 4) {
        // as art_shift with every r x (.) and (.) x r formed without the zero component of r
        const V3<R_T> x0 = cross_rp<OF>(r, v3(C[0], C[3], C[4])), x1 = cross_rp<OF>(r, v3(C[3], C[1], C[5])),
                        x2 = cross_rp<OF>(r, v3(C[4], C[5], C[2]));
        const R_T B2[9] = {B[0] + x0.x, B[1] + x1.x, B[2] + x2.x, B[3] + x0.y, B[4] + x1.y,
                             B[5] + x2.y, B[6] + x0.z, B[7] + x1.z, B[8] + x2.z};
        const V3<R_T> d0 = cross_rp<OF>(r, v3(B[0], B[1], B[2]));
        const V3<R_T> d1 = cross_rp<OF>(r, v3(B[3], B[4], B[5]));
        const V3<R_T> d2 = cross_rp<OF>(r, v3(B[6], B[7], B[8]));
        // f_i = (row i of B2) x r = -(r x row i)
        const V3<R_T> f0 = cross_rp<OF>(r, v3(B2[0], B2[1], B2[2]));
        const V3<R_T> f1 = cross_rp<OF>(r, v3(B2[3], B2[4], B2[5]));
        const V3<R_T> f2 = cross_rp<OF>(r, v3(B2[6], B2[7], B2[8]));
        out.A[0] = A[0] + d0.x + f0.x;
        out.A[1] = A[1] + d1.y + f1.y;
        out.A[2] = A[2] + d2.z + f2.z;
        out.A[3] = A[3] + d1.x + f0.y;
        out.A[4] = A[4] + d2.x + f0.z;
        out.A[5] = A[5] + d2.y + f1.z;
#pragma unroll
        for (int k = 0; k < 9; ++k) out.B[k] = B2[k];
#pragma unroll
        for (int k = 0; k < 6; ++k) out.C[k] = C[k];
    } else {
        const R_T rho = rlen<OF>(r);
        auto Cs = [&](int i, int j) -> R_T {
            return i == j ? C[i] : C[(i + j == 1) ? 3 : ((i + j == 2) ? 4 : 5)];
        };
        R_T B2[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                B2[3 * i + j] = i == OF ? B[3 * i + j] : B[3 * i + j] + (xk_sgn(OF, i) * rho) * Cs(xk_src(OF, i), j);
        // A'(i, j) = A(i, j) + (r x B_row_j)_i - (B2_row_i x r)_j
        //          = A(i, j) + [i != OF] s_i rho B(j, p_i) + [j != OF] s_j rho B2(i, p_j)
        const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
        for (int t = 0; t < 6; ++t) {
            const int i = ii[t], j = jj[t];
            R_T a = A[t];
            if (i != OF) a += (xk_sgn(OF, i) * rho) * B[3 * j + xk_src(OF, i)];
            if (j != OF) a += (xk_sgn(OF, j) * rho) * B2[3 * i + xk_src(OF, j)];
            out.A[t] = a;
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) out.B[k] = B2[k];
#pragma unroll
        for (int k = 0; k < 6; ++k) out.C[k] = C[k];
    }
}

template <int AX, int OF>
__device__ __forceinline__ void jart_to_parent(const Art<R_T>& Ia, const JRot<AX>& J, V3<R_T> r, Art<R_T>& out) {
    R_T A[6], B[9], C[6];
    jsym_rotate(J, Ia.A, A);
    jfull_rotate(J, Ia.B, B);
    jsym_rotate(J, Ia.C, C);
    art_shift_r<OF>(A, B, C, r, out);
}

// A body's constants, loaded once per rollout into registers (the step loop would
// otherwise re-read them from shared memory every step).
struct BodyConst {
    V3<R_T> a, r, mc;   // joint axis, joint position in the parent, mass * com
    R_T Ao[6];          // rotational inertia about the body origin
    R_T m, arm, kp, kd, tmax, qinit;
    int b;
};

__device__ __forceinline__ BodyConst load_body(const DevModel<R_T>& M, int b) {
    BodyConst C;
    C.a = v3(M.axis[0][b], M.axis[1][b], M.axis[2][b]);
    C.r = v3(M.jpos[0][b], M.jpos[1][b], M.jpos[2][b]);
    C.mc = v3(M.mc[0][b], M.mc[1][b], M.mc[2][b]);
#pragma unroll
    for (int t = 0; t < 6; ++t) C.Ao[t] = M.Ao[t][b];
    C.m = M.mass[b];
    C.arm = M.armature[b];
    C.kp = M.kp[b];
    C.kd = M.kd[b];
    C.tmax = M.tau_max[b];
    C.qinit = M.q_init[b];
    C.b = b;
    return C;
}

// Pins a loop-invariant value to a register: the empty asm makes it opaque, so the
// compiler keeps it instead of recomputing or reloading it inside the step loop.
__device__ __forceinline__ void pin(R_T& x) { asm volatile("" : R_PIN(x)); }
__device__ __forceinline__ void pin(V3<R_T>& v) {
    pin(v.x);
    pin(v.y);
    pin(v.z);
}
__device__ __forceinline__ void pin(BodyConst& C) {
    pin(C.a);
    pin(C.r);
    pin(C.mc);
#pragma unroll
    for (int t = 0; t < 6; ++t) pin(C.Ao[t]);
    pin(C.m);
    pin(C.arm);
    pin(C.kp);
    pin(C.kd);
    pin(C.tmax);
    pin(C.qinit);
}

// Axis-vector operations with a = the joint axis (component AX for a coordinate axis).
template <int AX>
__device__ __forceinline__ V3<R_T> add_ax(const BodyConst& C, V3<R_T> v, R_T x) {  // v + x a
    if constexpr (AX == 0) return v3(v.x + x, v.y, v.z);
    else if constexpr (AX == 1) return v3(v.x, v.y + x, v.z);
    else if constexpr (AX == 2) return v3(v.x, v.y, v.z + x);
    else return v + x * C.a;
}
template <int AX>
__device__ __forceinline__ V3<R_T> cross_ax(const BodyConst& C, V3<R_T> w, R_T x) {  // w x (x a)
    if constexpr (AX == 0) return v3(R_C(0.), w.z * x, -(w.y * x));
    else if constexpr (AX == 1) return v3(-(w.z * x), R_C(0.), w.x * x);
    else if constexpr (AX == 2) return v3(w.y * x, -(w.x * x), R_C(0.));
    else return cross(w, x * C.a);
}
template <int AX>
__device__ __forceinline__ R_T dot_ax(const BodyConst& C, V3<R_T> v) {  // a . v
    if constexpr (AX == 0) return v.x;
    else if constexpr (AX == 1) return v.y;
    else if constexpr (AX == 2) return v.z;
    else return dot(C.a, v);
}
template <int AX>
__device__ __forceinline__ V3<R_T> symcol_ax(const BodyConst& C, const R_T* S) {  // S a
    if constexpr (AX == 0) return v3(S[0], S[3], S[4]);
    else if constexpr (AX == 1) return v3(S[3], S[1], S[5]);
    else if constexpr (AX == 2) return v3(S[4], S[5], S[2]);
    else return sym_mul(S, C.a);
}
template <int AX>
__device__ __forceinline__ V3<R_T> btcol_ax(const BodyConst& C, const R_T* B) {  // B^T a
    if constexpr (AX >= 0) {
        return v3(B[3 * AX], B[3 * AX + 1], B[3 * AX + 2]);
    } else {
        const V3<R_T> a = C.a;
        return v3(B[0] * a.x + B[3] * a.y + B[6] * a.z, B[1] * a.x + B[4] * a.y + B[7] * a.z,
                  B[2] * a.x + B[5] * a.y + B[8] * a.z);
    }
}

// S v, B v and B^T v for a vector v whose component AX is zero (AX < 0: any v).
template <int AX>
__device__ __forceinline__ V3<R_T> sym_mul_z(const R_T* S, V3<R_T> v) {
    if constexpr (AX == 0) return v3(S[3] * v.y + S[4] * v.z, S[1] * v.y + S[5] * v.z, S[5] * v.y + S[2] * v.z);
    else if constexpr (AX == 1) return v3(S[0] * v.x + S[4] * v.z, S[3] * v.x + S[5] * v.z, S[4] * v.x + S[2] * v.z);
    else if constexpr (AX == 2) return v3(S[0] * v.x + S[3] * v.y, S[3] * v.x + S[1] * v.y, S[4] * v.x + S[5] * v.y);
    else return sym_mul(S, v);
}
template <int AX>
__device__ __forceinline__ V3<R_T> mul_z(const M3<R_T>& B, V3<R_T> v) {
    if constexpr (AX == 0)
        return v3(B.m[1] * v.y + B.m[2] * v.z, B.m[4] * v.y + B.m[5] * v.z, B.m[7] * v.y + B.m[8] * v.z);
    else if constexpr (AX == 1)
        return v3(B.m[0] * v.x + B.m[2] * v.z, B.m[3] * v.x + B.m[5] * v.z, B.m[6] * v.x + B.m[8] * v.z);
    else if constexpr (AX == 2)
        return v3(B.m[0] * v.x + B.m[1] * v.y, B.m[3] * v.x + B.m[4] * v.y, B.m[6] * v.x + B.m[7] * v.y);
    else return mul(B, v);
}
template <int AX>
__device__ __forceinline__ V3<R_T> mulT_z(const M3<R_T>& B, V3<R_T> v) {
    if constexpr (AX == 0)
        return v3(B.m[3] * v.y + B.m[6] * v.z, B.m[4] * v.y + B.m[7] * v.z, B.m[5] * v.y + B.m[8] * v.z);
    else if constexpr (AX == 1)
        return v3(B.m[0] * v.x + B.m[6] * v.z, B.m[1] * v.x + B.m[7] * v.z, B.m[2] * v.x + B.m[8] * v.z);
    else if constexpr (AX == 2)
        return v3(B.m[0] * v.x + B.m[3] * v.y, B.m[1] * v.x + B.m[4] * v.y, B.m[2] * v.x + B.m[5] * v.y);
    else return mulT(B, v);
}

template <bool KEEP, int AX>
__device__ __forceinline__ JRot<AX> joint_rot(const BodyConst& C, const BodyMem& m) {
    if constexpr (AX >= 0) {
        return JRot<AX>{m.s, m.c};
    } else {
        if (KEEP) return JRot<-1>{m.R};
        return JRot<-1>{axis_rotation(C.a, m.s, m.c)};
    }
}

struct Pose {
    M3<R_T> R;
    V3<R_T> p, w, v;
};


// Contact forces of body b's points; with the modular cost (PAPER), `count` lanes also
// add the points' running-cost terms to pcost (a replicated body counts on one lane).
template <bool PAPER>
__device__ __forceinline__ void body_contacts(const DevModel<R_T>& M, int b, const Pose& P, V3<R_T>& fen,
                                              V3<R_T>& fef, R_T& pcost, bool count) {
    const int c0 = M.cfirst[b], cn = M.ccount[b];
    const bool paper = PAPER && count;
    for (int c = 0; c < cn; ++c) {
        const int ci = c0 + c;
        const V3<R_T> rc = v3(M.cpos[0][ci], M.cpos[1][ci], M.cpos[2][ci]);
        const V3<R_T> pc = P.p + mul(P.R, rc);
        const R_T depth = -pc.z;
        if (depth > R_C(0.)) {
            const V3<R_T> vw = mul(P.R, P.v + cross(P.w, rc));
            const R_T fn = R_MAX(M.contact_k * depth - M.contact_c * vw.z, R_C(0.));
            const R_T sc = -M.mu * fn * R_RSQRT(vw.x * vw.x + vw.y * vw.y + M.eps_f * M.eps_f);
            const V3<R_T> F = v3(sc * vw.x, sc * vw.y, fn);
            const V3<R_T> fb = mulT(P.R, F);
            fef = fef + fb;
            fen = fen + cross(rc, fb);
            if (paper) pcost += contact_cost(M, vw, F);
        } else if (paper) {
            pcost += M.cf_off;
        }
    }
}

// v x* (I v) - f_ext for body b (see the warp kernel for the exact-cancellation form).
__device__ __forceinline__ void body_bias(const BodyConst& C, const Pose& P, V3<R_T> fen, V3<R_T> fef,
                                          V3<R_T>& pn, V3<R_T>& pf) {
    const R_T* Ao = C.Ao;
    const V3<R_T> mc = C.mc;
    const V3<R_T> mcw = cross(mc, P.w);
    const V3<R_T> hn = sym_mul(Ao, P.w) + cross(mc, P.v);
    const V3<R_T> hf = C.m * P.v - mcw;
    pn = cross(P.w, hn) - cross(P.v, mcw) - fen;
    pf = cross(P.w, hf) - fef;
}

__device__ __forceinline__ void body_inertia(const BodyConst& C, Art<R_T>& IA) {
    const V3<R_T> mc = C.mc;
#pragma unroll
    for (int t = 0; t < 6; ++t) IA.A[t] = C.Ao[t];
    IA.B[0] = R_C(0.);
    IA.B[1] = -mc.z;
    IA.B[2] = mc.y;
    IA.B[3] = mc.z;
    IA.B[4] = R_C(0.);
    IA.B[5] = -mc.x;
    IA.B[6] = -mc.y;
    IA.B[7] = mc.x;
    IA.B[8] = R_C(0.);
    IA.C[0] = IA.C[1] = IA.C[2] = C.m;
    IA.C[3] = IA.C[4] = IA.C[5] = R_C(0.);
}

// Pass 1 of revolute body b from its parent's pose P: its pose, the velocity product and
// the bias (contact forces included).
template <bool KEEP, bool PAPER, int AX, int OF, bool CONTACTS = true>
__device__ __forceinline__ void body_pass1(const DevModel<R_T>& M, const BodyConst& C, R_T q, R_T qd,
                                           const Pose& Pp, Pose& P, BodyMem& m, R_T& pcost, bool count) {
    const V3<R_T> r = C.r;
    R_SINCOS(q, &m.s, &m.c);
    JRot<AX> J;
    if constexpr (AX >= 0) {
        J.s = m.s;
        J.c = m.c;
    } else {
        J.R = axis_rotation(C.a, m.s, m.c);
        if (KEEP) m.R = J.R;
    }
    P.R = jcompose(Pp.R, J);
    if constexpr (OF == 5) P.p = Pp.p;
    else P.p = Pp.p + rot_r<OF>(Pp.R, r);
    P.w = add_ax<AX>(C, jrotT(J, Pp.w), qd);
    P.v = jrotT(J, add_rcross<OF>(Pp.v, r, Pp.w, -R_C(1.)));
    m.cw = cross_ax<AX>(C, P.w, qd);
    m.cv = cross_ax<AX>(C, P.v, qd);
    V3<R_T> fen = v3(R_C(0.), R_C(0.), R_C(0.)), fef = fen;
    if (CONTACTS) body_contacts<PAPER>(M, C.b, P, fen, fef, pcost, count);
    body_bias(C, P, fen, fef, m.x0, m.x1);
    if (PAPER && count) {
        const R_T dq = q - C.qinit;
        pcost += M.w_q * dq * dq;
    }
}

// The joint projection of an articulated inertia IA of a body (Featherstone's U = IA S,
// D = S^T U + armature, Ia = IA - U U^T / D). For a body without children it depends on the
// model only, so a rollout computes it once for the chain leaves.
struct ArtProj {
    Art<R_T> Ia;
    V3<R_T> ua, ul, x0, x1;  // U (angular, linear) and U / D
    R_T invD;
};

template <int AX>
__device__ __forceinline__ void art_project(const BodyConst& C, const Art<R_T>& IA, ArtProj& P) {
    P.ua = symcol_ax<AX>(C, IA.A);
    P.ul = btcol_ax<AX>(C, IA.B);
    P.invD = sc_rcp(dot_ax<AX>(C, P.ua) + C.arm);
    // x = U / D; Ia = IA - U x^T
    P.x0 = P.invD * P.ua;
    P.x1 = P.invD * P.ul;
    const V3<R_T> ua = P.ua, ul = P.ul, x0 = P.x0, x1 = P.x1;
    P.Ia.A[0] = IA.A[0] - ua.x * x0.x;
    P.Ia.A[1] = IA.A[1] - ua.y * x0.y;
    P.Ia.A[2] = IA.A[2] - ua.z * x0.z;
    P.Ia.A[3] = IA.A[3] - ua.x * x0.y;
    P.Ia.A[4] = IA.A[4] - ua.x * x0.z;
    P.Ia.A[5] = IA.A[5] - ua.y * x0.z;
    const R_T U[3] = {ua.x, ua.y, ua.z}, X1[3] = {x1.x, x1.y, x1.z};
#pragma unroll
    for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
        for (int j2 = 0; j2 < 3; ++j2) P.Ia.B[3 * i2 + j2] = IA.B[3 * i2 + j2] - U[i2] * X1[j2];
    P.Ia.C[0] = IA.C[0] - ul.x * x1.x;
    P.Ia.C[1] = IA.C[1] - ul.y * x1.y;
    P.Ia.C[2] = IA.C[2] - ul.z * x1.z;
    P.Ia.C[3] = IA.C[3] - ul.x * x1.y;
    P.Ia.C[4] = IA.C[4] - ul.x * x1.z;
    P.Ia.C[5] = IA.C[5] - ul.y * x1.z;
}

// PIN keeps the projection in registers for the whole rollout; without it the compiler may
// recompute it where registers are short.
template <int AX, bool PIN = true>
__device__ __forceinline__ ArtProj leaf_projection(const BodyConst& C) {
    Art<R_T> IA;
    body_inertia(C, IA);
    ArtProj P;
    art_project<AX>(C, IA, P);
    if (!PIN) return P;
#pragma unroll
    for (int t = 0; t < 6; ++t) pin(P.Ia.A[t]);
#pragma unroll
    for (int t = 0; t < 9; ++t) pin(P.Ia.B[t]);
#pragma unroll
    for (int t = 0; t < 6; ++t) pin(P.Ia.C[t]);
    pin(P.ua);
    pin(P.ul);
    pin(P.x0);
    pin(P.x1);
    pin(P.invD);
    return P;
}

// Pass 2 of body b: its articulated inertia (own + `carry` from its child when has_carry),
// then the carry to its parent; m.x0/x1/uu become U_ang/D, U_lin/D, u/D. LEAF: the body
// has no child and `leaf` holds its projection.
template <bool KEEP, int AX, int OF, bool LEAF = false>
__device__ __forceinline__ void body_pass2(const BodyConst& C, R_T tau, BodyMem& m, bool has_carry,
                                           Art<R_T>& carry, V3<R_T>& cpn, V3<R_T>& cpf,
                                           const ArtProj* leaf = nullptr) {
    const V3<R_T> r = C.r;
    V3<R_T> pAn = m.x0, pAf = m.x1;
    ArtProj Pj;
    if constexpr (LEAF) {
        Pj = *leaf;
    } else {
        Art<R_T> IA;
        body_inertia(C, IA);
        if (has_carry) {
#pragma unroll
            for (int t = 0; t < 6; ++t) IA.A[t] += carry.A[t];
#pragma unroll
            for (int t = 0; t < 9; ++t) IA.B[t] += carry.B[t];
#pragma unroll
            for (int t = 0; t < 6; ++t) IA.C[t] += carry.C[t];
            pAn = pAn + cpn;
            pAf = pAf + cpf;
        }
        art_project<AX>(C, IA, Pj);
    }
    const Art<R_T>& Ia = Pj.Ia;
    const R_T u = tau - dot_ax<AX>(C, pAn);
    const R_T ud = u * Pj.invD;
    const M3<R_T>& Bm = *reinterpret_cast<const M3<R_T>*>(Ia.B);
    // c = (cw, cv) has a zero component AX (it is a cross product with the joint axis)
    const V3<R_T> pan = pAn + sym_mul_z<AX>(Ia.A, m.cw) + mul_z<AX>(Bm, m.cv) + ud * Pj.ua;
    const V3<R_T> paf = pAf + mulT_z<AX>(Bm, m.cw) + sym_mul_z<AX>(Ia.C, m.cv) + ud * Pj.ul;
    const JRot<AX> J = joint_rot<KEEP, AX>(C, m);
    jart_to_parent<AX, OF>(Ia, J, r, carry);
    cpf = jrot(J, paf);
    cpn = add_rcross<OF>(jrot(J, pan), r, cpf, R_C(1.));
    m.x0 = Pj.x0;
    m.x1 = Pj.x1;
    m.uu = ud;
}

// Pass 3 of body b: from the parent's acceleration (apw, apv, offset by gravity) to its
// own, and its joint acceleration.
template <bool KEEP, int AX, int OF>
__device__ __forceinline__ R_T body_pass3(const BodyConst& C, const BodyMem& m, V3<R_T>& apw, V3<R_T>& apv) {
    const V3<R_T> r = C.r;
    const JRot<AX> J = joint_rot<KEEP, AX>(C, m);
    const V3<R_T> a1w = jrotT(J, apw) + m.cw;
    const V3<R_T> a1v = jrotT(J, add_rcross<OF>(apv, r, apw, -R_C(1.))) + m.cv;
    const R_T qdd = m.uu - dot(m.x0, a1w) - dot(m.x1, a1v);
    apw = add_ax<AX>(C, a1w, qdd);
    apv = a1v;
    return qdd;
}

struct SegKnots {
    R_T q0, v0, q1, v1;
};

__device__ __forceinline__ SegKnots seg_knots(const float* __restrict__ knots, int nj, int k, int b) {
    const int j = b - 1;
    return SegKnots{knots[(k * 2 + 0) * nj + j], knots[(k * 2 + 1) * nj + j], knots[((k + 1) * 2 + 0) * nj + j],
                    knots[((k + 1) * 2 + 1) * nj + j]};
}

// Power-basis form of one joint's Hermite segment (Eq. hermite_segment expanded in s, with
// m = dtk v): q(s) = ((c3 s + c2) s + c1) s + c0, c0 = q0, c1 = m0,
// c2 = 3 (q1 - q0) - 2 m0 - m1, c3 = -2 (q1 - q0) + m0 + m1; dq/dt = dq/ds / dtk. Formed
// once per segment, evaluated in 5 fused multiply-adds per step.
struct SegPoly {
    R_T c0, c1, c2, c3;
};

__device__ __forceinline__ SegPoly seg_poly(const SegKnots& K, R_T dtk) {
    const R_T m0 = dtk * K.v0, m1 = dtk * K.v1, dq = K.q1 - K.q0;
    return SegPoly{K.q0, m0, R_FMA(R_C(3.), dq, -R_FMA(R_C(2.), m0, m1)), R_FMA(-R_C(2.), dq, m0 + m1)};
}

__device__ __forceinline__ R_T poly_pd(const BodyConst& C, const SegPoly& P, R_T s, R_T inv_dtk, R_T q,
                                         R_T qd) {
    const R_T qref = R_FMA(R_FMA(R_FMA(P.c3, s, P.c2), s, P.c1), s, P.c0);
    const R_T vref = R_FMA(R_FMA(R_C(3.) * P.c3, s, R_C(2.) * P.c2), s, P.c1) * inv_dtk;
    return sc_clamp(C.kp * (qref - q) + C.kd * (vref - qd), -C.tmax, C.tmax);
}

__device__ __forceinline__ R_T hermite_pd(const BodyConst& C, const SegKnots& K, R_T s, R_T dtk,
                                            R_T inv_dtk, R_T q, R_T qd) {
    const R_T q0 = K.q0, v0 = K.v0, q1 = K.q1, v1 = K.v1;
    const R_T s2 = s * s, s3 = s2 * s;
    const R_T h00 = R_C(2.) * s3 - R_C(3.) * s2 + R_C(1.), h10 = s3 - R_C(2.) * s2 + s;
    const R_T h01 = -R_C(2.) * s3 + R_C(3.) * s2, h11 = s3 - s2;
    const R_T d00 = R_C(6.) * s2 - R_C(6.) * s, d10 = R_C(3.) * s2 - R_C(4.) * s + R_C(1.);
    const R_T d01 = -R_C(6.) * s2 + R_C(6.) * s, d11 = R_C(3.) * s2 - R_C(2.) * s;
    const R_T qref = h00 * q0 + h10 * dtk * v0 + h01 * q1 + h11 * dtk * v1;
    const R_T vref = (d00 * q0 + d01 * q1) * inv_dtk + d10 * v0 + d11 * v1;
    return sc_clamp(C.kp * (qref - q) + C.kd * (vref - qd), -C.tmax, C.tmax);
}

__device__ __forceinline__ void cost_terms(const DevModel<R_T>& M, const Pose& P, R_T& tz, R_T& tt) {
    const R_T dz = P.p.z - M.z_des;
    const R_T tilt = R_ATAN2P(R_SQRT(P.R.m[2] * P.R.m[2] + P.R.m[5] * P.R.m[5]), P.R.m[8]);
    tz = M.w_z * dz * dz;
    tt = M.w_tilt * tilt * tilt;
}

// One sample's rollout by the 4 lanes of its group (g = lane within the group).
// The lane plan (first body and length of each lane's chain, the branch body and which
// lanes carry it) is in the model: lane_b0, lane_len, branch. PAPER compiles the
// modular cost of Sec. IV-A in (models with any of its weights non-zero).
template <int LMAX, bool BRANCH, bool PAPER, int AXP>
__device__ __noinline__ R_T lanes_rollout(const DevModel<R_T>& M, int g, const double* __restrict__ x0,
                                            const float* __restrict__ knots, int H, int nk, R_T dt, R_T dtk,
                                            double* __restrict__ xf) {
    constexpr bool KEEP = LMAX <= 3;  // short chains keep rotations and segment knots in registers
    // under the x, y, y plan every contact point sits on a calf (model creation checks it),
    // so the base, hips and thighs skip the contact loop
    constexpr bool LEAF_CONTACTS = AXP == AXP_XYY;
    const int nj = M.nb - 1, nq = 7 + nj;
    const int b0 = M.lane_b0[g];
    // the x, y, y plan has 3 bodies in every chain: a compile-time length drops the
    // per-body length tests from the step loop (the launch got 9 % shorter)
    const int len = AXP == AXP_XYY ? LMAX : M.lane_len[g];
    const int bb = BRANCH ? M.branch_body : 0;
    const bool on_branch = BRANCH && g >= 2;  // lanes 2 and 3 carry the branch body
    // base (replicated), branch joint (replicated on lanes 2, 3), chain joints
    Pose B;
    V3<R_T> p = v3((R_T)x0[0], (R_T)x0[1], (R_T)x0[2]);
    const V3<R_T> p_start = p;
    R_T qw = (R_T)x0[3], qx = (R_T)x0[4], qy = (R_T)x0[5], qz = (R_T)x0[6];
    V3<R_T> vl = v3((R_T)x0[nq], (R_T)x0[nq + 1], (R_T)x0[nq + 2]);
    V3<R_T> w = v3((R_T)x0[nq + 3], (R_T)x0[nq + 4], (R_T)x0[nq + 5]);
    R_T qb = R_C(0.), qdb = R_C(0.);
    if (BRANCH) {
        qb = (R_T)x0[7 + bb - 1];
        qdb = (R_T)x0[nq + 6 + bb - 1];
    }
    R_T q[LMAX], qd[LMAX];
#pragma unroll
    for (int j = 0; j < LMAX; ++j) {
        q[j] = j < len ? (R_T)x0[7 + b0 - 1 + j] : R_C(0.);
        qd[j] = j < len ? (R_T)x0[nq + 6 + b0 - 1 + j] : R_C(0.);
    }
    const R_T inv_dtk = R_C(1.0) / dtk;
    R_T sum = R_C(0.), comp = R_C(0.);
    const int cb = M.cost_body;
    int cowner = 0;  // lane that owns the cost body (0 for the base: every lane has it)
    for (int l = 0; l < LANES; ++l)
        if (cb >= M.lane_b0[l] && cb < M.lane_b0[l] + M.lane_len[l]) cowner = l;
    if (BRANCH && cb == bb) cowner = 2;
    SegPoly kc[KEEP ? LMAX : 1];
    // short chains keep their bodies' constants (and the base's) in registers; long chains
    // re-read them from shared memory where they are used
    BodyConst bc[KEEP ? LMAX : 1];
    BodyConst bc0;
    if (KEEP) {
#pragma unroll
        for (int j = 0; j < LMAX; ++j) {
            bc[j] = load_body(M, j < len ? b0 + j : b0);
            pin(bc[j]);
        }
        bc0 = load_body(M, 0);
        pin(bc0);
    }
    auto body = [&](int j) -> BodyConst { return KEEP ? bc[KEEP ? j : 0] : load_body(M, b0 + j); };
    // under the x, y, y plan every chain has 3 bodies: the calf is the leaf
    ArtProj leafp;
    if constexpr (AXP == AXP_XYY) leafp = leaf_projection<chain_axis<AXP, 2>()>(bc[2]);
    auto base = [&]() -> BodyConst { return KEEP ? bc0 : load_body(M, 0); };
    int kcur = -1;
    // segment k = floor(h (nk - 1) / H) and its remainder rem = h (nk - 1) - k H, advanced
    // by integer steps instead of a division per step; s = rem / H
    const R_T inv_H = R_C(1.0) / (R_T)H;
    int k = 0, rem = -(nk - 1);
    pdl_wait();  // the knots (a solve's noise kernel may still be writing them)
    for (int h = 0; h < H; ++h) {
        rem += nk - 1;
        while (rem >= H) {
            rem -= H;
            ++k;
        }
        if (!MPPI_CHECK_OK(k + 1 < nk, CHECK_KNOT)) k = nk - 2;
        const R_T s = (R_T)rem * inv_H;
        if (KEEP && k != kcur) {
            kcur = k;
#pragma unroll
            for (int j = 0; j < (KEEP ? LMAX : 1); ++j)
                if (j < len) kc[j] = seg_poly(seg_knots(knots, nj, k, b0 + j), dtk);
        }
        R_T tau[LMAX], taub = R_C(0.);
#pragma unroll
        for (int j = 0; j < LMAX; ++j) {
            if (KEEP)
                tau[j] = j < len ? poly_pd(body(j), kc[KEEP ? j : 0], s, inv_dtk, q[j], qd[j]) : R_C(0.);
            else
                tau[j] = j < len ? hermite_pd(body(j), seg_knots(knots, nj, k, b0 + j), s, dtk, inv_dtk, q[j], qd[j])
                                 : R_C(0.);
        }
        if (on_branch) taub = hermite_pd(load_body(M, bb), seg_knots(knots, nj, k, bb), s, dtk, inv_dtk, qb, qdb);
        // ---- pass 1 ----
        B.R = quat_to_R(qw, qx, qy, qz);
        B.p = p;
        B.w = w;  // chain plans exist only for floating bases (model creation)
        B.v = vl;
        V3<R_T> p0n, p0f;
        R_T pcost = R_C(0.);  // this lane's share of the modular running cost
        {
            V3<R_T> fen = v3(R_C(0.), R_C(0.), R_C(0.)), fef = fen;
            if (!LEAF_CONTACTS) body_contacts<PAPER>(M, 0, B, fen, fef, pcost, g == 0);
            body_bias(base(), B, fen, fef, p0n, p0f);
        }
        if constexpr (PAPER) {  // every lane holds the base: no divergent branch, lane 0 counts it
            const R_T bcst = base_cost(M, B.R, B.p);
            pcost += g == 0 ? bcst : R_C(0.);
        }
        R_T tz = R_C(0.), tt = R_C(0.);
        // inputs of the cost terms (height and the rotation's last column) of this lane's
        // cost body, picked by selects along pass 1 (the base unless a chain body is it)
        R_T cpz = B.p.z, cr2 = B.R.m[2], cr5 = B.R.m[5], cr8 = B.R.m[8];
        BodyMem mb;
        Pose PB;
        if (on_branch) {
            body_pass1<KEEP, PAPER, -1, -1>(M, load_body(M, bb), qb, qdb, B, PB, mb, pcost, g == 2);
            if (cb == bb) cost_terms(M, PB, tz, tt);
        }
        BodyMem mem[LMAX];
        {
            Pose Pp = on_branch ? PB : B;
            static_for<0, LMAX>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                if (j < len) {
                    Pose P;
                    body_pass1<KEEP, PAPER, chain_axis<AXP, j>(), chain_offset<AXP, j>(), !LEAF_CONTACTS || j == 2>(
                        M, body(j), q[j], qd[j], Pp, P, mem[j], pcost, true);
                    if constexpr (AXP == AXP_XYY) {
                        const bool own = cb == b0 + j;
                        cpz = own ? P.p.z : cpz;
                        cr2 = own ? P.R.m[2] : cr2;
                        cr5 = own ? P.R.m[5] : cr5;
                        cr8 = own ? P.R.m[8] : cr8;
                    } else if (cb == b0 + j) {
                        cost_terms(M, P, tz, tt);
                    }
                    Pp = P;
                }
            });
        }
        if constexpr (AXP == AXP_XYY) {
            Pose Pc;
            Pc.p.z = cpz;
            Pc.R.m[2] = cr2;
            Pc.R.m[5] = cr5;
            Pc.R.m[8] = cr8;
            cost_terms(M, Pc, tz, tt);
        } else if (cb == 0) {
            cost_terms(M, B, tz, tt);
        }
        // from the lane that owns the cost body (lane 0 holds the base's terms like every lane)
        tz = __shfl_sync(0xffffffffu, tz, cowner, LANES);
        tt = __shfl_sync(0xffffffffu, tt, cowner, LANES);
        // ---- pass 2 ----
        Art<R_T> carry;
        V3<R_T> cpn = v3(R_C(0.), R_C(0.), R_C(0.)), cpf = cpn;
        static_for<0, LMAX>([&](auto ic) {
            constexpr int j = LMAX - 1 - decltype(ic)::value;
            if constexpr (AXP == AXP_XYY && j == 2)
                body_pass2<KEEP, chain_axis<AXP, j>(), chain_offset<AXP, j>(), true>(body(j), tau[j], mem[j], false,
                                                                                    carry, cpn, cpf, &leafp);
            else if (j < len)
                body_pass2<KEEP, chain_axis<AXP, j>(), chain_offset<AXP, j>()>(body(j), tau[j], mem[j], j < len - 1,
                                                                              carry, cpn, cpf);
        });
        if (BRANCH) {
            // arms meet at the branch body: own + partner (lanes 2 <-> 3), identical on both
            Art<R_T> sumc;
#pragma unroll
            for (int t = 0; t < 6; ++t) sumc.A[t] = carry.A[t] + __shfl_xor_sync(0xffffffffu, carry.A[t], 1, LANES);
#pragma unroll
            for (int t = 0; t < 9; ++t) sumc.B[t] = carry.B[t] + __shfl_xor_sync(0xffffffffu, carry.B[t], 1, LANES);
#pragma unroll
            for (int t = 0; t < 6; ++t) sumc.C[t] = carry.C[t] + __shfl_xor_sync(0xffffffffu, carry.C[t], 1, LANES);
            const V3<R_T> sn = v3(cpn.x + __shfl_xor_sync(0xffffffffu, cpn.x, 1, LANES),
                                    cpn.y + __shfl_xor_sync(0xffffffffu, cpn.y, 1, LANES),
                                    cpn.z + __shfl_xor_sync(0xffffffffu, cpn.z, 1, LANES));
            const V3<R_T> sf = v3(cpf.x + __shfl_xor_sync(0xffffffffu, cpf.x, 1, LANES),
                                    cpf.y + __shfl_xor_sync(0xffffffffu, cpf.y, 1, LANES),
                                    cpf.z + __shfl_xor_sync(0xffffffffu, cpf.z, 1, LANES));
            if (on_branch) {
                carry = sumc;
                cpn = sn;
                cpf = sf;
                body_pass2<KEEP, -1, -1>(load_body(M, bb), taub, mb, true, carry, cpn, cpf);
                if (g == 3) {  // lane 2 alone hands the branch to the base
#pragma unroll
                    for (int t = 0; t < 6; ++t) carry.A[t] = R_C(0.);
#pragma unroll
                    for (int t = 0; t < 9; ++t) carry.B[t] = R_C(0.);
#pragma unroll
                    for (int t = 0; t < 6; ++t) carry.C[t] = R_C(0.);
                    cpn = v3(R_C(0.), R_C(0.), R_C(0.));
                    cpf = cpn;
                }
            }
        }
        // ---- base: every lane's contribution (butterfly), solve ----
        Art<R_T> IA0;
        body_inertia(base(), IA0);
#pragma unroll
        for (int t = 0; t < 6; ++t) IA0.A[t] += lsum(carry.A[t]);
#pragma unroll
        for (int t = 0; t < 9; ++t) IA0.B[t] += lsum(carry.B[t]);
#pragma unroll
        for (int t = 0; t < 6; ++t) IA0.C[t] += lsum(carry.C[t]);
        p0n = p0n + v3(lsum(cpn.x), lsum(cpn.y), lsum(cpn.z));
        p0f = p0f + v3(lsum(cpf.x), lsum(cpf.y), lsum(cpf.z));
        const V3<R_T> g_b = v3(-M.gravity * B.R.m[6], -M.gravity * B.R.m[7], -M.gravity * B.R.m[8]);
        V3<R_T> aw, av;
        {
            const R_T rhs[6] = {-p0n.x, -p0n.y, -p0n.z, -p0f.x, -p0f.y, -p0f.z};
            R_T x[6];
            art_solve(IA0, rhs, x);
            aw = v3(x[0], x[1], x[2]);
            av = v3(x[3], x[4], x[5]);
        }
        // ---- pass 3 ----
        R_T qdd[LMAX], qddb = R_C(0.);
        {
            V3<R_T> apw = aw, apv = av;
            if (on_branch) qddb = body_pass3<KEEP, -1, -1>(load_body(M, bb), mb, apw, apv);
            static_for<0, LMAX>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                qdd[j] = j < len ? body_pass3<KEEP, chain_axis<AXP, j>(), chain_offset<AXP, j>()>(body(j), mem[j], apw, apv) : R_C(0.);
            });
        }
        // ---- running cost on the pre-step state ----
        R_T te = R_C(0.);
#pragma unroll
        for (int j = 0; j < LMAX; ++j) te += tau[j] * tau[j];
        if (g == 2) te += taub * taub;
        te = lsum(te);
        if (PAPER) pcost = lsum(pcost);
        {
            const R_T vx = B.R.m[0] * vl.x + B.R.m[1] * vl.y + B.R.m[2] * vl.z;
            const R_T dv = vx - M.vx_des;
            R_T c = tz + M.w_vx * dv * dv + tt + M.w_tau * te;
            if (PAPER) c += pcost;
            const R_T y = c - comp;
            const R_T t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
        // ---- semi-implicit Euler ----
#pragma unroll
        for (int j = 0; j < LMAX; ++j) {
            qd[j] += dt * qdd[j];
            q[j] += dt * qd[j];
        }
        if (on_branch) {
            qdb += dt * qddb;
            qb += dt * qdb;
        }
        {
            w = w + dt * aw;
            vl = vl + dt * (av + g_b);
            p = p + dt * mul(B.R, vl);
            const R_T wn = R_SQRT(dot(w, w));
            // both branches evaluated, one selected: no branch splits the step's last block
            const bool tiny = wn * dt < R_C(1e-12);
            R_T sh, ch;
            R_SINCOS(R_C(0.5) * wn * dt, &sh, &ch);
            const R_T dq0 = tiny ? R_C(1.) : ch;
            const R_T dqs = tiny ? R_C(0.5) * dt : R_FDIV(sh, wn);
            const R_T dx = dqs * w.x, dy = dqs * w.y, dz = dqs * w.z;
            const R_T nw = qw * dq0 - qx * dx - qy * dy - qz * dz;
            const R_T nx = qw * dx + qx * dq0 + qy * dz - qz * dy;
            const R_T ny = qw * dy - qx * dz + qy * dq0 + qz * dx;
            const R_T nz = qw * dz + qx * dy - qy * dx + qz * dq0;
            const R_T inv = R_RSQRT(nw * nw + nx * nx + ny * ny + nz * nz);
            qw = nw * inv;
            qx = nx * inv;
            qy = ny * inv;
            qz = nz * inv;
        }
    }
    if (PAPER) {  // terminal cost (every lane holds the base)
        const R_T y = terminal_cost(M, p, p_start, H, dt) - comp;
        const R_T t = sum + y;
        comp = (t - sum) - y;
        sum = t;
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
        if (BRANCH && g == 2) {
            xf[7 + bb - 1] = qb;
            xf[nq + 6 + bb - 1] = qdb;
        }
#pragma unroll
        for (int j = 0; j < LMAX; ++j)
            if (j < len) {
                xf[7 + b0 - 1 + j] = q[j];
                xf[nq + 6 + b0 - 1 + j] = qd[j];
            }
    }
    return sum;
}

R_NS_END

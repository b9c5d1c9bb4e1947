// Two-warp split of the lanes-per-chain rollout, for trees of the usual humanoid layout
// (axis plan AXP_HUM in common.cuh): a pair of warps rolls out 16 samples. The leg warp
// runs both leg chains of each sample (2 lanes per sample, one leg each) and owns the
// floating base; its partner, the arm warp, runs the waist body and both arm chains
// (2 lanes per sample, one arm each, the waist replicated on the two). Each warp's code
// is compiled for its own chains' joint axes and offsets; one warp holding both kinds of
// chain would have to run the two specialisations one after the other.
//
// Per step the warps meet three times in shared memory (records per sample, each part
// written by one warp and read by the other behind a 64-thread named barrier):
//   A  arm -> leg: the waist subtree's articulated inertia and bias force (Featherstone's
//      articulated-body recursion, carried to the base frame) plus the base's own
//      inertia and bias force, and the arm warp's share of the running cost (with the
//      base's terms), so the leg warp, whose chain is the longer one, only adds;
//   B  leg -> arm: the base acceleration of this step, from the leg warp's base solve;
//   C  arm -> leg: the base pose of the next step: the arm warp integrates the base while
//      the leg warp runs its third pass.
// The base is integrated once, by the arm warp, so every base quantity the two warps use
// is the same bits. A record part is written before a barrier and read after it, and its
// next write comes after a later barrier, so one buffer per direction suffices.
// Left and right chains meet by a pair shuffle (a commutative sum: both lanes of a pair
// hold the same bits). Equations as in the other rollout kernels: Sec. III-A Hermite
// setpoints, Sec. III-C PD tracking, the articulated-body algorithm, semi-implicit Euler,
// Kahan-summed running cost (Alg. 1).
//
// A body included after rollout_lanes.cuh by chain_f32.cuh (FP32) and by the FP64 check
// build's translation unit, with the scalar macros of scalar_macros.h.
R_NS_BEGIN

constexpr int SPLIT_SPP = 16;                                 // samples per warp pair
constexpr int SPLIT_REC = 36;                                 // values per record (16-B aligned, bank-spread)
constexpr int SPLIT_PAIR_FLOATS = 2 * SPLIT_SPP * SPLIT_REC;  // values: records A, then records B
constexpr int SPLIT_LEG = 6, SPLIT_ARM = 4;
constexpr int SPLIT_WAIST_AX = 2, SPLIT_WAIST_OF = 2;         // waist: about z, offset along z

// Joint axis and offset codes (as in rollout_lanes.cuh) of chain position J of the leg
// (ROLE 0: z, x, y, y, y, x; offsets yz-plane, z, 0, z, z, 0) and arm chains (ROLE 1:
// y, x, z, y; offsets yz-plane, y, 0, z).
template <int ROLE, int J>
__host__ __device__ constexpr int split_axis() {
    return ROLE == 0 ? (J == 0 ? 2 : ((J == 1 || J == 5) ? 0 : 1)) : (J == 0 ? 1 : (J == 1 ? 0 : (J == 2 ? 2 : 1)));
}
template <int ROLE, int J>
__host__ __device__ constexpr int split_offset() {
    return ROLE == 0 ? (J == 0 ? 4 : ((J == 2 || J == 5) ? 5 : 2)) : (J == 0 ? 4 : (J == 1 ? 1 : (J == 2 ? 5 : 2)));
}

// Named barrier of the two warps of a pair (ids 1.. ; 0 is __syncthreads). Its memory
// clobber makes the compiler reload the records after it: the record pointers must not be
// declared __restrict__, since the partner warp writes the same words.
__device__ __forceinline__ void pair_sync(int id) { asm volatile("barrier.sync %0, 64;" ::"r"(id) : "memory"); }

__device__ __forceinline__ R_T pair_sum(R_T v) { return v + __shfl_xor_sync(0xffffffffu, v, 1); }

__device__ __forceinline__ void pair_sum(Art<R_T>& c, V3<R_T>& n, V3<R_T>& f) {
#pragma unroll
    for (int t = 0; t < 6; ++t) c.A[t] = pair_sum(c.A[t]);
#pragma unroll
    for (int t = 0; t < 9; ++t) c.B[t] = pair_sum(c.B[t]);
#pragma unroll
    for (int t = 0; t < 6; ++t) c.C[t] = pair_sum(c.C[t]);
    n = v3(pair_sum(n.x), pair_sum(n.y), pair_sum(n.z));
    f = v3(pair_sum(f.x), pair_sum(f.y), pair_sum(f.z));
}

// N groups of 4 values of a record (one float4 each in FP32); both lanes of a pair write
// the same values to the same words
template <int N>
__device__ __forceinline__ void rec_store(R_T* rec, const R_T (&v)[4 * N]) {
    if constexpr (std::is_same<R_T, float>::value) {
        float4* d = reinterpret_cast<float4*>(rec);
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < 4 * N; ++k) rec[k] = v[k];
    }
}
template <int N>
__device__ __forceinline__ void rec_load(const R_T* rec, R_T (&v)[4 * N]) {
    if constexpr (std::is_same<R_T, float>::value) {
        const float4* s = reinterpret_cast<const float4*>(rec);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const float4 x = s[k];
            v[4 * k] = x.x;
            v[4 * k + 1] = x.y;
            v[4 * k + 2] = x.z;
            v[4 * k + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4 * N; ++k) v[k] = rec[k];
    }
}

// record B holds two parts with different writers: the base acceleration (aw, av) at
// floats [0, 8), written by the leg warp, and the next base pose (R, p, w, v) at [8, 28),
// written by the arm warp, which integrates the base.
__device__ __forceinline__ void put_acc(R_T* rec, V3<R_T> aw, V3<R_T> av) {
    const R_T v[8] = {aw.x, aw.y, aw.z, av.x, av.y, av.z, R_C(0.), R_C(0.)};
    rec_store<2>(rec, v);
}
__device__ __forceinline__ void get_acc(const R_T* rec, V3<R_T>& aw, V3<R_T>& av) {
    R_T v[8];
    rec_load<2>(rec, v);
    aw = v3(v[0], v[1], v[2]);
    av = v3(v[3], v[4], v[5]);
}
__device__ __forceinline__ void put_pose(R_T* rec, const Pose& B) {
    const R_T v[20] = {B.R.m[0], B.R.m[1], B.R.m[2], B.R.m[3], B.R.m[4], B.R.m[5], B.R.m[6],
                         B.R.m[7], B.R.m[8], B.p.x,    B.p.y,    B.p.z,    B.w.x,    B.w.y,
                         B.w.z,    B.v.x,    B.v.y,    B.v.z,    R_C(0.),      R_C(0.)};
    rec_store<5>(rec + 8, v);
}
__device__ __forceinline__ void get_pose(const R_T* rec, Pose& B) {
    R_T v[20];
    rec_load<5>(rec + 8, v);
#pragma unroll
    for (int t = 0; t < 9; ++t) B.R.m[t] = v[t];
    B.p = v3(v[9], v[10], v[11]);
    B.w = v3(v[12], v[13], v[14]);
    B.v = v3(v[15], v[16], v[17]);
}

// Contact forces of a foot's points, evaluated whether or not a point penetrates (no
// branch): a point above the ground gets fn = 0, so F = 0 and the sums are unchanged.
template <bool PAPER>
__device__ __forceinline__ void foot_contacts(const DevModel<R_T>& M, int b, const Pose& P, V3<R_T>& fen,
                                              V3<R_T>& fef, R_T& pcost) {
    const int c0 = M.cfirst[b], cn = M.ccount[b];
    for (int c = 0; c < cn; ++c) {
        const int ci = c0 + c;
        const V3<R_T> rc = v3(M.cpos[0][ci], M.cpos[1][ci], M.cpos[2][ci]);
        const V3<R_T> pc = P.p + mul(P.R, rc);
        const R_T depth = -pc.z;
        const bool touch = depth > R_C(0.);
        const V3<R_T> vw = mul(P.R, P.v + cross(P.w, rc));
        const R_T fn = touch ? R_MAX(M.contact_k * depth - M.contact_c * vw.z, R_C(0.)) : R_C(0.);
        const R_T sc = -M.mu * fn * R_RSQRT(vw.x * vw.x + vw.y * vw.y + M.eps_f * M.eps_f);
        const V3<R_T> F = v3(sc * vw.x, sc * vw.y, fn);
        const V3<R_T> fb = mulT(P.R, F);
        fef = fef + fb;
        fen = fen + cross(rc, fb);
        if (PAPER) pcost += touch ? contact_cost(M, vw, F) : M.cf_off;
    }
}

// Leg warp: both legs of one sample on lanes side = 0, 1, the base solve, the cost sum.
// Returns the sample's cost (the same on both lanes).
template <bool PAPER>
__device__ __noinline__ R_T split_legs(const DevModel<R_T>& M, int side, const R_T* recA, R_T* recB, int bar,
                                         const double* __restrict__ x0,
                                         const float* __restrict__ knots, int H, int nk, R_T dt, R_T dtk,
                                         double* __restrict__ xf) {
    constexpr int LEN = SPLIT_LEG;
    // the plan fixes the numbering: legs from bodies 1 and 7, the waist 13, arms from 14
    // and 18, 21 joints (compile-time, which shortens the launch)
    constexpr int nj = 21, nq = 7 + nj;
    const int b0 = 1 + 6 * side;
    const V3<R_T> p_start = v3((R_T)x0[0], (R_T)x0[1], (R_T)x0[2]);
    R_T q[LEN], qd[LEN];
#pragma unroll
    for (int j = 0; j < LEN; ++j) {
        q[j] = (R_T)x0[7 + b0 - 1 + j];
        qd[j] = (R_T)x0[nq + 6 + b0 - 1 + j];
    }
    const R_T inv_dtk = R_C(1.0) / dtk;
    R_T sum = R_C(0.), comp = R_C(0.);
    // the plan keeps the cost body off the legs (model creation checks it): no cost terms here
    const ArtProj leafp = leaf_projection<split_axis<0, LEN - 1>(), false>(load_body(M, b0 + LEN - 1));
    SegPoly kc[LEN];
    int kcur = -1;
    Pose B;
    pair_sync(bar);
    get_pose(recB, B);  // the first base pose, from the arm warp
    const R_T inv_H = R_C(1.0) / (R_T)H;
    int k = 0, rem = -(nk - 1);
    for (int h = 0; h < H; ++h) {
        rem += nk - 1;
        while (rem >= H) {
            rem -= H;
            ++k;
        }
        if (!MPPI_CHECK_OK(k + 1 < nk, CHECK_KNOT)) k = nk - 2;
        const R_T s = (R_T)rem * inv_H;
        // power-basis setpoints, formed once per segment (the registers they hold became
        // free once the base's integration moved to the arm warp)
        if (k != kcur) {
            kcur = k;
#pragma unroll
            for (int j = 0; j < LEN; ++j) kc[j] = seg_poly(seg_knots(knots, nj, k, b0 + j), dtk);
        }
        R_T tau[LEN];
#pragma unroll
        for (int j = 0; j < LEN; ++j) tau[j] = poly_pd(load_body(M, b0 + j), kc[j], s, inv_dtk, q[j], qd[j]);
        // ---- pass 1: base, then the leg ----
        R_T pc = R_C(0.);  // this lane's share of the modular running cost
        BodyMem mem[LEN];
        {
            Pose Pp = B;
            static_for<0, LEN>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                Pose P;
                body_pass1<false, PAPER, split_axis<0, j>(), split_offset<0, j>(), false>(
                    M, load_body(M, b0 + j), q[j], qd[j], Pp, P, mem[j], pc, true);
                if constexpr (j == LEN - 1) {  // the foot: its contact forces enter its bias
                    V3<R_T> fen = v3(R_C(0.), R_C(0.), R_C(0.)), fef = fen;
                    foot_contacts<PAPER>(M, b0 + j, P, fen, fef, pc);
                    mem[j].x0 = mem[j].x0 - fen;
                    mem[j].x1 = mem[j].x1 - fef;
                }
                Pp = P;
            });
        }
        // ---- pass 2: the leg inward, both legs summed at the base ----
        Art<R_T> carry;
        V3<R_T> cpn = v3(R_C(0.), R_C(0.), R_C(0.)), cpf = cpn;
        static_for<0, LEN>([&](auto ic) {
            constexpr int j = LEN - 1 - decltype(ic)::value;
            if constexpr (j == LEN - 1)
                body_pass2<false, split_axis<0, j>(), split_offset<0, j>(), true>(load_body(M, b0 + j), tau[j], mem[j],
                                                                                false, carry, cpn, cpf, &leafp);
            else
                body_pass2<false, split_axis<0, j>(), split_offset<0, j>()>(load_body(M, b0 + j), tau[j], mem[j], true,
                                                                          carry, cpn, cpf);
        });
        pair_sum(carry, cpn, cpf);
        R_T te = R_C(0.);
#pragma unroll
        for (int j = 0; j < LEN; ++j) te += tau[j] * tau[j];
        R_T lc = M.w_tau * te;
        if (PAPER) lc += pc;
        const R_T c_legs = pair_sum(lc);
        // ---- A: the waist subtree from the arm warp; base solve ----
        pair_sync(bar);
        R_T a[28];
        rec_load<7>(recA, a);
        // record A holds the waist subtree plus the base's own inertia and bias force
        Art<R_T> IA0;
#pragma unroll
        for (int t = 0; t < 6; ++t) IA0.A[t] = carry.A[t] + a[t];
#pragma unroll
        for (int t = 0; t < 9; ++t) IA0.B[t] = carry.B[t] + a[6 + t];
#pragma unroll
        for (int t = 0; t < 6; ++t) IA0.C[t] = carry.C[t] + a[15 + t];
        const V3<R_T> p0n = cpn + v3(a[21], a[22], a[23]);
        const V3<R_T> p0f = cpf + v3(a[24], a[25], a[26]);
        const R_T c_arms = a[27];
        V3<R_T> aw, av;
        {
            const R_T rhs[6] = {-p0n.x, -p0n.y, -p0n.z, -p0f.x, -p0f.y, -p0f.z};
            R_T x[6];
            art_solve(IA0, rhs, x);
            aw = v3(x[0], x[1], x[2]);
            av = v3(x[3], x[4], x[5]);
        }
        // ---- running cost on the pre-step state (the base terms came with record A) ----
        {
            const R_T c = c_legs + c_arms;
            const R_T y = c - comp;
            const R_T t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
        put_acc(recB, aw, av);
        pair_sync(bar);  // B: the arm warp integrates the base meanwhile
        // ---- pass 3 and the legs' joints ----
        R_T qdd[LEN];
        {
            V3<R_T> apw = aw, apv = av;
            static_for<0, LEN>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                qdd[j] = body_pass3<false, split_axis<0, j>(), split_offset<0, j>()>(load_body(M, b0 + j), mem[j], apw,
                                                                                   apv);
            });
        }
#pragma unroll
        for (int j = 0; j < LEN; ++j) {
            qd[j] += dt * qdd[j];
            q[j] += dt * qd[j];
        }
        pair_sync(bar);  // C: the next base pose is written
        get_pose(recB, B);
    }
    if (PAPER) {  // terminal cost (B holds the final base pose)
        const R_T y = terminal_cost(M, B.p, p_start, H, dt) - comp;
        const R_T t = sum + y;
        comp = (t - sum) - y;
        sum = t;
    }
    if (xf) {
#pragma unroll
        for (int j = 0; j < LEN; ++j) {
            xf[7 + b0 - 1 + j] = q[j];
            xf[nq + 6 + b0 - 1 + j] = qd[j];
        }
    }
    return sum;
}

// Arm warp: the waist (replicated on both lanes), one arm per lane, and the integration of
// the floating base (replicated on both lanes). Returns 0; the sample's cost is the leg
// warp's.
template <bool PAPER>
__device__ __noinline__ R_T split_arms(const DevModel<R_T>& M, int side, R_T* recA, R_T* recB, int bar,
                                         const double* __restrict__ x0,
                                         const float* __restrict__ knots, int H, int nk, R_T dt, R_T dtk,
                                         double* __restrict__ xf) {
    constexpr int LEN = SPLIT_ARM;
    constexpr int nj = 21, nq = 7 + nj;
    const int b0 = 14 + 4 * side;
    constexpr int bb = 13;
    const bool lead = side == 0;
    R_T qb = (R_T)x0[7 + bb - 1], qdb = (R_T)x0[nq + 6 + bb - 1];
    R_T q[LEN], qd[LEN];
#pragma unroll
    for (int j = 0; j < LEN; ++j) {
        q[j] = (R_T)x0[7 + b0 - 1 + j];
        qd[j] = (R_T)x0[nq + 6 + b0 - 1 + j];
    }
    const R_T inv_dtk = R_C(1.0) / dtk;
    const int cb = M.cost_body;
    const ArtProj leafp = leaf_projection<split_axis<1, LEN - 1>(), false>(load_body(M, b0 + LEN - 1));
    SegPoly kc[LEN], kb;
    int kcur = -1;
    // the floating base: integrated here, its pose handed to the leg warp each step
    V3<R_T> p = v3((R_T)x0[0], (R_T)x0[1], (R_T)x0[2]);
    R_T qw = (R_T)x0[3], qx = (R_T)x0[4], qy = (R_T)x0[5], qz = (R_T)x0[6];
    V3<R_T> vl = v3((R_T)x0[nq], (R_T)x0[nq + 1], (R_T)x0[nq + 2]);
    V3<R_T> w = v3((R_T)x0[nq + 3], (R_T)x0[nq + 4], (R_T)x0[nq + 5]);
    Pose B;
    B.R = quat_to_R(qw, qx, qy, qz);
    B.p = p;
    B.w = w;
    B.v = vl;
    put_pose(recB, B);
    pair_sync(bar);
    V3<R_T> aw, av;
    const R_T inv_H = R_C(1.0) / (R_T)H;
    int k = 0, rem = -(nk - 1);
    for (int h = 0; h < H; ++h) {
        rem += nk - 1;
        while (rem >= H) {
            rem -= H;
            ++k;
        }
        if (!MPPI_CHECK_OK(k + 1 < nk, CHECK_KNOT)) k = nk - 2;
        const R_T s = (R_T)rem * inv_H;
        if (k != kcur) {
            kcur = k;
#pragma unroll
            for (int j = 0; j < LEN; ++j) kc[j] = seg_poly(seg_knots(knots, nj, k, b0 + j), dtk);
            kb = seg_poly(seg_knots(knots, nj, k, bb), dtk);
        }
        R_T tau[LEN];
#pragma unroll
        for (int j = 0; j < LEN; ++j) tau[j] = poly_pd(load_body(M, b0 + j), kc[j], s, inv_dtk, q[j], qd[j]);
        const R_T taub = poly_pd(load_body(M, bb), kb, s, inv_dtk, qb, qdb);
        // ---- pass 1: waist, then the arm ----
        R_T pc = R_C(0.), tz = R_C(0.), tt = R_C(0.);
        BodyMem mb;
        Pose PB;
        body_pass1<false, PAPER, SPLIT_WAIST_AX, SPLIT_WAIST_OF, false>(M, load_body(M, bb), qb, qdb, B, PB, mb, pc,
                                                                        lead);
        if (cb == bb && lead) cost_terms(M, PB, tz, tt);
        BodyMem mem[LEN];
        {
            Pose Pp = PB;
            static_for<0, LEN>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                Pose P;
                body_pass1<false, PAPER, split_axis<1, j>(), split_offset<1, j>(), false>(
                    M, load_body(M, b0 + j), q[j], qd[j], Pp, P, mem[j], pc, true);
                if (cb == b0 + j) cost_terms(M, P, tz, tt);
                Pp = P;
            });
        }
        // ---- pass 2: the arm inward, both arms summed at the waist, the waist ----
        Art<R_T> carry;
        V3<R_T> cpn = v3(R_C(0.), R_C(0.), R_C(0.)), cpf = cpn;
        static_for<0, LEN>([&](auto ic) {
            constexpr int j = LEN - 1 - decltype(ic)::value;
            if constexpr (j == LEN - 1)
                body_pass2<false, split_axis<1, j>(), split_offset<1, j>(), true>(load_body(M, b0 + j), tau[j], mem[j],
                                                                                false, carry, cpn, cpf, &leafp);
            else
                body_pass2<false, split_axis<1, j>(), split_offset<1, j>()>(load_body(M, b0 + j), tau[j], mem[j], true,
                                                                          carry, cpn, cpf);
        });
        pair_sum(carry, cpn, cpf);
        body_pass2<false, SPLIT_WAIST_AX, SPLIT_WAIST_OF>(load_body(M, bb), taub, mb, true, carry, cpn, cpf);
        // the base's own inertia and bias force, and its cost terms, off the leg warp's path
        {
            Art<R_T> IB;
            body_inertia(load_body(M, 0), IB);
#pragma unroll
            for (int t = 0; t < 6; ++t) carry.A[t] += IB.A[t];
#pragma unroll
            for (int t = 0; t < 9; ++t) carry.B[t] += IB.B[t];
#pragma unroll
            for (int t = 0; t < 6; ++t) carry.C[t] += IB.C[t];
            V3<R_T> bn, bf;
            const V3<R_T> z0 = v3(R_C(0.), R_C(0.), R_C(0.));
            body_bias(load_body(M, 0), B, z0, z0, bn, bf);
            cpn = cpn + bn;
            cpf = cpf + bf;
        }
        if (PAPER && lead) pc += base_cost(M, B.R, B.p);
        if (cb == 0 && lead) cost_terms(M, B, tz, tt);
        R_T te = R_C(0.);
#pragma unroll
        for (int j = 0; j < LEN; ++j) te += tau[j] * tau[j];
        if (lead) te += taub * taub;
        R_T lc = (tz + tt) + M.w_tau * te;
        if (PAPER) lc += pc;
        if (lead) {
            const R_T vx = B.R.m[0] * B.v.x + B.R.m[1] * B.v.y + B.R.m[2] * B.v.z;
            const R_T dv = vx - M.vx_des;
            lc += M.w_vx * dv * dv;
        }
        {
            const R_T v[28] = {carry.A[0], carry.A[1], carry.A[2], carry.A[3], carry.A[4], carry.A[5], carry.B[0],
                                 carry.B[1], carry.B[2], carry.B[3], carry.B[4], carry.B[5], carry.B[6], carry.B[7],
                                 carry.B[8], carry.C[0], carry.C[1], carry.C[2], carry.C[3], carry.C[4], carry.C[5],
                                 cpn.x,      cpn.y,      cpn.z,      cpf.x,      cpf.y,      cpf.z,      pair_sum(lc)};
            rec_store<7>(recA, v);
        }
        pair_sync(bar);  // A: the leg warp may read
        pair_sync(bar);  // B: base acceleration written
        get_acc(recB, aw, av);
        // ---- base: semi-implicit Euler, quaternion exponential; the next pose to the leg warp ----
        {
            const V3<R_T> g_b = v3(-M.gravity * B.R.m[6], -M.gravity * B.R.m[7], -M.gravity * B.R.m[8]);
            w = w + dt * aw;
            vl = vl + dt * (av + g_b);
            p = p + dt * mul(B.R, vl);
            const R_T wn = R_SQRT(dot(w, w));
            // both branches evaluated, one selected (no branch in the step)
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
        Pose Bn;
        Bn.R = quat_to_R(qw, qx, qy, qz);
        Bn.p = p;
        Bn.w = w;
        Bn.v = vl;
        put_pose(recB, Bn);
        // ---- pass 3 and the waist's and arm's joints ----
        R_T qdd[LEN], qddb;
        {
            V3<R_T> apw = aw, apv = av;
            qddb = body_pass3<false, SPLIT_WAIST_AX, SPLIT_WAIST_OF>(load_body(M, bb), mb, apw, apv);
            static_for<0, LEN>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                qdd[j] = body_pass3<false, split_axis<1, j>(), split_offset<1, j>()>(load_body(M, b0 + j), mem[j], apw,
                                                                                   apv);
            });
        }
#pragma unroll
        for (int j = 0; j < LEN; ++j) {
            qd[j] += dt * qdd[j];
            q[j] += dt * qd[j];
        }
        qdb += dt * qddb;
        qb += dt * qdb;
        pair_sync(bar);  // C: the leg warp may read the next pose
        B = Bn;
    }
    if (xf) {
        if (lead) {
            xf[7 + bb - 1] = qb;
            xf[nq + 6 + bb - 1] = qdb;
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
        for (int j = 0; j < LEN; ++j) {
            xf[7 + b0 - 1 + j] = q[j];
            xf[nq + 6 + b0 - 1 + j] = qd[j];
        }
    }
    return R_C(0.);
}

// One warp pair's rollout of 16 samples: warp 2p + 0 the legs, 2p + 1 the waist and arms.
// rec = this pair's exchange area (SPLIT_PAIR_FLOATS floats of shared memory), bar its
// named barrier; every lane of both warps must call it the same number of times.
template <bool PAPER>
__device__ __forceinline__ R_T split_rollout(const DevModel<R_T>& M, int role, int lane, R_T* rec, int bar,
                                               const double* __restrict__ x0, const float* __restrict__ knots, int H,
                                               int nk, R_T dt, R_T dtk, double* __restrict__ xf) {
    const int i = lane >> 1, side = lane & 1;
    R_T* recA = rec + i * SPLIT_REC;
    R_T* recB = rec + (SPLIT_SPP + i) * SPLIT_REC;
    return role == 0 ? split_legs<PAPER>(M, side, recA, recB, bar, x0, knots, H, nk, dt, dtk, xf)
                     : split_arms<PAPER>(M, side, recA, recB, bar, x0, knots, H, nk, dt, dtk, xf);
}

R_NS_END

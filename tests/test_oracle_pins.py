"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test compares the oracle with something it does not compute: published known-answer
vectors, closed forms of mechanics, an independent numpy kinematics written here from
the model's data conventions, library routines (scipy), exact rational arithmetic, or
invariants of the method. CPU only.
"""
import math
import os

import numpy as np
import pytest
from scipy import special, stats

from paper_2511_19204_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------------------------
# Philox4x32-10 and the normal draws
# ------------------------------------------------------------------------------------
def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert list(orc.philox(ctr, key)) == out


def test_normals_are_standard_normal(orc):
    # 60k draws across elements, samples and iterations: KS against N(0, 1) and the
    # independence of the Box-Muller pair members.
    vals, pairs = [], []
    for n in range(1, 301):
        for e in range(0, 200, 2):
            a = orc.normal(7, 3, 0, n, e)
            b = orc.normal(7, 3, 0, n, e + 1)
            vals += [a, b]
            pairs.append((a, b))
    vals = np.array(vals)
    pairs = np.array(pairs)
    assert abs(vals.mean()) < 0.02
    assert abs(vals.std() - 1.0) < 0.02
    assert stats.kstest(vals, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(pairs[:, 0], pairs[:, 1])[0, 1]) < 0.02
    # different counters give different streams
    assert orc.normal(7, 3, 0, 1, 0) != orc.normal(7, 4, 0, 1, 0)
    assert orc.normal(7, 3, 0, 1, 0) != orc.normal(7, 3, 1, 1, 0)
    assert orc.normal(7, 3, 0, 1, 0) != orc.normal(8, 3, 0, 1, 0)


def test_box_muller_from_words(orc):
    # eps pair of element block 0 rebuilt from the published Box-Muller formulas and the
    # Philox words (u1 = ((w0 >> 8) + 1) 2^-24, u2 = (w1 >> 8) 2^-24).
    seed, it, inst, n = 0x1234_5678_9ABC, 5, 2, 9
    w = orc.philox([0, n, it, inst], [seed & 0xFFFFFFFF, seed >> 32])
    u1 = ((int(w[0]) >> 8) + 1) / 2.0**24
    u2 = (int(w[1]) >> 8) / 2.0**24
    r = math.sqrt(-2 * math.log(u1))
    assert orc.normal(seed, it, inst, n, 0) == pytest.approx(r * math.cos(2 * math.pi * u2), abs=1e-15)
    assert orc.normal(seed, it, inst, n, 1) == pytest.approx(r * math.sin(2 * math.pi * u2), abs=1e-15)
    u1 = ((int(w[2]) >> 8) + 1) / 2.0**24
    u2 = (int(w[3]) >> 8) / 2.0**24
    r = math.sqrt(-2 * math.log(u1))
    assert orc.normal(seed, it, inst, n, 2) == pytest.approx(r * math.cos(2 * math.pi * u2), abs=1e-15)
    assert orc.normal(seed, it, inst, n, 3) == pytest.approx(r * math.sin(2 * math.pi * u2), abs=1e-15)


def test_sample_knots_structure(orc):
    nu, nk, N, H, dt = 12, 6, 4000, 200, 0.005
    nom = np.random.default_rng(0).normal(size=(nk, 2, nu))
    sig = np.linspace(0.05, 0.3, nk)
    kn = orc.sample_knots(nu, nk, N, H, dt, nom, sig, scale_q=1.0, scale_v=0.0, seed=11)
    # sample 0 is the nominal (Alg. 1 samples n = 1..N-1)
    np.testing.assert_array_equal(kn[0], nom)
    d = kn[1:] - nom
    dtk = H * dt / (nk - 1)
    # per-knot std follows sigma_k * scale_p, scale_v default 1 / knot spacing
    std_q = d[:, :, 0, :].std(axis=(0, 2))
    std_v = d[:, :, 1, :].std(axis=(0, 2))
    np.testing.assert_allclose(std_q, sig, rtol=0.03)
    np.testing.assert_allclose(std_v, sig / dtk, rtol=0.03)
    # sigma = 0 reproduces the nominal everywhere
    kz = orc.sample_knots(nu, nk, 5, H, dt, nom, np.zeros(nk), seed=11)
    np.testing.assert_array_equal(kz, np.broadcast_to(nom, kz.shape))
    # explicit scales
    k2 = orc.sample_knots(nu, nk, 3, H, dt, nom, sig, scale_q=2.0, scale_v=0.5, seed=11)
    np.testing.assert_allclose((k2[1:, :, 0] - nom[:, 0]) / 2.0, d[:2, :, 0], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose((k2[1:, :, 1] - nom[:, 1]) / 0.5, d[:2, :, 1] * dtk, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------------------------
# Eq. (vel-clamp)
# ------------------------------------------------------------------------------------
def test_clamp_closed_form(orc):
    # one joint, limits [-1, 2], knot spacing 0.2 -> |v| <= min(2 - q, q + 1) / 0.1
    kn = np.array([[[0.5], [100.0]], [[1.9], [-5.0]], [[3.0], [1.0]], [[-0.5], [-2.0]]])
    out = orc.clamp(kn, 0.2, np.array([-1.0]), np.array([2.0]))
    np.testing.assert_allclose(out[:, 0, 0], [0.5, 1.9, 2.0, -0.5])
    np.testing.assert_allclose(out[:, 1, 0], [15.0, -1.0, 0.0, -2.0], atol=1e-12)
    # infinite limits: untouched
    out = orc.clamp(kn, 0.2, np.array([-np.inf]), np.array([np.inf]))
    np.testing.assert_array_equal(out, kn)
    # one-sided limit
    out = orc.clamp(kn, 0.2, np.array([-np.inf]), np.array([2.0]))
    np.testing.assert_allclose(out[:, 1, 0], [15.0, -1.0, 0.0, -2.0], atol=1e-12)


def test_clamp_feasible_set_is_convex(orc):
    # weighted means of clamped samples stay inside the clamp's feasible set, so the
    # nominal never needs re-clamping
    rng = np.random.default_rng(3)
    lo, hi = np.array([-0.5, -1.0, 0.0]), np.array([0.5, 2.0, 0.3])
    dtk = 0.2
    kn = np.stack([orc.clamp(rng.normal(scale=2.0, size=(5, 2, 3)), dtk, lo, hi) for _ in range(50)])
    w = rng.random(50)
    w /= w.sum()
    mean = np.tensordot(w, kn, axes=1)
    again = orc.clamp(mean, dtk, lo, hi)
    np.testing.assert_allclose(again, mean, atol=1e-12)
    # idempotent
    np.testing.assert_array_equal(orc.clamp(kn[0], dtk, lo, hi), kn[0])


# ------------------------------------------------------------------------------------
# Hermite spline (Eq. hermite_segment)
# ------------------------------------------------------------------------------------
def test_hermite_endpoints_and_partition(orc):
    rng = np.random.default_rng(1)
    for _ in range(20):
        q0, v0, q1, v1 = rng.normal(size=4)
        dtk = rng.uniform(0.05, 0.5)
        q, qd = orc.hermite(0.0, dtk, q0, v0, q1, v1)
        assert q == pytest.approx(q0, abs=1e-14) and qd == pytest.approx(v0, abs=1e-12)
        q, qd = orc.hermite(1.0, dtk, q0, v0, q1, v1)
        assert q == pytest.approx(q1, abs=1e-14) and qd == pytest.approx(v1, abs=1e-12)
        # h00 + h01 = 1: equal positions and zero slopes give a constant
        s = rng.random()
        q, qd = orc.hermite(s, dtk, 0.7, 0.0, 0.7, 0.0)
        assert q == pytest.approx(0.7, abs=1e-15) and qd == pytest.approx(0.0, abs=1e-13)


def test_hermite_reproduces_cubics(orc):
    # knots (p(t_j), p'(t_j)) of any cubic p reproduce p and p' at every step
    rng = np.random.default_rng(2)
    H, nk, dt = 200, 6, 0.005
    dtk = H * dt / (nk - 1)
    c = rng.normal(size=4)
    p = np.polynomial.Polynomial(c)
    dp = p.deriv()
    tk = np.arange(nk) * dtk
    for h in range(H):
        k, s = orc.segment(h, H, nk)
        t = h * dt
        assert 0 <= k <= nk - 2 and 0.0 <= s < 1.0
        assert s == pytest.approx((t - tk[k]) / dtk, abs=1e-12)
        q, qd = orc.hermite(s, dtk, p(tk[k]), dp(tk[k]), p(tk[k + 1]), dp(tk[k + 1]))
        assert q == pytest.approx(p(t), rel=1e-12, abs=1e-12)
        assert qd == pytest.approx(dp(t), rel=1e-11, abs=1e-11)


def test_segment_integer_exact(orc):
    for H, nk in [(50, 4), (200, 6), (200, 8), (7, 3), (1, 2), (199, 8)]:
        for h in range(H):
            k, s = orc.segment(h, H, nk)
            r = h * (nk - 1)
            assert k == min(r // H, nk - 2)
            assert s == (r - k * H) / H


# ------------------------------------------------------------------------------------
# Rigid-body dynamics
# ------------------------------------------------------------------------------------
def _rot(a, t):
    a = np.asarray(a, dtype=float)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(t) * K + (1 - math.cos(t)) * K @ K


def _quat_R(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _fk(m, R0, p0, q):
    """Independent forward kinematics from the model's data conventions."""
    R, P = [R0], [p0]
    for i in range(1, m.nb):
        l = m.parent[i]
        R.append(R[l] @ _rot(m.axis[i], q[i - 1]))
        P.append(P[l] + R[l] @ m.jpos[i])
    return R, P


def _kinetic_energy_matrix(m, x, eps=1e-6):
    """Mass matrix from T(u) = sum 1/2 m |v_com|^2 + 1/2 w^T Ic w (+ armature), with body
    velocities from central differences of the configuration along u. u = (base w,
    base v (body frame), qdot) for a floating base, qdot for a fixed one."""
    nj = m.nj
    R0 = _quat_R(x[3:7])
    p0 = x[0:3]
    q = x[7:7 + nj]
    off = 0 if m.fixed_base else 6
    n = off + nj

    def moved(u, e):
        if m.fixed_base:
            Rb, pb = R0, p0
        else:
            w, v = u[0:3], u[3:6]
            nw = np.linalg.norm(w)
            Rb = R0 @ (_rot(w / nw, e * nw) if nw > 0 else np.eye(3))
            pb = p0 + e * (R0 @ v)
        return _fk(m, Rb, pb, q + e * u[off:])

    def T(u):
        Rp, Pp = moved(u, eps)
        Rm, Pm = moved(u, -eps)
        t = 0.0
        for i in range(m.nb):
            cp = Pp[i] + Rp[i] @ m.com[i]
            cm = Pm[i] + Rm[i] @ m.com[i]
            vc = (cp - cm) / (2 * eps)
            Rd = (Rp[i] - Rm[i]) / (2 * eps)
            Ri = 0.5 * (Rp[i] + Rm[i])
            W = Ri.T @ Rd
            w = np.array([W[2, 1], W[0, 2], W[1, 0]])
            ic = m.inertia[i]
            Ic = np.array([[ic[0], ic[3], ic[4]], [ic[3], ic[1], ic[5]], [ic[4], ic[5], ic[2]]])
            t += 0.5 * m.mass[i] * vc @ vc + 0.5 * w @ Ic @ w
        t += 0.5 * np.sum(m.armature[1:] * u[off:] ** 2)
        return t

    M = np.zeros((n, n))
    E = np.eye(n)
    Tii = [T(E[i]) for i in range(n)]
    for i in range(n):
        M[i, i] = 2 * Tii[i]
        for j in range(i + 1, n):
            M[i, j] = M[j, i] = T(E[i] + E[j]) - Tii[i] - Tii[j]
    return M


ZOO = ["pendulum", "chain2", "free_body", "branch3", "quadruped", "humanoid"]


@pytest.mark.parametrize("name", ZOO)
def test_mass_matrix_against_kinetic_energy(orc, name):
    m = S.MODELS[name]()
    x = S.random_state(m, 17)
    M = orc.crba(m, x)
    Mk = _kinetic_energy_matrix(m, x)
    np.testing.assert_allclose(M, Mk, rtol=1e-6, atol=1e-8 * np.abs(Mk).max())


@pytest.mark.parametrize("name", ZOO)
def test_aba_against_crba_rnea(orc, name):
    # a = M^-1 (tau - h) by dense Cholesky (numpy) against the articulated-body recursion
    m = S.MODELS[name]()
    rng = np.random.default_rng(5)
    for seed in range(3):
        x = S.random_state(m, 100 + seed, height=0.05)   # low: contacts active
        tau = rng.normal(size=m.nj)
        acc = orc.forward_dynamics(m, x, tau)
        M = orc.crba(m, x)
        h = orc.rnea_bias(m, x)
        off = 0 if m.fixed_base else 6
        rhs = -h
        rhs[off:] += tau
        ref = np.linalg.solve(M, rhs)
        got = acc[6 - off:] if m.fixed_base else acc
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("theta,arm", [(0.3, 0.0), (-1.2, 0.0), (2.5, 0.05), (0.0, 0.1)])
def test_pendulum_closed_form(orc, theta, arm):
    m = S.pendulum(armature=arm)
    x = np.zeros(m.nx)
    x[3] = 1.0
    x[7] = theta
    x[m.nq + 6] = 0.7   # velocity does not enter a single hinge's acceleration
    acc = orc.forward_dynamics(m, x, np.zeros(1))
    ip = 0.02 + 1.3 * 0.4 ** 2 + arm
    assert acc[6] == pytest.approx(-1.3 * 9.81 * 0.4 * math.sin(theta) / ip, rel=1e-12, abs=1e-14)
    # with a torque
    acc = orc.forward_dynamics(m, x, np.array([0.9]))
    assert acc[6] == pytest.approx((0.9 - 1.3 * 9.81 * 0.4 * math.sin(theta)) / ip, rel=1e-12)


def test_free_fall_discrete_closed_form(orc):
    # semi-implicit Euler on a ballistic body: z_n = z0 + n dt v0 - g dt^2 n (n+1) / 2
    m = S.free_body()
    x = np.zeros(m.nx)
    q = np.array([0.9, 0.2, -0.3, 0.1])
    x[3:7] = q / np.linalg.norm(q)
    x[0:3] = [0.1, -0.2, 3.0]
    R = _quat_R(x[3:7])
    v0 = np.array([0.4, -0.3, 1.5])
    x[m.nq:m.nq + 3] = R.T @ v0
    dt = 0.01
    for n in range(1, 31):
        x = orc.step(m, x, np.zeros(0), dt)
        assert x[2] == pytest.approx(3.0 + n * dt * 1.5 - 9.81 * dt * dt * n * (n + 1) / 2, abs=1e-12)
        assert x[0] == pytest.approx(0.1 + n * dt * 0.4, abs=1e-12)
        np.testing.assert_allclose(x[3:7], q / np.linalg.norm(q), atol=1e-14)


def _momenta(m, x):
    R = _quat_R(x[3:7])
    v = x[m.nq:m.nq + 3]
    w = x[m.nq + 3:m.nq + 6]
    c = m.com[0]
    vcom_w = R @ (v + np.cross(w, c))
    ic = m.inertia[0]
    Ic = np.array([[ic[0], ic[3], ic[4]], [ic[3], ic[1], ic[5]], [ic[4], ic[5], ic[2]]])
    L = R @ (Ic @ w)
    return m.mass[0] * vcom_w, L


def test_free_body_conserves_momentum(orc):
    # torque-free asymmetric top without gravity: linear and angular momentum about the
    # centre of mass are constant; the integrator's error is first order in dt
    m = S.free_body().copy(gravity=0.0)
    x0 = np.zeros(m.nx)
    x0[3] = 1.0
    x0[m.nq:m.nq + 6] = [0.2, -0.1, 0.3, 1.5, -2.0, 0.7]
    P0, L0 = _momenta(m, x0)
    errs = []
    for dt in (2e-3, 1e-3):
        x = x0.copy()
        for _ in range(int(round(0.5 / dt))):
            x = orc.step(m, x, np.zeros(0), dt)
        P, L = _momenta(m, x)
        errs.append(max(np.linalg.norm(P - P0) / np.linalg.norm(P0), np.linalg.norm(L - L0) / np.linalg.norm(L0)))
    assert errs[1] < 5e-3
    assert 1.5 < errs[0] / errs[1] < 2.6


def _energy_np(m, x):
    """Kinetic + potential energy from the independent kinematics above."""
    u = np.concatenate([x[m.nq + 3:m.nq + 6], x[m.nq:m.nq + 3], x[m.nq + 6:]]) if not m.fixed_base \
        else x[m.nq + 6:]
    M = _kinetic_energy_matrix(m, x)
    R, P = _fk(m, _quat_R(x[3:7]), x[0:3], x[7:7 + m.nj])
    V = sum(m.mass[i] * m.gravity * (P[i] + R[i] @ m.com[i])[2] for i in range(m.nb))
    return 0.5 * u @ M @ u + V


@pytest.mark.parametrize("name", ["chain2", "branch3"])
def test_energy_error_first_order(orc, name):
    # contact, damping and PD off, gravity on: the energy error of the semi-implicit
    # Euler rollout is O(dt) (halving dt halves it) and small
    m = S.MODELS[name]()
    m = m.copy(kp=np.zeros(m.nj), kd=np.zeros(m.nj))
    x0 = S.random_state(m, 9, v_scale=1.0)
    E0 = _energy_np(m, x0)
    assert orc.energy(m, x0) == pytest.approx(E0, rel=1e-7)
    errs = []
    for dt in (1e-3, 5e-4):
        kn = np.zeros((2, 2, m.nj))
        H = int(round(0.4 / dt))
        _, xf, tr = orc.rollout(m, x0, kn, H, dt, traj=True)
        e = [abs(orc.energy(m, tr[h]) - E0) for h in range(0, H + 1, max(1, H // 20))]
        errs.append(max(e))
        assert abs(_energy_np(m, xf) - orc.energy(m, xf)) < 1e-6 * max(1.0, abs(E0))
    assert errs[1] < 1e-2 * max(1.0, abs(E0))
    assert 1.5 < errs[0] / errs[1] < 2.6


def test_contact_damped_oscillator(orc):
    # point mass resting on the spring-damper ground: m z'' = -k z - c z' - m g while in
    # contact; from 0.1 mm below equilibrium at rest the motion is the closed-form
    # underdamped oscillator, which the rollout approaches at first order in dt
    m = S.point_mass(m=1.0).copy(mu=0.0)
    k, c, g = m.contact_k, m.contact_c, m.gravity
    z_eq = -g / k
    d = -1e-4
    wn = math.sqrt(k)
    zeta = c / (2 * math.sqrt(k))
    wd = wn * math.sqrt(1 - zeta ** 2)

    def exact(t):
        return z_eq + math.exp(-zeta * wn * t) * (d * math.cos(wd * t) + d * zeta * wn / wd * math.sin(wd * t))

    errs = []
    for dt in (1e-5, 5e-6):
        x = np.zeros(m.nx)
        x[3] = 1.0
        x[2] = z_eq + d
        err = 0.0
        for n in range(1, int(round(0.02 / dt)) + 1):
            x = orc.step(m, x, np.zeros(0), dt)
            err = max(err, abs(x[2] - exact(n * dt)))
        errs.append(err / abs(d))
    assert errs[1] < 2e-2
    assert 1.6 < errs[0] / errs[1] < 2.4


@pytest.mark.parametrize("v", [0.05, 0.4, 3.0])
def test_smooth_coulomb_friction(orc, v):
    # in static penetration f_n = m g, so the sliding deceleration is
    # mu g v / sqrt(v^2 + eps^2) along -v
    m = S.point_mass(m=2.0, mu=0.8, eps_f=0.1)
    x = np.zeros(m.nx)
    x[3] = 1.0
    x[2] = -2.0 * m.gravity / m.contact_k
    x[m.nq:m.nq + 3] = [v * 0.6, v * 0.8, 0.0]
    acc = orc.forward_dynamics(m, x, np.zeros(0))
    mag = 0.8 * m.gravity * v / math.sqrt(v * v + 0.01)
    np.testing.assert_allclose(acc[3:6], [-0.6 * mag, -0.8 * mag, 0.0], atol=1e-9)
    f = orc.contact_forces(m, x)
    assert f[0, 2] == pytest.approx(2.0 * m.gravity, rel=1e-12)


def test_standing_contact_load(orc):
    # the standing pose penetrates m g / (4 k) per foot: the four normal forces carry the
    # weight exactly and the base starts in equilibrium vertically
    m = S.quadruped()
    x = S.standing_state(m)
    f = orc.contact_forces(m, x)
    np.testing.assert_allclose(f[:, 2], m.mass.sum() * m.gravity / 4, rtol=1e-9)
    np.testing.assert_allclose(f[:, :2], 0.0, atol=1e-12)
    _, cpos = orc.positions(m, x)
    np.testing.assert_allclose(cpos[:, 2], -m.mass.sum() * m.gravity / (4 * m.contact_k), atol=1e-12)


# ------------------------------------------------------------------------------------
# PD tracking and running cost through a rollout
# ------------------------------------------------------------------------------------
def test_pd_first_step_on_pendulum(orc):
    m = S.pendulum().copy(kp=np.array([30.0]), kd=np.array([2.0]), tau_max=np.array([5.0]))
    x = np.zeros(m.nx)
    x[3] = 1.0
    x[7] = 0.2
    x[m.nq + 6] = -0.5
    H, dt, nk = 10, 0.01, 2
    kn = np.array([[[0.5], [1.0]], [[0.9], [-0.3]]])
    dtk = H * dt
    # spline setpoint at t = 0 is the first knot (q 0.5, v 1.0)
    tau = min(5.0, max(-5.0, 30.0 * (0.5 - 0.2) + 2.0 * (1.0 + 0.5)))
    ip = 0.02 + 1.3 * 0.16
    a = (tau - 1.3 * 9.81 * 0.4 * math.sin(0.2)) / ip
    _, xf = orc.rollout(m, x, kn, 1, dt)
    assert xf[m.nq + 6] == pytest.approx(-0.5 + dt * a, rel=1e-12)
    assert xf[7] == pytest.approx(0.2 + dt * (-0.5 + dt * a), rel=1e-12)
    # saturated: a larger gain clips at tau_max
    m2 = m.copy(kp=np.array([300.0]))
    _, xf = orc.rollout(m2, x, kn, 1, dt)
    a2 = (5.0 - 1.3 * 9.81 * 0.4 * math.sin(0.2)) / ip
    assert xf[m.nq + 6] == pytest.approx(-0.5 + dt * a2, rel=1e-12)
    del dtk, nk


def test_running_cost_on_ballistic_body(orc):
    # a free body in free fall at a fixed tilt: the cost sum is the closed form over the
    # ballistic trajectory evaluated at the pre-step states
    m = S.free_body().copy(z_des=0.7, vx_des=0.2, w_z=2.0, w_vx=3.0, w_tilt=5.0, w_tau=0.0)
    x = np.zeros(m.nx)
    ang = 0.4
    x[3:7] = [math.cos(ang / 2), math.sin(ang / 2), 0.0, 0.0]   # tilt 0.4 rad about x
    x[2] = 2.0
    R = _quat_R(x[3:7])
    v0 = np.array([0.5, 0.0, 1.0])
    x[m.nq:m.nq + 3] = R.T @ v0
    H, dt = 25, 0.01
    kn = np.zeros((2, 2, 0))
    S_or, _ = orc.rollout(m, x, kn, H, dt)
    Sx = 0.0
    for h in range(H):
        z = 2.0 + h * dt * 1.0 - 9.81 * dt * dt * h * (h + 1) / 2
        vz = 1.0 - 9.81 * dt * h
        del vz
        Sx += 2.0 * (z - 0.7) ** 2 + 3.0 * (0.5 - 0.2) ** 2 + 5.0 * ang ** 2
    assert S_or == pytest.approx(Sx, rel=1e-12)


def _effort_only(m, w_tau):
    """The model with every cost term off except the effort term w_tau |tau|^2."""
    return m.copy(w_z=0.0, w_vx=0.0, w_tilt=0.0, w_tau=w_tau, w_h=0.0, w_orient=0.0, w_q=0.0,
                  w_cvel=0.0, w_cforce=0.0, w_term=0.0)


@pytest.mark.parametrize("target", [10.0, -10.0])
def test_effort_cost_saturated_torque(orc, target):
    # Sec. IV-A cost sum with only the effort term, Eq. (pd-controller) clipped to the
    # actuator limit: a setpoint 10 rad away saturates the PD torque at +-tau_max on every
    # step (the pendulum stays within 1 rad over 40 steps), so the sum is H w_tau tau_max^2.
    # An unclipped torque would give ~(Kp 10)^2 per step, a dropped weight tau_max^2.
    m = _effort_only(S.pendulum().copy(kp=np.array([30.0]), kd=np.array([2.0]), tau_max=np.array([0.5])), 0.37)
    x = np.zeros(m.nx)
    x[3] = 1.0
    x[7] = 0.1
    H, dt = 40, 0.01
    kn = np.array([[[target], [0.0]], [[target], [0.0]]])
    S_or, xf = orc.rollout(m, x, kn, H, dt)
    # |q| < 1 and |v| < 10 keep |Kp (q_ref - q) + Kd (v_ref - v)| >= 30 * 9 - 2 * 10 >> tau_max
    assert abs(xf[7]) < 1.0 and abs(xf[m.nq + 6]) < 10.0
    assert S_or == pytest.approx(H * 0.37 * 0.5 ** 2, rel=1e-12)


def test_effort_cost_charges_the_pre_step_torque(orc):
    # Two steps, unsaturated: c(x_h, u_h) is charged at the pre-step states x_0 and x_1.
    # The setpoint spline reproduces the line q(t) = 0.3 + 0.8 t exactly (knot values and
    # slopes of a line), so q_ref(t_h) and v_ref(t_h) are known without the Hermite basis;
    # x_1 is the pendulum's closed-form first step (semi-implicit Euler, Eq. for theta'' =
    # (tau - m g l_c sin theta) / I_pivot). A torque charged after the step, or a missing
    # square, changes the sum.
    kp, kd, wt = 30.0, 2.0, 0.37
    m = _effort_only(S.pendulum().copy(kp=np.array([kp]), kd=np.array([kd]), tau_max=np.array([50.0])), wt)
    x = np.zeros(m.nx)
    x[3] = 1.0
    q0, v0 = 0.2, -0.5
    x[7] = q0
    x[m.nq + 6] = v0
    H, dt = 2, 0.01
    T = H * dt
    a_line, b_line = 0.3, 0.8
    kn = np.array([[[a_line], [b_line]], [[a_line + b_line * T], [b_line]]])
    tau0 = kp * (a_line - q0) + kd * (b_line - v0)
    ip = 0.02 + 1.3 * 0.16
    acc = (tau0 - 1.3 * 9.81 * 0.4 * math.sin(q0)) / ip
    v1 = v0 + dt * acc
    q1 = q0 + dt * v1
    tau1 = kp * (a_line + b_line * dt - q1) + kd * (b_line - v1)
    assert max(abs(tau0), abs(tau1)) < 50.0
    S_or, _ = orc.rollout(m, x, kn, H, dt)
    assert S_or == pytest.approx(wt * (tau0 ** 2 + tau1 ** 2), rel=1e-12)
    # one step charges tau_0 alone
    S1, _ = orc.rollout(m, x, np.array([[[a_line], [b_line]], [[a_line + b_line * dt], [b_line]]]), 1, dt)
    assert S1 == pytest.approx(wt * tau0 ** 2, rel=1e-12)


def test_effort_cost_sums_joints_of_clipped_torques(orc):
    # One step on a 2-joint chain: the effort is w_tau sum_j clip(tau_j)^2 with the first
    # joint saturated and the second not (its setpoint is the current state plus a small
    # offset); the dynamics do not enter a one-step sum.
    kp = np.array([200.0, 3.0])
    kd = np.array([1.0, 0.5])
    tmax = np.array([0.8, 10.0])
    m = _effort_only(S.chain2().copy(kp=kp, kd=kd, tau_max=tmax), 1.9)
    x = np.zeros(m.nx)
    x[3] = 1.0
    q = np.array([0.1, -0.4])
    v = np.array([0.3, 0.2])
    x[7:9] = q
    x[m.nq + 6:m.nq + 8] = v
    qr = np.array([0.5, -0.35])
    vr = np.array([0.0, 0.25])
    kn = np.array([[qr, vr], [qr + vr * 0.01, vr]])
    S_or, _ = orc.rollout(m, x, kn, 1, 0.01)
    tau = np.clip(kp * (qr - q) + kd * (vr - v), -tmax, tmax)
    assert abs(tau[0]) == 0.8 and abs(tau[1]) < 10.0
    assert S_or == pytest.approx(1.9 * float(np.sum(tau ** 2)), rel=1e-12)


# ------------------------------------------------------------------------------------
# Weights (Eqs. omega-weights, softmax_minmax) and the average (Eq. update-nominal)
# ------------------------------------------------------------------------------------
def test_weights_match_library_softmax(orc):
    rng = np.random.default_rng(4)
    Sc = rng.uniform(10, 50, size=257)
    lam = 0.1
    st, w, info = orc.weights(Sc, lam, normalize=0)
    assert st == 0
    sh = (Sc - Sc.min()) / (Sc.max() - Sc.min())
    np.testing.assert_allclose(w, special.softmax(-sh / lam), rtol=1e-12)
    st, w, info = orc.weights(Sc, 3.0, normalize=1)
    np.testing.assert_allclose(w, special.softmax(-Sc / 3.0), rtol=1e-12)
    assert info["best"] == int(np.argmin(Sc))
    assert info["ess"] == pytest.approx(1.0 / np.sum(w ** 2), rel=1e-12)


def test_weights_invariants(orc):
    rng = np.random.default_rng(6)
    Sc = rng.uniform(0, 100, size=100)
    st, w, info = orc.weights(Sc, 0.2)
    assert w.sum() == pytest.approx(1.0, abs=1e-14)
    # min-max normalisation: invariant under S -> a S + b, a > 0
    _, w2, _ = orc.weights(3.7 * Sc + 1234.5, 0.2)
    np.testing.assert_allclose(w2, w, rtol=1e-12)
    # permutation invariance
    perm = rng.permutation(100)
    _, w3, _ = orc.weights(Sc[perm], 0.2)
    np.testing.assert_allclose(w3, w[perm], rtol=1e-13)
    # lambda -> 0: one-hot on the argmin; lambda -> inf: uniform
    _, w0, _ = orc.weights(Sc, 1e-6)
    np.testing.assert_allclose(w0, np.eye(100)[np.argmin(Sc)], atol=1e-12)
    _, wi, _ = orc.weights(Sc, 1e9)
    np.testing.assert_allclose(wi, np.full(100, 0.01), rtol=1e-7)
    # equal costs: uniform (S_max = S_min gives S_hat = 0)
    _, we, info = orc.weights(np.full(10, 4.2), 0.1)
    np.testing.assert_allclose(we, 0.1, rtol=1e-14)
    assert info["best"] == 0
    # N = 1
    _, w1, _ = orc.weights(np.array([5.0]), 0.1)
    assert w1[0] == 1.0
    # ties: lowest index
    _, _, info = orc.weights(np.array([3.0, 1.0, 2.0, 1.0]), 0.1)
    assert info["best"] == 1


def test_weights_non_finite(orc):
    Sc = np.array([np.nan, 2.0, np.inf, 1.0, 3.0])
    st, w, info = orc.weights(Sc, 0.1)
    assert st == 0
    assert w[0] == 0 and w[2] == 0
    ref = special.softmax(-(np.array([2.0, 1.0, 3.0]) - 1.0) / 2.0 / 0.1)
    np.testing.assert_allclose(w[[1, 3, 4]], ref, rtol=1e-12)
    assert info["n_finite"] == 3 and info["best"] == 3
    st, w, info = orc.weights(np.array([np.nan, np.inf]), 0.1)
    assert st == -3 and np.all(w == 0)


def test_average_exact_rational(orc):
    kn = np.array([[[[1.0, -2.0]], [[4.0, 8.0]]]]).reshape(1, 2, 1, 2)
    kn = np.concatenate([kn, 3 * kn + 1], axis=0)   # two samples
    out = orc.average(kn, np.array([0.25, 0.75]))
    np.testing.assert_array_equal(out, 0.25 * kn[0] + 0.75 * kn[1])   # exact in binary
    out = orc.average(kn, np.array([0.0, 1.0]))
    np.testing.assert_array_equal(out, kn[1])


def test_resampling_equals_knot_average(orc):
    # averaging trajectories and resampling at the knots equals averaging the knots:
    # the spline and its derivative are linear in the knots (Eq. update-nominal)
    rng = np.random.default_rng(8)
    H, nk, dt, N = 60, 4, 0.01, 7
    dtk = H * dt / (nk - 1)
    kn = rng.normal(size=(N, nk, 2, 1))
    w = rng.random(N)
    w /= w.sum()
    mean = orc.average(kn, w)
    for h in range(H):
        k, s = orc.segment(h, H, nk)
        traj = np.array([orc.hermite(s, dtk, kn[n, k, 0, 0], kn[n, k, 1, 0], kn[n, k + 1, 0, 0], kn[n, k + 1, 1, 0])
                         for n in range(N)])
        got = orc.hermite(s, dtk, mean[k, 0, 0], mean[k, 1, 0], mean[k + 1, 0, 0], mean[k + 1, 1, 0])
        np.testing.assert_allclose(got, w @ traj, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------------------------
# Alg. 1 as a whole
# ------------------------------------------------------------------------------------
def test_solve_fixed_points(orc):
    p = S.plain_quadruped(n=16)
    p.horizon = 20
    # sigma = 0: every sample is the nominal, the update returns it
    r = orc.solve(p.model, p.n, p.nk, p.horizon, 2, p.dt, p.lam, np.zeros((2, p.nk)), p.state, p.nominal)
    np.testing.assert_allclose(r["mean"], p.nominal, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["best"], p.nominal, rtol=0, atol=1e-12)
    # N = 1: only the nominal is simulated
    r = orc.solve(p.model, 1, p.nk, p.horizon, 1, p.dt, p.lam, p.sigma, p.state, p.nominal)
    np.testing.assert_array_equal(r["mean"], p.nominal)
    assert r["best_index"] == 0


def test_solve_best_tracking_and_update(orc):
    p = S.plain_quadruped(n=24)
    p.horizon = 30
    r = orc.solve(p.model, p.n, p.nk, p.horizon, 3, p.dt, p.lam, S.linear_sigma(p.nk, 3), p.state,
                  p.nominal, keep=True)
    costs = r["costs"]
    assert r["best_cost"] == pytest.approx(np.nanmin(costs))
    it, n = np.unravel_index(np.nanargmin(costs), costs.shape)
    np.testing.assert_array_equal(r["best"], r["knots"][it, n])
    # iteration i+1 samples around the weighted mean of iteration i
    st, w, _ = orc.weights(costs[0], p.lam)
    mean0 = orc.average(r["knots"][0], w)
    np.testing.assert_allclose(r["knots"][1, 0], mean0, rtol=1e-13, atol=1e-15)
    st, w, _ = orc.weights(costs[2], p.lam)
    np.testing.assert_allclose(r["mean"], orc.average(r["knots"][2], w), rtol=1e-13, atol=1e-15)
    # each sample's cost is its own rollout
    S1, _ = orc.rollout(p.model, p.state, r["knots"][1, 5], p.horizon, p.dt)
    assert S1 == pytest.approx(costs[1, 5], rel=1e-14)


def test_config_rollouts_finite(orc):
    # the chosen armature and friction regularisation keep every sampled rollout of the
    # plain quadruped configuration bounded (semi-implicit Euler at dt = 0.01)
    p = S.plain_quadruped()
    r = orc.solve_problem(p, keep=True)
    assert r["status"] == 0
    assert np.all(np.isfinite(r["costs"])) and np.all(r["costs"] < 1e4)


# ------------------------------------------------------------------------------------
# Eq. (overall-noise-kernel)
# ------------------------------------------------------------------------------------
def test_noise_schedule_structure(orc):
    I, K, b1, b2 = 3, 6, 0.7, 1.3
    s = orc.noise_schedule(I, K, b1, b2)
    # the first iteration (i = I) carries factor 1 on the trajectory term; the last knot
    # (k = K - 1) the largest action factor exp(-1 / (beta2 K))
    assert s[0, K - 1] == pytest.approx(math.exp(-1.0 / (b2 * K)), rel=1e-15)
    # multiplicative separability: constant ratios along knots and along iterations
    np.testing.assert_allclose(s[:, 1:] / s[:, :-1], math.exp(1.0 / (b2 * K)), rtol=1e-13)
    np.testing.assert_allclose(s[1:, :] / s[:-1, :], math.exp(-1.0 / (b1 * I)), rtol=1e-13)
    # larger variance for later knots and earlier iterations
    assert np.all(np.diff(s, axis=1) > 0) and np.all(np.diff(s, axis=0) < 0)
    # the scale multiplies every entry
    np.testing.assert_allclose(orc.noise_schedule(I, K, b1, b2, 0.3), 0.3 * s, rtol=1e-15)


def test_library_noise_schedule_matches_oracle(orc):
    # host-side helper of the library (no GPU needed)
    from paper_2511_19204_gb300 import build, mppi
    build.build()
    for I, K, b1, b2, sc in ((3, 6, 0.7, 1.3, 0.3), (1, 4, 2.0, 0.5, 1.0), (5, 8, 0.25, 4.0, 0.05)):
        got = mppi.noise_schedule(I, K, b1, b2, sc)
        np.testing.assert_allclose(got, orc.noise_schedule(I, K, b1, b2, sc), rtol=2e-7)
    with pytest.raises(mppi.MppiError):
        mppi.noise_schedule(0, 4, 1.0, 1.0)


# ------------------------------------------------------------------------------------
# Sec. III-E: state prediction and shift of tau_best
# ------------------------------------------------------------------------------------
def test_shift_identity_and_cubic(orc):
    rng = np.random.default_rng(21)
    H, nk, dt = 200, 6, 0.005
    T = H * dt
    dtk = T / (nk - 1)
    kn = rng.normal(size=(nk, 2, 3))
    np.testing.assert_array_equal(orc.shift_knots(kn, H, 0, dt), kn)       # no delay: unchanged
    # knots sampled from cubics: the shifted knots are the cubics at t_j + delay, and past
    # the horizon end the end point (value and slope at T) is held
    polys = [np.polynomial.Polynomial(rng.normal(size=4)) for _ in range(3)]
    for i, p in enumerate(polys):
        for j in range(nk):
            kn[j, 0, i] = p(j * dtk)
            kn[j, 1, i] = p.deriv()(j * dtk)
    for steps in (1, 7, 40, 199, 260):
        sh = orc.shift_knots(kn, H, steps, dt)
        for i, p in enumerate(polys):
            for j in range(nk):
                t = min(j * dtk + steps * dt, T)
                assert sh[j, 0, i] == pytest.approx(p(t), rel=1e-11, abs=1e-11)
                assert sh[j, 1, i] == pytest.approx(p.deriv()(t), rel=1e-10, abs=1e-10)


def test_prediction_is_the_rollout_prefix(orc):
    p = S.scale_quadruped(n=4)
    kn = orc.sample_knots(p.model.nj, p.nk, 4, p.horizon, p.dt, p.nominal, p.sigma[0], seed=3)[2]
    _, _, tr = orc.rollout(p.model, p.state, kn, p.horizon, p.dt, traj=True)
    for d in (0, 1, 4, 10, p.horizon):
        np.testing.assert_array_equal(orc.predict_state(p.model, p.state, kn, p.horizon, d, p.dt), tr[d])


# ------------------------------------------------------------------------------------
# Modular cost of Sec. IV-A (Eq. running cost, Eq. terminal cost)
# ------------------------------------------------------------------------------------
_NO_QUAD = dict(w_z=0.0, w_vx=0.0, w_tilt=0.0, w_tau=0.0)


def _axis_quat(axis, ang):
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    return np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * a])


def test_modular_cost_drifting_body(orc):
    # a free body without gravity drifts at constant velocity (zero acceleration, exact
    # under semi-implicit Euler): p_h = p0 + h dt v. Height term, terminal term and the
    # orientation term (fixed attitude alpha about an axis, R_des = identity) in closed form.
    alpha = 0.35
    m = S.free_body().copy(gravity=0.0, w_h=3.0, w_orient=2.0, w_term=7.0, z_des=0.4,
                           pdot_des=(0.2, -0.1, 0.05), **_NO_QUAD)
    x = np.zeros(m.nx)
    x[3:7] = _axis_quat((1.0, 2.0, -0.5), alpha)
    x[0:3] = [0.1, 0.2, 1.0]
    v = np.array([0.6, 0.3, -0.4])
    x[m.nq:m.nq + 3] = _quat_R(x[3:7]).T @ v
    H, dt = 40, 0.01
    S_or, xf = orc.rollout(m, x, np.zeros((2, 2, 0)), H, dt)
    Sx = sum(3.0 * abs(1.0 + h * dt * v[2] - 0.4) + 2.0 * alpha ** 2 for h in range(H))
    Sx += 7.0 * np.sum(np.abs(H * dt * (v - np.array([0.2, -0.1, 0.05]))))
    assert S_or == pytest.approx(Sx, rel=1e-12)
    np.testing.assert_allclose(xf[0:3], x[0:3] + H * dt * v, atol=1e-13)


def test_modular_cost_orientation_is_the_geodesic_angle(orc):
    # ||log3(R^T R_des)|| against scipy's rotation magnitude for random attitude pairs
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(8)
    H, dt = 1, 0.01
    for _ in range(20):
        qb = rng.normal(size=4)
        qd = rng.normal(size=4)
        qb /= np.linalg.norm(qb)
        qd /= np.linalg.norm(qd)
        m = S.free_body().copy(gravity=0.0, w_orient=1.0, quat_des=tuple(qd), **_NO_QUAD)
        x = np.zeros(m.nx)
        x[3:7] = qb
        S_or, _ = orc.rollout(m, x, np.zeros((2, 2, 0)), H, dt)
        rb = Rotation.from_quat([qb[1], qb[2], qb[3], qb[0]])
        rd = Rotation.from_quat([qd[1], qd[2], qd[3], qd[0]])
        th = (rb.inv() * rd).magnitude()
        assert S_or == pytest.approx(th * th, rel=1e-10, abs=1e-14)


def test_modular_cost_joint_term(orc):
    # a torque-free pendulum without gravity spins at constant rate: q_h = q(0) + h dt w
    m = S.pendulum().copy(gravity=0.0, w_q=1.5, q_stand=np.array([0.3]), **_NO_QUAD)
    x = np.zeros(m.nx)
    x[7] = -0.2
    x[m.nq + 6] = 2.0
    H, dt = 30, 0.01
    kn = np.zeros((2, 2, 1))
    S_or, _ = orc.rollout(m, x, kn, H, dt)
    Sx = sum(1.5 * (-0.2 + h * dt * 2.0 - 0.3) ** 2 for h in range(H))
    assert S_or == pytest.approx(Sx, rel=1e-12)


def test_modular_cost_contact_terms(orc):
    # a point mass resting at its equilibrium depth m g / k carries f_c = (0, 0, m g); with
    # no friction it slides at constant speed vx with contact velocity (vx, 0, 0)
    m0 = S.point_mass(mu=0.0)
    g, mass, k = m0.gravity, float(m0.mass[0]), m0.contact_k
    H, dt = 25, 0.005
    vx = 0.7
    x = np.zeros(m0.nx)
    x[3] = 1.0
    x[2] = -mass * g / k
    x[m0.nq] = vx
    kn = np.zeros((2, 2, 0))
    m = m0.copy(w_cforce=0.5, f0=(0.0, 0.0, 0.0), **_NO_QUAD)
    assert orc.rollout(m, x, kn, H, dt)[0] == pytest.approx(H * 0.5 * mass * g, rel=1e-9)
    m = m0.copy(w_cforce=0.5, f0=(0.1, -0.2, mass * g), **_NO_QUAD)
    assert orc.rollout(m, x, kn, H, dt)[0] == pytest.approx(H * 0.5 * 0.3, rel=1e-9)
    m = m0.copy(w_cvel=2.0, **_NO_QUAD)
    assert orc.rollout(m, x, kn, H, dt)[0] == pytest.approx(H * 2.0 * vx, rel=1e-9)
    # off the ground (no gravity, at rest above the plane): no contact velocity term, and
    # the force term is ||f0||_1 per step
    y = x.copy()
    y[2] = 0.5
    m = m0.copy(gravity=0.0, w_cvel=2.0, w_cforce=0.5, f0=(0.1, -0.2, 3.0), **_NO_QUAD)
    assert orc.rollout(m, y, kn, H, dt)[0] == pytest.approx(H * 0.5 * 3.3, rel=1e-12)


def test_terminal_cost_ballistic(orc):
    # terminal term on the discrete ballistic closed form z_H = z0 + H dt v0 - g dt^2 H (H + 1) / 2
    m = S.free_body().copy(w_term=4.0, pdot_des=(0.3, 0.0, 0.0), **_NO_QUAD)
    x = np.zeros(m.nx)
    x[3] = 1.0
    x[0:3] = [0.0, 0.1, 2.0]
    v0 = np.array([0.5, 0.0, 1.2])
    x[m.nq:m.nq + 3] = v0
    H, dt = 30, 0.01
    S_or, _ = orc.rollout(m, x, np.zeros((2, 2, 0)), H, dt)
    zH = 2.0 + H * dt * 1.2 - 9.81 * dt * dt * H * (H + 1) / 2
    Sx = 4.0 * (abs(H * dt * 0.5 - 0.3 * H * dt) + abs(zH - 2.0))
    assert S_or == pytest.approx(Sx, rel=1e-12)


def test_tab2_weights_and_standing_load():
    # the weight sets and the derived per-point standing load
    p = S.paper_walking(n=4)
    m = p.model
    assert (m.w_h, m.w_orient, m.w_q, m.w_cvel, m.w_cforce, m.w_term) == (1e2, 10.0, 0.0, 0.5, 5e-2, 2.5e3)
    assert m.w_z == m.w_vx == m.w_tilt == m.w_tau == 0.0
    assert m.f0[2] * m.nc == pytest.approx(float(np.sum(m.mass)) * m.gravity)
    assert m.pdot_des == (0.5, 0.0, 0.0)


# ------------------------------------------------------------------------------------
# Spline variants of the ablation (Sec. IV-D): setpoints and node slopes
# ------------------------------------------------------------------------------------
def _variant_knots(rng, nk, nu):
    kn = np.zeros((nk, 2, nu))
    kn[:, 0] = rng.normal(size=(nk, nu))
    kn[:, 1] = rng.normal(size=(nk, nu))     # ignored by the position-only variants
    return kn


@pytest.mark.parametrize("nk", [2, 3, 6, 16])
def test_natural_cubic_variant_against_scipy(orc, nk):
    from scipy.interpolate import CubicSpline
    rng = np.random.default_rng(nk)
    H, dt, nu = 200, 0.005, 3
    kn = _variant_knots(rng, nk, nu)
    tk = np.arange(nk) * H * dt / (nk - 1)
    q, v = orc.setpoints(kn, H, dt, orc.SPLINE_CUBIC)
    sl = orc.spline_slopes(kn, H, dt, orc.SPLINE_CUBIC)
    th = np.arange(H) * dt
    for j in range(nu):
        cs = CubicSpline(tk, kn[:, 0, j], bc_type="natural")
        np.testing.assert_allclose(q[:, j], cs(th), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(v[:, j], cs(th, 1), rtol=1e-11, atol=1e-11)
        np.testing.assert_allclose(sl[:, 1, j], cs(tk, 1), rtol=1e-11, atol=1e-11)
    np.testing.assert_array_equal(sl[:, 0], kn[:, 0])


def test_hermite_setpoints_against_scipy(orc):
    from scipy.interpolate import CubicHermiteSpline
    rng = np.random.default_rng(3)
    H, dt, nk, nu = 200, 0.005, 6, 2
    kn = _variant_knots(rng, nk, nu)
    tk = np.arange(nk) * H * dt / (nk - 1)
    q, v = orc.setpoints(kn, H, dt, orc.SPLINE_HERMITE)
    th = np.arange(H) * dt
    for j in range(nu):
        hs = CubicHermiteSpline(tk, kn[:, 0, j], kn[:, 1, j])
        np.testing.assert_allclose(q[:, j], hs(th), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(v[:, j], hs(th, 1), rtol=1e-11, atol=1e-11)


def test_quadratic_variant(orc):
    rng = np.random.default_rng(5)
    H, dt, nk, nu = 200, 0.005, 6, 2
    T = H * dt
    tk = np.arange(nk) * T / (nk - 1)
    th = np.arange(H) * dt
    # reproduces a quadratic that starts at rest: q(t) = a + c t^2
    a, c = rng.normal(size=nu), rng.normal(size=nu)
    kn = np.zeros((nk, 2, nu))
    kn[:, 0] = a + np.outer(tk ** 2, c)
    q, v = orc.setpoints(kn, H, dt, orc.SPLINE_QUADRATIC)
    np.testing.assert_allclose(q, a + np.outer(th ** 2, c), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(v, np.outer(2 * th, c), rtol=1e-11, atol=1e-11)
    # on random nodes: interpolates, is C1 at the nodes, piecewise quadratic, starts at rest
    kn = _variant_knots(rng, nk, nu)
    q, v = orc.setpoints(kn, H, dt, orc.SPLINE_QUADRATIC)
    step = H // (nk - 1)
    np.testing.assert_allclose(q[::step][:nk - 1], kn[:nk - 1, 0], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(v[0], 0.0, atol=1e-12)
    sl = orc.spline_slopes(kn, H, dt, orc.SPLINE_QUADRATIC)
    for k in range(nk - 1):
        seg = slice(k * step, (k + 1) * step)
        for j in range(nu):
            # the exact quadratic through the segment's end values with its start slope
            t0, h = tk[k], T / (nk - 1)
            s = (th[seg] - t0) / h
            a2 = kn[k + 1, 0, j] - kn[k, 0, j] - sl[k, 1, j] * h
            np.testing.assert_allclose(q[seg, j], kn[k, 0, j] + sl[k, 1, j] * h * s + a2 * s ** 2, rtol=1e-12,
                                       atol=1e-12)
            # C1: the segment's end slope is the next node's slope
            assert sl[k, 1, j] + 2 * a2 / h == pytest.approx(sl[k + 1, 1, j], rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("spline", [1, 2])
def test_variant_equals_hermite_with_its_node_slopes(orc, spline):
    # each segment of either variant is a polynomial of degree <= 3 with the variant's end
    # values and slopes, so the Hermite interpolant of those nodes is the same curve
    rng = np.random.default_rng(10 + spline)
    H, dt, nk, nu = 200, 0.005, 6, 3
    kn = _variant_knots(rng, nk, nu)
    qv, vv = orc.setpoints(kn, H, dt, spline)
    qh, vh = orc.setpoints(orc.spline_slopes(kn, H, dt, spline), H, dt, orc.SPLINE_HERMITE)
    np.testing.assert_allclose(qh, qv, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(vh, vv, rtol=1e-11, atol=1e-11)


def test_variant_solve_ignores_sampled_velocities(orc):
    # under a position-only variant the sampled velocity knots do not matter: the rollout
    # costs equal those of the same knots with zeroed velocity knots
    p = S.scale_quadruped(n=16)
    p.horizon = 60
    kn = orc.sample_knots(p.model.nj, p.nk, p.n, p.horizon, p.dt, p.nominal, p.sigma[0], seed=4)
    kz = kn.copy()
    kz[:, :, 1, :] = 0.0
    for spline in (1, 2):
        a = orc.rollout_batch(p.model, p.state, kn, p.horizon, p.dt, spline=spline)
        b = orc.rollout_batch(p.model, p.state, kz, p.horizon, p.dt, spline=spline)
        np.testing.assert_array_equal(a, b)
    r = orc.solve(p.model, p.n, p.nk, p.horizon, 1, p.dt, p.lam, p.sigma[:1], p.state, p.nominal, seed=2,
                  spline=2, keep=True)
    for n in range(p.n):
        np.testing.assert_allclose(r["knots"][0, n], orc.spline_slopes(r["knots"][0, n], p.horizon, p.dt, 2),
                                   rtol=0, atol=0)

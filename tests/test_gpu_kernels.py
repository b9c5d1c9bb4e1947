"""Kernel-level parity of the CUDA path with the FP64 oracle, through the C ABI.

Tolerances (FP32 product unless stated):
  Philox words                       bit-exact
  knot noise                         |d| <= 4 ulp(FP32)|sigma s eps| + 2 ulp(theta) + 1e-6
  single-step state derivative       1e-5 relative (to the largest component)
  50-step contact-free rollouts      1e-4 relative (costs, final states)
  FP64 check build                   1e-9 relative
  weights / average (FP64 on both)   1e-12 relative
"""
import numpy as np
import pytest

from paper_2511_19204_gb300 import flops as F
from paper_2511_19204_gb300 import synth as S

pytestmark = pytest.mark.gpu

F32_ULP = 2.0 ** -23


@pytest.fixture(scope="module")
def M():
    from paper_2511_19204_gb300 import build, mppi
    build.build()
    mppi.load()
    return mppi


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ------------------------------------------------------------------------------------
# Philox / noise
# ------------------------------------------------------------------------------------
def test_philox_words_bit_exact(M, orc):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    ctr[2] = [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]
    for key in ([0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [0xA4093822, 0x299F31D0], [12345, 678]):
        got = M.philox_words(ctr, key)
        ref = np.array([orc.philox(ctr[i], key) for i in range(ctr.shape[0])], dtype=np.uint32)
        np.testing.assert_array_equal(got, ref)     # every word of all 4096 counters


@pytest.mark.parametrize("name,nk,n", [("quadruped", 4, 37), ("quadruped", 6, 300), ("humanoid", 7, 50),
                                       ("humanoid", 8, 129)])
def test_sample_knots_match_oracle(M, orc, name, nk, n):
    m = S.MODELS[name]()
    H, dt = 200, 0.005
    sig = S.linear_sigma(nk, 2)
    sig[1] *= 0.5
    nom = S.random_knots(m, 1, nk, seed=3, scale=0.2)[0]
    mod = M.Model(m)
    c = M.Controller(mod, n, H, nk, 0.1, sig, iters=2, dt=dt, seed=0xABCDEF0123, instance=7,
                     mapping=M.MPPI_MAP_WARP)
    nom32 = nom.astype(np.float32)
    for it, ctrv in ((0, 5), (1, 77)):
        got = c.sample_knots(it, ctrv, nom32)
        ref = orc.sample_knots(m.nj, nk, n, H, dt, nom32.astype(np.float64), sig[it], seed=0xABCDEF0123,
                               iter_ctr=ctrv, inst=7)
        np.testing.assert_array_equal(got[0], nom32)            # sample 0 is the nominal
        dtk = H * dt / (nk - 1)
        scale = np.array([1.0, 1.0 / dtk])[None, None, :, None]
        dev = np.abs(ref - nom32.astype(np.float64)) + 0 * scale
        tol = 4 * F32_ULP * dev + 2 * F32_ULP * np.abs(ref) + 1e-6
        assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) - tol)


@pytest.mark.parametrize("robot", ["quadruped", "humanoid"])
def test_sample_knots_clamp(M, orc, robot):
    # the clamp of Eq. (vel-clamp) on a joint count divisible by 4 (the quadruped's 12: the
    # barrier-free noise kernel) and on one that is not (the humanoid's 21: the kernel that
    # stages the normals in shared memory)
    if robot == "quadruped":
        lo, hi = np.array([-0.3, 0.2, -2.0]), np.array([0.3, 1.5, -0.8])
        m = S.quadruped(limits=(lo, hi))
    else:
        h = S.humanoid()
        q0 = h.q_stand
        m = h.copy(q_min=q0 - 0.25 - 0.1 * np.arange(h.nj) / h.nj, q_max=q0 + 0.3)
    nk, n, H, dt = 5, 200, 100, 0.01
    sig = S.linear_sigma(nk, 1) * 4
    nom = S.nominal_knots(m, nk)
    c = M.Controller(M.Model(m), n, H, nk, 0.1, sig, iters=1, dt=dt, seed=9, mapping=M.MPPI_MAP_WARP)
    got = c.sample_knots(0, 3, nom.astype(np.float32)).astype(np.float64)
    ref = orc.sample_knots(m.nj, nk, n, H, dt, nom, sig[0], seed=9, iter_ctr=3, q_min=m.q_min, q_max=m.q_max)
    assert np.max(np.abs(got - ref)) < 2e-5
    q, v = got[:, :, 0, :], got[:, :, 1, :]
    assert np.all(q >= m.q_min - 1e-6) and np.all(q <= m.q_max + 1e-6)
    dtk = H * dt / (nk - 1)
    room = np.minimum(m.q_max - q, q - m.q_min)
    assert np.all(np.abs(v) <= 2 * room / dtk + 1e-5)


# ------------------------------------------------------------------------------------
# Dynamics
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["quadruped", "humanoid", "chain2", "branch3", "free_body", "pendulum",
                                  "point_mass"])
def test_forward_dynamics(M, orc, name):
    m = S.MODELS[name]()
    rng = np.random.default_rng(11)
    xs = np.stack([S.random_state(m, 50 + i, height=0.3 if i % 2 else 0.05) for i in range(24)])
    tau = rng.normal(scale=5.0, size=(24, m.nj))
    mod = M.Model(m)
    ref = np.stack([orc.forward_dynamics(m, xs[i], tau[i]) for i in range(24)])
    got32 = mod.forward_dynamics(xs, tau)
    got64 = mod.forward_dynamics(xs, tau, fp64=True)
    for i in range(24):
        assert _rel(got64[i], ref[i]) < 1e-9, (i, _rel(got64[i], ref[i]))
        assert _rel(got32[i], ref[i]) < 1e-5, (i, _rel(got32[i], ref[i]))


def _lifted(m, seed):
    x = S.standing_state(m, jitter=0.05, seed=seed)
    x[2] = 3.0 + 0.1 * (seed % 3)
    rng = np.random.default_rng(seed)
    x[m.nq:m.nq + 6] = rng.normal(scale=0.3, size=6)
    return x


@pytest.mark.parametrize("name,mapping", [("quadruped", 0), ("quadruped", 1), ("quadruped", 2), ("humanoid", 0),
                                          ("humanoid", 2)])
def test_rollout_contact_free(M, orc, name, mapping):
    # 50 steps in the air: no contact ever acts, so FP32 stays within 1e-4 of FP64
    m = S.MODELS[name]()
    nk, H, dt, n = 4, 50, 0.01, 40
    kn = S.random_knots(m, n, nk, seed=4, scale=0.2).astype(np.float32)
    x0 = _lifted(m, 1)
    c = M.Controller(M.Model(m), n, H, nk, 0.1, S.linear_sigma(nk), dt=dt, mapping=mapping)
    costs, fins = c.rollout_explicit(x0, kn, finals=True)
    ref_c, ref_f = orc.rollout_batch(m, x0, kn.astype(np.float64), H, dt, finals=True)
    _, cpos = orc.positions(m, ref_f[0])
    assert cpos[:, 2].min() > 0.0
    assert _rel(costs, ref_c) < 1e-4
    for i in range(n):
        assert _rel(fins[i], ref_f[i]) < 1e-4, i
    # the FP64 check build of the same mapping (for the chain mapping: the product's
    # specialised lanes / split kernels in double)
    c.set_fp64_check(True)
    costs64, fins64 = c.rollout_explicit(x0, kn, finals=True)
    assert _rel(costs64, ref_c) < 1e-9
    for i in range(n):
        assert _rel(fins64[i], ref_f[i]) < 1e-9, i


@pytest.mark.parametrize("cfg", ["scale", "humanoid", "plain"])
@pytest.mark.parametrize("mapping64", [0, 2])
def test_rollout_with_contact_fp64_check(M, orc, cfg, mapping64):
    # contact rollouts of the configurations: the FP64 check build within 1e-9 where the
    # dynamics are well conditioned (dt = 0.005), and within the oracle's own FP64
    # sensitivity envelope at dt = 0.01; the FP32 product's cost error is reported and
    # bounded by 1e-3 (median) or the FP32 envelope
    from _parity import rollout_envelope
    if cfg == "scale":
        p = S.scale_quadruped(n=64)
    elif cfg == "humanoid":
        p = S.humanoid_problem(n=32)
        p.horizon = 100
    else:
        p = S.plain_quadruped()
    m = p.model
    kn = orc.sample_knots(m.nj, p.nk, p.n, p.horizon, p.dt, p.nominal, p.sigma[0], seed=p.seed)
    kn32 = kn.astype(np.float32)
    kn64 = kn32.astype(np.float64)
    (ref_c, ref_f), env_c64, env_f64 = rollout_envelope(m, p.state, kn64, p.horizon, p.dt, 1e-15)
    # mapping64 0: the generic warp kernel in double; 2: the product's lanes-per-chain
    # kernel in double (the x, y, y quadruped plan; the humanoid's two-warp split)
    c = M.Controller.from_problem(M.Model(m), p, mapping=mapping64)
    c.set_fp64_check(True)
    c64, f64 = c.rollout_explicit(p.state, kn32, finals=True)
    scale_f = np.max(np.abs(ref_f), axis=1)
    err_f = np.max(np.abs(f64 - ref_f), axis=1) / scale_f
    err_c = np.abs(c64 - ref_c) / np.abs(ref_c)
    print(f"{cfg} mapping {mapping64}: FP64 check build rel. error costs max {err_c.max():.2e}, final states max {err_f.max():.2e}; "
          f"oracle FP64 envelope max {np.max(env_f64 / scale_f):.2e}")
    if cfg == "plain":
        assert np.all(np.abs(f64 - ref_f).max(axis=1) <= np.maximum(1e-9 * scale_f, 10 * env_f64))
        assert np.median(err_f) < 1e-9
    else:
        assert err_c.max() < 1e-9 and err_f.max() < 1e-9
    if mapping64 != 0:
        return
    c.set_fp64_check(False)
    c.set_mapping(M.MPPI_MAP_CHAIN)
    c32 = c.rollout_explicit(p.state, kn32)
    err = np.abs(c32 - ref_c) / np.abs(ref_c)
    print(f"{cfg}: FP32 contact-rollout cost rel. error median {np.median(err):.2e} max {err.max():.2e}")
    assert np.median(err) < 1e-3
    if cfg != "plain":
        assert err.max() < 1e-3
    else:
        # chaotic: FP32 rounding of every step is amplified ~1e5-fold, so most samples
        # agree closely and a tail does not; bound the bulk and the tail separately
        _, env_c32, _ = rollout_envelope(m, p.state, kn64, p.horizon, p.dt, 1e-6, draws=8)
        env = env_c32 / np.abs(ref_c)
        print(f"plain: oracle FP32-level envelope median {np.median(env):.2e} max {env.max():.2e}")
        assert np.median(err) <= 10 * np.median(env) + 1e-6
        assert err.max() <= 10 * env.max() + 1e-6


@pytest.mark.parametrize("robot,n,block", [("quadruped", 1, 0), ("quadruped", 37, 32), ("quadruped", 300, 64),
                                           ("quadruped", 1000, 128), ("quadruped", 2049, 256), ("humanoid", 1, 0),
                                           ("humanoid", 77, 64), ("humanoid", 513, 256)])
def test_mappings_agree(M, orc, robot, n, block):
    # every rollout mapping runs the same algorithm: on the well-conditioned dt = 0.005
    # workloads they agree with each other and with the oracle to FP32 accuracy
    p = S.scale_quadruped(n=n) if robot == "quadruped" else S.humanoid_problem(n=n)
    p.horizon = 120 if robot == "quadruped" else 60
    kn = orc.sample_knots(p.model.nj, p.nk, n, p.horizon, p.dt, p.nominal, p.sigma[0], seed=p.seed).astype(np.float32)
    c = M.Controller.from_problem(M.Model(p.model), p, mapping=0)
    maps = (0, 1, 2) if robot == "quadruped" else (0, 2)
    out = {}
    for mapping in maps:
        c.set_mapping(mapping, block if (block or mapping != 1) else 0)
        out[mapping], fin = c.rollout_explicit(p.state, kn, finals=True)
        assert np.all(np.isfinite(fin))
    idx = np.arange(n) if n <= 64 else np.r_[0:16, n - 16:n]
    ref = orc.rollout_batch(p.model, p.state, kn.astype(np.float64)[idx], p.horizon, p.dt)
    for mapping in maps:
        err = np.abs(out[mapping][idx] - ref) / np.abs(ref)
        assert err.max() < 1e-4, (mapping, err.max())
        assert np.max(np.abs(out[mapping] - out[0]) / np.abs(out[0])) < 1e-4


@pytest.mark.parametrize("tilt", [0.0, 0.05, -1.0, None])
def test_chain_axis_plans(M, orc, tilt):
    # the quadruped's x, y, y joint axes (contacts on the calves) select the axis-specialised
    # chain kernel; a tilted or reversed hip axis, or a contact point on a thigh (None), the
    # generic one; both agree with the oracle
    p = S.scale_quadruped(n=256)
    p.horizon = 120
    m = p.model
    if tilt is None:
        m = m.copy(contact_body=np.append(m.contact_body, 2).astype(np.int32),
                   contact_pos=np.vstack([m.contact_pos, [0.0, 0.0, -0.1]]))
        p.model = m
    elif tilt:
        axis = m.axis.copy()
        for b in range(1, m.nb, 3):
            a = np.array([1.0, 0.0, tilt]) if tilt > 0 else np.array([-1.0, 0.0, 0.0])
            axis[b] = a / np.linalg.norm(a)
        m = m.copy(axis=axis)
        p.model = m
    mod = M.Model(m)
    assert mod.info()["topology"] == 1
    assert mod.info()["axis_plan"] == (1 if tilt == 0.0 else 0)
    assert F.axis_plan_xyy(m) == (tilt == 0.0)
    kn = orc.sample_knots(m.nj, p.nk, p.n, p.horizon, p.dt, p.nominal, p.sigma[0], seed=p.seed).astype(np.float32)
    c = M.Controller.from_problem(mod, p, mapping=M.MPPI_MAP_CHAIN)
    got, fin = c.rollout_explicit(p.state, kn, finals=True)
    ref_c, ref_f = orc.rollout_batch(m, p.state, kn.astype(np.float64), p.horizon, p.dt, finals=True)
    err = np.abs(got - ref_c) / np.abs(ref_c)
    err_f = np.max(np.abs(fin - ref_f), axis=1) / np.max(np.abs(ref_f), axis=1)
    print(f"axis plan {mod.info()['axis_plan']}: cost rel. error median {np.median(err):.2e} max {err.max():.2e}, "
          f"final state max {err_f.max():.2e}")
    assert err.max() < 1e-4 and err_f.max() < 1e-4
    # the same plan's kernel in double: 1e-9
    c.set_fp64_check(True)
    g64, f64 = c.rollout_explicit(p.state, kn, finals=True)
    assert np.max(np.abs(g64 - ref_c) / np.abs(ref_c)) < 1e-9
    assert np.max(np.max(np.abs(f64 - ref_f), axis=1) / np.max(np.abs(ref_f), axis=1)) < 1e-9


@pytest.mark.parametrize("variant", ["layout", "tilted", "offset", "hand_contact", "leg_cost"])
def test_humanoid_axis_plans(M, orc, variant):
    # the humanoid's joint layout (legs z, x, y, y, y, x; waist z; arms y, x, z, y) selects
    # the two-warp split kernel (axis plan 2); a tilted hip axis or an elbow offset off its
    # axis selects the one-warp generic chain kernel. Both agree with the oracle, and the
    # split kernel gives the same bits at every block size and rejects 32-thread blocks.
    p = S.humanoid_problem(n=200)
    p.horizon = 60
    m = p.model
    if variant == "tilted":
        axis = m.axis.copy()
        axis[1] = np.array([0.05, 0.0, 1.0]) / np.linalg.norm([0.05, 0.0, 1.0])
        m = m.copy(axis=axis)
    elif variant == "offset":
        jpos = m.jpos.copy()
        jpos[m.nb - 1, 0] = 0.01
        m = m.copy(jpos=jpos)
    elif variant == "hand_contact":   # a contact point off the feet
        m = m.copy(contact_body=np.append(m.contact_body, m.nb - 1).astype(np.int32),
                   contact_pos=np.vstack([m.contact_pos, [0.0, 0.0, -0.2]]))
    elif variant == "leg_cost":       # the cost body on a leg
        m = m.copy(cost_body=4)
    p.model = m
    mod = M.Model(m)
    assert mod.info()["topology"] == 2
    assert mod.info()["axis_plan"] == (2 if variant == "layout" else 0)
    assert F.axis_plan_hum(m) == (variant == "layout")
    kn = orc.sample_knots(m.nj, p.nk, p.n, p.horizon, p.dt, p.nominal, p.sigma[0], seed=p.seed).astype(np.float32)
    c = M.Controller.from_problem(mod, p, mapping=M.MPPI_MAP_CHAIN)
    got, fin = c.rollout_explicit(p.state, kn, finals=True)
    ref_c, ref_f = orc.rollout_batch(m, p.state, kn.astype(np.float64), p.horizon, p.dt, finals=True)
    err = np.abs(got - ref_c) / np.abs(ref_c)
    err_f = np.max(np.abs(fin - ref_f), axis=1) / np.max(np.abs(ref_f), axis=1)
    print(f"humanoid {variant}, axis plan {mod.info()['axis_plan']}: cost rel. error median {np.median(err):.2e} "
          f"max {err.max():.2e}, final state max {err_f.max():.2e}")
    assert err.max() < 1e-4 and err_f.max() < 1e-4
    # the same plan's kernel in double (split or generic branch chain): 1e-9
    c.set_fp64_check(True)
    g64, f64 = c.rollout_explicit(p.state, kn, finals=True)
    assert np.max(np.abs(g64 - ref_c) / np.abs(ref_c)) < 1e-9
    assert np.max(np.max(np.abs(f64 - ref_f), axis=1) / np.max(np.abs(ref_f), axis=1)) < 1e-9
    c.set_fp64_check(False)
    if variant == "layout":
        for block in (64, 256):
            c.set_mapping(M.MPPI_MAP_CHAIN, block)
            g2, f2 = c.rollout_explicit(p.state, kn, finals=True)
            np.testing.assert_array_equal(g2, got)
            np.testing.assert_array_equal(f2, fin)
        with pytest.raises(M.MppiError):
            c.set_mapping(M.MPPI_MAP_CHAIN, 32)


# ------------------------------------------------------------------------------------
# Weights and average
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("n,norm", [(1, 0), (7, 0), (256, 0), (1000, 1), (8192, 0), (8193, 0)])
def test_weights_match_oracle(M, orc, n, norm):
    rng = np.random.default_rng(n)
    c = rng.uniform(100, 900, size=n).astype(np.float32)
    if n > 10:
        c[3] = np.nan
        c[5] = np.inf
        c[n // 2] = c.min()        # a tie: lowest index wins
    st, w, info = M.weights(c, 0.1 if norm == 0 else 50.0, norm)
    st_o, w_o, info_o = orc.weights(c.astype(np.float64), 0.1 if norm == 0 else 50.0, norm)
    assert st == st_o == 0
    np.testing.assert_allclose(w, w_o, rtol=1e-12, atol=1e-300)
    assert info["best_index"] == info_o["best"]
    assert info["n_finite"] == info_o["n_finite"]
    assert info["ess"] == pytest.approx(info_o["ess"], rel=1e-12)
    assert info["lse"] == pytest.approx(info_o["lse"], rel=1e-12, abs=1e-14)


def test_weights_all_non_finite(M):
    st, w, info = M.weights(np.array([np.nan, np.inf, -np.inf], np.float32), 0.1)
    assert st == -3 and np.all(w == 0) and info["best_index"] == -1


@pytest.mark.parametrize("n,E", [(1, 48), (64, 48), (65, 144), (1000, 336), (8192, 144)])
def test_average_matches_oracle(M, orc, n, E):
    rng = np.random.default_rng(E + n)
    kn = rng.normal(size=(n, E)).astype(np.float32)
    w = rng.random(n)
    w /= w.sum()
    got = M.average(kn, w)
    ref = orc.average(kn.astype(np.float64), w)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14)
    # exact on a rational case
    kn2 = np.array([[1.0, -2.0, 4.0], [3.0, 0.5, 8.0]], np.float32)
    np.testing.assert_array_equal(M.average(kn2, np.array([0.25, 0.75])), 0.25 * kn2[0] + 0.75 * kn2[1])


def test_rollout_elementary_functions(M):
    # the rollout's own sine/cosine and tilt arctangent against numpy's FP64 values of the
    # same FP32 arguments
    rng = np.random.default_rng(12)
    x = np.concatenate([np.linspace(-4 * np.pi, 4 * np.pi, 100001), rng.uniform(-100, 100, 100000),
                        [0.0, -0.0, np.pi / 4, np.pi / 2, np.pi, 1e-30, -1e-8]]).astype(np.float32)
    y = np.abs(rng.normal(size=x.shape)).astype(np.float32)
    y[::7] *= np.float32(1e-4)
    y[-7:] = [0.0, 0.0, 1.0, 0.0, 1e-20, 2.0, 0.0]
    out = M.selftest_math(x, y).astype(np.float64)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    err_sc = np.maximum(np.abs(out[:, 0] - np.sin(xd)), np.abs(out[:, 1] - np.cos(xd)))
    err_at = np.abs(out[:, 2] - np.arctan2(yd, xd))
    print(f"fast_sincos: max abs error {err_sc.max():.2e} over |x| <= 100; "
          f"fast_atan2_pos: max abs error {err_at.max():.2e}")
    assert err_sc.max() < 2.5e-7
    assert err_at.max() < 5e-7


def test_widening_is_the_exact_conversion(M):
    # The knot average converts FP32 knots to FP64 by integer operations only; every float
    # must come out as (double)x bit for bit: normals, signed zeros, subnormals, extremes,
    # infinities, and any bit pattern (NaNs compared as NaN).
    rng = np.random.default_rng(5)
    x = np.concatenate([
        rng.normal(size=4096).astype(np.float32),
        (rng.random(4096) * 1.2e-38).astype(np.float32),          # subnormals and the smallest normals
        np.array([0.0, -0.0, np.inf, -np.inf, 1e-45, -1e-45, 3.4028235e38, -3.4028235e38,
                  1.17549435e-38, 1.1754942e-38], dtype=np.float32),
        rng.integers(0, 2**32, size=65536, dtype=np.uint64).astype(np.uint32).view(np.float32)])
    got = M.selftest_widen(x)
    ref = x.astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    np.testing.assert_array_equal(got[~nan].view(np.uint64), ref[~nan].view(np.uint64))

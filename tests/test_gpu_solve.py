"""Whole-solve parity (Alg. 1) of the CUDA path with the FP64 oracle, and the solve API's
behaviour, through the C ABI.

Updated control points are compared at 1e-3 (relative to max(1, |x|)) on the contact
configurations: contact rollouts are chaotic, so FP32 rollouts differ from FP64 ones by
~1e-5..1e-3 in cost and the weights move accordingly.
"""
import os

import numpy as np
import pytest

from paper_2511_19204_gb300 import synth as S

pytestmark = pytest.mark.gpu
KNOT_TOL = 1e-3


@pytest.fixture(scope="module")
def M():
    from paper_2511_19204_gb300 import build, mppi
    build.build()
    mppi.load()
    return mppi


def _close(a, b, tol=KNOT_TOL):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    err = np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b)))
    return err, err <= tol


@pytest.mark.parametrize("mapping", [0, 1, 2])
def test_plain_quadruped_solve_matches_oracle(M, orc, mapping):
    # dt = 0.01 contact rollouts amplify FP32 rounding ~1e5-fold (see tests/_parity.py):
    # the updated control points must lie within 1e-3 or within 5x the oracle's own
    # spread under 1e-6 relative perturbations of the initial state (8 draws)
    from _parity import solve_envelope
    p = S.plain_quadruped()
    c = M.Controller.from_problem(M.Model(p.model), p, mapping=mapping)
    mean, best, info = c.solve(p.state, warm=p.nominal.astype(np.float32))
    ref, env = solve_envelope(p.model, p.n, p.nk, p.horizon, p.iters, p.dt, p.lam, p.sigma, p.state,
                              p.nominal.astype(np.float32).astype(np.float64), p.seed, 1e-6, draws=8)
    assert info["status"] == 0 and info["n_finite"] == p.n
    err, ok = _close(mean, ref["mean"])
    env_rel = np.max(env / np.maximum(1.0, np.abs(ref["mean"])))
    print(f"plain mapping {mapping}: mean knot error {err:.2e} (oracle FP32-level envelope {env_rel:.2e}), "
          f"best cost {info['best_cost']:.6f} vs {ref['best_cost']:.6f}")
    assert err <= max(KNOT_TOL, 5 * env_rel)
    assert abs(info["best_cost"] - ref["best_cost"]) <= max(1e-4 * ref["best_cost"], 5 * ref["best_cost_envelope"])
    assert info["cost_min"] == pytest.approx(ref["smin"], rel=1e-3)
    if info["best_index"] == ref["best_index"]:
        err, ok = _close(best, ref["best"], 1e-6)
        assert ok


def test_ragged_sizes_and_three_iterations(M, orc):
    # N not a multiple of any tile, nk = 5, 3 iterations with a decaying schedule
    m = S.quadruped()
    n, nk, H, it, dt = 77, 5, 60, 3, 0.005
    sig = S.linear_sigma(nk, it) * np.array([[1.0], [0.6], [0.3]])
    x0 = S.standing_state(m, jitter=0.02, base_vel=0.3, seed=5)
    nom = S.nominal_knots(m, nk)
    for mapping in (0, 1, 2):
        c = M.Controller(M.Model(m), n, H, nk, 0.2, sig, iters=it, dt=dt, seed=21, instance=3, mapping=mapping)
        mean, best, info = c.solve(x0, warm=nom.astype(np.float32))
        ref = orc.solve(m, n, nk, H, it, dt, 0.2, sig, x0, nom, seed=21, inst=3)
        err, ok = _close(mean, ref["mean"])
        assert ok, err
        assert info["best_cost"] == pytest.approx(ref["best_cost"], rel=1e-3)
        assert c.iter_counter == it


@pytest.mark.parametrize("mapping", [0, 2])
def test_humanoid_solve_matches_oracle(M, orc, mapping):
    p = S.humanoid_problem(n=256)
    p.horizon = 100
    c = M.Controller.from_problem(M.Model(p.model), p, mapping=mapping)
    mean, best, info = c.solve(p.state, warm=p.nominal.astype(np.float32))
    ref = orc.solve(p.model, p.n, p.nk, p.horizon, p.iters, p.dt, p.lam, p.sigma, p.state,
                    p.nominal.astype(np.float32).astype(np.float64), seed=p.seed)
    err, ok = _close(mean, ref["mean"])
    print(f"humanoid: mean knot error {err:.2e}")
    assert ok
    assert info["best_cost"] == pytest.approx(ref["best_cost"], rel=1e-3)


def test_scale_config_full_size_sampled(M, orc):
    # the benchmark's workload: N = 8192, H = 200, 3 iterations, in the bench's launch
    # configuration. Checked: every knot of iteration 0, 64 sampled rollouts, and the
    # full solve's updated control points.
    p = S.scale_quadruped(n=8192)
    mapping = int(os.environ.get("MPPI_BENCH_MAPPING", M.MPPI_MAP_AUTO))
    c = M.Controller.from_problem(M.Model(p.model), p, mapping=mapping)
    nom32 = p.nominal.astype(np.float32)
    kn = c.sample_knots(0, 0, nom32)
    ref_kn = orc.sample_knots(p.model.nj, p.nk, p.n, p.horizon, p.dt, nom32.astype(np.float64), p.sigma[0],
                              seed=p.seed, iter_ctr=0)
    assert np.max(np.abs(kn - ref_kn) / np.maximum(1.0, np.abs(ref_kn))) < 1e-5
    costs = c.rollout_explicit(p.state, ref_kn.astype(np.float32))
    idx = np.random.default_rng(0).choice(p.n, 64, replace=False)
    idx[0] = 0
    idx[1] = p.n - 1
    ref_c = orc.rollout_batch(p.model, p.state, ref_kn.astype(np.float32).astype(np.float64)[idx], p.horizon, p.dt)
    err = np.abs(costs[idx] - ref_c) / np.abs(ref_c)
    print(f"scale: sampled FP32 cost error median {np.median(err):.2e} max {err.max():.2e}")
    assert np.median(err) < 1e-3
    assert np.all(np.isfinite(costs))
    mean, best, info = c.solve(p.state, warm=nom32)
    ref = orc.solve(p.model, p.n, p.nk, p.horizon, p.iters, p.dt, p.lam, p.sigma, p.state,
                    nom32.astype(np.float64), seed=p.seed)
    err, ok = _close(mean, ref["mean"])
    print(f"scale: mean knot error {err:.2e}; best cost {info['best_cost']:.4f} vs {ref['best_cost']:.4f}")
    assert ok
    assert info["best_cost"] == pytest.approx(ref["best_cost"], rel=1e-3)


def test_humanoid_config_full_size_sampled(M, orc):
    # the humanoid workload at full size (K = 2048, H = 200) in the benchmark's launch
    # configuration (two-warp split kernel, 256-thread blocks): 32 sampled rollouts and the
    # full solve's updated control points against the oracle
    p = S.humanoid_problem()
    c = M.Controller.from_problem(M.Model(p.model), p, mapping=M.MPPI_MAP_CHAIN, block=256)
    assert c.info()["block"] == 256 and M.Model(p.model).info()["axis_plan"] == 2
    nom32 = p.nominal.astype(np.float32)
    kn = orc.sample_knots(p.model.nj, p.nk, p.n, p.horizon, p.dt, nom32.astype(np.float64), p.sigma[0],
                          seed=p.seed).astype(np.float32)
    costs = c.rollout_explicit(p.state, kn)
    idx = np.random.default_rng(1).choice(p.n, 32, replace=False)
    idx[0], idx[1] = 0, p.n - 1
    ref_c = orc.rollout_batch(p.model, p.state, kn.astype(np.float64)[idx], p.horizon, p.dt)
    err = np.abs(costs[idx] - ref_c) / np.abs(ref_c)
    print(f"humanoid: sampled FP32 cost error median {np.median(err):.2e} max {err.max():.2e}")
    assert err.max() < 1e-3 and np.all(np.isfinite(costs))
    mean, best, info = c.solve(p.state, warm=nom32)
    ref = orc.solve(p.model, p.n, p.nk, p.horizon, p.iters, p.dt, p.lam, p.sigma, p.state,
                    nom32.astype(np.float64), seed=p.seed)
    err, ok = _close(mean, ref["mean"])
    print(f"humanoid full size: mean knot error {err:.2e}; best cost {info['best_cost']:.4f} vs {ref['best_cost']:.4f}")
    assert ok
    assert info["best_cost"] == pytest.approx(ref["best_cost"], rel=1e-3)


# ------------------------------------------------------------------------------------
# API behaviour
# ------------------------------------------------------------------------------------
def test_counter_resident_warm_start_and_replay(M):
    p = S.plain_quadruped()
    c = M.Controller.from_problem(M.Model(p.model), p, mapping=0)
    blob = c.export_state()
    m1, b1, i1 = c.solve(p.state)
    assert c.iter_counter == 1
    m2, b2, i2 = c.solve(p.state)                 # resident warm start = best of solve 1
    assert c.iter_counter == 2
    assert not np.array_equal(m1, m2)
    c.import_state(blob)                          # replay from the exported state
    m1r, b1r, i1r = c.solve(p.state)
    np.testing.assert_array_equal(m1r, m1)
    np.testing.assert_array_equal(b1r, b1)
    m2r, _, _ = c.solve(p.state, warm=b1)         # explicit warm start = the resident one
    np.testing.assert_array_equal(m2r, m2)


@pytest.mark.parametrize("problem", ["scale", "humanoid"])
def test_programmatic_launches_change_no_bit(M, problem):
    # In a plain solve every lanes-per-chain rollout, weights kernel and later noise kernel
    # starts as a programmatic dependent of the kernel before it and waits for it before
    # reading its output; with profiling on, events sit between the kernels and every
    # kernel waits for the previous one to finish. Both must give the same bits (3
    # iterations, so the noise kernels of iterations 2 and 3 are dependents too).
    p = S.scale_quadruped(n=2048) if problem == "scale" else S.humanoid_problem(n=512)
    p.iters = 3
    p.sigma = S.linear_sigma(p.nk, 3)
    c = M.Controller.from_problem(M.Model(p.model), p, mapping=M.MPPI_MAP_CHAIN)
    warm = p.nominal.astype(np.float32)
    out = []
    for prof in (False, True, False):
        c.profile(prof)
        c.iter_counter = 0
        out.append(c.solve(p.state, warm=warm))
    for m, b, info in out[1:]:
        np.testing.assert_array_equal(m, out[0][0])
        np.testing.assert_array_equal(b, out[0][1])
        assert info["best_cost"] == out[0][2]["best_cost"]


def test_warm_from_mean(M):
    p = S.plain_quadruped()
    c = M.Controller.from_problem(M.Model(p.model), p, mapping=0, warm_from=M.MPPI_WARM_MEAN)
    m1, _, _ = c.solve(p.state)
    c.iter_counter = 0
    m_ref, _, _ = c.solve(p.state, warm=p.nominal.astype(np.float32))
    np.testing.assert_array_equal(m1, m_ref)
    blob = c.export_state()
    nominal = np.frombuffer(blob[20:], dtype=np.float32)
    np.testing.assert_array_equal(nominal, m_ref.reshape(-1))


def test_solve_device_matches_host(M):
    torch = pytest.importorskip("torch")
    p = S.plain_quadruped()
    c = M.Controller.from_problem(M.Model(p.model), p, mapping=0)
    mean_h, best_h, info_h = c.solve(p.state)
    c2 = M.Controller.from_problem(M.Model(p.model), p, mapping=0)
    x = torch.tensor(p.state, dtype=torch.float64, device="cuda")
    out = torch.zeros(c2.E, dtype=torch.float32, device="cuda")
    best = torch.zeros(c2.E, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    c2.solve_device(x.data_ptr(), out.data_ptr(), best.data_ptr())
    c2.sync()
    np.testing.assert_array_equal(out.cpu().numpy().reshape(mean_h.shape), mean_h)
    np.testing.assert_array_equal(best.cpu().numpy().reshape(best_h.shape), best_h)


def test_io_bytes_are_the_copies_of_a_host_solve(M):
    import ctypes as C
    p = S.scale_quadruped(n=64)
    c = M.Controller.from_problem(M.Model(p.model), p)
    h2d, d2h = c.io_bytes()
    assert h2d == 8 * p.model.nx
    assert d2h == 4 * 2 * c.E + C.sizeof(M.mppi_result)


def test_nonfinite_state_rejected(M):
    p = S.plain_quadruped()
    c = M.Controller.from_problem(M.Model(p.model), p, mapping=0)
    x = p.state.copy()
    x[5] = np.nan
    _, _, info = c.solve(x, check=False)
    assert info["return_status"] == M.MPPI_ERR_NONFINITE_STATE
    assert c.iter_counter == 0


def test_all_costs_non_finite_keeps_nominal(M):
    p = S.plain_quadruped()
    m = p.model.copy(w_tau=1e39)                  # infinite in FP32: every cost is inf or nan
    c = M.Controller.from_problem(M.Model(m), p, mapping=0)
    warm = p.nominal.astype(np.float32)
    mean, best, info = c.solve(p.state, warm=warm, check=False)
    assert info["return_status"] == M.MPPI_ERR_ALL_COSTS_NONFINITE
    assert info["n_finite"] == 0
    np.testing.assert_array_equal(mean, warm)
    np.testing.assert_array_equal(best, warm)


def test_single_sample_returns_nominal(M):
    p = S.plain_quadruped(n=1)
    c = M.Controller.from_problem(M.Model(p.model), p, mapping=0)
    warm = p.nominal.astype(np.float32)
    mean, best, info = c.solve(p.state, warm=warm)
    np.testing.assert_array_equal(mean, warm)
    assert info["best_index"] == 0 and info["ess"] == pytest.approx(1.0)


def test_zero_sigma_fixed_point(M):
    p = S.plain_quadruped()
    c = M.Controller(M.Model(p.model), p.n, p.horizon, p.nk, p.lam, np.zeros((1, p.nk)), dt=p.dt, mapping=0)
    warm = p.nominal.astype(np.float32)
    mean, best, info = c.solve(p.state, warm=warm)
    np.testing.assert_allclose(mean, warm, rtol=0, atol=1e-6)
    assert info["cost_min"] == info["cost_max"]

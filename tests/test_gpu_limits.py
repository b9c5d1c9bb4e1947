"""The library's size limits and degenerate shapes on the CUDA path against the FP64
oracle: the largest accepted model (32 bodies on a random tree, 32 contact points) with
the largest knot count (16), the shortest horizon (H = 1) with the fewest knots (2), and
the rejections one past each limit.

Tolerances: FP64 check build 1e-9; FP32 costs and control points 1e-3, or within 10x the
oracle's own spread under FP32-sized (1e-6) perturbations of the initial state
(tests/_parity.py) where contact makes the rollout sensitive.
"""
import numpy as np
import pytest

from paper_2511_19204_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_2511_19204_gb300 import build, mppi
    build.build()
    mppi.load()
    return mppi


def _tree_problem(n):
    m = S.random_tree(32, 32)
    nk, H, dt = 16, 40, 0.005
    return m, n, nk, H, dt, S.standing_state(m, jitter=0.05, base_vel=0.2, seed=9), S.nominal_knots(m, nk)


def test_largest_tree_rollouts(M, orc):
    from _parity import rollout_envelope
    m, n, nk, H, dt, x0, nom = _tree_problem(64)
    assert m.nb == 32 and m.nc == 32
    sig = S.linear_sigma(nk, 1)
    kn = orc.sample_knots(m.nj, nk, n, H, dt, nom, sig[0], seed=5).astype(np.float32)
    c = M.Controller(M.Model(m), n, H, nk, 0.1, sig, dt=dt, seed=5, mapping=M.MPPI_MAP_WARP)
    (ref_c, ref_f), env_c, _ = rollout_envelope(m, x0, kn.astype(np.float64), H, dt, 1e-6, draws=4)
    got, fin = c.rollout_explicit(x0, kn, finals=True)
    err = np.abs(got - ref_c) / np.abs(ref_c)
    print(f"32-body tree: FP32 cost rel. error median {np.median(err):.2e} max {err.max():.2e}")
    assert np.median(err) < 1e-4
    assert np.all(np.abs(got - ref_c) <= np.maximum(1e-3 * np.abs(ref_c), 10 * env_c))
    c.set_fp64_check(True)
    got64, fin64 = c.rollout_explicit(x0, kn, finals=True)
    scale = np.max(np.abs(ref_f), axis=1)
    assert np.max(np.abs(got64 - ref_c) / np.abs(ref_c)) < 1e-9
    assert np.max(np.max(np.abs(fin64 - ref_f), axis=1) / scale) < 1e-9


def test_largest_tree_solve(M, orc):
    m, n, nk, H, dt, x0, nom = _tree_problem(256)
    sig = S.linear_sigma(nk, 2)
    c = M.Controller(M.Model(m), n, H, nk, 0.1, sig, iters=2, dt=dt, seed=7, mapping=M.MPPI_MAP_WARP)
    mean, best, info = c.solve(x0, warm=nom.astype(np.float32))
    ref = orc.solve(m, n, nk, H, 2, dt, 0.1, sig, x0, nom.astype(np.float32).astype(np.float64), seed=7)
    err = np.max(np.abs(mean - ref["mean"]) / np.maximum(1.0, np.abs(ref["mean"])))
    print(f"32-body tree solve: mean knot error {err:.2e}; best cost {info['best_cost']:.4f} vs {ref['best_cost']:.4f}")
    assert err <= 1e-3
    assert info["best_cost"] == pytest.approx(ref["best_cost"], rel=1e-3)


@pytest.mark.parametrize("mapping", [0, 2])
def test_shortest_horizon_fewest_knots(M, orc, mapping):
    m = S.quadruped()
    n, nk, H, dt = 33, 2, 1, 0.005
    sig = S.linear_sigma(nk, 1)
    x0 = S.standing_state(m, jitter=0.02, seed=3)
    nom = S.nominal_knots(m, nk)
    c = M.Controller(M.Model(m), n, H, nk, 0.1, sig, dt=dt, seed=2, mapping=mapping)
    mean, best, info = c.solve(x0, warm=nom.astype(np.float32))
    ref = orc.solve(m, n, nk, H, 1, dt, 0.1, sig, x0, nom.astype(np.float32).astype(np.float64), seed=2)
    err = np.max(np.abs(mean - ref["mean"]) / np.maximum(1.0, np.abs(ref["mean"])))
    assert err <= 1e-4
    assert info["best_index"] == ref["best_index"]


def test_one_past_each_limit_is_rejected(M):
    with pytest.raises(M.MppiError):
        M.Model(S.random_tree(33, 4))
    with pytest.raises(M.MppiError):
        M.Model(S.random_tree(8, 33))
    mod = M.Model(S.quadruped())
    for nk in (1, 17):
        with pytest.raises(M.MppiError):
            M.Controller(mod, 8, 20, nk, 0.1, np.full((1, nk), 0.1), dt=0.005)
    with pytest.raises(M.MppiError):
        M.Controller(mod, 8, 0, 4, 0.1, np.full((1, 4), 0.1), dt=0.005)
    with pytest.raises(M.MppiError):
        M.Controller(mod, 0, 20, 4, 0.1, np.full((1, 4), 0.1), dt=0.005)

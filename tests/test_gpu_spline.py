"""Position-only spline variants of the ablation (Sec. IV-D) on the CUDA path against the
FP64 oracle, through the C ABI. The CUDA path turns each variant into Hermite knots (the
variant's node slopes in the velocity slots); the oracle evaluates each variant from its
own definition.

Tolerances:
  node slopes (FP32 Thomas solve vs FP64 dense solve)   1e-5 relative to max |slope|
  rollout costs                                         1e-3 (median 1e-4)
  updated control points                                1e-3 (relative to max(1, |x|))
  batched == alone                                      bit-exact
"""
import numpy as np
import pytest

from paper_2511_19204_gb300 import synth as S

pytestmark = pytest.mark.gpu
VARIANTS = [1, 2]   # MPPI_SPLINE_CUBIC, MPPI_SPLINE_QUADRATIC


@pytest.fixture(scope="module")
def M():
    from paper_2511_19204_gb300 import build, mppi
    build.build()
    mppi.load()
    return mppi


@pytest.mark.parametrize("spline", VARIANTS)
@pytest.mark.parametrize("nk", [2, 5, 16])
def test_noise_writes_variant_slopes(M, orc, spline, nk):
    p = S.scale_quadruped(n=77)
    c = M.Controller(M.Model(p.model), p.n, p.horizon, nk, p.lam, S.linear_sigma(nk, 1), dt=p.dt, seed=3,
                     spline=spline)
    nom = S.nominal_knots(p.model, nk).astype(np.float32)
    kn = c.sample_knots(0, 0, nom).astype(np.float64)
    ref_q = orc.sample_knots(p.model.nj, nk, p.n, p.horizon, p.dt, nom.astype(np.float64), S.linear_sigma(nk, 1)[0],
                             seed=3)[:, :, 0]
    assert np.max(np.abs(kn[:, :, 0] - ref_q) / np.maximum(1.0, np.abs(ref_q))) < 1e-5
    for n in range(p.n):
        ref = orc.spline_slopes(kn[n], p.horizon, p.dt, spline)
        scale = max(1.0, np.max(np.abs(ref[:, 1])))
        assert np.max(np.abs(kn[n, :, 1] - ref[:, 1])) / scale < 1e-5, n


@pytest.mark.parametrize("spline", VARIANTS)
@pytest.mark.parametrize("mapping", [0, 2])
def test_variant_rollouts_match_oracle(M, orc, spline, mapping):
    p = S.scale_quadruped(n=128)
    c = M.Controller.from_problem(M.Model(p.model), p, mapping=mapping, spline=spline)
    kn = c.sample_knots(0, 0, p.nominal.astype(np.float32))
    got = c.rollout_explicit(p.state, kn)
    ref = orc.rollout_batch(p.model, p.state, kn.astype(np.float64), p.horizon, p.dt, spline=spline)
    err = np.abs(got - ref) / np.abs(ref)
    print(f"spline {spline} mapping {mapping}: cost rel. error median {np.median(err):.2e} max {err.max():.2e}")
    assert np.median(err) < 1e-4 and err.max() < 1e-3


@pytest.mark.parametrize("spline", VARIANTS)
def test_variant_solve_matches_oracle(M, orc, spline):
    p = S.scale_quadruped(n=1024)
    c = M.Controller.from_problem(M.Model(p.model), p, spline=spline)
    nom32 = p.nominal.astype(np.float32)
    mean, best, info = c.solve(p.state, warm=nom32)
    ref = orc.solve(p.model, p.n, p.nk, p.horizon, p.iters, p.dt, p.lam, p.sigma, p.state, nom32.astype(np.float64),
                    seed=p.seed, spline=spline)
    scale = np.maximum(1.0, np.abs(ref["mean"]))
    err_q = np.max(np.abs(mean[:, 0] - ref["mean"][:, 0]) / scale[:, 0])
    err_v = np.max(np.abs(mean[:, 1] - ref["mean"][:, 1])) / max(1.0, np.max(np.abs(ref["mean"][:, 1])))
    print(f"spline {spline}: mean knot error q {err_q:.2e} v {err_v:.2e}; best cost {info['best_cost']:.4f} "
          f"vs {ref['best_cost']:.4f}")
    assert err_q <= 1e-3 and err_v <= 1e-3
    assert info["best_cost"] == pytest.approx(ref["best_cost"], rel=1e-3)


def test_variant_batch_equals_alone(M):
    from test_gpu_batch import _batch
    quad, hum = S.quadruped(), S.humanoid()
    mq, mh = M.Model(quad), M.Model(hum)
    specs = [(mq, quad, 2, 97, 60, 4, 1), (mq, quad, 0, 40, 40, 6, 2), (mh, hum, 2, 129, 30, 7, 1),
             (mh, hum, 0, 33, 50, 5, 2), (mq, quad, 2, 64, 50, 5, 0)]
    alone, batch, states, warms = [], [], [], []
    for i, (mod, rob, mp, K, H, nk, spline) in enumerate(specs):
        sig = S.linear_sigma(nk, 1)
        kw = dict(iters=1, dt=0.005, seed=31 + i, instance=i, mapping=mp, spline=spline)
        alone.append(M.Controller(mod, K, H, nk, 0.1, sig, **kw))
        batch.append(M.Controller(mod, K, H, nk, 0.1, sig, **kw))
        states.append(S.standing_state(rob, jitter=0.02, base_vel=0.2, seed=400 + i))
        warms.append(S.nominal_knots(rob, nk).astype(np.float32))
    ref = [c.solve(x, warm=w) for c, x, w in zip(alone, states, warms)]
    rc, means, bests, infos = _batch(M, batch, states, warms)
    assert rc == 0
    for i, (r, m, b, inf) in enumerate(zip(ref, means, bests, infos)):
        np.testing.assert_array_equal(m, r[0].reshape(-1), err_msg=f"instance {i}")
        np.testing.assert_array_equal(b, r[1].reshape(-1), err_msg=f"instance {i}")
        assert inf["best_cost"] == r[2]["best_cost"]


def test_bad_spline_rejected(M):
    p = S.scale_quadruped(n=8)
    with pytest.raises(M.MppiError):
        M.Controller.from_problem(M.Model(p.model), p, spline=3)

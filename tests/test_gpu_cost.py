"""The modular cost of Sec. IV-A (running terms, terminal term, Tab. II weights) on the
CUDA path against the FP64 oracle, through the C ABI.

Tolerances (as for the other contact rollouts at dt = 0.005):
  FP64 check build, each term alone and Tab. II sets     1e-9 relative (costs)
  FP32 product                                           1e-3 relative (costs), median 1e-4
  updated control points                                 1e-3 (relative to max(1, |x|))
  batched == alone                                       bit-exact

The contact terms switch with the contact set (||v_c||_1 counts only points in contact,
f_c jumps from 0 to the damping force at touchdown), so their sum is discontinuous in
the trajectory: where a contact point of a sample comes within an FP32 position error of
the ground at a step, FP32 and FP64 may place it on opposite sides and the costs differ
by that step's jump. A sample above 1e-3 must therefore lie within 3x the oracle's own
spread when its initial state is perturbed at FP32 precision (1e-6 relative, 16 draws;
tests/_parity.py), and at most 5 % of the samples may be above 1e-3.
"""
import numpy as np
import pytest

from paper_2511_19204_gb300 import synth as S

pytestmark = pytest.mark.gpu
TERMS = ["w_h", "w_orient", "w_q", "w_cvel", "w_cforce", "w_term"]


def _check_fp32(orc, p, kn64, got, ref, label):
    from _parity import rollout_envelope
    err = np.abs(got - ref) / np.abs(ref)
    bad = np.nonzero(err >= 1e-3)[0]
    msg = ""
    if len(bad):
        _, env, _ = rollout_envelope(p.model, p.state, kn64[bad], p.horizon, p.dt, 1e-6, draws=16)
        ratio = np.abs(got[bad] - ref[bad]) / np.maximum(env, 1e-300)
        msg = f"; {len(bad)} above 1e-3 at {ratio.max():.2f}x the oracle's FP32-level spread"
        assert np.all(np.abs(got[bad] - ref[bad]) <= 3 * env + 1e-3 * np.abs(ref[bad])), (bad, ratio)
    print(f"{label}: FP32 rel. error median {np.median(err):.2e} max {err.max():.2e}{msg}")
    assert np.median(err) < 1e-4
    assert len(bad) <= 0.05 * len(err)


@pytest.fixture(scope="module")
def M():
    from paper_2511_19204_gb300 import build, mppi
    build.build()
    mppi.load()
    return mppi


def _only(m, term, w=1.0):
    kw = {t: 0.0 for t in TERMS}
    kw.update(w_z=0.0, w_vx=0.0, w_tilt=0.0, w_tau=0.0)
    kw[term] = w
    total = float(np.sum(m.mass)) * m.gravity
    return m.copy(f0=(0.05, -0.1, total / max(m.nc, 1)), pdot_des=(0.4, 0.1, 0.0),
                  quat_des=(0.98, 0.05, -0.1, 0.15), q_stand=m.q_stand, **kw)


def _costs(M, orc, p, mapping, fp64=False):
    m = p.model
    kn = orc.sample_knots(m.nj, p.nk, p.n, p.horizon, p.dt, p.nominal, p.sigma[0], seed=p.seed)
    kn32 = kn.astype(np.float32)
    ref = orc.rollout_batch(m, p.state, kn32.astype(np.float64), p.horizon, p.dt)
    c = M.Controller.from_problem(M.Model(m), p, mapping=mapping)
    if fp64:
        c.set_fp64_check(True)
    got = c.rollout_explicit(p.state, kn32)
    return got, ref, kn32.astype(np.float64)


@pytest.mark.parametrize("term", TERMS)
@pytest.mark.parametrize("mapping", [0, 2])
def test_each_term_fp64_check(M, orc, term, mapping):
    # every term alone, FP64 check build (the warp kernel, and the product's lanes-per-chain
    # kernel with the modular cost compiled in): the algorithm, not FP32 rounding
    p = S.scale_quadruped(n=64)
    p.model = _only(p.model, term)
    got, ref, _ = _costs(M, orc, p, mapping=mapping, fp64=True)
    err = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
    print(f"{term}: FP64 check rel. error max {err.max():.2e}, cost median {np.median(ref):.3e}")
    assert np.all(ref > 0) and err.max() < 1e-9


@pytest.mark.parametrize("term", TERMS)
@pytest.mark.parametrize("mapping", [0, 2])
def test_each_term_fp32(M, orc, term, mapping):
    p = S.scale_quadruped(n=128)
    p.model = _only(p.model, term)
    got, ref, kn64 = _costs(M, orc, p, mapping=mapping)
    _check_fp32(orc, p, kn64, got, ref, f"{term} mapping {mapping}")


@pytest.mark.parametrize("task", sorted(S.TAB2_WEIGHTS))
@pytest.mark.parametrize("robot", ["quadruped", "humanoid"])
def test_tab2_weight_sets(M, orc, task, robot):
    if robot == "quadruped":
        p = S.scale_quadruped(n=96)
    else:
        p = S.humanoid_problem(n=64)
        p.horizon = 100
    p.model = S.with_paper_cost(p.model, task, pdot_des=(0.5, 0.0, 0.0), keep_quadratic=True)
    got64, ref, kn64 = _costs(M, orc, p, mapping=0, fp64=True)
    assert np.max(np.abs(got64 - ref) / np.abs(ref)) < 1e-9
    got64c, _, _ = _costs(M, orc, p, mapping=2, fp64=True)   # the product's chain / split kernel in double
    assert np.max(np.abs(got64c - ref) / np.abs(ref)) < 1e-9
    for mapping in ((0, 1, 2) if robot == "quadruped" else (0, 2)):   # half warp: <= 16 bodies
        got, _, _ = _costs(M, orc, p, mapping=mapping)
        _check_fp32(orc, p, kn64, got, ref, f"{robot} {task} mapping {mapping}")


def test_paper_walking_solve_matches_oracle(M, orc):
    p = S.paper_walking(n=1024)
    c = M.Controller.from_problem(M.Model(p.model), p)
    nom32 = p.nominal.astype(np.float32)
    mean, best, info = c.solve(p.state, warm=nom32)
    ref = orc.solve(p.model, p.n, p.nk, p.horizon, p.iters, p.dt, p.lam, p.sigma, p.state,
                    nom32.astype(np.float64), seed=p.seed)
    err = np.max(np.abs(mean - ref["mean"]) / np.maximum(1.0, np.abs(ref["mean"])))
    print(f"paper walking: mean knot error {err:.2e}; best cost {info['best_cost']:.3f} vs {ref['best_cost']:.3f}")
    assert err <= 1e-3
    assert info["best_cost"] == pytest.approx(ref["best_cost"], rel=1e-3)


def test_paper_cost_batch_equals_alone(M):
    from test_gpu_batch import _batch
    quad = S.with_paper_cost(S.quadruped(), "walking", pdot_des=(0.5, 0.0, 0.0))
    hum = S.with_paper_cost(S.humanoid(), "bipedal", pdot_des=(0.3, 0.0, 0.0), z_des=0.9)
    mq, mh = M.Model(quad), M.Model(hum)
    specs = [(mq, quad, 2, 97, 60, 4), (mq, quad, 0, 40, 40, 5), (mh, hum, 2, 129, 30, 7), (mh, hum, 0, 33, 50, 6)]
    alone, batch, states, warms = [], [], [], []
    for i, (mod, rob, mp, K, H, nk) in enumerate(specs):
        sig = S.linear_sigma(nk, 1)
        kw = dict(iters=1, dt=0.005, seed=11 + i, instance=i, mapping=mp)
        alone.append(M.Controller(mod, K, H, nk, 0.1, sig, **kw))
        batch.append(M.Controller(mod, K, H, nk, 0.1, sig, **kw))
        states.append(S.standing_state(rob, jitter=0.02, base_vel=0.2, seed=300 + i))
        warms.append(S.nominal_knots(rob, nk).astype(np.float32))
    ref = [c.solve(x, warm=w) for c, x, w in zip(alone, states, warms)]
    rc, means, bests, infos = _batch(M, batch, states, warms)
    assert rc == 0
    for i, (r, m, b, inf) in enumerate(zip(ref, means, bests, infos)):
        np.testing.assert_array_equal(m, r[0].reshape(-1), err_msg=f"instance {i}")
        np.testing.assert_array_equal(b, r[1].reshape(-1), err_msg=f"instance {i}")
        assert inf["best_cost"] == r[2]["best_cost"]


def test_model_rejects_negative_weights(M):
    with pytest.raises(M.MppiError):
        M.Model(S.quadruped().copy(w_cvel=-1.0))
    with pytest.raises(M.MppiError):
        M.Model(S.quadruped().copy(w_term=float("nan")))

"""Receding-horizon steps of Sec. III-E through the C ABI: state prediction over the
compute delay from the resident warm start, the shift of that warm start with the tail
padded, and a closed loop of predict -> shift -> solve, each against the FP64 oracle.

Tolerances:
  shift (FP64 evaluation of FP32 knots, one rounding)   1 ulp(FP32) + 1e-12
  prediction, FP64 check build                          1e-9 relative (largest component)
  prediction, FP32 product                              1e-4 relative up to 40 steps,
                                                        1e-3 over the whole horizon
  prediction over H steps vs the warp rollout's final   bit-exact (same device function)
  closed-loop solves                                    1e-3 on control points (solve tests)
"""
import numpy as np
import pytest

from paper_2511_19204_gb300 import synth as S

pytestmark = pytest.mark.gpu
F32_EPS = 2.0 ** -23


@pytest.fixture(scope="module")
def M():
    from paper_2511_19204_gb300 import build, mppi
    build.build()
    mppi.load()
    return mppi


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _solved(M, n=256, **kw):
    p = S.scale_quadruped(n=n)
    c = M.Controller.from_problem(M.Model(p.model), p, **kw)
    c.solve(p.state, warm=p.nominal.astype(np.float32))
    return p, c


def test_shift_matches_oracle(M, orc):
    p, c = _solved(M)
    blob = c.export_state()
    W = c.warm_start()
    assert not np.array_equal(W, p.nominal.astype(np.float32))   # tau_best moved
    c.shift_warm_start(0)
    np.testing.assert_array_equal(c.warm_start(), W)
    for steps in (1, 3, 17, 40, p.horizon - 1, p.horizon, p.horizon + 25):
        c.import_state(blob)
        c.shift_warm_start(steps)
        got = c.warm_start().astype(np.float64)
        ref = orc.shift_knots(W.astype(np.float64), p.horizon, steps, p.dt)
        bound = F32_EPS * np.abs(ref) + 1e-12
        assert np.all(np.abs(got - ref) <= bound), (steps, np.max(np.abs(got - ref) - bound))
    # on knots sampled from one cubic per joint the spline is that cubic, so shifts
    # compose: by 7 then by 5 is by 12 up to the rounding of the intermediate knots, on
    # every knot whose read time stays clear of the padded tail segment (all but the
    # second-to-last; the last is the held end point either way)
    rng = np.random.default_rng(4)
    T = p.horizon * p.dt
    tk = np.arange(p.nk) * T / (p.nk - 1)
    coef = rng.normal(size=(4, p.model.nj))
    cub = np.zeros((p.nk, 2, p.model.nj))
    cub[:, 0] = coef[0] + np.outer(tk, coef[1]) + np.outer(tk ** 2, coef[2]) + np.outer(tk ** 3, coef[3])
    cub[:, 1] = coef[1] + 2 * np.outer(tk, coef[2]) + 3 * np.outer(tk ** 2, coef[3])
    c.import_state(blob[:20] + cub.astype(np.float32).tobytes())
    c.shift_warm_start(7)
    c.shift_warm_start(5)
    ref = orc.shift_knots(cub.astype(np.float32).astype(np.float64), p.horizon, 12, p.dt)
    keep = [j for j in range(p.nk) if j != p.nk - 2]
    assert _rel(c.warm_start()[keep], ref[keep]) < 1e-5


def test_shift_rejects_negative_steps(M):
    p, c = _solved(M, n=64)
    with pytest.raises(M.MppiError):
        c.shift_warm_start(-1)


@pytest.mark.parametrize("robot", ["quadruped", "humanoid"])
def test_prediction_matches_oracle(M, orc, robot):
    if robot == "quadruped":
        p, c = _solved(M)
    else:
        p = S.humanoid_problem(n=128)
        p.horizon = 100
        c = M.Controller.from_problem(M.Model(p.model), p)
        c.solve(p.state, warm=p.nominal.astype(np.float32))
    W = c.warm_start().astype(np.float64)
    x = p.state
    np.testing.assert_array_equal(c.predict_state(x, 0), x)
    for steps in (1, 4, 10, 40, p.horizon):
        ref = orc.predict_state(p.model, x, W, p.horizon, steps, p.dt)
        got = c.predict_state(x, steps)
        err = _rel(got, ref)
        print(f"{robot}: prediction over {steps} steps, FP32 rel. error {err:.2e}")
        assert err < (1e-4 if steps <= 40 else 1e-3)
    c.set_fp64_check(True)
    for steps in (1, 10, p.horizon):
        ref = orc.predict_state(p.model, x, W, p.horizon, steps, p.dt)
        assert _rel(c.predict_state(x, steps), ref) < 1e-9
    c.set_fp64_check(False)


def test_prediction_over_horizon_is_rollout_final(M):
    p, c = _solved(M, n=64, mapping=0)
    W = c.warm_start()
    kn = np.broadcast_to(W, (p.n,) + W.shape).copy()
    _, fins = c.rollout_explicit(p.state, kn, finals=True)
    np.testing.assert_array_equal(c.predict_state(p.state, p.horizon), fins[0])


def test_prediction_rejects_bad_arguments(M):
    p, c = _solved(M, n=64)
    with pytest.raises(M.MppiError):
        c.predict_state(p.state, p.horizon + 1)
    with pytest.raises(M.MppiError):
        c.predict_state(p.state, -1)
    bad = p.state.copy()
    bad[0] = np.nan
    with pytest.raises(M.MppiError):
        c.predict_state(bad, 3)


def test_closed_loop_matches_oracle(M, orc):
    # three receding-horizon cycles (Sec. III-E with the loop of Alg. 1): predict the
    # state after the delay from the executed warm start, shift the warm start, solve from
    # the prediction. Each step is compared with the oracle given the same inputs.
    p = S.scale_quadruped(n=512)
    c = M.Controller.from_problem(M.Model(p.model), p)
    c.solve(p.state, warm=p.nominal.astype(np.float32))
    x = p.state.copy()
    delay = 6
    for cycle in range(3):
        W = c.warm_start().astype(np.float64)
        ctr = c.iter_counter
        x_pred = c.predict_state(x, delay)
        assert _rel(x_pred, orc.predict_state(p.model, x, W, p.horizon, delay, p.dt)) < 1e-4
        c.shift_warm_start(delay)
        W_shift = c.warm_start()
        ref_shift = orc.shift_knots(W, p.horizon, delay, p.dt)
        assert np.all(np.abs(W_shift - ref_shift) <= F32_EPS * np.abs(ref_shift) + 1e-12)
        mean, best, info = c.solve(x_pred)
        ref = orc.solve(p.model, p.n, p.nk, p.horizon, p.iters, p.dt, p.lam, p.sigma, x_pred,
                        W_shift.astype(np.float64), seed=p.seed, iter_base=ctr)
        err = np.max(np.abs(mean - ref["mean"]) / np.maximum(1.0, np.abs(ref["mean"])))
        print(f"cycle {cycle}: mean knot error {err:.2e}, best cost {info['best_cost']:.4f} "
              f"vs {ref['best_cost']:.4f}")
        assert err <= 1e-3
        assert info["best_cost"] == pytest.approx(ref["best_cost"], rel=1e-3)
        x = x_pred


def test_device_cycle_matches_host_cycle(M):
    # the device-resident cycle (no host round trip between the steps) gives the same bits
    torch = pytest.importorskip("torch")
    p = S.scale_quadruped(n=256)
    hosts, devs = [], []
    c1 = M.Controller.from_problem(M.Model(p.model), p)
    c2 = M.Controller.from_problem(M.Model(p.model), p)
    c1.solve(p.state, warm=p.nominal.astype(np.float32))
    c2.solve(p.state, warm=p.nominal.astype(np.float32))
    x = p.state.copy()
    dx = torch.tensor(p.state, dtype=torch.float64, device="cuda")
    dp = torch.zeros_like(dx)
    mean = torch.zeros(c2.E, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    for _ in range(2):
        x = c1.predict_state(x, 5)
        c1.shift_warm_start(5)
        hosts.append((x.copy(), c1.solve(x)[0]))
        c2.predict_state_device(dx.data_ptr(), 5, dp.data_ptr())
        c2.shift_warm_start(5)
        c2.solve_device(dp.data_ptr(), mean.data_ptr())
        c2.sync()
        devs.append((dp.cpu().numpy().copy(), mean.cpu().numpy().reshape(hosts[-1][1].shape)))
        dx.copy_(dp)
        torch.cuda.synchronize()
    for (xh, mh), (xd, md) in zip(hosts, devs):
        np.testing.assert_array_equal(xh, xd)
        np.testing.assert_array_equal(mh, md)

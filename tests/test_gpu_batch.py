"""Batched solves (one persistent launch over uneven instances) against per-instance
solves and the oracle, through the C ABI."""
import ctypes as C

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


def _mix(M):
    """Uneven instances: both robots, every batched mapping, ragged K, 1 and 3 iterations."""
    quad, hum = S.quadruped(), S.humanoid()
    mq, mh = M.Model(quad), M.Model(hum)
    specs = [  # (model, robot, mapping, K, H, nk, iters, lam, seed)
        (mq, quad, 2, 97, 60, 4, 1, 0.1, 1), (mq, quad, 2, 256, 120, 6, 3, 0.2, 2),
        (mq, quad, 1, 33, 50, 5, 1, 0.3, 3), (mq, quad, 0, 40, 40, 4, 2, 0.1, 4),
        (mh, hum, 0, 70, 50, 8, 1, 0.05, 5), (mh, hum, 2, 129, 30, 7, 2, 0.5, 6), (mh, hum, 2, 300, 40, 4, 1, 0.2, 9),
        (mq, quad, 2, 1, 20, 4, 1, 0.1, 7), (mq, quad, 2, 65, 100, 8, 1, 0.25, 8),
    ]
    out = []
    for i, (mod, rob, mp, K, H, nk, it, lam, seed) in enumerate(specs):
        sig = S.linear_sigma(nk, it)
        x0 = S.standing_state(rob, jitter=0.02, base_vel=0.2, seed=100 + i)
        warm = S.nominal_knots(rob, nk).astype(np.float32)
        kw = dict(iters=it, dt=0.005, seed=seed, instance=i, mapping=mp)
        out.append(dict(mod=mod, rob=rob, K=K, H=H, nk=nk, it=it, lam=lam, sig=sig, x0=x0, warm=warm, kw=kw))
    return out


def _batch(M, ctrls, states, warms):
    L = M.load()
    n = len(ctrls)
    hs = (C.c_void_p * n)(*[c.h for c in ctrls])
    st = [np.ascontiguousarray(s, dtype=np.float64) for s in states]
    wa = [np.ascontiguousarray(w, dtype=np.float32).reshape(-1) if w is not None else None for w in warms]
    means = [np.zeros(c.E, np.float32) for c in ctrls]
    bests = [np.zeros(c.E, np.float32) for c in ctrls]
    dp = C.POINTER(C.c_double)
    fp = C.POINTER(C.c_float)
    ps = (dp * n)(*[s.ctypes.data_as(dp) for s in st])
    pw = (fp * n)(*[w.ctypes.data_as(fp) if w is not None else None for w in wa])
    pm = (fp * n)(*[m.ctypes.data_as(fp) for m in means])
    pb = (fp * n)(*[b.ctypes.data_as(fp) for b in bests])
    info = (M.mppi_result * n)()
    rc = L.mppi_solve_batch(hs, n, ps, pw, pm, pb, info)
    return rc, means, bests, [info[i].as_dict() for i in range(n)]


def test_batch_equals_alone_bitwise(M):
    mix = _mix(M)
    alone = [M.Controller(d["mod"], d["K"], d["H"], d["nk"], d["lam"], d["sig"], **d["kw"]) for d in mix]
    batch = [M.Controller(d["mod"], d["K"], d["H"], d["nk"], d["lam"], d["sig"], **d["kw"]) for d in mix]
    ref = [c.solve(d["x0"], warm=d["warm"]) for c, d in zip(alone, mix)]
    rc, means, bests, infos = _batch(M, batch, [d["x0"] for d in mix], [d["warm"] for d in mix])
    assert rc == 0
    for i, (r, m, b, inf) in enumerate(zip(ref, means, bests, infos)):
        np.testing.assert_array_equal(m, r[0].reshape(-1), err_msg=f"instance {i}")
        np.testing.assert_array_equal(b, r[1].reshape(-1), err_msg=f"instance {i}")
        assert inf["best_cost"] == r[2]["best_cost"] and inf["best_index"] == r[2]["best_index"]
        assert inf["n_finite"] == r[2]["n_finite"] and inf["ess"] == r[2]["ess"]
    # the next solve of each: resident warm start and counters advance the same way
    ref2 = [c.solve(d["x0"]) for c, d in zip(alone, mix)]
    rc, means2, _, _ = _batch(M, batch, [d["x0"] for d in mix], [None] * len(mix))
    assert rc == 0
    for i, (r, m) in enumerate(zip(ref2, means2)):
        np.testing.assert_array_equal(m, r[0].reshape(-1), err_msg=f"second solve, instance {i}")
        assert batch[i].iter_counter == alone[i].iter_counter


def test_batch_matches_oracle(M, orc):
    mix = _mix(M)
    ctrls = [M.Controller(d["mod"], d["K"], d["H"], d["nk"], d["lam"], d["sig"], **d["kw"]) for d in mix]
    rc, means, _, infos = _batch(M, ctrls, [d["x0"] for d in mix], [d["warm"] for d in mix])
    assert rc == 0
    for i, d in enumerate(mix):
        ref = orc.solve(d["rob"], d["K"], d["nk"], d["H"], d["it"], 0.005, d["lam"], d["sig"], d["x0"],
                        d["warm"].astype(np.float64), seed=d["kw"]["seed"], inst=i)
        err = np.max(np.abs(means[i] - ref["mean"].reshape(-1)) / np.maximum(1.0, np.abs(ref["mean"].reshape(-1))))
        assert err < 1e-3, (i, err)
        assert infos[i]["best_cost"] == pytest.approx(ref["best_cost"], rel=1e-3)


def test_batch_rejects_bad_input(M):
    mix = _mix(M)[:2]
    c = [M.Controller(d["mod"], d["K"], d["H"], d["nk"], d["lam"], d["sig"], **d["kw"]) for d in mix]
    rc, *_ = _batch(M, [c[0], c[0]], [mix[0]["x0"], mix[0]["x0"]], [None, None])
    assert rc == M.MPPI_ERR_INVALID_ARG
    x = mix[1]["x0"].copy()
    x[0] = np.inf
    rc, *_ = _batch(M, c, [mix[0]["x0"], x], [None, None])
    assert rc == M.MPPI_ERR_NONFINITE_STATE


def test_every_rollout_variant_in_one_batch(M):
    # one batch holding an instance of every rollout variant (axis-specialised and generic
    # chain kernels for both robots, with and without the modular cost; half-warp and warp
    # mappings), so every group runs its own persistent kernel beside the others: each
    # instance gives the bits of its single solve
    quad, hum = S.quadruped(), S.humanoid()
    qaxis = quad.axis.copy()
    qaxis[1] = np.array([1.0, 0.0, 0.05]) / np.linalg.norm([1.0, 0.0, 0.05])
    hjpos = hum.jpos.copy()
    hjpos[hum.nb - 1, 0] = 0.01
    robots = {"xyy": quad, "quad_generic": quad.copy(axis=qaxis), "split": hum, "hum_generic": hum.copy(jpos=hjpos)}
    paper = {k: S.with_paper_cost(r, "walking", pdot_des=(0.4, 0.0, 0.0)) for k, r in robots.items()}
    specs = []   # (robot, mapping, K, H, nk)
    for k in robots:
        specs.append((robots[k], 2, 70, 30, 5))
        specs.append((paper[k], 2, 33, 25, 4))
    specs += [(quad, 1, 19, 30, 4), (quad, 0, 11, 20, 6), (hum, 0, 9, 20, 5)]
    models = {}
    alone, batch, states, warms = [], [], [], []
    for i, (rob, mp, K, H, nk) in enumerate(specs):
        mod = models.setdefault(id(rob), M.Model(rob))
        sig = S.linear_sigma(nk, 1)
        kw = dict(iters=1, dt=0.005, seed=70 + i, instance=i, mapping=mp)
        alone.append(M.Controller(mod, K, H, nk, 0.2, sig, **kw))
        batch.append(M.Controller(mod, K, H, nk, 0.2, sig, **kw))
        states.append(S.standing_state(rob, jitter=0.02, base_vel=0.2, seed=500 + i))
        warms.append(S.nominal_knots(rob, nk).astype(np.float32))
    plans = {models[id(r)].info()["axis_plan"] for r, *_ in specs}
    assert plans == {0, 1, 2}
    ref = [c.solve(x, warm=w) for c, x, w in zip(alone, states, warms)]
    rc, means, bests, infos = _batch(M, batch, states, warms)
    assert rc == 0
    for i, (r, m, b, inf) in enumerate(zip(ref, means, bests, infos)):
        np.testing.assert_array_equal(m, r[0].reshape(-1), err_msg=f"instance {i}")
        np.testing.assert_array_equal(b, r[1].reshape(-1), err_msg=f"instance {i}")
        assert inf["best_cost"] == r[2]["best_cost"]


@pytest.mark.parametrize("K", [4000, 12000])
def test_large_instances_batch_equals_alone_bitwise(M, orc, K):
    """Several chunk groups and a ragged last chunk, on both single-solve reductions: 4000
    samples (63 chunks, 4 groups) fit on the device at once and finish cooperatively,
    12000 (188 chunks, 12 groups) finish group by group. Both must equal the batched
    kernel's group-by-group reduction bit for bit, and the oracle at 1e-3."""
    quad = S.quadruped()
    mq = M.Model(quad)
    nk, H, it = 6, 40, 2
    sig = S.linear_sigma(nk, it)
    x0 = S.standing_state(quad, jitter=0.02, base_vel=0.2, seed=77)
    warm = S.nominal_knots(quad, nk).astype(np.float32)
    kw = dict(iters=it, dt=0.005, seed=5, instance=2, mapping=2)
    alone = M.Controller(mq, K, H, nk, 0.1, sig, **kw)
    batch = M.Controller(mq, K, H, nk, 0.1, sig, **kw)
    ref = alone.solve(x0, warm=warm)
    rc, means, bests, infos = _batch(M, [batch], [x0], [warm])
    assert rc == 0
    np.testing.assert_array_equal(means[0], ref[0].reshape(-1))
    np.testing.assert_array_equal(bests[0], ref[1].reshape(-1))
    assert infos[0]["ess"] == ref[2]["ess"] and infos[0]["best_cost"] == ref[2]["best_cost"]
    o = orc.solve(quad, K, nk, H, it, 0.005, 0.1, sig, x0, warm.astype(np.float64), seed=5, inst=2)
    err = float(np.max(np.abs(ref[0] - o["mean"]) / np.maximum(1.0, np.abs(o["mean"]))))
    assert err <= 1e-3, err
    assert ref[2]["best_cost"] == pytest.approx(o["best_cost"], rel=1e-3)

"""The continuous-batching request loop: results equal single solves bit for bit (alone
and in the mix), requests arriving during launches are admitted, memory admission, ticket
lifecycle. Through the C ABI."""
import time

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


def _controllers(M, count, seed=0):
    rng = np.random.default_rng(seed)
    quad, hum = S.quadruped(), S.humanoid()
    mods = {"q": M.Model(quad), "h": M.Model(hum)}
    out = []
    for i in range(count):
        is_q = rng.random() < 0.7
        rob = quad if is_q else hum
        K = int(rng.integers(40, 300))
        H = int(rng.integers(30, 80))
        nk = int(rng.integers(4, 9))
        kw = dict(iters=1, dt=0.005, seed=50 + i, instance=i)
        args = (mods["q" if is_q else "h"], K, H, nk, float(rng.uniform(0.05, 0.5)), S.linear_sigma(nk))
        x0 = S.standing_state(rob, jitter=0.02, seed=300 + i)
        out.append((args, kw, x0))
    return out


def test_served_results_equal_single_solves(M):
    specs = _controllers(M, 24)
    alone = [M.Controller(*a, **kw) for a, kw, _ in specs]
    served = [M.Controller(*a, **kw) for a, kw, _ in specs]
    srv = M.Server(mem_budget_bytes=8 << 30, max_inflight=3)
    for rnd in range(3):          # three control steps: resident warm starts carry over
        ref = [c.solve(x) for c, (_, _, x) in zip(alone, specs)]
        tickets = []
        for i, (c, (_, _, x)) in enumerate(zip(served, specs)):
            tickets.append(srv.submit(c, x))
            if i % 5 == 4:
                time.sleep(0.0005)    # later requests arrive while earlier launches run
        for i, t in enumerate(tickets):
            st, mean, best, info = srv.poll(t, served[i])
            assert st == 0
            np.testing.assert_array_equal(mean, ref[i][0], err_msg=f"round {rnd} controller {i}")
            np.testing.assert_array_equal(best, ref[i][1], err_msg=f"round {rnd} controller {i}")
            assert info["best_cost"] == ref[i][2]["best_cost"]
    stats = srv.stats()
    assert stats["submitted"] == stats["completed"] == 72
    assert stats["launches"] >= 3
    srv.close()


def test_memory_admission_and_tickets(M):
    specs = _controllers(M, 6, seed=1)
    ctrls = [M.Controller(*a, **kw) for a, kw, _ in specs]
    biggest = max(c.device_bytes for c in ctrls)
    # budget for one context at a time: every request still completes, admissions wait
    srv = M.Server(mem_budget_bytes=biggest, max_inflight=4)
    tickets = [srv.submit(c, x) for c, (_, _, x) in zip(ctrls, specs)]
    seen = set()
    while len(seen) < len(tickets):
        nc = srv.next_completed(timeout_us=2_000_000)
        assert nc is not None
        t, t_sub, t_done = nc
        assert t_done >= t_sub > 0
        seen.add(t)
    for c, t in zip(ctrls, tickets):
        st, *_ = srv.poll(t, c, timeout_us=0)
        assert st == 0
    with pytest.raises(M.MppiError) as e:
        srv.poll(tickets[0], ctrls[0])
    assert e.value.status == M.MPPI_ERR_NOT_FOUND
    stats = srv.stats()
    assert stats["peak_bytes"] <= biggest
    assert stats["launches"] >= 2 and stats["deferred"] >= 1
    srv.close()
    # a request larger than the whole budget is refused at submit time
    small = M.Server(mem_budget_bytes=1024, max_inflight=1)
    with pytest.raises(M.MppiError) as e:
        small.submit(ctrls[0], specs[0][2])
    assert e.value.status == M.MPPI_ERR_ADMISSION
    x = specs[0][2].copy()
    x[3] = np.nan
    with pytest.raises(M.MppiError) as e:
        M.Server().submit(ctrls[0], x)
    assert e.value.status == M.MPPI_ERR_NONFINITE_STATE
    small.close()


def test_pending_then_done(M):
    specs = _controllers(M, 1, seed=2)
    c = M.Controller(*specs[0][0], **specs[0][1])
    srv = M.Server()
    t = srv.submit(c, specs[0][2])
    r = srv.poll(t, c, timeout_us=0)      # may or may not be done yet; never blocks
    if r is None:
        r = srv.poll(t, c, timeout_us=-1)
    assert r[0] == 0
    srv.close()

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


def _slot_bytes(budget, max_inflight):
    """The documented launch-slot size: min(4 MiB, floor(budget / (4 max_inflight))) rounded
    down to 256 B."""
    return min(4 << 20, (budget // (4 * max_inflight)) & ~255)


def test_memory_admission_and_tickets(M):
    specs = _controllers(M, 6, seed=1)
    # one large context (1024 humanoid samples, 8 knots: > 1 MB) second in line, so it
    # arrives while the first request is admitted and must wait for its memory
    hum = S.humanoid()
    big = ((M.Model(hum), 1024, 30, 8, 0.2, S.linear_sigma(8)), dict(iters=1, dt=0.005, seed=77, instance=77),
           S.standing_state(hum, jitter=0.02, seed=77))
    specs.insert(1, big)
    ctrls = [M.Controller(*a, **kw) for a, kw, _ in specs]
    biggest = max(c.device_bytes for c in ctrls)
    assert biggest == ctrls[1].device_bytes > (1 << 20)
    smallest = min(c.device_bytes for c in ctrls)
    # a budget whose part left after the launch slots' reservation holds one context at a
    # time: every request still completes, admissions wait
    budget = (4 * biggest) // 3 + 4096
    while budget - 4 * _slot_bytes(budget, 4) < biggest:
        budget += 4096
    srv = M.Server(mem_budget_bytes=budget, max_inflight=4)
    st0 = srv.stats()
    assert st0["slot_bytes"] == _slot_bytes(budget, 4)
    assert st0["reserved_bytes"] == 4 * st0["slot_bytes"] <= budget // 4
    assert budget - st0["reserved_bytes"] < biggest + smallest
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
    # the peak charged to the budget: the slots' reservation plus the admitted contexts
    assert stats["reserved_bytes"] + biggest <= stats["peak_bytes"] <= budget
    assert stats["launches"] >= 2 and stats["deferred"] >= 1
    srv.close()
    # a request larger than the budget left after the reservation is refused at submit time
    small = M.Server(mem_budget_bytes=4 * 4 * (16 << 10), max_inflight=4)
    assert ctrls[1].device_bytes > small.stats()["slot_bytes"] * 12
    with pytest.raises(M.MppiError) as e:
        small.submit(ctrls[1], specs[1][2])
    assert e.value.status == M.MPPI_ERR_ADMISSION
    small.close()
    # a budget too small for the launch slots is refused at creation
    with pytest.raises(M.MppiError) as e:
        M.Server(mem_budget_bytes=4 * 4 * (16 << 10) - 4096, max_inflight=4)
    assert e.value.status == M.MPPI_ERR_INVALID_ARG
    x = specs[0][2].copy()
    x[3] = np.nan
    with pytest.raises(M.MppiError) as e:
        M.Server().submit(ctrls[0], x)
    assert e.value.status == M.MPPI_ERR_NONFINITE_STATE


def test_server_device_memory_is_the_reservation(M):
    # The device memory a server adds is its slots' reservation, taken at creation; serving
    # requests (many admissions, batches of every size) allocates nothing more.
    import torch
    specs = _controllers(M, 24, seed=3)
    ctrls = [M.Controller(*a, **kw) for a, kw, _ in specs]
    warm = M.Server(mem_budget_bytes=1 << 30, max_inflight=3)   # loads every kernel once
    for c, (_, _, x) in zip(ctrls, specs):
        warm.poll(warm.submit(c, x), c)
    warm.close()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    srv = M.Server(mem_budget_bytes=1 << 30, max_inflight=3)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    reserved = srv.stats()["reserved_bytes"]
    assert reserved == 3 * (4 << 20)
    slack = 4 << 20    # allocation granularity of the driver (2 MiB pages), stream bookkeeping
    assert abs((free0 - free1) - reserved) <= slack, (free0 - free1, reserved)
    lowest = free1
    for rnd in range(3):
        tickets = [srv.submit(c, x) for c, (_, _, x) in zip(ctrls, specs)]
        for t, c in zip(tickets, ctrls):
            assert srv.poll(t, c)[0] == 0
            lowest = min(lowest, torch.cuda.mem_get_info()[0])
    assert free1 - lowest <= slack, (free1 - lowest)
    stats = srv.stats()
    assert stats["peak_bytes"] <= (1 << 30)
    srv.close()


def test_deadline_sheds_requests_waiting_too_long(M):
    # One launch slot and two requests per controller (400-step horizons, so a launch
    # lasts well over a millisecond): a controller's second request cannot share a launch
    # with its first and waits for it, far longer than the 0.2 ms deadline set once all
    # are queued, so it is shed (MPPI_ERR_DEADLINE, nothing run). Every result that does
    # run equals the same controller's plain solves in order: a shed request changes
    # nothing in its context (warm start, noise counter).
    specs = []
    for a, kw, x in _controllers(M, 8, seed=4):
        specs.append(((a[0], a[1], 400) + tuple(a[3:]), kw, x))
    make = lambda i: M.Controller(*specs[i][0], **specs[i][1])
    served = [make(i) for i in range(len(specs))]
    srv = M.Server(mem_budget_bytes=1 << 30, max_inflight=1)
    tickets = [(i, srv.submit(served[i], specs[i][2])) for _ in range(2) for i in range(len(specs))]
    srv.set_deadline(200)     # 0.2 ms
    outcome = {i: [] for i in range(len(specs))}
    for i, t in tickets:
        st, mean, best, info = srv.poll(t, served[i])
        assert st in (0, M.MPPI_ERR_DEADLINE)
        outcome[i].append((st, mean))
    n_shed = sum(st != 0 for v in outcome.values() for st, _ in v)
    n_ran = sum(st == 0 for v in outcome.values() for st, _ in v)
    assert n_shed >= 1 and n_ran >= 1 and srv.stats()["shed"] == n_shed
    srv.set_deadline(0)
    for i in range(len(specs)):
        fresh = make(i)
        ran = [mean for st, mean in outcome[i] if st == 0]
        # one more served solve with shedding off: the sequence of results that ran equals
        # a fresh controller's sequence of plain solves
        st, mean, _, _ = srv.poll(srv.submit(served[i], specs[i][2]), served[i])
        assert st == 0
        ran.append(mean)
        for k, got in enumerate(ran):
            ref, _, _ = fresh.solve(specs[i][2])
            np.testing.assert_array_equal(got, ref, err_msg=f"controller {i}, solve {k}")
    with pytest.raises(M.MppiError):
        srv.set_deadline(-1)
    srv.close()


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


def test_served_results_match_oracle_at_serving_sizes(M, orc):
    # The serving workload's shapes (K log-uniform 256..2048, H 100..200, 4..8 knots, a
    # 70 / 30 quadruped / humanoid mix, 1 iteration, dt 0.005): a dozen controllers
    # submitted together, so their launches overlap on the device. Each served result
    # must equal the same controller's plain solve bit for bit (alone vs in the mix) and
    # the FP64 oracle's solve (Alg. 1) within 1e-3 on the updated control points.
    rng = np.random.default_rng(11)
    quad, hum = S.quadruped(), S.humanoid()
    mods = {"quadruped": M.Model(quad), "humanoid": M.Model(hum)}
    specs = []
    for i in range(12):
        rob = quad if rng.random() < 0.7 else hum
        K = int(np.floor(np.exp(rng.uniform(np.log(256), np.log(2048)))))
        H = int(rng.integers(100, 201))
        nk = int(rng.integers(4, 9))
        lam = float(rng.uniform(0.05, 0.5))
        x0 = S.standing_state(rob, jitter=0.02, seed=900 + i)
        specs.append((rob, K, H, nk, lam, x0, i))
    assert {s[0].name for s in specs} == {"quadruped", "humanoid"}
    make = lambda s: M.Controller(mods[s[0].name], s[1], s[2], s[3], s[4], S.linear_sigma(s[3]), dt=0.005,
                                  seed=4000 + s[6], instance=s[6])
    served = [make(s) for s in specs]
    alone = [make(s) for s in specs]
    srv = M.Server(mem_budget_bytes=8 << 30, max_inflight=4)
    tickets = [srv.submit(c, s[5]) for c, s in zip(served, specs)]
    results = [srv.poll(t, c) for t, c in zip(tickets, served)]
    srv.close()
    worst = 0.0
    for (rob, K, H, nk, lam, x0, i), c, (st, mean, best, info) in zip(specs, alone, results):
        assert st == 0
        ref_mean, ref_best, ref_info = c.solve(x0)
        np.testing.assert_array_equal(mean, ref_mean, err_msg=f"controller {i}")
        np.testing.assert_array_equal(best, ref_best, err_msg=f"controller {i}")
        nom = S.nominal_knots(rob, nk).astype(np.float32).astype(np.float64)
        ref = orc.solve(rob, K, nk, H, 1, 0.005, lam, S.linear_sigma(nk), x0, nom, seed=4000 + i, inst=i)
        err = float(np.max(np.abs(mean - ref["mean"]) / np.maximum(1.0, np.abs(ref["mean"]))))
        worst = max(worst, err)
        assert err <= 1e-3, f"controller {i} ({rob.name}, K {K}, H {H}, {nk} knots): {err:.2e}"
        assert info["best_cost"] == pytest.approx(ref["best_cost"], rel=1e-3)
    print(f"served vs oracle at serving sizes: worst control-point error {worst:.2e}")

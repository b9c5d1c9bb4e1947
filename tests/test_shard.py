"""The sample-shard merge of one iteration (Sec. III-C weights and the Eq. update-nominal
average over samples split into shards) on CPU: the library's host merges against the
FP64 oracle's unsharded weights and average, and the two-round exchange of
`paper_2511_19204_gb300.shard` on 2 and 4 gloo ranks. Each rank's local range and moments
are formed here from their definitions (the device versions are checked in
test_gpu_shard.py)."""
import itertools
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _local_range(M, costs, base):
    fin = np.isfinite(costs)
    if not fin.any():
        return M.shard_range()
    c = np.where(fin, costs, np.inf)
    i = int(np.argmin(c))   # the first smallest
    return M.shard_range(float(c[i]), float(costs[fin].max()), base + i, int(fin.sum()))


def _local_moments(costs, knots, g, lam, normalize):
    # Eq. softmax_minmax (normalize 0) or Eq. omega-weights (1) before the division by
    # the total, with the merged range
    span = g.s_max - g.s_min
    k = (1.0 / (span * lam) if span > 0 else 0.0) if normalize == 0 else 1.0 / lam
    c = costs.astype(np.float64)
    w = np.where(np.isfinite(c), np.exp(-(np.where(np.isfinite(c), c, 0.0) - g.s_min) * k), 0.0)
    return np.concatenate([[w.sum()], w @ knots.reshape(len(costs), -1).astype(np.float64)])


def _problem(orc, n=256, H=20):
    from paper_2511_19204_gb300 import synth as S
    p = S.scale_quadruped(n=n)
    p.horizon = H
    kn = orc.sample_knots(p.model.nj, p.nk, p.n, p.horizon, p.dt, p.nominal, p.sigma[0], seed=p.seed)
    costs = orc.rollout_batch(p.model, p.state, kn, p.horizon, p.dt).astype(np.float32)
    return kn.astype(np.float32).reshape(p.n, -1), costs, p.lam


def _reference(orc, knots, costs, lam, normalize):
    st, w, info = orc.weights(costs.astype(np.float64), lam, normalize)
    return st, orc.average(knots.astype(np.float64), w).reshape(-1), info


def test_range_merge_matches_the_oracle_in_any_order(orc):
    from paper_2511_19204_gb300 import mppi as M
    rng = np.random.default_rng(3)
    for trial in range(20):
        N = int(rng.integers(8, 300))
        costs = rng.normal(size=N).astype(np.float32)
        costs[rng.random(N) < 0.1] = np.nan
        costs[rng.random(N) < 0.05] = np.inf
        if trial % 3 == 0:   # a tie for the minimum, across shards
            i, j = sorted(rng.choice(N, 2, replace=False))
            costs[i] = costs[j] = np.float32(np.nanmin(np.where(np.isfinite(costs), costs, np.nan)) - 1.0)
        cuts = sorted(rng.choice(np.arange(1, N), size=int(rng.integers(1, 6)), replace=False))
        bounds = [0, *cuts, N]
        parts = [_local_range(M, costs[a:b], a) for a, b in zip(bounds[:-1], bounds[1:])]
        parts.append(M.shard_range())   # an empty shard changes nothing
        st, w, info = orc.weights(costs.astype(np.float64), 0.1, 0)
        for order in itertools.islice(itertools.permutations(range(len(parts))), 24):
            r = M.shard_range()
            for k in order:
                r = M.shard_range_merge(r, parts[k])
            assert r.n_finite == info["n_finite"]
            assert r.s_min == info["smin"] and r.s_max == info["smax"]
            assert r.best_index == info["best"]
        # a balanced tree gives the same range as a left fold (associativity)
        while len(parts) > 1:
            parts = [M.shard_range_merge(parts[i], parts[i + 1]) if i + 1 < len(parts) else parts[i]
                     for i in range(0, len(parts), 2)]
        assert parts[0].as_tuple() == r.as_tuple()


def test_all_non_finite_shards_merge_to_the_empty_range():
    from paper_2511_19204_gb300 import mppi as M
    a = _local_range(M, np.array([np.nan, np.inf], np.float32), 0)
    b = _local_range(M, np.array([-np.inf], np.float32), 2)
    r = M.shard_range_merge(a, b)
    assert r.n_finite == 0 and r.best_index == -1 and r.s_min == np.inf and r.s_max == -np.inf


@pytest.mark.parametrize("normalize", [0, 1])
def test_host_merge_of_moments_matches_the_unsharded_oracle(orc, normalize):
    from paper_2511_19204_gb300 import mppi as M
    knots, costs, lam = _problem(orc)
    st, ref, info = _reference(orc, knots, costs, lam, normalize)
    bounds = [0, 31, 32, 200, 256]
    rs = [_local_range(M, costs[a:b], a) for a, b in zip(bounds[:-1], bounds[1:])]
    g = M.shard_range()
    for r in rs:
        g = M.shard_range_merge(g, r)
    assert g.best_index == info["best"]
    m = None
    for a, b in zip(bounds[:-1], bounds[1:]):
        part = _local_moments(costs[a:b], knots[a:b], g, lam, normalize)
        m = part if m is None else M.shard_moments_merge(m, part)
    np.testing.assert_allclose(m[1:] / m[0], ref, rtol=1e-12, atol=1e-14)
    mean = M.shard_mean(m)
    np.testing.assert_allclose(mean, ref, rtol=2.0 ** -23, atol=1e-30)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, bounds, knots, costs, lam, normalize, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2511_19204_gb300 import mppi as M
    from paper_2511_19204_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    a, b = bounds[rank], bounds[rank + 1]
    c, k = costs[a:b], knots[a:b]
    st, mean, g, best = shard.sharded_update(lambda: _local_range(M, c, a),
                                             lambda gr: _local_moments(c, k, gr, lam, normalize),
                                             lambda n: k[n], a, b - a, k.shape[1])
    q.put((rank, st, None if mean is None else mean.tobytes(), g.as_tuple(), None if best is None else best.tobytes()))
    dist.destroy_process_group()


def _run_ranks(bounds, knots, costs, lam, normalize):
    world = len(bounds) - 1
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, bounds, knots, costs, lam, normalize, q))
             for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    return sorted(out)


@pytest.mark.parametrize("bounds,normalize", [([0, 128, 256], 0), ([0, 50, 150, 156, 256], 0), ([0, 50, 150, 156, 256], 1)])
def test_sharded_update_on_gloo_ranks(orc, bounds, normalize):
    knots, costs, lam = _problem(orc)
    if len(bounds) > 3:
        costs[150:156] = np.nan                      # one rank without a finite cost
        lo = np.float32(np.nanmin(costs) - 0.5)
        costs[60] = costs[200] = lo                  # a tie across ranks: the lower index wins
    st, ref, info = _reference(orc, knots, costs, lam, normalize)
    out = _run_ranks(bounds, knots, costs, lam, normalize)
    means = [np.frombuffer(o[2], np.float32) for o in out]
    bests = [np.frombuffer(o[4], np.float32) for o in out]
    for (rank, st, _, g, _), mean, best in zip(out, means, bests):
        assert st == 0
        assert g[2] == info["best"] and g[3] == info["n_finite"]
        np.testing.assert_array_equal(mean, means[0])       # identical bits on every rank
        np.testing.assert_allclose(mean, ref, rtol=2.0 ** -23, atol=1e-30)
        np.testing.assert_array_equal(best, knots[info["best"]])
    if len(bounds) > 3:
        assert info["best"] == 60


def test_sharded_update_without_finite_costs_leaves_the_nominal():
    knots = np.ones((8, 4), np.float32)
    costs = np.full(8, np.nan, np.float32)
    out = _run_ranks([0, 4, 8], knots, costs, 0.1, 0)
    from paper_2511_19204_gb300 import mppi as M
    for rank, st, mean, g, best in out:
        assert st == M.MPPI_ERR_ALL_COSTS_NONFINITE and mean is None and best is None

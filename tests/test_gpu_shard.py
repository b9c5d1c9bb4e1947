"""The device side of the sample-shard entry points on one GPU: a full-size iteration's
costs and knots (K = 8192, E = 144) cut into uneven shards, each scanned and summed by
mppi_shard_range_local / mppi_shard_moments on its own slice of device memory, merged by
the host merges, against the FP64 oracle's unsharded weights and average (Sec. III-C)
and the library's own single-instance weights and average."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_2511_19204_gb300 import build, mppi
    build.build()
    mppi.load()
    return mppi


def _case(K=8192, E=144, seed=17):
    rng = np.random.default_rng(seed)
    costs = (50.0 + 10.0 * rng.standard_normal(K)).astype(np.float32)
    costs[rng.random(K) < 0.02] = np.nan
    costs[rng.random(K) < 0.01] = np.inf
    lo = np.float32(np.nanmin(np.where(np.isfinite(costs), costs, np.nan)) - 1.0)
    i1, i2 = (4500, 7000) if K > 7000 else (K // 3, 2 * K // 3)
    costs[i1] = costs[i2] = lo            # the global minimum twice, in different shards
    knots = rng.normal(size=(K, E)).astype(np.float32)
    return knots, costs


def _sharded(M, torch, knots, costs, bounds, lam, normalize, stream=None):
    d_k = torch.tensor(knots, device="cuda")
    d_c = torch.tensor(costs, device="cuda")
    K, E = knots.shape
    ranges = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        ranges.append(M.shard_range_local(d_c.data_ptr() + 4 * a, b - a, a, stream))
    g = M.shard_range()
    for r in ranges:
        g = M.shard_range_merge(g, r)
    m = None
    for a, b in zip(bounds[:-1], bounds[1:]):
        part = M.shard_moments(d_k.data_ptr() + 4 * a * E, d_c.data_ptr() + 4 * a, b - a, E, g, lam, normalize, stream)
        m = part if m is None else M.shard_moments_merge(m, part)
    return ranges, g, m


@pytest.mark.parametrize("normalize", [0, 1])
def test_sharded_iteration_matches_oracle_and_single_instance(M, orc, normalize):
    torch = pytest.importorskip("torch")
    knots, costs = _case()
    lam = 0.1 if normalize == 0 else 5.0
    bounds = [0, 1, 3000, 4600, 8191, 8192]      # a 1-sample shard, uneven and odd-aligned slices
    ranges, g, m = _sharded(M, torch, knots, costs, bounds, lam, normalize)
    st, w, info = orc.weights(costs.astype(np.float64), lam, normalize)
    ref = orc.average(knots.astype(np.float64), w).reshape(-1)
    assert (g.s_min, g.s_max, g.best_index, g.n_finite) == (info["smin"], info["smax"], info["best"], info["n_finite"])
    assert g.best_index == 4500
    # each shard's scan against its own slice
    for (a, b), r in zip(zip(bounds[:-1], bounds[1:]), ranges):
        _, _, li = orc.weights(costs[a:b].astype(np.float64), lam, normalize)
        assert r.n_finite == li["n_finite"]
        if li["n_finite"]:
            assert r.best_index == a + li["best"] and r.s_min == li["smin"] and r.s_max == li["smax"]
    np.testing.assert_allclose(m[1:] / m[0], ref, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(M.shard_mean(m), ref, rtol=2.0 ** -23, atol=1e-30)
    # the library's single-instance weights and average of the same iteration
    st2, w2, _ = M.weights(costs, lam, normalize)
    np.testing.assert_allclose(m[1:] / m[0], M.average(knots, w2).reshape(-1), rtol=1e-12, atol=1e-14)


def test_uniform_weights_all_non_finite_and_bad_input(M):
    torch = pytest.importorskip("torch")
    knots = np.arange(24, dtype=np.float32).reshape(6, 4)
    costs = np.full(6, 3.0, np.float32)            # S_max = S_min: uniform weights
    ranges, g, m = _sharded(M, torch, knots, costs, [0, 2, 6], 0.1, 0)
    assert g.best_index == 0 and g.n_finite == 6
    np.testing.assert_allclose(M.shard_mean(m), knots.mean(axis=0), rtol=1e-7)
    d_k = torch.tensor(knots, device="cuda")
    d_c = torch.full((6,), float("nan"), device="cuda")
    r = M.shard_range_local(d_c.data_ptr(), 6, 0)
    assert r.n_finite == 0 and r.best_index == -1
    L = M.load()
    out = np.zeros(5)
    import ctypes as C
    st = L.mppi_shard_moments(6, 4, C.c_void_p(d_k.data_ptr()), C.c_void_p(d_c.data_ptr()), C.byref(r), 0.1, 0,
                              out.ctypes.data_as(C.POINTER(C.c_double)), None)
    assert st == M.MPPI_ERR_ALL_COSTS_NONFINITE
    bad = M.shard_range(0.1, 1.0, 0, 6)            # 0.1 is not an FP32 value
    st = L.mppi_shard_moments(6, 4, C.c_void_p(d_k.data_ptr()), C.c_void_p(d_c.data_ptr()), C.byref(bad), 0.1, 0,
                              out.ctypes.data_as(C.POINTER(C.c_double)), None)
    assert st == M.MPPI_ERR_INVALID_ARG
    assert L.mppi_shard_range_local(0, C.c_void_p(d_c.data_ptr()), 0, C.byref(r), None) == M.MPPI_ERR_INVALID_ARG


def test_shards_on_a_caller_stream(M, orc):
    torch = pytest.importorskip("torch")
    knots, costs = _case(K=3000, E=96, seed=5)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    ranges, g, m = _sharded(M, torch, knots, costs, [0, 1500, 3000], 0.2, 0, stream=s.cuda_stream)
    st, w, info = orc.weights(costs.astype(np.float64), 0.2, 0)
    np.testing.assert_allclose(m[1:] / m[0], orc.average(knots.astype(np.float64), w).reshape(-1), rtol=1e-12, atol=1e-14)


def _gpu_rank(rank, world, port, bounds, knots, costs, lam, q):
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    from paper_2511_19204_gb300 import mppi as M
    from paper_2511_19204_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    a, b = bounds[rank], bounds[rank + 1]
    K, E = b - a, knots.shape[1]
    d_k = torch.tensor(knots[a:b], device="cuda")
    d_c = torch.tensor(costs[a:b], device="cuda")
    st, mean, g, best = shard.sharded_update(lambda: M.shard_range_local(d_c.data_ptr(), K, a),
                                             lambda gr: M.shard_moments(d_k.data_ptr(), d_c.data_ptr(), K, E, gr, lam),
                                             lambda n: knots[a + n], a, K, E)
    q.put((rank, st, mean.tobytes(), g.as_tuple(), best.tobytes()))
    dist.destroy_process_group()


def test_sharded_update_through_the_device_on_two_ranks(M, orc):
    # The whole sharded iteration as two processes would run it on two GPUs: each rank's
    # range and moments by the device entry points (both ranks on this one GPU; nothing on
    # the device waits for the other rank), the two exchanges over gloo, against the FP64
    # oracle's unsharded weights and average.
    import socket
    import torch.multiprocessing as mp
    knots, costs = _case(K=8192, E=144, seed=23)
    lam = 0.1
    bounds = [0, 5000, 8192]
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_gpu_rank, args=(r, 2, port, bounds, knots, costs, lam, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    st, w, info = orc.weights(costs.astype(np.float64), lam, 0)
    ref = orc.average(knots.astype(np.float64), w).reshape(-1)
    means = [np.frombuffer(o[2], np.float32) for o in out]
    for (rank, st, _, g, best), mean in zip(out, means):
        assert st == 0 and g[2] == info["best"] == 4500
        np.testing.assert_array_equal(mean, means[0])
        np.testing.assert_allclose(mean, ref, rtol=2.0 ** -23, atol=1e-30)
        np.testing.assert_array_equal(np.frombuffer(best, np.float32), knots[info["best"]])

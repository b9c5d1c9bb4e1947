"""mppi_average_noalloc: the allocation-free variant of the FP64 knot average, for
callers that cannot call cudaMalloc where they need the average (real-time loops that
must not block on the allocator, fixed pre-reserved footprints, hosts whose allocator
belongs to another framework). Its scratch is a fixed device array shared by all calls,
so it is checked against the FP64 oracle's average and against mppi_average on two calls
in a row (the second must not see the first's leftovers), at the exact size limit of the
scratch, and on a caller's own stream. Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(M, torch, kn, w, stream=None):
    """Run the entry point on device copies of kn [K][E] and w [K]; with a torch stream,
    the work goes on that stream and only that stream is synchronised before reading."""
    L = M.load()
    K, E = kn.shape
    d_k = torch.tensor(kn, dtype=torch.float32, device="cuda")
    d_w = torch.tensor(w, dtype=torch.float64, device="cuda")
    d_o = torch.full((E,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    handle = C.c_void_p(stream.cuda_stream) if stream is not None else None
    st = L.mppi_average_noalloc(K, E, C.c_void_p(d_k.data_ptr()), C.c_void_p(d_w.data_ptr()),
                                C.c_void_p(d_o.data_ptr()), handle)
    if stream is not None:
        # read back on the same stream, so nothing waits on the default stream
        host = torch.empty(E, dtype=torch.float64, pin_memory=True)
        with torch.cuda.stream(stream):
            host.copy_(d_o, non_blocking=True)
        stream.synchronize()
        out = host.numpy().copy()
    else:
        torch.cuda.synchronize()
        out = d_o.cpu().numpy()
    return st, out


def _case(rng, K, E):
    kn = rng.normal(size=(K, E)).astype(np.float32)
    w = rng.random(K)
    w /= w.sum()
    return kn, w


def test_noalloc_average_matches_oracle_and_allocating_entry_point(orc):
    torch = pytest.importorskip("torch")
    from paper_2511_19204_gb300 import build, mppi as M
    build.build()
    rng = np.random.default_rng(123)
    for K, E in ((8192, 144), (1000, 336)):      # two calls in a row, different shapes
        kn, w = _case(rng, K, E)
        st, got = _noalloc(M, torch, kn, w)
        assert st == M.MPPI_OK
        ref = orc.average(kn.astype(np.float64), w).reshape(-1)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(got, M.average(kn, w).reshape(-1), rtol=1e-12, atol=1e-14)


def test_noalloc_at_the_scratch_limit_and_on_a_caller_stream(orc):
    torch = pytest.importorskip("torch")
    from paper_2511_19204_gb300 import mppi as M
    rng = np.random.default_rng(7)
    # ceil(K / 64) * E == 1048576 exactly: the largest accepted request
    K, E = 64 * 1024, 1024
    kn, w = _case(rng, K, E)
    st, got = _noalloc(M, torch, kn, w)
    assert st == M.MPPI_OK
    ref = orc.average(kn.astype(np.float64), w).reshape(-1)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14)
    # the stream argument is honoured: work on a side stream, only that stream synchronised
    s = torch.cuda.Stream()
    kn2, w2 = _case(rng, 3000, 144)
    st, got = _noalloc(M, torch, kn2, w2, stream=s)
    assert st == M.MPPI_OK
    np.testing.assert_allclose(got, orc.average(kn2.astype(np.float64), w2).reshape(-1), rtol=1e-12, atol=1e-14)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    from paper_2511_19204_gb300 import mppi as M
    L = M.load()
    d = torch.zeros(4, device="cuda")
    p = C.c_void_p(d.data_ptr())
    # ceil(K / 64) * E > 2^20 doubles: one chunk past the limit
    assert L.mppi_average_noalloc(64 * 1024 + 1, 1024, p, p, p, None) == M.MPPI_ERR_INVALID_ARG
    assert b"scratch" in L.mppi_last_error(None)
    assert L.mppi_average_noalloc(0, 8, p, p, p, None) == M.MPPI_ERR_INVALID_ARG

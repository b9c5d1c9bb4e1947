"""mppi_average_noalloc: the allocation-free variant of the FP64 knot average, for
callers that cannot call cudaMalloc where they need the average (real-time loops that
must not block on the allocator, fixed pre-reserved footprints, hosts whose allocator
belongs to another framework). Its scratch is a fixed device array shared by all calls,
so it is checked against mppi_average on two calls in a row: the second must not see
the first's leftovers. Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(M, torch, kn, w, stream=None):
    L = M.load()
    K, E = kn.shape
    d_k = torch.tensor(kn, dtype=torch.float32, device="cuda")
    d_w = torch.tensor(w, dtype=torch.float64, device="cuda")
    d_o = torch.full((E,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    st = L.mppi_average_noalloc(K, E, C.c_void_p(d_k.data_ptr()), C.c_void_p(d_w.data_ptr()),
                                C.c_void_p(d_o.data_ptr()), None)
    torch.cuda.synchronize()
    return st, d_o.cpu().numpy()


def test_noalloc_average_matches_allocating_entry_point():
    torch = pytest.importorskip("torch")
    from paper_2511_19204_gb300 import build, mppi as M
    build.build()
    rng = np.random.default_rng(123)
    for K, E in ((8192, 144), (1000, 336)):      # two calls in a row, different shapes
        kn = rng.normal(size=(K, E)).astype(np.float32)
        w = rng.random(K)
        w /= w.sum()
        st, got = _noalloc(M, torch, kn, w)
        assert st == M.MPPI_OK
        ref = M.average(kn, w).reshape(-1)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    from paper_2511_19204_gb300 import mppi as M
    L = M.load()
    d = torch.zeros(4, device="cuda")
    p = C.c_void_p(d.data_ptr())
    # ceil(K / 64) * E > 2^20 doubles
    assert L.mppi_average_noalloc(64 * 1025, 1024, p, p, p, None) == M.MPPI_ERR_INVALID_ARG
    assert b"scratch" in L.mppi_last_error(None)
    assert L.mppi_average_noalloc(0, 8, p, p, p, None) == M.MPPI_ERR_INVALID_ARG

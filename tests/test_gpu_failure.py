"""Failure detection on the GPU without a fault: the persistent kernel's bounded queue wait
gives up on an item nobody publishes and reports MPPI_ERR_TIMEOUT; the device stays
usable for ordinary solves afterwards."""
import ctypes as C
import time

import numpy as np
import pytest

from paper_2511_19204_gb300 import synth as S

pytestmark = pytest.mark.gpu


def test_queue_wait_times_out_and_device_recovers(orc):
    from paper_2511_19204_gb300 import build, mppi as M
    build.build()
    L = M.load()
    bits = C.c_int32(0)
    t0 = time.perf_counter()
    st = L.mppi_selftest_queue_timeout(200_000, C.byref(bits))   # 0.2 s budget
    el = time.perf_counter() - t0
    assert st == M.MPPI_ERR_TIMEOUT
    assert bits.value & 2
    assert 0.15 < el < 10.0
    # the context is intact: an ordinary solve still matches the oracle
    p = S.scale_quadruped(n=128)
    p.horizon = 60
    c = M.Controller.from_problem(M.Model(p.model), p)
    mean, _, info = c.solve(p.state, warm=p.nominal.astype(np.float32))
    ref = orc.solve(p.model, p.n, p.nk, p.horizon, p.iters, p.dt, p.lam, p.sigma, p.state,
                    p.nominal.astype(np.float32).astype(np.float64), seed=p.seed)
    assert info["status"] == 0
    assert np.max(np.abs(mean - ref["mean"]) / np.maximum(1.0, np.abs(ref["mean"]))) < 1e-3


def test_selftest_rejects_bad_budget():
    from paper_2511_19204_gb300 import mppi as M
    L = M.load()
    assert L.mppi_selftest_queue_timeout(0, None) == M.MPPI_ERR_INVALID_ARG

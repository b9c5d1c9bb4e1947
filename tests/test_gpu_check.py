"""The bounds-check build (-DMPPI_CHECK): device-side index checks on the noise, segment,
split-record, persistent-queue, chunk-sum and best-sample accesses, each of which records
a bit in a check word and skips or clamps the access instead of trapping. Small cases of
every kernel family run against that build in a child process (MPPI_LIBRARY): their
results must match the oracle and the product's bit-exact relations, and no check may
have fired."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounds_check_build_small_cases():
    from paper_2511_19204_gb300 import build, mppi
    lib = build.build(check=True)
    env = dict(os.environ, MPPI_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_check_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    print(out)
    assert out["library"] == os.path.basename(lib)
    assert out["check_word"] == 0
    for k in ("quadruped_solve", "quadruped_solve_warp", "humanoid_split_solve", "quadruped_solve_K4000",
              "quadruped_solve_K12000"):
        assert out[k] <= 1e-3, (k, out[k])
    assert out["quadruped_generic_rollout"] <= 1e-4
    assert out["batch_equal"] and out["served_equal"]
    # the product build has no checks
    import ctypes as C
    w = C.c_uint32(7)
    assert mppi.load().mppi_check_word(C.byref(w), 0) == mppi.MPPI_ERR_UNSUPPORTED and w.value == 0

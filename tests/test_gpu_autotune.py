"""The autotuner through the C ABI: it keeps a valid mapping, and its JSON cache file
round-trips (entries written by a tuning are read back by a later process, here
simulated by reloading an edited file)."""
import json

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


def _ctrl(M, model):
    # an unusual shape so that no other test has tuned it in this process
    return M.Controller(model, 200, 37, 5, 0.1, S.linear_sigma(5, 1), dt=0.005, seed=3)


def test_autotune_picks_a_valid_mapping_and_persists_it(M, tmp_path):
    path = tmp_path / "tune.json"
    M.autotune_cache_file(str(path))
    try:
        mod = M.Model(S.quadruped())
        c = _ctrl(M, mod)
        m, b, ms = c.autotune()
        assert m in (M.MPPI_MAP_WARP, M.MPPI_MAP_HALFWARP, M.MPPI_MAP_CHAIN) and b in (32, 64, 128, 256)
        assert c.info()["mapping"] == m and c.info()["block"] == b
        entries = json.loads(path.read_text())
        assert len(entries) >= 1
        e = [x for x in entries if x["K"] == 200 and x["H"] == 37 and x["knots"] == 5][0]
        assert (e["mapping"], e["block"]) == (m, b) and len(e["ms"]) == 16
        # a later process reads the file: edit the entry, reload, tune a new context
        e["mapping"], e["block"] = M.MPPI_MAP_WARP, 64
        path.write_text("[\n" + ",\n".join(json.dumps(x) for x in entries) + "\n]\n")
        M.autotune_cache_file(str(path))
        c2 = _ctrl(M, mod)
        m2, b2, _ = c2.autotune()
        assert (m2, b2) == (M.MPPI_MAP_WARP, 64)
        assert c2.info()["mapping"] == M.MPPI_MAP_WARP and c2.info()["block"] == 64
        # the tuned context still solves
        p = S.scale_quadruped(n=200)
        mean, best, info = c2.solve(p.state, warm=S.nominal_knots(p.model, 5).astype(np.float32))
        assert info["status"] == 0
    finally:
        M.autotune_cache_file(None)

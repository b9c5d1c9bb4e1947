"""The C-ABI library builds, loads and exports every entry point include/mppi.h declares;
host-side argument validation (no GPU needed: it fails before any CUDA call)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mppi.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mppi_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_19204_gb300 import build, mppi
    build.build()
    return mppi.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["mppi_model_create", "mppi_create", "mppi_solve", "mppi_submit", "mppi_poll",
              "mppi_rollout_explicit", "mppi_solve_batch", "mppi_autotune"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2511_19204_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (mppi_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(lib, n)


def test_binding_covers_every_symbol():
    from paper_2511_19204_gb300 import mppi
    bound = {s[0] for s in mppi.SIGNATURES}
    assert set(_declared()) <= bound


def test_status_strings(lib):
    assert lib.mppi_status_str(0) == b"ok"
    assert lib.mppi_status_str(-3) == b"no finite cost in an iteration"
    assert lib.mppi_status_str(12345) == b"unknown status"


def _desc(m, **over):
    from paper_2511_19204_gb300 import mppi
    k = dict(parent=np.ascontiguousarray(m.parent, dtype=np.int32), axis=np.ascontiguousarray(m.axis),
             jpos=np.ascontiguousarray(m.jpos), mass=np.ascontiguousarray(m.mass),
             com=np.ascontiguousarray(m.com), inertia=np.ascontiguousarray(m.inertia),
             armature=np.ascontiguousarray(m.armature), q_min=np.ascontiguousarray(m.q_min),
             q_max=np.ascontiguousarray(m.q_max), kp=np.ascontiguousarray(m.kp), kd=np.ascontiguousarray(m.kd),
             tau_max=np.ascontiguousarray(m.tau_max), contact_body=np.ascontiguousarray(m.contact_body, dtype=np.int32),
             contact_pos=np.ascontiguousarray(m.contact_pos))
    k.update(over)
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    d = mppi.mppi_model_desc(nb=int(k.get("nb", m.nb)), nc=int(k.get("nc", m.nc)), fixed_base=0,
                             cost_body=int(k.get("cost_body", 0)),
                             parent=k["parent"].ctypes.data_as(ip), axis=k["axis"].ctypes.data_as(dp),
                             jpos=k["jpos"].ctypes.data_as(dp), mass=k["mass"].ctypes.data_as(dp),
                             com=k["com"].ctypes.data_as(dp), inertia=k["inertia"].ctypes.data_as(dp),
                             armature=k["armature"].ctypes.data_as(dp), q_min=k["q_min"].ctypes.data_as(dp),
                             q_max=k["q_max"].ctypes.data_as(dp), kp=k["kp"].ctypes.data_as(dp),
                             kd=k["kd"].ctypes.data_as(dp), tau_max=k["tau_max"].ctypes.data_as(dp),
                             contact_body=k["contact_body"].ctypes.data_as(ip),
                             contact_pos=k["contact_pos"].ctypes.data_as(dp), q_init=None,
                             contact_k=1.0, contact_c=1.0, mu=0.5, eps_f=0.1, gravity=9.81)
    return d, k


@pytest.mark.parametrize("case", ["nb0", "nb_big", "bad_parent", "axis", "mass", "cost_body", "contact_body"])
def test_model_validation_rejects_before_cuda(lib, case):
    from paper_2511_19204_gb300 import synth
    m = synth.quadruped()
    over = {}
    if case == "nb0":
        over["nb"] = 0
    elif case == "nb_big":
        over["nb"] = 40
    elif case == "bad_parent":
        p = m.parent.copy()
        p[5] = 7
        over["parent"] = p
    elif case == "axis":
        a = m.axis.copy()
        a[3] *= 2.0
        over["axis"] = a
    elif case == "mass":
        mm = m.mass.copy()
        mm[2] = -1.0
        over["mass"] = mm
    elif case == "cost_body":
        over["cost_body"] = 13
    elif case == "contact_body":
        cb = m.contact_body.copy()
        cb[0] = 99
        over["contact_body"] = cb
    d, keep = _desc(m, **over)
    h = C.c_void_p()
    assert lib.mppi_model_create(C.byref(d), C.byref(h)) == -1
    assert not h.value
    assert len(lib.mppi_last_error(None)) > 0


def test_null_arguments(lib):
    assert lib.mppi_model_create(None, None) == -1
    assert lib.mppi_create(None, 1, 1, 2, 0.1, None, 1, None, None) == -1
    assert lib.mppi_solve(None, None, None, None, None, None) == -1
    assert lib.mppi_weights(0, None, 0.1, 0, None, None) == -1
    assert lib.mppi_average(0, 0, None, None, None) == -1
    assert lib.mppi_philox_words(0, None, None, None) == 0


def test_autotune_cache_file_format(lib, tmp_path):
    # host-side part of the autotune cache: a well-formed file loads, a malformed one is
    # refused, a missing one is accepted (created by the next tuning), NULL turns it off
    good = tmp_path / "tune.json"
    good.write_text('[\n{"device": "GPU X|152|10.3", "model": "00000000deadbeef", "K": 64, "H": 50, "knots": 4, '
                    '"mapping": 2, "block": 64, "ms": [' + ", ".join(["-1"] * 8 + ["0.5"] * 8) + ']}\n]\n')
    assert lib.mppi_autotune_cache_file(str(good).encode()) == 0
    bad = tmp_path / "bad.json"
    bad.write_text('[\n{"device": "GPU X", "model": "zz", "K": 1}\n]\n')
    assert lib.mppi_autotune_cache_file(str(bad).encode()) == -1
    assert lib.mppi_autotune_cache_file(str(tmp_path / "new.json").encode()) == 0
    assert lib.mppi_autotune_cache_file(None) == 0

"""ctypes binding of libmppi.so (include/mppi.h) with the C ABI's names.

Argument marshalling only: every step of the MPPI path runs in the library's CUDA
kernels. Loading fails loudly (``MppiError``) when the library is missing or no CUDA
device is present; there is no fallback.

Low-level functions mirror the C entry points one to one (``mppi_model_create``,
``mppi_create``, ``mppi_solve``, ...); ``Model`` and ``Controller`` wrap them for numpy /
torch callers.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# the library to load: MPPI_LIBRARY (e.g. the bounds-check build) or the in-tree build
LIB_PATH = os.environ.get("MPPI_LIBRARY") or os.path.join(_HERE, "libmppi.so")

MPPI_OK = 0
MPPI_PENDING = 1
MPPI_ERR_INVALID_ARG = -1
MPPI_ERR_NONFINITE_STATE = -2
MPPI_ERR_ALL_COSTS_NONFINITE = -3
MPPI_ERR_OUT_OF_MEMORY = -4
MPPI_ERR_ADMISSION = -5
MPPI_ERR_TIMEOUT = -6
MPPI_ERR_CUDA = -7
MPPI_ERR_UNSUPPORTED = -8
MPPI_ERR_NOT_FOUND = -9
MPPI_ERR_DEADLINE = -10

MPPI_MAP_AUTO = -1
MPPI_MAP_WARP = 0
MPPI_MAP_HALFWARP = 1
MPPI_MAP_CHAIN = 2
MPPI_MAP_THREAD = 3
MAPPING_NAMES = {MPPI_MAP_WARP: "warp-per-sample", MPPI_MAP_HALFWARP: "halfwarp-per-sample",
                 MPPI_MAP_CHAIN: "lanes-per-chain", MPPI_MAP_THREAD: "reserved"}
MPPI_NORM_MINMAX = 0
MPPI_NORM_RAW = 1
MPPI_WARM_BEST = 0
MPPI_WARM_MEAN = 1
MPPI_SPLINE_HERMITE = 0
MPPI_SPLINE_CUBIC = 1
MPPI_SPLINE_QUADRATIC = 2

_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int32)
_u32p = C.POINTER(C.c_uint32)
_u64p = C.POINTER(C.c_uint64)
_i64p = C.POINTER(C.c_int64)


class MppiError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"mppi status {status}: {msg}")
        self.status = status


class mppi_model_desc(C.Structure):
    _fields_ = [("nb", C.c_int32), ("nc", C.c_int32), ("fixed_base", C.c_int32), ("cost_body", C.c_int32),
                ("parent", _ip), ("axis", _dp), ("jpos", _dp), ("mass", _dp), ("com", _dp),
                ("inertia", _dp), ("armature", _dp), ("q_min", _dp), ("q_max", _dp), ("kp", _dp),
                ("kd", _dp), ("tau_max", _dp), ("contact_body", _ip), ("contact_pos", _dp),
                ("q_init", _dp),
                ("contact_k", C.c_double), ("contact_c", C.c_double), ("mu", C.c_double),
                ("eps_f", C.c_double), ("gravity", C.c_double), ("z_des", C.c_double),
                ("vx_des", C.c_double), ("w_z", C.c_double), ("w_vx", C.c_double),
                ("w_tilt", C.c_double), ("w_tau", C.c_double),
                ("w_h", C.c_double), ("w_orient", C.c_double), ("w_q", C.c_double),
                ("w_cvel", C.c_double), ("w_cforce", C.c_double), ("w_term", C.c_double),
                ("quat_des", C.c_double * 4), ("f0", C.c_double * 3), ("pdot_des", C.c_double * 3)]


class mppi_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("scale_q", C.c_double), ("scale_v", C.c_double),
                ("normalize", C.c_int32), ("warm_from", C.c_int32), ("seed", C.c_uint64),
                ("instance_id", C.c_uint32), ("mapping", C.c_int32), ("block_size", C.c_int32),
                ("spline", C.c_int32), ("stream", C.c_void_p)]


class mppi_result(C.Structure):
    _fields_ = [("cost_min", C.c_double), ("cost_max", C.c_double), ("best_cost", C.c_double),
                ("ess", C.c_double), ("lse", C.c_double), ("best_index", C.c_int32),
                ("best_iter", C.c_int32), ("n_finite", C.c_int32), ("status", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class mppi_shard_range(C.Structure):
    _fields_ = [("s_min", C.c_double), ("s_max", C.c_double), ("best_index", C.c_int64),
                ("n_finite", C.c_int64)]

    def as_tuple(self):
        return (self.s_min, self.s_max, self.best_index, self.n_finite)


_P = C.c_void_p
_SRP = C.POINTER(mppi_shard_range)
# (name, restype, argtypes) of every entry point in include/mppi.h
SIGNATURES = [
    ("mppi_model_create", C.c_int32, [C.POINTER(mppi_model_desc), C.POINTER(_P)]),
    ("mppi_model_destroy", None, [_P]),
    ("mppi_create", C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int32, C.c_double, _fp, C.c_int32,
                                C.POINTER(mppi_params), C.POINTER(_P)]),
    ("mppi_destroy", None, [_P]),
    ("mppi_noise_schedule", C.c_int32, [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double, _fp]),
    ("mppi_solve", C.c_int32, [_P, _dp, _fp, _fp, _fp, C.POINTER(mppi_result)]),
    ("mppi_solve_device", C.c_int32, [_P, _P, _P, _P, _P, _P]),
    ("mppi_sync", C.c_int32, [_P]),
    ("mppi_rollout_explicit", C.c_int32, [_P, _dp, _fp, _dp, _dp]),
    ("mppi_sample_knots", C.c_int32, [_P, C.c_int32, C.c_uint32, _fp, _fp]),
    ("mppi_get_iter_counter", C.c_int32, [_P, _u32p]),
    ("mppi_set_iter_counter", C.c_int32, [_P, C.c_uint32]),
    ("mppi_export_state", C.c_int32, [_P, _P, C.POINTER(C.c_size_t)]),
    ("mppi_import_state", C.c_int32, [_P, _P, C.c_size_t]),
    ("mppi_predict_state", C.c_int32, [_P, _dp, C.c_int32, _dp]),
    ("mppi_predict_state_device", C.c_int32, [_P, _P, C.c_int32, _P]),
    ("mppi_shift_warm_start", C.c_int32, [_P, C.c_int32]),
    ("mppi_get_warm_start", C.c_int32, [_P, _fp]),
    ("mppi_model_info", C.c_int32, [_P, _ip]),
    ("mppi_selftest_math", C.c_int32, [C.c_int32, _fp, _fp, _fp]),
    ("mppi_selftest_widen", C.c_int32, [C.c_int32, _fp, _dp]),
    ("mppi_check_word", C.c_int32, [_u32p, C.c_int32]),
    ("mppi_autotune_cache_file", C.c_int32, [C.c_char_p]),
    ("mppi_philox_words", C.c_int32, [C.c_int32, _u32p, _u32p, _u32p]),
    ("mppi_weights", C.c_int32, [C.c_int32, _fp, C.c_double, C.c_int32, _dp, C.POINTER(mppi_result)]),
    ("mppi_average", C.c_int32, [C.c_int32, C.c_int32, _fp, _dp, _dp]),
    ("mppi_average_noalloc", C.c_int32, [C.c_int32, C.c_int32, _P, _P, _P, _P]),
    ("mppi_shard_range_local", C.c_int32, [C.c_int32, _P, C.c_int64, _SRP, _P]),
    ("mppi_shard_range_merge", None, [_SRP, _SRP, _SRP]),
    ("mppi_shard_moments", C.c_int32, [C.c_int32, C.c_int32, _P, _P, _SRP, C.c_double, C.c_int32, _dp, _P]),
    ("mppi_shard_moments_merge", None, [C.c_int32, _dp, _dp, _dp]),
    ("mppi_shard_mean", C.c_int32, [C.c_int32, _dp, _fp]),
    ("mppi_forward_dynamics", C.c_int32, [_P, C.c_int32, _dp, _dp, _dp]),
    ("mppi_forward_dynamics_ex", C.c_int32, [_P, C.c_int32, _dp, _dp, _dp, C.c_int32]),
    ("mppi_solve_batch", C.c_int32, [C.POINTER(_P), C.c_int32, C.POINTER(_dp), C.POINTER(_fp),
                                     C.POINTER(_fp), C.POINTER(_fp), C.POINTER(mppi_result)]),
    ("mppi_selftest_queue_timeout", C.c_int32, [C.c_int64, _ip]),
    ("mppi_server_create", C.c_int32, [C.c_int32, C.c_size_t, C.c_int32, C.POINTER(_P)]),
    ("mppi_server_destroy", None, [_P]),
    ("mppi_submit", C.c_int32, [_P, _P, _dp, _fp, _u64p]),
    ("mppi_poll", C.c_int32, [_P, C.c_uint64, _fp, _fp, C.POINTER(mppi_result), C.c_int64]),
    ("mppi_next_completed", C.c_int32, [_P, C.c_int64, _u64p, _i64p]),
    ("mppi_server_stats", C.c_int32, [_P, _i64p]),
    ("mppi_server_stats_ex", C.c_int32, [_P, _i64p, C.c_int32]),
    ("mppi_server_set_deadline", C.c_int32, [_P, C.c_int64]),
    ("mppi_server_reset_timing", C.c_int32, [_P]),
    ("mppi_autotune", C.c_int32, [_P, _ip, _ip, _fp]),
    ("mppi_ctx_set_mapping", C.c_int32, [_P, C.c_int32, C.c_int32]),
    ("mppi_ctx_set_fp64_check", C.c_int32, [_P, C.c_int32]),
    ("mppi_ctx_profile", C.c_int32, [_P, C.c_int32]),
    ("mppi_ctx_rollout_ms", C.c_int32, [_P, _fp]),
    ("mppi_ctx_info", C.c_int32, [_P, _ip]),
    ("mppi_ctx_io_bytes", C.c_int32, [_P, _i64p]),
    ("mppi_ctx_device_bytes", C.c_size_t, [_P]),
    ("mppi_ctx_kernels_per_solve", C.c_int32, [_P]),
    ("mppi_status_str", C.c_char_p, [C.c_int32]),
    ("mppi_last_error", C.c_char_p, [_P]),
]

_lib = None


def load(path: str = LIB_PATH):
    """Load libmppi.so (raises MppiError if it is missing: build it with
    ``paper_2511_19204_gb300.build.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise MppiError(MPPI_ERR_UNSUPPORTED, f"{path} is missing; run the build first")
        L = C.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _err(status, ctx=None):
    L = load()
    msg = L.mppi_last_error(ctx).decode() if L else ""
    return MppiError(status, f"{L.mppi_status_str(status).decode()}: {msg}")


def _check(status, ctx=None, ok=(MPPI_OK,)):
    if status not in ok:
        raise _err(status, ctx)
    return status


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _pd(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _pf(a):
    return a.ctypes.data_as(_fp) if a is not None else None


# --------------------------------------------------------------------------------------
# One-to-one entry points
# --------------------------------------------------------------------------------------
def __getattr__(name):
    if name.startswith("mppi_"):
        return getattr(load(), name)
    raise AttributeError(name)


# --------------------------------------------------------------------------------------
# Wrappers
# --------------------------------------------------------------------------------------
class Model:
    """Device copy of a synth.RobotModel (mppi_model_create)."""

    def __init__(self, m):
        L = load()
        self.src = m
        self.nb, self.nj, self.nc = m.nb, m.nj, m.nc
        self.nx = m.nx
        self.nv = m.nv
        k = dict(parent=np.ascontiguousarray(m.parent, dtype=np.int32), axis=_d(m.axis), jpos=_d(m.jpos),
                 mass=_d(m.mass), com=_d(m.com), inertia=_d(m.inertia), armature=_d(m.armature),
                 q_min=_d(m.q_min) if m.nj else np.zeros(1), q_max=_d(m.q_max) if m.nj else np.zeros(1),
                 kp=_d(m.kp) if m.nj else np.zeros(1), kd=_d(m.kd) if m.nj else np.zeros(1),
                 tau_max=_d(m.tau_max) if m.nj else np.zeros(1),
                 contact_body=np.ascontiguousarray(m.contact_body, dtype=np.int32) if m.nc else np.zeros(1, np.int32),
                 contact_pos=_d(m.contact_pos).reshape(-1) if m.nc else np.zeros(3),
                 q_init=_d(m.q_stand) if m.q_stand is not None and m.nj else None)
        self._keep = k
        d = mppi_model_desc(nb=m.nb, nc=m.nc, fixed_base=int(m.fixed_base), cost_body=m.cost_body,
                            parent=k["parent"].ctypes.data_as(_ip), axis=_pd(k["axis"]), jpos=_pd(k["jpos"]),
                            mass=_pd(k["mass"]), com=_pd(k["com"]), inertia=_pd(k["inertia"]),
                            armature=_pd(k["armature"]), q_min=_pd(k["q_min"]), q_max=_pd(k["q_max"]),
                            kp=_pd(k["kp"]), kd=_pd(k["kd"]), tau_max=_pd(k["tau_max"]),
                            contact_body=k["contact_body"].ctypes.data_as(_ip),
                            contact_pos=_pd(k["contact_pos"]), q_init=_pd(k["q_init"]),
                            contact_k=m.contact_k, contact_c=m.contact_c, mu=m.mu, eps_f=m.eps_f,
                            gravity=m.gravity, z_des=m.z_des, vx_des=m.vx_des, w_z=m.w_z, w_vx=m.w_vx,
                            w_tilt=m.w_tilt, w_tau=m.w_tau, w_h=m.w_h, w_orient=m.w_orient, w_q=m.w_q,
                            w_cvel=m.w_cvel, w_cforce=m.w_cforce, w_term=m.w_term,
                            quat_des=(C.c_double * 4)(*m.quat_des), f0=(C.c_double * 3)(*m.f0),
                            pdot_des=(C.c_double * 3)(*m.pdot_des))
        h = _P()
        _check(L.mppi_model_create(C.byref(d), C.byref(h)))
        self.h = h

    def info(self):
        o = np.zeros(4, np.int32)
        _check(load().mppi_model_info(self.h, o.ctypes.data_as(_ip)))
        return dict(topology=int(o[0]), axis_plan=int(o[1]), paper_cost=int(o[2]), nb=int(o[3]))

    def forward_dynamics(self, states, tau, fp64=False):
        L = load()
        X = _d(states).reshape(-1, self.nx)
        n = X.shape[0]
        T = _d(tau).reshape(n, self.nj) if self.nj else np.zeros((n, 1))
        acc = np.zeros((n, self.nv))
        _check(L.mppi_forward_dynamics_ex(self.h, n, _pd(X), _pd(T), _pd(acc), int(fp64)))
        return acc

    def close(self):
        if getattr(self, "h", None):
            load().mppi_model_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Controller:
    """One MPC instance (mppi_create) on the current CUDA device."""

    def __init__(self, model: Model, n: int, horizon: int, nk: int, lam: float, sigma, iters: int = 1,
                 dt: float = 0.01, scale_q: float = 1.0, scale_v: float = 0.0, normalize: int = MPPI_NORM_MINMAX,
                 warm_from: int = MPPI_WARM_BEST, seed: int = 1, instance: int = 0,
                 mapping: int = MPPI_MAP_AUTO, block: int = 0, stream=None, spline: int = 0):
        L = load()
        self.model = model
        self.n, self.horizon, self.nk, self.iters = n, horizon, nk, iters
        self.nj = model.nj
        self.E = nk * 2 * model.nj
        self.nx = model.nx
        self.sigma = _f(sigma).reshape(iters, nk)
        p = mppi_params(dt=dt, scale_q=scale_q, scale_v=scale_v, normalize=normalize, warm_from=warm_from,
                        seed=seed, instance_id=instance, mapping=mapping, block_size=block, spline=spline,
                        stream=C.c_void_p(stream) if stream else None)
        h = _P()
        _check(L.mppi_create(model.h, n, horizon, nk, lam, _pf(self.sigma), iters, C.byref(p), C.byref(h)))
        self.h = h
        self._mean = np.zeros(self.E, np.float32)
        self._best = np.zeros(self.E, np.float32)

    @classmethod
    def from_problem(cls, model: Model, p, **kw):
        return cls(model, p.n, p.horizon, p.nk, p.lam, p.sigma, iters=p.iters, dt=p.dt, seed=p.seed,
                   instance=p.instance, **kw)

    # ---- solve ----
    def solve(self, state, warm=None, check=True):
        """Returns (mean [nk,2,nj], best [nk,2,nj], info dict)."""
        L = load()
        x = _d(state)
        w = _f(warm).reshape(-1) if warm is not None else None
        mean = np.zeros(self.E, np.float32)
        best = np.zeros(self.E, np.float32)
        info = mppi_result()
        st = L.mppi_solve(self.h, _pd(x), _pf(w), _pf(mean), _pf(best), C.byref(info))
        if check:
            _check(st, self.h, ok=(MPPI_OK, MPPI_ERR_ALL_COSTS_NONFINITE))
        d = info.as_dict()
        d["return_status"] = st
        return mean.reshape(self.nk, 2, self.nj), best.reshape(self.nk, 2, self.nj), d

    def solve_device(self, d_state, d_mean, d_best=None, d_warm=None, d_info=None):
        """Enqueue a solve on device pointers (ints, e.g. torch tensor.data_ptr())."""
        _check(load().mppi_solve_device(self.h, C.c_void_p(d_state), C.c_void_p(d_warm) if d_warm else None,
                                        C.c_void_p(d_mean), C.c_void_p(d_best) if d_best else None,
                                        C.c_void_p(d_info) if d_info else None), self.h)

    def sync(self):
        _check(load().mppi_sync(self.h), self.h)

    # ---- single steps ----
    def rollout_explicit(self, state, knots, finals=False):
        L = load()
        kn = _f(knots).reshape(self.n, self.E)
        costs = np.zeros(self.n)
        fin = np.zeros((self.n, self.nx)) if finals else None
        _check(L.mppi_rollout_explicit(self.h, _pd(_d(state)), _pf(kn), _pd(costs), _pd(fin)), self.h)
        return (costs, fin) if finals else costs

    def sample_knots(self, it, iter_counter, nominal):
        out = np.zeros((self.n, self.nk, 2, self.nj), np.float32)
        _check(load().mppi_sample_knots(self.h, it, iter_counter, _pf(_f(nominal).reshape(-1)), _pf(out)), self.h)
        return out

    @property
    def iter_counter(self):
        v = C.c_uint32()
        _check(load().mppi_get_iter_counter(self.h, C.byref(v)), self.h)
        return v.value

    @iter_counter.setter
    def iter_counter(self, value):
        _check(load().mppi_set_iter_counter(self.h, int(value)), self.h)

    def export_state(self) -> bytes:
        L = load()
        n = C.c_size_t()
        _check(L.mppi_export_state(self.h, None, C.byref(n)), self.h)
        buf = C.create_string_buffer(n.value)
        _check(L.mppi_export_state(self.h, buf, C.byref(n)), self.h)
        return buf.raw[:n.value]

    def import_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(load().mppi_import_state(self.h, buf, len(blob)), self.h)

    def predict_state(self, state, steps):
        """Sec. III-E: state after `steps` control steps of the resident warm start."""
        x = _d(state).copy()
        out = np.zeros(self.nx)
        _check(load().mppi_predict_state(self.h, _pd(x), int(steps), _pd(out)), self.h)
        return out

    def predict_state_device(self, d_state_ptr, steps, d_out_ptr):
        _check(load().mppi_predict_state_device(self.h, C.c_void_p(d_state_ptr), int(steps),
                                                C.c_void_p(d_out_ptr)), self.h)

    def shift_warm_start(self, steps):
        """Sec. III-E: shift the resident warm start by `steps` executed actions."""
        _check(load().mppi_shift_warm_start(self.h, int(steps)), self.h)

    def warm_start(self):
        out = np.zeros(self.E, np.float32)
        _check(load().mppi_get_warm_start(self.h, _pf(out)), self.h)
        return out.reshape(self.nk, 2, self.nj)

    def set_mapping(self, mapping, block=0):
        _check(load().mppi_ctx_set_mapping(self.h, mapping, block), self.h)

    def set_fp64_check(self, on=True):
        _check(load().mppi_ctx_set_fp64_check(self.h, int(on)), self.h)

    def autotune(self):
        m, b = C.c_int32(), C.c_int32()
        ms = np.zeros(16, np.float32)
        _check(load().mppi_autotune(self.h, C.byref(m), C.byref(b), _pf(ms)), self.h)
        return m.value, b.value, ms.reshape(4, 4)

    def profile(self, on=True):
        _check(load().mppi_ctx_profile(self.h, int(on)), self.h)

    def rollout_ms(self):
        ms = np.zeros(self.iters, np.float32)
        _check(load().mppi_ctx_rollout_ms(self.h, _pf(ms)), self.h)
        return ms

    def io_bytes(self):
        """(host -> device, device -> host) bytes of one solve() without a warm start."""
        o = np.zeros(2, np.int64)
        _check(load().mppi_ctx_io_bytes(self.h, o.ctypes.data_as(_i64p)), self.h)
        return int(o[0]), int(o[1])

    def info(self):
        o = np.zeros(8, np.int32)
        _check(load().mppi_ctx_info(self.h, o.ctypes.data_as(_ip)), self.h)
        return dict(n=int(o[0]), horizon=int(o[1]), nk=int(o[2]), iters=int(o[3]), nj=int(o[4]),
                    nx=int(o[5]), mapping=int(o[6]), block=int(o[7]))

    @property
    def device_bytes(self):
        return int(load().mppi_ctx_device_bytes(self.h))

    @property
    def kernels_per_solve(self):
        return int(load().mppi_ctx_kernels_per_solve(self.h))

    def close(self):
        if getattr(self, "h", None):
            load().mppi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def noise_schedule(iters, knots, beta1, beta2, scale=1.0):
    """mppi_noise_schedule: [iters][knots] float32 standard deviations."""
    out = np.zeros((iters, knots), np.float32)
    _check(load().mppi_noise_schedule(iters, knots, beta1, beta2, scale, _pf(out)))
    return out


def philox_words(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.zeros_like(c)
    _check(load().mppi_philox_words(c.shape[0], c.ctypes.data_as(_u32p), k.ctypes.data_as(_u32p),
                                    out.ctypes.data_as(_u32p)))
    return out


def weights(costs, lam, normalize=MPPI_NORM_MINMAX):
    c = _f(costs)
    w = np.zeros(c.shape[0])
    info = mppi_result()
    st = load().mppi_weights(c.shape[0], _pf(c), lam, normalize, _pd(w), C.byref(info))
    _check(st, ok=(MPPI_OK, MPPI_ERR_ALL_COSTS_NONFINITE))
    return st, w, info.as_dict()


def average(knots, w):
    k = _f(knots)
    K = k.shape[0]
    E = int(np.prod(k.shape[1:]))
    out = np.zeros(E)
    _check(load().mppi_average(K, E, _pf(k.reshape(K, E)), _pd(_d(w)), _pd(out)))
    return out.reshape(k.shape[1:])


# ------------------------------------------------------------------------------------
# Sample shards (one iteration's weights and average over samples split into shards)
# ------------------------------------------------------------------------------------
def shard_range(s_min=float("inf"), s_max=float("-inf"), best_index=-1, n_finite=0):
    """An mppi_shard_range from its four fields (the empty range by default)."""
    return mppi_shard_range(s_min, s_max, best_index, n_finite)


def shard_range_local(d_costs, K, index_base, stream=None):
    """First exchange, on the device: the range of a shard's K costs (device pointer d_costs)."""
    r = mppi_shard_range()
    _check(load().mppi_shard_range_local(K, _P(d_costs), index_base, C.byref(r), _P(stream) if stream else None))
    return r


def shard_range_merge(a, b):
    """Host merge of two ranges (associative, commutative)."""
    r = mppi_shard_range()
    load().mppi_shard_range_merge(C.byref(a), C.byref(b), C.byref(r))
    return r


def shard_moments(d_knots, d_costs, K, E, global_range, lam, normalize=MPPI_NORM_MINMAX, stream=None):
    """Second exchange, on the device: [sum w, sum w theta (E)] of a shard under the merged range."""
    out = np.zeros(E + 1)
    _check(load().mppi_shard_moments(K, E, _P(d_knots), _P(d_costs), C.byref(global_range), lam, normalize,
                                     _pd(out), _P(stream) if stream else None))
    return out


def shard_moments_merge(a, b):
    """Host merge of two moment vectors of length E + 1."""
    a, b = _d(a), _d(b)
    out = np.zeros_like(a)
    load().mppi_shard_moments_merge(a.shape[0] - 1, _pd(a), _pd(b), _pd(out))
    return out


def shard_mean(sums):
    """The updated nominal [E] (FP32) from merged moments."""
    s = _d(sums)
    out = np.zeros(s.shape[0] - 1, dtype=np.float32)
    _check(load().mppi_shard_mean(s.shape[0] - 1, _pd(s), _pf(out)))
    return out


def _packed(arrays, sizes, dtype, what):
    """One contiguous copy of `arrays` (each flattened) and each one's address in it."""
    buf = np.concatenate([np.asarray(a) for a in arrays], axis=None, dtype=dtype) if len(arrays) else \
        np.zeros(0, dtype)
    if buf.size != int(sizes.sum()):
        raise ValueError(f"solve_batch: a {what} has the wrong size")
    off = np.zeros(len(sizes), np.int64)
    np.cumsum(sizes[:-1], out=off[1:])
    return buf, (buf.__array_interface__["data"][0] + buf.itemsize * off).astype(np.uintp)


def _ptr_array(addrs, t):
    """A uintp address array passed as a C array of pointers to t (it must outlive the call)."""
    return C.cast(addrs.ctypes.data, C.POINTER(C.POINTER(t)))


def solve_batch(ctrls, states, warms=None, check=True):
    """mppi_solve_batch over Controllers: returns (status, means, bests, infos). Inputs
    and outputs are packed into one buffer each and the pointer arrays computed from
    offsets (a ctypes conversion per array cost ~10 us and dominated the host time of a
    256-instance batch)."""
    L = load()
    n = len(ctrls)
    hs = (C.c_void_p * n)(*[c.h for c in ctrls])
    nx = np.fromiter((c.nx for c in ctrls), dtype=np.int64, count=n)
    E = np.fromiter((c.E for c in ctrls), dtype=np.int64, count=n)
    xs, ps_a = _packed(states, nx, np.float64, "state")
    warms = warms or [None] * n
    has = [i for i, w in enumerate(warms) if w is not None]
    pw_a = np.zeros(n, np.uintp)
    if has:
        ws, addr = _packed([warms[i] for i in has], E[has], np.float32, "warm start")
        pw_a[has] = addr
    off = np.zeros(n, np.int64)
    np.cumsum(E[:-1], out=off[1:])
    tot = int(E.sum())
    out = np.zeros(2 * tot, np.float32)       # means, then bests
    base = out.__array_interface__["data"][0]
    pm_a = (base + 4 * off).astype(np.uintp)
    pb_a = (base + 4 * (tot + off)).astype(np.uintp)
    info = (mppi_result * n)()
    rc = L.mppi_solve_batch(hs, n, _ptr_array(ps_a, C.c_double), _ptr_array(pw_a, C.c_float),
                            _ptr_array(pm_a, C.c_float), _ptr_array(pb_a, C.c_float), info)
    if check:
        _check(rc, ok=(MPPI_OK, MPPI_ERR_ALL_COSTS_NONFINITE))
    offs, shapes = off.tolist(), [(c.nk, 2, c.nj) for c in ctrls]
    means = [out[o:o + e].reshape(sh) for o, e, sh in zip(offs, E.tolist(), shapes)]
    bests = [out[tot + o:tot + o + e].reshape(sh) for o, e, sh in zip(offs, E.tolist(), shapes)]
    names = [f for f, _ in mppi_result._fields_]
    infos = [dict(zip(names, r)) for r in np.ctypeslib.as_array(info).tolist()]
    return rc, means, bests, infos


class Server:
    """Continuous-batching request loop (mppi_server_create / submit / poll)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 8 << 30, max_inflight: int = 4):
        h = _P()
        _check(load().mppi_server_create(device, mem_budget_bytes, max_inflight, C.byref(h)))
        self.h = h

    def submit(self, ctrl: Controller, state, warm=None) -> int:
        t = C.c_uint64()
        x = _d(state)
        w = _f(warm).reshape(-1) if warm is not None else None
        _check(load().mppi_submit(self.h, ctrl.h, _pd(x), _pf(w), C.byref(t)), ctrl.h)
        return t.value

    def poll(self, ticket: int, ctrl: Controller, timeout_us: int = -1):
        """(status, mean, best, info) or None while pending."""
        mean = np.zeros(ctrl.E, np.float32)
        best = np.zeros(ctrl.E, np.float32)
        info = mppi_result()
        st = load().mppi_poll(self.h, ticket, _pf(mean), _pf(best), C.byref(info), timeout_us)
        if st == MPPI_PENDING:
            return None
        if st == MPPI_ERR_NOT_FOUND:
            raise _err(st)
        return st, mean.reshape(ctrl.nk, 2, ctrl.nj), best.reshape(ctrl.nk, 2, ctrl.nj), info.as_dict()

    def next_completed(self, timeout_us: int = 0):
        """(ticket, submit_ns, done_ns) or None."""
        t = C.c_uint64()
        tm = np.zeros(2, np.int64)
        st = load().mppi_next_completed(self.h, timeout_us, C.byref(t), tm.ctypes.data_as(_i64p))
        if st == MPPI_PENDING:
            return None
        _check(st)
        return t.value, int(tm[0]), int(tm[1])

    def set_deadline(self, deadline_us: int):
        """Shed requests still waiting for admission deadline_us after submission
        (they complete with MPPI_ERR_DEADLINE); 0 never sheds."""
        _check(load().mppi_server_set_deadline(self.h, int(deadline_us)))

    def stats(self):
        o = np.zeros(11, np.int64)
        _check(load().mppi_server_stats_ex(self.h, o.ctypes.data_as(_i64p), 11))
        return dict(submitted=int(o[0]), completed=int(o[1]), launches=int(o[2]), peak_bytes=int(o[3]),
                    deferred=int(o[4]), shed=int(o[5]), reserved_bytes=int(o[6]), slot_bytes=int(o[7]),
                    max_worker_pass_ns=int(o[8]), max_launch_ns=int(o[9]), max_unpack_ns=int(o[10]))

    def reset_timing(self):
        """Restart the worker-timing maxima reported by stats()."""
        _check(load().mppi_server_reset_timing(self.h))

    def close(self):
        if getattr(self, "h", None):
            load().mppi_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_math(x, y):
    """The rollout's FP32 (sin x, cos x, atan2(y, x)) for y >= 0, shape [n, 3]."""
    xs = _f(x).reshape(-1).copy()
    ys = _f(y).reshape(-1).copy()
    out = np.zeros((xs.shape[0], 3), np.float32)
    _check(load().mppi_selftest_math(xs.shape[0], _pf(xs), _pf(ys), _pf(out)))
    return out


def selftest_widen(x):
    """The knot average's integer FP32 -> FP64 widening of x (float32), as float64."""
    xs = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
    out = np.zeros(xs.shape[0], np.float64)
    _check(load().mppi_selftest_widen(xs.shape[0], _pf(xs), _pd(out)))
    return out


def autotune_cache_file(path):
    """Persist the autotuner's choices in the JSON file `path` (None: this process only)."""
    _check(load().mppi_autotune_cache_file(path.encode() if path else None))

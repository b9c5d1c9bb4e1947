"""FP64 CPU oracle of the Hermite-spline MPPI hot path (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import this
package. It loads ``liboracle.so`` compiled from ``oracle.c`` (plain C, FP64) and never
touches the CUDA library; the two share no code. Inputs come from the seeded
generators in ``paper_2511_19204_gb300.synth`` (data only).

Each wrapper cites the part of the paper it restates; see ``oracle.c`` for the
arithmetic.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_COUNT_SRC = os.path.join(_HERE, "count.cc")
_COUNT_LIB = os.path.join(_HERE, "liboracle_count.so")

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O3, portable flags, no fast-math and no contraction of a
    multiply and an add into a fused one, which GCC does by default where the target has
    it: the oracle computes each operation of its source rounded separately, on x86 and Arm
    alike) and its operation-counting build (g++, the same source with a counting scalar
    type)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O3", "-ffp-contract=off", "-std=gnu11", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm",
               "-lpthread"]
        subprocess.check_call(cmd)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_COUNT_SRC))
    if force or not os.path.exists(_COUNT_LIB) or os.path.getmtime(_COUNT_LIB) < newest:
        cmd = ["g++", "-O1", "-ffp-contract=off", "-std=c++17", "-fPIC", "-shared", "-o", _COUNT_LIB, _COUNT_SRC,
               "-lm", "-lpthread"]
        subprocess.check_call(cmd)
    return _LIB


class _Model(C.Structure):
    _fields_ = [("nb", C.c_int32), ("nc", C.c_int32), ("fixed_base", C.c_int32),
                ("cost_body", C.c_int32),
                ("parent", _ip), ("axis", _dp), ("jpos", _dp), ("mass", _dp), ("com", _dp),
                ("inertia", _dp), ("armature", _dp), ("q_min", _dp), ("q_max", _dp),
                ("kp", _dp), ("kd", _dp), ("tau_max", _dp), ("contact_body", _ip),
                ("contact_pos", _dp),
                ("contact_k", C.c_double), ("contact_c", C.c_double), ("mu", C.c_double),
                ("eps_f", C.c_double), ("gravity", C.c_double),
                ("z_des", C.c_double), ("vx_des", C.c_double), ("w_z", C.c_double),
                ("w_vx", C.c_double), ("w_tilt", C.c_double), ("w_tau", C.c_double),
                ("w_h", C.c_double), ("w_orient", C.c_double), ("w_q", C.c_double),
                ("w_cvel", C.c_double), ("w_cforce", C.c_double), ("w_term", C.c_double),
                ("quat_des", C.c_double * 4), ("f0", C.c_double * 3), ("pdot_des", C.c_double * 3),
                ("q0", _dp)]


_lib = None

SPLINE_HERMITE, SPLINE_CUBIC, SPLINE_QUADRATIC = 0, 1, 2   # Sec. IV-D variants


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        mp = C.POINTER(_Model)
        L.orc_philox.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.orc_normal.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]
        L.orc_normal.restype = C.c_double
        L.orc_clamp.argtypes = [C.c_int, C.c_int, C.c_double, _dp, _dp, _dp]
        L.orc_sample_knots.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, _dp, _dp,
                                       C.c_double, C.c_double, C.c_uint64, C.c_uint32, C.c_uint32,
                                       _dp, _dp, _dp]
        L.orc_noise_schedule.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, _dp]
        L.orc_segment.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), _dp]
        L.orc_hermite.argtypes = [C.c_double] * 6 + [_dp, _dp]
        L.orc_forward_dynamics.argtypes = [mp, _dp, _dp, _dp]
        L.orc_forward_dynamics.restype = C.c_int
        L.orc_crba.argtypes = [mp, _dp, _dp]
        L.orc_crba.restype = C.c_int
        L.orc_rnea_bias.argtypes = [mp, _dp, _dp]
        L.orc_rnea_bias.restype = C.c_int
        L.orc_contact_forces.argtypes = [mp, _dp, _dp]
        L.orc_positions.argtypes = [mp, _dp, _dp, _dp]
        L.orc_energy.argtypes = [mp, _dp]
        L.orc_energy.restype = C.c_double
        L.orc_step.argtypes = [mp, _dp, _dp, C.c_double]
        L.orc_step.restype = C.c_int
        L.orc_rollout.argtypes = [mp, _dp, _dp, C.c_int, C.c_int, C.c_double, _dp, _dp]
        L.orc_rollout.restype = C.c_double
        L.orc_rollout_ex.argtypes = [mp, _dp, _dp, C.c_int, C.c_int, C.c_double, C.c_int, _dp, _dp]
        L.orc_rollout_ex.restype = C.c_double
        L.orc_rollout_batch.argtypes = [mp, C.c_int, _dp, _dp, C.c_int, C.c_int, C.c_double, _dp,
                                        _dp, C.c_int]
        L.orc_rollout_batch_ex.argtypes = [mp, C.c_int, _dp, _dp, C.c_int, C.c_int, C.c_double, C.c_int,
                                           _dp, _dp, C.c_int]
        L.orc_spline_slopes.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, _dp]
        L.orc_setpoints.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, _dp, _dp, _dp]
        L.orc_predict_state.argtypes = [mp, _dp, _dp, C.c_int, C.c_int, C.c_int, C.c_double, _dp]
        L.orc_predict_state.restype = C.c_int
        L.orc_shift_knots.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, _dp, _dp]
        L.orc_weights.argtypes = [C.c_int, _dp, C.c_double, C.c_int, _dp, _dp]
        L.orc_weights.restype = C.c_int
        L.orc_average.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp]
        L.orc_solve.argtypes = [mp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                C.c_int, _dp, C.c_double, C.c_double, C.c_uint64, C.c_uint32,
                                C.c_uint32, _dp, _dp, _dp, _dp, _dp, C.c_int, _dp, _dp, C.c_int]
        L.orc_solve.restype = C.c_int
        _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


class OracleModel:
    """The oracle's own packing of a synthetic RobotModel (keeps the arrays alive)."""

    def __init__(self, m):
        self.src = m
        self._keep = dict(
            parent=np.ascontiguousarray(m.parent, dtype=np.int32), axis=_d(m.axis), jpos=_d(m.jpos),
            mass=_d(m.mass), com=_d(m.com), inertia=_d(m.inertia), armature=_d(m.armature),
            q_min=_d(m.q_min), q_max=_d(m.q_max), kp=_d(m.kp), kd=_d(m.kd), tau_max=_d(m.tau_max),
            contact_body=np.ascontiguousarray(m.contact_body, dtype=np.int32),
            contact_pos=_d(m.contact_pos).reshape(-1, 3) if m.nc else np.zeros((1, 3)))
        if m.nc == 0:
            self._keep["contact_body"] = np.zeros(1, dtype=np.int32)
        self._keep["q0"] = _d(m.q_stand) if m.q_stand is not None and m.nj else np.zeros(max(m.nj, 1))
        qd = np.asarray(getattr(m, "quat_des", (1.0, 0.0, 0.0, 0.0)), dtype=np.float64)
        qd = qd / np.linalg.norm(qd) if np.linalg.norm(qd) > 0 else np.array([1.0, 0.0, 0.0, 0.0])
        k = self._keep
        self.s = _Model(nb=m.nb, nc=m.nc, fixed_base=int(m.fixed_base), cost_body=m.cost_body,
                        parent=k["parent"].ctypes.data_as(_ip), axis=_ptr(k["axis"]),
                        jpos=_ptr(k["jpos"]), mass=_ptr(k["mass"]), com=_ptr(k["com"]),
                        inertia=_ptr(k["inertia"]), armature=_ptr(k["armature"]),
                        q_min=_ptr(k["q_min"]), q_max=_ptr(k["q_max"]), kp=_ptr(k["kp"]),
                        kd=_ptr(k["kd"]), tau_max=_ptr(k["tau_max"]),
                        contact_body=k["contact_body"].ctypes.data_as(_ip),
                        contact_pos=_ptr(k["contact_pos"]),
                        contact_k=m.contact_k, contact_c=m.contact_c, mu=m.mu, eps_f=m.eps_f,
                        gravity=m.gravity, z_des=m.z_des, vx_des=m.vx_des, w_z=m.w_z,
                        w_vx=m.w_vx, w_tilt=m.w_tilt, w_tau=m.w_tau,
                        w_h=m.w_h, w_orient=m.w_orient, w_q=m.w_q, w_cvel=m.w_cvel,
                        w_cforce=m.w_cforce, w_term=m.w_term,
                        quat_des=(C.c_double * 4)(*qd), f0=(C.c_double * 3)(*m.f0),
                        pdot_des=(C.c_double * 3)(*m.pdot_des), q0=_ptr(k["q0"]))
        self.ref = C.byref(self.s)
        self.nj = m.nj
        self.nx = m.nx
        self.nv = m.nv


def _om(m):
    return m if isinstance(m, OracleModel) else OracleModel(m)


# ------------------------------------------------------------------------------------
# Noise: Philox4x32-10 words, Box-Muller normals, Alg. 1 sampling + Eq. (vel-clamp)
# ------------------------------------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    u32p = C.POINTER(C.c_uint32)
    lib().orc_philox(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), out.ctypes.data_as(u32p))
    return out


def normal(seed: int, iter_ctr: int, inst: int, n: int, e: int) -> float:
    return lib().orc_normal(seed, iter_ctr, inst, n, e)


def sample_knots(nu, nk, N, H, dt, nominal, sigma_row, scale_q=1.0, scale_v=0.0, seed=1,
                 iter_ctr=0, inst=0, q_min=None, q_max=None) -> np.ndarray:
    out = np.zeros((N, nk, 2, nu))
    nom = _d(nominal).reshape(-1)
    sr = _d(sigma_row).reshape(-1)
    lo = _d(q_min) if q_min is not None else None
    hi = _d(q_max) if q_max is not None else None
    lib().orc_sample_knots(nu, nk, N, H, dt, _ptr(nom), _ptr(sr), scale_q, scale_v, seed, iter_ctr,
                           inst, _ptr(lo), _ptr(hi), _ptr(out))
    return out


def noise_schedule(iters, knots, beta1, beta2, scale=1.0) -> np.ndarray:
    """Sec. III-B Eq. (overall-noise-kernel) as a [iters][knots] standard-deviation table."""
    out = np.zeros((iters, knots))
    lib().orc_noise_schedule(iters, knots, beta1, beta2, scale, _ptr(out))
    return out


def clamp(knots, dtk, q_min, q_max) -> np.ndarray:
    k = _d(knots).copy()
    nk, _, nu = k.shape
    lib().orc_clamp(nu, nk, dtk, _ptr(_d(q_min)), _ptr(_d(q_max)), _ptr(k))
    return k


# ------------------------------------------------------------------------------------
# Spline
# ------------------------------------------------------------------------------------
def segment(h, H, nk):
    k = C.c_int()
    s = C.c_double()
    lib().orc_segment(h, H, nk, C.byref(k), C.byref(s))
    return k.value, s.value


def hermite(s, dtk, q0, v0, q1, v1):
    q = C.c_double()
    qd = C.c_double()
    lib().orc_hermite(s, dtk, q0, v0, q1, v1, C.byref(q), C.byref(qd))
    return q.value, qd.value


# ------------------------------------------------------------------------------------
# Dynamics
# ------------------------------------------------------------------------------------
def forward_dynamics(m, x, tau) -> np.ndarray:
    om = _om(m)
    acc = np.zeros(om.nv)
    t = _d(tau) if om.nj else np.zeros(1)
    rc = lib().orc_forward_dynamics(om.ref, _ptr(_d(x)), _ptr(t), _ptr(acc))
    if rc != 0:
        raise FloatingPointError("singular articulated inertia")
    return acc


def crba(m, x) -> np.ndarray:
    om = _om(m)
    n = om.nv - (6 if om.src.fixed_base else 0)
    M = np.zeros((n, n))
    lib().orc_crba(om.ref, _ptr(_d(x)), _ptr(M))
    return M


def rnea_bias(m, x) -> np.ndarray:
    om = _om(m)
    n = om.nv - (6 if om.src.fixed_base else 0)
    h = np.zeros(n)
    lib().orc_rnea_bias(om.ref, _ptr(_d(x)), _ptr(h))
    return h


def contact_forces(m, x) -> np.ndarray:
    om = _om(m)
    out = np.zeros((max(om.src.nc, 1), 3))
    lib().orc_contact_forces(om.ref, _ptr(_d(x)), _ptr(out))
    return out[:om.src.nc]


def positions(m, x):
    om = _om(m)
    b = np.zeros((om.src.nb, 3))
    c = np.zeros((max(om.src.nc, 1), 3))
    lib().orc_positions(om.ref, _ptr(_d(x)), _ptr(b), _ptr(c))
    return b, c[:om.src.nc]


def energy(m, x) -> float:
    om = _om(m)
    return lib().orc_energy(om.ref, _ptr(_d(x)))


def step(m, x, tau, dt) -> np.ndarray:
    om = _om(m)
    y = _d(x).copy()
    t = _d(tau) if om.nj else np.zeros(1)
    if lib().orc_step(om.ref, _ptr(y), _ptr(t), dt) != 0:
        raise FloatingPointError("singular articulated inertia")
    return y


def rollout(m, x0, knots, H, dt, traj=False, spline=0):
    """Returns (cost, x_final[, traj [H+1, nx]])."""
    om = _om(m)
    kn = _d(knots)
    nk = kn.shape[0]
    xf = np.zeros(om.nx)
    tr = np.zeros((H + 1, om.nx)) if traj else None
    S = lib().orc_rollout_ex(om.ref, _ptr(_d(x0)), _ptr(kn), nk, H, dt, spline, _ptr(xf), _ptr(tr))
    return (S, xf, tr) if traj else (S, xf)


def rollout_batch(m, x0, knots, H, dt, finals=False, nthreads=None, spline=0):
    om = _om(m)
    kn = _d(knots)
    N, nk = kn.shape[0], kn.shape[1]
    costs = np.zeros(N)
    fin = np.zeros((N, om.nx)) if finals else None
    nt = nthreads or os.cpu_count() or 1
    lib().orc_rollout_batch_ex(om.ref, N, _ptr(_d(x0)), _ptr(kn), nk, H, dt, spline, _ptr(costs), _ptr(fin), nt)
    return (costs, fin) if finals else costs


def setpoints(knots, H, dt, spline=0):
    """The (q_ref, v_ref) [H, nu] a rollout tracks for knots [nk, 2, nu]."""
    kn = _d(knots)
    nk, _, nu = kn.shape
    q = np.zeros((H, nu))
    v = np.zeros((H, nu))
    lib().orc_setpoints(spline, nu, nk, H, dt, _ptr(kn), _ptr(q), _ptr(v))
    return q, v


def spline_slopes(knots, H, dt, spline) -> np.ndarray:
    """Sec. IV-D variants: the velocity knots replaced by the variant spline's node
    derivatives of the position knots (knots [nk, 2, nu])."""
    kn = _d(knots).copy()
    nk, _, nu = kn.shape
    lib().orc_spline_slopes(spline, nu, nk, H * dt / (nk - 1), _ptr(kn))
    return kn


def predict_state(m, x0, knots, H, nsteps, dt) -> np.ndarray:
    """Sec. III-E: the state after the first nsteps steps of the knots' spline."""
    om = _om(m)
    kn = _d(knots)
    out = np.zeros(om.nx)
    lib().orc_predict_state(om.ref, _ptr(_d(x0)), _ptr(kn), kn.shape[0], H, nsteps, dt, _ptr(out))
    return out


def shift_knots(knots, H, steps, dt) -> np.ndarray:
    """Sec. III-E: shift by `steps` actions, tail held at the horizon end."""
    kn = _d(knots)
    nk, _, nu = kn.shape
    out = np.zeros_like(kn)
    lib().orc_shift_knots(nu, nk, H, steps, dt, _ptr(kn), _ptr(out))
    return out


# ------------------------------------------------------------------------------------
# Weights, average, solve
# ------------------------------------------------------------------------------------
def weights(costs, lam, normalize=0):
    """Returns (status, w [N], info dict)."""
    S = _d(costs)
    N = S.shape[0]
    w = np.zeros(N)
    info = np.zeros(6)
    st = lib().orc_weights(N, _ptr(S), lam, normalize, _ptr(w), _ptr(info))
    return st, w, dict(smin=info[0], smax=info[1], best=int(info[2]), ess=info[3],
                       n_finite=int(info[4]), lse=info[5])


def average(knots, w) -> np.ndarray:
    kn = _d(knots)
    N = kn.shape[0]
    E = int(np.prod(kn.shape[1:]))
    out = np.zeros(E)
    lib().orc_average(N, E, _ptr(kn), _ptr(_d(w)), _ptr(out))
    return out.reshape(kn.shape[1:])


def solve(m, n, nk, H, iters, dt, lam, sigma, state, nominal, seed=1, iter_base=0, inst=0,
          normalize=0, scale_q=1.0, scale_v=0.0, nthreads=None, keep=False, spline=0):
    """Alg. 1 from `state` and `nominal`. Returns dict(mean, best, info[, knots, costs])."""
    om = _om(m)
    nu = om.nj
    E = nk * 2 * nu
    mean = np.zeros(E)
    best = np.zeros(E)
    info = np.zeros(8)
    kn = np.zeros((iters, n, E)) if keep else None
    co = np.zeros((iters, n)) if keep else None
    nt = nthreads or os.cpu_count() or 1
    st = lib().orc_solve(om.ref, n, nk, H, iters, dt, lam, normalize, _ptr(_d(sigma)), scale_q,
                         scale_v, seed, iter_base, inst, _ptr(_d(state)), _ptr(_d(nominal)),
                         _ptr(mean), _ptr(best), _ptr(info), nt, _ptr(kn), _ptr(co), spline)
    out = dict(status=st, mean=mean.reshape(nk, 2, nu), best=best.reshape(nk, 2, nu),
               smin=info[0], smax=info[1], best_cost=info[2], best_index=int(info[3]),
               best_iter=int(info[4]), ess=info[5], n_finite=int(info[6]))
    if keep:
        out["knots"] = kn.reshape(iters, n, nk, 2, nu)
        out["costs"] = co
    return out


def solve_problem(p, iter_base=0, nthreads=None, keep=False, **kw):
    """Alg. 1 on a synth.Problem."""
    return solve(p.model, p.n, p.nk, p.horizon, p.iters, p.dt, p.lam, p.sigma, p.state, p.nominal,
                 seed=p.seed, iter_base=iter_base, inst=p.instance, nthreads=nthreads, keep=keep, **kw)


# ------------------------------------------------------------------------------------
# Operation counts of the algorithm as the oracle specifies it (count.cc)
# ------------------------------------------------------------------------------------
PHASES = ("spline", "pd", "pass1", "contact", "bias", "pass2", "solve", "pass3", "cost", "integrate", "other")
OP_KINDS = ("add", "mul", "div", "sqrt", "func", "cmp", "trivial_add", "trivial_mul", "trivial_div")
_count_lib = None


def _count():
    global _count_lib
    if _count_lib is None:
        build()
        L = C.CDLL(_COUNT_LIB)
        L.orc_count_rollout.argtypes = [C.POINTER(_Model), _dp, _dp, C.c_int, C.c_int, C.c_double, C.c_int, _dp]
        L.orc_count_rollout.restype = C.c_double
        L.orc_count_dims.argtypes = [_ip]
        dims = np.zeros(2, np.int32)
        L.orc_count_dims(dims.ctypes.data_as(_ip))
        assert (int(dims[0]), int(dims[1])) == (len(PHASES), len(OP_KINDS))
        _count_lib = L
    return _count_lib


def count_rollout(m, x0, knots, H, dt, spline=0):
    """Operations of one rollout of one sample, by phase and kind: (cost, counts [phase][kind])
    with counts a numpy array indexed by PHASES and OP_KINDS. Flops = add + mul + div +
    sqrt + func (a multiply-add is a mul and an add); the trivial_* columns count the
    operations among those whose result a structural 0 or +-1 operand fixes."""
    om = _om(m)
    kn = _d(knots)
    out = np.zeros((len(PHASES), len(OP_KINDS)))
    S = _count().orc_count_rollout(om.ref, _ptr(_d(x0)), _ptr(kn), kn.shape[0], H, dt, spline, _ptr(out))
    return S, out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

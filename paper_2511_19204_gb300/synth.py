"""Seeded synthetic inputs: robot models, initial states, nominal knots, noise schedules.

This module is the only code shared by the CUDA path and the FP64 oracle. It holds
data, never the method's arithmetic: it writes down masses, inertias, joint
placements, gains and contact points, and draws seeded random numbers. Everything the
controller computes from these inputs (noise, splines, dynamics, weights, averages)
lives separately on each side.

The paper's robots (Go2, G1) and its simulator are not available, so the two robot
families here stand in for its workloads (Sec. IV-A):

Armature (reflected rotor inertia) and the friction regularisation eps_f are model
parameters chosen so that semi-implicit Euler is stable at the workloads' time steps:
with armature 0.2 kg m^2 (quadruped) / 0.05 (humanoid) and eps_f = 1.5 m/s the
linearised one-step map at the standing pose has spectral radius 1.0 at dt = 0.01 and
0.005 for the quadruped, and only the physical falling mode (about 1.01) for the
humanoid. Smaller values leave period-2 contact-damping and friction modes above 1.

* ``quadruped()``: a 12-joint quadruped with a floating trunk (6 kg, 0.38 x 0.09 x
  0.11 m box), hip bodies (0.5 kg spheres, r = 0.04 m) at the trunk corners, and
  thigh/calf rods (0.21 m, 1.0/0.2 kg). Hip axis x, thigh and calf axes y. The foot is
  a point contact at the end of the calf. Standing pose hip 0, thigh 0.8, calf -1.6 rad
  puts each foot 0.2926 m below its hip joint.
* ``humanoid(seed)``: a floating pelvis with a waist-yaw torso, two 6-joint legs
  (hip yaw/roll/pitch, knee, ankle pitch/roll) and two 4-joint arms (shoulder
  pitch/roll/yaw, elbow): 21 joints, 22 bodies. Link masses U(0.5, 8) kg and lengths
  U(0.1, 0.45) m from the seed; thigh and shin lengths are drawn from U(0.35, 0.45) m
  and mirrored so a 1.0 m torso height is reachable. Feet are 0.2 x 0.08 m rectangles
  with four corner contacts each.
* a zoo of tiny trees for the dynamics pins: fixed-base pendulum, fixed-base 2-link
  chain, free body, floating base with a 2-body branch, and a point mass for the
  contact model.

Conventions shared by both sides (a data format, not code):

* body 0 is the base (floating unless ``fixed_base``); body i >= 1 hangs from
  ``parent[i] < i`` on a revolute joint. The joint frame sits at ``jpos[i]`` in the
  parent frame, parallel to the parent frame at q = 0, and rotates about the unit
  ``axis[i]`` (child-frame coordinates) by q_i.
* body inertia: ``mass``, centre of mass ``com`` (body frame) and rotational inertia
  about the centre of mass ``inertia`` = (Ixx, Iyy, Izz, Ixy, Ixz, Iyz).
* state = [p_base(3, world), quat(4: w,x,y,z, body->world), q(nj),
  v_base_lin(3, body frame), omega_base(3, body frame), qdot(nj)].
* knots = [knot][q|v][joint], knot j at t_j = j * H * dt / (nk - 1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GRAVITY = 9.81


@dataclasses.dataclass
class RobotModel:
    name: str
    parent: np.ndarray          # int32 [nb]
    axis: np.ndarray            # f64 [nb, 3]
    jpos: np.ndarray            # f64 [nb, 3]
    mass: np.ndarray            # f64 [nb]
    com: np.ndarray             # f64 [nb, 3]
    inertia: np.ndarray         # f64 [nb, 6]
    armature: np.ndarray        # f64 [nb] (entry 0 unused)
    q_min: np.ndarray           # f64 [nj]
    q_max: np.ndarray           # f64 [nj]
    kp: np.ndarray              # f64 [nj]
    kd: np.ndarray              # f64 [nj]
    tau_max: np.ndarray         # f64 [nj]
    contact_body: np.ndarray    # int32 [nc]
    contact_pos: np.ndarray     # f64 [nc, 3]
    contact_k: float = 2.0e4
    contact_c: float = 200.0
    mu: float = 0.8
    eps_f: float = 0.1
    gravity: float = GRAVITY
    fixed_base: bool = False
    cost_body: int = 0
    z_des: float = 0.30
    vx_des: float = 0.5
    w_z: float = 1.0
    w_vx: float = 1.0
    w_tilt: float = 1.0
    w_tau: float = 1.0e-3
    q_stand: np.ndarray = None  # f64 [nj]; also q0 of the w_q cost term
    base_z0: float = 0.0
    # modular cost of Sec. IV-A (zero weights disable a term)
    w_h: float = 0.0
    w_orient: float = 0.0
    w_q: float = 0.0
    w_cvel: float = 0.0
    w_cforce: float = 0.0
    w_term: float = 0.0
    quat_des: tuple = (1.0, 0.0, 0.0, 0.0)
    f0: tuple = (0.0, 0.0, 0.0)
    pdot_des: tuple = (0.0, 0.0, 0.0)

    @property
    def nb(self) -> int:
        return int(self.parent.shape[0])

    @property
    def nj(self) -> int:
        return self.nb - 1

    @property
    def nc(self) -> int:
        return int(self.contact_body.shape[0])

    @property
    def nq(self) -> int:
        return 7 + self.nj

    @property
    def nv(self) -> int:
        return 6 + self.nj

    @property
    def nx(self) -> int:
        return self.nq + self.nv

    def copy(self, **changes) -> "RobotModel":
        fields = {}
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            fields[f.name] = v.copy() if isinstance(v, np.ndarray) else v
        fields.update(changes)
        return RobotModel(**fields)


def _rod_inertia(m: float, length: float, radius: float, along: str = "z") -> np.ndarray:
    """Uniform rod/cylinder about its centre: transverse m L^2/12 + m r^2/4, axial m r^2/2."""
    tr = m * length * length / 12.0 + m * radius * radius / 4.0
    ax = 0.5 * m * radius * radius
    d = {"x": (ax, tr, tr), "y": (tr, ax, tr), "z": (tr, tr, ax)}[along]
    return np.array([d[0], d[1], d[2], 0.0, 0.0, 0.0])


def _box_inertia(m: float, sx: float, sy: float, sz: float) -> np.ndarray:
    return np.array([m * (sy * sy + sz * sz) / 12.0, m * (sx * sx + sz * sz) / 12.0,
                     m * (sx * sx + sy * sy) / 12.0, 0.0, 0.0, 0.0])


def _sphere_inertia(m: float, r: float) -> np.ndarray:
    i = 0.4 * m * r * r
    return np.array([i, i, i, 0.0, 0.0, 0.0])


def _finish(name, bodies, contacts, nj_limits=None, **kw) -> RobotModel:
    nb = len(bodies)
    parent = np.array([b["parent"] for b in bodies], dtype=np.int32)
    axis = np.array([b.get("axis", (0.0, 0.0, 1.0)) for b in bodies], dtype=np.float64)
    jpos = np.array([b.get("jpos", (0.0, 0.0, 0.0)) for b in bodies], dtype=np.float64)
    mass = np.array([b["mass"] for b in bodies], dtype=np.float64)
    com = np.array([b.get("com", (0.0, 0.0, 0.0)) for b in bodies], dtype=np.float64)
    inertia = np.array([b["inertia"] for b in bodies], dtype=np.float64)
    armature = np.array([b.get("armature", 0.0) for b in bodies], dtype=np.float64)
    nj = nb - 1
    inf = np.full(nj, np.inf)
    q_min = -inf.copy() if nj_limits is None else np.asarray(nj_limits[0], dtype=np.float64)
    q_max = inf.copy() if nj_limits is None else np.asarray(nj_limits[1], dtype=np.float64)
    kp = np.array([b.get("kp", 0.0) for b in bodies[1:]], dtype=np.float64)
    kd = np.array([b.get("kd", 0.0) for b in bodies[1:]], dtype=np.float64)
    tau_max = np.array([b.get("tau_max", np.inf) for b in bodies[1:]], dtype=np.float64)
    cb = np.array([c[0] for c in contacts], dtype=np.int32).reshape(-1)
    cp = np.array([c[1] for c in contacts], dtype=np.float64).reshape(-1, 3)
    return RobotModel(name=name, parent=parent, axis=axis, jpos=jpos, mass=mass, com=com,
                      inertia=inertia, armature=armature, q_min=q_min, q_max=q_max, kp=kp,
                      kd=kd, tau_max=tau_max, contact_body=cb, contact_pos=cp, **kw)


# --------------------------------------------------------------------------------------
# Quadruped (floating trunk + 4 legs x 3 revolute joints, 13 bodies, 4 point feet)
# --------------------------------------------------------------------------------------
QUAD_THIGH_L = 0.21
QUAD_CALF_L = 0.21
QUAD_STAND = (0.0, 0.8, -1.6)


def quadruped(kp: float = 40.0, kd: float = 1.0, tau_max: float = 40.0,
              armature: float = 0.2, eps_f: float = 1.5,
              limits: tuple | None = None) -> RobotModel:
    """The 18-DoF quadruped of the plain and scale workloads.

    Legs are ordered FL, FR, HL, HR; each leg is hip (axis x), thigh (axis y), calf
    (axis y). ``limits`` = (q_min[3], q_max[3]) per leg joint turns the knot clamp on.
    """
    bodies = [dict(parent=-1, mass=6.0, inertia=_box_inertia(6.0, 0.38, 0.09, 0.11))]
    contacts = []
    for sx, sy in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
        hip = len(bodies)
        bodies.append(dict(parent=0, axis=(1.0, 0.0, 0.0), jpos=(0.19 * sx, 0.045 * sy, 0.0),
                           mass=0.5, inertia=_sphere_inertia(0.5, 0.04), armature=armature,
                           kp=kp, kd=kd, tau_max=tau_max))
        thigh = len(bodies)
        bodies.append(dict(parent=hip, axis=(0.0, 1.0, 0.0), jpos=(0.0, 0.08 * sy, 0.0),
                           mass=1.0, com=(0.0, 0.0, -QUAD_THIGH_L / 2),
                           inertia=_rod_inertia(1.0, QUAD_THIGH_L, 0.02), armature=armature,
                           kp=kp, kd=kd, tau_max=tau_max))
        calf = len(bodies)
        bodies.append(dict(parent=thigh, axis=(0.0, 1.0, 0.0), jpos=(0.0, 0.0, -QUAD_THIGH_L),
                           mass=0.2, com=(0.0, 0.0, -QUAD_CALF_L / 2),
                           inertia=_rod_inertia(0.2, QUAD_CALF_L, 0.015), armature=armature,
                           kp=kp, kd=kd, tau_max=tau_max))
        contacts.append((calf, (0.0, 0.0, -QUAD_CALF_L)))
    lim = None
    if limits is not None:
        lo = np.tile(np.asarray(limits[0], dtype=np.float64), 4)
        hi = np.tile(np.asarray(limits[1], dtype=np.float64), 4)
        lim = (lo, hi)
    m = _finish("quadruped", bodies, contacts, nj_limits=lim,
                contact_k=2.0e4, contact_c=200.0, mu=0.8, eps_f=eps_f,
                cost_body=0, z_des=0.30, vx_des=0.5, w_z=1.0, w_vx=1.0, w_tilt=1.0, w_tau=1.0e-3)
    m.q_stand = np.tile(np.array(QUAD_STAND), 4)
    th, ca = QUAD_STAND[1], QUAD_STAND[1] + QUAD_STAND[2]
    foot_drop = QUAD_THIGH_L * math.cos(th) + QUAD_CALF_L * math.cos(ca)
    m.base_z0 = foot_drop - float(m.mass.sum()) * m.gravity / (4.0 * m.contact_k)
    return m


# --------------------------------------------------------------------------------------
# Humanoid (floating pelvis + 21 revolute joints, 22 bodies, 2 feet x 4 contacts)
# --------------------------------------------------------------------------------------
HUMANOID_SEED = 0x5EED


def humanoid(seed: int = HUMANOID_SEED, kp: float = 200.0, kd: float = 5.0,
             tau_max: float = 150.0, armature: float = 0.05, eps_f: float = 1.5) -> RobotModel:
    rng = np.random.default_rng(seed)

    def mass():
        return float(rng.uniform(0.5, 8.0))

    def length():
        return float(rng.uniform(0.1, 0.45))

    X, Y, Z = (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)
    jkw = dict(armature=armature, kp=kp, kd=kd, tau_max=tau_max)
    m_pelvis = mass()
    bodies = [dict(parent=-1, mass=m_pelvis, inertia=_box_inertia(m_pelvis, 0.15, 0.25, 0.12))]
    contacts = []
    l_thigh = float(rng.uniform(0.35, 0.45))
    l_shin = float(rng.uniform(0.35, 0.45))
    foot_h = 0.05
    leg_masses = [mass() for _ in range(6)]
    for sy in (1.0, -1.0):
        b_yaw = len(bodies)
        bodies.append(dict(parent=0, axis=Z, jpos=(0.0, 0.1 * sy, -0.05), mass=leg_masses[0],
                           inertia=_sphere_inertia(leg_masses[0], 0.05), **jkw))
        b_roll = len(bodies)
        bodies.append(dict(parent=b_yaw, axis=X, jpos=(0.0, 0.0, -0.05), mass=leg_masses[1],
                           inertia=_sphere_inertia(leg_masses[1], 0.05), **jkw))
        b_thigh = len(bodies)
        bodies.append(dict(parent=b_roll, axis=Y, jpos=(0.0, 0.0, 0.0), mass=leg_masses[2],
                           com=(0.0, 0.0, -l_thigh / 2),
                           inertia=_rod_inertia(leg_masses[2], l_thigh, 0.05), **jkw))
        b_shin = len(bodies)
        bodies.append(dict(parent=b_thigh, axis=Y, jpos=(0.0, 0.0, -l_thigh), mass=leg_masses[3],
                           com=(0.0, 0.0, -l_shin / 2),
                           inertia=_rod_inertia(leg_masses[3], l_shin, 0.04), **jkw))
        b_ankle = len(bodies)
        bodies.append(dict(parent=b_shin, axis=Y, jpos=(0.0, 0.0, -l_shin), mass=leg_masses[4],
                           inertia=_sphere_inertia(leg_masses[4], 0.04), **jkw))
        b_foot = len(bodies)
        bodies.append(dict(parent=b_ankle, axis=X, jpos=(0.0, 0.0, 0.0), mass=leg_masses[5],
                           com=(0.03, 0.0, -foot_h / 2),
                           inertia=_box_inertia(leg_masses[5], 0.2, 0.08, foot_h), **jkw))
        for cx in (0.13, -0.07):
            for cy in (0.04, -0.04):
                contacts.append((b_foot, (cx, cy, -foot_h)))
    l_waist = length()
    m_torso = mass()
    l_torso = length()
    b_torso = len(bodies)
    bodies.append(dict(parent=0, axis=Z, jpos=(0.0, 0.0, l_waist / 2), mass=m_torso,
                       com=(0.0, 0.0, l_torso / 2),
                       inertia=_box_inertia(m_torso, 0.2, 0.3, max(l_torso, 0.1)), **jkw))
    l_upper, l_fore = length(), length()
    arm_masses = [mass() for _ in range(4)]
    for sy in (1.0, -1.0):
        b_sp = len(bodies)
        bodies.append(dict(parent=b_torso, axis=Y, jpos=(0.0, 0.18 * sy, l_torso), mass=arm_masses[0],
                           inertia=_sphere_inertia(arm_masses[0], 0.05), **jkw))
        b_sr = len(bodies)
        bodies.append(dict(parent=b_sp, axis=X, jpos=(0.0, 0.05 * sy, 0.0), mass=arm_masses[1],
                           inertia=_sphere_inertia(arm_masses[1], 0.05), **jkw))
        b_upper = len(bodies)
        bodies.append(dict(parent=b_sr, axis=Z, jpos=(0.0, 0.0, 0.0), mass=arm_masses[2],
                           com=(0.0, 0.0, -l_upper / 2),
                           inertia=_rod_inertia(arm_masses[2], l_upper, 0.04), **jkw))
        bodies.append(dict(parent=b_upper, axis=Y, jpos=(0.0, 0.0, -l_upper), mass=arm_masses[3],
                           com=(0.0, 0.0, -l_fore / 2),
                           inertia=_rod_inertia(arm_masses[3], l_fore, 0.035), **jkw))
    m = _finish("humanoid", bodies, contacts, contact_k=2.0e4, contact_c=200.0, mu=0.8, eps_f=eps_f,
                cost_body=b_torso, z_des=1.0, vx_des=0.3, w_z=1.0, w_vx=1.0, w_tilt=1.0,
                w_tau=1.0e-3)
    # standing pose: slight knee bend, arms down
    leg = [0.0, 0.0, -0.2, 0.4, -0.2, 0.0]
    q = leg + leg + [0.0] + [0.0, 0.0, 0.0, -0.3] + [0.0, 0.0, 0.0, -0.3]
    m.q_stand = np.array(q, dtype=np.float64)
    hip_drop = 0.05 + 0.05
    knee_drop = l_thigh * math.cos(0.2)
    shin_drop = l_shin * math.cos(0.2)
    total = float(m.mass.sum())
    m.base_z0 = hip_drop + knee_drop + shin_drop + foot_h - total * m.gravity / (8.0 * m.contact_k)
    return m


# --------------------------------------------------------------------------------------
# Tiny trees for the dynamics pins
# --------------------------------------------------------------------------------------
def pendulum(m: float = 1.3, lc: float = 0.4, ic: float = 0.02, armature: float = 0.0) -> RobotModel:
    """Fixed base + one link on a y-axis hinge, centre of mass lc below the hinge."""
    bodies = [dict(parent=-1, mass=1.0, inertia=_sphere_inertia(1.0, 0.1)),
              dict(parent=0, axis=(0.0, 1.0, 0.0), jpos=(0.0, 0.0, 0.0), mass=m,
                   com=(0.0, 0.0, -lc), inertia=np.array([ic, ic, ic, 0, 0, 0.0]),
                   armature=armature)]
    return _finish("pendulum", bodies, [], fixed_base=True, w_tau=0.0)


def chain2(seed: int = 11) -> RobotModel:
    """Fixed base + 2 links with skewed axes and offset centres of mass."""
    rng = np.random.default_rng(seed)
    a1 = rng.normal(size=3)
    a2 = rng.normal(size=3)
    bodies = [dict(parent=-1, mass=1.0, inertia=_sphere_inertia(1.0, 0.1)),
              dict(parent=0, axis=tuple(a1 / np.linalg.norm(a1)), jpos=(0.05, -0.02, 0.1),
                   mass=1.7, com=tuple(rng.normal(scale=0.1, size=3)),
                   inertia=np.array([0.03, 0.02, 0.025, 0.002, -0.001, 0.0015]), armature=0.01),
              dict(parent=1, axis=tuple(a2 / np.linalg.norm(a2)), jpos=(0.0, 0.1, -0.3),
                   mass=0.9, com=tuple(rng.normal(scale=0.1, size=3)),
                   inertia=np.array([0.012, 0.018, 0.01, -0.001, 0.0005, 0.002]), armature=0.02)]
    return _finish("chain2", bodies, [], fixed_base=True, w_tau=0.0)


def random_tree(nb: int = 32, nc: int = 32, seed: int = 17, fixed_base: bool = False) -> RobotModel:
    """A floating (or fixed) base with nb - 1 revolute bodies on a random tree (each body's
    parent drawn among the earlier ones), skewed unit axes, random offsets, masses and
    inertias, and nc contact points on random bodies: the largest model the library
    accepts at nb = nc = 32."""
    rng = np.random.default_rng(seed)
    bodies = [dict(parent=-1, mass=float(rng.uniform(2.0, 6.0)), com=tuple(rng.normal(scale=0.02, size=3)),
                   inertia=_box_inertia(4.0, 0.3, 0.2, 0.1))]
    for b in range(1, nb):
        a = rng.normal(size=3)
        ms = float(rng.uniform(0.2, 1.5))
        bodies.append(dict(parent=int(rng.integers(0, b)), axis=tuple(a / np.linalg.norm(a)),
                           jpos=tuple(rng.normal(scale=0.08, size=3)), mass=ms,
                           com=tuple(rng.normal(scale=0.04, size=3)),
                           inertia=_sphere_inertia(ms, float(rng.uniform(0.03, 0.08))),
                           armature=0.05, kp=20.0, kd=0.8, tau_max=30.0))
    contacts = [(int(rng.integers(0, nb)), tuple(rng.normal(scale=0.05, size=3))) for _ in range(nc)]
    m = _finish(f"random_tree_{nb}", bodies, contacts, fixed_base=fixed_base, contact_k=2.0e4, contact_c=200.0,
                mu=0.8, eps_f=1.5, z_des=0.5, vx_des=0.0, w_z=1.0, w_vx=0.5, w_tilt=0.5, w_tau=1e-3)
    m.q_stand = np.zeros(nb - 1)
    m.base_z0 = 0.5
    return m


def free_body(m: float = 2.5) -> RobotModel:
    """A single floating rigid body with an asymmetric inertia and an offset centre of mass."""
    bodies = [dict(parent=-1, mass=m, com=(0.03, -0.02, 0.05),
                   inertia=np.array([0.05, 0.08, 0.11, 0.004, -0.003, 0.002]))]
    return _finish("free_body", bodies, [], w_tau=0.0)


def branch3(seed: int = 5) -> RobotModel:
    """Floating base with two children on skewed hinges (a 3-body branch)."""
    rng = np.random.default_rng(seed)
    bodies = [dict(parent=-1, mass=3.0, com=(0.01, 0.02, -0.01),
                   inertia=np.array([0.04, 0.05, 0.06, 0.003, 0.001, -0.002]))]
    for k in range(2):
        a = rng.normal(size=3)
        bodies.append(dict(parent=0, axis=tuple(a / np.linalg.norm(a)),
                           jpos=tuple(rng.normal(scale=0.15, size=3)), mass=float(rng.uniform(0.5, 1.5)),
                           com=tuple(rng.normal(scale=0.08, size=3)),
                           inertia=np.array([0.01, 0.012, 0.008, 0.001, -0.0005, 0.0007]),
                           armature=0.01, kp=10.0, kd=0.5, tau_max=20.0))
    return _finish("branch3", bodies, [], w_tau=0.0)


def point_mass(m: float = 1.0, k: float = 2.0e4, c: float = 200.0, mu: float = 0.8,
               eps_f: float = 0.1) -> RobotModel:
    """A floating point-like mass (tiny inertia) with one contact at its centre of mass."""
    bodies = [dict(parent=-1, mass=m, inertia=_sphere_inertia(m, 0.05))]
    return _finish("point_mass", bodies, [(0, (0.0, 0.0, 0.0))], contact_k=k, contact_c=c, mu=mu,
                   eps_f=eps_f, w_tau=0.0)


# --------------------------------------------------------------------------------------
# The modular cost of Sec. IV-A with the weight sets of Tab. II
# --------------------------------------------------------------------------------------
# (w_h, w_orient, w_q, w_c,vel, w_c,force, w_H) per task, Tab. II
TAB2_WEIGHTS = {
    "walking": (1e2, 10.0, 0.0, 0.5, 5e-2, 2.5e3),
    "jumping": (1.0, 0.5, 0.3, 1.0, 5e-4, 2e3),
    "handstand": (50.0, 10.0, 0.3, 1.0, 5e-4, 0.0),
    "backflip": (1.0, 0.5, 0.3, 1.0, 5e-4, 2e3),
    "bipedal": (10.0, 1.0, 0.3, 1.0, 5e-4, 2e2),
}


def with_paper_cost(m: RobotModel, task: str, pdot_des=(0.0, 0.0, 0.0), z_des: float | None = None,
                    quat_des=(1.0, 0.0, 0.0, 0.0), keep_quadratic: bool = False) -> RobotModel:
    """A copy of m costed by the modular running and terminal cost with Tab. II's weights
    for `task`; f0 is the standing load per contact point (total weight / nc, vertical)
    and the quadratic terms are switched off unless keep_quadratic."""
    w = TAB2_WEIGHTS[task]
    total = float(np.sum(m.mass)) * m.gravity
    kw = dict(w_h=w[0], w_orient=w[1], w_q=w[2], w_cvel=w[3], w_cforce=w[4], w_term=w[5],
              quat_des=tuple(float(v) for v in quat_des), pdot_des=tuple(float(v) for v in pdot_des),
              f0=(0.0, 0.0, total / max(m.nc, 1)))
    if z_des is not None:
        kw["z_des"] = float(z_des)
    if not keep_quadratic:
        kw.update(w_z=0.0, w_vx=0.0, w_tilt=0.0, w_tau=0.0)
    return dataclasses.replace(m, name=m.name + "_" + task, **kw)


MODELS = {"quadruped": quadruped, "humanoid": humanoid, "pendulum": pendulum, "chain2": chain2,
          "free_body": free_body, "branch3": branch3, "point_mass": point_mass, "random_tree": random_tree}


# --------------------------------------------------------------------------------------
# States, knots and schedules
# --------------------------------------------------------------------------------------
def standing_state(model: RobotModel, jitter: float = 0.0, base_vel: float = 0.0,
                   seed: int = 2) -> np.ndarray:
    """Standing pose (+ seeded U(-jitter, jitter) on joint q, U(-base_vel, base_vel) on
    each body-frame base linear velocity component)."""
    rng = np.random.default_rng(seed)
    nj = model.nj
    x = np.zeros(model.nx, dtype=np.float64)
    x[2] = model.base_z0
    x[3] = 1.0
    q0 = model.q_stand if model.q_stand is not None else np.zeros(nj)
    x[7:7 + nj] = q0 + (rng.uniform(-jitter, jitter, size=nj) if jitter > 0 else 0.0)
    if base_vel > 0:
        x[model.nq:model.nq + 3] = rng.uniform(-base_vel, base_vel, size=3)
    return x


def random_state(model: RobotModel, seed: int, q_scale: float = 0.5, v_scale: float = 1.0,
                 height: float = 0.5) -> np.ndarray:
    """A generic seeded state (random unit quaternion, joint angles and velocities)."""
    rng = np.random.default_rng(seed)
    x = np.zeros(model.nx, dtype=np.float64)
    x[0:3] = rng.normal(scale=0.1, size=3) + np.array([0.0, 0.0, height])
    qu = rng.normal(size=4)
    x[3:7] = qu / np.linalg.norm(qu)
    nj = model.nj
    x[7:7 + nj] = rng.uniform(-q_scale, q_scale, size=nj)
    x[model.nq:model.nq + 6] = rng.normal(scale=v_scale, size=6)
    x[model.nq + 6:] = rng.normal(scale=v_scale, size=nj)
    return x


def nominal_knots(model: RobotModel, nk: int) -> np.ndarray:
    """theta^q = standing pose, theta^v = 0 (Alg. 1 initialisation). Shape [nk, 2, nu]."""
    k = np.zeros((nk, 2, model.nj), dtype=np.float64)
    q0 = model.q_stand if model.q_stand is not None else np.zeros(model.nj)
    k[:, 0, :] = q0
    return k


def linear_sigma(nk: int, iters: int = 1, lo: float = 0.05, hi: float = 0.3) -> np.ndarray:
    """Per-knot standard deviation growing linearly lo -> hi, identical for every
    iteration. Shape [iters, nk]."""
    row = lo + (hi - lo) * np.arange(nk) / max(nk - 1, 1)
    return np.tile(row, (iters, 1))


def random_knots(model: RobotModel, n: int, nk: int, seed: int, scale: float = 0.3) -> np.ndarray:
    """Seeded knots around the standing pose, shape [n, nk, 2, nu]."""
    rng = np.random.default_rng(seed)
    base = nominal_knots(model, nk)
    noise = rng.normal(size=(n, nk, 2, model.nj)) * scale
    noise[:, :, 1, :] *= 3.0
    return base[None] + noise


# --------------------------------------------------------------------------------------
# Workloads (configurations of the plain, scale, humanoid, batched and serving runs)
# --------------------------------------------------------------------------------------
@dataclasses.dataclass
class Problem:
    model: RobotModel
    n: int            # samples (sample 0 is the unperturbed nominal)
    nk: int           # knots
    horizon: int      # simulation steps H
    iters: int        # MPPI iterations per solve
    dt: float
    lam: float
    sigma: np.ndarray  # [iters, nk]
    state: np.ndarray  # [nx]
    nominal: np.ndarray  # [nk, 2, nu]
    seed: int = 1
    instance: int = 0


def plain_quadruped(seed_noise: int = 1, seed_jitter: int = 2, n: int = 32) -> Problem:
    """Plain single iteration: 32 samples, 4 knots over 0.5 s, dt 0.01, lambda 0.1."""
    m = quadruped()
    return Problem(model=m, n=n, nk=4, horizon=50, iters=1, dt=0.01, lam=0.1,
                   sigma=linear_sigma(4, 1), state=standing_state(m, jitter=0.02, seed=seed_jitter),
                   nominal=nominal_knots(m, 4), seed=seed_noise)


def scale_quadruped(n: int = 8192, seed_state: int = 20, seed_noise: int = 1) -> Problem:
    """Single-instance scale: 6 knots over 1.0 s, dt 0.005 (200 steps), 3 iterations,
    random base velocity U(-0.5, 0.5) m/s per component."""
    m = quadruped()
    return Problem(model=m, n=n, nk=6, horizon=200, iters=3, dt=0.005, lam=0.1,
                   sigma=linear_sigma(6, 3),
                   state=standing_state(m, jitter=0.02, base_vel=0.5, seed=seed_state),
                   nominal=nominal_knots(m, 6), seed=seed_noise)


def paper_walking(n: int = 8192, v: float = 0.5, seed_state: int = 20, seed_noise: int = 1) -> Problem:
    """The scale workload (6 knots over 1.0 s, dt 0.005, 3 iterations) costed by the
    modular cost with Tab. II's walking weights, forward target velocity v."""
    p = scale_quadruped(n=n, seed_state=seed_state, seed_noise=seed_noise)
    p.model = with_paper_cost(p.model, "walking", pdot_des=(v, 0.0, 0.0))
    return p


def humanoid_problem(n: int = 2048, seed_noise: int = 3) -> Problem:
    """Humanoid tree: 2048 samples, 8 knots over 1.0 s, dt 0.005 (200 steps)."""
    m = humanoid()
    return Problem(model=m, n=n, nk=8, horizon=200, iters=1, dt=0.005, lam=0.1,
                   sigma=linear_sigma(8, 1), state=standing_state(m, jitter=0.02, seed=4),
                   nominal=nominal_knots(m, 8), seed=seed_noise)


def batched_problems(count: int = 256, seed: int = 1000, quad_frac: float = 0.7,
                     n_lo: int = 64, n_hi: int = 2048, h_lo: int = 50, h_hi: int = 200,
                     dt: float = 0.005) -> list:
    """Uneven independent instances: 70 % quadruped / 30 % humanoid, samples
    log-uniform in [n_lo, n_hi], horizons U{h_lo..h_hi}, knots U{4..8}, lambda
    U(0.05, 0.5), linear sigma 0.05 -> 0.3, one iteration each. Instance i draws from
    seed + i."""
    quad = quadruped()
    hum = humanoid()
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed + i)
        m = quad if rng.random() < quad_frac else hum
        n = int(math.floor(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        h = int(rng.integers(h_lo, h_hi + 1))
        nk = int(rng.integers(4, 9))
        lam = float(rng.uniform(0.05, 0.5))
        st = standing_state(m, jitter=0.02, seed=seed + i)
        out.append(Problem(model=m, n=n, nk=nk, horizon=h, iters=1, dt=dt, lam=lam,
                           sigma=linear_sigma(nk, 1), state=st, nominal=nominal_knots(m, nk),
                           seed=seed + i, instance=i))
    return out

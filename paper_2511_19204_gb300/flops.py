"""Algorithmic floating-point work of one rollout step of one sample (one unit).

Counted from the formulation the kernels evaluate (articulated-body algorithm with
spatial quantities split into 3-vector / 3x3 blocks, symmetric 6x6 inertias stored as
21 numbers), per primitive, with a fused multiply-add counted as 2 flops and an add,
multiply, divide, square root, sine/cosine pair or arctangent as 1. The same numbers
are derived in the design notes; they do not depend on the lane mapping.

Per joint body (revolute):
  Hermite setpoint + derivative (Eq. hermite_segment) + PD (Eq. pd-controller)   55
  joint rotation (sincos + Rodrigues)                                            31
  pass 1: world rotation 45, origin 18, angular 21 and linear 27 velocity       111
  velocity product c                                                             21
  bias force v x* (I v)                                                          78
  pass 2: U, D, u (28), articulated inertia update (63), Ia c (66),
          bias update (24), congruence X^T Ia X (342), force transform (42)     565
  child -> parent accumulation                                                   27
  pass 3: acceleration transform (48), joint acceleration (13), update (6)       67
  semi-implicit Euler                                                             4
  effort term tau^2                                                               2
Per contact point in penetration: position 18, velocity 27, normal force 4,
  regularised friction 12, body-frame force 15, moment 12                       88
Per floating base: rotation from quaternion 25, bias 78, 6x6 Cholesky solve 161,
  gravity 6, integration 94 (velocities 12, position 21, quaternion exponential
  and product 61), running cost 42                                              406
With the modular cost of Sec. IV-A on (any of its weights non-zero), in addition:
  per joint: (q - q0)^2 weighted and accumulated                                   4
  per contact point: ||v_c||_1 5, ||f_c - f0||_1 8, weights and accumulation 4    17
  per base: height term 3, R^T R_des 54, rotation angle (vee 3, norm 6, trace 3,
  arctangent 1), theta^2 term 2, reduction 3                                      75
  (the terminal term, ~15 flops per rollout, is not counted per step)
Quadrupeds whose chains turn about +x, +y, +y (hip in the base's xy-plane, thigh joint
along y from the hip, knee along z from the thigh) run the specialised chain kernel, which
applies joint rotations to two components, forms products with the offsets from their
non-zero components only, skips the zero component of the velocity product, reuses U / D
in the projection, computes the leaf's projection once per rollout and evaluates each
setpoint from a power-basis form of its segment (formed once per segment). Per step:
  hip   (x axis, offset in the xy-plane, has a child): setpoint + PD 20 (qref 6, vref 5,
        PD 5, clamp 2, segment form amortised ~0), sincos 1, pass 1 51 (composition 18,
        origin 12, angular velocity 7, linear velocity 14), velocity product 4, bias 78,
        child accumulation 27, pass 2 306 (D and u 3, projection 48, bias products and
        update 61, congruence 174 = rotations 108 + shift 66, force transform 20), pass 3
        40, Euler 4, effort 2                                                        533
  thigh (y axis, offset along y, has a child): pass 1 41 (origin 6, linear velocity
        10), shift 32, force transform 16, pass 3 36, the rest as the hip               481
  calf  (y axis, offset along z, leaf): as the thigh without the child accumulation,
        D and the projection (u 1 instead of 3 + 48)                                  404
Humanoids of the usual layout (legs turning about z, x, y, y, y, x; a waist about z; arms
about y, x, z, y; offsets in the yz-plane, on one axis or zero) run the two-warp split
kernel with the same specialisations; a zero offset drops the origin, the offset cross
products and the congruence shift, and every body evaluates its setpoint from the
power-basis form of its segment (20). Per step:
  leg:   yaw 533, roll 481, thigh 431, shin 481, ankle 481, foot (leaf) 354           2761
  arm:   shoulder pitch 533, shoulder roll 481, upper arm 431, forearm (leaf) 404    1849
  waist: two children (54), offset along z                                             508

The method's own count (the FP64 oracle with an operation-counting scalar type, at the end
of this file) is the roofline's numerator; these per-primitive counts of the kernels'
formulations are reported beside it.
"""
from __future__ import annotations

PER_JOINT = 55 + 31 + 111 + 21 + 78 + 565 + 27 + 67 + 4 + 2
PER_CONTACT = 18 + 27 + 4 + 12 + 15 + 12
PER_BASE_SOLVE = 161 + 6   # 6x6 Cholesky solve and the gravity offset
PER_BASE = 25 + 78 + 161 + 6 + 94 + 42
MOD_JOINT = 4
MOD_CONTACT = 5 + 8 + 4
MOD_BASE = 3 + 54 + 3 + 6 + 3 + 1 + 2 + 3
MOD_WEIGHTS = ("w_h", "w_orient", "w_q", "w_cvel", "w_cforce", "w_term")
PER_JOINT_XYY_HIP = 20 + 1 + 51 + 4 + 78 + 27 + (3 + 48 + 61 + 174 + 20) + 40 + 4 + 2
PER_JOINT_XYY_THIGH = 20 + 1 + 41 + 4 + 78 + 27 + (3 + 48 + 61 + 140 + 16) + 36 + 4 + 2
PER_JOINT_XYY_CALF = 20 + 1 + 41 + 4 + 78 + 0 + (1 + 0 + 61 + 140 + 16) + 36 + 4 + 2

# split humanoid kernel: (setpoint, pass 1, child accumulation, pass 2, pass 3) per body,
# each plus sincos 1, velocity product 4, bias 78, Euler 4, effort 2
_SPLIT_FIXED = 1 + 4 + 78 + 4 + 2
PER_JOINT_HUM_LEG = [20 + 51 + 27 + 306 + 40, 20 + 41 + 27 + 268 + 36, 20 + 31 + 27 + 232 + 32,
                     20 + 41 + 27 + 268 + 36, 20 + 41 + 27 + 268 + 36, 20 + 31 + 0 + 182 + 32]
PER_JOINT_HUM_ARM = [20 + 51 + 27 + 306 + 40, 20 + 41 + 27 + 268 + 36, 20 + 31 + 27 + 232 + 32,
                     20 + 41 + 0 + 218 + 36]
PER_JOINT_HUM_WAIST = 20 + 41 + 54 + 268 + 36


def axis_plan_hum(model) -> bool:
    """True when the model runs the two-warp split kernel: a floating base with 2 legs of 6
    bodies, a waist body on the base carrying 2 arms of 4, axes and offsets as above,
    contact points only on the feet and the cost body not on a leg."""
    import numpy as np
    if model.fixed_base or model.nb != 22:
        return False
    e = np.eye(3)
    par = list(model.parent)
    if par[13] != 0 or any(par[1 + 6 * l] != 0 for l in range(2)) or any(par[14 + 4 * l] != 13 for l in range(2)):
        return False

    def chain(b0, n):
        return all(par[b0 + j] == b0 + j - 1 for j in range(1, n))

    def off(b, kind):   # kind: axis index, "yz" or "zero"
        r = model.jpos[b]
        if kind == "zero":
            return not np.any(r)
        if kind == "yz":
            return r[0] == 0.0
        return all(r[i] == 0.0 for i in range(3) if i != kind)

    legs = [(2, "yz"), (0, 2), (1, "zero"), (1, 2), (1, 2), (0, "zero")]
    arms = [(1, "yz"), (0, 1), (2, "zero"), (1, 2)]
    for b0, plan in [(1, legs), (7, legs), (14, arms), (18, arms)]:
        if not chain(b0, len(plan)):
            return False
        for j, (ax, kind) in enumerate(plan):
            if not (np.array_equal(model.axis[b0 + j], e[ax]) and off(b0 + j, kind)):
                return False
    feet = {6, 12}
    return bool(np.array_equal(model.axis[13], e[2]) and off(13, 2)
                and all(int(b) in feet for b in model.contact_body) and not 1 <= model.cost_body <= 12)


def axis_plan_xyy(model) -> bool:
    """True when the model runs the axis-specialised chain kernel: a floating base with 4
    chains of 3 bodies whose joint axes are exactly +x, +y, +y, with the hip in the base's
    xy-plane, the thigh joint along y from the hip, the knee along z from the thigh, and
    contact points only on the calves."""
    import numpy as np
    if model.fixed_base or model.nb != 13:
        return False
    ex, ey = np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0])
    for leg in range(4):
        b0 = 1 + 3 * leg
        if list(model.parent[b0:b0 + 3]) != [0, b0, b0 + 1]:
            return False
        if not (np.array_equal(model.axis[b0], ex) and np.array_equal(model.axis[b0 + 1], ey)
                and np.array_equal(model.axis[b0 + 2], ey)):
            return False
        if model.jpos[b0][2] != 0.0:
            return False
        if model.jpos[b0 + 1][0] != 0.0 or model.jpos[b0 + 1][2] != 0.0:
            return False
        if model.jpos[b0 + 2][0] != 0.0 or model.jpos[b0 + 2][1] != 0.0:
            return False
    calves = {3, 6, 9, 12}
    return all(int(b) in calves for b in model.contact_body)


def flops_per_step(model, contacts_active=None, mapping_chain=True) -> int:
    """Flops of one step of one sample. ``contacts_active`` defaults to every contact
    point (the standing / walking regime); pass a number for another regime.
    ``mapping_chain``: the rollout runs the lanes-per-chain kernel (which specialises the
    axes of x, y, y quadrupeds and of the usual humanoid layout)."""
    nc = model.nc if contacts_active is None else contacts_active
    if mapping_chain and axis_plan_xyy(model):
        joints = 4 * (PER_JOINT_XYY_HIP + PER_JOINT_XYY_THIGH + PER_JOINT_XYY_CALF)
    elif mapping_chain and axis_plan_hum(model):
        joints = (2 * sum(PER_JOINT_HUM_LEG) + 2 * sum(PER_JOINT_HUM_ARM) + PER_JOINT_HUM_WAIST
                  + 21 * _SPLIT_FIXED)
    else:
        joints = PER_JOINT * model.nj
    f = joints + PER_CONTACT * nc + PER_BASE
    if any(getattr(model, w, 0.0) for w in MOD_WEIGHTS):
        f += MOD_JOINT * model.nj + MOD_CONTACT * model.nc + MOD_BASE
    return f


# Algorithmic work per step-sample as the method specifies it: the FP64 oracle (which
# restates Alg. 1's rollout with dense 6x6 spatial algebra) run with an operation-counting
# scalar type on the workloads' own samples (16 of each, the configurations' seeds),
# averaged per step. "dense" counts every operation (add/sub, mul, div, sqrt and the
# elementary functions one each; a multiply-add is two); "nontrivial" leaves out those
# whose result a structural operand fixes (an added 0, a factor 0 or +-1, a divisor +-1):
# multiplying by the zeros of a 6x6 spatial transform is not work of the algorithm, and
# the dense figure divided by the measured rollout time would exceed the FP32 peak.
# The non-trivial figure is the roofline's numerator; the kernels' own formulations
# (above) do a little less (they hoist the model-constant body inertias and form 1 / D
# once per body where the oracle divides per element).
METHOD_FLOPS = {
    # workload: (dense, nontrivial) per step-sample
    "scale_quadruped": (24157.7, 6767.4),
    "plain_quadruped": (24173.9, 6747.7),
    "humanoid": (41946.6, 13160.5),
}


def method_flops_per_step(workload: str):
    """(dense, nontrivial) oracle operation counts per step-sample of a workload, or None."""
    return METHOD_FLOPS.get(workload)


def fp32_peak_tflops(sms: int = 152, clock_mhz: float = 2070.0) -> float:
    """FP32 ALU peak: SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return sms * 128 * 2 * clock_mhz * 1e6 / 1e12

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
"""
from __future__ import annotations

PER_JOINT = 55 + 31 + 111 + 21 + 78 + 565 + 27 + 67 + 4 + 2
PER_CONTACT = 18 + 27 + 4 + 12 + 15 + 12
PER_BASE = 25 + 78 + 161 + 6 + 94 + 42
MOD_JOINT = 4
MOD_CONTACT = 5 + 8 + 4
MOD_BASE = 3 + 54 + 3 + 6 + 3 + 1 + 2 + 3
MOD_WEIGHTS = ("w_h", "w_orient", "w_q", "w_cvel", "w_cforce", "w_term")
PER_JOINT_XYY_HIP = 20 + 1 + 51 + 4 + 78 + 27 + (3 + 48 + 61 + 174 + 20) + 40 + 4 + 2
PER_JOINT_XYY_THIGH = 20 + 1 + 41 + 4 + 78 + 27 + (3 + 48 + 61 + 140 + 16) + 36 + 4 + 2
PER_JOINT_XYY_CALF = 20 + 1 + 41 + 4 + 78 + 0 + (1 + 0 + 61 + 140 + 16) + 36 + 4 + 2


def axis_plan_xyy(model) -> bool:
    """True when the model runs the axis-specialised chain kernel: a floating base with 4
    chains of 3 bodies whose joint axes are exactly +x, +y, +y, with the hip in the base's
    xy-plane, the thigh joint along y from the hip and the knee along z from the thigh."""
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
    return True


def flops_per_step(model, contacts_active=None, mapping_chain=True) -> int:
    """Flops of one step of one sample. ``contacts_active`` defaults to every contact
    point (the standing / walking regime); pass a number for another regime.
    ``mapping_chain``: the rollout runs the lanes-per-chain kernel (which specialises the
    axes of x, y, y quadrupeds)."""
    nc = model.nc if contacts_active is None else contacts_active
    if mapping_chain and axis_plan_xyy(model):
        joints = 4 * (PER_JOINT_XYY_HIP + PER_JOINT_XYY_THIGH + PER_JOINT_XYY_CALF)
    else:
        joints = PER_JOINT * model.nj
    f = joints + PER_CONTACT * nc + PER_BASE
    if any(getattr(model, w, 0.0) for w in MOD_WEIGHTS):
        f += MOD_JOINT * model.nj + MOD_CONTACT * model.nc + MOD_BASE
    return f


def fp32_peak_tflops(sms: int = 152, clock_mhz: float = 2070.0) -> float:
    """FP32 ALU peak: SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return sms * 128 * 2 * clock_mhz * 1e6 / 1e12

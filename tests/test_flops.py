"""Flop counts behind the roofline figures: the specialised kernels' per-body totals and
which models they apply to (a perturbed axis or offset falls back to the generic count)."""
import numpy as np

from paper_2511_19204_gb300 import flops as F
from paper_2511_19204_gb300 import synth as S


def test_quadruped_counts():
    q = S.quadruped()
    assert F.axis_plan_xyy(q)
    assert F.PER_JOINT_XYY_HIP + F.PER_JOINT_XYY_THIGH + F.PER_JOINT_XYY_CALF == 533 + 481 + 404
    assert F.flops_per_step(q) == 4 * (533 + 481 + 404) + 4 * F.PER_CONTACT + F.PER_BASE == 6430
    assert F.flops_per_step(q, mapping_chain=False) == 12 * F.PER_JOINT + 4 * F.PER_CONTACT + F.PER_BASE


def test_humanoid_counts():
    h = S.humanoid()
    assert F.axis_plan_hum(h) and not F.axis_plan_xyy(h)
    fixed = F._SPLIT_FIXED
    assert [c + fixed for c in F.PER_JOINT_HUM_LEG] == [568, 516, 466, 516, 516, 389]
    assert [c + fixed for c in F.PER_JOINT_HUM_ARM] == [533, 481, 431, 404]
    assert F.PER_JOINT_HUM_WAIST + fixed == 508
    assert F.flops_per_step(h) == 2 * 2971 + 2 * 1849 + 508 + 8 * F.PER_CONTACT + F.PER_BASE == 11258
    assert F.flops_per_step(h, mapping_chain=False) == 21 * F.PER_JOINT + 8 * F.PER_CONTACT + F.PER_BASE


def test_perturbed_layouts_use_the_generic_count():
    h = S.humanoid()
    axis = h.axis.copy()
    axis[1] = np.array([0.05, 0.0, 1.0]) / np.linalg.norm([0.05, 0.0, 1.0])
    jpos = h.jpos.copy()
    jpos[h.nb - 1, 0] = 0.01
    jpos2 = h.jpos.copy()
    jpos2[3, 2] = 0.02          # the thigh joint's offset must be zero
    for m in (h.copy(axis=axis), h.copy(jpos=jpos), h.copy(jpos=jpos2)):
        assert not F.axis_plan_hum(m)
        assert F.flops_per_step(m) == 21 * F.PER_JOINT + 8 * F.PER_CONTACT + F.PER_BASE
    hand = h.copy(contact_body=np.append(h.contact_body, h.nb - 1).astype(np.int32),
                  contact_pos=np.vstack([h.contact_pos, [0.0, 0.0, -0.2]]))
    assert not F.axis_plan_hum(hand)
    assert not F.axis_plan_hum(h.copy(cost_body=4))
    assert F.axis_plan_hum(h.copy(cost_body=0))
    q = S.quadruped()
    jq = q.jpos.copy()
    jq[1, 2] = 0.01
    assert not F.axis_plan_xyy(q.copy(jpos=jq))
    thigh = q.copy(contact_body=np.append(q.contact_body, 2).astype(np.int32),
                   contact_pos=np.vstack([q.contact_pos, [0.0, 0.0, -0.1]]))
    assert not F.axis_plan_xyy(thigh)

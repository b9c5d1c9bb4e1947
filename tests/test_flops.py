"""Flop counts behind the roofline figures: the specialised kernels' per-body totals and
which models they apply to (a perturbed axis or offset falls back to the generic count)."""
import numpy as np
import pytest

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
    assert [c + fixed for c in F.PER_JOINT_HUM_LEG] == [533, 481, 431, 481, 481, 354]
    assert [c + fixed for c in F.PER_JOINT_HUM_ARM] == [533, 481, 431, 404]
    assert F.PER_JOINT_HUM_WAIST + fixed == 508
    assert F.flops_per_step(h) == 2 * 2761 + 2 * 1849 + 508 + 8 * F.PER_CONTACT + F.PER_BASE == 10838
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


# ------------------------------------------------------------------------------------
# The method's own count: the FP64 oracle with an operation-counting scalar type
# ------------------------------------------------------------------------------------
def _workload_counts(orc, p, nsamp=16):
    """Per-step (dense, nontrivial) counts over nsamp samples of a workload, and the
    per-phase breakdown [phase][kind]."""
    kn = orc.sample_knots(p.model.nj, p.nk, p.n, p.horizon, p.dt, p.nominal, p.sigma[0], seed=p.seed)
    per = np.zeros((len(orc.PHASES), len(orc.OP_KINDS)))
    for i in range(nsamp):
        _, cnt = orc.count_rollout(p.model, p.state, kn[i], p.horizon, p.dt)
        per += cnt / p.horizon
    per /= nsamp
    dense = per[:, :5].sum()
    return dense, dense - per[:, 6:9].sum(), per


def test_counting_build_runs_the_oracle(orc):
    # the counting build evaluates the same arithmetic: identical rollout costs
    for p in (S.scale_quadruped(n=8), S.humanoid_problem(n=8)):
        p.horizon = 40
        kn = orc.sample_knots(p.model.nj, p.nk, p.n, p.horizon, p.dt, p.nominal, p.sigma[0], seed=p.seed)
        for i in range(3):
            c, _ = orc.count_rollout(p.model, p.state, kn[i], p.horizon, p.dt)
            ref, _ = orc.rollout(p.model, p.state, kn[i], p.horizon, p.dt)
            assert c == ref


def test_counts_are_linear_in_the_tree(orc):
    # the articulated-body algorithm is O(bodies): without contacts, the dense count of a
    # step grows by the same amount for each added body of a random tree, and a joint costs
    # the same in every phase wherever it sits
    counts = {}
    for nb in (5, 9, 13):
        m = S.random_tree(nb=nb, nc=0, seed=3)
        x0 = S.random_state(m, seed=1)
        kn = S.random_knots(m, 1, 4, seed=2)[0]
        _, cnt = orc.count_rollout(m, x0, kn, 10, 0.005)
        counts[nb] = cnt / 10
    d1 = counts[9] - counts[5]
    d2 = counts[13] - counts[9]
    dense = slice(0, 5)
    np.testing.assert_allclose(d1[:, dense], d2[:, dense], atol=1e-9)
    per_body = d1[:, dense].sum() / 4
    print(f"dense operations per added body per step: {per_body:.0f}")
    assert 1500 < per_body < 2500


def test_stored_method_counts_reproduce(orc):
    for name, p in (("scale_quadruped", S.scale_quadruped(n=64)), ("plain_quadruped", S.plain_quadruped()),
                    ("humanoid", S.humanoid_problem(n=64))):
        dense, nontrivial, _ = _workload_counts(orc, p)
        sd, sn = F.method_flops_per_step(name)
        assert dense == pytest.approx(sd, abs=0.06) and nontrivial == pytest.approx(sn, abs=0.06), name


def test_kernel_counts_against_the_method(orc):
    # phase by phase, the specialised kernels' own counts (the formulation they evaluate)
    # against the oracle's non-trivial operations: the kernels do less where they hoist
    # model constants (body inertias, a body's 1 / D instead of a division per element of
    # the rank-one update) and evaluate setpoints from a power basis; they never do less
    # than half, and the totals agree within 25 % (quadruped 5 %, humanoid 21 %)
    for name, p, kernel in (("scale_quadruped", S.scale_quadruped(n=64), 6430),
                            ("humanoid", S.humanoid_problem(n=64), 10838)):
        dense, nontrivial, per = _workload_counts(orc, p)
        assert F.flops_per_step(p.model) == kernel
        assert kernel <= nontrivial <= dense / 3
        assert nontrivial / kernel < 1.25
        # the base's 6x6 solve: the same Cholesky work (the kernel counts 161 with gravity)
        solve = per[orc.PHASES.index("solve"), :5].sum() - per[orc.PHASES.index("solve"), 6:9].sum()
        assert abs(solve - F.PER_BASE_SOLVE) < 0.1 * F.PER_BASE_SOLVE
        # the oracle's rank-one update divides every element by D; the kernel multiplies by 1 / D
        pass2 = orc.PHASES.index("pass2")
        assert per[pass2, 2] == pytest.approx(42 * p.model.nj, abs=0.5)

"""Small cases of every kernel family, run by test_gpu_check.py in a child process whose
MPPI_LIBRARY is the bounds-check build: each result against the FP64 oracle (or the
product's own bit-exact relations), then the check word. Prints one JSON line."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2511_19204_gb300 import mppi as M  # noqa: E402
from paper_2511_19204_gb300 import synth as S  # noqa: E402


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))))


def solve_case(p, mapping):
    c = M.Controller.from_problem(M.Model(p.model), p, mapping=mapping)
    warm = p.nominal.astype(np.float32)
    mean, _, info = c.solve(p.state, warm=warm)
    ref = oracle.solve(p.model, p.n, p.nk, p.horizon, p.iters, p.dt, p.lam, p.sigma, p.state,
                       warm.astype(np.float64), seed=p.seed, inst=p.instance)
    return rel(mean, ref["mean"])


def main():
    import ctypes as C
    L = M.load()
    out = {"library": os.path.basename(M.LIB_PATH)}
    w = C.c_uint32(0)
    L.mppi_check_word(C.byref(w), 1)             # start clean
    q = S.scale_quadruped(n=256)
    q.horizon = 60
    out["quadruped_solve"] = solve_case(q, M.MPPI_MAP_CHAIN)
    out["quadruped_solve_warp"] = solve_case(q, M.MPPI_MAP_WARP)
    h = S.humanoid_problem(n=64)
    h.horizon = 60
    out["humanoid_split_solve"] = solve_case(h, M.MPPI_MAP_CHAIN)
    for K in (4000, 12000):                      # the cooperative and the group-by-group finish
        p = S.scale_quadruped(n=K)
        p.horizon, p.iters, p.sigma = 20, 2, p.sigma[:2]
        out[f"quadruped_solve_K{K}"] = solve_case(p, M.MPPI_MAP_CHAIN)
    # batched: uneven instances, every rollout variant, bit-equal to single solves
    specs = [(S.quadruped(), 2, 97, 60, 4), (S.quadruped(), 1, 33, 50, 5), (S.quadruped(), 0, 40, 40, 4),
             (S.humanoid(), 2, 129, 30, 7), (S.humanoid(), 0, 70, 50, 8)]
    mods = {}
    alone, batch, states = [], [], []
    for i, (rob, mp, K, H, nk) in enumerate(specs):
        mod = mods.setdefault(rob.name, M.Model(rob))
        kw = dict(iters=1, dt=0.005, seed=10 + i, instance=i, mapping=mp)
        alone.append(M.Controller(mod, K, H, nk, 0.2, S.linear_sigma(nk), **kw))
        batch.append(M.Controller(mod, K, H, nk, 0.2, S.linear_sigma(nk), **kw))
        states.append(S.standing_state(rob, jitter=0.02, seed=40 + i))
    ref = [c.solve(x)[0] for c, x in zip(alone, states)]
    st, means, _, _ = M.solve_batch(batch, states)
    out["batch_equal"] = bool(st == 0 and all(np.array_equal(np.asarray(m).reshape(-1), a.reshape(-1))
                                              for m, a in zip(means, ref)))
    # served
    srv = M.Server(mem_budget_bytes=1 << 30, max_inflight=2)
    ref2 = [c.solve(x)[0] for c, x in zip(alone, states)]
    tickets = [srv.submit(c, x) for c, x in zip(batch, states)]
    served = [srv.poll(t, c) for t, c in zip(tickets, batch)]
    srv.close()
    out["served_equal"] = bool(all(s[0] == 0 and np.array_equal(s[1], r) for s, r in zip(served, ref2)))
    # explicit rollouts of the generic chain plans
    m = S.quadruped()
    axis = m.axis.copy()
    axis[1] = np.array([1.0, 0.0, 0.05]) / np.linalg.norm([1.0, 0.0, 0.05])
    m = m.copy(axis=axis)
    kn = S.random_knots(m, 40, 5, seed=3).astype(np.float32)
    x0 = S.standing_state(m, jitter=0.02, seed=4)
    c = M.Controller(M.Model(m), 40, 50, 5, 0.1, S.linear_sigma(5), dt=0.005, mapping=M.MPPI_MAP_CHAIN)
    got = c.rollout_explicit(x0, kn)
    out["quadruped_generic_rollout"] = rel(got, oracle.rollout_batch(m, x0, kn.astype(np.float64), 50, 0.005))
    L.mppi_check_word(C.byref(w), 0)
    out["check_word"] = int(w.value)
    print(json.dumps(out))


if __name__ == "__main__":
    main()

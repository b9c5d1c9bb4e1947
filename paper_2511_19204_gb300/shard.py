"""Sample shards over torch.distributed: one MPPI iteration's weights and knot average
when the samples of one instance are split across ranks.

Sec. III-C's min-max weights (Eq. softmax_minmax) need the global S_min and S_max before
any exponential, so an iteration exchanges twice: an all-gather of each rank's cost range
(4 numbers), merged by the library's host merge, then an all-gather of each rank's weight
sum and weighted knot sums (E + 1 FP64 numbers) under the merged range, merged the same
way and divided into the updated nominal (Eq. update-nominal). Every rank folds the
gathered parts in rank order, so all ranks hold identical bits. The sample with the
global best index (Sec. III-D) lives on one rank, which contributes its knots.

The local steps are callables, so the same exchange serves ranks whose shards are on a
GPU (mppi.shard_range_local / mppi.shard_moments on the rank's device buffers) and any
other producer of the two local results. This module only moves and merges them.
"""
from __future__ import annotations

import numpy as np

from . import mppi as M


def _gather(t, group):
    import torch.distributed as dist
    parts = [t.new_empty(t.shape) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, t, group=group)
    return parts


def allgather_merge_range(local, group=None, device="cpu"):
    """Merged mppi_shard_range of every rank's local range (rank order)."""
    import torch
    t = torch.tensor([local.s_min, local.s_max, float(local.best_index), float(local.n_finite)],
                     dtype=torch.float64, device=device)
    r = M.shard_range()
    for p in _gather(t, group):
        v = p.cpu().tolist()
        r = M.shard_range_merge(r, M.shard_range(v[0], v[1], int(v[2]), int(v[3])))
    return r


def allgather_merge_moments(local, group=None, device="cpu"):
    """Merged [sum w, sum w theta] of every rank's local moments (rank order)."""
    import torch
    t = torch.as_tensor(np.ascontiguousarray(local, dtype=np.float64), device=device)
    parts = [p.cpu().numpy() for p in _gather(t, group)]
    m = parts[0]
    for p in parts[1:]:
        m = M.shard_moments_merge(m, p)
    return m


def sharded_update(range_fn, moments_fn, knots_row_fn, index_base, K, E, group=None, device="cpu"):
    """One iteration's update over the ranks of `group`. This rank holds global samples
    index_base .. index_base + K - 1; range_fn() returns its mppi_shard_range,
    moments_fn(global_range) its [E + 1] moments, knots_row_fn(n) the knots [E] of its
    local sample n. Returns (status, mean [E] FP32 or None, global range, best knots [E]
    FP32 or None); status is MPPI_ERR_ALL_COSTS_NONFINITE when no rank has a finite cost
    (the iteration leaves the nominal unchanged)."""
    import torch
    g = allgather_merge_range(range_fn(), group, device)
    if g.n_finite == 0:
        return M.MPPI_ERR_ALL_COSTS_NONFINITE, None, g, None
    mean = M.shard_mean(allgather_merge_moments(moments_fn(g), group, device))
    own = index_base <= g.best_index < index_base + K
    row = np.zeros(E + 1, dtype=np.float64)
    if own:
        row[0] = 1.0
        row[1:] = np.asarray(knots_row_fn(int(g.best_index - index_base)), dtype=np.float32).reshape(-1)
    parts = [p.cpu().numpy() for p in _gather(torch.as_tensor(row, device=device), group)]
    owners = [p for p in parts if p[0] == 1.0]
    if len(owners) != 1:
        raise M.MppiError(M.MPPI_ERR_INVALID_ARG, f"{len(owners)} ranks own the best sample: the shards overlap or leave a gap")
    return M.MPPI_OK, mean, g, owners[0][1:].astype(np.float32)

"""Assignment of independent meshes to ranks for batched stepping on several
GPUs.  Members never exchange data, so each rank steps its own batch; the
only cross-rank traffic is bookkeeping (timing, optional gathers)."""
from __future__ import annotations

import numpy as np


def shard_members(dofs, world_size):
    """Greedy longest-first bin packing of member DOF counts onto ranks.
    Returns one ascending list of member indices per rank; deterministic.
    With more ranks than members the extra ranks get empty lists (their
    caller has nothing to step)."""
    if int(world_size) < 1:
        raise ValueError(f"world_size must be >= 1, got {world_size}")
    dofs = np.asarray(dofs, dtype=np.int64)
    if dofs.ndim != 1 or np.any(dofs < 0):
        raise ValueError("dofs must be a 1-D list of non-negative counts")
    order = sorted(range(len(dofs)), key=lambda k: (-int(dofs[k]), k))
    load = [0] * world_size
    out = [[] for _ in range(world_size)]
    for k in order:
        r = min(range(world_size), key=lambda i: (load[i], i))
        out[r].append(k)
        load[r] += int(dofs[k])
    return [sorted(x) for x in out]

"""CPU tests of batched contexts (S11): member layout, the block-diagonal
pattern against the oracle's per-member patterns, and the rank sharding of
members over gloo processes (world size 2)."""
import os

import numpy as np
import pytest

import fe_inputs as fi
from oracle import fe_oracle as O


@pytest.fixture(scope="module")
def fe():
    from paper_2306_05893_gb300 import build
    build.build()
    import paper_2306_05893_gb300 as fe
    fe.load()
    return fe


def _members(k=5, seed=7):
    return fi.batch_workload(k, seed=seed)


def test_batch_layout_and_block_diagonal_pattern(fe):
    mem = _members()
    b = fe.FEBatch([(m.mesh.elem_type, m.mesh.X, m.mesh.conn, m.mesh.fixed_nodes, m.model, m.params)
                    for m in mem], 0.01, 0.1, 0.01, 1000.0)
    models = [mem[k].model for k in b.member]
    assert models == sorted(models)                     # grouped by model, stable
    assert sorted(b.member.tolist()) == list(range(len(mem)))
    sizes = [mem[k].mesh.n_nodes for k in b.member]
    assert np.array_equal(np.diff(b.node_off), sizes)
    # pattern = union of the members' patterns shifted by their DOF offsets
    rows, cols = [], []
    for s, k in enumerate(b.member):
        m = mem[k].mesh
        fixed = (3 * m.fixed_nodes[:, None] + np.arange(3)).reshape(-1)
        rp, ci, _ = O.csr_pattern(3 * m.n_nodes, m.conn, fixed)
        r = np.repeat(np.arange(3 * m.n_nodes), np.diff(rp))
        off = 3 * b.node_off[s]
        rows.append(r + off)
        cols.append(ci.astype(np.int64) + off)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    slot_row = np.repeat(np.arange(b.n), np.diff(b.rowptr))
    assert np.array_equal(slot_row, rows) and np.array_equal(b.colind, cols)
    o = b.ordering()
    assert o["perm"].size == sum(3 * (mem[k].mesh.n_nodes - mem[k].mesh.fixed_nodes.size) for k in b.member)
    b.close()


def test_shard_members_balanced_cover():
    from paper_2306_05893_gb300.sharding import shard_members
    dofs = [3 * m.mesh.n_nodes for m in _members(64)]
    for ws in (1, 2, 3, 8):
        parts = shard_members(dofs, ws)
        flat = sorted(x for p in parts for x in p)
        assert flat == list(range(64))
        loads = [sum(dofs[k] for k in p) for p in parts]
        assert max(loads) - min(loads) <= max(dofs)


def test_shard_members_edge_cases():
    from paper_2306_05893_gb300.sharding import shard_members
    # more ranks than members: one member each, the rest empty
    assert shard_members([5, 9, 7], 5) == [[1], [2], [0], [], []]
    assert shard_members([], 3) == [[], [], []]
    # equal sizes go round-robin in index order (deterministic ties)
    assert shard_members([4, 4, 4, 4], 2) == [[0, 2], [1, 3]]
    for bad in (0, -1):
        with pytest.raises(ValueError):
            shard_members([1, 2], bad)
    with pytest.raises(ValueError):
        shard_members([1, -2], 2)


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    import paper_2306_05893_gb300 as fe
    from paper_2306_05893_gb300.sharding import shard_members
    mem = fi.batch_workload(12, seed=7)
    parts = shard_members([3 * m.mesh.n_nodes for m in mem], world)
    mine = parts[rank]
    b = fe.FEBatch([(mem[k].mesh.elem_type, mem[k].mesh.X, mem[k].mesh.conn, mem[k].mesh.fixed_nodes,
                     mem[k].model, mem[k].params) for k in mine], 0.01, 0.1, 0.01, 1000.0)
    t = torch.tensor([len(mine), b.n], dtype=torch.int64)
    allt = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(allt, t)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        np.save(os.path.join(out_dir, "shards.npy"), np.array([x.tolist() for x in allt]))
        with open(os.path.join(out_dir, "members.txt"), "w") as f:
            f.write(repr(gathered))
    b.close()
    dist.destroy_process_group()


def test_sharded_batches_over_gloo(tmp_path, fe):
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    counts = np.load(tmp_path / "shards.npy")
    members = eval((tmp_path / "members.txt").read_text())
    mem = fi.batch_workload(12, seed=7)
    assert sorted(members[0] + members[1]) == list(range(12))
    assert counts[:, 0].tolist() == [len(members[0]), len(members[1])]
    for r in range(2):
        assert counts[r, 1] == sum(3 * mem[k].mesh.n_nodes for k in members[r])

"""Subinterval sharding (paper_1509_04567_gb300.shard) on CPU ranks with the gloo backend:
each rank solves its block of subintervals with the oracle (solve_linear restricted to
those subproblems), the partial solutions are summed onto the owner of each time slab,
and every rank's slab equals the oracle's one-process solve (Sec. 2.2, eq. superposition)."""
import os
import socket

import numpy as np
import pytest

from paper_1509_04567_gb300 import shard


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_rank_ranges_and_slabs_cover_everything_once():
    for P, world in ((8, 2), (7, 3), (64, 8), (5, 5)):
        idx = shard.partition_boundaries(16 * P + 3, P)
        ranges = [shard.rank_range(P, world, r) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == P
        assert all(ranges[r][1] == ranges[r + 1][0] for r in range(world - 1))
        assert max(b - a for a, b in ranges) - min(b - a for a, b in ranges) <= 1
        rows = [shard.slab_rows(idx, a, b) for a, b in ranges]
        assert rows[0][0] == 0 and rows[-1][1] == idx[-1] + 1
        assert all(rows[r][1] == rows[r + 1][0] for r in range(world - 1))
    with pytest.raises(ValueError):
        shard.rank_range(2, 3, 0)


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    import oracle.pebk as ob
    from paper_1509_04567_gb300 import workloads as wl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pr = wl.adv_diff_1d(n=128, nu=1e-2, P=6, n_out=31, T=0.5, tol=1e-12, restart_len=30)

    def solve_range(a, b):
        Y, _ = ob.solve_linear(pr.op, pr.opts, pr.u0, pr.G, subintervals=list(range(a + 1, b + 1)))
        if a == 0:
            Y = Y + pr.u0[None, :]
        return torch.from_numpy(Y)

    (r0, r1), slab = shard.solve_sharded(solve_range, pr.opts["n_out"], pr.opts["P"], world, rank, dist)
    Yfull, _ = ob.solve_linear(pr.op, pr.opts, pr.u0, pr.G)
    err = float(np.max(np.abs(slab.numpy() - Yfull[r0:r1])))
    q.put((rank, r0, r1, err))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_sum_their_subproblems_onto_the_slab_owners(world):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0] * world
    assert out[0][1] == 0 and out[-1][2] == 31
    for rank, r0, r1, err in out:
        assert r1 > r0 and err < 1e-12, (rank, err)

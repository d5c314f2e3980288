"""Subinterval sharding of one Paraexp solve over several GPUs (Sec. 2.2, Fig. 3).

The subproblems of eq. linivpSubproblem are independent: rank r of `world` takes a
contiguous block of subintervals [a_r, b_r), solves their nonhomogeneous parts and carries
their summed solution to T (the library's sub_first / sub_last options).  The only exchange
the method has is the superposition sum (eq. superposition): rank s owns the output times of
its own subintervals, and the ranks' partial solutions are summed onto the owner, one time
slab at a time -- a reduce-scatter over time slabs.  A rank r > s has nothing at the times
of slab s (its solution is zero before T_{a_r}), so its share there is zeros.

Host logic only: the per-rank solve is a callable, so the same code runs the CUDA path on
GPUs (NCCL) and any other solver on CPU ranks (gloo).
"""
from __future__ import annotations


def rank_range(P: int, world: int, rank: int) -> tuple[int, int]:
    """Subintervals [a, b) (0-based) of `rank`: contiguous blocks whose sizes differ by <= 1."""
    if not (0 <= rank < world) or world < 1 or P < world:
        raise ValueError("need 0 <= rank < world <= P")
    q, r = divmod(P, world)
    a = rank * q + min(rank, r)
    return a, a + q + (1 if rank < r else 0)


def slab_rows(idx: list[int], a: int, b: int) -> tuple[int, int]:
    """Output rows [r0, r1) owned by the holder of subintervals [a, b): the samples of those
    subintervals, the first subinterval's first sample only when a = 0 (a shared boundary
    sample belongs to the subinterval that ends there)."""
    return (0 if a == 0 else idx[a] + 1), idx[b] + 1


def partition_boundaries(n_out: int, P: int) -> list[int]:
    """Grid indices of the subinterval boundaries, T_j = t_floor(j (n_out - 1) / P)."""
    return [(j * (n_out - 1)) // P for j in range(P + 1)]


def reduce_slabs(Y, idx: list[int], world: int, rank: int, dist):
    """Sums the ranks' partial solutions Y (n_out x n, this rank's) onto the owner of each
    time slab; returns this rank's slab of the full solution (rows slab_rows(...) of it)."""
    P = len(idx) - 1
    mine = None
    for s in range(world):
        r0, r1 = slab_rows(idx, *rank_range(P, world, s))
        buf = Y[r0:r1].clone().contiguous()
        dist.reduce(buf, dst=s, op=dist.ReduceOp.SUM)
        if s == rank:
            mine = buf
    return mine


def solve_sharded(solve_range, n_out: int, P: int, world: int, rank: int, dist):
    """One sharded solve: solve_range(a, b) returns this rank's partial solution (n_out x n,
    zero up to T_a, u0 included only when a = 0); returns (rows, slab of the full solution)."""
    idx = partition_boundaries(n_out, P)
    a, b = rank_range(P, world, rank)
    Y = solve_range(a, b)
    return slab_rows(idx, a, b), reduce_slabs(Y, idx, world, rank, dist)


def gpu_solve_range(ctx, op: dict, opts: dict, y0, G, Y):
    """solve_range for the CUDA path: the library solve restricted to subintervals [a, b)."""
    def run(a: int, b: int):
        ctx.solve_linear(op, dict(opts, sub_first=a, sub_last=b), y0, G, Y)
        return Y
    return run

"""Batched solves of independent problems of uneven size (pexp_solve_batched), the
batched workload's recipe with the mesh sizes scaled down so that the oracle finishes:
every problem against oracle.solve_linear (FP64 1e-10, mixed 1e-6, against the solution's
scale over the interval), and the autotuner's table written and read back."""
import json
import os

import numpy as np
import pytest

import oracle.pebk as ob
from gpu_util import ctx
from paper_1509_04567_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
COUNT = 16


@pytest.fixture(scope="module")
def c():
    cc = ctx()
    yield cc
    cc.close()


@pytest.fixture(scope="module")
def problems():
    # n in [4096, 8192] (the low end of the batched workload's range), P capped at 8 (the
    # oracle's homogeneous parts grow as P^2), the largest step budget
    prs = [wl.batched_instance(i, n_min_log2=12, n_max_log2=13, tol=1e-12, P_max=8) for i in range(COUNT)]
    for pr in prs:
        pr.opts["restart_len"] = 40
    refs = [ob.solve_linear(pr.op, pr.opts, pr.u0, pr.G)[0] for pr in prs]
    return prs, refs


def _items(prs, precision):
    import torch
    dt = torch.float32 if precision else torch.float64
    items = []
    for pr in prs:
        opts = dict(pr.opts, precision=precision, tol=1e-7 if precision else 1e-12)
        items.append((pr.op, opts, torch.from_numpy(pr.u0).cuda(), torch.from_numpy(pr.G).to("cuda", dt),
                      torch.full((opts["n_out"], pr.n), float("nan"), dtype=dt, device="cuda")))
    return items


def _err_scale(Y, ref):
    """max_i ||Y_i - ref_i|| / max_i ||ref_i||: the error against the solution's scale over
    the interval (the stopping rule's scale).  Some instances of the recipe decay by a
    large factor over [0, 1], where an error relative to each time's own norm would measure
    the decay more than the solve."""
    return float(np.max(np.linalg.norm(Y - ref, axis=1)) / np.max(np.linalg.norm(ref, axis=1)))


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_batched_matches_oracle(c, problems, precision):
    import torch
    prs, refs = problems
    assert len({pr.n for pr in prs}) > 8 and len({pr.opts["P"] for pr in prs}) >= 2   # uneven sizes
    items = _items(prs, precision)
    reps = c.solve_batched(items)
    torch.cuda.synchronize()
    for k, (pr, ref, it, rep) in enumerate(zip(prs, refs, items, reps)):
        assert rep["rc"] == 0, (k, rep["rc"])
        err = _err_scale(it[4].double().cpu().numpy(), ref)
        assert err < (1e-6 if precision else 1e-10), (k, pr.n, pr.opts["P"], err)


def test_autotune_writes_and_reads_its_table(c, problems, tmp_path):
    import torch
    prs, refs = problems
    items = _items(prs[:8], 1)
    path = str(tmp_path / "pexp_tune.json")
    c.autotune(items, path)
    tab = json.load(open(path))
    assert tab["batch_workers"] in (1, 2, 4, 8, 16) and len(tab["timings_ms"]) == 5
    assert torch.cuda.get_device_name(0) in tab["device"]
    mtime = os.path.getmtime(path)
    c.autotune(items, path)              # read back, not re-timed
    assert os.path.getmtime(path) == mtime
    reps = c.solve_batched(items)        # the tuned count solves as before
    for (pr, ref, it, rep) in zip(prs[:8], refs[:8], items, reps):
        assert rep["rc"] == 0 and _err_scale(it[4].double().cpu().numpy(), ref) < 1e-6

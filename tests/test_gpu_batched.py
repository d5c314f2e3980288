"""Batched solves of independent problems of uneven size (pexp_solve_batched), the
batched workload's recipe with the mesh sizes scaled down so that the oracle finishes:
every problem against oracle.solve_linear (FP64 1e-10, mixed 1e-6), and the autotuner's
table written and read back."""
import json
import os

import numpy as np
import pytest

import oracle.pebk as ob
from gpu_util import ctx, relerr_rows
from paper_1509_04567_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
COUNT = 20


@pytest.fixture(scope="module")
def c():
    cc = ctx()
    yield cc
    cc.close()


@pytest.fixture(scope="module")
def problems():
    # n in [256, 2048], P capped at 16 (the oracle's homogeneous parts grow as P^2)
    prs = [wl.batched_instance(i, n_min_log2=8, n_max_log2=11, tol=1e-12, P_max=16) for i in range(COUNT)]
    for pr in prs:
        pr.opts["restart_len"] = 30
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


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_batched_matches_oracle(c, problems, precision):
    import torch
    prs, refs = problems
    assert len({pr.n for pr in prs}) > 10 and len({pr.opts["P"] for pr in prs}) >= 3   # uneven sizes
    items = _items(prs, precision)
    reps = c.solve_batched(items)
    torch.cuda.synchronize()
    for k, (pr, ref, it, rep) in enumerate(zip(prs, refs, items, reps)):
        assert rep["rc"] == 0, (k, rep["rc"])
        err = relerr_rows(it[4].double().cpu().numpy(), ref)
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
        assert rep["rc"] == 0 and relerr_rows(it[4].double().cpu().numpy(), ref) < 1e-6

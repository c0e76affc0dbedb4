"""Batched solves: many independent instances in one persistent launch give
each instance the result of its own single solve, and small instances match
the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1809_03745_gb300 import workloads as W

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1809_03745_gb300 import ebpoisson as E


def _instances(count, max_cells, seed):
    return W.batched_instances(count=count, seed=seed, n2=(64, 512), n3=(32, 64), max_cells=max_cells)


def test_batch_equals_single_solves():
    inst = _instances(12, 300000, 1809 + 4)
    geoms = [E.Geometry(d) for d, _, _ in inst]
    solvers = [E.Poisson(g, precision="mixed", tol=1e-10, max_cycles=400) for g in geoms]
    rhs = [torch.from_numpy(S) for _, S, _ in inst]
    sig = [torch.from_numpy(s) for _, _, s in inst]
    phis, infos = E.solve_batched(solvers, rhs, sig)
    for k, P in enumerate(solvers):
        assert infos[k]["status"] == 0 and infos[k]["rel_res"] <= 1e-10, (k, infos[k])
        single, si = P.solve(rhs[k], sig[k])
        assert si["vcycles"] == infos[k]["vcycles"]
        # same per-cell arithmetic and order-independent reductions: bitwise equal
        assert torch.equal(single, phis[k]), (k, (single - phis[k]).abs().max().item())


def test_batch_small_instances_match_oracle():
    inst = _instances(6, 40000, 1809 + 40)
    solvers, rhs, sig = [], [], []
    for d, S, s in inst:
        solvers.append(E.Poisson(E.Geometry(d), precision="mixed", tol=1e-12, max_cycles=600))
        rhs.append(torch.from_numpy(S))
        sig.append(torch.from_numpy(s))
    phis, infos = E.solve_batched(solvers, rhs, sig)
    for k, (d, S, s) in enumerate(inst):
        assert infos[k]["status"] == 0, infos[k]
        og, ophi, A, b, data = oracle.solve(d, s=S, sigma=s)
        got = phis[k].cpu().numpy()
        assert np.abs(got - ophi).max() <= 1e-9 * np.abs(ophi).max(), (k, d["dim"], d["n"])


def test_batch_more_instances_than_ctas():
    """More instances than CTAs: the batch is split over several launches."""
    inst = _instances(200, 5000, 1809 + 41)
    solvers = [E.Poisson(E.Geometry(d), precision="mixed", tol=1e-10, max_cycles=600) for d, _, _ in inst]
    phis, infos = E.solve_batched(solvers, [torch.from_numpy(S) for _, S, _ in inst],
                                  [torch.from_numpy(s) for _, _, s in inst])
    assert all(i["status"] == 0 for i in infos)

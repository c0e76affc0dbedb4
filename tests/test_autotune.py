"""Autotuner: selection and caching logic on the CPU with a fake timer; on
the GPU, a tuned schedule converges and is cached for the size class."""
import json

import numpy as np
import pytest
import torch

from paper_1809_03745_gb300 import autotune as A


def test_select_fastest_converging_and_cache_roundtrip(tmp_path):
    path = str(tmp_path / "tune.json")
    t = A.Autotuner(path, candidates=[(2, 2, 2), (4, 4, 2), (6, 6, 2)])
    times = {(2, 2, 2): (9.0, True), (4, 4, 2): (5.0, False), (6, 6, 2): (7.0, True)}
    best = t.select("3d-2^21-ph2-mixed", lambda s: times[tuple(s)])
    assert best == (6, 6, 2)  # the faster (4,4,2) did not converge
    data = json.load(open(path))
    assert data["3d-2^21-ph2-mixed"]["schedule"] == [6, 6, 2]
    assert len(data["3d-2^21-ph2-mixed"]["trials"]) == 3
    t2 = A.Autotuner(path)
    assert t2.lookup("3d-2^21-ph2-mixed") == (6, 6, 2)
    assert t2.lookup("2d-2^20-ph2-mixed") is None


def test_ties_prefer_fewer_sweeps_and_nothing_cached_without_convergence(tmp_path):
    t = A.Autotuner(str(tmp_path / "t.json"), candidates=[(4, 4, 2), (2, 2, 2)])
    assert t.select("k", lambda s: (1.0, True)) == (2, 2, 2)
    t3 = A.Autotuner(None, candidates=[(3, 3, 2), (2, 2, 2)])
    assert t3.select("x", lambda s: (1.0, False)) == (3, 3, 2)
    assert t3.lookup("x") is None


def test_size_class_and_defaults():
    assert A.size_class(2, 1024 * 1024, 2, "mixed") == "2d-2^20-ph2-mixed"
    assert A.size_class(3, 128 ** 3, 1, "fp64") == "3d-2^21-ph1-fp64"
    assert A.default_schedule(2) == (2, 2, 2)
    assert A.default_schedule(3) == (6, 6, 2)


@pytest.mark.gpu
def test_tune_on_gpu_converges_and_caches(tmp_path):
    from paper_1809_03745_gb300 import ebpoisson as E
    from paper_1809_03745_gb300 import workloads as W
    d, S, sig = W.c3_inputs(32)
    g = E.Geometry(d)
    t = A.Autotuner(str(tmp_path / "t.json"), candidates=[(2, 2, 2), (6, 6, 2)])
    best = t.tune(g, torch.from_numpy(S), torch.from_numpy(sig), reps=1)
    assert best in [(2, 2, 2), (6, 6, 2)]
    P = t.solver(g, tol=1e-10, max_cycles=400)
    phi, info = P.solve(torch.from_numpy(S), torch.from_numpy(sig))
    assert info["status"] == 0 and info["rel_res"] <= 1e-10
    assert t.schedule(g) == best

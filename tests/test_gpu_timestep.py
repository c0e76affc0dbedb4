"""Poisson solves inside the time step (Sec. 3.6): three solves per step on
charges that move between them, each started from the previous potential.
Every solve reaches the oracle's direct solution of its own charges, and the
warm start saves V-cycles against starting from zero."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1809_03745_gb300 import timestep as TS


def test_every_solve_of_the_step_matches_the_oracle():
    r = TS.run(n=64, steps=2, dt=0.01, tol=1e-12, keep=True)
    sols = r["solutions"]
    assert len(sols) == 6
    k = 0
    for step in r["inputs"]:
        for S, sig in step:
            _, ophi, _, _, _ = oracle.solve(r["desc"], s=S, sigma=sig)
            assert np.abs(sols[k] - ophi).max() <= 1e-9 * np.abs(ophi).max(), k
            k += 1


def test_warm_start_saves_vcycles():
    warm = TS.run(n=256, steps=4, dt=0.005, warm=True)
    cold = TS.run(n=256, steps=4, dt=0.005, warm=False)
    vw = [v for x in warm["rows"][1:] for v in x["vcycles"]]
    vc = [v for x in cold["rows"][1:] for v in x["vcycles"]]
    assert np.mean(vw) < np.mean(vc), (vw, vc)
    # same charges, same tolerance: the two runs end at potentials that agree
    # to the solve tolerance's reach
    a, b = warm["phi"].cpu().numpy(), cold["phi"].cpu().numpy()
    assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max()

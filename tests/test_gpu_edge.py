"""Edge cases on the GPU: zero data gives the zero solution without a
V-cycle (single, batched, composite); the largest grids the benchmark
workloads reach converge and keep the mirror symmetry the geometry and data
have (a property that holds at any size, where the oracle cannot follow)."""
import numpy as np
import pytest
import torch

from paper_1809_03745_gb300 import workloads as W

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1809_03745_gb300 import ebpoisson as E


def _zero(desc):
    d = dict(desc, phi_E=0.0, phi_wall=[0.0] * 6, electrodes=None)
    n = W.ncells(d)
    return d, np.zeros((2, n)), np.zeros(n)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_zero_data_gives_zero_solution(precision):
    for desc in (W.rod_plane_2d(64, dielectric=True), W.pin_plane_3d(32)):
        d, S, s = _zero(desc)
        P = E.Poisson(E.Geometry(d), precision=precision)
        phi0 = torch.ones(2, W.ncells(d), dtype=torch.float64, device="cuda")
        phi, info = P.solve(torch.from_numpy(S), torch.from_numpy(s), phi=phi0)
        assert info["status"] == 0 and info["vcycles"] == 0 and info["bnorm"] == 0.0
        assert torch.count_nonzero(phi).item() == 0


def test_zero_data_batched_and_composite():
    d, S, s = _zero(W.rod_plane_2d(64))
    P = [E.Poisson(E.Geometry(d)) for _ in range(3)]
    phis, infos = E.solve_batched(P, [torch.from_numpy(S)] * 3, [torch.from_numpy(s)] * 3)
    assert all(i["status"] == 0 and i["vcycles"] == 0 for i in infos)
    assert all(torch.count_nonzero(p).item() == 0 for p in phis)
    G = E.Composite(d, [24, 24], [40, 40])
    Sf = np.zeros((2, G.n_fine))
    pc, pf, info = G.solve(S, Sf)
    assert info["status"] == 0 and info["bnorm"] == 0.0
    assert torch.count_nonzero(pc).item() == 0 and torch.count_nonzero(pf).item() == 0


def test_largest_2d_grid_converges_and_is_mirror_symmetric():
    n = 4096
    d = W.rod_plane_2d(n)
    x, y, _ = W.cell_centres(d)
    S = np.zeros((2, x.size))
    S[0] = 100.0 * np.exp(-((x - 0.5) ** 2 + (y - 0.45) ** 2) / (2 * 0.03 ** 2))
    # red and black swap under the mirror, so only the converged solution is
    # symmetric: solve far below the benchmark tolerance
    P = E.Poisson(E.Geometry(d), precision="mixed", tol=1e-12, max_cycles=300)
    phi, info = P.solve(torch.from_numpy(S))
    assert info["status"] == 0 and info["rel_res"] <= 1e-12, info
    r = P.residual(torch.from_numpy(S), None, phi)
    assert r.abs().max().item() <= 1.01e-12 * info["bnorm"]
    f = phi[0].reshape(n, n)
    assert (f - f.flip(1)).abs().max().item() <= 1e-9 * f.abs().max().item()


def test_largest_3d_grid_converges_and_has_fourfold_symmetry():
    n = 384
    d, S, s = W.c3_inputs(n)
    P = E.Poisson(E.Geometry(d), precision="mixed", tol=1e-12, max_cycles=600)
    phi, info = P.solve(torch.from_numpy(S), torch.from_numpy(s))
    assert info["status"] == 0 and info["rel_res"] <= 1e-12, info
    f = phi[0].reshape(n, n, n)  # [z][y][x]
    m = f.abs().max().item()
    assert (f - f.flip(2)).abs().max().item() <= 1e-9 * m
    assert (f - f.flip(1)).abs().max().item() <= 1e-9 * m
    assert (f - f.transpose(1, 2)).abs().max().item() <= 1e-9 * m

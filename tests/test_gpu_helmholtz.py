"""GPU parity of the Helmholtz shift and the Robin conditions (row f1).

The operator lam phi - div(eps grad phi) with Robin walls and electrodes
(Sec. 3.3, Eq. helmholtz; Sec. 3.3.1, Eq. robin) through the C ABI against
the oracle: the residual b - A phi per cell to 1e-12 relative, solves to the
oracle's direct solution to 1e-9 relative, in FP64 and mixed precision.  The
cases: the three Eddington photon groups of the photoionisation model on the
2D rod-plane and 3D pin-plane geometries (Robin outflow on every boundary,
lam from 3 (kappa L)^2 = 276 to 71610), a two-phase problem with a shift per
phase and Robin walls of several kinds (one a pure flux condition, a1 = 0),
and a disk electrode with Robin data a3 != 0.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1809_03745_gb300 import workloads as W

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1809_03745_gb300 import ebpoisson as E


def _two_phase(n):
    d = W.rod_plane_2d(n, dielectric=True)
    d["lam"] = (5.0, 2.0)
    d["bc"] = [W.ROBIN, W.ROBIN, W.DIRICHLET, W.ROBIN, 0, 0]
    d["robin"] = [(2.0, 0.5), (0.0, 1.0), (0.0, 0.0), (1.0, 0.2), (0.0, 0.0), (0.0, 0.0)]
    d["phi_wall"] = [0.3, -0.4, 0.0, 1.1, 0.0, 0.0]
    x, y, _ = W.cell_centres(d)
    S = np.zeros((2, x.size))
    S[0] = 60.0 * np.exp(-((x - 0.5) ** 2 + (y - 0.4) ** 2) / 0.01)
    S[1] = 5.0 * np.sin(3.0 * x)
    return d, S, np.where(y < 0.3, 0.4, 0.0)


def _disk(n):
    c = (0.52, 0.47)
    d = W._desc(2, (n, n), (0, 0), 1.0 / n, [(W.PRIM_SPHERE, [c[0], c[1], 0.0, 0.21])], [(0, 0, 0)], 0, -1,
                (1.0, 1.0), [W.ROBIN] * 4 + [0, 0], 0.7, [0.2, 0.0, -0.3, 0.5, 0.0, 0.0])
    d["robin"] = [(1.0, 0.4), (2.0, 0.5), (1.5, 0.25), (0.5, 1.0), (0.0, 0.0), (0.0, 0.0)]
    d["eb_robin"] = (1.5, 1.0)
    d["lam"] = (4.0, 0.0)
    x, y, _ = W.cell_centres(d)
    S = np.zeros((2, x.size))
    S[0] = 4.0 * (np.cos(2 * x) * np.exp(y) + x * y) + 3.0 * np.cos(2 * x) * np.exp(y)
    return d, S, np.zeros(x.size)


def _cases():
    out = []
    groups, _ = W.photo_inputs(2, 128)
    for gi, (d, S, sig) in enumerate(groups):
        out.append((f"rte2d_128_g{gi + 1}", d, S, sig))
    groups, _ = W.photo_inputs(3, 32)
    for gi, (d, S, sig) in enumerate(groups):
        out.append((f"rte3d_32_g{gi + 1}", d, S, sig))
    out.append(("two_phase_robin_200",) + _two_phase(200))
    out.append(("robin_disk_96",) + _disk(96))
    return out


CASES = _cases()
IDS = [c[0] for c in CASES]


@pytest.fixture(scope="module")
def oracles():
    return {name: oracle.solve(d, s=S, sigma=sig) for name, d, S, sig in CASES}


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_helmholtz_robin_geometry_and_residual_parity(case, oracles):
    """Same unknowns as the oracle; r = b - A phi for a random phi per cell."""
    name, d, S, sig = case
    og, _, A, b, data = oracles[name]
    g = E.Geometry(d)
    flags = g.export()["flags"].cpu().numpy()
    dofbits = (og.dof[0] >= 0).astype(np.uint8) | ((og.dof[1] >= 0).astype(np.uint8) << 1)
    assert np.array_equal(flags & 3, dofbits)
    rng = np.random.default_rng(13)
    phi = og.to_cells(rng.normal(size=og.ndof))
    P = E.Poisson(g, precision="fp64")
    r = P.residual(torch.from_numpy(S), torch.from_numpy(sig), torch.from_numpy(phi)).cpu().numpy()
    ro = og.to_cells(b - A @ og.to_dofs(phi))
    scale = np.abs(b).max() + abs(A).max() * np.abs(phi).max()
    assert np.abs(r - ro).max() <= 1e-12 * scale


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_helmholtz_robin_solve_parity(case, precision, oracles):
    name, d, S, sig = case
    og, ophi = oracles[name][:2]
    g = E.Geometry(d)
    P = E.Poisson(g, precision=precision, tol=1e-12, max_cycles=200)
    phi, info = P.solve(torch.from_numpy(S), torch.from_numpy(sig))
    assert info["status"] == 0, info
    got = phi.cpu().numpy()
    assert np.abs(got - ophi).max() <= 1e-9 * np.abs(ophi).max(), info
    for p in range(2):
        assert np.all(got[p][og.dof[p] < 0] == 0.0)


def test_photoionisation_rate_matches_oracle():
    """S_ph = nu_eff p_O2 sum_gamma A_gamma Psi_gamma from the three GPU group
    solves against the same sum over the oracle's solutions (2D, 128^2)."""
    groups, w = W.photo_inputs(2, 128)
    sg, so = 0.0, 0.0
    for (d, S, sig), wg in zip(groups, w):
        ophi = oracle.solve(d, s=S, sigma=sig)[1]
        P = E.Poisson(E.Geometry(d), precision="mixed", tol=1e-10)
        phi, info = P.solve(torch.from_numpy(S), torch.from_numpy(sig))
        assert info["status"] == 0, info
        sg = sg + wg * phi.cpu().numpy()[0]
        so = so + wg * ophi[0]
    assert np.abs(sg - so).max() <= 1e-8 * np.abs(so).max()


@pytest.mark.parametrize("bad", ["robin_zero", "robin_negative", "eb_robin_zero", "lam_negative"])
def test_invalid_helmholtz_robin_coefficients_are_rejected(bad):
    d = W.rte_desc(2, 32, 10.0)
    if bad == "robin_zero":
        d["robin"] = [(0.0, 0.0)] + [(1.0, 1.0)] * 5
    elif bad == "robin_negative":
        d["robin"] = [(1.0, -0.5)] + [(1.0, 1.0)] * 5
    elif bad == "eb_robin_zero":
        d["eb_robin"] = (0.0, 0.0)
    else:
        d["lam"] = (-1.0, 0.0)
    with pytest.raises(E.EBError) as ei:
        E.Geometry(d)
    assert ei.value.status == E.EB_ERR_INVALID

"""Pins of the oracle's TGA diffusion step (row f2; Sec. 3.4, Eq. tga).

None restates the step's formulas:
  - exact conservation: with Neumann walls and no Dirichlet boundary the
    operator's integrated flux vanishes, so sum(kappa phi) grows by exactly
    dt sum(kappa rho) per step (the integral form of Sec. 3.3), cut cells and
    a dielectric interface included;
  - the steady state: for a fixed source the scheme's fixed point is the
    steady problem's solution (its mu's make it so), and it is L-stable, so
    many large steps reach the oracle's steady solve (a separate code path);
  - second order in time: against the exact evolution of the semi-discrete
    system, exp(-M^-1 A0 t) phi0 (a matrix exponential), the error falls by 4
    per halving of dt;
  - planted mistakes (mu3 and mu4 swapped; M dropped from the second stage)
    each fail one of these.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import tga as T
from paper_1809_03745_gb300 import workloads as W


def _neumann_two_phase(n=32):
    """A dielectric disk (eps 3) in a box with Neumann walls and no electrode."""
    return W._desc(2, (n, n), (0, 0), 1.0 / n, [(W.PRIM_SPHERE, [0.46, 0.53, 0.0, 0.23])], [(0, 0, 0)], -1, 0,
                   (1.0, 3.0), [0, 0, 0, 0, 0, 0], 0.0, [0.0] * 6)


def _disk_electrode(n=16):
    """A disk electrode (zero potential) in a box with Dirichlet walls."""
    return W._desc(2, (n, n), (0, 0), 1.0 / n, [(W.PRIM_SPHERE, [0.47, 0.52, 0.0, 0.2])], [(0, 0, 0)], 0, -1,
                   (1.0, 1.0), [1, 1, 1, 1, 0, 0], 0.0, [0.0] * 6)


def test_tga_step_conserves_the_integral():
    D = T.Diffusion(_neumann_two_phase())
    rng = np.random.default_rng(21)
    phi = rng.normal(size=D.g.ndof)
    rho = rng.normal(size=D.g.ndof)
    assert np.any((D.kappa > 0) & (D.kappa < 1))  # cut cells take part
    for dt in (1e-3, 0.1):
        new = D.step(phi, rho, dt)
        gain = np.dot(D.kappa, new) - np.dot(D.kappa, phi)
        want = dt * np.dot(D.kappa, rho)
        assert abs(gain - want) <= 1e-11 * (np.abs(D.kappa * phi).sum() + dt * np.abs(D.kappa * rho).sum())


def test_tga_reaches_the_steady_solution():
    """Rod-plane with a dielectric (homogeneous boundary data): 40 steps of
    dt = 5 from zero end at the oracle's solution of A0 phi = kappa rho."""
    d = W.rod_plane_2d(32, dielectric=True)
    D = T.Diffusion(d)
    X, Y, _ = D.g.cell_centres()
    rho_c = np.stack([50.0 * np.exp(-((X - 0.5) ** 2 + (Y - 0.45) ** 2) / 0.01), 3.0 * np.cos(2 * X)])
    rho = D.g.to_dofs(rho_c)
    phi = np.zeros(D.g.ndof)
    for _ in range(40):
        phi = D.step(phi, rho, 5.0)
    ss = oracle.solve_system(D.A0, D.kappa * rho)
    assert np.abs(phi - ss).max() <= 1e-9 * np.abs(ss).max()


@pytest.mark.parametrize("case", ["box", "disk_electrode"])
def test_tga_is_second_order_in_time(case):
    """Against the exact semi-discrete evolution exp(-M^-1 A0 t) phi0 (no
    source), the error at t = 0.04 falls by about 4 per halving of dt."""
    import scipy.linalg as la
    if case == "box":
        d = W._desc(2, (16, 16), (0, 0), 1.0 / 16, [], [], -1, -1, (1.0, 1.0), [1, 1, 1, 1, 0, 0], 0.0, [0.0] * 6)
    else:
        d = _disk_electrode(16)
    D = T.Diffusion(d)
    assert np.all(D.kappa > 0)
    X, Y, _ = D.g.cell_centres()
    phi0 = D.g.to_dofs(np.stack([np.sin(math.pi * X) * np.sin(math.pi * Y) + 0.3 * np.sin(3 * math.pi * X),
                                 np.zeros_like(X)]))
    t_end = 0.04
    exact = la.expm(-t_end * (D.A0.toarray() / D.kappa[:, None])) @ phi0
    errs = []
    for steps in (4, 8, 16):
        phi = phi0.copy()
        for _ in range(steps):
            phi = D.step(phi, np.zeros_like(phi), t_end / steps)
        errs.append(np.abs(phi - exact).max())
    rates = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert min(rates) >= 1.8, (errs, rates)


def test_plant_swapped_mu3_mu4_breaks_the_steady_state(monkeypatch):
    monkeypatch.setattr(T, "PLANT", 1)
    with pytest.raises(AssertionError):
        test_tga_reaches_the_steady_solution()


def test_plant_without_mass_in_stage_two_breaks_conservation(monkeypatch):
    monkeypatch.setattr(T, "PLANT", 2)
    with pytest.raises(AssertionError):
        test_tga_step_conserves_the_integral()

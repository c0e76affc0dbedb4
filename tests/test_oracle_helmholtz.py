"""Pins of the oracle's Helmholtz shift and Robin conditions (row f1).

The operator is alpha a phi - div(eps grad phi) = rho (Sec. 3.3, Eq. helmholtz,
with beta b = -eps and a constant shift lam = alpha a per phase); Robin
conditions a1 phi + a2 dphi/dn = a3, n out of the fluid, sit on domain walls
and electrode boundaries (Sec. 3.3.1, Eq. robin; Sec. 2.3's outflow condition
of the Eddington photon densities).  The paper imposes them by extrapolating
phi to the boundary with the stencils the Dirichlet condition uses.  The
pins, none of which restates the oracle's formulas:
  - every stencil involved is exact for quadratics (the one-sided wall
    formula, the centred flux, the ray-cast EB derivative on grid-aligned
    surfaces), so the discrete solution of a quadratic manufactured problem
    with Robin data equals the quadratic at every unknown;
  - a Robin condition with a2 = 0 is the Dirichlet condition and one with
    a1 = 0, a3 = 0 the homogeneous Neumann condition, each built by an
    independent branch of the oracle: the systems must agree;
  - on a curved electrode the scheme stays second order (Sec. 4.2's test of
    the discretisation), for a smooth manufactured solution.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1809_03745_gb300 import workloads as W


def _wall_data(g, phi, grad, kinds, robin):
    """Per wall face: phi (Dirichlet sides) or a1 phi + a2 dphi/dn_out (Robin
    sides), n_out = -e_a on a low side and +e_a on a high side."""
    out = []
    for side, x, y, z in g.wall_face_centres():
        a, hi = side // 2, side % 2
        if kinds[side] == 2:
            a1, a2 = robin[side]
            dn = (1.0 if hi else -1.0) * grad(x, y, z)[a]
            out.append(a1 * phi(x, y, z) + a2 * dn)
        else:
            out.append(phi(x, y, z))
    return np.concatenate(out)


def _quadratic(dim):
    co = np.array([0.4, -0.7, 1.1, 0.8, -0.6, 0.5, 0.4 if dim == 3 else 0.0, 0.3 if dim == 3 else 0.0,
                   -0.2 if dim == 3 else 0.0])

    def phi(x, y, z):
        return (co[0] + co[1] * x + co[2] * y + co[3] * x * x + co[4] * x * y + co[5] * y * y + co[6] * z * z
                + co[7] * y * z + co[8] * z)

    def grad(x, y, z):
        return (co[1] + 2 * co[3] * x + co[4] * y,
                co[2] + co[4] * x + 2 * co[5] * y + co[7] * z,
                2 * co[6] * z + co[7] * y + co[8])
    lap = 2 * co[3] + 2 * co[5] + 2 * co[6]
    return phi, grad, lap


ROBIN = [(1.0, 0.3), (2.0, 0.5), (0.0, 1.0), (1.0, 0.0), (0.7, 0.2), (1.5, 1.0)]


@pytest.mark.parametrize("dim", [2, 3])
def test_quadratic_exactness_with_robin_walls_and_helmholtz_shift(dim):
    """A box without boundaries inside: Robin walls of several kinds (one with
    a1 = 0, a pure flux condition; one with a2 = 0, a Dirichlet condition
    written as Robin) and one Dirichlet wall, eps = 2, shift lam = 3.  With
    rho = lam phi - eps lap(phi) sampled at cell centres and a3 from the exact
    phi at the wall faces, the solution is the quadratic itself."""
    n = 24 if dim == 2 else 12
    h = 1.0 / n
    kinds = [2, 2, 2, 1, 2, 2] if dim == 3 else [2, 2, 2, 1, 0, 0]
    d = W._desc(dim, (n,) * dim, (0,) * dim, h, [], [], -1, -1, (2.0, 1.0), kinds, 0.0, [0] * 6)
    d["robin"] = ROBIN
    d["lam"] = (3.0, 0.0)
    g = oracle.Geometry(d)
    phi, grad, lap = _quadratic(dim)
    X, Y, Z = g.cell_centres()
    s = np.zeros((2, g.ncell))
    s[0] = 3.0 * phi(X, Y, Z) - 2.0 * lap
    pd = _wall_data(g, phi, grad, kinds, ROBIN)
    data = g.data(s=s, phidom=np.stack([pd, pd]))
    A, b = g.assemble(data)
    x = g.to_cells(oracle.solve_system(A, b))[0]
    ex = phi(X, Y, Z)
    assert np.abs(x - ex).max() <= 1e-11 * np.abs(ex).max()


def _rod_plane(n):
    return W.rod_plane_2d(n, dielectric=True)


@pytest.mark.parametrize("n", [32])
def test_robin_with_a2_zero_is_dirichlet_and_with_a1_zero_is_neumann(n):
    """The 2D rod-plane problem (electrodes, a dielectric slab, Dirichlet and
    Neumann walls).  Written with Robin conditions of a2 = 0 on the Dirichlet
    walls and the electrodes (a3 = a1 times the Dirichlet value), and of a1 = 0,
    a3 = 0 on the Neumann walls, it assembles to the same system."""
    d = _rod_plane(n)
    g0 = oracle.Geometry(d)
    S = np.zeros((2, g0.ncell))
    X, Y, _ = g0.cell_centres()
    S[0] = 50.0 * np.exp(-((X - 0.5) ** 2 + (Y - 0.6) ** 2) / 0.01)
    sig = np.where(g0.ebkind == oracle.EB_INTERFACE, 0.3, 0.0)
    A0, b0 = g0.assemble(g0.data(s=S, sigma=sig))
    r = dict(d)
    a1 = 2.5
    r["bc"] = [2] * 6
    r["robin"] = [(a1, 0.0) if k == 1 else (0.0, 1.0) for k in d["bc"]]
    r["phi_wall"] = [a1 * v if k == 1 else 0.0 for k, v in zip(d["bc"], d["phi_wall"])]
    r["eb_robin"] = (a1, 0.0)
    r["electrodes"] = [(root, a1 * v) for root, v in d["electrodes"]]
    r["phi_E"] = a1 * d["phi_E"]
    g1 = oracle.Geometry(r)
    assert np.array_equal(g1.dof, g0.dof)
    A1, b1 = g1.assemble(g1.data(s=S, sigma=sig))
    assert abs(A1 - A0).max() <= 1e-13 * abs(A0).max()
    assert np.abs(b1 - b0).max() <= 1e-13 * np.abs(b0).max()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("offset", [0.0, 1e-10])
def test_quadratic_exactness_with_robin_electrode_on_grid_faces(dim, offset):
    """An electrode filling the half space below a plane of cell faces (exactly,
    or within the crossing snap distance above it), carrying a Robin condition
    a1 phi + a2 dphi/dn = a3 with n pointing into the electrode; Robin and
    Dirichlet walls; shift lam = 2.  The ray-cast EB derivative and the wall
    formula are exact for quadratics there, so eliminating the boundary value
    keeps the discrete solution equal to the quadratic at every unknown,
    including the zero-volume fragments on the plane (whose rows carry no
    shift: it scales with the volume fraction)."""
    n = 32 if dim == 2 else 16
    h = 1.0 / n
    y0 = 0.5 + offset
    kinds = [2, 1, 1, 1, 0, 0] if dim == 2 else [2, 1, 1, 1, 2, 2]
    d = W._desc(dim, (n,) * dim, (0,) * dim, h, [(W.PRIM_HALFSPACE, [0.0, 1.0, 0.0, y0])], [(0, 0, 0)], 0, -1,
                (1.0, 1.0), kinds, 0.0, [0] * 6)
    d["robin"] = ROBIN
    d["eb_robin"] = (0.8, 0.35)
    d["lam"] = (2.0, 0.0)
    g = oracle.Geometry(d)
    phi, grad, lap = _quadratic(dim)
    X, Y, Z = g.cell_centres()
    s = np.zeros((2, g.ncell))
    s[0] = 2.0 * phi(X, Y, Z) - lap
    xb = g.ebx
    gx = grad(xb[:, 0], xb[:, 1], xb[:, 2])
    a3 = 0.8 * phi(xb[:, 0], xb[:, 1], xb[:, 2]) + 0.35 * (-gx[1])  # n = -e_y, into the electrode
    pd = _wall_data(g, phi, grad, kinds, ROBIN)
    data = g.data(s=s, phiE=a3, phidom=np.stack([pd, pd]))
    A, b = g.assemble(data)
    x = g.to_cells(oracle.solve_system(A, b))[0]
    ex = phi(X, Y, Z)
    m = g.dof[0] >= 0
    assert np.abs(x[m] - ex[m]).max() <= 1e-11 * np.abs(ex).max()


def _disk_errors(n):
    """A disk electrode of radius 0.21 at (0.52, 0.47) with a Robin condition,
    Robin walls, lam = 4: the smooth phi = cos(2x) e^y + x y, its exact data."""
    h = 1.0 / n
    c = (0.52, 0.47)
    kinds = [2, 2, 2, 2, 0, 0]
    rob = [(1.0, 0.4), (2.0, 0.5), (1.5, 0.25), (0.5, 1.0), (0.0, 0.0), (0.0, 0.0)]
    d = W._desc(2, (n, n), (0, 0), h, [(W.PRIM_SPHERE, [c[0], c[1], 0.0, 0.21])], [(0, 0, 0)], 0, -1,
                (1.0, 1.0), kinds, 0.0, [0] * 6)
    d["robin"] = rob
    d["eb_robin"] = (1.5, 1.0)
    d["lam"] = (4.0, 0.0)
    g = oracle.Geometry(d)

    def phi(x, y, z):
        return np.cos(2 * x) * np.exp(y) + x * y

    def grad(x, y, z):
        return (-2 * np.sin(2 * x) * np.exp(y) + y, np.cos(2 * x) * np.exp(y) + x, 0.0 * x)
    X, Y, Z = g.cell_centres()
    lap = -3.0 * np.cos(2 * X) * np.exp(Y)
    s = np.zeros((2, g.ncell))
    s[0] = 4.0 * phi(X, Y, Z) - lap
    xb = g.ebx
    r = np.hypot(xb[:, 0] - c[0], xb[:, 1] - c[1])
    nx, ny = -(xb[:, 0] - c[0]) / np.where(r > 0, r, 1.0), -(xb[:, 1] - c[1]) / np.where(r > 0, r, 1.0)
    gx, gy, _ = grad(xb[:, 0], xb[:, 1], xb[:, 2])
    a3 = 1.5 * phi(xb[:, 0], xb[:, 1], 0.0) + 1.0 * (gx * nx + gy * ny)
    pd = _wall_data(g, phi, grad, kinds, rob)
    data = g.data(s=s, phiE=a3, phidom=np.stack([pd, pd]))
    A, b = g.assemble(data)
    x = g.to_cells(oracle.solve_system(A, b))[0]
    m = g.dof[0] >= 0
    e = np.abs(x[m] - phi(X, Y, Z)[m])
    return e.max(), math.sqrt(np.mean(e ** 2))


def test_robin_disk_electrode_second_order():
    """Curved Robin boundary: the errors fall at second order from 32^2 to 128^2
    (rates from the successive halvings of h, max and RMS)."""
    errs = [_disk_errors(n) for n in (32, 64, 128)]
    for (m0, r0), (m1, r1) in zip(errs, errs[1:]):
        assert math.log2(r0 / r1) >= 1.8, errs
        assert math.log2(m0 / m1) >= 1.5, errs
    assert errs[-1][0] <= 1e-3, errs

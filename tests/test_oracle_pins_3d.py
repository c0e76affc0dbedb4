"""3D pins of the CPU oracle.

In 3D a curved boundary cut by a cell is a non-planar polygon, so exactness for
quadratics only holds for planar boundaries (Sec. 3.1 linearises the boundary
inside each cell).  For planar electrodes and a planar dielectric interface
the local truncation error of a quadratic solution vanishes on every row whose
stencil stays off the domain walls (cut cells at a wall may fall back to the
two-point wall formula); concentric spheres with a dielectric shell converge
at second order to their closed form; the conservation identity holds.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1809_03745_gb300 import workloads as W


def _wall_values(g, f):
    return np.concatenate([f(x, y, z) for _, x, y, z in g.wall_face_centres()])


def _interior_rows(g, margin=3):
    n = g.n[0]
    idx = np.arange(g.ncell)
    i, j, k = idx % n, (idx // n) % n, idx // (n * n)
    inner = (i >= margin) & (i < n - margin) & (j >= margin) & (j < n - margin) & (k >= margin) & (k < n - margin)
    rows = []
    for p in range(2):
        m = inner & (g.dof[p] >= 0)
        rows.append(g.dof[p][m])
    return np.concatenate(rows)


@pytest.mark.parametrize("n", [12, 16])
def test_planar_electrode_truncation_zero(n):
    rng = np.random.default_rng(n)
    c = rng.normal(size=10)

    def phi(x, y, z):
        return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * y + c[6] * z * z + c[7] * x * y
                + c[8] * y * z + c[9] * x * z)
    lap = 2 * (c[4] + c[5] + c[6])
    nv = np.array([0.3, 0.5, 0.81])
    nv /= np.linalg.norm(nv)
    dd = nv @ np.array([0.37, 0.41, 0.45])
    d = W._desc(3, (n, n, n), (0, 0, 0), 1.0 / n, [(W.PRIM_HALFSPACE, [nv[0], nv[1], nv[2], dd])], [(0, 0, 0)], 0,
                -1, (1.0, 1.0), [1] * 6, 0.0, [0] * 6)
    g = oracle.Geometry(d)
    pd = _wall_values(g, phi)
    data = g.data(s=np.full((2, g.ncell), -lap), phiE=phi(g.ebx[:, 0], g.ebx[:, 1], g.ebx[:, 2]),
                  phidom=np.stack([pd, pd]))
    A, b = g.assemble(data)
    X, Y, Z = g.cell_centres()
    xe = g.to_dofs(np.stack([phi(X, Y, Z), phi(X, Y, Z)]))
    rows = _interior_rows(g)
    cut_rows = np.concatenate([g.dof[p][(g.cut == 1) & (g.dof[p] >= 0)] for p in range(2)])
    assert len(np.intersect1d(rows, cut_rows)) > n  # the check covers many cut cells
    r = (A @ xe - b)[rows]
    assert np.abs(r).max() <= 1e-10 * np.abs(b).max()


@pytest.mark.parametrize("n", [12, 16])
def test_planar_interface_truncation_zero(n):
    """Tilted planar dielectric interface with surface charge: the piecewise
    quadratic with eps_g A_g - eps_d A_d = -sigma/eps0 has zero truncation error
    on every row off the walls (Eq. matching with phi_B eliminated, in 3D)."""
    eg, ed, sigma, Ad = 1.0, 4.0, 0.7, 1.3
    nv = np.array([0.25, 0.15, 0.95])
    nv /= np.linalg.norm(nv)
    x0 = np.array([0.45, 0.5, 0.52])
    c0 = nv @ x0
    d = W._desc(3, (n, n, n), (0, 0, 0), 1.0 / n, [(W.PRIM_HALFSPACE, [nv[0], nv[1], nv[2], c0])], [(0, 0, 0)], -1,
                0, (eg, ed), [1] * 6, 0.0, [0] * 6)
    Ag = (-sigma + ed * Ad) / eg

    def ph(q, x, y, z):
        u = nv[0] * x + nv[1] * y + nv[2] * z - c0
        return (Ag if q == 0 else Ad) * u + (x - x0[0]) ** 2 + (y - x0[1]) ** 2 + (z - x0[2]) ** 2
    g = oracle.Geometry(d)
    s = np.zeros((2, g.ncell))
    s[0] = -eg * 6.0
    s[1] = -ed * 6.0
    pd = np.stack([_wall_values(g, lambda x, y, z: ph(0, x, y, z)), _wall_values(g, lambda x, y, z: ph(1, x, y, z))])
    data = g.data(s=s, sigma=np.full(g.ncell, sigma), phidom=pd)
    A, b = g.assemble(data)
    X, Y, Z = g.cell_centres()
    xe = g.to_dofs(np.stack([ph(0, X, Y, Z), ph(1, X, Y, Z)]))
    rows = _interior_rows(g)
    iface = np.concatenate([g.dof[p][(g.ebkind == oracle.EB_INTERFACE) & (g.dof[p] >= 0)] for p in range(2)])
    assert len(np.intersect1d(rows, iface)) > n
    r = (A @ xe - b)[rows]
    assert np.abs(r).max() <= 1e-10 * np.abs(b).max()
    # the same problem with the surface charge sign flipped is not reproduced
    data2 = g.data(s=s, sigma=np.full(g.ncell, -sigma), phidom=pd)
    A2, b2 = g.assemble(data2)
    assert np.abs((A2 @ xe - b2)[rows]).max() > 1e-3 * np.abs(b2).max()


def _concentric(n, sigma, R0=0.3, R1=0.6, R2=0.9, eg=1.0, ed=4.0, phi0=1.0):
    h = 2.0 / n
    prims = [(W.PRIM_SPHERE, [0, 0, 0, R0]), (W.PRIM_SPHERE, [0, 0, 0, R2]), (W.PRIM_SPHERE, [0, 0, 0, R1])]
    nodes = [(0, 0, 0), (0, 1, 0), (3, 1, 0), (1, 0, 2), (0, 2, 0)]
    d = W._desc(3, (n, n, n), (-1, -1, -1), h, prims, nodes, 3, 4, (eg, ed), [1] * 6, phi0, [0] * 6,
                electrodes=[(0, phi0), (2, 0.0)])
    g = oracle.Geometry(d)
    data = g.data(sigma=np.full(g.ncell, sigma))
    A, b = g.assemble(data)
    P = g.to_cells(oracle.solve_system(A, b))
    X, Y, Z = g.cell_centres()
    r = np.sqrt(X * X + Y * Y + Z * Z)
    # eps_q r^2 phi_q' = c_q, c_g - c_d = -sigma R1^2
    cd = (-phi0 - sigma * R1 * R1 * (1 / R2 - 1 / R1) / eg) / ((1 / R0 - 1 / R1) / ed - (1 / R2 - 1 / R1) / eg)
    cg = cd - sigma * R1 * R1
    pd_ = -cd / (ed * r) + phi0 + cd / (ed * R0)
    pg_ = -cg / (eg * r) + cg / (eg * R2)
    e = np.concatenate([np.abs(P[0][g.dof[0] >= 0] - pg_[g.dof[0] >= 0]),
                        np.abs(P[1][g.dof[1] >= 0] - pd_[g.dof[1] >= 0])])
    return e.max(), math.sqrt(np.mean(e * e))


@pytest.mark.parametrize("sigma", [0.0, 0.7])
def test_concentric_spheres_second_order(sigma):
    errs = [_concentric(n, sigma) for n in (16, 32)]
    r2 = math.log2(errs[0][1] / errs[1][1])
    rinf = math.log2(errs[0][0] / errs[1][0])
    assert r2 > 1.8, errs
    assert rinf > 1.5, errs
    assert errs[1][0] < 0.05


def test_conservation_identity_3d():
    desc = W.pin_plane_3d(16, radius=0.12)
    g = oracle.Geometry(desc)
    data = g.data(s=np.zeros((2, g.ncell)))
    A, b = g.assemble(data)
    rng = np.random.default_rng(3)
    phi = rng.normal(size=g.ndof)
    Lphi = -(A @ phi) + b
    lhs = g.h ** 3 * Lphi.sum()
    rhs = g.boundary_flux(data, phi)
    assert abs(lhs - rhs) < 1e-12 * g.h ** 3 * np.abs(Lphi).sum()


def test_dense_solve_matches_3d():
    desc = W.pin_plane_3d(8, radius=0.15, disk_r=0.35, disk_t=0.2)
    g = oracle.Geometry(desc)
    A, b = g.assemble(g.data())
    x1 = oracle.solve_system(A, b)
    x2 = np.linalg.solve(A.toarray(), b)
    assert np.abs(x1 - x2).max() <= 1e-12 * np.abs(x2).max()


def test_sphere_volume_second_order():
    errs = []
    for n in (16, 32):
        d = W._desc(3, (n, n, n), (0, 0, 0), 1.0 / n, [(W.PRIM_SPHERE, [0.52, 0.47, 0.5, 0.31])], [(0, 0, 0)], 0, -1,
                    (1.0, 1.0), [1] * 6, 0.0, [0] * 6)
        g = oracle.Geometry(d)
        vol = g.kappa[0].sum() * g.h ** 3
        errs.append(abs(vol - (1.0 - 4.0 / 3.0 * math.pi * 0.31 ** 3)))
    assert math.log2(errs[0] / errs[1]) > 1.8, errs


def test_pin_plane_solution_mirror_symmetric():
    """The pin-plane geometry and line charge are symmetric under x -> 1-x,
    y -> 1-y and x <-> y; so is the discrete solution (the EB centroid of a
    curved cut is fanned about the crossing loop's vertex mean, independent of
    where the loop starts)."""
    n = 24
    d, S, s = W.c3_inputs(n)
    g, phi, A, b, data = oracle.solve(d, s=S, sigma=s)
    f = phi[0].reshape(n, n, n)
    m = np.abs(f).max()
    assert np.abs(f - f[:, :, ::-1]).max() <= 1e-12 * m
    assert np.abs(f - f[:, ::-1, :]).max() <= 1e-12 * m
    assert np.abs(f - f.transpose(0, 2, 1)).max() <= 1e-12 * m
    k = g.kappa[0].reshape(n, n, n)
    assert np.abs(k - k[:, :, ::-1]).max() <= 1e-13


def test_field_exact_for_quadratic_3d():
    """E = -grad phi (Sec. 2.1) of a full quadratic (cross terms included) with a
    tilted planar electrode: centred differences at cell centres and the ray-cast
    EB stencil at electrode centroids away from the walls are exact."""
    n = 16
    c = np.random.default_rng(7).normal(size=10)

    def phi(x, y, z):
        return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * y + c[6] * z * z + c[7] * x * y
                + c[8] * y * z + c[9] * x * z)

    def grad(x, y, z):
        return np.stack([c[1] + 2 * c[4] * x + c[7] * y + c[9] * z, c[2] + 2 * c[5] * y + c[7] * x + c[8] * z,
                         c[3] + 2 * c[6] * z + c[8] * y + c[9] * x])
    nv = np.array([0.3, 0.5, 0.81])
    nv /= np.linalg.norm(nv)
    dd = nv @ np.array([0.37, 0.41, 0.45])
    d = W._desc(3, (n, n, n), (0, 0, 0), 1.0 / n, [(W.PRIM_HALFSPACE, [nv[0], nv[1], nv[2], dd])], [(0, 0, 0)], 0,
                -1, (1.0, 1.0), [1] * 6, 0.0, [0] * 6)
    g = oracle.Geometry(d)
    pd = _wall_values(g, phi)
    data = g.data(s=np.zeros((2, g.ncell)), phiE=phi(g.ebx[:, 0], g.ebx[:, 1], g.ebx[:, 2]),
                  phidom=np.stack([pd, pd]))
    X, Y, Z = g.cell_centres()
    E, En = g.field(data, g.to_dofs(np.stack([phi(X, Y, Z)] * 2)))
    idx = np.arange(g.ncell)
    i, j, k = idx % n, (idx // n) % n, idx // (n * n)
    dof = g.dof[0]
    inner = idx[(i > 0) & (i < n - 1) & (j > 0) & (j < n - 1) & (k > 0) & (k < n - 1) & (dof >= 0) & (g.cut == 0)]
    both = inner[(dof[inner - 1] >= 0) & (dof[inner + 1] >= 0) & (dof[inner - n] >= 0) & (dof[inner + n] >= 0)
                 & (dof[inner - n * n] >= 0) & (dof[inner + n * n] >= 0)]
    assert len(both) > 1000
    assert np.abs(E[:, 0, both] + grad(X, Y, Z)[:, both]).max() < 1e-12
    m = 3
    eb = np.nonzero((g.ebkind == oracle.EB_ELECTRODE) & (i >= m) & (i < n - m) & (j >= m) & (j < n - m)
                    & (k >= m) & (k < n - m))[0]
    assert len(eb) > 100
    dn = (grad(g.ebx[eb, 0], g.ebx[eb, 1], g.ebx[eb, 2]).T * -g.ebn[eb]).sum(1)
    assert np.abs(En[eb, 0] + dn).max() < 1e-12 * np.abs(dn).max() + 1e-13

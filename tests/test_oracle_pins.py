"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Every check here is independent of the oracle's own formulas: closed-form
solutions (Sec. 4.2), exactness for quadratics (the discretisation of
Sec. 3.3 is second order, so every stencil in it reproduces quadratics), exact
polygon clipping for planar cuts (Sec. 3.1 linearises the boundary), the
telescoping of conservative fluxes (the integral form, Eq. poisson_integral),
a dense LAPACK solve, and mirror symmetry.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1809_03745_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _wall_values(g, f):
    return np.concatenate([f(x, y, z) for _, x, y, z in g.wall_face_centres()])


def _coax_errors(n, sigma, gold):
    desc = W.coaxial_2d(n, R0=gold["R0"], R1=gold["R1"], R2=gold["R2"], eps=gold["eps_dielectric"],
                        phi0=gold["phi0"])
    g = oracle.Geometry(desc)
    data = g.data(sigma=np.full(g.ncell, sigma))
    A, b = g.assemble(data)
    phi = g.to_cells(oracle.solve_system(A, b))
    X, Y, _ = g.cell_centres()
    pg, pd = W.coaxial_exact(np.hypot(X, Y), R0=gold["R0"], R1=gold["R1"], R2=gold["R2"],
                             eps_d=gold["eps_dielectric"], phi0=gold["phi0"], sigma=sigma)
    e = np.concatenate([np.abs(phi[p][g.dof[p] >= 0] - ex[g.dof[p] >= 0]) for p, ex in ((0, pg), (1, pd))])
    return e.max(), math.sqrt(np.mean(e ** 2)), g


@pytest.mark.parametrize("sigma", [0.0, 0.7, -1.3])
def test_coaxial_closed_form_second_order(sigma):
    """Sec. 4.2: the coaxial multi-fluid problem converges at second order to the
    closed form; with a surface charge on R1 the closed form pins the sign of
    the matching condition (eps_g d/dn_g + eps_d d/dn_d = -sigma/eps0)."""
    gold = json.load(open(os.path.join(GOLDEN, "coaxial_sec4_2.json")))
    errs = [_coax_errors(n, sigma, gold) for n in (64, 128, 256)]
    linf = [e[0] for e in errs]
    l2 = [e[1] for e in errs]
    r_l2 = math.log2(l2[0] / l2[2]) / 2
    r_inf = math.log2(linf[1] / linf[2])
    assert r_l2 > 1.8, (l2, r_l2)
    assert r_inf > 1.8, (linf, r_inf)
    assert linf[2] < 2e-4
    for _, _, g in errs:
        assert g.stencil_counts["order1"] == 0 and g.stencil_counts["ls"] == 0


def _quad_single(desc, coef):
    a, b, c, d, e, f = coef
    phi = lambda x, y, z: a + b * x + c * y + d * x * x + e * x * y + f * y * y  # noqa: E731
    g = oracle.Geometry(desc)
    eps = desc["eps"][0]
    s = np.full((2, g.ncell), -eps * (2 * d + 2 * f))
    pe = phi(g.ebx[:, 0], g.ebx[:, 1], 0)
    pd = _wall_values(g, phi)
    data = g.data(s=s, phiE=pe, phidom=np.stack([pd, pd]))
    A, bb = g.assemble(data)
    x = oracle.solve_system(A, bb)
    X, Y, Z = g.cell_centres()
    ex = phi(X, Y, Z)
    m = g.dof[0] >= 0
    return g, data, x, np.abs(g.to_cells(x)[0][m] - ex[m]).max() / np.abs(ex).max()


@pytest.mark.parametrize("n", [32, 64])
@pytest.mark.parametrize("geom", ["circle", "rod"])
def test_quadratic_exactness_single_phase(n, geom):
    """Face-centred differences, centroid interpolation (Sec. 3.3), the one-sided
    wall formula and the ray-cast EB derivative (Sec. 3.3.1) are all exact for
    quadratics, and the moments are divergence-consistent: the discrete solution
    equals the quadratic at cell centres when no fallback stencil fires."""
    rng = np.random.default_rng(n + len(geom))
    if geom == "circle":
        desc = W._desc(2, (n, n), (0, 0), 1.0 / n, [(W.PRIM_SPHERE, [0.52, 0.47, 0, 0.23])], [(0, 0, 0)], 0, -1,
                       (1.0, 1.0), [1, 1, 1, 1, 0, 0], 0.0, [0] * 6)
    else:
        desc = W.rod_plane_2d(n, all_dirichlet=True)
    g, _, _, err = _quad_single(desc, rng.normal(size=6))
    assert g.stencil_counts["order1"] == 0 and g.stencil_counts["ls"] == 0
    assert err < 1e-12, err


def _tilted(n, th=0.25, px=0.45, py=0.5, sigma=0.7, eg=1.0, ed=4.0, Ad=1.3):
    nx, ny = math.cos(th), math.sin(th)
    c0 = px * nx + py * ny
    desc = W._desc(2, (n, n), (0, 0), 1.0 / n, [(W.PRIM_HALFSPACE, [nx, ny, 0, c0])], [(0, 0, 0)], -1, 0,
                   (eg, ed), [1, 1, 1, 1, 0, 0], 0.0, [0] * 6)
    Ag = (-sigma + ed * Ad) / eg

    def ph(q, x, y, z):
        u = nx * x + ny * y - c0
        return (Ag if q == 0 else Ad) * u + (x - px) ** 2 + (y - py) ** 2
    g = oracle.Geometry(desc)
    s = np.zeros((2, g.ncell))
    s[0] = -eg * 4.0
    s[1] = -ed * 4.0
    pd = np.stack([_wall_values(g, lambda x, y, z: ph(0, x, y, z)), _wall_values(g, lambda x, y, z: ph(1, x, y, z))])
    data = g.data(s=s, sigma=np.full(g.ncell, sigma), phidom=pd)
    return g, data, ph


@pytest.mark.parametrize("n", [32, 48, 64])
def test_quadratic_exactness_multifluid(n):
    """Piecewise quadratic across a tilted planar dielectric interface, continuous,
    with eps_g A_g - eps_d A_d = -sigma/eps0: the matching condition Eq. (matching)
    with phi_B eliminated (Sec. 3.3.1) reproduces it exactly."""
    g, data, ph = _tilted(n)
    A, b = g.assemble(data)
    x = oracle.solve_system(A, b)
    X, Y, Z = g.cell_centres()
    P = g.to_cells(x)
    assert g.stencil_counts["order1"] == 0 and g.stencil_counts["ls"] == 0
    assert (g.ebkind == oracle.EB_INTERFACE).sum() > n // 2
    for q in (0, 1):
        m = g.dof[q] >= 0
        assert np.abs(P[q][m] - ph(q, X, Y, Z)[m]).max() < 1e-12


def test_multifluid_sign_plant():
    """The same tilted-interface problem with the surface-charge sign flipped in
    the data is *not* reproduced: the exactness pin is sensitive to the sign."""
    g, data, ph = _tilted(32)
    dt, keep = data
    flipped = g.data(s=keep[0].reshape(2, -1), sigma=-keep[1], phidom=keep[3].reshape(2, -1))
    A, b = g.assemble(flipped)
    P = g.to_cells(oracle.solve_system(A, b))
    X, Y, Z = g.cell_centres()
    m = g.dof[0] >= 0
    assert np.abs(P[0][m] - ph(0, X, Y, Z)[m]).max() > 1e-3


def _clip(poly, nx, ny, c):
    """Sutherland-Hodgman: keep the part of poly with nx*x + ny*y >= c."""
    out = []
    for k in range(len(poly)):
        P, Q = poly[k], poly[(k + 1) % len(poly)]
        fp, fq = nx * P[0] + ny * P[1] - c, nx * Q[0] + ny * Q[1] - c
        if fp >= 0:
            out.append(P)
        if (fp >= 0) != (fq >= 0):
            t = fp / (fp - fq)
            out.append((P[0] + t * (Q[0] - P[0]), P[1] + t * (Q[1] - P[1])))
    return out


def _area(poly):
    return 0.5 * sum(poly[k][0] * poly[(k + 1) % len(poly)][1] - poly[(k + 1) % len(poly)][0] * poly[k][1]
                     for k in range(len(poly)))


def test_planar_cut_moments_exact():
    """Sec. 3.1: inside a cut cell the boundary is a straight line, so for a planar
    electrode the volume fraction, the face apertures and the EB area are the
    exact clipped-polygon values."""
    n = 24
    th = 0.7
    nx, ny = math.cos(th), math.sin(th)
    c = 0.31 * nx + 0.58 * ny
    # electrode where n.x < c  -> fluid where n.x >= c
    desc = W._desc(2, (n, n), (0, 0), 1.0 / n, [(W.PRIM_HALFSPACE, [nx, ny, 0, c])], [(0, 0, 0)], 0, -1,
                   (1.0, 1.0), [1, 1, 1, 1, 0, 0], 1.0, [0] * 6)
    g = oracle.Geometry(desc)
    h = 1.0 / n
    ax, fx = g.faces(0)
    ay, fy = g.faces(1)
    checked = 0
    for cidx in np.nonzero(g.cut)[0]:
        i, j = cidx % n, cidx // n
        sq = [(i * h, j * h), ((i + 1) * h, j * h), ((i + 1) * h, (j + 1) * h), (i * h, (j + 1) * h)]
        poly = _clip(sq, nx, ny, c)
        kap = _area(poly) / h ** 2 if len(poly) >= 3 else 0.0
        assert abs(g.kappa[0, cidx] - kap) < 1e-12
        # EB chord length
        pts = [p for p in poly if abs(nx * p[0] + ny * p[1] - c) < 1e-12]
        if len(pts) == 2:
            chord = math.hypot(pts[0][0] - pts[1][0], pts[0][1] - pts[1][1]) / h
            assert abs(g.eba[cidx] - chord) < 1e-12
            assert abs(g.ebn[cidx, 0] + nx) < 1e-12 and abs(g.ebn[cidx, 1] + ny) < 1e-12
            checked += 1
        # apertures of the lo x-face and lo y-face: clipped segment lengths
        x0 = i * h
        lo_x = ((j + 1) * h - max(j * h, min((j + 1) * h, (c - nx * x0) / ny))) / h
        assert abs(ax[0, i + (n + 1) * j] - lo_x) < 1e-12, (i, j)
    assert checked > n // 2


def test_volume_of_annulus_second_order():
    """Sum of volume fractions over the coaxial annulus converges to
    pi (R2^2 - R0^2) at second order (linearised circle)."""
    errs = []
    for n in (64, 128, 256):
        g = oracle.Geometry(W.coaxial_2d(n))
        area = (g.kappa[0].sum() + g.kappa[1].sum()) * g.h ** 2
        errs.append(abs(area - math.pi * (0.9 ** 2 - 0.3 ** 2)))
        diel = g.kappa[1].sum() * g.h ** 2
        assert abs(diel - math.pi * (0.6 ** 2 - 0.3 ** 2)) < 20 * g.h ** 2
    assert math.log2(errs[0] / errs[2]) / 2 > 1.8, errs


def test_conservation_identity():
    """Integral form Eq. (poisson_integral): for ANY phi, h^D sum_i (L phi)_i equals
    the net outward flux through the walls and electrode EBs plus the interface
    surface charge; interior centroid fluxes cancel face by face."""
    desc, S, sig = W.c2_inputs(64)
    g = oracle.Geometry(desc)
    data = g.data(s=np.zeros((2, g.ncell)), sigma=sig)
    A, b = g.assemble(data)
    rng = np.random.default_rng(7)
    for _ in range(3):
        phi = rng.normal(size=g.ndof)
        Lphi = -(A @ phi) + b          # s = 0, so b holds only the data terms
        lhs = g.h ** 2 * Lphi.sum()
        rhs = g.boundary_flux(data, phi)
        scale = g.h ** 2 * np.abs(Lphi).sum()
        assert abs(lhs - rhs) < 1e-12 * scale, (lhs, rhs, scale)


@pytest.mark.parametrize("which", ["c2", "coax"])
def test_dense_solve_matches(which):
    """A dense LAPACK solve and the sparse LU agree on small grids (<= 32^2)."""
    if which == "c2":
        desc, S, sig = W.c2_inputs(32)
    else:
        desc, S, sig = W.coaxial_2d(32), None, None
    g = oracle.Geometry(desc)
    data = g.data(s=S, sigma=sig)
    A, b = g.assemble(data)
    x1 = oracle.solve_system(A, b)
    x2 = np.linalg.solve(A.toarray(), b)
    assert np.abs(x1 - x2).max() <= 1e-12 * np.abs(x2).max()


def test_mirror_symmetry_rod_plane():
    """The rod-plane problem without noise is symmetric about x = 1/2."""
    n = 64
    desc, S, sig = W.c1_inputs(n, noise=0.0)
    g, phi, A, b, data = oracle.solve(desc, s=S, sigma=sig)
    P = phi[0].reshape(n, n)
    assert np.abs(P - P[:, ::-1]).max() < 1e-12


def test_field_exact_for_quadratic():
    """Centred differences and the EB ray stencil are exact for quadratics: the
    cell-centre field and the EB normal field of the quadratic solution match
    -grad phi exactly where both neighbours exist / at EB centroids."""
    n = 48
    coef = (0.3, -1.1, 0.7, 0.9, -0.4, 1.6)
    a, b_, c, d, e, f = coef
    desc = W._desc(2, (n, n), (0, 0), 1.0 / n, [(W.PRIM_SPHERE, [0.52, 0.47, 0, 0.23])], [(0, 0, 0)], 0, -1,
                   (1.0, 1.0), [1, 1, 1, 1, 0, 0], 0.0, [0] * 6)
    g, data, x, err = _quad_single(desc, coef)
    E, En = g.field(data, x)
    X, Y, _ = g.cell_centres()
    gx = b_ + 2 * d * X + e * Y
    gy = c + e * X + 2 * f * Y
    dof = g.dof[0]
    # cells whose both x- and y-neighbours carry dofs (centred differences)
    ii, jj = np.arange(g.ncell) % n, np.arange(g.ncell) // n
    inner = (dof >= 0) & (ii > 0) & (ii < n - 1) & (jj > 0) & (jj < n - 1)
    idx = np.nonzero(inner)[0]
    both = idx[(dof[idx - 1] >= 0) & (dof[idx + 1] >= 0) & (dof[idx - n] >= 0) & (dof[idx + n] >= 0)
               & (g.cut[idx] == 0)]
    assert np.abs(E[0, 0, both] + gx[both]).max() < 1e-9
    assert np.abs(E[1, 0, both] + gy[both]).max() < 1e-9
    eb = np.nonzero(g.ebkind == oracle.EB_ELECTRODE)[0]
    xb, yb = g.ebx[eb, 0], g.ebx[eb, 1]
    nin = -g.ebn[eb, :2]
    dn = (b_ + 2 * d * xb + e * yb) * nin[:, 0] + (c + e * xb + 2 * f * yb) * nin[:, 1]
    assert np.abs(En[eb, 0] + dn).max() < 1e-9


def test_manufactured_harmonic_convergence():
    """phi = sin(pi x) cosh(pi y) (harmonic) on the rod-plane geometry with
    Dirichlet data on every wall and on the rod: second order in L-infinity."""
    errs = []
    for n in (64, 128, 256):
        desc = W.rod_plane_2d(n, all_dirichlet=True)
        f = lambda x, y, z: np.sin(np.pi * x) * np.cosh(np.pi * y)  # noqa: E731
        g = oracle.Geometry(desc)
        pe = f(g.ebx[:, 0], g.ebx[:, 1], 0)
        pd = _wall_values(g, f)
        data = g.data(s=np.zeros((2, g.ncell)), phiE=pe, phidom=np.stack([pd, pd]))
        A, b = g.assemble(data)
        x = oracle.solve_system(A, b)
        X, Y, Z = g.cell_centres()
        m = g.dof[0] >= 0
        errs.append(np.abs(g.to_cells(x)[0][m] - f(X, Y, Z)[m]).max())
    assert math.log2(errs[0] / errs[1]) > 1.8 and math.log2(errs[1] / errs[2]) > 1.8, errs


def test_rejects_cell_cut_by_both_interfaces():
    """A cell cut by the electrode and by the dielectric at once is outside the
    method's single-interface-per-cell model and is rejected."""
    desc = W.rod_plane_2d(32, dielectric=True, tip_y=0.21, slab_y=0.2, rough_amp=0.0)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.Geometry(desc)
    assert ei.value.status == oracle.UNSUPPORTED


@pytest.mark.parametrize("dim", [2, 3])
def test_interface_field_satisfies_matching_condition(dim):
    """Eq. (matching): eps_g dphi/dn_g + eps_d dphi/dn_d = -sigma/eps0 at every
    dielectric EB.  With phi_B eliminated (Sec. 3.3.1) the two one-sided normal
    derivatives satisfy it for any phi, so the EB normal field En = -dphi/dn_in
    of both phases must give eps_g En_g + eps_d En_d = sigma/eps0 exactly, for
    random phi and a random sigma per cell; eps_g != eps_d catches a swap."""
    eg, ed = 1.0, 4.0
    if dim == 2:
        n = 32
        desc = W._desc(2, (n, n), (0, 0), 1.0 / n, [(W.PRIM_SPHERE, [0.48, 0.53, 0, 0.27])], [(0, 0, 0)], -1, 0,
                       (eg, ed), [1, 1, 1, 1, 0, 0], 0.0, [0] * 6)
    else:
        n = 16
        desc = W._desc(3, (n, n, n), (0, 0, 0), 1.0 / n, [(W.PRIM_SPHERE, [0.48, 0.53, 0.51, 0.3])], [(0, 0, 0)],
                       -1, 0, (eg, ed), [1] * 6, 0.0, [0] * 6)
    g = oracle.Geometry(desc)
    rng = np.random.default_rng(dim)
    sigma = rng.uniform(-1.0, 1.0, size=g.ncell)
    data = g.data(sigma=sigma)
    E, En = g.field(data, rng.normal(size=g.ndof))
    ib = np.nonzero((g.ebkind == oracle.EB_INTERFACE) & (g.dof[0] >= 0) & (g.dof[1] >= 0))[0]
    assert len(ib) > 20
    r = eg * En[ib, 0] + ed * En[ib, 1] - sigma[ib]
    assert np.abs(r).max() <= 1e-10 * np.abs(En[ib]).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_exactness_with_first_order_eb_stencils(dim):
    """A tilted slot between two electrodes, 1.3 cells wide in 2D and 1.6 in 3D:
    most EB stencils fall back to first order (one plane, (bi)linear transverse
    interpolation; Sec. 3.3.1 allows it where the second plane is not in the
    fluid), which is still exact for linear phi.  The truncation error and the
    EB normal field of a linear phi vanish."""
    n = 32 if dim == 2 else 16
    h = 1.0 / n
    if dim == 2:
        nv, p0, width = np.array([-math.sin(0.2), math.cos(0.2), 0.0]), np.array([0.5, 0.45, 0.0]), 1.3 * h
    else:
        nv, p0, width = np.array([0.15, -0.2, 1.0]), np.array([0.5, 0.5, 0.45]), 1.6 * h
        nv /= np.linalg.norm(nv)
    # electrode: below the plane through p0 or above its copy `width` higher
    prims = [(W.PRIM_HALFSPACE, [nv[0], nv[1], nv[2], nv @ p0]),
             (W.PRIM_HALFSPACE, [-nv[0], -nv[1], -nv[2], -(nv @ p0 + width)])]
    bc = [1, 1, 0, 0, 0, 0] if dim == 2 else [1, 1, 1, 1, 0, 0]
    d = W._desc(dim, (n,) * dim, (0,) * dim, h, prims, [(0, 0, 0), (0, 1, 0), (1, 0, 1)], 2, -1, (1.0, 1.0), bc,
                0.0, [0] * 6)
    g = oracle.Geometry(d)
    assert g.stencil_counts["order1"] > 40
    a = np.array([0.3, -1.7, 2.3, 0.9 if dim == 3 else 0.0])

    def phi(x, y, z):
        return a[0] + a[1] * x + a[2] * y + a[3] * z
    pd = _wall_values(g, phi)
    data = g.data(s=np.zeros((2, g.ncell)), phiE=phi(g.ebx[:, 0], g.ebx[:, 1], g.ebx[:, 2]),
                  phidom=np.stack([pd, pd]))
    A, b = g.assemble(data)
    X, Y, Z = g.cell_centres()
    xe = g.to_dofs(np.stack([phi(X, Y, Z)] * 2))
    assert np.abs(A @ xe - b).max() <= 1e-12 * np.abs(b).max()
    E, En = g.field(data, xe)
    eb = np.nonzero(g.ebkind == oracle.EB_ELECTRODE)[0]
    dn = -(g.ebn[eb] @ a[1:])
    assert np.abs(En[eb, 0] + dn).max() <= 1e-12 * np.abs(dn).max()


def _wedge(dim):
    if dim == 2:
        return W.fluid_wedge(2, 32)
    return W.fluid_wedge(3, 16, half=0.45, angle=1.2, tilt=0.2)


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_exactness_with_least_squares_eb_stencils(dim):
    """At the apex of an acute fluid wedge neither ray stencil of Sec. 3.3.1
    finds its interpolation cells in the fluid, and the EB normal derivative
    falls back to the least-squares fit of phi_B + g.(x - x_B) over the fluid
    neighbours on the fluid side.  That fit reproduces any linear phi, so the
    truncation error and the EB normal field of a linear phi vanish there too.
    The same geometry also carries first-order and ray stencils."""
    g = oracle.Geometry(_wedge(dim))
    c = g.stencil_counts
    assert c["ls"] >= (2 if dim == 2 else 30) and c["order1"] > 0 and c["order2"] > 0, c
    order = g.stencil_order()
    ls_cells = np.nonzero(order[0] == 3)[0]
    assert len(ls_cells) == c["ls"]
    a = np.array([0.3, -1.7, 2.3, 0.9 if dim == 3 else 0.0])

    def phi(x, y, z):
        return a[0] + a[1] * x + a[2] * y + a[3] * z
    pd = _wall_values(g, phi)
    data = g.data(s=np.zeros((2, g.ncell)), phiE=phi(g.ebx[:, 0], g.ebx[:, 1], g.ebx[:, 2]),
                  phidom=np.stack([pd, pd]))
    A, b = g.assemble(data)
    X, Y, Z = g.cell_centres()
    xe = g.to_dofs(np.stack([phi(X, Y, Z)] * 2))
    assert np.abs(A @ xe - b).max() <= 1e-12 * np.abs(b).max()
    # the least-squares cells' own rows, checked on their own as well
    rows = g.dof[0, ls_cells]
    assert np.abs((A @ xe - b)[rows]).max() <= 1e-12 * np.abs(b).max()
    E, En = g.field(data, xe)
    dn = -(g.ebn[ls_cells] @ a[1:])
    assert np.abs(En[ls_cells, 0] + dn).max() <= 1e-12 * np.abs(a).max()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("offset", [0.0, -1e-10, 1e-10])
def test_quadratic_exactness_with_eb_on_grid_faces(dim, offset):
    """An electrode whose surface lies on a plane of cell faces, exactly or
    within the crossing snap distance (1e-8 h).  Just below that plane each
    cell keeps a fluid fragment of zero volume whose top face is open: it
    carries an unknown whose row equates the face flux with the EB flux
    (reading: a fragment has an unknown when it has an open face).  Above
    the plane the cells are full, and where the surface lies just above the
    plane (offset +1e-10) the EB sits on their bottom faces instead.  In both
    forms the face flux (phi_above - phi_below)/h is the derivative at the
    face for a quadratic, so the discrete solution equals a quadratic phi at
    every unknown, the zero-volume ones included."""
    n = 32 if dim == 2 else 16
    h = 1.0 / n
    y0 = 0.5 + offset
    prims = [(W.PRIM_HALFSPACE, [0.0, 1.0, 0.0, y0])]
    bc = [1, 1, 1, 1, 0, 0] if dim == 2 else [1] * 6
    d = W._desc(dim, (n,) * dim, (0,) * dim, h, prims, [(0, 0, 0)], 0, -1, (1.0, 1.0), bc, 0.0, [0] * 6)
    g = oracle.Geometry(d)
    sliver = np.nonzero((g.dof[0] >= 0) & (g.kappa[0] < 1e-12))[0]
    nplane = n ** (dim - 1)
    assert len(sliver) == (0 if offset > 0 else nplane)
    assert g.n_eb == nplane
    co = np.array([0.3, -0.7, 1.1, 0.8, -0.6, 0.5, 0.4 if dim == 3 else 0.0, 0.2 if dim == 3 else 0.0])

    def phi(x, y, z):
        return (co[0] + co[1] * x + co[2] * y + co[3] * x * x + co[4] * x * y + co[5] * y * y + co[6] * z * z
                + co[7] * y * z)
    lap = 2 * co[3] + 2 * co[5] + 2 * co[6]
    s = np.full((2, g.ncell), -lap)
    pd = _wall_values(g, phi)
    data = g.data(s=s, phiE=phi(g.ebx[:, 0], g.ebx[:, 1], g.ebx[:, 2]), phidom=np.stack([pd, pd]))
    A, bb = g.assemble(data)
    x = g.to_cells(oracle.solve_system(A, bb))[0]
    X, Y, Z = g.cell_centres()
    ex = phi(X, Y, Z)
    m = g.dof[0] >= 0
    assert np.abs(x[m] - ex[m]).max() <= 1e-12 * np.abs(ex).max()
    if len(sliver):
        assert np.abs(x[sliver] - ex[sliver]).max() <= 1e-12 * np.abs(ex).max()

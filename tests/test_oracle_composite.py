"""Pins of the oracle's composite (one refined box) operator.

- quadratic exactness in 2D with an electrode off the box: tangential and
  normal CF interpolation are exact for quadratics, the refluxed coarse flux
  is the exact face mean, so the truncation error vanishes on every row;
- in 3D the same for quadratics without cross terms (the tangential step
  adds the two 1-D corrections, no cross term);
- exact conservation for arbitrary phi with the rod crossing the box sides
  (cut CF faces): the fine fluxes through every CF face enter the coarse row
  with the opposite sign; the same in 3D with a pin through the top side, and
  a planted mistake (the coarse operator's own CF-side flux kept) breaks it;
- second-order convergence of the coaxial closed form (Sec. 4.2) with a box
  in the gas shell;
- a box covering the whole domain reduces to the plain fine-grid problem;
- a dielectric unknown next to a CF side is rejected;
- planted mistakes (linear tangential weights, a linear normal step) break
  the exactness pin.
"""
import math

import numpy as np
import pytest

import oracle
from oracle.composite import Composite
from paper_1809_03745_gb300 import workloads as W


def _walls(g, f):
    return np.concatenate([f(x, y, z) for _, x, y, z in g.wall_face_centres()])


def _quadratic_truncation(C, phi, lap):
    gc, gf = C.gc, C.gf
    pdc, pdf = _walls(gc, phi), _walls(gf, phi)
    A, b = C.assemble(sc=np.full((2, gc.ncell), -lap), sf=np.full((2, gf.ncell), -lap),
                      phiEc=phi(gc.ebx[:, 0], gc.ebx[:, 1], gc.ebx[:, 2]),
                      phiEf=phi(gf.ebx[:, 0], gf.ebx[:, 1], gf.ebx[:, 2]),
                      phidomc=np.stack([pdc, pdc]), phidomf=np.stack([pdf, pdf]))
    Xc, Yc, Zc = gc.cell_centres()
    Xf, Yf, Zf = gf.cell_centres()
    x = C.join(np.stack([phi(Xc, Yc, Zc)] * 2), np.stack([phi(Xf, Yf, Zf)] * 2))
    return np.abs(A @ x - b).max() / np.abs(b).max(), A, b, x


def test_composite_quadratic_exactness_2d():
    n = 32
    d = W._desc(2, (n, n), (0, 0), 1.0 / n, [(W.PRIM_SPHERE, [0.2, 0.2, 0.0, 0.1])], [(0, 0, 0)], 0, -1,
                (1.0, 1.0), [1] * 4 + [0, 0], 0.0, [0] * 6)
    C = Composite(d, [16, 16], [24, 24])
    c = np.array([0.3, -0.7, 0.4, 1.1, -0.6, 0.9])

    def phi(x, y, z):
        return c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * y * y + c[5] * x * y
    rel, A, b, x = _quadratic_truncation(C, phi, 2 * (c[3] + c[4]))
    assert len(C.faces) == 4 * 16
    assert rel <= 1e-12
    assert np.abs(oracle.solve_system(A, b) - x).max() <= 1e-11


def test_composite_quadratic_exactness_3d_no_cross_terms():
    n = 16
    d = W._desc(3, (n, n, n), (0, 0, 0), 1.0 / n, [], [], -1, -1, (1.0, 1.0), [1] * 6, 0.0, [0] * 6)
    C = Composite(d, [4, 6, 5], [12, 10, 11])
    c = np.array([0.2, 0.5, -0.3, 0.8, 1.3, -0.4, 0.7])

    def phi(x, y, z):
        return c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * y + c[6] * z * z
    rel, A, b, x = _quadratic_truncation(C, phi, 2 * (c[4] + c[5] + c[6]))
    assert rel <= 1e-12


def test_composite_conservation_with_cut_cf_faces():
    d = W.rod_plane_2d(32)
    C = Composite(d, [12, 12], [20, 20])
    gc, gf = C.gc, C.gf
    assert any(gf.cut[f[2]] for f in C.faces)  # the rod crosses a CF side
    A, b = C.assemble(sc=np.zeros((2, gc.ncell)), sf=np.zeros((2, gf.ncell)))
    x = np.random.default_rng(1).normal(size=C.n)
    vol = np.concatenate([np.full(C.nco, gc.h ** 2), np.full(gf.ndof, gf.h ** 2)])
    terms = vol * (b - A @ x)
    assert abs(terms.sum() - C.boundary_flux(x)) <= 1e-12 * np.abs(terms).sum()


def test_composite_coaxial_second_order():
    errs = []
    for n in (128, 256):
        d = W.coaxial_2d(n)
        h = 2.0 / n
        lo = [int(round(1.69 / h)), int(round(0.875 / h))]
        hi = [int(round(1.815 / h)), int(round(1.125 / h))]
        C = Composite(d, lo, hi)
        x, (pc, pf) = C.solve()
        e_all, e_box = 0.0, 0.0
        for g, P in ((C.gc, pc), (C.gf, pf)):
            X, Y, _ = g.cell_centres()
            ex = W.coaxial_exact(np.sqrt(X * X + Y * Y))
            for p in range(2):
                m = g.dof[p] >= 0
                if g is C.gc:
                    m &= ~C.under
                if m.any():
                    e = np.abs(P[p][m] - ex[p][m]).max()
                    e_all = max(e_all, e)
                    if g is C.gf:
                        e_box = max(e_box, e)
        errs.append((e_all, e_box))
    assert math.log2(errs[0][0] / errs[1][0]) > 1.8, errs
    assert math.log2(errs[0][1] / errs[1][1]) > 1.8, errs
    assert errs[1][0] < 2e-4


def test_box_over_the_whole_domain_is_the_fine_problem():
    d = W.rod_plane_2d(16)
    C = Composite(d, [0, 0], [16, 16])
    assert C.nco == 0 and len(C.faces) == 0
    x, (pc, pf) = C.solve()
    _, phi_f, *_ = oracle.solve(W.rod_plane_2d(32))
    assert np.abs(pf - phi_f).max() <= 1e-12


def test_dielectric_at_cf_side_rejected():
    d = W.coaxial_2d(64)
    with pytest.raises(oracle.OracleError):
        Composite(d, [40, 28], [48, 36])  # crosses the dielectric shell


def test_planted_linear_tangential_interpolation_breaks_exactness(monkeypatch):
    """Plant a mistake in the oracle: linear instead of quadratic tangential
    weights.  The quadratic-exactness pin must then fail, so it does test the
    coarse-fine interpolation."""
    import oracle.composite as OC
    monkeypatch.setattr(OC, "_tangential_weights", lambda off: (-off if off < 0 else 0.0, 1.0 - abs(off),
                                                                off if off > 0 else 0.0))
    n = 32
    d = W._desc(2, (n, n), (0, 0), 1.0 / n, [(W.PRIM_SPHERE, [0.2, 0.2, 0.0, 0.1])], [(0, 0, 0)], 0, -1,
                (1.0, 1.0), [1] * 4 + [0, 0], 0.0, [0] * 6)
    C = OC.Composite(d, [16, 16], [24, 24])
    c = np.array([0.3, -0.7, 0.4, 1.1, -0.6, 0.9])

    def phi(x, y, z):
        return c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * y * y + c[5] * x * y
    rel, *_ = _quadratic_truncation(C, phi, 2 * (c[3] + c[4]))
    assert rel > 1e-8


def _conservation_gap_3d(C):
    gc, gf = C.gc, C.gf
    A, b = C.assemble(sc=np.zeros((2, gc.ncell)), sf=np.zeros((2, gf.ncell)))
    x = np.random.default_rng(2).normal(size=C.n)
    vol = np.concatenate([np.full(C.nco, gc.h ** 3), np.full(gf.ndof, gf.h ** 3)])
    terms = vol * (b - A @ x)
    return abs(terms.sum() - C.boundary_flux(x)) / np.abs(terms).sum()


def test_composite_conservation_3d_pin_crossing_cf_side():
    """3D: a pin of radius 0.1 through the top side of the box [4, 12)^3 of a
    16^3 grid cuts CF faces; for arbitrary phi the volume-weighted residuals
    still sum to the wall and EB fluxes alone."""
    d = W.pin_plane_3d(16, radius=0.1, disk=False)
    C = Composite(d, [4, 4, 4], [12, 12, 12])
    assert any(C.gf.cut[f[2]] for f in C.faces)
    assert _conservation_gap_3d(C) <= 1e-12


def test_planted_missing_coarse_flux_removal_breaks_conservation(monkeypatch):
    """Plant a mistake in the oracle: keep the coarse operator's own flux
    through the CF sides next to the box.  The conservation pin must then fail."""
    import oracle.composite as OC
    monkeypatch.setattr(OC.Composite, "coarse_cf_faces", lambda self: [])
    d = W.pin_plane_3d(16, radius=0.1, disk=False)
    C = OC.Composite(d, [4, 4, 4], [12, 12, 12])
    assert _conservation_gap_3d(C) > 1e-6


def test_planted_linear_normal_interpolation_breaks_exactness(monkeypatch):
    """Plant a mistake in the oracle: the linear normal step (fine cell at -1/2
    and coarse value only) everywhere.  The 2D quadratic-exactness pin must fail."""
    import oracle.composite as OC
    monkeypatch.setattr(OC, "_normal_weights", lambda quadratic: (1.0 / 3.0, 0.0, 2.0 / 3.0))
    n = 32
    d = W._desc(2, (n, n), (0, 0), 1.0 / n, [(W.PRIM_SPHERE, [0.2, 0.2, 0.0, 0.1])], [(0, 0, 0)], 0, -1,
                (1.0, 1.0), [1] * 4 + [0, 0], 0.0, [0] * 6)
    C = OC.Composite(d, [16, 16], [24, 24])
    c = np.array([0.3, -0.7, 0.4, 1.1, -0.6, 0.9])

    def phi(x, y, z):
        return c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * y * y + c[5] * x * y
    rel, *_ = _quadratic_truncation(C, phi, 2 * (c[3] + c[4]))
    assert rel > 1e-8

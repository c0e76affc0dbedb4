"""Pins of the oracle's multi-level composite operator (nested refined boxes).

- one box reduces exactly to the two-level operator (same A and b);
- quadratic exactness over three levels in 2D and (without cross terms) in 3D:
  the CF interpolation of every level pair is exact for quadratics and the
  refluxed flux is the exact face mean, so the truncation error vanishes on
  every row of the composite system and its solution is the quadratic;
- exact conservation over three levels with the rod crossing the CF sides of
  both boxes (2D) and a pin crossing both boxes' top sides (3D);
- proper nesting is enforced;
- values under the boxes are the composed kappa-weighted means (exact for a
  linear phi on regular cells);
- planted mistakes: the inner pair keeping the coarse operator's own CF flux
  breaks conservation; the inner pair scaled by the outer pair's spacing
  breaks exactness; means not composed through the inner box break the
  composition pin.
"""
import numpy as np
import pytest

import oracle
from oracle.composite import Composite
from oracle.multilevel import MultiLevel
from paper_1809_03745_gb300 import workloads as W


def _walls(g, f):
    return np.concatenate([f(x, y, z) for _, x, y, z in g.wall_face_centres()])


def _truncation(M, phi, lap):
    s, phiE, phidom, xs = [], [], [], []
    for g in M.g:
        s.append(np.full((2, g.ncell), -lap))
        phiE.append(phi(g.ebx[:, 0], g.ebx[:, 1], g.ebx[:, 2]))
        pd = _walls(g, phi)
        phidom.append(np.stack([pd, pd]))
        X, Y, Z = g.cell_centres()
        xs.append(np.stack([phi(X, Y, Z)] * 2))
    A, b = M.assemble(s=s, phiE=phiE, phidom=phidom)
    x = M.join(xs)
    return np.abs(A @ x - b).max() / np.abs(b).max(), A, b, x


def _sphere_2d(n=32):
    return W._desc(2, (n, n), (0, 0), 1.0 / n, [(W.PRIM_SPHERE, [0.2, 0.2, 0.0, 0.1])], [(0, 0, 0)], 0, -1,
                   (1.0, 1.0), [1] * 4 + [0, 0], 0.0, [0] * 6)


C2 = np.array([0.3, -0.7, 0.4, 1.1, -0.6, 0.9])


def _quad2(x, y, z):
    c = C2
    return c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * y * y + c[5] * x * y


def test_one_box_is_the_two_level_operator():
    d = W.rod_plane_2d(32)
    M = MultiLevel(d, [([12, 12], [20, 20])])
    A, b = M.assemble()
    C = Composite(d, [12, 12], [20, 20])
    A2, b2 = C.assemble()
    assert M.n == C.n
    assert abs(A - A2).max() == 0.0 and np.abs(b - b2).max() == 0.0


def test_three_levels_quadratic_exactness_2d():
    M = MultiLevel(_sphere_2d(), [([12, 12], [28, 28]), ([4, 8], [24, 20])])
    assert M.L == 3 and all(len(P.faces) > 0 for P in M.pairs)
    rel, A, b, x = _truncation(M, _quad2, 2 * (C2[3] + C2[4]))
    assert rel <= 1e-12
    assert np.abs(oracle.solve_system(A, b) - x).max() <= 1e-11


def test_three_levels_quadratic_exactness_3d_no_cross_terms():
    n = 16
    d = W._desc(3, (n, n, n), (0, 0, 0), 1.0 / n, [], [], -1, -1, (1.0, 1.0), [1] * 6, 0.0, [0] * 6)
    M = MultiLevel(d, [([4, 4, 4], [12, 12, 12]), ([4, 4, 8], [12, 12, 12])])
    c = np.array([0.2, 0.5, -0.3, 0.8, 1.3, -0.4, 0.7])

    def phi(x, y, z):
        return c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * y + c[6] * z * z
    rel, *_ = _truncation(M, phi, 2 * (c[4] + c[5] + c[6]))
    assert rel <= 1e-12


def _conservation_gap(M, seed=1):
    A, b = M.assemble()
    x = np.random.default_rng(seed).normal(size=M.n)
    terms = M.volumes() * (b - A @ x)
    return abs(terms.sum() - M.boundary_flux(x)) / np.abs(terms).sum()


def test_three_levels_conservation_2d_rod_crossing_both_boxes():
    d = W.rod_plane_2d(32)
    M = MultiLevel(d, [([8, 8], [24, 24]), ([8, 8], [24, 24])])
    for P in M.pairs:
        assert any(P.gf.cut[f[2]] for f in P.faces)  # the rod crosses a CF side of each box
    assert _conservation_gap(M) <= 1e-12


def test_three_levels_conservation_3d_pin_crossing_both_boxes():
    d = W.pin_plane_3d(16, radius=0.1, disk=False)
    M = MultiLevel(d, [([4, 4, 4], [12, 12, 12]), ([4, 4, 4], [12, 12, 12])])
    for P in M.pairs:
        assert any(P.gf.cut[f[2]] for f in P.faces)
    assert _conservation_gap(M, 2) <= 1e-12


def test_nesting_is_enforced():
    d = W.rod_plane_2d(32)
    with pytest.raises(oracle.OracleError):
        MultiLevel(d, [([8, 8], [24, 24]), ([0, 8], [16, 24])])  # touches the parent's low-x CF side
    # a side on the domain boundary may be shared
    M = MultiLevel(_sphere_2d(), [([12, 16], [28, 32]), ([4, 8], [24, 32])])
    assert M.L == 3


def test_planted_inner_pair_keeps_coarse_flux_breaks_conservation(monkeypatch):
    """Plant a mistake in the oracle: the inner level pair keeps the coarse
    operator's own flux through its CF sides.  The conservation pin must fail."""
    orig = Composite.coarse_cf_faces
    h0 = 1.0 / 32

    def planted(self):
        return [] if self.gc.h < h0 else orig(self)
    monkeypatch.setattr(Composite, "coarse_cf_faces", planted)
    d = W.rod_plane_2d(32)
    M = MultiLevel(d, [([8, 8], [24, 24]), ([8, 8], [24, 24])])
    assert _conservation_gap(M) > 1e-6


def test_planted_inner_pair_spacing_breaks_exactness(monkeypatch):
    """Plant a mistake in the oracle: the inner pair's fine level takes the
    spacing of the outer pair's fine level in its CF flux.  The exactness pin
    must fail."""
    M = MultiLevel(_sphere_2d(), [([12, 12], [28, 28]), ([4, 8], [24, 20])])
    M.h[2] = M.h[1]
    rel, *_ = _truncation(M, _quad2, 2 * (C2[3] + C2[4]))
    assert rel > 1e-6


def test_four_levels_quadratic_exactness_and_conservation_2d():
    M = MultiLevel(_sphere_2d(), [([12, 12], [28, 28]), ([4, 8], [28, 24]), ([8, 8], [40, 24])])
    assert M.L == 4 and all(len(P.faces) > 0 for P in M.pairs)
    rel, A, b, x = _truncation(M, _quad2, 2 * (C2[3] + C2[4]))
    assert rel <= 1e-12
    d = W.rod_plane_2d(32)
    assert _conservation_gap(MultiLevel(d, [([8, 8], [24, 24])] * 3)) <= 1e-12


def test_values_under_boxes_are_composed_means():
    """A linear phi given on every level's own cells: split() reports, under
    each box, the kappa-weighted mean of the children, composed level by
    level, which for a linear phi on regular cells is phi at the cell centre
    exactly.  Level 0 cells under box 2 get their values only through level
    1's means, so a map that skipped the composition would report 0 there."""
    M = MultiLevel(_sphere_2d(), [([12, 12], [28, 28]), ([4, 8], [28, 24])])

    def lin(x, y, z):
        return 0.3 + 1.7 * x - 0.9 * y
    phis = []
    for g in M.g:
        X, Y, Z = g.cell_centres()
        phis.append(np.stack([lin(X, Y, Z)] * 2))
    out = M.split(M.join(phis))
    g0 = M.g[0]
    X, Y, Z = g0.cell_centres()
    m = (g0.dof[0] >= 0) & M.under(0) & (g0.kappa[0] == 1.0)
    # level-0 cells whose children are under box 2: box 2 covers level-1 cells [4, 28) x [8, 24),
    # i.e. level-0 cells [14, 26) x [16, 24)
    deep = m & (X > (12 + 2) / 32) & (X < (12 + 14) / 32) & (Y > (12 + 4) / 32) & (Y < (12 + 12) / 32)
    assert deep.sum() > 0
    assert np.abs(out[0][0][m] - lin(X, Y, Z)[m]).max() <= 1e-13


def test_planted_uncomposed_means_fail_the_composition_pin():
    """Plant a mistake in the oracle: level 0's values under box 1 taken from
    level 1's own unknowns alone (no composition through box 2).  The
    composition pin must then fail."""
    import scipy.sparse as sp
    M = MultiLevel(_sphere_2d(), [([12, 12], [28, 28]), ([4, 8], [28, 24])])
    g1, own1 = M.g[1], M.own[1]
    E1 = sp.csr_matrix((np.ones(len(own1)), (own1, M.off[1] + np.arange(len(own1)))), shape=(g1.ndof, M.n))
    own0 = M.own[0]
    E0 = sp.csr_matrix((np.ones(len(own0)), (own0, M.off[0] + np.arange(len(own0)))), shape=(M.g[0].ndof, M.n))
    M.T[0] = (E0 + M.M[0] @ E1).tocsr()

    def lin(x, y, z):
        return 0.3 + 1.7 * x - 0.9 * y
    phis = []
    for g in M.g:
        X, Y, Z = g.cell_centres()
        phis.append(np.stack([lin(X, Y, Z)] * 2))
    out = M.split(M.join(phis))
    g0 = M.g[0]
    X, Y, Z = g0.cell_centres()
    m = (g0.dof[0] >= 0) & M.under(0) & (g0.kappa[0] == 1.0)
    assert np.abs(out[0][0][m] - lin(X, Y, Z)[m]).max() > 1e-3

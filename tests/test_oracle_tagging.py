"""Pins of the oracle's refinement tags (Sec. 6 tracer criteria) and regrid box.

- closed forms on synthetic fields: |E| = y^2 gives |grad T| dx / T = 2h/y
  exactly at interior cells (centred differences are exact for quadratics)
  and (2 y h + h^2)/y^2 at the bottom row (one-sided), and the refine and
  coarsen sets follow from the thresholds by hand;
- a 3D point-charge field |E| = 1/r^2, whose continuous ratio is 2h/r: cells
  well inside r = 2h/eps1 are tagged along every axis and cells well outside
  are not (a gradient that drops an axis fails along it);
- covered cells carry no tag; scaling E by 2 changes nothing;
- hand-worked regrid boxes: growth by the buffer, rounding to the blocking
  factor, clipping at coarse-fine sides, the keep rule;
- planted mistakes (the tracer not normalised, the centred difference not
  halved, the z term dropped) each fail a pin.
"""
import numpy as np

import oracle
from oracle import tagging as TG
from paper_1809_03745_gb300 import workloads as W


def _box(D, n):
    return oracle.Geometry(W._desc(D, (n,) * D, (0,) * D, 1.0 / n, [], [], -1, -1, (1.0, 1.0), [1] * 6, 0.0,
                                   [0] * 6))


def _field_y2(g):
    X, Y, Z = g.cell_centres()
    E = np.zeros((2, 2, g.ncell))
    E[1][0] = Y * Y  # |E| = y^2 in the gas phase
    return E, Y


def test_quadratic_profile_ratio_closed_form():
    n = 64
    g = _box(2, n)
    h = 1.0 / n
    E, Y = _field_y2(g)
    T, ratio = TG.gradient_ratio(g, E)
    ymax = 1.0 - h / 2
    assert np.abs(T - Y * Y / ymax ** 2).max() <= 1e-15
    j = np.rint(Y / h - 0.5).astype(int)
    want = np.where(j == 0, (2 * Y * h + h * h) / (Y * Y),
                    np.where(j == n - 1, (2 * Y * h - h * h) / (Y * Y), 2 * h / Y))
    assert np.abs(ratio - want).max() <= 1e-12 * want.max()


def test_quadratic_profile_tags_by_hand():
    n = 128
    g = _box(2, n)
    h = 1.0 / n
    E, Y = _field_y2(g)
    t = TG.tags(g, E)
    j = np.rint(Y / h - 0.5).astype(int)
    ymax = 1.0 - h / 2
    # interior: ratio 2h/y > 0.1 iff y < 20h; T > 0.8 iff y > sqrt(0.8) ymax; coarsen iff
    # 2h/y < 0.1 and y^2 < 0.2 ymax^2
    y = Y[(j > 0) & (j < n - 1)]
    tt = t[(j > 0) & (j < n - 1)]
    refine = (y < 20 * h) | (y > np.sqrt(0.8) * ymax)
    coarsen = (y > 20 * h) & (y < np.sqrt(0.2) * ymax)
    assert np.array_equal((tt & TG.REFINE) != 0, refine)
    assert np.array_equal((tt & TG.COARSEN) != 0, coarsen)
    assert refine.sum() > 0 and coarsen.sum() > 0


def _point_charge(g, c):
    X, Y, Z = g.cell_centres()
    R = np.stack([X - c[0], Y - c[1], Z - c[2]])
    r = np.sqrt((R * R).sum(axis=0))
    E = np.zeros((3, 2, g.ncell))
    for a in range(3):
        E[a][0] = R[a] / r ** 3
    return E, r, R


def test_point_charge_tags_every_axis():
    n = 32
    g = _box(3, n)
    h = 1.0 / n
    c = (0.5 + 0.3 * h, 0.5 - 0.2 * h, 0.5 + 0.1 * h)
    E, r, R = _point_charge(g, c)
    t = TG.tags(g, E, eps=(0.2, 0.8, 0.1, 0.2))  # continuous ratio 2h/r: refine inside r = 10h
    near = (r > 2 * h) & (r < 7 * h)
    far = r > 13 * h
    assert ((t[near] & TG.REFINE) != 0).all()
    assert ((t[far] & TG.REFINE) == 0).all()
    # the cells on the z axis through the charge are among the tagged ones
    onz = near & (np.abs(R[0]) < h) & (np.abs(R[1]) < h)
    assert onz.sum() >= 6


def test_covered_cells_carry_no_tags_and_scale_invariance():
    d = W.rod_plane_2d(64)
    g, phi, A, b, data = oracle.solve(d)
    E, _ = g.field(data, g.to_dofs(phi))
    t = TG.tags(g, E)
    covered = (g.dof[0] < 0) & (g.dof[1] < 0)
    assert covered.any() and (t[covered] == 0).all()
    assert (t & TG.REFINE).any()
    assert np.array_equal(TG.tags(g, 2.0 * E), t)


def test_regrid_box_by_hand():
    n = (32, 32)
    tag = np.zeros(32 * 32, np.uint8)
    live = np.ones(32 * 32, bool)
    tag[13 * 32 + 10] = TG.REFINE  # cell (10, 13)
    # bbox [10, 11) x [13, 14) -> grown by 2: [8, 13) x [11, 16) -> rounded to 4: [8, 16) x [8, 16)
    assert TG.regrid_box(tag, live, n, 2, [False, False], [False, False]) == ([8, 8], [16, 16])
    # a cell by the low-x edge: [0, 4) x [8, 16) on a domain side; clipped to [4, ...) on a CF side
    tag[:] = 0
    tag[13 * 32 + 1] = TG.REFINE
    assert TG.regrid_box(tag, live, n, 2, [False, False], [False, False]) == ([0, 8], [4, 16])
    assert TG.regrid_box(tag, live, n, 2, [True, False], [False, False]) == ([4, 8], [8, 16])
    # keep rule: cells under the current finer box stay refined unless tagged for coarsening
    tag[:] = 0
    keep = ([20, 20], [24, 28])
    assert TG.regrid_box(tag, live, n, 2, [False] * 2, [False] * 2, keep=keep) == ([16, 16], [28, 32])
    idx = np.arange(32 * 32)
    inside = (idx % 32 >= 20) & (idx % 32 < 24) & (idx // 32 >= 20) & (idx // 32 < 28)
    tag[inside] = TG.COARSEN
    assert TG.regrid_box(tag, live, n, 2, [False] * 2, [False] * 2, keep=keep) is None
    tag[inside & (idx // 32 >= 26)] = 0  # rows 26, 27 no longer released
    assert TG.regrid_box(tag, live, n, 2, [False] * 2, [False] * 2, keep=keep) == ([16, 24], [28, 32])


def test_planted_unnormalised_tracer_fails(monkeypatch):
    """Plant a mistake in the oracle: T = |E| without the division by max|E|."""
    monkeypatch.setattr(TG, "tracer", TG.field_magnitude)
    n = 64
    g = _box(2, n)
    E, Y = _field_y2(g)
    T, _ = TG.gradient_ratio(g, 0.5 * E)
    ymax = 1.0 - 0.5 / n
    assert np.abs(T - Y * Y / ymax ** 2).max() > 1e-3


def test_planted_unhalved_difference_fails(monkeypatch):
    """Plant a mistake in the oracle: the centred difference T+ - T- not halved."""
    orig = TG._axis_difference

    def planted(Tg, Lg, ax):
        return orig(Tg, Lg, ax) * np.where(orig(Tg, Lg, ax) == 0, 1.0, 2.0)
    monkeypatch.setattr(TG, "_axis_difference", planted)
    n = 64
    g = _box(2, n)
    h = 1.0 / n
    E, Y = _field_y2(g)
    _, ratio = TG.gradient_ratio(g, E)
    assert np.abs(ratio - 2 * h / Y).max() > 1e-3


def test_planted_dropped_z_term_fails(monkeypatch):
    """Plant a mistake in the oracle: the z difference left out of |grad T|."""
    orig = TG._axis_difference
    monkeypatch.setattr(TG, "_axis_difference", lambda Tg, Lg, ax: orig(Tg, Lg, ax) * (ax != 0))
    n = 32
    g = _box(3, n)
    h = 1.0 / n
    c = (0.5 + 0.3 * h, 0.5 - 0.2 * h, 0.5 + 0.1 * h)
    E, r, R = _point_charge(g, c)
    t = TG.tags(g, E, eps=(0.2, 0.8, 0.1, 0.2))
    near = (r > 2 * h) & (r < 7 * h)
    assert not ((t[near] & TG.REFINE) != 0).all()

"""Refinement tags of the oracle (Sec. 6: the tracer field and its criteria)
and the box that a regrid step derives from them.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): only tests/ and the
baseline legs of bench.py may use it.

Sec. 6 regrids on the tracer T = |E| / max |E|.  A cell is tagged for
refinement when |grad T| dx / T exceeds eps1 or T exceeds eps2, and for
coarsening when |grad T| dx / T is below eps3 and T below eps4 (the paper's
values: 0.1, 0.8, 0.1, 0.2).  The paper leaves the discrete details open;
this module reads them as follows.

  * |E| of a cell is the largest field magnitude over the phases that have an
    unknown there; the maximum runs over the cells of the grid being tagged
    (one level).  Covered cells carry no T and no tag.
  * grad T by differences over cell neighbours along each axis: centred
    where both neighbours carry T, one-sided where one does, zero where none
    does.  dx cancels: |grad T| dx = sqrt(sum_a d_a^2) with d_a the difference
    in index units ((T+ - T-)/2, T+ - T or T - T-).
  * The ratio |grad T| dx / T is taken as 0 where T and the gradient are both
    zero, and as infinite where only T is zero.
  * Bits of a tag: 1 refine, 2 coarsen.

Regrid box (one box per level, reading of the patch-based regrid of Sec. 3):
the cells to refine are the refine-tagged ones plus, when a finer box exists,
the cells under it that are not tagged for coarsening (a refined cell is kept
until the coarsening test releases it).  Their bounding box is grown by
`buf` cells per side, its corners are rounded outward to multiples of
`block`, and it is clipped to the grid, `block` cells short of every side that
is a coarse-fine side of the grid (proper nesting); a box that clipping left
thinner than `block` cells is widened to `block` cells away from the side it
was clipped at.  No box results when no cell is to be refined or the grid
has no room for a box.
"""
from __future__ import annotations

import numpy as np

REFINE, COARSEN = 1, 2
PAPER_EPS = (0.1, 0.8, 0.1, 0.2)


def field_magnitude(g, E):
    """|E| per cell: the largest magnitude over the phases with an unknown (0 where covered)."""
    D = g.dim
    E = np.asarray(E).reshape(D, 2, g.ncell)
    mag = np.zeros(g.ncell)
    for p in range(2):
        m2 = E[0][p] * E[0][p]
        for a in range(1, D):
            m2 = m2 + E[a][p] * E[a][p]
        m = np.sqrt(m2)
        has = g.dof[p] >= 0
        mag = np.where(has & (m > mag), m, mag)
    return mag


def tracer(g, E):
    """T = |E| / max |E| on the cells of the grid (0 where covered or when E = 0 everywhere)."""
    mag = field_magnitude(g, E)
    mx = mag.max() if mag.size else 0.0
    return mag / mx if mx > 0.0 else np.zeros_like(mag)


def _axis_difference(Tg, Lg, ax):
    """d_a of every cell along array axis ax: centred, one-sided or zero."""
    Tp = np.zeros_like(Tg)
    Tm = np.zeros_like(Tg)
    lp = np.zeros_like(Lg)
    lm = np.zeros_like(Lg)
    sl_hi = [slice(None)] * 3
    sl_lo = [slice(None)] * 3
    sl_hi[ax] = slice(1, None)
    sl_lo[ax] = slice(None, -1)
    Tp[tuple(sl_lo)] = Tg[tuple(sl_hi)]
    lp[tuple(sl_lo)] = Lg[tuple(sl_hi)]
    Tm[tuple(sl_hi)] = Tg[tuple(sl_lo)]
    lm[tuple(sl_hi)] = Lg[tuple(sl_lo)]
    return np.where(lp & lm, (Tp - Tm) * 0.5, np.where(lp, Tp - Tg, np.where(lm, Tg - Tm, 0.0)))


def gradient_ratio(g, E):
    """(T, |grad T| dx / T) per cell."""
    D = g.dim
    n = g.n
    T = tracer(g, E)
    live = (g.dof[0] >= 0) | (g.dof[1] >= 0)
    Tg = T.reshape(n[2], n[1], n[0])
    Lg = live.reshape(n[2], n[1], n[0])
    s2 = np.zeros_like(Tg)
    for a in range(D):
        d = _axis_difference(Tg, Lg, 2 - a)  # array axis of grid axis a (x fastest)
        s2 = s2 + d * d
    gdx = np.sqrt(s2).reshape(-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(T > 0.0, gdx / np.where(T > 0.0, T, 1.0), np.where(gdx > 0.0, np.inf, 0.0))
    return T, ratio


def tags(g, E, eps=PAPER_EPS):
    """Tag bits per cell (REFINE, COARSEN) by the criteria of Sec. 6."""
    eps1, eps2, eps3, eps4 = eps
    T, ratio = gradient_ratio(g, E)
    live = (g.dof[0] >= 0) | (g.dof[1] >= 0)
    refine = (ratio > eps1) | (T > eps2)
    coarsen = (ratio < eps3) & (T < eps4)
    out = np.where(refine, REFINE, 0) | np.where(coarsen, COARSEN, 0)
    return np.where(live, out, 0).astype(np.uint8)


def regrid_box(tag, live, n, D, cf_lo, cf_hi, keep=None, buf=2, block=4):
    """The next finer box over a grid of n cells from its tags (reading above).

    live: cells that carry T (an unknown of some phase).  cf_lo / cf_hi: per
    axis, whether the grid's low / high side is a coarse-fine side.  keep:
    (lo, hi) of the current finer box, or None.  Returns (lo, hi) lists of D
    entries, or None."""
    n = [int(v) for v in n][:D]
    tg = np.asarray(tag).reshape([int(v) for v in n[::-1]] if D == 3 else [n[1], n[0]])
    lv = np.asarray(live, bool).reshape(tg.shape)
    want = (tg & REFINE) != 0
    if keep is not None:
        klo, khi = keep
        idx = np.indices(tg.shape)
        inside = np.ones(tg.shape, bool)
        for a in range(D):
            ia = idx[D - 1 - a]
            inside &= (ia >= klo[a]) & (ia < khi[a])
        want |= inside & lv & ((tg & COARSEN) == 0)
    if not want.any():
        return None
    lo, hi = [], []
    for a in range(D):
        ax = D - 1 - a
        other = tuple(k for k in range(D) if k != ax)
        hit = np.nonzero(want.any(axis=other))[0]
        l, h = int(hit[0]) - buf, int(hit[-1]) + 1 + buf
        l = (l // block) * block
        h = -((-h) // block) * block
        lmin = block if cf_lo[a] else 0
        hmax = n[a] - block if cf_hi[a] else n[a]
        l, h = max(l, lmin), min(h, hmax)
        if h - l < block:  # widened away from the clipped side to one block
            if l == lmin:
                h = l + block
            else:
                l = h - block
            if l < lmin or h > hmax:
                return None
        lo.append(l)
        hi.append(h)
    return lo, hi

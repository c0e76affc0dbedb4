"""Regrid driver: refine nested boxes where the tracer criteria of Sec. 6 ask.

Level by level: solve on the current hierarchy (level 0 alone at first),
evaluate E = -grad phi on the finest level, tag its cells (eb_tag_cells: the
tracer T = |E| / max |E|, refine where |grad T| dx / T > eps1 or T > eps2),
turn the marked cells' bounding box into the next box (eb_regrid_box: buffer,
blocking factor, proper nesting) and rebuild the composite grid with it.  The
composite grid lets only the gas phase touch a coarse-fine side; when a box
would cut through a dielectric, its coarse-fine sides move outward by the
blocking factor until the set-up accepts it (or the box reaches the grid).
Every step runs in the library; this module only sequences the calls.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ebpoisson as E
from . import workloads as W

PAPER_EPS = (0.1, 0.8, 0.1, 0.2)


def level_sources(desc_l, source):
    """[2][n] right-hand side of one level: source(x, y, z) in the gas phase."""
    x, y, z = W.cell_centres(desc_l)
    S = np.zeros((2, x.size))
    S[0] = source(x, y, z)
    return S


def cf_sides(boxes, parent_n, D):
    """Which sides of the finest level are coarse-fine sides (inside their parent grid)."""
    if not boxes:
        return [0, 0, 0], [0, 0, 0]
    lo, hi = boxes[-1]
    return ([int(lo[a] > 0) if a < D else 0 for a in range(3)],
            [int(hi[a] < parent_n[a]) if a < D else 0 for a in range(3)])


def same_boxes(a, b):
    """Do two box lists place the same levels (box l of a equals box l of b for every l)?"""
    key = lambda bs: [([int(v) for v in lo], [int(v) for v in hi]) for lo, hi in bs]  # noqa: E731
    return len(a) == len(b) and key(a) == key(b)


def _grow(box, n, cflo, cfhi, D, block):
    """The box with every side that is not at its limit moved out by `block` cells (None if none can)."""
    lo, hi = list(box[0]), list(box[1])
    moved = False
    for a in range(D):
        lmin = block if cflo[a] else 0
        hmax = n[a] - block if cfhi[a] else n[a]
        if lo[a] > lmin:
            lo[a] = max(lmin, lo[a] - block)
            moved = True
        if hi[a] < hmax:
            hi[a] = min(hmax, hi[a] + block)
            moved = True
    return (lo, hi) if moved else None


def _hierarchy(desc, boxes, n, cflo, cfhi, D, block, **kw):
    """Set up the composite grid, growing the newest box while a dielectric cuts its CF sides."""
    while True:
        try:
            return E.Hierarchy(desc, boxes, **kw), boxes
        except E.EBError as exc:
            if exc.status != E.EB_ERR_UNSUPPORTED:
                raise
            grown = _grow(boxes[-1], n, cflo, cfhi, D, block)
            if grown is None:
                raise
            boxes = boxes[:-1] + [grown]


def build_hierarchy(desc, source, *, max_levels=3, eps=PAPER_EPS, buf=2, block=4, keep=None, precision="mixed",
                    tol=1e-10, device=None):
    """Refine from level 0 up to max_levels levels.

    keep: boxes of an earlier hierarchy of the same problem; where the grid a
    box is tagged on is unchanged, the earlier finer box's cells stay marked
    unless tagged for coarsening.  Returns dict(hierarchy (or None when
    nothing was refined), boxes, phis, info, steps)."""
    D = int(desc["dim"])
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    g = E.Geometry(desc, device=dev)
    P = E.Poisson(g, precision=precision, tol=tol)
    S0 = level_sources(desc, source)
    phi, info = P.solve(torch.from_numpy(S0))
    Ef = P.field(phi)[0]
    boxes, steps, H = [], [], None
    phis = [phi]
    grid_n = list(desc["n"])[:D]
    keep_box = keep[0] if keep else None
    while True:
        _, blo, bhi, nm, emax = E.tag_cells(g if H is None else H.level_geom(len(boxes)), Ef, eps, keep=keep_box,
                                            want_tags=False)
        parent_n = list(H.levels[len(boxes) - 1]["n"]) if H is not None else grid_n
        cflo, cfhi = cf_sides(boxes, parent_n, D)
        n_here = grid_n if H is None else list(H.levels[len(boxes)]["n"])[:D]
        box = E.regrid_box(D, n_here, cflo, cfhi, blo, bhi, nm, buf, block)
        steps.append(dict(level=len(boxes), n_marked=nm, bbox=(blo[:D], bhi[:D]), e_max=emax, box=box))
        if box is None or len(boxes) + 1 >= max_levels:
            break
        if H is not None:
            H.close()
        H, boxes = _hierarchy(desc, boxes + [box], n_here, cflo, cfhi, D, block, precision=precision, tol=tol,
                              device=dev)
        steps[-1]["box"] = boxes[-1]
        S = [level_sources(H.level_desc(l), source) for l in range(H.L)]
        phis, info = H.solve([torch.from_numpy(s) for s in S])
        Ef = H.field(H.L - 1, phis[-1])[0]
        # the earlier finer box is kept only while the grid it sits on is unchanged
        k = len(boxes)
        keep_box = keep[k] if keep and len(keep) > k and same_boxes(keep[:k], boxes) else None
    return dict(hierarchy=H, boxes=boxes, phis=phis, info=info, steps=steps)

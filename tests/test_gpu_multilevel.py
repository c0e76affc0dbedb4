"""Nested refined levels and regrid tags on the GPU against the oracle.

- the composite residual over three levels equals the oracle's multi-level
  operator (2D rod crossing both boxes' CF sides; 3D pin through both boxes),
  and over four levels (2D, the rod crossing all three boxes);
- those solves equal the oracle's direct solution (FP64 and mixed);
- two levels through the nested-level calls equal the two-level calls bitwise;
- the tags of eb_tag_cells equal the oracle's bit for bit on the same E
  (2D and 3D, with and without a kept box), and so do the marked count, the
  bounding box and max |E|;
- the regrid driver's boxes equal the oracle's regrid chain on the 2D
  rod-plane, and its three-level solution matches the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import tagging as TG
from oracle.multilevel import MultiLevel
from paper_1809_03745_gb300 import workloads as W

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1809_03745_gb300 import ebpoisson as E
    from paper_1809_03745_gb300 import regrid as R


def _src2(x, y, z):
    return 100 * np.exp(-((x - 0.5) ** 2 + (y - 0.45) ** 2) / (2 * 0.03 ** 2))


def _src3(x, y, z):
    return W.line_charge(x, y, z, 1e3)


def _case(name):
    if name == "rod2d":
        return W.rod_plane_2d(32), [([8, 8], [24, 24]), ([8, 8], [24, 24])], _src2
    if name == "rod2d_4lev":
        return W.rod_plane_2d(32), [([8, 8], [24, 24])] * 3, _src2
    return W.pin_plane_3d(16, radius=0.1, disk=False), [([4, 4, 4], [12, 12, 12]), ([4, 4, 4], [12, 12, 12])], _src3


def _sources(grids, src):
    out = []
    for g in grids:
        X, Y, Z = g.cell_centres()
        s = np.zeros((2, g.ncell))
        s[0] = src(X, Y, Z)
        out.append(s)
    return out


CASES = ["rod2d", "pin3d", "rod2d_4lev"]


@pytest.fixture(scope="module")
def oracles():
    out = {}
    for name in CASES:
        d, boxes, src = _case(name)
        M = MultiLevel(d, boxes)
        S = _sources(M.g, src)
        A, b = M.assemble(s=S)
        out[name] = (M, S, A, b, oracle.solve_system(A, b))
    return out


@pytest.mark.parametrize("name", CASES)
def test_nested_level_residual_parity(name, oracles):
    d, boxes, _ = _case(name)
    M, S, A, b, _ = oracles[name]
    H = E.Hierarchy(d, boxes, precision="fp64")
    assert H.L == len(boxes) + 1 and [H.levels[l]["n_cells"] for l in range(H.L)] == [g.ncell for g in M.g]
    x = np.random.default_rng(5).normal(size=M.n)
    phis = M.split(x)
    r = [t.cpu().numpy() for t in H.residual(S, None, phis)]
    ro = M.split(b - A @ x)
    scale = np.abs(b).max() + abs(A).max() * np.abs(x).max()
    for l, g in enumerate(M.g):
        for p in range(2):
            m = (g.dof[p] >= 0) & ~M.under(l)
            if m.any():
                assert np.abs(r[l][p][m] - ro[l][p][m]).max() <= 1e-12 * scale, (l, p)
            mu = M.under(l)
            assert np.abs(r[l][p][mu]).max(initial=0.0) == 0.0


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nested_level_solve_parity(name, precision, oracles):
    d, boxes, _ = _case(name)
    M, S, A, b, xo = oracles[name]
    H = E.Hierarchy(d, boxes, precision=precision, tol=1e-12, max_cycles=200)
    phis, info = H.solve(S)
    assert info["status"] == 0 and info["rel_res"] <= 1e-12, info
    ref = M.split(xo)
    scale = max(np.abs(v).max() for v in ref)
    for l, g in enumerate(M.g):
        got = phis[l].cpu().numpy()
        for p in range(2):
            m = g.dof[p] >= 0
            if m.any():
                assert np.abs(got[p][m] - ref[l][p][m]).max() <= 1e-9 * scale, (l, p)


def test_two_levels_match_the_two_level_calls_bitwise():
    d = W.rod_plane_2d(64)
    lo, hi = [24, 24], [40, 40]
    C = E.Composite(d, lo, hi, precision="mixed", tol=1e-11)
    H = E.Hierarchy(d, [(lo, hi)], precision="mixed", tol=1e-11)
    fd = W.refined_box_desc(d, lo, hi)
    Sc = R.level_sources(d, _src2)
    Sf = R.level_sources(fd, _src2)
    pc, pf, i1 = C.solve(Sc, Sf)
    phis, i2 = H.solve([Sc, Sf])
    assert i1["outer_iters"] == i2["outer_iters"] and i1["vcycles"] == i2["vcycles"]
    assert torch.equal(pc, phis[0]) and torch.equal(pf, phis[1])


def _oracle_field(desc, src):
    x, y, z = W.cell_centres(desc)
    S = np.zeros((2, x.size))
    S[0] = src(x, y, z)
    g, phi, A, b, data = oracle.solve(desc, s=S)
    Ef, _ = g.field(data, g.to_dofs(phi))
    return g, Ef


@pytest.mark.parametrize("dim", [2, 3])
def test_tags_bitwise_against_oracle(dim):
    if dim == 2:
        desc, src = W.rod_plane_2d(64, dielectric=True), _src2
        keep = ([24, 28], [40, 48])
    else:
        desc, src = W.pin_plane_3d(32), _src3
        keep = ([12, 12, 12], [20, 20, 24])
    g, Ef = _oracle_field(desc, src)
    G = E.Geometry(desc)
    Ed = torch.from_numpy(Ef).cuda()
    live = (g.dof[0] >= 0) | (g.dof[1] >= 0)
    for eps in (TG.PAPER_EPS, (0.05, 0.6, 0.02, 0.3)):
        for kp in (None, keep):
            tags, blo, bhi, nm, emax = E.tag_cells(G, Ed, eps, keep=kp)
            want_t = TG.tags(g, Ef, eps)
            assert np.array_equal(tags.cpu().numpy(), want_t)
            assert emax == TG.field_magnitude(g, Ef).max()
            want = (want_t & TG.REFINE) != 0
            if kp is not None:
                idx = np.arange(g.ncell)
                I = [idx % g.n[0], (idx // g.n[0]) % g.n[1], idx // (g.n[0] * g.n[1])]
                inside = live.copy()
                for a in range(dim):
                    inside &= (I[a] >= kp[0][a]) & (I[a] < kp[1][a])
                want |= inside & ((want_t & TG.COARSEN) == 0)
            assert nm == int(want.sum()) and nm > 0
            idx = np.nonzero(want)[0]
            I = [idx % g.n[0], (idx // g.n[0]) % g.n[1], idx // (g.n[0] * g.n[1])]
            assert blo[:dim] == [int(I[a].min()) for a in range(dim)]
            assert bhi[:dim] == [int(I[a].max()) + 1 for a in range(dim)]
            box = E.regrid_box(dim, g.n[:dim], [0] * 3, [0] * 3, blo, bhi, nm)
            assert box == TG.regrid_box(want_t, live, g.n, dim, [False] * dim, [False] * dim, keep=kp)


def _oracle_regrid(desc, source, max_levels):
    D = desc["dim"]
    g, Ef = _oracle_field(desc, source)
    boxes, grid, M = [], g, None
    while True:
        t = TG.tags(grid, Ef)
        live = (grid.dof[0] >= 0) | (grid.dof[1] >= 0)
        if boxes:
            lo, hi = boxes[-1]
            pn = M.g[len(boxes) - 1].n
            cflo, cfhi = [lo[a] > 0 for a in range(D)], [hi[a] < pn[a] for a in range(D)]
        else:
            cflo = cfhi = [False] * D
        box = TG.regrid_box(t, live, grid.n, D, cflo, cfhi)
        if box is None or len(boxes) + 1 >= max_levels:
            return boxes, M, None
        boxes.append(box)
        M = MultiLevel(desc, boxes)
        x, _ = M.solve(s=_sources(M.g, source))
        grid = M.g[-1]
        Ef, _ = grid.field(M.data[-1], M.T[-1] @ x)
        if len(boxes) + 1 >= max_levels:
            return boxes, M, x


def test_regrid_driver_matches_oracle_chain():
    desc = W.rod_plane_2d(64)
    out = R.build_hierarchy(desc, _src2, max_levels=3, precision="mixed", tol=1e-12)
    boxes, M, x = _oracle_regrid(desc, _src2, 3)
    assert len(boxes) == 2
    assert [(list(lo), list(hi)) for lo, hi in out["boxes"]] == [(list(lo), list(hi)) for lo, hi in boxes]
    assert out["info"]["status"] == 0
    ref = M.split(x)
    scale = max(np.abs(v).max() for v in ref)
    for l, g in enumerate(M.g):
        got = out["phis"][l].cpu().numpy()
        for p in range(2):
            m = g.dof[p] >= 0
            if m.any():
                assert np.abs(got[p][m] - ref[l][p][m]).max() <= 1e-9 * scale, (l, p)

"""Composite two-level operator of the oracle: one ratio-2 refined box.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): only tests/ and the
baseline legs of bench.py may use it.

The paper's solver runs on refined grids (Sec. 3.3.2; the coarse-fine
operator follows its refluxing description in Sec. 3.3).  The paper does not
spell out the coarse-fine interpolation, so this module takes the following
reading, one plain step at a time:

  * The coarse grid covers the domain; the fine grid covers the coarse cells
    [lo, hi) per axis at half the spacing and is a grid of its own, computed
    from the same implicit functions.  A box side on the domain boundary keeps
    the domain's boundary condition; every other box side is a coarse-fine
    (CF) side, a homogeneous Neumann wall of the fine grid to which the CF
    flux below is added.
  * Unknowns: the coarse unknowns of cells outside the box and all fine
    unknowns.  A coarse cell under the box carries no equation; where a coarse
    stencil reaches it, its value is the kappa-weighted mean of its children
    that carry the phase (0 if none does).
  * Ghost value behind a CF face of fine cell F (phase 0):
      - tangential step: quadratic Lagrange interpolation through the coarse
        cells C-1, C, C+1 along each tangential axis, evaluated at the ghost's
        offset +-1/4 (coarse units): weights (-3/32, 15/16, 5/32) and mirrored;
        in 3D the two tangential corrections are added to phi_C (no cross
        term).  C is the coarse cell across the face.  A direction whose
        outer cell is outside the domain, under the box, covered, cut or
        without the phase falls back to linear (3/4, 1/4) toward the offset,
        then to phi_C alone.
      - normal step: quadratic through the fine cells at -3/2 and -1/2 (fine
        units from the face) and the tangential value at +1, evaluated at +1/2:
        weights (-1/5, 2/3, 8/15); linear (1/3 at -1/2, 2/3 at +1) when the cell
        at -3/2 is cut, covered or outside the fine grid.
  * CF flux out of F: eps_0 (phi_ghost - phi_F)/h_f times the fine face
    aperture, added to F's row as alpha_f F / h_f.
  * Refluxing: the coarse row of C loses the coarse operator's own flux
    through the CF face and gains minus the mean of the fine fluxes through
    the 2^(D-1) fine faces covering it, so the composite operator conserves
    exactly.
  * Only phase 0 (gas) may touch a CF side: a fine cell next to a CF side or
    its coarse neighbour with a dielectric unknown is rejected.
"""
from __future__ import annotations

import numpy as np

from . import Geometry, OracleError, solve_system


def fine_desc(desc: dict, box_lo, box_hi) -> dict:
    """Description of the fine grid over coarse cells [box_lo, box_hi)."""
    D = int(desc["dim"])
    n = list(desc["n"]) + [1] * (3 - len(desc["n"]))
    lo = list(desc["lo"]) + [0.0] * (3 - len(desc["lo"]))
    h = float(desc["h"])
    nf, lof = [1, 1, 1], [0.0, 0.0, 0.0]
    bc = list(desc["bc"])
    wall = list(desc["phi_wall"])
    for a in range(D):
        nf[a] = 2 * (box_hi[a] - box_lo[a])
        lof[a] = lo[a] + box_lo[a] * h
        if box_lo[a] > 0:
            bc[2 * a], wall[2 * a] = 0, 0.0
        if box_hi[a] < n[a]:
            bc[2 * a + 1], wall[2 * a + 1] = 0, 0.0
    out = dict(desc)
    out.update(n=tuple(nf), lo=tuple(lof), h=h / 2.0, bc=bc, phi_wall=wall)
    return out


def _tangential_weights(off):
    """Quadratic Lagrange weights at offset off (+-1/4) for nodes -1, 0, +1."""
    return (off * (off - 1.0) / 2.0, 1.0 - off * off, off * (off + 1.0) / 2.0)


def _normal_weights(quadratic):
    """Weights (fine cell at -1/2, fine cell at -3/2, coarse value at +1) of the
    ghost at +1/2 along the CF normal, in fine-cell units: quadratic Lagrange
    through the three, or linear through the first and the last."""
    return (2.0 / 3.0, -1.0 / 5.0, 8.0 / 15.0) if quadratic else (1.0 / 3.0, 0.0, 2.0 / 3.0)


class Composite:
    def __init__(self, desc: dict, box_lo, box_hi):
        self.D = D = int(desc["dim"])
        self.desc = desc
        self.box_lo = [int(v) for v in box_lo] + [0] * (3 - len(box_lo))
        self.box_hi = [int(v) for v in box_hi] + [1] * (3 - len(box_hi))
        self.gc = Geometry(desc)
        self.fdesc = fine_desc(desc, self.box_lo, self.box_hi)
        self.gf = Geometry(self.fdesc)
        gc, gf = self.gc, self.gf
        nc = list(gc.n) + [1] * (3 - len(gc.n))
        for a in range(D):
            if not (0 <= self.box_lo[a] < self.box_hi[a] <= nc[a]):
                raise OracleError(1)
        self.nc, self.nf = nc, list(gf.n) + [1] * (3 - len(gf.n))
        # coarse cells under the box
        idx = np.arange(gc.ncell)
        I = [idx % nc[0], (idx // nc[0]) % nc[1], idx // (nc[0] * nc[1])]
        under = np.ones(gc.ncell, bool)
        for a in range(D):
            under &= (I[a] >= self.box_lo[a]) & (I[a] < self.box_hi[a])
        self.under = under
        # composite numbering: coarse dofs outside the box, then fine dofs
        self.cmap = -np.ones(gc.ndof, np.int64)
        keep = []
        for p in range(2):
            m = (gc.dof[p] >= 0) & ~under
            keep.append(gc.dof[p][m])
        keep = np.sort(np.concatenate(keep))
        self.cmap[keep] = np.arange(len(keep))
        self.nco = len(keep)
        self.n = self.nco + gf.ndof
        self._cf_faces()

    # ---------------------------------------------------------------- indexing
    def ccell(self, I):
        return int(I[0] + self.nc[0] * (I[1] + self.nc[1] * I[2]))

    def fcell(self, I):
        return int(I[0] + self.nf[0] * (I[1] + self.nf[1] * I[2]))

    def _c_available(self, I):
        """A coarse cell usable by the tangential interpolation (phase 0)."""
        for a in range(3):
            if not (0 <= I[a] < self.nc[a]):
                return False
        c = self.ccell(I)
        return (not self.under[c]) and self.gc.dof[0][c] >= 0 and not self.gc.cut[c]

    def _f_available(self, I):
        for a in range(3):
            if not (0 <= I[a] < self.nf[a]):
                return False
        c = self.fcell(I)
        return self.gf.dof[0][c] >= 0 and not self.gf.cut[c]

    # ---------------------------------------------------------------- CF faces
    def _cf_faces(self):
        """Every fine face on a CF side with its ghost stencil.  Entries:
        (a, s, fine cell F, fine face index J, coarse cell C, alpha_f,
        terms: list of (space, index, weight) of the ghost value) where space
        is 'f' (fine dof) or 'c' (coarse dof)."""
        D, gc, gf = self.D, self.gc, self.gf
        faces = []
        for a in range(D):
            t = [k for k in range(D) if k != a]
            for s in (0, 1):  # low / high side of the box
                if s == 0 and self.box_lo[a] == 0:
                    continue
                if s == 1 and self.box_hi[a] == self.nc[a]:
                    continue
                ranges = [range(self.nf[k]) if k < D else range(1) for k in range(3)]
                ranges[a] = [0] if s == 0 else [self.nf[a] - 1]
                al_f = gf.faces(a)[0]  # [phase][face]
                for i0 in ranges[0]:
                    for i1 in ranges[1]:
                        for i2 in ranges[2]:
                            FI = [i0, i1, i2]
                            fc = self.fcell(FI)
                            CI = [self.box_lo[k] + FI[k] // 2 for k in range(3)]
                            CI[a] += -1 if s == 0 else 1
                            if D == 2:
                                CI[2] = 0
                            cc = self.ccell(CI)
                            if gf.dof[1][fc] >= 0 or gc.dof[1][cc] >= 0:
                                raise OracleError(6)  # dielectric at a CF side
                            if gf.dof[0][fc] < 0 or gc.dof[0][cc] < 0:
                                continue
                            J = list(FI)
                            J[a] += s
                            al = al_f[0][self._face_index(gf, a, J)]
                            if not (al > 0.0):
                                continue
                            # tangential value at the ghost's position
                            terms_c = {cc: 1.0}
                            for k in t:
                                off = -0.25 if FI[k] % 2 == 0 else 0.25
                                lo_I, hi_I = list(CI), list(CI)
                                lo_I[k] -= 1
                                hi_I[k] += 1
                                if self._c_available(lo_I) and self._c_available(hi_I):
                                    w = _tangential_weights(off)
                                    corr = [(self.ccell(lo_I), w[0]), (cc, w[1] - 1.0), (self.ccell(hi_I), w[2])]
                                else:
                                    side = hi_I if off > 0 else lo_I
                                    if self._c_available(side):
                                        corr = [(cc, -0.25), (self.ccell(side), 0.25)]
                                    else:
                                        corr = []
                                for c2, w2 in corr:
                                    terms_c[c2] = terms_c.get(c2, 0.0) + w2
                            # normal step
                            F2 = list(FI)
                            F2[a] += 1 if s == 0 else -1
                            wf, wf2, wc = _normal_weights(self._f_available(F2))
                            terms = [("f", int(gf.dof[0][fc]), wf)]
                            if wf2 != 0.0:
                                terms.append(("f", int(gf.dof[0][self.fcell(F2)]), wf2))
                            for c2, w2 in terms_c.items():
                                if w2 != 0.0:
                                    terms.append(("c", int(gc.dof[0][c2]), wc * w2))
                            faces.append((a, s, fc, J, cc, CI, al, terms))
        self.faces = faces

    def coarse_cf_faces(self):
        """(a, s, coarse cell index triple) of every coarse cell across a CF side."""
        out = []
        for a in range(self.D):
            for s in (0, 1):
                if (s == 0 and self.box_lo[a] == 0) or (s == 1 and self.box_hi[a] == self.nc[a]):
                    continue
                ranges = [range(self.box_lo[k], self.box_hi[k]) if k < self.D else range(1) for k in range(3)]
                ranges[a] = [self.box_lo[a] - 1] if s == 0 else [self.box_hi[a]]
                for i0 in ranges[0]:
                    for i1 in ranges[1]:
                        for i2 in ranges[2]:
                            out.append((a, s, [i0, i1, i2]))
        return out

    @staticmethod
    def _face_index(g, a, J):
        n = list(g.n) + [1] * (3 - len(g.n))
        m = list(n)
        m[a] += 1
        return int(J[0] + m[0] * (J[1] + m[1] * J[2]))

    # ---------------------------------------------------------------- operator
    def averaging(self):
        """Sparse map from fine dofs to the coarse dofs under the box
        (kappa-weighted mean of the children carrying the phase)."""
        import scipy.sparse as sp
        gc, gf, D = self.gc, self.gf, self.D
        rows, cols, vals = [], [], []
        for c in np.nonzero(self.under)[0]:
            I = [c % self.nc[0], (c // self.nc[0]) % self.nc[1], c // (self.nc[0] * self.nc[1])]
            for p in range(2):
                r = gc.dof[p][c]
                if r < 0:
                    continue
                kids = []
                for k in range(1 << D):
                    FI = [2 * (I[a] - self.box_lo[a]) + ((k >> a) & 1) if a < D else 0 for a in range(3)]
                    fc = self.fcell(FI)
                    if gf.dof[p][fc] >= 0:
                        kids.append((gf.dof[p][fc], gf.kappa[p][fc]))
                tot = sum(w for _, w in kids)
                if tot > 0.0:
                    for f, w in kids:
                        rows.append(r)
                        cols.append(f)
                        vals.append(w / tot)
        return sp.csr_matrix((vals, (rows, cols)), shape=(gc.ndof, gf.ndof))

    def assemble(self, sc=None, sigc=None, sf=None, sigf=None, phiEc=None, phiEf=None, phidomc=None, phidomf=None):
        """Composite A (CSR) and b: A x = b over [coarse dofs outside the box, fine dofs]."""
        import scipy.sparse as sp
        gc, gf, D = self.gc, self.gf, self.D
        self.dc = gc.data(s=sc, sigma=sigc, phiE=phiEc, phidom=phidomc)
        self.df = gf.data(s=sf, sigma=sigf, phiE=phiEf, phidom=phidomf)
        Ac, bc = gc.assemble(self.dc)
        Af, bf = gf.assemble(self.df)
        M = self.averaging()
        # coarse dofs as a function of the composite vector: outside cells
        # directly, under-box cells through the averaging map
        keep = np.nonzero(self.cmap >= 0)[0]
        E = sp.csr_matrix((np.ones(len(keep)), (keep, self.cmap[keep])), shape=(gc.ndof, self.nco))
        Tc = sp.hstack([E, M]).tocsr()  # coarse dof values = Tc x
        Rc = sp.csr_matrix((np.ones(len(keep)), (self.cmap[keep], keep)), shape=(self.nco, gc.ndof))
        Ac_comp = Rc @ Ac @ Tc
        Af_comp = sp.hstack([sp.csr_matrix((gf.ndof, self.nco)), Af]).tocsr()
        A = sp.vstack([Ac_comp, Af_comp]).tolil()
        b = np.concatenate([Rc @ bc, bf])
        hf, hc = gf.h, gc.h
        # CF fluxes and refluxing
        for (a, s, fc, J, cc, CI, al, terms) in self.faces:
            eps0 = float(self.desc["eps"][0])
            # F_cf = eps0 (ghost - phi_F)/h_f as a row over the composite vector
            row = {}
            for space, i, w in terms:
                col = (self.nco + i) if space == "f" else int(self.cmap[i])
                row[col] = row.get(col, 0.0) + eps0 * w / hf
            colF = self.nco + int(gf.dof[0][fc])
            row[colF] = row.get(colF, 0.0) - eps0 / hf
            rf = self.nco + int(gf.dof[0][fc])
            rcr = int(self.cmap[gc.dof[0][cc]])
            for col, w in row.items():
                A[rf, col] -= al * w / hf                       # r_F += alpha F / h_f
                A[rcr, col] += al * w / hc / (1 << (D - 1))     # r_C -= mean fine flux / h_c
        # every coarse row next to a CF side loses the coarse operator's own
        # flux through that side (the box has no coarse equation to balance it)
        for (a, s, CI) in self.coarse_cf_faces():
            cc = self.ccell(CI)
            if gc.dof[0][cc] < 0:
                continue
            rcr = int(self.cmap[gc.dof[0][cc]])
            JC = list(CI)
            if s == 0:
                JC[a] += 1  # C below the box: the face is C's high face
            sign = 1.0 if s == 0 else -1.0
            idx, w, c0 = gc.face_flux(self.dc, a, JC, 0)
            # r_C contains sign * (w . phi + c0); remove it
            for i, wk in zip(idx, w):
                r_i = int(self.cmap[i])
                if r_i >= 0:
                    A[rcr, r_i] += sign * wk
                else:  # a coarse dof under the box: through the averaging map
                    mrow = M.getrow(i)
                    for j, mv in zip(mrow.indices, mrow.data):
                        A[rcr, self.nco + j] += sign * wk * mv
            b[rcr] -= sign * c0
        self.A, self.b = A.tocsr(), b
        return self.A, self.b

    # ---------------------------------------------------------------- helpers
    def split(self, x):
        """Composite vector -> (coarse [2][cell] with the box filled by averages, fine [2][cell])."""
        gc, gf = self.gc, self.gf
        xf = x[self.nco:]
        xc = np.zeros(gc.ndof)
        keep = np.nonzero(self.cmap >= 0)[0]
        xc[keep] = x[self.cmap[keep]]
        M = self.averaging()
        under_dofs = M.getnnz(axis=1) > 0
        xc[under_dofs] = (M @ xf)[under_dofs]
        return gc.to_cells(xc), gf.to_cells(xf)

    def join(self, phic, phif):
        """(coarse [2][cell], fine [2][cell]) -> composite vector."""
        xc = self.gc.to_dofs(phic)
        keep = np.nonzero(self.cmap >= 0)[0]
        x = np.zeros(self.n)
        x[self.cmap[keep]] = xc[keep]
        x[self.nco:] = self.gf.to_dofs(phif)
        return x

    def solve(self, sc=None, sigc=None, sf=None, sigf=None):
        A, b = self.assemble(sc, sigc, sf, sigf)
        x = solve_system(A, b)
        return x, self.split(x)

    def boundary_flux(self, x):
        """Wall and EB fluxes of the composite grid: coarse cells outside the box and all fine cells."""
        gc, gf = self.gc, self.gf
        xc = np.zeros(gc.ndof)
        keep = np.nonzero(self.cmap >= 0)[0]
        xc[keep] = x[self.cmap[keep]]
        xc += self.averaging() @ x[self.nco:]
        return (gc.boundary_flux_masked(self.dc, xc, (~self.under).astype(np.uint8))
                + gf.boundary_flux(self.df, x[self.nco:]))

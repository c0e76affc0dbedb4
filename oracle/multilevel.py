"""Composite operator of the oracle over several nested refined levels.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): only tests/ and the
baseline legs of bench.py may use it.

The paper runs its solves on a hierarchy of refined levels (Sec. 3.3.2; the
refluxing of Sec. 3.3 couples each pair of levels; Sec. 6 refines where a
tracer field asks for it).  This module takes the following reading, written
out plainly on top of the two-level operator of oracle/composite.py:

  * Level 0 covers the domain.  Level l >= 1 is one box at ratio 2 over the
    cells [lo_l, hi_l) of level l-1, counted in level l-1's own grid (whose
    cell 0 is its box's lower corner); it is a grid of its own, computed from
    the same implicit functions, with homogeneous Neumann walls on its
    coarse-fine (CF) sides and the domain's conditions on sides that lie on
    the domain boundary.
  * Proper nesting: on every side of level l-1 that is a CF side, level l
    keeps at least one level-(l-1) cell away from it, so every coarse cell
    across a CF face of level l is a cell of level l-1 that carries its own
    equation.
  * Unknowns: every level's unknowns outside the next finer box; all of the
    finest level's.  A cell under the next finer box carries no equation;
    where a stencil reaches it, its value is the kappa-weighted mean of its
    children carrying the phase, whose values are in turn such means where
    they lie under a still finer box.
  * Each pair of consecutive levels is coupled exactly as in the two-level
    operator: ghost values behind the CF faces of the finer level by the
    quadratic tangential and normal Lagrange steps, the CF flux added to the
    fine rows, and the coarse row across a CF face losing the coarse
    operator's own flux through it and gaining minus the mean fine flux.
"""
from __future__ import annotations

import numpy as np

from . import OracleError, solve_system
from .composite import Composite


class MultiLevel:
    def __init__(self, desc: dict, boxes):
        """boxes: [(lo, hi), ...] for levels 1..L-1, each over its parent's grid."""
        self.D = D = int(desc["dim"])
        self.desc = desc
        if len(boxes) < 1:
            raise OracleError(1)
        self.pairs = []
        d = desc
        for lo, hi in boxes:
            lo = [int(v) for v in lo] + [0] * (3 - len(lo))
            hi = [int(v) for v in hi] + [1] * (3 - len(hi))
            if self.pairs:
                # proper nesting: one parent cell between the box and every CF side of the parent
                par = self.pairs[-1]
                n = par.nf
                for a in range(D):
                    if par.box_lo[a] > 0 and lo[a] < 1:
                        raise OracleError(1)
                    if par.box_hi[a] < par.nc[a] and hi[a] > n[a] - 1:
                        raise OracleError(1)
            P = Composite(d, lo, hi)
            self.pairs.append(P)
            d = P.fdesc
        self.L = len(self.pairs) + 1
        self.g = [P.gc for P in self.pairs] + [self.pairs[-1].gf]
        self.h = [g.h for g in self.g]
        # own unknowns of every level: outside the next finer box (all on the finest)
        self.own = []
        for l, g in enumerate(self.g):
            if l < self.L - 1:
                under = self.pairs[l].under
                keep = np.sort(np.concatenate([g.dof[p][(g.dof[p] >= 0) & ~under] for p in range(2)]))
            else:
                keep = np.arange(g.ndof)
            self.own.append(keep)
        self.off = np.concatenate([[0], np.cumsum([len(k) for k in self.own])]).astype(np.int64)
        self.n = int(self.off[-1])
        self._maps()

    def _maps(self):
        """T[l]: level l's full dof values as a linear map of the composite vector."""
        import scipy.sparse as sp
        L, n = self.L, self.n
        self.T = [None] * L
        self.M = [P.averaging() for P in self.pairs]
        for l in range(L - 1, -1, -1):
            g, keep = self.g[l], self.own[l]
            E = sp.csr_matrix((np.ones(len(keep)), (keep, self.off[l] + np.arange(len(keep)))), shape=(g.ndof, n))
            if l == L - 1:
                self.T[l] = E
            else:
                self.T[l] = (E + self.M[l] @ self.T[l + 1]).tocsr()
        # composite row of each own dof of a level
        self.row = []
        for l, g in enumerate(self.g):
            r = -np.ones(g.ndof, np.int64)
            r[self.own[l]] = self.off[l] + np.arange(len(self.own[l]))
            self.row.append(r)

    def assemble(self, s=None, sigma=None, phiE=None, phidom=None):
        """Composite A (CSR) and b over [level 0 own dofs, level 1 own dofs, ...].
        s, sigma, phiE, phidom: per-level lists (or None)."""
        import scipy.sparse as sp
        L, D = self.L, self.D

        def at(v, l):
            return None if v is None else v[l]
        self.data = [g.data(s=at(s, l), sigma=at(sigma, l), phiE=at(phiE, l), phidom=at(phidom, l))
                     for l, g in enumerate(self.g)]
        blocks, bs = [], []
        for l, g in enumerate(self.g):
            Al, bl = g.assemble(self.data[l])
            own = self.own[l]
            R = sp.csr_matrix((np.ones(len(own)), (np.arange(len(own)), own)), shape=(len(own), g.ndof))
            blocks.append(R @ Al @ self.T[l])
            bs.append(R @ bl)
        A = sp.vstack(blocks).tocsr()
        b = np.concatenate(bs)
        eps0 = float(self.desc["eps"][0])
        for l, P in enumerate(self.pairs):
            gc, gf = self.g[l], self.g[l + 1]
            hc, hf = self.h[l], self.h[l + 1]
            nface = len(P.faces)
            if nface:
                # CF flux of every fine face, eps0 (ghost - phi_F)/h_f, as rows over
                # the level dofs, then over the composite vector
                fr, fc_, fv = [], [], []
                cr, cc_, cv = [], [], []
                srow, scol, sval = [], [], []
                for k, (a, s_, fcell, J, ccell, CI, al, terms) in enumerate(P.faces):
                    for space, i, w in terms:
                        if space == "f":
                            fr.append(k)
                            fc_.append(i)
                            fv.append(eps0 * w / hf)
                        else:
                            cr.append(k)
                            cc_.append(i)
                            cv.append(eps0 * w / hf)
                    dF = int(gf.dof[0][fcell])
                    fr.append(k)
                    fc_.append(dF)
                    fv.append(-eps0 / hf)
                    rF = int(self.row[l + 1][dF])
                    rC = int(self.row[l][gc.dof[0][ccell]])
                    if rF < 0 or rC < 0:
                        raise OracleError(1)  # nesting violated
                    srow += [rF, rC]
                    scol += [k, k]
                    sval += [-al / hf, al / hc / (1 << (D - 1))]
                Gf = sp.csr_matrix((fv, (fr, fc_)), shape=(nface, gf.ndof))
                Gc = sp.csr_matrix((cv, (cr, cc_)), shape=(nface, gc.ndof))
                flux = Gf @ self.T[l + 1] + Gc @ self.T[l]
                S = sp.csr_matrix((sval, (srow, scol)), shape=(self.n, nface))
                A = (A + S @ flux).tocsr()
            # the coarse operator's own flux through each CF side is removed
            wr, wc, wv, rr, rc, rv = [], [], [], [], [], []
            for k, (a, s_, CI) in enumerate(P.coarse_cf_faces()):
                cc = P.ccell(CI)
                if gc.dof[0][cc] < 0:
                    continue
                rC = int(self.row[l][gc.dof[0][cc]])
                JC = list(CI)
                if s_ == 0:
                    JC[a] += 1
                sign = 1.0 if s_ == 0 else -1.0
                idx, w, c0 = gc.face_flux(self.data[l], a, JC, 0)
                for i, wk in zip(idx, w):
                    wr.append(k)
                    wc.append(int(i))
                    wv.append(wk)
                rr.append(rC)
                rc.append(k)
                rv.append(sign)
                b[rC] -= sign * c0
            if rr:
                nk = len(P.coarse_cf_faces())
                W = sp.csr_matrix((wv, (wr, wc)), shape=(nk, gc.ndof))
                S = sp.csr_matrix((rv, (rr, rc)), shape=(self.n, nk))
                A = (A + S @ (W @ self.T[l])).tocsr()
        self.A, self.b = A.tocsr(), b
        return self.A, self.b

    # ---------------------------------------------------------------- helpers
    def split(self, x):
        """Composite vector -> per-level [2][cell] arrays (cells under a finer box hold the means)."""
        return [g.to_cells(self.T[l] @ x) for l, g in enumerate(self.g)]

    def join(self, phis):
        """Per-level [2][cell] arrays -> composite vector (own cells only)."""
        x = np.zeros(self.n)
        for l, g in enumerate(self.g):
            xl = g.to_dofs(phis[l])
            x[self.off[l]:self.off[l + 1]] = xl[self.own[l]]
        return x

    def under(self, l):
        """Cells of level l under the next finer box (none on the finest)."""
        return self.pairs[l].under if l < self.L - 1 else np.zeros(self.g[l].ncell, bool)

    def volumes(self):
        """Cell volume h_l^D of every composite unknown."""
        return np.concatenate([np.full(len(self.own[l]), self.h[l] ** self.D) for l in range(self.L)])

    def solve(self, s=None, sigma=None):
        A, b = self.assemble(s=s, sigma=sigma)
        x = solve_system(A, b)
        return x, self.split(x)

    def boundary_flux(self, x):
        """Wall and EB fluxes of the composite grid (each level outside the next finer box)."""
        tot = 0.0
        for l, g in enumerate(self.g):
            xl = self.T[l] @ x
            if l < self.L - 1:
                tot += g.boundary_flux_masked(self.data[l], xl, (~self.pairs[l].under).astype(np.uint8))
            else:
                tot += g.boundary_flux(self.data[l], xl)
        return tot

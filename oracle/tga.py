"""TGA implicit Runge-Kutta diffusion step, on the oracle's operator.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/`` may
import it.  Shares no code with the CUDA path.

Sec. 3.4 advances a parabolic equation d phi/dt = L phi + rho by the scheme
of Twizell, Gumel and Arigu (Eq. tga): two Helmholtz solves per step,

    (I - mu1 L)(I - mu2 L) phi^{n+1} = (I + mu3 L) phi^n + dt (I + mu4 L) rho,
    mu1, mu2 = (a -+ sqrt(a^2 - 4a + 2)) dt / 2,  mu3 = (1 - a) dt,
    mu4 = (1/2 - a) dt,  a = 2 - sqrt(2) - eps  (eps the machine precision).

The printed equation drops the factor dt on the source and writes the model
equation as d phi/dt + L phi = rho while using I - mu L on the left; we read
it as above, the form of the scheme's source (McCorquodale et al.), whose
mu's make it second order and exact at steady state.  On cut cells the
finite-volume semi-discretisation is kappa d phi/dt = L_c phi + kappa rho per
cell (L_c = -A0, the operator integrated over the cell), so I becomes the
mass matrix M = diag(kappa) and the step is two solves:

    (M - mu1 L_c) psi = (M + mu3 L_c) phi^n + dt (M + mu4 L_c) rho,
    (M - mu2 L_c) phi^{n+1} = M psi.

A fragment of zero volume has M = 0: its rows are the constraint L_c phi = 0
at both stages, and its psi never reaches phi^{n+1}.  Boundary conditions are
homogeneous (the operator's boundary data is zero).  Vectors are over the
oracle's dofs.
"""
from __future__ import annotations

import math
import sys

import numpy as np

from . import Geometry, solve_system

PLANT = 0  # a planted mistake for the tests that show the pins catch it: 1 mu3 / mu4 swapped, 2 no M in stage 2


def coefficients(dt: float):
    """mu1, mu2, mu3, mu4 of one step of length dt."""
    a = 2.0 - math.sqrt(2.0) - sys.float_info.epsilon
    r = math.sqrt(a * a - 4.0 * a + 2.0)
    return (a - r) / 2.0 * dt, (a + r) / 2.0 * dt, (1.0 - a) * dt, (0.5 - a) * dt


class Diffusion:
    """The shift-free operator A0 (homogeneous data) and the mass matrix of a
    geometry; eps plays the diffusion coefficient."""

    def __init__(self, desc: dict):
        d = dict(desc)
        d["lam"] = (0.0, 0.0)
        self.g = Geometry(d)
        data = self.g.data(s=np.zeros((2, self.g.ncell)), sigma=np.zeros(self.g.ncell), phiE=0.0,
                           phidom=np.zeros((2, self.g.nwall)))
        self.A0, _ = self.g.assemble(data)
        kap = np.zeros(self.g.ndof)
        for p in range(2):
            m = self.g.dof[p] >= 0
            kap[self.g.dof[p][m]] = self.g.kappa[p][m]
        self.kappa = kap

    def step(self, phi: np.ndarray, rho: np.ndarray, dt: float) -> np.ndarray:
        """phi^{n+1} from phi^n, with the source rho (both over dofs, per unit volume)."""
        import scipy.sparse as sp
        mu1, mu2, mu3, mu4 = coefficients(dt)
        if PLANT == 1:
            mu3, mu4 = mu4, mu3
        M = sp.diags(self.kappa)
        Lphi = -(self.A0 @ phi)
        Lrho = -(self.A0 @ rho)
        R = self.kappa * phi + mu3 * Lphi + dt * (self.kappa * rho + mu4 * Lrho)
        psi = solve_system((M + mu1 * self.A0).tocsr(), R)
        rhs2 = psi if PLANT == 2 else self.kappa * psi
        return solve_system((M + mu2 * self.A0).tocsr(), rhs2)

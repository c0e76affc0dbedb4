"""Poisson solves inside the time step (arXiv:1809.03745, Sec. 3.6).

The paper's second-order fractional step advances the plasma in stages and
solves the Poisson equation three times per step: after the first
Runge-Kutta stage (charges rho*, sigma*), after the second (rho dagger,
sigma^{k+1}) and after the implicit diffusion (rho^{k+1}, sigma^{k+1}).  The
charges move little between solves, so each solve starts from the previous
potential.  This driver reproduces that regime for the solver: the transport
itself is out of scope, so the charges follow a prescribed synthetic motion
(a space-charge head drifting from the tip towards the plane and growing,
surface charge building up on the dielectric), evaluated at the stage times
of each step; the potential is carried from solve to solve on the device.

Usage: python -m paper_1809_03745_gb300.timestep [--n 1024] [--steps 20] [--dt 0.005]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import workloads as W

# where the synthetic motion stands at each solve of a step, in units of dt:
# the first solve sees the charges of the Euler predictor (a full step), the
# second those of the Heun average (modelled as half a step), the third those
# after the diffusion (a full step), so the charge moves back and forth
# within a step as the stages do
STAGES = (1.0, 0.5, 1.0)


def charges(desc, t: float, peak=100.0, speed=0.4, growth=2.0, sigma_rate=0.5, seed=W.SEED_BASE + 6):
    """Space charge s = rho/eps0 [2][cells] and surface charge sigma/eps0
    [cells] of the synthetic discharge at time t: a Gaussian head of width
    0.03 starting 0.05 below the tip and drifting towards the plane at
    `speed` while its peak grows by `growth` per unit time, a fixed seeded
    pattern of surface charge growing linearly at `sigma_rate`."""
    x, y, z = W.cell_centres(desc)
    tip = desc["prims"][0][1][1] - desc["prims"][0][1][6]  # the capsule's lower end minus its radius
    yc = max(tip - 0.05 - speed * t, 0.05)
    amp = peak * (1.0 + growth * t)
    s = amp * np.exp(-((x - 0.5) ** 2 + (y - yc) ** 2) / (2 * 0.03 ** 2))
    S = np.zeros((2, s.size))
    S[0] = s
    rng = np.random.default_rng(seed)
    pattern = rng.uniform(-1.0, 1.0, size=s.size)
    return S, sigma_rate * t * pattern


def step_inputs(desc, step: int, dt: float):
    """The (s, sigma) of the three solves of step `step`."""
    t0 = step * dt
    out = []
    for frac in STAGES:
        out.append(charges(desc, t0 + frac * dt))
    return out


def run(n=1024, steps=20, dt=0.005, device="cuda", warm=True, tol=1e-10, keep=False):
    """Advances `steps` steps of three solves each on the 2D multi-material
    rod-plane problem at n^2, each solve warm-started from the last
    potential (warm=False: from zero); returns per-step figures."""
    import torch

    from . import ebpoisson as E
    desc = W.rod_plane_2d(n, dielectric=True)
    g = E.Geometry(desc, device=device)
    P = E.Poisson(g, precision="mixed", tol=tol, max_cycles=200)
    inputs = [step_inputs(desc, k, dt) for k in range(steps)]
    dev = [[(torch.from_numpy(S).to(device), torch.from_numpy(sg).to(device)) for S, sg in st] for st in inputs]
    phi = torch.zeros(2, g.ncell, dtype=torch.float64, device=device)
    rows, kept = [], []
    for k in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vc = []
        for S, sg in dev[k]:
            if not warm:
                phi.zero_()
            _, info = P.solve(S, sg, phi)
            if info["status"] != 0:
                raise RuntimeError(f"step {k}: solve failed: {info}")
            vc.append(info["vcycles"])
            if keep:
                kept.append(phi.cpu().numpy())
        torch.cuda.synchronize()
        rows.append({"step": k, "ms": (time.perf_counter() - t0) * 1e3, "vcycles": vc})
    return {"cells": g.ncell, "rows": rows, "phi": phi, "desc": desc, "inputs": inputs, "solutions": kept}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--dt", type=float, default=0.005)
    args = ap.parse_args()
    out = {}
    for warm in (True, False):
        r = run(args.n, args.steps, args.dt, warm=warm)
        body = r["rows"][2:]  # the first steps include the start from zero
        ms = float(np.median([x["ms"] for x in body]))
        out["warm" if warm else "cold"] = {
            "ms_per_step": ms, "solves_per_step": 3, "cells": r["cells"],
            "cells_per_s": 3 * r["cells"] / (ms / 1e3),
            "vcycles_per_solve": float(np.mean([v for x in body for v in x["vcycles"]]))}
    print(json.dumps({"workload": f"2D multi-material rod-plane {args.n}^2, three Poisson solves per time step "
                                  f"(mixed, tol 1e-10), synthetic charge motion, dt {args.dt}", **out}), flush=True)


if __name__ == "__main__":
    main()

"""Implicit diffusion by TGA steps on the paper's geometries.

The drift-diffusion update of Sec. 3.4 advances the diffusion part with the
TGA scheme: two Helmholtz solves on the Poisson multigrid per step and
species.  This driver diffuses one species in the gas of the rod-plane (2D) or
pin-plane (3D) geometry (workloads.diffusion_inputs: absorbing solid, no flux
through the walls, a Gaussian seed and source below the tip) at a chosen
diffusion number r = D dt / h^2, and reports the time per step and the
V-cycles of its two stage solves.  The explicit limit is r = 1/(2 dim); the
implicit step is meant for r well above it (refined cells near the tip).

Usage: python -m paper_1809_03745_gb300.diffusion [--dim 2] [--n 1024] [--r 10] [--steps 10]
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import workloads as W


def run(dim=2, n=1024, r=10.0, steps=10, tol=1e-10, device="cuda"):
    import torch

    from . import ebpoisson as E
    d, phi0, rho0 = W.diffusion_inputs(dim, n)
    dt = r / float(n) ** 2
    T = E.TGA(d, dt, tol=tol, device=device)
    kap = T.geom.export()["kappa"]
    phi = torch.from_numpy(phi0).to(device) * (kap > 0)
    rho = torch.from_numpy(rho0).to(device) * (kap > 0)
    out = torch.empty_like(phi)
    for _ in range(3):  # warm-up steps, not timed
        T.step(phi, rho, out)
    stream = torch.cuda.current_stream()
    rows = []
    cur = phi.clone()
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        _, infos = T.step(cur, rho, out)
        b.record(stream)
        torch.cuda.synchronize()
        if any(i["status"] != 0 for i in infos):
            raise RuntimeError(f"stage solve failed: {infos}")
        cur, out = out, cur
        rows.append({"ms": a.elapsed_time(b), "vcycles": [i["vcycles"] for i in infos]})
    # the solid absorbs: the share of seed and source that has left the gas
    fed = float((kap * phi).sum()) + float((kap * rho).sum()) * dt * steps
    absorbed = 1.0 - float((kap * cur).sum()) / fed
    return {"cells": T.geom.ncell, "dt": dt, "mu": T.mu, "rows": rows, "absorbed": absorbed}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--r", type=float, default=10.0, help="diffusion number D dt / h^2")
    ap.add_argument("--steps", type=int, default=10)
    args = ap.parse_args()
    res = run(args.dim, args.n, args.r, args.steps)
    ms = float(np.median([x["ms"] for x in res["rows"]]))
    print(json.dumps({"workload": f"{args.dim}D TGA diffusion step at {args.n}^{args.dim}, D dt/h^2 = {args.r:g} "
                                  "(absorbing solid, Neumann walls, mixed, tol 1e-10)",
                      "cells": res["cells"], "dt": res["dt"], "ms_per_step": ms, "solves_per_step": 2,
                      "cells_per_s": res["cells"] / (ms / 1e3), "vcycles": res["rows"][-1]["vcycles"],
                      "absorbed": res["absorbed"]}), flush=True)


if __name__ == "__main__":
    main()

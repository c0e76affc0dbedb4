"""Three-group photoionisation update: three Helmholtz solves with Robin outflow.

The paper's photoionisation model solves the stationary Eddington (SP1)
equation for three photon groups, kappa_g Psi_g - div(grad Psi_g / (3 kappa_g))
= eta / c, with the outflow condition dPsi/dn + 3 kappa_g / 2 Psi = 0 on every
boundary of the gas, and forms S_ph = nu_eff p_O2 sum_g A_g Psi_g (Sec. 2.3;
the appendix on photoionisation, with its table of lambda_g and A_g).  Each
update therefore runs the Poisson multigrid three times with a diagonal shift
and Robin boundaries.  This driver builds the three group problems on the
rod-plane (2D) or pin-plane (3D) geometry (workloads.photo_inputs), solves
them on the device and reports the time per update, from zero and
warm-started from the previous update's Psi_g with the emission grown by 2%
(it changes little between updates).

Usage: python -m paper_1809_03745_gb300.photoionization [--dim 2] [--n 1024] [--updates 5]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import workloads as W


def setup(dim, n, L=0.02, device="cuda", tol=1e-10):
    """The three group solvers with their sources on the device."""
    import torch

    from . import ebpoisson as E
    groups, w = W.photo_inputs(dim, n, L=L)
    solvers = []
    for d, S, sig in groups:
        g = E.Geometry(d, device=device)
        P = E.Poisson(g, precision="mixed", tol=tol, max_cycles=200)
        solvers.append((g, P, torch.from_numpy(S).to(device), torch.from_numpy(sig).to(device)))
    return solvers, w


def update(solvers, w, psi=None, grow=1.0):
    """One photoionisation update: the three group solves with the emission
    scaled by `grow` (warm-started from psi when given) and S_ph = sum_g w_g
    Psi_g on the device."""
    import torch
    out, infos = [], []
    for k, (g, P, S, sig) in enumerate(solvers):
        phi0 = psi[k] if psi is not None else torch.zeros(2, g.ncell, dtype=torch.float64, device=S.device)
        phi, info = P.solve(S * grow if grow != 1.0 else S, sig, phi0)
        if info["status"] != 0:
            raise RuntimeError(f"group {k + 1}: solve failed: {info}")
        out.append(phi)
        infos.append(info)
    sph = sum(wg * p[0] for wg, p in zip(w, out))
    return out, sph, infos


def run(dim=2, n=1024, updates=5, L=0.02, device="cuda"):
    import torch
    solvers, w = setup(dim, n, L, device)
    psi, _, infos = update(solvers, w)  # from zero
    rows = []
    for k in range(updates):
        # the emission grows by 2% per update, so each warm start has work to do
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        psi, sph, infos = update(solvers, w, [p.clone() for p in psi], grow=1.02 ** (k + 1))
        torch.cuda.synchronize()
        rows.append({"ms": (time.perf_counter() - t0) * 1e3, "vcycles": [i["vcycles"] for i in infos]})
    cold = []
    for _ in range(max(1, updates // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, ci = update(solvers, w)
        torch.cuda.synchronize()
        cold.append({"ms": (time.perf_counter() - t0) * 1e3, "vcycles": [i["vcycles"] for i in ci]})
    ncell = solvers[0][0].ncell
    return {"cells": ncell, "lam": [W.rte_desc(2, 8, W.photo_kappa(k) * L)["lam"][0] for k in range(3)],
            "warm": rows, "cold": cold, "sph_max": float(sph.abs().max())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--updates", type=int, default=5)
    ap.add_argument("--L", type=float, default=0.02, help="box side in metres")
    args = ap.parse_args()
    r = run(args.dim, args.n, args.updates, args.L)
    warm = float(np.median([x["ms"] for x in r["warm"]]))
    cold = float(np.median([x["ms"] for x in r["cold"]]))
    print(json.dumps({"workload": f"{args.dim}D three-group photoionisation update at {args.n}^{args.dim} "
                                  f"({args.L * 100:g} cm box, Robin outflow, mixed, tol 1e-10)",
                      "cells": r["cells"], "lam": r["lam"], "ms_per_update_warm": warm,
                      "ms_per_update_cold": cold, "solves_per_update": 3,
                      "cells_per_s_warm": 3 * r["cells"] / (warm / 1e3),
                      "vcycles_warm": r["warm"][-1]["vcycles"], "vcycles_cold": r["cold"][-1]["vcycles"],
                      "sph_max": r["sph_max"]}), flush=True)


if __name__ == "__main__":
    main()

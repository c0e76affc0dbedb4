"""Replays a seeded request trace against the solve server and against
one-at-a-time plain FP64 solves.

Requests: 90% drawn like the batched instances (2D 64^2..1024^2 or 3D
32^3..192^3, seeded geometry, permittivity, voltage and charge), 10% large 3D
pin-plane grids (`large_n`^3, single level of the finest grid, the pin-plane
geometry with a drawn voltage and charge peak).  Arrivals are a Poisson
process of rate lambda (seeded); lambda is `load` times the server's measured
capacity in requests/s from a closed-loop run of the same requests.

Server side: the requests are submitted at their arrival times from a client
thread, and latency runs from submission to the result being ready.
Baseline: every request is timed alone with the plain FP64 path (geometry,
setup and solve, multi-launch), and its latency is that of a single FIFO
server fed the same arrivals, computed from those service times.

Usage: python -m paper_1809_03745_gb300.serve_trace --requests 200 --load 0.7
"""
from __future__ import annotations

import argparse
import json
import math
import threading
import time

import numpy as np


def make_requests(count, seed=1815, large_frac=0.1, large_n=384):
    from . import workloads as W
    rng = np.random.Generator(np.random.PCG64(seed))
    is_large = rng.uniform(size=count) < large_frac
    small = W.batched_instances(count=int((~is_large).sum()), seed=seed + 1)
    reqs, it = [], iter(small)
    base = None
    for k in range(count):
        if is_large[k]:
            if base is None:
                d = W.pin_plane_3d(large_n)
                x, y, z = W.cell_centres(d)
                r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2
                dz = np.where(z < 0.05, 0.05 - z, np.where(z > 0.5, z - 0.5, 0.0))
                base = (d, np.exp(-r2 / (2 * 0.02 ** 2)) * np.exp(-dz ** 2 / (2 * 0.02 ** 2)))
                del x, y, z, r2, dz
            V = float(rng.uniform(0.5, 2.0))
            peak = float(math.exp(rng.uniform(math.log(10.0), math.log(1e3))))
            reqs.append((W.pin_plane_3d(large_n, V=V), ("large", peak), None))
        else:
            reqs.append(next(it))
    return reqs, base


def _fields(req, base):
    d, S, s = req
    if isinstance(S, tuple):  # large request: scaled shared charge profile
        g = base[1]
        S = np.zeros((2, g.size))
        S[0] = req[1][1] * g
        s = np.zeros(g.size)
    return d, S, s


def _ncell(d):
    return int(np.prod([int(d["n"][k]) for k in range(int(d["dim"]))]))


def run_server(reqs, base, arrivals, **opts):
    from . import ebpoisson as E
    srv = E.Server(**opts)
    lat = [None] * len(reqs)
    status = [None] * len(reqs)
    t_sub = [0.0] * len(reqs)
    tickets = {}
    lock = threading.Lock()
    t0 = time.perf_counter()

    def client():
        for k, req in enumerate(reqs):
            d, S, s = _fields(req, base)
            wait = t0 + arrivals[k] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            t = srv.submit(d, S, s)
            with lock:
                t_sub[k] = time.perf_counter()
                tickets[k] = t

    th = threading.Thread(target=client)
    th.start()
    remaining = set(range(len(reqs)))
    while remaining:
        for k in list(remaining):
            with lock:
                t = tickets.get(k)
            if t is None:
                continue
            r = srv.poll(t)
            if r is not None:
                lat[k] = (time.perf_counter() - t_sub[k]) * 1e3
                status[k] = r[1]["status"]
                remaining.discard(k)
        time.sleep(0.0005)
    th.join()
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    return lat, status, wall, st


def run_baseline(reqs, base, precision="fp64", launch_mode=2, tol=1e-10):
    """Service time of every request alone: geometry, setup and solve."""
    import torch
    from . import ebpoisson as E
    svc = []
    for req in reqs:
        d, S, s = _fields(req, base)
        torch.cuda.synchronize()
        t = time.perf_counter()
        g = E.Geometry(d)
        P = E.Poisson(g, precision=precision, tol=tol, max_cycles=400, launch_mode=launch_mode)
        phi, info = P.solve(torch.from_numpy(S), torch.from_numpy(s))
        out = phi.cpu()
        svc.append((time.perf_counter() - t) * 1e3)
        del P, g, phi, out
    return svc


def fifo_latency(arrivals_s, svc_ms):
    free = 0.0
    lat = []
    for a, s in zip(arrivals_s, svc_ms):
        start = max(a * 1e3, free)
        free = start + s
        lat.append(free - a * 1e3)
    return lat


def pct(x, q):
    x = sorted(x)
    return x[min(len(x) - 1, max(0, int(math.ceil(q * len(x))) - 1))]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--load", type=float, nargs="+", default=[0.5, 0.7, 0.9])
    ap.add_argument("--large-n", type=int, default=384)
    ap.add_argument("--seed", type=int, default=1815)
    ap.add_argument("--max-slots", type=int, default=64)
    ap.add_argument("--step-iters", type=int, default=1)
    ap.add_argument("--no-baseline", action="store_true")
    args = ap.parse_args()
    reqs, base = make_requests(args.requests, args.seed, large_n=args.large_n)
    cells = [_ncell(r[0]) for r in reqs]
    opts = dict(max_slots=args.max_slots, step_iters=args.step_iters, tol=1e-10, max_cycles=400)
    # capacity: everything submitted at once
    lat, status, wall, st = run_server(reqs, base, [0.0] * len(reqs), **opts)
    cap_rps = len(reqs) / wall
    out = {"requests": len(reqs), "cells": int(sum(cells)), "large_n": args.large_n,
           "closed_loop": {"wall_s": wall, "cells_per_s": sum(cells) / wall, "req_per_s": cap_rps,
                           "failed": int(sum(1 for s in status if s != 0)), "steps": st["steps"],
                           "hbm_peak": st["hbm_peak"], "hbm_budget": st["hbm_budget"]}}
    rng = np.random.Generator(np.random.PCG64(args.seed + 100))
    out["open_loop"] = []
    for load in args.load:
        lam = load * cap_rps
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=len(reqs)))
        arrivals -= arrivals[0]
        lat, status, wall, st = run_server(reqs, base, list(arrivals), **opts)
        ok = [l for l, s in zip(lat, status) if s == 0]
        row = {"load": load, "lambda_req_per_s": lam, "p50_ms": pct(ok, 0.5), "p99_ms": pct(ok, 0.99),
               "cells_per_s": sum(cells) / wall, "failed": int(sum(1 for s in status if s != 0)),
               "hbm_peak": st["hbm_peak"]}
        if not args.no_baseline:
            if "svc" not in out:
                svc = run_baseline(reqs, base)
                out["svc"] = {"fp64_plain_total_s": sum(svc) / 1e3,
                              "fp64_plain_cells_per_s": sum(cells) / (sum(svc) / 1e3)}
                out["_svc_ms"] = svc
            bl = fifo_latency(arrivals, out["_svc_ms"])
            row["baseline_p50_ms"], row["baseline_p99_ms"] = pct(bl, 0.5), pct(bl, 0.99)
        out["open_loop"].append(row)
        print(json.dumps(row), flush=True)
    out.pop("_svc_ms", None)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

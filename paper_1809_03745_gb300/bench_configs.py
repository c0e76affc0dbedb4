"""Measures every workload configuration on one GPU and prints one JSON line each.

  C1  2D rod-plane 128^2, single phase: FP64 V-cycles and mixed precision
  C2  2D multi-material 1024^2: FP64 V-cycles against FP32 V-cycles in FP64
      defect correction, and the plain multi-launch FP64 path
  C3  3D pin-plane 256^3 with a ratio-2 128^3 box around the tip (composite
      solve), and the 256^3 single level
  C4  64 seeded instances (2D 64^2..1024^2, 3D 32^3..192^3): one batched
      persistent launch (mixed) against one-at-a-time solves, plain FP64
      multi-launch and mixed persistent

Times are wall-clock around the solve calls after warm-up (device work
synchronised on both sides); inputs are resident on the device; all solves
run to max|r| <= 1e-10 max|b|.

With --trace c1|c2|c3 it instead prints where one V-cycle's time goes: the
persistent kernel's phase stamps of the first V-cycle (eb_poisson_trace),
summed per level and phase kind, and the grid-barrier cost.

With --regrid N it refines the N^3 pin-plane (C3 geometry and line charge)
by the Sec. 6 tracer criteria up to three levels (regrid.build_hierarchy),
then times a solve of the final hierarchy and the tagging kernels on its
finest level; with --regrid2d N the same on the N^2 C2 rod-plane.

With --composite N it runs one C3 composite solve at N^3 + (N/2)^3 (after
the set-up, no warm-up), and with --kernels N the large-grid kernels on their
own on the N^3 pin-plane finest level (the tile-streamed sweep, one colour
pass, the tile-streamed and the block residual + restriction, the block
prolongation, `--reps` launches each): the small, bounded programs the ncu captures run.

Usage: python -m paper_1809_03745_gb300.bench_configs [--only C1 C2 C3 C4]
       python -m paper_1809_03745_gb300.bench_configs --trace c2 [--n N] [--precision mixed|fp64]
       python -m paper_1809_03745_gb300.bench_configs --peaks   (measured FP64 / FP32 FMA rates)
       python -m paper_1809_03745_gb300.bench_configs --composite 256
       python -m paper_1809_03745_gb300.bench_configs --regrid 128
       python -m paper_1809_03745_gb300.bench_configs --tags 192 [--reps 20]
       python -m paper_1809_03745_gb300.bench_configs --bottom-ab 256   (bottom sweeps 64, 32, 24, 16)
       python -m paper_1809_03745_gb300.bench_configs --kernels 384 [--reps 20]
"""
from __future__ import annotations

import argparse
import collections
import json
import time

import numpy as np
import torch

from . import ebpoisson as E
from . import workloads as W


def _timed(fn, reps=3):
    fn()
    best, out = float("inf"), None
    for _ in range(reps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t)
    return best, out


def single(name, desc, S, sig, **kw):
    g = E.Geometry(desc)
    P = E.Poisson(g, **kw)
    rhs, sg = torch.from_numpy(S).cuda(), torch.from_numpy(sig).cuda()
    dt, (phi, info) = _timed(lambda: P.solve(rhs, sg))
    n = W.ncells(desc)
    return {"config": name, "cells": n, "ms": dt * 1e3, "cells_per_s": n / dt, "vcycles": info["vcycles"],
            "outer": info["outer_iters"], "rel_res": info["rel_res"], "status": info["status"],
            "opts": {k: v for k, v in kw.items()}}


def c1():
    d, S, sig = W.c1_inputs(128)
    yield single("C1 128^2 FP64", d, S, sig, precision="fp64", tol=1e-10, max_cycles=200)
    yield single("C1 128^2 mixed", d, S, sig, precision="mixed", tol=1e-10, max_cycles=200)


def c2():
    d, S, sig = W.c2_inputs(1024)
    yield single("C2 1024^2 FP64 V-cycles (persistent)", d, S, sig, precision="fp64", tol=1e-10, max_cycles=200)
    yield single("C2 1024^2 FP32 V-cycles in FP64 defect correction (persistent)", d, S, sig, precision="mixed",
                 tol=1e-10, max_cycles=200)
    yield single("C2 1024^2 FP64 plain multi-launch", d, S, sig, precision="fp64", tol=1e-10, max_cycles=200,
                 launch_mode=2)


def c3():
    d, lo, hi, Sc, sc, Sf, sf = W.c3_amr_inputs(256)
    t = time.perf_counter()
    G = E.Composite(d, lo, hi, precision="mixed", tol=1e-10, max_cycles=200)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t
    args = [torch.from_numpy(a).cuda() for a in (Sc, Sf, sc, sf)]
    dt, (pc, pf, info) = _timed(lambda: G.solve(*args), reps=2)
    n = 256 ** 3 - 64 ** 3 + 128 ** 3
    yield {"config": "C3 256^3 + 128^3 box composite, mixed", "cells": n, "ms": dt * 1e3, "cells_per_s": n / dt,
           "composite_iters": info["outer_iters"], "vcycles": info["vcycles"], "rel_res": info["rel_res"],
           "status": info["status"], "setup_s": setup}
    del G, args
    dd, S, sig = W.c3_inputs(256)
    yield single("C3 256^3 single level, mixed", dd, S, sig, precision="mixed", tol=1e-10, max_cycles=400)


def c4(count=64):
    inst = W.batched_instances(count=count)
    cells = sum(W.ncells(d) for d, _, _ in inst)
    geoms = [E.Geometry(d) for d, _, _ in inst]
    rhs = [torch.from_numpy(S).cuda() for _, S, _ in inst]
    sig = [torch.from_numpy(s).cuda() for _, _, s in inst]
    Pb = [E.Poisson(g, precision="mixed", tol=1e-10, max_cycles=600) for g in geoms]
    dt, (phis, infos) = _timed(lambda: E.solve_batched(Pb, rhs, sig), reps=2)
    yield {"config": f"C4 {count} instances, one batched persistent launch, mixed", "cells": cells,
           "ms": dt * 1e3, "cells_per_s": cells / dt, "statuses": sorted(set(i["status"] for i in infos)),
           "max_vcycles": max(i["vcycles"] for i in infos), "kernel_ms": infos[0]["kernel_ms"],
           "n_2d": sum(d["dim"] == 2 for d, _, _ in inst)}

    def one_by_one(Ps):
        return [P.solve(rhs[k], sig[k])[1] for k, P in enumerate(Ps)]
    dt1, inf1 = _timed(lambda: one_by_one(Pb), reps=1)
    yield {"config": f"C4 {count} instances one at a time, mixed persistent", "cells": cells, "ms": dt1 * 1e3,
           "cells_per_s": cells / dt1, "statuses": sorted(set(i["status"] for i in inf1))}
    del Pb
    torch.cuda.empty_cache()
    Pp = [E.Poisson(g, precision="fp64", tol=1e-10, max_cycles=600, launch_mode=2) for g in geoms]
    dt2, inf2 = _timed(lambda: one_by_one(Pp), reps=1)
    yield {"config": f"C4 {count} instances one at a time, plain FP64 multi-launch", "cells": cells,
           "ms": dt2 * 1e3, "cells_per_s": cells / dt2, "statuses": sorted(set(i["status"] for i in inf2))}


TRACE_KIND = {1: "red", 2: "rows", 3: "black", 4: "write", 5: "resrows", 6: "restrict", 7: "prolong",
              8: "coarseend", 9: "bottom", 12: "update", 13: "sweep"}


def trace(workload, n=None, precision="mixed"):
    """Phase trace of the first V-cycle of one solve (after two warm-up solves)."""
    gen = {"c1": (W.c1_inputs, 128), "c2": (W.c2_inputs, 1024), "c3": (W.c3_inputs, 128)}[workload]
    d, S, sig = gen[0](n or gen[1])
    P = E.Poisson(E.Geometry(d), precision=precision, tol=1e-10, max_cycles=400)
    rhs, sg = torch.from_numpy(S).cuda(), torch.from_numpy(sig).cuda()
    for _ in range(2):
        P.solve(rhs, sg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, info = P.solve(rhs, sg)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    print(f"{workload} n={n or gen[1]} {precision}: {info['vcycles']} V-cycles, {info['outer_iters']} outer, "
          f"rel_res {info['rel_res']:.2e}, wall {wall * 1e3:.2f} ms, kernel {info['kernel_ms']:.2f} ms")
    tr = P.trace()
    agg = collections.OrderedDict()
    for lev, k, ms in tr:
        key = (lev, TRACE_KIND.get(k, str(k)))
        cnt, t = agg.get(key, (0, 0.0))
        agg[key] = (cnt + 1, t + ms)
    print(f"  first V-cycle: {len(tr)} phases, {sum(ms for _, _, ms in tr) * 1e3:.1f} us")
    for (lev, k), (cnt, t) in agg.items():
        print(f"    L{lev:2d} {k:10s} n={cnt:3d} {t * 1e3:8.1f} us  avg {t * 1e3 / cnt:6.2f}")
    print(f"  grid barrier: {P.profile(2, 1000)[0] * 1e3:.2f} us")


def composite_once(n):
    """One C3 composite solve at n^3 + (n/2)^3 right after the set-up."""
    d, lo, hi, Sc, sc, Sf, sf = W.c3_amr_inputs(n)
    G = E.Composite(d, lo, hi, precision="mixed", tol=1e-10, max_cycles=200)
    args = [torch.from_numpy(a).cuda() for a in (Sc, Sf, sc, sf)]
    _, _, info = G.solve(*args)
    torch.cuda.synchronize()
    print(json.dumps({"workload": f"C3 composite {n}^3 + {n // 2}^3 box, one solve", "status": info["status"],
                      "outer_iters": info["outer_iters"], "vcycles": info["vcycles"], "rel_res": info["rel_res"],
                      "kernel_launches": info["kernel_launches"], "kernel_stats": G.kernel_stats()}), flush=True)


def composite_bottom_ab(n, sweeps):
    """The C3 composite solve at n^3 + (n/2)^3 with each bottom sweep count (set-up, one warm-up, best of 2)."""
    d, lo, hi, Sc, sc, Sf, sf = W.c3_amr_inputs(n)
    args = [torch.from_numpy(a).cuda() for a in (Sc, Sf, sc, sf)]
    for bs in sweeps:
        G = E.Composite(d, lo, hi, precision="mixed", tol=1e-10, max_cycles=200, bottom_sweeps=bs)
        dt, (_, _, info) = _timed(lambda: G.solve(*args), reps=2)
        print(json.dumps({"workload": f"C3 composite {n}^3 + {n // 2}^3 box", "bottom_sweeps": bs, "ms": dt * 1e3,
                          "outer_iters": info["outer_iters"], "vcycles": info["vcycles"], "rel_res": info["rel_res"],
                          "status": info["status"], "kernel_stats": G.kernel_stats()}), flush=True)
        G.close()


def kernels_once(n, reps):
    """The large-grid kernels of the n^3 pin-plane finest level, each launched
    on its own (eb_poisson_profile kernels 4, 0, 5, 1)."""
    P = E.Poisson(E.Geometry(W.pin_plane_3d(n)), precision="mixed", tol=1e-10, max_cycles=1)
    names = {4: "streamed sweep", 0: "colour pass", 5: "streamed residual + restriction",
             1: "block residual + restriction", 6: "block prolongation"}
    for k in (4, 0, 5, 1, 6):
        try:
            ms, by = P.profile(k, reps=reps)
        except E.EBError as exc:  # no streamed level below 2^25 cells
            print(json.dumps({"kernel": names[k], "n": n, "skipped": str(exc)}), flush=True)
            continue
        print(json.dumps({"kernel": names[k], "n": n, "ms": ms, "gbs": by / ms / 1e6}), flush=True)


def regrid_once(n, dim):
    """Sec. 6 regrid of the pin-plane (3D) or rod-plane (2D) to three levels, then timings."""
    from . import regrid as R
    if dim == 3:
        desc = W.pin_plane_3d(n)
        src = lambda x, y, z: W.line_charge(x, y, z, 1e3)  # noqa: E731
    else:
        desc = W.rod_plane_2d(n, dielectric=True)
        src = lambda x, y, z: 100 * np.exp(-((x - 0.5) ** 2 + (y - 0.45) ** 2) / (2 * 0.03 ** 2))  # noqa: E731
    torch.cuda.synchronize()
    t = time.perf_counter()
    out = R.build_hierarchy(desc, src, max_levels=3, precision="mixed", tol=1e-10)
    torch.cuda.synchronize()
    t_regrid = time.perf_counter() - t
    H = out["hierarchy"]
    rec = {"workload": f"regrid {'pin-plane' if dim == 3 else 'rod-plane'} {n}^{dim}, three levels by Sec. 6 tags",
           "boxes": out["boxes"], "steps": [{k: v for k, v in st.items() if k != "e_max"} for st in out["steps"]],
           "regrid_s": t_regrid}
    if H is not None:
        cells = [H.levels[l]["n_cells"] for l in range(H.L)]
        S = [torch.from_numpy(R.level_sources(H.level_desc(l), src)).cuda() for l in range(H.L)]
        dt, (phis, info) = _timed(lambda: H.solve(S), reps=2)
        own = sum(cells) - sum(int(np.prod([hi - lo for lo, hi in zip(*b)])) for b in out["boxes"])
        rec.update(level_cells=cells, composite_cells=own, solve_ms=dt * 1e3, cells_per_s=own / dt,
                   composite_iters=info["outer_iters"], vcycles=info["vcycles"], rel_res=info["rel_res"])
        Ef = H.field(H.L - 1, phis[-1])[0]
        g = H.level_geom(H.L - 1)
        reps = 20
        E.tag_cells(g, Ef, want_tags=True)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(reps):
            E.tag_cells(g, Ef, want_tags=True)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t) / reps * 1e3
        nf = cells[-1]
        rec.update(tag_ms=ms, tag_cells=nf, tag_gbs=(dim * 2 * 8 + 1 + 1) * nf / ms / 1e6)
    print(json.dumps(rec), flush=True)


def tags_once(n, reps):
    """The tagging kernels on the N^3 pin-plane's single-level field, `reps` launches."""
    desc = W.pin_plane_3d(n)
    x, y, z = W.cell_centres(desc)
    S = np.zeros((2, x.size))
    S[0] = W.line_charge(x, y, z, 1e3)
    g = E.Geometry(desc)
    P = E.Poisson(g, precision="mixed", tol=1e-10, max_cycles=400)
    phi, _ = P.solve(torch.from_numpy(S))
    Ef = P.field(phi)[0]
    E.tag_cells(g, Ef)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(reps):
        _, blo, bhi, nm, emax = E.tag_cells(g, Ef)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t) / reps * 1e3
    by = (3 * 2 * 8 + 1 + 1) * g.ncell
    print(json.dumps({"workload": f"tags of the {n}^3 pin-plane field", "cells": g.ncell, "ms_per_call": ms,
                      "bytes_model": "per cell: E read once (3 x 2 x 8 B), flags 1 B, tag 1 B",
                      "gbs": by / ms / 1e6, "n_marked": nm, "bbox": [blo, bhi]}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="+", default=["C1", "C2", "C3", "C4"])
    ap.add_argument("--trace", choices=["c1", "c2", "c3"], default=None)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--peaks", action="store_true")
    ap.add_argument("--composite", type=int, default=None)
    ap.add_argument("--kernels", type=int, default=None)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--regrid", type=int, default=None)
    ap.add_argument("--regrid2d", type=int, default=None)
    ap.add_argument("--tags", type=int, default=None)
    ap.add_argument("--bottom-ab", type=int, default=None)
    args = ap.parse_args()
    E.load()
    if args.composite:
        composite_once(args.composite)
        return
    if args.bottom_ab:
        composite_bottom_ab(args.bottom_ab, (64, 32, 24, 16))
        return
    if args.tags:
        tags_once(args.tags, args.reps)
        return
    if args.regrid or args.regrid2d:
        regrid_once(args.regrid or args.regrid2d, 3 if args.regrid else 2)
        return
    if args.kernels:
        kernels_once(args.kernels, args.reps)
        return
    if args.peaks:
        f64, f32 = E.device_fma_rates(torch.cuda.current_device())
        print(json.dumps({"fp64_fma_tflops": f64, "fp32_fma_tflops": f32}), flush=True)
        return
    if args.trace:
        trace(args.trace, args.n, args.precision)
        return
    for name, fn in (("C1", c1), ("C2", c2), ("C3", c3), ("C4", c4)):
        if name in args.only:
            for line in fn():
                print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()

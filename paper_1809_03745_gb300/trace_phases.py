"""Phase trace of the persistent solve kernel: where one V-cycle's time goes.

Solves a workload once (after two warm-up solves) and prints, from
`eb_poisson_trace`, the time of the first V-cycle's phases summed per level
and kind, the solve's wall and kernel time, and the grid-barrier cost.

Usage: python -m paper_1809_03745_gb300.trace_phases [c1|c2|c3] [--n N] [--precision mixed|fp64]
"""
from __future__ import annotations

import argparse
import collections
import time

import torch

from . import ebpoisson as E
from . import workloads as W

KIND = {1: "red", 2: "rows", 3: "black", 4: "write", 5: "resrows", 6: "restrict", 7: "prolong", 8: "coarseend",
        9: "bottom", 12: "update"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", nargs="?", default="c2", choices=["c1", "c2", "c3"])
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    args = ap.parse_args()
    gen = {"c1": (W.c1_inputs, 128), "c2": (W.c2_inputs, 1024), "c3": (W.c3_inputs, 128)}[args.workload]
    d, S, sig = gen[0](args.n or gen[1])
    P = E.Poisson(E.Geometry(d), precision=args.precision, tol=1e-10, max_cycles=400)
    rhs, sg = torch.from_numpy(S).cuda(), torch.from_numpy(sig).cuda()
    for _ in range(2):
        P.solve(rhs, sg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, info = P.solve(rhs, sg)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    print(f"{args.workload} n={args.n or gen[1]} {args.precision}: {info['vcycles']} V-cycles, {info['outer_iters']} "
          f"outer, rel_res {info['rel_res']:.2e}, wall {wall * 1e3:.2f} ms, kernel {info['kernel_ms']:.2f} ms")
    tr = P.trace()
    agg = collections.OrderedDict()
    for lev, k, ms in tr:
        key = (lev, KIND.get(k, str(k)))
        n, t = agg.get(key, (0, 0.0))
        agg[key] = (n + 1, t + ms)
    print(f"  first V-cycle: {len(tr)} phases, {sum(ms for _, _, ms in tr) * 1e3:.1f} us")
    for (lev, k), (n, t) in agg.items():
        print(f"    L{lev:2d} {k:10s} n={n:3d} {t * 1e3:8.1f} us  avg {t * 1e3 / n:6.2f}")
    print(f"  grid barrier: {P.profile(2, 1000)[0] * 1e3:.2f} us")


if __name__ == "__main__":
    main()

"""Autotuner for the multigrid schedule: smoother sweeps and inner V-cycles.

The paper fixes no sweep counts (Sec. 3.3.2 only names red-black
Gauss-Seidel V-cycles), and the best choice depends on the dimension and on
the cut-cell content: on two-phase rod-plane grids 2+2 sweeps are fastest,
on 3D pin-plane grids 6+6 sweeps need a sixth of the V-cycles.  The tuner
times complete solves (device time of the persistent solve kernel, from
CUDA events) for a small set of candidate schedules on a sample problem of a
size class, keeps the fastest that converges, and caches it in a JSON file
keyed by the class: dimension, log2 of the cell count, phase count and
precision.  Solvers for later problems of the class take the cached choice.

The search itself is host logic; every solve it times runs through the C
ABI.  `measure` can be replaced (tests use a fake) so the selection and
caching logic runs without a GPU.
"""
from __future__ import annotations

import json
import math
import os
import threading

# (nu1, nu2, inner V-cycles per FP64 outer iteration)
CANDIDATES = [(2, 2, 2), (2, 2, 3), (3, 3, 2), (4, 4, 2), (4, 4, 3), (6, 6, 2), (8, 8, 2)]


def default_schedule(dim: int):
    """The library's own choice when nothing is cached (nu1 = nu2 = -1)."""
    return (6, 6, 2) if dim == 3 else (2, 2, 2)


def size_class(dim: int, ncell: int, n_phase: int, precision: str) -> str:
    return f"{dim}d-2^{int(round(math.log2(max(ncell, 1))))}-ph{n_phase}-{precision}"


class Autotuner:
    def __init__(self, path: str | None = None, candidates=None):
        self.path = path
        self.candidates = list(candidates or CANDIDATES)
        self.table: dict[str, dict] = {}
        self._lock = threading.Lock()
        if path and os.path.exists(path):
            with open(path) as f:
                self.table = json.load(f)

    # ------------------------------------------------------------ cache
    def lookup(self, key: str):
        with self._lock:
            e = self.table.get(key)
        return tuple(e["schedule"]) if e else None

    def _store(self, key: str, schedule, trials):
        with self._lock:
            self.table[key] = {"schedule": list(schedule), "trials": trials}
            if self.path:
                tmp = self.path + ".tmp"
                with open(tmp, "w") as f:
                    json.dump(self.table, f, indent=1, sort_keys=True)
                os.replace(tmp, self.path)

    # ------------------------------------------------------------ search
    def select(self, key: str, measure):
        """measure(schedule) -> (ms, converged).  Returns the fastest
        converging schedule (ties: fewer sweeps) and caches it; if none
        converges, the first candidate is returned and nothing is cached."""
        trials = []
        for sch in self.candidates:
            ms, ok = measure(sch)
            trials.append({"schedule": list(sch), "ms": float(ms), "converged": bool(ok)})
        good = [t for t in trials if t["converged"] and math.isfinite(t["ms"])]
        if not good:
            return tuple(self.candidates[0])
        best = min(good, key=lambda t: (t["ms"], t["schedule"][0] + t["schedule"][1]))
        self._store(key, best["schedule"], trials)
        return tuple(best["schedule"])

    # ------------------------------------------------------------ GPU use
    def tune(self, geom, rhs, sigma=None, *, precision="mixed", tol=1e-10, max_cycles=400, reps=2):
        """Times every candidate on (geom, rhs, sigma) and caches the winner
        for the problem's size class; returns the schedule."""
        from . import ebpoisson as E
        key = size_class(geom.dim, geom.ncell, int(geom.info["n_phase"]), precision)

        def measure(sch):
            P = E.Poisson(geom, precision=precision, tol=tol, max_cycles=max_cycles, nu1=sch[0], nu2=sch[1],
                          inner_cycles=sch[2])
            try:
                P.solve(rhs, sigma)  # warm-up
                ms = []
                ok = True
                for _ in range(reps):
                    _, info = P.solve(rhs, sigma)
                    ok = ok and info["status"] == 0
                    ms.append(info["kernel_ms"] if info["kernel_ms"] > 0 else float("inf"))
                return min(ms), ok
            finally:
                P.close()

        return self.select(key, measure)

    def schedule(self, geom, precision="mixed"):
        key = size_class(geom.dim, geom.ncell, int(geom.info["n_phase"]), precision)
        return self.lookup(key) or default_schedule(geom.dim)

    def solver(self, geom, *, precision="mixed", **kw):
        """A Poisson solver with the cached (else default) schedule of the class."""
        from . import ebpoisson as E
        nu1, nu2, inner = self.schedule(geom, precision)
        return E.Poisson(geom, precision=precision, nu1=nu1, nu2=nu2, inner_cycles=inner, **kw)

"""Host-side logic on the CPU: the bench's algorithmic-bytes model, the
serving trace's FIFO baseline and percentiles, and the batched-instance
sampler's stated readings (sizes, seeds, thickness clamps)."""
import json
import math
import os

import numpy as np
import pytest

import bench
from paper_1809_03745_gb300 import serve_trace as T
from paper_1809_03745_gb300 import workloads as W


def test_solve_bytes_model():
    # per fine cell and V-cycle, FP32 2D with 2+2 sweeps: 4 sweeps x (read x, b, write x: 12 B + flag byte)
    # + residual/restriction (read x, b 8 B, flags 1 B, write coarse b and x 2 x 4 / 4 B) + prolongation
    # (coarse x 4 / 4 B, read and write x 8 B, flags 1 B) = 52 + 11 + 10 = 73 B, times the level sum 4/3
    assert bench.vcycle_bytes(2, 4, 4) == pytest.approx(73.0 * 4 / 3)
    # FP64: 4 x 25 + (16 + 1 + 4) + (2 + 16 + 1) = 140 B
    assert bench.vcycle_bytes(2, 8, 4) == pytest.approx(140.0 * 4 / 3)
    # 3D, FP32, 3+3 sweeps: 6 x 13 + (8 + 1 + 1) + (0.5 + 8 + 1) = 97.5 B, level sum 8/7
    assert bench.vcycle_bytes(3, 4, 6) == pytest.approx(97.5 * 8 / 7)
    # a solve adds 44 B per FP64 outer iteration and 24 B per launch; linear in cells
    v = bench.vcycle_bytes(2, 4, 4)
    assert bench.solve_bytes(1000, 2, True, 14, 7) == pytest.approx(1000 * (14 * v + 7 * 44 + 24))
    assert bench.solve_bytes(10, 3, True, 5, 3, sweeps=6, launches=2) == pytest.approx(
        10 * (5 * bench.vcycle_bytes(3, 4, 6) + 3 * 44 + 48))
    # the composite grid: coarse cells outside the quarter-width box plus the ratio-2 fine cells
    assert bench.composite_cells(256) == 256 ** 3 - 64 ** 3 + 128 ** 3 == 18612224


def test_fifo_latency_and_percentiles():
    # arrivals (s) and service times (ms): a single FIFO server
    lat = T.fifo_latency([0.0, 0.001, 0.5], [10.0, 10.0, 10.0])
    assert lat == pytest.approx([10.0, 19.0, 10.0])
    x = list(range(1, 101))
    assert T.pct(x, 0.5) == 50 and T.pct(x, 0.99) == 99 and T.pct(x, 1.0) == 100
    assert T.pct([7.0], 0.99) == 7.0


def test_batched_instances_follow_their_readings():
    inst = W.batched_instances(count=40)
    again = W.batched_instances(count=40)
    dims = set()
    for (d, S, s), (d2, S2, s2) in zip(inst, again):
        assert d == d2 and np.array_equal(S, S2)  # seeded: identical on every call
        n, D = d["n"][0], d["dim"]
        dims.add(D)
        assert n % 16 == 0 and all(d["n"][k] == n for k in range(D))
        lo, hi = (32, 192) if D == 3 else (64, 1024)
        assert lo - 8 <= n <= hi + 8
        h = d["h"]
        assert math.isclose(h, 1.0 / n)
        tip_r = d["prims"][0][1][-1]
        assert tip_r >= 3 * h - 1e-12  # tip radius clamped to at least 3 cells
        assert S.shape == (2, W.ncells(d)) and np.all(S[1] == 0.0) and S[0].max() > 0.0
    assert dims == {2, 3}
    small = W.batched_instances(count=20, max_cells=40000)
    assert all(W.ncells(d) <= 40000 for d, _, _ in small)


def test_refined_box_description():
    d = W.pin_plane_3d(64)
    f = W.refined_box_desc(d, [24, 24, 24], [40, 40, 40])
    assert f["n"] == (32, 32, 32) and f["h"] == d["h"] / 2
    assert f["lo"] == pytest.approx((24 / 64, 24 / 64, 24 / 64))


def test_traffic_record_is_tied_to_kernel_sources():
    """The DRAM traffic of profiles/traffic.json counts only for the sources it
    was captured on: the hash changes with any one of them."""
    import bench
    files = {n: n.encode() * 3 for n in bench.KERNEL_SOURCES}
    h0 = bench.kernel_sources_sha256(lambda n: files[n])
    assert h0 == bench.kernel_sources_sha256(lambda n: files[n])
    for n in bench.KERNEL_SOURCES:
        changed = dict(files, **{n: files[n] + b" "})
        assert bench.kernel_sources_sha256(lambda m: changed[m]) != h0
    rec = json.load(open(os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.json")))
    assert len(rec["sources_sha256"]) == 64
    assert any(k.startswith("k_solve_fp32") and v > 0 for k, v in rec.items() if isinstance(v, (int, float)))

"""Serving loop: continuous batching through the C ABI.

Each result of a mixed stream of requests equals the single solve of the
same problem with the same options (bitwise: the batched steps replay the
single solve's iterates); admission keeps the accounted device memory within
the budget; a request whose geometry is rejected completes with its error
and leaves the others untouched; a full queue refuses submissions."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1809_03745_gb300 import workloads as W

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1809_03745_gb300 import ebpoisson as E


def _single(d, S, s, **kw):
    P = E.Poisson(E.Geometry(d), **kw)
    phi, info = P.solve(torch.from_numpy(S), torch.from_numpy(s))
    return phi.cpu().numpy(), info


def test_results_same_alone_and_in_the_mix():
    inst = W.batched_instances(count=10, seed=1809 + 50, n2=(64, 384), n3=(32, 64), max_cells=150000)
    srv = E.Server(max_slots=4, step_iters=1, tol=1e-10, max_cycles=400)
    try:
        tickets = []
        for k, (d, S, s) in enumerate(inst):
            tickets.append(srv.submit(d, S, s))
            if k % 3 == 2:
                time.sleep(0.01)  # later requests arrive while earlier ones run
        res = [srv.wait(t, 300.0) for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    for (d, S, s), r in zip(inst, res):
        assert r is not None
        phi, info = r
        assert info["status"] == 0 and info["rel_res"] <= 1e-10, info
        alone, ai = _single(d, S, s, tol=1e-10, max_cycles=400)
        assert ai["vcycles"] == info["vcycles"]
        assert np.array_equal(alone, phi), np.abs(alone - phi).max()
    assert st["completed"] == len(inst) and st["failed"] == 0
    assert st["steps"] >= max(r[1]["outer_iters"] for r in res)
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    assert st["cells_per_s"] > 0 and st["estimate_misses"] == 0


def test_small_results_match_oracle():
    inst = W.batched_instances(count=4, seed=1809 + 51, n2=(64, 160), n3=(32, 40), max_cells=40000)
    srv = E.Server(max_slots=8, step_iters=2, tol=1e-12, max_cycles=600)
    try:
        tickets = [srv.submit(d, S, s) for d, S, s in inst]
        res = [srv.wait(t, 300.0) for t in tickets]
    finally:
        srv.close()
    for (d, S, s), (phi, info) in zip(inst, res):
        assert info["status"] == 0, info
        og, ophi, A, b, data = oracle.solve(d, s=S, sigma=s)
        assert np.abs(phi - ophi).max() <= 1e-9 * np.abs(ophi).max()


def test_admission_respects_memory_budget():
    inst = W.batched_instances(count=6, seed=1809 + 52, n2=(256, 256), n3=(32, 32), p3d=0.0)
    # the server's pre-build estimate of one 256^2 instance (including the
    # bound on a dense bottom inverse); an admitted instance is then accounted
    # at its measured size, so 1.2 estimates of budget hold a few at a time
    per = 256 * 256 * 200 + 257 * 257 + (8 << 20) + 1024 * 1024 * 8
    srv = E.Server(max_slots=16, hbm_budget_bytes=1.2 * per, tol=1e-10, max_cycles=400)
    try:
        tickets = [srv.submit(d, S, s) for d, S, s in inst]
        peak_active = 0
        while True:
            st = srv.stats()
            peak_active = max(peak_active, st["active"])
            if st["completed"] + st["failed"] == len(inst):
                break
            time.sleep(0.002)
        res = [srv.wait(t, 60.0) for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    assert all(r[1]["status"] == 0 for r in res)
    assert st["hbm_peak"] <= st["hbm_budget"], st
    assert st["estimate_misses"] == 0
    assert peak_active < len(inst)  # the budget, not the slot count, limited admission
    assert st["hbm_used"] == 0


def test_failed_request_does_not_disturb_others():
    good = W.batched_instances(count=3, seed=1809 + 53, n2=(64, 128), n3=(32, 32), p3d=0.0)
    bad = W.rod_plane_2d(32, dielectric=True, tip_y=0.21, slab_y=0.2, rough_amp=0.0)  # electrode cuts the slab
    n = W.ncells(bad)
    srv = E.Server(max_slots=4, tol=1e-10, max_cycles=400)
    try:
        t0 = srv.submit(*good[0])
        tb = srv.submit(bad, np.zeros((2, n)), np.zeros(n))
        t1 = srv.submit(*good[1])
        t2 = srv.submit(*good[2])
        out = {t: srv.wait(t, 120.0) for t in (t0, tb, t1, t2)}
        st = srv.stats()
    finally:
        srv.close()
    assert out[tb][1]["status"] == E.EB_ERR_UNSUPPORTED
    for t, (d, S, s) in zip((t0, t1, t2), good):
        phi, info = out[t]
        assert info["status"] == 0
        alone, _ = _single(d, S, s, tol=1e-10, max_cycles=400)
        assert np.array_equal(alone, phi)
    assert st["failed"] == 1 and st["completed"] == 3


def test_full_queue_refuses_and_poll_before_ready():
    d, S, s = W.c2_inputs(512)
    srv = E.Server(max_slots=1, queue_cap=1, tol=1e-10, max_cycles=400)
    try:
        t1 = srv.submit(d, S, s)
        t_end = time.time() + 30
        while srv.stats()["active"] < 1 and time.time() < t_end:  # t1 admitted: the queue is empty again
            time.sleep(0.001)
        t2 = srv.submit(d, S, s)
        busy = 0
        try:
            srv.submit(d, S, s)
            srv.submit(d, S, s)
        except E.EBError as e:
            assert e.status == E.EB_ERR_BUSY
            busy += 1
        assert busy == 1
        assert srv.poll(t2) is None  # queued or running
        r1, r2 = srv.wait(t1, 120.0), srv.wait(t2, 120.0)
        assert r1[1]["status"] == 0 and np.array_equal(r1[0], r2[0])
        with pytest.raises(E.EBError):
            srv.poll(t1)  # a ticket is forgotten once its result was taken
    finally:
        srv.close()

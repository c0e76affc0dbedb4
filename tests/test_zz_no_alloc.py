"""The allocation-free residual entry point.

Callers that cannot allocate device memory where they need a residual (a
fully carved-up memory pool, an allocator-free real-time loop) call
eb_poisson_residual_noalloc, which keeps its scratch in a static device array.
This checks, through the C ABI, that it returns what eb_poisson_residual
returns on two calls in a row with different inputs, in 2D and 3D (the static
array keeps the previous call's contents, which must not leak into the next
result); that a problem with more cells or more sparse rows than the array
holds is refused before any device work; and that a call made with another
device current than the geometry's is refused.
This file is collected last so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1809_03745_gb300 import workloads as W

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1809_03745_gb300 import ebpoisson as E


def _pin3d(n):
    d = W.pin_plane_3d(n, radius=0.08)
    x, y, z = W.cell_centres(d)
    S = np.zeros((2, W.ncells(d)))
    S[0] = 50.0 * np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.4) ** 2) / (2 * 0.05 ** 2))
    return d, S, np.zeros(W.ncells(d))


def _corrugated_slabs(n=96, ns=12, amp=0.03, periods=4.0, thick=2.3):
    """ns thin electrode slabs, each between two sine sheets: about 36% of the
    884,736 cells of a 96^3 grid are cut, beyond the static array's 2^19 sparse
    rows (two per cut cell) while the cell count stays under 2^20."""
    h = 1.0 / n
    prims, nodes, slabs = [], [], []
    for i in range(ns):
        c = (i + 0.5) / ns + 0.0123
        prims.append((W.PRIM_SINE, [2, c + 0.5 * thick * h, amp, periods, 0.7 * i, 0]))
        prims.append((W.PRIM_SINE, [2, c - 0.5 * thick * h, amp, periods, 0.7 * i, 0]))
        nodes += [(0, 2 * i, 0), (0, 2 * i + 1, 0)]
        nodes.append((3, len(nodes) - 1, 0))
        nodes.append((2, len(nodes) - 3, len(nodes) - 1))
        slabs.append(len(nodes) - 1)
    root = slabs[0]
    for s_ in slabs[1:]:
        nodes.append((1, root, s_))
        root = len(nodes) - 1
    return W._desc(3, (n, n, n), (0, 0, 0), h, prims, nodes, root, -1, (1.0, 1.0), [1] * 6, 1.0, [0] * 6)


def _noalloc(lib, g, rhs, sg, phi, out):
    return lib.eb_poisson_residual_noalloc(g._h, ctypes.c_void_p(rhs.data_ptr()),
                                           ctypes.c_void_p(sg.data_ptr()) if sg is not None else None,
                                           ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("case", ["c2_256", "pin3d_64"])
def test_noalloc_residual_matches_allocating_residual_twice(case):
    lib = E.load()
    d, S, sig = W.c2_inputs(256) if case == "c2_256" else _pin3d(64)
    g = E.Geometry(d)
    P = E.Poisson(g, precision="fp64")
    rng = np.random.default_rng(21)
    for call in range(2):
        phi = torch.from_numpy(rng.normal(size=(2, g.ncell)) * (call + 1)).cuda()
        rhs = torch.from_numpy(S * (1.0 + call)).cuda()
        sg = torch.from_numpy(sig * (1.0 - 2.0 * call)).cuda()
        ref = P.residual(rhs, sg, phi)
        out = torch.full_like(ref, float("nan"))
        st = _noalloc(lib, g, rhs, sg, phi, out)
        assert st == E.EB_OK, lib.eb_last_error()
        scale = ref.abs().max().item()
        assert torch.isfinite(out).all()
        assert (out - ref).abs().max().item() <= 1e-12 * scale


def test_noalloc_residual_rejects_oversize_problem():
    lib = E.load()
    d = W.rod_plane_2d(1032)  # 1032^2 > 2^20 cells
    g = E.Geometry(d)
    z = torch.zeros(2, g.ncell, dtype=torch.float64, device="cuda")
    st = lib.eb_poisson_residual_noalloc(g._h, ctypes.c_void_p(z.data_ptr()), None, ctypes.c_void_p(z.data_ptr()),
                                         ctypes.c_void_p(z.data_ptr()), None)
    assert st == E.EB_ERR_INVALID
    assert b"static scratch" in lib.eb_last_error()


def test_noalloc_residual_rejects_too_many_sparse_rows():
    lib = E.load()
    g = E.Geometry(_corrugated_slabs())
    assert g.ncell <= 1 << 20 and 2 * g.info["n_irregular"] > 1 << 19, g.info
    z = torch.zeros(2, g.ncell, dtype=torch.float64, device="cuda")
    st = _noalloc(lib, g, z, None, z, z)
    assert st == E.EB_ERR_INVALID
    assert b"sparse-row limit" in lib.eb_last_error()


@pytest.mark.skipif(torch.cuda.device_count() < 2, reason="needs a second GPU to make current")
def test_noalloc_residual_rejects_another_current_device():
    """The geometry lives on device 0; with device 1 current the call is refused
    on the host, before any launch."""
    lib = E.load()
    d, S, sig = W.c2_inputs(64)
    g = E.Geometry(d, device="cuda:0")
    z = torch.zeros(2, g.ncell, dtype=torch.float64, device="cuda:0")
    with torch.cuda.device(1):
        st = lib.eb_poisson_residual_noalloc(g._h, ctypes.c_void_p(z.data_ptr()), None,
                                             ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(z.data_ptr()), None)
    assert st == E.EB_ERR_INVALID
    assert b"not the geometry's device" in lib.eb_last_error()

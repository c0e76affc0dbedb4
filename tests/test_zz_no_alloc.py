"""The allocation-free residual entry point.

Callers that cannot allocate device memory where they need a residual (a
fully carved-up memory pool, an allocator-free real-time loop) call
eb_poisson_residual_noalloc, which keeps its scratch in a static device array.
This checks, through the C ABI, that it returns what eb_poisson_residual
returns on two calls in a row with different inputs (the static array keeps
the previous call's contents, which must not leak into the next result), and
that a problem larger than the array is refused before any device work.
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


def test_noalloc_residual_matches_allocating_residual_twice():
    lib = E.load()
    d, S, sig = W.c2_inputs(256)
    g = E.Geometry(d)
    P = E.Poisson(g, precision="fp64")
    rng = np.random.default_rng(21)
    for call in range(2):
        phi = torch.from_numpy(rng.normal(size=(2, g.ncell)) * (call + 1)).cuda()
        rhs = torch.from_numpy(S * (1.0 + call)).cuda()
        sg = torch.from_numpy(sig * (1.0 - 2.0 * call)).cuda()
        ref = P.residual(rhs, sg, phi)
        out = torch.full_like(ref, float("nan"))
        st = lib.eb_poisson_residual_noalloc(g._h, ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(sg.data_ptr()),
                                             ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
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

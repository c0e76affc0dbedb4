"""Host-side regrid logic of the library, without a GPU: the box rule of
eb_regrid_box equals the oracle's regrid box on random tag patterns (the
bounding box taken on the host), and eb_amr_setup_levels refuses badly nested
or badly sized boxes before any device work."""
import ctypes

import numpy as np
import pytest

from oracle import tagging as TG
from paper_1809_03745_gb300 import ebpoisson as E
from paper_1809_03745_gb300 import workloads as W


def _bbox(want, n, D):
    idx = np.nonzero(want)[0]
    I = [idx % n[0], (idx // n[0]) % n[1], idx // (n[0] * n[1])]
    return [int(I[a].min()) for a in range(D)], [int(I[a].max()) + 1 for a in range(D)], len(idx)


@pytest.mark.parametrize("D", [2, 3])
def test_regrid_box_rule_matches_oracle(D):
    E.load(build_if_missing=True)
    rng = np.random.default_rng(11 + D)
    for trial in range(200):
        n = [int(v) for v in rng.choice([8, 12, 16, 24, 32], size=D)] + [1] * (3 - D)
        ncell = int(np.prod(n))
        tag = np.zeros(ncell, np.uint8)
        k = int(rng.integers(0, 4))
        if k:
            c = rng.integers(0, ncell, size=k)
            tag[c] = TG.REFINE
        live = np.ones(ncell, bool)
        cflo = [bool(v) for v in rng.integers(0, 2, size=D)]
        cfhi = [bool(v) for v in rng.integers(0, 2, size=D)]
        buf, block = int(rng.integers(0, 4)), int(rng.choice([2, 4]))
        want = TG.regrid_box(tag, live, n, D, cflo, cfhi, buf=buf, block=block)
        if k:
            blo, bhi, nm = _bbox((tag & TG.REFINE) != 0, n, D)
        else:
            blo, bhi, nm = [0] * D, [0] * D, 0
        got = E.regrid_box(D, n, [int(v) for v in cflo], [int(v) for v in cfhi], blo, bhi, nm, buf, block)
        assert got == want, (trial, n, cflo, cfhi, buf, block, blo, bhi)


def test_setup_levels_refuses_bad_boxes_before_device_work():
    lib = E.load(build_if_missing=True)
    d, keep = E.make_desc(W.rod_plane_2d(32))
    o = E.eb_solver_opts_default()
    h = ctypes.c_void_p()

    def setup(boxes):
        lo = (ctypes.c_int * (3 * len(boxes)))(*[v for b in boxes for v in b[0]])
        hi = (ctypes.c_int * (3 * len(boxes)))(*[v for b in boxes for v in b[1]])
        return lib.eb_amr_setup_levels(ctypes.byref(d), len(boxes) + 1, lo, hi, ctypes.byref(o), None,
                                       ctypes.byref(h))
    # level 2 touching the low-x CF side of level 1
    assert setup([([8, 8, 0], [24, 24, 1]), ([0, 8, 0], [16, 24, 1])]) == E.EB_ERR_INVALID
    assert b"coarse-fine side" in lib.eb_last_error()
    # a box side that is not a multiple of 4 parent cells
    assert setup([([8, 8, 0], [22, 24, 1])]) == E.EB_ERR_INVALID
    # too many levels
    assert setup([([8, 8, 0], [24, 24, 1])] * 4) == E.EB_ERR_INVALID


def test_regrid_driver_grows_boxes_to_their_limits():
    from paper_1809_03745_gb300 import regrid as R
    # CF sides in x (limits 4 and n - 4), domain sides in y (limits 0 and n)
    box = ([8, 2], [20, 30])
    assert R._grow(box, [32, 32], [1, 0], [1, 0], 2, 4) == ([4, 0], [24, 32])
    assert R._grow(([4, 0], [28, 32]), [32, 32], [1, 0], [1, 0], 2, 4) is None


def test_tag_and_box_calls_refuse_bad_arguments_without_device_work():
    lib = E.load(build_if_missing=True)
    eps = (ctypes.c_double * 4)(0.1, 0.8, 0.1, 0.2)
    lo, hi = (ctypes.c_int * 3)(), (ctypes.c_int * 3)()
    nm, em = ctypes.c_longlong(), ctypes.c_double()
    assert lib.eb_tag_cells(None, None, eps, None, None, None, lo, hi, ctypes.byref(nm), ctypes.byref(em),
                            None) == E.EB_ERR_INVALID
    i3 = lambda *v: (ctypes.c_int * 3)(*v)  # noqa: E731
    has = ctypes.c_int()
    assert lib.eb_regrid_box(2, i3(32, 32, 1), i3(0, 0, 0), i3(0, 0, 0), i3(1, 1, 0), i3(2, 2, 1), 1, 2, 0,
                             lo, hi, ctypes.byref(has)) == E.EB_ERR_INVALID  # block < 1
    assert lib.eb_regrid_box(4, i3(32, 32, 1), i3(0, 0, 0), i3(0, 0, 0), i3(1, 1, 0), i3(2, 2, 1), 1, 2, 4,
                             lo, hi, ctypes.byref(has)) == E.EB_ERR_INVALID  # dim


def test_keep_rule_needs_every_coarser_box_unchanged():
    from paper_1809_03745_gb300 import regrid as R
    a = [([8, 8], [24, 24]), ([4, 4], [20, 28])]
    assert R.same_boxes(a[:1], [([8, 8], [24, 24])])
    assert R.same_boxes(a, [((8, 8), (24, 24)), ((4, 4), (20, 28))])
    assert not R.same_boxes(a, [([8, 8], [24, 28]), ([4, 4], [20, 28])])  # level 1 moved: level 2's grid differs
    assert not R.same_boxes(a, a[:1])

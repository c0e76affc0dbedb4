"""GPU parity of the TGA implicit diffusion step (row f2; Sec. 3.4, Eq. tga).

`eb_tga_step` through the C ABI (a stepper over three solver handles with
shifts 0, 1/mu1, 1/mu2; the right-hand sides formed on the device) against the oracle's step
(oracle/tga.py, its own operator and sparse solves): one step to 1e-9
relative, several steps in 3D to 1e-8, exact conservation of sum(kappa phi)
on a box with Neumann walls, and geometries whose shifts or grids do not
match are rejected.
"""
import numpy as np
import pytest
import torch

from oracle import tga as OT
from paper_1809_03745_gb300 import workloads as W

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1809_03745_gb300 import ebpoisson as E


def _inputs(d, seed):
    x, y, z = W.cell_centres(d)
    rng = np.random.default_rng(seed)
    phi = np.stack([np.sin(3 * x) * np.cos(2 * y) + 0.1 * rng.normal(size=x.size), 0.5 * np.cos(x + z)])
    rho = np.stack([40.0 * np.exp(-((x - 0.5) ** 2 + (y - 0.45) ** 2 + (z - 0.4) ** 2) / 0.01), np.sin(4 * y)])
    return phi, rho


def _oracle_steps(d, phi, rho, dt, steps):
    D = OT.Diffusion(d)
    p = D.g.to_dofs(phi)
    r = D.g.to_dofs(rho)
    for _ in range(steps):
        p = D.step(p, r, dt)
    return D.g.to_cells(p), D


@pytest.mark.parametrize("dt", [1e-3, 0.1])
def test_tga_step_matches_oracle_2d_two_phase(dt):
    d = W.rod_plane_2d(64, dielectric=True)
    phi, rho = _inputs(d, 3)
    want, D = _oracle_steps(d, phi, rho, dt, 1)
    T = E.TGA(d, dt, tol=1e-12)
    got, infos = T.step(torch.from_numpy(phi).cuda(), torch.from_numpy(rho).cuda())
    got = got.cpu().numpy()
    assert all(i["status"] == 0 for i in infos), infos
    assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()
    for p in range(2):
        assert np.all(got[p][D.g.dof[p] < 0] == 0.0)


def test_tga_steps_match_oracle_3d():
    d = W.pin_plane_3d(32)
    phi, rho = _inputs(d, 5)
    want, _ = _oracle_steps(d, phi, rho, 0.01, 5)
    T = E.TGA(d, 0.01, tol=1e-12)
    cur = torch.from_numpy(phi).cuda()
    r = torch.from_numpy(rho).cuda()
    for _ in range(5):
        cur, infos = T.step(cur, r)
        assert all(i["status"] == 0 for i in infos), infos
    got = cur.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-8 * np.abs(want).max()


def test_tga_step_conserves_on_device():
    d = W._desc(2, (96, 96), (0, 0), 1.0 / 96, [(W.PRIM_SPHERE, [0.46, 0.53, 0.0, 0.23])], [(0, 0, 0)], -1, 0,
                (1.0, 3.0), [0, 0, 0, 0, 0, 0], 0.0, [0.0] * 6)
    phi, rho = _inputs(d, 7)
    T = E.TGA(d, 0.05, tol=1e-12)
    kap = T.geom.export()["kappa"].cpu().numpy()
    phi = phi * (kap > 0)
    rho = rho * (kap > 0)
    got, _ = T.step(torch.from_numpy(phi).cuda(), torch.from_numpy(rho).cuda())
    gain = (kap * got.cpu().numpy()).sum() - (kap * phi).sum()
    want = 0.05 * (kap * rho).sum()
    assert abs(gain - want) <= 1e-9 * (np.abs(kap * phi).sum() + 0.05 * np.abs(kap * rho).sum())


def test_tga_rejects_handles_of_another_dt():
    d = W.rod_plane_2d(32)
    T = E.TGA(d, 0.01)
    gh = [P.geom._h for P in T.handles]
    ph = [P._h for P in T.handles]
    with pytest.raises(E.EBError) as ei:
        E.eb_tga_create(*gh, *ph, 0.02)
    assert ei.value.status == E.EB_ERR_INVALID
    # the shifted geometries in the wrong order
    with pytest.raises(E.EBError) as ei:
        E.eb_tga_create(gh[0], gh[2], gh[1], ph[0], ph[2], ph[1], 0.01)
    assert ei.value.status == E.EB_ERR_INVALID
    # another grid
    other = E.Geometry(W.rod_plane_2d(16))
    with pytest.raises(E.EBError) as ei:
        E.eb_tga_create(other._h, gh[1], gh[2], ph[0], ph[1], ph[2], 0.01)
    assert ei.value.status == E.EB_ERR_INVALID


def test_diffusion_driver_runs_and_absorbs():
    """The timed driver on the absorbing rod-plane: both stages converge, and
    the solid takes a share of the seed and source in (0, 1)."""
    from paper_1809_03745_gb300 import diffusion
    res = diffusion.run(dim=2, n=64, r=10.0, steps=3)
    assert len(res["rows"]) == 3 and all(min(r["vcycles"]) >= 1 for r in res["rows"])
    assert 0.0 < res["absorbed"] < 1.0

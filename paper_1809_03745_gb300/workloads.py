"""Seeded synthetic workloads: geometry descriptions and input fields.

This module only *describes* problems (primitives, CSG trees, boundary
conditions) and draws seeded random inputs sampled at cell centres.  It holds
none of the discretisation's arithmetic and imports neither the CUDA binding
nor the oracle, so both sides can take the same inputs from it.

Problem description format (a plain dict):
    dim            2 or 3
    n              cells per axis (3 ints; n[2] = 1 in 2D)
    lo, h          lower domain corner and the (isotropic) cell size
    prims          list of (kind, params) -- see PRIM_* below
    nodes          list of (op, a, b) CSG nodes, children before parents
    root_E         CSG node whose negative set is the union of all electrodes (-1: none)
    electrodes     list of (root, V): each electrode's own CSG node and potential; a
                   cut cell takes the V of the electrode whose implicit function is
                   smallest at its EB centroid.  Default [(root_E, phi_E)].
    root_D         CSG node whose negative set is the dielectric (-1: none)
    eps            (eps_gas, eps_dielectric), relative permittivities
    bc             6 ints per wall xlo,xhi,ylo,yhi,zlo,zhi: 0 Neumann, 1 Dirichlet
    phi_E          electrode potential
    phi_wall       6 floats, Dirichlet value per wall

Workloads follow the paper's examples: the rod/pin-plane electrode of
Sec. 4.4 and 6.2, the rough dielectric surface of Sec. 6.1 and the coaxial
multi-fluid problem of Sec. 4.2.  Seeds: base 1809, config k uses 1809 + k.
"""
from __future__ import annotations

import math

import numpy as np

# primitive kinds (parameters in brackets; every implicit function is negative inside)
PRIM_SPHERE = 0     # [cx, cy, cz, r]                      |x - c| - r
PRIM_CAPSULE = 1    # [ax, ay, az, bx, by, bz, r]          dist(x, segment ab) - r
PRIM_HALFSPACE = 2  # [nx, ny, nz, d]                      n.x - d
PRIM_SINE = 3       # [up, c, A, k, ph, t]                 x[up] - (c + A sin(2 pi k x[t] + ph))
PRIM_CYLINDER = 4   # [axis, px, py, pz, r, lo, hi]        max(dist_to_axis - r, lo - x[axis], x[axis] - hi)
PRIM_BOX = 5        # [lox, loy, loz, hix, hiy, hiz]       max_k max(lo_k - x_k, x_k - hi_k)

CSG_PRIM, CSG_UNION, CSG_INTERSECT, CSG_NEGATE = 0, 1, 2, 3

NEUMANN, DIRICHLET, ROBIN = 0, 1, 2
SEED_BASE = 1809

# Three-group photoionisation model for oxygen (the paper's photoionisation
# table): per group lambda_gamma and A_gamma in 1/(m Pa); kappa_gamma =
# lambda_gamma p_O2 / sqrt(3) with p_O2 = 0.2 bar; S_ph = nu_eff p_O2 sum
# A_gamma Psi_gamma with nu_eff = 0.1.
PHOTO_GROUPS = ((4.15e-2, 1.12e-4), (1.09e-1, 2.88e-3), (6.69e-1, 2.76e-1))
PHOTO_P_O2 = 2.0e4
PHOTO_NU_EFF = 0.1


def _desc(dim, n, lo, h, prims, nodes, root_E, root_D, eps, bc, phi_E, phi_wall, electrodes=None):
    n = list(n) + [1] * (3 - len(n))
    lo = list(lo) + [0.0] * (3 - len(lo))
    if electrodes is None:
        electrodes = [(root_E, phi_E)] if root_E >= 0 else []
    return dict(dim=dim, n=tuple(int(v) for v in n), lo=tuple(float(v) for v in lo), h=float(h),
                prims=[(int(k), [float(v) for v in p]) for k, p in prims],
                nodes=[tuple(int(v) for v in q) for q in nodes], root_E=int(root_E), root_D=int(root_D),
                eps=(float(eps[0]), float(eps[1])), bc=[int(v) for v in bc], phi_E=float(phi_E),
                phi_wall=[float(v) for v in phi_wall],
                electrodes=[(int(r), float(v)) for r, v in electrodes])


def cell_centres(desc):
    n, lo, h = desc["n"], desc["lo"], desc["h"]
    if desc["dim"] == 2:
        j, i = np.meshgrid(np.arange(n[1]), np.arange(n[0]), indexing="ij")
        x = lo[0] + (i.reshape(-1) + 0.5) * h
        y = lo[1] + (j.reshape(-1) + 0.5) * h
        return x, y, np.zeros_like(x)
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    x = lo[0] + (i.reshape(-1) + 0.5) * h
    y = lo[1] + (j.reshape(-1) + 0.5) * h
    z = lo[2] + (k.reshape(-1) + 0.5) * h
    return x, y, z


def ncells(desc):
    n = desc["n"]
    return int(n[0]) * int(n[1]) * (int(n[2]) if desc["dim"] == 3 else 1)


# --------------------------------------------------------------- 2D workloads

def rod_plane_2d(n=128, *, dielectric=False, tip_y=0.5, half_width=0.05, V=1.0, eps_d=4.0,
                 slab_y=0.2, rough_amp=0.005, rough_periods=20.0, all_dirichlet=False):
    """Rod electrode with a hemispherical tip over a grounded plane on [0,1]^2.

    The rod is a capsule on the axis x = 0.5 whose apex is at y = tip_y, running
    out through the top wall.  Walls: y = 0 grounded, y = 1 at the rod voltage
    V, x = 0, 1 homogeneous Neumann.  With ``dielectric`` a slab of
    eps_r = eps_d fills y < slab_y + rough_amp sin(2 pi rough_periods x).
    """
    h = 1.0 / n
    prims = [(PRIM_CAPSULE, [0.5, tip_y + half_width, 0.0, 0.5, 2.0, 0.0, half_width])]
    nodes = [(CSG_PRIM, 0, 0)]
    root_E, root_D = 0, -1
    if dielectric:
        prims.append((PRIM_SINE, [1, slab_y, rough_amp, rough_periods, 0.0, 0]))
        nodes.append((CSG_PRIM, 1, 0))
        root_D = 1
    bc = [NEUMANN, NEUMANN, DIRICHLET, DIRICHLET, NEUMANN, NEUMANN]
    if all_dirichlet:
        bc = [DIRICHLET] * 4 + [NEUMANN] * 2
    return _desc(2, (n, n), (0.0, 0.0), h, prims, nodes, root_E, root_D, (1.0, eps_d), bc, V,
                 [0.0, 0.0, 0.0, V, 0.0, 0.0])


def c1_inputs(n=128, seed=SEED_BASE + 1, noise=1e-3):
    """Rod-plane, vacuum, Gaussian blob of peak 100 and width 0.03 centred 0.05
    below the tip, plus seeded uniform noise of amplitude ``noise``."""
    desc = rod_plane_2d(n)
    x, y, _ = cell_centres(desc)
    rng = np.random.Generator(np.random.PCG64(seed))
    s = 100.0 * np.exp(-((x - 0.5) ** 2 + (y - 0.45) ** 2) / (2 * 0.03 ** 2))
    if noise:
        s = s + rng.uniform(-noise, noise, size=s.shape)
    S = np.zeros((2, s.size))
    S[0] = s
    return desc, S, np.zeros(s.size)


def c2_inputs(n=1024, seed=SEED_BASE + 2, peak=100.0):
    """Rod-plane over a rough dielectric slab (eps_r = 4, y < 0.2 + 0.005 sin(40 pi x)),
    seeded surface charge sigma/eps0 ~ U(-1, 1) per cell (read on interface cells),
    and a Gaussian space-charge filament of radius 0.02 on the axis from
    y = 0.2 to the tip at y = 0.5, with Gaussian caps beyond."""
    desc = rod_plane_2d(n, dielectric=True)
    x, y, _ = cell_centres(desc)
    rng = np.random.Generator(np.random.PCG64(seed))
    r = 0.02
    dy = np.where(y < 0.2, 0.2 - y, np.where(y > 0.5, y - 0.5, 0.0))
    s = peak * np.exp(-(x - 0.5) ** 2 / (2 * r * r)) * np.exp(-dy ** 2 / (2 * r * r))
    S = np.zeros((2, s.size))
    S[0] = s
    sigma = rng.uniform(-1.0, 1.0, size=s.size)
    return desc, S, sigma


def coaxial_2d(n=256, *, R0=0.3, R1=0.6, R2=0.9, eps=4.0, phi0=1.0):
    """The multi-fluid coaxial problem of Sec. 4.2 on (-1,1)^2: inner electrode
    r < R0 at phi0, outer electrode r > R2 grounded, dielectric R0 < r < R1."""
    h = 2.0 / n
    prims = [(PRIM_SPHERE, [0.0, 0.0, 0.0, R0]), (PRIM_SPHERE, [0.0, 0.0, 0.0, R2]),
             (PRIM_SPHERE, [0.0, 0.0, 0.0, R1])]
    # electrode = inner disk U complement of outer disk
    nodes = [(CSG_PRIM, 0, 0), (CSG_PRIM, 1, 0), (CSG_NEGATE, 1, 0), (CSG_UNION, 0, 2), (CSG_PRIM, 2, 0)]
    bc = [DIRICHLET] * 4 + [NEUMANN] * 2
    return _desc(2, (n, n), (-1.0, -1.0), h, prims, nodes, 3, 4, (1.0, eps), bc, phi0, [0.0] * 6,
                 electrodes=[(0, phi0), (2, 0.0)])


def coaxial_exact(r, *, R0=0.3, R1=0.6, R2=0.9, eps_g=1.0, eps_d=4.0, phi0=1.0, sigma=0.0):
    """Closed form of the coaxial problem (Sec. 4.2, Eq. poisson_coaxial_exact),
    with an optional uniform surface charge sigma/eps0 on r = R1.  Returns the
    gas-phase and dielectric-phase expressions, each continued past R1."""
    cg = (phi0 + sigma * R1 / eps_d * math.log(R1 / R0)) / (math.log(R1 / R2) / eps_g - math.log(R1 / R0) / eps_d)
    cd = cg + sigma * R1
    phi_g = cg / eps_g * np.log(r / R2)
    phi_d = phi0 + cd / eps_d * np.log(r / R0)
    return phi_g, phi_d


def fluid_wedge(dim=2, n=32, *, half=0.6, angle=1.3, apex=(0.3123, 0.4571, 0.5213), tilt=0.0, V=1.0):
    """An acute fluid wedge cut out of a planar electrode: the electrode is the
    union of two half-spaces whose boundary planes meet at `apex`, making
    angles angle +- half with the x axis (in 3D both planes are tilted by
    +-tilt out of the z axis).  Near the apex neither ray stencil of the EB
    normal derivative finds its cells in the fluid, so the least-squares
    fallback (Sec. 3.3.1) is used there.  Electrode at V, walls Dirichlet 0."""
    h = 1.0 / n
    a1, a2 = angle + half, angle - half
    n1 = np.array([math.sin(a1), -math.cos(a1), 0.0])
    n2 = np.array([-math.sin(a2), math.cos(a2), 0.0])
    if dim == 3:
        n1[2], n2[2] = tilt, -tilt
        n1 /= np.linalg.norm(n1)
        n2 /= np.linalg.norm(n2)
    p = np.array(list(apex[:dim]) + [0.5] * (3 - dim))
    prims = [(PRIM_HALFSPACE, [n1[0], n1[1], n1[2], float(n1 @ p)]),
             (PRIM_HALFSPACE, [n2[0], n2[1], n2[2], float(n2 @ p)])]
    nodes = [(CSG_PRIM, 0, 0), (CSG_PRIM, 1, 0), (CSG_UNION, 0, 1)]
    bc = [DIRICHLET] * 4 + ([NEUMANN] * 2 if dim == 2 else [DIRICHLET] * 2)
    return _desc(dim, (n,) * dim, (0.0,) * dim, h, prims, nodes, 2, -1, (1.0, 1.0), bc, V, [0.0] * 6)


# --------------------------------------------------------------- 3D workloads

def pin_plane_3d(n=256, *, tip_z=0.5, radius=0.02, V=1.0, disk=True, eps_d=3.0, disk_r=0.3, disk_t=0.05):
    """Cylindrical pin with a hemispherical tip above a grounded plane on [0,1]^3,
    with an optional dielectric disk of eps_r = eps_d on the plane (Sec. 6.2)."""
    h = 1.0 / n
    prims = [(PRIM_CAPSULE, [0.5, 0.5, tip_z + radius, 0.5, 0.5, 2.0, radius])]
    nodes = [(CSG_PRIM, 0, 0)]
    root_D = -1
    if disk:
        prims.append((PRIM_CYLINDER, [2, 0.5, 0.5, 0.0, disk_r, -1.0, disk_t]))
        nodes.append((CSG_PRIM, 1, 0))
        root_D = 1
    bc = [NEUMANN, NEUMANN, NEUMANN, NEUMANN, DIRICHLET, DIRICHLET]
    return _desc(3, (n, n, n), (0.0, 0.0, 0.0), h, prims, nodes, 0, root_D, (1.0, eps_d), bc, V,
                 [0.0, 0.0, 0.0, 0.0, 0.0, V])


def line_charge(x, y, z, peak=1e3):
    """Gaussian line charge of radius 0.02 along the pin axis for z in [0.05, 0.5]."""
    r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2
    dz = np.where(z < 0.05, 0.05 - z, np.where(z > 0.5, z - 0.5, 0.0))
    return peak * np.exp(-r2 / (2 * 0.02 ** 2)) * np.exp(-dz ** 2 / (2 * 0.02 ** 2))


def c3_inputs(n=256, seed=SEED_BASE + 3, peak=1e3):
    desc = pin_plane_3d(n)
    x, y, z = cell_centres(desc)
    s = line_charge(x, y, z, peak)
    S = np.zeros((2, s.size))
    S[0] = s
    return desc, S, np.zeros(s.size)


def refined_box_desc(desc, box_lo, box_hi):
    """The fine grid of a ratio-2 box over coarse cells [box_lo, box_hi) (for cell centres)."""
    D = desc["dim"]
    n = [2 * (box_hi[k] - box_lo[k]) if k < D else 1 for k in range(3)]
    lo = [desc["lo"][k] + box_lo[k] * desc["h"] if k < D else 0.0 for k in range(3)]
    return dict(desc, n=tuple(n), lo=tuple(lo), h=desc["h"] / 2.0)


def c3_amr_inputs(n=256, peak=1e3, box_frac=(0.375, 0.625)):
    """The 3D pin-plane workload with a ratio-2 refined box around the tip:
    coarse cells [3n/8, 5n/8)^3 (physical [0.375, 0.625]^3), so 256^3 + 128^3.
    Returns (desc, box_lo, box_hi, S_c, sig_c, S_f, sig_f)."""
    desc = pin_plane_3d(n)
    lo = [int(round(box_frac[0] * n))] * 3
    hi = [int(round(box_frac[1] * n))] * 3
    x, y, z = cell_centres(desc)
    Sc = np.zeros((2, x.size))
    Sc[0] = line_charge(x, y, z, peak)
    xf, yf, zf = cell_centres(refined_box_desc(desc, lo, hi))
    Sf = np.zeros((2, xf.size))
    Sf[0] = line_charge(xf, yf, zf, peak)
    return desc, lo, hi, Sc, np.zeros(x.size), Sf, np.zeros(xf.size)


# --------------------------------------------------------------- batched instances

def batched_instances(count=64, seed=SEED_BASE + 4, *, n2=(64, 1024), n3=(32, 192), p3d=0.5, max_cells=None):
    """Independent solves with seeded geometry and sizes: 2D or 3D by a
    Bernoulli draw, n log-uniform in the given range rounded to a multiple of
    16, tip radius U[0.01, 0.05] clamped to >= 3h, gap U[0.3, 0.7], eps_r
    U[2, 8] for a dielectric slab (2D, thickness 0.1) or disk (3D, radius 0.3,
    thickness 0.05), each kept at least three cells thick, voltage U[0.5, 2]
    and a Gaussian blob of peak log-U[10, 1e3] 0.05 below the apex."""
    root = np.random.SeedSequence(seed)
    out = []
    for child in root.spawn(count):
        rng = np.random.Generator(np.random.PCG64(child))
        is3d = rng.uniform() < p3d
        lo_n, hi_n = n3 if is3d else n2
        n = int(round(math.exp(rng.uniform(math.log(lo_n), math.log(hi_n))) / 16.0)) * 16
        n = max(16, n)
        if max_cells is not None:
            while n ** (3 if is3d else 2) > max_cells and n > 16:
                n -= 16
        h = 1.0 / n
        tip_r = max(rng.uniform(0.01, 0.05), 3 * h)
        gap = rng.uniform(0.3, 0.7)
        eps_d = rng.uniform(2.0, 8.0)
        V = rng.uniform(0.5, 2.0)
        peak = math.exp(rng.uniform(math.log(10.0), math.log(1e3)))
        if is3d:
            # a disk at least three cells thick, its top off the node planes
            desc = pin_plane_3d(n, tip_z=gap, radius=tip_r, V=V, eps_d=eps_d,
                                disk_t=max(min(0.05, gap - 10 * h), 3 * h) + 0.3 * h)
            x, y, z = cell_centres(desc)
            s = peak * np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - (gap - 0.05)) ** 2) / (2 * 0.03 ** 2))
        else:
            slab = max(min(0.1, gap - 10 * h), 3 * h) + 0.3 * h  # >= 3 cells, top off the node rows
            desc = rod_plane_2d(n, dielectric=True, tip_y=gap, half_width=tip_r, V=V, eps_d=eps_d, slab_y=slab,
                                rough_amp=0.0)
            x, y, _ = cell_centres(desc)
            s = peak * np.exp(-((x - 0.5) ** 2 + (y - (gap - 0.05)) ** 2) / (2 * 0.03 ** 2))
        S = np.zeros((2, s.size))
        S[0] = s
        out.append((desc, S, np.zeros(s.size)))
    return out


def photo_kappa(group):
    """kappa_gamma [1/m] of photoionisation group 0, 1 or 2."""
    return PHOTO_GROUPS[group][0] * PHOTO_P_O2 / math.sqrt(3.0)


def rte_desc(dim, n, kappa_L):
    """One Eddington (SP1) photon group in the stationary form of Sec. 2.3 on
    the rod-plane (2D) or pin-plane (3D) geometry scaled to the unit box:
    kappa Psi - div(grad Psi / (3 kappa)) = eta / c becomes, per unit length
    L of the box and after a factor 3 kappa L^2, lam Psi - lap Psi = s with
    lam = 3 (kappa L)^2 (eps = 1).  Photons leave through every boundary of
    the gas: the walls, the electrode and the dielectric (merged with the
    electrode into one solid here), with the outflow condition dPsi/dn + 3
    kappa / 2 Psi = 0, i.e. Robin a1 = 1.5 kappa L, a2 = 1, a3 = 0."""
    if dim == 2:
        d = rod_plane_2d(n, dielectric=True)
    else:
        d = pin_plane_3d(n)
    # the electrode and the dielectric as one solid: union of the two primitives
    d["nodes"] = list(d["nodes"]) + [(CSG_UNION, 0, 1)]
    d["root_E"], d["root_D"] = len(d["nodes"]) - 1, -1
    d["electrodes"] = [(d["root_E"], 0.0)]
    d["phi_E"] = 0.0
    d["eps"] = (1.0, 1.0)
    a1 = 1.5 * kappa_L
    d["bc"] = [ROBIN] * (2 * dim) + [NEUMANN] * (6 - 2 * dim)
    d["robin"] = [(a1, 1.0)] * 6
    d["phi_wall"] = [0.0] * 6
    d["eb_robin"] = (a1, 1.0)
    d["lam"] = (3.0 * kappa_L ** 2, 0.0)
    return d


def photo_inputs(dim, n, L=0.02, peak=1.0):
    """The three photon groups on an L-sized box: per group (desc, S, sigma)
    with the source s = 3 kappa L^2 eta / c of a Gaussian emission region of
    width 0.03 below the tip (peak eta / c = peak), and the weights w_gamma =
    nu_eff p_O2 A_gamma of S_ph = sum w_gamma Psi_gamma."""
    out, w = [], []
    for gi in range(3):
        kap = photo_kappa(gi)
        d = rte_desc(dim, n, kap * L)
        x, y, z = cell_centres(d)
        if dim == 2:
            eta = peak * np.exp(-((x - 0.5) ** 2 + (y - 0.42) ** 2) / (2 * 0.03 ** 2))
        else:
            eta = peak * np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.42) ** 2) / (2 * 0.03 ** 2))
        S = np.zeros((2, eta.size))
        S[0] = 3.0 * kap * L * L * eta
        out.append((d, S, np.zeros(eta.size)))
        w.append(PHOTO_NU_EFF * PHOTO_P_O2 * PHOTO_GROUPS[gi][1])
    return out, w


def diffusion_inputs(dim, n, peak=1.0):
    """A species diffusing in the gas of the rod-plane (2D) or pin-plane (3D)
    geometry, the diffusion part of the drift-diffusion step of Sec. 3.4 in a
    unit box with eps = D = 1: the electrode and the dielectric as one
    absorbing solid (homogeneous Dirichlet on its surface), no flux through the
    walls.  Returns (desc, phi0, rho): a Gaussian seed of width 0.03 below the
    tip and a Gaussian source of width 0.05 around it, [2][n_cells] each (the
    solid's phase 1 is empty)."""
    d = rod_plane_2d(n, dielectric=True) if dim == 2 else pin_plane_3d(n)
    d["nodes"] = list(d["nodes"]) + [(CSG_UNION, 0, 1)]
    d["root_E"], d["root_D"] = len(d["nodes"]) - 1, -1
    d["electrodes"] = [(d["root_E"], 0.0)]
    d["phi_E"] = 0.0
    d["eps"] = (1.0, 1.0)
    d["bc"] = [NEUMANN] * 6
    d["phi_wall"] = [0.0] * 6
    x, y, z = cell_centres(d)
    r2 = (x - 0.5) ** 2 + ((y - 0.42) ** 2 + z ** 2 if dim == 2 else (y - 0.5) ** 2 + (z - 0.42) ** 2)
    phi = np.zeros((2, x.size))
    rho = np.zeros((2, x.size))
    phi[0] = peak * np.exp(-r2 / (2 * 0.03 ** 2))
    rho[0] = 10.0 * peak * np.exp(-r2 / (2 * 0.05 ** 2))
    return d, phi, rho

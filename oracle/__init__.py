"""Plain FP64 CPU oracle for the EB multi-material Poisson discretisation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
product path (``paper_1809_03745_gb300``) never imports it and shares no code
with it.

The arithmetic lives in ``eb_oracle.c`` (geometry, stencils, assembly, field);
this module compiles it with gcc, marshals a problem description into it, and
solves the assembled sparse system with SciPy's sparse LU (a library routine
used as one step, Sec. 3.3.2 only asks for *a* solution of L(phi) = rho).

Problem description (a plain dict, the same one the CUDA binding accepts):
    dim, n (3 ints), lo (3 floats), h,
    prims: list of (kind, params[<=10]), nodes: list of (op, a, b),
    root_E, root_D (-1 = none), eps (gas, dielectric), bc (6 ints, 0 Neumann
    1 Dirichlet, 2 Robin per side xlo,xhi,ylo,yhi,zlo,zhi), phi_E, phi_wall (6 floats).
Helmholtz and Robin (optional keys): lam (2 floats, the shift alpha a per phase),
    robin (6 pairs a1, a2 for the Robin sides; phi_wall then holds a3), eb_robin
    (a pair a1, a2: electrodes carry a1 phi + a2 dphi/dn = a3 with phi_E as a3).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eb_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libeb_oracle.so")
_lock = threading.Lock()
_lib = None

OK, INVALID, UNSUPPORTED = 0, 1, 6
EB_NONE, EB_ELECTRODE, EB_INTERFACE = 0, 1, 2


def build(force: bool = False, plant: int = 0) -> str:
    """Compile the oracle into oracle/_build/libeb_oracle.so (gcc, no FMA contraction).
    plant = k > 0 builds the variant with planted mistake k (see eb_oracle.c) into
    its own library, for the tests that show the pins catch it."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    lib = _LIB if plant == 0 else os.path.join(_LIB_DIR, f"libeb_oracle_plant{int(plant)}.so")
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               f"-DOR_PLANT={int(plant)}", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, lib)
    return lib


class _Desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("h", C.c_double),
                ("n_prims", C.c_int), ("prim_kind", C.POINTER(C.c_int)), ("prim_par", C.POINTER(C.c_double)),
                ("n_nodes", C.c_int), ("node_op", C.POINTER(C.c_int)), ("node_a", C.POINTER(C.c_int)),
                ("node_b", C.POINTER(C.c_int)), ("root_E", C.c_int), ("root_D", C.c_int),
                ("eps", C.c_double * 2), ("bc", C.c_int * 6), ("robin", C.c_double * 12),
                ("eb_robin", C.c_int), ("eb_robin_a", C.c_double * 2), ("lam", C.c_double * 2)]


class _Data(C.Structure):
    _fields_ = [("phiE", C.POINTER(C.c_double)), ("sigma", C.POINTER(C.c_double)),
                ("phidom", C.POINTER(C.c_double)), ("s", C.POINTER(C.c_double))]


def planted(k: int):
    """The oracle library with planted mistake k, bound like the real one (tests only)."""
    return _bind(C.CDLL(build(plant=k)))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(C.CDLL(build()))
    return _lib


def _bind(lib):
    P = C.c_void_p
    lib.or_geom_build.restype = P
    lib.or_geom_build.argtypes = [C.POINTER(_Desc), C.POINTER(C.c_int)]
    lib.or_geom_free.argtypes = [P]
    for name in ("or_ndof", "or_ncell", "or_n_eb", "or_wall_total", "or_bad_cell"):
        getattr(lib, name).restype = C.c_long
        getattr(lib, name).argtypes = [P]
    lib.or_status.restype = C.c_int
    lib.or_status.argtypes = [P]
    lib.or_nface.restype = C.c_long
    lib.or_nface.argtypes = [P, C.c_int]
    lib.or_counts.argtypes = [P, C.c_void_p]
    lib.or_cells.argtypes = [P] + [C.c_void_p] * 7
    lib.or_faces.argtypes = [P, C.c_int, C.c_void_p, C.c_void_p]
    lib.or_labels.argtypes = [P, C.c_void_p]
    lib.or_stencil_order.argtypes = [P, C.c_void_p]
    lib.or_assemble.restype = C.c_long
    lib.or_assemble.argtypes = [P, C.POINTER(_Data), C.c_void_p, C.c_void_p, C.c_void_p, C.c_long,
                                C.c_void_p]
    lib.or_boundary_flux.restype = C.c_double
    lib.or_boundary_flux.argtypes = [P, C.POINTER(_Data), C.c_void_p]
    lib.or_field.argtypes = [P, C.POINTER(_Data), C.c_void_p, C.c_void_p, C.c_void_p]
    lib.or_boundary_flux_masked.restype = C.c_double
    lib.or_boundary_flux_masked.argtypes = [P, C.POINTER(_Data), C.c_void_p, C.c_void_p]
    lib.or_face_flux.restype = C.c_long
    lib.or_face_flux.argtypes = [P, C.POINTER(_Data), C.c_int, C.c_void_p, C.c_int, C.c_void_p,
                                 C.c_void_p, C.c_void_p]
    lib.or_eval_implicit.restype = C.c_double
    lib.or_eval_implicit.argtypes = [C.POINTER(_Desc), C.c_int, C.c_void_p]
    return lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, status, cell=-1):
        super().__init__(f"oracle geometry status {status} at cell {cell}")
        self.status = status
        self.cell = cell


class Geometry:
    """Cut-cell geometry, dofs and EB stencils of one problem (Sec. 3.1, 3.3.1)."""

    def __init__(self, desc: dict):
        lib = self._lib = _load()  # kept: the geometry lives in this library's memory
        self.desc = desc
        self.dim = int(desc["dim"])
        n = list(desc["n"]) + [1] * (3 - len(desc["n"]))
        if self.dim == 2:
            n[2] = 1
        self.n = tuple(int(v) for v in n)
        self.h = float(desc["h"])
        self.lo = tuple(float(v) for v in (list(desc["lo"]) + [0.0] * (3 - len(desc["lo"]))))
        prims = desc.get("prims", [])
        nodes = desc.get("nodes", [])
        self._kind = np.array([p[0] for p in prims] or [0], dtype=np.int32)
        par = np.zeros((max(len(prims), 1), 10))
        for i, p in enumerate(prims):
            par[i, :len(p[1])] = p[1]
        self._par = np.ascontiguousarray(par.reshape(-1))
        self._op = np.array([q[0] for q in nodes] or [0], dtype=np.int32)
        self._a = np.array([q[1] for q in nodes] or [0], dtype=np.int32)
        self._b = np.array([q[2] for q in nodes] or [0], dtype=np.int32)
        d = _Desc()
        d.dim = self.dim
        for k in range(3):
            d.n[k] = self.n[k]
            d.lo[k] = self.lo[k]
        d.h = self.h
        d.n_prims = len(prims)
        d.prim_kind = self._kind.ctypes.data_as(C.POINTER(C.c_int))
        d.prim_par = self._par.ctypes.data_as(C.POINTER(C.c_double))
        d.n_nodes = len(nodes)
        d.node_op = self._op.ctypes.data_as(C.POINTER(C.c_int))
        d.node_a = self._a.ctypes.data_as(C.POINTER(C.c_int))
        d.node_b = self._b.ctypes.data_as(C.POINTER(C.c_int))
        d.root_E = int(desc.get("root_E", -1))
        d.root_D = int(desc.get("root_D", -1))
        eps = desc.get("eps", (1.0, 1.0))
        d.eps[0], d.eps[1] = float(eps[0]), float(eps[1])
        for k in range(6):
            d.bc[k] = int(desc["bc"][k])
        rob = desc.get("robin")
        if rob is not None:
            for k in range(6):
                d.robin[2 * k], d.robin[2 * k + 1] = float(rob[k][0]), float(rob[k][1])
        ebr = desc.get("eb_robin")
        if ebr is not None:
            d.eb_robin = 1
            d.eb_robin_a[0], d.eb_robin_a[1] = float(ebr[0]), float(ebr[1])
        lam = desc.get("lam", (0.0, 0.0))
        d.lam[0], d.lam[1] = float(lam[0]), float(lam[1])
        self._d = d
        st = C.c_int(0)
        self._g = lib.or_geom_build(C.byref(d), C.byref(st))
        if st.value != OK:
            cell = lib.or_bad_cell(self._g)
            lib.or_geom_free(self._g)
            self._g = None
            raise OracleError(st.value, cell)
        self.ncell = lib.or_ncell(self._g)
        self.ndof = lib.or_ndof(self._g)
        self.n_eb = lib.or_n_eb(self._g)
        self.nwall = lib.or_wall_total(self._g)
        nc = self.ncell
        self.cut = np.zeros(nc, np.uint8)
        self.ebkind = np.zeros(nc, np.uint8)
        self.kappa = np.zeros((2, nc))
        self.dof = np.zeros((2, nc), np.int64)
        self.eba = np.zeros(nc)
        self.ebn = np.zeros((nc, 3))
        self.ebx = np.zeros((nc, 3))
        lib.or_cells(self._g, _ptr(self.cut), _ptr(self.ebkind), _ptr(self.kappa), _ptr(self.dof), _ptr(self.eba),
                     _ptr(self.ebn), _ptr(self.ebx))
        cnt = np.zeros(4, np.int64)
        lib.or_counts(self._g, _ptr(cnt))
        self.stencil_counts = {"order2": int(cnt[1]), "order1": int(cnt[2]), "ls": int(cnt[3])}
        self.eb_cells = np.nonzero(self.cut.astype(bool) & ((self.dof[0] >= 0) | (self.dof[1] >= 0)))[0]

    def __del__(self):
        if getattr(self, "_g", None) is not None and getattr(self, "_lib", None) is not None:
            self._lib.or_geom_free(self._g)
            self._g = None

    # -- geometry queries ------------------------------------------------
    def faces(self, a: int):
        """(alpha[2][faces], centroid offsets[2][faces][2]) for faces normal to axis a."""
        nf = self._lib.or_nface(self._g, a)
        al = np.zeros((2, nf))
        fc = np.zeros((2, nf, 2))
        self._lib.or_faces(self._g, a, _ptr(al), _ptr(fc))
        return al, fc

    def labels(self):
        nn = [self.n[k] + 1 if k < self.dim else 1 for k in range(3)]
        lab = np.zeros(nn[0] * nn[1] * nn[2], np.uint8)
        self._lib.or_labels(self._g, _ptr(lab))
        return lab

    def stencil_order(self):
        o = np.zeros((2, self.ncell), np.int32)
        self._lib.or_stencil_order(self._g, _ptr(o))
        return o

    def cell_centres(self):
        idx = np.arange(self.ncell)
        i = idx % self.n[0]
        j = (idx // self.n[0]) % self.n[1]
        k = idx // (self.n[0] * self.n[1])
        x = self.lo[0] + (i + 0.5) * self.h
        y = self.lo[1] + (j + 0.5) * self.h
        z = self.lo[2] + (k + 0.5) * self.h if self.dim == 3 else np.zeros_like(x)
        return x, y, z

    def wall_face_centres(self):
        """Centres of all wall faces in the oracle's wall ordering: list of (side, x, y, z arrays)."""
        out = []
        for a in range(self.dim):
            t = [k for k in range(self.dim) if k != a]
            shape = [self.n[k] for k in t]
            for hi in (0, 1):
                if self.dim == 2:
                    it = np.arange(shape[0])
                    coords = {t[0]: self.lo[t[0]] + (it + 0.5) * self.h}
                else:
                    i0, i1 = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
                    i0 = i0.T.reshape(-1)  # fastest over t[0]
                    i1 = i1.T.reshape(-1)
                    coords = {t[0]: self.lo[t[0]] + (i0 + 0.5) * self.h, t[1]: self.lo[t[1]] + (i1 + 0.5) * self.h}
                m = len(next(iter(coords.values())))
                coords[a] = np.full(m, self.lo[a] + (self.n[a] if hi else 0) * self.h)
                xyz = [coords.get(k, np.zeros(m)) for k in range(3)]
                out.append((2 * a + hi, *xyz))
        return out

    # -- data --------------------------------------------------------------
    def data(self, s=None, sigma=None, phiE=None, phidom=None):
        """Marshal problem data.  s: [2][cell] (or [cell] gas only); sigma: [cell];
        phiE: scalar or [cell]; phidom: [2][nwall] or None (per-side constants)."""
        nc = self.ncell
        S = np.zeros((2, nc))
        if s is not None:
            s = np.asarray(s, dtype=np.float64)
            if s.ndim == 1:
                S[0] = s
            else:
                S[:] = s
        sig = np.zeros(nc) if sigma is None else np.ascontiguousarray(sigma, dtype=np.float64).reshape(nc)
        if phiE is None:
            pe = self.electrode_potential()
        elif np.isscalar(phiE):
            pe = np.full(nc, float(phiE))
        else:
            pe = np.ascontiguousarray(phiE, dtype=np.float64)
        if phidom is None:
            wall = self.desc.get("phi_wall", [0.0] * 6)
            vals = []
            for side, x, _, _ in self.wall_face_centres():
                vals.append(np.full(len(x), float(wall[side])))
            pd1 = np.concatenate(vals)
            pd = np.stack([pd1, pd1])
        else:
            pd = np.asarray(phidom, dtype=np.float64).reshape(2, self.nwall)
        keep = (np.ascontiguousarray(S.reshape(-1)), sig, np.ascontiguousarray(pe),
                np.ascontiguousarray(pd.reshape(-1)))
        dt = _Data()
        dt.s = keep[0].ctypes.data_as(C.POINTER(C.c_double))
        dt.sigma = keep[1].ctypes.data_as(C.POINTER(C.c_double))
        dt.phiE = keep[2].ctypes.data_as(C.POINTER(C.c_double))
        dt.phidom = keep[3].ctypes.data_as(C.POINTER(C.c_double))
        return (dt, keep)

    def electrode_potential(self):
        """Per-cell electrode potential: on electrode cut cells, the V of the electrode
        whose implicit function is smallest at the EB centroid (lowest index on ties)."""
        pe = np.zeros(self.ncell)
        elec = self.desc.get("electrodes")
        if elec is None:
            elec = [(self.desc.get("root_E", -1), self.desc.get("phi_E", 0.0))]
        cells = np.nonzero(self.ebkind == EB_ELECTRODE)[0]
        if len(cells) == 0 or len(elec) == 0:
            return pe
        if len(elec) == 1:
            pe[cells] = elec[0][1]
            return pe
        vals = np.stack([eval_implicit(self.desc, r, self.ebx[cells]) for r, _ in elec])
        k = np.argmin(vals, axis=0)
        pe[cells] = np.array([v for _, v in elec])[k]
        return pe

    # -- operator ------------------------------------------------------------
    def assemble(self, data):
        """Sparse A (CSR) and b with A phi = b  (A = -linear part of L, b = kappa s + data part)."""
        import scipy.sparse as sp
        dt, _keep = data
        cap = self.ndof * 160 + 16
        rows = np.zeros(cap, np.int64)
        cols = np.zeros(cap, np.int64)
        vals = np.zeros(cap)
        b = np.zeros(self.ndof)
        nnz = self._lib.or_assemble(self._g, C.byref(dt), _ptr(rows), _ptr(cols), _ptr(vals), cap, _ptr(b))
        if nnz > cap:
            raise RuntimeError("triplet capacity exceeded")
        A = sp.coo_matrix((vals[:nnz], (rows[:nnz], cols[:nnz])), shape=(self.ndof, self.ndof)).tocsr()
        A.sum_duplicates()
        return A, b

    def boundary_flux(self, data, phi_dof):
        dt, _keep = data
        phi_dof = np.ascontiguousarray(phi_dof, dtype=np.float64)
        return self._lib.or_boundary_flux(self._g, C.byref(dt), _ptr(phi_dof))

    def boundary_flux_masked(self, data, phi_dof, mask):
        dt, _keep = data
        phi_dof = np.ascontiguousarray(phi_dof, dtype=np.float64)
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        return self._lib.or_boundary_flux_masked(self._g, C.byref(dt), _ptr(phi_dof), _ptr(m))

    def face_flux(self, data, a, J, p):
        """(dof indices, weights, constant) of alpha/h x the +e_a centroid flux of face (a, J)."""
        dt, _keep = data
        Jv = np.array([J[0], J[1], J[2] if len(J) > 2 else 0], dtype=np.int64)
        idx = np.zeros(512, np.int64)
        w = np.zeros(512)
        c = np.zeros(1)
        n = self._lib.or_face_flux(self._g, C.byref(dt), a, _ptr(Jv), p, _ptr(idx), _ptr(w), _ptr(c))
        return idx[:n].copy(), w[:n].copy(), float(c[0])

    def field(self, data, phi_dof):
        """E[D][2][cell] at cell centres and En[cell][2] = -dphi/dn_in at EB centroids."""
        dt, _keep = data
        phi_dof = np.ascontiguousarray(phi_dof, dtype=np.float64)
        E = np.zeros((self.dim, 2, self.ncell))
        En = np.zeros((self.ncell, 2))
        self._lib.or_field(self._g, C.byref(dt), _ptr(phi_dof), _ptr(E), _ptr(En))
        return E, En

    # -- layout helpers --------------------------------------------------------
    def to_cells(self, x_dof):
        """dof vector -> [2][cell] array, 0 where a phase has no dof."""
        out = np.zeros((2, self.ncell))
        for p in range(2):
            m = self.dof[p] >= 0
            out[p, m] = x_dof[self.dof[p, m]]
        return out

    def to_dofs(self, x_cells):
        x_cells = np.asarray(x_cells).reshape(2, self.ncell)
        out = np.zeros(self.ndof)
        for p in range(2):
            m = self.dof[p] >= 0
            out[self.dof[p, m]] = x_cells[p, m]
        return out


def solve_system(A, b):
    """Direct sparse LU solve (SuperLU through SciPy)."""
    import scipy.sparse.linalg as spla
    lu = spla.splu(A.tocsc(), permc_spec="COLAMD")
    return lu.solve(b)


def solve(desc: dict, s=None, sigma=None, phiE=None, phidom=None):
    """Geometry + assembly + direct solve.  Returns (geometry, phi[2][cell], A, b)."""
    g = Geometry(desc)
    data = g.data(s=s, sigma=sigma, phiE=phiE, phidom=phidom)
    A, b = g.assemble(data)
    x = solve_system(A, b)
    return g, g.to_cells(x), A, b, data


def eval_implicit(desc: dict, root: int, pts: np.ndarray) -> np.ndarray:
    """Evaluate CSG node `root` of desc at points [m][3] (for tests)."""
    g = Geometry.__new__(Geometry)
    lib = _load()
    prims = desc.get("prims", [])
    nodes = desc.get("nodes", [])
    kind = np.array([p[0] for p in prims] or [0], dtype=np.int32)
    par = np.zeros((max(len(prims), 1), 10))
    for i, p in enumerate(prims):
        par[i, :len(p[1])] = p[1]
    par = np.ascontiguousarray(par.reshape(-1))
    op = np.array([q[0] for q in nodes] or [0], dtype=np.int32)
    a = np.array([q[1] for q in nodes] or [0], dtype=np.int32)
    b = np.array([q[2] for q in nodes] or [0], dtype=np.int32)
    d = _Desc()
    d.dim = int(desc["dim"])
    d.n_prims = len(prims)
    d.prim_kind = kind.ctypes.data_as(C.POINTER(C.c_int))
    d.prim_par = par.ctypes.data_as(C.POINTER(C.c_double))
    d.n_nodes = len(nodes)
    d.node_op = op.ctypes.data_as(C.POINTER(C.c_int))
    d.node_a = a.ctypes.data_as(C.POINTER(C.c_int))
    d.node_b = b.ctypes.data_as(C.POINTER(C.c_int))
    out = np.zeros(len(pts))
    for i, p in enumerate(np.asarray(pts, dtype=np.float64)):
        x = np.ascontiguousarray(p[:3])
        out[i] = lib.or_eval_implicit(C.byref(d), int(root), _ptr(x))
    del g
    return out

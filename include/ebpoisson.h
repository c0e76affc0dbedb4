/*
 * ebpoisson.h -- C ABI of the GB300 embedded-boundary multi-material Poisson
 * solver.
 *
 * The library solves the electrostatic equation of Marskar, arXiv:1809.03745,
 * Sec. 2.1, Eq. (poisson):
 *
 *     div(eps_r grad phi) = -rho / eps0
 *
 * on a Cartesian grid whose cells may be cut by embedded boundaries (EBs):
 * electrodes (Dirichlet, held at a potential) and dielectric interfaces across
 * which eps_r jumps and on which a surface charge sigma sits (Sec. 3.3.1,
 * Eq. matching).  The discretisation is the cut-cell finite-volume method of
 * Sec. 3.1 and 3.3 (integral form Eq. poisson_integral, centroid-interpolated
 * face fluxes, ray-cast EB normal-derivative stencils Eq. bndry_stencil,
 * multifluid boundary state eliminated); the linear system is solved by
 * geometric multigrid V-cycles with red-black Gauss-Seidel smoothing
 * (Sec. 3.3.2), optionally in FP32 inside an FP64 defect-correction loop.
 *
 * Conventions shared by every entry point:
 *   - Cells are indexed x fastest, then y, then z: c = i + n0*(j + n1*k).
 *     Cell i covers [lo + i h, lo + (i+1) h]; its centre is lo + (i + 1/2) h.
 *   - Two phases: 0 = gas (eps_gas), 1 = dielectric (eps_diel).  Per-phase
 *     fields are laid out [phase][cell].  Single-phase problems (no dielectric)
 *     still use two phase slots; slot 1 is ignored on input and zero on output.
 *   - "d_" arguments are DEVICE pointers owned by the caller, on the device
 *     that was current when the handle was created; "h_" arguments are host
 *     pointers.  The library never keeps a caller pointer past the call.
 *   - Work is enqueued on the given CUDA stream (a cudaStream_t passed as
 *     void*, NULL = legacy default stream).  Calls that return information
 *     (counts, convergence) synchronise that stream before returning.
 *   - Every call returns an eb_status; no exception crosses the ABI.  On error
 *     the outputs are unspecified and eb_last_error() describes the failure.
 *   - Handles are not thread-safe: one host thread per handle at a time.
 */
#ifndef EBPOISSON_H
#define EBPOISSON_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EB_OK = 0,
  EB_ERR_INVALID = 1,       /* bad argument or description */
  EB_ERR_OOM = 2,           /* device allocation failed or budget exceeded */
  EB_ERR_NOT_CONVERGED = 3, /* cycle cap reached before the tolerance */
  EB_ERR_CUDA = 4,          /* a CUDA runtime call failed */
  EB_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
  EB_ERR_UNSUPPORTED = 6,   /* geometry outside the method's model (see eb_geom_build) */
  EB_ERR_BUSY = 7           /* serving queue full / result not ready */
} eb_status;

/* Static description of a status code; never freed. */
const char* eb_status_str(eb_status s);
/* Detail of the last error raised on the calling thread; valid until the next call. */
const char* eb_last_error(void);

/* ------------------------------------------------------------- geometry
 * Implicit functions (Sec. 3.1, 3.2): each region is the NEGATIVE set of a
 * function s(x) built by CSG from primitives.  All formulas below are
 * evaluated in double precision in the stated order; 2D problems use z = 0.
 */
enum {
  EB_PRIM_SPHERE = 0,    /* p = [cx, cy, cz, r]:              |x - c| - r */
  EB_PRIM_CAPSULE = 1,   /* p = [ax, ay, az, bx, by, bz, r]:  dist(x, segment ab) - r */
  EB_PRIM_HALFSPACE = 2, /* p = [nx, ny, nz, d]:              n.x - d */
  EB_PRIM_SINE = 3,      /* p = [up, c, A, k, ph, t]:         x[up] - (c + A sin(2 pi k x[t] + ph)) */
  EB_PRIM_CYLINDER = 4,  /* p = [axis, px, py, pz, r, lo, hi]: max(dist_to_axis - r, lo - x[axis], x[axis] - hi) */
  EB_PRIM_BOX = 5        /* p = [lox, loy, loz, hix, hiy, hiz]: max_k max(lo_k - x_k, x_k - hi_k) */
};
enum { EB_CSG_PRIM = 0, EB_CSG_UNION = 1, EB_CSG_INTERSECT = 2, EB_CSG_NEGATE = 3 };
enum { EB_BC_NEUMANN = 0, EB_BC_DIRICHLET = 1, EB_BC_ROBIN = 2 };

#define EB_MAX_PRIMS 32
#define EB_MAX_NODES 64
#define EB_MAX_ELECTRODES 4

typedef struct {
  int kind;      /* EB_PRIM_* */
  double p[10];  /* parameters, see above */
} eb_prim;

typedef struct {
  int op;   /* EB_CSG_*: PRIM -> primitive a; UNION -> min(a,b); INTERSECT -> max(a,b); NEGATE -> -a */
  int a, b; /* primitive index (PRIM) or child node indices, children listed before parents */
} eb_csg;

typedef struct {
  int dim;        /* 2 or 3 */
  int n[3];       /* cells per axis; each a multiple of 8 and >= 8; n[2] ignored in 2D */
  double lo[3];   /* lower domain corner */
  double h;       /* cell size, the same on every axis */
  const eb_prim* prims;
  int n_prims;    /* <= EB_MAX_PRIMS */
  const eb_csg* nodes;
  int n_nodes;    /* <= EB_MAX_NODES */
  int electrode_root;                       /* node whose negative set is all electrodes, -1 = none */
  int n_electrodes;                         /* <= EB_MAX_ELECTRODES */
  int electrode_node[EB_MAX_ELECTRODES];    /* each electrode's own node */
  double electrode_phi[EB_MAX_ELECTRODES];  /* each electrode's potential */
  int dielectric_root;                      /* node whose negative set is the dielectric, -1 = none */
  double eps_gas, eps_diel;                 /* relative permittivities */
  int bc_type[6];     /* EB_BC_* per wall: xlo, xhi, ylo, yhi, zlo, zhi */
  double bc_value[6]; /* Dirichlet value per wall, or a3 of a Robin wall (Neumann walls are homogeneous) */
  /* Helmholtz and Robin terms (Sec. 3.3, Eq. helmholtz; Sec. 3.3.1, Eq. robin); all zero gives the
   * Poisson problem.  The operator becomes lam_p phi - div(eps grad phi) in phase p (each cell's
   * balance gains kappa lam_p phi).  A Robin wall imposes a1 phi + a2 dphi/dn = a3 with n out of the
   * domain; Robin electrodes impose the same with n into the electrode, electrode_phi giving each
   * electrode's a3.  The boundary value is eliminated through the one-sided wall formula or the EB
   * ray stencil that the Dirichlet condition uses.  Coefficients >= 0, a1 + a2 > 0, lam >= 0;
   * EB_ERR_INVALID otherwise. */
  double bc_robin[6][2];       /* a1, a2 per Robin wall */
  int electrode_robin;         /* 1: every electrode carries the Robin condition instead of a potential */
  double electrode_robin_a[2]; /* its a1, a2 */
  double helmholtz_lam[2];     /* lam per phase (gas, dielectric) */
} eb_geom_desc;

typedef struct eb_geom eb_geom;

#define EB_MAX_LEVELS 16
typedef struct {
  int dim;
  int n_phase;                   /* 1 without a dielectric, else 2 */
  long long n_cells;             /* finest level */
  long long n_dof;               /* fluid fragments with an unknown, finest level */
  long long n_eb;                /* cut cells with at least one unknown (the EB list) */
  long long n_irregular;         /* cells with a sparse operator row, finest level */
  int n_levels;                  /* multigrid levels (finest = 0) */
  int level_n[EB_MAX_LEVELS][3]; /* cells per axis on each level */
  long long stencil_order[3];    /* EB stencils of order 2, order 1, least squares */
  long long device_bytes;        /* device memory held by the handle */
} eb_geom_info;

/* Cut-cell geometry pass (Sec. 3.1): node labels, edge crossings (exactly 60
 * bisection halvings on the implicit function, midpoint of the final bracket),
 * face apertures and centroids, EB area, normal and centroid (EB normal from
 * the apertures by the divergence theorem), volume fractions by the divergence
 * theorem; then the coarsened multigrid hierarchy (Sec. 3.1, 3.3.2), stopping
 * where a coarse cell would be multi-valued or hold two kinds of boundary.
 * A node with s = 0 belongs to the non-negative side.
 * Errors: EB_ERR_INVALID (bad sizes, h, tree), EB_ERR_UNSUPPORTED (a cell cut
 * by an electrode and the dielectric at once, a face with four crossings, a
 * cell whose crossings do not form one loop, an EB stencil with no candidate
 * cells), EB_ERR_OOM, EB_ERR_CUDA.  *out is NULL on error. */
eb_status eb_geom_build(const eb_geom_desc* desc, void* stream, eb_geom** out);
eb_status eb_geom_query(const eb_geom* g, eb_geom_info* out);
void eb_geom_destroy(eb_geom* g);

/* Device copies of the finest-level geometry, for inspection.  Any pointer
 * may be NULL to skip it.  Sizes: flags [n_cells] (bit0 gas unknown, bit1
 * dielectric unknown, bit2 sparse row); kappa [2][n_cells]; eb_cell [n_eb]
 * ascending cell indices of the EB list; eb_area [n_eb] (units of h^{D-1});
 * eb_normal [n_eb][3] (unit, out of the gas fragment, or out of the fluid for
 * an electrode); eb_centroid [n_eb][3] (physical); eb_kind [n_eb] (1 electrode,
 * 2 dielectric interface); stencil_order [n_eb][2] (2, 1, 3 = least squares,
 * 0 = phase absent). */
typedef struct {
  uint8_t* flags;
  double* kappa;
  int32_t* eb_cell;
  double* eb_area;
  double* eb_normal;
  double* eb_centroid;
  uint8_t* eb_kind;
  int32_t* stencil_order;
} eb_geom_arrays;
eb_status eb_geom_export(const eb_geom* g, eb_geom_arrays* out, void* stream);

/* ------------------------------------------------------------- solver */
enum { EB_PREC_FP64 = 0, EB_PREC_MIXED = 1 };

typedef struct {
  double tol;        /* stop when max|r| <= tol * max|b| (Sec. 3.3.2), default 1e-10 */
  int max_cycles;    /* cap on V-cycles in total, default 100 */
  int nu1, nu2;      /* red-black Gauss-Seidel sweeps before / after the coarse correction;
                        -1 (the default) = by dimension: 2 in 2D, 6 in 3D, the fastest
                        to 1e-10 on the rod-plane and pin-plane workloads */
  int precision;     /* EB_PREC_FP64: FP64 V-cycles; EB_PREC_MIXED: FP32 V-cycles inside FP64 defect correction */
  int inner_cycles;  /* FP32 V-cycles per FP64 outer iteration (mixed), default 2 */
  int bottom_sweeps; /* relaxation sweeps on the coarsest level, default 64 */
  int launch_mode;   /* 0 (default): the whole solve in one persistent cooperative kernel (falls back to 1
                        when the device cannot launch cooperatively); 1: per-phase kernels, one iteration
                        replayed through a captured CUDA graph; 2: per-phase kernels, plain launches */
} eb_solver_opts;

/* Fill opts with the defaults listed above. */
void eb_solver_opts_default(eb_solver_opts* opts);

typedef struct {
  int status;       /* eb_status of the solve */
  int outer_iters;  /* FP64 residual evaluations after the initial one */
  int vcycles;      /* V-cycles in total */
  double rel_res;   /* final max|r| / max|b| in FP64 */
  double bnorm;     /* max|b| */
  long long kernel_launches; /* kernels this call launched (graph nodes counted per replay) */
  double kernel_ms; /* device time of the persistent solve kernel(s) of this call, from CUDA
                       events on the stream they ran on; 0 on the multi-launch paths */
  int bottom;       /* how the coarsest level was solved: EB_BOTTOM_* */
  int levels;       /* multigrid levels of the V-cycle */
  int sweep_levels; /* levels relaxed by tile-streamed sweeps (FP32 3D levels of at least 2^25 cells,
                       x extent a multiple of 16, y and z multiples of 4: both colours in one pass
                       over the level, tiles staged in shared memory by TMA); the others use one
                       pass per colour.  The environment variable EBP_SWEEP=0 turns them off,
                       EBP_SWEEP_MIN_CELLS=n moves the threshold, EBP_SWEEP_RESTRICT=1 also
                       restricts these levels by a tile-streamed residual + restriction pass */
} eb_solve_info;

/* Bottom solves of the V-cycle (Sec. 3.3.2 solves the coarsest level directly
 * or by relaxation; which one applies follows from the coarsest level's size):
 * an exact FP64 inverse for at most 256 unknowns, applied inside one CTA; an
 * FP32 Gauss-Jordan inverse for at most 1024 unknowns, applied by the whole
 * grid; BiCGStab over the whole grid when coarsening stopped above 4096 cells;
 * else red-black relaxation sweeps inside one CTA (also the bottom of the
 * per-phase launch paths). */
enum { EB_BOTTOM_RELAX = 1, EB_BOTTOM_INV64 = 2, EB_BOTTOM_INV32 = 3, EB_BOTTOM_KRYLOV = 4 };

typedef struct eb_poisson eb_poisson;

/* Builds the finite-volume operator on every multigrid level (Sec. 3.3):
 * regular cells use the implicit 2D+1-point stencil eps_p/h^2 with
 * second-order one-sided Dirichlet walls; cut cells get a sparse FP64 row with
 * centroid-interpolated face fluxes, ray-cast EB derivatives (order 2, then
 * first order, then least squares) and the multifluid boundary state
 * eliminated.  The handle keeps a reference to g; destroy the solver first. */
eb_status eb_poisson_setup(const eb_geom* g, const eb_solver_opts* opts, void* stream, eb_poisson** out);
void eb_poisson_destroy(eb_poisson* P);

/* r = b - A phi in FP64 on the finest level, [2][n_cells], for given
 * d_rhs = rho/eps0 [2][n_cells] sampled at cell centres and d_sigma =
 * sigma/eps0 [n_cells] (read only on dielectric-interface cells; may be NULL
 * for zero).  b = kappa * rhs + the boundary data (electrode and wall
 * potentials, surface charge).  With d_phi = 0 this returns b. */
eb_status eb_poisson_residual(eb_poisson* P, const double* d_rhs, const double* d_sigma, const double* d_phi,
                              double* d_r, void* stream);

/* Allocation-free variant of eb_poisson_residual (the paper has no
 * counterpart: this serves callers that cannot allocate device memory where
 * they need the residual, e.g. inside a fully carved-up memory pool or an
 * allocator-free real-time loop).  Same inputs and output as
 * eb_poisson_residual, but it takes the geometry handle (built earlier) and
 * needs no solver handle; its scratch (right-hand side and sparse-row
 * residuals) lives in one file-scope device array of 2^21 + 2^19 + 8 doubles
 * (about 20.1 MB), held on every device that loads the library until the
 * process exits.  Limits: at most 2^20 finest-level cells and 2^19 sparse
 * rows, else EB_ERR_INVALID before any device work; EB_ERR_INVALID too when
 * the current device is not the one g was built on.  d_phi is read as given
 * (no masked copy): its entries without an unknown must be finite.  It calls
 * no cudaMalloc or cudaFree.  Every call looks up the array's address on the
 * current device (cudaGetSymbolAddress, so a context created afresh after
 * cudaDeviceReset is handled); the first call on a device may load the
 * module and should come before any stream capture.  Every call shares the
 * one array: calls whose work overlaps on the device race and give undefined
 * results.  Synchronises the stream before returning. */
eb_status eb_poisson_residual_noalloc(const eb_geom* g, const double* d_rhs, const double* d_sigma,
                                      const double* d_phi, double* d_r, void* stream);

/* Solves A phi = b to max|r| <= tol max|b|.  d_phi [2][n_cells] holds the
 * initial guess on entry and the solution on exit (entries without an unknown
 * are written as 0).  info may be NULL.  Returns EB_ERR_NOT_CONVERGED when the
 * cycle cap is reached (d_phi then holds the last iterate). */
eb_status eb_poisson_solve(eb_poisson* P, const double* d_rhs, const double* d_sigma, double* d_phi,
                           eb_solve_info* info, void* stream);

/* Solves n independent problems (each with its own geometry and solver
 * handle, all of one precision on one device) in one persistent cooperative
 * launch: every instance gets a group of CTAs in proportion to its cell
 * count and runs its own multigrid solve and convergence test with a barrier
 * of its own, so instances finish independently.  P, d_rhs, d_sigma and d_phi
 * are host arrays of n entries (d_sigma may be NULL, or hold NULL entries);
 * infos (n entries) may be NULL.  Each result equals the single solve of the
 * same instance up to rounding.  A handle may appear once per batch
 * (EB_ERR_INVALID otherwise).  Returns the first non-OK instance status. */
eb_status eb_poisson_solve_batched(eb_poisson* const* P, int n, const double* const* d_rhs,
                                   const double* const* d_sigma, double* const* d_phi, eb_solve_info* infos,
                                   void* stream);

/* E = -grad phi (Sec. 2.1) at cell centres per phase, d_E [D][2][n_cells]:
 * centred differences where both face neighbours carry an unknown of the
 * phase across an open face, one-sided where one does, else the EB normal
 * derivative times the normal; and the normal field -dphi/dn_in at each EB
 * centroid per phase, d_En [n_eb][2] (EB list order), using the eliminated
 * boundary state on dielectric interfaces. */
eb_status eb_field_eval(eb_poisson* P, const double* d_phi, const double* d_sigma, double* d_E, double* d_En,
                        void* stream);

/* The constants of one TGA step of length dt (Sec. 3.4, Eq. tga; Twizell, Gumel
 * and Arigu): mu[0..3] = mu1, mu2, mu3, mu4 with a = 2 - sqrt(2) - (machine
 * precision), mu1,2 = (a -+ sqrt(a^2 - 4a + 2)) dt / 2, mu3 = (1 - a) dt,
 * mu4 = (1/2 - a) dt.  EB_ERR_INVALID unless dt > 0 and finite. */
eb_status eb_tga_coefficients(double dt, double mu[4]);

/* Opaque handle of a TGA diffusion stepper (Sec. 3.4, Eq. tga). */
typedef struct eb_tga eb_tga;

/* A stepper for the implicit diffusion d phi/dt = L phi + rho with
 * L phi = div(eps grad phi) on the cut-cell grid, where each cell's balance is
 * kappa d phi/dt = (L phi integrated over the cell) + kappa rho.  One step of
 * length dt solves
 *   (M - mu1 L) psi = (M + mu3 L) phi + dt (M + mu4 L) rho,
 *   (M - mu2 L) phi_next = M psi,       M = diag(kappa).
 * We read the printed equation this way: it omits dt on the source and writes
 * the model equation with +L while the scheme's operators carry -L.
 * G0, G1, G2 are geometries built from one description whose helmholtz_lam is
 * 0, 1/mu1 and 1/mu2 of this dt (eb_tga_coefficients; both phases when there
 * are two; eps is the diffusion coefficient); P0, P1, P2 are persistent solver
 * handles on them (only P0's operator is applied).  EB_ERR_INVALID when the grids differ or a shift does not match dt.  Boundary
 * conditions are the description's types with homogeneous data (its values
 * are not used).  The stepper borrows the six handles (they must outlive it)
 * and owns 10 x n_cells doubles of device memory; kappa is computed on
 * `stream` here.  *out is null on failure. */
eb_status eb_tga_create(const eb_geom* G0, const eb_geom* G1, const eb_geom* G2, eb_poisson* P0, eb_poisson* P1,
                        eb_poisson* P2, double dt, void* stream, eb_tga** out);

/* One step of the stepper T.  d_phi, d_rho, d_out: FP64 [2][n_cells] device
 * arrays (d_out may be d_phi); entries without an unknown must be finite and
 * come out 0.  Each stage is solved to max|r| <= tol max|b| from zero
 * (0 < tol < 1); info[0] and info[1] (may be null) report the two stage
 * solves.  The step is enqueued on `stream` and returns after the stages; one
 * stepper runs one step at a time.  Returns the first stage status that is not
 * EB_OK (EB_ERR_NOT_CONVERGED when an iteration limit is reached). */
eb_status eb_tga_step(eb_tga* T, const double* d_phi, const double* d_rho, double* d_out, double tol,
                      eb_solve_info* info, void* stream);

/* Frees the stepper's device memory (not the borrowed handles); null is a
 * no-op. */
void eb_tga_destroy(eb_tga* T);

/* Benchmark hook (no counterpart in the paper): launches one kernel of the
 * finest multigrid level `reps` times on `stream` between CUDA events and
 * reports the mean duration per launch and the algorithmic bytes one launch
 * must move.  It relaxes the solver's own work arrays (left as the last solve
 * left them); the caller's fields are not touched.  Both run the persistent
 * solve kernel's own phase code in its grid shape.  kernel 0: one colour of
 * the red-black Gauss-Seidel sweep (regular cells) of the inner-precision finest level
 * (bytes: half of read x, read b, write x, read flags per cell); kernel 1: the
 * fused residual + restriction of that level (read x, b, flags per fine cell,
 * write coarse b and x); kernel 6: the prolongation of the next level's
 * correction onto it (read and write x, read the flags per fine cell, read
 * the coarse x and flags). */
eb_status eb_poisson_profile(eb_poisson* P, int kernel, int reps, double* ms_per_launch, double* bytes_per_launch,
                             void* stream);
/* kernel 2 of eb_poisson_profile times `reps` grid barriers of the persistent
 * solve kernel (bytes_per_launch receives the number of CTAs).  kernel 3 is
 * the bounded-wait self-test: two CTAs wait at a grid barrier sized for
 * three, so the wait ends only by its clock bound (about 2 s); the call then
 * returns EB_ERR_TIMEOUT with ms_per_launch the kernel's duration, and the
 * context stays usable.  Kernels 4 and 5 need a finest level relaxed by
 * tile-streamed sweeps (EB_ERR_UNSUPPORTED otherwise): 4 is one such sweep,
 * both colours in one pass (bytes: read x, b, flags, write x per cell), 5 the
 * tile-streamed residual + restriction (read x, b, flags per fine cell, write
 * coarse b and x); a wait of theirs that gives up returns EB_ERR_TIMEOUT. */

/* Benchmark hook (no counterpart in the paper): the device's measured rate
 * of fused multiply-adds in FP64 and in FP32, in TFLOP/s (two flops per
 * FMA): eight independent FMA chains per thread over eight CTAs of 256
 * threads per SM, timed with CUDA events.  The roofline of an FP64 kernel is
 * the lesser of the memory bound and this rate times its flops per byte. */
eb_status eb_device_fma_rates(int device, double* fp64_tflops, double* fp32_tflops);

/* Diagnostics (no counterpart in the paper): the phases of the first V-cycle
 * of the last persistent solve.  out[0] = number of phases m; then for each
 * phase i, out[1+2i] = its code ((level << 4) | kind; kinds 1 red regular
 * cells, 3 black regular cells (each also writes the sparse-row values of
 * its colour), 2 sparse rows computed, 5 sparse residual rows, 6 residual +
 * restriction, 7 prolongation,
 * 8 end of the one-CTA levels, 9 bottom solve) and
 * out[2+2i] its duration in ms.  n is the capacity of out. */
eb_status eb_poisson_trace(eb_poisson* P, double* out, int n);

/* ---------------------------------------------------------------- composite grid
 * One ratio-2 refined box over the coarse grid (Sec. 3.3.2 solves on refined
 * levels; coarse-fine coupling by refluxing, Sec. 3.3).  The box covers
 * coarse cells [box_lo, box_hi) per axis (sides a positive multiple of 4
 * cells); the fine grid has 2 (box_hi - box_lo) cells per axis at h/2 and is
 * built from the same description.  Composite operator: fine cells next to a
 * coarse-fine (CF) side get the flux eps_gas (ghost - phi)/h_f through it,
 * the ghost by quadratic tangential interpolation of coarse values (weights
 * -3/32, 15/16, 5/32) and quadratic normal interpolation (-1/5, 2/3, 8/15),
 * falling back to linear, then constant, where a needed cell is outside the
 * domain, under the box, covered or cut; the coarse cell across a CF face
 * has the coarse flux through it replaced by minus the mean of the fine
 * fluxes (exact conservation); coarse cells under the box carry no equation
 * and take the kappa-weighted mean of their children.  Only the gas phase may
 * touch a CF side (EB_ERR_UNSUPPORTED otherwise).
 * Fields: coarse [2][n_coarse], fine [2][n_fine] (layout as elsewhere). */
typedef struct eb_amr eb_amr;
eb_status eb_amr_setup(const eb_geom_desc* coarse, const int box_lo[3], const int box_hi[3],
                       const eb_solver_opts* opts, void* stream, eb_amr** out);
eb_status eb_amr_query(const eb_amr* A, long long* n_coarse, long long* n_fine, int fine_n[3], long long* cf_faces);
/* Composite residual b - A phi (FP64): d_r_c is 0 under the box and where a
 * cell has no unknown; phi_c values under the box are ignored (replaced by
 * the fine means). */
eb_status eb_amr_residual(eb_amr* A, const double* d_rhs_c, const double* d_sig_c, const double* d_rhs_f,
                          const double* d_sig_f, const double* d_phi_c, const double* d_phi_f, double* d_r_c,
                          double* d_r_f, void* stream);
/* Composite solve to max|r| <= tol max|b| (opts of setup; max_cycles caps the
 * composite iterations): restarted FGMRES (restart 12, FP64) preconditioned
 * by one FAC step: a coarse correction over the domain (fine part averaged
 * under the box), constant per parent on the fine grid, then a fine
 * correction on the box with zero Dirichlet data on its CF sides, each one V-cycle
 * of the persistent multigrid solve (3+3 sweeps, a relaxed bottom at most 32
 * sweeps).  d_phi_c / d_phi_f hold the guess on
 * entry; on return d_phi_c under the box holds the fine means.  info:
 * outer_iters = FGMRES iterations, vcycles = V-cycles of the corrections.
 * The work space (27 composite vectors) is allocated at the first call. */
eb_status eb_amr_solve(eb_amr* A, const double* d_rhs_c, const double* d_sig_c, const double* d_rhs_f,
                       const double* d_sig_f, double* d_phi_c, double* d_phi_f, eb_solve_info* info, void* stream);
/* Benchmark hook (no counterpart in the paper): the persistent multigrid
 * launches of the last eb_amr_solve, for the coarse correction solver
 * (out[0..3]) and the fine one (out[4..7]): launches, their summed device
 * time in ms (CUDA events on their stream), V-cycles, FP64 outer iterations.
 * info->kernel_ms of eb_amr_solve is the summed time of those launches;
 * info->kernel_launches counts every kernel the call launched. */
eb_status eb_amr_kernel_stats(const eb_amr* A, double out[8]);
void eb_amr_destroy(eb_amr* A);

/* ---------------------------------------------------------------- nested levels
 * A composite grid of n_levels levels (2 .. EB_AMR_MAX_LEVELS; Sec. 3.3.2
 * solves on a hierarchy of refined levels, Sec. 6 refines where the tracer
 * criteria ask).  Level 0 is the grid of `base`; level l >= 1 is one ratio-2
 * box over cells [box_lo[l-1][k], box_hi[l-1][k]) of level l-1's grid,
 * counted from that grid's lower corner (sides a positive multiple of 4
 * parent cells).  Every pair of consecutive levels is coupled as in the
 * two-level grid above; a cell under the next finer box carries no equation
 * and takes the kappa-weighted mean of its children (themselves such means
 * under a still finer box).  Proper nesting: a box keeps at least one parent
 * cell away from each coarse-fine side of its parent (EB_ERR_INVALID
 * otherwise); sides on the domain boundary keep the domain's conditions.
 * box_lo / box_hi: host arrays of 3 (n_levels - 1) ints.  The two-level calls
 * above are this with n_levels = 2 (eb_amr_residual / eb_amr_solve refuse
 * more levels; eb_amr_query reports levels 0 and 1). */
#define EB_AMR_MAX_LEVELS 4
eb_status eb_amr_setup_levels(const eb_geom_desc* base, int n_levels, const int* box_lo, const int* box_hi,
                              const eb_solver_opts* opts, void* stream, eb_amr** out);
/* Level `level`'s grid: number of levels, cells, cells per axis, physical
 * lower corner, spacing, and fine CF faces towards its parent (0 on level 0).
 * Any output may be NULL. */
eb_status eb_amr_level_query(const eb_amr* A, int level, int* n_levels, long long* n_cells, int n[3],
                             double lo[3], double* h, long long* cf_faces);
/* The geometry of level `level` (owned by A; CF sides as Neumann walls), for
 * eb_geom_query / eb_geom_export / eb_tag_cells. */
eb_status eb_amr_level_geom(const eb_amr* A, int level, const eb_geom** out);
/* Composite residual b - A phi (FP64) over all levels: d_rhs, d_sig, d_phi,
 * d_r are host arrays of n_levels device pointers, each level [2][n_cells]
 * (d_sig or its entries may be NULL).  d_r is 0 under the next finer box and
 * where a cell has no unknown; phi values under a finer box are ignored. */
eb_status eb_amr_residual_levels(eb_amr* A, const double* const* d_rhs, const double* const* d_sig,
                                 const double* const* d_phi, double* const* d_r, void* stream);
/* Composite solve over all levels to max|r| <= tol max|b|: restarted FGMRES
 * (restart 12, FP64) preconditioned by one multiplicative FAC sweep from
 * level 0 up (a level-0 correction over the domain with the finer remainders
 * restricted under the boxes, constant per parent on level 1, then on every
 * finer level a correction of what remains there with zero Dirichlet data on
 * its CF sides), each correction one V-cycle of the persistent multigrid
 * solve (3+3 sweeps, a relaxed bottom at most 32 sweeps).  d_phi holds the
 * guess on entry; on return every level's values
 * under the next finer box hold the finer means.  info as eb_amr_solve. */
eb_status eb_amr_solve_levels(eb_amr* A, const double* const* d_rhs, const double* const* d_sig,
                              double* const* d_phi, eb_solve_info* info, void* stream);
/* E = -grad phi on level `level`'s grid alone (as eb_field_eval; the level's CF
 * sides act as Neumann walls, so cells next to them take one-sided values). */
eb_status eb_amr_field_eval(eb_amr* A, int level, const double* d_phi, const double* d_sigma, double* d_E,
                            double* d_En, void* stream);

/* ---------------------------------------------------------------- regrid tags
 * Refinement tags of Sec. 6 on one grid (a plain geometry or a level of a
 * composite grid): the tracer T = |E| / max |E|, |E| per cell the largest
 * field magnitude over the phases with an unknown, the maximum over the
 * grid's cells; a cell is tagged for refinement (tag value 1) when
 * |grad T| dx / T > eps[0] or T > eps[1], for coarsening (value 2) when
 * |grad T| dx / T < eps[2] and T < eps[3] (the paper uses 0.1, 0.8, 0.1, 0.2).
 * grad T by differences over the axis neighbours that carry T: centred
 * ((T+ - T-)/2 in index units, dx cancels), one-sided where one neighbour
 * does, 0 where none does; the ratio is 0 where T and the gradient are 0 and
 * infinite where only T is 0.  Covered cells get no tag.  All arithmetic is
 * FP64 without contraction, so the tags are a function of d_E alone.
 * d_E: [D][2][n_cells] as eb_field_eval writes it.  keep_lo / keep_hi (both
 * or neither NULL): the current finer box on this grid; its cells that carry
 * T and are not tagged for coarsening are marked as well (a refined region is
 * kept until the coarsening test releases it).  d_tags (may be NULL):
 * [n_cells] tag bytes.  On return bbox_lo / bbox_hi (host, 3 ints; hi
 * exclusive) bound the marked cells (refine-tagged or kept), *n_marked counts
 * them (0: bbox undefined) and *e_max is max |E|.  The call allocates a
 * scratch of n_cells doubles (T) for its duration and synchronises the
 * stream.  EB_ERR_INVALID for a NULL argument, an eps that is not finite, or
 * a current device other than the geometry's (checked before any launch). */
eb_status eb_tag_cells(const eb_geom* G, const double* d_E, const double eps[4], const int* keep_lo,
                       const int* keep_hi, unsigned char* d_tags, int bbox_lo[3], int bbox_hi[3],
                       long long* n_marked, double* e_max, void* stream);
/* The next finer box from the marked cells' bounding box (host arithmetic, no
 * device work): grown by `buf` cells per side, rounded outward to multiples
 * of `block`, clipped to the grid n[dim] and `block` cells short of every side
 * that is a coarse-fine side (cf_lo / cf_hi per axis, nonzero for CF), then
 * widened to `block` cells away from the side it was clipped at if clipping
 * left it thinner.  *has_box = 0 when n_marked is 0 or the grid has no room;
 * else box_lo / box_hi hold the box (the next level's box_lo / box_hi).
 * EB_ERR_INVALID for buf < 0, block < 1 or dim outside 2..3. */
eb_status eb_regrid_box(int dim, const int n[3], const int cf_lo[3], const int cf_hi[3], const int bbox_lo[3],
                        const int bbox_hi[3], long long n_marked, int buf, int block, int box_lo[3],
                        int box_hi[3], int* has_box);

/* ---------------------------------------------------------------- serving
 * Continuous-batching solve server (no counterpart in the paper, whose
 * solves run one per time step inside a plasma code).  Requests (a geometry
 * description and host fields) are queued on submit; a worker thread admits
 * them in arrival order while the device-memory budget and the slot count
 * allow, builds their geometry and hierarchy on the device, and advances
 * every admitted instance together in batched persistent launches of
 * `step_iters` FP64 outer iterations each.  Instances join and leave at those
 * boundaries, so a request that arrives while others run starts at the next
 * step and a converged one frees its slot and memory at once.  An instance's
 * iterates are those of its single solve (a resumed step recomputes the same
 * residual), so its result equals the single solve with the same options.
 * A request whose build or solve fails completes with that status; the
 * others are not affected. */
typedef struct {
  double hbm_budget_bytes; /* device bytes the admitted instances may hold; <= 0: half the free memory */
  int max_slots;           /* instances on the device at once, 1..1024 */
  int queue_cap;           /* requests waiting for admission before submit returns EB_ERR_BUSY */
  int step_iters;          /* FP64 outer iterations per batched launch (>= 1) */
  int device;              /* CUDA device */
  eb_solver_opts solver;   /* options of every instance (persistent path; launch_mode ignored) */
} eb_server_opts;

typedef struct {
  long long submitted, completed, failed, queued, active;
  double p50_ms, p99_ms;      /* latency from submit to result ready, completed requests */
  double cells_per_s;         /* cells of completed requests / time from first admission to last completion */
  long long cells_completed;
  long long hbm_budget, hbm_used, hbm_peak; /* bytes accounted to admitted instances */
  long long steps;            /* batched launches */
  long long estimate_misses;  /* admissions whose measured bytes exceeded the pre-build estimate */
} eb_server_stats;

typedef struct eb_server eb_server;

void eb_server_opts_default(eb_server_opts* o);
/* Starts the worker thread.  Errors: EB_ERR_INVALID, EB_ERR_CUDA. */
eb_status eb_server_create(const eb_server_opts* o, eb_server** out);
/* Queues one solve.  desc (and its arrays), h_rhs [2][n_cells] and h_sigma
 * [n_cells] (may be NULL) are copied before the call returns.  *ticket
 * names the request.  EB_ERR_BUSY when the queue holds queue_cap requests;
 * EB_ERR_INVALID for a description rejected on the host. */
eb_status eb_server_submit(eb_server* S, const eb_geom_desc* desc, const double* h_rhs, const double* h_sigma,
                           unsigned long long* ticket);
/* EB_ERR_BUSY while the request is queued or running.  When it is done:
 * copies phi [2][n_cells] into h_phi (may be NULL) and the solve's info,
 * returns EB_OK, and forgets the ticket.  A failed request returns EB_OK
 * with info->status holding its error.  EB_ERR_INVALID for an unknown ticket. */
eb_status eb_server_poll(eb_server* S, unsigned long long ticket, double* h_phi, eb_solve_info* info);
/* eb_server_poll that blocks up to timeout_s seconds (EB_ERR_BUSY after that);
 * timeout_s is clamped to [0, 1e7] (NaN counts as 0, +inf as 1e7). */
eb_status eb_server_wait(eb_server* S, unsigned long long ticket, double timeout_s, double* h_phi,
                         eb_solve_info* info);
eb_status eb_server_query(eb_server* S, eb_server_stats* out);
/* Finishes the admitted and queued requests, stops the worker, frees everything. */
void eb_server_destroy(eb_server* S);

#ifdef __cplusplus
}
#endif
#endif /* EBPOISSON_H */

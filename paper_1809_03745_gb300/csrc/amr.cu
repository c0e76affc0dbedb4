// amr.cu -- composite two-level solve: one ratio-2 refined box over a coarse
// grid (Sec. 3.3.2 runs its multigrid over refined levels; the coarse-fine
// coupling follows the refluxing of Sec. 3.3).
//
// Composite operator (the same reading as the oracle's):
//   * the fine box is a grid of its own whose coarse-fine (CF) sides are
//     homogeneous Neumann walls; the CF flux eps0 (ghost - phi_F)/h_f times the
//     fine aperture is added to each fine cell next to a CF side, the ghost by
//     quadratic tangential then quadratic normal Lagrange steps (fallbacks to
//     linear, then constant) precomputed per face at set-up;
//   * a coarse cell outside the box next to a CF side loses the coarse
//     operator's own flux through that face and gains minus the mean of the
//     fine fluxes through it (refluxing: exact conservation);
//   * coarse cells under the box carry no equation; where a coarse stencil
//     reaches one, its value is the kappa-weighted mean of its children.
// Solve: restarted FGMRES in FP64 on the composite system, right-
// preconditioned by one FAC step: a coarse correction over the whole domain
// (the fine part of the vector averaged onto the coarse cells under the box),
// added constant per parent on the fine grid, then a fine correction of what
// remains on the box with zero Dirichlet data on its CF sides.  Both
// corrections run one V-cycle of the persistent multigrid kernel; dot products are
// summed in a fixed order (deterministic).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "eb_internal.h"

using namespace ebp;

namespace {

constexpr int TBA = 256;
int nb(long long n) { return (int)std::max<long long>(1, (n + TBA - 1) / TBA); }

struct BoxIdx {
  int D;
  int nc[3], nf[3], lo[3], hi[3];
};

// cell indices of linear index c (grids of fewer than 2^32 cells: 32-bit
// divisions, several times cheaper than 64-bit ones in these memory-bound
// passes over every coarse cell)
__device__ __forceinline__ void ijk3(const int n[3], long long c, int I[3]) {
  const unsigned cu = (unsigned)c, n0 = (unsigned)n[0], n1 = (unsigned)n[1];
  const unsigned r = cu / n0;
  I[0] = (int)(cu - r * n0);
  const unsigned k = r / n1;
  I[1] = (int)(r - k * n1);
  I[2] = (int)k;
}
__device__ __forceinline__ long long lin3(const int n[3], const int I[3]) {
  return (long long)I[0] + (long long)n[0] * ((long long)I[1] + (long long)n[1] * I[2]);
}
__device__ __forceinline__ bool under_box(const BoxIdx& B, const int I[3]) {
  for (int k = 0; k < B.D; ++k)
    if (I[k] < B.lo[k] || I[k] >= B.hi[k]) return false;
  return true;
}

// coarse values under the box: kappa-weighted mean of the children with the phase
__global__ void k_avg_down(BoxIdx B, const uint8_t* cflags, const uint8_t* fflags, const double* kf, const double* pf,
                           double* pc, long long ncc, long long nff) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncc) return;
  int I[3];
  ijk3(B.nc, c, I);
  if (!under_box(B, I)) return;
  for (int p = 0; p < 2; ++p) {
    if (!((cflags[c] >> p) & 1)) {
      pc[p * ncc + c] = 0.0;
      continue;
    }
    double num = 0.0, den = 0.0;
    for (int k = 0; k < (1 << B.D); ++k) {
      int F[3] = {0, 0, 0};
      for (int a = 0; a < B.D; ++a) F[a] = 2 * (I[a] - B.lo[a]) + ((k >> a) & 1);
      long long f = lin3(B.nf, F);
      if ((fflags[f] >> p) & 1) {
        double w = kf[p * nff + f];
        num += w * pf[p * nff + f];
        den += w;
      }
    }
    pc[p * ncc + c] = den > 0.0 ? num / den : 0.0;
  }
}

// alpha_f times the CF flux out of the fine cell, per fine CF face
__global__ void k_cf_flux(const CFFace* faces, long long nface, const double* pc, const double* pf, double eps0,
                          double hf, double* fl) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nface) return;
  const CFFace f = faces[t];
  double v = 0.0;
  if (f.al > 0.0) {
    double tv = 0.0;
    for (int k = 0; k < f.nc; ++k) tv += f.cw[k] * pc[f.cc[k]];
    double ghost = f.wf * pf[f.fcell] + f.wc * tv;
    if (f.f2 >= 0) ghost += f.wf2 * pf[f.f2];
    v = f.al * eps0 * (ghost - pf[f.fcell]) / hf;
  }
  fl[t] = v;
}

// fine rows of one CF side (one face per fine cell within a side)
__global__ void k_cf_fine_apply(const CFFace* faces, long long t0, long long t1, const double* fl, double hf,
                                double* rf) {
  long long t = t0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= t1) return;
  const CFFace& f = faces[t];
  if (f.al > 0.0) rf[f.fcell] += fl[t] / hf;
}

// coarse rows next to the box: take the coarse face flux out, put minus the
// mean fine flux in
__global__ void k_cf_coarse_apply(const CFCoarse* cf, long long n, const double* fl, const double* pc, long long ncc,
                                  double hc, int D, double* rc) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const CFCoarse& c = cf[t];
  if (c.ccell < 0) return;
  double own = 0.0;
  for (int k = 0; k < c.n; ++k) {
    unsigned cl = (unsigned)c.col[k];
    own += c.w[k] * pc[(long long)(cl >> 30) * ncc + (cl & 0x3fffffffu)];
  }
  double fsum = 0.0;
  for (int k = 0; k < c.nfine; ++k) fsum += fl[c.fine[k]];
  rc[c.ccell] += -own - fsum / (hc * (double)(1 << (D - 1)));
}

__global__ void k_zero_under(BoxIdx B, double* rc, long long ncc) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncc) return;
  int I[3];
  ijk3(B.nc, c, I);
  if (under_box(B, I)) rc[c] = rc[ncc + c] = 0.0;
}

// coarse correction right-hand side under the box: mean fine residual of the
// children carrying the phase
__global__ void k_restrict_under(BoxIdx B, const uint8_t* fflags, const double* rf, double* rc, long long ncc,
                                 long long nff) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncc) return;
  int I[3];
  ijk3(B.nc, c, I);
  if (!under_box(B, I)) return;
  for (int p = 0; p < 2; ++p) {
    double s = 0.0;
    int m = 0;
    for (int k = 0; k < (1 << B.D); ++k) {
      int F[3] = {0, 0, 0};
      for (int a = 0; a < B.D; ++a) F[a] = 2 * (I[a] - B.lo[a]) + ((k >> a) & 1);
      long long f = lin3(B.nf, F);
      if ((fflags[f] >> p) & 1) {
        s += rf[p * nff + f];
        ++m;
      }
    }
    rc[p * ncc + c] = m ? s / m : 0.0;
  }
}

// phi_c += e_c outside the box; phi_f += e_c of the parent where the fine cell has the phase
__global__ void k_add_coarse(BoxIdx B, const double* ec, double* pc, long long ncc) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncc) return;
  int I[3];
  ijk3(B.nc, c, I);
  if (under_box(B, I)) return;
  pc[c] += ec[c];
  pc[ncc + c] += ec[ncc + c];
}
__global__ void k_prolong_const(BoxIdx B, const uint8_t* fflags, const double* ec, double* pf, long long ncc,
                                long long nff) {
  long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nff) return;
  int F[3];
  ijk3(B.nf, f, F);
  int I[3] = {0, 0, 0};
  for (int a = 0; a < B.D; ++a) I[a] = B.lo[a] + F[a] / 2;
  long long c = lin3(B.nc, I);
  for (int p = 0; p < 2; ++p)
    if ((fflags[f] >> p) & 1) pf[p * nff + f] += ec[p * ncc + c];
}
__global__ void k_axpy_masked(const uint8_t* flags, long long n, const double* x, double* y) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int p = 0; p < 2; ++p)
    if ((flags[c] >> p) & 1) y[p * n + c] += x[p * n + c];
}
__global__ void k_absmax2(const uint8_t* flags, long long n, const double* v, unsigned long long* out) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  if (c < n)
    for (int p = 0; p < 2; ++p)
      if ((flags[c] >> p) & 1) m = fmax(m, fabs(v[p * n + c]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// Composite vectors: coarse [2][ncc] (entries under the box and without an
// unknown ignored) and fine [2][nff].  Partial sums per block, added on the
// host in block order, so every dot product is deterministic.
constexpr int DOT_BLOCKS = 512;
__global__ void k_cv_dot(BoxIdx B, const uint8_t* flags, long long n, int coarse, const double* a, const double* b,
                         double* part) {
  __shared__ double sh[TBA];
  double acc = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    if (coarse) {
      int I[3];
      ijk3(B.nc, c, I);
      if (under_box(B, I)) continue;
    }
    for (int p = 0; p < 2; ++p)
      if ((flags[c] >> p) & 1) acc += a[p * n + c] * b[p * n + c];
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
    if ((int)threadIdx.x < s2) sh[threadIdx.x] += sh[threadIdx.x + s2];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
// Dot products of w with m vectors at once (m <= CV_MAXV): per block the m
// partial sums, part[i * gridDim.x + block]; the caller adds the blocks in
// order (deterministic).  Coarse entries under the box are skipped.
constexpr int CV_MAXV = 14;
struct CVPtrs {
  const double* v[CV_MAXV];
  double a[CV_MAXV];
};
__global__ void k_cv_mdot(BoxIdx B, const uint8_t* flags, long long n, int coarse, int m, CVPtrs V, const double* w,
                          double* part) {
  __shared__ double sh[CV_MAXV][TBA / 32];
  double acc[CV_MAXV];
#pragma unroll
  for (int i = 0; i < CV_MAXV; ++i) acc[i] = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    if (coarse) {
      int I[3];
      ijk3(B.nc, c, I);
      if (under_box(B, I)) continue;
    }
    const unsigned f = flags[c];
    for (int p = 0; p < 2; ++p) {
      if (!((f >> p) & 1u)) continue;
      const double wv = w[p * n + c];
#pragma unroll
      for (int i = 0; i < CV_MAXV; ++i)
        if (i < m) acc[i] += V.v[i][p * n + c] * wv;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < CV_MAXV; ++i) {
    double a = acc[i];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) sh[i][wid] = a;
  }
  __syncthreads();
  if (threadIdx.x < m) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[threadIdx.x][k];
    part[threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
}
// w -= sum_i a_i v_i on the entries with an unknown (others 0)
__global__ void k_cv_maxpy(const uint8_t* flags, long long n, int m, CVPtrs V, double* w) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const unsigned f = flags[c];
  for (int p = 0; p < 2; ++p) {
    if (!((f >> p) & 1u)) {
      w[p * n + c] = 0.0;
      continue;
    }
    double t = w[p * n + c];
    for (int i = 0; i < m; ++i) t -= V.a[i] * V.v[i][p * n + c];
    w[p * n + c] = t;
  }
}

// y = a x + b y on the entries with an unknown
__global__ void k_cv_axpby(const uint8_t* flags, long long n, double a, const double* x, double b, double* y) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int p = 0; p < 2; ++p)
    if ((flags[c] >> p) & 1) y[p * n + c] = a * x[p * n + c] + b * y[p * n + c];
    else y[p * n + c] = 0.0;
}
// w = b - r (the operator applied to the vector whose residual r was formed)
__global__ void k_cv_sub(const uint8_t* flags, long long n, const double* b, const double* r, double* w) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int p = 0; p < 2; ++p) w[p * n + c] = ((flags[c] >> p) & 1) ? b[p * n + c] - r[p * n + c] : 0.0;
}

}  // namespace

struct CVec {
  double* c = nullptr;
  double* f = nullptr;
};

struct eb_amr {
  int D = 2;
  BoxIdx B{};
  CFBox cfb{};
  eb_geom_desc dc{}, df{}, df0{};
  std::vector<eb_prim> prims;
  std::vector<eb_csg> nodes;
  eb_geom *Gc = nullptr, *Gf = nullptr, *Gf0 = nullptr;
  eb_poisson *Pc = nullptr, *Pf = nullptr, *Pf0 = nullptr;
  eb_solver_opts o{};
  long long ncc = 0, nff = 0, nface = 0, ncface = 0;
  double hc = 0.0, hf = 0.0, eps0 = 1.0;
  const uint8_t *cflags = nullptr, *fflags = nullptr;  // finest-level flags (owned by the geometries)
  CFFace* faces = nullptr;
  CFCoarse* cfaces = nullptr;
  double *fl = nullptr, *kf = nullptr, *pcf = nullptr, *rc = nullptr, *rf = nullptr, *ec = nullptr, *ef = nullptr;
  int* d_status = nullptr;
  unsigned long long* d_norm = nullptr;
  // FGMRES work space (allocated at the first solve)
  std::vector<CVec> V, Z;
  CVec bvec, tmp;
  double* d_part = nullptr;
  std::vector<void*> allocs;
  long long bytes = 0;
  double *bc0 = nullptr, *bf0 = nullptr;  // b of the coarse and fine operators for the current data
  // persistent solve launches of the last composite solve, coarse [0] and
  // fine [1] correction solvers: launches, kernel ms, V-cycles, FP64 outer iterations
  double kstat[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
};

static void amr_count(eb_amr* A, int which, int cyc, int outer, double ms) {
  A->kstat[which][0] += 1.0;
  A->kstat[which][1] += ms;
  A->kstat[which][2] += cyc;
  A->kstat[which][3] += outer;
}

static eb_status amr_fail(eb_amr* A, eb_status st) {
  eb_amr_destroy(A);
  return st;
}

extern "C" void eb_amr_destroy(eb_amr* A) {
  if (!A) return;
  cudaDeviceSynchronize();
  eb_poisson_destroy(A->Pc);
  eb_poisson_destroy(A->Pf);
  eb_poisson_destroy(A->Pf0);
  eb_geom_destroy(A->Gc);
  eb_geom_destroy(A->Gf);
  eb_geom_destroy(A->Gf0);
  for (void* p : A->allocs) cudaFree(p);
  delete A;
}

extern "C" eb_status eb_amr_setup(const eb_geom_desc* desc, const int box_lo[3], const int box_hi[3],
                                  const eb_solver_opts* opts, void* stream, eb_amr** out) {
  if (!desc || !box_lo || !box_hi || !out) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  *out = nullptr;
  if (desc->n_prims < 0 || desc->n_prims > EB_MAX_PRIMS || desc->n_nodes < 0 || desc->n_nodes > EB_MAX_NODES ||
      (desc->n_prims && !desc->prims) || (desc->n_nodes && !desc->nodes)) {
    set_error("invalid primitive or CSG node list");
    return EB_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  eb_amr* A = new eb_amr();
  A->D = desc->dim;
  const int D = A->D;
  if (D < 2 || D > 3) {
    delete A;
    set_error("dimension must be 2 or 3");
    return EB_ERR_INVALID;
  }
  if (opts) A->o = *opts;
  else eb_solver_opts_default(&A->o);
  A->o.launch_mode = 0;
  A->prims.assign(desc->prims, desc->prims + desc->n_prims);
  A->nodes.assign(desc->nodes, desc->nodes + desc->n_nodes);
  A->dc = *desc;
  A->dc.prims = A->prims.data();
  A->dc.nodes = A->nodes.data();
  BoxIdx& B = A->B;
  B.D = D;
  for (int k = 0; k < 3; ++k) {
    B.nc[k] = k < D ? desc->n[k] : 1;
    B.lo[k] = k < D ? box_lo[k] : 0;
    B.hi[k] = k < D ? box_hi[k] : 1;
    B.nf[k] = k < D ? 2 * (B.hi[k] - B.lo[k]) : 1;
    if (k < D && (B.lo[k] < 0 || B.hi[k] > B.nc[k] || B.hi[k] - B.lo[k] < 4 || (B.hi[k] - B.lo[k]) % 4)) {
      delete A;
      set_error("refined box must lie in the domain with sides a positive multiple of 4 coarse cells");
      return EB_ERR_INVALID;
    }
  }
  // fine grid descriptions: CF sides Neumann (operator) or zero Dirichlet (corrections)
  A->df = A->dc;
  for (int k = 0; k < D; ++k) {
    A->df.n[k] = B.nf[k];
    A->df.lo[k] = desc->lo[k] + B.lo[k] * desc->h;
  }
  A->df.h = desc->h / 2.0;
  A->df0 = A->df;
  for (int k = 0; k < D; ++k)
    for (int s2 = 0; s2 < 2; ++s2) {
      bool cf = s2 == 0 ? B.lo[k] > 0 : B.hi[k] < B.nc[k];
      if (!cf) continue;
      A->df.bc_type[2 * k + s2] = EB_BC_NEUMANN;
      A->df.bc_value[2 * k + s2] = 0.0;
      A->df0.bc_type[2 * k + s2] = EB_BC_DIRICHLET;
      A->df0.bc_value[2 * k + s2] = 0.0;
    }
  A->df0.n_electrodes = desc->n_electrodes;
  for (int e = 0; e < desc->n_electrodes; ++e) A->df0.electrode_phi[e] = 0.0;
  eb_status st = eb_geom_build(&A->dc, stream, &A->Gc);
  if (st == EB_OK) st = eb_geom_build(&A->df, stream, &A->Gf);
  if (st == EB_OK) st = eb_geom_build(&A->df0, stream, &A->Gf0);
  if (st != EB_OK) return amr_fail(A, st);
  A->ncc = A->Gc->L[0].g.ncell;
  A->nff = A->Gf->L[0].g.ncell;
  if (A->ncc >= (1LL << 32) || A->nff >= (1LL << 32)) {  // the composite kernels index cells in 32 bits
    set_error("composite grids are limited to 2^32 cells per level");
    return amr_fail(A, EB_ERR_INVALID);
  }
  A->hc = desc->h;
  A->hf = desc->h / 2.0;
  A->eps0 = desc->eps_gas;
  A->cflags = A->Gc->L[0].flags;
  A->fflags = A->Gf->L[0].flags;
  // CF sides and face counts
  CFBox& cb = A->cfb;
  std::memset(&cb, 0, sizeof(cb));
  for (int k = 0; k < 3; ++k) {
    cb.lo[k] = B.lo[k];
    cb.hi[k] = B.hi[k];
  }
  long long off = 0, coff = 0;
  for (int a = 0; a < D; ++a)
    for (int s2 = 0; s2 < 2; ++s2) {
      bool cf = s2 == 0 ? B.lo[a] > 0 : B.hi[a] < B.nc[a];
      if (!cf) continue;
      long long nfa = 1, nca = 1;
      for (int k = 0; k < D; ++k)
        if (k != a) {
          nfa *= B.nf[k];
          nca *= B.hi[k] - B.lo[k];
        }
      cb.side_a[cb.nside] = a;
      cb.side_s[cb.nside] = s2;
      cb.off[cb.nside] = off;
      cb.coff[cb.nside] = coff;
      ++cb.nside;
      off += nfa;
      coff += nca;
    }
  cb.off[cb.nside] = off;
  cb.coff[cb.nside] = coff;
  A->nface = off;
  A->ncface = coff;
  auto alloc = [&](size_t bytes) { return dev_alloc(A->allocs, std::max<size_t>(bytes, 16), &A->bytes, &st); };
  A->faces = (CFFace*)alloc(sizeof(CFFace) * off);
  A->cfaces = (CFCoarse*)alloc(sizeof(CFCoarse) * coff);
  A->fl = (double*)alloc(sizeof(double) * off);
  A->kf = (double*)alloc(sizeof(double) * 2 * A->nff);
  A->pcf = (double*)alloc(sizeof(double) * 2 * A->ncc);
  A->rc = (double*)alloc(sizeof(double) * 2 * A->ncc);
  A->bc0 = (double*)alloc(sizeof(double) * 2 * A->ncc);
  A->bf0 = (double*)alloc(sizeof(double) * 2 * A->nff);
  A->ec = (double*)alloc(sizeof(double) * 2 * A->ncc);
  A->rf = (double*)alloc(sizeof(double) * 2 * A->nff);
  A->ef = (double*)alloc(sizeof(double) * 2 * A->nff);
  A->d_status = (int*)alloc(sizeof(int));
  A->d_norm = (unsigned long long*)alloc(sizeof(unsigned long long) * 2);
  if (st != EB_OK) return amr_fail(A, st);
  st = build_cf(A->Gf, A->Gc, cb, A->faces, A->cfaces, A->d_status, s);
  if (st != EB_OK) return amr_fail(A, st);
  eb_geom_arrays ga;
  std::memset(&ga, 0, sizeof(ga));
  ga.kappa = A->kf;
  st = eb_geom_export(A->Gf, &ga, stream);
  // a correction inside the preconditioner is one V-cycle of 3+3 sweeps: one
  // inner V-cycle per defect-correction step and a loose tolerance (on the
  // 256^3 + 128^3 pin-plane grid: 21 FGMRES iterations and 285 ms, against 19
  // and 447 ms with two 6+6 V-cycles to 1e-2; 2+2 sweeps needed 23 iterations)
  eb_solver_opts oc = A->o;
  oc.inner_cycles = 1;
  oc.nu1 = oc.nu2 = 3;
  if (st == EB_OK) st = eb_poisson_setup(A->Gc, &oc, stream, &A->Pc);
  if (st == EB_OK) st = eb_poisson_setup(A->Gf, &A->o, stream, &A->Pf);
  if (st == EB_OK) st = eb_poisson_setup(A->Gf0, &oc, stream, &A->Pf0);
  if (st != EB_OK) return amr_fail(A, st);
  if (cudaStreamSynchronize(s) != cudaSuccess) return amr_fail(A, cuda_fail(cudaGetLastError(), "amr setup"));
  *out = A;
  return EB_OK;
}

extern "C" eb_status eb_amr_query(const eb_amr* A, long long* n_coarse, long long* n_fine, int fine_n[3],
                                  long long* cf_faces) {
  if (!A) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  if (n_coarse) *n_coarse = A->ncc;
  if (n_fine) *n_fine = A->nff;
  if (fine_n)
    for (int k = 0; k < 3; ++k) fine_n[k] = A->B.nf[k];
  if (cf_faces) *cf_faces = A->nface;
  return EB_OK;
}

// composite residual into A->rc / A->rf (phi_c values under the box are replaced by fine means)
// b of both operators for the given data, into A->bc0 / A->bf0
static eb_status amr_rhs(eb_amr* A, const double* rhs_c, const double* sig_c, const double* rhs_f,
                         const double* sig_f, cudaStream_t s) {
  eb_status st = poisson_rhs(A->Pc, rhs_c, sig_c, A->bc0, s);
  if (st == EB_OK) st = poisson_rhs(A->Pf, rhs_f, sig_f, A->bf0, s);
  return st;
}

static eb_status amr_resid(eb_amr* A, const double* phi_c, const double* phi_f, cudaStream_t s) {
  cudaMemcpyAsync(A->pcf, phi_c, 2 * A->ncc * sizeof(double), cudaMemcpyDeviceToDevice, s);
  k_avg_down<<<nb(A->ncc), TBA, 0, s>>>(A->B, A->cflags, A->fflags, A->kf, phi_f, A->pcf, A->ncc, A->nff);
  note_launch();
  eb_status st = poisson_residual_view(A->Pc, A->bc0, A->pcf, A->rc, s);
  if (st == EB_OK) st = poisson_residual_view(A->Pf, A->bf0, phi_f, A->rf, s);
  if (st != EB_OK) return st;
  if (A->nface) {
    k_cf_flux<<<nb(A->nface), TBA, 0, s>>>(A->faces, A->nface, A->pcf, phi_f, A->eps0, A->hf, A->fl);
    note_launch();
    for (int sd = 0; sd < A->cfb.nside; ++sd) {
      long long t0 = A->cfb.off[sd], t1 = A->cfb.off[sd + 1];
      k_cf_fine_apply<<<nb(t1 - t0), TBA, 0, s>>>(A->faces, t0, t1, A->fl, A->hf, A->rf);
      note_launch();
    }
    k_cf_coarse_apply<<<nb(A->ncface), TBA, 0, s>>>(A->cfaces, A->ncface, A->fl, A->pcf, A->ncc, A->hc, A->D,
                                                     A->rc);
    note_launch();
  }
  k_zero_under<<<nb(A->ncc), TBA, 0, s>>>(A->B, A->rc, A->ncc);
  note_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? EB_OK : cuda_fail(e, "composite residual");
}

static eb_status amr_norm(eb_amr* A, cudaStream_t s, double* out) {
  cudaMemsetAsync(A->d_norm, 0, sizeof(unsigned long long), s);
  k_absmax2<<<nb(A->ncc), TBA, 0, s>>>(A->cflags, A->ncc, A->rc, A->d_norm);
  note_launch();
  k_absmax2<<<nb(A->nff), TBA, 0, s>>>(A->fflags, A->nff, A->rf, A->d_norm);
  note_launch();
  unsigned long long v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, A->d_norm, sizeof(v), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "composite norm");
  std::memcpy(out, &v, sizeof(double));
  return EB_OK;
}

extern "C" eb_status eb_amr_residual(eb_amr* A, const double* d_rhs_c, const double* d_sig_c, const double* d_rhs_f,
                                     const double* d_sig_f, const double* d_phi_c, const double* d_phi_f,
                                     double* d_r_c, double* d_r_f, void* stream) {
  if (!A || !d_rhs_c || !d_rhs_f || !d_phi_c || !d_phi_f || !d_r_c || !d_r_f) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  eb_status st = amr_rhs(A, d_rhs_c, d_sig_c, d_rhs_f, d_sig_f, s);
  if (st == EB_OK) st = amr_resid(A, d_phi_c, d_phi_f, s);
  if (st != EB_OK) return st;
  cudaMemcpyAsync(d_r_c, A->rc, 2 * A->ncc * sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(d_r_f, A->rf, 2 * A->nff * sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaError_t e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? EB_OK : cuda_fail(e, "composite residual");
}

static double cv_dot(eb_amr* A, const CVec& a, const CVec& b, cudaStream_t s) {
  k_cv_dot<<<DOT_BLOCKS, TBA, 0, s>>>(A->B, A->cflags, A->ncc, 1, a.c, b.c, A->d_part);
  note_launch();
  k_cv_dot<<<DOT_BLOCKS, TBA, 0, s>>>(A->B, A->fflags, A->nff, 0, a.f, b.f, A->d_part + DOT_BLOCKS);
  note_launch();
  double h[2 * DOT_BLOCKS];
  cudaMemcpyAsync(h, A->d_part, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  double t = 0.0;
  for (int i = 0; i < 2 * DOT_BLOCKS; ++i) t += h[i];
  return t;
}
static void cv_axpby(eb_amr* A, double a, const CVec& x, double b, const CVec& y, cudaStream_t s) {
  k_cv_axpby<<<nb(A->ncc), TBA, 0, s>>>(A->cflags, A->ncc, a, x.c, b, y.c);
  note_launch();
  k_cv_axpby<<<nb(A->nff), TBA, 0, s>>>(A->fflags, A->nff, a, x.f, b, y.f);
  note_launch();
}

// h[i] = (V[i], w) for i < m, both grids, one launch per grid and one sync;
// with `self` also h[m] = (w, w), from the same pass over w
static void cv_mdot(eb_amr* A, int m, const CVec& w, double* h, cudaStream_t s, bool self = false) {
  CVPtrs pc{}, pf{};
  for (int i = 0; i < m; ++i) {
    pc.v[i] = A->V[i].c;
    pf.v[i] = A->V[i].f;
  }
  if (self) {
    pc.v[m] = w.c;
    pf.v[m] = w.f;
    ++m;
  }
  k_cv_mdot<<<DOT_BLOCKS, TBA, 0, s>>>(A->B, A->cflags, A->ncc, 1, m, pc, w.c, A->d_part);
  note_launch();
  k_cv_mdot<<<DOT_BLOCKS, TBA, 0, s>>>(A->B, A->fflags, A->nff, 0, m, pf, w.f, A->d_part + CV_MAXV * DOT_BLOCKS);
  note_launch();
  std::vector<double> hp(2 * CV_MAXV * DOT_BLOCKS);
  cudaMemcpyAsync(hp.data(), A->d_part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  for (int i = 0; i < m; ++i) {
    double t = 0.0;
    for (int b = 0; b < DOT_BLOCKS; ++b) t += hp[i * DOT_BLOCKS + b];
    for (int b = 0; b < DOT_BLOCKS; ++b) t += hp[CV_MAXV * DOT_BLOCKS + i * DOT_BLOCKS + b];
    h[i] = t;
  }
}
// w -= sum_{i < m} h[i] V[i]
static void cv_maxpy(eb_amr* A, int m, const double* h, const CVec& w, cudaStream_t s) {
  CVPtrs pc{}, pf{};
  for (int i = 0; i < m; ++i) {
    pc.v[i] = A->V[i].c;
    pf.v[i] = A->V[i].f;
    pc.a[i] = pf.a[i] = h[i];
  }
  k_cv_maxpy<<<nb(A->ncc), TBA, 0, s>>>(A->cflags, A->ncc, m, pc, w.c);
  note_launch();
  k_cv_maxpy<<<nb(A->nff), TBA, 0, s>>>(A->fflags, A->nff, m, pf, w.f);
  note_launch();
}

// accuracy asked of the two multigrid corrections inside one FAC step: loose
// enough that each stops after its first V-cycle
constexpr double FAC_TOL = 3e-1;

// z = M^-1 v: one FAC step from zero (coarse correction over the domain,
// constant per parent on the box, then a fine correction of what remains);
// uses A->rc / rf / ec / ef / tmp as scratch.
static eb_status fac_apply(eb_amr* A, const CVec& v, const CVec& z, int* cycles, cudaStream_t s) {
  const double tol = FAC_TOL;
  cudaMemcpyAsync(A->rc, v.c, 2 * A->ncc * sizeof(double), cudaMemcpyDeviceToDevice, s);
  k_zero_under<<<nb(A->ncc), TBA, 0, s>>>(A->B, A->rc, A->ncc);
  note_launch();
  k_restrict_under<<<nb(A->ncc), TBA, 0, s>>>(A->B, A->fflags, v.f, A->rc, A->ncc, A->nff);
  note_launch();
  int cyc = 0, outer = 0;
  double kms = 0.0;
  eb_status st = poisson_solve_b(A->Pc, A->rc, A->ec, tol, &cyc, s, &outer, &kms);
  *cycles += cyc;
  amr_count(A, 0, cyc, outer, kms);
  if (st != EB_OK) return st;
  cudaMemsetAsync(z.c, 0, 2 * A->ncc * sizeof(double), s);
  cudaMemsetAsync(z.f, 0, 2 * A->nff * sizeof(double), s);
  k_add_coarse<<<nb(A->ncc), TBA, 0, s>>>(A->B, A->ec, z.c, A->ncc);
  note_launch();
  k_prolong_const<<<nb(A->nff), TBA, 0, s>>>(A->B, A->fflags, A->ec, z.f, A->ncc, A->nff);
  note_launch();
  // what remains on the box: v_f - (A z)_f = v_f - b_f + r_f(z)
  st = amr_resid(A, z.c, z.f, s);
  if (st != EB_OK) return st;
  k_cv_sub<<<nb(A->nff), TBA, 0, s>>>(A->fflags, A->nff, A->bvec.f, A->rf, A->tmp.f);  // (A z)_f
  note_launch();
  k_cv_axpby<<<nb(A->nff), TBA, 0, s>>>(A->fflags, A->nff, 1.0, v.f, -1.0, A->tmp.f);  // v_f - (A z)_f
  note_launch();
  st = poisson_solve_b(A->Pf0, A->tmp.f, A->ef, tol, &cyc, s, &outer, &kms);
  *cycles += cyc;
  amr_count(A, 1, cyc, outer, kms);
  if (st != EB_OK) return st;
  k_axpy_masked<<<nb(A->nff), TBA, 0, s>>>(A->fflags, A->nff, A->ef, z.f);
  note_launch();
  return EB_OK;
}

// w = A z (homogeneous operator) = b - r(z)
static eb_status op_apply(eb_amr* A, const CVec& z, const CVec& w, cudaStream_t s) {
  eb_status st = amr_resid(A, z.c, z.f, s);
  if (st != EB_OK) return st;
  k_cv_sub<<<nb(A->ncc), TBA, 0, s>>>(A->cflags, A->ncc, A->bvec.c, A->rc, w.c);
  note_launch();
  k_zero_under<<<nb(A->ncc), TBA, 0, s>>>(A->B, w.c, A->ncc);
  note_launch();
  k_cv_sub<<<nb(A->nff), TBA, 0, s>>>(A->fflags, A->nff, A->bvec.f, A->rf, w.f);
  note_launch();
  return EB_OK;
}

static constexpr int GM = 12;  // FGMRES restart length

static eb_status amr_workspace(eb_amr* A) {
  if (!A->V.empty()) return EB_OK;
  eb_status st = EB_OK;
  auto vec = [&]() {
    CVec v;
    v.c = (double*)dev_alloc(A->allocs, 2 * A->ncc * sizeof(double), &A->bytes, &st);
    v.f = (double*)dev_alloc(A->allocs, 2 * A->nff * sizeof(double), &A->bytes, &st);
    return v;
  };
  for (int i = 0; i <= GM; ++i) A->V.push_back(vec());
  for (int i = 0; i < GM; ++i) A->Z.push_back(vec());
  A->bvec = vec();
  A->tmp = vec();
  A->d_part = (double*)dev_alloc(A->allocs, 2 * CV_MAXV * DOT_BLOCKS * sizeof(double), &A->bytes, &st);
  if (st != EB_OK) {
    A->V.clear();
    A->Z.clear();
  }
  return st;
}

extern "C" eb_status eb_amr_solve(eb_amr* A, const double* d_rhs_c, const double* d_sig_c, const double* d_rhs_f,
                                  const double* d_sig_f, double* d_phi_c, double* d_phi_f, eb_solve_info* info,
                                  void* stream) {
  if (!A || !d_rhs_c || !d_rhs_f || !d_phi_c || !d_phi_f) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  eb_solve_info inf;
  std::memset(&inf, 0, sizeof(inf));
  std::memset(A->kstat, 0, sizeof(A->kstat));
  const long long launches0 = launch_total();
  eb_status st = amr_workspace(A);
  if (st != EB_OK) return st;
  // b: the composite residual at phi = 0
  cudaMemsetAsync(A->ec, 0, 2 * A->ncc * sizeof(double), s);
  cudaMemsetAsync(A->ef, 0, 2 * A->nff * sizeof(double), s);
  st = amr_rhs(A, d_rhs_c, d_sig_c, d_rhs_f, d_sig_f, s);
  if (st == EB_OK) st = amr_resid(A, A->ec, A->ef, s);
  double bn = 0.0, r = 0.0;
  if (st == EB_OK) st = amr_norm(A, s, &bn);
  if (st != EB_OK) return st;
  cudaMemcpyAsync(A->bvec.c, A->rc, 2 * A->ncc * sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(A->bvec.f, A->rf, 2 * A->nff * sizeof(double), cudaMemcpyDeviceToDevice, s);
  const CVec x{d_phi_c, d_phi_f};
  int it = 0, cycles = 0;
  const int max_it = std::max(1, A->o.max_cycles);
  // restarted FGMRES, right-preconditioned by one FAC step (Sec. 3.3.2's
  // multigrid as the inner solver of every correction)
  st = EB_ERR_NOT_CONVERGED;
  while (it < max_it) {
    eb_status s2 = amr_resid(A, x.c, x.f, s);
    if (s2 == EB_OK) s2 = amr_norm(A, s, &r);
    if (s2 != EB_OK) {
      st = s2;
      break;
    }
    if (bn == 0.0 || r <= A->o.tol * bn) {
      st = EB_OK;
      break;
    }
    if (!(r == r) || r > 1e6 * bn) break;
    // v0 = r / |r|_2
    cudaMemcpyAsync(A->V[0].c, A->rc, 2 * A->ncc * sizeof(double), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(A->V[0].f, A->rf, 2 * A->nff * sizeof(double), cudaMemcpyDeviceToDevice, s);
    k_zero_under<<<nb(A->ncc), TBA, 0, s>>>(A->B, A->V[0].c, A->ncc);
    note_launch();
    double beta = std::sqrt(cv_dot(A, A->V[0], A->V[0], s));
    if (!(beta > 0.0)) {
      st = EB_OK;
      break;
    }
    cv_axpby(A, 0.0, A->V[0], 1.0 / beta, A->V[0], s);
    // this cycle's target in the 2-norm estimate: the reduction the max norm
    // still needs, with a factor 1/2 of margin
    const double target = 0.5 * (A->o.tol * bn / r) * beta;
    double H[GM + 1][GM], cs[GM], sn[GM], g[GM + 1];
    std::memset(H, 0, sizeof(H));
    std::memset(g, 0, sizeof(g));
    g[0] = beta;
    int k = 0;
    for (; k < GM && it < max_it; ++k, ++it) {
      s2 = fac_apply(A, A->V[k], A->Z[k], &cycles, s);
      if (s2 == EB_OK) s2 = op_apply(A, A->Z[k], A->V[k + 1], s);
      if (s2 != EB_OK) break;
      // classical Gram-Schmidt, all k + 1 projections in one pass, repeated
      // only when the pass removed most of w (the criterion of Daniel, Gragg,
      // Kaufman and Stewart: the new norm below 1/sqrt(2) of the old one,
      // where cancellation may have left w short of orthogonal)
      for (int i = 0; i <= k; ++i) H[i][k] = 0.0;
      double hp[CV_MAXV];
      cv_mdot(A, k + 1, A->V[k + 1], hp, s, true);  // (V_i, w) and (w, w)
      const double w0 = std::sqrt(std::max(hp[k + 1], 0.0));
      cv_maxpy(A, k + 1, hp, A->V[k + 1], s);
      for (int i = 0; i <= k; ++i) H[i][k] += hp[i];
      double w1 = std::sqrt(cv_dot(A, A->V[k + 1], A->V[k + 1], s));
      if (w1 < w0 / std::sqrt(2.0)) {
        cv_mdot(A, k + 1, A->V[k + 1], hp, s);
        cv_maxpy(A, k + 1, hp, A->V[k + 1], s);
        for (int i = 0; i <= k; ++i) H[i][k] += hp[i];
        w1 = std::sqrt(cv_dot(A, A->V[k + 1], A->V[k + 1], s));
      }
      H[k + 1][k] = w1;
      if (H[k + 1][k] > 0.0) cv_axpby(A, 0.0, A->V[k + 1], 1.0 / H[k + 1][k], A->V[k + 1], s);
      for (int i = 0; i < k; ++i) {  // earlier rotations
        double t = cs[i] * H[i][k] + sn[i] * H[i + 1][k];
        H[i + 1][k] = -sn[i] * H[i][k] + cs[i] * H[i + 1][k];
        H[i][k] = t;
      }
      double den = std::hypot(H[k][k], H[k + 1][k]);
      cs[k] = den > 0.0 ? H[k][k] / den : 1.0;
      sn[k] = den > 0.0 ? H[k + 1][k] / den : 0.0;
      H[k][k] = den;
      H[k + 1][k] = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      // the 2-norm estimate far below the target: stop the cycle and check the true max norm
      if (std::fabs(g[k + 1]) <= target) {
        ++k;
        ++it;
        break;
      }
    }
    if (s2 != EB_OK) {
      st = s2;
      break;
    }
    // x += Z y with H y = g (upper triangular)
    double y[GM];
    for (int i = k - 1; i >= 0; --i) {
      double t = g[i];
      for (int j = i + 1; j < k; ++j) t -= H[i][j] * y[j];
      y[i] = H[i][i] != 0.0 ? t / H[i][i] : 0.0;
    }
    for (int i = 0; i < k; ++i) cv_axpby(A, y[i], A->Z[i], 1.0, x, s);
  }
  // report phi_c under the box as the fine means
  if (st == EB_OK || st == EB_ERR_NOT_CONVERGED) {
    k_avg_down<<<nb(A->ncc), TBA, 0, s>>>(A->B, A->cflags, A->fflags, A->kf, d_phi_f, d_phi_c, A->ncc, A->nff);
    note_launch();
    if (st == EB_ERR_NOT_CONVERGED) set_error("composite iteration cap reached");
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess && st == EB_OK) st = cuda_fail(e, "composite solve");
  inf.status = st;
  inf.outer_iters = it;
  inf.vcycles = cycles;
  inf.bnorm = bn;
  inf.rel_res = bn > 0.0 ? r / bn : 0.0;
  inf.kernel_ms = A->kstat[0][1] + A->kstat[1][1];
  inf.kernel_launches = launch_total() - launches0;
  if (info) *info = inf;
  return st;
}

extern "C" eb_status eb_amr_kernel_stats(const eb_amr* A, double out[8]) {
  if (!A || !out) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  for (int w = 0; w < 2; ++w)
    for (int k = 0; k < 4; ++k) out[4 * w + k] = A->kstat[w][k];
  return EB_OK;
}

// amr.cu -- composite multi-level solve: nested ratio-2 refined boxes, one
// per level (Sec. 3.3.2 runs its multigrid over refined levels; the
// coarse-fine coupling of each pair of levels follows the refluxing of
// Sec. 3.3).
//
// Composite operator (the same reading as the oracle's):
//   * every box is a grid of its own whose coarse-fine (CF) sides are
//     homogeneous Neumann walls; the CF flux eps0 (ghost - phi_F)/h_f times the
//     fine aperture is added to each fine cell next to a CF side, the ghost by
//     quadratic tangential then quadratic normal Lagrange steps (fallbacks to
//     linear, then constant) precomputed per face at set-up;
//   * a coarse cell outside the box next to a CF side loses the coarse
//     operator's own flux through that face and gains minus the mean of the
//     fine fluxes through it (refluxing: exact conservation);
//   * cells under the next finer box carry no equation; where a stencil
//     reaches one, its value is the kappa-weighted mean of its children, which
//     are such means themselves under a still finer box;
//   * each box keeps one parent cell away from its parent's CF sides (proper
//     nesting), so every coarse cell across a CF face carries an equation.
// Solve: restarted FGMRES in FP64 on the composite system, right-
// preconditioned by one multiplicative FAC sweep from level 0 up: a level-0
// correction over the whole domain (the finer parts of the vector restricted
// under the boxes), added constant per parent on level 1, then on every finer
// level a correction of what remains there with zero Dirichlet data on its CF
// sides.  Every correction runs one V-cycle of the persistent multigrid
// kernel; dot products are summed in a fixed order (deterministic).
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
// coarse cells under the box: the launch size of the passes that touch only them
long long box_cells(const BoxIdx& B) {
  return (long long)(B.hi[0] - B.lo[0]) * (B.hi[1] - B.lo[1]) * (B.hi[2] - B.lo[2]);
}

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
// the t-th coarse cell under the box (x fastest); false past the last one.
// Passes that only touch the cells under the box launch over these alone.
__device__ __forceinline__ bool box_cell(const BoxIdx& B, long long t, int I[3]) {
  const unsigned e0 = (unsigned)(B.hi[0] - B.lo[0]), e1 = (unsigned)(B.hi[1] - B.lo[1]);
  const unsigned e2 = (unsigned)(B.hi[2] - B.lo[2]);
  if (t >= (long long)e0 * e1 * e2) return false;
  const unsigned tu = (unsigned)t, r = tu / e0;
  I[0] = B.lo[0] + (int)(tu - r * e0);
  I[1] = B.lo[1] + (int)(r % e1);
  I[2] = B.lo[2] + (int)(r / e1);
  return true;
}

// coarse values under the box: kappa-weighted mean of the children with the phase
__global__ void k_avg_down(BoxIdx B, const uint8_t* cflags, const uint8_t* fflags, const double* kf, const double* pf,
                           double* pc, long long ncc, long long nff) {
  int I[3];
  if (!box_cell(B, (long long)blockIdx.x * blockDim.x + threadIdx.x, I)) return;
  const long long c = lin3(B.nc, I);
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
  int I[3];
  if (!box_cell(B, (long long)blockIdx.x * blockDim.x + threadIdx.x, I)) return;
  const long long c = lin3(B.nc, I);
  rc[c] = rc[ncc + c] = 0.0;
}

// coarse correction right-hand side under the box: mean fine residual of the
// children carrying the phase
__global__ void k_restrict_under(BoxIdx B, const uint8_t* fflags, const double* rf, double* rc, long long ncc,
                                 long long nff) {
  int I[3];
  if (!box_cell(B, (long long)blockIdx.x * blockDim.x + threadIdx.x, I)) return;
  const long long c = lin3(B.nc, I);
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
// w -= sum_i a_i v_i on the entries with an unknown (others 0), and from the
// same pass the per-block partial sums of the new w . w over the entries a
// dot product counts (the caller adds the blocks in order: deterministic)
__global__ void k_cv_maxpy_norm(BoxIdx B, const uint8_t* flags, long long n, int coarse, int m, CVPtrs V, double* w,
                                double* part) {
  __shared__ double sh[TBA];
  double acc = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    bool counted = true;
    if (coarse) {
      int I[3];
      ijk3(B.nc, c, I);
      counted = !under_box(B, I);
    }
    const unsigned f = flags[c];
    for (int p = 0; p < 2; ++p) {
      if (!((f >> p) & 1u)) {
        w[p * n + c] = 0.0;
        continue;
      }
      double t = w[p * n + c];
#pragma unroll
      for (int i = 0; i < CV_MAXV; ++i)
        if (i < m) t -= V.a[i] * V.v[i][p * n + c];
      w[p * n + c] = t;
      if (counted) acc += t * t;
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
    if ((int)threadIdx.x < s2) sh[threadIdx.x] += sh[threadIdx.x + s2];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
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

constexpr int AMR_MAXL = EB_AMR_MAX_LEVELS;

// A composite vector: one [2][n_l] array per level (entries under the next
// finer box and without an unknown ignored)
struct CVec {
  double* v[AMR_MAXL] = {};
};

// One level: its grid as an operator (CF sides homogeneous Neumann) and, from
// level 1 on, as a correction grid (CF sides zero Dirichlet)
struct AmrLevel {
  eb_geom_desc d{}, d0{};
  eb_geom *G = nullptr, *G0 = nullptr;
  eb_poisson *P = nullptr, *P0 = nullptr;  // level 0: P0 == P
  long long n = 0;
  double h = 0.0;
  const uint8_t* flags = nullptr;  // finest-level flags of G (owned by G)
  double *pc = nullptr;            // phi with the cells under the next box replaced by the finer means
  double *r = nullptr, *b0 = nullptr, *e = nullptr, *kap = nullptr;
};

// The coupling of levels l-1 (coarse) and l (fine), stored at index l
struct AmrPair {
  BoxIdx B{};
  CFBox cfb{};
  long long nface = 0, ncface = 0;
  CFFace* faces = nullptr;
  CFCoarse* cfaces = nullptr;
  double* fl = nullptr;
};

struct eb_amr {
  int D = 2, L = 2;
  AmrLevel lv[AMR_MAXL];
  AmrPair pr[AMR_MAXL];
  std::vector<eb_prim> prims;
  std::vector<eb_csg> nodes;
  eb_solver_opts o{};
  double eps0 = 1.0;
  int* d_status = nullptr;
  unsigned long long* d_norm = nullptr;
  // FGMRES work space (allocated at the first solve)
  std::vector<CVec> V, Z;
  CVec bvec, tmp;
  double* d_part = nullptr;
  std::vector<void*> allocs;
  long long bytes = 0;
  // persistent solve launches of the last composite solve, coarse [0] and
  // finer levels' [1] correction solvers: launches, kernel ms, V-cycles, FP64 outer iterations
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
  for (int l = 0; l < AMR_MAXL; ++l) {
    AmrLevel& v = A->lv[l];
    if (v.P0 != v.P) eb_poisson_destroy(v.P0);
    eb_poisson_destroy(v.P);
    eb_geom_destroy(v.G0);
    eb_geom_destroy(v.G);
  }
  for (void* p : A->allocs) cudaFree(p);
  delete A;
}

// is side s2 of axis k of the box of pair B a CF side (inside its parent grid)?
static bool cf_side(const BoxIdx& B, int k, int s2) { return s2 == 0 ? B.lo[k] > 0 : B.hi[k] < B.nc[k]; }

extern "C" eb_status eb_amr_setup_levels(const eb_geom_desc* desc, int n_levels, const int* box_lo,
                                         const int* box_hi, const eb_solver_opts* opts, void* stream,
                                         eb_amr** out) {
  if (!desc || !box_lo || !box_hi || !out) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  *out = nullptr;
  if (n_levels < 2 || n_levels > AMR_MAXL) {
    set_error("a composite grid has 2 to " + std::to_string(AMR_MAXL) + " levels");
    return EB_ERR_INVALID;
  }
  if (desc->n_prims < 0 || desc->n_prims > EB_MAX_PRIMS || desc->n_nodes < 0 || desc->n_nodes > EB_MAX_NODES ||
      (desc->n_prims && !desc->prims) || (desc->n_nodes && !desc->nodes)) {
    set_error("invalid primitive or CSG node list");
    return EB_ERR_INVALID;
  }
  if (desc->dim < 2 || desc->dim > 3) {
    set_error("dimension must be 2 or 3");
    return EB_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  eb_amr* A = new eb_amr();
  A->D = desc->dim;
  A->L = n_levels;
  const int D = A->D, L = A->L;
  if (opts) A->o = *opts;
  else eb_solver_opts_default(&A->o);
  A->o.launch_mode = 0;
  A->prims.assign(desc->prims, desc->prims + desc->n_prims);
  A->nodes.assign(desc->nodes, desc->nodes + desc->n_nodes);
  A->lv[0].d = *desc;
  A->lv[0].d.prims = A->prims.data();
  A->lv[0].d.nodes = A->nodes.data();
  // level descriptions: each box over cells [lo, hi) of its parent's grid
  for (int l = 1; l < L; ++l) {
    const eb_geom_desc& pd = A->lv[l - 1].d;
    BoxIdx& B = A->pr[l].B;
    const int* lo = box_lo + 3 * (l - 1);
    const int* hi = box_hi + 3 * (l - 1);
    B.D = D;
    for (int k = 0; k < 3; ++k) {
      B.nc[k] = k < D ? pd.n[k] : 1;
      B.lo[k] = k < D ? lo[k] : 0;
      B.hi[k] = k < D ? hi[k] : 1;
      B.nf[k] = k < D ? 2 * (B.hi[k] - B.lo[k]) : 1;
      if (k < D && (B.lo[k] < 0 || B.hi[k] > B.nc[k] || B.hi[k] - B.lo[k] < 4 || (B.hi[k] - B.lo[k]) % 4)) {
        delete A;
        set_error("the box of level " + std::to_string(l) +
                  " must lie in its parent grid with sides a positive multiple of 4 parent cells");
        return EB_ERR_INVALID;
      }
    }
    // proper nesting: one parent cell between the box and each CF side of the parent
    if (l >= 2)
      for (int k = 0; k < D; ++k) {
        const BoxIdx& PB = A->pr[l - 1].B;
        if ((cf_side(PB, k, 0) && B.lo[k] < 1) || (cf_side(PB, k, 1) && B.hi[k] > B.nc[k] - 1)) {
          delete A;
          set_error("the box of level " + std::to_string(l) +
                    " must keep one parent cell away from every coarse-fine side of its parent");
          return EB_ERR_INVALID;
        }
      }
    eb_geom_desc& d = A->lv[l].d;
    d = pd;
    for (int k = 0; k < D; ++k) {
      d.n[k] = B.nf[k];
      d.lo[k] = pd.lo[k] + B.lo[k] * pd.h;
    }
    d.h = pd.h / 2.0;
    // sides on the domain boundary keep the parent's (domain) conditions
    eb_geom_desc& d0 = A->lv[l].d0;
    d0 = d;
    for (int k = 0; k < D; ++k)
      for (int s2 = 0; s2 < 2; ++s2) {
        if (!cf_side(B, k, s2)) continue;
        d.bc_type[2 * k + s2] = EB_BC_NEUMANN;
        d.bc_value[2 * k + s2] = 0.0;
        d0.bc_type[2 * k + s2] = EB_BC_DIRICHLET;
        d0.bc_value[2 * k + s2] = 0.0;
      }
    d0.n_electrodes = pd.n_electrodes;
    for (int e = 0; e < pd.n_electrodes; ++e) d0.electrode_phi[e] = 0.0;
  }
  eb_status st = EB_OK;
  for (int l = 0; l < L && st == EB_OK; ++l) {
    st = eb_geom_build(&A->lv[l].d, stream, &A->lv[l].G);
    if (st == EB_OK && l > 0) st = eb_geom_build(&A->lv[l].d0, stream, &A->lv[l].G0);
  }
  if (st != EB_OK) return amr_fail(A, st);
  for (int l = 0; l < L; ++l) {
    AmrLevel& v = A->lv[l];
    v.n = v.G->L[0].g.ncell;
    v.h = v.d.h;
    v.flags = v.G->L[0].flags;
    if (v.n >= (1LL << 32)) {  // the composite kernels index cells in 32 bits
      set_error("composite grids are limited to 2^32 cells per level");
      return amr_fail(A, EB_ERR_INVALID);
    }
  }
  A->eps0 = desc->eps_gas;
  auto alloc = [&](size_t bytes) { return dev_alloc(A->allocs, std::max<size_t>(bytes, 16), &A->bytes, &st); };
  // CF sides and face counts of every pair
  for (int l = 1; l < L; ++l) {
    AmrPair& P = A->pr[l];
    const BoxIdx& B = P.B;
    CFBox& cb = P.cfb;
    std::memset(&cb, 0, sizeof(cb));
    for (int k = 0; k < 3; ++k) {
      cb.lo[k] = B.lo[k];
      cb.hi[k] = B.hi[k];
    }
    long long off = 0, coff = 0;
    for (int a = 0; a < D; ++a)
      for (int s2 = 0; s2 < 2; ++s2) {
        if (!cf_side(B, a, s2)) continue;
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
    P.nface = off;
    P.ncface = coff;
    P.faces = (CFFace*)alloc(sizeof(CFFace) * off);
    P.cfaces = (CFCoarse*)alloc(sizeof(CFCoarse) * coff);
    P.fl = (double*)alloc(sizeof(double) * off);
  }
  for (int l = 0; l < L; ++l) {
    AmrLevel& v = A->lv[l];
    const size_t b2 = sizeof(double) * 2 * v.n;
    if (l < L - 1) v.pc = (double*)alloc(b2);
    if (l > 0) v.kap = (double*)alloc(b2);
    v.r = (double*)alloc(b2);
    v.b0 = (double*)alloc(b2);
    v.e = (double*)alloc(b2);
  }
  A->d_status = (int*)alloc(sizeof(int));
  A->d_norm = (unsigned long long*)alloc(sizeof(unsigned long long) * 2);
  if (st != EB_OK) return amr_fail(A, st);
  for (int l = 1; l < L && st == EB_OK; ++l) {
    AmrPair& P = A->pr[l];
    st = build_cf(A->lv[l].G, A->lv[l - 1].G, P.cfb, P.faces, P.cfaces, A->d_status, s);
    if (st != EB_OK) break;
    eb_geom_arrays ga;
    std::memset(&ga, 0, sizeof(ga));
    ga.kappa = A->lv[l].kap;
    st = eb_geom_export(A->lv[l].G, &ga, stream);
  }
  if (st != EB_OK) return amr_fail(A, st);
  // a correction inside the preconditioner is one V-cycle of 3+3 sweeps: one
  // inner V-cycle per defect-correction step and a loose tolerance (on the
  // 256^3 + 128^3 pin-plane grid: 21 FGMRES iterations and 285 ms, against 19
  // and 447 ms with two 6+6 V-cycles to 1e-2; 2+2 sweeps needed 23 iterations).
  // A relaxed bottom takes at most 32 sweeps there: the same 21 iterations in
  // 243 ms against 252 ms with 64; 16 sweeps needed 23 iterations (261 ms).
  eb_solver_opts oc = A->o;
  oc.inner_cycles = 1;
  oc.nu1 = oc.nu2 = 3;
  oc.bottom_sweeps = std::min(oc.bottom_sweeps, 32);
  st = eb_poisson_setup(A->lv[0].G, &oc, stream, &A->lv[0].P);
  A->lv[0].P0 = A->lv[0].P;
  for (int l = 1; l < L && st == EB_OK; ++l) {
    st = eb_poisson_setup(A->lv[l].G, &A->o, stream, &A->lv[l].P);
    if (st == EB_OK) st = eb_poisson_setup(A->lv[l].G0, &oc, stream, &A->lv[l].P0);
  }
  if (st != EB_OK) return amr_fail(A, st);
  if (cudaStreamSynchronize(s) != cudaSuccess) return amr_fail(A, cuda_fail(cudaGetLastError(), "amr setup"));
  *out = A;
  return EB_OK;
}

extern "C" eb_status eb_amr_setup(const eb_geom_desc* desc, const int box_lo[3], const int box_hi[3],
                                  const eb_solver_opts* opts, void* stream, eb_amr** out) {
  return eb_amr_setup_levels(desc, 2, box_lo, box_hi, opts, stream, out);
}

extern "C" eb_status eb_amr_query(const eb_amr* A, long long* n_coarse, long long* n_fine, int fine_n[3],
                                  long long* cf_faces) {
  if (!A) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  if (n_coarse) *n_coarse = A->lv[0].n;
  if (n_fine) *n_fine = A->lv[1].n;
  if (fine_n)
    for (int k = 0; k < 3; ++k) fine_n[k] = A->pr[1].B.nf[k];
  if (cf_faces) *cf_faces = A->pr[1].nface;
  return EB_OK;
}

extern "C" eb_status eb_amr_level_query(const eb_amr* A, int level, int* n_levels, long long* n_cells, int n[3],
                                        double lo[3], double* h, long long* cf_faces) {
  if (!A || level < 0 || level >= A->L) {
    set_error(A ? "level out of range" : "null argument");
    return EB_ERR_INVALID;
  }
  const AmrLevel& v = A->lv[level];
  if (n_levels) *n_levels = A->L;
  if (n_cells) *n_cells = v.n;
  for (int k = 0; k < 3; ++k) {
    if (n) n[k] = k < A->D ? v.d.n[k] : 1;
    if (lo) lo[k] = k < A->D ? v.d.lo[k] : 0.0;
  }
  if (h) *h = v.h;
  if (cf_faces) *cf_faces = level > 0 ? A->pr[level].nface : 0;
  return EB_OK;
}

extern "C" eb_status eb_amr_level_geom(const eb_amr* A, int level, const eb_geom** out) {
  if (!A || !out || level < 0 || level >= A->L) {
    set_error(A && out ? "level out of range" : "null argument");
    return EB_ERR_INVALID;
  }
  *out = A->lv[level].G;
  return EB_OK;
}

// b of every level's operator for the given data, into lv[l].b0
static eb_status amr_rhs(eb_amr* A, const double* const* rhs, const double* const* sig, cudaStream_t s) {
  eb_status st = EB_OK;
  for (int l = 0; l < A->L && st == EB_OK; ++l)
    st = poisson_rhs(A->lv[l].P, rhs[l], sig ? sig[l] : nullptr, A->lv[l].b0, s);
  return st;
}

// composite residual into lv[l].r: every level's values under the next finer
// box are first replaced by the finer level's means, finest first
static eb_status amr_resid(eb_amr* A, const double* const* phi, cudaStream_t s) {
  const int L = A->L;
  const double* val[AMR_MAXL];
  val[L - 1] = phi[L - 1];
  for (int l = L - 2; l >= 0; --l) {
    AmrLevel &c = A->lv[l], &f = A->lv[l + 1];
    cudaMemcpyAsync(c.pc, phi[l], 2 * c.n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    k_avg_down<<<nb(box_cells(A->pr[l + 1].B)), TBA, 0, s>>>(A->pr[l + 1].B, c.flags, f.flags, f.kap, val[l + 1],
                                                            c.pc, c.n, f.n);
    note_launch();
    val[l] = c.pc;
  }
  eb_status st = EB_OK;
  for (int l = 0; l < L && st == EB_OK; ++l) st = poisson_residual_view(A->lv[l].P, A->lv[l].b0, val[l], A->lv[l].r, s);
  if (st != EB_OK) return st;
  for (int l = 1; l < L; ++l) {
    const AmrPair& P = A->pr[l];
    AmrLevel &c = A->lv[l - 1], &f = A->lv[l];
    if (!P.nface) continue;
    k_cf_flux<<<nb(P.nface), TBA, 0, s>>>(P.faces, P.nface, val[l - 1], val[l], A->eps0, f.h, P.fl);
    note_launch();
    for (int sd = 0; sd < P.cfb.nside; ++sd) {
      long long t0 = P.cfb.off[sd], t1 = P.cfb.off[sd + 1];
      k_cf_fine_apply<<<nb(t1 - t0), TBA, 0, s>>>(P.faces, t0, t1, P.fl, f.h, f.r);
      note_launch();
    }
    k_cf_coarse_apply<<<nb(P.ncface), TBA, 0, s>>>(P.cfaces, P.ncface, P.fl, val[l - 1], c.n, c.h, A->D, c.r);
    note_launch();
  }
  for (int l = 1; l < L; ++l) {
    k_zero_under<<<nb(box_cells(A->pr[l].B)), TBA, 0, s>>>(A->pr[l].B, A->lv[l - 1].r, A->lv[l - 1].n);
    note_launch();
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? EB_OK : cuda_fail(e, "composite residual");
}

static eb_status amr_norm(eb_amr* A, cudaStream_t s, double* out) {
  cudaMemsetAsync(A->d_norm, 0, sizeof(unsigned long long), s);
  for (int l = 0; l < A->L; ++l) {
    k_absmax2<<<nb(A->lv[l].n), TBA, 0, s>>>(A->lv[l].flags, A->lv[l].n, A->lv[l].r, A->d_norm);
    note_launch();
  }
  unsigned long long v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, A->d_norm, sizeof(v), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "composite norm");
  std::memcpy(out, &v, sizeof(double));
  return EB_OK;
}

static bool all_set(const double* const* p, int n) {
  if (!p) return false;
  for (int l = 0; l < n; ++l)
    if (!p[l]) return false;
  return true;
}

extern "C" eb_status eb_amr_residual_levels(eb_amr* A, const double* const* d_rhs, const double* const* d_sig,
                                            const double* const* d_phi, double* const* d_r, void* stream) {
  if (!A || !all_set(d_rhs, A->L) || !all_set(d_phi, A->L) || !d_r || !all_set(d_r, A->L)) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  eb_status st = amr_rhs(A, d_rhs, d_sig, s);
  if (st == EB_OK) st = amr_resid(A, d_phi, s);
  if (st != EB_OK) return st;
  for (int l = 0; l < A->L; ++l)
    cudaMemcpyAsync(d_r[l], A->lv[l].r, 2 * A->lv[l].n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaError_t e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? EB_OK : cuda_fail(e, "composite residual");
}

extern "C" eb_status eb_amr_residual(eb_amr* A, const double* d_rhs_c, const double* d_sig_c, const double* d_rhs_f,
                                     const double* d_sig_f, const double* d_phi_c, const double* d_phi_f,
                                     double* d_r_c, double* d_r_f, void* stream) {
  if (A && A->L != 2) {
    set_error("eb_amr_residual serves two-level grids; use eb_amr_residual_levels");
    return EB_ERR_INVALID;
  }
  const double* rhs[2] = {d_rhs_c, d_rhs_f};
  const double* sig[2] = {d_sig_c, d_sig_f};
  const double* phi[2] = {d_phi_c, d_phi_f};
  double* r[2] = {d_r_c, d_r_f};
  return eb_amr_residual_levels(A, rhs, sig, phi, r, stream);
}

// level l's cells under the next finer box are skipped by the dot products
static const BoxIdx& dot_box(const eb_amr* A, int l) { return A->pr[l + 1 < A->L ? l + 1 : l].B; }

static double cv_dot(eb_amr* A, const CVec& a, const CVec& b, cudaStream_t s) {
  const int L = A->L;
  for (int l = 0; l < L; ++l) {
    const AmrLevel& v = A->lv[l];
    k_cv_dot<<<DOT_BLOCKS, TBA, 0, s>>>(dot_box(A, l), v.flags, v.n, l < L - 1, a.v[l], b.v[l],
                                        A->d_part + l * DOT_BLOCKS);
    note_launch();
  }
  std::vector<double> h(L * DOT_BLOCKS);
  cudaMemcpyAsync(h.data(), A->d_part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  double t = 0.0;
  for (int i = 0; i < L * DOT_BLOCKS; ++i) t += h[i];
  return t;
}
static void cv_axpby(eb_amr* A, double a, const CVec& x, double b, const CVec& y, cudaStream_t s) {
  for (int l = 0; l < A->L; ++l) {
    k_cv_axpby<<<nb(A->lv[l].n), TBA, 0, s>>>(A->lv[l].flags, A->lv[l].n, a, x.v[l], b, y.v[l]);
    note_launch();
  }
}
static void cv_copy(eb_amr* A, const CVec& x, const CVec& y, cudaStream_t s) {
  for (int l = 0; l < A->L; ++l)
    cudaMemcpyAsync(y.v[l], x.v[l], 2 * A->lv[l].n * sizeof(double), cudaMemcpyDeviceToDevice, s);
}

// h[i] = (V[i], w) for i < m, all levels, one launch per level and one sync;
// with `self` also h[m] = (w, w), from the same pass over w
static void cv_mdot(eb_amr* A, int m, const CVec& w, double* h, cudaStream_t s, bool self = false) {
  const int L = A->L;
  CVPtrs p[AMR_MAXL] = {};
  for (int l = 0; l < L; ++l) {
    for (int i = 0; i < m; ++i) p[l].v[i] = A->V[i].v[l];
    if (self) p[l].v[m] = w.v[l];
  }
  if (self) ++m;
  for (int l = 0; l < L; ++l) {
    const AmrLevel& v = A->lv[l];
    k_cv_mdot<<<DOT_BLOCKS, TBA, 0, s>>>(dot_box(A, l), v.flags, v.n, l < L - 1, m, p[l], w.v[l],
                                         A->d_part + l * CV_MAXV * DOT_BLOCKS);
    note_launch();
  }
  std::vector<double> hp(L * CV_MAXV * DOT_BLOCKS);
  cudaMemcpyAsync(hp.data(), A->d_part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  for (int i = 0; i < m; ++i) {
    double t = 0.0;
    for (int l = 0; l < L; ++l)
      for (int b = 0; b < DOT_BLOCKS; ++b) t += hp[l * CV_MAXV * DOT_BLOCKS + i * DOT_BLOCKS + b];
    h[i] = t;
  }
}
// w -= sum_{i < m} h[i] V[i], returning the new (w, w) from the same pass
static double cv_maxpy_norm(eb_amr* A, int m, const double* h, const CVec& w, cudaStream_t s) {
  const int L = A->L;
  for (int l = 0; l < L; ++l) {
    CVPtrs p{};
    for (int i = 0; i < m; ++i) {
      p.v[i] = A->V[i].v[l];
      p.a[i] = h[i];
    }
    const AmrLevel& v = A->lv[l];
    k_cv_maxpy_norm<<<DOT_BLOCKS, TBA, 0, s>>>(dot_box(A, l), v.flags, v.n, l < L - 1, m, p, w.v[l],
                                               A->d_part + l * DOT_BLOCKS);
    note_launch();
  }
  std::vector<double> hp(L * DOT_BLOCKS);
  cudaMemcpyAsync(hp.data(), A->d_part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  double t = 0.0;
  for (int i = 0; i < L * DOT_BLOCKS; ++i) t += hp[i];
  return t;
}

// accuracy asked of the multigrid corrections inside one FAC step: loose
// enough that each stops after its first V-cycle
constexpr double FAC_TOL = 3e-1;

// w[l] for l = L-2 .. lmin: cells under the next finer box take the mean of
// that level's children (finest first, so every level sees the whole remainder)
static void restrict_down(eb_amr* A, const CVec& w, int lmin, cudaStream_t s) {
  for (int l = A->L - 2; l >= lmin; --l) {
    const AmrLevel &c = A->lv[l], &f = A->lv[l + 1];
    k_zero_under<<<nb(box_cells(A->pr[l + 1].B)), TBA, 0, s>>>(A->pr[l + 1].B, w.v[l], c.n);
    note_launch();
    k_restrict_under<<<nb(box_cells(A->pr[l + 1].B)), TBA, 0, s>>>(A->pr[l + 1].B, f.flags, w.v[l + 1], w.v[l], c.n,
                                                                   f.n);
    note_launch();
  }
}

// z = M^-1 v: one multiplicative FAC sweep from zero, coarse to fine: a
// correction of level 0 over the domain (the finer parts of v restricted
// under the boxes), added constant per parent on level 1; then on every finer
// level a correction of what remains there (zero Dirichlet CF sides), the
// remainder of the still finer levels restricted under its box, added to the
// level and constant per parent on the next.  Uses lv[].r / e and tmp.
static eb_status fac_apply(eb_amr* A, const CVec& v, const CVec& z, int* cycles, cudaStream_t s) {
  const double tol = FAC_TOL;
  const int L = A->L;
  cv_copy(A, v, A->tmp, s);
  restrict_down(A, A->tmp, 0, s);
  int cyc = 0, outer = 0;
  double kms = 0.0;
  eb_status st = poisson_solve_b(A->lv[0].P, A->tmp.v[0], A->lv[0].e, tol, &cyc, s, &outer, &kms);
  *cycles += cyc;
  amr_count(A, 0, cyc, outer, kms);
  if (st != EB_OK) return st;
  for (int l = 0; l < L; ++l) cudaMemsetAsync(z.v[l], 0, 2 * A->lv[l].n * sizeof(double), s);
  for (int l = 0; l < L; ++l) {
    if (l > 0) {
      // what remains on levels l and finer: v - A z, restricted into level l
      st = amr_resid(A, z.v, s);
      if (st != EB_OK) return st;
      for (int k = l; k < L; ++k) {
        const AmrLevel& q = A->lv[k];
        k_cv_sub<<<nb(q.n), TBA, 0, s>>>(q.flags, q.n, A->bvec.v[k], q.r, A->tmp.v[k]);  // (A z)_k
        note_launch();
        k_cv_axpby<<<nb(q.n), TBA, 0, s>>>(q.flags, q.n, 1.0, v.v[k], -1.0, A->tmp.v[k]);  // v_k - (A z)_k
        note_launch();
      }
      restrict_down(A, A->tmp, l, s);
      st = poisson_solve_b(A->lv[l].P0, A->tmp.v[l], A->lv[l].e, tol, &cyc, s, &outer, &kms);
      *cycles += cyc;
      amr_count(A, 1, cyc, outer, kms);
      if (st != EB_OK) return st;
    }
    const AmrLevel& c = A->lv[l];
    if (l < L - 1) {
      const AmrLevel& f = A->lv[l + 1];
      k_add_coarse<<<nb(c.n), TBA, 0, s>>>(A->pr[l + 1].B, c.e, z.v[l], c.n);
      note_launch();
      k_prolong_const<<<nb(f.n), TBA, 0, s>>>(A->pr[l + 1].B, f.flags, c.e, z.v[l + 1], c.n, f.n);
      note_launch();
    } else {
      k_axpy_masked<<<nb(c.n), TBA, 0, s>>>(c.flags, c.n, c.e, z.v[l]);
      note_launch();
    }
  }
  return EB_OK;
}

// w = A z (homogeneous operator) = b - r(z)
static eb_status op_apply(eb_amr* A, const CVec& z, const CVec& w, cudaStream_t s) {
  eb_status st = amr_resid(A, z.v, s);
  if (st != EB_OK) return st;
  for (int l = 0; l < A->L; ++l) {
    const AmrLevel& q = A->lv[l];
    k_cv_sub<<<nb(q.n), TBA, 0, s>>>(q.flags, q.n, A->bvec.v[l], q.r, w.v[l]);
    note_launch();
    if (l < A->L - 1) {
      k_zero_under<<<nb(box_cells(A->pr[l + 1].B)), TBA, 0, s>>>(A->pr[l + 1].B, w.v[l], q.n);
      note_launch();
    }
  }
  return EB_OK;
}

static constexpr int GM = 12;  // FGMRES restart length

static eb_status amr_workspace(eb_amr* A) {
  if (!A->V.empty()) return EB_OK;
  eb_status st = EB_OK;
  auto vec = [&]() {
    CVec v;
    for (int l = 0; l < A->L; ++l)
      v.v[l] = (double*)dev_alloc(A->allocs, 2 * A->lv[l].n * sizeof(double), &A->bytes, &st);
    return v;
  };
  for (int i = 0; i <= GM; ++i) A->V.push_back(vec());
  for (int i = 0; i < GM; ++i) A->Z.push_back(vec());
  A->bvec = vec();
  A->tmp = vec();
  A->d_part = (double*)dev_alloc(A->allocs, A->L * CV_MAXV * DOT_BLOCKS * sizeof(double), &A->bytes, &st);
  if (st != EB_OK) {
    A->V.clear();
    A->Z.clear();
  }
  return st;
}

extern "C" eb_status eb_amr_solve_levels(eb_amr* A, const double* const* d_rhs, const double* const* d_sig,
                                         double* const* d_phi, eb_solve_info* info, void* stream) {
  if (!A || !all_set(d_rhs, A->L) || !d_phi || !all_set(d_phi, A->L)) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  const int L = A->L;
  cudaStream_t s = (cudaStream_t)stream;
  eb_solve_info inf;
  std::memset(&inf, 0, sizeof(inf));
  std::memset(A->kstat, 0, sizeof(A->kstat));
  const long long launches0 = launch_total();
  eb_status st = amr_workspace(A);
  if (st != EB_OK) return st;
  // b: the composite residual at phi = 0
  CVec zero;
  for (int l = 0; l < L; ++l) {
    zero.v[l] = A->lv[l].e;
    cudaMemsetAsync(A->lv[l].e, 0, 2 * A->lv[l].n * sizeof(double), s);
  }
  st = amr_rhs(A, d_rhs, d_sig, s);
  if (st == EB_OK) st = amr_resid(A, zero.v, s);
  double bn = 0.0, r = 0.0;
  if (st == EB_OK) st = amr_norm(A, s, &bn);
  if (st != EB_OK) return st;
  CVec res, x;
  for (int l = 0; l < L; ++l) {
    res.v[l] = A->lv[l].r;
    x.v[l] = d_phi[l];
  }
  cv_copy(A, res, A->bvec, s);
  int it = 0, cycles = 0;
  const int max_it = std::max(1, A->o.max_cycles);
  // restarted FGMRES, right-preconditioned by one FAC sweep (Sec. 3.3.2's
  // multigrid as the inner solver of every correction)
  st = EB_ERR_NOT_CONVERGED;
  while (it < max_it) {
    eb_status s2 = amr_resid(A, x.v, s);
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
    cv_copy(A, res, A->V[0], s);
    for (int l = 0; l < L - 1; ++l) {
      k_zero_under<<<nb(box_cells(A->pr[l + 1].B)), TBA, 0, s>>>(A->pr[l + 1].B, A->V[0].v[l], A->lv[l].n);
      note_launch();
    }
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
      double w1 = std::sqrt(std::max(cv_maxpy_norm(A, k + 1, hp, A->V[k + 1], s), 0.0));
      for (int i = 0; i <= k; ++i) H[i][k] += hp[i];
      if (w1 < w0 / std::sqrt(2.0)) {
        cv_mdot(A, k + 1, A->V[k + 1], hp, s);
        w1 = std::sqrt(std::max(cv_maxpy_norm(A, k + 1, hp, A->V[k + 1], s), 0.0));
        for (int i = 0; i <= k; ++i) H[i][k] += hp[i];
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
  // report every level's phi under the next finer box as the finer means (finest first)
  if (st == EB_OK || st == EB_ERR_NOT_CONVERGED) {
    for (int l = L - 2; l >= 0; --l) {
      const AmrLevel &c = A->lv[l], &f = A->lv[l + 1];
      k_avg_down<<<nb(box_cells(A->pr[l + 1].B)), TBA, 0, s>>>(A->pr[l + 1].B, c.flags, f.flags, f.kap,
                                                              d_phi[l + 1], d_phi[l], c.n, f.n);
      note_launch();
    }
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

extern "C" eb_status eb_amr_solve(eb_amr* A, const double* d_rhs_c, const double* d_sig_c, const double* d_rhs_f,
                                  const double* d_sig_f, double* d_phi_c, double* d_phi_f, eb_solve_info* info,
                                  void* stream) {
  if (A && A->L != 2) {
    set_error("eb_amr_solve serves two-level grids; use eb_amr_solve_levels");
    return EB_ERR_INVALID;
  }
  const double* rhs[2] = {d_rhs_c, d_rhs_f};
  const double* sig[2] = {d_sig_c, d_sig_f};
  double* phi[2] = {d_phi_c, d_phi_f};
  return eb_amr_solve_levels(A, rhs, sig, phi, info, stream);
}

extern "C" eb_status eb_amr_field_eval(eb_amr* A, int level, const double* d_phi, const double* d_sigma,
                                       double* d_E, double* d_En, void* stream) {
  if (!A || level < 0 || level >= A->L) {
    set_error(A ? "level out of range" : "null argument");
    return EB_ERR_INVALID;
  }
  return eb_field_eval(A->lv[level].P, d_phi, d_sigma, d_E, d_En, stream);
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

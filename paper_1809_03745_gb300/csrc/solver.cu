// solver.cu -- multigrid driver and the C ABI of the EB Poisson library
// (arXiv:1809.03745, Sec. 3.3.2).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "eb_internal.h"
#include "persistent.cuh"

// ----------------------------------------------------------------- errors

namespace ebp {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

eb_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return EB_ERR_OOM;
  return EB_ERR_CUDA;
}

void* dev_alloc(std::vector<void*>& owner, size_t bytes, long long* counter, eb_status* st) {
  if (*st != EB_OK) return nullptr;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *st = EB_ERR_OOM;
    set_error("device allocation of " + std::to_string(bytes) + " bytes failed");
    return nullptr;
  }
  owner.push_back(p);
  if (counter) *counter += (long long)bytes;
  return p;
}

}  // namespace ebp

using namespace ebp;

extern "C" const char* eb_status_str(eb_status s) {
  switch (s) {
    case EB_OK: return "ok";
    case EB_ERR_INVALID: return "invalid argument";
    case EB_ERR_OOM: return "out of device memory";
    case EB_ERR_NOT_CONVERGED: return "not converged";
    case EB_ERR_CUDA: return "CUDA error";
    case EB_ERR_TIMEOUT: return "timeout";
    case EB_ERR_UNSUPPORTED: return "unsupported geometry";
    case EB_ERR_BUSY: return "busy";
  }
  return "unknown status";
}

extern "C" const char* eb_last_error(void) { return g_last_error.c_str(); }

// --------------------------------------------------------------- geometry

static eb_status validate(const eb_geom_desc* d) {
  auto bad = [](const char* m) {
    set_error(m);
    return EB_ERR_INVALID;
  };
  if (!d) return bad("null description");
  if (d->dim != 2 && d->dim != 3) return bad("dim must be 2 or 3");
  long long cells = 1;
  for (int k = 0; k < d->dim; ++k) {
    if (d->n[k] < 8 || d->n[k] % 8) return bad("cells per axis must be a multiple of 8 and at least 8");
    cells *= d->n[k];
  }
  if (cells >= (1LL << 30)) return bad("at most 2^30 cells");
  if (!(d->h > 0.0) || !std::isfinite(d->h)) return bad("h must be positive");
  if (d->n_prims < 0 || d->n_prims > EB_MAX_PRIMS) return bad("too many primitives");
  if (d->n_nodes < 0 || d->n_nodes > EB_MAX_NODES) return bad("too many CSG nodes");
  if ((d->n_prims && !d->prims) || (d->n_nodes && !d->nodes)) return bad("null primitive/node array");
  for (int i = 0; i < d->n_prims; ++i)
    if (d->prims[i].kind < 0 || d->prims[i].kind > 5) return bad("unknown primitive kind");
  for (int i = 0; i < d->n_nodes; ++i) {
    const eb_csg& c = d->nodes[i];
    if (c.op == EB_CSG_PRIM) {
      if (c.a < 0 || c.a >= d->n_prims) return bad("CSG primitive index out of range");
    } else if (c.op == EB_CSG_NEGATE) {
      if (c.a < 0 || c.a >= i) return bad("CSG child must precede its parent");
    } else if (c.op == EB_CSG_UNION || c.op == EB_CSG_INTERSECT) {
      if (c.a < 0 || c.a >= i || c.b < 0 || c.b >= i) return bad("CSG child must precede its parent");
    } else {
      return bad("unknown CSG op");
    }
  }
  if (d->electrode_root >= d->n_nodes || d->dielectric_root >= d->n_nodes) return bad("root out of range");
  if (d->n_electrodes < 0 || d->n_electrodes > EB_MAX_ELECTRODES) return bad("too many electrodes");
  for (int e = 0; e < d->n_electrodes; ++e)
    if (d->electrode_node[e] < 0 || d->electrode_node[e] >= d->n_nodes) return bad("electrode node out of range");
  if (d->electrode_root >= 0 && d->n_electrodes == 0) return bad("an electrode root needs at least one electrode");
  if (!(d->eps_gas > 0.0) || (d->dielectric_root >= 0 && !(d->eps_diel > 0.0))) return bad("permittivity must be > 0");
  for (int k = 0; k < 2 * d->dim; ++k) {
    if (d->bc_type[k] != EB_BC_NEUMANN && d->bc_type[k] != EB_BC_DIRICHLET && d->bc_type[k] != EB_BC_ROBIN)
      return bad("unknown wall type");
    if (d->bc_type[k] == EB_BC_ROBIN) {
      const double a1 = d->bc_robin[k][0], a2 = d->bc_robin[k][1];
      if (!(a1 >= 0.0 && a2 >= 0.0 && a1 + a2 > 0.0 && std::isfinite(a1 + a2)))
        return bad("Robin wall coefficients must be >= 0, not both 0");
    }
  }
  if (d->electrode_robin) {
    const double a1 = d->electrode_robin_a[0], a2 = d->electrode_robin_a[1];
    if (!(a1 >= 0.0 && a2 >= 0.0 && a1 + a2 > 0.0 && std::isfinite(a1 + a2)))
      return bad("Robin electrode coefficients must be >= 0, not both 0");
  }
  for (int p = 0; p < 2; ++p)
    if (!(d->helmholtz_lam[p] >= 0.0 && std::isfinite(d->helmholtz_lam[p]))) return bad("Helmholtz shift must be >= 0");
  return EB_OK;
}

extern "C" eb_status eb_geom_build(const eb_geom_desc* d, void* stream, eb_geom** out) {
  if (!out) {
    set_error("null output handle");
    return EB_ERR_INVALID;
  }
  *out = nullptr;
  eb_status st = validate(d);
  if (st != EB_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  eb_geom* G = new eb_geom();
  cudaGetDevice(&G->device);
  Csg& c = G->csg;
  std::memset(&c, 0, sizeof(c));
  c.n_prims = d->n_prims;
  c.n_nodes = d->n_nodes;
  for (int i = 0; i < d->n_prims; ++i) {
    c.kind[i] = d->prims[i].kind;
    for (int k = 0; k < NPAR; ++k) c.par[i][k] = d->prims[i].p[k];
  }
  for (int i = 0; i < d->n_nodes; ++i) {
    c.op[i] = d->nodes[i].op;
    c.a[i] = d->nodes[i].a;
    c.b[i] = d->nodes[i].b;
  }
  c.root_E = d->electrode_root;
  c.root_D = d->dielectric_root;
  c.n_elec = d->n_electrodes;
  for (int e = 0; e < d->n_electrodes; ++e) {
    c.elec_node[e] = d->electrode_node[e];
    c.elec_phi[e] = d->electrode_phi[e];
  }
  G->n_phase = d->dielectric_root >= 0 ? 2 : 1;
  DevLevel L0;
  Grid& g = L0.g;
  g.D = d->dim;
  for (int k = 0; k < 3; ++k) {
    g.n[k] = k < d->dim ? d->n[k] : 1;
    g.lo[k] = k < d->dim ? d->lo[k] : 0.0;
  }
  g.h = d->h;
  g.ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  for (int k = 0; k < 6; ++k) {
    g.bc[k] = (k < 2 * d->dim) ? d->bc_type[k] : 0;
    g.bcv[k] = (k < 2 * d->dim && g.bc[k]) ? d->bc_value[k] : 0.0;
    g.rob[k][0] = g.bc[k] == EB_BC_ROBIN ? d->bc_robin[k][0] : 0.0;
    g.rob[k][1] = g.bc[k] == EB_BC_ROBIN ? d->bc_robin[k][1] : 0.0;
  }
  g.eps[0] = d->eps_gas;
  g.eps[1] = d->dielectric_root >= 0 ? d->eps_diel : d->eps_gas;
  g.lam[0] = d->helmholtz_lam[0];
  g.lam[1] = d->dielectric_root >= 0 ? d->helmholtz_lam[1] : d->helmholtz_lam[0];
  g.eb_robin = d->electrode_robin ? 1 : 0;
  g.eb_ra[0] = g.eb_robin ? d->electrode_robin_a[0] : 0.0;
  g.eb_ra[1] = g.eb_robin ? d->electrode_robin_a[1] : 0.0;
  G->L.push_back(L0);
  std::vector<void*> misc;
  G->d_csg = (Csg*)dev_alloc(G->L[0].allocs, sizeof(Csg), &G->bytes, &st);
  G->d_status = (int*)dev_alloc(G->L[0].allocs, sizeof(int), &G->bytes, &st);
  if (st == EB_OK) {
    cudaError_t e = cudaMemcpyAsync(G->d_csg, &c, sizeof(Csg), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) st = cuda_fail(e, "description upload");
  }
  if (st == EB_OK) st = build_finest_geometry(G, s);
  if (st == EB_OK) st = build_rows(G, 0, s);
  // coarsen while every axis keeps at least 8 cells and stays even
  while (st == EB_OK) {
    const Grid& f = G->L.back().g;
    bool ok = true;
    for (int k = 0; k < f.D; ++k)
      if (f.n[k] % 2 || f.n[k] / 2 < 8) ok = false;
    if (!ok || (int)G->L.size() >= EB_MAX_LEVELS) break;
    bool stopped = false;
    st = build_coarse_geometry(G, (int)G->L.size() - 1, s, &stopped);
    if (st != EB_OK || stopped) break;
    st = build_rows(G, (int)G->L.size() - 1, s);
    if (st == EB_ERR_UNSUPPORTED) {  // a coarse stencil that cannot be built ends the hierarchy
      free_level(G->L.back());
      G->L.pop_back();
      st = EB_OK;
      break;
    }
  }
  if (st == EB_OK) {
    // dof and stencil-order counts of the finest level
    const DevLevel& F = G->L[0];
    std::vector<uint8_t> flags(F.g.ncell);
    cudaMemcpy(flags.data(), F.flags, F.g.ncell, cudaMemcpyDeviceToHost);
    long long nd = 0;
    for (uint8_t f : flags) nd += (f & 1) + ((f >> 1) & 1);
    G->n_dof = nd;
    long long nq = F.R.ncut;
    std::vector<uint8_t> ord(2 * std::max<long long>(nq, 1)), dofm(std::max<long long>(nq, 1));
    if (nq) {
      cudaMemcpy(ord.data(), F.order, 2 * nq, cudaMemcpyDeviceToHost);
      cudaMemcpy(dofm.data(), F.R.dofm, nq, cudaMemcpyDeviceToHost);
    }
    for (long long q = 0; q < nq; ++q)
      for (int p = 0; p < 2; ++p) {
        if (!((dofm[q] >> p) & 1)) continue;
        int o = ord[p * nq + q];
        if (o == 2) G->stencil_counts[0]++;
        if (o == 1) G->stencil_counts[1]++;
        if (o == 3) G->stencil_counts[2]++;
      }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "geometry summary");
  }
  if (st != EB_OK) {
    eb_geom_destroy(G);
    return st;
  }
  *out = G;
  return EB_OK;
}

extern "C" void eb_geom_destroy(eb_geom* G) {
  if (!G) return;
  for (auto& L : G->L) free_level(L);
  delete G;
}

extern "C" eb_status eb_geom_query(const eb_geom* G, eb_geom_info* out) {
  if (!G || !out) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  std::memset(out, 0, sizeof(*out));
  const DevLevel& F = G->L[0];
  out->dim = F.g.D;
  out->n_phase = G->n_phase;
  out->n_cells = F.g.ncell;
  out->n_dof = G->n_dof;
  out->n_eb = F.n_eb;
  out->n_irregular = F.nirr;
  out->n_levels = (int)G->L.size();
  for (size_t l = 0; l < G->L.size(); ++l)
    for (int k = 0; k < 3; ++k) out->level_n[l][k] = G->L[l].g.n[k];
  for (int k = 0; k < 3; ++k) out->stencil_order[k] = G->stencil_counts[k];
  out->device_bytes = G->bytes;
  return EB_OK;
}

extern "C" eb_status eb_geom_export(const eb_geom* G, eb_geom_arrays* out, void* stream) {
  if (!G || !out) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  return export_geometry(G, out, (cudaStream_t)stream);
}

// ----------------------------------------------------------------- solver

struct eb_poisson {
  const eb_geom* G = nullptr;
  eb_solver_opts o{};
  int nlev = 0;
  std::vector<Op<double>> op64;
  std::vector<Op<float>> op32;
  double* phi64 = nullptr;
  double* b64 = nullptr;
  unsigned long long* d_norm = nullptr;  // [0] residual max, [1] rhs max
  unsigned long long* h_norm = nullptr;  // pinned
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  long long launches = 0;   // kernels launched by the current call
  long long per_iter = 0;   // kernels in one iteration
  // persistent solve
  bool persistent = false;
  int grid = 0;
  void* d_hier = nullptr;     // Hier<float> or Hier<double>
  Op<double>* d_fine = nullptr;
  unsigned* d_bar = nullptr;  // count, gen, err
  int* d_out = nullptr;       // status, iterations, cycles, slot
  int* h_out = nullptr;       // pinned
  unsigned long long* d_norms = nullptr;
  unsigned long long* d_stamps = nullptr;  // [8] first-V-cycle timestamps of the last solve
  void* d_binv = nullptr;
  int bm = 0;
  int bottom = EB_BOTTOM_RELAX;  // EB_BOTTOM_* of the persistent hierarchy
  int sweep_levels = 0;          // grid levels relaxed by tile-streamed sweeps
  int sweep_bytes = 0;           // their shared memory per CTA
  int sweep_ns = 0;              // ring slots
  int sweep_first = -1;          // the finest of them
  std::vector<int*> sweep_ticks;  // their ticket counters (4 ints per level)
  int smem_bytes = 0;  // dynamic shared memory of the persistent kernel
  cudaEvent_t kev[2] = {nullptr, nullptr};  // bracket the persistent kernel
  double kernel_ms = 0.0;                   // its device time in the last call
  std::vector<void*> allocs;
  long long bytes = 0;
};

extern "C" void eb_solver_opts_default(eb_solver_opts* o) {
  if (!o) return;
  o->tol = 1e-10;
  o->max_cycles = 100;
  o->nu1 = -1;
  o->nu2 = -1;
  o->precision = EB_PREC_MIXED;
  o->inner_cycles = 2;
  o->bottom_sweeps = 64;
  o->launch_mode = 0;
}

// The regular stencil's wall weights, Helmholtz shift and reciprocal
// interior diagonal (Op::wr, lh, idg) on a level with grid g.  A Robin wall's
// weight a1 / (a1 + 8 a2 / (3h)) is what is left of the one-sided wall
// formula once the wall value is eliminated; it depends on the level's h.
template <class T>
static void set_stencil_terms(Op<T>& o, const Grid& g) {
  o.intdg = 1;
  for (int k = 0; k < 6; ++k) {
    double w = 0.0;
    if (k < 2 * g.D) {
      if (g.bc[k] == 1) w = 1.0;
      else if (g.bc[k] == 2) w = g.rob[k][0] / (g.rob[k][0] + g.rob[k][1] * 8.0 / (3.0 * g.h));
    }
    o.wr[k] = (T)w;
    o.w3[k] = (T)w * (T(1) / T(3));
    if (w != 0.0 && w != 1.0) o.intdg = 0;
  }
  for (int p = 0; p < 2; ++p) {
    const T lh = (T)(g.lam[p] * g.h * g.h / g.eps[p]);
    o.lh[p] = lh;
    o.idg[p] = T(1) / (T(2 * g.D) + lh);
    if (lh != T(0)) o.intdg = 0;
  }
}

template <class T>
static Op<T> make_op(const DevLevel& L, std::vector<void*>& owner, long long* bytes, eb_status* st, int nphase,
                     T* x0 = nullptr, T* b0 = nullptr, T* x1 = nullptr, T* b1 = nullptr) {
  Op<T> o;
  std::memset(&o, 0, sizeof(o));
  o.D = L.g.D;
  for (int k = 0; k < 3; ++k) o.n[k] = L.g.n[k];
  o.dn0 = make_fastdiv((unsigned)L.g.n[0]);
  o.dn1 = make_fastdiv((unsigned)L.g.n[1]);
  o.dhx = make_fastdiv((unsigned)((L.g.n[0] + 1) / 2));
  o.dq = make_fastdiv((unsigned)std::max(1, L.g.n[0] / 4));
  o.ncell = L.g.ncell;
  set_stencil_terms(o, L.g);
  size_t n = (size_t)L.g.ncell;
  o.x[0] = x0 ? x0 : (T*)dev_alloc(owner, n * sizeof(T), bytes, st);
  o.b[0] = b0 ? b0 : (T*)dev_alloc(owner, n * sizeof(T), bytes, st);
  if (nphase == 2) {
    o.x[1] = x1 ? x1 : (T*)dev_alloc(owner, n * sizeof(T), bytes, st);
    o.b[1] = b1 ? b1 : (T*)dev_alloc(owner, n * sizeof(T), bytes, st);
  }
  o.flags = L.flags;
  o.irr_cell = L.irr_cell;
  o.irr_of_cell = L.irr_of_cell;
  o.row_ptr = L.row_ptr;
  o.col = L.col;
  o.val = L.val;
  o.diag = L.diag;
  o.tmp = (T*)dev_alloc(owner, sizeof(T) * std::max<long long>(2 * L.nirr, 1), bytes, st);
  o.nirr = L.nirr;
  o.nirr_red = L.nirr_red;
  for (int p = 0; p < 2; ++p) {
    double e = L.g.eps[p], h2 = L.g.h * L.g.h;
    o.ceps[p] = (T)(e / h2);
    o.h2e[p] = (T)(h2 / e);
  }
  if (*st == EB_OK) {
    cudaMemset(o.x[0], 0, n * sizeof(T));
    cudaMemset(o.b[0], 0, n * sizeof(T));
    if (nphase == 2) {
      cudaMemset(o.x[1], 0, n * sizeof(T));
      cudaMemset(o.b[1], 0, n * sizeof(T));
    }
  }
  return o;
}

static inline int blocks(long long n, int tb = 256) { return (int)std::max<long long>(1, (n + tb - 1) / tb); }

static thread_local long long* g_count = nullptr;  // launch counter of the current call
static thread_local long long g_total = 0;         // every launch of this thread
namespace ebp {
void note_launch(int k) { g_total += k; }
long long launch_total() { return g_total; }
}  // namespace ebp
static inline void counted(int k = 1) {
  g_total += k;
  if (g_count) *g_count += k;
}

template <class T>
static void smooth(const Op<T>& o, cudaStream_t s) {
  long long work = (o.ncell / o.n[0]) * ((o.n[0] + 1) / 2);
  for (int colour = 0; colour < 2; ++colour) {
    k_smooth_dense<T><<<blocks(work), 256, 0, s>>>(o, colour);
    counted();
    long long rb = colour == 0 ? 0 : 2 * o.nirr_red, re = colour == 0 ? 2 * o.nirr_red : 2 * o.nirr;
    if (re <= rb) continue;
    if (re - rb <= 16384) {
      k_rows_gs_cta<T><<<1, 1024, 0, s>>>(o, rb, re);
      counted();
    } else {
      k_rows<T><<<blocks(re - rb), 256, 0, s>>>(o, rb, re, 0);
      k_scatter_rows<T><<<blocks(re - rb), 256, 0, s>>>(o, rb, re);
      counted(2);
    }
  }
}

template <class T>
static void vcycle(eb_poisson* P, std::vector<Op<T>>& ops, int l, cudaStream_t s) {
  const Op<T>& o = ops[l];
  if (l == P->nlev - 1) {
    k_bottom<T><<<1, 1024, 0, s>>>(o, P->o.bottom_sweeps);
    counted();
    return;
  }
  for (int i = 0; i < P->o.nu1; ++i) smooth(o, s);
  if (o.nirr) {
    k_rows<T><<<blocks(2 * o.nirr), 256, 0, s>>>(o, 0, 2 * o.nirr, 1);
    counted();
  }
  k_resid_restrict<T><<<blocks(ops[l + 1].ncell), 256, 0, s>>>(o, ops[l + 1]);
  counted();
  vcycle(P, ops, l + 1, s);
  k_prolong<T><<<blocks(o.ncell), 256, 0, s>>>(o, ops[l + 1]);
  counted();
  for (int i = 0; i < P->o.nu2; ++i) smooth(o, s);
}

// FP64 residual of the finest level; writes the FP32 inner rhs in mixed mode
static void resid64(eb_poisson* P, cudaStream_t s, bool to32) {
  const Op<double>& o = P->op64[0];
  cudaMemsetAsync(P->d_norm, 0, sizeof(unsigned long long), s);
  if (o.nirr) {
    k_rows<double><<<blocks(2 * o.nirr), 256, 0, s>>>(o, 0, 2 * o.nirr, 1);
    counted();
  }
  float *b0 = nullptr, *b1 = nullptr, *e0 = nullptr, *e1 = nullptr;
  if (to32) {
    const Op<float>& f = P->op32[0];
    b0 = f.b[0];
    b1 = f.b[1];
    e0 = f.x[0];
    e1 = f.x[1];
  }
  k_resid64_out<<<blocks(o.ncell), 256, 0, s>>>(o, b0, b1, e0, e1, P->d_norm);
  counted();
}

// one iteration: mixed -> inner FP32 V-cycles, FP64 update, FP64 residual;
// FP64 -> one V-cycle and the residual
static void iteration(eb_poisson* P, cudaStream_t s) {
  if (P->o.precision == EB_PREC_MIXED) {
    for (int i = 0; i < P->o.inner_cycles; ++i) vcycle(P, P->op32, 0, s);
    const Op<float>& f = P->op32[0];
    k_update64<<<blocks(P->op64[0].ncell), 256, 0, s>>>(P->op64[0], f.x[0], f.x[1]);
    counted();
    resid64(P, s, true);
  } else {
    vcycle(P, P->op64, 0, s);
    resid64(P, s, false);
  }
}


// ------------------------------------------------- tile-streamed sweeps (sweep3d.cuh)

static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  });
  return fn;
}

// a 3D tensor map over one level array (x fastest), boxes of bx x by x bz
static bool tmap3(CUtensorMap* m, CUtensorMapDataType type, int esize, const void* base, const int n[3], int bx,
                  int by, int bz) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
  if (!enc) return false;
  cuuint64_t dim[3] = {(cuuint64_t)n[0], (cuuint64_t)n[1], (cuuint64_t)n[2]};
  cuuint64_t str[2] = {(cuuint64_t)n[0] * esize, (cuuint64_t)n[0] * n[1] * esize};
  cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(m, type, 3, const_cast<void*>(base), dim, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Levels of at least 2^25 cells (about 322^3) relax by tile-streamed sweeps:
// measured on a GB300 at 384^3 a streamed sweep takes 0.39 ms against 0.53 ms
// for the two colour passes, at 256^3 0.19 ms against 0.17 ms.  The streamed
// residual + restriction is slower than the block restriction at both sizes
// (0.36 / 0.31 ms, 0.19 / 0.10 ms) and is used only on request
// (EBP_SWEEP_RESTRICT=1).
static constexpr long long SW_MIN_CELLS = 1LL << 25;

// Items of a level cut into z-chunks of zc planes: tile t = it % ntiles,
// chunk it / ntiles.  An item holds dielectric unknowns when its tile's box
// does in one of the planes it loads (z0 - 2 .. z1 + 1) or the coarse cells
// under it do in one of its coarse planes (z0 / 2 .. z1 / 2 - 1); plane1
// gives that per (tile, plane), fine planes first (ntiles x n2), then coarse
// (ntiles x cn2, cn2 = 0 without a coarse level).
static std::vector<int> sweep_items1(const std::vector<uint8_t>& plane1, int ntiles, int n2, int cn2, int zc) {
  std::vector<int> out;
  const int nzc = (n2 + zc - 1) / zc;
  for (int q = 0; q < nzc; ++q) {
    const int z0 = q * zc, z1 = std::min(z0 + zc, n2);
    for (int t = 0; t < ntiles; ++t) {
      bool has = false;
      for (int z = std::max(z0 - 2, 0); z < std::min(z1 + 2, n2) && !has; ++z) has = plane1[(size_t)t * n2 + z] != 0;
      for (int z = z0 / 2; z < std::min(z1 / 2, cn2) && !has; ++z)
        has = plane1[(size_t)ntiles * n2 + (size_t)t * cn2 + z] != 0;
      if (has) out.push_back(q * ntiles + t);
    }
  }
  return out;
}

// z-chunk of a level for `workers` CTAs: the least of (rounds of items per
// CTA, the dielectric phase's items included) x (steps per item: two planes
// each, two more for the ends), over chunks of 4..n2 planes in steps of 4.
static int sweep_chunk(const int n[3], int workers, const std::vector<uint8_t>* plane1, int cn2) {
  const long long ntx = (n[0] + SW_TX - 1) / SW_TX, nty = (n[1] + SW_TY - 1) / SW_TY;
  long long best = -1;
  int zc_best = 4;
  for (int zc = 4; zc <= n[2] + 3; zc += 4) {
    const long long nzc = (n[2] + zc - 1) / zc;
    long long items = ntx * nty * nzc;
    if (plane1) items += (long long)sweep_items1(*plane1, (int)(ntx * nty), n[2], cn2, zc).size();
    const long long rounds = (items + workers - 1) / workers;
    const long long cost = rounds * (zc / 2 + 2);
    if (best < 0 || cost < best) {
      best = cost;
      zc_best = zc;
    }
  }
  return zc_best;
}

// Marks the FP32 3D grid levels of at least SW_MIN_CELLS cells (each extent
// a multiple of 4, x a multiple of 16) for tile-streamed passes: a second x
// buffer per phase, tensor maps of x, the second buffer, b and the flags with
// two-plane boxes, and the list of items that hold dielectric unknowns.
// Levels stay on the colour passes when any of it fails.
template <class T>
static eb_status setup_sweeps(eb_poisson* P, std::vector<Op<T>>& ops, Hier<T>& H, int smem_cap) {
  if (!std::is_same<T, float>::value) return EB_OK;
  if (const char* env = std::getenv("EBP_SWEEP"))
    if (std::atoi(env) == 0) return EB_OK;
  if (SW_HEAD + 128 + SW_NS * SwSlot<T>::BYTES > smem_cap) return EB_OK;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P->G->device);
  const int workers = std::max(1, nsm - 1);
  long long min_cells = SW_MIN_CELLS;  // EBP_SWEEP_MIN_CELLS lowers it (tests run small grids through the path)
  if (const char* env = std::getenv("EBP_SWEEP_MIN_CELLS")) min_cells = std::max(1LL, std::atoll(env));
  int restrict_streamed = 0;
  if (const char* env = std::getenv("EBP_SWEEP_RESTRICT")) restrict_streamed = std::atoi(env) != 0;
  eb_status st = EB_OK;
  for (int l = 0; l < H.lc; ++l) {
    Op<T>& o = ops[l];
    if (o.D != 3 || o.ncell < min_cells || (o.n[0] % 16) || (o.n[1] % 4) || (o.n[2] % 4)) continue;
    SweepLev<T>& sw = H.sw[l];
    const DevLevel& Lv = P->G->L[l];
    const int two = o.x[1] != nullptr;
    sw.ntx = (o.n[0] + SW_TX - 1) / SW_TX;
    sw.nty = (o.n[1] + SW_TY - 1) / SW_TY;
    // where the dielectric phase's unknowns sit, per (tile, plane)
    std::vector<uint8_t> plane1;
    const bool has_c = l + 1 < (int)P->G->L.size();
    const int cn2 = has_c ? P->G->L[l + 1].g.n[2] : 0;
    if (two) {
      const int ntiles = sw.ntx * sw.nty;
      const size_t nb = (size_t)ntiles * (o.n[2] + cn2);
      std::vector<void*> tmp;
      uint8_t* d_p1 = (uint8_t*)dev_alloc(tmp, nb, nullptr, &st);
      if (st != EB_OK) return st;
      cudaMemsetAsync(d_p1, 0, nb, P->s);
      const uint8_t* cfl = has_c ? P->G->L[l + 1].flags : nullptr;
      const int* cn = has_c ? P->G->L[l + 1].g.n : o.n;
      k_sweep_has1<<<(unsigned)(cfl ? nb : (size_t)ntiles * o.n[2]), 256, 0, P->s>>>(
          Lv.flags, o.n[0], o.n[1], o.n[2], sw.ntx, sw.nty, cfl, cn[0], cn[1], cn2, d_p1);
      plane1.resize(nb);
      cudaError_t e = cudaMemcpyAsync(plane1.data(), d_p1, nb, cudaMemcpyDeviceToHost, P->s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(P->s);
      for (void* q : tmp) cudaFree(q);
      if (e != cudaSuccess) return cuda_fail(e, "sweep setup");
    }
    sw.zc = sweep_chunk(o.n, workers, two ? &plane1 : nullptr, cn2);
    sw.nzc = (o.n[2] + sw.zc - 1) / sw.zc;
    sw.nitems = sw.ntx * sw.nty * sw.nzc;
    CUtensorMap maps[7];
    std::memset(maps, 0, sizeof(maps));
    for (int p = 0; p < 2; ++p) {
      sw.alt[p] = nullptr;
      if (o.x[p]) {
        sw.alt[p] = (T*)dev_alloc(P->allocs, sizeof(T) * (size_t)o.ncell, &P->bytes, &st);
        if (st == EB_OK) cudaMemsetAsync(sw.alt[p], 0, sizeof(T) * (size_t)o.ncell, P->s);
      }
    }
    CUtensorMap* dmaps = (CUtensorMap*)dev_alloc(P->allocs, sizeof(CUtensorMap) * 7, &P->bytes, &st);
    if (st != EB_OK) return st;
    sw.tick = (int*)dev_alloc(P->allocs, 4 * sizeof(int), &P->bytes, &st);
    if (st != EB_OK) return st;
    cudaMemsetAsync(sw.tick, 0, 4 * sizeof(int), P->s);
    P->sweep_ticks.push_back(sw.tick);
    const int by = SW_TY + 2 * SW_HY;
    const CUtensorMapDataType ft = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    bool ok = tmap3(&maps[0], ft, 4, o.x[0], o.n, SW_BX, by, 2) && tmap3(&maps[2], ft, 4, sw.alt[0], o.n, SW_BX, by, 2) &&
              tmap3(&maps[4], ft, 4, o.b[0], o.n, SW_BX, by, 2) &&
              tmap3(&maps[6], CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, Lv.flags, o.n, SW_FBX, by, 2);
    if (ok && two)
      ok = tmap3(&maps[1], ft, 4, o.x[1], o.n, SW_BX, by, 2) && tmap3(&maps[3], ft, 4, sw.alt[1], o.n, SW_BX, by, 2) &&
           tmap3(&maps[5], ft, 4, o.b[1], o.n, SW_BX, by, 2);
    if (!ok) continue;  // this level keeps the colour passes
    // the items whose boxes (or coarse cells) hold dielectric unknowns
    const std::vector<int> list1 =
        two ? sweep_items1(plane1, sw.ntx * sw.nty, o.n[2], cn2, sw.zc) : std::vector<int>();
    int* dlist = (int*)dev_alloc(P->allocs, sizeof(int) * std::max<size_t>(list1.size(), 1), &P->bytes, &st);
    if (st != EB_OK) return st;
    cudaError_t e = cudaSuccess;
    if (!list1.empty())
      e = cudaMemcpyAsync(dlist, list1.data(), sizeof(int) * list1.size(), cudaMemcpyHostToDevice, P->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dmaps, maps, sizeof(maps), cudaMemcpyHostToDevice, P->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->s);
    if (e != cudaSuccess) return cuda_fail(e, "sweep setup");
    sw.maps = dmaps;
    sw.list1 = dlist;
    sw.n1items = (int)list1.size();
    sw.par = 0;
    sw.on = 1;
    sw.rs = restrict_streamed;
    ++P->sweep_levels;
    if (P->sweep_first < 0) P->sweep_first = l;
  }
  if (P->sweep_levels) {
    P->sweep_ns = SW_NS;
    P->sweep_bytes = SW_HEAD + 128 + SW_NS * SwSlot<T>::BYTES;
  }
  return EB_OK;
}

// After a launch in which a wait gave up, the streamed passes' ticket
// counters may be left in the middle of a pass: zero them for the next one.
static void sweep_reset(eb_poisson* P, cudaStream_t s) {
  for (int* t : P->sweep_ticks) cudaMemsetAsync(t, 0, 4 * sizeof(int), s);
}

template <class T>
static eb_status build_hier(eb_poisson* P, std::vector<Op<T>>& ops) {
  Hier<T> H;
  std::memset(&H, 0, sizeof(H));
  H.nlev = P->nlev;
  H.nu1 = P->o.nu1;
  H.nu2 = P->o.nu2;
  H.bsweeps = P->o.bottom_sweeps;
  // levels of at most 4096 cells run inside one CTA, their data in its shared
  // memory when it fits in SMEM_CAP bytes
  const int SMEM_CAP = 112 * 1024;
  H.lc = P->nlev - 1;
  for (int l = 0; l < P->nlev; ++l)
    if (ops[l].ncell <= 4096) {
      H.lc = std::min(l, P->nlev - 1);
      break;
    }
  auto layout = [&](int l0, bool write) {
    long long off = 0;
    auto take = [&](long long bytes) {
      long long o = off;
      off += (bytes + 15) / 16 * 16;
      return (int)o;
    };
    for (int l = l0; l < P->nlev; ++l) {
      long long n = ops[l].ncell;
      for (int p = 0; p < 2; ++p) {
        int ox = ops[l].x[p] ? take(n * (long long)sizeof(T)) : 0;
        int ob = ops[l].b[p] ? take(n * (long long)sizeof(T)) : 0;
        if (write) {
          H.off_x[l][p] = ox;
          H.off_b[l][p] = ob;
        }
      }
      int of = take(n);
      int ot = take(std::max<long long>(2 * ops[l].nirr, 1) * (long long)sizeof(T));
      if (write) {
        H.off_f[l] = of;
        H.off_t[l] = ot;
      }
    }
    return off;
  };
  const Op<T>& ob = ops[P->nlev - 1];
  const int m = (int)(P->G->n_phase * ob.ncell);
  // a bottom of 256 < m <= 1024 unknowns gets a dense inverse applied by the
  // whole grid: every level is then a grid level, the bottom in global memory.
  // (Set-up costs ~2 m^3 flops through L2: ~7 ms at m = 1024, ~260 ms at
  // m = 3500, which a serving loop pays per admitted request.)
  const bool big_bottom = m > 256 && m <= 1024;
  // a bottom of more than 4096 cells (coarsening stopped early) and no inverse
  // is solved by BiCGStab over the whole grid
  const bool krylov_bottom = m > 1024 && ob.ncell > 4096;
  if (big_bottom || krylov_bottom) H.lc = P->nlev - 1;
  while (H.lc < P->nlev - 1 && layout(H.lc, false) > SMEM_CAP) ++H.lc;
  long long sb = layout(H.lc, false);
  H.smem = (sb <= SMEM_CAP && !big_bottom && !krylov_bottom) ? 1 : 0;
  H.smem_bytes = H.smem ? (int)sb : 0;
  if (H.smem) layout(H.lc, true);
  // the sparse rows of those levels (constant over a solve) join them while
  // the total stays under ROWS_CAP, level by level from the finest of them:
  // the row phases inside CTA 0 then make no L2 round trip
  if (H.smem) {
    const long long ROWS_CAP = 200 * 1024;
    auto al = [](long long b) { return (b + 15) / 16 * 16; };
    long long off = sb;
    for (int l = H.lc; l < P->nlev; ++l) {
      const long long nirr = ops[l].nirr, nr = 2 * nirr, nnz = P->G->L[l].nnz, nc = ops[l].ncell;
      if (nr == 0) continue;
      const long long need = al(4 * (nr + 1)) + al(4 * nnz) + al(8 * nnz) + al(8 * nr) + al(4 * nirr) + al(4 * nc);
      if (off + need > ROWS_CAP) continue;
      H.off_rp[l] = (int)off;
      H.off_col[l] = (int)(off += al(4 * (nr + 1)));
      H.off_val[l] = (int)(off += al(4 * nnz));
      H.off_dg[l] = (int)(off += al(8 * nnz));
      H.off_ic[l] = (int)(off += al(8 * nr));
      H.off_io[l] = (int)(off += al(4 * nirr));
      off += al(4 * nc);
      H.rnnz[l] = (int)nnz;
      H.srows[l] = 1;
    }
    H.smem_bytes = (int)off;
  }
  for (int l = 0; l < P->nlev; ++l) H.op[l] = ops[l];
  eb_status st = EB_OK;
  // dense inverse of the coarsest operator (FP64 Gauss-Jordan on the device)
  if (m <= 256) {
    std::vector<void*> tmp;
    double* M = (double*)dev_alloc(tmp, sizeof(double) * m * m, nullptr, &st);
    double* Mi = (double*)dev_alloc(tmp, sizeof(double) * m * m, nullptr, &st);
    int* stat = (int*)dev_alloc(tmp, sizeof(int), nullptr, &st);
    T* binv = (T*)dev_alloc(P->allocs, sizeof(T) * m * m, &P->bytes, &st);
    if (st == EB_OK) {
      const DevLevel& Lb = P->G->L[P->nlev - 1];
      double h2 = Lb.g.h * Lb.g.h;
      cudaMemsetAsync(stat, 0, sizeof(int), P->s);
      cudaMemsetAsync(M, 0, sizeof(double) * m * m, P->s);
      k_bottom_matrix<T><<<blocks(m), 256, 0, P->s>>>(ob, Lb.g.eps[0] / h2, Lb.g.eps[1] / h2, m, M);
      k_gauss_jordan<<<1, 1024, 0, P->s>>>(M, Mi, m, stat);
      k_convert<T><<<blocks((long long)m * m), 256, 0, P->s>>>(Mi, binv, (long long)m * m);
      int hs = 0;
      cudaError_t e = cudaMemcpyAsync(&hs, stat, sizeof(int), cudaMemcpyDeviceToHost, P->s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(P->s);
      if (e != cudaSuccess) st = cuda_fail(e, "bottom inverse");
      if (st == EB_OK && hs == 0) {
        H.bm = m;
        H.binv = binv;
      }
    }
    for (void* p : tmp) cudaFree(p);
  } else if (m <= 1024) {
    // larger bottoms: FP32 Gauss-Jordan with partial pivoting, one pivot step
    // per pair of launches (an approximate inverse is enough for a bottom
    // solve inside the V-cycle; a failed pivot keeps the relaxation bottom)
    std::vector<void*> tmp;
    double* M = (double*)dev_alloc(tmp, sizeof(double) * m * m, nullptr, &st);
    float* Af = (float*)dev_alloc(tmp, sizeof(float) * m * m, nullptr, &st);
    float* Ai = (float*)dev_alloc(tmp, sizeof(float) * m * m, nullptr, &st);
    int* stat = (int*)dev_alloc(tmp, sizeof(int), nullptr, &st);
    T* binv = st == EB_OK ? (T*)dev_alloc(P->allocs, sizeof(T) * m * m, &P->bytes, &st) : nullptr;
    if (st == EB_OK) {
      const DevLevel& Lb = P->G->L[P->nlev - 1];
      double h2 = Lb.g.h * Lb.g.h;
      long long mm = (long long)m * m;
      cudaMemsetAsync(stat, 0, sizeof(int), P->s);
      cudaMemsetAsync(M, 0, sizeof(double) * m * m, P->s);
      k_bottom_matrix<T><<<blocks(m), 256, 0, P->s>>>(ob, Lb.g.eps[0] / h2, Lb.g.eps[1] / h2, m, M);
      k_to_float<<<blocks(mm), 256, 0, P->s>>>(M, Af, mm);
      k_identity<<<blocks(mm), 256, 0, P->s>>>(Ai, m);
      const int eb = (int)(((long long)m * 32 + 255) / 256);
      for (int k = 0; k < m; ++k) {
        k_gj_pivot<<<1, 1024, 0, P->s>>>(Af, Ai, m, k, stat);
        k_gj_elim<<<eb, 256, 0, P->s>>>(Af, Ai, m, k, stat);
      }
      k_from_float<T><<<blocks(mm), 256, 0, P->s>>>(Ai, binv, mm);  // row-major for ph_bottom_grid
      int hs = 0;
      cudaError_t e = cudaMemcpyAsync(&hs, stat, sizeof(int), cudaMemcpyDeviceToHost, P->s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(P->s);
      if (e != cudaSuccess) st = cuda_fail(e, "bottom inverse");
      if (st == EB_OK && hs == 0) {
        H.bm = m;
        H.binv = binv;
        H.gbot = 1;
      }
    }
    for (void* p : tmp) cudaFree(p);
    st = st == EB_ERR_OOM ? EB_OK : st;  // no room for the inverse: relaxation bottom
    if (st == EB_OK && H.bm == 0) cudaGetLastError();
  }
  if (st != EB_OK) return st;
  if (krylov_bottom && H.bm == 0) {
    H.kry = (T*)dev_alloc(P->allocs, sizeof(T) * 12 * (size_t)ob.ncell, &P->bytes, &st);
    H.kpart = (double*)dev_alloc(P->allocs, sizeof(double) * 2 * 2 * 1024, &P->bytes, &st);  // up to 1024 CTAs
    H.kry_iters = std::max(16, P->o.bottom_sweeps);
    H.gkry = st == EB_OK ? 1 : 0;
    if (st != EB_OK) return st;
  }
  P->bm = H.bm;
  P->bottom = H.gkry ? EB_BOTTOM_KRYLOV : H.gbot ? EB_BOTTOM_INV32 : H.bm ? EB_BOTTOM_INV64 : EB_BOTTOM_RELAX;
  {
    // dynamic shared memory the persistent kernel may take (the device's
    // opt-in maximum less room for its static shared memory)
    int smax = 0;
    cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->G->device);
    st = setup_sweeps<T>(P, ops, H, smax - 16 * 1024);
    if (st != EB_OK) return st;
  }
  // CTA 0 keeps the coarse levels in its dynamic shared memory and sits the
  // streamed sweeps out; the other CTAs use the same bytes for the sweep ring
  P->smem_bytes = std::max(H.smem_bytes, P->sweep_bytes);
  P->d_hier = dev_alloc(P->allocs, sizeof(Hier<T>), &P->bytes, &st);
  if (st == EB_OK) {
    cudaError_t e = cudaMemcpy(P->d_hier, &H, sizeof(Hier<T>), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = cuda_fail(e, "hierarchy upload");
  }
  return st;
}

// The persistent kernels in two builds: with the tile-streamed passes (FP32
// hierarchies that have streamed levels) and without them, so that every
// other solve runs the lean build.
static const void* solve_kernel(bool mixed, bool sw) {
  if (!mixed) return (const void*)k_solve<double, false>;
  return sw ? (const void*)k_solve<float, true> : (const void*)k_solve<float, false>;
}
static const void* batch_kernel(bool mixed, bool sw) {
  if (!mixed) return (const void*)k_solve_batch<double, false>;
  return sw ? (const void*)k_solve_batch<float, true> : (const void*)k_solve_batch<float, false>;
}

static eb_status setup_persistent(eb_poisson* P) {
  int dev = P->G->device, coop = 0, nsm = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  eb_status st = EB_OK;
  bool mixed = P->o.precision == EB_PREC_MIXED;
  st = mixed ? build_hier<float>(P, P->op32) : build_hier<double>(P, P->op64);
  if (st != EB_OK) return st;
  P->d_fine = (Op<double>*)dev_alloc(P->allocs, sizeof(Op<double>), &P->bytes, &st);
  P->d_bar = (unsigned*)dev_alloc(P->allocs, 4 * sizeof(unsigned), &P->bytes, &st);
  P->d_out = (int*)dev_alloc(P->allocs, 4 * sizeof(int), &P->bytes, &st);
  P->d_norms = (unsigned long long*)dev_alloc(P->allocs, sizeof(unsigned long long) * (P->o.max_cycles + 2),
                                              &P->bytes, &st);
  P->d_stamps = (unsigned long long*)dev_alloc(P->allocs, sizeof(unsigned long long) * (TRMAX + 1), &P->bytes, &st);
  if (st == EB_OK) cudaMemset(P->d_stamps, 0, sizeof(unsigned long long) * (TRMAX + 1));
  if (st != EB_OK) return st;
  cudaError_t e = cudaMemcpy(P->d_fine, &P->op64[0], sizeof(Op<double>), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMallocHost(&P->h_out, 4 * sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "persistent setup");
  if (!coop || P->o.launch_mode != 0) return EB_OK;  // per-phase kernels
  int per_sm = 0, smax = 0;
  const bool sw = P->sweep_levels > 0;
  const void* fn = solve_kernel(mixed, sw);
  // the attribute is per kernel, shared by every handle: allow the device maximum once
  cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  smax -= 16 * 1024;  // headroom for the kernel's static shared memory
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_kernel(mixed, sw), cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  if (e == cudaSuccess && P->sweep_levels)
    e = cudaFuncSetAttribute((const void*)k_sweep_phase<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  if (e == cudaSuccess && P->sweep_levels)
    e = cudaFuncSetAttribute((const void*)k_restrict3d_phase<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smax);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PT, P->smem_bytes);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return EB_OK;
  }
  // CTAs per SM of the persistent kernel: fewer CTAs make the grid barrier
  // cheaper, more hide memory latency on the largest levels
  int want = 1;
  if (const char* env = std::getenv("EBP_CTAS_PER_SM")) want = std::max(1, std::atoi(env));
  P->grid = nsm * std::min(per_sm, want);
  P->persistent = true;
  return EB_OK;
}

static cudaError_t kernel_events(eb_poisson* P) {
  cudaError_t e = cudaSuccess;
  for (cudaEvent_t& k : P->kev)
    if (!k && e == cudaSuccess) e = cudaEventCreate(&k);
  return e;
}

static eb_status solve_persistent(eb_poisson* P, double* r, int* iters, int* cycles, int* status) {
  cudaStream_t s = P->s;
  cudaMemsetAsync(P->d_bar, 0, 4 * sizeof(unsigned), s);
  cudaMemsetAsync(P->d_norms, 0, sizeof(unsigned long long) * (P->o.max_cycles + 2), s);
  size_t dyn = (size_t)P->smem_bytes;
  SolveCtl ctl;
  ctl.tol = P->o.tol;
  ctl.max_cycles = P->o.max_cycles;
  ctl.mixed = P->o.precision == EB_PREC_MIXED;
  ctl.inner = ctl.mixed ? P->o.inner_cycles : 1;
  ctl.bnorm = (const double*)(P->d_norm + 1);
  ctl.norms = P->d_norms;
  ctl.out = P->d_out;
  ctl.trace = P->d_stamps;
  ctl.max_iters = 0;
  Barrier B{P->d_bar, (int*)(P->d_bar + 2)};
  void* args[4];
  cudaError_t e = kernel_events(P);
  if (e != cudaSuccess) return cuda_fail(e, "event");
  cudaEventRecord(P->kev[0], s);
  if (ctl.mixed) {
    const Hier<float>* H = (const Hier<float>*)P->d_hier;
    const Op<double>* F = P->d_fine;
    args[0] = (void*)&H;
    args[1] = (void*)&F;
    args[2] = (void*)&ctl;
    args[3] = (void*)&B;
    e = cudaLaunchCooperativeKernel(solve_kernel(true, P->sweep_levels > 0), dim3(P->grid), dim3(PT), args, dyn, s);
  } else {
    const Hier<double>* H = (const Hier<double>*)P->d_hier;
    const Op<double>* F = P->d_fine;
    args[0] = (void*)&H;
    args[1] = (void*)&F;
    args[2] = (void*)&ctl;
    args[3] = (void*)&B;
    e = cudaLaunchCooperativeKernel(solve_kernel(false, false), dim3(P->grid), dim3(PT), args, dyn, s);
  }
  counted();
  cudaEventRecord(P->kev[1], s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P->h_out, P->d_out, 4 * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "persistent solve");
  float kt = 0.0f;
  if (cudaEventElapsedTime(&kt, P->kev[0], P->kev[1]) == cudaSuccess) P->kernel_ms = kt;
  unsigned long long nv = 0;
  e = cudaMemcpy(&nv, P->d_norms + P->o.max_cycles + 1, sizeof(nv), cudaMemcpyDeviceToHost);
  unsigned bar[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(bar, P->d_bar, sizeof(bar), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "persistent readback");
  std::memcpy(r, &nv, sizeof(double));
  *iters = P->h_out[1];
  *cycles = P->h_out[2];
  *status = bar[2] ? EB_ERR_TIMEOUT : P->h_out[0];
  if (bar[2]) sweep_reset(P, s);
  return EB_OK;
}

extern "C" eb_status eb_poisson_setup(const eb_geom* G, const eb_solver_opts* opts, void* stream, eb_poisson** out) {
  if (!G || !out) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  *out = nullptr;
  eb_poisson* P = new eb_poisson();
  P->G = G;
  if (opts) P->o = *opts;
  else eb_solver_opts_default(&P->o);
  eb_solver_opts& o = P->o;
  const int nu_auto = G->L[0].g.D == 3 ? 6 : 2;
  if (o.nu1 == -1) o.nu1 = nu_auto;
  if (o.nu2 == -1) o.nu2 = nu_auto;
  if (!(o.tol > 0.0) || o.max_cycles < 1 || o.nu1 < 0 || o.nu2 < 0 || o.inner_cycles < 1 || o.bottom_sweeps < 1 ||
      (o.precision != EB_PREC_FP64 && o.precision != EB_PREC_MIXED) || o.launch_mode < 0 || o.launch_mode > 2) {
    delete P;
    set_error("invalid solver options");
    return EB_ERR_INVALID;
  }
  P->nlev = (int)G->L.size();
  eb_status st = EB_OK;
  int np = G->n_phase;
  const DevLevel& F = G->L[0];
  size_t n0 = (size_t)F.g.ncell;
  P->phi64 = (double*)dev_alloc(P->allocs, 2 * n0 * sizeof(double), &P->bytes, &st);
  P->b64 = (double*)dev_alloc(P->allocs, 2 * n0 * sizeof(double), &P->bytes, &st);
  P->d_norm = (unsigned long long*)dev_alloc(P->allocs, 2 * sizeof(unsigned long long), &P->bytes, &st);
  if (st == EB_OK) {
    cudaMemset(P->phi64, 0, 2 * n0 * sizeof(double));
    cudaMemset(P->b64, 0, 2 * n0 * sizeof(double));
  }
  // finest FP64 operator over the solver's own phi and b
  P->op64.push_back(make_op<double>(F, P->allocs, &P->bytes, &st, np, P->phi64, P->b64, P->phi64 + n0, P->b64 + n0));
  if (o.precision == EB_PREC_FP64) {
    for (int l = 1; l < P->nlev; ++l) P->op64.push_back(make_op<double>(G->L[l], P->allocs, &P->bytes, &st, np));
  } else {
    for (int l = 0; l < P->nlev; ++l) P->op32.push_back(make_op<float>(G->L[l], P->allocs, &P->bytes, &st, np));
  }
  if (st == EB_OK) {
    cudaError_t e = cudaStreamCreateWithFlags(&P->s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&P->h_norm, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = cuda_fail(e, "solver setup");
  }
  if (st == EB_OK) st = setup_persistent(P);
  if (st == EB_OK && o.launch_mode != 2 && !P->persistent) {
    cudaError_t e = cudaStreamBeginCapture(P->s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      g_count = &P->per_iter;
      iteration(P, P->s);
      g_count = nullptr;
      e = cudaStreamEndCapture(P->s, &P->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&P->gexec, P->graph, 0);
    if (e != cudaSuccess) st = cuda_fail(e, "graph capture");
  }
  (void)stream;
  if (st != EB_OK) {
    eb_poisson_destroy(P);
    return st;
  }
  *out = P;
  return EB_OK;
}

extern "C" void eb_poisson_destroy(eb_poisson* P) {
  if (!P) return;
  if (P->s) cudaStreamSynchronize(P->s);
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  if (P->graph) cudaGraphDestroy(P->graph);
  if (P->ev) cudaEventDestroy(P->ev);
  for (cudaEvent_t k : P->kev)
    if (k) cudaEventDestroy(k);
  if (P->s) cudaStreamDestroy(P->s);
  if (P->h_norm) cudaFreeHost(P->h_norm);
  if (P->h_out) cudaFreeHost(P->h_out);
  for (void* p : P->allocs) cudaFree(p);
  delete P;
}

static double as_double(unsigned long long v) {
  double d;
  std::memcpy(&d, &v, sizeof(d));
  return d;
}

// the solver's stream waits for the caller's, and the other way round at the end
static void join_in(eb_poisson* P, cudaStream_t user) {
  cudaEventRecord(P->ev, user);
  cudaStreamWaitEvent(P->s, P->ev, 0);
}
static void join_out(eb_poisson* P, cudaStream_t user) {
  cudaEventRecord(P->ev, P->s);
  cudaStreamWaitEvent(user, P->ev, 0);
}

static eb_status read_norms(eb_poisson* P, double* r, double* b) {
  cudaError_t e = cudaMemcpyAsync(P->h_norm, P->d_norm, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, P->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->s);
  if (e != cudaSuccess) return cuda_fail(e, "norm readback");
  *r = as_double(P->h_norm[0]);
  if (b) *b = as_double(P->h_norm[1]);
  return EB_OK;
}

__global__ void k_resid_field(Op<double> o, double* r) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= o.ncell) return;
  uint8_t f = o.flags[c];
  int I[3];
  ijk(o, c, I);
  for (int p = 0; p < 2; ++p) r[p * o.ncell + c] = ((f >> p) & 1) ? cell_residual(o, c, p, I) : 0.0;
}

// b (FP64 [2][n_cells]) of the finest level for the given data: kappa rhs
// plus the boundary and surface-charge terms; enqueued on s, no sync.
eb_status poisson_rhs(eb_poisson* P, const double* d_rhs, const double* d_sigma, double* d_b, cudaStream_t s) {
  cudaMemsetAsync(P->d_norm + 1, 0, sizeof(unsigned long long), s);
  return launch_rhs64(P->G, d_rhs, d_sigma, d_b, (double*)(P->d_norm + 1), s);
}

// r = b - A phi on the finest level for a b formed by poisson_rhs; phi is
// read as given (its entries without an unknown must be finite), the sparse
// rows use the handle's row scratch; enqueued on s, no sync.
eb_status poisson_residual_view(eb_poisson* P, const double* d_b, const double* d_phi, double* d_r, cudaStream_t s) {
  Op<double> o = P->op64[0];
  const long long n = o.ncell;
  o.x[0] = const_cast<double*>(d_phi);
  o.b[0] = const_cast<double*>(d_b);
  if (o.x[1]) {
    o.x[1] = const_cast<double*>(d_phi) + n;
    o.b[1] = const_cast<double*>(d_b) + n;
  }
  if (o.nirr) k_rows<double><<<blocks(2 * o.nirr), 256, 0, s>>>(o, 0, 2 * o.nirr, 1);
  k_resid_field<<<blocks(n), 256, 0, s>>>(o, d_r);
  counted(o.nirr ? 2 : 1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? EB_OK : cuda_fail(e, "residual");
}

extern "C" eb_status eb_poisson_residual(eb_poisson* P, const double* d_rhs, const double* d_sigma,
                                         const double* d_phi, double* d_r, void* stream) {
  if (!P || !d_rhs || !d_phi || !d_r) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  cudaStream_t user = (cudaStream_t)stream;
  const DevLevel& F = P->G->L[0];
  long long n = F.g.ncell;
  join_in(P, user);
  cudaMemsetAsync(P->d_norm + 1, 0, sizeof(unsigned long long), P->s);
  eb_status st = launch_rhs64(P->G, d_rhs, d_sigma, P->b64, (double*)(P->d_norm + 1), P->s);
  if (st != EB_OK) return st;
  k_copy_masked<<<blocks(n), 256, 0, P->s>>>(F.flags, n, d_phi, P->phi64);
  const Op<double>& o = P->op64[0];
  if (o.nirr) k_rows<double><<<blocks(2 * o.nirr), 256, 0, P->s>>>(o, 0, 2 * o.nirr, 1);
  k_resid_field<<<blocks(n), 256, 0, P->s>>>(o, d_r);
  counted(o.nirr ? 3 : 2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->s);
  join_out(P, user);
  return e == cudaSuccess ? EB_OK : cuda_fail(e, "residual");
}

extern "C" eb_status eb_poisson_solve(eb_poisson* P, const double* d_rhs, const double* d_sigma, double* d_phi,
                                      eb_solve_info* info, void* stream) {
  if (!P || !d_rhs || !d_phi) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  cudaStream_t user = (cudaStream_t)stream;
  const DevLevel& F = P->G->L[0];
  long long n = F.g.ncell;
  eb_solve_info inf;
  std::memset(&inf, 0, sizeof(inf));
  P->launches = 0;
  g_count = &P->launches;
  join_in(P, user);
  cudaMemsetAsync(P->d_norm + 1, 0, sizeof(unsigned long long), P->s);
  eb_status st = launch_rhs64(P->G, d_rhs, d_sigma, P->b64, (double*)(P->d_norm + 1), P->s);
  if (st != EB_OK) {
    g_count = nullptr;
    return st;
  }
  k_copy_masked<<<blocks(n), 256, 0, P->s>>>(F.flags, n, d_phi, P->phi64);
  counted(2);
  bool mixed = P->o.precision == EB_PREC_MIXED;
  if (P->persistent) {
    double r = 0.0, b = 0.0;
    int iters = 0, cycles = 0, status = 0;
    st = solve_persistent(P, &r, &iters, &cycles, &status);
    if (st == EB_OK) {
      cudaMemcpy(&b, P->d_norm + 1, sizeof(double), cudaMemcpyDeviceToHost);
      if (status == EB_ERR_NOT_CONVERGED) set_error("cycle cap reached or residual diverged");
      if (status == EB_ERR_TIMEOUT) set_error("a grid barrier wait gave up");
      st = (eb_status)status;
    }
    k_copy_masked<<<blocks(n), 256, 0, P->s>>>(F.flags, n, P->phi64, d_phi);
    counted();
    g_count = nullptr;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->s);
    if (e != cudaSuccess && st == EB_OK) st = cuda_fail(e, "solve");
    join_out(P, user);
    inf.kernel_launches = P->launches;
    inf.kernel_ms = P->kernel_ms;
    inf.status = st;
    inf.outer_iters = iters;
    inf.vcycles = cycles;
    inf.bnorm = b;
    inf.rel_res = b > 0.0 ? r / b : 0.0;
    inf.bottom = P->bottom;
    inf.levels = P->nlev;
    inf.sweep_levels = P->sweep_levels;
    if (info) *info = inf;
    return st;
  }
  resid64(P, P->s, mixed);
  double r = 0.0, b = 0.0;
  st = read_norms(P, &r, &b);
  if (st != EB_OK) return st;
  inf.bnorm = b;
  double r0 = r;
  int cycles = 0, outer = 0;
  st = EB_OK;
  if (b == 0.0) {
    cudaMemsetAsync(P->phi64, 0, 2 * n * sizeof(double), P->s);
    r = 0.0;
  } else {
    int per = mixed ? P->o.inner_cycles : 1;
    while (r > P->o.tol * b) {
      if (cycles + per > P->o.max_cycles || !std::isfinite(r) || r > 1e6 * r0) {
        st = EB_ERR_NOT_CONVERGED;
        set_error("cycle cap reached or residual diverged");
        break;
      }
      cudaError_t e = P->gexec ? cudaGraphLaunch(P->gexec, P->s) : cudaSuccess;
      if (!P->gexec) iteration(P, P->s);
      else counted((int)P->per_iter);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess) {
        st = cuda_fail(e, "iteration");
        break;
      }
      cycles += per;
      ++outer;
      eb_status rs = read_norms(P, &r, nullptr);
      if (rs != EB_OK) {
        st = rs;
        break;
      }
    }
  }
  k_copy_masked<<<blocks(n), 256, 0, P->s>>>(F.flags, n, P->phi64, d_phi);
  counted();
  g_count = nullptr;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->s);
  if (e != cudaSuccess && st == EB_OK) st = cuda_fail(e, "solve");
  join_out(P, user);
  inf.kernel_launches = P->launches;
  inf.status = st;
  inf.outer_iters = outer;
  inf.vcycles = cycles;
  inf.rel_res = b > 0.0 ? r / b : 0.0;
  inf.bottom = EB_BOTTOM_RELAX;  // the per-phase paths relax the coarsest level
  inf.levels = P->nlev;
  inf.sweep_levels = 0;  // the per-phase paths relax by colour passes
  if (info) *info = inf;
  return st;
}


// ------------------------------------------------------------------ batches

// CTAs per instance for a batch on `total` CTAs: one each, the rest in
// proportion to the instances' cell counts (largest remainders), at most
// `cap` per instance.
// An instance with tile-streamed sweeps takes at least two CTAs (its CTA 0
// sits the sweeps out), given in `mins`.
static std::vector<int> split_ctas(const std::vector<long long>& cells, int total, int cap,
                                   const std::vector<int>& mins) {
  int n = (int)cells.size();
  std::vector<int> size(mins);
  long long sum = 0;
  int used = 0;
  for (long long c : cells) sum += c;
  for (int m : mins) used += m;
  int left = total - used;
  if (left <= 0 || sum <= 0) return size;
  std::vector<std::pair<double, int>> rem;
  int given = 0;
  for (int i = 0; i < n; ++i) {
    double share = (double)left * (double)cells[i] / (double)sum;
    int whole = std::max(0, std::min((int)share, cap - size[i]));
    size[i] += whole;
    given += whole;
    rem.push_back({share - whole, i});
  }
  std::sort(rem.begin(), rem.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
    return a.first > b.first || (a.first == b.first && a.second < b.second);
  });
  for (int k = 0; k < (int)rem.size() && given < left; ++k) {
    int i = rem[k].second;
    if (size[i] < cap) {
      ++size[i];
      ++given;
    }
  }
  return size;
}

template <class T>
static eb_status launch_batch_t(eb_poisson* const* P, int n, int max_iters, int grid_total, int smem, cudaStream_t s,
                                double* kernel_ms) {
  std::vector<long long> cells(n);
  for (int i = 0; i < n; ++i) cells[i] = P[i]->G->L[0].g.ncell;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P[0]->G->device);
  std::vector<int> mins(n);
  for (int i = 0; i < n; ++i) mins[i] = P[i]->sweep_levels ? 2 : 1;
  std::vector<int> size = split_ctas(cells, grid_total, std::max(2, nsm), mins);
  std::vector<BatchItem<T>> items(n);
  std::vector<int> cta_item;
  int start = 0;
  for (int i = 0; i < n; ++i) {
    eb_poisson* Q = P[i];
    BatchItem<T>& it = items[i];
    it.H = (const Hier<T>*)Q->d_hier;
    it.F = Q->d_fine;
    SolveCtl& c = it.ctl;
    c.tol = Q->o.tol;
    c.max_cycles = Q->o.max_cycles;
    c.mixed = Q->o.precision == EB_PREC_MIXED;
    c.inner = c.mixed ? Q->o.inner_cycles : 1;
    c.bnorm = (const double*)(Q->d_norm + 1);
    c.norms = Q->d_norms;
    c.out = Q->d_out;
    c.trace = Q->d_stamps;
    c.max_iters = max_iters;
    it.B = Barrier{Q->d_bar, (int*)(Q->d_bar + 2)};
    it.start = start;
    it.size = size[i];
    for (int k = 0; k < size[i]; ++k) cta_item.push_back(i);
    start += size[i];
    cudaMemsetAsync(Q->d_bar, 0, 4 * sizeof(unsigned), s);
    cudaMemsetAsync(Q->d_norms, 0, sizeof(unsigned long long) * (Q->o.max_cycles + 2), s);
  }
  BatchItem<T>* d_items = nullptr;
  int* d_cta = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d_items, sizeof(BatchItem<T>) * n, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_cta, sizeof(int) * cta_item.size(), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_items, items.data(), sizeof(BatchItem<T>) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_cta, cta_item.data(), sizeof(int) * cta_item.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = kernel_events(P[0]);
  if (e == cudaSuccess) {
    void* args[2] = {(void*)&d_items, (void*)&d_cta};
    cudaEventRecord(P[0]->kev[0], s);
    bool sw = false;
    for (int i = 0; i < n; ++i) sw = sw || P[i]->sweep_levels > 0;
    e = cudaLaunchCooperativeKernel(batch_kernel(std::is_same<T, float>::value, sw), dim3(start), dim3(PT), args,
                                    (size_t)smem, s);
    cudaEventRecord(P[0]->kev[1], s);
    counted();
  }
  if (d_items) cudaFreeAsync(d_items, s);
  if (d_cta) cudaFreeAsync(d_cta, s);
  // the host vectors must outlive the copies above
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  float kt = 0.0f;
  if (e == cudaSuccess && cudaEventElapsedTime(&kt, P[0]->kev[0], P[0]->kev[1]) == cudaSuccess && kernel_ms)
    *kernel_ms += kt;
  return e == cudaSuccess ? EB_OK : cuda_fail(e, "batched solve");
}

// An instance's right-hand side assembled into b and its guess copied in,
// ready for batch_step(fresh = false).
eb_status batch_prepare(eb_poisson* P, const double* rhs, const double* sigma, const double* phi, cudaStream_t s) {
  const DevLevel& F = P->G->L[0];
  cudaMemsetAsync(P->d_norm + 1, 0, sizeof(unsigned long long), s);
  eb_status st = launch_rhs64(P->G, rhs, sigma, P->b64, (double*)(P->d_norm + 1), s);
  if (st != EB_OK) return st;
  k_copy_masked<<<blocks(F.g.ncell), 256, 0, s>>>(F.flags, F.g.ncell, phi, P->phi64);
  counted(2);
  return EB_OK;
}

// The instance's current iterate copied out (entries without an unknown = 0).
eb_status batch_copy_out(eb_poisson* P, double* phi, cudaStream_t s) {
  const DevLevel& F = P->G->L[0];
  k_copy_masked<<<blocks(F.g.ncell), 256, 0, s>>>(F.flags, F.g.ncell, P->phi64, phi);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? EB_OK : cuda_fail(e, "copy out");
}

long long poisson_device_bytes(const eb_poisson* P) { return P->bytes; }

// A x = b for a right-hand side given in integrated form (boundary data not
// added: a correction equation with homogeneous data), from x = 0, to
// max|r| <= tol max|b|.  d_b and d_x are [2][ncell] on `user`'s stream.
eb_status poisson_solve_b(eb_poisson* P, const double* d_b, double* d_x, double tol, int* cycles, cudaStream_t user,
                          int* outer, double* kernel_ms) {
  if (!P->persistent) {
    set_error("correction solves need the persistent path");
    return EB_ERR_UNSUPPORTED;
  }
  const DevLevel& F = P->G->L[0];
  long long n = F.g.ncell;
  join_in(P, user);
  k_copy_masked<<<blocks(n), 256, 0, P->s>>>(F.flags, n, d_b, P->b64);
  cudaMemsetAsync(P->d_norm + 1, 0, sizeof(unsigned long long), P->s);
  k_absmax_masked<<<blocks(n), 256, 0, P->s>>>(F.flags, n, P->b64, P->d_norm + 1);
  counted(2);
  cudaMemsetAsync(P->phi64, 0, 2 * n * sizeof(double), P->s);
  double keep = P->o.tol;
  P->o.tol = tol;
  double r = 0.0;
  int iters = 0, cyc = 0, status = 0;
  eb_status st = solve_persistent(P, &r, &iters, &cyc, &status);
  P->o.tol = keep;
  if (st == EB_OK && status != EB_OK && status != EB_ERR_NOT_CONVERGED) st = (eb_status)status;
  k_copy_masked<<<blocks(n), 256, 0, P->s>>>(F.flags, n, P->phi64, d_x);
  counted();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess && st == EB_OK) st = cuda_fail(e, "correction solve");
  join_out(P, user);
  if (cycles) *cycles = cyc;
  if (outer) *outer = iters;
  if (kernel_ms) *kernel_ms = P->kernel_ms;
  return st;
}

// One cooperative launch over instances that share precision and device.
// fresh: assemble b and copy the guess in first; max_iters: outer iterations
// allowed (0: until convergence).  Results (status, iterations, V-cycles,
// residual) are read into each handle's pinned h_out / h_norm.
eb_status batch_step(eb_poisson* const* P, int n, const double* const* rhs, const double* const* sigma,
                     double* const* phi, bool fresh, bool copy_out, int max_iters, cudaStream_t s,
                     double* kernel_ms) {
  if (n < 1) return EB_OK;
  bool mixed = P[0]->o.precision == EB_PREC_MIXED;
  int smem = 0;
  for (int i = 0; i < n; ++i) {
    if ((P[i]->o.precision == EB_PREC_MIXED) != mixed || !P[i]->persistent || P[i]->G->device != P[0]->G->device) {
      set_error("a batch needs persistent solvers of one precision on one device");
      return EB_ERR_INVALID;
    }
    smem = std::max(smem, P[i]->smem_bytes);
  }
  int nsm = 0, per_sm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P[0]->G->device);
  cudaError_t e = cudaSuccess;
  bool sw = false;
  for (int i = 0; i < n; ++i) sw = sw || P[i]->sweep_levels > 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel(mixed, sw), PT, smem);
  if (e != cudaSuccess || per_sm < 1) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidConfiguration : e, "batch occupancy");
  int total = nsm * std::min(per_sm, 1);
  if (fresh)
    for (int i = 0; i < n; ++i) {
      eb_status st = batch_prepare(P[i], rhs[i], sigma ? sigma[i] : nullptr, phi[i], s);
      if (st != EB_OK) return st;
    }
  // as many instances per launch as their minimum CTA counts allow
  for (int b0 = 0, m = 0; b0 < n; b0 += m) {
    int need = 0;
    for (m = 0; b0 + m < n; ++m) {
      const int c = P[b0 + m]->sweep_levels ? 2 : 1;
      if (need + c > total) break;
      need += c;
    }
    if (m == 0) m = 1;  // (total >= 2 on every device with a persistent kernel)
    eb_status st = mixed ? launch_batch_t<float>(P + b0, m, max_iters, total, smem, s, kernel_ms)
                         : launch_batch_t<double>(P + b0, m, max_iters, total, smem, s, kernel_ms);
    if (st != EB_OK) return st;
  }
  for (int i = 0; i < n; ++i) {
    if (copy_out) {
      const DevLevel& F = P[i]->G->L[0];
      k_copy_masked<<<blocks(F.g.ncell), 256, 0, s>>>(F.flags, F.g.ncell, P[i]->phi64, phi[i]);
      counted();
    }
    cudaMemcpyAsync(P[i]->h_out, P[i]->d_out, 4 * sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(P[i]->h_norm, P[i]->d_norms + P[i]->o.max_cycles + 1, sizeof(unsigned long long),
                    cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(P[i]->h_norm + 1, P[i]->d_norm + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "batched solve");
  for (int i = 0; i < n; ++i)
    if (P[i]->h_out[0] == EB_ERR_TIMEOUT) sweep_reset(P[i], s);
  return EB_OK;
}

void batch_info(eb_poisson* Q, eb_solve_info* inf) {
  std::memset(inf, 0, sizeof(*inf));
  double r = as_double(Q->h_norm[0]), b = as_double(Q->h_norm[1]);
  inf->status = Q->h_out[0];
  inf->outer_iters = Q->h_out[1];
  inf->vcycles = Q->h_out[2];
  inf->bnorm = b;
  inf->rel_res = b > 0.0 ? r / b : 0.0;
  inf->bottom = Q->bottom;
  inf->levels = Q->nlev;
  inf->sweep_levels = Q->sweep_levels;
}

extern "C" eb_status eb_poisson_solve_batched(eb_poisson* const* P, int n, const double* const* d_rhs,
                                              const double* const* d_sigma, double* const* d_phi,
                                              eb_solve_info* infos, void* stream) {
  if (!P || n < 0 || (n && (!d_rhs || !d_phi))) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  for (int i = 0; i < n; ++i)
    if (!P[i] || !d_rhs[i] || !d_phi[i]) {
      set_error("null instance");
      return EB_ERR_INVALID;
    }
  {  // a handle twice in one batch would have two CTA groups share its work arrays and barrier
    std::vector<eb_poisson*> h(P, P + n);
    std::sort(h.begin(), h.end());
    if (std::adjacent_find(h.begin(), h.end()) != h.end()) {
      set_error("a solver handle appears twice in the batch");
      return EB_ERR_INVALID;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  long long launches = 0;
  g_count = &launches;
  double kms = 0.0;
  eb_status st = batch_step(P, n, d_rhs, d_sigma, d_phi, true, true, 0, s, &kms);
  g_count = nullptr;
  if (st != EB_OK) return st;
  eb_status worst = EB_OK;
  for (int i = 0; i < n; ++i) {
    eb_solve_info inf;
    batch_info(P[i], &inf);
    inf.kernel_launches = launches;
    inf.kernel_ms = kms;
    if (infos) infos[i] = inf;
    if (inf.status != EB_OK && worst == EB_OK) worst = (eb_status)inf.status;
  }
  if (worst == EB_ERR_NOT_CONVERGED) set_error("an instance reached its cycle cap");
  if (worst == EB_ERR_TIMEOUT) set_error("a grid barrier wait gave up");
  return worst;
}

extern "C" eb_status eb_field_eval(eb_poisson* P, const double* d_phi, const double* d_sigma, double* d_E,
                                   double* d_En, void* stream) {
  if (!P || !d_phi) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  cudaStream_t user = (cudaStream_t)stream;
  join_in(P, user);
  eb_status st = launch_field(P->G, d_phi, d_sigma, d_E, d_En, P->s);
  cudaError_t e = cudaStreamSynchronize(P->s);
  join_out(P, user);
  if (st != EB_OK) return st;
  return e == cudaSuccess ? EB_OK : cuda_fail(e, "field");
}

extern "C" eb_status eb_poisson_profile(eb_poisson* P, int kernel, int reps, double* ms, double* bytes, void* stream) {
  if (P && kernel == 2 && reps >= 1 && ms && bytes) {
    if (!P->persistent) {
      set_error("no persistent kernel on this device");
      return EB_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(P->d_bar, 0, 4 * sizeof(unsigned), s);
    Barrier B{P->d_bar, (int*)(P->d_bar + 2)};
    void* args[2] = {(void*)&B, (void*)&reps};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_barrier_bench, dim3(P->grid), dim3(PT), args, 0, s);
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "barrier benchmark");
    *ms = (double)t / reps;
    *bytes = (double)P->grid;
    return EB_OK;
  }
  if (P && kernel == 3 && ms && bytes) {
    // a grid barrier that nobody completes: the bounded wait must expire and
    // report EB_ERR_TIMEOUT with the context still usable
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(P->d_bar, 0, 4 * sizeof(unsigned), s);
    Barrier B{P->d_bar, (int*)(P->d_bar + 2)};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    k_barrier_expiry<<<2, PT, 0, s>>>(B);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    unsigned bar[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(bar, P->d_bar, sizeof(bar), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "barrier expiry test");
    *ms = (double)t;
    *bytes = 0.0;
    if (bar[2]) {
      set_error("a grid barrier wait gave up");
      return EB_ERR_TIMEOUT;
    }
    return EB_OK;
  }
  if (P && (kernel == 4 || kernel == 5) && reps >= 1 && ms && bytes) {
    // kernel 4: one tile-streamed sweep (both colours) of the finest level on
    // its own; kernel 5: the streamed residual + restriction of that level
    if (!P->persistent || P->o.precision != EB_PREC_MIXED || P->sweep_first != 0 || P->nlev < 2) {
      set_error("the finest level has no tile-streamed sweep");
      return EB_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(P->d_bar, 0, 4 * sizeof(unsigned), s);
    int* err = (int*)(P->d_bar + 2);
    const Hier<float>* H = (const Hier<float>*)P->d_hier;
    const size_t dyn = (size_t)P->sweep_bytes;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto go = [&]() {
      if (kernel == 4) k_sweep_phase<float><<<P->grid, PT, dyn, s>>>(H, 0, err);
      else k_restrict3d_phase<float><<<P->grid, PT, dyn, s>>>(H, 0, err);
    };
    go();
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps; ++i) go();
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    unsigned bar[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(bar, P->d_bar, sizeof(bar), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "sweep profile");
    if (bar[2]) {
      sweep_reset(P, s);
      set_error("a sweep wait gave up");
      return EB_ERR_TIMEOUT;
    }
    *ms = (double)t / reps;
    // sweep: read x and b, write x (4 bytes each), read the flag byte, per cell;
    // restriction: read x and b, the flag byte, write coarse b and x (8 / 8 bytes)
    *bytes = (double)P->G->L[0].g.ncell * (kernel == 4 ? 13.0 : 10.0);
    return EB_OK;
  }
  if (!P || reps < 1 || (kernel != 0 && kernel != 1 && kernel != 6) || !ms || !bytes) {
    set_error("invalid argument");
    return EB_ERR_INVALID;
  }
  if ((kernel == 1 || kernel == 6) && P->nlev < 2) {
    set_error("no coarse level");
    return EB_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  bool mixed = P->o.precision == EB_PREC_MIXED;
  long long n = P->G->L[0].g.ncell;
  int D = P->G->L[0].g.D;
  double tb = mixed ? 4.0 : 8.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // the persistent kernel's own phase code, in its grid shape when it has one
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P->G->device);
  const int grid = P->persistent ? P->grid : nsm;
  auto launch = [&](int i) {
    if (kernel == 0) {
      if (mixed) k_dense_phase<float><<<grid, PT, 0, s>>>(P->op32[0], i & 1);
      else k_dense_phase<double><<<grid, PT, 0, s>>>(P->op64[0], i & 1);
    } else if (kernel == 1) {
      if (mixed) k_restrict_phase<float><<<grid, PT, 0, s>>>(P->op32[0], P->op32[1]);
      else k_restrict_phase<double><<<grid, PT, 0, s>>>(P->op64[0], P->op64[1]);
    } else {
      if (mixed) k_prolong_phase<float><<<grid, PT, 0, s>>>(P->op32[0], P->op32[1]);
      else k_prolong_phase<double><<<grid, PT, 0, s>>>(P->op64[0], P->op64[1]);
    }
  };
  launch(0);
  cudaEventRecord(e0, s);
  for (int i = 0; i < reps; ++i) launch(i);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "profile");
  *ms = (double)t / reps;
  if (kernel == 0) *bytes = (double)n * (3.0 * tb + 1.0) / 2.0;
  else if (kernel == 1) *bytes = (double)n * (2.0 * tb + 1.0) + (double)n / (double)(1 << D) * 2.0 * tb;
  else *bytes = (double)n * (2.0 * tb + 1.0) + (double)n / (double)(1 << D) * (tb + 1.0);
  return EB_OK;
}

// ------------------------------------------------------- arithmetic peaks

// 8 independent fused multiply-add chains per thread, `iters` steps each;
// the result is stored so that no chain is dead code
template <class T>
__global__ void k_fma_rate(T* out, int iters, T a, T b) {
  T v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = fma(v[k], a, b);
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += v[k];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
static eb_status fma_rate(int device, double* tflops) {
  int nsm = 0, dev0 = 0;
  cudaGetDevice(&dev0);
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  const int blocks = nsm * 8, threads = 256, iters = 1 << 14;
  T* out = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.0f;
  if (e == cudaSuccess) {
    k_fma_rate<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e0);
    for (int r = 0; r < 5; ++r) k_fma_rate<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  cudaSetDevice(dev0);
  if (e != cudaSuccess) return cuda_fail(e, "arithmetic rate");
  // two flops per fused multiply-add
  *tflops = 2.0 * 8.0 * iters * (double)blocks * threads * 5.0 / (ms * 1e-3) / 1e12;
  return EB_OK;
}

extern "C" eb_status eb_device_fma_rates(int device, double* fp64_tflops, double* fp32_tflops) {
  if (!fp64_tflops || !fp32_tflops) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  eb_status st = fma_rate<double>(device, fp64_tflops);
  if (st == EB_OK) st = fma_rate<float>(device, fp32_tflops);
  return st;
}

extern "C" eb_status eb_poisson_trace(eb_poisson* P, double* out, int n) {
  if (!P || !out || n < 1) {
    set_error("invalid argument");
    return EB_ERR_INVALID;
  }
  if (!P->d_stamps || !P->persistent) {
    set_error("no trace on this path");
    return EB_ERR_UNSUPPORTED;
  }
  std::vector<unsigned long long> t(TRMAX + 1);
  cudaError_t e = cudaMemcpy(t.data(), P->d_stamps, sizeof(unsigned long long) * (TRMAX + 1), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "trace");
  long long cnt = std::min<long long>((long long)t[0], TRMAX);
  // entry k > 0: phase that ended at stamp k, duration since stamp k-1
  int m = 0;
  for (long long k = 1; k < cnt && 1 + 2 * (m + 1) <= n; ++k) {
    unsigned long long a = t[k] & 0xffffffffffffULL, b = t[1 + k] & 0xffffffffffffULL;
    out[1 + 2 * m] = (double)(t[1 + k] >> 48);
    out[2 + 2 * m] = (double)(b - a) * 1e-6;
    ++m;
  }
  out[0] = m;
  return EB_OK;
}

// ------------------------------------------------------- allocation-free residual
//
// Some callers cannot allocate device memory at the point where they need a
// residual: code running inside a region that forbids cudaMalloc (a memory
// pool that is already fully carved up, a real-time loop that must not touch
// the allocator, a host thread that holds the device only between other
// users' allocations).  For them the residual below keeps its right-hand side
// and sparse-row scratch in one file-scope device array instead of memory
// owned by a solver handle.  The array is NA_MAX_CELLS * 2 + NA_MAX_ROWS + 8
// doubles (about 20.1 MB) and stays allocated on every device that loads the
// library until the process exits.

static constexpr long long NA_MAX_CELLS = 1LL << 20;  // cells of the finest level (e.g. 1024^2)
static constexpr long long NA_MAX_ROWS = 1LL << 19;   // sparse rows (two per irregular cell)
static __device__ __align__(256) double g_na_scratch[NA_MAX_CELLS * 2 + NA_MAX_ROWS + 8];

// Resolves the device address of the static array on the current device.
// It is looked up on every call (a cheap host call): an address cached per
// device ordinal would go stale once the context is torn down and created
// again (cudaDeviceReset), since the module is then loaded afresh.  The first
// call on a device may load the module, so it should come before any stream
// capture.
static eb_status na_scratch(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "static scratch address");
  *out = (double*)p;
  return EB_OK;
}

extern "C" eb_status eb_poisson_residual_noalloc(const eb_geom* G, const double* d_rhs, const double* d_sigma,
                                                 const double* d_phi, double* d_r, void* stream) {
  if (!G || !d_rhs || !d_phi || !d_r) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  const DevLevel& F = G->L[0];
  long long n = F.g.ncell, nrow = 2 * F.nirr;
  if (n > NA_MAX_CELLS) {
    set_error("problem exceeds the static scratch of the allocation-free residual: " + std::to_string(n) +
              " cells, at most " + std::to_string(NA_MAX_CELLS));
    return EB_ERR_INVALID;
  }
  if (nrow > NA_MAX_ROWS) {
    set_error("problem exceeds the static scratch of the allocation-free residual: " + std::to_string(nrow) +
              " sparse rows, at most " + std::to_string(NA_MAX_ROWS) + " (the sparse-row limit)");
    return EB_ERR_INVALID;
  }
  // the geometry's arrays live on the device it was built on; the static
  // array used is the current device's, so the two must be the same device
  int dev = -1;
  cudaError_t ed = cudaGetDevice(&dev);
  if (ed != cudaSuccess) return cuda_fail(ed, "device query");
  if (dev != G->device) {
    set_error("the current device (" + std::to_string(dev) + ") is not the geometry's device (" +
              std::to_string(G->device) + ")");
    return EB_ERR_INVALID;
  }
  double* base = nullptr;
  eb_status st = na_scratch(&base);
  if (st != EB_OK) return st;
  double* b = base;                       // [2][n] right-hand side
  double* tmp = base + 2 * NA_MAX_CELLS;  // [nrow] sparse-row residuals
  double* bnorm = tmp + NA_MAX_ROWS;      // max|b| (not returned)
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(bnorm, 0, sizeof(double), s);
  if (e != cudaSuccess) return cuda_fail(e, "scratch clear");
  st = launch_rhs64(G, d_rhs, d_sigma, b, bnorm, s);
  if (st != EB_OK) return st;
  // a view of the finest operator over the caller's phi and the static b
  Op<double> o;
  std::memset(&o, 0, sizeof(o));
  o.D = F.g.D;
  for (int k = 0; k < 3; ++k) o.n[k] = F.g.n[k];
  o.dn0 = make_fastdiv((unsigned)F.g.n[0]);
  o.dn1 = make_fastdiv((unsigned)F.g.n[1]);
  o.dhx = make_fastdiv((unsigned)((F.g.n[0] + 1) / 2));
  o.dq = make_fastdiv((unsigned)std::max(1, F.g.n[0] / 4));
  o.ncell = n;
  set_stencil_terms(o, F.g);
  o.x[0] = const_cast<double*>(d_phi);
  o.x[1] = const_cast<double*>(d_phi) + n;
  o.b[0] = b;
  o.b[1] = b + n;
  o.flags = F.flags;
  o.irr_cell = F.irr_cell;
  o.irr_of_cell = F.irr_of_cell;
  o.row_ptr = F.row_ptr;
  o.col = F.col;
  o.val = F.val;
  o.diag = F.diag;
  o.tmp = tmp;
  o.nirr = F.nirr;
  o.nirr_red = F.nirr_red;
  for (int p = 0; p < 2; ++p) {
    double h2 = F.g.h * F.g.h;
    o.ceps[p] = F.g.eps[p] / h2;
    o.h2e[p] = h2 / F.g.eps[p];
  }
  if (nrow) k_rows<double><<<blocks(nrow), 256, 0, s>>>(o, 0, nrow, 1);
  k_resid_field<<<blocks(n), 256, 0, s>>>(o, d_r);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? EB_OK : cuda_fail(e, "allocation-free residual");
}

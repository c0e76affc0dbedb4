// geometry.cu -- cut-cell geometry, multigrid coarsening and operator rows
// (arXiv:1809.03745, Sec. 3.1, 3.3, 3.3.1).  Setup-time work: compiled
// without FMA contraction so the geometry is reproducible bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "eb_internal.h"
#include "coarsen_impl.cuh"
#include "stencil_impl.cuh"

namespace ebp {

// ------------------------------------------------------------ compaction
// Stream compaction in ascending index order: per-block counts, one-block
// exclusive scan of the counts, per-block ballot scan and write.

constexpr int CB = 1024;

template <class Pred>
__global__ void k_pred_count(Pred pred, long long n, int* counts) {
  long long i = (long long)blockIdx.x * CB + threadIdx.x;
  int v = (i < n) && pred(i);
  int c = __syncthreads_count(v);
  if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

__global__ void k_scan_counts(int* counts, int nb, long long* total) {
  __shared__ long long sh[CB];
  int t = threadIdx.x;
  int per = (nb + CB - 1) / CB;
  int beg = t * per, end = min(nb, beg + per);
  long long s = 0;
  for (int i = beg; i < end; ++i) s += counts[i];
  sh[t] = s;
  __syncthreads();
  for (int off = 1; off < CB; off <<= 1) {
    long long v = t >= off ? sh[t - off] : 0;
    __syncthreads();
    sh[t] += v;
    __syncthreads();
  }
  long long run = sh[t] - s;
  for (int i = beg; i < end; ++i) {
    int c = counts[i];
    counts[i] = (int)run;
    run += c;
  }
  if (t == CB - 1) *total = sh[CB - 1];
}

template <class Pred>
__global__ void k_pred_write(Pred pred, long long n, const int* offsets, int* out) {
  __shared__ int wc[CB / 32];
  long long i = (long long)blockIdx.x * CB + threadIdx.x;
  int v = (i < n) && pred(i);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned mask = __ballot_sync(0xffffffffu, v);
  int wpre = __popc(mask & ((1u << lane) - 1u));
  if (lane == 0) wc[warp] = __popc(mask);
  __syncthreads();
  if (warp == 0) {
    int x = wc[lane];
    int inc = x;
    for (int off = 1; off < 32; off <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += y;
    }
    wc[lane] = inc - x;
  }
  __syncthreads();
  if (v) out[offsets[blockIdx.x] + wc[warp] + wpre] = (int)i;
}

struct Scratch {
  std::vector<void*> bufs;
  ~Scratch() {
    for (void* p : bufs) cudaFree(p);
  }
  template <class T>
  T* get(size_t n) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return nullptr;
    bufs.push_back(p);
    return (T*)p;
  }
};

// Compacts the indices i < n with pred(i) into a new device array; returns count.
template <class Pred>
eb_status compact(Pred pred, long long n, int** out, long long* count, std::vector<void*>& owner,
                  long long* bytes, cudaStream_t s) {
  Scratch S;
  int nb = (int)((n + CB - 1) / CB);
  if (nb < 1) nb = 1;
  int* counts = S.get<int>(nb);
  long long* total = S.get<long long>(1);
  if (!counts || !total) return EB_ERR_OOM;
  k_pred_count<<<nb, CB, 0, s>>>(pred, n, counts);
  k_scan_counts<<<1, CB, 0, s>>>(counts, nb, total);
  long long tot = 0;
  cudaError_t e = cudaMemcpyAsync(&tot, total, sizeof(tot), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "compaction");
  eb_status st = EB_OK;
  int* o = (int*)dev_alloc(owner, (size_t)std::max<long long>(tot, 1) * sizeof(int), bytes, &st);
  if (st != EB_OK) return st;
  k_pred_write<<<nb, CB, 0, s>>>(pred, n, counts, o);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "compaction write");
  *out = o;
  *count = tot;
  return EB_OK;
}

// exclusive scan of an int array of length n into out[0..n] (out[n] = total)
__global__ void k_block_sums(const int* in, long long n, long long* sums) {
  __shared__ long long sh[CB];
  long long i = (long long)blockIdx.x * CB + threadIdx.x;
  sh[threadIdx.x] = i < n ? in[i] : 0;
  __syncthreads();
  for (int off = CB / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = sh[0];
}
__global__ void k_scan_sums(long long* sums, int nb) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    long long run = 0;
    for (int b = 0; b < nb; ++b) {
      long long v = sums[b];
      sums[b] = run;
      run += v;
    }
    sums[nb] = run;
  }
}
__global__ void k_block_scan(const int* in, long long n, const long long* sums, int* out, int nb) {
  __shared__ long long sh[CB];
  long long i = (long long)blockIdx.x * CB + threadIdx.x;
  long long v = i < n ? in[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < CB; off <<= 1) {
    long long y = (int)threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += y;
    __syncthreads();
  }
  if (i < n) out[i] = (int)(sums[blockIdx.x] + sh[threadIdx.x] - v);
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (int)sums[nb];
}

eb_status exclusive_scan(const int* in, long long n, int* out, long long* total, cudaStream_t s) {
  Scratch S;
  int nb = (int)((n + CB - 1) / CB);
  if (nb < 1) nb = 1;
  long long* sums = S.get<long long>(nb + 1);
  if (!sums) return EB_ERR_OOM;
  k_block_sums<<<nb, CB, 0, s>>>(in, n, sums);
  k_scan_sums<<<1, 32, 0, s>>>(sums, nb);
  k_block_scan<<<nb, CB, 0, s>>>(in, n, sums, out, nb);
  cudaError_t e = cudaMemcpyAsync(total, sums + nb, sizeof(long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "scan");
  return EB_OK;
}

// ------------------------------------------------------------- predicates

struct PredEq {
  const uint8_t* v;
  uint8_t val;
  __device__ bool operator()(long long i) const { return v[i] == val; }
};
struct PredNonzero {
  const uint8_t* v;
  __device__ bool operator()(long long i) const { return v[i] != 0; }
};
struct PredIrrColour {
  Grid g;
  const uint8_t* flags;
  int colour;
  __device__ bool operator()(long long c) const {
    if (!(flags[c] & F_IRR)) return false;
    int I[3];
    cell_ijk(g, c, I);
    return ((I[0] + I[1] + I[2]) & 1) == colour;
  }
};

// ------------------------------------------------------------- kernels

constexpr int TB = 256;
inline int nblk(long long n, int tb = TB) { return (int)std::max<long long>(1, (n + tb - 1) / tb); }

__global__ void k_labels(const Csg* csg, Grid g, uint8_t* lab) {
  long long nn = node_count(g);
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  long long nx = g.n[0] + 1, ny = g.n[1] + 1;
  int I[3] = {(int)(i % nx), (int)((i / nx) % ny), (int)(i / (nx * ny))};
  double x[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < g.D; ++k) x[k] = node_x(g, k, I[k]);
  lab[i] = (uint8_t)label_at(*csg, x);
}

// 0 covered, 1 regular gas, 2 regular dielectric, 3 cut
__global__ void k_preclass(Grid g, const uint8_t* lab, uint8_t* pre) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  int I[3];
  cell_ijk(g, c, I);
  int nc = 1 << g.D;
  int first = -1;
  bool uni = true;
  for (int k = 0; k < nc; ++k) {
    int N[3] = {I[0] + (k & 1), I[1] + ((k >> 1) & 1), I[2] + ((k >> 2) & 1)};
    int l = lab[node_index(g, N)];
    if (first < 0) first = l;
    else if (l != first) uni = false;
  }
  pre[c] = uni ? (uint8_t)first : (uint8_t)3;
}

__global__ void k_map(const int* list, long long n, int* map) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) map[list[i]] = (int)i;
}

__global__ void k_cut_geom(const Csg* csg, Grid g, const uint8_t* lab, CutRecords R, int* status) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= R.ncut) return;
  int st = cut_cell_geometry(*csg, g, lab, R.cell[q], R, q);
  if (st) atomicOr(status, st);
}

// unknowns of cut fragments: an open interior or Dirichlet face (a fragment
// of zero volume with such a face carries its EB's boundary condition)
__global__ void k_dofs(Grid g, CutRecords R) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= R.ncut) return;
  int I[3];
  cell_ijk(g, R.cell[q], I);
  uint8_t m = 0;
  for (int p = 0; p < 2; ++p)
    if (record_open_face(g, R, q, I, p)) m |= (uint8_t)(1 << p);
  R.dofm[q] = m;
  // an interface cell that keeps a single fragment (the interface runs
  // through a node, or the other fragment has no open face) carries no
  // interface flux
  if (R.ebk[q] == EBK_IFACE && (m == 1 || m == 2)) R.ebk[q] = EBK_NONE;
}

__global__ void k_flags(Grid g, const uint8_t* pre, const int* cut_of_cell, const uint8_t* dofm, uint8_t* flags) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  int q = cut_of_cell[c];
  uint8_t f;
  if (q >= 0) f = dofm[q];
  else f = pre[c] == 1 ? F_GAS : (pre[c] == 2 ? F_DIEL : 0);
  flags[c] = f;
}

// a cell gets a sparse row when it is cut, or when a face neighbour inside
// the domain lacks the unknown of its phase (the implicit stencil would not apply)
__global__ void k_irr_mark(Grid g, const int* cut_of_cell, uint8_t* flags) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  uint8_t f = flags[c];
  if (!(f & 3)) return;
  bool irr = cut_of_cell[c] >= 0;
  if (!irr) {
    int I[3];
    cell_ijk(g, c, I);
    for (int a = 0; a < g.D && !irr; ++a)
      for (int s = -1; s <= 1 && !irr; s += 2) {
        int J[3] = {I[0], I[1], I[2]};
        J[a] += s;
        if (!in_domain(g, J)) continue;
        uint8_t fn = flags[cell_index(g, J[0], J[1], J[2])] & 3;
        if (!(fn & (f & 3))) irr = true;
      }
  }
  if (irr) flags[c] = (uint8_t)(f | F_IRR);
}

__global__ void k_fill_int(int* a, long long n, int v) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

// ----------------------------------------------------------- coarsening

// coarse classification: 0 covered, 1 regular gas, 2 regular dielectric, 3 cut
__global__ void k_coarse_preclass(LevelGeom F, Grid gc, uint8_t* pre) {
  long long C = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (C >= gc.ncell) return;
  pre[C] = coarse_preclass(F, gc, C);
}

__global__ void k_coarse_geom(LevelGeom F, Grid gc, CutRecords Rc, int* status) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Rc.ncut) return;
  int st = coarse_cut_geometry(F, gc, Rc, q);
  if (st) atomicOr(status, st);
}

// ------------------------------------------------------------------ rows

__global__ void k_row_count(LevelGeom L, int* counts, int* status) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= 2 * L.nirr) return;
  long long cell = L.irr_cell[r >> 1];
  int p = (int)(r & 1);
  counts[r] = 0;
  if (!((L.flags[cell] >> p) & 1)) return;
  Form<MAXE> R;
  int orders[2];
  int st = build_row_form(L, cell, p, R, orders);
  if (st) {
    atomicOr(status, st);
    return;
  }
  int self = col_encode(p, cell), n = 0;
  for (int k = 0; k < R.n; ++k)
    if (R.col[k] != self) ++n;
  counts[r] = n;
}

__global__ void k_row_fill(LevelGeom L, const int* row_ptr, int* col, double* val, double* diag, double* bconst,
                           double* bsig, uint8_t* order) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= 2 * L.nirr) return;
  long long cell = L.irr_cell[r >> 1];
  int p = (int)(r & 1);
  diag[r] = 0.0;
  bconst[r] = 0.0;
  bsig[r] = 0.0;
  if (!((L.flags[cell] >> p) & 1)) return;
  Form<MAXE> R;
  int orders[2];
  if (build_row_form(L, cell, p, R, orders)) return;
  int self = col_encode(p, cell);
  int e = row_ptr[r];
  for (int k = 0; k < R.n; ++k) {
    if (R.col[k] == self) {
      diag[r] = -R.w[k];
    } else {
      col[e] = R.col[k];
      val[e] = -R.w[k];
      ++e;
    }
  }
  bconst[r] = R.c;
  bsig[r] = R.sig;
  long long q = L.cut_of_cell[cell];
  if (q >= 0) order[p * L.R.ncut + q] = (uint8_t)orders[p];
}

// ------------------------------------------------------- rhs, field, export

__device__ __forceinline__ void rhs_cell(const LevelGeom& L, long long c, const double* s, const double* sigma,
                                         const double* bconst, const double* bsig, double* b, double& mx) {
  const Grid& g = L.g;
  uint8_t f = L.flags[c];
  for (int p = 0; p < 2; ++p) {
    double v = 0.0;
    if ((f >> p) & 1) {
      if (f & F_IRR) {
        long long k = L.irr_of_cell[c];
        long long r = 2 * k + p;
        int q = L.cut_of_cell[c];
        double kap = q >= 0 ? L.R.kappa[p * L.R.ncut + q] : 1.0;
        v = kap * s[p * g.ncell + c] + bconst[r];
        if (sigma) v = v + bsig[r] * sigma[c];
      } else {
        v = s[p * g.ncell + c];
        int I[3];
        cell_ijk(g, c, I);
        double e = g.eps[p], h2 = g.h * g.h;
        // wall data: Dirichlet 8 eps phi0 / (3 h^2); Robin the same with a3
        // divided by a1 + 8 a2 / (3h) (the wall value eliminated)
        for (int a = 0; a < g.D; ++a)
          for (int hi = 0; hi < 2; ++hi) {
            const int sd = 2 * a + hi;
            if (I[a] != (hi ? g.n[a] - 1 : 0) || !g.bc[sd]) continue;
            double d = 8.0 * e * g.bcv[sd] / (3.0 * h2);
            if (g.bc[sd] == 2) d = d / (g.rob[sd][0] + g.rob[sd][1] * 8.0 / (3.0 * g.h));
            v = v + d;
          }
      }
    }
    b[p * g.ncell + c] = v;
    mx = fmax(mx, fabs(v));
  }
}

// b = kappa s + boundary data + sigma terms, and max|b| (one atomic per warp)
__global__ void k_rhs64(LevelGeom L, const double* s, const double* sigma, const double* bconst, const double* bsig,
                        double* b, unsigned long long* bnorm) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double mx = 0.0;
  if (c < L.g.ncell) rhs_cell(L, c, s, sigma, bconst, bsig, b, mx);
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(bnorm, (unsigned long long)__double_as_longlong(mx));
}

__device__ double eval_dn(const LevelGeom& L, long long q, const int I[3], int p, const double* phi,
                          const double* sigma, long long cell) {
  Form<MAXE> R;
  R.zero();
  int orders[2];
  if (add_eb_dphidn(L, q, I, p, L.R.phiE[q], 1.0, R, orders)) return 0.0;
  double v = R.c;
  for (int k = 0; k < R.n; ++k) v += R.w[k] * phi[(long long)col_phase(R.col[k]) * L.g.ncell + col_cell(R.col[k])];
  if (sigma) v += R.sig * sigma[cell];
  return v;
}

__global__ void k_field_cells(LevelGeom L, const double* phi, const double* sigma, double* E) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const Grid& g = L.g;
  if (c >= g.ncell) return;
  uint8_t f = L.flags[c];
  int I[3];
  cell_ijk(g, c, I);
  for (int p = 0; p < 2; ++p) {
    bool has = (f >> p) & 1;
    double nin[3] = {0.0, 0.0, 0.0}, dn = 0.0;
    bool dn_done = false;
    long long q = L.cut_of_cell[c];
    for (int a = 0; a < g.D; ++a) {
      double v = 0.0;
      if (has) {
        int Jl[3] = {I[0], I[1], I[2]}, Jh[3] = {I[0], I[1], I[2]};
        Jh[a] += 1;
        FaceInfo fl, fh;
        bool lo = I[a] > 0 && face_open(L, a, Jl, p, fl);
        bool hi = I[a] < g.n[a] - 1 && face_open(L, a, Jh, p, fh);
        const double* ph = phi + (long long)p * g.ncell;
        long long sa = (a == 0) ? 1 : (a == 1 ? g.n[0] : (long long)g.n[0] * g.n[1]);
        if (lo && hi) v = -(ph[c + sa] - ph[c - sa]) / (2.0 * g.h);
        else if (hi) v = -(ph[c + sa] - ph[c]) / g.h;
        else if (lo) v = -(ph[c] - ph[c - sa]) / g.h;
        else if (q >= 0 && L.R.ebk[q] != EBK_NONE) {
          if (!dn_done) {
            double xB[3];
            record_nin(L, q, p, xB, nin);
            dn = eval_dn(L, q, I, p, phi, sigma, c);
            dn_done = true;
          }
          v = -dn * nin[a];
        }
      }
      E[((long long)a * 2 + p) * g.ncell + c] = v;
    }
  }
}

__global__ void k_field_eb(LevelGeom L, const int* eb_q, long long n_eb, const double* phi, const double* sigma,
                           double* En) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_eb) return;
  long long q = eb_q[i];
  long long cell = L.R.cell[q];
  int I[3];
  cell_ijk(L.g, cell, I);
  uint8_t f = L.flags[cell];
  for (int p = 0; p < 2; ++p) {
    double v = 0.0;
    if (((f >> p) & 1) && L.R.ebk[q] != EBK_NONE) v = -eval_dn(L, q, I, p, phi, sigma, cell);
    En[2 * i + p] = v;
  }
}

__global__ void k_export_kappa(LevelGeom L, double* kappa) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const Grid& g = L.g;
  if (c >= g.ncell) return;
  int q = L.cut_of_cell[c];
  for (int p = 0; p < 2; ++p) {
    double v;
    if (q >= 0) v = L.R.kappa[p * L.R.ncut + q];
    else v = ((L.flags[c] >> p) & 1) ? 1.0 : 0.0;
    kappa[p * g.ncell + c] = v;
  }
}

__global__ void k_export_eb(LevelGeom L, const int* eb_q, long long n_eb, const uint8_t* order, int32_t* cell,
                            double* area, double* normal, double* centroid, uint8_t* kind, int32_t* ord) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_eb) return;
  long long q = eb_q[i], nq = L.R.ncut;
  if (cell) cell[i] = L.R.cell[q];
  if (area) area[i] = L.R.eba[q];
  for (int d = 0; d < 3; ++d) {
    if (normal) normal[3 * i + d] = L.R.ebn[d * nq + q];
    if (centroid) centroid[3 * i + d] = L.R.ebx[d * nq + q];
  }
  if (kind) kind[i] = L.R.ebk[q];
  if (ord)
    for (int p = 0; p < 2; ++p) ord[2 * i + p] = ((L.flags[L.R.cell[q]] >> p) & 1) ? order[p * nq + q] : 0;
}

// ------------------------------------------------- composite CF faces

__device__ void cf_side_of(const CFBox& B, const long long* off, long long t, int& side, long long& local) {
  side = 0;
  while (side + 1 < B.nside && t >= off[side + 1]) ++side;
  local = t - off[side];
}

__device__ void cf_tangential(int D, int a, int t[2]) {
  int k = 0;
  for (int d = 0; d < D; ++d)
    if (d != a) t[k++] = d;
  if (D == 2) t[1] = 2;
}

// a coarse cell the tangential interpolation may use (gas unknown, not cut,
// inside the domain and outside the box)
__device__ bool cf_coarse_ok(const LevelGeom& Lc, const CFBox& B, const int I[3]) {
  const Grid& g = Lc.g;
  bool under = true;
  for (int k = 0; k < g.D; ++k) {
    if (I[k] < 0 || I[k] >= g.n[k]) return false;
    if (I[k] < B.lo[k] || I[k] >= B.hi[k]) under = false;
  }
  if (under) return false;
  long long c = cell_index(g, I[0], I[1], I[2]);
  return (Lc.flags[c] & 1) && Lc.cut_of_cell[c] < 0;
}

__device__ bool cf_fine_ok(const LevelGeom& Lf, const int I[3]) {
  const Grid& g = Lf.g;
  for (int k = 0; k < g.D; ++k)
    if (I[k] < 0 || I[k] >= g.n[k]) return false;
  long long c = cell_index(g, I[0], I[1], I[2]);
  return (Lf.flags[c] & 1) && Lf.cut_of_cell[c] < 0;
}

__global__ void k_cf_fine(LevelGeom Lf, LevelGeom Lc, CFBox B, CFFace* faces, int* status) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B.off[B.nside]) return;
  int side;
  long long loc;
  cf_side_of(B, B.off, t, side, loc);
  const int D = Lf.g.D, a = B.side_a[side], s = B.side_s[side];
  int tg[2];
  cf_tangential(D, a, tg);
  int FI[3] = {0, 0, 0};
  FI[a] = s ? Lf.g.n[a] - 1 : 0;
  FI[tg[0]] = (int)(loc % Lf.g.n[tg[0]]);
  if (D == 3) FI[tg[1]] = (int)(loc / Lf.g.n[tg[0]]);
  int CI[3] = {0, 0, 0};
  for (int k = 0; k < D; ++k) CI[k] = B.lo[k] + FI[k] / 2;
  CI[a] += s ? 1 : -1;
  CFFace f;
  f.fcell = (int)cell_index(Lf.g, FI[0], FI[1], FI[2]);
  f.ccell = (int)cell_index(Lc.g, CI[0], CI[1], CI[2]);
  f.f2 = -1;
  f.nc = 0;
  f.wf = f.wf2 = f.wc = f.al = 0.0;
  const uint8_t ff = Lf.flags[f.fcell], fcf = Lc.flags[f.ccell];
  if ((ff & 2) || (fcf & 2)) atomicExch(status, 1);  // a dielectric unknown at a CF side
  FaceInfo fi;
  int J[3] = {FI[0], FI[1], FI[2]};
  J[a] += s;
  if ((ff & 1) && (fcf & 1) && face_open(Lf, a, J, 0, fi)) {
    f.al = fi.al;
    // tangential value: phi_C plus one 1-D correction per tangential axis
    f.nc = 1;
    f.cc[0] = f.ccell;
    f.cw[0] = 1.0;
    for (int q = 0; q < D - 1; ++q) {
      const int k = tg[q];
      const double o = (FI[k] % 2 == 0) ? -0.25 : 0.25;
      int lo_I[3] = {CI[0], CI[1], CI[2]}, hi_I[3] = {CI[0], CI[1], CI[2]};
      lo_I[k] -= 1;
      hi_I[k] += 1;
      if (cf_coarse_ok(Lc, B, lo_I) && cf_coarse_ok(Lc, B, hi_I)) {
        f.cc[f.nc] = (int)cell_index(Lc.g, lo_I[0], lo_I[1], lo_I[2]);
        f.cw[f.nc++] = o * (o - 1.0) / 2.0;
        f.cw[0] = f.cw[0] + ((1.0 - o * o) - 1.0);
        f.cc[f.nc] = (int)cell_index(Lc.g, hi_I[0], hi_I[1], hi_I[2]);
        f.cw[f.nc++] = o * (o + 1.0) / 2.0;
      } else {
        const int* sd = o > 0.0 ? hi_I : lo_I;
        if (cf_coarse_ok(Lc, B, sd)) {
          f.cw[0] = f.cw[0] + (-0.25);
          f.cc[f.nc] = (int)cell_index(Lc.g, sd[0], sd[1], sd[2]);
          f.cw[f.nc++] = 0.25;
        }
      }
    }
    int F2[3] = {FI[0], FI[1], FI[2]};
    F2[a] += s ? -1 : 1;
    if (cf_fine_ok(Lf, F2)) {
      f.f2 = (int)cell_index(Lf.g, F2[0], F2[1], F2[2]);
      f.wf = 2.0 / 3.0;
      f.wf2 = -1.0 / 5.0;
      f.wc = 8.0 / 15.0;
    } else {
      f.wf = 1.0 / 3.0;
      f.wc = 2.0 / 3.0;
    }
  }
  faces[t] = f;
}

__global__ void k_cf_coarse2(LevelGeom Lc, CFBox B, int nf0, int nf1, int nf2, CFCoarse* out, int* status) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B.coff[B.nside]) return;
  int side;
  long long loc;
  cf_side_of(B, B.coff, t, side, loc);
  const int D = Lc.g.D, a = B.side_a[side], s = B.side_s[side];
  const int nf[3] = {nf0, nf1, nf2};
  int tg[2];
  cf_tangential(D, a, tg);
  const int w0 = B.hi[tg[0]] - B.lo[tg[0]];
  const int U = (int)(loc % w0), V = D == 3 ? (int)(loc / w0) : 0;
  int CI[3] = {0, 0, 0};
  CI[a] = s ? B.hi[a] : B.lo[a] - 1;
  CI[tg[0]] = B.lo[tg[0]] + U;
  if (D == 3) CI[tg[1]] = B.lo[tg[1]] + V;
  CFCoarse c;
  c.ccell = -1;
  c.nfine = 0;
  c.n = 0;
  const long long cc = cell_index(Lc.g, CI[0], CI[1], CI[2]);
  for (int j = 0; j < (D == 3 ? 2 : 1); ++j)
    for (int i = 0; i < 2; ++i) {
      long long u = 2 * U + i, v = 2 * V + j;
      c.fine[c.nfine++] = (int)(B.off[side] + u + (D == 3 ? (long long)nf[tg[0]] * v : 0));
    }
  if (Lc.flags[cc] & 1) {
    c.ccell = (int)cc;
    int JC[3] = {CI[0], CI[1], CI[2]};
    if (s == 0) JC[a] += 1;  // the cell below the box: its high face
    FaceInfo fi;
    if (face_open(Lc, a, JC, 0, fi)) {
      Form<24> R;
      R.zero();
      add_centroid_flux(Lc, a, JC, 0, (s == 0 ? 1.0 : -1.0) * fi.al / Lc.g.h, R);
      if (R.overflow) atomicExch(status, 2);
      c.n = R.n;
      for (int k = 0; k < R.n; ++k) {
        c.col[k] = R.col[k];
        c.w[k] = R.w[k];
      }
    }
  }
  out[t] = c;
}

// ------------------------------------------------------------------ host

static LevelGeom view(const DevLevel& L) {
  LevelGeom v;
  v.g = L.g;
  v.coarse = L.coarse;
  v.flags = L.flags;
  v.cut_of_cell = L.cut_of_cell;
  v.R = L.R;
  v.nirr = L.nirr;
  v.nirr_red = L.nirr_red;
  v.irr_cell = L.irr_cell;
  v.irr_of_cell = L.irr_of_cell;
  return v;
}

static eb_status check(cudaStream_t s, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, what);
  return EB_OK;
}

static eb_status read_status(eb_geom* G, cudaStream_t s, int* out) {
  cudaError_t e = cudaMemcpyAsync(out, G->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  return EB_OK;
}

static eb_status alloc_records(DevLevel& L, long long ncut, long long* bytes) {
  eb_status st = EB_OK;
  long long n = std::max<long long>(ncut, 1);
  int D = L.g.D, nf = 2 * D;
  CutRecords& R = L.R;
  R.ncut = ncut;
  R.kappa = (double*)dev_alloc(L.allocs, sizeof(double) * 2 * n, bytes, &st);
  R.alpha = (double*)dev_alloc(L.allocs, sizeof(double) * nf * 2 * n, bytes, &st);
  R.fcen = (double*)dev_alloc(L.allocs, sizeof(double) * nf * 4 * n, bytes, &st);
  R.ebk = (uint8_t*)dev_alloc(L.allocs, n, bytes, &st);
  R.eba = (double*)dev_alloc(L.allocs, sizeof(double) * n, bytes, &st);
  R.ebn = (double*)dev_alloc(L.allocs, sizeof(double) * 3 * n, bytes, &st);
  R.ebx = (double*)dev_alloc(L.allocs, sizeof(double) * 3 * n, bytes, &st);
  R.phiE = (double*)dev_alloc(L.allocs, sizeof(double) * n, bytes, &st);
  R.dofm = (uint8_t*)dev_alloc(L.allocs, n, bytes, &st);
  L.order = (uint8_t*)dev_alloc(L.allocs, 2 * n, bytes, &st);
  if (st == EB_OK) {
    cudaMemset(L.order, 0, 2 * n);
    cudaMemset(R.alpha, 0, sizeof(double) * nf * 2 * n);
    cudaMemset(R.fcen, 0, sizeof(double) * nf * 4 * n);
  }
  return st;
}

// flags, irregular marking and the colour-sorted irregular list of a level
// whose cut records and dof masks are in place; pre = preclass array.
static eb_status finish_level(eb_geom* G, DevLevel& L, const uint8_t* pre, cudaStream_t s) {
  long long n = L.g.ncell;
  k_flags<<<nblk(n), TB, 0, s>>>(L.g, pre, L.cut_of_cell, L.R.dofm, L.flags);
  k_irr_mark<<<nblk(n), TB, 0, s>>>(L.g, L.cut_of_cell, L.flags);
  eb_status st = check(s, "flags");
  if (st != EB_OK) return st;
  int *red = nullptr, *black = nullptr;
  long long nr = 0, nbk = 0;
  std::vector<void*> tmp;
  st = compact(PredIrrColour{L.g, L.flags, 0}, n, &red, &nr, tmp, nullptr, s);
  if (st == EB_OK) st = compact(PredIrrColour{L.g, L.flags, 1}, n, &black, &nbk, tmp, nullptr, s);
  if (st == EB_OK) {
    L.nirr = nr + nbk;
    L.nirr_red = nr;
    L.irr_cell = (int*)dev_alloc(L.allocs, sizeof(int) * std::max<long long>(L.nirr, 1), &G->bytes, &st);
  }
  if (st == EB_OK) {
    if (nr) cudaMemcpyAsync(L.irr_cell, red, sizeof(int) * nr, cudaMemcpyDeviceToDevice, s);
    if (nbk) cudaMemcpyAsync(L.irr_cell + nr, black, sizeof(int) * nbk, cudaMemcpyDeviceToDevice, s);
    k_fill_int<<<nblk(n), TB, 0, s>>>(L.irr_of_cell, n, -1);
    k_map<<<nblk(L.nirr), TB, 0, s>>>(L.irr_cell, L.nirr, L.irr_of_cell);
    st = check(s, "irregular list");
  }
  for (void* p : tmp) cudaFree(p);
  return st;
}

static eb_status alloc_level_dense(eb_geom* G, DevLevel& L) {
  eb_status st = EB_OK;
  long long n = L.g.ncell;
  L.flags = (uint8_t*)dev_alloc(L.allocs, n, &G->bytes, &st);
  L.cut_of_cell = (int*)dev_alloc(L.allocs, sizeof(int) * n, &G->bytes, &st);
  L.irr_of_cell = (int*)dev_alloc(L.allocs, sizeof(int) * n, &G->bytes, &st);
  return st;
}

eb_status build_finest_geometry(eb_geom* G, cudaStream_t s) {
  DevLevel& L = G->L[0];
  const Grid& g = L.g;
  eb_status st = alloc_level_dense(G, L);
  if (st != EB_OK) return st;
  long long nn = node_count(g);
  std::vector<void*> tmp;
  G->d_lab = (uint8_t*)dev_alloc(L.allocs, nn, &G->bytes, &st);
  uint8_t* pre = (uint8_t*)dev_alloc(tmp, g.ncell, nullptr, &st);
  if (st != EB_OK) {
    for (void* p : tmp) cudaFree(p);
    return st;
  }
  cudaMemsetAsync(G->d_status, 0, sizeof(int), s);
  k_labels<<<nblk(nn), TB, 0, s>>>(G->d_csg, g, G->d_lab);
  k_preclass<<<nblk(g.ncell), TB, 0, s>>>(g, G->d_lab, pre);
  st = check(s, "labels");
  long long ncut = 0;
  int* cut = nullptr;
  if (st == EB_OK) st = compact(PredEq{pre, 3}, g.ncell, &cut, &ncut, L.allocs, &G->bytes, s);
  if (st == EB_OK) st = alloc_records(L, ncut, &G->bytes);
  if (st == EB_OK) {
    L.R.cell = cut;
    k_fill_int<<<nblk(g.ncell), TB, 0, s>>>(L.cut_of_cell, g.ncell, -1);
    k_map<<<nblk(ncut), TB, 0, s>>>(cut, ncut, L.cut_of_cell);
    k_cut_geom<<<nblk(ncut, 64), 64, 0, s>>>(G->d_csg, g, G->d_lab, L.R, G->d_status);
    k_dofs<<<nblk(ncut), TB, 0, s>>>(g, L.R);
    st = check(s, "cut-cell geometry");
  }
  int status = 0;
  if (st == EB_OK) st = read_status(G, s, &status);
  if (st == EB_OK && status) {
    set_error("geometry outside the method's model: a cell cut by an electrode and the dielectric, a face with "
              "four crossings, or an interface cell that keeps only one fragment");
    st = EB_ERR_UNSUPPORTED;
  }
  if (st == EB_OK) st = finish_level(G, L, pre, s);
  // EB list: cut cells with at least one unknown, ascending
  if (st == EB_OK) st = compact(PredNonzero{L.R.dofm}, ncut, &L.eb_q, &L.n_eb, L.allocs, &G->bytes, s);
  for (void* p : tmp) cudaFree(p);
  return st;
}

eb_status build_coarse_geometry(eb_geom* G, int fine, cudaStream_t s, bool* stopped) {
  *stopped = false;
  DevLevel& F = G->L[fine];
  DevLevel C;
  C.g = F.g;
  C.coarse = 1;
  for (int k = 0; k < F.g.D; ++k) C.g.n[k] = F.g.n[k] / 2;
  C.g.h = F.g.h * 2.0;
  C.g.ncell = (long long)C.g.n[0] * C.g.n[1] * (C.g.D == 3 ? C.g.n[2] : 1);
  for (int k = 0; k < 6; ++k) C.g.bcv[k] = 0.0;
  eb_status st = alloc_level_dense(G, C);
  std::vector<void*> tmp;
  uint8_t* pre = (uint8_t*)dev_alloc(tmp, C.g.ncell, nullptr, &st);
  long long ncut = 0;
  int* cut = nullptr;
  LevelGeom fv = view(F);
  if (st == EB_OK) {
    cudaMemsetAsync(G->d_status, 0, sizeof(int), s);
    k_coarse_preclass<<<nblk(C.g.ncell), TB, 0, s>>>(fv, C.g, pre);
    st = check(s, "coarse classification");
  }
  if (st == EB_OK) st = compact(PredEq{pre, 3}, C.g.ncell, &cut, &ncut, C.allocs, &G->bytes, s);
  if (st == EB_OK) st = alloc_records(C, ncut, &G->bytes);
  if (st == EB_OK) {
    C.R.cell = cut;
    k_fill_int<<<nblk(C.g.ncell), TB, 0, s>>>(C.cut_of_cell, C.g.ncell, -1);
    k_map<<<nblk(ncut), TB, 0, s>>>(cut, ncut, C.cut_of_cell);
    k_coarse_geom<<<nblk(ncut, 64), 64, 0, s>>>(fv, C.g, C.R, G->d_status);
    k_dofs<<<nblk(ncut), TB, 0, s>>>(C.g, C.R);
    st = check(s, "coarse geometry");
  }
  int status = 0;
  if (st == EB_OK) st = read_status(G, s, &status);
  if (st == EB_OK && status) {
    *stopped = true;
    for (void* p : tmp) cudaFree(p);
    free_level(C);
    return EB_OK;
  }
  if (st == EB_OK) st = finish_level(G, C, pre, s);
  for (void* p : tmp) cudaFree(p);
  if (st != EB_OK) {
    free_level(C);
    return st;
  }
  G->L.push_back(C);
  return EB_OK;
}

eb_status build_rows(eb_geom* G, int level, cudaStream_t s) {
  DevLevel& L = G->L[level];
  long long nrow = 2 * L.nirr;
  eb_status st = EB_OK;
  std::vector<void*> tmp;
  int* counts = (int*)dev_alloc(tmp, sizeof(int) * std::max<long long>(nrow, 1), nullptr, &st);
  L.row_ptr = (int*)dev_alloc(L.allocs, sizeof(int) * (nrow + 1), &G->bytes, &st);
  L.diag = (double*)dev_alloc(L.allocs, sizeof(double) * std::max<long long>(nrow, 1), &G->bytes, &st);
  L.bconst = (double*)dev_alloc(L.allocs, sizeof(double) * std::max<long long>(nrow, 1), &G->bytes, &st);
  L.bsig = (double*)dev_alloc(L.allocs, sizeof(double) * std::max<long long>(nrow, 1), &G->bytes, &st);
  if (st != EB_OK) {
    for (void* p : tmp) cudaFree(p);
    return st;
  }
  LevelGeom v = view(L);
  cudaMemsetAsync(G->d_status, 0, sizeof(int), s);
  k_row_count<<<nblk(nrow, 64), 64, 0, s>>>(v, counts, G->d_status);
  st = check(s, "row count");
  int status = 0;
  if (st == EB_OK) st = read_status(G, s, &status);
  if (st == EB_OK && status) {
    set_error(level == 0 ? "no EB normal-derivative stencil could be built for a cut cell (too few fluid cells "
                           "nearby) or a stencil overflowed"
                         : "coarse stencil failure");
    st = EB_ERR_UNSUPPORTED;
  }
  long long nnz = 0;
  if (st == EB_OK) st = exclusive_scan(counts, nrow, L.row_ptr, &nnz, s);
  if (st == EB_OK) {
    L.nnz = nnz;
    L.col = (int*)dev_alloc(L.allocs, sizeof(int) * std::max<long long>(nnz, 1), &G->bytes, &st);
    L.val = (double*)dev_alloc(L.allocs, sizeof(double) * std::max<long long>(nnz, 1), &G->bytes, &st);
  }
  if (st == EB_OK) {
    k_row_fill<<<nblk(nrow, 64), 64, 0, s>>>(v, L.row_ptr, L.col, L.val, L.diag, L.bconst, L.bsig, L.order);
    st = check(s, "row fill");
  }
  for (void* p : tmp) cudaFree(p);
  return st;
}

void free_level(DevLevel& L) {
  for (void* p : L.allocs) cudaFree(p);
  L.allocs.clear();
}

eb_status launch_rhs64(const eb_geom* G, const double* s_rhs, const double* sigma, double* b, double* bnorm,
                       cudaStream_t s) {
  const DevLevel& L = G->L[0];
  k_rhs64<<<nblk(L.g.ncell), TB, 0, s>>>(view(L), s_rhs, sigma, L.bconst, L.bsig, b, (unsigned long long*)bnorm);
  note_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? EB_OK : cuda_fail(e, "rhs");
}

eb_status launch_field(const eb_geom* G, const double* phi, const double* sigma, double* E, double* En,
                       cudaStream_t s) {
  const DevLevel& L = G->L[0];
  LevelGeom v = view(L);
  if (E) k_field_cells<<<nblk(L.g.ncell, 128), 128, 0, s>>>(v, phi, sigma, E);
  if (En && L.n_eb) k_field_eb<<<nblk(L.n_eb, 64), 64, 0, s>>>(v, L.eb_q, L.n_eb, phi, sigma, En);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? EB_OK : cuda_fail(e, "field");
}

eb_status build_cf(const eb_geom* Gf, const eb_geom* Gc, const CFBox& B, CFFace* faces, CFCoarse* cfaces,
                   int* d_status, cudaStream_t s) {
  const DevLevel& F = Gf->L[0];
  const DevLevel& C = Gc->L[0];
  cudaMemsetAsync(d_status, 0, sizeof(int), s);
  if (B.off[B.nside] > 0)
    k_cf_fine<<<nblk(B.off[B.nside]), TB, 0, s>>>(view(F), view(C), B, faces, d_status);
  if (B.coff[B.nside] > 0)
    k_cf_coarse2<<<nblk(B.coff[B.nside], 64), 64, 0, s>>>(view(C), B, F.g.n[0], F.g.n[1], F.g.n[2], cfaces,
                                                          d_status);
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "coarse-fine faces");
  if (h == 1) {
    set_error("a dielectric unknown touches a coarse-fine side of the refined box");
    return EB_ERR_UNSUPPORTED;
  }
  if (h == 2) {
    set_error("coarse face flux stencil too long");
    return EB_ERR_UNSUPPORTED;
  }
  return check(s, "coarse-fine faces");
}

// kappa [2][ncell] of the finest level (volume fraction per phase, 0 where
// the phase has no unknown), enqueued on s
eb_status launch_kappa(const eb_geom* G, double* kappa, cudaStream_t s) {
  const DevLevel& L = G->L[0];
  k_export_kappa<<<nblk(L.g.ncell), TB, 0, s>>>(view(L), kappa);
  return check(s, "kappa");
}

eb_status export_geometry(const eb_geom* G, eb_geom_arrays* out, cudaStream_t s) {
  const DevLevel& L = G->L[0];
  LevelGeom v = view(L);
  if (out->flags) cudaMemcpyAsync(out->flags, L.flags, L.g.ncell, cudaMemcpyDeviceToDevice, s);
  if (out->kappa) k_export_kappa<<<nblk(L.g.ncell), TB, 0, s>>>(v, out->kappa);
  if (L.n_eb)
    k_export_eb<<<nblk(L.n_eb), TB, 0, s>>>(v, L.eb_q, L.n_eb, L.order, out->eb_cell, out->eb_area, out->eb_normal,
                                            out->eb_centroid, out->eb_kind, out->stencil_order);
  return check(s, "export");
}

}  // namespace ebp

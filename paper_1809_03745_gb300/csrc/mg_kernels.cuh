// mg_kernels.cuh -- multigrid kernels (arXiv:1809.03745, Sec. 3.3.2):
// red-black Gauss-Seidel, residual fused with conservative restriction,
// prolongation with correction, the single-CTA bottom relaxation, and the FP64
// defect-correction kernels.  Templated on the V-cycle precision T; sparse
// rows of cut cells always carry FP64 coefficients.
#pragma once

#include <cuda_runtime.h>

#include "eb_common.cuh"

namespace ebp {

// Division of 32-bit unsigned values by a fixed divisor with a multiply-high
// and a shift (Granlund-Montgomery round-up method); exact for every 32-bit x.
struct FastDiv {
  unsigned d, m, s;
};
inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f;
  f.d = d;
  unsigned s = 0;
  while ((1ull << s) < d) ++s;
  f.s = s;
  f.m = (unsigned)((((1ull << s) - d) << 32) / d + 1);
  return f;
}
__device__ __forceinline__ unsigned fdiv(unsigned x, const FastDiv& f) {
  return (unsigned)(((unsigned long long)__umulhi(x, f.m) + x) >> f.s);
}

template <class T>
struct Op {
  FastDiv dn0, dn1, dhx;  // n[0], n[1] and the cells of one colour per x row, (n[0] + 1) / 2
  FastDiv dq;             // groups of four cells per x row, n[0] / 4 (used when n[0] % 4 == 0)
  int D;
  int n[3];
  long long ncell;
  // wall weight per side (xlo, xhi, ylo, yhi, zlo, zhi): 1 on a Dirichlet
  // wall, 0 on a Neumann wall, a1 / (a1 + 8 a2 / (3h)) on a Robin wall
  T wr[6];
  T w3[6];   // wr / 3: the weight of the inward neighbour of a wall cell
  T lh[2];   // the Helmholtz shift per phase in the stencil's units: lam_p h^2 / eps_p
  T idg[2];  // 1 / (2D + lh[p]): the reciprocal diagonal of a cell away from the walls
  int intdg;  // 1: every wall weight is 0 or 1 and no shift, so every diagonal is a small integer
  T* x[2];  // unknown per phase
  T* b[2];  // right-hand side per phase
  const uint8_t* flags;
  const int* irr_cell;
  const int* irr_of_cell;
  const int* row_ptr;
  const int* col;
  const double* val;
  const double* diag;
  T* tmp;  // [2 nirr] row scratch
  long long nirr, nirr_red;
  T ceps[2];  // eps_p / h^2
  T h2e[2];   // h^2 / eps_p
};

// Implicit stencil of a regular cell: A x = (eps/h^2)((dg + lh) x_c - sum).
// Every open face adds 1 to dg and its neighbour to sum.  A wall face with
// weight w adds 3w to dg and w x_inward / 3 to sum.  This is the one-sided
// second-order wall flux: w = 1 for Dirichlet; for Robin the wall value is
// eliminated through the same formula.  A Neumann wall face (w = 0) adds
// nothing.
// The diagonal is counted as an integer (open faces, and 3 per Dirichlet
// wall face when every weight is 0 or 1) and only fractional wall weights are
// accumulated in T: on the FP64 path every extra operation per cell runs on
// GB300's narrow FP64 pipe.
template <class T>
__device__ __forceinline__ void wall_term(const Op<T>& o, int side, T xin, T& sum, int& nf, T& wd) {
  sum += xin * o.w3[side];
  if (o.intdg) nf += 3;
  else wd += T(3) * o.wr[side];
}

template <class T>
__device__ __forceinline__ void reg_stencil(const Op<T>& o, const T* x, const int I[3], long long c, T& sum, T& dg) {
  sum = T(0);
  int nf = 0;
  T wd = T(0);
  long long st = 1;
  for (int a = 0; a < o.D; ++a) {
    if (I[a] > 0) {
      sum += x[c - st];
      ++nf;
    } else if (o.wr[2 * a] != T(0)) {
      wall_term(o, 2 * a, x[c + st], sum, nf, wd);
    }
    if (I[a] < o.n[a] - 1) {
      sum += x[c + st];
      ++nf;
    } else if (o.wr[2 * a + 1] != T(0)) {
      wall_term(o, 2 * a + 1, x[c - st], sum, nf, wd);
    }
    st *= o.n[a];
  }
  dg = T(nf) + wd;
}

// Correctly rounded reciprocals (the same value as 1 / x, without a general
// division's code inlined at every call site).
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

// 1 / (dg + lh[p]), the reciprocal diagonal of a regular cell of phase p
// whose stencil gave dg: the stored value for a cell away from the walls.
// Reciprocals of the possible integer diagonals (faces + 3 per Dirichlet
// wall face), as constants.
__device__ __forceinline__ float inv_count(int d, float) { return 1.0f / (float)d; }
__device__ __forceinline__ double inv_count(int d, double) {
  switch (d) {
    case 1: return 1.0;
    case 2: return 0.5;
    case 3: return 1.0 / 3.0;
    case 4: return 0.25;
    case 5: return 0.2;
    case 6: return 1.0 / 6.0;
    case 7: return 1.0 / 7.0;
    case 8: return 0.125;
    case 9: return 1.0 / 9.0;
    case 10: return 0.1;
    case 11: return 1.0 / 11.0;
    case 12: return 1.0 / 12.0;
    default: return 1.0 / (double)d;
  }
}

template <class T>
__device__ __forceinline__ T diag_inv(const Op<T>& o, int p, T dg) {
  if (dg == T(2 * o.D)) return o.idg[p];
  if (o.intdg) return inv_count((int)dg, T(0));
  return rcp_rn(dg + o.lh[p]);
}

template <class T>
__device__ __forceinline__ void ijk(const Op<T>& o, long long c, int I[3]) {
  unsigned cu = (unsigned)c;
  unsigned r = fdiv(cu, o.dn0);
  unsigned k = fdiv(r, o.dn1);
  I[0] = (int)(cu - r * (unsigned)o.n[0]);
  I[1] = (int)(r - k * (unsigned)o.n[1]);
  I[2] = (int)k;
}

// one colour of red-black Gauss-Seidel on regular cells; thread per cell pair along x
template <class T>
__global__ void k_smooth_dense(Op<T> o, int colour) {
  int hx = (o.n[0] + 1) >> 1;  // cells of one colour per x row (either parity of n0)
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (o.ncell / o.n[0]) * hx) return;
  long long row = t / hx;
  int j = (int)(row % o.n[1]);
  int k = (int)(row / o.n[1]);
  int i = 2 * (int)(t % hx) + ((j + k + colour) & 1);
  if (i >= o.n[0]) return;
  long long c = (long long)i + (long long)o.n[0] * row;
  uint8_t f = o.flags[c];
  if ((f & F_IRR) || !(f & 3)) return;
  int p = (f & 1) ? 0 : 1;
  T* x = o.x[p];
  int I[3] = {i, j, k};
  T sum, dg;
  reg_stencil(o, x, I, c, sum, dg);
  x[c] = (o.h2e[p] * o.b[p][c] + sum) * diag_inv(o, p, dg);
}

// sum over the off-diagonal entries of sparse row r; entries are taken eight
// at a time with every load of a batch issued before the products
template <class T>
__device__ __forceinline__ double row_dot(const Op<T>& o, long long r) {
  double s = 0.0;
  const int e0 = o.row_ptr[r], e1 = o.row_ptr[r + 1];
  for (int e = e0; e < e1; e += 8) {
    unsigned cl[8];
    double v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      cl[k] = 0u;
      v[k] = 0.0;
      if (e + k < e1) {
        cl[k] = (unsigned)o.col[e + k];
        v[k] = o.val[e + k];
      }
    }
    T xv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) xv[k] = (e + k < e1) ? o.x[cl[k] >> 30][cl[k] & 0x3fffffffu] : T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k] * (double)xv[k];
  }
  return s;
}

// The same sum in the arithmetic of T: the FP32 V-cycle's levels inside one
// CTA, where a single SM does every row and FP64 issues at a small fraction
// of the FP32 rate.  The coefficients are rounded to T on load; the result
// is rounded to T in either case.
template <class T>
__device__ __forceinline__ T row_dot_t(const Op<T>& o, long long r) {
  T s = T(0);
  const int e0 = o.row_ptr[r], e1 = o.row_ptr[r + 1];
  for (int e = e0; e < e1; e += 8) {
    unsigned cl[8];
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      cl[k] = 0u;
      v[k] = T(0);
      if (e + k < e1) {
        cl[k] = (unsigned)o.col[e + k];
        v[k] = (T)o.val[e + k];
      }
    }
    T xv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) xv[k] = (e + k < e1) ? o.x[cl[k] >> 30][cl[k] & 0x3fffffffu] : T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k] * xv[k];
  }
  return s;
}

// sparse rows [rb, re): mode 0 writes the Gauss-Seidel value, mode 1 the residual, into tmp
template <class T>
__global__ void k_rows(Op<T> o, long long rb, long long re, int mode) {
  long long r = rb + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= re) return;
  double d = o.diag[r];
  if (d == 0.0) return;
  long long cell = o.irr_cell[r >> 1];
  int p = (int)(r & 1);
  double s = (double)o.b[p][cell] - row_dot(o, r);
  o.tmp[r] = mode == 0 ? (T)(s / d) : (T)(s - d * (double)o.x[p][cell]);
}

template <class T>
__global__ void k_scatter_rows(Op<T> o, long long rb, long long re) {
  long long r = rb + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= re) return;
  if (o.diag[r] == 0.0) return;
  o.x[r & 1][o.irr_cell[r >> 1]] = o.tmp[r];
}

// Gauss-Seidel of rows [rb, re) by one CTA: all new values from the current
// iterate first (rows of one colour may couple through EB stencils), then written.
template <class T>
__global__ void k_rows_gs_cta(Op<T> o, long long rb, long long re) {
  for (long long r = rb + threadIdx.x; r < re; r += blockDim.x) {
    double d = o.diag[r];
    if (d == 0.0) continue;
    long long cell = o.irr_cell[r >> 1];
    int p = (int)(r & 1);
    o.tmp[r] = (T)(((double)o.b[p][cell] - row_dot(o, r)) / d);
  }
  __syncthreads();
  for (long long r = rb + threadIdx.x; r < re; r += blockDim.x) {
    if (o.diag[r] == 0.0) continue;
    o.x[r & 1][o.irr_cell[r >> 1]] = o.tmp[r];
  }
}

template <class T>
__device__ __forceinline__ T cell_residual(const Op<T>& o, long long c, int p, const int I[3]) {
  uint8_t f = o.flags[c];
  if (f & F_IRR) return o.tmp[2 * (long long)o.irr_of_cell[c] + p];
  T sum, dg;
  reg_stencil(o, o.x[p], I, c, sum, dg);
  return o.b[p][c] - o.ceps[p] * ((dg + o.lh[p]) * o.x[p][c] - sum);
}

// r = b - A x on the fine level, averaged over the 2^D children into the
// coarse right-hand side (the integral form makes restriction a sum; per unit
// volume it is the mean); the coarse unknown is zeroed.  Thread per coarse cell.
template <class T>
__global__ void k_resid_restrict(Op<T> f, Op<T> c) {
  long long C = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (C >= c.ncell) return;
  int IC[3];
  ijk(c, C, IC);
  int nch = 1 << f.D;
  T acc[2] = {T(0), T(0)};
  for (int k = 0; k < nch; ++k) {
    int I[3] = {2 * IC[0] + (k & 1), 2 * IC[1] + ((k >> 1) & 1), f.D == 3 ? 2 * IC[2] + ((k >> 2) & 1) : 0};
    long long cf = (long long)I[0] + (long long)f.n[0] * ((long long)I[1] + (long long)f.n[1] * I[2]);
    uint8_t fl = f.flags[cf];
    for (int p = 0; p < 2; ++p)
      if ((fl >> p) & 1) acc[p] += cell_residual(f, cf, p, I);
  }
  uint8_t cf = c.flags[C];
  T scale = T(1) / T(nch);
  for (int p = 0; p < 2; ++p) {
    if (c.b[p] == nullptr) continue;
    c.b[p][C] = ((cf >> p) & 1) ? acc[p] * scale : T(0);
    c.x[p][C] = T(0);
  }
}

// x_fine += P x_coarse: (bi/tri)linear where every coarse cell of the
// interpolation carries an unknown of the phase, piecewise constant otherwise.
template <class T>
__global__ void k_prolong(Op<T> f, Op<T> c) {
  long long cf = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cf >= f.ncell) return;
  uint8_t fl = f.flags[cf];
  if (!(fl & 3)) return;
  int I[3];
  ijk(f, cf, I);
  int IC[3] = {I[0] >> 1, I[1] >> 1, f.D == 3 ? I[2] >> 1 : 0};
  int sdir[3];
  bool inside = true;
  for (int a = 0; a < 3; ++a) {
    sdir[a] = (I[a] & 1) ? 1 : -1;
    if (a < f.D) {
      int nb = IC[a] + sdir[a];
      if (nb < 0 || nb >= c.n[a]) inside = false;
    }
  }
  long long C = (long long)IC[0] + (long long)c.n[0] * ((long long)IC[1] + (long long)c.n[1] * IC[2]);
  long long st[3] = {1, c.n[0], (long long)c.n[0] * c.n[1]};
  int ncn = 1 << f.D;
  for (int p = 0; p < 2; ++p) {
    if (!((fl >> p) & 1)) continue;
    const T* xc = c.x[p];
    T v = xc[C];
    bool lin = inside;
    if (lin)
      for (int k = 1; k < ncn && lin; ++k) {
        long long n = C;
        for (int a = 0; a < f.D; ++a)
          if ((k >> a) & 1) n += sdir[a] * st[a];
        if (!((c.flags[n] >> p) & 1)) lin = false;
      }
    if (lin) {
      // weights 3/4 (own) and 1/4 (neighbour) per axis
      T acc = T(0);
      for (int k = 0; k < ncn; ++k) {
        long long n = C;
        T w = T(1);
        for (int a = 0; a < f.D; ++a) {
          if ((k >> a) & 1) {
            n += sdir[a] * st[a];
            w *= T(0.25);
          } else {
            w *= T(0.75);
          }
        }
        acc += w * xc[n];
      }
      v = acc;
    }
    f.x[p][cf] += v;
  }
}

// Coarsest level: red-black Gauss-Seidel sweeps by one CTA (Sec. 3.3.2: a
// relaxation bottom solver for multiphase problems).
template <class T>
__global__ void k_bottom(Op<T> o, int sweeps) {
  int hx = (o.n[0] + 1) >> 1;
  long long work = (o.ncell / o.n[0]) * hx;
  for (int it = 0; it < sweeps; ++it) {
    for (int colour = 0; colour < 2; ++colour) {
      for (long long t = threadIdx.x; t < work; t += blockDim.x) {
        long long row = t / hx;
        int j = (int)(row % o.n[1]);
        int k = (int)(row / o.n[1]);
        int i = 2 * (int)(t % hx) + ((j + k + colour) & 1);
        if (i >= o.n[0]) continue;
        long long c = (long long)i + (long long)o.n[0] * row;
        uint8_t f = o.flags[c];
        if ((f & F_IRR) || !(f & 3)) continue;
        int p = (f & 1) ? 0 : 1;
        int I[3] = {i, j, k};
        T sum, dg;
        reg_stencil(o, o.x[p], I, c, sum, dg);
        o.x[p][c] = (o.h2e[p] * o.b[p][c] + sum) * diag_inv(o, p, dg);
      }
      __syncthreads();
      long long rb = colour == 0 ? 0 : 2 * o.nirr_red, re = colour == 0 ? 2 * o.nirr_red : 2 * o.nirr;
      for (long long r = rb + threadIdx.x; r < re; r += blockDim.x) {
        double d = o.diag[r];
        if (d == 0.0) continue;
        long long cell = o.irr_cell[r >> 1];
        int p = (int)(r & 1);
        o.tmp[r] = (T)(((double)o.b[p][cell] - row_dot(o, r)) / d);
      }
      __syncthreads();
      for (long long r = rb + threadIdx.x; r < re; r += blockDim.x) {
        if (o.diag[r] == 0.0) continue;
        o.x[r & 1][o.irr_cell[r >> 1]] = o.tmp[r];
      }
      __syncthreads();
    }
  }
}

// FP64 residual of the finest level (irregular rows already in o.tmp) and its
// max norm; with b32/e32 given, the residual becomes the FP32 inner
// right-hand side and the FP32 correction is zeroed.
__global__ void k_resid64_out(Op<double> o, float* b32_0, float* b32_1, float* e32_0, float* e32_1,
                              unsigned long long* norm) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double mx = 0.0;
  if (c < o.ncell) {
    uint8_t f = o.flags[c];
    int I[3];
    ijk(o, c, I);
    float* bo[2] = {b32_0, b32_1};
    float* eo[2] = {e32_0, e32_1};
    for (int p = 0; p < 2; ++p) {
      double r = 0.0;
      if ((f >> p) & 1) r = cell_residual(o, c, p, I);
      mx = fmax(mx, fabs(r));
      if (bo[p]) bo[p][c] = (float)r;
      if (eo[p]) eo[p][c] = 0.0f;
    }
  }
  // warp max then one atomic per warp (max is order independent)
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) atomicMax(norm, (unsigned long long)__double_as_longlong(mx));
}

__global__ void k_update64(Op<double> o, const float* e0, const float* e1) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= o.ncell) return;
  uint8_t f = o.flags[c];
  if (f & 1) o.x[0][c] += (double)e0[c];
  if ((f & 2) && e1) o.x[1][c] += (double)e1[c];
}

// masked copy of a [2][ncell] field: entries without an unknown become 0
// max |v| over the entries that carry an unknown, into *out (bit pattern of a
// non-negative double, so an integer atomicMax orders it)
__global__ void k_absmax_masked(const uint8_t* flags, long long ncell, const double* v, unsigned long long* out) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  if (c < ncell) {
    uint8_t f = flags[c];
    for (int p = 0; p < 2; ++p)
      if ((f >> p) & 1) m = fmax(m, fabs(v[p * ncell + c]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_copy_masked(const uint8_t* flags, long long ncell, const double* src, double* dst) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  uint8_t f = flags[c];
  for (int p = 0; p < 2; ++p) dst[p * ncell + c] = ((f >> p) & 1) ? src[p * ncell + c] : 0.0;
}

}  // namespace ebp

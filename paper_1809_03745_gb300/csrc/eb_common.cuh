// eb_common.cuh -- shared definitions of the GB300 EB Poisson library.
//
// Per-item logic (one node, face, cell or operator row) is written as
// host+device inline functions so that the kernels stay thin wrappers; the
// kernels themselves live in the .cu files.
#pragma once

#include <cmath>
#include <cstdint>

#ifdef __CUDACC__
#define EBP_HD __host__ __device__ __forceinline__
// large setup-time functions stay out of line: inlining them into every
// caller multiplies compile time without helping run time
#define EBP_HDN static __host__ __device__ __noinline__
#else
#define EBP_HD inline
#define EBP_HDN static inline
#endif

namespace ebp {

// node labels
constexpr int LAB_E = 0;  // inside an electrode (solid)
constexpr int LAB_G = 1;  // gas
constexpr int LAB_D = 2;  // dielectric

// cell flags: bit0 gas unknown, bit1 dielectric unknown, bit2 sparse (irregular) row
constexpr uint8_t F_GAS = 1, F_DIEL = 2, F_IRR = 4;

// EB kind of a cut cell
constexpr uint8_t EBK_NONE = 0, EBK_ELEC = 1, EBK_IFACE = 2;

constexpr int MAX_PRIMS = 32, MAX_NODES = 64, MAX_ELEC = 4, NPAR = 10;

// status bits raised by setup kernels
constexpr int ST_UNSUPPORTED = 1;  // geometry outside the model
constexpr int ST_STOP = 2;         // coarsening must stop at this level
constexpr int ST_OVERFLOW = 4;     // a per-row buffer overflowed

// Implicit-function description, copied to device memory once per geometry.
struct Csg {
  int n_prims, n_nodes;
  int kind[MAX_PRIMS];
  double par[MAX_PRIMS][NPAR];
  int op[MAX_NODES], a[MAX_NODES], b[MAX_NODES];
  int root_E, root_D;
  int n_elec;
  int elec_node[MAX_ELEC];
  double elec_phi[MAX_ELEC];
};

// Grid of one multigrid level.
struct Grid {
  int D;
  int n[3];
  double lo[3];
  double h;
  long long ncell;
  int bc[6];        // 0 = Neumann wall (homogeneous), 1 = Dirichlet, 2 = Robin
  double bcv[6];    // Dirichlet values, or a3 of a Robin wall (finest level only; 0 on coarse levels)
  double eps[2];
  double rob[6][2];  // Robin walls: a1, a2 of a1 phi + a2 dphi/dn_out = a3
  double lam[2];     // Helmholtz shift per phase: kappa lam phi joins each cell's balance
  int eb_robin;      // 1: electrode boundaries carry a1 phi + a2 dphi/dn_out = a3 (a3 in phiE)
  double eb_ra[2];   // their a1, a2
};

EBP_HD long long cell_index(const Grid& g, int i, int j, int k) {
  return (long long)i + (long long)g.n[0] * ((long long)j + (long long)g.n[1] * k);
}
EBP_HD void cell_ijk(const Grid& g, long long c, int I[3]) {
  I[0] = (int)(c % g.n[0]);
  I[1] = (int)((c / g.n[0]) % g.n[1]);
  I[2] = (int)(c / ((long long)g.n[0] * g.n[1]));
}
EBP_HD bool in_domain(const Grid& g, const int I[3]) {
  for (int k = 0; k < g.D; ++k)
    if (I[k] < 0 || I[k] >= g.n[k]) return false;
  return true;
}
EBP_HD long long node_index(const Grid& g, const int I[3]) {
  long long nx = g.n[0] + 1, ny = g.n[1] + 1;
  return (long long)I[0] + nx * ((long long)I[1] + ny * (g.D == 3 ? I[2] : 0));
}
EBP_HD long long node_count(const Grid& g) {
  return (long long)(g.n[0] + 1) * (g.n[1] + 1) * (g.D == 3 ? (g.n[2] + 1) : 1);
}
EBP_HD double node_x(const Grid& g, int k, int i) { return g.lo[k] + (double)i * g.h; }
EBP_HD double cell_x(const Grid& g, int k, int i) { return g.lo[k] + ((double)i + 0.5) * g.h; }
EBP_HD void transverse_axes(int D, int a, int t[2]) {
  int m = 0;
  for (int k = 0; k < D; ++k)
    if (k != a) t[m++] = k;
  if (D == 2) t[1] = -1;
}

// Per-cut-cell geometry records, structure of arrays indexed by the cut index
// q in [0, ncut).  Faces are numbered f = 2*a + side (side 0 = lo).
struct CutRecords {
  long long ncut;
  int* cell;        // [ncut]
  double* kappa;    // [2][ncut]
  double* alpha;    // [2D faces][2 phases][ncut]
  double* fcen;     // [2D faces][2 phases][2][ncut] centroid offsets along the transverse axes (units of h)
  uint8_t* ebk;     // [ncut]
  double* eba;      // [ncut]   EB area in units of h^{D-1}
  double* ebn;      // [3][ncut] unit normal out of the gas (electrode: fluid) fragment
  double* ebx;      // [3][ncut] EB centroid, physical
  double* phiE;     // [ncut]   electrode potential at the centroid (finest level)
  uint8_t* dofm;    // [ncut]   bit p: fragment of phase p carries an unknown
};

EBP_HD long long rec_alpha_index(long long ncut, int f, int p, long long q) { return ((long long)f * 2 + p) * ncut + q; }
EBP_HD long long rec_fcen_index(long long ncut, int f, int p, int t, long long q) {
  return (((long long)f * 2 + p) * 2 + t) * ncut + q;
}

}  // namespace ebp

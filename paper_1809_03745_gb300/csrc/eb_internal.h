// eb_internal.h -- host-side structures shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/ebpoisson.h"
#include "eb_common.cuh"

namespace ebp {

// One multigrid level on the device.
struct DevLevel {
  Grid g{};
  int coarse = 0;               // 1 below the finest level
  uint8_t* flags = nullptr;     // [ncell]
  int* cut_of_cell = nullptr;   // [ncell]
  int* irr_of_cell = nullptr;   // [ncell]
  CutRecords R{};               // records of cut cells
  uint8_t* order = nullptr;     // [2][ncut] EB stencil order per phase
  int* irr_cell = nullptr;      // [nirr]
  long long nirr = 0, nirr_red = 0;
  // sparse rows, two slots per irregular cell: row = 2k + phase
  int* row_ptr = nullptr;       // [2 nirr + 1]
  int* col = nullptr;           // [nnz]
  double* val = nullptr;        // [nnz]
  double* diag = nullptr;       // [2 nirr]; 0 marks an absent phase
  double* bconst = nullptr;     // [2 nirr] boundary data moved to b (finest level)
  double* bsig = nullptr;       // [2 nirr] coefficient of sigma/eps0 (finest level)
  long long nnz = 0;
  int* eb_q = nullptr;          // finest level: cut-record index of each EB-list cell
  long long n_eb = 0;
  std::vector<void*> allocs;
};

}  // namespace ebp

struct eb_geom {
  int device = 0;
  ebp::Csg csg{};
  ebp::Csg* d_csg = nullptr;
  uint8_t* d_lab = nullptr;
  std::vector<ebp::DevLevel> L;
  int n_phase = 1;
  long long n_dof = 0;
  long long stencil_counts[3] = {0, 0, 0};
  long long bytes = 0;
  int* d_status = nullptr;
};

namespace ebp {

// ------------------------------------------------- composite (one refined box)
// Box of coarse cells [lo, hi) refined by 2 and its coarse-fine (CF) sides.
struct CFBox {
  int lo[3], hi[3];
  int nside;
  int side_a[6], side_s[6];  // normal axis, 0 = low side / 1 = high side of the box
  long long off[7];          // first fine CF face of each side
  long long coff[7];         // first coarse CF face of each side
};

// One fine face on a CF side: the ghost value behind it is
// wf phi_F + wf2 phi_F2 + wc sum_k cw_k phi_coarse(cc_k); al = 0 marks a face
// without flux.
struct CFFace {
  int fcell, f2;  // fine cell, fine cell 3/2 h_f inside (-1: linear normal step)
  int ccell;      // coarse cell across the face
  int nc;
  int cc[5];
  double cw[5];
  double wf, wf2, wc, al;
};

// One coarse face on a CF side: the coarse cell outside the box (-1 when it
// has no gas unknown), its fine faces, and the coarse operator's own flux
// through the face as it enters the cell's row (sum w phi[col], cols encoded
// (phase << 30 | cell)).
struct CFCoarse {
  int ccell;
  int nfine;
  int fine[4];
  int n;
  int col[24];
  double w[24];
};

// Builds the CF face lists on the device from the fine (box) and coarse
// finest levels; EB_ERR_UNSUPPORTED when a dielectric unknown touches a CF side.
eb_status build_cf(const eb_geom* Gf, const eb_geom* Gc, const CFBox& B, CFFace* faces, CFCoarse* cfaces,
                   int* d_status, cudaStream_t s);

// kernels launched by the calling host thread since it started (every launch
// site of the library adds to it); a call's launches are the difference
void note_launch(int k = 1);
long long launch_total();

// error reporting
void set_error(const std::string& msg);
eb_status cuda_fail(cudaError_t e, const char* what);

// device memory owned by a level or handle
void* dev_alloc(std::vector<void*>& owner, size_t bytes, long long* counter, eb_status* st);

// geometry and operator construction (geometry.cu)
eb_status build_finest_geometry(eb_geom* G, cudaStream_t s);
eb_status build_coarse_geometry(eb_geom* G, int fine, cudaStream_t s, bool* stopped);
eb_status build_rows(eb_geom* G, int level, cudaStream_t s);
void free_level(DevLevel& L);
eb_status export_geometry(const eb_geom* G, eb_geom_arrays* out, cudaStream_t s);
eb_status launch_field(const eb_geom* G, const double* phi, const double* sigma, double* E, double* En,
                       cudaStream_t s);
eb_status launch_rhs64(const eb_geom* G, const double* s_rhs, const double* sigma, double* b, double* bnorm,
                       cudaStream_t s);
eb_status launch_kappa(const eb_geom* G, double* kappa, cudaStream_t s);

}  // namespace ebp

// solver internals used by the serving loop (server.cu)
struct eb_poisson;
eb_status batch_prepare(eb_poisson* P, const double* rhs, const double* sigma, const double* phi, cudaStream_t s);
eb_status batch_step(eb_poisson* const* P, int n, const double* const* rhs, const double* const* sigma,
                     double* const* phi, bool fresh, bool copy_out, int max_iters, cudaStream_t s,
                     double* kernel_ms);
void batch_info(eb_poisson* Q, eb_solve_info* inf);
eb_status batch_copy_out(eb_poisson* P, double* phi, cudaStream_t s);
long long poisson_device_bytes(const eb_poisson* P);
eb_status poisson_solve_b(eb_poisson* P, const double* d_b, double* d_x, double tol, int* cycles, cudaStream_t user,
                          int* outer = nullptr, double* kernel_ms = nullptr);
eb_status poisson_rhs(eb_poisson* P, const double* d_rhs, const double* d_sigma, double* d_b, cudaStream_t s);
eb_status poisson_residual_view(eb_poisson* P, const double* d_b, const double* d_phi, double* d_r, cudaStream_t s);

// tga.cu -- implicit diffusion by the TGA scheme (arXiv:1809.03745, Sec. 3.4,
// Eq. tga): two Helmholtz solves per step on the multigrid of the Poisson
// path, the operators applied and the right-hand sides formed on the device.
//
// For d phi/dt = L phi + rho with L phi = div(eps grad phi), each cut cell's
// balance is kappa d phi/dt = (L phi)_c + kappa rho (L_c integrated over the
// cell, M = diag(kappa)), and one step of length dt is
//   (M - mu1 L_c) psi = (M + mu3 L_c) phi + dt (M + mu4 L_c) rho,
//   (M - mu2 L_c) phi' = M psi.
// A handle with the Helmholtz shift lam solves (A0 + M lam) x = b, A0 = -L_c,
// so the stages run on handles shifted by 1/mu1 and 1/mu2 with right-hand
// sides divided by mu1 and mu2; L_c phi is minus the shift-free handle's
// operator applied with no boundary data (its residual for b = 0).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "eb_internal.h"

using namespace ebp;

namespace {

constexpr int TBT = 256;
inline unsigned nbt(long long n) { return (unsigned)((n + TBT - 1) / TBT); }

// R / mu1 with R = kappa phi + mu3 L phi + dt (kappa rho + mu4 L rho), on the
// entries with an unknown (0 elsewhere): the first stage's right-hand side
__global__ void k_tga_rhs(const uint8_t* flags, long long n, const double* kap, const double* phi,
                          const double* Lphi, const double* rho, const double* Lrho, double mu3, double mu4, double dt,
                          double inv_mu1, double* R) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int p = 0; p < 2; ++p) {
    const long long i = p * n + c;
    R[i] = ((flags[c] >> p) & 1)
               ? (kap[i] * phi[i] + mu3 * Lphi[i] + dt * (kap[i] * rho[i] + mu4 * Lrho[i])) * inv_mu1
               : 0.0;
  }
}

// kappa psi / mu2: the second stage's right-hand side
__global__ void k_tga_mass(const uint8_t* flags, long long n, const double* kap, const double* psi, double inv_mu2,
                           double* b) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int p = 0; p < 2; ++p) {
    const long long i = p * n + c;
    b[i] = ((flags[c] >> p) & 1) ? kap[i] * psi[i] * inv_mu2 : 0.0;
  }
}

}  // namespace

struct eb_tga {
  const eb_geom* G0 = nullptr;
  eb_poisson *P0 = nullptr, *P1 = nullptr, *P2 = nullptr;
  double dt = 0.0, mu[4] = {0.0, 0.0, 0.0, 0.0};
  double* kap = nullptr;  // [2][ncell] volume fractions
  double* work = nullptr;  // L phi, L rho, R, psi: [4][2][ncell]
  std::vector<void*> allocs;
  long long bytes = 0;
};

extern "C" eb_status eb_tga_coefficients(double dt, double mu[4]) {
  if (!mu || !(dt > 0.0) || !std::isfinite(dt)) {
    set_error("dt must be > 0 and finite, mu non-null");
    return EB_ERR_INVALID;
  }
  const double a = 2.0 - std::sqrt(2.0) - 2.220446049250313e-16;  // 2 - sqrt(2) less the machine precision
  const double r = std::sqrt(a * a - 4.0 * a + 2.0);
  mu[0] = 0.5 * (a - r) * dt;
  mu[1] = 0.5 * (a + r) * dt;
  mu[2] = (1.0 - a) * dt;
  mu[3] = (0.5 - a) * dt;
  return EB_OK;
}

extern "C" eb_status eb_tga_create(const eb_geom* G0, const eb_geom* G1, const eb_geom* G2, eb_poisson* P0,
                                   eb_poisson* P1, eb_poisson* P2, double dt, void* stream, eb_tga** out) {
  if (!out || !G0 || !G1 || !G2 || !P0 || !P1 || !P2) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  *out = nullptr;
  double mu[4];
  eb_status st = eb_tga_coefficients(dt, mu);
  if (st != EB_OK) return st;
  const Grid& g0 = G0->L[0].g;
  for (const eb_geom* G : {G1, G2}) {
    const Grid& g = G->L[0].g;
    if (g.ncell != g0.ncell || g.D != g0.D || g.n[0] != g0.n[0] || g.n[1] != g0.n[1] || g.n[2] != g0.n[2] ||
        G->n_phase != G0->n_phase || G->n_dof != G0->n_dof || G->device != G0->device) {
      set_error("the three geometries must come from one description");
      return EB_ERR_INVALID;
    }
  }
  auto near = [](double a, double b) { return std::fabs(a - b) <= 1e-12 * std::fabs(b); };
  const Grid &g1 = G1->L[0].g, &g2 = G2->L[0].g;
  bool ok = g0.lam[0] == 0.0 && g0.lam[1] == 0.0 && near(g1.lam[0], 1.0 / mu[0]) && near(g2.lam[0], 1.0 / mu[1]);
  if (G0->n_phase == 2) ok = ok && near(g1.lam[1], 1.0 / mu[0]) && near(g2.lam[1], 1.0 / mu[1]);
  if (!ok) {
    set_error("the geometries' Helmholtz shifts must be 0, 1/mu1 and 1/mu2 of this dt (eb_tga_coefficients)");
    return EB_ERR_INVALID;
  }
  eb_tga* T = new eb_tga();
  T->G0 = G0;
  T->P0 = P0;
  T->P1 = P1;
  T->P2 = P2;
  T->dt = dt;
  std::memcpy(T->mu, mu, sizeof(mu));
  const size_t n2 = 2 * (size_t)g0.ncell;
  T->kap = (double*)dev_alloc(T->allocs, sizeof(double) * n2, &T->bytes, &st);
  if (st == EB_OK) T->work = (double*)dev_alloc(T->allocs, sizeof(double) * 4 * n2, &T->bytes, &st);
  if (st == EB_OK) st = launch_kappa(G0, T->kap, (cudaStream_t)stream);
  if (st != EB_OK) {
    eb_tga_destroy(T);
    return st;
  }
  *out = T;
  return EB_OK;
}

extern "C" eb_status eb_tga_step(eb_tga* T, const double* d_phi, const double* d_rho, double* d_out, double tol,
                                 eb_solve_info* info, void* stream) {
  if (!T || !d_phi || !d_rho || !d_out) {
    set_error("null argument");
    return EB_ERR_INVALID;
  }
  if (!(tol > 0.0 && tol < 1.0)) {
    set_error("tol must lie in (0, 1)");
    return EB_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const DevLevel& F = T->G0->L[0];
  const long long n = F.g.ncell, n2 = 2 * n;
  double *Lphi = T->work, *Lrho = Lphi + n2, *R = Lrho + n2, *psi = R + n2;
  // L phi and L rho: the shift-free operator's residual for b = 0, no boundary data
  cudaMemsetAsync(R, 0, sizeof(double) * n2, s);
  eb_status st = poisson_residual_view(T->P0, R, d_phi, Lphi, s);
  if (st == EB_OK) st = poisson_residual_view(T->P0, R, d_rho, Lrho, s);
  if (st != EB_OK) return st;
  const double* mu = T->mu;
  k_tga_rhs<<<nbt(n), TBT, 0, s>>>(F.flags, n, T->kap, d_phi, Lphi, d_rho, Lrho, mu[2], mu[3], T->dt, 1.0 / mu[0], R);
  // stage 1 on the handle shifted by 1/mu1: (A0 + M / mu1) psi = R / mu1
  int cyc[2] = {0, 0}, outer[2] = {0, 0};
  double kms[2] = {0.0, 0.0};
  eb_status st1 = poisson_solve_b(T->P1, R, psi, tol, &cyc[0], s, &outer[0], &kms[0]);
  eb_status st2 = st1;
  if (st1 == EB_OK || st1 == EB_ERR_NOT_CONVERGED) {
    // stage 2 on the handle shifted by 1/mu2: (A0 + M / mu2) phi' = M psi / mu2
    k_tga_mass<<<nbt(n), TBT, 0, s>>>(F.flags, n, T->kap, psi, 1.0 / mu[1], R);
    st2 = poisson_solve_b(T->P2, R, d_out, tol, &cyc[1], s, &outer[1], &kms[1]);
  }
  if (info) {
    const eb_status sts[2] = {st1, st2};
    for (int k = 0; k < 2; ++k) {
      std::memset(&info[k], 0, sizeof(info[k]));
      info[k].status = sts[k];
      info[k].vcycles = cyc[k];
      info[k].outer_iters = outer[k];
      info[k].kernel_ms = kms[k];
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "tga step");
  return st1 != EB_OK ? st1 : st2;
}

extern "C" void eb_tga_destroy(eb_tga* T) {
  if (!T) return;
  for (void* p : T->allocs) cudaFree(p);
  delete T;
}

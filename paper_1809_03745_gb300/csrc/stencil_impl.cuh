// stencil_impl.cuh -- finite-volume operator rows of cut cells and the EB
// normal-derivative stencils (arXiv:1809.03745, Sec. 3.3 and 3.3.1).
//
// A level's operator is A = -(linear part of L) with
//   (L phi)_i = h^{-D} [ sum_faces alpha_f h^{D-1} F_f + alpha_EB h^{D-1} F_EB ]
// (integral form, Eq. poisson_integral).  Regular cells use the implicit
// 2D+1-point stencil; every other cell with an unknown gets a sparse row built
// here, one thread per (cell, phase).
#pragma once

#include "geom_impl.cuh"

namespace ebp {

constexpr int MAXS = 128;  // entries of one EB stencil
constexpr int MAXE = 192;  // entries of one operator row before the diagonal is split off

// Device view of one level's geometry.
struct LevelGeom {
  Grid g;
  int coarse;              // 1 on multigrid levels below the finest
  const uint8_t* flags;    // [ncell]
  const int* cut_of_cell;  // [ncell], -1 when not cut
  CutRecords R;
  long long nirr, nirr_red;
  const int* irr_cell;     // [nirr], red cells first, ascending within a colour
  const int* irr_of_cell;  // [ncell], -1 when the cell has no sparse row
};

EBP_HD int col_encode(int p, long long cell) { return (int)(((unsigned)p << 30) | (unsigned)cell); }
EBP_HD int col_phase(int col) { return (int)(((unsigned)col) >> 30); }
EBP_HD long long col_cell(int col) { return (long long)(((unsigned)col) & 0x3fffffffu); }

EBP_HD bool has_dof(const LevelGeom& L, const int I[3], int p) {
  if (!in_domain(L.g, I)) return false;
  return (L.flags[cell_index(L.g, I[0], I[1], I[2])] >> p) & 1;
}

struct FaceInfo {
  double al, t0, t1;
};

// Face normal to a with index J (J[a] in [0, n_a]): open for phase p when its
// aperture is positive and every adjacent cell inside the domain carries a
// phase-p unknown.  Aperture and centroid come from the record of an adjacent
// cut cell, else the face is a full face.
EBP_HDN bool face_open(const LevelGeom& L, int a, const int J[3], int p, FaceInfo& fi) {
  const Grid& g = L.g;
  for (int k = 0; k < g.D; ++k) {
    if (k == a) {
      if (J[k] < 0 || J[k] > g.n[k]) return false;
    } else if (J[k] < 0 || J[k] >= g.n[k]) {
      return false;
    }
  }
  int lo[3] = {J[0], J[1], J[2]};
  lo[a] -= 1;
  bool lo_in = J[a] > 0, hi_in = J[a] < g.n[a];
  if (lo_in && !has_dof(L, lo, p)) return false;
  if (hi_in && !has_dof(L, J, p)) return false;
  fi.al = 1.0;
  fi.t0 = 0.0;
  fi.t1 = 0.0;
  long long q = -1;
  int f = 0;
  if (hi_in) {
    q = L.cut_of_cell[cell_index(g, J[0], J[1], J[2])];
    f = 2 * a;
  }
  if (q < 0 && lo_in) {
    q = L.cut_of_cell[cell_index(g, lo[0], lo[1], lo[2])];
    f = 2 * a + 1;
  }
  if (q >= 0) {
    fi.al = L.R.alpha[rec_alpha_index(L.R.ncut, f, p, q)];
    fi.t0 = L.R.fcen[rec_fcen_index(L.R.ncut, f, p, 0, q)];
    fi.t1 = L.R.fcen[rec_fcen_index(L.R.ncut, f, p, 1, q)];
  }
  return fi.al > 0.0;
}

// Linear form: sum w_k phi[col_k] + c + sig * sigma_cell
template <int N>
struct Form {
  int n;
  int col[N];
  double w[N];
  double c, sig;
  int overflow;
  EBP_HD void zero() {
    n = 0;
    c = 0.0;
    sig = 0.0;
    overflow = 0;
  }
  EBP_HD void add(int cl, double v) {
    for (int k = 0; k < n; ++k)
      if (col[k] == cl) {
        w[k] = w[k] + v;
        return;
      }
    if (n < N) {
      col[n] = cl;
      w[n] = v;
      ++n;
    } else {
      overflow = 1;
    }
  }
};

// face-centred flux through face (a, J) in the +e_a direction, phase p
struct CFlux {
  int n;
  int col[2];
  double w[2];
  double c;
};

// Interior: eps (phi_hi - phi_lo)/h.  Dirichlet wall with value phi0: the
// outward derivative (8 phi0 - 9 phi1 + phi2)/(3h), phi1 the wall cell, phi2
// the next cell inward (the order of indices that makes it second order), or
// 2 (phi0 - phi1)/h when phi2 is not reachable through an open face.  Robin
// wall (a1 phi0 + a2 dphi/dn_out = a3, Sec. 3.3.1): the same formula, written
// Aw phi0 + R, fixes the wall value phi0 = (a3 - a2 R) / (a1 + a2 Aw); the
// flux is then eps (Aw a3 + a1 R) / (a1 + a2 Aw).
EBP_HDN bool centred_flux(const LevelGeom& L, int a, const int J[3], int p, CFlux& F) {
  FaceInfo fi;
  if (!face_open(L, a, J, p, fi)) return false;
  const Grid& g = L.g;
  double eps = g.eps[p], h = g.h;
  F.n = 0;
  F.c = 0.0;
  bool lo_wall = J[a] == 0, hi_wall = J[a] == g.n[a];
  if (!lo_wall && !hi_wall) {
    F.n = 2;
    F.col[0] = col_encode(p, cell_index(g, J[0], J[1], J[2]));
    F.w[0] = eps / h;
    int lo[3] = {J[0], J[1], J[2]};
    lo[a] -= 1;
    F.col[1] = col_encode(p, cell_index(g, lo[0], lo[1], lo[2]));
    F.w[1] = -eps / h;
    return true;
  }
  int hi = hi_wall ? 1 : 0;
  if (!g.bc[2 * a + hi]) return false;
  int C[3] = {J[0], J[1], J[2]};
  if (hi) C[a] -= 1;
  int C2[3] = {C[0], C[1], C[2]};
  C2[a] += hi ? -1 : 1;
  int between[3] = {C[0], C[1], C[2]};
  if (!hi) between[a] += 1;
  FaceInfo fb;
  bool has2 = face_open(L, a, between, p, fb);
  double phi0 = g.bcv[2 * a + hi];
  double sgn = hi ? 1.0 : -1.0;  // outward is +e_a on the hi wall
  long long c1 = cell_index(g, C[0], C[1], C[2]);
  if (g.bc[2 * a + hi] == 2) {
    const double a1 = g.rob[2 * a + hi][0], a2 = g.rob[2 * a + hi][1];
    const double Aw = has2 ? 8.0 / (3.0 * h) : 2.0 / h, den = a1 + a2 * Aw;
    const double f = sgn * eps * a1 / den;  // phi0 holds a3 here
    F.col[0] = col_encode(p, c1);
    if (has2) {
      F.n = 2;
      F.w[0] = f * (-9.0 / (3.0 * h));
      F.col[1] = col_encode(p, cell_index(g, C2[0], C2[1], C2[2]));
      F.w[1] = f * (1.0 / (3.0 * h));
    } else {
      F.n = 1;
      F.w[0] = f * (-2.0 / h);
    }
    F.c = sgn * eps * Aw * phi0 / den;
    return true;
  }
  if (has2) {
    F.n = 2;
    F.col[0] = col_encode(p, c1);
    F.w[0] = sgn * (-9.0 * eps / (3.0 * h));
    F.col[1] = col_encode(p, cell_index(g, C2[0], C2[1], C2[2]));
    F.w[1] = sgn * (eps / (3.0 * h));
    F.c = sgn * (8.0 * eps * phi0 / (3.0 * h));
  } else {
    F.n = 1;
    F.col[0] = col_encode(p, c1);
    F.w[0] = sgn * (-2.0 * eps / h);
    F.c = sgn * (2.0 * eps * phi0 / h);
  }
  return true;
}

template <int N>
EBP_HD void form_add_cflux(Form<N>& L, double s, const CFlux& F) {
  for (int k = 0; k < F.n; ++k) L.add(F.col[k], s * F.w[k]);
  L.c = L.c + s * F.c;
}

// Adds scale * (flux through the centroid of face (a, J), +e_a direction):
// linear interpolation of face-centred fluxes toward the centroid (Sec. 3.3),
// bilinear in 3D; planar 3-point form, then 1-D, then none when a neighbouring
// face carries no flux.
template <int N>
EBP_HDN void add_centroid_flux(const LevelGeom& L, int a, const int J[3], int p, double scale, Form<N>& R) {
  CFlux F00, F10, F01, F11;
  if (!centred_flux(L, a, J, p, F00)) return;
  FaceInfo fi;
  face_open(L, a, J, p, fi);
  int t[2];
  transverse_axes(L.g.D, a, t);
  double t1 = fi.t0, t2 = (L.g.D == 3) ? fi.t1 : 0.0;
  double a1 = fabs(t1), a2 = fabs(t2);
  int s1 = t1 > 0.0 ? 1 : -1, s2 = t2 > 0.0 ? 1 : -1;
  bool need10 = a1 > 0.0, need01 = a2 > 0.0, need11 = need10 && need01;
  bool have10 = false, have01 = false, have11 = false;
  if (need10) {
    int K[3] = {J[0], J[1], J[2]};
    K[t[0]] += s1;
    have10 = centred_flux(L, a, K, p, F10);
  }
  if (need01) {
    int K[3] = {J[0], J[1], J[2]};
    K[t[1]] += s2;
    have01 = centred_flux(L, a, K, p, F01);
  }
  if (need11) {
    int K[3] = {J[0], J[1], J[2]};
    K[t[0]] += s1;
    K[t[1]] += s2;
    have11 = centred_flux(L, a, K, p, F11);
  }
  if ((!need10 || have10) && (!need01 || have01) && (!need11 || have11)) {
    form_add_cflux(R, scale * ((1.0 - a1) * (1.0 - a2)), F00);
    if (need10) form_add_cflux(R, scale * (a1 * (1.0 - a2)), F10);
    if (need01) form_add_cflux(R, scale * ((1.0 - a1) * a2), F01);
    if (need11) form_add_cflux(R, scale * (a1 * a2), F11);
  } else if ((!need10 || have10) && (!need01 || have01)) {
    form_add_cflux(R, scale * (1.0 - a1 - a2), F00);
    if (need10) form_add_cflux(R, scale * a1, F10);
    if (need01) form_add_cflux(R, scale * a2, F01);
  } else if (need10 && have10) {
    form_add_cflux(R, scale * (1.0 - a1), F00);
    form_add_cflux(R, scale * a1, F10);
  } else if (need01 && have01) {
    form_add_cflux(R, scale * (1.0 - a2), F00);
    form_add_cflux(R, scale * a2, F01);
  } else {
    form_add_cflux(R, scale, F00);
  }
}

// ------------------------------------------------------------ EB stencils

struct Stencil {
  int order;  // 2, 1, 3 = least squares, 0 = none
  int n;
  double w0;
  long long cell[MAXS];
  double w[MAXS];
};

// dphi/dn_in = w0 phi_B + sum_k w_k phi_k at the EB centroid xB of cell I,
// phase p, n_in pointing into phase p (Eq. bndry_stencil).  The cut cell
// itself never enters.  Order 2: rays to the planes of cell centres one and
// two cells away along the dominant axis of n_in (lowest axis on ties),
// quadratic tensor interpolation over three cells per transverse axis centred
// on the cell holding the intersection (shifted inward at a wall), one-sided
// three-point derivative along the ray.  Order 1: the first plane only, two
// bracketing cells per transverse axis.  Least squares: phi_B + g.(x - x_B)
// fitted over the fluid-side cells of the 3^D, then 5^D, neighbourhood.
EBP_HDN int build_stencil(const LevelGeom& L, const int I[3], int p, const double xB[3], const double nin[3],
                         Stencil& S) {
  const Grid& g = L.g;
  const int D = g.D;
  const double h = g.h;
  int a = 0;
  for (int k = 1; k < D; ++k)
    if (fabs(nin[k]) > fabs(nin[a])) a = k;
  int sg = nin[a] > 0.0 ? 1 : -1;
  int t[2];
  transverse_axes(D, a, t);
  int nt = D - 1;
  S.order = 0;
  S.n = 0;
  S.w0 = 0.0;
  {  // second order
    bool ok = true;
    double ell[3];
    int base = 0;
    for (int m = 1; m <= 2 && ok; ++m) {
      double P = cell_x(g, a, I[a]) + (double)(m * sg) * h;
      double l = (P - xB[a]) / nin[a];
      ell[m] = l;
      int ka[2] = {0, 0};
      double w3[2][3];
      for (int q = 0; q < nt; ++q) {
        int tt = t[q];
        double y = xB[tt] + l * nin[tt];
        int k = (int)floor((y - g.lo[tt]) / h);
        if (k < 1) k = 1;
        if (k > g.n[tt] - 2) k = g.n[tt] - 2;
        double xi = (y - cell_x(g, tt, k)) / h;
        ka[q] = k;
        w3[q][0] = 0.5 * xi * (xi - 1.0);
        w3[q][1] = 1.0 - xi * xi;
        w3[q][2] = 0.5 * xi * (xi + 1.0);
      }
      int nz = (nt == 2) ? 3 : 1;
      for (int iz = 0; iz < nz && ok; ++iz)
        for (int iy = 0; iy < 3 && ok; ++iy) {
          int Jc[3] = {I[0], I[1], I[2]};
          Jc[a] = I[a] + m * sg;
          Jc[t[0]] = ka[0] + iy - 1;
          double w = w3[0][iy];
          if (nt == 2) {
            Jc[t[1]] = ka[1] + iz - 1;
            w = w * w3[1][iz];
          }
          if (!has_dof(L, Jc, p)) {
            ok = false;
            break;
          }
          S.cell[S.n] = cell_index(g, Jc[0], Jc[1], Jc[2]);
          S.w[S.n] = w;
          ++S.n;
        }
      if (m == 1) base = S.n;
    }
    if (ok) {
      double l1 = ell[1], l2 = ell[2];
      double c1 = (l2 / l1) / (l2 - l1), c2 = -(l1 / l2) / (l2 - l1);
      for (int k = 0; k < S.n; ++k) S.w[k] = (k < base ? c1 : c2) * S.w[k];
      S.w0 = -(c1 + c2);
      S.order = 2;
      return 0;
    }
    S.n = 0;
  }
  {  // first order
    double P = cell_x(g, a, I[a]) + (double)sg * h;
    double l = (P - xB[a]) / nin[a];
    int ka[2] = {0, 0};
    double w2[2][2];
    for (int q = 0; q < nt; ++q) {
      int tt = t[q];
      double y = xB[tt] + l * nin[tt];
      int k = (int)floor((y - g.lo[tt]) / h - 0.5);
      if (k < 0) k = 0;
      if (k > g.n[tt] - 2) k = g.n[tt] - 2;
      double xi = (y - cell_x(g, tt, k)) / h;
      ka[q] = k;
      w2[q][0] = 1.0 - xi;
      w2[q][1] = xi;
    }
    bool ok = true;
    int nz = (nt == 2) ? 2 : 1;
    for (int iz = 0; iz < nz && ok; ++iz)
      for (int iy = 0; iy < 2 && ok; ++iy) {
        int Jc[3] = {I[0], I[1], I[2]};
        Jc[a] = I[a] + sg;
        Jc[t[0]] = ka[0] + iy;
        double w = w2[0][iy];
        if (nt == 2) {
          Jc[t[1]] = ka[1] + iz;
          w = w * w2[1][iz];
        }
        if (!has_dof(L, Jc, p)) {
          ok = false;
          break;
        }
        S.cell[S.n] = cell_index(g, Jc[0], Jc[1], Jc[2]);
        S.w[S.n] = w / l;
        ++S.n;
      }
    if (ok) {
      S.w0 = -1.0 / l;
      S.order = 1;
      return 0;
    }
    S.n = 0;
  }
  for (int rad = 1; rad <= 2; ++rad) {  // least squares
    double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    int w = 2 * rad + 1, nz = (D == 3) ? w : 1;
    S.n = 0;
    bool full = false;
    for (int oz = 0; oz < nz; ++oz)
      for (int oy = 0; oy < w; ++oy)
        for (int ox = 0; ox < w; ++ox) {
          int Jc[3] = {I[0] + ox - rad, I[1] + oy - rad, I[2] + (D == 3 ? oz - rad : 0)};
          if (Jc[0] == I[0] && Jc[1] == I[1] && Jc[2] == I[2]) continue;
          if (!has_dof(L, Jc, p)) continue;
          double dx[3] = {0.0, 0.0, 0.0}, dn = 0.0;
          for (int k = 0; k < D; ++k) {
            dx[k] = cell_x(g, k, Jc[k]) - xB[k];
            dn = dn + dx[k] * nin[k];
          }
          if (!(dn > 0.0)) continue;
          if (S.n >= MAXS) {
            full = true;
            continue;
          }
          for (int r = 0; r < D; ++r)
            for (int s = 0; s < D; ++s) M[r][s] = M[r][s] + dx[r] * dx[s];
          S.cell[S.n] = cell_index(g, Jc[0], Jc[1], Jc[2]);
          S.w[S.n] = 0.0;
          ++S.n;
        }
    if (full) return ST_OVERFLOW;
    if (S.n < D) continue;
    double u[3] = {0.0, 0.0, 0.0};
    if (D == 2) {
      double det = M[0][0] * M[1][1] - M[0][1] * M[1][0];
      if (!(fabs(det) > 1e-12 * h * h * h * h)) continue;
      u[0] = (nin[0] * M[1][1] - M[0][1] * nin[1]) / det;
      u[1] = (M[0][0] * nin[1] - nin[0] * M[1][0]) / det;
    } else {
      double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                   M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
      if (!(fabs(det) > 1e-12 * h * h * h * h * h * h)) continue;
      for (int col = 0; col < 3; ++col) {
        double Mc[3][3];
        for (int r = 0; r < 3; ++r)
          for (int s = 0; s < 3; ++s) Mc[r][s] = (s == col) ? nin[r] : M[r][s];
        double dc = Mc[0][0] * (Mc[1][1] * Mc[2][2] - Mc[1][2] * Mc[2][1]) -
                    Mc[0][1] * (Mc[1][0] * Mc[2][2] - Mc[1][2] * Mc[2][0]) +
                    Mc[0][2] * (Mc[1][0] * Mc[2][1] - Mc[1][1] * Mc[2][0]);
        u[col] = dc / det;
      }
    }
    double sw = 0.0;
    for (int k = 0; k < S.n; ++k) {
      int Jc[3];
      cell_ijk(g, S.cell[k], Jc);
      double wk = 0.0;
      for (int r = 0; r < D; ++r) wk = wk + u[r] * (cell_x(g, r, Jc[r]) - xB[r]);
      S.w[k] = wk;
      sw = sw + wk;
    }
    S.w0 = -sw;
    S.order = 3;
    return 0;
  }
  S.n = 0;
  return ST_UNSUPPORTED;
}

// inward normal of phase p at cut record q
EBP_HD void record_nin(const LevelGeom& L, long long q, int p, double xB[3], double nin[3]) {
  long long nq = L.R.ncut;
  double sgn = (L.R.ebk[q] == EBK_IFACE && p == 1) ? 1.0 : -1.0;
  for (int k = 0; k < 3; ++k) {
    xB[k] = L.R.ebx[k * nq + q];
    nin[k] = sgn * L.R.ebn[k * nq + q];
  }
}

// dphi/dn_in of fragment (cell, p) with the boundary value substituted, as a
// form over the unknowns: electrode -> phi_E; dielectric interface -> phi_B
// eliminated from eps_g dphi/dn_g + eps_d dphi/dn_d = -sigma/eps0 (Eq.
// matching with normals pointing into each fluid; Gauss's law fixes the sign).
// A Robin electrode (a1 phi_B + a2 dphi/dn_out = a3, phiE holding a3; Sec.
// 3.3.1): with the ray stencil dphi/dn_in = w0 phi_B + S and dn_out = -dn_in,
// phi_B = (a3 + a2 S) / (a1 - a2 w0) and dphi/dn_in = (w0 a3 + a1 S) / (a1 - a2 w0).
// Scaled by `scale` and added to R; returns a status.  `orders` gets the
// stencil order of each phase.
template <int N>
EBP_HDN int add_eb_dphidn(const LevelGeom& L, long long q, const int I[3], int p, double phiE, double scale, Form<N>& R,
                         int orders[2]) {
  Stencil S;
  double xB[3], nin[3];
  orders[0] = orders[1] = 0;
  if (L.R.ebk[q] == EBK_ELEC) {
    record_nin(L, q, p, xB, nin);
    int st = build_stencil(L, I, p, xB, nin, S);
    if (st) return st;
    orders[p] = S.order;
    if (L.g.eb_robin) {
      const double a1 = L.g.eb_ra[0], a2 = L.g.eb_ra[1], den = a1 - a2 * S.w0;
      for (int k = 0; k < S.n; ++k) R.add(col_encode(p, S.cell[k]), scale * (a1 / den) * S.w[k]);
      R.c = R.c + scale * (S.w0 * phiE / den);
      return 0;
    }
    for (int k = 0; k < S.n; ++k) R.add(col_encode(p, S.cell[k]), scale * S.w[k]);
    R.c = R.c + scale * (S.w0 * phiE);
    return 0;
  }
  // interface: w0 of both phases first
  double w0[2];
  for (int ph = 0; ph < 2; ++ph) {
    record_nin(L, q, ph, xB, nin);
    int st = build_stencil(L, I, ph, xB, nin, S);
    if (st) return st;
    w0[ph] = S.w0;
    orders[ph] = S.order;
  }
  double eg = L.g.eps[0], ed = L.g.eps[1];
  double Dn = eg * w0[0] + ed * w0[1];
  if (!(fabs(Dn) > 0.0)) return ST_UNSUPPORTED;
  // dn_p = S_p + w0_p phi_B,  phi_B = (-sigma - eg S_g - ed S_d) / Dn
  for (int ph = 0; ph < 2; ++ph) {
    record_nin(L, q, ph, xB, nin);
    build_stencil(L, I, ph, xB, nin, S);
    double coef = ((ph == p) ? 1.0 : 0.0) - w0[p] * (ph == 0 ? eg : ed) / Dn;
    for (int k = 0; k < S.n; ++k) R.add(col_encode(ph, S.cell[k]), scale * (coef * S.w[k]));
  }
  R.sig = R.sig + scale * (-w0[p] / Dn);
  return 0;
}

// Row (L phi)_cell for phase p as a form.  Returns a status; orders receives
// the EB stencil orders.
template <int N>
EBP_HDN int build_row_form(const LevelGeom& L, long long cell, int p, Form<N>& R, int orders[2]) {
  const Grid& g = L.g;
  int I[3];
  cell_ijk(g, cell, I);
  R.zero();
  orders[0] = orders[1] = 0;
  for (int a = 0; a < g.D; ++a)
    for (int s = 0; s < 2; ++s) {
      int J[3] = {I[0], I[1], I[2]};
      J[a] += s;
      FaceInfo fi;
      if (!face_open(L, a, J, p, fi)) continue;
      add_centroid_flux(L, a, J, p, (s ? 1.0 : -1.0) * fi.al / g.h, R);
    }
  long long q = L.cut_of_cell[cell];
  if (q >= 0 && L.R.ebk[q] != EBK_NONE) {
    double scale = -g.eps[p] * L.R.eba[q] / g.h;  // F_EB = -eps dphi/dn_in
    int st = add_eb_dphidn(L, q, I, p, L.R.phiE[q], scale, R, orders);
    if (st) return st;
  }
  // the Helmholtz shift kappa lam phi (R holds minus the operator's linear part)
  if (g.lam[p] != 0.0) {
    const double kap = q >= 0 ? L.R.kappa[p * L.R.ncut + q] : 1.0;
    R.add(col_encode(p, cell), -kap * g.lam[p]);
  }
  return R.overflow ? ST_OVERFLOW : 0;
}

}  // namespace ebp

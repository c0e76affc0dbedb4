// coarsen_impl.cuh -- coarse multigrid geometry from the fine level
// (arXiv:1809.03745, Sec. 3.1: the EB graph is generated on the finest level
// and coarsened through the hierarchy; Sec. 3.3.2: coarsening may lose
// features and the bottom is reached sooner).
#pragma once

#include "stencil_impl.cuh"

namespace ebp {

// reasons for stopping the coarsening (ORed with ST_STOP)
constexpr int STOP_TWO_KINDS = 8;     // electrode and dielectric interface in one coarse cell
constexpr int STOP_PHASES = 16;       // both phases without a dielectric interface
constexpr int STOP_THIN = 32;         // a feature thinner than the coarse cell (EB areas cancel)

// 0 covered, 1 regular gas, 2 regular dielectric, 3 cut
EBP_HD uint8_t coarse_preclass(const LevelGeom& F, const Grid& gc, long long C) {
  int IC[3];
  cell_ijk(gc, C, IC);
  int nch = 1 << gc.D;
  uint8_t any = 0, all_reg = 1, ph = 0xff;
  for (int k = 0; k < nch; ++k) {
    int I[3] = {2 * IC[0] + (k & 1), 2 * IC[1] + ((k >> 1) & 1), gc.D == 3 ? 2 * IC[2] + ((k >> 2) & 1) : 0};
    long long c = cell_index(F.g, I[0], I[1], I[2]);
    uint8_t f = F.flags[c] & 3;
    any |= f;
    if (F.cut_of_cell[c] >= 0 || (f != 1 && f != 2)) all_reg = 0;
    if (ph == 0xff) ph = f;
    else if (f != ph) all_reg = 0;
  }
  if (!any) return 0;
  if (all_reg) return ph;
  return 3;
}

// Coarse cut cell q from its children: the volume fraction is the mean of the
// children's, a coarse face aperture the mean of its child faces, face
// centroids and the EB centroid are aperture / area weighted means, and the
// EB normal follows from the coarse apertures.  Children of one phase form a
// single coarse unknown even when they do not touch inside the coarse cell
// (the coarse operator only steers the multigrid correction).  Returns ST_STOP
// (with a reason bit) where a coarse cell would hold both an electrode and the
// dielectric interface, or both phases without an interface.
EBP_HDN int coarse_cut_geometry(const LevelGeom& F, const Grid& gc, const CutRecords& Rc, long long q) {
  const Grid& gf = F.g;
  const int D = gf.D;
  const long long nq = Rc.ncut, nqf = F.R.ncut;
  int IC[3];
  cell_ijk(gc, Rc.cell[q], IC);
  int nch = 1 << D;
  double kap[2] = {0.0, 0.0};
  int kindmask = 0;
  double wsum = 0.0, xs[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < nch; ++k) {
    int I[3] = {2 * IC[0] + (k & 1), 2 * IC[1] + ((k >> 1) & 1), D == 3 ? 2 * IC[2] + ((k >> 2) & 1) : 0};
    long long c = cell_index(gf, I[0], I[1], I[2]);
    uint8_t f = F.flags[c];
    int cq = F.cut_of_cell[c];
    for (int p = 0; p < 2; ++p)
      if ((f >> p) & 1) kap[p] += (cq >= 0) ? F.R.kappa[p * nqf + cq] : 1.0;
    if (cq >= 0 && (f & 3)) {
      uint8_t ek = F.R.ebk[cq];
      if (ek == EBK_ELEC) kindmask |= 1;
      if (ek == EBK_IFACE) kindmask |= 2;
      if (ek != EBK_NONE) {
        double w = F.R.eba[cq];
        wsum += w;
        for (int d = 0; d < 3; ++d) xs[d] += w * F.R.ebx[d * nqf + cq];
      }
    }
  }
  for (int p = 0; p < 2; ++p) kap[p] /= (double)nch;
  Rc.kappa[q] = kap[0];
  Rc.kappa[nq + q] = kap[1];
  Rc.phiE[q] = 0.0;
  Rc.dofm[q] = 0;
  Rc.ebk[q] = EBK_NONE;
  Rc.eba[q] = 0.0;
  for (int d = 0; d < 3; ++d) {
    Rc.ebn[d * nq + q] = 0.0;
    Rc.ebx[d * nq + q] = 0.0;
  }
  if (kindmask == 3) return ST_STOP | STOP_TWO_KINDS;
  uint8_t kind = (kindmask & 2) ? EBK_IFACE : ((kindmask & 1) ? EBK_ELEC : EBK_NONE);
  bool hasp[2] = {kap[0] > 0.0, kap[1] > 0.0};
  if (hasp[0] && hasp[1] && kind != EBK_IFACE) return ST_STOP | STOP_PHASES;
  double alc[6][2];
  int nfc = 1 << (D - 1);
  for (int a = 0; a < D; ++a) {
    int t[2];
    transverse_axes(D, a, t);
    for (int s = 0; s < 2; ++s) {
      int fidx = 2 * a + s;
      for (int p = 0; p < 2; ++p) {
        double sa = 0.0, s0 = 0.0, s1 = 0.0;
        for (int k = 0; k < nch; ++k) {
          int o[3] = {k & 1, (k >> 1) & 1, D == 3 ? (k >> 2) & 1 : 0};
          if (o[a] != s) continue;
          int J[3] = {2 * IC[0] + o[0], 2 * IC[1] + o[1], D == 3 ? 2 * IC[2] + o[2] : 0};
          J[a] += s;
          FaceInfo fi;
          if (!face_open(F, a, J, p, fi)) continue;
          double off0 = ((double)o[t[0]] - 0.5) * 0.5 + 0.5 * fi.t0;
          double off1 = (D == 3) ? ((double)o[t[1]] - 0.5) * 0.5 + 0.5 * fi.t1 : 0.0;
          sa += fi.al;
          s0 += fi.al * off0;
          s1 += fi.al * off1;
        }
        double al = sa / (double)nfc;
        alc[fidx][p] = al;
        Rc.alpha[rec_alpha_index(nq, fidx, p, q)] = al;
        Rc.fcen[rec_fcen_index(nq, fidx, p, 0, q)] = sa > 0.0 ? s0 / sa : 0.0;
        Rc.fcen[rec_fcen_index(nq, fidx, p, 1, q)] = sa > 0.0 ? s1 / sa : 0.0;
      }
    }
  }
  int p0 = (kind == EBK_IFACE) ? 0 : ((hasp[1] && !hasp[0]) ? 1 : 0);
  double vec[3] = {0.0, 0.0, 0.0}, len2 = 0.0;
  for (int a = 0; a < D; ++a) {
    vec[a] = -(alc[2 * a + 1][p0] - alc[2 * a][p0]);
    len2 += vec[a] * vec[a];
  }
  double ar = sqrt(len2);
  // children's EB pieces facing opposite ways (both sides of a feature thinner
  // than this cell) cancel in the coarse normal: the coarse level cannot
  // represent the feature, so coarsening stops here
  if (kind != EBK_NONE && ar * (double)(1 << (D - 1)) < 0.5 * wsum) return ST_STOP | STOP_THIN;
  if (kind != EBK_NONE && ar > 0.0 && wsum > 0.0) {
    Rc.ebk[q] = kind;
    Rc.eba[q] = ar;
    for (int d = 0; d < 3; ++d) {
      Rc.ebn[d * nq + q] = vec[d] / ar;
      Rc.ebx[d * nq + q] = xs[d] / wsum;
    }
  } else {
    for (int d = 0; d < D; ++d) Rc.ebx[d * nq + q] = cell_x(gc, d, IC[d]);
  }
  return 0;
}

}  // namespace ebp

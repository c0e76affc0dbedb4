// geom_impl.cuh -- per-item cut-cell geometry (arXiv:1809.03745, Sec. 3.1).
//
// Every function here works on one node, face or cell and is called from the
// geometry kernels.  The translation units that include this header are
// compiled without FMA contraction so that each product and sum is rounded
// on its own: the geometry is then reproducible across devices and hosts.
#pragma once

#include "eb_common.cuh"

namespace ebp {

// --------------------------------------------------------- implicit functions

EBP_HDN double prim_eval(const Csg& c, int p, const double x[3]) {
  const double* q = c.par[p];
  switch (c.kind[p]) {
    case 0: {  // sphere: |x - c| - r
      double dx = x[0] - q[0], dy = x[1] - q[1], dz = x[2] - q[2];
      return sqrt(dx * dx + dy * dy + dz * dz) - q[3];
    }
    case 1: {  // capsule: distance to segment a->b minus r
      double ab0 = q[3] - q[0], ab1 = q[4] - q[1], ab2 = q[5] - q[2];
      double ap0 = x[0] - q[0], ap1 = x[1] - q[1], ap2 = x[2] - q[2];
      double num = ap0 * ab0 + ap1 * ab1 + ap2 * ab2;
      double den = ab0 * ab0 + ab1 * ab1 + ab2 * ab2;
      double t = num / den;
      if (t < 0.0) t = 0.0;
      if (t > 1.0) t = 1.0;
      double c0 = x[0] - (q[0] + t * ab0), c1 = x[1] - (q[1] + t * ab1), c2 = x[2] - (q[2] + t * ab2);
      double dd = c0 * c0 + c1 * c1 + c2 * c2;
      return sqrt(dd) - q[6];
    }
    case 2:  // half space: n.x - d
      return q[0] * x[0] + q[1] * x[1] + q[2] * x[2] - q[3];
    case 3: {  // sinusoidal surface: x[up] - (c + A sin(2 pi k x[t] + ph))
      int up = (int)q[0], ta = (int)q[5];
      double arg = 6.283185307179586 * q[3] * x[ta] + q[4];
      return x[up] - (q[1] + q[2] * sin(arg));
    }
    case 4: {  // finite cylinder along an axis
      int a = (int)q[0];
      double r2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        if (k == a) continue;
        double dk = x[k] - q[1 + k];
        r2 = r2 + dk * dk;
      }
      double m = sqrt(r2) - q[4];
      double e1 = q[5] - x[a], e2 = x[a] - q[6];
      if (e1 > m) m = e1;
      if (e2 > m) m = e2;
      return m;
    }
    case 5: {  // box
      double m = -1e300;
      for (int k = 0; k < 3; ++k) {
        double a1 = q[k] - x[k], a2 = x[k] - q[3 + k];
        if (a1 > m) m = a1;
        if (a2 > m) m = a2;
      }
      return m;
    }
  }
  return 1e300;
}

// Evaluates CSG nodes 0..root in order (children precede parents).
EBP_HDN double csg_eval(const Csg& c, int root, const double x[3]) {
  double v[MAX_NODES];
  for (int i = 0; i <= root; ++i) {
    int op = c.op[i];
    double r;
    if (op == 0) {
      r = prim_eval(c, c.a[i], x);
    } else if (op == 3) {
      r = -v[c.a[i]];
    } else {
      double A = v[c.a[i]], B = v[c.b[i]];
      if (op == 1) r = A < B ? A : B;
      else r = A > B ? A : B;
    }
    v[i] = r;
  }
  return v[root];
}

EBP_HD int label_at(const Csg& c, const double x[3]) {
  if (c.root_E >= 0 && csg_eval(c, c.root_E, x) < 0.0) return LAB_E;
  if (c.root_D >= 0 && csg_eval(c, c.root_D, x) < 0.0) return LAB_D;
  return LAB_G;
}

// Crossing on the edge from node I along axis a, as a fraction of h from node
// I: bisection on the implicit function separating the two end labels, exactly
// 60 halvings, midpoint of the final bracket.
EBP_HDN double edge_crossing(const Csg& c, const Grid& g, const uint8_t* lab, const int I[3], int a) {
  int J[3] = {I[0], I[1], I[2]};
  J[a] += 1;
  int la = lab[node_index(g, I)], lb = lab[node_index(g, J)];
  bool elec = (la == LAB_E || lb == LAB_E);
  int root = elec ? c.root_E : c.root_D;
  int inside_lab = elec ? LAB_E : LAB_D;
  int in_a = (la == inside_lab);
  double x[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < g.D; ++k) x[k] = node_x(g, k, I[k]);
  double lo = node_x(g, a, I[a]), hi = node_x(g, a, I[a] + 1);
  for (int it = 0; it < 60; ++it) {
    double m = 0.5 * (lo + hi);
    x[a] = m;
    int in = csg_eval(c, root, x) < 0.0;
    if (in == in_a) lo = m;
    else hi = m;
  }
  double cr = 0.5 * (lo + hi);
  double fr = (cr - node_x(g, a, I[a])) / g.h;
  // a crossing within 1e-8 h of a node is put on the node: the boundary moves
  // by less than 1e-8 h, and fragments of vanishing size become exactly empty
  if (fr < 1e-8) fr = 0.0;
  if (fr > 1.0 - 1e-8) fr = 1.0;
  return fr;
}

// ------------------------------------------------------------------ faces

struct FaceGeom {
  double al[2];     // aperture per phase
  double fc[2][2];  // centroid offsets per phase along the transverse axes, units of h
  int status;
};

// Face normal to a whose lowest corner node is J.  2D: an edge along the
// transverse axis.  3D: marching squares on the square without saddles; the
// fluid part of each phase is the polygon through its corners and the two
// edge crossings, integrated by the shoelace formula.
EBP_HDN FaceGeom face_geometry(const Csg& c, const Grid& g, const uint8_t* lab, int a, const int J[3]) {
  FaceGeom F;
  F.status = 0;
  for (int p = 0; p < 2; ++p) {
    F.al[p] = 0.0;
    F.fc[p][0] = 0.0;
    F.fc[p][1] = 0.0;
  }
  int t[2];
  transverse_axes(g.D, a, t);
  if (g.D == 2) {
    int K[3] = {J[0], J[1], J[2]};
    K[t[0]] += 1;
    int la = lab[node_index(g, J)], lb = lab[node_index(g, K)];
    if (la == lb) {
      if (la != LAB_E) F.al[la - 1] = 1.0;
      return F;
    }
    double fr = edge_crossing(c, g, lab, J, t[0]);
    if (la != LAB_E) {
      F.al[la - 1] = fr;
      F.fc[la - 1][0] = 0.5 * fr - 0.5;
    }
    if (lb != LAB_E) {
      F.al[lb - 1] = 1.0 - fr;
      F.fc[lb - 1][0] = 0.5 * fr;
    }
    return F;
  }
  int C[4][3];
  for (int k = 0; k < 4; ++k) {
    C[k][0] = J[0];
    C[k][1] = J[1];
    C[k][2] = J[2];
  }
  C[1][t[0]] += 1;
  C[2][t[0]] += 1;
  C[2][t[1]] += 1;
  C[3][t[1]] += 1;
  const double cu[4] = {-0.5, 0.5, 0.5, -0.5}, cv[4] = {-0.5, -0.5, 0.5, 0.5};
  int L[4], cutk[4], ncut = 0;
  double pu[4] = {0, 0, 0, 0}, pv[4] = {0, 0, 0, 0};
  for (int k = 0; k < 4; ++k) L[k] = lab[node_index(g, C[k])];
  for (int k = 0; k < 4; ++k) {
    int k1 = (k + 1) & 3;
    cutk[k] = L[k] != L[k1];
    if (!cutk[k]) continue;
    ++ncut;
    if (k == 0) { pu[0] = edge_crossing(c, g, lab, C[0], t[0]) - 0.5; pv[0] = -0.5; }
    if (k == 1) { pu[1] = 0.5; pv[1] = edge_crossing(c, g, lab, C[1], t[1]) - 0.5; }
    if (k == 2) { pu[2] = edge_crossing(c, g, lab, C[3], t[0]) - 0.5; pv[2] = 0.5; }
    if (k == 3) { pu[3] = -0.5; pv[3] = edge_crossing(c, g, lab, C[0], t[1]) - 0.5; }
  }
  if (ncut == 0) {
    if (L[0] != LAB_E) F.al[L[0] - 1] = 1.0;
    return F;
  }
  if (ncut != 2) {
    F.status = ST_UNSUPPORTED;
    return F;
  }
  for (int p = 0; p < 2; ++p) {
    int lp = p + 1;
    bool has = false;
    for (int k = 0; k < 4; ++k) has = has || (L[k] == lp);
    if (!has) continue;
    double u[8], v[8];
    int m = 0;
    for (int k = 0; k < 4; ++k) {
      if (L[k] == lp) { u[m] = cu[k]; v[m] = cv[k]; ++m; }
      if (cutk[k]) { u[m] = pu[k]; v[m] = pv[k]; ++m; }
    }
    double A = 0.0, Su = 0.0, Sv = 0.0;
    for (int k = 0; k < m; ++k) {
      int k1 = (k + 1) % m;
      double cr = u[k] * v[k1] - u[k1] * v[k];
      A = A + cr;
      Su = Su + (u[k] + u[k1]) * cr;
      Sv = Sv + (v[k] + v[k1]) * cr;
    }
    A = 0.5 * A;
    F.al[p] = A;
    if (A > 0.0) {
      F.fc[p][0] = Su / (6.0 * A);
      F.fc[p][1] = Sv / (6.0 * A);
    }
  }
  return F;
}

// ------------------------------------------------------------------ cells

// Local coordinates (units of h, cell-centre origin) of the crossing on the
// cell edge along axis a starting at corner offset o (o[a] = 0).
EBP_HDN void edge_point_local(const Csg& c, const Grid& g, const uint8_t* lab, const int I[3], int a, const int o[3],
                             double P[3]) {
  int N[3] = {I[0] + o[0], I[1] + o[1], I[2] + o[2]};
  double fr = edge_crossing(c, g, lab, N, a);
  P[0] = P[1] = P[2] = 0.0;
  for (int k = 0; k < g.D; ++k) P[k] = (k == a) ? fr - 0.5 : (o[k] ? 0.5 : -0.5);
}

// EB centroid in local coordinates.  2D: midpoint of the two crossings.  3D:
// the crossings ordered into one loop through the cell faces, area centroid
// of the fan of triangles about the vertex mean of the loop.
EBP_HDN int eb_centroid_local(const Csg& c, const Grid& g, const uint8_t* lab, const int I[3], double u[3]) {
  u[0] = u[1] = u[2] = 0.0;
  if (g.D == 2) {
    double P[2][3];
    int m = 0;
    for (int a = 0; a < 2; ++a) {
      int b = 1 - a;
      for (int s = 0; s < 2; ++s) {
        int o[3] = {0, 0, 0};
        o[b] = s;
        int N0[3] = {I[0] + o[0], I[1] + o[1], 0}, N1[3] = {N0[0], N0[1], 0};
        N1[a] += 1;
        if (lab[node_index(g, N0)] == lab[node_index(g, N1)]) continue;
        if (m >= 2) return ST_UNSUPPORTED;
        edge_point_local(c, g, lab, I, a, o, P[m]);
        ++m;
      }
    }
    if (m != 2) return ST_UNSUPPORTED;
    for (int k = 0; k < 2; ++k) u[k] = 0.5 * (P[0][k] + P[1][k]);
    return 0;
  }
  double P[12][3];
  int cutE[12], eax[12], eo[12][3], ncut = 0;
  for (int a = 0; a < 3; ++a) {
    int t[2];
    transverse_axes(3, a, t);
    for (int k = 0; k < 4; ++k) {
      int e = 4 * a + k;
      int o[3] = {0, 0, 0};
      o[t[0]] = k & 1;
      o[t[1]] = (k >> 1) & 1;
      int N0[3] = {I[0] + o[0], I[1] + o[1], I[2] + o[2]}, N1[3] = {N0[0], N0[1], N0[2]};
      N1[a] += 1;
      eax[e] = a;
      eo[e][0] = o[0];
      eo[e][1] = o[1];
      eo[e][2] = o[2];
      cutE[e] = lab[node_index(g, N0)] != lab[node_index(g, N1)];
      if (cutE[e]) {
        edge_point_local(c, g, lab, I, a, o, P[e]);
        ++ncut;
      }
    }
  }
  if (ncut < 3) return ST_UNSUPPORTED;
  int nb[12][2], nnb[12];
  for (int e = 0; e < 12; ++e) nnb[e] = 0;
  for (int fa = 0; fa < 3; ++fa)
    for (int s = 0; s < 2; ++s) {
      int on[4], m = 0;
      for (int e = 0; e < 12; ++e) {
        if (!cutE[e] || eax[e] == fa) continue;
        if (eo[e][fa] != s) continue;
        if (m < 4) on[m] = e;
        ++m;
      }
      if (m == 0) continue;
      if (m != 2) return ST_UNSUPPORTED;
      for (int q = 0; q < 2; ++q) {
        int e = on[q], o2 = on[1 - q];
        if (nnb[e] >= 2) return ST_UNSUPPORTED;
        nb[e][nnb[e]++] = o2;
      }
    }
  int start = -1;
  for (int e = 0; e < 12; ++e)
    if (cutE[e]) { start = e; break; }
  for (int e = 0; e < 12; ++e)
    if (cutE[e] && nnb[e] != 2) return ST_UNSUPPORTED;
  int loop[13], len = 0, prev = -1, cur = start;
  int first_next = nb[start][0] < nb[start][1] ? nb[start][0] : nb[start][1];
  while (true) {
    loop[len++] = cur;
    int nx = (prev < 0) ? first_next : ((nb[cur][0] == prev) ? nb[cur][1] : nb[cur][0]);
    prev = cur;
    cur = nx;
    if (cur == start || len > 12) break;
  }
  if (len != ncut) return ST_UNSUPPORTED;
  // area centroid of the fan of triangles about the loop's vertex mean: for a
  // planar (convex) loop the polygon's centroid; for a curved boundary it does
  // not depend on where the loop starts or which way it runs
  double vm[3];
  for (int q = 0; q < 3; ++q) {
    double t = 0.0;
    for (int k = 0; k < len; ++k) t = t + P[loop[k]][q];
    vm[q] = t / (double)len;
  }
  double W = 0.0, S[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < len; ++k) {
    const double* v1 = P[loop[k]];
    const double* v2 = P[loop[(k + 1) % len]];
    double e1[3], e2[3], cr[3];
    for (int q = 0; q < 3; ++q) {
      e1[q] = v1[q] - vm[q];
      e2[q] = v2[q] - vm[q];
    }
    cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double ar = 0.5 * sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    W = W + ar;
    for (int q = 0; q < 3; ++q) S[q] = S[q] + ar * ((vm[q] + v1[q] + v2[q]) / 3.0);
  }
  if (W > 0.0) {
    for (int q = 0; q < 3; ++q) u[q] = S[q] / W;
  } else {  // all crossings on one line or point: their mean
    for (int q = 0; q < 3; ++q) u[q] = vm[q];
  }
  return 0;
}

// Geometry of one cut cell of the finest level, written to record q.
// Volume fractions by the divergence theorem with the cell centre as origin:
// kappa = (1/D) [ 1/2 sum_faces alpha_f + alpha_EB (u_B . n_EB) ].
EBP_HDN int cut_cell_geometry(const Csg& c, const Grid& g, const uint8_t* lab, long long cell, const CutRecords& R,
                             long long q) {
  int I[3];
  cell_ijk(g, cell, I);
  const long long nq = R.ncut;
  bool has[3] = {false, false, false};
  int ncorner = 1 << g.D;
  for (int k = 0; k < ncorner; ++k) {
    int N[3] = {I[0] + (k & 1), I[1] + ((k >> 1) & 1), I[2] + ((k >> 2) & 1)};
    has[lab[node_index(g, N)]] = true;
  }
  for (int p = 0; p < 2; ++p) R.kappa[p * nq + q] = 0.0;
  R.eba[q] = 0.0;
  for (int k = 0; k < 3; ++k) {
    R.ebn[k * nq + q] = 0.0;
    R.ebx[k * nq + q] = 0.0;
  }
  R.phiE[q] = 0.0;
  R.ebk[q] = EBK_NONE;
  if (has[LAB_E] && has[LAB_G] && has[LAB_D]) return ST_UNSUPPORTED;
  uint8_t kind = has[LAB_E] ? EBK_ELEC : EBK_IFACE;
  R.ebk[q] = kind;
  // faces
  double al[6][2];
  for (int a = 0; a < g.D; ++a)
    for (int s = 0; s < 2; ++s) {
      int J[3] = {I[0], I[1], I[2]};
      J[a] += s;
      FaceGeom F = face_geometry(c, g, lab, a, J);
      if (F.status) return F.status;
      int f = 2 * a + s;
      for (int p = 0; p < 2; ++p) {
        al[f][p] = F.al[p];
        R.alpha[rec_alpha_index(nq, f, p, q)] = F.al[p];
        R.fcen[rec_fcen_index(nq, f, p, 0, q)] = F.fc[p][0];
        R.fcen[rec_fcen_index(nq, f, p, 1, q)] = F.fc[p][1];
      }
    }
  int p0 = (kind == EBK_ELEC && has[LAB_D]) ? 1 : 0;
  double vec[3] = {0.0, 0.0, 0.0}, len2 = 0.0;
  for (int a = 0; a < g.D; ++a) {
    vec[a] = -(al[2 * a + 1][p0] - al[2 * a][p0]);
    len2 = len2 + vec[a] * vec[a];
  }
  double ar = sqrt(len2);
  double u[3];
  int st = eb_centroid_local(c, g, lab, I, u);
  if (st) return st;
  if (!(ar > 0.0)) {  // the boundary runs through a node only: a cut cell without an EB
    kind = EBK_NONE;
    R.ebk[q] = kind;
    ar = 0.0;
  }
  R.eba[q] = ar;
  double n[3];
  for (int k = 0; k < 3; ++k) {
    n[k] = ar > 0.0 ? vec[k] / ar : 0.0;
    R.ebn[k * nq + q] = n[k];
    R.ebx[k * nq + q] = (k < g.D) ? cell_x(g, k, I[k]) + g.h * u[k] : 0.0;
  }
  for (int p = 0; p < 2; ++p) {
    if (!has[p + 1]) continue;
    double sgn = (kind == EBK_IFACE && p == 1) ? -1.0 : 1.0;
    double sf = 0.0, un = 0.0;
    for (int a = 0; a < g.D; ++a) {
      sf = sf + al[2 * a][p];
      sf = sf + al[2 * a + 1][p];
    }
    for (int a = 0; a < g.D; ++a) un = un + u[a] * (sgn * n[a]);
    R.kappa[p * nq + q] = (0.5 * sf + ar * un) / (double)g.D;
  }
  // electrode potential: the electrode whose function is smallest at x_B
  if (kind == EBK_ELEC && c.n_elec > 0) {
    double xb[3] = {R.ebx[q], R.ebx[nq + q], R.ebx[2 * nq + q]};
    int best = 0;
    double bv = csg_eval(c, c.elec_node[0], xb);
    for (int e = 1; e < c.n_elec; ++e) {
      double v = csg_eval(c, c.elec_node[e], xb);
      if (v < bv) {
        bv = v;
        best = e;
      }
    }
    R.phiE[q] = c.elec_phi[best];
  }
  return 0;
}

// Does the phase-p fragment of cut record q have an open interior face or an
// open Dirichlet wall face?
EBP_HD bool record_open_face(const Grid& g, const CutRecords& R, long long q, const int I[3], int p) {
  for (int a = 0; a < g.D; ++a)
    for (int s = 0; s < 2; ++s) {
      if (!(R.alpha[rec_alpha_index(R.ncut, 2 * a + s, p, q)] > 0.0)) continue;
      bool wall = s ? (I[a] == g.n[a] - 1) : (I[a] == 0);
      if (!wall) return true;
      if (g.bc[2 * a + s]) return true;
    }
  return false;
}

}  // namespace ebp

/*
 * eb_oracle.c -- plain, slow, FP64 CPU oracle for the embedded-boundary (EB)
 * multi-material Poisson discretisation of Marskar, arXiv:1809.03745.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this code.  It
 * shares no code, header or table with the CUDA library: it is a separate
 * restatement of the same discretisation so that the two can be compared.
 *
 * What it computes (paper section in brackets):
 *   - node labels from two implicit functions s_E (electrode) and s_D
 *     (dielectric), each a CSG tree of primitives  [Sec. 3.1, Sec. 3.2]
 *   - edge crossings, face apertures and face centroids, EB area, normal and
 *     centroid, volume fractions by the divergence theorem  [Sec. 3.1]
 *   - the finite-volume operator of the integral form of Eq. (poisson) with
 *     centroid-interpolated face fluxes, second-order one-sided domain
 *     Dirichlet fluxes, ray-cast EB normal-derivative stencils with first-order
 *     and least-squares fallbacks, and the multifluid matching condition
 *     Eq. (matching) with the boundary state eliminated  [Sec. 3.3, 3.3.1]
 *   - the Helmholtz generalisation alpha a phi - div(eps grad phi) = rho with
 *     a constant shift lam = alpha a per phase, entering each cell's balance
 *     as kappa lam phi  [Sec. 3.3, Eq. helmholtz, with beta b = -eps]
 *   - Robin conditions a1 phi + a2 dphi/dn = a3 (n out of the fluid) on
 *     domain walls and on electrode boundaries, imposed by extrapolating phi
 *     to the boundary with the same one-sided wall formula or ray-cast EB
 *     stencil the Dirichlet condition uses and eliminating the boundary value
 *     [Sec. 3.3.1, Eq. robin; the outflow condition of Eq. (RTE robin)]
 *   - the cell-centred field E = -grad(phi)  [Sec. 2.1]
 * The linear system is handed back as COO triplets; the caller solves it with
 * a library sparse direct solver.
 *
 * Every part is pinned by the tests' closed forms, exactness, conservation
 * and symmetry checks; the least-squares fallback of the EB normal-derivative
 * stencil by linear exactness at the apex of acute fluid wedges, where
 * neither ray stencil finds its cells; the Helmholtz shift and the Robin
 * conditions by quadratic exactness (Robin walls; a Robin electrode on grid
 * faces), their reduction to the Dirichlet and Neumann branches, and
 * second-order convergence on a curved Robin electrode.
 *
 * Everything is written dimension-generic over D = 2 or 3, one cell or face
 * at a time, with no blocking or fusion.  Compile with -ffp-contract=off so
 * that a*b+c is never fused: the geometry is meant to be reproducible to the
 * last bit on any host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Planted mistakes, for the tests that show each pin catches one: a separate
 * build with -DOR_PLANT=k (the oracle itself is built with 0, no plant).
 *   1  the first-order Dirichlet wall flux even where the second-order one applies
 *   2  face-centre fluxes instead of their interpolation to the face centroid
 *   3  right-hand side s instead of kappa s in cut cells
 *   4  the two permittivities swapped in the boundary-state elimination
 *   5  the first-order EB stencil divided by h instead of the ray length
 *   6  the least-squares EB stencil with the boundary weight's sign dropped
 *   7  the least-squares fit taken about the cell centre instead of the EB centroid
 *   8  no unknown on a fragment of zero volume (treated as covered)
 *   9  the Robin wall elimination with a2 entering with the wrong sign
 *  10  the Helmholtz shift without the volume fraction (lam instead of kappa lam)
 *  11  the Robin EB elimination with the inward derivative taken as outward */
#ifndef OR_PLANT
#define OR_PLANT 0
#endif

/* ---------------------------------------------------------------- inputs */

enum { PR_SPHERE = 0, PR_CAPSULE = 1, PR_HALFSPACE = 2, PR_SINE = 3, PR_CYLINDER = 4, PR_BOX = 5 };
enum { CSG_PRIM = 0, CSG_UNION = 1, CSG_INTERSECT = 2, CSG_NEGATE = 3 };
enum { LAB_E = 0, LAB_G = 1, LAB_D = 2 };         /* electrode (solid), gas, dielectric */
enum { EB_NONE = 0, EB_ELECTRODE = 1, EB_INTERFACE = 2 };
enum { OR_OK = 0, OR_INVALID = 1, OR_UNSUPPORTED = 6 };

#define NPAR 10
#define MAXT 512

typedef struct {
  int dim;
  int n[3];
  double lo[3];
  double h;
  int n_prims;
  const int* prim_kind;
  const double* prim_par; /* NPAR per primitive */
  int n_nodes;
  const int* node_op;
  const int* node_a;
  const int* node_b;
  int root_E; /* -1: no electrode */
  int root_D; /* -1: no dielectric */
  double eps[2]; /* relative permittivity of gas (phase 0) and dielectric (phase 1) */
  int bc[6];     /* per domain side 2*d+hi: 0 homogeneous Neumann, 1 Dirichlet, 2 Robin */
  double robin[6][2]; /* Robin sides: a1, a2 of a1 phi + a2 dphi/dn_out = a3 (a3: the wall data) */
  int eb_robin;       /* 1: electrode boundaries carry a Robin condition instead of Dirichlet */
  double eb_robin_a[2]; /* its a1, a2 (a3: the electrode data, per cell) */
  double lam[2];      /* Helmholtz shift per phase: kappa lam phi joins each cell's balance */
} or_desc;

/* one EB normal-derivative stencil: dphi/dn_in = w0*phi_B + sum w[k]*phi[cell[k]] */
typedef struct {
  int order; /* 2, 1 (first-order ray), 3 = least squares, 0 = none */
  int n;
  double w0;
  int cell[125];
  double w[125];
} or_stencil;

typedef struct {
  or_desc d;
  int D;
  long ncell, nnode, nface[3];
  long nn[3];   /* nodes per direction */
  long nf[3][3]; /* face-array extents per direction */
  uint8_t* lab; /* [nnode] */
  double* cross[3]; /* [nnode], fraction along edge from node I in direction a; NAN when uncut */
  double* alpha[3][2]; /* [face] aperture per phase */
  double* fcen[3][2];  /* [face][2] centroid offsets along the transverse axes, units of h */
  uint8_t* cut;     /* [cell] 1 when the corner labels are not all equal */
  uint8_t* ebkind;  /* [cell] */
  double* kappa[2]; /* [cell] */
  double* eba;      /* [cell] EB area fraction */
  double* ebn;      /* [cell][3] unit normal out of the gas fragment (electrode: out of the fluid) */
  double* ebx;      /* [cell][3] EB centroid, physical */
  long* dof[2];     /* [cell] */
  long ndof;
  or_stencil* st[2]; /* [cell] stencils for EB cells */
  long counts[4];    /* stencils of order none / 2 / 1 / LS */
  long n_eb;         /* EB cells with at least one dof */
  int status;
  long bad_cell;
} or_geom;

/* ------------------------------------------------------- implicit functions */

static double prim_eval(const or_desc* d, int p, const double x[3])
{
  const double* q = d->prim_par + NPAR * p;
  switch (d->prim_kind[p]) {
  case PR_SPHERE: {
    /* distance to centre q[0..2] minus radius q[3] */
    double dx = x[0] - q[0], dy = x[1] - q[1], dz = x[2] - q[2];
    return sqrt(dx * dx + dy * dy + dz * dz) - q[3];
  }
  case PR_CAPSULE: {
    /* distance to the segment q[0..2] -> q[3..5] minus radius q[6] */
    double ab[3], ap[3], t, c[3], dd = 0.0, num = 0.0, den = 0.0;
    for (int k = 0; k < 3; ++k) { ab[k] = q[3 + k] - q[k]; ap[k] = x[k] - q[k]; }
    num = ap[0] * ab[0] + ap[1] * ab[1] + ap[2] * ab[2];
    den = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
    t = num / den;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    for (int k = 0; k < 3; ++k) { c[k] = x[k] - (q[k] + t * ab[k]); }
    dd = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    return sqrt(dd) - q[6];
  }
  case PR_HALFSPACE:
    /* q[0..2].x - q[3]: negative on the side the normal points away from */
    return q[0] * x[0] + q[1] * x[1] + q[2] * x[2] - q[3];
  case PR_SINE: {
    /* x[up] - (c + A sin(2 pi k x[t] + ph)); up = q[0], c = q[1], A = q[2], k = q[3], ph = q[4], t = q[5] */
    int up = (int)q[0], ta = (int)q[5];
    double arg = 6.283185307179586 * q[3] * x[ta] + q[4];
    return x[up] - (q[1] + q[2] * sin(arg));
  }
  case PR_CYLINDER: {
    /* axis q[0]; point on axis q[1..3]; radius q[4]; extent [q[5], q[6]] along the axis */
    int a = (int)q[0];
    double r2 = 0.0, rad, e1, e2, m;
    for (int k = 0; k < 3; ++k) {
      if (k == a) continue;
      double dk = x[k] - q[1 + k];
      r2 = r2 + dk * dk;
    }
    rad = sqrt(r2) - q[4];
    e1 = q[5] - x[a];
    e2 = x[a] - q[6];
    m = rad;
    if (e1 > m) m = e1;
    if (e2 > m) m = e2;
    return m;
  }
  case PR_BOX: {
    /* q[0..2] lo, q[3..5] hi: max over axes of the two slab functions */
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

static double csg_eval(const or_desc* d, int node, const double x[3])
{
  int op = d->node_op[node];
  if (op == CSG_PRIM) return prim_eval(d, d->node_a[node], x);
  if (op == CSG_NEGATE) return -csg_eval(d, d->node_a[node], x);
  double a = csg_eval(d, d->node_a[node], x);
  double b = csg_eval(d, d->node_b[node], x);
  if (op == CSG_UNION) return a < b ? a : b;
  return a > b ? a : b; /* intersection */
}

/* ---------------------------------------------------------------- indexing */

static long cell_id(const or_geom* g, const long I[3]) { return I[0] + g->d.n[0] * (I[1] + (long)g->d.n[1] * I[2]); }
static long node_id(const or_geom* g, const long I[3]) { return I[0] + g->nn[0] * (I[1] + g->nn[1] * I[2]); }
static long face_id(const or_geom* g, int a, const long I[3])
{
  return I[0] + g->nf[a][0] * (I[1] + g->nf[a][1] * I[2]);
}
static void cell_ijk(const or_geom* g, long c, long I[3])
{
  I[0] = c % g->d.n[0];
  I[1] = (c / g->d.n[0]) % g->d.n[1];
  I[2] = c / ((long)g->d.n[0] * g->d.n[1]);
}
static int in_domain(const or_geom* g, const long I[3])
{
  for (int k = 0; k < g->D; ++k)
    if (I[k] < 0 || I[k] >= g->d.n[k]) return 0;
  return 1;
}
static double node_x(const or_geom* g, int k, long i) { return g->d.lo[k] + (double)i * g->d.h; }
static double cell_x(const or_geom* g, int k, long i) { return g->d.lo[k] + ((double)i + 0.5) * g->d.h; }

/* transverse axes of direction a, in increasing order */
static void transverse(int D, int a, int t[2])
{
  int m = 0;
  for (int k = 0; k < D; ++k)
    if (k != a) t[m++] = k;
  if (D == 2) t[1] = -1;
}

/* ------------------------------------------------------- geometry: labels */

static int label_at(const or_desc* d, const double x[3])
{
  if (d->root_E >= 0 && csg_eval(d, d->root_E, x) < 0.0) return LAB_E;
  if (d->root_D >= 0 && csg_eval(d, d->root_D, x) < 0.0) return LAB_D;
  return LAB_G;
}

/* Edge crossing by bisection on the implicit function that separates the two
 * end labels: exactly 60 halvings, the midpoint of the final bracket.  Returned
 * as the fraction of h from the lower node. */
static double edge_crossing(const or_geom* g, const long I[3], int a, int la)
{
  const or_desc* d = &g->d;
  int lb;
  long J[3] = {I[0], I[1], I[2]};
  J[a] += 1;
  lb = g->lab[node_id(g, J)];
  int root = (la == LAB_E || lb == LAB_E) ? d->root_E : d->root_D;
  int inside_lab = (la == LAB_E || lb == LAB_E) ? LAB_E : LAB_D;
  int in_a = (la == inside_lab);
  double x[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < g->D; ++k) x[k] = node_x(g, k, I[k]);
  double lo = node_x(g, a, I[a]), hi = node_x(g, a, I[a] + 1);
  for (int it = 0; it < 60; ++it) {
    double m = 0.5 * (lo + hi);
    x[a] = m;
    int in = csg_eval(d, root, x) < 0.0;
    if (in == in_a) lo = m;
    else hi = m;
  }
  double c = 0.5 * (lo + hi);
  double fr = (c - node_x(g, a, I[a])) / d->h;
  /* a crossing within 1e-8 h of a node is put on the node: the boundary moves
   * by less than 1e-8 h, and fragments of vanishing size become exactly empty */
  if (fr < 1e-8) fr = 0.0;
  if (fr > 1.0 - 1e-8) fr = 1.0;
  return fr;
}

/* ---------------------------------------------------- geometry: one face */

/* Face (a, I): the cell face normal to a whose lowest corner is node I.  In 2D
 * it is an edge along the transverse axis; in 3D a square whose fluid part per
 * phase is the polygon through its same-label corners and edge crossings
 * (marching squares without saddles). */
static int face_geometry(or_geom* g, int a, const long I[3])
{
  int D = g->D, t[2];
  long f = face_id(g, a, I);
  transverse(D, a, t);
  for (int p = 0; p < 2; ++p) {
    g->alpha[a][p][f] = 0.0;
    g->fcen[a][p][2 * f] = 0.0;
    g->fcen[a][p][2 * f + 1] = 0.0;
  }
  if (D == 2) {
    long J[3] = {I[0], I[1], I[2]};
    J[t[0]] += 1;
    int la = g->lab[node_id(g, I)], lb = g->lab[node_id(g, J)];
    if (la == lb) {
      if (la != LAB_E) g->alpha[a][la - 1][f] = 1.0;
      return OR_OK;
    }
    double fr = g->cross[t[0]][node_id(g, I)];
    if (la != LAB_E) {
      g->alpha[a][la - 1][f] = fr;
      g->fcen[a][la - 1][2 * f] = 0.5 * fr - 0.5;
    }
    if (lb != LAB_E) {
      g->alpha[a][lb - 1][f] = 1.0 - fr;
      g->fcen[a][lb - 1][2 * f] = 0.5 * fr;
    }
    return OR_OK;
  }
  /* 3D: corners in counter-clockwise order in the (t0, t1) plane */
  long C[4][3];
  for (int k = 0; k < 4; ++k) { C[k][0] = I[0]; C[k][1] = I[1]; C[k][2] = I[2]; }
  C[1][t[0]] += 1;
  C[2][t[0]] += 1; C[2][t[1]] += 1;
  C[3][t[1]] += 1;
  static const double cu[4] = {-0.5, 0.5, 0.5, -0.5}, cv[4] = {-0.5, -0.5, 0.5, 0.5};
  int lab[4], ncut = 0;
  double pu[4], pv[4];
  int cutk[4];
  for (int k = 0; k < 4; ++k) lab[k] = g->lab[node_id(g, C[k])];
  /* crossing on the edge from corner k to corner k+1 */
  for (int k = 0; k < 4; ++k) {
    int k1 = (k + 1) & 3;
    cutk[k] = lab[k] != lab[k1];
    if (!cutk[k]) continue;
    ++ncut;
    if (k == 0) { pu[k] = g->cross[t[0]][node_id(g, C[0])] - 0.5; pv[k] = -0.5; }
    if (k == 1) { pu[k] = 0.5; pv[k] = g->cross[t[1]][node_id(g, C[1])] - 0.5; }
    if (k == 2) { pu[k] = g->cross[t[0]][node_id(g, C[3])] - 0.5; pv[k] = 0.5; }
    if (k == 3) { pu[k] = -0.5; pv[k] = g->cross[t[1]][node_id(g, C[0])] - 0.5; }
  }
  if (ncut == 0) {
    if (lab[0] != LAB_E) g->alpha[a][lab[0] - 1][f] = 1.0;
    return OR_OK;
  }
  if (ncut != 2) return OR_UNSUPPORTED; /* saddle or three labels on one face */
  for (int p = 0; p < 2; ++p) {
    int L = p + 1;
    double u[8], v[8];
    int m = 0;
    for (int k = 0; k < 4; ++k) {
      if (lab[k] == L) { u[m] = cu[k]; v[m] = cv[k]; ++m; }
      if (cutk[k]) { u[m] = pu[k]; v[m] = pv[k]; ++m; }
    }
    int has = 0;
    for (int k = 0; k < 4; ++k) has |= lab[k] == L;
    if (!has) continue;
    double A = 0.0, Su = 0.0, Sv = 0.0;
    for (int k = 0; k < m; ++k) {
      int k1 = (k + 1) % m;
      double cr = u[k] * v[k1] - u[k1] * v[k];
      A = A + cr;
      Su = Su + (u[k] + u[k1]) * cr;
      Sv = Sv + (v[k] + v[k1]) * cr;
    }
    A = 0.5 * A;
    g->alpha[a][p][f] = A;
    if (A > 0.0) {
      g->fcen[a][p][2 * f] = Su / (6.0 * A);
      g->fcen[a][p][2 * f + 1] = Sv / (6.0 * A);
    }
  }
  return OR_OK;
}

/* ----------------------------------------------------- geometry: one cell */

/* local coordinates (units of h, origin at the cell centre) of the crossing
 * on cell edge along axis a whose lowest node is the cell's corner with
 * offsets o[] (o[a] = 0). */
static void edge_point(const or_geom* g, const long I[3], int a, const int o[3], double P[3])
{
  long N[3] = {I[0] + o[0], I[1] + o[1], I[2] + o[2]};
  double fr = g->cross[a][node_id(g, N)];
  for (int k = 0; k < 3; ++k) P[k] = 0.0;
  for (int k = 0; k < g->D; ++k) P[k] = (k == a) ? fr - 0.5 : (o[k] ? 0.5 : -0.5);
}

static int eb_centroid(or_geom* g, const long I[3], double u[3])
{
  int D = g->D;
  if (D == 2) {
    double P[4][3];
    int m = 0;
    for (int a = 0; a < 2; ++a) {
      int b = 1 - a;
      for (int s = 0; s < 2; ++s) {
        int o[3] = {0, 0, 0};
        o[b] = s;
        long N0[3] = {I[0] + o[0], I[1] + o[1], 0}, N1[3] = {N0[0], N0[1], 0};
        N1[a] += 1;
        if (g->lab[node_id(g, N0)] == g->lab[node_id(g, N1)]) continue;
        if (m >= 2) return OR_UNSUPPORTED;
        edge_point(g, I, a, o, P[m]);
        ++m;
      }
    }
    if (m != 2) return OR_UNSUPPORTED;
    for (int k = 0; k < 3; ++k) u[k] = 0.5 * (P[0][k] + P[1][k]);
    u[2] = 0.0;
    return OR_OK;
  }
  /* 3D: the 12 edges, axis-major, then corner offsets (o_t0, o_t1) = 00,10,01,11 */
  double P[12][3];
  int cutE[12], eax[12], eo[12][3];
  int ncut = 0;
  for (int a = 0; a < 3; ++a) {
    int t[2];
    transverse(3, a, t);
    for (int k = 0; k < 4; ++k) {
      int e = 4 * a + k;
      int o[3] = {0, 0, 0};
      o[t[0]] = k & 1;
      o[t[1]] = (k >> 1) & 1;
      long N0[3] = {I[0] + o[0], I[1] + o[1], I[2] + o[2]}, N1[3] = {N0[0], N0[1], N0[2]};
      N1[a] += 1;
      eax[e] = a;
      eo[e][0] = o[0]; eo[e][1] = o[1]; eo[e][2] = o[2];
      cutE[e] = g->lab[node_id(g, N0)] != g->lab[node_id(g, N1)];
      if (cutE[e]) { edge_point(g, I, a, o, P[e]); ++ncut; }
    }
  }
  if (ncut < 3) return OR_UNSUPPORTED;
  /* two cut edges are neighbours on the loop when they lie on a common face
   * of the cell; every face carries zero or two crossings (no saddles). */
  int nb[12][2], nnb[12];
  for (int e = 0; e < 12; ++e) nnb[e] = 0;
  for (int fa = 0; fa < 3; ++fa) {
    for (int s = 0; s < 2; ++s) {
      int on[4], m = 0;
      for (int e = 0; e < 12; ++e) {
        if (!cutE[e] || eax[e] == fa) continue;
        if (eo[e][fa] != s) continue;
        if (m < 4) on[m] = e;
        ++m;
      }
      if (m == 0) continue;
      if (m != 2) return OR_UNSUPPORTED;
      for (int q = 0; q < 2; ++q) {
        int e = on[q], o2 = on[1 - q];
        if (nnb[e] >= 2) return OR_UNSUPPORTED;
        nb[e][nnb[e]++] = o2;
      }
    }
  }
  int loop[12], len = 0, start = -1;
  for (int e = 0; e < 12; ++e)
    if (cutE[e]) { start = e; break; }
  for (int e = 0; e < 12; ++e)
    if (cutE[e] && nnb[e] != 2) return OR_UNSUPPORTED;
  int prev = -1, cur = start;
  int first_next = nb[start][0] < nb[start][1] ? nb[start][0] : nb[start][1];
  while (1) {
    loop[len++] = cur;
    int nx;
    if (prev < 0) nx = first_next;
    else nx = (nb[cur][0] == prev) ? nb[cur][1] : nb[cur][0];
    prev = cur;
    cur = nx;
    if (cur == start || len > 12) break;
  }
  if (len != ncut) return OR_UNSUPPORTED; /* more than one loop */
  /* area centroid of the fan of triangles about the loop's vertex mean: for a
   * planar (convex) loop the polygon's centroid; for a curved boundary it does
   * not depend on where the loop starts or which way it runs */
  double c[3];
  for (int q = 0; q < 3; ++q) {
    double t = 0.0;
    for (int k = 0; k < len; ++k) t = t + P[loop[k]][q];
    c[q] = t / (double)len;
  }
  double W = 0.0, S[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < len; ++k) {
    const double* v1 = P[loop[k]];
    const double* v2 = P[loop[(k + 1) % len]];
    double e1[3], e2[3], cr[3];
    for (int q = 0; q < 3; ++q) {
      e1[q] = v1[q] - c[q];
      e2[q] = v2[q] - c[q];
    }
    cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double ar = 0.5 * sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    W = W + ar;
    for (int q = 0; q < 3; ++q) S[q] = S[q] + ar * ((c[q] + v1[q] + v2[q]) / 3.0);
  }
  if (W > 0.0) {
    for (int q = 0; q < 3; ++q) u[q] = S[q] / W;
  } else { /* all crossings on one line or point: their mean */
    for (int q = 0; q < 3; ++q) u[q] = c[q];
  }
  return OR_OK;
}

/* aperture of the lo (s=0) or hi (s=1) face of cell I in direction a, phase p */
static double cell_face_alpha(const or_geom* g, const long I[3], int a, int s, int p)
{
  long J[3] = {I[0], I[1], I[2]};
  J[a] += s;
  return g->alpha[a][p][face_id(g, a, J)];
}

static int cell_geometry(or_geom* g, long c)
{
  int D = g->D;
  long I[3];
  cell_ijk(g, c, I);
  int has[3] = {0, 0, 0}, nc = 1 << D;
  for (int k = 0; k < nc; ++k) {
    long N[3] = {I[0] + (k & 1), I[1] + ((k >> 1) & 1), I[2] + ((k >> 2) & 1)};
    has[g->lab[node_id(g, N)]] = 1;
  }
  g->cut[c] = (has[0] + has[1] + has[2]) > 1;
  g->ebkind[c] = EB_NONE;
  g->kappa[0][c] = 0.0;
  g->kappa[1][c] = 0.0;
  g->eba[c] = 0.0;
  for (int k = 0; k < 3; ++k) { g->ebn[3 * c + k] = 0.0; g->ebx[3 * c + k] = 0.0; }
  if (!g->cut[c]) {
    if (has[LAB_G]) g->kappa[0][c] = 1.0;
    if (has[LAB_D]) g->kappa[1][c] = 1.0;
    return OR_OK;
  }
  if (has[LAB_E] && has[LAB_G] && has[LAB_D]) return OR_UNSUPPORTED;
  g->ebkind[c] = has[LAB_E] ? EB_ELECTRODE : EB_INTERFACE;
  /* EB normal and area from the apertures of the gas fragment (interface) or
   * of the single fluid fragment (electrode): A n = -sum_d (a_hi - a_lo) e_d */
  int p0 = (g->ebkind[c] == EB_ELECTRODE && has[LAB_D]) ? 1 : 0;
  double vec[3] = {0.0, 0.0, 0.0}, len2 = 0.0;
  for (int a = 0; a < D; ++a) {
    vec[a] = -(cell_face_alpha(g, I, a, 1, p0) - cell_face_alpha(g, I, a, 0, p0));
    len2 = len2 + vec[a] * vec[a];
  }
  double ar = sqrt(len2);
  double u[3] = {0.0, 0.0, 0.0};
  int st = eb_centroid(g, I, u);
  if (st != OR_OK) return st;
  if (!(ar > 0.0)) {
    /* the boundary runs through a node only: a cut cell without an EB */
    g->ebkind[c] = EB_NONE;
    ar = 0.0;
  }
  g->eba[c] = ar;
  for (int k = 0; k < 3; ++k) {
    g->ebn[3 * c + k] = ar > 0.0 ? vec[k] / ar : 0.0;
    g->ebx[3 * c + k] = (k < D) ? cell_x(g, k, I[k]) + g->d.h * u[k] : 0.0;
  }
  /* volume fractions by the divergence theorem, cell-centre origin, units of h:
   * kappa = (1/D) [ 1/2 sum_faces alpha_f + alpha_EB (u_B . n_EB) ] */
  for (int p = 0; p < 2; ++p) {
    if (!has[p + 1]) continue;
    double sgn = (g->ebkind[c] == EB_INTERFACE && p == 1) ? -1.0 : 1.0;
    double sf = 0.0, un = 0.0;
    for (int a = 0; a < D; ++a) {
      sf = sf + cell_face_alpha(g, I, a, 0, p);
      sf = sf + cell_face_alpha(g, I, a, 1, p);
    }
    for (int a = 0; a < D; ++a) un = un + u[a] * (sgn * g->ebn[3 * c + a]);
    g->kappa[p][c] = (0.5 * sf + ar * un) / (double)D;
  }
  return OR_OK;
}

/* does fragment (c, p) have an open face that is interior or a Dirichlet wall */
static int open_face(const or_geom* g, const long I[3], int p)
{
  for (int a = 0; a < g->D; ++a)
    for (int s = 0; s < 2; ++s) {
      if (!(cell_face_alpha(g, I, a, s, p) > 0.0)) continue;
      long wall = s ? (I[a] == g->d.n[a] - 1) : (I[a] == 0);
      if (!wall) return 1;
      if (g->d.bc[2 * a + s] == 1 || g->d.bc[2 * a + s] == 2) return 1;
    }
  return 0;
}

static long dof_of(const or_geom* g, const long I[3], int p)
{
  if (!in_domain(g, I)) return -1;
  return g->dof[p][cell_id(g, I)];
}

/* ------------------------------------------------- EB normal-derivative */

/* Stencil for dphi/dn_in at the EB centroid x_B of cell I, phase p, with
 * n_in the unit normal pointing into phase p:
 *  order 2: rays to the planes of cell centres one and two cells away along
 *           the dominant axis, quadratic (tensor) interpolation transverse,
 *           one-sided 3-point derivative along the ray;
 *  order 1: the first plane only, (bi)linear interpolation;
 *  LS:      unweighted least squares of phi_B + g.(x - x_B) over the 3^D
 *           neighbourhood on the fluid side.
 * The cut cell itself never enters (Sec. 3.3.1, Eq. bndry_stencil). */
static int build_stencil(const or_geom* g, const long I[3], int p, const double xB[3], const double nin[3],
                         or_stencil* S)
{
  int D = g->D;
  double h = g->d.h;
  int a = 0;
  for (int k = 1; k < D; ++k)
    if (fabs(nin[k]) > fabs(nin[a])) a = k;
  int sg = nin[a] > 0.0 ? 1 : -1;
  int t[2];
  transverse(D, a, t);
  int nt = D - 1;
  double ell[3];
  S->order = 0;
  S->n = 0;
  /* second order */
  {
    int ok = 1, m_;
    int cells[2][9];
    double wts[2][9];
    int cnt[2] = {0, 0};
    for (m_ = 1; m_ <= 2 && ok; ++m_) {
      double P = cell_x(g, a, I[a]) + (double)(m_ * sg) * h;
      double l = (P - xB[a]) / nin[a];
      ell[m_] = l;
      long ka[2];
      double w3[2][3];
      for (int q = 0; q < nt; ++q) {
        int tt = t[q];
        double y = xB[tt] + l * nin[tt];
        long k = (long)floor((y - g->d.lo[tt]) / h);
        /* three cells centred on the cell holding y, shifted inward at a wall */
        if (k < 1) k = 1;
        if (k > g->d.n[tt] - 2) k = g->d.n[tt] - 2;
        double xi = (y - cell_x(g, tt, k)) / h;
        ka[q] = k;
        w3[q][0] = 0.5 * xi * (xi - 1.0);
        w3[q][1] = 1.0 - xi * xi;
        w3[q][2] = 0.5 * xi * (xi + 1.0);
      }
      int ny = 3, nz = (nt == 2) ? 3 : 1;
      for (int iz = 0; iz < nz && ok; ++iz)
        for (int iy = 0; iy < ny && ok; ++iy) {
          long J[3] = {I[0], I[1], I[2]};
          J[a] = I[a] + m_ * sg;
          J[t[0]] = ka[0] + iy - 1;
          double w = w3[0][iy];
          if (nt == 2) { J[t[1]] = ka[1] + iz - 1; w = w * w3[1][iz]; }
          long dd = dof_of(g, J, p);
          if (dd < 0) { ok = 0; break; }
          cells[m_ - 1][cnt[m_ - 1]] = (int)cell_id(g, J);
          wts[m_ - 1][cnt[m_ - 1]] = w;
          cnt[m_ - 1]++;
        }
    }
    if (ok) {
      double l1 = ell[1], l2 = ell[2];
      double c1 = (l2 / l1) / (l2 - l1), c2 = -(l1 / l2) / (l2 - l1);
      S->order = 2;
      S->w0 = -(c1 + c2);
      for (int k = 0; k < cnt[0]; ++k) { S->cell[S->n] = cells[0][k]; S->w[S->n] = c1 * wts[0][k]; S->n++; }
      for (int k = 0; k < cnt[1]; ++k) { S->cell[S->n] = cells[1][k]; S->w[S->n] = c2 * wts[1][k]; S->n++; }
      return OR_OK;
    }
  }
  /* first order */
  {
    double P = cell_x(g, a, I[a]) + (double)sg * h;
    double l = (P - xB[a]) / nin[a];
    long ka[2];
    double w2[2][2];
    int ok = 1, cnt = 0, nz = (nt == 2) ? 2 : 1;
    for (int q = 0; q < nt; ++q) {
      int tt = t[q];
      double y = xB[tt] + l * nin[tt];
      /* two cells bracketing y, shifted inward at a wall */
      long k = (long)floor((y - g->d.lo[tt]) / h - 0.5);
      if (k < 0) k = 0;
      if (k > g->d.n[tt] - 2) k = g->d.n[tt] - 2;
      double xi = (y - cell_x(g, tt, k)) / h;
      ka[q] = k;
      w2[q][0] = 1.0 - xi;
      w2[q][1] = xi;
    }
    int cells[4];
    double wts[4];
    for (int iz = 0; iz < nz && ok; ++iz)
      for (int iy = 0; iy < 2 && ok; ++iy) {
        long J[3] = {I[0], I[1], I[2]};
        J[a] = I[a] + sg;
        J[t[0]] = ka[0] + iy;
        double w = w2[0][iy];
        if (nt == 2) { J[t[1]] = ka[1] + iz; w = w * w2[1][iz]; }
        if (dof_of(g, J, p) < 0) { ok = 0; break; }
        cells[cnt] = (int)cell_id(g, J);
        wts[cnt] = w;
        cnt++;
      }
    if (ok) {
      if (OR_PLANT == 5) l = h;
      S->order = 1;
      S->w0 = -1.0 / l;
      for (int k = 0; k < cnt; ++k) { S->cell[S->n] = cells[k]; S->w[S->n] = wts[k] / l; S->n++; }
      return OR_OK;
    }
  }
  /* least squares over the fluid-side neighbourhood: radius 1, then 2 */
  for (int rad = 1; rad <= 2; ++rad) {
    double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double dv[125][3];
    int cells[125], cnt = 0;
    int w = 2 * rad + 1, nz = (D == 3) ? w : 1;
    for (int oz = 0; oz < nz; ++oz)
      for (int oy = 0; oy < w; ++oy)
        for (int ox = 0; ox < w; ++ox) {
          long J[3] = {I[0] + ox - rad, I[1] + oy - rad, I[2] + (D == 3 ? oz - rad : 0)};
          if (J[0] == I[0] && J[1] == I[1] && J[2] == I[2]) continue;
          if (dof_of(g, J, p) < 0) continue;
          double dx[3] = {0.0, 0.0, 0.0}, dn = 0.0;
          for (int k = 0; k < D; ++k) { dx[k] = cell_x(g, k, J[k]) - xB[k]; dn = dn + dx[k] * nin[k]; }
          if (OR_PLANT == 7)
            for (int k = 0; k < D; ++k) dx[k] = cell_x(g, k, J[k]) - cell_x(g, k, I[k]);
          if (!(dn > 0.0)) continue;
          for (int k = 0; k < 3; ++k) dv[cnt][k] = dx[k];
          cells[cnt++] = (int)cell_id(g, J);
        }
    if (cnt < D) continue;
    for (int k = 0; k < cnt; ++k)
      for (int r = 0; r < D; ++r)
        for (int s = 0; s < D; ++s) M[r][s] = M[r][s] + dv[k][r] * dv[k][s];
    /* u = M^{-1} n_in by Cramer's rule */
    double u[3] = {0.0, 0.0, 0.0};
    if (D == 2) {
      double det = M[0][0] * M[1][1] - M[0][1] * M[1][0];
      if (!(fabs(det) > 1e-12 * h * h * h * h)) continue;
      u[0] = (nin[0] * M[1][1] - M[0][1] * nin[1]) / det;
      u[1] = (M[0][0] * nin[1] - nin[0] * M[1][0]) / det;
    } else {
      double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                   M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                   M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
      if (!(fabs(det) > 1e-12 * h * h * h * h * h * h)) continue;
      for (int col = 0; col < 3; ++col) {
        double Mc[3][3];
        memcpy(Mc, M, sizeof(Mc));
        for (int r = 0; r < 3; ++r) Mc[r][col] = nin[r];
        double dc = Mc[0][0] * (Mc[1][1] * Mc[2][2] - Mc[1][2] * Mc[2][1]) -
                    Mc[0][1] * (Mc[1][0] * Mc[2][2] - Mc[1][2] * Mc[2][0]) +
                    Mc[0][2] * (Mc[1][0] * Mc[2][1] - Mc[1][1] * Mc[2][0]);
        u[col] = dc / det;
      }
    }
    S->order = 3;
    double sw = 0.0;
    for (int k = 0; k < cnt; ++k) {
      double wk = 0.0;
      for (int r = 0; r < D; ++r) wk = wk + u[r] * dv[k][r];
      S->cell[S->n] = cells[k];
      S->w[S->n] = wk;
      S->n++;
      sw = sw + wk;
    }
    S->w0 = (OR_PLANT == 6) ? sw : -sw;
    return OR_OK;
  }
  return OR_UNSUPPORTED;
}

/* ------------------------------------------------------------- build */

static void* xmalloc(size_t n)
{
  void* p = malloc(n ? n : 1);
  if (p) memset(p, 0, n ? n : 1);
  return p;
}

void or_geom_free(or_geom* g)
{
  if (!g) return;
  free(g->lab);
  for (int a = 0; a < 3; ++a) {
    free(g->cross[a]);
    for (int p = 0; p < 2; ++p) { free(g->alpha[a][p]); free(g->fcen[a][p]); }
  }
  free(g->cut);
  free(g->ebkind);
  for (int p = 0; p < 2; ++p) { free(g->kappa[p]); free(g->dof[p]); free(g->st[p]); }
  free(g->eba);
  free(g->ebn);
  free(g->ebx);
  free(g);
}

or_geom* or_geom_build(const or_desc* d, int* status)
{
  or_geom* g = (or_geom*)xmalloc(sizeof(or_geom));
  g->d = *d;
  g->status = OR_OK;
  g->bad_cell = -1;
  int D = d->dim;
  g->D = D;
  if (D != 2 && D != 3) { *status = OR_INVALID; g->status = OR_INVALID; return g; }
  if (D == 2) g->d.n[2] = 1;
  for (int k = 0; k < 3; ++k) g->nn[k] = (k < D) ? d->n[k] + 1 : 1;
  g->ncell = (long)g->d.n[0] * g->d.n[1] * g->d.n[2];
  g->nnode = g->nn[0] * g->nn[1] * g->nn[2];
  for (int a = 0; a < 3; ++a) {
    for (int k = 0; k < 3; ++k) g->nf[a][k] = (k < D) ? g->d.n[k] + (k == a ? 1 : 0) : 1;
    g->nface[a] = (a < D) ? g->nf[a][0] * g->nf[a][1] * g->nf[a][2] : 0;
  }
  g->lab = (uint8_t*)xmalloc(g->nnode);
  for (int a = 0; a < D; ++a) {
    g->cross[a] = (double*)xmalloc(sizeof(double) * g->nnode);
    for (int p = 0; p < 2; ++p) {
      g->alpha[a][p] = (double*)xmalloc(sizeof(double) * g->nface[a]);
      g->fcen[a][p] = (double*)xmalloc(sizeof(double) * 2 * g->nface[a]);
    }
  }
  g->cut = (uint8_t*)xmalloc(g->ncell);
  g->ebkind = (uint8_t*)xmalloc(g->ncell);
  g->eba = (double*)xmalloc(sizeof(double) * g->ncell);
  g->ebn = (double*)xmalloc(sizeof(double) * 3 * g->ncell);
  g->ebx = (double*)xmalloc(sizeof(double) * 3 * g->ncell);
  for (int p = 0; p < 2; ++p) {
    g->kappa[p] = (double*)xmalloc(sizeof(double) * g->ncell);
    g->dof[p] = (long*)xmalloc(sizeof(long) * g->ncell);
    g->st[p] = (or_stencil*)xmalloc(sizeof(or_stencil) * g->ncell);
  }
  /* 1. node labels */
  for (long z = 0; z < g->nn[2]; ++z)
    for (long y = 0; y < g->nn[1]; ++y)
      for (long x = 0; x < g->nn[0]; ++x) {
        long I[3] = {x, y, z};
        double X[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < D; ++k) X[k] = node_x(g, k, I[k]);
        g->lab[node_id(g, I)] = (uint8_t)label_at(d, X);
      }
  /* 2. edge crossings */
  for (int a = 0; a < D; ++a)
    for (long z = 0; z < g->nn[2]; ++z)
      for (long y = 0; y < g->nn[1]; ++y)
        for (long x = 0; x < g->nn[0]; ++x) {
          long I[3] = {x, y, z};
          long nid = node_id(g, I);
          g->cross[a][nid] = NAN;
          if (I[a] >= g->nn[a] - 1) continue;
          long J[3] = {x, y, z};
          J[a] += 1;
          int la = g->lab[nid], lb = g->lab[node_id(g, J)];
          if (la != lb) g->cross[a][nid] = edge_crossing(g, I, a, la);
        }
  /* 3. faces */
  for (int a = 0; a < D; ++a)
    for (long z = 0; z < g->nf[a][2]; ++z)
      for (long y = 0; y < g->nf[a][1]; ++y)
        for (long x = 0; x < g->nf[a][0]; ++x) {
          long I[3] = {x, y, z};
          int st = face_geometry(g, a, I);
          if (st != OR_OK) { g->status = st; *status = st; return g; }
        }
  /* 4. cells */
  for (long c = 0; c < g->ncell; ++c) {
    int st = cell_geometry(g, c);
    if (st != OR_OK) { g->status = st; g->bad_cell = c; *status = st; return g; }
  }
  /* 5. degrees of freedom: a fragment with an open face that is interior or a
   * Dirichlet wall (a fragment of zero volume with such a face carries the
   * boundary condition of its EB into the neighbouring cell) */
  g->ndof = 0;
  for (long c = 0; c < g->ncell; ++c) {
    long I[3];
    cell_ijk(g, c, I);
    for (int p = 0; p < 2; ++p) {
      g->dof[p][c] = -1;
      if (open_face(g, I, p) && !(OR_PLANT == 8 && !(g->kappa[p][c] > 0.0))) g->dof[p][c] = g->ndof++;
    }
  }
  /* 6. EB stencils */
  for (int k = 0; k < 4; ++k) g->counts[k] = 0;
  g->n_eb = 0;
  for (long c = 0; c < g->ncell; ++c) {
    if (!g->cut[c]) continue;
    if (g->dof[0][c] < 0 && g->dof[1][c] < 0) continue;
    g->n_eb++;
    /* an interface cell that keeps a single fragment (the other has no volume
     * or no open face: the interface runs through a node) carries no
     * interface flux; its EB is dropped */
    if (g->ebkind[c] == EB_INTERFACE && (g->dof[0][c] < 0 || g->dof[1][c] < 0)) g->ebkind[c] = EB_NONE;
    if (g->ebkind[c] == EB_NONE) continue;
    long I[3];
    cell_ijk(g, c, I);
    for (int p = 0; p < 2; ++p) {
      if (g->dof[p][c] < 0) continue;
      double nin[3];
      double sgn = (g->ebkind[c] == EB_INTERFACE && p == 1) ? 1.0 : -1.0;
      for (int k = 0; k < 3; ++k) nin[k] = sgn * g->ebn[3 * c + k];
      int st = build_stencil(g, I, p, g->ebx + 3 * c, nin, &g->st[p][c]);
      if (st != OR_OK) { g->status = st; g->bad_cell = c; *status = st; return g; }
      int o = g->st[p][c].order;
      g->counts[o == 2 ? 1 : (o == 1 ? 2 : 3)]++;
    }
  }
  *status = OR_OK;
  return g;
}

/* --------------------------------------------------------- linear forms */

typedef struct {
  int n;
  long idx[MAXT];
  double w[MAXT];
  double c;
} lform;

static void lf_zero(lform* f) { f->n = 0; f->c = 0.0; }
static void lf_add(lform* f, long idx, double w)
{
  for (int k = 0; k < f->n; ++k)
    if (f->idx[k] == idx) { f->w[k] = f->w[k] + w; return; }
  if (f->n < MAXT) { f->idx[f->n] = idx; f->w[f->n] = w; f->n++; }
}
static void lf_axpy(lform* y, double s, const lform* x)
{
  for (int k = 0; k < x->n; ++k) lf_add(y, x->idx[k], s * x->w[k]);
  y->c = y->c + s * x->c;
}

typedef struct {
  const double* phiE;   /* [cell] electrode potential at the EB centroid */
  const double* sigma;  /* [cell] surface charge sigma/eps0 on interface cells */
  const double* phidom; /* [2][sum of side sizes] Dirichlet value per wall face, per phase */
  const double* s;      /* [2][cell] rho/eps0 per phase, sampled at cell centres */
} or_data;

/* index of a wall face in phidom: side = 2a + hi, position = linear index of
 * the cell over the transverse axes */
static long wall_index(const or_geom* g, int a, int hi, const long I[3])
{
  long off = 0;
  for (int side = 0; side < 2 * a + hi; ++side) {
    int aa = side / 2;
    long sz = 1;
    for (int k = 0; k < g->D; ++k)
      if (k != aa) sz *= g->d.n[k];
    off += sz;
  }
  int t[2];
  transverse(g->D, a, t);
  long pos = I[t[0]];
  if (g->D == 3) pos += (long)g->d.n[t[0]] * I[t[1]];
  return off + pos;
}
static long wall_total(const or_geom* g)
{
  long tot = 0;
  for (int a = 0; a < g->D; ++a) {
    long sz = 1;
    for (int k = 0; k < g->D; ++k)
      if (k != a) sz *= g->d.n[k];
    tot += 2 * sz;
  }
  return tot;
}

/* Face-centred flux in the +e_a direction through face (a, J), phase p, as a
 * linear form in the dofs.  Interior faces: eps (phi_hi - phi_lo)/h.  Wall
 * faces with Dirichlet data phi0: the outward derivative
 * (8 phi0 - 9 phi1 + phi2)/(3h) (phi1 adjacent, phi2 next inward; Sec. 3.3.1
 * with the indices put in the order that makes it second order), or
 * 2(phi0 - phi1)/h when phi2 is unavailable.  Robin walls (a1 phi0 + a2
 * dphi/dn_out = a3, a3 the wall data): the same formula written as
 * dphi/dn_out = Aw phi0 + R (Aw = 8/(3h) or 2/h), solved with the condition
 * for the wall value phi0 = (a3 - a2 R) / (a1 + a2 Aw), so that
 * dphi/dn_out = (Aw a3 + a1 R) / (a1 + a2 Aw).  Returns 0 when the face
 * carries no flux for phase p. */
static int centred_flux(const or_geom* g, const or_data* dt, int a, const long J[3], int p, lform* F)
{
  lf_zero(F);
  for (int k = 0; k < g->D; ++k) {
    if (k == a) { if (J[k] < 0 || J[k] > g->d.n[k]) return 0; }
    else if (J[k] < 0 || J[k] >= g->d.n[k]) return 0;
  }
  double al = g->alpha[a][p][face_id(g, a, J)];
  if (!(al > 0.0)) return 0;
  double eps = g->d.eps[p], h = g->d.h;
  long L[3] = {J[0], J[1], J[2]};
  L[a] -= 1;
  int lo_wall = J[a] == 0, hi_wall = J[a] == g->d.n[a];
  if (!lo_wall && !hi_wall) {
    long dl = dof_of(g, L, p), dh = dof_of(g, J, p);
    if (dl < 0 || dh < 0) return 0;
    lf_add(F, dh, eps / h);
    lf_add(F, dl, -eps / h);
    return 1;
  }
  int hi = hi_wall;
  const int bct = g->d.bc[2 * a + hi];
  if (bct != 1 && bct != 2) return 0;
  long C[3] = {J[0], J[1], J[2]}, C2[3];
  if (hi) C[a] -= 1;
  long d1 = dof_of(g, C, p);
  if (d1 < 0) return 0;
  memcpy(C2, C, sizeof(C2));
  C2[a] += hi ? -1 : 1;
  long d2 = dof_of(g, C2, p);
  long between[3] = {C[0], C[1], C[2]};
  if (!hi) between[a] += 1; /* face shared by C and C2 */
  if (d2 >= 0 && !(g->alpha[a][p][face_id(g, a, between)] > 0.0)) d2 = -1;
  double phi0 = dt->phidom[(long)p * wall_total(g) + wall_index(g, a, hi, C)];
  lform O;
  lf_zero(&O);
  if (bct == 2) {
    /* R and Aw of the one-sided formula, then the Robin elimination */
    lform R;
    lf_zero(&R);
    double Aw;
    if (d2 >= 0) {
      lf_add(&R, d1, -9.0 / (3.0 * h));
      lf_add(&R, d2, 1.0 / (3.0 * h));
      Aw = 8.0 / (3.0 * h);
    } else {
      lf_add(&R, d1, -2.0 / h);
      Aw = 2.0 / h;
    }
    const double a1 = g->d.robin[2 * a + hi][0];
    const double a2 = (OR_PLANT == 9 ? -1.0 : 1.0) * g->d.robin[2 * a + hi][1];
    const double den = a1 + a2 * Aw; /* phi0 is the Robin data a3 here */
    lf_axpy(&O, eps * a1 / den, &R);
    O.c = eps * Aw * phi0 / den;
  } else if (d2 >= 0 && OR_PLANT != 1) {
    lf_add(&O, d1, -9.0 * eps / (3.0 * h));
    lf_add(&O, d2, eps / (3.0 * h));
    O.c = 8.0 * eps * phi0 / (3.0 * h);
  } else {
    lf_add(&O, d1, -2.0 * eps / h);
    O.c = 2.0 * eps * phi0 / h;
  }
  /* outward is -e_a on the lo wall and +e_a on the hi wall */
  lf_axpy(F, hi ? 1.0 : -1.0, &O);
  return 1;
}

/* Flux through the centroid of face (a, J), +e_a direction: linear
 * interpolation of face-centred fluxes (Sec. 3.3, the F_2 formula), bilinear
 * in 3D, dropping to the planar 3-point form, then 1-D, then none, when a
 * neighbouring face carries no flux. */
static int centroid_flux(const or_geom* g, const or_data* dt, int a, const long J[3], int p, lform* F)
{
  lform F00, F10, F01, F11;
  if (!centred_flux(g, dt, a, J, p, &F00)) { lf_zero(F); return 0; }
  if (OR_PLANT == 2) { *F = F00; return 1; }
  long f = face_id(g, a, J);
  int t[2];
  transverse(g->D, a, t);
  double t1 = g->fcen[a][p][2 * f], t2 = (g->D == 3) ? g->fcen[a][p][2 * f + 1] : 0.0;
  double a1 = fabs(t1), a2 = fabs(t2);
  int s1 = t1 > 0.0 ? 1 : -1, s2 = t2 > 0.0 ? 1 : -1;
  int have10 = 0, have01 = 0, have11 = 0;
  if (a1 > 0.0) {
    long K[3] = {J[0], J[1], J[2]};
    K[t[0]] += s1;
    have10 = centred_flux(g, dt, a, K, p, &F10);
  }
  if (a2 > 0.0) {
    long K[3] = {J[0], J[1], J[2]};
    K[t[1]] += s2;
    have01 = centred_flux(g, dt, a, K, p, &F01);
  }
  if (a1 > 0.0 && a2 > 0.0) {
    long K[3] = {J[0], J[1], J[2]};
    K[t[0]] += s1;
    K[t[1]] += s2;
    have11 = centred_flux(g, dt, a, K, p, &F11);
  }
  int need10 = a1 > 0.0, need01 = a2 > 0.0, need11 = need10 && need01;
  lf_zero(F);
  if ((!need10 || have10) && (!need01 || have01) && (!need11 || have11)) {
    lf_axpy(F, (1.0 - a1) * (1.0 - a2), &F00);
    if (need10) lf_axpy(F, a1 * (1.0 - a2), &F10);
    if (need01) lf_axpy(F, (1.0 - a1) * a2, &F01);
    if (need11) lf_axpy(F, a1 * a2, &F11);
    return 1;
  }
  if ((!need10 || have10) && (!need01 || have01)) {
    lf_axpy(F, 1.0 - a1 - a2, &F00);
    if (need10) lf_axpy(F, a1, &F10);
    if (need01) lf_axpy(F, a2, &F01);
    return 1;
  }
  if (need10 && have10) {
    lf_axpy(F, 1.0 - a1, &F00);
    lf_axpy(F, a1, &F10);
    return 1;
  }
  if (need01 && have01) {
    lf_axpy(F, 1.0 - a2, &F00);
    lf_axpy(F, a2, &F01);
    return 1;
  }
  lf_axpy(F, 1.0, &F00);
  return 1;
}

/* stencil sum_k w_k phi_k as a form (phase p dofs) */
static void stencil_form(const or_geom* g, const or_stencil* S, int p, lform* f)
{
  lf_zero(f);
  for (int k = 0; k < S->n; ++k) lf_add(f, g->dof[p][S->cell[k]], S->w[k]);
}

/* dphi/dn_in for fragment (c, p) with the boundary value substituted:
 * electrode -> phi_E; interface -> phi_B eliminated from
 * eps_g dphi/dn_g + eps_d dphi/dn_d = -sigma (Eq. matching, physical sign).
 * A Robin electrode (a1 phi_B + a2 dphi/dn_out = a3, a3 the electrode data,
 * dn_out = -dn_in): with dphi/dn_in = w0 phi_B + S, the condition gives
 * phi_B = (a3 + a2 S) / (a1 - a2 w0), so dphi/dn_in = (w0 a3 + a1 S) / (a1 - a2 w0). */
static void eb_dphidn(const or_geom* g, const or_data* dt, long c, int p, lform* out)
{
  lform S;
  stencil_form(g, &g->st[p][c], p, &S);
  if (g->ebkind[c] == EB_ELECTRODE && g->d.eb_robin) {
    const double w0 = g->st[p][c].w0, a1 = g->d.eb_robin_a[0];
    const double a2 = (OR_PLANT == 11 ? -1.0 : 1.0) * g->d.eb_robin_a[1];
    const double den = a1 - a2 * w0;
    lf_zero(out);
    lf_axpy(out, a1 / den, &S);
    out->c = out->c + w0 * dt->phiE[c] / den;
    return;
  }
  if (g->ebkind[c] == EB_ELECTRODE) {
    lf_zero(out);
    lf_axpy(out, 1.0, &S);
    out->c = out->c + g->st[p][c].w0 * dt->phiE[c];
    return;
  }
  lform Sg, Sd, phiB;
  stencil_form(g, &g->st[0][c], 0, &Sg);
  stencil_form(g, &g->st[1][c], 1, &Sd);
  double eg = g->d.eps[OR_PLANT == 4 ? 1 : 0], ed = g->d.eps[OR_PLANT == 4 ? 0 : 1];
  double Dn = eg * g->st[0][c].w0 + ed * g->st[1][c].w0;
  lf_zero(&phiB);
  lf_axpy(&phiB, -eg / Dn, &Sg);
  lf_axpy(&phiB, -ed / Dn, &Sd);
  phiB.c = phiB.c - dt->sigma[c] / Dn;
  lf_zero(out);
  lf_axpy(out, 1.0, &S);
  lf_axpy(out, g->st[p][c].w0, &phiB);
}

/* (L phi)_c for phase p: (1/h^D)[sum_faces alpha_f h^{D-1} F_out + alpha_EB h^{D-1} F_EB]
 * - kappa lam phi_c */
static void row_form(const or_geom* g, const or_data* dt, long c, int p, lform* L)
{
  long I[3];
  cell_ijk(g, c, I);
  double h = g->d.h;
  lf_zero(L);
  for (int a = 0; a < g->D; ++a)
    for (int s = 0; s < 2; ++s) {
      long J[3] = {I[0], I[1], I[2]};
      J[a] += s;
      double al = g->alpha[a][p][face_id(g, a, J)];
      if (!(al > 0.0)) continue;
      lform F;
      if (!centroid_flux(g, dt, a, J, p, &F)) continue;
      lf_axpy(L, (s ? 1.0 : -1.0) * al / h, &F);
    }
  if (g->ebkind[c] != EB_NONE && g->cut[c]) {
    lform dn;
    eb_dphidn(g, dt, c, p, &dn);
    /* F_EB = eps dphi/dn_out = -eps dphi/dn_in */
    lf_axpy(L, -g->d.eps[p] * g->eba[c] / h, &dn);
  }
  /* the Helmholtz shift: kappa lam phi, (1/h^D)(kappa h^D lam phi); L holds
   * minus the operator's linear part */
  if (g->d.lam[p] != 0.0) lf_add(L, g->dof[p][c], -(OR_PLANT == 10 ? 1.0 : g->kappa[p][c]) * g->d.lam[p]);
}

/* Assemble A phi = b with A = -(linear part of L) and b = kappa s + (data part
 * of L); triplets written up to cap, the count returned. */
long or_assemble(const or_geom* g, const or_data* dt, long* rows, long* cols, double* vals, long cap, double* b)
{
  long nnz = 0;
  for (long c = 0; c < g->ncell; ++c)
    for (int p = 0; p < 2; ++p) {
      long r = g->dof[p][c];
      if (r < 0) continue;
      lform L;
      row_form(g, dt, c, p, &L);
      for (int k = 0; k < L.n; ++k) {
        if (nnz < cap) { rows[nnz] = r; cols[nnz] = L.idx[k]; vals[nnz] = -L.w[k]; }
        ++nnz;
      }
      b[r] = (OR_PLANT == 3 ? 1.0 : g->kappa[p][c]) * dt->s[(long)p * g->ncell + c] + L.c;
    }
  return nnz;
}

/* total outward boundary flux, integrated: sum over wall faces and EBs of
 * alpha h^{D-1} F_out, interface EBs contributing sigma alpha h^{D-1}. */
static double boundary_flux(const or_geom* g, const or_data* dt, const double* phi_dof, const uint8_t* mask)
{
  double tot = 0.0, h = g->d.h, hd1 = (g->D == 3) ? h * h : h;
  for (long c = 0; c < g->ncell; ++c) {
    if (mask && !mask[c]) continue;
    long I[3];
    cell_ijk(g, c, I);
    for (int p = 0; p < 2; ++p) {
      if (g->dof[p][c] < 0) continue;
      for (int a = 0; a < g->D; ++a)
        for (int s = 0; s < 2; ++s) {
          int wall = s ? (I[a] == g->d.n[a] - 1) : (I[a] == 0);
          if (!wall) continue;
          long J[3] = {I[0], I[1], I[2]};
          J[a] += s;
          double al = g->alpha[a][p][face_id(g, a, J)];
          if (!(al > 0.0)) continue;
          lform F;
          if (!centroid_flux(g, dt, a, J, p, &F)) continue;
          double v = F.c;
          for (int k = 0; k < F.n; ++k) v = v + F.w[k] * phi_dof[F.idx[k]];
          tot = tot + (s ? 1.0 : -1.0) * al * hd1 * v;
        }
      if (g->ebkind[c] == EB_ELECTRODE && g->cut[c]) {
        lform dn;
        eb_dphidn(g, dt, c, p, &dn);
        double v = dn.c;
        for (int k = 0; k < dn.n; ++k) v = v + dn.w[k] * phi_dof[dn.idx[k]];
        tot = tot + g->eba[c] * hd1 * (-g->d.eps[p] * v);
      }
    }
    if (g->ebkind[c] == EB_INTERFACE && g->dof[0][c] >= 0 && g->dof[1][c] >= 0)
      tot = tot + dt->sigma[c] * g->eba[c] * hd1;
  }
  return tot;
}

double or_boundary_flux(const or_geom* g, const or_data* dt, const double* phi_dof)
{
  return boundary_flux(g, dt, phi_dof, NULL);
}

/* The same sum over the cells whose mask entry is non-zero (a composite grid
 * counts the coarse cells outside a refined box only). */
double or_boundary_flux_masked(const or_geom* g, const or_data* dt, const double* phi_dof, const uint8_t* mask)
{
  return boundary_flux(g, dt, phi_dof, mask);
}

/* The flux of face (a, J), phase p, as it enters the row of the cell on the
 * face's low side: alpha/h times the centroid flux in the +e_a direction, a
 * linear form in the dofs plus a constant.  Returns the number of terms, 0
 * when the face carries no flux.  A composite operator uses it to take a
 * coarse flux out of a coarse row before putting the fine fluxes through the
 * same face in its place (refluxing). */
long or_face_flux(const or_geom* g, const or_data* dt, int a, const long* Jin, int p, long* idx, double* w,
                  double* c)
{
  long J[3] = {Jin[0], Jin[1], Jin[2]};
  *c = 0.0;
  double al = g->alpha[a][p][face_id(g, a, J)];
  if (!(al > 0.0)) return 0;
  lform F;
  if (!centroid_flux(g, dt, a, J, p, &F)) return 0;
  for (int k = 0; k < F.n; ++k) {
    idx[k] = F.idx[k];
    w[k] = F.w[k] * al / g->d.h;
  }
  *c = F.c * al / g->d.h;
  return F.n;
}

/* E = -grad phi at cell centres per phase ([D][2][cell]) and the normal
 * field -dphi/dn_in at EB centroids per phase ([cell][2]). */
void or_field(const or_geom* g, const or_data* dt, const double* phi_dof, double* E, double* En)
{
  double h = g->d.h;
  long nc = g->ncell;
  for (long c = 0; c < nc; ++c) {
    long I[3];
    cell_ijk(g, c, I);
    for (int p = 0; p < 2; ++p) {
      En[2 * c + p] = 0.0;
      for (int a = 0; a < g->D; ++a) E[((long)a * 2 + p) * nc + c] = 0.0;
      long r = g->dof[p][c];
      if (r < 0) continue;
      double dn_val = 0.0;
      int has_eb = g->cut[c] && g->ebkind[c] != EB_NONE;
      if (has_eb) {
        lform dn;
        eb_dphidn(g, dt, c, p, &dn);
        dn_val = dn.c;
        for (int k = 0; k < dn.n; ++k) dn_val = dn_val + dn.w[k] * phi_dof[dn.idx[k]];
        En[2 * c + p] = -dn_val;
      }
      for (int a = 0; a < g->D; ++a) {
        long Lo[3] = {I[0], I[1], I[2]}, Hi[3] = {I[0], I[1], I[2]};
        Lo[a] -= 1;
        Hi[a] += 1;
        long dl = dof_of(g, Lo, p), dh = dof_of(g, Hi, p);
        long Jl[3] = {I[0], I[1], I[2]}, Jh[3] = {I[0], I[1], I[2]};
        Jh[a] += 1;
        if (dl >= 0 && !(g->alpha[a][p][face_id(g, a, Jl)] > 0.0)) dl = -1;
        if (dh >= 0 && !(g->alpha[a][p][face_id(g, a, Jh)] > 0.0)) dh = -1;
        double v;
        if (dl >= 0 && dh >= 0) v = -(phi_dof[dh] - phi_dof[dl]) / (2.0 * h);
        else if (dh >= 0) v = -(phi_dof[dh] - phi_dof[r]) / h;
        else if (dl >= 0) v = -(phi_dof[r] - phi_dof[dl]) / h;
        else if (has_eb) {
          double sgn = (g->ebkind[c] == EB_INTERFACE && p == 1) ? 1.0 : -1.0;
          v = -dn_val * (sgn * g->ebn[3 * c + a]);
        } else v = 0.0;
        E[((long)a * 2 + p) * nc + c] = v;
      }
    }
  }
}

/* ------------------------------------------------------------- queries */

int or_status(const or_geom* g) { return g->status; }
long or_bad_cell(const or_geom* g) { return g->bad_cell; }
long or_ndof(const or_geom* g) { return g->ndof; }
long or_ncell(const or_geom* g) { return g->ncell; }
long or_n_eb(const or_geom* g) { return g->n_eb; }
long or_wall_total(const or_geom* g) { return wall_total(g); }
void or_counts(const or_geom* g, long* out)
{
  for (int k = 0; k < 4; ++k) out[k] = g->counts[k];
}
void or_cells(const or_geom* g, uint8_t* cut, uint8_t* ebkind, double* kappa, long* dof, double* eba, double* ebn,
              double* ebx)
{
  memcpy(cut, g->cut, g->ncell);
  memcpy(ebkind, g->ebkind, g->ncell);
  for (int p = 0; p < 2; ++p) {
    memcpy(kappa + p * g->ncell, g->kappa[p], sizeof(double) * g->ncell);
    memcpy(dof + p * g->ncell, g->dof[p], sizeof(long) * g->ncell);
  }
  memcpy(eba, g->eba, sizeof(double) * g->ncell);
  memcpy(ebn, g->ebn, sizeof(double) * 3 * g->ncell);
  memcpy(ebx, g->ebx, sizeof(double) * 3 * g->ncell);
}
long or_nface(const or_geom* g, int a) { return g->nface[a]; }
void or_faces(const or_geom* g, int a, double* alpha, double* fcen)
{
  for (int p = 0; p < 2; ++p) {
    memcpy(alpha + p * g->nface[a], g->alpha[a][p], sizeof(double) * g->nface[a]);
    memcpy(fcen + 2 * p * g->nface[a], g->fcen[a][p], sizeof(double) * 2 * g->nface[a]);
  }
}
void or_labels(const or_geom* g, uint8_t* lab) { memcpy(lab, g->lab, g->nnode); }
void or_stencil_order(const or_geom* g, int* order)
{
  for (int p = 0; p < 2; ++p)
    for (long c = 0; c < g->ncell; ++c) order[p * g->ncell + c] = g->st[p][c].order;
}
double or_eval_implicit(const or_desc* d, int root, const double* x) { return csg_eval(d, root, x); }

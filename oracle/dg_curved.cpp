/*
 * ORACLE — test infrastructure only (see dg_oracle.h).
 *
 * The curvilinear form of the same sliding-mesh DGSEM operator: every element carries its
 * own metric terms Ja^i_n and Jacobian J at the LGL nodes (Sec. 3.1, Eq.
 * transformed_equation), so that curved elements and a rotating sub-domain are covered:
 *   geom 1: the cylindrical sliding interface of Sec. 3.3 (rotor inside the circle,
 *           stator outside, relative motion a rotation), the "rotation with a
 *           cylindrical radial interface" geometry of the paper's overview figure;
 *   geom 2: the plane two-block box of dg_oracle.cpp, written through general metrics;
 *   geom 3: the plane annular interface normal to the rotation axis (the "rotation with a
 *           plane annular axial interface" geometry of the paper's overview figure): rotor
 *           z in [x0, x1] below the stator z in [x1, x2], both annular sectors with radii
 *           [z0, z1] (xi^2 runs from r = z1 to r = z0, which keeps the map (theta, r, z)
 *           right-handed); slip walls at both radii and at the axial ends;
 *   geom 4: the conical interface about the rotation axis (a rotor inside the cone, the
 *           stator outside): radius s sin(alpha) + n cos(alpha), height s cos(alpha) -
 *           n sin(alpha) for generator coordinate s and normal offset n; slip walls at
 *           the ends of s and n.
 *
 * Readings (the paper does not print them):
 *   - metrics: conservative curl form of Kopriva (2006), antisymmetrised,
 *       Ja^i_n = -1/2 [curl_xi (X_l grad_xi X_m - X_m grad_xi X_l)]_i,  (n, m, l) cyclic,
 *     from the node coordinates of the analytic map (relative to the element's centre,
 *     which the form does not see: it is translation invariant); J = a_1 . (a_2 x a_3) with
 *     a_d = D_d X.  The discrete metric identities sum_i D_i Ja^i_n = 0 hold, and the
 *     form commutes with a rotation of the mesh;
 *   - the rotor (block 0 of geom 1) turns about the z axis by phi(t) = fma(omega, t, phi0):
 *     X(t) = R(phi) X(0), Ja^i(t) = R(phi) Ja^i(0), v^g = omega e_z x X(t);
 *   - the relative displacement of the stator seen from the rotor is Delta = -phi, in
 *     angle units with face length l = h_theta (Sec. 4.3);
 *   - the periodic sector: a state read across its ends, or across the interface from a
 *     periodic image of a stator face, is rotated by the sector angle per wrap;
 *   - mortar geometry: the static (rotor) face's Ja^3 projected onto the mortar nodes; the
 *     grid velocity normal to the interface is zero (the motion is tangential);
 *   - slip walls at r = x0 and r = x2: the exterior state is the interior state with its
 *     normal velocity reflected, the wall's normal grid velocity is zero (it moves
 *     tangentially); the viscous wall flux is zero (adiabatic, no shear);
 *   - conforming faces: each element uses its own face metric; the two neighbours agree to
 *     rounding (watertight faces).
 */
#include "dg_oracle.h"

#include <cmath>
#include <cstring>
#include <vector>

namespace {

struct Curved {
  int kind = 1;              /* matches the first member of the Cartesian oracle's handle */
  orc_problem p;
  int N, np, nn;
  long long Es, Em, E;
  int ny, nz;                /* faces along xi^1 (sliding) and xi^2 (perpendicular) */
  double h1, h2, h3[2];      /* element sizes along xi^1, xi^2, xi^3 (per block) */
  bool cyl, ns;              /* cyl: a rotor turning about z (geom 1 and 3) */
  bool annular;              /* geom 3: reference axes (theta, r, z) instead of (theta, z, r) */
  bool cone;                 /* geom 4: reference axes (theta, s, n) across a cone */
  double sa, ca;             /* sin, cos of the cone's half-angle */
  double Theta;              /* periodic sector angle (geom 1) */
  std::vector<double> x, w, D, Dhat;
  double A[5], B[5], c[5];
  std::vector<double> X0, Ja0, J0;   /* [E][3][nn], [E][3][3][nn], [E][nn] at t = 0 */
};

struct Id { int blk, ix, iy, iz; };

Id elem_id(const Curved& o, long long e) {
  Id id;
  long long loc = e;
  int nx = o.p.nel_s[0];
  id.blk = 0;
  if (e >= o.Es) { id.blk = 1; loc = e - o.Es; nx = o.p.nel_m[0]; }
  id.ix = (int)(loc % nx);
  id.iy = (int)((loc / nx) % o.ny);
  id.iz = (int)(loc / ((long long)nx * o.ny));
  return id;
}

long long elem_index(const Curved& o, int blk, int ix, int iy, int iz) {
  int nx = blk == 0 ? o.p.nel_s[0] : o.p.nel_m[0];
  return (blk == 0 ? 0 : o.Es) + ix + (long long)nx * (iy + (long long)o.ny * iz);
}

int wrap(long long i, int n) { long long r = i % n; if (r < 0) r += n; return (int)r; }
long long floor_div(long long a, long long b) { long long q = a / b; if ((a % b != 0) && ((a < 0) != (b < 0))) --q; return q; }

int node(const Curved& o, int i, int j, int k) { return i + o.np * (j + o.np * k); }

/* node of face (d, side) with in-face indices (a, b): d=0 (a,b)=(j,k), d=1 (i,k), d=2 (i,j) */
int face_node(const Curved& o, int d, int side, int a, int b) {
  int f = side ? o.N : 0;
  if (d == 0) return node(o, f, a, b);
  if (d == 1) return node(o, a, f, b);
  return node(o, a, b, f);
}

/* ---- motion ---- */
double rotor_angle(const Curved& o, double t) { return std::fma(o.p.v, t, o.p.delta0); }
/* displacement of block 1 relative to block 0 along xi^1, as the mapper takes it */
double rel_displacement(const Curved& o, double t) {
  return o.cyl ? std::fma(-o.p.v, t, -o.p.delta0) : std::fma(o.p.v, t, o.p.delta0);
}
bool moves(const Curved& o, int blk) { return o.cyl ? blk == 0 : blk == 1; }

void rotate_z(double c, double s, const double* a, double* b) {
  double x = c * a[0] - s * a[1], y = s * a[0] + c * a[1];
  b[0] = x; b[1] = y; b[2] = a[2];
}
/* momentum components of a conservative state */
void rotate_state(double ang, double* U) {
  if (ang == 0.0) return;
  double m[3] = {U[1], U[2], U[3]}, r[3];
  rotate_z(std::cos(ang), std::sin(ang), m, r);
  U[1] = r[0]; U[2] = r[1]; U[3] = r[2];
}
/* gradients g[a*5 + c] of the primitives: vector index a, and c = 1..3 a vector too */
void rotate_grad(double ang, double* g) {
  if (ang == 0.0) return;
  double c = std::cos(ang), s = std::sin(ang), R[3][3] = {{c, -s, 0}, {s, c, 0}, {0, 0, 1}};
  double h[15];
  for (int cc = 0; cc < 5; ++cc)
    for (int a = 0; a < 3; ++a) {
      double acc = 0.0;
      for (int b = 0; b < 3; ++b) acc += R[a][b] * g[b * 5 + cc];
      h[a * 5 + cc] = acc;
    }
  for (int a = 0; a < 3; ++a) {
    double v[3];
    for (int cc = 0; cc < 3; ++cc) {
      double acc = 0.0;
      for (int d = 0; d < 3; ++d) acc += R[cc][d] * h[a * 5 + 1 + d];
      v[cc] = acc;
    }
    for (int cc = 0; cc < 3; ++cc) h[a * 5 + 1 + cc] = v[cc];
  }
  std::memcpy(g, h, sizeof(h));
}

/* physical node position at time t and the node's geometry */
void node_X(const Curved& o, long long e, int nd, double t, double* X) {
  const double* X0 = &o.X0[e * 3 * o.nn];
  double a[3] = {X0[nd], X0[o.nn + nd], X0[2 * o.nn + nd]};
  Id id = elem_id(o, e);
  if (!moves(o, id.blk)) { X[0] = a[0]; X[1] = a[1]; X[2] = a[2]; return; }
  if (o.cyl) {
    double ph = rotor_angle(o, t);
    rotate_z(std::cos(ph), std::sin(ph), a, X);
  } else {
    X[0] = a[0]; X[1] = a[1] + rel_displacement(o, t); X[2] = a[2];
  }
}

/* Ja^i (3 components) at node nd of element e at time t */
void node_Ja(const Curved& o, long long e, int i, int nd, double t, double* Ja) {
  const double* J0 = &o.Ja0[(e * 9 + i * 3) * o.nn];
  double a[3] = {J0[nd], J0[o.nn + nd], J0[2 * o.nn + nd]};
  Id id = elem_id(o, e);
  if (o.cyl && moves(o, id.blk)) {
    double ph = rotor_angle(o, t);
    rotate_z(std::cos(ph), std::sin(ph), a, Ja);
  } else {
    Ja[0] = a[0]; Ja[1] = a[1]; Ja[2] = a[2];
  }
}

void node_vg(const Curved& o, long long e, int nd, double t, double* vg) {
  Id id = elem_id(o, e);
  vg[0] = vg[1] = vg[2] = 0.0;
  if (!moves(o, id.blk)) return;
  if (o.cyl) {
    double X[3];
    node_X(o, e, nd, t, X);
    vg[0] = -o.p.v * X[1];
    vg[1] = o.p.v * X[0];
  } else {
    vg[1] = o.p.v;
  }
}

/* ---- geometry at t = 0 (analytic map, curl-form metrics) ---- */
void build_geometry(Curved& o) {
  int np = o.np, nn = o.nn;
  o.X0.assign(o.E * 3 * nn, 0.0);
  o.Ja0.assign(o.E * 9 * nn, 0.0);
  o.J0.assign(o.E * nn, 0.0);
  #pragma omp parallel for schedule(static)
  for (long long e = 0; e < o.E; ++e) {
    Id id = elem_id(o, e);
    double lo3 = id.blk == 0 ? o.p.x0 : o.p.x1;
    std::vector<double> X(3 * nn);
    for (int k = 0; k < np; ++k)
      for (int j = 0; j < np; ++j)
        for (int i = 0; i < np; ++i) {
          double s1 = o.p.y0 + id.iy * o.h1 + (o.x[i] + 1.0) * 0.5 * o.h1;
          double s2 = o.p.z0 + id.iz * o.h2 + (o.x[j] + 1.0) * 0.5 * o.h2;
          double s3 = lo3 + id.ix * o.h3[id.blk] + (o.x[k] + 1.0) * 0.5 * o.h3[id.blk];
          int nd = node(o, i, j, k);
          if (o.cone) {             /* xi^1 -> theta, xi^2 -> s (generator), xi^3 -> n (across) */
            double rr = s2 * o.sa + s3 * o.ca;
            X[nd] = rr * std::cos(s1);
            X[nn + nd] = rr * std::sin(s1);
            X[2 * nn + nd] = s2 * o.ca - s3 * o.sa;
            continue;
          }
          if (o.annular) {          /* xi^1 -> theta, xi^2 -> -r (right-handed), xi^3 -> z */
            double rr = o.p.z0 + o.p.z1 - s2;
            X[nd] = rr * std::cos(s1);
            X[nn + nd] = rr * std::sin(s1);
            X[2 * nn + nd] = s3;
            continue;
          }
          if (o.cyl) {              /* xi^1 -> theta, xi^2 -> z, xi^3 -> r */
            X[nd] = s3 * std::cos(s1);
            X[nn + nd] = s3 * std::sin(s1);
          } else {
            X[nd] = s3;
            X[nn + nd] = s1;
          }
          X[2 * nn + nd] = s2;
        }
    /* coordinates relative to the element's centre: the curl form is invariant under a
     * translation of X (the D_d commute), and local coordinates keep its products from
     * cancelling digits */
    double Xc[3];
    {
      double s1 = o.p.y0 + (id.iy + 0.5) * o.h1, s2 = o.p.z0 + (id.iz + 0.5) * o.h2;
      double s3 = lo3 + (id.ix + 0.5) * o.h3[id.blk];
      double rc = o.p.z0 + o.p.z1 - s2;
      Xc[0] = o.annular ? rc * std::cos(s1) : (o.cyl ? s3 * std::cos(s1) : s3);
      Xc[1] = o.annular ? rc * std::sin(s1) : (o.cyl ? s3 * std::sin(s1) : s1);
      Xc[2] = o.annular ? s3 : s2;
      if (o.cone) {
        double rk = s2 * o.sa + s3 * o.ca;
        Xc[0] = rk * std::cos(s1);
        Xc[1] = rk * std::sin(s1);
        Xc[2] = s2 * o.ca - s3 * o.sa;
      }
    }
    for (int n = 0; n < 3; ++n)
      for (int nd = 0; nd < nn; ++nd) X[n * nn + nd] -= Xc[n];
    /* derivative along reference direction d of a nodal field f */
    auto Dd = [&](int d, const double* f, double* out) {
      for (int k = 0; k < np; ++k)
        for (int j = 0; j < np; ++j)
          for (int i = 0; i < np; ++i) {
            double acc = 0.0;
            for (int l = 0; l < np; ++l) {
              int src = d == 0 ? node(o, l, j, k) : (d == 1 ? node(o, i, l, k) : node(o, i, j, l));
              int row = d == 0 ? i : (d == 1 ? j : k);
              acc += o.D[row * np + l] * f[src];
            }
            out[node(o, i, j, k)] = acc;
          }
    };
    /* covariant basis a_d = D_d X and the Jacobian */
    std::vector<double> dX(9 * nn);    /* dX[(d*3 + n)*nn] = d X_n / d xi^d */
    for (int d = 0; d < 3; ++d)
      for (int n = 0; n < 3; ++n) Dd(d, &X[n * nn], &dX[(d * 3 + n) * nn]);
    for (int nd = 0; nd < nn; ++nd) {
      const double* a1 = &dX[0]; const double* a2 = &dX[3 * nn]; const double* a3 = &dX[6 * nn];
      double A1[3] = {a1[nd], a1[nn + nd], a1[2 * nn + nd]};
      double A2[3] = {a2[nd], a2[nn + nd], a2[2 * nn + nd]};
      double A3[3] = {a3[nd], a3[nn + nd], a3[2 * nn + nd]};
      double cx = A2[1] * A3[2] - A2[2] * A3[1], cy = A2[2] * A3[0] - A2[0] * A3[2], cz = A2[0] * A3[1] - A2[1] * A3[0];
      o.J0[e * nn + nd] = A1[0] * cx + A1[1] * cy + A1[2] * cz;
    }
    /* curl form: for each Cartesian component n with (n, m, l) cyclic,
     * V_k = X_l D_k X_m - X_m D_k X_l, Ja^i_n = -1/2 (D_j V_k - D_k V_j), (i, j, k) cyclic */
    std::vector<double> V(3 * nn), T1(nn), T2(nn);
    for (int n = 0; n < 3; ++n) {
      int m = (n + 1) % 3, l = (n + 2) % 3;
      for (int k = 0; k < 3; ++k)
        for (int nd = 0; nd < nn; ++nd)
          V[k * nn + nd] = X[l * nn + nd] * dX[(k * 3 + m) * nn + nd] - X[m * nn + nd] * dX[(k * 3 + l) * nn + nd];
      for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3, k = (i + 2) % 3;
        Dd(j, &V[k * nn], T1.data());
        Dd(k, &V[j * nn], T2.data());
        for (int nd = 0; nd < nn; ++nd) o.Ja0[(e * 9 + i * 3 + n) * nn + nd] = -0.5 * (T1[nd] - T2[nd]);
      }
    }
    for (int n = 0; n < 3; ++n)
      for (int nd = 0; nd < nn; ++nd) o.X0[(e * 3 + n) * nn + nd] = X[n * nn + nd] + Xc[n];
  }
}

/* ---- neighbours ---- */
/* kind 0: conforming (nb, and the rotation angle of the neighbour's state into this
 * element's frame), 1: boundary, 2: sliding interface */
int neighbour(const Curved& o, const Id& id, int d, int side, long long* nb, double* ang) {
  *ang = 0.0;
  int nx = id.blk == 0 ? o.p.nel_s[0] : o.p.nel_m[0];
  if (d == 0) {
    int iy = id.iy + (side ? 1 : -1);
    if (o.cyl && iy >= o.ny) *ang = o.Theta;      /* image across theta = y1 */
    if (o.cyl && iy < 0) *ang = -o.Theta;
    *nb = elem_index(o, id.blk, id.ix, wrap(iy, o.ny), id.iz);
    return 0;
  }
  if (d == 1) {
    int iz = id.iz + (side ? 1 : -1);
    if ((o.annular || o.cone) && (iz < 0 || iz >= o.nz)) return 1;   /* slip walls at the xi^2 ends */
    *nb = elem_index(o, id.blk, id.ix, id.iy, wrap(iz, o.nz));
    return 0;
  }
  int jx = id.ix + (side ? 1 : -1);
  if (jx >= 0 && jx < nx) { *nb = elem_index(o, id.blk, jx, id.iy, id.iz); return 0; }
  if ((id.blk == 0 && side == 0) || (id.blk == 1 && side == 1)) return 1;
  if (o.p.interface_conforming) {
    int b2 = 1 - id.blk;
    *nb = elem_index(o, b2, b2 == 0 ? o.p.nel_s[0] - 1 : 0, id.iy, id.iz);
    return 0;
  }
  return 2;
}

void cons_to_prim(const double* U, double g, double* Q) {
  Q[0] = U[0]; Q[1] = U[1] / U[0]; Q[2] = U[2] / U[0]; Q[3] = U[3] / U[0];
  Q[4] = (g - 1.0) * (U[4] - 0.5 * U[0] * (Q[1] * Q[1] + Q[2] * Q[2] + Q[3] * Q[3]));
}

/* exterior state of a boundary face node: plane -> the flow's state at the node's position
 * (weak Dirichlet), cylinder -> slip-wall mirror of the interior state (outward unit normal n) */
void boundary_state(const Curved& o, long long e, int nd, double t, const double* uin, const double* n, double* uout) {
  if (!o.cyl) {
    double X[3];
    node_X(o, e, nd, t, X);
    orc_flow_state(&o.p, X, t, 1, uout);
    return;
  }
  double mn = uin[1] * n[0] + uin[2] * n[1] + uin[3] * n[2];
  uout[0] = uin[0];
  for (int a = 0; a < 3; ++a) uout[1 + a] = uin[1 + a] - 2.0 * mn * n[a];
  uout[4] = uin[4];
}

void viscous_dot(const Curved& o, const double* U, const double* g15, const double* N, double* Fn) {
  double Fv[15];
  orc_viscous_flux(U, g15, o.p.mu, o.p.Pr, o.p.Rgas, o.p.gamma, Fv);
  for (int c = 0; c < 5; ++c) Fn[c] = Fv[c] * N[0] + Fv[5 + c] * N[1] + Fv[10 + c] * N[2];
}

/* ---------------------- sliding interface (Sec. 3.3) ---------------------- */
struct Iface {
  long long n; double s, sig_s, sig_m;
  std::vector<double> Ps_lo, Ps_hi, Bs_lo, Bs_hi, Pm_lo, Pm_hi, Bm_lo, Bm_hi;
};

void iface_config(const Curved& o, double t, Iface& I) {
  orc_map_closed(rel_displacement(o, t), o.h1, &I.n, &I.s);
  I.sig_s = 2.0 * I.s - 1.0;
  I.sig_m = 1.0 - 2.0 * I.s;
  int nq = o.np * o.np;
  for (auto* v : {&I.Ps_lo, &I.Ps_hi, &I.Bs_lo, &I.Bs_hi, &I.Pm_lo, &I.Pm_hi, &I.Bm_lo, &I.Bm_hi}) v->assign(nq, 0.0);
  orc_mortar_mats(o.N, I.sig_s, I.Ps_lo.data(), I.Ps_hi.data(), I.Bs_lo.data(), I.Bs_hi.data());
  orc_mortar_mats(o.N, I.sig_m, I.Pm_lo.data(), I.Pm_hi.data(), I.Bm_lo.data(), I.Bm_hi.data());
}

/* the element of face (ipar, iperp) on side blk of the interface and its face layer */
long long iface_elem(const Curved& o, int blk, int ipar, int iperp) {
  return elem_index(o, blk, blk == 0 ? o.p.nel_s[0] - 1 : 0, ipar, iperp);
}

/* per-node fields of a face: f[(c*np + q)*np + p] = field component c at node (p, q) */
void face_field(const Curved& o, int blk, int ipar, int iperp, int ncomp,
                const std::vector<double>& src, int stride_e, double* f) {
  long long e = iface_elem(o, blk, ipar, iperp);
  int side = blk == 0 ? 1 : 0;
  for (int c = 0; c < ncomp; ++c)
    for (int q = 0; q < o.np; ++q)
      for (int p = 0; p < o.np; ++p)
        f[(c * o.np + q) * o.np + p] = src[(e * stride_e + c) * o.nn + face_node(o, 2, side, p, q)];
}

void project(const Curved& o, const double* P, const double* tr, double* Q, int ncomp) {
  for (int v = 0; v < ncomp; ++v)
    for (int q = 0; q < o.np; ++q)
      for (int j = 0; j < o.np; ++j) {
        double acc = 0.0;
        for (int i = 0; i < o.np; ++i) acc += P[j * o.np + i] * tr[(v * o.np + q) * o.np + i];
        Q[(v * o.np + q) * o.np + j] = acc;
      }
}

void back_project(const Curved& o, const double* Blo, const double* Flo, const double* Bhi, const double* Fhi,
                  double sign, double* F, int ncomp) {
  for (int v = 0; v < ncomp; ++v)
    for (int q = 0; q < o.np; ++q)
      for (int i = 0; i < o.np; ++i) {
        double acc = 0.0;
        for (int j = 0; j < o.np; ++j) acc += Blo[i * o.np + j] * Flo[(v * o.np + q) * o.np + j];
        for (int j = 0; j < o.np; ++j) acc += Bhi[i * o.np + j] * Fhi[(v * o.np + q) * o.np + j];
        F[(v * o.np + q) * o.np + i] = sign * acc;
      }
}

/* angle that carries the moving partner of mortar (ipar, isub) into the static frame */
double mortar_angle(const Curved& o, const Iface& I, int ipar, int isub) {
  if (!o.cyl) return 0.0;
  long long itu = (long long)ipar - I.n + isub - 1;
  return (double)floor_div(itu, o.ny) * o.Theta;
}

/* the static face's Ja^3 at time t, per face node: N[(a*np + q)*np + p] */
void static_face_normal(const Curved& o, int ipar, int iperp, double t, double* N) {
  long long e = iface_elem(o, 0, ipar, iperp);
  for (int q = 0; q < o.np; ++q)
    for (int p = 0; p < o.np; ++p) {
      double Ja[3];
      node_Ja(o, e, 2, face_node(o, 2, 1, p, q), t, Ja);
      for (int a = 0; a < 3; ++a) N[(a * o.np + q) * o.np + p] = Ja[a];
    }
}

/* primitive trace of a face, from the conservative state */
void prim_face(const Curved& o, const double* U, int blk, int ipar, int iperp, double* pr) {
  long long e = iface_elem(o, blk, ipar, iperp);
  int side = blk == 0 ? 1 : 0, nq = o.np * o.np;
  for (int q = 0; q < o.np; ++q)
    for (int p = 0; p < o.np; ++p) {
      double u[5], qq[5];
      int nd = face_node(o, 2, side, p, q);
      for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * o.nn + nd];
      cons_to_prim(u, o.p.gamma, qq);
      for (int v = 0; v < 5; ++v) pr[v * nq + q * o.np + p] = qq[v];
    }
}

/* Steps 2-4 on mortar (ipar, iperp, isub): projected traces of both sides (the moving one
 * rotated into the static frame), Riemann flux with the projected static normal, times
 * the projected surface element.  mode 0: flux (grad may be null), mode 1: lifting face
 * values q* N_a (15 values per node, [a*5 + c]). */
void mortar_values(const Curved& o, const Iface& I, const double* U, const double* grad, double t, int ipar, int iperp,
                   int isub, int mode, double* Fm) {
  int np = o.np, nq = np * np;
  const double* Ps = isub == 0 ? I.Ps_lo.data() : I.Ps_hi.data();
  const double* Pm = isub == 0 ? I.Pm_hi.data() : I.Pm_lo.data();
  int it = wrap((long long)ipar - I.n + isub - 1, o.ny);
  double ang = mortar_angle(o, I, ipar, isub);
  std::vector<double> tr(15 * nq), QL(5 * nq), QR(5 * nq), GL(15 * nq), GR(15 * nq), Nf(3 * nq), Nm(3 * nq);
  if (mode == 1) {
    prim_face(o, U, 0, ipar, iperp, tr.data());
    project(o, Ps, tr.data(), QL.data(), 5);
    prim_face(o, U, 1, it, iperp, tr.data());
    project(o, Pm, tr.data(), QR.data(), 5);
  } else {
    long long es = iface_elem(o, 0, ipar, iperp), em = iface_elem(o, 1, it, iperp);
    for (int v = 0; v < 5; ++v)
      for (int q = 0; q < np; ++q)
        for (int p = 0; p < np; ++p) tr[(v * np + q) * np + p] = U[(es * 5 + v) * o.nn + face_node(o, 2, 1, p, q)];
    project(o, Ps, tr.data(), QL.data(), 5);
    for (int v = 0; v < 5; ++v)
      for (int q = 0; q < np; ++q)
        for (int p = 0; p < np; ++p) tr[(v * np + q) * np + p] = U[(em * 5 + v) * o.nn + face_node(o, 2, 0, p, q)];
    project(o, Pm, tr.data(), QR.data(), 5);
    if (grad) {
      for (int k = 0; k < 15; ++k)
        for (int q = 0; q < np; ++q)
          for (int p = 0; p < np; ++p) {
            tr[(k * np + q) * np + p] = grad[(es * 15 + k) * o.nn + face_node(o, 2, 1, p, q)];
          }
      project(o, Ps, tr.data(), GL.data(), 15);
      for (int k = 0; k < 15; ++k)
        for (int q = 0; q < np; ++q)
          for (int p = 0; p < np; ++p) tr[(k * np + q) * np + p] = grad[(em * 15 + k) * o.nn + face_node(o, 2, 0, p, q)];
      project(o, Pm, tr.data(), GR.data(), 15);
    }
  }
  static_face_normal(o, ipar, iperp, t, Nf.data());
  project(o, Ps, Nf.data(), Nm.data(), 3);
  for (int q = 0; q < np; ++q)
    for (int j = 0; j < np; ++j) {
      int ab = q * np + j;
      double N[3] = {Nm[ab], Nm[nq + ab], Nm[2 * nq + ab]};
      double sJ = std::sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
      double n[3] = {N[0] / sJ, N[1] / sJ, N[2] / sJ};
      double ul[5], ur[5];
      for (int v = 0; v < 5; ++v) { ul[v] = QL[v * nq + ab]; ur[v] = QR[v * nq + ab]; }
      if (mode == 1) {
        /* primitive traces: rotate the moving side's velocity */
        if (ang != 0.0) {
          double vv[3] = {ur[1], ur[2], ur[3]}, r[3];
          rotate_z(std::cos(ang), std::sin(ang), vv, r);
          ur[1] = r[0]; ur[2] = r[1]; ur[3] = r[2];
        }
        for (int a = 0; a < 3; ++a)
          for (int c = 0; c < 5; ++c) Fm[((a * 5 + c) * np + q) * np + j] = 0.5 * (ul[c] + ur[c]) * N[a];
        continue;
      }
      rotate_state(ang, ur);
      double f[5];
      orc_riemann(o.p.riemann, ul, ur, n, 0.0, o.p.gamma, f);
      for (int v = 0; v < 5; ++v) f[v] *= sJ;
      if (grad) {
        double gl[15], gr[15], fl[5], fr[5];
        for (int k = 0; k < 15; ++k) { gl[k] = GL[k * nq + ab]; gr[k] = GR[k * nq + ab]; }
        rotate_grad(ang, gr);
        viscous_dot(o, ul, gl, N, fl);
        viscous_dot(o, ur, gr, N, fr);
        for (int v = 0; v < 5; ++v) f[v] -= 0.5 * (fl[v] + fr[v]);
      }
      for (int v = 0; v < 5; ++v) Fm[(v * np + q) * np + j] = f[v];
    }
}

/* rotate face values back into the moving face's frame: state-like (5) or lifting (15) */
void unrotate_face(int ncomp, int np, double ang, double* F) {
  if (ang == 0.0) return;
  int nq = np * np;
  for (int ab = 0; ab < nq; ++ab) {
    if (ncomp == 5) {
      double u[5];
      for (int v = 0; v < 5; ++v) u[v] = F[v * nq + ab];
      rotate_state(-ang, u);
      for (int v = 0; v < 5; ++v) F[v * nq + ab] = u[v];
    } else {
      double g[15];
      for (int k = 0; k < 15; ++k) g[k] = F[k * nq + ab];
      rotate_grad(-ang, g);
      for (int k = 0; k < 15; ++k) F[k * nq + ab] = g[k];
    }
  }
}

/* All interface face values: mode 0 fluxes (5 per node), mode 1 lifting values (15). */
void all_interface(const Curved& o, const Iface& I, const double* U, const double* grad, double t, int mode,
                   std::vector<double>& Fs, std::vector<double>& Fm) {
  int nq = o.np * o.np, nc = mode == 1 ? 15 : 5;
  long long nf = (long long)o.ny * o.nz;
  std::vector<double> Fsm(nf * 2 * nc * nq);
  #pragma omp parallel for schedule(dynamic)
  for (long long f = 0; f < nf; ++f)
    for (int isub = 0; isub < 2; ++isub)
      mortar_values(o, I, U, grad, t, (int)(f % o.ny), (int)(f / o.ny), isub, mode, Fsm.data() + (f * 2 + isub) * nc * nq);
  Fs.assign(nf * nc * nq, 0.0);
  Fm.assign(nf * nc * nq, 0.0);
  #pragma omp parallel for schedule(dynamic)
  for (long long f = 0; f < nf; ++f) {
    int ipar = (int)(f % o.ny);
    long long row = (f / o.ny) * o.ny;
    back_project(o, I.Bs_lo.data(), Fsm.data() + (f * 2 + 0) * nc * nq, I.Bs_hi.data(),
                 Fsm.data() + (f * 2 + 1) * nc * nq, 1.0, Fs.data() + f * nc * nq, nc);
    /* moving face ipar: lower part = mortar (ipar + n, 1), upper part = mortar (ipar + n + 1, 0) */
    int plo = wrap((long long)ipar + I.n, o.ny), phi = wrap((long long)ipar + I.n + 1, o.ny);
    std::vector<double> lo(Fsm.begin() + (row + plo) * 2 * nc * nq + nc * nq, Fsm.begin() + (row + plo) * 2 * nc * nq + 2 * nc * nq);
    std::vector<double> hi(Fsm.begin() + (row + phi) * 2 * nc * nq, Fsm.begin() + (row + phi) * 2 * nc * nq + nc * nq);
    unrotate_face(nc, o.np, mortar_angle(o, I, plo, 1), lo.data());
    unrotate_face(nc, o.np, mortar_angle(o, I, phi, 0), hi.data());
    back_project(o, I.Bm_lo.data(), lo.data(), I.Bm_hi.data(), hi.data(), -1.0, Fm.data() + f * nc * nq, nc);
  }
}

/* ------------------------------ element operator ------------------------------ */

/* Outward face flux (times surface element) of element e on face (d, side). */
void face_flux(const Curved& o, const double* U, const double* grad, double t, long long e, int d, int side,
               const std::vector<double>* Fs, const std::vector<double>* Fm, double* Fout) {
  Id id = elem_id(o, e);
  int np = o.np, nq = np * np;
  long long nb = -1;
  double ang = 0.0;
  int kind = neighbour(o, id, d, side, &nb, &ang);
  if (kind == 2) {
    const std::vector<double>& src = id.blk == 0 ? *Fs : *Fm;
    const double* F = src.data() + ((long long)id.iz * o.ny + id.iy) * 5 * nq;
    for (int k = 0; k < 5 * nq; ++k) Fout[k] = F[k];
    return;
  }
  double sg = side ? 1.0 : -1.0;
  for (int b = 0; b < np; ++b)
    for (int a = 0; a < np; ++a) {
      int vn = face_node(o, d, side, a, b);
      double Ja[3], vg[3];
      node_Ja(o, e, d, vn, t, Ja);
      node_vg(o, e, vn, t, vg);
      double sJ = std::sqrt(Ja[0] * Ja[0] + Ja[1] * Ja[1] + Ja[2] * Ja[2]);
      double np_[3] = {Ja[0] / sJ, Ja[1] / sJ, Ja[2] / sJ};     /* unit normal along +xi^d */
      double nout[3] = {sg * np_[0], sg * np_[1], sg * np_[2]};
      double vgn = vg[0] * np_[0] + vg[1] * np_[1] + vg[2] * np_[2];
      double uin[5], uout[5], gin[15], gout[15];
      for (int v = 0; v < 5; ++v) uin[v] = U[(e * 5 + v) * o.nn + vn];
      bool wall = false;
      if (kind == 1) {
        boundary_state(o, e, vn, t, uin, nout, uout);
        wall = o.cyl;
        if (wall) vgn = 0.0;     /* the walls move tangentially */
      } else {
        int vnn = face_node(o, d, 1 - side, a, b);
        for (int v = 0; v < 5; ++v) uout[v] = U[(nb * 5 + v) * o.nn + vnn];
        rotate_state(ang, uout);
        if (grad) {
          for (int k = 0; k < 15; ++k) gout[k] = grad[(nb * 15 + k) * o.nn + vnn];
          rotate_grad(ang, gout);
        }
      }
      double f[5];
      if (side == 1) orc_riemann(o.p.riemann, uin, uout, np_, vgn, o.p.gamma, f);
      else orc_riemann(o.p.riemann, uout, uin, np_, vgn, o.p.gamma, f);
      for (int v = 0; v < 5; ++v) f[v] *= sg * sJ;
      if (grad && !wall) {
        for (int k = 0; k < 15; ++k) gin[k] = grad[(e * 15 + k) * o.nn + vn];
        if (kind == 1) for (int k = 0; k < 15; ++k) gout[k] = gin[k];
        double N[3] = {sg * Ja[0], sg * Ja[1], sg * Ja[2]}, fi[5], fo[5];
        viscous_dot(o, uin, gin, N, fi);
        viscous_dot(o, uout, gout, N, fo);
        for (int v = 0; v < 5; ++v) f[v] -= 0.5 * (fi[v] + fo[v]);
      }
      for (int v = 0; v < 5; ++v) Fout[v * nq + a + np * b] = f[v];
    }
}

/* Contravariant two-point volume flux of the split form (Sec. 3.1) along one reference
 * direction, between nodes a and b with metric vectors Ja_a, Ja_b (Ja^d at each node) and
 * normal grid speeds V_a = Ja_a . v^g, V_b (reading, the curvilinear form of Pirozzoli's
 * products): kind 0 the products of means of Pirozzoli's flux with the averaged metric
 * m = {{Ja}} in place of the unit normal and the averaged V in place of the normal grid
 * speed; kind 1 the central flux {{Ja . F(U) - V U}}.  For equal nodes both reduce to the
 * contravariant ALE flux Ja . F(U) - V U. */
void curved_two_point(int kind, const double* Ua, const double* Ub, const double* Jaa, const double* Jab,
                      double Va, double Vb, double gamma, double* F) {
  if (kind == 1) {
    double Fa[5], Fb[5];
    orc_euler_flux(Ua, Jaa, Va, gamma, Fa);
    orc_euler_flux(Ub, Jab, Vb, gamma, Fb);
    for (int v = 0; v < 5; ++v) F[v] = 0.5 * (Fa[v] + Fb[v]);
    return;
  }
  double m[3] = {0.5 * (Jaa[0] + Jab[0]), 0.5 * (Jaa[1] + Jab[1]), 0.5 * (Jaa[2] + Jab[2])};
  orc_two_point_flux(0, Ua, Ub, m, 0.5 * (Va + Vb), gamma, F);
}

/* Split-form residual of a curved element (Sec. 3.1, the split formulation with Pirozzoli's
 * flux), strong form:
 *   J dU/dt = - sum_d sum_l 2 D_il F~#^d(U_node, U_l)  - sum_faces ell(+-1)/w (F* . N sJ - F~^d(U_node)) ,
 * F~^d(U) = Ja^d . F(U) - (Ja^d . v^g) U the node's own contravariant flux.  Navier-Stokes
 * (grad given, the BR1 gradients): the viscous flux keeps the weak form of the weak-form
 * residual, + sum_d sum_l Dhat_il Ja^d . F^v(U_l, grad_l), and the face flux F* carries the
 * BR1 viscous mean (the node's own flux subtracted is the advective one only). */
void split_residual(const Curved& o, const double* U, const double* grad, double t, long long e,
                    const std::vector<double>* Fs, const std::vector<double>* Fm, double* Ut) {
  int np = o.np, nn = o.nn, nq = np * np;
  int kind = o.p.volume == 2 ? 1 : 0;
  std::vector<double> Ja(9 * nn), V(3 * nn);       /* Ja[(d*3 + c)*nn + nd], V[d*nn + nd] */
  for (int nd = 0; nd < nn; ++nd) {
    double vg[3];
    node_vg(o, e, nd, t, vg);
    for (int d = 0; d < 3; ++d) {
      double a[3];
      node_Ja(o, e, d, nd, t, a);
      for (int c = 0; c < 3; ++c) Ja[(d * 3 + c) * nn + nd] = a[c];
      V[d * nn + nd] = a[0] * vg[0] + a[1] * vg[1] + a[2] * vg[2];
    }
  }
  auto ja = [&](int d, int nd, double* out) { for (int c = 0; c < 3; ++c) out[c] = Ja[(d * 3 + c) * nn + nd]; };
  for (int k = 0; k < np; ++k)
    for (int j = 0; j < np; ++j)
      for (int i = 0; i < np; ++i) {
        int nd = node(o, i, j, k);
        double u[5], ul[5], f[5], acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * nn + nd];
        for (int d = 0; d < 3; ++d) {
          int row = d == 0 ? i : (d == 1 ? j : k);
          double Jn[3];
          ja(d, nd, Jn);
          for (int l = 0; l < np; ++l) {
            int nl = d == 0 ? node(o, l, j, k) : (d == 1 ? node(o, i, l, k) : node(o, i, j, l));
            double Jl[3];
            ja(d, nl, Jl);
            for (int v = 0; v < 5; ++v) ul[v] = U[(e * 5 + v) * nn + nl];
            curved_two_point(kind, u, ul, Jn, Jl, V[d * nn + nd], V[d * nn + nl], o.p.gamma, f);
            for (int v = 0; v < 5; ++v) acc[v] += 2.0 * o.D[row * np + l] * f[v];
          }
        }
        for (int v = 0; v < 5; ++v) Ut[v * nn + nd] = -acc[v];
      }
  if (grad) {
    std::vector<double> Gt(15 * nn);         /* Ja^d . F^v, [(d*5 + v)*nn + nd] */
    for (int nd = 0; nd < nn; ++nd) {
      double u[5], g15[15], Fv[15];
      for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * nn + nd];
      for (int k = 0; k < 15; ++k) g15[k] = grad[(e * 15 + k) * nn + nd];
      orc_viscous_flux(u, g15, o.p.mu, o.p.Pr, o.p.Rgas, o.p.gamma, Fv);
      for (int d = 0; d < 3; ++d) {
        double a[3];
        ja(d, nd, a);
        for (int v = 0; v < 5; ++v) Gt[(d * 5 + v) * nn + nd] = a[0] * Fv[v] + a[1] * Fv[5 + v] + a[2] * Fv[10 + v];
      }
    }
    for (int v = 0; v < 5; ++v)
      for (int k = 0; k < np; ++k)
        for (int j = 0; j < np; ++j)
          for (int i = 0; i < np; ++i) {
            double acc = 0.0;
            for (int l = 0; l < np; ++l) {
              acc += o.Dhat[i * np + l] * Gt[(0 * 5 + v) * nn + node(o, l, j, k)];
              acc += o.Dhat[j * np + l] * Gt[(1 * 5 + v) * nn + node(o, i, l, k)];
              acc += o.Dhat[k * np + l] * Gt[(2 * 5 + v) * nn + node(o, i, j, l)];
            }
            Ut[v * nn + node(o, i, j, k)] += acc;
          }
  }
  std::vector<double> Fout(5 * nq);
  for (int d = 0; d < 3; ++d)
    for (int side = 0; side < 2; ++side) {
      face_flux(o, U, grad, t, e, d, side, Fs, Fm, Fout.data());
      double wend = o.w[side ? o.N : 0], sg = side ? 1.0 : -1.0;
      for (int b = 0; b < np; ++b)
        for (int a = 0; a < np; ++a) {
          int nd = face_node(o, d, side, a, b);
          double u[5], Jn[3], f[5];
          for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * nn + nd];
          ja(d, nd, Jn);
          orc_euler_flux(u, Jn, V[d * nn + nd], o.p.gamma, f);
          for (int v = 0; v < 5; ++v) Ut[v * nn + nd] -= (Fout[v * nq + a + np * b] - sg * f[v]) / wend;
        }
    }
  for (int v = 0; v < 5; ++v)
    for (int nd = 0; nd < nn; ++nd) Ut[v * nn + nd] /= o.J0[e * nn + nd];
}

void residual(const Curved& o, const double* U, const double* grad, double t, long long e,
              const std::vector<double>* Fs, const std::vector<double>* Fm, double* Ut) {
  if (o.p.volume != 0) {
    split_residual(o, U, grad, t, e, Fs, Fm, Ut);
    return;
  }
  int np = o.np, nn = o.nn, nq = np * np;
  std::vector<double> Ft(15 * nn);
  for (int nd = 0; nd < nn; ++nd) {
    double u[5], vg[3], F[3][5], Fv[15];
    for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * nn + nd];
    node_vg(o, e, nd, t, vg);
    for (int a = 0; a < 3; ++a) {
      double n[3] = {0, 0, 0};
      n[a] = 1.0;
      orc_euler_flux(u, n, vg[a], o.p.gamma, F[a]);
    }
    if (grad) {
      double g15[15];
      for (int k = 0; k < 15; ++k) g15[k] = grad[(e * 15 + k) * nn + nd];
      orc_viscous_flux(u, g15, o.p.mu, o.p.Pr, o.p.Rgas, o.p.gamma, Fv);
      for (int a = 0; a < 3; ++a)
        for (int v = 0; v < 5; ++v) F[a][v] -= Fv[a * 5 + v];
    }
    for (int i = 0; i < 3; ++i) {
      double Ja[3];
      node_Ja(o, e, i, nd, t, Ja);
      for (int v = 0; v < 5; ++v) Ft[(i * 5 + v) * nn + nd] = Ja[0] * F[0][v] + Ja[1] * F[1][v] + Ja[2] * F[2][v];
    }
  }
  for (int v = 0; v < 5; ++v)
    for (int k = 0; k < np; ++k)
      for (int j = 0; j < np; ++j)
        for (int i = 0; i < np; ++i) {
          double acc = 0.0;
          for (int l = 0; l < np; ++l) {
            acc += o.Dhat[i * np + l] * Ft[(0 * 5 + v) * nn + node(o, l, j, k)];
            acc += o.Dhat[j * np + l] * Ft[(1 * 5 + v) * nn + node(o, i, l, k)];
            acc += o.Dhat[k * np + l] * Ft[(2 * 5 + v) * nn + node(o, i, j, l)];
          }
          Ut[v * nn + node(o, i, j, k)] = -acc;
        }
  std::vector<double> Fout(5 * nq);
  for (int d = 0; d < 3; ++d)
    for (int side = 0; side < 2; ++side) {
      face_flux(o, U, grad, t, e, d, side, Fs, Fm, Fout.data());
      double wend = o.w[side ? o.N : 0];
      for (int v = 0; v < 5; ++v)
        for (int b = 0; b < np; ++b)
          for (int a = 0; a < np; ++a) Ut[v * nn + face_node(o, d, side, a, b)] -= Fout[v * nq + a + np * b] / wend;
    }
  for (int v = 0; v < 5; ++v)
    for (int nd = 0; nd < nn; ++nd) Ut[v * nn + nd] /= o.J0[e * nn + nd];
}

/* BR1 lifting with metrics: grad_a q = (1/J) [ sum_i Dhat_i (Ja^i_a q) + sum_faces q* N_a / w ]. */
void lifting(const Curved& o, const Iface& I, const double* U, double t, double* grad) {
  int np = o.np, nn = o.nn, nq = np * np;
  std::vector<double> Ls, Lm;
  if (!o.p.interface_conforming) all_interface(o, I, U, nullptr, t, 1, Ls, Lm);
  #pragma omp parallel for schedule(static)
  for (long long e = 0; e < o.E; ++e) {
    Id id = elem_id(o, e);
    std::vector<double> Q(5 * nn), Gt(15 * nn);
    for (int nd = 0; nd < nn; ++nd) {
      double u[5], q[5];
      for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * nn + nd];
      cons_to_prim(u, o.p.gamma, q);
      for (int v = 0; v < 5; ++v) Q[v * nn + nd] = q[v];
    }
    double* g = grad + e * 15 * nn;
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 5; ++c)
        for (int k = 0; k < np; ++k)
          for (int j = 0; j < np; ++j)
            for (int i = 0; i < np; ++i) {
              double acc = 0.0;
              for (int l = 0; l < np; ++l) {
                int n1 = node(o, l, j, k), n2 = node(o, i, l, k), n3 = node(o, i, j, l);
                double J1[3], J2[3], J3[3];
                node_Ja(o, e, 0, n1, t, J1);
                node_Ja(o, e, 1, n2, t, J2);
                node_Ja(o, e, 2, n3, t, J3);
                acc += o.Dhat[i * np + l] * J1[a] * Q[c * nn + n1];
                acc += o.Dhat[j * np + l] * J2[a] * Q[c * nn + n2];
                acc += o.Dhat[k * np + l] * J3[a] * Q[c * nn + n3];
              }
              g[(a * 5 + c) * nn + node(o, i, j, k)] = acc;
            }
    for (int d = 0; d < 3; ++d)
      for (int side = 0; side < 2; ++side) {
        long long nb = -1;
        double ang = 0.0;
        int kind = neighbour(o, id, d, side, &nb, &ang);
        double wend = o.w[side ? o.N : 0], sg = side ? 1.0 : -1.0;
        for (int b = 0; b < np; ++b)
          for (int aa = 0; aa < np; ++aa) {
            int vn = face_node(o, d, side, aa, b);
            double L[15];
            if (kind == 2) {
              const std::vector<double>& S = id.blk == 0 ? Ls : Lm;
              long long f = (long long)id.iz * o.ny + id.iy;
              for (int k = 0; k < 15; ++k) L[k] = S[(f * 15 + k) * nq + aa + np * b];
            } else {
              double Ja[3];
              node_Ja(o, e, d, vn, t, Ja);
              double N[3] = {sg * Ja[0], sg * Ja[1], sg * Ja[2]};
              double uo[5], qo[5];
              if (kind == 1) {
                double sJ = std::sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
                double nout[3] = {N[0] / sJ, N[1] / sJ, N[2] / sJ}, uin[5];
                for (int v = 0; v < 5; ++v) uin[v] = U[(e * 5 + v) * nn + vn];
                boundary_state(o, e, vn, t, uin, nout, uo);
              } else {
                int vnn = face_node(o, d, 1 - side, aa, b);
                for (int v = 0; v < 5; ++v) uo[v] = U[(nb * 5 + v) * nn + vnn];
                rotate_state(ang, uo);
              }
              cons_to_prim(uo, o.p.gamma, qo);
              for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 5; ++c) L[a * 5 + c] = 0.5 * (Q[c * nn + vn] + qo[c]) * N[a];
            }
            for (int k = 0; k < 15; ++k) g[k * nn + vn] += L[k] / wend;
          }
      }
    for (int k = 0; k < 15; ++k)
      for (int nd = 0; nd < nn; ++nd) g[k * nn + nd] /= o.J0[e * nn + nd];
  }
}

}  // namespace

/* ---- entry points used by dg_oracle.cpp's dispatch ---- */
void* orc_curved_create(const orc_problem* p) {
  if (p->N < 1 || p->N > 15) return nullptr;
  if (p->nel_s[1] != p->nel_m[1] || p->nel_s[2] != p->nel_m[2]) return nullptr;
  Curved* o = new Curved();
  o->p = *p;
  o->N = p->N; o->np = p->N + 1; o->nn = o->np * o->np * o->np;
  o->ny = p->nel_s[1]; o->nz = p->nel_s[2];
  o->Es = (long long)p->nel_s[0] * o->ny * o->nz;
  o->Em = (long long)p->nel_m[0] * o->ny * o->nz;
  o->E = o->Es + o->Em;
  if (p->geom < 1 || p->geom > 4) { delete o; return nullptr; }
  o->cyl = p->geom == 1 || p->geom == 3 || p->geom == 4;
  o->annular = p->geom == 3;
  o->cone = p->geom == 4;
  o->sa = std::sin(p->cone_angle);
  o->ca = std::cos(p->cone_angle);
  o->ns = p->physics == 1;
  o->h1 = (p->y1 - p->y0) / o->ny;
  o->h2 = (p->z1 - p->z0) / o->nz;
  o->h3[0] = (p->x1 - p->x0) / p->nel_s[0];
  o->h3[1] = (p->x2 - p->x1) / p->nel_m[0];
  o->Theta = p->y1 - p->y0;
  o->x.resize(o->np); o->w.resize(o->np);
  orc_lgl(o->N, o->x.data(), o->w.data());
  o->D.resize(o->np * o->np); o->Dhat.resize(o->np * o->np);
  orc_dmatrix(o->N, o->x.data(), o->D.data());
  for (int i = 0; i < o->np; ++i)
    for (int l = 0; l < o->np; ++l) o->Dhat[i * o->np + l] = -(o->w[l] / o->w[i]) * o->D[l * o->np + i];
  orc_lsrk_coeffs(o->A, o->B, o->c);
  build_geometry(*o);
  return o;
}

void orc_curved_destroy(void* h) { delete (Curved*)h; }
long long orc_curved_nelem(void* h) { return ((Curved*)h)->E; }

void orc_curved_coords(void* h, double t, double* xyz) {
  Curved& o = *(Curved*)h;
  for (long long e = 0; e < o.E; ++e)
    for (int nd = 0; nd < o.nn; ++nd) {
      double X[3];
      node_X(o, e, nd, t, X);
      for (int a = 0; a < 3; ++a) xyz[(e * 3 + a) * o.nn + nd] = X[a];
    }
}

void orc_curved_fill(void* h, double t, double* U) {
  Curved& o = *(Curved*)h;
  for (long long e = 0; e < o.E; ++e)
    for (int nd = 0; nd < o.nn; ++nd) {
      double X[3], u[5];
      node_X(o, e, nd, t, X);
      orc_flow_state(&o.p, X, t, 0, u);
      for (int v = 0; v < 5; ++v) U[(e * 5 + v) * o.nn + nd] = u[v];
    }
}

void orc_curved_metrics(void* h, double t, double* Ja, double* J) {
  Curved& o = *(Curved*)h;
  for (long long e = 0; e < o.E; ++e)
    for (int nd = 0; nd < o.nn; ++nd) {
      for (int i = 0; i < 3; ++i) {
        double v[3];
        node_Ja(o, e, i, nd, t, v);
        for (int n = 0; n < 3; ++n) Ja[((e * 3 + i) * 3 + n) * o.nn + nd] = v[n];
      }
      J[e * o.nn + nd] = o.J0[e * o.nn + nd];
    }
}

void orc_curved_lifting(void* h, const double* U, double t, double* grad) {
  Curved& o = *(Curved*)h;
  Iface I;
  iface_config(o, t, I);
  lifting(o, I, U, t, grad);
}

void orc_curved_interface(void* h, const double* U, double t, double* Fs_out, double* Fm_out) {
  Curved& o = *(Curved*)h;
  Iface I;
  iface_config(o, t, I);
  std::vector<double> grad;
  if (o.ns) { grad.assign(o.E * 15 * o.nn, 0.0); lifting(o, I, U, t, grad.data()); }
  std::vector<double> Fs, Fm;
  all_interface(o, I, U, o.ns ? grad.data() : nullptr, t, 0, Fs, Fm);
  std::memcpy(Fs_out, Fs.data(), sizeof(double) * Fs.size());
  std::memcpy(Fm_out, Fm.data(), sizeof(double) * Fm.size());
}

void orc_curved_rhs(void* h, const double* U, double t, const long long* elems, int count, double* Ut) {
  Curved& o = *(Curved*)h;
  Iface I;
  iface_config(o, t, I);
  std::vector<double> grad;
  if (o.ns) { grad.assign(o.E * 15 * o.nn, 0.0); lifting(o, I, U, t, grad.data()); }
  const double* g = o.ns ? grad.data() : nullptr;
  std::vector<double> Fs, Fm;
  if (!o.p.interface_conforming) all_interface(o, I, U, g, t, 0, Fs, Fm);
  long long n = elems ? count : o.E;
  #pragma omp parallel for schedule(dynamic)
  for (long long m = 0; m < n; ++m)
    residual(o, U, g, t, elems ? elems[m] : m, &Fs, &Fm, Ut + m * 5 * o.nn);
}

void orc_curved_step(void* h, double* U, double* G, double* t, double dt, int nsteps) {
  Curved& o = *(Curved*)h;
  long long ndof = o.E * 5 * o.nn;
  std::vector<double> Ut(ndof);
  for (int s = 0; s < nsteps; ++s) {
    for (int k = 0; k < 5; ++k) {
      orc_curved_rhs(h, U, std::fma(o.c[k], dt, *t), nullptr, 0, Ut.data());
      for (long long m = 0; m < ndof; ++m) {
        G[m] = (k == 0) ? dt * Ut[m] : o.A[k] * G[m] + dt * Ut[m];
        U[m] = U[m] + o.B[k] * G[m];
      }
    }
    *t = *t + dt;
  }
}

void orc_curved_totals(void* h, const double* U, double* tot5) {
  Curved& o = *(Curved*)h;
  for (int v = 0; v < 5; ++v) tot5[v] = 0.0;
  for (long long e = 0; e < o.E; ++e)
    for (int k = 0; k < o.np; ++k)
      for (int j = 0; j < o.np; ++j)
        for (int i = 0; i < o.np; ++i) {
          int nd = node(o, i, j, k);
          double wq = o.J0[e * o.nn + nd] * o.w[i] * o.w[j] * o.w[k];
          for (int v = 0; v < 5; ++v) tot5[v] += wq * U[(e * 5 + v) * o.nn + nd];
        }
}

double orc_curved_l2_error_rho(void* h, const double* U, double t) {
  Curved& o = *(Curved*)h;
  std::vector<double> Ue(o.E * 5 * o.nn);
  orc_curved_fill(h, t, Ue.data());
  double err = 0.0, vol = 0.0;
  for (long long e = 0; e < o.E; ++e)
    for (int k = 0; k < o.np; ++k)
      for (int j = 0; j < o.np; ++j)
        for (int i = 0; i < o.np; ++i) {
          int nd = node(o, i, j, k);
          double wq = o.J0[e * o.nn + nd] * o.w[i] * o.w[j] * o.w[k];
          double d = U[e * 5 * o.nn + nd] - Ue[e * 5 * o.nn + nd];
          err += wq * d * d;
          vol += wq;
        }
  return std::sqrt(err / vol);
}

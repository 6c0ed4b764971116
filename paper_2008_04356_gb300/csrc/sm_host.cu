// Host side of the C-ABI (include/slidemesh.h): solver set-up, stage sequencing and CUDA
// graph replay of whole Runge-Kutta steps.
//
// Per step of a single solve (Carpenter-Kennedy five-stage RK4, Sec. 3.1): one step_params
// launch builds, for all five stages k, t_k = fma(c_k, dt, t), Delta(t_k), (n, s) and the
// mortar operators (Sec. 4.3, 3.2); then per stage k
//   1. sliding_interface: both sides' interface face fluxes (Sec. 3.3 steps 3-5)
//   2. dg_element: volume + surface integral and G = A_k G + dt R, U' = U + B_k G.
// Batched solves take one stage_params launch per stage over the group.
// U ping-pongs between two buffers because neighbour traces are read from the state of the
// previous stage while the element kernel writes the new one.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/slidemesh.h"
#include "sm_launch.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* what, cudaError_t e = cudaSuccess) {
  char buf[512];
  if (e != cudaSuccess)
    snprintf(buf, sizeof(buf), "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  else
    snprintf(buf, sizeof(buf), "%s", what);
  g_last_error = buf;
  return code;
}

#define SM_CK(call, what)                                          \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return fail(SM_ERR_CUDA, what, e_);     \
  } while (0)

// Legendre polynomial P_n and derivative (three-term recurrence).
void legendre_pd(int n, double x, double* p, double* dp) {
  double a = 1.0, b = x, da = 0.0, db = 1.0;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
    double dc = k * b + x * db;   // P_k' = k P_{k-1} + x P_{k-1}'
    a = b; b = c; da = db; db = dc;
  }
  (void)da;
  *p = b;
  *dp = db;
}

// LGL nodes: the N+1 roots of q(x) = P_{N+1}(x) - P_{N-1}(x) (which vanishes at +-1 and at
// the roots of P_N'), found by Newton from Chebyshev-Gauss-Lobatto points, symmetrised.
void lgl_basis(int N, BasisDev& b) {
  memset(&b, 0, sizeof(b));
  const int np = N + 1;
  for (int j = 0; j < np; ++j) {
    double x = -cos(M_PI * j / N);
    for (int it = 0; it < 60; ++it) {
      double p1, d1, p0, d0;
      legendre_pd(N + 1, x, &p1, &d1);
      legendre_pd(N - 1, x, &p0, &d0);
      double dx = (p1 - p0) / (d1 - d0);
      x -= dx;
      if (fabs(dx) < 1e-17) break;
    }
    b.x[j] = x;
  }
  for (int j = 0; j < np / 2; ++j) {
    double a = 0.5 * (b.x[N - j] - b.x[j]);
    b.x[j] = -a;
    b.x[N - j] = a;
  }
  b.x[0] = -1.0;
  b.x[N] = 1.0;
  if (np % 2 == 1) b.x[N / 2] = 0.0;
  for (int j = 0; j < np; ++j) {
    double p, dp;
    legendre_pd(N, b.x[j], &p, &dp);
    b.w[j] = 2.0 / (N * (N + 1.0) * p * p);
  }
  for (int i = 0; i < np; ++i) {
    double prod = 1.0;
    for (int k = 0; k < np; ++k)
      if (k != i) prod *= (b.x[i] - b.x[k]);
    b.lam[i] = 1.0 / prod;
  }
  // exact mass matrix of the Lagrange basis, M = V^-T diag(2/(2k+1)) V^-1 and its inverse
  // M^-1 = V diag((2k+1)/2) V^T, with the Legendre Vandermonde V_ik = P_k(x_i)
  double V[SM_MAXNP][SM_MAXNP], Vi[SM_MAXNP][SM_MAXNP];
  for (int i = 0; i < np; ++i)
    for (int k = 0; k < np; ++k) {
      double p, dp;
      legendre_pd(k, b.x[i], &p, &dp);
      V[i][k] = p;
    }
  // invert V (Gauss-Jordan, partial pivoting)
  double A[SM_MAXNP][2 * SM_MAXNP];
  for (int i = 0; i < np; ++i)
    for (int k = 0; k < 2 * np; ++k) A[i][k] = k < np ? V[i][k] : (k - np == i ? 1.0 : 0.0);
  for (int c = 0; c < np; ++c) {
    int piv = c;
    for (int r = c + 1; r < np; ++r)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    for (int k = 0; k < 2 * np; ++k) { double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
    double d = A[c][c];
    for (int k = 0; k < 2 * np; ++k) A[c][k] /= d;
    for (int r = 0; r < np; ++r)
      if (r != c) {
        double f = A[r][c];
        for (int k = 0; k < 2 * np; ++k) A[r][k] -= f * A[c][k];
      }
  }
  for (int i = 0; i < np; ++i)
    for (int k = 0; k < np; ++k) Vi[i][k] = A[i][np + k];
  for (int i = 0; i < np; ++i)
    for (int j = 0; j < np; ++j) {
      double m = 0.0, mi = 0.0;
      for (int k = 0; k < np; ++k) {
        m += Vi[k][i] * (2.0 / (2 * k + 1)) * Vi[k][j];
        mi += V[i][k] * ((2 * k + 1) / 2.0) * V[j][k];
      }
      b.M[i * SM_MAXNP + j] = m;
      b.Minv[i * SM_MAXNP + j] = mi;
    }
  // D_ij = ell_j'(x_i) from barycentric weights; Dhat_il = -(w_l / w_i) D_li
  double D[SM_MAXNP][SM_MAXNP];
  for (int i = 0; i < np; ++i) {
    double diag = 0.0;
    for (int j = 0; j < np; ++j)
      if (j != i) {
        D[i][j] = (b.lam[j] / b.lam[i]) / (b.x[i] - b.x[j]);
        diag -= D[i][j];
      }
    D[i][i] = diag;
  }
  for (int i = 0; i < np; ++i)
    for (int l = 0; l < np; ++l) {
      double dh = -(b.w[l] / b.w[i]) * D[l][i];
      b.Dhat[i * SM_MAXNP + l] = dh;
      b.Dhat_f[i * SM_MAXNP + l] = (float)dh;
    }
  // split form: Ds = 2 D - M^-1 B with the LGL weights, zero on the diagonal (D_ii = 0 at the
  // interior nodes of the symmetric LGL set, 2 D_00 = -1/w_0 and 2 D_NN = 1/w_N at the ends)
  for (int i = 0; i < np; ++i)
    for (int l = 0; l < np; ++l) b.Dsplit[i * SM_MAXNP + l] = i == l ? 0.0 : 2.0 * D[i][l];
  for (int j = 0; j < np; ++j) {
    b.x_f[j] = (float)b.x[j];
    b.w_f[j] = (float)b.w[j];
  }
}

// Carpenter & Kennedy (1994), five-stage fourth-order 2N-storage scheme.
const double RK_A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double RK_B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};
const double RK_C[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                        2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

// Curvilinear geometry at t = 0 for MeshDev::geom 1 and 2: node coordinates of the analytic
// map (cylinder: (r cos theta, r sin theta, z) with xi^1 -> theta, xi^2 -> z, xi^3 -> r;
// plane: xi^1 -> y, xi^2 -> z, xi^3 -> x; relative to the element's centre), the Jacobian
// J = a_1 . (a_2 x a_3) with
// a_d = D_d X, and the metric terms in Kopriva's conservative curl form, antisymmetrised,
//   Ja^i_n = -1/2 (D_j V_k - D_k V_j),  V_k = X_l D_k X_m - X_m D_k X_l,
// (i, j, k) and (n, m, l) cyclic: the discrete metric identities sum_i D_i Ja^i_n = 0 hold
// and the form commutes with a rotation of the mesh.  Per node 13 values: Ja^i_n (3 i + n),
// J (9), Ja^i . v^g / |v| of the moving block (10 + i; the rotor's v^g / omega = e_z x X,
// the plane's v^g / v = e_y).
void curvilinear_geometry(const MeshDev& m, const BasisDev& b, int N, std::vector<double>& geo) {
  const int np = N + 1, nn = np * np * np;
  double D[SM_MAXNP][SM_MAXNP];
  for (int i = 0; i < np; ++i) {
    double diag = 0.0;
    for (int j = 0; j < np; ++j)
      if (j != i) {
        D[i][j] = (b.lam[j] / b.lam[i]) / (b.x[i] - b.x[j]);
        diag -= D[i][j];
      }
    D[i][i] = diag;
  }
  auto idx = [np](int i, int j, int k) { return i + np * (j + np * k); };
  // derivative along reference direction d of nodal data f
  auto deriv = [&](int d, const double* f, double* out) {
    for (int k = 0; k < np; ++k)
      for (int j = 0; j < np; ++j)
        for (int i = 0; i < np; ++i) {
          double acc = 0.0;
          for (int l = 0; l < np; ++l) {
            const int row = d == 0 ? i : (d == 1 ? j : k);
            const int src = d == 0 ? idx(l, j, k) : (d == 1 ? idx(i, l, k) : idx(i, j, l));
            acc += D[row][l] * f[src];
          }
          out[idx(i, j, k)] = acc;
        }
  };
  geo.assign((size_t)m.E * 13 * nn, 0.0);
  std::vector<double> X(3 * nn), dX(9 * nn), V(3 * nn), T1(nn), T2(nn);
  for (long long e = 0; e < m.E; ++e) {
    const ElemPos p = decode_elem(m, e);
    const double h3 = p.blk ? m.hx1 : m.hx0, lo3 = p.blk ? m.x1 : m.x0;
    for (int k = 0; k < np; ++k)
      for (int j = 0; j < np; ++j)
        for (int i = 0; i < np; ++i) {
          const double s1 = m.y0 + p.iy * m.hy + (b.x[i] + 1.0) * 0.5 * m.hy;
          const double s2 = m.z0 + p.iz * m.hz + (b.x[j] + 1.0) * 0.5 * m.hz;
          const double s3 = lo3 + p.ix * h3 + (b.x[k] + 1.0) * 0.5 * h3;
          const int q = idx(i, j, k);
          if (m.geom == 4) {        // cone: (theta, s along the generator, n across)
            const double r = s2 * m.cone_s + s3 * m.cone_c;
            X[q] = r * cos(s1);
            X[nn + q] = r * sin(s1);
            X[2 * nn + q] = s2 * m.cone_c - s3 * m.cone_s;
            continue;
          }
          if (m.geom == 3) {        // annular: (theta, r from z1 down to z0, z), right-handed
            const double r = 2.0 * m.z0 + m.nz * m.hz - s2;
            X[q] = r * cos(s1);
            X[nn + q] = r * sin(s1);
            X[2 * nn + q] = s3;
            continue;
          }
          if (m.geom == 1) {
            X[q] = s3 * cos(s1);
            X[nn + q] = s3 * sin(s1);
          } else {
            X[q] = s3;
            X[nn + q] = s1;
          }
          X[2 * nn + q] = s2;
        }
    // the curl form is translation invariant: evaluate it on coordinates relative to the
    // element's centre so that its products do not cancel digits
    double Xc[3];
    {
      const double s1 = m.y0 + (p.iy + 0.5) * m.hy, s2 = m.z0 + (p.iz + 0.5) * m.hz, s3 = lo3 + (p.ix + 0.5) * h3;
      const double rc = 2.0 * m.z0 + m.nz * m.hz - s2;
      Xc[0] = m.geom == 3 ? rc * cos(s1) : (m.geom == 1 ? s3 * cos(s1) : s3);
      Xc[1] = m.geom == 3 ? rc * sin(s1) : (m.geom == 1 ? s3 * sin(s1) : s1);
      Xc[2] = m.geom == 3 ? s3 : s2;
      if (m.geom == 4) {
        const double rk = s2 * m.cone_s + s3 * m.cone_c;
        Xc[0] = rk * cos(s1);
        Xc[1] = rk * sin(s1);
        Xc[2] = s2 * m.cone_c - s3 * m.cone_s;
      }
    }
    std::vector<double> Xg(X);   // global coordinates for the grid-velocity factors
    for (int c = 0; c < 3; ++c)
      for (int q = 0; q < nn; ++q) X[c * nn + q] -= Xc[c];
    for (int d = 0; d < 3; ++d)
      for (int c = 0; c < 3; ++c) deriv(d, &X[c * nn], &dX[(d * 3 + c) * nn]);
    double* g = &geo[(size_t)e * 13 * nn];
    for (int q = 0; q < nn; ++q) {
      const double* a1 = &dX[0]; const double* a2 = &dX[3 * nn]; const double* a3 = &dX[6 * nn];
      const double c0 = a2[nn + q] * a3[2 * nn + q] - a2[2 * nn + q] * a3[nn + q];
      const double c1 = a2[2 * nn + q] * a3[q] - a2[q] * a3[2 * nn + q];
      const double c2 = a2[q] * a3[nn + q] - a2[nn + q] * a3[q];
      g[9 * nn + q] = a1[q] * c0 + a1[nn + q] * c1 + a1[2 * nn + q] * c2;
    }
    for (int n = 0; n < 3; ++n) {
      const int mm = (n + 1) % 3, l = (n + 2) % 3;
      for (int k = 0; k < 3; ++k)
        for (int q = 0; q < nn; ++q)
          V[k * nn + q] = X[l * nn + q] * dX[(k * 3 + mm) * nn + q] - X[mm * nn + q] * dX[(k * 3 + l) * nn + q];
      for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3, k = (i + 2) % 3;
        deriv(j, &V[k * nn], T1.data());
        deriv(k, &V[j * nn], T2.data());
        for (int q = 0; q < nn; ++q) g[(3 * i + n) * nn + q] = -0.5 * (T1[q] - T2[q]);
      }
    }
    const bool moving = rotating_geom(m.geom) ? p.blk == 0 : p.blk == 1;
    if (moving)
      for (int i = 0; i < 3; ++i)
        for (int q = 0; q < nn; ++q)
          g[(10 + i) * nn + q] = rotating_geom(m.geom) ? -Xg[nn + q] * g[(3 * i) * nn + q] + Xg[q] * g[(3 * i + 1) * nn + q]
                                            : g[(3 * i + 1) * nn + q];
  }
}

// Fills the per-precision constant block of the kernels (FP64 values, rounded once for FP32).
void fill_constants(MeshDev& m, const BasisDev& b, const double* fpar) {
  double c[MC_COUNT] = {0};
  const double hx[2] = {m.hx0, m.hx1};
  for (int blk = 0; blk < 2; ++blk) {
    c[MC_METRIC + 3 * blk + 0] = m.hz * hx[blk] * 0.25;
    c[MC_METRIC + 3 * blk + 1] = hx[blk] * m.hy * 0.25;
    c[MC_METRIC + 3 * blk + 2] = m.hy * m.hz * 0.25;
    c[MC_MINVJ + blk] = -1.0 / (hx[blk] * m.hy * m.hz * 0.125);
  }
  c[MC_VG] = m.v;
  c[MC_GAMMA] = m.gamma;
  c[MC_IW0] = 1.0 / b.w[0];
  c[MC_SJ_IF] = m.hy * m.hz * 0.25;
  const double* P = fpar;   // background primitive state of flows 0 and 2
  c[MC_BC + 0] = P[0];
  c[MC_BC + 1] = P[0] * P[1];
  c[MC_BC + 2] = P[0] * P[2];
  c[MC_BC + 3] = P[0] * P[3];
  c[MC_BC + 4] = P[4] / (m.gamma - 1.0) + 0.5 * P[0] * (P[1] * P[1] + P[2] * P[2] + P[3] * P[3]);
  c[MC_H + 0] = m.hx0;
  c[MC_H + 1] = m.hx1;
  c[MC_H + 2] = m.hy;
  c[MC_H + 3] = m.hz;
  c[MC_X + 0] = m.x0;
  c[MC_X + 1] = m.x1;
  c[MC_X + 2] = m.y0;
  c[MC_X + 3] = m.z0;
  c[MC_MU] = m.mu;
  c[MC_R] = m.Rgas;
  c[MC_K] = m.Pr > 0.0 ? m.mu * m.gamma * m.Rgas / ((m.gamma - 1.0) * m.Pr) : 0.0;
  c[MC_PCOS] = cos(m.Theta);
  c[MC_PSIN] = sin(m.Theta);
  for (int k = 0; k < MC_COUNT; ++k) {
    m.cd[k] = c[k];
    m.cf[k] = (float)c[k];
  }
  for (int k = 0; k < 16; ++k) m.fparf[k] = (float)fpar[k];
}

// Once per device: the Dhat tables of every degree in each element-kernel unit's constant
// memory.
std::mutex g_dhat_mu;
bool g_dhat_done[256] = {false};

cudaError_t ensure_dhat_constants() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_dhat_mu);
  if (g_dhat_done[dev]) return cudaSuccess;
  static float f[7][SM_MAXNP * SM_MAXNP], fs[7][SM_MAXNP * SM_MAXNP];
  static double d[7][SM_MAXNP * SM_MAXNP], ds[7][SM_MAXNP * SM_MAXNP];
  for (int n = 1; n <= 7; ++n) {
    BasisDev b;
    lgl_basis(n, b);
    for (int k = 0; k < SM_MAXNP * SM_MAXNP; ++k) {
      d[n - 1][k] = b.Dhat[k];
      f[n - 1][k] = b.Dhat_f[k];
      ds[n - 1][k] = b.Dsplit[k];
      fs[n - 1][k] = (float)b.Dsplit[k];
    }
  }
  if ((e = upload_split_ns_constants_f32(&f[0][0], &d[0][0], &fs[0][0], &ds[0][0])) != cudaSuccess) return e;
  if ((e = upload_split_ns_constants_f64(&f[0][0], &d[0][0], &fs[0][0], &ds[0][0])) != cudaSuccess) return e;
  if ((e = upload_dsplit_f32(&fs[0][0], &ds[0][0])) != cudaSuccess) return e;
  if ((e = upload_dsplit_f64(&fs[0][0], &ds[0][0])) != cudaSuccess) return e;
  if ((e = upload_dhat_f32(&f[0][0], &d[0][0])) != cudaSuccess) return e;
  if ((e = upload_dhat_f64(&f[0][0], &d[0][0])) != cudaSuccess) return e;
  if ((e = upload_dhat_batch(&f[0][0], &d[0][0])) != cudaSuccess) return e;
  if ((e = upload_dhat_ns_f32(&f[0][0], &d[0][0])) != cudaSuccess) return e;
  if ((e = upload_dhat_ns_f64(&f[0][0], &d[0][0])) != cudaSuccess) return e;
  if ((e = upload_dhat_curved_f32(&f[0][0], &d[0][0])) != cudaSuccess) return e;
  if ((e = upload_dhat_curved_f64(&f[0][0], &d[0][0])) != cudaSuccess) return e;
  if ((e = upload_dhat_curved_ns_f32(&f[0][0], &d[0][0])) != cudaSuccess) return e;
  if ((e = upload_dhat_curved_ns_f64(&f[0][0], &d[0][0])) != cudaSuccess) return e;
  if ((e = upload_dhat_curved_split_ns_f32(&f[0][0], &d[0][0])) != cudaSuccess) return e;
  if ((e = upload_dhat_curved_split_ns_f64(&f[0][0], &d[0][0])) != cudaSuccess) return e;
  g_dhat_done[dev] = true;
  return cudaSuccess;
}

struct GraphEntry {
  double dt;
  int cur;
  cudaGraphExec_t exec;
};

}  // namespace

struct sm_solver {
  sm_mesh_desc desc;
  sm_motion motion;
  int N, np, prec, sb;
  long long nn, nstate, nface_vals;
  MeshDev m;
  BasisDev basis_h;
  BasisDev* basis_d = nullptr;
  double* modes_d = nullptr;
  void* U[2] = {nullptr, nullptr};
  void* G = nullptr;
  void* Fs = nullptr;
  void* Fm = nullptr;
  StageParams* sp = nullptr;   // five blocks: the stages of a step (block 0 for sm_rhs & co.)
  int sp_last = 0;              // the block of the last evaluated stage
  unsigned* ticket_d = nullptr; // counter of the step-parameter launch
  double* t_d = nullptr;
  double* red_d = nullptr;      // partial sums [nblk][5] + outputs [3][5]
  int4* topo_d = nullptr;       // per-element neighbour table (2 int4 per element)
  void* Gr = nullptr;           // lifted gradients [E][15][NN] (Navier-Stokes)
  void* Ls = nullptr;           // interface lifting face values, static side (Navier-Stokes)
  void* Lm = nullptr;           // ... moving side
  void* Ts = nullptr;           // interface traces of the current state (Euler, sliding interface)
  void* Tm = nullptr;
  void* Ts2 = nullptr;          // periodic x: traces and face fluxes of the second interface
  void* Tm2 = nullptr;          // (x-mirrored, see MeshDev)
  void* Fs2 = nullptr;
  void* Fm2 = nullptr;
  bool traces_ok = false;       // Ts / Tm hold the traces of U[cur]
  void* geo = nullptr;          // curvilinear geometry per node (MeshDev::geom != 0)
  int red_blocks = 0;
  int cur = 0;
  double t_host = 0.0;
  cudaStream_t cap = nullptr;
  std::vector<GraphEntry> graphs;
  // sm_stream_jobs: state-sized staging buffers, copy streams and their events (first call)
  void* stage_in = nullptr;
  void* stage_out = nullptr;
  double* t0_d = nullptr;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t in_ready = nullptr, in_free = nullptr, out_ready = nullptr, out_free = nullptr;
};

namespace {

bool is_ns(const sm_solver* s) { return s->desc.physics == SM_NAVIER_STOKES; }

// Caller device arrays are read and written with 8- and 16-byte vector accesses.
bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// After the stage parameters: everything the element kernel reads besides U.  Navier-Stokes:
// lifting face values on the interface, the lifted gradients, then the interface fluxes with
// their viscous part; Euler: the interface fluxes.
// from_traces: the interface kernel reads the compact traces Ts / Tm (of U[cur]) instead of U.
cudaError_t enqueue_flux_inputs(sm_solver* s, const StageParams* sp, const void* dU, void* Fs, void* Fm, cudaStream_t st,
                                bool from_traces = false) {
  cudaError_t e = cudaSuccess;
  const bool sliding = !s->desc.interface_conforming;
  if (is_ns(s) && s->m.geom != 0) {
    const bool f64 = s->prec == SM_FP64;
    if (sliding && (e = f64 ? launch_curved_interface_lift_f64(s->N, s->m, sp, dU, s->Ls, s->Lm, st)
                            : launch_curved_interface_lift_f32(s->N, s->m, sp, dU, s->Ls, s->Lm, st)) != cudaSuccess)
      return e;
    e = f64 ? launch_curved_lift_f64(s->N, s->m, sp, dU, s->Gr, s->Ls, s->Lm, st)
            : launch_curved_lift_f32(s->N, s->m, sp, dU, s->Gr, s->Ls, s->Lm, st);
    if (e != cudaSuccess || !sliding) return e;
    return f64 ? launch_curved_interface_ns_f64(s->N, s->desc.riemann, s->m, sp, dU, s->Gr, Fs, Fm, st)
               : launch_curved_interface_ns_f32(s->N, s->desc.riemann, s->m, sp, dU, s->Gr, Fs, Fm, st);
  }
  if (is_ns(s)) {
    if (sliding && (e = launch_interface_lift(s->N, s->prec, s->m, sp, dU, s->Ls, s->Lm, st)) != cudaSuccess) return e;
    e = s->prec == SM_FP64 ? launch_lift_f64(s->N, s->m, sp, dU, s->Gr, s->Ls, s->Lm, st)
                           : launch_lift_f32(s->N, s->m, sp, dU, s->Gr, s->Ls, s->Lm, st);
    if (e != cudaSuccess) return e;
    if (sliding) e = launch_interface_ns(s->N, s->prec, s->desc.riemann, s->m, sp, dU, s->Gr, Fs, Fm, st);
    return e;
  }
  if (sliding && s->m.geom != 0)
    return s->prec == SM_FP64 ? launch_curved_interface_f64(s->N, s->desc.riemann, s->m, sp, dU, Fs, Fm, st)
                              : launch_curved_interface_f32(s->N, s->desc.riemann, s->m, sp, dU, Fs, Fm, st);
  if (sliding)
    e = launch_interface(s->N, s->prec, s->desc.riemann, s->m, sp, dU, Fs, Fm, st, from_traces ? s->Ts : nullptr,
                         from_traces ? s->Tm : nullptr);
  if (e == cudaSuccess && sliding && s->m.Ts2) {
    // the second interface (periodic x), solved as the x-mirrored first one from its traces
    if (!from_traces) {
      e = launch_gather_traces(s->N, s->prec, s->m, dU, s->m.Ts2, s->m.Tm2, st, 1);
      s->traces_ok = false;           // Ts2 / Tm2 now hold the traces of dU
      if (e != cudaSuccess) return e;
    }
    e = launch_interface(s->N, s->prec, s->desc.riemann, s->m, sp, dU, const_cast<void*>(s->m.Fs2),
                         const_cast<void*>(s->m.Fm2), st, s->m.Ts2, s->m.Tm2);
  }
  return e;
}

// Stepping keeps the interface traces of the current state in Ts / Tm: each stage's element
// kernel writes those of the state it produces; after a new state they are gathered once.
bool use_traces(const sm_solver* s) { return s->Ts != nullptr; }

cudaError_t ensure_traces(sm_solver* s, cudaStream_t st) {
  if (!use_traces(s) || s->traces_ok) return cudaSuccess;
  cudaError_t e = launch_gather_traces(s->N, s->prec, s->m, s->U[s->cur], s->Ts, s->Tm, st);
  if (e == cudaSuccess && s->m.Ts2) e = launch_gather_traces(s->N, s->prec, s->m, s->U[s->cur], s->m.Ts2, s->m.Tm2, st, 1);
  if (e == cudaSuccess) s->traces_ok = true;
  return e;
}

cudaError_t enqueue_rhs_parts(sm_solver* s, double t, const void* dU, void* Fs, void* Fm, cudaStream_t st) {
  cudaError_t e = launch_stage_params(s->m, s->np, s->sp, s->t_d, t, 0.0, 0.0, 0, st);
  if (e != cudaSuccess) return e;
  s->sp_last = 0;
  return enqueue_flux_inputs(s, s->sp, dU, Fs, Fm, st);
}

cudaError_t launch_elem(sm_solver* s, int mode, const ElemArgs& a0, cudaStream_t st) {
  ElemArgs a = a0;
  if (s->m.geom != 0 && is_ns(s) && s->desc.volume == SM_VOLUME_SPLIT) {
    a.Gr = s->Gr;
    return s->prec == SM_FP64 ? launch_curved_split_ns_f64(s->N, s->desc.riemann, mode, a, st)
                              : launch_curved_split_ns_f32(s->N, s->desc.riemann, mode, a, st);
  }
  if (s->m.geom != 0 && is_ns(s)) {
    a.Gr = s->Gr;
    return s->prec == SM_FP64 ? launch_curved_element_ns_f64(s->N, s->desc.riemann, mode, a, st)
                              : launch_curved_element_ns_f32(s->N, s->desc.riemann, mode, a, st);
  }
  if (s->m.geom != 0 && s->desc.volume == SM_VOLUME_SPLIT)
    return s->prec == SM_FP64 ? launch_curved_split_f64(s->N, s->desc.riemann, mode, a, st)
                              : launch_curved_split_f32(s->N, s->desc.riemann, mode, a, st);
  if (s->m.geom != 0)
    return s->prec == SM_FP64 ? launch_curved_element_f64(s->N, s->desc.riemann, mode, a, st)
                              : launch_curved_element_f32(s->N, s->desc.riemann, mode, a, st);
  if (is_ns(s) && s->desc.volume == SM_VOLUME_SPLIT) {
    a.Gr = s->Gr;
    return s->prec == SM_FP64 ? launch_element_split_ns_f64(s->N, s->desc.riemann, mode, a, st)
                              : launch_element_split_ns_f32(s->N, s->desc.riemann, mode, a, st);
  }
  if (is_ns(s)) {
    a.Gr = s->Gr;
    return s->prec == SM_FP64 ? launch_element_ns_f64(s->N, s->desc.riemann, mode, a, st)
                              : launch_element_ns_f32(s->N, s->desc.riemann, mode, a, st);
  }
  if (s->desc.volume == SM_VOLUME_SPLIT)
    return s->prec == SM_FP64 ? launch_element_split_f64(s->N, s->desc.riemann, mode, a, st)
                              : launch_element_split_f32(s->N, s->desc.riemann, mode, a, st);
  return s->prec == SM_FP64 ? launch_element_f64(s->N, s->desc.riemann, mode, a, st)
                            : launch_element_f32(s->N, s->desc.riemann, mode, a, st);
}

// One RK step: the five stages' parameters in one launch, then per stage the interface
// inputs and the element kernel.
cudaError_t enqueue_step(sm_solver* s, double dt, int cur, cudaStream_t st) {
  int c = cur;
  cudaError_t e = launch_step_params(s->m, s->np, s->sp, s->t_d, RK_C, dt, s->ticket_d, st);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < 5; ++k) {
    const StageParams* sp = s->sp + k;
    if ((e = enqueue_flux_inputs(s, sp, s->U[c], s->Fs, s->Fm, st, use_traces(s))) != cudaSuccess) return e;
    ElemArgs a{s->m, sp, s->U[c], s->U[1 - c], s->G, s->Fs, s->Fm, RK_A[k], RK_B[k], dt};
    a.Ts = s->Ts;
    a.Tm = s->Tm;
    e = launch_elem(s, k == 0 ? ELEM_STAGE_FIRST : ELEM_STAGE, a, st);
    if (e != cudaSuccess) return e;
    c ^= 1;
  }
  return cudaSuccess;
}

void clear_graphs(sm_solver* s) {
  for (auto& g : s->graphs) cudaGraphExecDestroy(g.exec);
  s->graphs.clear();
}

int get_graph(sm_solver* s, double dt, int cur, cudaGraphExec_t* out) {
  for (auto& g : s->graphs)
    if (g.dt == dt && g.cur == cur) { *out = g.exec; return SM_OK; }
  if (s->graphs.size() >= 8) clear_graphs(s);
  SM_CK(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t e = enqueue_step(s, dt, cur, s->cap);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s->cap, &graph);
  if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return fail(SM_ERR_CUDA, "capture step", e); }
  if (e2 != cudaSuccess) return fail(SM_ERR_CUDA, "end capture", e2);
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(SM_ERR_CUDA, "instantiate step graph", e);
  s->graphs.push_back({dt, cur, exec});
  *out = exec;
  return SM_OK;
}

void free_solver(sm_solver* s) {
  if (!s) return;
  clear_graphs(s);
  if (s->cap) cudaStreamDestroy(s->cap);
  if (s->h2d) cudaStreamDestroy(s->h2d);
  if (s->d2h) cudaStreamDestroy(s->d2h);
  for (cudaEvent_t ev : {s->in_ready, s->in_free, s->out_ready, s->out_free})
    if (ev) cudaEventDestroy(ev);
  void* ptrs[] = {s->basis_d, s->modes_d, s->U[0], s->U[1], s->G, s->Fs, s->Fm, s->sp, s->ticket_d, s->t_d, s->red_d, s->topo_d,
                  s->Gr, s->Ls, s->Lm, s->Ts, s->Tm, s->Ts2, s->Tm2, s->Fs2, s->Fm2, s->geo, s->stage_in, s->stage_out,
                  s->t0_d};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete s;
}

int valid_desc(const sm_mesh_desc* d) {
  if (!d) return fail(SM_ERR_ARG, "desc is NULL");
  if (d->N < 1 || d->N > 7) return fail(SM_ERR_UNSUPPORTED, "N must be in 1..7");
  if (d->geom != SM_GEOM_PLANE && d->geom != SM_GEOM_CYLINDER && d->geom != SM_GEOM_PLANE_CURVILINEAR &&
      d->geom != SM_GEOM_ANNULAR && d->geom != SM_GEOM_CONE)
    return fail(SM_ERR_UNSUPPORTED, "unknown interface geometry");
  if (d->geom == SM_GEOM_CONE) {
    if (!(d->cone_angle >= 0.0 && d->cone_angle < 0.5 * M_PI)) return fail(SM_ERR_ARG, "cone half-angle in [0, pi/2)");
    const double sa = sin(d->cone_angle), ca = cos(d->cone_angle);
    if (!(d->z0 * sa + d->x0 * ca > 0.0 && d->z1 * sa + d->x0 * ca > 0.0))
      return fail(SM_ERR_ARG, "the conical mesh must stay off the axis (positive radii)");
    if (!(d->y1 - d->y0 <= 2.0 * M_PI + 1e-12)) return fail(SM_ERR_ARG, "the angular sector exceeds 2 pi");
    if (d->flow != SM_FLOW_CONSTANT && d->flow != SM_FLOW_AXIAL_PULSE && d->flow != SM_FLOW_RIGID_ROTATION)
      return fail(SM_ERR_ARG, "cone flows: constant, axial pulse, rigid rotation");
  } else if (d->geom == SM_GEOM_ANNULAR) {
    if (!(d->z0 > 0.0)) return fail(SM_ERR_ARG, "annular radii must be positive");
    if (!(d->y1 - d->y0 <= 2.0 * M_PI + 1e-12)) return fail(SM_ERR_ARG, "the angular sector exceeds 2 pi");
    if (d->flow != SM_FLOW_CONSTANT && d->flow != SM_FLOW_AXIAL_PULSE && d->flow != SM_FLOW_RIGID_ROTATION)
      return fail(SM_ERR_ARG, "annular flows: constant, axial pulse, rigid rotation");
  } else if (d->geom == SM_GEOM_CYLINDER) {
    if (!(d->x0 > 0.0)) return fail(SM_ERR_ARG, "cylinder radii must be positive");
    if (!(d->y1 - d->y0 <= 2.0 * M_PI + 1e-12)) return fail(SM_ERR_ARG, "the angular sector exceeds 2 pi");
    if (d->flow != SM_FLOW_CONSTANT && d->flow != SM_FLOW_AXIAL_PULSE && d->flow != SM_FLOW_RIGID_ROTATION)
      return fail(SM_ERR_ARG, "cylinder flows: constant, axial pulse, rigid rotation");
  } else if (d->flow > SM_FLOW_SHEAR_X) {
    return fail(SM_ERR_ARG, "the axial pulse and rigid rotation flows need the cylinder");
  }
  for (int k = 0; k < 3; ++k)
    if (d->nel_static[k] < 1 || d->nel_moving[k] < 1) return fail(SM_ERR_ARG, "element counts must be >= 1");
  if (d->nel_static[1] != d->nel_moving[1] || d->nel_static[2] != d->nel_moving[2])
    return fail(SM_ERR_ARG, "interface faces must match: nel_static[1..2] == nel_moving[1..2]");
  if (!(d->x1 > d->x0 && d->x2 > d->x1 && d->y1 > d->y0 && d->z1 > d->z0)) return fail(SM_ERR_ARG, "empty block extent");
  if (!(d->gamma > 1.0)) return fail(SM_ERR_ARG, "gamma must exceed 1");
  if (d->riemann != SM_RUSANOV && d->riemann != SM_ROE_HH) return fail(SM_ERR_ARG, "unknown Riemann solver");
  if (d->precision != SM_FP64 && d->precision != SM_FP32) return fail(SM_ERR_ARG, "unknown precision");
  if (d->flow < 0 || d->flow > SM_FLOW_RIGID_ROTATION) return fail(SM_ERR_ARG, "unknown flow");
  if (d->physics != SM_EULER && d->physics != SM_NAVIER_STOKES) return fail(SM_ERR_ARG, "unknown physics");
  if (d->physics == SM_NAVIER_STOKES && !(d->mu >= 0.0 && d->Pr > 0.0 && d->Rgas > 0.0))
    return fail(SM_ERR_ARG, "Navier-Stokes needs mu >= 0, Pr > 0, Rgas > 0");
  if (d->volume != SM_VOLUME_WEAK && d->volume != SM_VOLUME_SPLIT) return fail(SM_ERR_ARG, "unknown volume integral");
  if (d->periodic_x != 0 && d->periodic_x != 1) return fail(SM_ERR_ARG, "periodic_x must be 0 or 1");
  if (d->periodic_x && (d->geom != SM_GEOM_PLANE || d->physics != SM_EULER))
    return fail(SM_ERR_UNSUPPORTED, "the second sliding interface (periodic x) takes the plane geometry and Euler physics");
  long long E = (long long)(d->nel_static[0] + d->nel_moving[0]) * d->nel_static[1] * d->nel_static[2];
  if (E > (1LL << 31)) return fail(SM_ERR_ARG, "too many elements");
  return SM_OK;
}

// The mesh, flow and physics fields of the kernels' mesh description from the C-ABI
// description (shared by sm_init_mesh and sm_rhs_static); device pointers, the motion and
// the per-precision constants are set by the callers.
void mesh_from_desc(const sm_mesh_desc* desc, MeshDev& m) {
  memset(&m, 0, sizeof(m));
  m.nxs = desc->nel_static[0];
  m.nxm = desc->nel_moving[0];
  m.ny = desc->nel_static[1];
  m.nz = desc->nel_static[2];
  m.Es = (long long)m.nxs * m.ny * m.nz;
  m.E = m.Es + (long long)m.nxm * m.ny * m.nz;
  m.hx0 = (desc->x1 - desc->x0) / m.nxs;
  m.hx1 = (desc->x2 - desc->x1) / m.nxm;
  m.hy = (desc->y1 - desc->y0) / m.ny;
  m.hz = (desc->z1 - desc->z0) / m.nz;
  m.x0 = desc->x0;
  m.x1 = desc->x1;
  m.y0 = desc->y0;
  m.z0 = desc->z0;
  m.gamma = desc->gamma;
  m.conforming = desc->interface_conforming;
  m.flow = desc->flow;
  m.physics = desc->physics;
  m.mu = desc->mu;
  m.Pr = desc->Pr;
  m.Rgas = desc->Rgas;
  m.geom = desc->geom;
  m.Theta = desc->y1 - desc->y0;
  m.cone_s = sin(desc->cone_angle);
  m.cone_c = cos(desc->cone_angle);
  for (int k = 0; k < 16; ++k) m.fpar[k] = desc->fpar[k];
}

}  // namespace

extern "C" {

const char* sm_status_string(int st) {
  switch (st) {
    case SM_OK: return "ok";
    case SM_PENDING: return "pending";
    case SM_ERR_ARG: return "invalid argument";
    case SM_ERR_OOM: return "out of device memory";
    case SM_ERR_CUDA: return "CUDA error";
    case SM_ERR_NONFINITE: return "non-finite state";
    case SM_ERR_TIMEOUT: return "timeout";
    case SM_ERR_BUSY: return "busy";
    case SM_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

const char* sm_last_error(void) { return g_last_error.c_str(); }

int sm_init_mesh(const sm_mesh_desc* desc, sm_solver** out) {
  if (!out) return fail(SM_ERR_ARG, "out is NULL");
  *out = nullptr;
  int rc = valid_desc(desc);
  if (rc != SM_OK) return rc;
  sm_solver* s = new (std::nothrow) sm_solver();
  if (!s) return fail(SM_ERR_OOM, "host allocation");
  s->desc = *desc;
  s->motion = {0.0, 0.0, 0.0};
  s->N = desc->N;
  s->np = desc->N + 1;
  s->nn = (long long)s->np * s->np * s->np;
  s->prec = desc->precision;
  s->sb = s->prec == SM_FP64 ? 8 : 4;
  lgl_basis(s->N, s->basis_h);
  MeshDev& m = s->m;
  mesh_from_desc(desc, m);
  s->nstate = m.E * 5 * s->nn;
  s->nface_vals = (long long)m.ny * m.nz * 5 * s->np * s->np;
  s->red_blocks = 304;
  const size_t sbytes = (size_t)s->nstate * s->sb, fbytes = (size_t)s->nface_vals * s->sb;
  cudaError_t e;
#define SM_ALLOC(ptr, bytes)                                                        \
  e = cudaMalloc((void**)&(ptr), (bytes));                                          \
  if (e != cudaSuccess) {                                                           \
    cudaGetLastError();                                                             \
    free_solver(s);                                                                 \
    return fail(e == cudaErrorMemoryAllocation ? SM_ERR_OOM : SM_ERR_CUDA, "cudaMalloc", e); \
  }
  SM_ALLOC(s->basis_d, sizeof(BasisDev));
  SM_ALLOC(s->modes_d, sizeof(double) * 160);
  SM_ALLOC(s->U[0], sbytes);
  SM_ALLOC(s->U[1], sbytes);
  SM_ALLOC(s->G, sbytes);
  SM_ALLOC(s->Fs, fbytes);
  SM_ALLOC(s->Fm, fbytes);
  SM_ALLOC(s->sp, 5 * sizeof(StageParams));
  SM_ALLOC(s->ticket_d, sizeof(unsigned));
  SM_ALLOC(s->t_d, sizeof(double));
  SM_ALLOC(s->red_d, sizeof(double) * (s->red_blocks * 5 + 15));
  SM_ALLOC(s->topo_d, sizeof(int4) * 2 * (size_t)m.E);
  if (desc->physics == SM_NAVIER_STOKES) {
    // lifting values per interface face node: 5 on the plane (normal +x), 15 (q* N_a) curved
    const size_t lbytes = desc->geom == SM_GEOM_PLANE ? fbytes : 3 * fbytes;
    SM_ALLOC(s->Gr, (size_t)m.E * 15 * s->nn * s->sb);
    SM_ALLOC(s->Ls, lbytes);
    SM_ALLOC(s->Lm, lbytes);
  } else if (!desc->interface_conforming && desc->geom == SM_GEOM_PLANE) {
    SM_ALLOC(s->Ts, fbytes);
    SM_ALLOC(s->Tm, fbytes);
    if (desc->periodic_x) {
      SM_ALLOC(s->Ts2, fbytes);
      SM_ALLOC(s->Tm2, fbytes);
      SM_ALLOC(s->Fs2, fbytes);
      SM_ALLOC(s->Fm2, fbytes);
    }
  }
  if (desc->geom != SM_GEOM_PLANE) SM_ALLOC(s->geo, (size_t)m.E * 13 * s->nn * s->sb);
#undef SM_ALLOC
  m.basis = s->basis_d;
  m.modes = s->modes_d;
  m.topo = s->topo_d;
  m.periodic_x = desc->periodic_x;
  m.Ts2 = s->Ts2;
  m.Tm2 = s->Tm2;
  m.Fs2 = s->Fs2;
  m.Fm2 = s->Fm2;
  fill_constants(m, s->basis_h, desc->fpar);
  // static mesh topology: neighbour codes and packed position of every element
  std::vector<int4> topo(2 * (size_t)m.E);
  for (long long e = 0; e < m.E; ++e) {
    ElemPos p = decode_elem(m, e);
    int nb[6];
    for (int fc = 0; fc < 6; ++fc) {
      long long q = 0;
      int kind = face_neighbor(m, p, fc >> 1, fc & 1, &q);
      nb[fc] = kind == 0 ? (int)q : (kind == 1 ? -1 : (kind == 2 ? -2 : -3));
    }
    topo[2 * e] = make_int4(nb[0], nb[1], nb[2], nb[3]);
    topo[2 * e + 1] = make_int4(nb[4], nb[5], (p.ix << 1) | p.blk, p.iz * m.ny + p.iy);
  }
  const char* what = nullptr;
  if (s->geo) {
    std::vector<double> g;
    curvilinear_geometry(m, s->basis_h, s->N, g);
    if (s->prec == SM_FP64) {
      e = cudaMemcpy(s->geo, g.data(), sizeof(double) * g.size(), cudaMemcpyHostToDevice);
    } else {
      std::vector<float> gf(g.begin(), g.end());
      e = cudaMemcpy(s->geo, gf.data(), sizeof(float) * gf.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) what = "upload geometry";
    m.geo = s->geo;
  }
  if (what) {
  } else if ((e = cudaMemcpy(s->basis_d, &s->basis_h, sizeof(BasisDev), cudaMemcpyHostToDevice)) != cudaSuccess) what = "upload basis";
  else if ((e = cudaMemcpy(s->modes_d, &desc->modes[0][0][0], sizeof(double) * 160, cudaMemcpyHostToDevice)) != cudaSuccess) what = "upload modes";
  else if ((e = cudaMemcpy(s->topo_d, topo.data(), sizeof(int4) * topo.size(), cudaMemcpyHostToDevice)) != cudaSuccess) what = "upload topology";
  else if ((e = cudaMemset(s->G, 0, sbytes)) != cudaSuccess) what = "clear G";
  else if ((e = cudaMemset(s->U[0], 0, sbytes)) != cudaSuccess) what = "clear U";
  else if ((e = cudaMemset(s->Fs, 0, fbytes)) != cudaSuccess || (e = cudaMemset(s->Fm, 0, fbytes)) != cudaSuccess) what = "clear F";
  else if ((e = cudaMemset(s->t_d, 0, sizeof(double))) != cudaSuccess) what = "clear t";
  else if ((e = cudaMemset(s->sp, 0, 5 * sizeof(StageParams))) != cudaSuccess) what = "clear stage params";
  else if ((e = cudaMemset(s->ticket_d, 0, sizeof(unsigned))) != cudaSuccess) what = "clear step counter";
  else if ((e = (s->prec == SM_FP64 ? prepare_element_f64(s->N) : prepare_element_f32(s->N))) != cudaSuccess) what = "element kernel attributes";
  else if (desc->volume == SM_VOLUME_SPLIT &&
           (e = (s->prec == SM_FP64 ? prepare_element_split_f64(s->N) : prepare_element_split_f32(s->N))) != cudaSuccess)
    what = "split-form kernel attributes";
  else if (desc->volume == SM_VOLUME_SPLIT && desc->physics == SM_NAVIER_STOKES && desc->geom == SM_GEOM_PLANE &&
           (e = (s->prec == SM_FP64 ? prepare_element_split_ns_f64(s->N) : prepare_element_split_ns_f32(s->N))) != cudaSuccess)
    what = "split-form Navier-Stokes kernel attributes";
  else if ((e = ensure_dhat_constants()) != cudaSuccess) what = "derivative constants";
  else if ((e = prepare_interface(s->N, s->prec)) != cudaSuccess) what = "interface kernel attributes";
  else if (desc->geom != SM_GEOM_PLANE &&
           (e = (s->prec == SM_FP64 ? prepare_curved_f64(s->N) : prepare_curved_f32(s->N))) != cudaSuccess)
    what = "curvilinear kernel attributes";
  else if (desc->geom != SM_GEOM_PLANE && desc->volume == SM_VOLUME_SPLIT &&
           (e = (s->prec == SM_FP64 ? prepare_curved_split_f64(s->N) : prepare_curved_split_f32(s->N))) != cudaSuccess)
    what = "curvilinear split-form kernel attributes";
  else if (desc->geom != SM_GEOM_PLANE && desc->physics == SM_NAVIER_STOKES &&
           (e = (s->prec == SM_FP64 ? prepare_curved_ns_f64(s->N) : prepare_curved_ns_f32(s->N))) != cudaSuccess)
    what = "curvilinear Navier-Stokes kernel attributes";
  else if (desc->geom != SM_GEOM_PLANE && desc->physics == SM_NAVIER_STOKES && desc->volume == SM_VOLUME_SPLIT &&
           (e = (s->prec == SM_FP64 ? prepare_curved_split_ns_f64(s->N) : prepare_curved_split_ns_f32(s->N))) != cudaSuccess)
    what = "curvilinear split-form Navier-Stokes kernel attributes";
  else if (desc->physics == SM_NAVIER_STOKES &&
           ((e = (s->prec == SM_FP64 ? prepare_ns_f64(s->N) : prepare_ns_f32(s->N))) != cudaSuccess ||
            (e = prepare_interface_ns(s->N, s->prec)) != cudaSuccess)) what = "Navier-Stokes kernel attributes";
  else if ((e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking)) != cudaSuccess) what = "capture stream";
  else if ((e = cudaDeviceSynchronize()) != cudaSuccess) what = "init sync";
  if (what) {
    free_solver(s);
    return fail(SM_ERR_CUDA, what, e);
  }
  *out = s;
  return SM_OK;
}

int sm_set_motion(sm_solver* s, const sm_motion* mo) {
  if (!s || !mo) return fail(SM_ERR_ARG, "NULL argument");
  const bool cyl = rotating_geom(s->desc.geom);
  if (!cyl && mo->omega != 0.0) return fail(SM_ERR_UNSUPPORTED, "rotation needs a rotating geometry");
  if (cyl && mo->v != 0.0) return fail(SM_ERR_UNSUPPORTED, "the cylinder's rotor rotates (omega), it does not translate");
  if (!std::isfinite(mo->v) || !std::isfinite(mo->omega) || !std::isfinite(mo->delta0))
    return fail(SM_ERR_ARG, "non-finite motion");
  const double speed = cyl ? mo->omega : mo->v;
  if (s->desc.interface_conforming && (speed != 0.0 || mo->delta0 != 0.0))
    return fail(SM_ERR_ARG, "a conforming interface cannot move");
  s->motion = *mo;
  // the mapper takes the displacement of block 1 relative to block 0: the rotor (block 0)
  // turning by phi = delta0 + omega t displaces the stator by -phi
  s->m.v = cyl ? -mo->omega : mo->v;
  s->m.delta0 = cyl ? -mo->delta0 : mo->delta0;
  s->m.cd[MC_VG] = speed;
  s->m.cf[MC_VG] = (float)speed;
  clear_graphs(s);
  return SM_OK;
}

long long sm_state_size(const sm_solver* s) { return s ? s->nstate : -1; }
int sm_scalar_bytes(const sm_solver* s) { return s ? s->sb : -1; }
void* sm_state_ptr(sm_solver* s) { return s ? s->U[s->cur] : nullptr; }

int sm_init_state(sm_solver* s, void* stream) {
  if (!s) return fail(SM_ERR_ARG, "NULL solver");
  cudaStream_t st = (cudaStream_t)stream;
  SM_CK(launch_init_state(s->N, s->prec, s->m, s->U[s->cur], st), "init state");
  s->traces_ok = false;
  SM_CK(cudaMemsetAsync(s->G, 0, (size_t)s->nstate * s->sb, st), "clear G");
  s->t_host = 0.0;
  SM_CK(cudaMemsetAsync(s->t_d, 0, sizeof(double), st), "clear t");
  return SM_OK;
}

int sm_set_state(sm_solver* s, const void* U, int on_device, double t, void* stream) {
  if (!s || !U) return fail(SM_ERR_ARG, "NULL argument");
  if (!std::isfinite(t)) return fail(SM_ERR_ARG, "non-finite time");
  cudaStream_t st = (cudaStream_t)stream;
  SM_CK(cudaMemcpyAsync(s->U[s->cur], U, (size_t)s->nstate * s->sb,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st), "copy state in");
  s->traces_ok = false;
  s->t_host = t;
  SM_CK(cudaMemcpyAsync(s->t_d, &s->t_host, sizeof(double), cudaMemcpyHostToDevice, st), "copy time in");
  SM_CK(cudaMemsetAsync(s->G, 0, (size_t)s->nstate * s->sb, st), "clear G");
  return SM_OK;
}

int sm_get_state(sm_solver* s, void* U, int on_device, double* t, void* stream) {
  if (!s) return fail(SM_ERR_ARG, "NULL solver");
  cudaStream_t st = (cudaStream_t)stream;
  double tt = 0.0;
  if (U)
    SM_CK(cudaMemcpyAsync(U, s->U[s->cur], (size_t)s->nstate * s->sb,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st), "copy state out");
  SM_CK(cudaMemcpyAsync(&tt, s->t_d, sizeof(double), cudaMemcpyDeviceToHost, st), "copy time out");
  SM_CK(cudaStreamSynchronize(st), "sync");
  s->t_host = tt;
  if (t) *t = tt;
  return SM_OK;
}

int sm_rhs(sm_solver* s, double t, const void* dU, void* dUt, void* stream) {
  if (!s || !dU || !dUt) return fail(SM_ERR_ARG, "NULL argument");
  if (dU == dUt) return fail(SM_ERR_ARG, "dU and dUt must not overlap");
  if (!aligned16(dU) || !aligned16(dUt)) return fail(SM_ERR_ARG, "device arrays must be 16-byte aligned");
  if (!std::isfinite(t)) return fail(SM_ERR_ARG, "non-finite time");
  cudaStream_t st = (cudaStream_t)stream;
  SM_CK(enqueue_rhs_parts(s, t, dU, s->Fs, s->Fm, st), "stage params / interface");
  ElemArgs a{s->m, s->sp, dU, dUt, nullptr, s->Fs, s->Fm, 0.0, 0.0, 0.0};
  SM_CK(launch_elem(s, ELEM_RHS, a, st), "element kernel");
  return SM_OK;
}

int sm_interface(sm_solver* s, double t, const void* dU, void* dFs, void* dFm, void* stream) {
  if (!s || !dU || !dFs || !dFm) return fail(SM_ERR_ARG, "NULL argument");
  if (!aligned16(dU) || !aligned16(dFs) || !aligned16(dFm))
    return fail(SM_ERR_ARG, "device arrays must be 16-byte aligned");
  if (s->desc.interface_conforming) return fail(SM_ERR_ARG, "the interface is conforming");
  if (!std::isfinite(t)) return fail(SM_ERR_ARG, "non-finite time");
  SM_CK(enqueue_rhs_parts(s, t, dU, dFs, dFm, (cudaStream_t)stream), "interface");
  return SM_OK;
}

int sm_gradients(sm_solver* s, double t, const void* dU, void* dGrad, void* stream) {
  if (!s || !dU || !dGrad) return fail(SM_ERR_ARG, "NULL argument");
  if (!aligned16(dU) || !aligned16(dGrad)) return fail(SM_ERR_ARG, "device arrays must be 16-byte aligned");
  if (!is_ns(s)) return fail(SM_ERR_ARG, "gradients are lifted for Navier-Stokes solvers only");
  if (!std::isfinite(t)) return fail(SM_ERR_ARG, "non-finite time");
  cudaStream_t st = (cudaStream_t)stream;
  SM_CK(launch_stage_params(s->m, s->np, s->sp, s->t_d, t, 0.0, 0.0, 0, st), "stage parameters");
  s->sp_last = 0;
  if (s->m.geom != 0) {
    const bool f64 = s->prec == SM_FP64;
    if (!s->desc.interface_conforming)
      SM_CK(f64 ? launch_curved_interface_lift_f64(s->N, s->m, s->sp, dU, s->Ls, s->Lm, st)
                : launch_curved_interface_lift_f32(s->N, s->m, s->sp, dU, s->Ls, s->Lm, st), "interface lifting");
    SM_CK(f64 ? launch_curved_lift_f64(s->N, s->m, s->sp, dU, dGrad, s->Ls, s->Lm, st)
              : launch_curved_lift_f32(s->N, s->m, s->sp, dU, dGrad, s->Ls, s->Lm, st), "lifting");
    return SM_OK;
  }
  if (!s->desc.interface_conforming)
    SM_CK(launch_interface_lift(s->N, s->prec, s->m, s->sp, dU, s->Ls, s->Lm, st), "interface lifting");
  SM_CK(s->prec == SM_FP64 ? launch_lift_f64(s->N, s->m, s->sp, dU, dGrad, s->Ls, s->Lm, st)
                           : launch_lift_f32(s->N, s->m, s->sp, dU, dGrad, s->Ls, s->Lm, st), "lifting");
  return SM_OK;
}

int sm_step(sm_solver* s, double dt, int nsteps, void* stream) {
  if (!s) return fail(SM_ERR_ARG, "NULL solver");
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return fail(SM_ERR_ARG, "dt must be positive, nsteps >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  if (nsteps > 0) SM_CK(ensure_traces(s, st), "gather interface traces");
  for (int n = 0; n < nsteps; ++n) {
    cudaGraphExec_t exec;
    int rc = get_graph(s, dt, s->cur, &exec);
    if (rc != SM_OK) return rc;
    SM_CK(cudaGraphLaunch(exec, st), "graph launch");
    s->cur ^= 1;
    s->t_host += dt;
    s->sp_last = 4;
  }
  return SM_OK;
}

namespace {

// The copies and steps of sm_stream_jobs (staging buffers and copy streams in place).
int stream_jobs_enqueue(sm_solver* s, const char* in, long long in_stride, char* out, long long out_stride, int count,
                        double t0, double dt, int nsteps, void* stream) {
  const size_t bytes = (size_t)s->nstate * s->sb;
  cudaStream_t cs = (cudaStream_t)stream;
  // the start time, once, in device memory (a per-job device-to-device copy of 8 bytes)
  SM_CK(cudaMemcpy(s->t0_d, &t0, sizeof(double), cudaMemcpyHostToDevice), "copy start time");
  SM_CK(cudaMemcpyAsync(s->stage_in, in, bytes, cudaMemcpyHostToDevice, s->h2d), "copy job in");
  SM_CK(cudaEventRecord(s->in_ready, s->h2d), "event");
  for (int k = 0; k < count; ++k) {
    // job k's state into the solver; the staging buffer is then free for job k + 1
    SM_CK(cudaStreamWaitEvent(cs, s->in_ready, 0), "wait job in");
    SM_CK(cudaMemcpyAsync(s->U[s->cur], s->stage_in, bytes, cudaMemcpyDeviceToDevice, cs), "state in");
    SM_CK(cudaMemcpyAsync(s->t_d, s->t0_d, sizeof(double), cudaMemcpyDeviceToDevice, cs), "time in");
    SM_CK(cudaEventRecord(s->in_free, cs), "event");
    s->traces_ok = false;
    s->t_host = t0;
    if (k + 1 < count) {
      SM_CK(cudaStreamWaitEvent(s->h2d, s->in_free, 0), "wait staging (in)");
      SM_CK(cudaMemcpyAsync(s->stage_in, in + (size_t)(k + 1) * (size_t)in_stride, bytes, cudaMemcpyHostToDevice, s->h2d),
            "copy job in");
      SM_CK(cudaEventRecord(s->in_ready, s->h2d), "event");
    }
    // the first stage of a step writes the RK register before reading it: G needs no reset
    const int rc = sm_step(s, dt, nsteps, stream);
    if (rc != SM_OK) return rc;
    // the result out through the second staging buffer, once job k - 1 has left it
    if (k > 0) SM_CK(cudaStreamWaitEvent(cs, s->out_free, 0), "wait staging (out)");
    SM_CK(cudaMemcpyAsync(s->stage_out, s->U[s->cur], bytes, cudaMemcpyDeviceToDevice, cs), "state out");
    SM_CK(cudaEventRecord(s->out_ready, cs), "event");
    SM_CK(cudaStreamWaitEvent(s->d2h, s->out_ready, 0), "wait job out");
    SM_CK(cudaMemcpyAsync(out + (size_t)k * (size_t)out_stride, s->stage_out, bytes, cudaMemcpyDeviceToHost, s->d2h),
          "copy job out");
    SM_CK(cudaEventRecord(s->out_free, s->d2h), "event");
  }
  return SM_OK;
}

}  // namespace

int sm_stream_jobs(sm_solver* s, const void* in_host, long long in_stride, void* out_host, long long out_stride,
                   int count, double t0, double dt, int nsteps, void* stream) {
  if (!s || !in_host || !out_host) return fail(SM_ERR_ARG, "NULL argument");
  if (count < 0 || nsteps < 1 || in_stride < 0 || out_stride < 0)
    return fail(SM_ERR_ARG, "count >= 0, nsteps >= 1, strides >= 0");
  if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(t0)) return fail(SM_ERR_ARG, "dt > 0 and t0 finite");
  if (count == 0) return SM_OK;
  const size_t bytes = (size_t)s->nstate * s->sb;
  if (!s->stage_in) {
    SM_CK(cudaMalloc(&s->stage_in, bytes), "staging buffer (in)");
    SM_CK(cudaMalloc(&s->stage_out, bytes), "staging buffer (out)");
    SM_CK(cudaMalloc(&s->t0_d, sizeof(double)), "start time");
    SM_CK(cudaStreamCreateWithFlags(&s->h2d, cudaStreamNonBlocking), "copy stream (in)");
    SM_CK(cudaStreamCreateWithFlags(&s->d2h, cudaStreamNonBlocking), "copy stream (out)");
    for (cudaEvent_t* ev : {&s->in_ready, &s->in_free, &s->out_ready, &s->out_free})
      SM_CK(cudaEventCreateWithFlags(ev, cudaEventDisableTiming), "event");
  }
  const int rc = stream_jobs_enqueue(s, static_cast<const char*>(in_host), in_stride, static_cast<char*>(out_host),
                                     out_stride, count, t0, dt, nsteps, stream);
  // every copy has finished before the call returns, also after a failure: none may touch
  // the caller's host buffers later
  const cudaError_t e1 = cudaStreamSynchronize(s->h2d);
  const cudaError_t e2 = cudaStreamSynchronize(s->d2h);
  const cudaError_t e3 = cudaStreamSynchronize((cudaStream_t)stream);
  if (rc != SM_OK) return rc;
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
    return fail(SM_ERR_CUDA, "sync", e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3));
  return SM_OK;
}

int sm_step_profiled(sm_solver* s, double dt, int nsteps, void* stream, double* ms_out, int* launches_out) {
  if (!s) return fail(SM_ERR_ARG, "NULL solver");
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return fail(SM_ERR_ARG, "dt must be positive, nsteps >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t ev[6];
  for (int k = 0; k < 6; ++k) SM_CK(cudaEventCreate(&ev[k]), "event create");
  double ms[3] = {0, 0, 0};
  int cnt[3] = {0, 0, 0};
  int rc = SM_OK;
  if (nsteps > 0 && ensure_traces(s, st) != cudaSuccess) rc = fail(SM_ERR_CUDA, "gather interface traces");
  for (int n = 0; n < nsteps && rc == SM_OK; ++n) {
    // the step's five stage-parameter blocks in one launch, then per stage the interface
    // inputs and the element kernel, with events around each part
    cudaError_t e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = launch_step_params(s->m, s->np, s->sp, s->t_d, RK_C, dt, s->ticket_d, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float a0 = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&a0, ev[0], ev[1]);
    if (e != cudaSuccess) { rc = fail(SM_ERR_CUDA, "profiled step", e); break; }
    ms[0] += a0;
    cnt[0] += 1;
    for (int k = 0; k < 5; ++k) {
      const StageParams* sp = s->sp + k;
      e = cudaEventRecord(ev[1], st);
      if (e == cudaSuccess) e = enqueue_flux_inputs(s, sp, s->U[s->cur], s->Fs, s->Fm, st, use_traces(s));
      if (e == cudaSuccess) e = cudaEventRecord(ev[2], st);
      ElemArgs a{s->m, sp, s->U[s->cur], s->U[1 - s->cur], s->G, s->Fs, s->Fm, RK_A[k], RK_B[k], dt};
      a.Ts = s->Ts;
      a.Tm = s->Tm;
      if (e == cudaSuccess) e = launch_elem(s, k == 0 ? ELEM_STAGE_FIRST : ELEM_STAGE, a, st);
      if (e == cudaSuccess) e = cudaEventRecord(ev[3], st);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
      float a1 = 0, a2 = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&a1, ev[1], ev[2]);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&a2, ev[2], ev[3]);
      if (e != cudaSuccess) { rc = fail(SM_ERR_CUDA, "profiled step", e); break; }
      ms[1] += a1; ms[2] += a2;
      cnt[1] += s->desc.interface_conforming ? 0 : 1; cnt[2] += 1;
      s->cur ^= 1;
    }
    if (rc == SM_OK) { s->t_host += dt; s->sp_last = 4; }
  }
  for (int k = 0; k < 6; ++k) cudaEventDestroy(ev[k]);
  if (ms_out) for (int k = 0; k < 3; ++k) ms_out[k] = ms[k];
  if (launches_out) for (int k = 0; k < 3; ++k) launches_out[k] = cnt[k];
  return rc;
}

int sm_diag(sm_solver* s, sm_diag_out* out, void* stream) {
  if (!s || !out) return fail(SM_ERR_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  double* part = s->red_d;
  double* res = s->red_d + s->red_blocks * 5;
  SM_CK(launch_totals(s->N, s->prec, s->m, s->U[s->cur], part, s->red_blocks, res, st), "totals");
  SM_CK(launch_face_sums(s->N, s->prec, s->m, s->Fs, part, s->red_blocks, res + 5, st), "face sums static");
  SM_CK(launch_face_sums(s->N, s->prec, s->m, s->Fm, part, s->red_blocks, res + 10, st), "face sums moving");
  double h[15];
  long long n = 0;
  double sfrac = 0.0, tt = 0.0;
  SM_CK(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st), "diag copy");
  const StageParams* spl = s->sp + s->sp_last;
  SM_CK(cudaMemcpyAsync(&n, &spl->n, sizeof(n), cudaMemcpyDeviceToHost, st), "diag copy n");
  SM_CK(cudaMemcpyAsync(&sfrac, &spl->s, sizeof(sfrac), cudaMemcpyDeviceToHost, st), "diag copy s");
  SM_CK(cudaMemcpyAsync(&tt, s->t_d, sizeof(tt), cudaMemcpyDeviceToHost, st), "diag copy t");
  SM_CK(cudaStreamSynchronize(st), "diag sync");
  out->n_delta = n;
  out->s_delta = sfrac;
  out->t = tt;
  int finite = 1;
  for (int v = 0; v < 5; ++v) {
    out->totals[v] = h[v];
    out->iface_sum_static[v] = h[5 + v];
    out->iface_sum_moving[v] = h[10 + v];
    if (!std::isfinite(h[v])) finite = 0;
  }
  return finite ? SM_OK : fail(SM_ERR_NONFINITE, "state totals are not finite");
}

void sm_destroy(sm_solver* s) { free_solver(s); }

int sm_map(const double* d_delta, int count, double l, int n_par, long long* d_n, double* d_s, int* d_pairs,
           void* stream) {
  if (count < 0 || n_par < 1 || !(l > 0.0) || (count > 0 && (!d_delta || !d_n || !d_s)))
    return fail(SM_ERR_ARG, "invalid sm_map arguments");
  SM_CK(launch_map_batch(d_delta, count, l, n_par, d_n, d_s, d_pairs, (cudaStream_t)stream), "map kernel");
  return SM_OK;
}

int sm_fp64_fma_probe(int blocks, int threads, int iters, double* d_out, void* stream) {
  if (blocks < 1 || threads < 32 || threads > 1024 || threads % 32 || iters < 1 || !d_out)
    return fail(SM_ERR_ARG, "sm_fp64_fma_probe: blocks >= 1, threads a multiple of 32 in 32..1024, iters >= 1, d_out");
  SM_CK(launch_fp64_fma_probe(blocks, threads, iters, d_out, (cudaStream_t)stream), "FP64 FMA probe");
  return SM_OK;
}

int sm_mortar_matrices(int N, double sigma, double* d_out, void* stream) {
  static std::mutex mu;
  static BasisDev* cache[8] = {nullptr};
  if (N < 1 || N > 7 || !d_out || !(sigma >= -1.0 && sigma <= 1.0)) return fail(SM_ERR_ARG, "invalid sm_mortar_matrices arguments");
  BasisDev* b;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!cache[N]) {
      BasisDev h;
      lgl_basis(N, h);
      SM_CK(cudaMalloc((void**)&cache[N], sizeof(BasisDev)), "basis alloc");
      SM_CK(cudaMemcpy(cache[N], &h, sizeof(BasisDev), cudaMemcpyHostToDevice), "basis upload");
    }
    b = cache[N];
  }
  SM_CK(launch_mortar_ops(b, N + 1, sigma, d_out, (cudaStream_t)stream), "mortar kernel");
  return SM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Batched stepping (sm_batch_*).
// ---------------------------------------------------------------------------------------
struct sm_batch {
  struct Group {
    int N = 0, riem = 0;
    std::vector<int> members;
    std::vector<BatchSolveDev> host;
    BatchSolveDev* d_bs = nullptr;
    int* d_offs_el = nullptr;
    int* d_offs_if = nullptr;
    int total_el = 0, total_if = 0;
    int grid_el = 0, grid_if = 0, tf = 8;
  };
  std::vector<sm_solver*> solvers;
  std::vector<double> dt;
  std::vector<Group> groups;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph = nullptr;
  int sms = 152;
};

namespace {

struct TuneKey { int N, riem, size_class; };
struct TuneVal { int tf, grid_if_per_sm, grid_el_per_sm; };
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, TuneVal>> g_tune;

int size_class(long long elems) { int c = 0; while (elems > 1) { elems >>= 1; ++c; } return c / 2; }

bool tune_lookup(const TuneKey& k, TuneVal* v) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto& p : g_tune)
    if (p.first.N == k.N && p.first.riem == k.riem && p.first.size_class == k.size_class) { *v = p.second; return true; }
  return false;
}
void tune_store(const TuneKey& k, const TuneVal& v) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto& p : g_tune)
    if (p.first.N == k.N && p.first.riem == k.riem && p.first.size_class == k.size_class) { p.second = v; return; }
  g_tune.push_back({k, v});
}

long long group_elems(const sm_batch& b, const sm_batch::Group& g) {
  long long e = 0;
  for (int i : g.members) e += b.solvers[i]->m.E;
  return e;
}

// interface work-item offsets for tile width tf
cudaError_t upload_if_offsets(sm_batch::Group& g, const sm_batch& b, int tf_req) {
  const int tf = batch_interface_tile(g.N, tf_req);
  std::vector<int> offs(g.members.size() + 1, 0);
  for (size_t q = 0; q < g.members.size(); ++q) {
    const MeshDev& m = b.solvers[g.members[q]]->m;
    offs[q + 1] = offs[q] + ((m.ny + tf - 1) / tf) * m.nz;
  }
  g.total_if = offs.back();
  g.tf = tf;
  return cudaMemcpy(g.d_offs_if, offs.data(), sizeof(int) * offs.size(), cudaMemcpyHostToDevice);
}

void free_batch(sm_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (auto& g : b->groups) {
    if (g.d_bs) cudaFree(g.d_bs);
    if (g.d_offs_el) cudaFree(g.d_offs_el);
    if (g.d_offs_if) cudaFree(g.d_offs_if);
  }
  delete b;
}

cudaError_t enqueue_batch_step(sm_batch* b, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 5; ++k)
    for (auto& g : b->groups) {
      const int n = (int)g.members.size();
      if ((e = launch_batch_stage_params(g.N, g.d_bs, n, RK_C[k], k == 4 ? 2 : 1, st)) != cudaSuccess) return e;
      if ((e = launch_batch_interface(g.N, g.riem, g.tf, g.d_bs, g.d_offs_if, n, g.grid_if, k, st)) != cudaSuccess) return e;
      if ((e = launch_batch_element(g.N, g.riem, k == 0 ? ELEM_STAGE_FIRST : ELEM_STAGE, g.d_bs, g.d_offs_el, n, g.grid_el,
                                    k, RK_A[k], RK_B[k], st)) != cudaSuccess)
        return e;
    }
  for (auto& g : b->groups)
    if ((e = launch_batch_flip(g.d_bs, (int)g.members.size(), st)) != cudaSuccess) return e;
  return e;
}

}  // namespace

extern "C" int sm_batch_create(sm_solver* const* solvers, const double* dt, int count, sm_batch** out) {
  if (!out || !solvers || !dt) return fail(SM_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (count < 1 || count > SM_MAX_BATCH) return fail(SM_ERR_ARG, "batch size must be in 1..1024");
  for (int i = 0; i < count; ++i) {
    if (!solvers[i]) return fail(SM_ERR_ARG, "NULL solver in batch");
    if (!(dt[i] > 0.0) || !std::isfinite(dt[i])) return fail(SM_ERR_ARG, "batch time steps must be positive");
    if (solvers[i]->prec != SM_FP32) return fail(SM_ERR_UNSUPPORTED, "batched kernels are FP32; step FP64 solvers with sm_step");
    if (solvers[i]->desc.physics != SM_EULER) return fail(SM_ERR_UNSUPPORTED, "batched kernels are Euler; step Navier-Stokes solvers with sm_step");
    if (solvers[i]->desc.geom != SM_GEOM_PLANE) return fail(SM_ERR_UNSUPPORTED, "batched kernels are for the plane interface");
    if (solvers[i]->desc.volume != SM_VOLUME_WEAK) return fail(SM_ERR_UNSUPPORTED, "batched kernels take the weak-form volume integral");
    if (solvers[i]->desc.periodic_x) return fail(SM_ERR_UNSUPPORTED, "batched kernels take one sliding interface");
  }
  sm_batch* b = new (std::nothrow) sm_batch();
  if (!b) return fail(SM_ERR_OOM, "host allocation");
  b->solvers.assign(solvers, solvers + count);
  b->dt.assign(dt, dt + count);
  int dev = 0;
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, (cudaGetDevice(&dev), dev));
  for (int i = 0; i < count; ++i) {
    const int N = solvers[i]->N, riem = solvers[i]->desc.riemann;
    sm_batch::Group* g = nullptr;
    for (auto& q : b->groups)
      if (q.N == N && q.riem == riem) g = &q;
    if (!g) {
      b->groups.emplace_back();
      g = &b->groups.back();
      g->N = N;
      g->riem = riem;
    }
    g->members.push_back(i);
  }
  cudaError_t e = cudaSuccess;
  for (auto& g : b->groups) {
    const int n = (int)g.members.size();
    std::vector<int> offs(n + 1, 0);
    const int epb = batch_elements_per_block(g.N);
    g.host.resize(n);
    for (int q = 0; q < n; ++q) {
      sm_solver* s = b->solvers[g.members[q]];
      BatchSolveDev& d = g.host[q];
      memset(&d, 0, sizeof(d));
      d.m = s->m;
      d.sp = s->sp;
      d.U[0] = s->U[0];
      d.U[1] = s->U[1];
      d.G = s->G;
      d.Fs = s->Fs;
      d.Fm = s->Fm;
      d.Ts = s->Ts;
      d.Tm = s->Tm;
      d.t_d = s->t_d;
      d.dt = b->dt[g.members[q]];
      d.cur = s->cur;
      offs[q + 1] = offs[q] + (int)((s->m.E + epb - 1) / epb);
    }
    g.total_el = offs.back();
    if ((e = cudaMalloc((void**)&g.d_bs, sizeof(BatchSolveDev) * n)) != cudaSuccess ||
        (e = cudaMalloc((void**)&g.d_offs_el, sizeof(int) * (n + 1))) != cudaSuccess ||
        (e = cudaMalloc((void**)&g.d_offs_if, sizeof(int) * (n + 1))) != cudaSuccess ||
        (e = cudaMemcpy(g.d_bs, g.host.data(), sizeof(BatchSolveDev) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(g.d_offs_el, offs.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = prepare_batch(g.N)) != cudaSuccess)
      break;
    TuneVal tv{8, 8, 0};
    const bool known = tune_lookup({g.N, g.riem, size_class(group_elems(*b, g))}, &tv);
    if ((e = upload_if_offsets(g, *b, known ? tv.tf : 8)) != cudaSuccess) break;
    g.grid_if = std::min(g.total_if, b->sms * (known ? tv.grid_if_per_sm : 8));
    g.grid_el = known && tv.grid_el_per_sm > 0 ? std::min(g.total_el, b->sms * tv.grid_el_per_sm) : g.total_el;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    free_batch(b);
    return fail(e == cudaErrorMemoryAllocation ? SM_ERR_OOM : SM_ERR_CUDA, "batch set-up", e);
  }
  *out = b;
  return SM_OK;
}

static int batch_autotune(sm_batch* b, void* stream, bool only_missing) {
  if (!b) return fail(SM_ERR_ARG, "NULL batch");
  cudaStream_t st = (cudaStream_t)stream;
  // the timed interface launches read the compact traces
  for (sm_solver* s : b->solvers) SM_CK(ensure_traces(s, st), "gather interface traces");
  cudaEvent_t e0, e1;
  SM_CK(cudaEventCreate(&e0), "event");
  SM_CK(cudaEventCreate(&e1), "event");
  auto timed = [&](auto&& launch) -> float {
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(e0, st);
      launch();
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best) best = ms;     // first launch is the warm-up
    }
    return best;
  };
  cudaError_t err = cudaSuccess;
  bool tuned = false;
  for (auto& g : b->groups) {
    const int n = (int)g.members.size();
    TuneVal known;
    if (only_missing && tune_lookup({g.N, g.riem, size_class(group_elems(*b, g))}, &known)) continue;
    tuned = true;
    // the stage parameters at each solve's current time (mode 1 with c = 0 writes only them)
    if ((err = launch_batch_stage_params(g.N, g.d_bs, n, 0.0, 1, st)) != cudaSuccess) break;
    int best_tf = g.tf, best_gif = g.grid_if;
    float best_if = 1e30f;
    for (int tf : {4, 8, 16}) {
      if (batch_interface_tile(g.N, tf) != tf) continue;   // the same kernel as a wider tile
      if ((err = upload_if_offsets(g, *b, tf)) != cudaSuccess) break;
      for (int per_sm : {2, 4, 8, 16, 0}) {
        const int grid = per_sm ? std::min(g.total_if, b->sms * per_sm) : g.total_if;
        const float ms = timed([&] { launch_batch_interface(g.N, g.riem, tf, g.d_bs, g.d_offs_if, n, grid, 0, st); });
        if (ms < best_if) { best_if = ms; best_tf = tf; best_gif = grid; }
      }
    }
    if (err != cudaSuccess) break;
    if ((err = upload_if_offsets(g, *b, best_tf)) != cudaSuccess) break;
    g.grid_if = best_gif;
    // element kernel in first-stage mode: writes only G and the other state buffer
    int best_gel = g.grid_el;
    float best_el = 1e30f;
    for (int per_sm : {2, 4, 6, 8, 12, 0}) {
      const int grid = per_sm ? std::min(g.total_el, b->sms * per_sm) : g.total_el;
      const float ms = timed([&] {
        launch_batch_element(g.N, g.riem, ELEM_STAGE_FIRST, g.d_bs, g.d_offs_el, n, grid, 0, RK_A[0], RK_B[0], st);
      });
      if (ms < best_el) { best_el = ms; best_gel = grid; }
    }
    g.grid_el = best_gel;
    const int gif_per_sm = best_gif >= g.total_if ? 0 : best_gif / b->sms;
    const int gel_per_sm = best_gel >= g.total_el ? 0 : best_gel / b->sms;
    tune_store({g.N, g.riem, size_class(group_elems(*b, g))}, {best_tf, gif_per_sm ? gif_per_sm : 1 << 20, gel_per_sm});
    if ((err = cudaGetLastError()) != cudaSuccess) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return fail(SM_ERR_CUDA, "autotune", err);
  if (tuned && b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  // the timed first-stage element launches wrote the traces of the spare buffer
  for (sm_solver* s : b->solvers) s->traces_ok = false;
  SM_CK(cudaStreamSynchronize(st), "autotune sync");
  return SM_OK;
}

extern "C" int sm_batch_autotune(sm_batch* b, void* stream) { return batch_autotune(b, stream, false); }

// Tunes only the groups whose (N, Riemann solver, size class) has no remembered shape.
int sm_batch_autotune_missing(sm_batch* b, void* stream) { return batch_autotune(b, stream, true); }

extern "C" int sm_batch_step(sm_batch* b, int nsteps, void* stream) {
  if (!b) return fail(SM_ERR_ARG, "NULL batch");
  if (nsteps < 0) return fail(SM_ERR_ARG, "nsteps must be >= 0");
  if (nsteps == 0) return SM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // the device copy of every solve's buffer parity follows the solver (it may have been
  // given a new state between batched steps)
  for (auto& g : b->groups) {
    bool changed = false;
    for (size_t q = 0; q < g.members.size(); ++q)
      if (g.host[q].cur != b->solvers[g.members[q]]->cur) { g.host[q].cur = b->solvers[g.members[q]]->cur; changed = true; }
    if (changed)
      SM_CK(cudaMemcpyAsync(g.d_bs, g.host.data(), sizeof(BatchSolveDev) * g.host.size(), cudaMemcpyHostToDevice, st),
            "batch parity upload");
  }
  for (sm_solver* s : b->solvers) SM_CK(ensure_traces(s, st), "gather interface traces");
  if (!b->graph) {
    SM_CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = enqueue_batch_step(b, b->cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return fail(SM_ERR_CUDA, "capture batch step", e); }
    if (e2 != cudaSuccess) return fail(SM_ERR_CUDA, "end capture", e2);
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { b->graph = nullptr; return fail(SM_ERR_CUDA, "instantiate batch graph", e); }
  }
  for (int n = 0; n < nsteps; ++n) {
    SM_CK(cudaGraphLaunch(b->graph, st), "batch graph launch");
    for (size_t i = 0; i < b->solvers.size(); ++i) {
      b->solvers[i]->cur ^= 1;
      b->solvers[i]->t_host += b->dt[i];
    }
    for (auto& g : b->groups)
      for (auto& h : g.host) h.cur ^= 1;
  }
  return SM_OK;
}

extern "C" int sm_batch_shapes(const sm_batch* b, int g, int* shape) {
  if (!b || !shape || g < 0 || g >= (int)b->groups.size()) return fail(SM_ERR_ARG, "invalid group");
  const auto& q = b->groups[g];
  shape[0] = q.N;
  shape[1] = q.tf;
  shape[2] = q.grid_if;
  shape[3] = q.grid_el;
  return (int)b->groups.size();
}

extern "C" void sm_batch_destroy(sm_batch* b) { free_batch(b); }

// ---------------------------------------------------------------------------------------
// Right-hand side without any device allocation (sm_rhs_static).
//
// Some callers cannot call cudaMalloc: code that runs while a framework owns the device
// memory through its own pool (allocating behind it breaks its accounting or fails once
// it has reserved the device), code inside regions where an allocation would synchronise
// the device (cudaMalloc and cudaFree wait for outstanding work), and embedders that
// forbid allocations after start-up.  For them the scratch of the right-hand side — the
// basis tables, the stage parameters (interface configuration and mortar operators) and
// both sides' interface face fluxes — lives in one file-scope device array of fixed size
// that every GPU loading this library holds until the process exits.
// ---------------------------------------------------------------------------------------
#define SM_STATIC_SCRATCH_BYTES (16u << 20)

static __device__ __align__(256) unsigned char g_static_scratch[SM_STATIC_SCRATCH_BYTES];
// The LGL basis tables of N = 1..7, written once per device when the entry point sets the
// device up, so that a call copies nothing from the host.
static __device__ BasisDev g_static_basis[7];

namespace {

std::mutex g_static_mu;
struct StaticDevice { unsigned char* scratch; BasisDev* basis; };
StaticDevice g_static_dev[256] = {};

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

// Once per device, with that device current: the device addresses of the scratch array and
// of the basis tables (filled here by a synchronous copy), and the kernels' attributes.
int static_device_setup(int dev, StaticDevice* out) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (dev < 0 || dev >= 256) return fail(SM_ERR_ARG, "device ordinal out of range");
  if (!g_static_dev[dev].scratch) {
    void* p = nullptr;
    void* pb = nullptr;
    SM_CK(cudaGetSymbolAddress(&p, g_static_scratch), "cudaGetSymbolAddress of the static scratch");
    SM_CK(cudaGetSymbolAddress(&pb, g_static_basis), "cudaGetSymbolAddress of the static basis tables");
    static BasisDev tables[7];
    for (int n = 1; n <= 7; ++n) lgl_basis(n, tables[n - 1]);
    SM_CK(cudaMemcpyToSymbol(g_static_basis, tables, sizeof(tables)), "upload the static basis tables");
    SM_CK(ensure_dhat_constants(), "derivative constants");
    for (int n = 1; n <= 7; ++n) {
      SM_CK(prepare_element_f64(n), "element kernel attributes");
      SM_CK(prepare_element_f32(n), "element kernel attributes");
      SM_CK(prepare_interface(n, SM_FP64), "interface kernel attributes");
      SM_CK(prepare_interface(n, SM_FP32), "interface kernel attributes");
    }
    g_static_dev[dev].basis = (BasisDev*)pb;
    g_static_dev[dev].scratch = (unsigned char*)p;
  }
  *out = g_static_dev[dev];
  return SM_OK;
}

size_t static_scratch_bytes(const sm_mesh_desc* desc) {
  if (!desc || desc->N < 1 || desc->N > 7) return 0;
  const size_t np = desc->N + 1, sb = desc->precision == SM_FP64 ? 8 : 4;
  const size_t faces = (size_t)desc->nel_static[1] * (size_t)desc->nel_static[2];
  return align256(sizeof(StageParams)) + 2 * align256(faces * 5 * np * np * sb);
}

}  // namespace

extern "C" int sm_rhs_static(const sm_mesh_desc* desc, const sm_motion* motion, double t, const void* dU,
                             void* dUt, void* stream) {
  int rc = valid_desc(desc);
  if (rc != SM_OK) return rc;
  if (desc->physics != SM_EULER) return fail(SM_ERR_UNSUPPORTED, "sm_rhs_static computes the Euler operator only");
  if (desc->geom != SM_GEOM_PLANE) return fail(SM_ERR_UNSUPPORTED, "sm_rhs_static computes the plane interface only");
  if (desc->volume != SM_VOLUME_WEAK) return fail(SM_ERR_UNSUPPORTED, "sm_rhs_static computes the weak-form operator only");
  if (desc->periodic_x) return fail(SM_ERR_UNSUPPORTED, "sm_rhs_static computes one sliding interface only");
  if (!motion || !dU || !dUt) return fail(SM_ERR_ARG, "NULL argument");
  if (dU == dUt) return fail(SM_ERR_ARG, "dU and dUt must not overlap");
  if (!aligned16(dU) || !aligned16(dUt)) return fail(SM_ERR_ARG, "device arrays must be 16-byte aligned");
  if (motion->omega != 0.0) return fail(SM_ERR_UNSUPPORTED, "rotation needs a rotating geometry");
  if (!std::isfinite(motion->v) || !std::isfinite(motion->delta0) || !std::isfinite(t))
    return fail(SM_ERR_ARG, "non-finite motion or time");
  if (desc->interface_conforming && (motion->v != 0.0 || motion->delta0 != 0.0))
    return fail(SM_ERR_ARG, "a conforming interface cannot move");
  const size_t need = static_scratch_bytes(desc);
  if (need > SM_STATIC_SCRATCH_BYTES) {
    char buf[200];
    snprintf(buf, sizeof(buf), "sm_rhs_static: needs %zu bytes of scratch, more than its fixed %u bytes "
             "(reduce the interface face count or use sm_rhs)", need, (unsigned)SM_STATIC_SCRATCH_BYTES);
    return fail(SM_ERR_ARG, buf);
  }
  int dev = 0;
  SM_CK(cudaGetDevice(&dev), "cudaGetDevice");
  StaticDevice sd;
  rc = static_device_setup(dev, &sd);
  if (rc != SM_OK) return rc;
  const int N = desc->N, np = N + 1, prec = desc->precision, sb = prec == SM_FP64 ? 8 : 4;
  StageParams* d_sp = (StageParams*)sd.scratch;
  unsigned char* d_fs = sd.scratch + align256(sizeof(StageParams));
  const size_t fbytes = (size_t)desc->nel_static[1] * desc->nel_static[2] * 5 * np * np * sb;
  unsigned char* d_fm = d_fs + align256(fbytes);
  // the mesh description as sm_init_mesh builds it for the plane interface, with the
  // device's basis table of degree N; the modes of the initial flow are not read by the
  // right-hand side's kernels (the weak Dirichlet state of that flow is its background)
  BasisDev basis;
  lgl_basis(N, basis);
  MeshDev m;
  mesh_from_desc(desc, m);
  m.v = motion->v;
  m.delta0 = motion->delta0;
  m.basis = sd.basis + (N - 1);
  m.modes = nullptr;
  fill_constants(m, basis, desc->fpar);
  // Every byte of the scratch the kernels read is written by this call first (the stage
  // parameters by the mapper kernel, every interface face by the interface kernel), so
  // nothing of a previous call's contents is used.  The call enqueues kernel launches only.
  cudaStream_t st = (cudaStream_t)stream;
  SM_CK(launch_stage_params(m, np, d_sp, nullptr, t, 0.0, 0.0, 0, st), "stage parameters");
  if (!desc->interface_conforming)
    SM_CK(launch_interface(N, prec, desc->riemann, m, d_sp, dU, d_fs, d_fm, st), "interface kernel");
  ElemArgs a{m, d_sp, dU, dUt, nullptr, d_fs, d_fm, 0.0, 0.0, 0.0};
  SM_CK(prec == SM_FP64 ? launch_element_f64(N, desc->riemann, ELEM_RHS, a, st)
                        : launch_element_f32(N, desc->riemann, ELEM_RHS, a, st), "element kernel");
  return SM_OK;
}

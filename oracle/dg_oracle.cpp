/*
 * ORACLE — test infrastructure only (see dg_oracle.h).
 *
 * Plain FP64 restatement of the sliding-mesh DGSEM method of arXiv 2008.04356:
 * compressible Euler equations in ALE form (Sec. 2, Eq. fluxes_written_out), weak-form
 * DGSEM on Legendre-Gauss-Lobatto nodes (Sec. 3.1, Eqs. transformed_equation,
 * weak_formulation), mortar projections for non-conforming faces (Sec. 3.2) and the
 * five-step sliding interface procedure (Sec. 3.3) with the displacement decomposition
 * and index relations of Sec. 4.3 (Eqs. subim, indices).
 *
 * Deliberately slow: no blocking, no fusion, loops written the way the formulas read.
 * Compiled with -ffp-contract=off so that no multiply-add is fused behind our back;
 * where the method needs a fused multiply-add (stage time, displacement) it calls fma().
 */
#include "dg_oracle.h"

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------------------ */
/* Legendre polynomials: three-term recurrence, value and first derivative.             */
/* ------------------------------------------------------------------------------------ */
void legendre(int n, double x, double* P, double* dP) {
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    double d2 = d0 + (2.0 * k - 1.0) * p1;   /* P_k' = P_{k-2}' + (2k-1) P_{k-1} */
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *P = p1; *dP = d1;
}

void invert(int n, const double* A, double* Ainv) {
  /* Gauss-Jordan elimination with partial pivoting. */
  std::vector<double> a(A, A + n * n), b(n * n, 0.0);
  for (int i = 0; i < n; ++i) b[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[r * n + c]) > std::fabs(a[piv * n + c])) piv = r;
    if (piv != c)
      for (int k = 0; k < n; ++k) { std::swap(a[c * n + k], a[piv * n + k]); std::swap(b[c * n + k], b[piv * n + k]); }
    double d = a[c * n + c];
    for (int k = 0; k < n; ++k) { a[c * n + k] /= d; b[c * n + k] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = a[r * n + c];
      for (int k = 0; k < n; ++k) { a[r * n + k] -= f * a[c * n + k]; b[r * n + k] -= f * b[c * n + k]; }
    }
  }
  std::memcpy(Ainv, b.data(), sizeof(double) * n * n);
}

long long floordiv128(__int128 a, __int128 b) {
  __int128 q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
  return (long long)q;
}

}  // namespace

extern "C" {

/* ====================================================================================
 * 1-D basis (Sec. 3.1: tensor-product Lagrange basis on LGL points, collocated
 * integration and interpolation).
 * ==================================================================================== */

/* N+1 Legendre-Gauss-Lobatto nodes: x_0=-1, x_N=+1 and the roots of P_N'.
 * Weights w_j = 2 / (N (N+1) P_N(x_j)^2). */
int orc_lgl(int N, double* x, double* w) {
  if (N < 1) return -1;
  for (int j = 0; j <= N; ++j) {
    double xj = -std::cos(PI * j / N);             /* Chebyshev-Lobatto start value */
    if (j > 0 && j < N) {
      for (int it = 0; it < 100; ++it) {
        double P, dP;
        legendre(N, xj, &P, &dP);
        /* Legendre ODE: (1-x^2) P'' = 2x P' - N(N+1) P */
        double ddP = (2.0 * xj * dP - N * (N + 1.0) * P) / (1.0 - xj * xj);
        double dx = dP / ddP;
        xj -= dx;
        if (std::fabs(dx) < 1e-16) break;
      }
    }
    x[j] = xj;
  }
  if (N % 2 == 0) x[N / 2] = 0.0;
  for (int j = 0; j <= N; ++j) {
    double P, dP;
    legendre(N, x[j], &P, &dP);
    w[j] = 2.0 / (N * (N + 1.0) * P * P);
  }
  return 0;
}

/* N+1 Legendre-Gauss nodes: roots of P_{N+1}; weights 2 / ((1-x^2) P_{N+1}'(x)^2). */
int orc_gl(int N, double* x, double* w) {
  int n = N + 1;
  for (int j = 0; j < n; ++j) {
    double xj = -std::cos(PI * (j + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(n, xj, &P, &dP);
      double dx = P / dP;
      xj -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double P, dP;
    legendre(n, xj, &P, &dP);
    x[j] = xj;
    w[j] = 2.0 / ((1.0 - xj * xj) * dP * dP);
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
  return 0;
}

/* ell_i(x) = prod_{k != i} (x - x_k) / (x_i - x_k), written out as the product. */
void orc_lagrange(int N, const double* nodes, double x, double* l) {
  for (int i = 0; i <= N; ++i) {
    double v = 1.0;
    for (int k = 0; k <= N; ++k)
      if (k != i) v *= (x - nodes[k]) / (nodes[i] - nodes[k]);
    l[i] = v;
  }
}

/* D[i][j] = ell_j'(x_i), from the product rule applied to the product above. */
void orc_dmatrix(int N, const double* nodes, double* D) {
  int np = N + 1;
  for (int i = 0; i < np; ++i) {
    double x = nodes[i];
    for (int j = 0; j < np; ++j) {
      double sum = 0.0;
      for (int m = 0; m < np; ++m) {
        if (m == j) continue;
        double prod = 1.0 / (nodes[j] - nodes[m]);
        for (int k = 0; k < np; ++k)
          if (k != j && k != m) prod *= (x - nodes[k]) / (nodes[j] - nodes[k]);
        sum += prod;
      }
      D[i * np + j] = sum;
    }
  }
}

/* Eq. proj_M: M_ij = int_{-1}^{1} ell_i ell_j dz, integrated exactly with N+1 Gauss points
 * (the integrand has degree 2N). */
void orc_mass_exact(int N, double* M) {
  int np = N + 1;
  std::vector<double> xl(np), wl(np), xg(np), wg(np), li(np);
  orc_lgl(N, xl.data(), wl.data());
  orc_gl(N, xg.data(), wg.data());
  for (int i = 0; i < np * np; ++i) M[i] = 0.0;
  for (int q = 0; q < np; ++q) {
    orc_lagrange(N, xl.data(), xg[q], li.data());
    for (int i = 0; i < np; ++i)
      for (int j = 0; j < np; ++j) M[i * np + j] += wg[q] * li[i] * li[j];
  }
}

/* ====================================================================================
 * Interface configuration (Sec. 4.3).
 *   Delta = (n + s) l,  n integer  -- reading: n = floor(Delta/l), s in [0,1).
 *   i_sub = 0 for the part of static face i with eta - i l < s l, else 1  (Eq. subim)
 *   moving partner of mortar (i, i_sub):  i~ = i - n + i_sub - 1           (Eq. indices)
 * ==================================================================================== */

void orc_map_closed(double delta, double l, long long* n, double* s) {
  double q = delta / l;
  double fq = std::floor(q);
  *n = (long long)fq;
  *s = q - fq;
}

void orc_map_pairs(long long n, int n_par, int* pairs) {
  for (int i = 0; i < n_par; ++i)
    for (int isub = 0; isub < 2; ++isub) {
      long long it = (long long)i - n + isub - 1;
      long long r = it % n_par;
      if (r < 0) r += n_par;
      pairs[2 * i + isub] = (int)r;
    }
}

/* Brute-force overlap search in exact integer arithmetic.  q = Delta/l is the same
 * rounded quotient as above; it is written as Q * 2^-K with integer Q, and all face
 * end points are then exact integers in units of 2^-K face lengths.  For every static
 * face i = [i, i+1] and every periodic image [a, a+1] of every moving face, the search
 * records which image covers the lower end of face i (the lower mortar, i_sub = 0) and
 * which image starts inside [i, i+1) (the upper mortar, i_sub = 1), checks that the
 * overlaps of positive length are exactly these, and reads n and s off the geometry.
 * Returns 0 on success, -1 outside the supported range (|q| >= 2^60 or ulp(q) < 2^-100),
 * -2 if the faces disagree on (n, s) (which would contradict equispaced faces). */
int orc_map_bruteforce(double delta, double l, int n_par, long long* n_out, double* s_out, int* pairs) {
  double q = delta / l;
  if (!(std::fabs(q) < 1152921504606846976.0)) return -1;  /* 2^60 */
  int e = 0;
  double m = std::frexp(q, &e);
  long long M = (long long)std::ldexp(m, 53);
  int K = 53 - e;
  __int128 Q = M;
  if (q == 0.0) { Q = 0; K = 0; }
  if (K < 0) { Q = Q << (-K); K = 0; }
  if (K > 100) return -1;
  const __int128 ONE = (__int128)1 << K;
  const __int128 PER = (__int128)n_par * ONE;
  long long n_ref = 0; __int128 s_ref = -1;
  for (int i = 0; i < n_par; ++i) {
    __int128 lo = (__int128)i * ONE, hi = lo + ONE;
    int lower = -1, upper = -1, npos = 0, pos_ok = 1;
    long long n_i = 0; __int128 s_i = 0;
    for (int j = 0; j < n_par; ++j) {
      /* images a_w = (j + w n_par) ONE + Q that can touch [lo - ONE, hi + ONE] */
      long long wc = floordiv128(lo - (__int128)j * ONE - Q, PER);
      for (long long w = wc - 2; w <= wc + 2; ++w) {
        __int128 a = ((__int128)j + (__int128)w * n_par) * ONE + Q, b = a + ONE;
        __int128 olo = a > lo ? a : lo, ohi = b < hi ? b : hi;
        int is_lower = (a < lo && lo <= b);
        int is_upper = (lo <= a && a < hi);
        if (ohi > olo) { ++npos; if (!is_lower && !is_upper) pos_ok = 0; }
        if (is_lower) { if (lower >= 0) return -2; lower = j; }
        if (is_upper) {
          if (upper >= 0) return -2;
          upper = j;
          n_i = i - (j + w * n_par);
          s_i = a - lo;
        }
      }
    }
    if (lower < 0 || upper < 0 || !pos_ok) return -2;
    if (npos != (s_i == 0 ? 1 : 2)) return -2;
    if (i == 0) { n_ref = n_i; s_ref = s_i; }
    else if (n_i != n_ref || s_i != s_ref) return -2;
    pairs[2 * i + 0] = lower;
    pairs[2 * i + 1] = upper;
  }
  *n_out = n_ref;
  *s_out = std::ldexp((double)s_ref, -K);   /* s < 1 carries at most q's 53 bits: exact */
  return 0;
}

/* ====================================================================================
 * Mortar operators (Sec. 3.2) for a face with hanging node sigma.
 *   lower mortar (xi <= sigma):  xi = -1    + (1+sigma)/2 (z+1),  Jacobian (1+sigma)/2
 *   upper mortar (xi >  sigma):  xi = sigma + (1-sigma)/2 (z+1),  Jacobian (1-sigma)/2
 *   S_ij = int ell_i(xi(z)) ell_j(z) dz (Eq. proj_S), exact with N+1 Gauss points.
 *   forward  P = M^-1 S^T  (Eq. projection_domain_mortar; reading: the face index i of S
 *            is summed against the face coefficients, so S enters transposed)
 *   backward B = J M^-1 S  (Eq. projection_mortar_domain, J the mortar's Jacobian)
 * Storage: P[j*np+i] maps face node i to mortar node j; B[i*np+j] maps mortar node j to
 * face node i.  At sigma = -1 or +1 one mortar is the whole face and the other has zero
 * length (Sec. 3.3); reading: the whole-face operators are then exactly the identity and
 * the zero-length mortar's B is exactly zero.
 * ==================================================================================== */
void orc_mortar_mats(int N, double sigma, double* P_lo, double* P_hi, double* B_lo, double* B_hi) {
  int np = N + 1;
  std::vector<double> xl(np), wl(np), xg(np), wg(np), M(np * np), Minv(np * np);
  std::vector<double> S_lo(np * np, 0.0), S_hi(np * np, 0.0), la(np), lb(np);
  orc_lgl(N, xl.data(), wl.data());
  orc_gl(N, xg.data(), wg.data());
  orc_mass_exact(N, M.data());
  invert(np, M.data(), Minv.data());
  double J_lo = (1.0 + sigma) / 2.0, J_hi = (1.0 - sigma) / 2.0;
  for (int qd = 0; qd < np; ++qd) {
    double z = xg[qd];
    orc_lagrange(N, xl.data(), z, lb.data());                        /* ell_j(z) */
    orc_lagrange(N, xl.data(), -1.0 + J_lo * (z + 1.0), la.data());  /* ell_i(xi_lo(z)) */
    for (int i = 0; i < np; ++i)
      for (int j = 0; j < np; ++j) S_lo[i * np + j] += wg[qd] * la[i] * lb[j];
    orc_lagrange(N, xl.data(), sigma + J_hi * (z + 1.0), la.data());  /* ell_i(xi_hi(z)) */
    for (int i = 0; i < np; ++i)
      for (int j = 0; j < np; ++j) S_hi[i * np + j] += wg[qd] * la[i] * lb[j];
  }
  for (int j = 0; j < np; ++j)
    for (int i = 0; i < np; ++i) {
      double plo = 0.0, phi = 0.0;
      for (int k = 0; k < np; ++k) { plo += Minv[j * np + k] * S_lo[i * np + k]; phi += Minv[j * np + k] * S_hi[i * np + k]; }
      P_lo[j * np + i] = plo;
      P_hi[j * np + i] = phi;
    }
  for (int i = 0; i < np; ++i)
    for (int j = 0; j < np; ++j) {
      double blo = 0.0, bhi = 0.0;
      for (int k = 0; k < np; ++k) { blo += Minv[i * np + k] * S_lo[k * np + j]; bhi += Minv[i * np + k] * S_hi[k * np + j]; }
      B_lo[i * np + j] = J_lo * blo;
      B_hi[i * np + j] = J_hi * bhi;
    }
  if (sigma == -1.0 || sigma == 1.0) {
    double* P_full = sigma == -1.0 ? P_hi : P_lo;
    double* B_full = sigma == -1.0 ? B_hi : B_lo;
    double* B_zero = sigma == -1.0 ? B_lo : B_hi;
    for (int a = 0; a < np; ++a)
      for (int b = 0; b < np; ++b) {
        P_full[a * np + b] = (a == b) ? 1.0 : 0.0;
        B_full[a * np + b] = (a == b) ? 1.0 : 0.0;
        B_zero[a * np + b] = 0.0;
      }
  }
}

/* ====================================================================================
 * Point fluxes.  Sec. 2, Eq. fluxes_written_out: convective flux in direction n minus the
 * grid-velocity transport (v^g . n) U; perfect gas p = (gamma-1)(rho e - rho |v|^2 / 2).
 * ==================================================================================== */
void orc_euler_flux(const double* U, const double* n, double vgn, double gamma, double* F) {
  double rho = U[0], u = U[1] / rho, v = U[2] / rho, w = U[3] / rho, E = U[4];
  double p = (gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v + w * w));
  double un = u * n[0] + v * n[1] + w * n[2];
  F[0] = rho * un - vgn * U[0];
  F[1] = U[1] * un + p * n[0] - vgn * U[1];
  F[2] = U[2] * un + p * n[1] - vgn * U[2];
  F[3] = U[3] * un + p * n[2] - vgn * U[3];
  F[4] = (E + p) * un - vgn * U[4];
}

/* Riemann solvers (Sec. 3.1) for a unit normal n pointing from L to R, ALE form.
 * kind 0: Rusanov, F* = (F_L + F_R)/2 - lambda_max (U_R - U_L)/2,
 *         lambda_max = max(|u_n - v^g_n| + c) over both states.
 * kind 1: Roe's approximate solver with the Harten-Hyman entropy fix; reading of the fix:
 *         for the two acoustic waves delta = max(0, lam_hat - lam_L, lam_R - lam_hat) and
 *         |lam_hat| is replaced by (lam_hat^2 + delta^2)/(2 delta) where |lam_hat| < delta.
 *         The grid velocity shifts every eigenvalue by -v^g_n; the eigenvectors are those of
 *         the fixed-grid Roe matrix. */
void orc_riemann(int kind, const double* UL, const double* UR, const double* n, double vgn,
                 double gamma, double* F) {
  double FL[5], FR[5];
  orc_euler_flux(UL, n, vgn, gamma, FL);
  orc_euler_flux(UR, n, vgn, gamma, FR);
  double rL = UL[0], uL = UL[1] / rL, vL = UL[2] / rL, wL = UL[3] / rL;
  double rR = UR[0], uR = UR[1] / rR, vR = UR[2] / rR, wR = UR[3] / rR;
  double pL = (gamma - 1.0) * (UL[4] - 0.5 * rL * (uL * uL + vL * vL + wL * wL));
  double pR = (gamma - 1.0) * (UR[4] - 0.5 * rR * (uR * uR + vR * vR + wR * wR));
  double cL = std::sqrt(gamma * pL / rL), cR = std::sqrt(gamma * pR / rR);
  double unL = uL * n[0] + vL * n[1] + wL * n[2];
  double unR = uR * n[0] + vR * n[1] + wR * n[2];
  if (kind == 0) {
    double a = std::fmax(std::fabs(unL - vgn) + cL, std::fabs(unR - vgn) + cR);
    for (int k = 0; k < 5; ++k) F[k] = 0.5 * (FL[k] + FR[k]) - 0.5 * a * (UR[k] - UL[k]);
    return;
  }
  /* Roe averages */
  double sL = std::sqrt(rL), sR = std::sqrt(rR);
  double HL = (UL[4] + pL) / rL, HR = (UR[4] + pR) / rR;
  double rh = sL * sR;
  double uh = (sL * uL + sR * uR) / (sL + sR);
  double vh = (sL * vL + sR * vR) / (sL + sR);
  double wh = (sL * wL + sR * wR) / (sL + sR);
  double Hh = (sL * HL + sR * HR) / (sL + sR);
  double q2 = uh * uh + vh * vh + wh * wh;
  double ch = std::sqrt((gamma - 1.0) * (Hh - 0.5 * q2));
  double unh = uh * n[0] + vh * n[1] + wh * n[2];
  double dr = rR - rL, dp = pR - pL, dun = unR - unL;
  double du = uR - uL, dv = vR - vL, dw = wR - wL;
  /* wave strengths */
  double a1 = (dp - rh * ch * dun) / (2.0 * ch * ch);
  double a5 = (dp + rh * ch * dun) / (2.0 * ch * ch);
  double a2 = dr - dp / (ch * ch);
  /* eigenvalues on the moving grid */
  double l1 = unh - ch - vgn, l2 = unh - vgn, l5 = unh + ch - vgn;
  double l1L = unL - cL - vgn, l1R = unR - cR - vgn;
  double l5L = unL + cL - vgn, l5R = unR + cR - vgn;
  double al1 = std::fabs(l1), al2 = std::fabs(l2), al5 = std::fabs(l5);
  double d1 = std::fmax(0.0, std::fmax(l1 - l1L, l1R - l1));
  if (al1 < d1) al1 = (l1 * l1 + d1 * d1) / (2.0 * d1);
  double d5 = std::fmax(0.0, std::fmax(l5 - l5L, l5R - l5));
  if (al5 < d5) al5 = (l5 * l5 + d5 * d5) / (2.0 * d5);
  /* |A| dU = sum of |lambda_k| alpha_k r_k */
  double D[5];
  double dutn = du - dun * n[0], dvtn = dv - dun * n[1], dwtn = dw - dun * n[2];
  D[0] = al1 * a1 + al2 * a2 + al5 * a5;
  D[1] = al1 * a1 * (uh - ch * n[0]) + al2 * (a2 * uh + rh * dutn) + al5 * a5 * (uh + ch * n[0]);
  D[2] = al1 * a1 * (vh - ch * n[1]) + al2 * (a2 * vh + rh * dvtn) + al5 * a5 * (vh + ch * n[1]);
  D[3] = al1 * a1 * (wh - ch * n[2]) + al2 * (a2 * wh + rh * dwtn) + al5 * a5 * (wh + ch * n[2]);
  D[4] = al1 * a1 * (Hh - unh * ch) + al2 * (a2 * 0.5 * q2 + rh * (uh * du + vh * dv + wh * dw - unh * dun))
       + al5 * a5 * (Hh + unh * ch);
  for (int k = 0; k < 5; ++k) F[k] = 0.5 * (FL[k] + FR[k]) - 0.5 * D[k];
}

/* Viscous fluxes (Sec. 2, Eqs. fluxes_written_out, stress_tensor, heat_flux): columns
 * i = x, y, z of F^v = (0, tau_1i, tau_2i, tau_3i, tau_ij v_j - q_i), Stokes' hypothesis
 * lambda = -2/3 mu, q = -k grad T with k = mu c_p / Pr, c_p = gamma R / (gamma - 1),
 * T = p / (rho R).  grad15[d*5 + c] is the derivative along x_d of primitive c of
 * (rho, v1, v2, v3, p); Fv15[i*5 + c] is component c of column i. */
void orc_viscous_flux(const double* U, const double* g, double mu, double Pr, double Rgas, double gamma,
                      double* Fv) {
  double rho = U[0], v[3] = {U[1] / rho, U[2] / rho, U[3] / rho};
  double p = (gamma - 1.0) * (U[4] - 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
  double T = p / (rho * Rgas);
  double k = mu * gamma * Rgas / ((gamma - 1.0) * Pr);
  double dv[3][3], dT[3];            /* dv[a][d] = d v_a / d x_d */
  for (int d = 0; d < 3; ++d) {
    for (int a = 0; a < 3; ++a) dv[a][d] = g[d * 5 + 1 + a];
    /* grad T = (grad p - T R grad rho) / (rho R) */
    dT[d] = (g[d * 5 + 4] - T * Rgas * g[d * 5 + 0]) / (rho * Rgas);
  }
  double div = dv[0][0] + dv[1][1] + dv[2][2];
  for (int i = 0; i < 3; ++i) {
    double tau[3];
    for (int a = 0; a < 3; ++a) tau[a] = mu * (dv[a][i] + dv[i][a]) + (a == i ? -2.0 / 3.0 * mu * div : 0.0);
    Fv[i * 5 + 0] = 0.0;
    for (int a = 0; a < 3; ++a) Fv[i * 5 + 1 + a] = tau[a];
    Fv[i * 5 + 4] = tau[0] * v[0] + tau[1] * v[1] + tau[2] * v[2] + k * dT[i];
  }
}

/* Two-point volume fluxes of the split-form DGSEM (Sec. 3.1: the split formulation of
 * Pirozzoli).  Reading: Pirozzoli's split of the convective terms d(rho w phi)/dx_n with
 * phi in {1, v, H}, the advecting velocity w = v.n - v^g.n being the velocity relative to
 * the moving grid (the ALE form of Sec. 2), written in two-point form as products of
 * arithmetic means {{a}} = (a_L + a_R) / 2:
 *   F#_rho = {{rho}} {{w}},   F#_rho v = F#_rho {{v}} + {{p}} n,   F#_rho e = F#_rho {{H}} + {{p}} v^g.n,
 * with the total enthalpy H = (rho e + p) / rho.  For U_L = U_R this is the ALE flux of
 * Eq. fluxes_written_out, F.n - (v^g.n) U, because rho H v^g.n - p v^g.n = rho e v^g.n.
 * kind 1 is the central flux (F(U_L) + F(U_R)) / 2, with which the split form equals the
 * weak form (summation-by-parts property of the LGL derivative). */
void orc_two_point_flux(int kind, const double* UL, const double* UR, const double* n, double vgn,
                        double gamma, double* F) {
  if (kind == 1) {
    double FL[5], FR[5];
    orc_euler_flux(UL, n, vgn, gamma, FL);
    orc_euler_flux(UR, n, vgn, gamma, FR);
    for (int k = 0; k < 5; ++k) F[k] = 0.5 * (FL[k] + FR[k]);
    return;
  }
  const double* S[2] = {UL, UR};
  double rho[2], vel[2][3], p[2], H[2];
  for (int s = 0; s < 2; ++s) {
    rho[s] = S[s][0];
    for (int a = 0; a < 3; ++a) vel[s][a] = S[s][1 + a] / rho[s];
    double q2 = vel[s][0] * vel[s][0] + vel[s][1] * vel[s][1] + vel[s][2] * vel[s][2];
    p[s] = (gamma - 1.0) * (S[s][4] - 0.5 * rho[s] * q2);
    H[s] = (S[s][4] + p[s]) / rho[s];
  }
  double rho_m = 0.5 * (rho[0] + rho[1]), p_m = 0.5 * (p[0] + p[1]), H_m = 0.5 * (H[0] + H[1]);
  double v_m[3];
  for (int a = 0; a < 3; ++a) v_m[a] = 0.5 * (vel[0][a] + vel[1][a]);
  double w_m = v_m[0] * n[0] + v_m[1] * n[1] + v_m[2] * n[2] - vgn;
  double f_rho = rho_m * w_m;
  F[0] = f_rho;
  for (int a = 0; a < 3; ++a) F[1 + a] = f_rho * v_m[a] + p_m * n[a];
  F[4] = f_rho * H_m + p_m * vgn;
}

/* Carpenter & Kennedy (1994) five-stage fourth-order 2N-storage coefficients, the scheme
 * Sec. 3.1 names for time integration (values are not printed in the paper):
 *   G = A_k G + dt R(U, t + c_k dt);  U = U + B_k G. */
void orc_lsrk_coeffs(double* A, double* B, double* c) {
  const double a[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                       -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
  const double b[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                       1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                       2277821191437.0 / 14882151754819.0};
  const double cc[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                        2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};
  for (int k = 0; k < 5; ++k) { A[k] = a[k]; B[k] = b[k]; c[k] = cc[k]; }
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  /* extern "C" */

/* ====================================================================================
 * The discrete operator on the two-block mesh.
 *   Element (ix, iy, iz) of a block maps its reference coordinates as
 *   xi^1 -> y (sliding direction), xi^2 -> z (perpendicular), xi^3 -> x (interface normal),
 *   node index i + np (j + np k) with i along xi^1, j along xi^2, k along xi^3.
 *   Global element id: static block first, e = ix + nx (iy + ny iz), then the moving block.
 *   State layout: U[(e*5 + var)*np^3 + node], conservative (rho, rho v1..3, rho e).
 * ==================================================================================== */
/* the curvilinear operator (dg_curved.cpp) */
void* orc_curved_create(const orc_problem* p);
void orc_curved_destroy(void* h);
long long orc_curved_nelem(void* h);
void orc_curved_coords(void* h, double t, double* xyz);
void orc_curved_fill(void* h, double t, double* U);
void orc_curved_metrics(void* h, double t, double* Ja, double* J);
void orc_curved_lifting(void* h, const double* U, double t, double* grad);
void orc_curved_interface(void* h, const double* U, double t, double* Fs, double* Fm);
void orc_curved_rhs(void* h, const double* U, double t, const long long* elems, int count, double* Ut);
void orc_curved_step(void* h, double* U, double* G, double* t, double dt, int nsteps);
void orc_curved_totals(void* h, const double* U, double* tot5);
double orc_curved_l2_error_rho(void* h, const double* U, double t);

namespace {

struct Oracle {
  int kind = 0;          /* 0: this Cartesian operator; 1: the curvilinear one (dg_curved.cpp) */
  orc_problem p;
  int N, np, nn;
  long long Es, Em, E;
  int ny, nz;
  double hy, hz, hx[2];
  std::vector<double> x, w, D, Dhat;
  double A[5], B[5], c[5];
  bool ns;   /* Navier-Stokes with BR1 lifting */
};

struct ElemId { int blk, ix, iy, iz; };

ElemId elem_id(const Oracle& o, long long e) {
  ElemId id;
  long long loc = e;
  id.blk = 0;
  int nx = o.p.nel_s[0];
  if (e >= o.Es) { id.blk = 1; loc = e - o.Es; nx = o.p.nel_m[0]; }
  id.ix = (int)(loc % nx);
  id.iy = (int)((loc / nx) % o.ny);
  id.iz = (int)(loc / ((long long)nx * o.ny));
  return id;
}

long long elem_index(const Oracle& o, int blk, int ix, int iy, int iz) {
  int nx = blk == 0 ? o.p.nel_s[0] : o.p.nel_m[0];
  long long base = blk == 0 ? 0 : o.Es;
  return base + ix + (long long)nx * (iy + (long long)o.ny * iz);
}

/* Displacement of the moving block at time t, fused as fma(v, t, delta0). */
double displacement(const Oracle& o, double t) { return std::fma(o.p.v, t, o.p.delta0); }

/* Physical position of node (i,j,k) of element id at time t. */
void node_xyz(const Oracle& o, const ElemId& id, int i, int j, int k, double t, double* X) {
  double xlo = id.blk == 0 ? o.p.x0 : o.p.x1;
  double hx = o.hx[id.blk];
  X[0] = xlo + id.ix * hx + (o.x[k] + 1.0) * 0.5 * hx;
  X[1] = o.p.y0 + id.iy * o.hy + (o.x[i] + 1.0) * 0.5 * o.hy;
  X[2] = o.p.z0 + id.iz * o.hz + (o.x[j] + 1.0) * 0.5 * o.hz;
  if (id.blk == 1) X[1] += displacement(o, t);
}

void prim_to_cons(const double* P, double gamma, double* U) {
  U[0] = P[0];
  U[1] = P[0] * P[1];
  U[2] = P[0] * P[2];
  U[3] = P[0] * P[3];
  U[4] = P[4] / (gamma - 1.0) + 0.5 * P[0] * (P[1] * P[1] + P[2] * P[2] + P[3] * P[3]);
}

void cons_to_prim(const double* U, double gamma, double* Q) {
  Q[0] = U[0];
  Q[1] = U[1] / U[0];
  Q[2] = U[2] / U[0];
  Q[3] = U[3] / U[0];
  Q[4] = (gamma - 1.0) * (U[4] - 0.5 * U[0] * (Q[1] * Q[1] + Q[2] * Q[2] + Q[3] * Q[3]));
}

/* The flows used as initial data and as Dirichlet boundary states.
 *  0: constant primitive state fpar[0..4].
 *  1: entropy wave rho = fpar0 + fpar1 sin(2 pi k.(x - u t)), k = fpar2..4, u = fpar5..7,
 *     p = fpar8 (an exact solution of the Euler equations).
 *  2: background primitive state fpar[0..4] plus, per primitive variable, 8 modes
 *     amp sin(2 pi (ky y + kz z) + phase); the boundary state is the background.
 *  3: rho = fpar0 + fpar1 x' + fpar2 x'^2 + fpar3 x'^3 with x' = x - fpar4 t,
 *     velocity fpar4..6, p = fpar7 (exact solution; polynomial in x). */
void flow_state(const orc_problem& p, const double* X, double t, int boundary, double* U) {
  double P[5];
  const double* f = p.fpar;
  switch (p.flow) {
    case 0: for (int k = 0; k < 5; ++k) P[k] = f[k]; break;
    case 1: {
      double ph = f[2] * (X[0] - f[5] * t) + f[3] * (X[1] - f[6] * t) + f[4] * (X[2] - f[7] * t);
      P[0] = f[0] + f[1] * std::sin(2.0 * PI * ph);
      P[1] = f[5]; P[2] = f[6]; P[3] = f[7]; P[4] = f[8];
      break;
    }
    case 2: {
      for (int k = 0; k < 5; ++k) P[k] = f[k];
      if (!boundary)
        for (int k = 0; k < 5; ++k)
          for (int m = 0; m < 8; ++m) {
            const double* md = p.modes[k][m];
            P[k] += md[0] * std::sin(2.0 * PI * (md[1] * X[1] + md[2] * X[2]) + md[3]);
          }
      break;
    }
    case 3: {
      double xs = X[0] - f[4] * t;
      P[0] = f[0] + xs * (f[1] + xs * (f[2] + xs * f[3]));
      P[1] = f[4]; P[2] = f[5]; P[3] = f[6]; P[4] = f[7];
      break;
    }
    case 4: {
      /* rho = fpar0, p = fpar1, velocity (0, 0, w(x)) with w = fpar2 + fpar3 x + fpar4 x^2 */
      P[0] = f[0];
      P[1] = 0.0; P[2] = 0.0;
      P[3] = f[2] + X[0] * (f[3] + X[0] * f[4]);
      P[4] = f[1];
      break;
    }
    case 5: {
      /* axial stream (0, 0, fpar2) with a Gaussian pressure pulse of amplitude fpar3 and
       * width fpar7 centred at (r, theta, z) = (fpar4, fpar5, fpar6) */
      double xc = f[4] * std::cos(f[5]), yc = f[4] * std::sin(f[5]), zc = f[6];
      double d2 = (X[0] - xc) * (X[0] - xc) + (X[1] - yc) * (X[1] - yc) + (X[2] - zc) * (X[2] - zc);
      P[0] = f[0];
      P[1] = 0.0; P[2] = 0.0; P[3] = f[2];
      P[4] = f[1] + (boundary ? 0.0 : f[3] * std::exp(-d2 / (2.0 * f[7] * f[7])));
      break;
    }
    default: {
      /* 6: rigid rotation with angular speed fpar2 about the z axis */
      double r2 = X[0] * X[0] + X[1] * X[1];
      P[0] = f[0];
      P[1] = -f[2] * X[1]; P[2] = f[2] * X[0]; P[3] = 0.0;
      P[4] = f[1] + 0.5 * f[0] * f[2] * f[2] * r2;
      break;
    }
  }
  prim_to_cons(P, p.gamma, U);
}

/* Face geometry helpers.  dir d in {0,1,2} is the reference direction xi^{d+1};
 * its physical axis is y, z, x respectively.  Face nodes are numbered a + np b:
 *   d=0: (a,b) = (j,k);  d=1: (a,b) = (i,k);  d=2: (a,b) = (i,j). */
int phys_axis(int d) { return d == 0 ? 1 : (d == 1 ? 2 : 0); }

int face_node_to_vol(const Oracle& o, int d, int side, int a, int b) {
  int f = side == 0 ? 0 : o.N;
  if (d == 0) return f + o.np * (a + o.np * b);
  if (d == 1) return a + o.np * (f + o.np * b);
  return a + o.np * (b + o.np * f);
}

/* |Ja^d|: surface element of the xi^{d+1} faces; Jacobian det = hx hy hz / 8. */
double metric(const Oracle& o, int blk, int d) {
  double hx = o.hx[blk];
  if (d == 0) return o.hz * hx / 4.0;
  if (d == 1) return hx * o.hy / 4.0;
  return o.hy * o.hz / 4.0;
}
double jacobian(const Oracle& o, int blk) { return o.hx[blk] * o.hy * o.hz / 8.0; }

/* Grid velocity (v^g) component along the physical axis of direction d. */
double grid_vel(const Oracle& o, int blk, int d) {
  return (blk == 1 && phys_axis(d) == 1) ? o.p.v : 0.0;
}

void unit_normal(int d, double* n) {
  n[0] = n[1] = n[2] = 0.0;
  n[phys_axis(d)] = 1.0;
}

/* ---------------------- Sliding interface (Sec. 3.3, five steps) ------------------- */
struct Interface {
  long long n; double s, sig_s, sig_m;
  std::vector<double> Ps_lo, Ps_hi, Bs_lo, Bs_hi, Pm_lo, Pm_hi, Bm_lo, Bm_hi;
};

/* Step 1: dynamic definition of the interface at time t (Sec. 4.3). */
void interface_config(const Oracle& o, double t, Interface& I) {
  double delta = displacement(o, t);
  orc_map_closed(delta, o.hy, &I.n, &I.s);
  I.sig_s = 2.0 * I.s - 1.0;      /* hanging node in the static face's reference coordinate */
  I.sig_m = 1.0 - 2.0 * I.s;      /* ... and in the moving face's */
  int nq = o.np * o.np;
  for (auto* v : {&I.Ps_lo, &I.Ps_hi, &I.Bs_lo, &I.Bs_hi, &I.Pm_lo, &I.Pm_hi, &I.Bm_lo, &I.Bm_hi}) v->assign(nq, 0.0);
  orc_mortar_mats(o.N, I.sig_s, I.Ps_lo.data(), I.Ps_hi.data(), I.Bs_lo.data(), I.Bs_hi.data());
  orc_mortar_mats(o.N, I.sig_m, I.Pm_lo.data(), I.Pm_hi.data(), I.Bm_lo.data(), I.Bm_hi.data());
}

int wrap(long long i, int n) { long long r = i % n; if (r < 0) r += n; return (int)r; }

/* Face trace on interface ifc.  Interface 0 (x = x1): static face (i, iperp) is the
 * xi^3 = +1 face of static element (nx-1, i, iperp), moving face (i~, iperp) the xi^3 = -1
 * face of moving element (0, i~, iperp).  Interface 1 (x = x0 = x2, periodic x): static face
 * the xi^3 = -1 face of static element (0, i, iperp), moving face the xi^3 = +1 face of
 * moving element (nx-1, i~, iperp).  tr[(v*np + q)*np + p], p along xi^1 (sliding), q along
 * xi^2. */
void interface_trace(const Oracle& o, const double* U, int blk, int ipar, int iperp, double* tr, int ifc = 0) {
  int ix = ifc == 0 ? (blk == 0 ? o.p.nel_s[0] - 1 : 0) : (blk == 0 ? 0 : o.p.nel_m[0] - 1);
  int side = (blk == 0) == (ifc == 0) ? 1 : 0;
  long long e = elem_index(o, blk, ix, ipar, iperp);
  for (int v = 0; v < 5; ++v)
    for (int q = 0; q < o.np; ++q)
      for (int p = 0; p < o.np; ++p)
        tr[(v * o.np + q) * o.np + p] = U[(e * 5 + v) * o.nn + face_node_to_vol(o, 2, side, p, q)];
}

/* Trace of the lifted gradients on the interface: grad[((e*3 + d)*5 + c)*nn + node],
 * tr[(k*np + q)*np + p] with k = 5 d + c (15 components). */
void interface_grad_trace(const Oracle& o, const double* grad, int blk, int ipar, int iperp, double* tr) {
  int ix = blk == 0 ? o.p.nel_s[0] - 1 : 0;
  int side = blk == 0 ? 1 : 0;
  long long e = elem_index(o, blk, ix, ipar, iperp);
  for (int k = 0; k < 15; ++k)
    for (int q = 0; q < o.np; ++q)
      for (int p = 0; p < o.np; ++p)
        tr[(k * o.np + q) * o.np + p] = grad[(e * 15 + k) * o.nn + face_node_to_vol(o, 2, side, p, q)];
}

/* Normal viscous flux (F^v . e_axis) at a point from state U and the 15 gradients. */
void viscous_normal(const Oracle& o, const double* U, const double* g15, int axis, double* Fn) {
  double Fv[15];
  orc_viscous_flux(U, g15, o.p.mu, o.p.Pr, o.p.Rgas, o.p.gamma, Fv);
  for (int c = 0; c < 5; ++c) Fn[c] = Fv[axis * 5 + c];
}

/* Step 3: L2 projection of a face trace onto a mortar, along the sliding direction only
 * (the mortar and face nodes line up along the perpendicular lines, Sec. 3.2). */
void project_to_mortar(const Oracle& o, const double* P, const double* tr, double* Q, int ncomp = 5) {
  for (int v = 0; v < ncomp; ++v)
    for (int q = 0; q < o.np; ++q)
      for (int j = 0; j < o.np; ++j) {
        double acc = 0.0;
        for (int i = 0; i < o.np; ++i) acc += P[j * o.np + i] * tr[(v * o.np + q) * o.np + i];
        Q[(v * o.np + q) * o.np + j] = acc;
      }
}

/* Steps 2-4 for one mortar (ipar, iperp, isub) of interface ifc (mortar index of Sec. 4.3,
 * with the interface as the outermost key): primary (static) and replica (moving) states on
 * the mortar, then the Riemann flux along the static face's outward normal (+x on interface
 * 0, -x on interface 1), scaled by the static face's surface element.  Both interfaces see
 * the same displacement, hence the same partners (Eq. indices) and operators. */
void mortar_flux(const Oracle& o, const Interface& I, const double* U, const double* grad, int ipar, int iperp,
                 int isub, double* Fm, int ifc = 0) {
  int nq = o.np * o.np;
  std::vector<double> tr(15 * nq), QL(5 * nq), QR(5 * nq), GL(15 * nq), GR(15 * nq);
  const double* Ps = isub == 0 ? I.Ps_lo.data() : I.Ps_hi.data();
  /* the static lower mortar is the upper part of the moving face, and vice versa */
  const double* Pm = isub == 0 ? I.Pm_hi.data() : I.Pm_lo.data();
  int it = wrap((long long)ipar - I.n + isub - 1, o.ny);          /* Eq. indices */
  interface_trace(o, U, 0, ipar, iperp, tr.data(), ifc);
  project_to_mortar(o, Ps, tr.data(), QL.data());
  interface_trace(o, U, 1, it, iperp, tr.data(), ifc);
  project_to_mortar(o, Pm, tr.data(), QR.data());
  if (grad) {   /* gradients projected onto the mortars like the solution (Sec. 3.2) */
    interface_grad_trace(o, grad, 0, ipar, iperp, tr.data());
    project_to_mortar(o, Ps, tr.data(), GL.data(), 15);
    interface_grad_trace(o, grad, 1, it, iperp, tr.data());
    project_to_mortar(o, Pm, tr.data(), GR.data(), 15);
  }
  double n[3] = {1.0, 0.0, 0.0}, sJ = metric(o, 0, 2);
  for (int q = 0; q < o.np; ++q)
    for (int j = 0; j < o.np; ++j) {
      double ul[5], ur[5], f[5];
      for (int v = 0; v < 5; ++v) { ul[v] = QL[(v * o.np + q) * o.np + j]; ur[v] = QR[(v * o.np + q) * o.np + j]; }
      if (ifc == 0) orc_riemann(o.p.riemann, ul, ur, n, 0.0, o.p.gamma, f);
      else {
        /* x = x0 = x2: the moving state is on the minus side; the flux in canonical
         * orientation (minus side left, normal +x), negated for the static outward normal */
        orc_riemann(o.p.riemann, ur, ul, n, 0.0, o.p.gamma, f);
        for (int v = 0; v < 5; ++v) f[v] = -f[v];
      }
      if (grad) {   /* BR1: mean of both sides' viscous fluxes */
        double gl[15], gr[15], fl[5], fr[5];
        for (int k = 0; k < 15; ++k) { gl[k] = GL[(k * o.np + q) * o.np + j]; gr[k] = GR[(k * o.np + q) * o.np + j]; }
        viscous_normal(o, ul, gl, 0, fl);
        viscous_normal(o, ur, gr, 0, fr);
        for (int v = 0; v < 5; ++v) f[v] -= 0.5 * (fl[v] + fr[v]);
      }
      for (int v = 0; v < 5; ++v) Fm[(v * o.np + q) * o.np + j] = f[v] * sJ;
    }
}

/* BR1 lifting on one mortar: mean of both sides' projected primitive traces, times the
 * static face's surface element (its outward normal is +x). */
void mortar_lift(const Oracle& o, const Interface& I, const double* U, int ipar, int iperp, int isub, double* Lm) {
  int nq = o.np * o.np;
  std::vector<double> tr(5 * nq), pr(5 * nq), QL(5 * nq), QR(5 * nq);
  auto prim_trace = [&](int blk, int i) {
    interface_trace(o, U, blk, i, iperp, tr.data());
    for (int ab = 0; ab < nq; ++ab) {
      double u[5], q[5];
      for (int v = 0; v < 5; ++v) u[v] = tr[v * nq + ab];
      cons_to_prim(u, o.p.gamma, q);
      for (int v = 0; v < 5; ++v) pr[v * nq + ab] = q[v];
    }
  };
  prim_trace(0, ipar);
  project_to_mortar(o, isub == 0 ? I.Ps_lo.data() : I.Ps_hi.data(), pr.data(), QL.data());
  prim_trace(1, wrap((long long)ipar - I.n + isub - 1, o.ny));
  project_to_mortar(o, isub == 0 ? I.Pm_hi.data() : I.Pm_lo.data(), pr.data(), QR.data());
  double sJ = metric(o, 0, 2);
  for (int k = 0; k < 5 * nq; ++k) Lm[k] = sJ * 0.5 * (QL[k] + QR[k]);
}

/* Step 5: projection of the mortar fluxes back onto a face, F = B_lo F_lo + B_hi F_hi. */
void project_to_face(const Oracle& o, const double* B_lo, const double* F_lo, const double* B_hi,
                     const double* F_hi, double sign, double* F) {
  for (int v = 0; v < 5; ++v)
    for (int q = 0; q < o.np; ++q)
      for (int i = 0; i < o.np; ++i) {
        double acc = 0.0;
        for (int j = 0; j < o.np; ++j) acc += B_lo[i * o.np + j] * F_lo[(v * o.np + q) * o.np + j];
        for (int j = 0; j < o.np; ++j) acc += B_hi[i * o.np + j] * F_hi[(v * o.np + q) * o.np + j];
        F[(v * o.np + q) * o.np + i] = sign * acc;
      }
}

/* Outward flux (times surface element) on static face (ipar, iperp) of interface ifc. */
void static_face_flux(const Oracle& o, const Interface& I, const double* U, const double* grad, int ipar, int iperp,
                      double* F, int ifc = 0) {
  int nq = o.np * o.np;
  std::vector<double> F0(5 * nq), F1(5 * nq);
  mortar_flux(o, I, U, grad, ipar, iperp, 0, F0.data(), ifc);
  mortar_flux(o, I, U, grad, ipar, iperp, 1, F1.data(), ifc);
  project_to_face(o, I.Bs_lo.data(), F0.data(), I.Bs_hi.data(), F1.data(), 1.0, F);
}

/* Outward flux on moving face (it, iperp) of interface ifc: its lower part (xi~ <= sigma~)
 * is mortar (it + n, 1), its upper part mortar (it + n + 1, 0); the moving side's outward
 * normal is opposite to the static side's, hence the sign. */
void moving_face_flux(const Oracle& o, const Interface& I, const double* U, const double* grad, int it, int iperp,
                      double* F, int ifc = 0) {
  int nq = o.np * o.np;
  std::vector<double> Flo(5 * nq), Fhi(5 * nq);
  mortar_flux(o, I, U, grad, wrap((long long)it + I.n, o.ny), iperp, 1, Flo.data(), ifc);
  mortar_flux(o, I, U, grad, wrap((long long)it + I.n + 1, o.ny), iperp, 0, Fhi.data(), ifc);
  project_to_face(o, I.Bm_lo.data(), Flo.data(), I.Bm_hi.data(), Fhi.data(), -1.0, F);
}

/* ------------------------------ DGSEM element operator ------------------------------ */

/* Outward surface flux (times |Ja^d|) on face (d, side) of element e, at the face nodes.
 * Conforming faces use the flux in canonical orientation (minus element left, normal
 * +axis) so that both neighbours see the same number; Dirichlet faces use the exact flow
 * state outside (weak boundary condition); interface faces come from the mortars. */
void face_flux_out(const Oracle& o, const Interface* I, const double* U, const double* grad, double t, long long e,
                   int d, int side, const std::vector<double>* Fsl_static, const std::vector<double>* Fsl_moving,
                   double* Fout) {
  ElemId id = elem_id(o, e);
  int np = o.np, nq = np * np;
  int nx = id.blk == 0 ? o.p.nel_s[0] : o.p.nel_m[0];
  double sJ = metric(o, id.blk, d), vgn = grid_vel(o, id.blk, d);
  double n[3];
  unit_normal(d, n);
  /* classify the neighbour */
  long long nb = -1; int nb_blk = id.blk; int kind = 0;  /* 0 conforming, 1 boundary, 2 interface */
  int ifc = 0;                                           /* interface 0 (x = x1) or 1 (x = x0 = x2) */
  if (d == 0) nb = elem_index(o, id.blk, id.ix, wrap(id.iy + (side ? 1 : -1), o.ny), id.iz);
  else if (d == 1) nb = elem_index(o, id.blk, id.ix, id.iy, wrap(id.iz + (side ? 1 : -1), o.nz));
  else {
    int jx = id.ix + (side ? 1 : -1);
    bool outer = (id.blk == 0 && side == 0) || (id.blk == 1 && side == 1);
    if (jx >= 0 && jx < nx) nb = elem_index(o, id.blk, jx, id.iy, id.iz);
    else if (outer && !o.p.periodic_x) kind = 1;
    else if (o.p.interface_conforming) {
      /* the other block's element across the interface: across x = x1 the static
       * element nx-1 meets moving element 0; across x = x0 = x2 static element 0 meets
       * moving element nx-1 */
      nb_blk = 1 - id.blk;
      int nb_ix = nb_blk == 0 ? (outer ? 0 : o.p.nel_s[0] - 1) : (outer ? o.p.nel_m[0] - 1 : 0);
      nb = elem_index(o, nb_blk, nb_ix, id.iy, id.iz);
    } else {
      kind = 2;
      ifc = outer ? 1 : 0;
    }
  }
  if (kind == 2) {
    const std::vector<double>* src = id.blk == 0 ? Fsl_static : Fsl_moving;
    if (src) {
      long long nf = (long long)o.ny * o.nz;
      const double* F = src->data() + ((long long)ifc * nf + (long long)id.iz * o.ny + id.iy) * 5 * nq;
      for (int v = 0; v < 5; ++v)
        for (int ab = 0; ab < nq; ++ab) Fout[v * nq + ab] = F[v * nq + ab];
    } else if (id.blk == 0) static_face_flux(o, *I, U, grad, id.iy, id.iz, Fout, ifc);
    else moving_face_flux(o, *I, U, grad, id.iy, id.iz, Fout, ifc);
    return;
  }
  for (int b = 0; b < np; ++b)
    for (int a = 0; a < np; ++a) {
      double uin[5], uout[5], f[5];
      int vn = face_node_to_vol(o, d, side, a, b);
      for (int v = 0; v < 5; ++v) uin[v] = U[(e * 5 + v) * o.nn + vn];
      if (kind == 1) {
        int i = vn % np, j = (vn / np) % np, k = vn / nq;
        double X[3];
        node_xyz(o, id, i, j, k, t, X);
        flow_state(o.p, X, t, 1, uout);
      } else {
        int vnn = face_node_to_vol(o, d, 1 - side, a, b);
        for (int v = 0; v < 5; ++v) uout[v] = U[(nb * 5 + v) * o.nn + vnn];
      }
      if (side == 1) orc_riemann(o.p.riemann, uin, uout, n, vgn, o.p.gamma, f);
      else orc_riemann(o.p.riemann, uout, uin, n, vgn, o.p.gamma, f);
      if (grad) {
        /* BR1 viscous face flux: mean of both sides' viscous fluxes; at a weak Dirichlet
         * face the exterior flux takes the exterior state with the interior gradients */
        double gin[15], gout[15], fi[5], fo[5];
        for (int k = 0; k < 15; ++k) {
          gin[k] = grad[(e * 15 + k) * o.nn + vn];
          gout[k] = kind == 1 ? gin[k] : grad[(nb * 15 + k) * o.nn + face_node_to_vol(o, d, 1 - side, a, b)];
        }
        viscous_normal(o, uin, gin, phys_axis(d), fi);
        viscous_normal(o, uout, gout, phys_axis(d), fo);
        for (int v = 0; v < 5; ++v) f[v] -= 0.5 * (fi[v] + fo[v]);
      }
      double sg = side == 1 ? 1.0 : -1.0;
      for (int v = 0; v < 5; ++v) Fout[v * nq + a + np * b] = sg * sJ * f[v];
    }
}

/* Split-form DGSEM residual of one element (Sec. 3.1, the split formulation with
 * Pirozzoli's flux), on a Cartesian element, where the contravariant two-point flux of
 * direction xi^{d+1} is |Ja^d| F#(U_a, U_b) along that direction's physical axis.  Strong
 * form, the volume term carried by the two-point flux:
 *   J dU/dt = - sum_d sum_l 2 D_il |Ja^d| F#^d(U_node, U_l)        (l along xi^{d+1})
 *             - sum_faces ell(+-1)/w (F* . N - F(U_node) . N) sJ ,
 * the surface term being the Riemann flux minus the node's own flux.  Navier-Stokes (grad
 * given, the BR1 gradients): the viscous flux keeps the weak form of the weak-form residual,
 *   + sum_d sum_l Dhat_il |Ja^d| F^v_d(U_l, grad_l),
 * and the face flux F* carries the BR1 viscous mean, F* = F*_adv - {{F^v}} . N (the node's
 * own flux subtracted is the advective one only). */
void split_element_residual(const Oracle& o, const Interface* I, const double* U, const double* grad, double t,
                            long long e, const std::vector<double>* Fs, const std::vector<double>* Fm,
                            double* Ut_e) {
  ElemId id = elem_id(o, e);
  int np = o.np, nn = o.nn, nq = np * np;
  int kind = o.p.volume == 2 ? 1 : 0;
  for (int k = 0; k < np; ++k)
    for (int j = 0; j < np; ++j)
      for (int i = 0; i < np; ++i) {
        int node = i + np * (j + np * k);
        double u[5], ul[5], f[5], n[3], acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * nn + node];
        for (int d = 0; d < 3; ++d) {
          unit_normal(d, n);
          double vgn = grid_vel(o, id.blk, d), a = metric(o, id.blk, d);
          int row = d == 0 ? i : (d == 1 ? j : k);
          for (int l = 0; l < np; ++l) {
            int nl = d == 0 ? l + np * (j + np * k) : (d == 1 ? i + np * (l + np * k) : i + np * (j + np * l));
            for (int v = 0; v < 5; ++v) ul[v] = U[(e * 5 + v) * nn + nl];
            orc_two_point_flux(kind, u, ul, n, vgn, o.p.gamma, f);
            for (int v = 0; v < 5; ++v) acc[v] += 2.0 * o.D[row * np + l] * a * f[v];
          }
        }
        for (int v = 0; v < 5; ++v) Ut_e[v * nn + node] = -acc[v];
      }
  if (grad) {
    std::vector<double> Fvt(3 * 5 * nn);     /* |Ja^d| F^v along xi^{d+1}'s physical axis */
    for (int node = 0; node < nn; ++node) {
      double u[5], g15[15], Fv[15];
      for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * nn + node];
      for (int k = 0; k < 15; ++k) g15[k] = grad[(e * 15 + k) * nn + node];
      orc_viscous_flux(u, g15, o.p.mu, o.p.Pr, o.p.Rgas, o.p.gamma, Fv);
      for (int d = 0; d < 3; ++d)
        for (int v = 0; v < 5; ++v) Fvt[(d * 5 + v) * nn + node] = metric(o, id.blk, d) * Fv[phys_axis(d) * 5 + v];
    }
    for (int v = 0; v < 5; ++v)
      for (int k = 0; k < np; ++k)
        for (int j = 0; j < np; ++j)
          for (int i = 0; i < np; ++i) {
            double acc = 0.0;
            for (int l = 0; l < np; ++l) {
              acc += o.Dhat[i * np + l] * Fvt[(0 * 5 + v) * nn + l + np * (j + np * k)];
              acc += o.Dhat[j * np + l] * Fvt[(1 * 5 + v) * nn + i + np * (l + np * k)];
              acc += o.Dhat[k * np + l] * Fvt[(2 * 5 + v) * nn + i + np * (j + np * l)];
            }
            Ut_e[v * nn + i + np * (j + np * k)] += acc;
          }
  }
  std::vector<double> Fout(5 * nq);
  for (int d = 0; d < 3; ++d)
    for (int side = 0; side < 2; ++side) {
      face_flux_out(o, I, U, grad, t, e, d, side, Fs, Fm, Fout.data());
      double wend = o.w[side == 0 ? 0 : o.N], sJ = metric(o, id.blk, d), sg = side == 1 ? 1.0 : -1.0;
      double n[3], u[5], f[5];
      unit_normal(d, n);
      for (int b = 0; b < np; ++b)
        for (int a = 0; a < np; ++a) {
          int node = face_node_to_vol(o, d, side, a, b);
          for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * nn + node];
          orc_euler_flux(u, n, grid_vel(o, id.blk, d), o.p.gamma, f);
          for (int v = 0; v < 5; ++v) Ut_e[v * nn + node] -= (Fout[v * nq + a + np * b] - sg * sJ * f[v]) / wend;
        }
    }
  double invJ = 1.0 / jacobian(o, id.blk);
  for (int k = 0; k < 5 * nn; ++k) Ut_e[k] *= invJ;
}

/* Weak-form DGSEM residual of one element (Eq. weak_formulation with LGL collocation):
 *   J dU/dt = - [ sum_l Dhat_il F~1_ljk + sum_l Dhat_jl F~2_ilk + sum_l Dhat_kl F~3_ijl ]
 *             - sum_faces ell(+-1)/w * (F* . N) sJ ,
 * with Dhat_il = -(w_l / w_i) D_li and contravariant fluxes F~d = |Ja^d| (F - v^g U) . e. */
void element_residual(const Oracle& o, const Interface* I, const double* U, const double* grad, double t, long long e,
                      const std::vector<double>* Fs, const std::vector<double>* Fm, double* Ut_e) {
  if (o.p.volume != 0) {
    split_element_residual(o, I, U, grad, t, e, Fs, Fm, Ut_e);
    return;
  }
  ElemId id = elem_id(o, e);
  int np = o.np, nn = o.nn, nq = np * np;
  std::vector<double> Ft(3 * 5 * nn);
  for (int node = 0; node < nn; ++node) {
    double u[5], f[5], n[3];
    for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * nn + node];
    double Fv[15];
    if (grad) {
      double g15[15];
      for (int k = 0; k < 15; ++k) g15[k] = grad[(e * 15 + k) * nn + node];
      orc_viscous_flux(u, g15, o.p.mu, o.p.Pr, o.p.Rgas, o.p.gamma, Fv);
    }
    for (int d = 0; d < 3; ++d) {
      unit_normal(d, n);
      orc_euler_flux(u, n, grid_vel(o, id.blk, d), o.p.gamma, f);
      if (grad)   /* total flux F^c - F^v (Sec. 2, Eq. navier_stokes) */
        for (int v = 0; v < 5; ++v) f[v] -= Fv[phys_axis(d) * 5 + v];
      for (int v = 0; v < 5; ++v) Ft[(d * 5 + v) * nn + node] = metric(o, id.blk, d) * f[v];
    }
  }
  double invJ = 1.0 / jacobian(o, id.blk);
  for (int v = 0; v < 5; ++v)
    for (int k = 0; k < np; ++k)
      for (int j = 0; j < np; ++j)
        for (int i = 0; i < np; ++i) {
          double acc = 0.0;
          for (int l = 0; l < np; ++l) {
            acc += o.Dhat[i * np + l] * Ft[(0 * 5 + v) * nn + l + np * (j + np * k)];
            acc += o.Dhat[j * np + l] * Ft[(1 * 5 + v) * nn + i + np * (l + np * k)];
            acc += o.Dhat[k * np + l] * Ft[(2 * 5 + v) * nn + i + np * (j + np * l)];
          }
          Ut_e[v * nn + i + np * (j + np * k)] = -acc;
        }
  std::vector<double> Fout(5 * nq);
  for (int d = 0; d < 3; ++d)
    for (int side = 0; side < 2; ++side) {
      face_flux_out(o, I, U, grad, t, e, d, side, Fs, Fm, Fout.data());
      double wend = o.w[side == 0 ? 0 : o.N];
      for (int v = 0; v < 5; ++v)
        for (int b = 0; b < np; ++b)
          for (int a = 0; a < np; ++a)
            Ut_e[v * nn + face_node_to_vol(o, d, side, a, b)] -= Fout[v * nq + a + np * b] / wend;
    }
  for (int k = 0; k < 5 * nn; ++k) Ut_e[k] *= invJ;
}

/* All interface face fluxes, via the mortar arrays of Sec. 4.2: first every mortar flux
 * (indexed by (i_par, i_perp, i_sub)), then the projections onto both sides' faces. */
void all_interface_fluxes(const Oracle& o, const Interface& I, const double* U, const double* grad,
                          std::vector<double>& Fs, std::vector<double>& Fm) {
  int nq = o.np * o.np;
  long long nf = (long long)o.ny * o.nz;
  int nifc = o.p.periodic_x ? 2 : 1;           /* interface 0 first, then interface 1 */
  std::vector<double> Fsm(nifc * nf * 2 * 5 * nq);
  #pragma omp parallel for schedule(dynamic)
  for (long long g = 0; g < nifc * nf; ++g) {
    int ifc = (int)(g / nf);
    long long f = g - ifc * nf;
    int ipar = (int)(f % o.ny), iperp = (int)(f / o.ny);
    for (int isub = 0; isub < 2; ++isub)
      mortar_flux(o, I, U, grad, ipar, iperp, isub, Fsm.data() + (g * 2 + isub) * 5 * nq, ifc);
  }
  Fs.assign(nifc * nf * 5 * nq, 0.0);
  Fm.assign(nifc * nf * 5 * nq, 0.0);
  #pragma omp parallel for schedule(dynamic)
  for (long long g = 0; g < nifc * nf; ++g) {
    int ifc = (int)(g / nf);
    long long f = g - ifc * nf;
    int ipar = (int)(f % o.ny), iperp = (int)(f / o.ny);
    long long row = ifc * nf + (long long)iperp * o.ny;
    project_to_face(o, I.Bs_lo.data(), Fsm.data() + (g * 2 + 0) * 5 * nq, I.Bs_hi.data(),
                    Fsm.data() + (g * 2 + 1) * 5 * nq, 1.0, Fs.data() + g * 5 * nq);
    long long flo = row + wrap((long long)ipar + I.n, o.ny), fhi = row + wrap((long long)ipar + I.n + 1, o.ny);
    project_to_face(o, I.Bm_lo.data(), Fsm.data() + (flo * 2 + 1) * 5 * nq, I.Bm_hi.data(),
                    Fsm.data() + (fhi * 2 + 0) * 5 * nq, -1.0, Fm.data() + g * 5 * nq);
  }
}


/* BR1 lifting ("first method" of Bassi and Rebay, Sec. 3.1): the gradient of each primitive
 * variable (rho, v1, v2, v3, p) along each physical axis by the same weak DG operator as the
 * flux divergence, applied to the "flux" Q e_axis with face value the mean of both sides'
 * traces; on the sliding interface the mean is taken on the mortars between the projected
 * primitive traces and projected back (Sec. 3.2).  grad[((e*3 + a)*5 + c)*nn + node]. */
void compute_lifting(const Oracle& o, const Interface& I, const double* U, double t, double* grad) {
  int np = o.np, nn = o.nn, nq = np * np;
  long long nf = (long long)o.ny * o.nz;
  std::vector<double> Ls, Lm;
  if (!o.p.interface_conforming) {
    std::vector<double> Lsm(nf * 2 * 5 * nq);
    for (long long f = 0; f < nf; ++f)
      for (int isub = 0; isub < 2; ++isub)
        mortar_lift(o, I, U, (int)(f % o.ny), (int)(f / o.ny), isub, Lsm.data() + (f * 2 + isub) * 5 * nq);
    Ls.assign(nf * 5 * nq, 0.0);
    Lm.assign(nf * 5 * nq, 0.0);
    for (long long f = 0; f < nf; ++f) {
      int ipar = (int)(f % o.ny);
      long long row = (f / o.ny) * o.ny;
      project_to_face(o, I.Bs_lo.data(), Lsm.data() + (f * 2 + 0) * 5 * nq, I.Bs_hi.data(),
                      Lsm.data() + (f * 2 + 1) * 5 * nq, 1.0, Ls.data() + f * 5 * nq);
      long long flo = row + wrap((long long)ipar + I.n, o.ny), fhi = row + wrap((long long)ipar + I.n + 1, o.ny);
      project_to_face(o, I.Bm_lo.data(), Lsm.data() + (flo * 2 + 1) * 5 * nq, I.Bm_hi.data(),
                      Lsm.data() + (fhi * 2 + 0) * 5 * nq, -1.0, Lm.data() + f * 5 * nq);
    }
  }
  #pragma omp parallel for schedule(static)
  for (long long e = 0; e < o.E; ++e) {
    ElemId id = elem_id(o, e);
    std::vector<double> Q(5 * nn);
    for (int node = 0; node < nn; ++node) {
      double u[5], q[5];
      for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * nn + node];
      cons_to_prim(u, o.p.gamma, q);
      for (int v = 0; v < 5; ++v) Q[v * nn + node] = q[v];
    }
    double invJ = 1.0 / jacobian(o, id.blk);
    int nx = id.blk == 0 ? o.p.nel_s[0] : o.p.nel_m[0];
    for (int d = 0; d < 3; ++d) {
      int a = phys_axis(d);
      double sJ = metric(o, id.blk, d);
      double* g = grad + (e * 15 + a * 5) * nn;
      /* volume: sum_l Dhat_il |Ja^d| Q along direction d */
      for (int v = 0; v < 5; ++v)
        for (int k = 0; k < np; ++k)
          for (int j = 0; j < np; ++j)
            for (int i = 0; i < np; ++i) {
              double acc = 0.0;
              for (int l = 0; l < np; ++l) {
                int nl = d == 0 ? l + np * (j + np * k) : (d == 1 ? i + np * (l + np * k) : i + np * (j + np * l));
                int il = d == 0 ? i : (d == 1 ? j : k);
                acc += o.Dhat[il * np + l] * sJ * Q[v * nn + nl];
              }
              g[v * nn + i + np * (j + np * k)] = acc;
            }
      /* surface: the two faces of direction d */
      for (int side = 0; side < 2; ++side) {
        long long nb = -1; int kind = 0, nb_blk = id.blk;
        if (d == 0) nb = elem_index(o, id.blk, id.ix, wrap(id.iy + (side ? 1 : -1), o.ny), id.iz);
        else if (d == 1) nb = elem_index(o, id.blk, id.ix, id.iy, wrap(id.iz + (side ? 1 : -1), o.nz));
        else {
          int jx = id.ix + (side ? 1 : -1);
          if (jx >= 0 && jx < nx) nb = elem_index(o, id.blk, jx, id.iy, id.iz);
          else if ((id.blk == 0 && side == 0) || (id.blk == 1 && side == 1)) kind = 1;
          else if (o.p.interface_conforming) {
            nb_blk = 1 - id.blk;
            nb = elem_index(o, nb_blk, nb_blk == 0 ? o.p.nel_s[0] - 1 : 0, id.iy, id.iz);
          } else kind = 2;
        }
        double wend = o.w[side == 0 ? 0 : o.N];
        for (int b = 0; b < np; ++b)
          for (int aa = 0; aa < np; ++aa) {
            int vn = face_node_to_vol(o, d, side, aa, b);
            double Fo[5];
            if (kind == 2) {
              const std::vector<double>& L = id.blk == 0 ? Ls : Lm;
              long long f = (long long)id.iz * o.ny + id.iy;
              for (int v = 0; v < 5; ++v) Fo[v] = L[(f * 5 + v) * nq + aa + np * b];
            } else {
              double qo[5], uo[5];
              if (kind == 1) {
                int i = vn % np, j = (vn / np) % np, k = vn / nq;
                double X[3];
                node_xyz(o, id, i, j, k, t, X);
                flow_state(o.p, X, t, 1, uo);
              } else {
                int vnn = face_node_to_vol(o, d, 1 - side, aa, b);
                for (int v = 0; v < 5; ++v) uo[v] = U[(nb * 5 + v) * nn + vnn];
              }
              cons_to_prim(uo, o.p.gamma, qo);
              double sg = side == 1 ? 1.0 : -1.0;
              for (int v = 0; v < 5; ++v) Fo[v] = sg * sJ * 0.5 * (Q[v * nn + vn] + qo[v]);
            }
            for (int v = 0; v < 5; ++v) g[v * nn + vn] += Fo[v] / wend;
          }
      }
      for (int k = 0; k < 5 * nn; ++k) g[k] *= invJ;
    }
  }
}
}  // namespace

extern "C" {

static bool curved(void* h) { return *(int*)h == 1; }

void* orc_create(const orc_problem* p) {
  if (p->volume < 0 || p->volume > 2) return nullptr;
  if (p->geom != 0) return p->periodic_x ? nullptr : orc_curved_create(p);
  if (p->N < 1 || p->N > 15) return nullptr;
  if (p->nel_s[1] != p->nel_m[1] || p->nel_s[2] != p->nel_m[2]) return nullptr;
  if (p->periodic_x && p->physics != 0) return nullptr;
  Oracle* o = new Oracle();
  o->p = *p;
  o->N = p->N; o->np = p->N + 1; o->nn = o->np * o->np * o->np;
  o->ny = p->nel_s[1]; o->nz = p->nel_s[2];
  o->Es = (long long)p->nel_s[0] * o->ny * o->nz;
  o->Em = (long long)p->nel_m[0] * o->ny * o->nz;
  o->E = o->Es + o->Em;
  o->hy = (p->y1 - p->y0) / o->ny;
  o->hz = (p->z1 - p->z0) / o->nz;
  o->hx[0] = (p->x1 - p->x0) / p->nel_s[0];
  o->hx[1] = (p->x2 - p->x1) / p->nel_m[0];
  o->x.resize(o->np); o->w.resize(o->np);
  orc_lgl(o->N, o->x.data(), o->w.data());
  o->D.resize(o->np * o->np); o->Dhat.resize(o->np * o->np);
  orc_dmatrix(o->N, o->x.data(), o->D.data());
  for (int i = 0; i < o->np; ++i)
    for (int l = 0; l < o->np; ++l) o->Dhat[i * o->np + l] = -(o->w[l] / o->w[i]) * o->D[l * o->np + i];
  orc_lsrk_coeffs(o->A, o->B, o->c);
  o->ns = p->physics == 1;
  return o;
}

void orc_destroy(void* h) {
  if (curved(h)) orc_curved_destroy(h);
  else delete (Oracle*)h;
}
long long orc_nelem(void* h) { return curved(h) ? orc_curved_nelem(h) : ((Oracle*)h)->E; }

void orc_node_coords(void* h, double t, double* xyz) {
  if (curved(h)) { orc_curved_coords(h, t, xyz); return; }
  Oracle& o = *(Oracle*)h;
  for (long long e = 0; e < o.E; ++e) {
    ElemId id = elem_id(o, e);
    for (int k = 0; k < o.np; ++k)
      for (int j = 0; j < o.np; ++j)
        for (int i = 0; i < o.np; ++i) {
          double X[3];
          node_xyz(o, id, i, j, k, t, X);
          int nd = i + o.np * (j + o.np * k);
          for (int a = 0; a < 3; ++a) xyz[(e * 3 + a) * o.nn + nd] = X[a];
        }
  }
}

static void fill_flow(Oracle& o, double t, double* U) {
  #pragma omp parallel for
  for (long long e = 0; e < o.E; ++e) {
    ElemId id = elem_id(o, e);
    for (int k = 0; k < o.np; ++k)
      for (int j = 0; j < o.np; ++j)
        for (int i = 0; i < o.np; ++i) {
          double X[3], u[5];
          node_xyz(o, id, i, j, k, t, X);
          flow_state(o.p, X, t, 0, u);
          int nd = i + o.np * (j + o.np * k);
          for (int v = 0; v < 5; ++v) U[(e * 5 + v) * o.nn + nd] = u[v];
        }
  }
}

void orc_init_state(void* h, double* U) {
  if (curved(h)) orc_curved_fill(h, 0.0, U);
  else fill_flow(*(Oracle*)h, 0.0, U);
}
void orc_exact_state(void* h, double t, double* U) {
  if (curved(h)) orc_curved_fill(h, t, U);
  else fill_flow(*(Oracle*)h, t, U);
}

void orc_flow_state(const orc_problem* p, const double* X, double t, int boundary, double* U) {
  flow_state(*p, X, t, boundary, U);
}

void orc_metrics(void* h, double t, double* Ja, double* J) {
  if (curved(h)) { orc_curved_metrics(h, t, Ja, J); return; }
  Oracle& o = *(Oracle*)h;
  for (long long e = 0; e < o.E; ++e) {
    int blk = elem_id(o, e).blk;
    for (int nd = 0; nd < o.nn; ++nd) {
      for (int i = 0; i < 3; ++i)
        for (int n = 0; n < 3; ++n)
          Ja[((e * 3 + i) * 3 + n) * o.nn + nd] = n == phys_axis(i) ? metric(o, blk, i) : 0.0;
      J[e * o.nn + nd] = jacobian(o, blk);
    }
  }
}

void orc_rhs(void* h, const double* U, double t, double* Ut) {
  if (curved(h)) { orc_curved_rhs(h, U, t, nullptr, 0, Ut); return; }
  Oracle& o = *(Oracle*)h;
  Interface I;
  interface_config(o, t, I);
  std::vector<double> grad;
  if (o.ns) { grad.assign(o.E * 15 * o.nn, 0.0); compute_lifting(o, I, U, t, grad.data()); }
  const double* g = o.ns ? grad.data() : nullptr;
  std::vector<double> Fs, Fm;
  const std::vector<double>* ps = nullptr, *pm = nullptr;
  if (!o.p.interface_conforming) { all_interface_fluxes(o, I, U, g, Fs, Fm); ps = &Fs; pm = &Fm; }
  #pragma omp parallel for schedule(static)
  for (long long e = 0; e < o.E; ++e) element_residual(o, &I, U, g, t, e, ps, pm, Ut + e * 5 * o.nn);
}

void orc_rhs_elements(void* h, const double* U, double t, const long long* elems, int count, double* Ut) {
  if (curved(h)) { orc_curved_rhs(h, U, t, elems, count, Ut); return; }
  Oracle& o = *(Oracle*)h;
  Interface I;
  interface_config(o, t, I);
  std::vector<double> grad;
  if (o.ns) { grad.assign(o.E * 15 * o.nn, 0.0); compute_lifting(o, I, U, t, grad.data()); }
  const double* g = o.ns ? grad.data() : nullptr;
  #pragma omp parallel for schedule(dynamic)
  for (int m = 0; m < count; ++m) element_residual(o, &I, U, g, t, elems[m], nullptr, nullptr, Ut + (long long)m * 5 * o.nn);
}

void orc_lifting(void* h, const double* U, double t, double* grad) {
  if (curved(h)) { orc_curved_lifting(h, U, t, grad); return; }
  Oracle& o = *(Oracle*)h;
  Interface I;
  interface_config(o, t, I);
  compute_lifting(o, I, U, t, grad);
}

void orc_interface_fluxes(void* h, const double* U, double t, double* F_static, double* F_moving) {
  if (curved(h)) { orc_curved_interface(h, U, t, F_static, F_moving); return; }
  Oracle& o = *(Oracle*)h;
  Interface I;
  interface_config(o, t, I);
  std::vector<double> grad;
  if (o.ns) { grad.assign(o.E * 15 * o.nn, 0.0); compute_lifting(o, I, U, t, grad.data()); }
  std::vector<double> Fs, Fm;
  all_interface_fluxes(o, I, U, o.ns ? grad.data() : nullptr, Fs, Fm);
  /* interface 0 (x = x1) first; with periodic x, interface 1 (x = x0 = x2) follows */
  std::memcpy(F_static, Fs.data(), sizeof(double) * Fs.size());
  std::memcpy(F_moving, Fm.data(), sizeof(double) * Fm.size());
}

/* Low-storage RK: per step, stages k = 0..4 at t_k = fma(c_k, dt, t); t advances by dt. */
void orc_step(void* h, double* U, double* G, double* t, double dt, int nsteps) {
  if (curved(h)) { orc_curved_step(h, U, G, t, dt, nsteps); return; }
  Oracle& o = *(Oracle*)h;
  long long ndof = o.E * 5 * o.nn;
  std::vector<double> Ut(ndof);
  for (int s = 0; s < nsteps; ++s) {
    for (int k = 0; k < 5; ++k) {
      double tk = std::fma(o.c[k], dt, *t);
      orc_rhs(h, U, tk, Ut.data());
      #pragma omp parallel for
      for (long long m = 0; m < ndof; ++m) {
        G[m] = (k == 0) ? dt * Ut[m] : o.A[k] * G[m] + dt * Ut[m];
        U[m] = U[m] + o.B[k] * G[m];
      }
    }
    *t = *t + dt;
  }
}

void orc_totals(void* h, const double* U, double* tot5) {
  if (curved(h)) { orc_curved_totals(h, U, tot5); return; }
  Oracle& o = *(Oracle*)h;
  for (int v = 0; v < 5; ++v) tot5[v] = 0.0;
  for (long long e = 0; e < o.E; ++e) {
    double J = jacobian(o, elem_id(o, e).blk);
    for (int v = 0; v < 5; ++v)
      for (int k = 0; k < o.np; ++k)
        for (int j = 0; j < o.np; ++j)
          for (int i = 0; i < o.np; ++i)
            tot5[v] += J * o.w[i] * o.w[j] * o.w[k] * U[(e * 5 + v) * o.nn + i + o.np * (j + o.np * k)];
  }
}

void orc_face_flux_sums(const orc_problem* p, const double* F_static, const double* F_moving,
                        double* ss, double* sm) {
  int np = p->N + 1, nq = np * np;
  std::vector<double> x(np), w(np);
  orc_lgl(p->N, x.data(), w.data());
  long long nf = (long long)p->nel_s[1] * p->nel_s[2];
  for (int v = 0; v < 5; ++v) { ss[v] = 0.0; sm[v] = 0.0; }
  for (long long f = 0; f < nf; ++f)
    for (int v = 0; v < 5; ++v)
      for (int q = 0; q < np; ++q)
        for (int i = 0; i < np; ++i) {
          ss[v] += w[i] * w[q] * F_static[(f * 5 + v) * nq + q * np + i];
          sm[v] += w[i] * w[q] * F_moving[(f * 5 + v) * nq + q * np + i];
        }
}

double orc_l2_error_rho(void* h, const double* U, double t) {
  if (curved(h)) return orc_curved_l2_error_rho(h, U, t);
  Oracle& o = *(Oracle*)h;
  double err = 0.0, vol = 0.0;
  for (long long e = 0; e < o.E; ++e) {
    ElemId id = elem_id(o, e);
    double J = jacobian(o, id.blk);
    for (int k = 0; k < o.np; ++k)
      for (int j = 0; j < o.np; ++j)
        for (int i = 0; i < o.np; ++i) {
          double X[3], u[5];
          node_xyz(o, id, i, j, k, t, X);
          flow_state(o.p, X, t, 0, u);
          double d = U[(e * 5 + 0) * o.nn + i + o.np * (j + o.np * k)] - u[0];
          double wq = J * o.w[i] * o.w[j] * o.w[k];
          err += wq * d * d;
          vol += wq;
        }
  }
  return std::sqrt(err / vol);
}

}  /* extern "C" */

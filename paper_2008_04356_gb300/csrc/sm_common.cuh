// Device-side building blocks of the sliding-mesh DGSEM hot path (sm_103a).
//
// Geometry of the two-block plane interface, the ALE Euler fluxes of Sec. 2
// (Eq. fluxes_written_out), the Rusanov and Roe/Harten-Hyman Riemann solvers named in
// Sec. 3.1, and the flows used for initial and weak Dirichlet data.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define SM_MAXNP 8
#define SM_PI 3.14159265358979323846

// Basis of degree N on Legendre-Gauss-Lobatto nodes, built in FP64 on the host once per
// solver.  Dhat_il = -(w_l / w_i) D_li is the weak-form derivative of Sec. 3.1
// (Eq. weak_formulation with collocated LGL quadrature).
struct BasisDev {
  double x[SM_MAXNP], w[SM_MAXNP], lam[SM_MAXNP];   // nodes, weights, barycentric weights
  double M[SM_MAXNP * SM_MAXNP], Minv[SM_MAXNP * SM_MAXNP];  // exact mass matrix, inverse
  double Dhat[SM_MAXNP * SM_MAXNP];
  float Dhat_f[SM_MAXNP * SM_MAXNP];
  float x_f[SM_MAXNP], w_f[SM_MAXNP];
  double Dsplit[SM_MAXNP * SM_MAXNP];   // split form: 2 D - M^-1 B (zero diagonal)
};

// Per-stage interface configuration (Sec. 4.3) and mortar operators (Sec. 3.2), written by
// the mapper kernel before the interface kernel runs.  Matrix order: 0 Ps_lo, 1 Ps_hi,
// 2 Pm_lo, 3 Pm_hi (forward, [mortar node][face node]), 4 Bs_lo, 5 Bs_hi, 6 Bm_lo, 7 Bm_hi
// (back, [face node][mortar node]); s = static face (hanging node sigma_s = 2s - 1),
// m = moving face (sigma_m = 1 - 2s).
struct StageParams {
  double t;            // stage time
  double delta;        // displacement of the moving block
  long long n;         // integer face offset
  int n_mod;           // n mod n_par in [0, n_par): the partner shift of the interface kernels
  int pad_;
  double s;            // sub-face fraction
  double sig_s, sig_m;
  double mat[8][SM_MAXNP * SM_MAXNP];
  float mat_f[8][SM_MAXNP * SM_MAXNP];
  // the FP32 operators as the FP32 interface kernel reads them (np even): the entries of
  // rows 2 h and 2 h + 1 of matrix k at column c, each duplicated into a float pair (its
  // operand for two node rows at once), as one float4:
  // pair_f[4 ((k np/2 + h) np + c) + {0, 1, 2, 3}] = mat_f[k] at (2h, c), (2h, c), (2h+1, c), (2h+1, c)
  alignas(16) float pair_f[16 * SM_MAXNP * SM_MAXNP];
  // cylindrical interface: cos, sin of the rotor angle phi = -delta, and of the angles
  // w Theta - phi that carry a stator face seen through w periodic wraps into the rotor's
  // frame, for w = w0 and w0 + 1 (w0 = floor((-n-1) / n_par), the smallest wrap count)
  double rot[2];
  double arot[2][2];
  long long w0;
  float rot_f[2];
  float arot_f[2][2];
};

// Offset of node (i, q) (i along the sliding direction, q across it) in one variable's block
// of a compact interface trace: rows q in order (i fastest), except for FP32 states with an
// even number of nodes per row, whose rows are interleaved in pairs (2 qp, 2 qp + 1) so that
// the FP32 interface kernel loads the same node of two rows as one float pair:
// (q / 2) 2 np + 2 i + q mod 2.
template <typename T, int NP>
__host__ __device__ constexpr int trace_node(int i, int q) {
  return (sizeof(T) == 4 && NP % 2 == 0) ? (q >> 1) * 2 * NP + 2 * i + (q & 1) : i + NP * q;
}

// Per-precision constants of the discrete operator, precomputed on the host so that the
// kernels do no FP64 arithmetic in FP32 mode.
enum {
  MC_METRIC = 0,      // [blk*3 + d]: |Ja^d|, surface element of the xi^{d+1} faces
  MC_MINVJ = 6,       // [blk]: -1 / J
  MC_VG = 8,          // grid velocity of the moving block (along y)
  MC_GAMMA = 9,
  MC_IW0 = 10,        // 1 / w_0 (LGL end-point weight)
  MC_SJ_IF = 11,      // surface element of the interface faces
  MC_BC = 12,         // [5]: constant boundary state (flows 0 and 2)
  MC_H = 17,          // [4]: hx (static), hx (moving), hy, hz
  MC_X = 21,          // [4]: x0, x1, y0, z0
  MC_MU = 25,         // dynamic viscosity
  MC_K = 26,          // heat conductivity mu gamma R / ((gamma - 1) Pr)
  MC_R = 27,          // gas constant
  MC_PCOS = 28,       // cos, sin of the periodic sector angle Theta (cylinder)
  MC_PSIN = 29,
  MC_COUNT = 30
};

// Mesh and physics description passed to kernels by value.
struct MeshDev {
  int nxs, nxm, ny, nz;
  long long Es, E;
  double hx0, hx1, hy, hz;
  double x0, x1, y0, z0;
  double gamma;
  double v, delta0;
  int conforming;
  int flow;
  int physics;                // 0 Euler, 1 Navier-Stokes
  double mu, Pr, Rgas;
  double fpar[16];
  const double* modes;        // [5][8][4] device
  const BasisDev* basis;      // device
  float cf[MC_COUNT];
  double cd[MC_COUNT];
  float fparf[16];
  // Optional precomputed topology, two int4 per element: (nb0, nb1, nb2, nb3) and
  // (nb4, nb5, (ix << 1) | blk, iz * ny + iy), neighbour codes as in the element kernel
  // (>= 0 element, -1 weak Dirichlet face, -2 sliding interface x = x1, -3 sliding
  // interface x = x0 = x2).  NULL: computed on the fly.
  const int4* topo;
  // Curvilinear geometries: 0 plane interface (Cartesian kernels), 1 cylindrical interface
  // (rotor = block 0 inside, slip walls at the radial ends, periodic angular sector of
  // angle Theta), 2 the plane box through the curvilinear kernels.
  int geom;
  double Theta;
  double cone_s, cone_c;      // geom 4: sin, cos of the cone's half-angle
  // per-node geometry [E][13][NN] in solver precision: Ja^i_n at t = 0 (slot 3 i + n),
  // J (slot 9), and the grid-velocity factors Ja^i . v^g / |v| of the moving block
  // (slots 10..12; the grid speed is MC_VG)
  const void* geo;
  // Periodic x (plane geometry): the moving block's face x = x2 meets the static block's
  // face x = x0 in a second sliding interface.  Its traces Ts2 / Tm2 and face fluxes Fs2 /
  // Fm2 use the layout of the first interface's arrays and hold the x-mirrored problem
  // (x-momentum negated), so that the first interface's kernel, whose static outward normal
  // is +x, solves it unchanged; the element kernels mirror the fluxes back when they read
  // them.  NULL pointers: one interface.
  int periodic_x;
  void* Ts2;
  void* Tm2;
  const void* Fs2;
  const void* Fm2;
};

template <typename T> struct Prec;
template <> struct Prec<double> {
  static __device__ __forceinline__ double sqrt_(double a) { return sqrt(a); }
  static __device__ __forceinline__ double rcp(double a) { return 1.0 / a; }
  static __device__ __forceinline__ const double* c(const MeshDev& m);
  static __device__ __forceinline__ double fpar(const MeshDev& m, int k);
  static __device__ __forceinline__ const double* dhat(const BasisDev* b) { return b->Dhat; }
  static __device__ __forceinline__ const double* w(const BasisDev* b) { return b->w; }
  static __device__ __forceinline__ const double* x(const BasisDev* b) { return b->x; }
  static __device__ __forceinline__ const double* mat(const StageParams* p, int k) { return p->mat[k]; }
  static __device__ __forceinline__ const double* rot(const StageParams* p) { return p->rot; }
  static __device__ __forceinline__ const double* arot(const StageParams* p, int k) { return p->arot[k]; }
};
// FP32 mode uses the hardware reciprocal and reciprocal square root (about 1-2 ulp), well
// inside the 1e-5 relative tolerance of the FP32 path; FP64 mode keeps IEEE division/sqrt.
template <> struct Prec<float> {
  static __device__ __forceinline__ float sqrt_(float a) { return a * rsqrtf(a); }
  static __device__ __forceinline__ float rcp(float a) { return __fdividef(1.0f, a); }
  static __device__ __forceinline__ const float* c(const MeshDev& m);
  static __device__ __forceinline__ float fpar(const MeshDev& m, int k);
  static __device__ __forceinline__ const float* dhat(const BasisDev* b) { return b->Dhat_f; }
  static __device__ __forceinline__ const float* w(const BasisDev* b) { return b->w_f; }
  static __device__ __forceinline__ const float* x(const BasisDev* b) { return b->x_f; }
  static __device__ __forceinline__ const float* mat(const StageParams* p, int k) { return p->mat_f[k]; }
  static __device__ __forceinline__ const float* rot(const StageParams* p) { return p->rot_f; }
  static __device__ __forceinline__ const float* arot(const StageParams* p, int k) { return p->arot_f[k]; }
};

__device__ __forceinline__ const double* Prec<double>::c(const MeshDev& m) { return m.cd; }
__device__ __forceinline__ const float* Prec<float>::c(const MeshDev& m) { return m.cf; }
__device__ __forceinline__ double Prec<double>::fpar(const MeshDev& m, int k) { return m.fpar[k]; }
__device__ __forceinline__ float Prec<float>::fpar(const MeshDev& m, int k) { return m.fparf[k]; }

// ---------------------------------------------------------------------------------------
// Element / face geometry.  Element e: static block first (e < Es), local index
// ix + nx (iy + ny iz).  Reference axes: xi^1 -> y, xi^2 -> z, xi^3 -> x.
// Faces of an element are f = 2 d + side, d the reference direction, side 0 = minus.
// Face nodes a + np b:  d=0: (a,b)=(j,k);  d=1: (a,b)=(i,k);  d=2: (a,b)=(i,j).
// ---------------------------------------------------------------------------------------
struct ElemPos { int blk, ix, iy, iz; };

// Geometries with a rotor turning about the z axis: 1 the cylindrical interface, 3 the plane
// annular interface normal to the axis (reference axes xi^1 -> theta, xi^2 -> r from the outer
// radius z1 down to z0, xi^3 -> z), 4 the conical interface (xi^1 -> theta, xi^2 -> s along
// the generator, xi^3 -> n across: radius s sin(alpha) + n cos(alpha), height
// s cos(alpha) - n sin(alpha)).
__host__ __device__ __forceinline__ bool rotating_geom(int geom) { return geom == 1 || geom == 3 || geom == 4; }

// Element counts stay below 2^31 (checked when a solver is created): 32-bit arithmetic.
__host__ __device__ __forceinline__ ElemPos decode_elem(const MeshDev& m, long long e64) {
  ElemPos p;
  int loc = (int)e64;
  int nx = m.nxs;
  p.blk = 0;
  if (e64 >= m.Es) { p.blk = 1; loc = (int)(e64 - m.Es); nx = m.nxm; }
  const int r = loc / nx;
  p.ix = loc - r * nx;
  p.iy = r % m.ny;
  p.iz = r / m.ny;
  return p;
}

__host__ __device__ __forceinline__ long long encode_elem(const MeshDev& m, int blk, int ix, int iy, int iz) {
  int nx = blk ? m.nxm : m.nxs;
  return (blk ? m.Es : 0) + ix + (long long)nx * (iy + (long long)m.ny * iz);
}

template <int NP>
__device__ __forceinline__ int face_vol_node(int d, int side, int a, int b) {
  const int f = side ? NP - 1 : 0;
  return d == 0 ? f + NP * (a + NP * b) : (d == 1 ? a + NP * (f + NP * b) : a + NP * (b + NP * f));
}

// Neighbour across face (d, side): kind 0 conforming (returns element), 1 weak Dirichlet
// boundary (x = x0 of the static block, x = x2 of the moving block), 2 sliding interface
// x = x1, 3 the second sliding interface x = x0 = x2 (periodic x).
__host__ __device__ __forceinline__ int face_neighbor(const MeshDev& m, const ElemPos& p, int d, int side, long long* nb) {
  if (d == 0) {
    int iy = p.iy + (side ? 1 : -1);
    iy = iy < 0 ? iy + m.ny : (iy >= m.ny ? iy - m.ny : iy);
    *nb = encode_elem(m, p.blk, p.ix, iy, p.iz);
    return 0;
  }
  if (d == 1) {
    int iz = p.iz + (side ? 1 : -1);
    if ((m.geom == 3 || m.geom == 4) && (iz < 0 || iz >= m.nz)) return 1;   // slip walls at the xi^2 ends
    iz = iz < 0 ? iz + m.nz : (iz >= m.nz ? iz - m.nz : iz);
    *nb = encode_elem(m, p.blk, p.ix, p.iy, iz);
    return 0;
  }
  int nx = p.blk ? m.nxm : m.nxs;
  int jx = p.ix + (side ? 1 : -1);
  if (jx >= 0 && jx < nx) { *nb = encode_elem(m, p.blk, jx, p.iy, p.iz); return 0; }
  const bool outer = (p.blk == 0 && side == 0) || (p.blk == 1 && side == 1);
  if (outer && !m.periodic_x) return 1;
  if (m.conforming) {
    // across x = x1 static element nx-1 meets moving element 0; across x = x0 = x2 (periodic
    // x) static element 0 meets moving element nx-1
    int ob = 1 - p.blk;
    *nb = encode_elem(m, ob, ob == 0 ? (outer ? 0 : m.nxs - 1) : (outer ? m.nxm - 1 : 0), p.iy, p.iz);
    return 0;
  }
  return outer ? 3 : 2;
}

// |Ja^d| (surface element of the xi^{d+1} faces) and the Jacobian of a Cartesian element.
__device__ __forceinline__ double face_metric(const MeshDev& m, int blk, int d) {
  double hx = blk ? m.hx1 : m.hx0;
  return d == 0 ? m.hz * hx * 0.25 : (d == 1 ? hx * m.hy * 0.25 : m.hy * m.hz * 0.25);
}
__device__ __forceinline__ double elem_jacobian(const MeshDev& m, int blk) {
  return (blk ? m.hx1 : m.hx0) * m.hy * m.hz * 0.125;
}

// ---------------------------------------------------------------------------------------
// Physics (Sec. 2).  U = (rho, rho v, rho e); perfect gas p = (gamma-1)(rho e - m.v/2).
// ---------------------------------------------------------------------------------------
template <typename T> struct Prim { T ir, u[3], p; };   // 1/rho, velocity, pressure

template <typename T>
__device__ __forceinline__ Prim<T> primitives(const T U[5], T gamma) {
  Prim<T> q;
  q.ir = Prec<T>::rcp(U[0]);
  q.u[0] = U[1] * q.ir;
  q.u[1] = U[2] * q.ir;
  q.u[2] = U[3] * q.ir;
  q.p = (gamma - T(1)) * (U[4] - T(0.5) * (U[1] * q.u[0] + U[2] * q.u[1] + U[3] * q.u[2]));
  return q;
}

template <typename T>
__device__ __forceinline__ T pressure(const T U[5], T gamma) { return primitives(U, gamma).p; }

// Flux along physical axis AX (0 = x, 1 = y, 2 = z) minus grid transport vg * U.
template <typename T, int AX>
__device__ __forceinline__ void axis_flux(const T U[5], const Prim<T>& q, T vg, T F[5]) {
  const T ua = q.u[AX];
  const T un = ua - vg;
  F[0] = U[0] * un;
  F[1] = U[1] * un + (AX == 0 ? q.p : T(0));
  F[2] = U[2] * un + (AX == 1 ? q.p : T(0));
  F[3] = U[3] * un + (AX == 2 ? q.p : T(0));
  F[4] = U[4] * un + q.p * ua;
}

// Riemann flux across a face with unit normal along +AX, grid normal velocity vgn.
// RIEM 0: Rusanov (local Lax-Friedrichs); RIEM 1: Roe with the Harten-Hyman entropy fix.
template <typename T, int AX, int RIEM>
__device__ __forceinline__ void riemann_axis(const T UL[5], const T UR[5], T vgn, T gamma, T F[5]) {
  const Prim<T> qL = primitives(UL, gamma), qR = primitives(UR, gamma);
  T FL[5], FR[5];
  axis_flux<T, AX>(UL, qL, vgn, FL);
  axis_flux<T, AX>(UR, qR, vgn, FR);
  const T unL = qL.u[AX], unR = qR.u[AX];
  const T cL = Prec<T>::sqrt_(gamma * qL.p * qL.ir), cR = Prec<T>::sqrt_(gamma * qR.p * qR.ir);
  if (RIEM == 0) {
    const T a = fmax(fabs(unL - vgn) + cL, fabs(unR - vgn) + cR);
#pragma unroll
    for (int k = 0; k < 5; ++k) F[k] = T(0.5) * (FL[k] + FR[k]) - T(0.5) * a * (UR[k] - UL[k]);
    return;
  }
  // Roe-averaged state
  const T sL = Prec<T>::sqrt_(UL[0]), sR = Prec<T>::sqrt_(UR[0]);
  const T iss = Prec<T>::rcp(sL + sR);
  T uh[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) uh[d] = (sL * qL.u[d] + sR * qR.u[d]) * iss;
  const T HL = (UL[4] + qL.p) * qL.ir, HR = (UR[4] + qR.p) * qR.ir;
  const T Hh = (sL * HL + sR * HR) * iss;
  const T q2 = uh[0] * uh[0] + uh[1] * uh[1] + uh[2] * uh[2];
  const T ch = Prec<T>::sqrt_((gamma - T(1)) * (Hh - T(0.5) * q2));
  const T rh = sL * sR;
  const T unh = uh[AX];
  const T dp = qR.p - qL.p, dr = UR[0] - UL[0], dun = unR - unL;
  const T ic2 = Prec<T>::rcp(ch * ch);
  const T a1 = T(0.5) * (dp - rh * ch * dun) * ic2;   // left acoustic wave
  const T a5 = T(0.5) * (dp + rh * ch * dun) * ic2;   // right acoustic wave
  const T a2 = dr - dp * ic2;                          // entropy wave
  const T l1 = unh - ch - vgn, l2 = unh - vgn, l5 = unh + ch - vgn;
  T al1 = fabs(l1), al5 = fabs(l5);
  const T al2 = fabs(l2);
  // Harten-Hyman: widen |lambda| of an acoustic wave that opens across zero
  const T d1 = fmax(T(0), fmax(l1 - (unL - cL - vgn), (unR - cR - vgn) - l1));
  if (al1 < d1) al1 = (l1 * l1 + d1 * d1) / (T(2) * d1);
  const T d5 = fmax(T(0), fmax(l5 - (unL + cL - vgn), (unR + cR - vgn) - l5));
  if (al5 < d5) al5 = (l5 * l5 + d5 * d5) / (T(2) * d5);
  const T w1 = al1 * a1, w5 = al5 * a5, w2 = al2 * a2;
  T du[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) du[d] = qR.u[d] - qL.u[d];
  T D[5];
  D[0] = w1 + w2 + w5;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T shear = du[d] - (d == AX ? dun : T(0));
    const T nd = d == AX ? ch : T(0);
    D[1 + d] = w1 * (uh[d] - nd) + w2 * uh[d] + al2 * rh * shear + w5 * (uh[d] + nd);
  }
  const T udu = uh[0] * du[0] + uh[1] * du[1] + uh[2] * du[2];
  D[4] = w1 * (Hh - unh * ch) + w2 * T(0.5) * q2 + al2 * rh * (udu - unh * dun) + w5 * (Hh + unh * ch);
#pragma unroll
  for (int k = 0; k < 5; ++k) F[k] = T(0.5) * (FL[k] + FR[k]) - T(0.5) * D[k];
}

// Rusanov flux along the outward normal n = sgn e_ax (sgn = +-1) of the element holding
// uin, ALE form with the normal grid speed vgn = v^g . n:
//   F* = (F(uin).n + F(uout).n) / 2 - a (uout - uin) / 2,
//   a = max(|v_in.n - vgn| + c_in, |v_out.n - vgn| + c_out).
// Every term changes sign exactly when the two states trade places and n and vgn change
// sign, and the same operations run for both neighbours of a face, so both obtain the same
// flux bit for bit (conservation) without a canonical orientation.
template <typename T>
__device__ __forceinline__ void rusanov_outward(const T uin[5], const T uout[5], const int ax, const T sgn,
                                                const T vgn, const T gamma, T F[5]) {
  const Prim<T> qi = primitives(uin, gamma), qo = primitives(uout, gamma);
  const T uni = sgn * (ax == 0 ? qi.u[0] : (ax == 1 ? qi.u[1] : qi.u[2]));
  const T uno = sgn * (ax == 0 ? qo.u[0] : (ax == 1 ? qo.u[1] : qo.u[2]));
  const T wi = uni - vgn, wo = uno - vgn;
  const T pni = sgn * qi.p, pno = sgn * qo.p;
  T Fi[5], Fo[5];
  Fi[0] = uin[0] * wi;
  Fo[0] = uout[0] * wo;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    Fi[1 + k] = uin[1 + k] * wi + (k == ax ? pni : T(0));
    Fo[1 + k] = uout[1 + k] * wo + (k == ax ? pno : T(0));
  }
  Fi[4] = uin[4] * wi + qi.p * uni;
  Fo[4] = uout[4] * wo + qo.p * uno;
  const T ci = Prec<T>::sqrt_(gamma * qi.p * qi.ir), co = Prec<T>::sqrt_(gamma * qo.p * qo.ir);
  const T a = fmax(fabs(wi) + ci, fabs(wo) + co);
#pragma unroll
  for (int k = 0; k < 5; ++k) F[k] = T(0.5) * (Fi[k] + Fo[k]) - T(0.5) * a * (uout[k] - uin[k]);
}

// ---- packed FP32 arithmetic (fma/add/mul.rn.f32x2: two IEEE operations per instruction) ----
__device__ __forceinline__ float2 p2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b as fma(b, -1, a): exact product, one rounding, the same as the subtraction
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, p2(-1.0f), a); }

struct Prim2 { float2 ir, u[3], p; };

// Primitives of two states at once (the FP32 reciprocal of Prec<float>::rcp per component).
__device__ __forceinline__ Prim2 primitives2(const float2 (&U)[5], const float gm1) {
  Prim2 q;
  q.ir = make_float2(Prec<float>::rcp(U[0].x), Prec<float>::rcp(U[0].y));
  q.u[0] = mul2(U[1], q.ir);
  q.u[1] = mul2(U[2], q.ir);
  q.u[2] = mul2(U[3], q.ir);
  float2 ke = mul2(U[1], q.u[0]);
  ke = fma2(U[2], q.u[1], ke);
  ke = fma2(U[3], q.u[2], ke);
  q.p = mul2(p2(gm1), fma2(p2(-0.5f), ke, U[4]));
  return q;
}

// Rusanov flux of two independent face nodes at once along the outward normal n = sgn e_ax
// of the element that holds uin, ALE form with the normal grid speed vgn (each component the
// same IEEE operations as a one-node evaluation of these formulas):
//   F* = (F(uin).n + F(uout).n) / 2 - a (uout - uin) / 2,
//   a = max(|v_in.n - vgn| + c_in, |v_out.n - vgn| + c_out).
__device__ __forceinline__ void rusanov_outward2(const float2 (&uin)[5], const float2 (&uout)[5], const int ax,
                                                 const float sgn, const float vgn, const float gamma,
                                                 float2 (&F)[5]) {
  const Prim2 qi = primitives2(uin, gamma - 1.0f), qo = primitives2(uout, gamma - 1.0f);
  const float2 sg = p2(sgn);
  const float2 uni = mul2(sg, ax == 0 ? qi.u[0] : (ax == 1 ? qi.u[1] : qi.u[2]));
  const float2 uno = mul2(sg, ax == 0 ? qo.u[0] : (ax == 1 ? qo.u[1] : qo.u[2]));
  const float2 wi = sub2(uni, p2(vgn)), wo = sub2(uno, p2(vgn));
  const float2 pni = mul2(sg, qi.p), pno = mul2(sg, qo.p);
  float2 t[5];
  t[0] = add2(mul2(uin[0], wi), mul2(uout[0], wo));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float2 fi = k == ax ? fma2(uin[1 + k], wi, pni) : mul2(uin[1 + k], wi);
    const float2 fo = k == ax ? fma2(uout[1 + k], wo, pno) : mul2(uout[1 + k], wo);
    t[1 + k] = add2(fi, fo);
  }
  t[4] = add2(fma2(qi.p, uni, mul2(uin[4], wi)), fma2(qo.p, uno, mul2(uout[4], wo)));
  const float2 ai = mul2(mul2(p2(gamma), qi.p), qi.ir), ao = mul2(mul2(p2(gamma), qo.p), qo.ir);
  const float cix = Prec<float>::sqrt_(ai.x), ciy = Prec<float>::sqrt_(ai.y);
  const float cox = Prec<float>::sqrt_(ao.x), coy = Prec<float>::sqrt_(ao.y);
  const float2 mha = make_float2(-0.5f * fmaxf(fabsf(wi.x) + cix, fabsf(wo.x) + cox),
                                 -0.5f * fmaxf(fabsf(wi.y) + ciy, fabsf(wo.y) + coy));
#pragma unroll
  for (int k = 0; k < 5; ++k) F[k] = fma2(mha, sub2(uout[k], uin[k]), mul2(p2(0.5f), t[k]));
}

// Cyclic rotation of the momentum components that brings physical axis ax (0 = x, 1 = y,
// 2 = z) to the first slot: (m_ax, m_ax+1, m_ax+2) (indices mod 3).  A cyclic permutation
// is a proper rotation, under which the Riemann fluxes are invariant, so every face is
// solved as an x-normal face by one code path.
template <typename T>
__device__ __forceinline__ void rotate_to_x(const T U[5], int ax, T R[5]) {
  R[0] = U[0];
  R[4] = U[4];
  R[1] = ax == 0 ? U[1] : (ax == 1 ? U[2] : U[3]);
  R[2] = ax == 0 ? U[2] : (ax == 1 ? U[3] : U[1]);
  R[3] = ax == 0 ? U[3] : (ax == 1 ? U[1] : U[2]);
}
template <typename T>
__device__ __forceinline__ void rotate_from_x(const T R[5], int ax, T U[5]) {
  U[0] = R[0];
  U[4] = R[4];
  U[1] = ax == 0 ? R[1] : (ax == 1 ? R[3] : R[2]);
  U[2] = ax == 0 ? R[2] : (ax == 1 ? R[1] : R[3]);
  U[3] = ax == 0 ? R[3] : (ax == 1 ? R[2] : R[1]);
}

// Flux along a unit normal n minus grid transport vgn * U (curvilinear faces).
template <typename T>
__device__ __forceinline__ void normal_flux(const T U[5], const Prim<T>& q, const T n[3], T vgn, T F[5]) {
  const T un = q.u[0] * n[0] + q.u[1] * n[1] + q.u[2] * n[2];
  const T w = un - vgn;
  F[0] = U[0] * w;
  F[1] = U[1] * w + q.p * n[0];
  F[2] = U[2] * w + q.p * n[1];
  F[3] = U[3] * w + q.p * n[2];
  F[4] = U[4] * w + q.p * un;
}

// Riemann flux across a face with unit normal n (from L to R), grid normal velocity vgn:
// the same Rusanov and Roe / Harten-Hyman solvers as riemann_axis, for any direction.
template <typename T, int RIEM>
__device__ __forceinline__ void riemann_normal(const T UL[5], const T UR[5], const T n[3], T vgn, T gamma, T F[5]) {
  const Prim<T> qL = primitives(UL, gamma), qR = primitives(UR, gamma);
  T FL[5], FR[5];
  normal_flux(UL, qL, n, vgn, FL);
  normal_flux(UR, qR, n, vgn, FR);
  const T unL = qL.u[0] * n[0] + qL.u[1] * n[1] + qL.u[2] * n[2];
  const T unR = qR.u[0] * n[0] + qR.u[1] * n[1] + qR.u[2] * n[2];
  const T cL = Prec<T>::sqrt_(gamma * qL.p * qL.ir), cR = Prec<T>::sqrt_(gamma * qR.p * qR.ir);
  if (RIEM == 0) {
    const T a = fmax(fabs(unL - vgn) + cL, fabs(unR - vgn) + cR);
#pragma unroll
    for (int k = 0; k < 5; ++k) F[k] = T(0.5) * (FL[k] + FR[k]) - T(0.5) * a * (UR[k] - UL[k]);
    return;
  }
  const T sL = Prec<T>::sqrt_(UL[0]), sR = Prec<T>::sqrt_(UR[0]);
  const T iss = Prec<T>::rcp(sL + sR);
  T uh[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) uh[d] = (sL * qL.u[d] + sR * qR.u[d]) * iss;
  const T HL = (UL[4] + qL.p) * qL.ir, HR = (UR[4] + qR.p) * qR.ir;
  const T Hh = (sL * HL + sR * HR) * iss;
  const T q2 = uh[0] * uh[0] + uh[1] * uh[1] + uh[2] * uh[2];
  const T ch = Prec<T>::sqrt_((gamma - T(1)) * (Hh - T(0.5) * q2));
  const T rh = sL * sR;
  const T unh = uh[0] * n[0] + uh[1] * n[1] + uh[2] * n[2];
  const T dp = qR.p - qL.p, dr = UR[0] - UL[0], dun = unR - unL;
  const T ic2 = Prec<T>::rcp(ch * ch);
  const T a1 = T(0.5) * (dp - rh * ch * dun) * ic2;
  const T a5 = T(0.5) * (dp + rh * ch * dun) * ic2;
  const T a2 = dr - dp * ic2;
  const T l1 = unh - ch - vgn, l2 = unh - vgn, l5 = unh + ch - vgn;
  T al1 = fabs(l1), al5 = fabs(l5);
  const T al2 = fabs(l2);
  const T d1 = fmax(T(0), fmax(l1 - (unL - cL - vgn), (unR - cR - vgn) - l1));
  if (al1 < d1) al1 = (l1 * l1 + d1 * d1) / (T(2) * d1);
  const T d5 = fmax(T(0), fmax(l5 - (unL + cL - vgn), (unR + cR - vgn) - l5));
  if (al5 < d5) al5 = (l5 * l5 + d5 * d5) / (T(2) * d5);
  const T w1 = al1 * a1, w5 = al5 * a5, w2 = al2 * a2;
  T du[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) du[d] = qR.u[d] - qL.u[d];
  T D[5];
  D[0] = w1 + w2 + w5;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T shear = du[d] - dun * n[d];
    const T nd = ch * n[d];
    D[1 + d] = w1 * (uh[d] - nd) + w2 * uh[d] + al2 * rh * shear + w5 * (uh[d] + nd);
  }
  const T udu = uh[0] * du[0] + uh[1] * du[1] + uh[2] * du[2];
  D[4] = w1 * (Hh - unh * ch) + w2 * T(0.5) * q2 + al2 * rh * (udu - unh * dun) + w5 * (Hh + unh * ch);
#pragma unroll
  for (int k = 0; k < 5; ++k) F[k] = T(0.5) * (FL[k] + FR[k]) - T(0.5) * D[k];
}

// Rotation about the z axis by the angle with cosine c and sine s: of the momentum of a
// state, and of the 15 primitive gradients g[a*5 + p] (a the derivative direction; the
// velocity components p = 1..3 turn too).
template <typename T>
__device__ __forceinline__ void rotate_state_z(T U[5], T c, T s) {
  const T x = c * U[1] - s * U[2], y = s * U[1] + c * U[2];
  U[1] = x;
  U[2] = y;
}
template <typename T>
__device__ __forceinline__ void rotate_grad_z(T g[15], T c, T s) {
#pragma unroll
  for (int p = 0; p < 5; ++p) {
    const T x = c * g[p] - s * g[5 + p], y = s * g[p] + c * g[5 + p];
    g[p] = x;
    g[5 + p] = y;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T x = c * g[a * 5 + 1] - s * g[a * 5 + 2], y = s * g[a * 5 + 1] + c * g[a * 5 + 2];
    g[a * 5 + 1] = x;
    g[a * 5 + 2] = y;
  }
}

// Viscous flux along physical axis a (Sec. 2, Eqs. stress_tensor, heat_flux) from the state
// and the 15 lifted gradients g[d*5 + c] = d(primitive c)/dx_d, primitives (rho, v, p):
// (0, tau_1a, tau_2a, tau_3a, tau_aj v_j + k dT/dx_a), tau with Stokes' lambda = -2/3 mu,
// T = p / (rho R).
template <typename T>
__device__ __forceinline__ void viscous_flux_axis(const T U[5], const T* g, int a, const T* c, T Fv[5]) {
  const T ir = Prec<T>::rcp(U[0]);
  const T v0 = U[1] * ir, v1 = U[2] * ir, v2 = U[3] * ir;
  const T mu = c[MC_MU];
  // column a of the velocity gradient and its transpose
  const T da0 = g[a * 5 + 1], da1 = g[a * 5 + 2], da2 = g[a * 5 + 3];          // d v_b / d x_a
  const T d0a = g[0 * 5 + 1 + a], d1a = g[1 * 5 + 1 + a], d2a = g[2 * 5 + 1 + a];  // d v_a / d x_b
  const T div = g[0 * 5 + 1] + g[1 * 5 + 2] + g[2 * 5 + 3];
  T t0 = mu * (da0 + d0a), t1 = mu * (da1 + d1a), t2 = mu * (da2 + d2a);
  const T lam = T(-2.0 / 3.0) * mu * div;
  t0 += a == 0 ? lam : T(0);
  t1 += a == 1 ? lam : T(0);
  t2 += a == 2 ? lam : T(0);
  const T p = (c[MC_GAMMA] - T(1)) * (U[4] - T(0.5) * (U[1] * v0 + U[2] * v1 + U[3] * v2));
  const T Tt = p * ir / c[MC_R];
  const T dT = (g[a * 5 + 4] - Tt * c[MC_R] * g[a * 5 + 0]) * ir / c[MC_R];
  Fv[0] = T(0);
  Fv[1] = t0;
  Fv[2] = t1;
  Fv[3] = t2;
  Fv[4] = t0 * v0 + t1 * v1 + t2 * v2 + c[MC_K] * dT;
}

// Exterior state of a weak Dirichlet face at physical position X and time t, in the
// kernel's precision: the constant background (flows 0 and 2, precomputed) or the exact
// solution (flows 1 and 3).
__device__ __forceinline__ float sin_t(float a) { return sinf(a); }
__device__ __forceinline__ double sin_t(double a) { return sin(a); }

template <typename T>
__device__ __forceinline__ void boundary_state(const MeshDev& m, const T X[3], T t, T U[5]) {
  const T* c = Prec<T>::c(m);
  if (m.flow == 0 || m.flow == 2) {
#pragma unroll
    for (int k = 0; k < 5; ++k) U[k] = c[MC_BC + k];
    return;
  }
  T P[5];
  if (m.flow == 1) {
    const T ph = Prec<T>::fpar(m, 2) * (X[0] - Prec<T>::fpar(m, 5) * t) +
                 Prec<T>::fpar(m, 3) * (X[1] - Prec<T>::fpar(m, 6) * t) +
                 Prec<T>::fpar(m, 4) * (X[2] - Prec<T>::fpar(m, 7) * t);
    P[0] = Prec<T>::fpar(m, 0) + Prec<T>::fpar(m, 1) * sin_t(T(2.0 * SM_PI) * ph);
    P[1] = Prec<T>::fpar(m, 5); P[2] = Prec<T>::fpar(m, 6); P[3] = Prec<T>::fpar(m, 7);
    P[4] = Prec<T>::fpar(m, 8);
  } else if (m.flow == 3) {
    const T xs = X[0] - Prec<T>::fpar(m, 4) * t;
    P[0] = Prec<T>::fpar(m, 0) + xs * (Prec<T>::fpar(m, 1) + xs * (Prec<T>::fpar(m, 2) + xs * Prec<T>::fpar(m, 3)));
    P[1] = Prec<T>::fpar(m, 4); P[2] = Prec<T>::fpar(m, 5); P[3] = Prec<T>::fpar(m, 6);
    P[4] = Prec<T>::fpar(m, 7);
  } else {
    P[0] = Prec<T>::fpar(m, 0); P[1] = T(0); P[2] = T(0);
    P[3] = Prec<T>::fpar(m, 2) + X[0] * (Prec<T>::fpar(m, 3) + X[0] * Prec<T>::fpar(m, 4));
    P[4] = Prec<T>::fpar(m, 1);
  }
  const T g = c[MC_GAMMA];
  U[0] = P[0];
  U[1] = P[0] * P[1];
  U[2] = P[0] * P[2];
  U[3] = P[0] * P[3];
  U[4] = P[4] / (g - T(1)) + T(0.5) * P[0] * (P[1] * P[1] + P[2] * P[2] + P[3] * P[3]);
}

// ---------------------------------------------------------------------------------------
// Flows: initial data and the weak Dirichlet boundary state (boundary = 1).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void flow_state(const MeshDev& m, double x, double y, double z, double t,
                                           int boundary, double U[5]) {
  double P[5];
  const double* f = m.fpar;
  if (m.flow == 0) {
    for (int k = 0; k < 5; ++k) P[k] = f[k];
  } else if (m.flow == 1) {
    double ph = f[2] * (x - f[5] * t) + f[3] * (y - f[6] * t) + f[4] * (z - f[7] * t);
    P[0] = f[0] + f[1] * sin(2.0 * SM_PI * ph);
    P[1] = f[5]; P[2] = f[6]; P[3] = f[7]; P[4] = f[8];
  } else if (m.flow == 2) {
    for (int k = 0; k < 5; ++k) P[k] = f[k];
    if (!boundary)
      for (int k = 0; k < 5; ++k)
        for (int q = 0; q < 8; ++q) {
          const double* md = m.modes + (k * 8 + q) * 4;
          P[k] += md[0] * sin(2.0 * SM_PI * (md[1] * y + md[2] * z) + md[3]);
        }
  } else if (m.flow == 3) {
    double xs = x - f[4] * t;
    P[0] = f[0] + xs * (f[1] + xs * (f[2] + xs * f[3]));
    P[1] = f[4]; P[2] = f[5]; P[3] = f[6]; P[4] = f[7];
  } else if (m.flow == 4) {
    P[0] = f[0]; P[1] = 0.0; P[2] = 0.0; P[3] = f[2] + x * (f[3] + x * f[4]); P[4] = f[1];
  } else if (m.flow == 5) {
    // axial stream (0, 0, f2) with a Gaussian pressure pulse (amplitude f3, width f7) at
    // (r, theta, z) = (f4, f5, f6)
    const double xc = f[4] * cos(f[5]), yc = f[4] * sin(f[5]), zc = f[6];
    const double d2 = (x - xc) * (x - xc) + (y - yc) * (y - yc) + (z - zc) * (z - zc);
    P[0] = f[0]; P[1] = 0.0; P[2] = 0.0; P[3] = f[2];
    P[4] = f[1] + (boundary ? 0.0 : f[3] * exp(-d2 / (2.0 * f[7] * f[7])));
  } else {
    // rigid rotation with angular speed f2 about the z axis
    P[0] = f[0]; P[1] = -f[2] * y; P[2] = f[2] * x; P[3] = 0.0;
    P[4] = f[1] + 0.5 * f[0] * f[2] * f[2] * (x * x + y * y);
  }
  U[0] = P[0];
  U[1] = P[0] * P[1];
  U[2] = P[0] * P[2];
  U[3] = P[0] * P[3];
  U[4] = P[4] / (m.gamma - 1.0) + 0.5 * P[0] * (P[1] * P[1] + P[2] * P[2] + P[3] * P[3]);
}

// Physical position of node (i, j, k) of element p; the moving block is shifted by delta
// (cylinder: the rotor, block 0, is turned by phi = -delta).
__device__ __forceinline__ void node_position(const MeshDev& m, const ElemPos& p, int i, int j, int k,
                                              double delta, double X[3]) {
  const double* xi = m.basis->x;
  double hx = p.blk ? m.hx1 : m.hx0;
  double xlo = p.blk ? m.x1 : m.x0;
  if (rotating_geom(m.geom)) {
    const double s3 = xlo + p.ix * hx + (xi[k] + 1.0) * 0.5 * hx;
    const double s2 = m.z0 + p.iz * m.hz + (xi[j] + 1.0) * 0.5 * m.hz;
    const double th = m.y0 + p.iy * m.hy + (xi[i] + 1.0) * 0.5 * m.hy;
    // cylinder: r = s3, z = s2; annular: r = z0 + z1 - s2, z = s3; cone: r = s2 sin(alpha) +
    // s3 cos(alpha), z = s2 cos(alpha) - s3 sin(alpha)
    const double r = m.geom == 1 ? s3 : (m.geom == 3 ? 2.0 * m.z0 + m.nz * m.hz - s2 : s2 * m.cone_s + s3 * m.cone_c);
    const double a0 = r * cos(th), a1 = r * sin(th);
    double c = 1.0, s = 0.0;
    if (p.blk == 0) sincos(-delta, &s, &c);
    X[0] = c * a0 - s * a1;
    X[1] = s * a0 + c * a1;
    X[2] = m.geom == 1 ? s2 : (m.geom == 3 ? s3 : s2 * m.cone_c - s3 * m.cone_s);
    return;
  }
  X[0] = xlo + p.ix * hx + (xi[k] + 1.0) * 0.5 * hx;
  X[1] = m.y0 + p.iy * m.hy + (xi[i] + 1.0) * 0.5 * m.hy + (p.blk ? delta : 0.0);
  X[2] = m.z0 + p.iz * m.hz + (xi[j] + 1.0) * 0.5 * m.hz;
}

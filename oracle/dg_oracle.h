/*
 * ORACLE — test infrastructure only.
 *
 * Plain, slow, FP64 CPU restatement of the sliding-mesh DGSEM operator of
 * Duerrwaechter, Kurz, Kopper, Kempf, Munz, Beck, "An Efficient Sliding Mesh
 * Interface Method for High-Order Discontinuous Galerkin Schemes"
 * (arXiv 2008.04356).  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg may load it.  It shares no code, header or table with the
 * CUDA library under paper_2008_04356_gb300/.
 *
 * Every function cites the passage of the paper it follows.  Readings where the
 * paper is silent or garbled are marked "reading:".
 */
#ifndef SLIDEMESH_DG_ORACLE_H
#define SLIDEMESH_DG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Problem description of the oracle: two structured hexahedral blocks that meet
 * at the plane x = x1 (the sliding interface, Sec. 3.3).  The static block spans
 * x in [x0, x1], the moving block x in [x1, x2]; both span y in [y0, y1] and
 * z in [z0, z1], periodic in y and z.  The moving block translates along +y with
 * speed v: its displacement is Delta(t) = delta0 + v t.  Faces along the
 * interface are equispaced: both blocks have the same element counts in y and z. */
typedef struct {
  int N;                 /* polynomial degree, 1..7 */
  int nel_s[3];          /* static block elements along x, y, z */
  int nel_m[3];          /* moving block elements along x, y, z (y, z equal to static) */
  double x0, x1, x2, y0, y1, z0, z1;
  double v, delta0;      /* grid velocity of the moving block along +y; initial displacement */
  double gamma;          /* ratio of specific heats */
  int riemann;           /* 0 = Rusanov (local Lax-Friedrichs), 1 = Roe with Harten-Hyman fix */
  int interface_conforming; /* 1: treat the interface as ordinary conforming faces (Delta must be 0) */
  int flow;              /* 0 constant state, 1 entropy wave, 2 Fourier modes (see fpar) */
  double fpar[16];
  double modes[5][8][4]; /* flow 2: per primitive variable, 8 modes of (amp, ky, kz, phase) */
  int physics;           /* 0 Euler, 1 Navier-Stokes with BR1 lifting */
  double mu, Pr, Rgas;   /* viscosity, Prandtl number, gas constant (Navier-Stokes) */
  int geom;              /* 0 plane interface (Cartesian operator); 1 cylindrical interface
                            (curvilinear operator); 2 plane interface through the
                            curvilinear operator (general metrics); 3 plane annular interface
                            normal to the rotation axis; 4 conical interface about the axis
                            (both curvilinear operator) */
  int volume;            /* volume integral (Sec. 3.1): 0 weak form; 1 split form with
                            Pirozzoli's two-point flux; 2 split form with the central
                            two-point flux (equal to the weak form by summation by parts).
                            With Navier-Stokes physics the viscous flux keeps the weak form
                            and the face flux carries the BR1 viscous mean; on curved
                            geometries the two-point flux uses the averaged metric terms of
                            its two nodes. */
  int periodic_x;        /* 1: x periodic with period x2 - x0, so that the moving block's face
                            x = x2 meets the static block's face x = x0 in a second sliding
                            interface (several interfaces, Sec. 4.3); geom 0, Euler physics */
  double cone_angle;     /* geom 4: half-angle alpha of the conical interface from the z axis */
} orc_problem;

/* geom 4, the conical sliding interface of Sec. 3.3 about the rotation axis: a point of
 * reference coordinates (theta, s, n) lies at radius rho = s sin(alpha) + n cos(alpha) and
 * height z = s cos(alpha) - n sin(alpha) (alpha = cone_angle), so s runs along the cone's
 * generator and n across it; x0 < x1 < x2 are values of n (block 0 = rotor, n in [x0, x1],
 * inside; block 1 = stator, n in [x1, x2]), [y0, y1] the periodic angular sector, [z0, z1]
 * the range of s; slip walls at s = z0, z1 and n = x0, x2; reference axes xi^1 -> theta
 * (sliding), xi^2 -> s, xi^3 -> n (J = rho h_theta h_s h_n / 8 > 0).  alpha = 0 is the
 * cylinder's map.  Motion and flows as for geom 1. */
/* geom 3, the plane annular interface of Sec. 3.3 normal to the rotation axis: x0 < x1 < x2
 * are axial positions (block 0 = rotor, z in [x0, x1]; block 1 = stator, z in [x1, x2]),
 * [y0, y1] the periodic angular sector, [z0, z1] the radii (z0 > 0); slip walls at both radii
 * and at z = x0, x2; reference axes xi^1 -> theta (sliding), xi^2 -> r (from r = z1 down to
 * r = z0: a right-handed map), xi^3 -> z.  Motion,
 * flows and the periodic sector as for geom 1. */
/* geom 1, the cylindrical sliding interface of Sec. 3.3 (a rotor inside the circle):
 * x0 < x1 < x2 are the radii (block 0 = rotor, r in [x0, x1]; block 1 = stator, r in
 * [x1, x2]), [y0, y1] the periodic angular sector (the state crosses its ends rotated by
 * the sector angle), [z0, z1] the periodic axial extent; v is the rotor's angular speed
 * omega and delta0 its angle at t = 0.  Reference axes: xi^1 -> theta (sliding), xi^2 -> z,
 * xi^3 -> r.  Walls r = x0 and r = x2 are slip walls.  Flows for the cylinder: 0 constant
 * (axial velocity only), 5 axial stream with a Gaussian pressure pulse (fpar: rho, p, w,
 * amplitude, r_c, theta_c, z_c, width), 6 rigid rotation about z (fpar: rho, p0, Omega;
 * p = p0 + rho Omega^2 r^2 / 2, a steady solution of the Euler equations). */

/* ---- 1-D basis (Sec. 3.1) ---- */
int  orc_lgl(int N, double* x, double* w);           /* N+1 Legendre-Gauss-Lobatto nodes/weights */
int  orc_gl(int N, double* x, double* w);            /* N+1 Legendre-Gauss nodes/weights */
void orc_lagrange(int N, const double* nodes, double x, double* l);  /* l[i] = ell_i(x) */
void orc_dmatrix(int N, const double* nodes, double* D);  /* D[i*(N+1)+j] = ell_j'(x_i) */
void orc_mass_exact(int N, double* M);               /* M_ij = int ell_i ell_j, exact */

/* ---- interface configuration (Sec. 4.3, Eqs. subim, indices) ---- */
void orc_map_closed(double delta, double l, long long* n, double* s);
void orc_map_pairs(long long n, int n_par, int* pairs);       /* pairs[2*i+isub] = moving partner */
int  orc_map_bruteforce(double delta, double l, int n_par, long long* n, double* s, int* pairs);

/* ---- mortar operators (Sec. 3.2, Eqs. proj_M, proj_S, projection_domain_mortar,
 *      projection_mortar_domain) ---- */
void orc_mortar_mats(int N, double sigma, double* P_lo, double* P_hi, double* B_lo, double* B_hi);

/* ---- point fluxes (Sec. 2 Eq. fluxes_written_out; Riemann solvers of Sec. 3.1) ---- */
void orc_euler_flux(const double* U, const double* n, double vgn, double gamma, double* F);
void orc_riemann(int kind, const double* UL, const double* UR, const double* n, double vgn,
                 double gamma, double* F);
/* two-point volume flux of the split form (kind 0 Pirozzoli, 1 central), Sec. 3.1 */
void orc_two_point_flux(int kind, const double* UL, const double* UR, const double* n, double vgn,
                        double gamma, double* F);

/* ---- low-storage RK (Carpenter & Kennedy (5,4), Sec. 3.1) ---- */
void orc_lsrk_coeffs(double* A, double* B, double* c);

/* ---- the discrete operator ---- */
void*     orc_create(const orc_problem* p);
void      orc_destroy(void* h);
long long orc_nelem(void* h);
void      orc_node_coords(void* h, double t, double* xyz);          /* [E][3][np^3] physical */
void      orc_init_state(void* h, double* U);                      /* U(t=0) at the nodes */
void      orc_exact_state(void* h, double t, double* U);           /* exact solution (flows 0,1) */
void      orc_rhs(void* h, const double* U, double t, double* Ut);  /* dU/dt at all nodes */
void      orc_rhs_elements(void* h, const double* U, double t, const long long* elems, int count,
                           double* Ut);                            /* dU/dt of listed elements */
void      orc_interface_fluxes(void* h, const double* U, double t, double* F_static,
                               double* F_moving);                  /* [nz][ny][5][np][np] */
void      orc_step(void* h, double* U, double* G, double* t, double dt, int nsteps);
void      orc_lifting(void* h, const double* U, double t, double* grad);  /* [E][3][5][np^3] */
void      orc_viscous_flux(const double* U, const double* grad15, double mu, double Pr, double Rgas,
                           double gamma, double* Fv15);                    /* [3][5] at one point */
void      orc_totals(void* h, const double* U, double* tot5);      /* sum J w w w U */
void      orc_metrics(void* h, double t, double* Ja, double* J);   /* Ja[E][3 (i)][3 (n)][np^3] = Ja^i_n, J[E][np^3] */
void      orc_flow_state(const orc_problem* p, const double* X, double t, int boundary, double* U);
void      orc_face_flux_sums(const orc_problem* p, const double* F_static, const double* F_moving,
                             double* sum_static5, double* sum_moving5);
double    orc_l2_error_rho(void* h, const double* U, double t);
int       orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif

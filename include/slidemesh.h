/*
 * slidemesh — sliding-mesh DGSEM hot path for one NVIDIA GB300 (sm_103a).
 *
 * The operator is the per-Runge-Kutta-stage right-hand side of the compressible Euler
 * equations in ALE form (Duerrwaechter et al., arXiv 2008.04356, Sec. 2 Eq.
 * fluxes_written_out), discretised by weak-form DGSEM on Legendre-Gauss-Lobatto nodes
 * (Sec. 3.1), with a plane sliding interface between a static and a moving block handled
 * by two mortars per face (Sec. 3.2 and 3.3; displacement decomposition and index relation
 * of Sec. 4.3, Eqs. subim and indices), advanced by the Carpenter-Kennedy low-storage RK4
 * (Sec. 3.1).
 *
 * Conventions of every call:
 *  - Every call returns an sm_status (0 = SM_OK, negative = error); no call aborts, and no
 *    kernel traps.  CUDA errors are returned as SM_ERR_CUDA; sm_last_error() gives text.
 *  - "stream" is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Calls that take a stream are asynchronous on it unless stated otherwise.
 *  - State layout (host or device): U[e][var][k][j][i], var = (rho, rho v1, rho v2, rho v3,
 *    rho e) conservative, (i, j, k) the LGL node indices along the element's reference
 *    axes xi^1 = y (sliding direction), xi^2 = z, xi^3 = x (interface normal).  Elements:
 *    static block first, e = ix + nx (iy + ny iz), then the moving block likewise.
 *    Scalars are double for SM_FP64 solvers and float for SM_FP32 solvers.
 *  - Interface face-flux layout: F[iz][iy][var][q][p], p along y (sliding), q along z;
 *    the outward normal flux of that side's face times its surface element.
 *  - A solver is not thread-safe; distinct solvers may be used from distinct threads.
 */
#ifndef SLIDEMESH_H
#define SLIDEMESH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SM_OK = 0,
  SM_PENDING = 1,
  SM_ERR_ARG = -1,
  SM_ERR_OOM = -2,
  SM_ERR_CUDA = -3,
  SM_ERR_NONFINITE = -4,
  SM_ERR_TIMEOUT = -5,
  SM_ERR_BUSY = -6,
  SM_ERR_UNSUPPORTED = -7
} sm_status;

enum { SM_FP64 = 0, SM_FP32 = 1 };
enum { SM_RUSANOV = 0, SM_ROE_HH = 1 };
enum { SM_GEOM_PLANE = 0, SM_GEOM_CYLINDER = 1, SM_GEOM_PLANE_CURVILINEAR = 2, SM_GEOM_ANNULAR = 3,
       SM_GEOM_CONE = 4 };
enum { SM_EULER = 0, SM_NAVIER_STOKES = 1 };
/* Volume integral of the element operator (Sec. 3.1):
 *  SM_VOLUME_WEAK   weak-form DGSEM, sum-factorised flux divergence with Dhat = -M^-1 D^T M;
 *  SM_VOLUME_SPLIT  split form with Pirozzoli's two-point flux (the scheme of all of the
 *                   paper's computations, used there with SM_ROE_HH): strong form, volume
 *                   term sum_l (2 D - M^-1 B)_il F#(U_i, U_l) per direction with
 *                   F#_rho = {{rho}}{{w}}, F#_rho v = F#_rho {{v}} + {{p}} n,
 *                   F#_rho e = F#_rho {{H}} + {{p}} v^g.n, {{a}} the arithmetic mean,
 *                   w = v.n - v^g.n the velocity relative to the grid, H the total enthalpy;
 *                   on curved elements n and v^g.n are the means of the two nodes' metric
 *                   vectors Ja^d and of Ja^d.v^g.  Euler physics, every geometry. */
enum { SM_VOLUME_WEAK = 0, SM_VOLUME_SPLIT = 1 };
/* Flows used as initial data (sm_init_state) and as the weak Dirichlet state at x = x0, x2
 * (SM_FLOW_SHEAR_X: rho = fpar0, p = fpar1, velocity (0, 0, fpar2 + fpar3 x + fpar4 x^2)):
 *  SM_FLOW_CONSTANT      primitive (rho, v1, v2, v3, p) = fpar[0..4]
 *  SM_FLOW_ENTROPY_WAVE  rho = fpar0 + fpar1 sin(2 pi k.(x - u t)), k = fpar2..4,
 *                        u = fpar5..7, p = fpar8
 *  SM_FLOW_MODES         background fpar[0..4] plus, per primitive variable, 8 modes
 *                        modes[var][m] = (amp, ky, kz, phase): amp sin(2 pi (ky y + kz z) + phase);
 *                        the boundary state is the background
 *  SM_FLOW_POLY_X        rho = fpar0 + fpar1 x' + fpar2 x'^2 + fpar3 x'^3, x' = x - fpar4 t,
 *                        velocity fpar4..6, p = fpar7
 *  SM_FLOW_AXIAL_PULSE   (cylinder) rho = fpar0, velocity (0, 0, fpar2), p = fpar1 plus a
 *                        Gaussian of amplitude fpar3 and width fpar7 centred at
 *                        (r, theta, z) = (fpar4, fpar5, fpar6)
 *  SM_FLOW_RIGID_ROTATION (cylinder) rho = fpar0, velocity fpar2 e_z x X,
 *                        p = fpar1 + rho fpar2^2 r^2 / 2 (a steady Euler solution) */
enum { SM_FLOW_CONSTANT = 0, SM_FLOW_ENTROPY_WAVE = 1, SM_FLOW_MODES = 2, SM_FLOW_POLY_X = 3, SM_FLOW_SHEAR_X = 4,
       SM_FLOW_AXIAL_PULSE = 5, SM_FLOW_RIGID_ROTATION = 6 };

/* Two structured hexahedral blocks sharing the plane sliding interface x = x1 (Sec. 3.3,
 * first geometry of Fig. sm_meshes_overview).  Static block x in [x0, x1], moving block
 * x in [x1, x2]; both y in [y0, y1] and z in [z0, z1], periodic in y and z.  The faces
 * along the interface are equispaced (Sec. 3.3): nel_static[1..2] must equal
 * nel_moving[1..2].  interface_conforming = 1 couples the two blocks as an ordinary
 * conforming face instead (valid only while the displacement is zero).
 *
 * geom SM_GEOM_CYLINDER: the cylindrical sliding interface (Sec. 3.3, a rotor inside the
 * circle and a stator outside, relative motion a rotation): x0 < x1 < x2 are radii (the
 * static-block slot holds the rotor, r in [x0, x1]; the moving-block slot the stator, r in
 * [x1, x2]), [y0, y1] is the periodic angular sector (states crossing its ends turn by the
 * sector angle), [z0, z1] the periodic axial extent; r = x0 and r = x2 are slip walls.
 * Curved elements from the analytic map, metric terms in conservative curl form; Euler.
 * geom SM_GEOM_PLANE_CURVILINEAR: the plane box through the same curvilinear kernels.
 *
 * geom SM_GEOM_ANNULAR: the plane annular sliding interface normal to the rotation axis (Sec.
 * 3.3, the third rotating geometry of the paper's overview figure): x0 < x1 < x2 are axial
 * positions (the static-block slot holds the rotor, z in [x0, x1]; the moving-block slot the
 * stator, z in [x1, x2]), [y0, y1] is the periodic angular sector, [z0, z1] the radii
 * (z0 > 0; element index iz runs from the outer radius inwards, which keeps the map right-
 * handed); slip walls at both radii and at z = x0, x2.  Motion, flows and curved elements
 * as for the cylinder; Euler or Navier-Stokes.
 *
 * geom SM_GEOM_CONE: the conical sliding interface about the rotation axis (Sec. 3.3, the
 * conical geometry of the overview figure): a node of angle theta, generator coordinate s in
 * [z0, z1] and normal offset n lies at radius s sin(cone_angle) + n cos(cone_angle) and height
 * s cos(cone_angle) - n sin(cone_angle); n in [x0, x1] is the rotor (inside the cone), n in
 * [x1, x2] the stator; [y0, y1] is the periodic angular sector; slip walls at s = z0, z1 and
 * n = x0, x2.  cone_angle = 0 gives the cylinder's map (with walls instead of periodic ends). */
typedef struct {
  int N;                   /* polynomial degree, 1..7 */
  int geom;                /* SM_GEOM_PLANE */
  int nel_static[3];       /* elements along x, y, z */
  int nel_moving[3];
  double x0, x1, x2, y0, y1, z0, z1;
  double gamma;            /* ratio of specific heats */
  int riemann;             /* SM_RUSANOV | SM_ROE_HH */
  int precision;           /* SM_FP64 | SM_FP32 for U, G, fluxes; mapping and mortar
                              matrices are always built in FP64 */
  int interface_conforming;
  int flow;                /* SM_FLOW_* */
  double fpar[16];
  double modes[5][8][4];
  int physics;             /* SM_EULER | SM_NAVIER_STOKES (BR1 lifting, Sec. 3.1) */
  double mu, Pr, Rgas;     /* dynamic viscosity, Prandtl number, gas constant */
  int volume;              /* SM_VOLUME_WEAK | SM_VOLUME_SPLIT */
  int periodic_x;          /* 1: x periodic with period x2 - x0 (plane geometry, Euler): the
                              moving block's face x = x2 meets the static block's face x = x0
                              in a second sliding interface with the same displacement
                              (several interfaces, Sec. 4.3); no Dirichlet faces remain.
                              sm_interface and sm_diag's interface sums cover the interface
                              x = x1 only.  Not for batches or sm_rhs_static. */
  double cone_angle;       /* SM_GEOM_CONE: half-angle of the cone from the z axis, [0, pi/2) */
} sm_mesh_desc;

/* Motion of the moving block: displacement Delta(t) = delta0 + v t along +y (Sec. 4.3,
 * Fig. coordinates); omega must be 0.  Cylinder and annulus: the rotor turns about the z axis by the
 * angle delta0 + omega t (v must be 0); the stator's displacement seen from the rotor is
 * minus that angle, in units of the angular face size. */
typedef struct {
  double v;
  double omega;
  double delta0;
} sm_motion;

typedef struct {
  long long n_delta;          /* integer face offset of the last evaluated stage */
  double s_delta;             /* sub-face fraction of the last evaluated stage, in [0, 1] */
  double t;                   /* solver time */
  double totals[5];           /* sum_e sum_ijk J w_i w_j w_k U (conserved totals) */
  double iface_sum_static[5]; /* sum over static interface faces of w_p w_q F, last stage */
  double iface_sum_moving[5]; /* same on the moving side; conservation: the two cancel */
} sm_diag_out;

typedef struct sm_solver sm_solver;

/* Creates a solver: validates desc, builds the LGL basis (FP64, host), allocates the
 * device state (two state buffers, the RK register, interface fluxes, stage parameters)
 * on the current device.  *out is library-owned; free it with sm_destroy.
 * Errors: SM_ERR_ARG (invalid desc), SM_ERR_UNSUPPORTED (N outside 1..7, geometry),
 * SM_ERR_OOM, SM_ERR_CUDA. */
int sm_init_mesh(const sm_mesh_desc* desc, sm_solver** out);

/* Sets the motion (Sec. 4.3: Delta = (n + s) l).  Takes effect at the next stage. */
int sm_set_motion(sm_solver* s, const sm_motion* motion);

/* Number of scalars of the state U (elements * 5 * (N+1)^3) and bytes per scalar. */
long long sm_state_size(const sm_solver* s);
int sm_scalar_bytes(const sm_solver* s);

/* Evaluates the desc's flow at t = 0 at every node into the solver state (on the device),
 * sets t = 0 and clears the RK register.  Asynchronous on stream. */
int sm_init_state(sm_solver* s, void* stream);

/* Copies a state in (U: host or device pointer in the solver's precision and layout;
 * on_device = 0 for host memory) and sets the solver time t.  Host copies go through the
 * given stream and the call returns after the copy has been issued; the caller keeps U
 * unchanged until the stream reaches this point (pinned host memory makes the copy
 * asynchronous, pageable memory makes it synchronous). */
int sm_set_state(sm_solver* s, const void* U, int on_device, double t, void* stream);

/* Copies the state out (host or device pointer) and returns the solver time in *t.
 * Synchronises the stream before returning. */
int sm_get_state(sm_solver* s, void* U, int on_device, double* t, void* stream);

/* Streams count independent jobs through the solver from host memory: job i takes the
 * state at in_host + i * in_stride bytes (the solver layout and precision; in_stride 0
 * reuses one input), sets the solver time to t0, advances it by nsteps RK steps of dt
 * (sm_step, Sec. 3.3 and 3.1) and writes the resulting state to out_host + i * out_stride
 * bytes (out_stride 0: every job overwrites the same output).  The copies overlap the
 * compute: while job i steps, the host-to-device copy of job i+1 and the device-to-host copy
 * of job i-1 run on two copy streams of their own, through two state-sized device staging
 * buffers that the solver allocates at the first call and keeps until sm_destroy.  Host
 * buffers should be pinned (pageable memory serialises the copies).  stream orders the
 * compute; the call returns when every result is in host memory.  The solver's state and
 * time afterwards are those of the last job.  Results equal those of sm_set_state +
 * sm_step + sm_get_state per job.  Arguments are checked before any CUDA call (NULL
 * pointers, count < 0, nsteps < 1, negative strides, dt <= 0 or non-finite t0: SM_ERR_ARG). */
int sm_stream_jobs(sm_solver* s, const void* in_host, long long in_stride, void* out_host, long long out_stride,
                   int count, double t0, double dt, int nsteps, void* stream);

/* dU/dt = R(U, t) for a caller-owned device state dU into caller-owned dUt (same layout
 * and precision), on stream: mapper and mortar matrices at time t (Sec. 4.3, 3.2), the
 * fused interface kernel (Sec. 3.3 steps 3-5), then volume + surface (Sec. 3.1).
 * dU and dUt must not overlap and must be 16-byte aligned (as cudaMalloc and PyTorch
 * allocations are; the kernels move them in 8- and 16-byte vectors), else SM_ERR_ARG before
 * any launch.  The solver's own state is not touched. */
int sm_rhs(sm_solver* s, double t, const void* dU, void* dUt, void* stream);

/* The interface operator alone (Sec. 3.3 steps 1-5) for the device state dU at time t:
 * writes both sides' face fluxes (layout above, 5 (N+1)^2 scalars per face) into the
 * caller-owned device arrays dF_static and dF_moving.  All three 16-byte aligned (else
 * SM_ERR_ARG). */
int sm_interface(sm_solver* s, double t, const void* dU, void* dF_static, void* dF_moving, void* stream);

/* Navier-Stokes solvers: the BR1-lifted gradients (Sec. 3.1) of the primitive variables
 * (rho, v1, v2, v3, p) of the device state dU at time t, into caller-owned dGrad laid out
 * [e][axis][primitive][k][j][i] (axis x, y, z), solver precision.  SM_ERR_ARG for an Euler
 * solver or arrays that are not 16-byte aligned. */
int sm_gradients(sm_solver* s, double t, const void* dU, void* dGrad, void* stream);

/* Advances the solver state by nsteps low-storage RK4 steps of size dt (five stages each,
 * stage time t + c_k dt computed on the device as fma(c_k, dt, t); the five stages'
 * interface configurations and mortar operators (Sec. 4.3, 3.2) are built in one launch at
 * the start of each step).  Asynchronous on stream; the steps are replayed from a CUDA graph
 * captured per (dt, buffer parity).  The solver time advances by dt per step. */
int sm_step(sm_solver* s, double dt, int nsteps, void* stream);

/* The same stage sequence as sm_step, launched kernel by kernel (no graph) with a CUDA
 * event pair around every launch on stream; synchronises.  ms_out[3] receives the summed
 * device time of the mapper (one launch per step), interface and element kernels,
 * launches_out[3] their launch counts (either may be NULL).  For measurement only: the state advances exactly as with
 * sm_step. */
int sm_step_profiled(sm_solver* s, double dt, int nsteps, void* stream, double* ms_out, int* launches_out);

/* Diagnostics of the current state (synchronises stream).  Returns SM_ERR_NONFINITE if
 * a total is not finite. */
int sm_diag(sm_solver* s, sm_diag_out* out, void* stream);

/* Device pointer to the solver's current state buffer (valid until the next sm_step). */
void* sm_state_ptr(sm_solver* s);

void sm_destroy(sm_solver* s);

/* sm_rhs without any device allocation.  The paper has no counterpart: this exists for
 * callers that cannot call cudaMalloc, e.g. code running while another framework owns
 * the device memory through its own pool, code in regions where an allocation (which
 * synchronises the device) is not acceptable, or embedders that forbid allocations after
 * start-up.  It computes dU/dt = R(U, t) for the mesh desc and motion into dUt exactly
 * as sm_init_mesh + sm_set_motion + sm_rhs would, but needs no solver: its scratch (stage
 * parameters, both sides' interface face fluxes) lives in one fixed 16 MiB device array
 * inside the library, and the LGL basis tables of N = 1..7 in a second fixed array; every
 * GPU that loads the library holds both until the process exits.  The caller owns dU and
 * dUt (device pointers, the solver layout and precision of desc, not overlapping, 16-byte
 * aligned; SM_ERR_ARG otherwise, before any CUDA call).
 * Plane interface, Euler, weak form, one interface (SM_ERR_UNSUPPORTED otherwise).
 *  - Sizes: the scratch needed is about 2 * faces * 5 (N+1)^2 * bytes-per-scalar plus
 *    ~10 KB (faces = nel_static[1] * nel_static[2]); larger problems are rejected with
 *    SM_ERR_ARG and a message naming both sizes (use sm_rhs for them).
 *  - The first call on a device sets that device up (looks up both arrays' device
 *    addresses, writes the basis tables with a synchronous copy, sets kernel attributes);
 *    make that first call before any stream capture.  After it, a call enqueues kernel
 *    launches on stream and copies nothing between host and device.
 *  - It calls no cudaMalloc, cudaFree or other allocating routine.
 *  - All calls share the one scratch array, whose contents persist from the last call:
 *    every byte a call reads is written by that same call first, so nothing needs
 *    clearing, but calls whose work overlaps on the GPU (other streams, other host threads)
 *    race with each other; serialise them, e.g. on one stream. */
int sm_rhs_static(const sm_mesh_desc* desc, const sm_motion* motion, double t, const void* dU, void* dUt,
                  void* stream);

/* ---- batched stepping: several solves advanced by shared launches ---- */

/* A batch advances count FP32 solvers (each with its own mesh, degree, motion and time
 * step dt[i]) together: per RK stage, one persistent launch of each kernel kind per group
 * of solvers sharing N and the Riemann solver, over a work list of (solve, CTA block)
 * items; a whole step replays from one CUDA graph.  Each solve's arithmetic is the same as
 * in a batch of one.  The solvers stay owned by the caller and must outlive the batch;
 * while in a batch a solver must be advanced only through it (sm_rhs and the state calls
 * remain usable between steps).  Errors: SM_ERR_ARG (count outside 1..1024, NULL solver,
 * non-positive dt), SM_ERR_UNSUPPORTED (an FP64 solver: the batched kernels are FP32). */
typedef struct sm_batch sm_batch;
int sm_batch_create(sm_solver* const* solvers, const double* dt, int count, sm_batch** out);

/* Chooses the launch shapes of every group (interface tile width 4/8/16 faces, persistent
 * grid sizes of the interface and element kernels) by timing the candidates on this
 * batch's own data, without changing any state; the choices are remembered per (N,
 * Riemann solver, size class) for later batches.  Synchronises stream. */
int sm_batch_autotune(sm_batch* b, void* stream);

/* nsteps batched RK steps on stream (asynchronous). */
int sm_batch_step(sm_batch* b, int nsteps, void* stream);

/* Launch shapes in use: for group g (0-based, groups ordered by first member), writes N,
 * interface tile width, interface grid and element grid into shape[4]; returns the number
 * of groups (or a negative status). */
int sm_batch_shapes(const sm_batch* b, int g, int* shape);

void sm_batch_destroy(sm_batch* b);

/* ---- serving: continuous batching of many solves ---- */

/* A request: one sliding-mesh solve of nsteps RK steps of size dt, from the desc's flow at
 * t = 0 (sm_init_state), with the given motion. */
typedef struct {
  sm_mesh_desc desc;
  sm_motion motion;
  double dt;
  int nsteps;
  int keep_state;      /* 1: keep a host copy of the final state (sm_result.state) */
} sm_request;

typedef struct {
  int status;          /* SM_OK when done, SM_PENDING while queued or running, else the error */
  double t_submit;     /* seconds on the server clock (steady clock since sm_server_create) */
  double t_admit;      /* when the solve got its slot and device memory */
  double t_done;       /* when its last step finished on the device */
  double sim_time;     /* solver time reached */
  long long dof;       /* elements * (N+1)^3 */
  int steps;
  double totals[5];    /* conserved totals of the final state */
  const void* state;   /* final state (host, solver precision and layout), owned by the server,
                          valid until sm_server_destroy; NULL unless keep_state */
  long long state_bytes;
} sm_result;

typedef struct {
  long long submitted, completed, failed, running, queued;
  long long batched_steps;       /* batched RK steps launched */
  long long dof_updates;         /* sum over completed solves of dof * 5 * steps */
  double busy_seconds;           /* wall time with at least one solve running */
  size_t bytes_in_use, peak_bytes;
  int max_concurrent;
} sm_server_stats_out;

typedef struct sm_server sm_server;

/* Starts a server on the current device with a worker thread.  Requests are admitted in
 * arrival order whenever a slot is free (at most max_slots solves resident) and the
 * solve's device memory fits in hbm_budget_bytes next to the ones already resident; all
 * resident solves are advanced together (FP32 solves through one batch per degree N and
 * Riemann solver, FP64 solves one at a time), and new requests join between steps. */
int sm_server_create(size_t hbm_budget_bytes, int max_slots, sm_server** out);

/* Queues a request (thread-safe, returns immediately); *ticket identifies it.
 * SM_ERR_ARG for an invalid request; SM_ERR_OOM if it could never fit the budget. */
int sm_submit(sm_server* s, const sm_request* req, uint64_t* ticket);

/* Status of a request (thread-safe): SM_PENDING until its last step is done. */
int sm_poll(sm_server* s, uint64_t ticket, sm_result* out);

/* Waits until every submitted request is done or timeout_s passes (SM_ERR_TIMEOUT). */
int sm_server_wait(sm_server* s, double timeout_s);

int sm_server_stats(sm_server* s, sm_server_stats_out* out);

/* Stops the worker (finishing no further steps), frees every solve and result. */
void sm_server_destroy(sm_server* s);

/* ---- building blocks exposed for testing ---- */

/* Interface configuration for count displacements (Sec. 4.3): for each d_delta[m],
 * q = delta / l, n = floor(q), s = q - n (IEEE FP64, no contraction), and the moving
 * partners of every static face i of a line of n_par faces by Eq. indices,
 * d_pairs[(m * n_par + i) * 2 + i_sub] = (i - n + i_sub - 1) mod n_par.
 * All pointers are device pointers; d_pairs may be NULL. */
int sm_map(const double* d_delta, int count, double l, int n_par, long long* d_n, double* d_s,
           int* d_pairs, void* stream);

/* Mortar operators for a face whose hanging node sits at sigma (Sec. 3.2, Eqs.
 * projection_domain_mortar and projection_mortar_domain), built in FP64 on the device:
 * d_out (device) receives P_lo, P_hi, B_lo, B_hi, each (N+1)^2 row-major, where
 * P[j][i] maps face node i to mortar node j and B[i][j] maps mortar node j to face
 * node i; lo is the mortar xi <= sigma (Jacobian (1+sigma)/2), hi the mortar xi > sigma. */
int sm_mortar_matrices(int N, double sigma, double* d_out, void* stream);

/* ---- measurement aid ---- */

/* FP64 fused multiply-add throughput probe for the roofline of the FP64 path (the paper
 * has no counterpart): launches blocks x threads threads, each running eight independent
 * chains x <- fma(x, a, b) for iters rounds, i.e. 16 * iters * blocks * threads FP64
 * flop, and writes one double per thread to d_out (device, blocks * threads doubles,
 * caller-owned).  Time it with events on stream.  Errors: SM_ERR_ARG (blocks < 1, threads
 * not a multiple of 32 in 32..1024, iters < 1, NULL d_out), SM_ERR_CUDA. */
int sm_fp64_fma_probe(int blocks, int threads, int iters, double* d_out, void* stream);

const char* sm_status_string(int status);
const char* sm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif

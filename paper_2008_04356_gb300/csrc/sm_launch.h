// Launch entry points of the kernels, shared by the translation units of the library.
#pragma once

#include "sm_common.cuh"

// Per-stage mapper + mortar operators (sm_mapper.cu).
cudaError_t launch_stage_params(const MeshDev& m, int np, StageParams* sp, double* t_dev, double t_arg,
                                double ck, double dt, int mode, cudaStream_t st);
// The five stage-parameter blocks of one RK step (sp5[0..4], stage times fma(ck[k], dt, t))
// in one launch, which then advances the stored time t_dev by dt; ticket: a zeroed counter.
struct StepCoeffs { double c[5]; };
cudaError_t launch_step_params(const MeshDev& m, int np, StageParams* sp5, double* t_dev, const double* ck, double dt,
                               unsigned* ticket, cudaStream_t st);
cudaError_t launch_map_batch(const double* d_delta, int count, double l, int n_par, long long* d_n,
                             double* d_s, int* d_pairs, cudaStream_t st);
cudaError_t launch_mortar_ops(const BasisDev* b, int np, double sigma, double* d_out, cudaStream_t st);

// Element kernel modes.
enum { ELEM_RHS = 0, ELEM_STAGE = 1, ELEM_STAGE_FIRST = 2 };

struct ElemArgs {
  MeshDev m;
  const StageParams* sp;
  const void* U;     // state read (neighbour traces come from here too)
  void* out;         // ELEM_RHS: dU/dt;  ELEM_STAGE*: updated state
  void* G;           // RK register (stage modes)
  const void* Fs;    // interface face fluxes, static side
  const void* Fm;    // interface face fluxes, moving side
  double rkA, rkB, dt;
  const void* Gr = nullptr;   // lifted gradients (Navier-Stokes)
  void* Ts = nullptr;         // stage modes: interface traces of the updated state, static side
  void* Tm = nullptr;         // ... moving side ([n_perp][n_par][5][(N+1)^2], nullptr: not written)
};

// sm_curved_f32.cu / sm_curved_f64.cu: curvilinear geometries (MeshDev::geom != 0)
cudaError_t launch_curved_element_f32(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st);
cudaError_t launch_curved_element_f64(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st);
cudaError_t launch_curved_interface_f32(int N, int riemann, const MeshDev& m, const StageParams* sp, const void* U,
                                        void* Fs, void* Fm, cudaStream_t st);
cudaError_t launch_curved_interface_f64(int N, int riemann, const MeshDev& m, const StageParams* sp, const void* U,
                                        void* Fs, void* Fm, cudaStream_t st);
cudaError_t prepare_curved_f32(int N);
// sm_curved_split_f32.cu / sm_curved_split_f64.cu: the split-form volume integral on curved
// elements (Euler), same faces, surface integral and RK update as the curved element kernel
cudaError_t launch_curved_split_f32(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st);
cudaError_t launch_curved_split_f64(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st);
cudaError_t prepare_curved_split_f32(int N);
cudaError_t prepare_curved_split_f64(int N);
// sm_curved_split_ns_f32.cu / sm_curved_split_ns_f64.cu: the same with Navier-Stokes physics
// (advective terms split, viscous terms weak, BR1 lifted gradients a.Gr)
cudaError_t launch_curved_split_ns_f32(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st);
cudaError_t launch_curved_split_ns_f64(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st);
cudaError_t prepare_curved_split_ns_f32(int N);
cudaError_t prepare_curved_split_ns_f64(int N);
cudaError_t upload_dhat_curved_split_ns_f32(const float* f, const double* d);
cudaError_t upload_dhat_curved_split_ns_f64(const float* f, const double* d);
cudaError_t prepare_curved_f64(int N);
cudaError_t upload_dhat_curved_f32(const float* f, const double* d);
cudaError_t upload_dhat_curved_f64(const float* f, const double* d);
// sm_curved_ns_f32.cu / sm_curved_ns_f64.cu: curvilinear Navier-Stokes (lifting values per
// interface face node: 15, a * 5 + c)
#define SM_CURVED_NS_DECL(S)                                                                                       \
  cudaError_t launch_curved_element_ns_##S(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st);     \
  cudaError_t launch_curved_lift_##S(int N, const MeshDev& m, const StageParams* sp, const void* U, void* Gr,     \
                                     const void* Ls, const void* Lm, cudaStream_t st);                            \
  cudaError_t launch_curved_interface_lift_##S(int N, const MeshDev& m, const StageParams* sp, const void* U,     \
                                               void* Ls, void* Lm, cudaStream_t st);                              \
  cudaError_t launch_curved_interface_ns_##S(int N, int riemann, const MeshDev& m, const StageParams* sp,         \
                                             const void* U, const void* Gr, void* Fs, void* Fm, cudaStream_t st); \
  cudaError_t prepare_curved_ns_##S(int N);                                                                        \
  cudaError_t upload_dhat_curved_ns_##S(const float* f, const double* d);
SM_CURVED_NS_DECL(f32)
SM_CURVED_NS_DECL(f64)
#undef SM_CURVED_NS_DECL

// sm_elem_f32.cu / sm_elem_f64.cu
cudaError_t launch_element_f32(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st);
cudaError_t launch_element_f64(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st);
cudaError_t prepare_element_f32(int N);
cudaError_t prepare_element_f64(int N);

// sm_elem_split_f32.cu / sm_elem_split_f64.cu: the split-form volume integral (Pirozzoli's
// two-point flux) with the same faces, surface integral and RK update
cudaError_t launch_element_split_f32(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st);
cudaError_t launch_element_split_f64(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st);
cudaError_t prepare_element_split_f32(int N);
cudaError_t prepare_element_split_f64(int N);
// sm_elem_split_ns_f32.cu / sm_elem_split_ns_f64.cu: the split form with Navier-Stokes physics
// (advective terms split, viscous terms weak, BR1 lifted gradients a.Gr)
cudaError_t launch_element_split_ns_f32(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st);
cudaError_t launch_element_split_ns_f64(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st);
cudaError_t prepare_element_split_ns_f32(int N);
cudaError_t prepare_element_split_ns_f64(int N);
// their constant memory: the Dhat tables (viscous terms) and the Ds tables (advective terms)
cudaError_t upload_split_ns_constants_f32(const float* dhf, const double* dhd, const float* dsf, const double* dsd);
cudaError_t upload_split_ns_constants_f64(const float* dhf, const double* dhd, const float* dsf, const double* dsd);
// constant-memory Ds = 2 D - M^-1 B tables of the split kernels ([7][64], N = 1..7)
cudaError_t upload_dsplit_f32(const float* f, const double* d);
cudaError_t upload_dsplit_f64(const float* f, const double* d);

// constant-memory Dhat tables of the element kernels ([7][64], N = 1..7), one copy per unit
cudaError_t upload_dhat_f32(const float* f, const double* d);
cudaError_t upload_dhat_f64(const float* f, const double* d);
cudaError_t upload_dhat_batch(const float* f, const double* d);

// Navier-Stokes (sm_elem_ns_f32.cu / sm_elem_ns_f64.cu / sm_iface_ns.cu)
cudaError_t launch_element_ns_f32(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st);
cudaError_t launch_element_ns_f64(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st);
cudaError_t launch_lift_f32(int N, const MeshDev& m, const StageParams* sp, const void* U, void* Gr, const void* Ls,
                            const void* Lm, cudaStream_t st);
cudaError_t launch_lift_f64(int N, const MeshDev& m, const StageParams* sp, const void* U, void* Gr, const void* Ls,
                            const void* Lm, cudaStream_t st);
cudaError_t prepare_ns_f32(int N);
cudaError_t prepare_ns_f64(int N);
cudaError_t upload_dhat_ns_f32(const float* f, const double* d);
cudaError_t upload_dhat_ns_f64(const float* f, const double* d);
cudaError_t launch_interface_ns(int N, int prec, int riemann, const MeshDev& m, const StageParams* sp, const void* U,
                                const void* Gr, void* Fs, void* Fm, cudaStream_t st);
cudaError_t launch_interface_lift(int N, int prec, const MeshDev& m, const StageParams* sp, const void* U, void* Ls,
                                  void* Lm, cudaStream_t st);
cudaError_t prepare_interface_ns(int N, int prec);

// sm_iface.cu
// Ts / Tm: the interface traces of U in the compact layout of the face fluxes (written by
// the stage-mode element kernel or launch_gather_traces), or nullptr to read them from U.
cudaError_t launch_interface(int N, int prec, int riemann, const MeshDev& m, const StageParams* sp, const void* U,
                             void* Fs, void* Fm, cudaStream_t st, const void* Ts = nullptr, const void* Tm = nullptr);
// sm_aux.cu: the interface traces of U into Ts / Tm (ifc 1: the second interface of a
// periodic x direction, x-momentum mirrored)
cudaError_t launch_gather_traces(int N, int prec, const MeshDev& m, const void* U, void* Ts, void* Tm, cudaStream_t st,
                                 int ifc = 0);
cudaError_t prepare_interface(int N, int prec);

// sm_aux.cu: initial data, reductions
cudaError_t launch_init_state(int N, int prec, const MeshDev& m, void* U, cudaStream_t st);
cudaError_t launch_fp64_fma_probe(int blocks, int threads, int iters, double* out, cudaStream_t st);
cudaError_t launch_totals(int N, int prec, const MeshDev& m, const void* U, double* partial, int nblk,
                          double* out5, cudaStream_t st);
cudaError_t launch_face_sums(int N, int prec, const MeshDev& m, const void* F, double* partial, int nblk,
                             double* out5, cudaStream_t st);

// ---- batched execution (sm_batch.cu): several FP32 solves of one degree N per launch ----
// One entry per solve, in device memory.  cur is the state buffer at the start of the next
// batched step; a stage k reads U[cur ^ (k & 1)] and writes the other buffer.
struct BatchSolveDev {
  MeshDev m;
  StageParams* sp;
  void* U[2];
  void* G;
  void* Fs;
  void* Fm;
  void* Ts;          // interface traces of the current state (static, moving side)
  void* Tm;
  double* t_d;
  double dt;
  int cur;
  int pad;
};

#define SM_MAX_BATCH 1024

cudaError_t launch_batch_stage_params(int N, const BatchSolveDev* d_bs, int nsolve, double ck, int mode, cudaStream_t st);
cudaError_t launch_batch_interface(int N, int riemann, int tf, const BatchSolveDev* d_bs, const int* d_offs, int nsolve,
                                   int grid, int stage, cudaStream_t st);
cudaError_t launch_batch_element(int N, int riemann, int mode, const BatchSolveDev* d_bs, const int* d_offs, int nsolve,
                                 int grid, int stage, double rkA, double rkB, cudaStream_t st);
cudaError_t launch_batch_flip(BatchSolveDev* d_bs, int nsolve, cudaStream_t st);
cudaError_t prepare_batch(int N);
int batch_elements_per_block(int N);
// tile width (static faces per work item) the batched interface kernel uses for a requested tf
int batch_interface_tile(int N, int tf);

// Curvilinear Navier-Stokes kernels, double state: element kernel with viscous terms
// (PHYS 1), BR1 lifting with metric terms, interface lifting values and viscous interface
// fluxes on the cylindrical interface (N = 1..7).
#include "sm_curved_impl.cuh"

cudaError_t launch_curved_element_ns_f64(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st) {
#define SM_CALL(n) launch_ce_n<n, double, 1>(riemann, mode, a, st)
  SM_CURVED_SWITCH(SM_CALL)
#undef SM_CALL
}

cudaError_t launch_curved_lift_f64(int N, const MeshDev& m, const StageParams* sp, const void* U, void* Gr,
                                   const void* Ls, const void* Lm, cudaStream_t st) {
#define SM_CALL(n) launch_cl_n<n, double>(m, sp, U, Gr, Ls, Lm, st)
  SM_CURVED_SWITCH(SM_CALL)
#undef SM_CALL
}

cudaError_t launch_curved_interface_lift_f64(int N, const MeshDev& m, const StageParams* sp, const void* U, void* Ls,
                                             void* Lm, cudaStream_t st) {
#define SM_CALL(n) launch_ci_n<n, double, CV_LIFT>(0, m, sp, U, Ls, Lm, nullptr, st)
  SM_CURVED_SWITCH(SM_CALL)
#undef SM_CALL
}

cudaError_t launch_curved_interface_ns_f64(int N, int riemann, const MeshDev& m, const StageParams* sp, const void* U,
                                           const void* Gr, void* Fs, void* Fm, cudaStream_t st) {
#define SM_CALL(n) launch_ci_n<n, double, CV_NS>(riemann, m, sp, U, Fs, Fm, Gr, st)
  SM_CURVED_SWITCH(SM_CALL)
#undef SM_CALL
}

namespace {
template <int N>
cudaError_t prepare_all() {
  cudaError_t r[4] = {prepare_ce_n<N, double, 1>(), prepare_cl_n<N, double>(), prepare_ci_n<N, double, CV_LIFT>(),
                      prepare_ci_n<N, double, CV_NS>()};
  for (cudaError_t e : r)
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}
}  // namespace

cudaError_t prepare_curved_ns_f64(int N) {
#define SM_CALL(n) prepare_all<n>()
  SM_CURVED_SWITCH(SM_CALL)
#undef SM_CALL
}

cudaError_t upload_dhat_curved_ns_f64(const float* f, const double* d) { return upload_dhat_here(f, d); }

// Split-form element kernel with Navier-Stokes physics, float state (N = 1..7, Rusanov / Roe,
// three modes): the advective terms in the split form, the viscous terms of the BR1-lifted
// gradients in the weak form.
#include "sm_split.cuh"

cudaError_t launch_element_split_ns_f32(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st) {
  SM_SPLIT_DISPATCH(float, N, riemann, mode, a, st, 1)
}

cudaError_t prepare_element_split_ns_f32(int N) { SM_SPLIT_PREPARE(float, N, 1) }

cudaError_t upload_split_ns_constants_f32(const float* dhf, const double* dhd, const float* dsf, const double* dsd) {
  cudaError_t e = upload_dsplit_here(dsf, dsd);
  if (e != cudaSuccess) return e;
  return upload_dhat_here(dhf, dhd);
}

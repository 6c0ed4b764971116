// Split-form element kernel on curved elements with Navier-Stokes physics, double state
// (N = 1..7, Rusanov / Roe, three modes): advective terms split, viscous terms weak.
#include "sm_curved_split.cuh"

cudaError_t launch_curved_split_ns_f64(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st) {
#define SM_CALL(n) launch_cs_n<n, double, 1>(riemann, mode, a, st)
  SM_CURVED_SPLIT_SWITCH(SM_CALL)
#undef SM_CALL
}

cudaError_t prepare_curved_split_ns_f64(int N) {
#define SM_CALL(n) prepare_cs_n<n, double, 1>()
  SM_CURVED_SPLIT_SWITCH(SM_CALL)
#undef SM_CALL
}

cudaError_t upload_dhat_curved_split_ns_f64(const float* f, const double* d) { return upload_dhat_here(f, d); }

// Split-form element kernel instantiations, float state (N = 1..7, Rusanov / Roe, three modes).
#include "sm_split.cuh"

cudaError_t launch_element_split_f32(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st) {
  SM_SPLIT_DISPATCH(float, N, riemann, mode, a, st, 0)
}

cudaError_t prepare_element_split_f32(int N) { SM_SPLIT_PREPARE(float, N, 0) }

cudaError_t upload_dsplit_f32(const float* f, const double* d) { return upload_dsplit_here(f, d); }

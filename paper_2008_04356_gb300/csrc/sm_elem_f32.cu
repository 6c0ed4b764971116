// Element kernel instantiations, float state (N = 1..7, Rusanov / Roe, three modes).
#include "sm_element.cuh"

cudaError_t launch_element_f32(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st) {
  SM_ELEM_DISPATCH(float, N, riemann, mode, a, st)
}

cudaError_t prepare_element_f32(int N) { SM_ELEM_PREPARE(float, N) }

cudaError_t upload_dhat_f32(const float* f, const double* d) { return upload_dhat_here(f, d); }

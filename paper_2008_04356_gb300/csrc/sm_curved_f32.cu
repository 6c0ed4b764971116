// Curvilinear kernels (cylindrical sliding interface, curved elements), float state:
// element kernel (Euler, N = 1..7, Rusanov / Roe, three modes) and interface kernel.
#include "sm_curved_impl.cuh"

cudaError_t launch_curved_element_f32(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st) {
#define SM_CALL(n) launch_ce_n<n, float, 0>(riemann, mode, a, st)
  SM_CURVED_SWITCH(SM_CALL)
#undef SM_CALL
}

cudaError_t launch_curved_interface_f32(int N, int riemann, const MeshDev& m, const StageParams* sp, const void* U,
                                       void* Fs, void* Fm, cudaStream_t st) {
#define SM_CALL(n) launch_ci_n<n, float, CV_EULER>(riemann, m, sp, U, Fs, Fm, nullptr, st)
  SM_CURVED_SWITCH(SM_CALL)
#undef SM_CALL
}

cudaError_t prepare_curved_f32(int N) {
#define SM_CALL(n) (prepare_ce_n<n, float, 0>() != cudaSuccess ? prepare_ce_n<n, float, 0>() : prepare_ci_n<n, float, CV_EULER>())
  SM_CURVED_SWITCH(SM_CALL)
#undef SM_CALL
}

cudaError_t upload_dhat_curved_f32(const float* f, const double* d) { return upload_dhat_here(f, d); }

// Split-form element kernel on curved elements, float state (N = 1..7, Rusanov / Roe, three modes).
#include "sm_curved_split.cuh"

cudaError_t launch_curved_split_f32(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st) {
#define SM_CALL(n) launch_cs_n<n, float>(riemann, mode, a, st)
  SM_CURVED_SPLIT_SWITCH(SM_CALL)
#undef SM_CALL
}

cudaError_t prepare_curved_split_f32(int N) {
#define SM_CALL(n) prepare_cs_n<n, float>()
  SM_CURVED_SPLIT_SWITCH(SM_CALL)
#undef SM_CALL
}

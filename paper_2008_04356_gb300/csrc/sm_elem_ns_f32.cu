// Navier-Stokes instantiations, float state: element kernel with viscous terms (PHYS 1) and
// the BR1 lifting kernel, N = 1..7.
#include "sm_lift.cuh"

namespace {

template <int N>
__global__ void __launch_bounds__(ElemCfg<N>::THREADS)
lift_kernel(const MeshDev m, const StageParams* __restrict__ sp, const float* __restrict__ U, float* __restrict__ Gr,
            const float* __restrict__ Ls, const float* __restrict__ Lm) {
  lift_block<N, float>(m, sp, U, Gr, Ls, Lm, (long long)blockIdx.x * ElemCfg<N>::EPB);
}

template <int N>
cudaError_t launch_lift_n(const MeshDev& m, const StageParams* sp, const void* U, void* Gr, const void* Ls,
                          const void* Lm, cudaStream_t st) {
  using C = ElemCfg<N>;
  const long long blocks = (m.E + C::EPB - 1) / C::EPB;
  if (blocks <= 0) return cudaSuccess;
  lift_kernel<N><<<(unsigned)blocks, C::THREADS, C::template smem_bytes<float>(), st>>>(
      m, sp, (const float*)U, (float*)Gr, (const float*)Ls, (const float*)Lm);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_ns_n(int riemann, int mode, const ElemArgs& a, cudaStream_t st) {
  if (riemann == 0) {
    if (mode == ELEM_RHS) return launch_elem_t<N, float, 0, ELEM_RHS, 1>(a, st);
    if (mode == ELEM_STAGE) return launch_elem_t<N, float, 0, ELEM_STAGE, 1>(a, st);
    return launch_elem_t<N, float, 0, ELEM_STAGE_FIRST, 1>(a, st);
  }
  if (mode == ELEM_RHS) return launch_elem_t<N, float, 1, ELEM_RHS, 1>(a, st);
  if (mode == ELEM_STAGE) return launch_elem_t<N, float, 1, ELEM_STAGE, 1>(a, st);
  return launch_elem_t<N, float, 1, ELEM_STAGE_FIRST, 1>(a, st);
}

template <int N>
cudaError_t prepare_ns_n() {
  cudaError_t r[7] = {prepare_elem_t<N, float, 0, ELEM_RHS, 1>(), prepare_elem_t<N, float, 0, ELEM_STAGE, 1>(),
                      prepare_elem_t<N, float, 0, ELEM_STAGE_FIRST, 1>(), prepare_elem_t<N, float, 1, ELEM_RHS, 1>(),
                      prepare_elem_t<N, float, 1, ELEM_STAGE, 1>(), prepare_elem_t<N, float, 1, ELEM_STAGE_FIRST, 1>(),
                      cudaFuncSetAttribute(lift_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)ElemCfg<N>::template smem_bytes<float>())};
  for (cudaError_t e : r)
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

}  // namespace

#define SM_NS_SWITCH(call)                  \
  switch (N) {                              \
    case 1: return call(1);                 \
    case 2: return call(2);                 \
    case 3: return call(3);                 \
    case 4: return call(4);                 \
    case 5: return call(5);                 \
    case 6: return call(6);                 \
    case 7: return call(7);                 \
    default: return cudaErrorInvalidValue;  \
  }

cudaError_t launch_element_ns_f32(int N, int riemann, int mode, const ElemArgs& a, cudaStream_t st) {
#define C_(n) launch_ns_n<n>(riemann, mode, a, st)
  SM_NS_SWITCH(C_)
#undef C_
}

cudaError_t launch_lift_f32(int N, const MeshDev& m, const StageParams* sp, const void* U, void* Gr, const void* Ls,
                         const void* Lm, cudaStream_t st) {
#define C_(n) launch_lift_n<n>(m, sp, U, Gr, Ls, Lm, st)
  SM_NS_SWITCH(C_)
#undef C_
}

cudaError_t prepare_ns_f32(int N) {
#define C_(n) prepare_ns_n<n>()
  SM_NS_SWITCH(C_)
#undef C_
}

cudaError_t upload_dhat_ns_f32(const float* f, const double* d) { return upload_dhat_here(f, d); }

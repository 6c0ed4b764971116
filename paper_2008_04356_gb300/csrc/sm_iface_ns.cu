// Interface kernel instantiations for the Navier-Stokes flux mode (tile of TF_NS faces,
// gradient traces staged) and the BR1 lifting mode.
#include "sm_iface.cuh"

namespace {

template <int N, typename T, int RIEM, int TF, int MODE>
__global__ void __launch_bounds__(IfCfg<N>::THREADS)
interface_mode_kernel(const MeshDev m, const StageParams* __restrict__ sp, const T* __restrict__ U, T* __restrict__ Fs,
                      T* __restrict__ Fm, const T* __restrict__ Gr) {
  interface_tile<N, T, RIEM, TF, MODE>(m, sp, U, Fs, Fm, blockIdx.x, blockIdx.y, Gr);
}

template <int N, typename T, int RIEM, int TF, int MODE>
cudaError_t launch_mode_t(const MeshDev& m, const StageParams* sp, const void* U, const void* Gr, void* Fs, void* Fm,
                          cudaStream_t st) {
  dim3 grid((m.ny + TF - 1) / TF, m.nz);
  interface_mode_kernel<N, T, RIEM, TF, MODE><<<grid, IfCfg<N>::THREADS, IfCfg<N>::template smem_bytes<T, TF, MODE>(), st>>>(
      m, sp, (const T*)U, (T*)Fs, (T*)Fm, (const T*)Gr);
  return cudaGetLastError();
}

template <int N, typename T, int RIEM, int TF, int MODE>
cudaError_t prep_mode_t() {
  return cudaFuncSetAttribute(interface_mode_kernel<N, T, RIEM, TF, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)IfCfg<N>::template smem_bytes<T, TF, MODE>());
}

template <int N>
cudaError_t launch_ns_n(int prec, int riemann, const MeshDev& m, const StageParams* sp, const void* U, const void* Gr,
                        void* Fs, void* Fm, cudaStream_t st) {
  constexpr int TF = IfCfg<N>::TF_NS;
  if (prec == 0)
    return riemann ? launch_mode_t<N, double, 1, TF, IF_NS>(m, sp, U, Gr, Fs, Fm, st)
                   : launch_mode_t<N, double, 0, TF, IF_NS>(m, sp, U, Gr, Fs, Fm, st);
  return riemann ? launch_mode_t<N, float, 1, TF, IF_NS>(m, sp, U, Gr, Fs, Fm, st)
                 : launch_mode_t<N, float, 0, TF, IF_NS>(m, sp, U, Gr, Fs, Fm, st);
}

template <int N>
cudaError_t launch_lift_n(int prec, const MeshDev& m, const StageParams* sp, const void* U, void* Ls, void* Lm,
                          cudaStream_t st) {
  constexpr int TF = IfCfg<N>::TF;
  if (prec == 0) return launch_mode_t<N, double, 0, TF, IF_LIFT>(m, sp, U, nullptr, Ls, Lm, st);
  return launch_mode_t<N, float, 0, TF, IF_LIFT>(m, sp, U, nullptr, Ls, Lm, st);
}

template <int N>
cudaError_t prep_n(int prec) {
  constexpr int TF = IfCfg<N>::TF, TFN = IfCfg<N>::TF_NS;
  cudaError_t r[3];
  if (prec == 0) {
    r[0] = prep_mode_t<N, double, 0, TFN, IF_NS>();
    r[1] = prep_mode_t<N, double, 1, TFN, IF_NS>();
    r[2] = prep_mode_t<N, double, 0, TF, IF_LIFT>();
  } else {
    r[0] = prep_mode_t<N, float, 0, TFN, IF_NS>();
    r[1] = prep_mode_t<N, float, 1, TFN, IF_NS>();
    r[2] = prep_mode_t<N, float, 0, TF, IF_LIFT>();
  }
  for (cudaError_t e : r)
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

}  // namespace

#define SM_IFNS_SWITCH(call)                \
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

cudaError_t launch_interface_ns(int N, int prec, int riemann, const MeshDev& m, const StageParams* sp, const void* U,
                                const void* Gr, void* Fs, void* Fm, cudaStream_t st) {
#define C_(n) launch_ns_n<n>(prec, riemann, m, sp, U, Gr, Fs, Fm, st)
  SM_IFNS_SWITCH(C_)
#undef C_
}

cudaError_t launch_interface_lift(int N, int prec, const MeshDev& m, const StageParams* sp, const void* U, void* Ls,
                                  void* Lm, cudaStream_t st) {
#define C_(n) launch_lift_n<n>(prec, m, sp, U, Ls, Lm, st)
  SM_IFNS_SWITCH(C_)
#undef C_
}

cudaError_t prepare_interface_ns(int N, int prec) {
#define C_(n) prep_n<n>(prec)
  SM_IFNS_SWITCH(C_)
#undef C_
}

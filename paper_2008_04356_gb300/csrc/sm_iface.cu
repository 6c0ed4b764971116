// Single-solve launch of the fused sliding-interface kernel (bodies in sm_iface.cuh): for FP32
// states at odd N the warp-owned rows, the staged tile otherwise.
#include "sm_iface.cuh"

namespace {

// persistent grid of the FP32 interface kernel: CTAs per SM x SMs of the current device
int fused_sms() {
  static int sms[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (sms[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    sms[dev] = v;
  }
  return sms[dev];
}

template <int N, typename T, int RIEM>
__global__ void __launch_bounds__(IfCfg<N>::THREADS, sizeof(T) == 4 ? IfCfg<N>::MINB : 1)
sliding_interface_kernel(const MeshDev m, const StageParams* __restrict__ sp, const T* __restrict__ U,
                         T* __restrict__ Fs, T* __restrict__ Fm, const T* __restrict__ Ts, const T* __restrict__ Tm) {
  interface_tile<N, T, RIEM, IfCfg<N>::TF>(m, sp, U, Fs, Fm, blockIdx.x, blockIdx.y, nullptr, Ts, Tm);
}

template <int N, int RIEM, int TF>
int warp_ctas_per_sm() {
  static int n = 0;
  if (n == 0) {
    using W = IfWarpCfg<N, TF>;
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, sliding_interface_warp_kernel<N, RIEM, TF>, W::THREADS,
                                                      W::smem_bytes) != cudaSuccess || v <= 0)
      v = 1;
    n = v;
  }
  return n;
}

template <int N, typename T, int RIEM>
cudaError_t launch_if_t(const MeshDev& m, const StageParams* sp, const void* U, void* Fs, void* Fm, cudaStream_t st,
                        const void* Ts, const void* Tm) {
  if constexpr (sizeof(T) == 4 && N % 2 == 1) {
    using W = IfWarpCfg<N, SM_IF_WARP_TF>;
    const long long tiles = (long long)((m.ny + W::TF - 1) / W::TF) * m.nz;
    if (tiles <= 0) return cudaSuccess;
    const long long cap = (long long)warp_ctas_per_sm<N, RIEM, W::TF>() * fused_sms();
    const long long grid = tiles < cap ? tiles : cap;
    sliding_interface_warp_kernel<N, RIEM, W::TF><<<(unsigned)grid, W::THREADS, W::smem_bytes, st>>>(
        m, sp, (const float*)U, (float*)Fs, (float*)Fm, (const float*)Ts, (const float*)Tm);
    return cudaGetLastError();
  } else {
    using C = IfCfg<N>;
    dim3 grid((m.ny + C::TF - 1) / C::TF, m.nz);
    sliding_interface_kernel<N, T, RIEM><<<grid, C::THREADS, C::template smem_bytes<T>(), st>>>(
        m, sp, (const T*)U, (T*)Fs, (T*)Fm, (const T*)Ts, (const T*)Tm);
    return cudaGetLastError();
  }
}

template <int N, typename T>
cudaError_t prepare_if_t() {
  if constexpr (sizeof(T) == 4 && N % 2 == 1) {
    using W = IfWarpCfg<N, SM_IF_WARP_TF>;
    const cudaError_t r[2] = {
        cudaFuncSetAttribute(sliding_interface_warp_kernel<N, 0, W::TF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)W::smem_bytes),
        cudaFuncSetAttribute(sliding_interface_warp_kernel<N, 1, W::TF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)W::smem_bytes)};
    for (cudaError_t e : r)
      if (e != cudaSuccess) return e;
    return cudaSuccess;
  } else {
    using C = IfCfg<N>;
    cudaError_t e0 = cudaFuncSetAttribute(sliding_interface_kernel<N, T, 0>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::template smem_bytes<T>());
    cudaError_t e1 = cudaFuncSetAttribute(sliding_interface_kernel<N, T, 1>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::template smem_bytes<T>());
    return e0 != cudaSuccess ? e0 : e1;
  }
}

template <int N>
cudaError_t launch_if_n(int prec, int riemann, const MeshDev& m, const StageParams* sp, const void* U, void* Fs,
                        void* Fm, cudaStream_t st, const void* Ts, const void* Tm) {
  if (prec == 0)
    return riemann ? launch_if_t<N, double, 1>(m, sp, U, Fs, Fm, st, Ts, Tm)
                   : launch_if_t<N, double, 0>(m, sp, U, Fs, Fm, st, Ts, Tm);
  return riemann ? launch_if_t<N, float, 1>(m, sp, U, Fs, Fm, st, Ts, Tm)
                 : launch_if_t<N, float, 0>(m, sp, U, Fs, Fm, st, Ts, Tm);
}

template <int N>
cudaError_t prepare_if_n(int prec) {
  return prec == 0 ? prepare_if_t<N, double>() : prepare_if_t<N, float>();
}

}  // namespace

cudaError_t launch_interface(int N, int prec, int riemann, const MeshDev& m, const StageParams* sp, const void* U,
                             void* Fs, void* Fm, cudaStream_t st, const void* Ts, const void* Tm) {
  switch (N) {
    case 1: return launch_if_n<1>(prec, riemann, m, sp, U, Fs, Fm, st, Ts, Tm);
    case 2: return launch_if_n<2>(prec, riemann, m, sp, U, Fs, Fm, st, Ts, Tm);
    case 3: return launch_if_n<3>(prec, riemann, m, sp, U, Fs, Fm, st, Ts, Tm);
    case 4: return launch_if_n<4>(prec, riemann, m, sp, U, Fs, Fm, st, Ts, Tm);
    case 5: return launch_if_n<5>(prec, riemann, m, sp, U, Fs, Fm, st, Ts, Tm);
    case 6: return launch_if_n<6>(prec, riemann, m, sp, U, Fs, Fm, st, Ts, Tm);
    case 7: return launch_if_n<7>(prec, riemann, m, sp, U, Fs, Fm, st, Ts, Tm);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t prepare_interface(int N, int prec) {
  switch (N) {
    case 1: return prepare_if_n<1>(prec);
    case 2: return prepare_if_n<2>(prec);
    case 3: return prepare_if_n<3>(prec);
    case 4: return prepare_if_n<4>(prec);
    case 5: return prepare_if_n<5>(prec);
    case 6: return prepare_if_n<6>(prec);
    case 7: return prepare_if_n<7>(prec);
    default: return cudaErrorInvalidValue;
  }
}

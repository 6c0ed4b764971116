// Kernels and launchers of the curvilinear path for one state precision SM_CURVED_T
// (included by sm_curved_f32.cu / sm_curved_f64.cu with SM_CURVED_T and SM_CURVED_SUFFIX).
#pragma once

#include "sm_curved.cuh"

namespace {

// Resident CTAs per SM asked of the register allocator for the element kernel: FP32 at N = 7
// two CTAs of 512 threads (64 registers), so that 32 warps hide the global-load latency of the
// state, geometry and neighbour traces instead of 16.
template <int N, typename T>
__host__ __device__ constexpr int curved_elem_minb() {
#ifdef SM_CURVED_MINB_OVERRIDE
  return SM_CURVED_MINB_OVERRIDE;
#else
  return sizeof(T) == 4 && N == 7 ? 2 : 1;
#endif
}

template <int N, typename T, int RIEM, int MODE, int PHYS>
__global__ void __launch_bounds__(ElemCfg<N>::THREADS, curved_elem_minb<N, T>())
curved_element_kernel(const MeshDev m, const StageParams* __restrict__ sp, const T* __restrict__ U,
                      T* __restrict__ out, T* __restrict__ G, const T* __restrict__ Fs, const T* __restrict__ Fm,
                      const T rkA, const T rkB, const T dt, const T* __restrict__ Gr) {
  curved_element_block<N, T, RIEM, MODE, PHYS>(m, sp, U, out, G, Fs, Fm, rkA, rkB, dt,
                                               (long long)blockIdx.x * ElemCfg<N>::EPB, Gr);
}

template <int N, typename T, int RIEM, int MODE>
__global__ void __launch_bounds__(CurvedIfCfg<N>::THREADS)
curved_interface_kernel(const MeshDev m, const StageParams* __restrict__ sp, const T* __restrict__ U,
                        T* __restrict__ Fs, T* __restrict__ Fm, const T* __restrict__ Gr) {
  curved_interface_tile<N, T, RIEM, MODE>(m, sp, U, Fs, Fm, blockIdx.x, blockIdx.y, Gr);
}

template <int N, typename T>
__global__ void __launch_bounds__(ElemCfg<N>::THREADS)
curved_lift_kernel(const MeshDev m, const StageParams* __restrict__ sp, const T* __restrict__ U, T* __restrict__ Gr,
                   const T* __restrict__ Ls, const T* __restrict__ Lm) {
  curved_lift_block<N, T>(m, sp, U, Gr, Ls, Lm, (long long)blockIdx.x * ElemCfg<N>::EPB);
}

template <int N, typename T, int RIEM, int MODE, int PHYS>
cudaError_t launch_ce(const ElemArgs& a, cudaStream_t st) {
  using C = ElemCfg<N>;
  const long long blocks = (a.m.E + C::EPB - 1) / C::EPB;
  if (blocks <= 0) return cudaSuccess;
  curved_element_kernel<N, T, RIEM, MODE, PHYS><<<(unsigned)blocks, C::THREADS, C::template smem_bytes<T>(), st>>>(
      a.m, a.sp, (const T*)a.U, (T*)a.out, (T*)a.G, (const T*)a.Fs, (const T*)a.Fm, (T)a.rkA, (T)a.rkB, (T)a.dt,
      (const T*)a.Gr);
  return cudaGetLastError();
}

template <int N, typename T, int RIEM, int MODE, int PHYS>
cudaError_t prepare_ce() {
  return cudaFuncSetAttribute(curved_element_kernel<N, T, RIEM, MODE, PHYS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)ElemCfg<N>::template smem_bytes<T>());
}

template <int N, typename T, int PHYS>
cudaError_t launch_ce_n(int riemann, int mode, const ElemArgs& a, cudaStream_t st) {
  if (riemann == 0) {
    if (mode == ELEM_RHS) return launch_ce<N, T, 0, ELEM_RHS, PHYS>(a, st);
    if (mode == ELEM_STAGE) return launch_ce<N, T, 0, ELEM_STAGE, PHYS>(a, st);
    return launch_ce<N, T, 0, ELEM_STAGE_FIRST, PHYS>(a, st);
  }
  if (mode == ELEM_RHS) return launch_ce<N, T, 1, ELEM_RHS, PHYS>(a, st);
  if (mode == ELEM_STAGE) return launch_ce<N, T, 1, ELEM_STAGE, PHYS>(a, st);
  return launch_ce<N, T, 1, ELEM_STAGE_FIRST, PHYS>(a, st);
}

template <int N, typename T, int PHYS>
cudaError_t prepare_ce_n() {
  cudaError_t r[6] = {prepare_ce<N, T, 0, ELEM_RHS, PHYS>(), prepare_ce<N, T, 0, ELEM_STAGE, PHYS>(),
                      prepare_ce<N, T, 0, ELEM_STAGE_FIRST, PHYS>(), prepare_ce<N, T, 1, ELEM_RHS, PHYS>(),
                      prepare_ce<N, T, 1, ELEM_STAGE, PHYS>(), prepare_ce<N, T, 1, ELEM_STAGE_FIRST, PHYS>()};
  for (cudaError_t e : r)
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

template <int N, typename T, int MODE>
cudaError_t launch_ci_n(int riemann, const MeshDev& m, const StageParams* sp, const void* U, void* Fs, void* Fm,
                        const void* Gr, cudaStream_t st) {
  using C = CurvedIfCfg<N>;
  dim3 grid((m.ny + C::TF - 1) / C::TF, m.nz);
  const size_t sm = C::template smem_bytes<T, MODE>();
  if (riemann)
    curved_interface_kernel<N, T, 1, MODE><<<grid, C::THREADS, sm, st>>>(m, sp, (const T*)U, (T*)Fs, (T*)Fm, (const T*)Gr);
  else
    curved_interface_kernel<N, T, 0, MODE><<<grid, C::THREADS, sm, st>>>(m, sp, (const T*)U, (T*)Fs, (T*)Fm, (const T*)Gr);
  return cudaGetLastError();
}

template <int N, typename T, int MODE>
cudaError_t prepare_ci_n() {
  const int sm = (int)CurvedIfCfg<N>::template smem_bytes<T, MODE>();
  cudaError_t e = cudaFuncSetAttribute(curved_interface_kernel<N, T, 0, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(curved_interface_kernel<N, T, 1, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

template <int N, typename T>
cudaError_t launch_cl_n(const MeshDev& m, const StageParams* sp, const void* U, void* Gr, const void* Ls,
                        const void* Lm, cudaStream_t st) {
  using C = ElemCfg<N>;
  const long long blocks = (m.E + C::EPB - 1) / C::EPB;
  if (blocks <= 0) return cudaSuccess;
  curved_lift_kernel<N, T><<<(unsigned)blocks, C::THREADS, CurvedLiftCfg<N>::template smem_bytes<T>(), st>>>(
      m, sp, (const T*)U, (T*)Gr, (const T*)Ls, (const T*)Lm);
  return cudaGetLastError();
}

template <int N, typename T>
cudaError_t prepare_cl_n() {
  return cudaFuncSetAttribute(curved_lift_kernel<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)CurvedLiftCfg<N>::template smem_bytes<T>());
}

}  // namespace

#define SM_CURVED_SWITCH(call)              \
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

// Batched persistent kernels: one launch per kernel kind and RK stage advances every FP32
// solve of a degree-N group together.  Work items are (solve, CTA block) pairs numbered by
// per-solve prefix offsets; a CTA loops over items grid-stride, finds its solve by binary
// search in the offsets (held in shared memory) and runs the same per-block bodies as the
// single-solve kernels, so a solve's arithmetic does not depend on the other solves.
#include "sm_element.cuh"
#include "sm_iface.cuh"
#include "sm_mapper.cuh"

namespace {

__device__ __forceinline__ int find_solve(const int* s_off, int nsolve, int item) {
  int lo = 0, hi = nsolve - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (s_off[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(64) batch_stage_params_kernel(const BatchSolveDev* __restrict__ bs, int np, double ck,
                                                                int mode) {
  const BatchSolveDev& b = bs[blockIdx.x];
  stage_params_body(b.m, np, b.sp, b.t_d, 0.0, ck, b.dt, mode);
}

__global__ void batch_flip_kernel(BatchSolveDev* bs, int nsolve) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nsolve) bs[i].cur ^= 1;
}

template <int N, int RIEM, int MODE>
__global__ void __launch_bounds__(ElemCfg<N>::THREADS, ElemCfg<N>::MINB)
dg_element_batch_kernel(const BatchSolveDev* __restrict__ bs, const int* __restrict__ offs, int nsolve, int stage,
                        float rkA, float rkB) {
  __shared__ int s_off[SM_MAX_BATCH + 1];
  for (int i = threadIdx.x; i <= nsolve; i += blockDim.x) s_off[i] = offs[i];
  __syncthreads();
  const int total = s_off[nsolve];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int s = find_solve(s_off, nsolve, item);
    const BatchSolveDev& b = bs[s];
    const int c = b.cur ^ (stage & 1);
    element_block<N, float, RIEM, MODE>(b.m, b.sp, (const float*)b.U[c], (float*)b.U[1 - c], (float*)b.G,
                                        (const float*)b.Fs, (const float*)b.Fm, rkA, rkB, (float)b.dt,
                                        (long long)(item - s_off[s]) * ElemCfg<N>::EPB, nullptr, (float*)b.Ts,
                                        (float*)b.Tm);
    __syncthreads();
  }
}

// Interface tiles of every solve of the group: odd N takes the register-fused tile (TF 8 or
// 16) in persistent CTAs that prefetch the next tile; even N the staged tile.
template <int N, int TF> struct BatchIfCfg {
  static constexpr bool FUSED = N % 2 == 1;
  static constexpr int TFF = TF < 8 ? 8 : TF;
  static constexpr int THREADS = FUSED ? IfFusedCfg<(FUSED ? N : 1), TFF>::THREADS : IfCfg<N>::THREADS;
  static constexpr int MINB = FUSED ? IfFusedCfg<(FUSED ? N : 1), TFF>::MINB : IfCfg<N>::MINB;
  static constexpr size_t smem = FUSED ? IfFusedCfg<(FUSED ? N : 1), TFF>::smem_bytes : IfCfg<N>::template smem_bytes<float, TF>();
  static constexpr int TILE = FUSED ? TFF : TF;
};

template <int N, int RIEM, int TF>
__global__ void __launch_bounds__(BatchIfCfg<N, TF>::THREADS, BatchIfCfg<N, TF>::MINB)
sliding_interface_batch_kernel(const BatchSolveDev* __restrict__ bs, const int* __restrict__ offs, int nsolve, int stage) {
  using B = BatchIfCfg<N, TF>;
  constexpr int TL = B::TILE;
  __shared__ int s_off[SM_MAX_BATCH + 1];
  const int tid = threadIdx.x;
  for (int i = tid; i <= nsolve; i += blockDim.x) s_off[i] = offs[i];
  __syncthreads();
  const int total = s_off[nsolve];
  if constexpr (B::FUSED) {
    using C = IfFusedCfg<N, TL>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* smem = reinterpret_cast<float*>(smem_raw);   // table and trace buffers, mortar fluxes
    float* sF = smem + C::NTAB * C::TAB + C::NBUF * C::TBUF;
    // a work item's solve, its buffers at this stage and its tile coordinates
    auto locate = [&](int item, int* ty, int* tz) -> const BatchSolveDev& {
      const int s = find_solve(s_off, nsolve, item);
      const BatchSolveDev& b = bs[s];
      const int ntx = (b.m.ny + TL - 1) / TL;
      divmod_small(item - s_off[s], ntx, 1.0f / (float)ntx, tz, ty);
      return b;
    };
    fused_pipeline<N, TL>(
        blockIdx.x, gridDim.x, total, smem,
        [&](int item, float* tab, float* tr) {
          int ty, tz;
          const BatchSolveDev& b = locate(item, &ty, &tz);
          const int c = b.cur ^ (stage & 1);
          fused_tile_stage<N, TL>(b.m, b.sp, (const float*)b.U[c], (const float*)b.Ts, (const float*)b.Tm, ty, tz,
                                  tab, tr, tid);
        },
        [&](int item, const float* tab, const float* tr) {
          int ty, tz;
          const BatchSolveDev& b = locate(item, &ty, &tz);
          fused_tile_compute<N, RIEM, TL>(b.m, b.sp, (float*)b.Fs, (float*)b.Fm, ty, tz, tab, tr, sF, tid);
        });
  } else {
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
      const int s = find_solve(s_off, nsolve, item);
      const BatchSolveDev& b = bs[s];
      const int local = item - s_off[s];
      const int ntx = (b.m.ny + TL - 1) / TL;
      const int c = b.cur ^ (stage & 1);
      interface_tile<N, float, RIEM, TL>(b.m, b.sp, (const float*)b.U[c], (float*)b.Fs, (float*)b.Fm, local % ntx,
                                         local / ntx, nullptr, (const float*)b.Ts, (const float*)b.Tm);
      __syncthreads();
    }
  }
}

template <int N, int RIEM, int MODE>
cudaError_t launch_el(const BatchSolveDev* bs, const int* offs, int nsolve, int grid, int stage, double A, double B,
                      cudaStream_t st) {
  using C = ElemCfg<N>;
  dg_element_batch_kernel<N, RIEM, MODE><<<grid, C::THREADS, C::template smem_bytes<float>(), st>>>(
      bs, offs, nsolve, stage, (float)A, (float)B);
  return cudaGetLastError();
}

template <int N, int RIEM, int TF>
cudaError_t launch_if(const BatchSolveDev* bs, const int* offs, int nsolve, int grid, int stage, cudaStream_t st) {
  using C = BatchIfCfg<N, TF>;
  sliding_interface_batch_kernel<N, RIEM, TF><<<grid, C::THREADS, C::smem, st>>>(
      bs, offs, nsolve, stage);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_el_n(int riemann, int mode, const BatchSolveDev* bs, const int* offs, int nsolve, int grid, int stage,
                        double A, double B, cudaStream_t st) {
  if (riemann == 0)
    return mode == ELEM_STAGE_FIRST ? launch_el<N, 0, ELEM_STAGE_FIRST>(bs, offs, nsolve, grid, stage, A, B, st)
                                    : launch_el<N, 0, ELEM_STAGE>(bs, offs, nsolve, grid, stage, A, B, st);
  return mode == ELEM_STAGE_FIRST ? launch_el<N, 1, ELEM_STAGE_FIRST>(bs, offs, nsolve, grid, stage, A, B, st)
                                  : launch_el<N, 1, ELEM_STAGE>(bs, offs, nsolve, grid, stage, A, B, st);
}

template <int N, int RIEM>
cudaError_t launch_if_tf(int tf, const BatchSolveDev* bs, const int* offs, int nsolve, int grid, int stage,
                         cudaStream_t st) {
  if (tf == 4) return launch_if<N, RIEM, 4>(bs, offs, nsolve, grid, stage, st);
  if (tf == 16) return launch_if<N, RIEM, 16>(bs, offs, nsolve, grid, stage, st);
  return launch_if<N, RIEM, 8>(bs, offs, nsolve, grid, stage, st);
}

template <int N, int RIEM, int TF>
cudaError_t prep_if() {
  return cudaFuncSetAttribute(sliding_interface_batch_kernel<N, RIEM, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)BatchIfCfg<N, TF>::smem);
}

template <int N, int RIEM, int MODE>
cudaError_t prep_el() {
  cudaError_t e = cudaFuncSetAttribute(dg_element_batch_kernel<N, RIEM, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)ElemCfg<N>::template smem_bytes<float>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(dg_element_batch_kernel<N, RIEM, MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutDefault);
}

template <int N>
cudaError_t prep_n() {
  cudaError_t r[10] = {prep_if<N, 0, 4>(), prep_if<N, 0, 8>(), prep_if<N, 0, 16>(), prep_if<N, 1, 4>(),
                       prep_if<N, 1, 8>(), prep_if<N, 1, 16>(), prep_el<N, 0, ELEM_STAGE>(),
                       prep_el<N, 0, ELEM_STAGE_FIRST>(), prep_el<N, 1, ELEM_STAGE>(), prep_el<N, 1, ELEM_STAGE_FIRST>()};
  for (cudaError_t e : r)
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

}  // namespace

#define SM_BATCH_SWITCH(N, call)          \
  switch (N) {                            \
    case 1: return call(1);               \
    case 2: return call(2);               \
    case 3: return call(3);               \
    case 4: return call(4);               \
    case 5: return call(5);               \
    case 6: return call(6);               \
    case 7: return call(7);               \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_batch_stage_params(int N, const BatchSolveDev* d_bs, int nsolve, double ck, int mode, cudaStream_t st) {
  if (nsolve <= 0) return cudaSuccess;
  batch_stage_params_kernel<<<nsolve, 64, 0, st>>>(d_bs, N + 1, ck, mode);
  return cudaGetLastError();
}

cudaError_t launch_batch_flip(BatchSolveDev* d_bs, int nsolve, cudaStream_t st) {
  if (nsolve <= 0) return cudaSuccess;
  batch_flip_kernel<<<(nsolve + 127) / 128, 128, 0, st>>>(d_bs, nsolve);
  return cudaGetLastError();
}

cudaError_t launch_batch_interface(int N, int riemann, int tf, const BatchSolveDev* d_bs, const int* d_offs, int nsolve,
                                   int grid, int stage, cudaStream_t st) {
  if (nsolve <= 0 || grid <= 0) return cudaSuccess;
#define SM_IF_CALL(n) (riemann ? launch_if_tf<n, 1>(tf, d_bs, d_offs, nsolve, grid, stage, st) \
                               : launch_if_tf<n, 0>(tf, d_bs, d_offs, nsolve, grid, stage, st))
  SM_BATCH_SWITCH(N, SM_IF_CALL)
#undef SM_IF_CALL
}

cudaError_t launch_batch_element(int N, int riemann, int mode, const BatchSolveDev* d_bs, const int* d_offs, int nsolve,
                                 int grid, int stage, double rkA, double rkB, cudaStream_t st) {
  if (nsolve <= 0 || grid <= 0) return cudaSuccess;
#define SM_EL_CALL(n) launch_el_n<n>(riemann, mode, d_bs, d_offs, nsolve, grid, stage, rkA, rkB, st)
  SM_BATCH_SWITCH(N, SM_EL_CALL)
#undef SM_EL_CALL
}

cudaError_t prepare_batch(int N) {
#define SM_PREP_CALL(n) prep_n<n>()
  SM_BATCH_SWITCH(N, SM_PREP_CALL)
#undef SM_PREP_CALL
}

int batch_interface_tile(int N, int tf) { return (N % 2 == 1 && tf < 8) ? 8 : tf; }

int batch_elements_per_block(int N) {
  switch (N) {
    case 1: return ElemCfg<1>::EPB;
    case 2: return ElemCfg<2>::EPB;
    case 3: return ElemCfg<3>::EPB;
    case 4: return ElemCfg<4>::EPB;
    case 5: return ElemCfg<5>::EPB;
    case 6: return ElemCfg<6>::EPB;
    case 7: return ElemCfg<7>::EPB;
    default: return 1;
  }
}

cudaError_t upload_dhat_batch(const float* f, const double* d) { return upload_dhat_here(f, d); }

// Initial data and deterministic diagnostics (not on the per-stage path).
//   - init_state: the flow's state at every node at t = 0 (moving block displaced by delta0);
//   - totals: sum_e sum_ijk J w_i w_j w_k U (the conserved integrals of Sec. 3.1's weak form);
//   - face sums: sum over interface faces of w_p w_q F (discrete mortar conservation);
//   - gather traces: the interface node layers of a state in the face-flux layout.
// Reductions are two-pass in FP64 with a fixed order, so repeated calls agree bit for bit.
#include <algorithm>

#include "sm_launch.h"

namespace {

template <typename T>
__global__ void init_state_kernel(const MeshDev m, int np, T* U) {
  const long long nn = (long long)np * np * np;
  const long long total = m.E * nn;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
    const long long e = g / nn;
    const int nd = (int)(g - e * nn);
    const int i = nd % np, j = (nd / np) % np, k = nd / (np * np);
    ElemPos p = decode_elem(m, e);
    double X[3], u[5];
    node_position(m, p, i, j, k, __fma_rn(m.v, 0.0, m.delta0), X);
    flow_state(m, X[0], X[1], X[2], 0.0, 0, u);
    for (int v = 0; v < 5; ++v) U[(e * 5 + v) * nn + nd] = (T)u[v];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) totals_kernel(const MeshDev m, int np, const T* U, double* partial) {
  __shared__ double red[5][256];
  const long long nn = (long long)np * np * np;
  const long long total = m.E * nn;
  double acc[5] = {0, 0, 0, 0, 0};
  const double* w = m.basis->w;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
    const long long e = g / nn;
    const int nd = (int)(g - e * nn);
    const int i = nd % np, j = (nd / np) % np, k = nd / (np * np);
    const double J = m.geom ? (double)reinterpret_cast<const T*>(m.geo)[(e * 13 + 9) * nn + nd] : elem_jacobian(m, e >= m.Es);
    const double wq = J * w[i] * w[j] * w[k];
    for (int v = 0; v < 5; ++v) acc[v] += wq * (double)U[(e * 5 + v) * nn + nd];
  }
  for (int v = 0; v < 5; ++v) red[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int v = 0; v < 5; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 5) partial[blockIdx.x * 5 + threadIdx.x] = red[threadIdx.x][0];
}

template <typename T>
__global__ void __launch_bounds__(256) face_sums_kernel(const MeshDev m, int np, const T* F, double* partial) {
  __shared__ double red[5][256];
  const int n2 = np * np;
  const long long total = (long long)m.ny * m.nz * n2;
  double acc[5] = {0, 0, 0, 0, 0};
  const double* w = m.basis->w;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
    const long long f = g / n2;
    const int ab = (int)(g - f * n2);
    const double wq = w[ab % np] * w[ab / np];
    for (int v = 0; v < 5; ++v) acc[v] += wq * (double)F[(f * 5 + v) * n2 + ab];
  }
  for (int v = 0; v < 5; ++v) red[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int v = 0; v < 5; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 5) partial[blockIdx.x * 5 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void finish_sum_kernel(const double* partial, int nblk, double* out5) {
  if (threadIdx.x < 5) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[b * 5 + threadIdx.x];
    out5[threadIdx.x] = s;
  }
}

// Interface traces of U: static face (iy, iz) is the xi^3 = +1 layer of static element
// (nxs-1, iy, iz), moving face the xi^3 = -1 layer of moving element (0, iy, iz); output
// [iz][iy][var][(N+1)^2] per side.  ifc = 1, the second interface x = x0 = x2 of a periodic x
// direction: the xi^3 = -1 layer of static element (0, iy, iz) and the xi^3 = +1 layer of
// moving element (nxm-1, iy, iz), x-momentum negated (the mirrored problem).
template <typename T>
__global__ void gather_traces_kernel(const MeshDev m, int np, const T* __restrict__ U, T* __restrict__ Ts,
                                     T* __restrict__ Tm, const int ifc) {
  const long long np2 = (long long)np * np, nn = np2 * np;
  const long long per_side = (long long)m.ny * m.nz * 5 * np2;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < 2 * per_side;
       g += (long long)gridDim.x * blockDim.x) {
    const int side = g >= per_side;
    const long long w = g - side * per_side;
    const long long f = w / (5 * np2);
    const int r = (int)(w - f * 5 * np2);
    const int v = r / (int)np2, ab = r - v * (int)np2;
    const int iy = (int)(f % m.ny), iz = (int)(f / m.ny);
    const int ix = ifc == 0 ? (side ? 0 : m.nxs - 1) : (side ? m.nxm - 1 : 0);
    const bool upper = (side == 0) == (ifc == 0);     // the element's xi^3 = +1 layer
    const long long e = encode_elem(m, side, ix, iy, iz);
    const T val = U[(e * 5 + v) * nn + (upper ? np2 * (np - 1) : 0) + ab];
    // FP32 with an even row length: rows interleaved in pairs (trace_node)
    const int i = ab % np, q = ab / np;
    const int node = (sizeof(T) == 4 && (np & 1) == 0) ? (q >> 1) * 2 * np + 2 * i + (q & 1) : ab;
    (side ? Tm : Ts)[w - ab + node] = (ifc == 1 && v == 1) ? -val : val;
  }
}

// FP64 fused multiply-add throughput probe, a measurement aid for the roofline of the FP64
// path (not part of the method): every thread runs eight independent dependency chains
// x <- x a + b for iters rounds (2 flop per link) and stores their sum so that none is
// removed.  With a = 1 - 1e-7, b = 1e-7 the chains stay near 1.
__global__ void fp64_fma_probe_kernel(const int iters, const double a, const double b, double* __restrict__ out) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + 8 * k);
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

cudaError_t launch_fp64_fma_probe(int blocks, int threads, int iters, double* out, cudaStream_t st) {
  fp64_fma_probe_kernel<<<blocks, threads, 0, st>>>(iters, 1.0 - 1e-7, 1e-7, out);
  return cudaGetLastError();
}

cudaError_t launch_gather_traces(int N, int prec, const MeshDev& m, const void* U, void* Ts, void* Tm, cudaStream_t st,
                                 int ifc) {
  const int np = N + 1;
  const long long total = 2LL * m.ny * m.nz * 5 * np * np;
  const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
  if (prec == 0)
    gather_traces_kernel<double><<<grid, 256, 0, st>>>(m, np, (const double*)U, (double*)Ts, (double*)Tm, ifc);
  else gather_traces_kernel<float><<<grid, 256, 0, st>>>(m, np, (const float*)U, (float*)Ts, (float*)Tm, ifc);
  return cudaGetLastError();
}

cudaError_t launch_init_state(int N, int prec, const MeshDev& m, void* U, cudaStream_t st) {
  const int np = N + 1;
  const int blocks = 152 * 8;
  if (prec == 0) init_state_kernel<double><<<blocks, 256, 0, st>>>(m, np, (double*)U);
  else init_state_kernel<float><<<blocks, 256, 0, st>>>(m, np, (float*)U);
  return cudaGetLastError();
}

cudaError_t launch_totals(int N, int prec, const MeshDev& m, const void* U, double* partial, int nblk, double* out5,
                          cudaStream_t st) {
  const int np = N + 1;
  if (prec == 0) totals_kernel<double><<<nblk, 256, 0, st>>>(m, np, (const double*)U, partial);
  else totals_kernel<float><<<nblk, 256, 0, st>>>(m, np, (const float*)U, partial);
  finish_sum_kernel<<<1, 32, 0, st>>>(partial, nblk, out5);
  return cudaGetLastError();
}

cudaError_t launch_face_sums(int N, int prec, const MeshDev& m, const void* F, double* partial, int nblk,
                             double* out5, cudaStream_t st) {
  const int np = N + 1;
  if (prec == 0) face_sums_kernel<double><<<nblk, 256, 0, st>>>(m, np, (const double*)F, partial);
  else face_sums_kernel<float><<<nblk, 256, 0, st>>>(m, np, (const float*)F, partial);
  finish_sum_kernel<<<1, 32, 0, st>>>(partial, nblk, out5);
  return cudaGetLastError();
}

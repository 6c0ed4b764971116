// Split-form element kernel on curved elements: the volume integral of the split formulation
// with Pirozzoli's two-point flux (Sec. 3.1) through per-node metric terms, for the rotating
// geometries and the plane box through general metrics; faces, surface integral and RK update
// as in the curved weak-form kernel.
//
// Strong form with the contravariant two-point flux of direction xi^d between nodes a and l
// of a line (reading, the curvilinear form of Pirozzoli's products): with the averaged metric
// vector m = {{Ja^d}} and normal grid speed V = {{Ja^d . v^g}},
//   w = {{v}} . m - V,  F~#_rho = {{rho}} w,  F~#_rho v = F~#_rho {{v}} + {{p}} m,
//   F~#_rho e = F~#_rho {{H}} + {{p}} V,
// the node's volume term is sum_d sum_l Ds_il F~#^d(U_i, U_l), Ds = 2 D - M^-1 B (zero diagonal
// on LGL nodes; the strong form's boundary correction sits on it).  For equal nodes the flux is
// the contravariant ALE flux Ja^d . F(U) - (Ja^d . v^g) U.
//
// Frames as in the weak-form kernel: a rotor element works in its own frame (state turned by
// -phi on load, metric terms of t = 0, Ja^d . v^g time-independent), the residual is turned
// back before the update.  One thread per node stores the halved primitives (rho, v1, v2, v3,
// p, H) / 2 and, per direction, the halved (Ja^d, Ja^d . v^g) / 2 in shared memory, so that a
// mean is one addition; after a barrier every thread sums the two-point fluxes of the three
// lines through its node.
//
// Navier-Stokes (PHYS 1, the paper's production scheme: split form with BR1): the advective
// terms as above, the viscous terms in the weak form of the curved weak-form kernel (the
// contravariant viscous fluxes Ja^d . F^v of the lifted gradients, contracted with Dhat), and
// the face flux minus the BR1 mean of both sides' viscous fluxes, so that the own-flux
// correction in Ds is the advective flux only:
//   J dU/dt = -[ sum_d sum_l Ds_il F~#^d(U_i, U_l) ] + sum_d sum_l Dhat_il Ja^d . F^v(U_l, grad_l)
//             - (1 / w_0) ((F*_adv - {{F^v}}) . N sJ) at face nodes.
#pragma once

#include "sm_curved.cuh"

template <int N> struct CurvedSplitCfg {
  using C = ElemCfg<N>;
  static constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN, EPB = C::EPB, THREADS = C::THREADS;
  // resident CTAs per SM asked of the register allocator: FP32 at N = 7 two CTAs of 512
  // threads (64 registers), so that 32 warps hide the global-load latency instead of 16
#ifdef SM_CSPLIT_MINB_OVERRIDE
  template <typename T> __host__ __device__ static constexpr int minb() { return SM_CSPLIT_MINB_OVERRIDE; }
#else
  template <typename T> __host__ __device__ static constexpr int minb() { return sizeof(T) == 4 && N == 7 ? 2 : 1; }
#endif
  template <typename T, int PHYS = 0> static constexpr size_t smem_bytes() {
    // primitives, metric quadruples per direction, face fluxes, the Ds table (PHYS 1: the
    // contravariant viscous fluxes)
    return sizeof(T) * (size_t)(EPB * 6 * NN + EPB * 12 * NN + EPB * 30 * NP2 + NP * NP + (PHYS ? EPB * 15 * NN : 0));
  }
};

template <int N, typename T, int RIEM, int MODE, int PHYS = 0>
__device__ __forceinline__ void curved_split_block(const MeshDev& m, const StageParams* __restrict__ sp,
                                                   const T* __restrict__ U, T* __restrict__ out,
                                                   T* __restrict__ G, const T* __restrict__ Fs,
                                                   const T* __restrict__ Fm, const T rkA, const T rkB,
                                                   const T dt, const long long e0, const T* __restrict__ Gr = nullptr) {
  using C = CurvedSplitCfg<N>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN, EPB = C::EPB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sQ = reinterpret_cast<T*>(smem_raw);        // [EPB][6][NN] halved primitives
  T* sM = sQ + EPB * 6 * NN;                     // [EPB][3][4][NN] halved (Ja^d, Ja^d . v^g)
  T* sS = sM + EPB * 12 * NN;                    // [EPB][6][5][NP2] outward face fluxes
  T* sD = sS + EPB * 30 * NP2;                   // [NP][NP] Ds
  T* sW = sD + NP * NP;                          // PHYS 1: [EPB][3][5][NN] -Ja^d . F^v
  const T* c = Prec<T>::c(m);
  const T* geo = reinterpret_cast<const T*>(m.geo);
  const int tid = threadIdx.x;
  const int le = tid / NN, nd = tid - le * NN;
  const long long e = e0 + le;
  const bool active = e < m.E;
  const long long base = e * 5 * NN + nd;
  const int blk = active && e >= m.Es;
  T fc, fs;
  block_frame<T>(m, sp, blk, fc, fs);
  if (tid < NP * NP) sD[tid] = (T)m.basis->Dsplit[(tid / NP) * SM_MAXNP + tid % NP];

  T u[5], g[5];
  if (active) {
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = U[base + v * NN];
    if (MODE == ELEM_STAGE) {
#pragma unroll
      for (int v = 0; v < 5; ++v) g[v] = G[base + v * NN];
    }
    T ub[5] = {u[0], u[1], u[2], u[3], u[4]};
    rotate_state_z(ub, fc, -fs);
    const Prim<T> q = primitives(ub, c[MC_GAMMA]);
    T* Q = sQ + le * 6 * NN + nd;
    Q[0] = T(0.5) * ub[0];
    Q[NN] = T(0.5) * q.u[0];
    Q[2 * NN] = T(0.5) * q.u[1];
    Q[3 * NN] = T(0.5) * q.u[2];
    Q[4 * NN] = T(0.5) * q.p;
    Q[5 * NN] = T(0.5) * ((ub[4] + q.p) * q.ir);
    const T* ge = geo + e * 13 * NN + nd;
    const T vs = moving_block(m, blk) ? c[MC_VG] : T(0);
    T* M = sM + le * 12 * NN + nd;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int a = 0; a < 3; ++a) M[(4 * d + a) * NN] = T(0.5) * ge[(3 * d + a) * NN];
      M[(4 * d + 3) * NN] = T(0.5) * vs * ge[(10 + d) * NN];
    }
    if (PHYS) {
      // the viscous fluxes of the lifted gradients (turned into the element's frame) along
      // the axes, contracted with each direction's metric vector, negated
      T gn[15], fv[3][5];
#pragma unroll
      for (int kk = 0; kk < 15; ++kk) gn[kk] = Gr[(e * 15 + kk) * NN + nd];
      rotate_grad_z(gn, fc, -fs);
#pragma unroll
      for (int a = 0; a < 3; ++a) viscous_flux_axis(ub, gn, a, c, fv[a]);
      T* W = sW + le * 15 * NN + nd;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T J0 = ge[(3 * d) * NN], J1 = ge[(3 * d + 1) * NN], J2 = ge[(3 * d + 2) * NN];
#pragma unroll
        for (int v = 0; v < 5; ++v) W[(5 * d + v) * NN] = -(J0 * fv[0][v] + J1 * fv[1][v] + J2 * fv[2][v]);
      }
    }
  }

  curved_face_fluxes<N, T, RIEM, PHYS>(m, sp, U, Fs, Fm, Gr, e0, sS, tid);

  __syncthreads();
  if (PHYS) {
    contract_lines_inplace<N, T>(sW, tid);
    __syncthreads();
  }
  if (!active) return;
  const int i = nd % NP, j = (nd / NP) % NP, k = nd / NP2;
  const T* Qe = sQ + le * 6 * NN;
  const T* Me = sM + le * 12 * NN;
  T qa[6];
#pragma unroll
  for (int s2 = 0; s2 < 6; ++s2) qa[s2] = Qe[s2 * NN + nd];
  T acc[5] = {T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int row = d == 0 ? i : (d == 1 ? j : k);
    const int stride = d == 0 ? 1 : (d == 1 ? NP : NP2);
    const int lbase = nd - row * stride;              // the line's first node
    T ma[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) ma[a] = Me[(4 * d + a) * NN + nd];
#pragma unroll
    for (int l = 0; l < NP; ++l) {
      const int nl = lbase + l * stride;
      const T dil = sD[row * NP + l];
      const T rm = qa[0] + Qe[nl];
      const T u0 = qa[1] + Qe[NN + nl], u1 = qa[2] + Qe[2 * NN + nl], u2 = qa[3] + Qe[3 * NN + nl];
      const T pm = qa[4] + Qe[4 * NN + nl], hm = qa[5] + Qe[5 * NN + nl];
      const T m0 = ma[0] + Me[(4 * d) * NN + nl], m1 = ma[1] + Me[(4 * d + 1) * NN + nl];
      const T m2 = ma[2] + Me[(4 * d + 2) * NN + nl], vm = ma[3] + Me[(4 * d + 3) * NN + nl];
      const T fr = rm * (u0 * m0 + u1 * m1 + u2 * m2 - vm);
      acc[0] += dil * fr;
      acc[1] += dil * (fr * u0 + pm * m0);
      acc[2] += dil * (fr * u1 + pm * m1);
      acc[3] += dil * (fr * u2 + pm * m2);
      acc[4] += dil * (fr * hm + pm * vm);
    }
  }
  if (PHYS) {
    const T* W = sW + le * 15 * NN + nd;
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += W[v * NN] + W[(5 + v) * NN] + W[(10 + v) * NN];
  }
  curved_surface_update<N, T, MODE>(m, sS + le * 30 * NP2, acc, nd, e, base, u, g, fc, fs, out, G, rkA, rkB, dt);
}

namespace {

template <int N, typename T, int RIEM, int MODE, int PHYS>
__global__ void __launch_bounds__(ElemCfg<N>::THREADS, CurvedSplitCfg<N>::template minb<T>())
curved_split_kernel(const MeshDev m, const StageParams* __restrict__ sp, const T* __restrict__ U,
                    T* __restrict__ out, T* __restrict__ G, const T* __restrict__ Fs, const T* __restrict__ Fm,
                    const T rkA, const T rkB, const T dt, const T* __restrict__ Gr) {
  curved_split_block<N, T, RIEM, MODE, PHYS>(m, sp, U, out, G, Fs, Fm, rkA, rkB, dt,
                                             (long long)blockIdx.x * ElemCfg<N>::EPB, Gr);
}

template <int N, typename T, int RIEM, int MODE, int PHYS>
cudaError_t launch_cs(const ElemArgs& a, cudaStream_t st) {
  using C = CurvedSplitCfg<N>;
  const long long blocks = (a.m.E + C::EPB - 1) / C::EPB;
  if (blocks <= 0) return cudaSuccess;
  curved_split_kernel<N, T, RIEM, MODE, PHYS><<<(unsigned)blocks, C::THREADS, C::template smem_bytes<T, PHYS>(), st>>>(
      a.m, a.sp, (const T*)a.U, (T*)a.out, (T*)a.G, (const T*)a.Fs, (const T*)a.Fm, (T)a.rkA, (T)a.rkB, (T)a.dt,
      (const T*)a.Gr);
  return cudaGetLastError();
}

template <int N, typename T, int RIEM, int MODE, int PHYS>
cudaError_t prepare_cs() {
  return cudaFuncSetAttribute(curved_split_kernel<N, T, RIEM, MODE, PHYS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)CurvedSplitCfg<N>::template smem_bytes<T, PHYS>());
}

template <int N, typename T, int PHYS = 0>
cudaError_t launch_cs_n(int riemann, int mode, const ElemArgs& a, cudaStream_t st) {
  if (riemann == 0) {
    if (mode == ELEM_RHS) return launch_cs<N, T, 0, ELEM_RHS, PHYS>(a, st);
    if (mode == ELEM_STAGE) return launch_cs<N, T, 0, ELEM_STAGE, PHYS>(a, st);
    return launch_cs<N, T, 0, ELEM_STAGE_FIRST, PHYS>(a, st);
  }
  if (mode == ELEM_RHS) return launch_cs<N, T, 1, ELEM_RHS, PHYS>(a, st);
  if (mode == ELEM_STAGE) return launch_cs<N, T, 1, ELEM_STAGE, PHYS>(a, st);
  return launch_cs<N, T, 1, ELEM_STAGE_FIRST, PHYS>(a, st);
}

template <int N, typename T, int PHYS = 0>
cudaError_t prepare_cs_n() {
  cudaError_t r[6] = {prepare_cs<N, T, 0, ELEM_RHS, PHYS>(), prepare_cs<N, T, 0, ELEM_STAGE, PHYS>(),
                      prepare_cs<N, T, 0, ELEM_STAGE_FIRST, PHYS>(), prepare_cs<N, T, 1, ELEM_RHS, PHYS>(),
                      prepare_cs<N, T, 1, ELEM_STAGE, PHYS>(), prepare_cs<N, T, 1, ELEM_STAGE_FIRST, PHYS>()};
  for (cudaError_t e : r)
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

}  // namespace

#define SM_CURVED_SPLIT_SWITCH(CALL)   \
  switch (N) {                         \
    case 1: return CALL(1);            \
    case 2: return CALL(2);            \
    case 3: return CALL(3);            \
    case 4: return CALL(4);            \
    case 5: return CALL(5);            \
    case 6: return CALL(6);            \
    case 7: return CALL(7);            \
    default: return cudaErrorInvalidValue; \
  }

// Element kernel: weak-form DGSEM volume + surface integral and the low-storage RK update
// (Sec. 3.1, Eqs. transformed_equation and weak_formulation; LGL collocation):
//
//   J dU/dt = -[ sum_l Dhat_il F~1_ljk + sum_l Dhat_jl F~2_ilk + sum_l Dhat_kl F~3_ijl ]
//             - (1 / w_0) (F* . N sJ) at the face nodes of the element,
//
// with contravariant ALE fluxes F~d = |Ja^d| (F(U) - v^g U) . e_axis(d) (Sec. 2) and the
// face fluxes from the Riemann solver (conforming neighbours and weak Dirichlet faces,
// computed here in canonical orientation so both neighbours obtain identical values) or
// from the interface kernel (sliding faces).  One CTA holds EPB whole elements, one
// thread per volume node; neighbour face traces are read from the same state array (L2
// serves them: the DRAM traffic stays at the state's own reads and writes).
#pragma once

#include "sm_launch.h"

template <int N> struct ElemCfg {
  static constexpr int NP = N + 1, NP2 = NP * NP, NN = NP * NP * NP;
  static constexpr int EPB = N == 1 ? 32 : (N == 2 ? 8 : (N == 3 ? 4 : (N == 4 ? 2 : 1)));
  static constexpr int THREADS = EPB * NN;
  template <typename T> static constexpr size_t smem_bytes() {
    return sizeof(T) * (size_t)(EPB * 5 * NN + EPB * 15 * NN + EPB * 30 * NP2 + NP2 + 8);
  }
};

// Neighbour codes of the per-CTA face table: >= 0 element index, -1 weak Dirichlet face,
// -2 sliding interface face.
enum { NB_BOUNDARY = -1, NB_INTERFACE = -2 };

template <int N, typename T, int RIEM, int MODE>
__global__ void __launch_bounds__(ElemCfg<N>::THREADS)
dg_element_kernel(const MeshDev m, const StageParams* __restrict__ sp, const T* __restrict__ U,
                  T* __restrict__ out, T* __restrict__ G, const T* __restrict__ Fs,
                  const T* __restrict__ Fm, const T rkA, const T rkB, const T dt) {
  using C = ElemCfg<N>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN, EPB = C::EPB, THREADS = C::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sU = reinterpret_cast<T*>(smem_raw);        // [EPB][5][NN]
  T* sF = sU + EPB * 5 * NN;                     // [EPB][3][5][NN] contravariant fluxes
  T* sS = sF + EPB * 15 * NN;                    // [EPB][6][5][NP2] outward face fluxes
  T* sD = sS + EPB * 30 * NP2;                   // [NP][NP] Dhat
  __shared__ int4 s_pos[EPB];
  __shared__ int s_nb[EPB][6];
  __shared__ T s_t, s_delta;

  const T* c = Prec<T>::c(m);
  const int tid = threadIdx.x;
  const int le = tid / NN, nd = tid - le * NN;
  const long long e0 = (long long)blockIdx.x * EPB;
  const long long e = e0 + le;
  const bool active = e < m.E;
  const long long base = e * 5 * NN + nd;

  // ---- prologue: element positions, face-neighbour table, Dhat, state, early G fetch ----
  if (tid < NP2) sD[tid] = Prec<T>::dhat(m.basis)[(tid / NP) * SM_MAXNP + (tid % NP)];
  if (tid < 6 * EPB) {
    const int l2 = tid / 6, fc = tid - l2 * 6;
    if (e0 + l2 < m.E) {
      const ElemPos p = decode_elem(m, e0 + l2);
      if (fc == 0) s_pos[l2] = make_int4(p.blk, p.ix, p.iy, p.iz);
      long long nb = 0;
      const int kind = face_neighbor(m, p, fc >> 1, fc & 1, &nb);
      s_nb[l2][fc] = kind == 0 ? (int)nb : (kind == 1 ? NB_BOUNDARY : NB_INTERFACE);
    }
  }
  if (tid == THREADS - 1) { s_t = (T)sp->t; s_delta = (T)sp->delta; }
  T u[5], g[5];
  if (active) {
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = U[base + v * NN];
    if (MODE == ELEM_STAGE) {
#pragma unroll
      for (int v = 0; v < 5; ++v) g[v] = G[base + v * NN];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) sU[(le * 5 + v) * NN + nd] = u[v];
  }
  __syncthreads();
  const T gamma = c[MC_GAMMA];
  if (active) {
    const int blk = s_pos[le].x;
    const Prim<T> q = primitives(u, gamma);
    T f[5];
    T* Fe = sF + le * 15 * NN + nd;
    const T a0 = c[MC_METRIC + 3 * blk], a1 = c[MC_METRIC + 3 * blk + 1], a2 = c[MC_METRIC + 3 * blk + 2];
    axis_flux<T, 1>(u, q, blk ? c[MC_VG] : T(0), f);          // xi^1 -> y (grid velocity)
#pragma unroll
    for (int v = 0; v < 5; ++v) Fe[v * NN] = a0 * f[v];
    axis_flux<T, 2>(u, q, T(0), f);                             // xi^2 -> z
#pragma unroll
    for (int v = 0; v < 5; ++v) Fe[(5 + v) * NN] = a1 * f[v];
    axis_flux<T, 0>(u, q, T(0), f);                             // xi^3 -> x
#pragma unroll
    for (int v = 0; v < 5; ++v) Fe[(10 + v) * NN] = a2 * f[v];
  }

  // ---- face fluxes: one work item per (element, face, face node) ----
  for (int w = tid; w < EPB * 6 * NP2; w += THREADS) {
    const int l2 = w / (6 * NP2);
    const int r = w - l2 * 6 * NP2;
    const int fc = r / NP2, ab = r - fc * NP2;
    if (e0 + l2 >= m.E) continue;
    const int d = fc >> 1, side = fc & 1;
    const int a = ab % NP, b = ab / NP;
    const int vn = face_vol_node<NP>(d, side, a, b);
    const int nb = s_nb[l2][fc];
    const int4 q4 = s_pos[l2];
    T Fo[5];
    if (nb == NB_INTERFACE) {
      const T* src = (q4.x ? Fm : Fs) + ((long long)q4.w * m.ny + q4.z) * 5 * NP2 + ab;
#pragma unroll
      for (int v = 0; v < 5; ++v) Fo[v] = src[v * NP2];
    } else {
      T uin[5], uout[5], fs[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) uin[v] = sU[(l2 * 5 + v) * NN + vn];
      if (nb >= 0) {
        const T* Un = U + (long long)nb * 5 * NN + face_vol_node<NP>(d, 1 - side, a, b);
#pragma unroll
        for (int v = 0; v < 5; ++v) uout[v] = Un[v * NN];
      } else {
        // weak Dirichlet face (x = x0 or x = x2): node position at the stage time
        const T* xi = Prec<T>::x(m.basis);
        const int i = vn % NP, j = (vn / NP) % NP, k = vn / NP2;
        const T hx = c[MC_H + q4.x];
        T X[3];
        X[0] = c[MC_X + q4.x] + (T)q4.y * hx + (xi[k] + T(1)) * T(0.5) * hx;
        X[1] = c[MC_X + 2] + (T)q4.z * c[MC_H + 2] + (xi[i] + T(1)) * T(0.5) * c[MC_H + 2] + (q4.x ? s_delta : T(0));
        X[2] = c[MC_X + 3] + (T)q4.w * c[MC_H + 3] + (xi[j] + T(1)) * T(0.5) * c[MC_H + 3];
        boundary_state<T>(m, X, s_t, uout);
      }
      const T vgn = (d == 0 && q4.x) ? c[MC_VG] : T(0);
      const T* L = side ? uin : uout;
      const T* R = side ? uout : uin;
      if (d == 0) riemann_axis<T, 1, RIEM>(L, R, vgn, gamma, fs);
      else if (d == 1) riemann_axis<T, 2, RIEM>(L, R, vgn, gamma, fs);
      else riemann_axis<T, 0, RIEM>(L, R, vgn, gamma, fs);
      const T sJ = c[MC_METRIC + 3 * q4.x + d];
      const T sg = side ? sJ : -sJ;
#pragma unroll
      for (int v = 0; v < 5; ++v) Fo[v] = sg * fs[v];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) sS[((l2 * 6 + fc) * 5 + v) * NP2 + ab] = Fo[v];
  }
  __syncthreads();
  if (!active) return;

  // ---- volume integral (sum factorisation) + surface integral ----
  const int i = nd % NP, j = (nd / NP) % NP, k = nd / NP2;
  T acc[5] = {T(0), T(0), T(0), T(0), T(0)};
  const T* F1 = sF + le * 15 * NN;
  const T* F2 = F1 + 5 * NN;
  const T* F3 = F1 + 10 * NN;
#pragma unroll
  for (int l = 0; l < NP; ++l) {
    const T d1 = sD[i * NP + l], d2 = sD[j * NP + l], d3 = sD[k * NP + l];
    const int n1 = l + NP * (j + NP * k), n2 = i + NP * (l + NP * k), n3 = i + NP * (j + NP * l);
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += d1 * F1[v * NN + n1] + d2 * F2[v * NN + n2] + d3 * F3[v * NN + n3];
  }
  const T iw0 = c[MC_IW0];
  const T* Se = sS + le * 30 * NP2;
  if (i == 0 || i == N) {
    const T* s = Se + (i == 0 ? 0 : 1) * 5 * NP2 + j + NP * k;
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += iw0 * s[v * NP2];
  }
  if (j == 0 || j == N) {
    const T* s = Se + (j == 0 ? 2 : 3) * 5 * NP2 + i + NP * k;
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += iw0 * s[v * NP2];
  }
  if (k == 0 || k == N) {
    const T* s = Se + (k == 0 ? 4 : 5) * 5 * NP2 + i + NP * j;
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += iw0 * s[v * NP2];
  }
  const T mInvJ = c[MC_MINVJ + s_pos[le].x];
  if (MODE == ELEM_RHS) {
#pragma unroll
    for (int v = 0; v < 5; ++v) out[base + v * NN] = acc[v] * mInvJ;
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const T ut = acc[v] * mInvJ;
      const T gn = (MODE == ELEM_STAGE_FIRST) ? dt * ut : rkA * g[v] + dt * ut;
      G[base + v * NN] = gn;
      out[base + v * NN] = u[v] + rkB * gn;
    }
  }
}

template <int N, typename T, int RIEM, int MODE>
static cudaError_t launch_elem_t(const ElemArgs& a, cudaStream_t st) {
  using C = ElemCfg<N>;
  const size_t smem = C::template smem_bytes<T>();
  const long long blocks = (a.m.E + C::EPB - 1) / C::EPB;
  if (blocks <= 0) return cudaSuccess;
  dg_element_kernel<N, T, RIEM, MODE><<<(unsigned)blocks, C::THREADS, smem, st>>>(
      a.m, a.sp, (const T*)a.U, (T*)a.out, (T*)a.G, (const T*)a.Fs, (const T*)a.Fm, (T)a.rkA, (T)a.rkB, (T)a.dt);
  return cudaGetLastError();
}

template <int N, typename T, int RIEM, int MODE>
static cudaError_t prepare_elem_t() {
  using C = ElemCfg<N>;
  cudaError_t e = cudaFuncSetAttribute(dg_element_kernel<N, T, RIEM, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::template smem_bytes<T>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(dg_element_kernel<N, T, RIEM, MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

template <int N, typename T>
static cudaError_t launch_elem_n(int riemann, int mode, const ElemArgs& a, cudaStream_t st) {
  if (riemann == 0) {
    if (mode == ELEM_RHS) return launch_elem_t<N, T, 0, ELEM_RHS>(a, st);
    if (mode == ELEM_STAGE) return launch_elem_t<N, T, 0, ELEM_STAGE>(a, st);
    return launch_elem_t<N, T, 0, ELEM_STAGE_FIRST>(a, st);
  }
  if (mode == ELEM_RHS) return launch_elem_t<N, T, 1, ELEM_RHS>(a, st);
  if (mode == ELEM_STAGE) return launch_elem_t<N, T, 1, ELEM_STAGE>(a, st);
  return launch_elem_t<N, T, 1, ELEM_STAGE_FIRST>(a, st);
}

template <int N, typename T>
static cudaError_t prepare_elem_n() {
  cudaError_t e = cudaSuccess, r;
  if ((r = prepare_elem_t<N, T, 0, ELEM_RHS>()) != cudaSuccess) e = r;
  if ((r = prepare_elem_t<N, T, 0, ELEM_STAGE>()) != cudaSuccess) e = r;
  if ((r = prepare_elem_t<N, T, 0, ELEM_STAGE_FIRST>()) != cudaSuccess) e = r;
  if ((r = prepare_elem_t<N, T, 1, ELEM_RHS>()) != cudaSuccess) e = r;
  if ((r = prepare_elem_t<N, T, 1, ELEM_STAGE>()) != cudaSuccess) e = r;
  if ((r = prepare_elem_t<N, T, 1, ELEM_STAGE_FIRST>()) != cudaSuccess) e = r;
  return e;
}

#define SM_ELEM_DISPATCH(T, N, riemann, mode, a, st)            \
  switch (N) {                                                  \
    case 1: return launch_elem_n<1, T>(riemann, mode, a, st);   \
    case 2: return launch_elem_n<2, T>(riemann, mode, a, st);   \
    case 3: return launch_elem_n<3, T>(riemann, mode, a, st);   \
    case 4: return launch_elem_n<4, T>(riemann, mode, a, st);   \
    case 5: return launch_elem_n<5, T>(riemann, mode, a, st);   \
    case 6: return launch_elem_n<6, T>(riemann, mode, a, st);   \
    case 7: return launch_elem_n<7, T>(riemann, mode, a, st);   \
    default: return cudaErrorInvalidValue;                      \
  }

#define SM_ELEM_PREPARE(T, N)                   \
  switch (N) {                                  \
    case 1: return prepare_elem_n<1, T>();      \
    case 2: return prepare_elem_n<2, T>();      \
    case 3: return prepare_elem_n<3, T>();      \
    case 4: return prepare_elem_n<4, T>();      \
    case 5: return prepare_elem_n<5, T>();      \
    case 6: return prepare_elem_n<6, T>();      \
    case 7: return prepare_elem_n<7, T>();      \
    default: return cudaErrorInvalidValue;      \
  }

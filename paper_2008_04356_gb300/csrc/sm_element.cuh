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
  // resident CTAs per SM asked of the register allocator in FP32 mode (about 48 registers)
#ifdef SM_ELEM_MINB_OVERRIDE
  static constexpr int MINB = SM_ELEM_MINB_OVERRIDE;
#else
  static constexpr int MINB = N == 1 ? 4 : (N == 6 ? 4 : (N == 7 ? 2 : (N == 2 || N == 3 || N == 4 ? 5 : 6)));
#endif
  template <typename T> static constexpr size_t smem_bytes() {
    return sizeof(T) * (size_t)(EPB * 15 * NN + EPB * 30 * NP2);
  }
};

// Neighbour codes of the per-CTA face table: >= 0 element index, -1 weak Dirichlet face,
// -2 face of the sliding interface x = x1, -3 face of the sliding interface x = x0 = x2.
enum { NB_BOUNDARY = -1, NB_INTERFACE = -2, NB_INTERFACE2 = -3 };

// Contraction line of NP values starting at p (shared memory), read with vector loads when
// the line length allows aligned pairs or quadruples.
template <typename T, int NP>
__device__ __forceinline__ void load_line(const T* p, T (&r)[NP]) {
  if constexpr (sizeof(T) == 4 && NP % 4 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int h = 0; h < NP / 4; ++h) {
      const float4 x = q[h];
      r[4 * h] = x.x; r[4 * h + 1] = x.y; r[4 * h + 2] = x.z; r[4 * h + 3] = x.w;
    }
  } else if constexpr (sizeof(T) == 4 && NP % 2 == 0) {
    const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
    for (int h = 0; h < NP / 2; ++h) {
      const float2 x = q[h];
      r[2 * h] = x.x; r[2 * h + 1] = x.y;
    }
  } else if constexpr (sizeof(T) == 8 && NP % 2 == 0) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int h = 0; h < NP / 2; ++h) {
      const double2 x = q[h];
      r[2 * h] = x.x; r[2 * h + 1] = x.y;
    }
  } else {
#pragma unroll
    for (int l = 0; l < NP; ++l) r[l] = p[l];
  }
}

// Stores a line with the vector widths of load_line (scalar stores at a line stride of NP
// words would hit each bank twice per warp).
template <typename T, int NP>
__device__ __forceinline__ void store_line(T* p, const T (&r)[NP]) {
  if constexpr (sizeof(T) == 4 && NP % 4 == 0) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int h = 0; h < NP / 4; ++h) q[h] = make_float4(r[4 * h], r[4 * h + 1], r[4 * h + 2], r[4 * h + 3]);
  } else if constexpr (sizeof(T) == 4 && NP % 2 == 0) {
    float2* q = reinterpret_cast<float2*>(p);
#pragma unroll
    for (int h = 0; h < NP / 2; ++h) q[h] = make_float2(r[2 * h], r[2 * h + 1]);
  } else if constexpr (sizeof(T) == 8 && NP % 2 == 0) {
    double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
    for (int h = 0; h < NP / 2; ++h) q[h] = make_double2(r[2 * h], r[2 * h + 1]);
  } else {
#pragma unroll
    for (int l = 0; l < NP; ++l) p[l] = r[l];
  }
}

// Weak-form derivative matrices Dhat for N = 1..7 in constant memory, [N-1][i*8 + l]; the
// line contractions below index them with compile-time constants, so every Dhat entry is
// an operand of the multiply-add itself.  Each translation unit that instantiates the
// element kernels has its own copy, filled once per device through upload_dhat_here().
static __constant__ float c_dhat_f[7][SM_MAXNP * SM_MAXNP];
static __constant__ double c_dhat_d[7][SM_MAXNP * SM_MAXNP];
// the FP32 entries duplicated into float pairs (operands of the paired line contractions)
static __constant__ float2 c_dhat_f2[7][SM_MAXNP * SM_MAXNP];

static inline cudaError_t upload_dhat_here(const float* f, const double* d) {
  cudaError_t e = cudaMemcpyToSymbol(c_dhat_f, f, sizeof(float) * 7 * SM_MAXNP * SM_MAXNP);
  if (e != cudaSuccess) return e;
  float2 f2[7 * SM_MAXNP * SM_MAXNP];
  for (int r = 0; r < 7 * SM_MAXNP * SM_MAXNP; ++r) f2[r] = make_float2(f[r], f[r]);
  e = cudaMemcpyToSymbol(c_dhat_f2, f2, sizeof(f2));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_dhat_d, d, sizeof(double) * 7 * SM_MAXNP * SM_MAXNP);
}

template <typename T> __device__ __forceinline__ T dhat_c(int n, int idx);
template <> __device__ __forceinline__ float dhat_c<float>(int n, int idx) { return c_dhat_f[n - 1][idx]; }
template <> __device__ __forceinline__ double dhat_c<double>(int n, int idx) { return c_dhat_d[n - 1][idx]; }

// Every contraction line (direction, variable, line) of the CTA's EPB elements once: read
// its NP values, write sum_l Dhat_al value_l back in place (Dhat as constant-memory operands).
// The three flux arrays of an element are in node order [v][k][j][i]: xi^1 lines are
// contiguous (vector accesses), xi^2 and xi^3 lines have strides NP and NP^2 and are
// numbered so that consecutive lanes take consecutive words (no bank conflicts).
template <int N, typename T, int EPB = ElemCfg<N>::EPB, int THREADS = ElemCfg<N>::THREADS>
__device__ __forceinline__ void contract_lines_inplace(T* sF, int tid) {
  using C = ElemCfg<N>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN;
  for (int w = tid; w < EPB * 5 * NP2; w += THREADS) {
    const int l2 = w / (5 * NP2);
    const int rr = w - l2 * 5 * NP2;
    T* line = sF + l2 * 15 * NN + (rr / NP2) * NN + (rr % NP2) * NP;
    T rv[NP], ov[NP];
    load_line<T, NP>(line, rv);
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      T s = T(0);
#pragma unroll
      for (int l = 0; l < NP; ++l) s += dhat_c<T>(N, a * SM_MAXNP + l) * rv[l];
      ov[a] = s;
    }
    store_line<T, NP>(line, ov);
  }
  if constexpr (sizeof(T) == 4 && NP == 6) {
    // FP32, N = 5: the xi^2 and xi^3 lines of nodes i and i + 1 (i even) are adjacent in
    // memory, so a thread takes both as float pairs (one 8-byte access per node) and
    // contracts them with packed multiply-adds (the same per-line operations in order).
    // Measured: 2.520 -> 2.478 ms per element launch at N = 5; at N = 7 the same form made
    // the curved lifting kernel (three contractions per launch) 1.8x slower, so other
    // degrees keep the one-line form.
#pragma unroll
    for (int d = 1; d < 3; ++d) {
      constexpr int NPH = NP2 / 2;
      const int stride2 = d == 1 ? NP / 2 : NP2 / 2;
      for (int w = tid; w < EPB * 5 * NPH; w += THREADS) {
        const int l2 = w / (5 * NPH);
        const int rr = w - l2 * 5 * NPH;
        const int v = rr / NPH, q = 2 * (rr - v * NPH);
        // xi^2 lines (i, k), (i+1, k): base i + NP^2 k; xi^3 lines (i, j), (i+1, j): base i + NP j
        const int base = d == 1 ? (q % NP) + NP2 * (q / NP) : q;
        float2* line = reinterpret_cast<float2*>(sF + l2 * 15 * NN + (5 * d + v) * NN + base);
        float2 rv[NP];
#pragma unroll
        for (int l = 0; l < NP; ++l) rv[l] = line[l * stride2];
#pragma unroll
        for (int a = 0; a < NP; ++a) {
          float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
          for (int l = 0; l < NP; ++l) s2 = __ffma2_rn(c_dhat_f2[N - 1][a * SM_MAXNP + l], rv[l], s2);
          line[a * stride2] = s2;
        }
      }
    }
    return;
  }
#pragma unroll
  for (int d = 1; d < 3; ++d) {
    const int stride = d == 1 ? NP : NP2;
    for (int w = tid; w < EPB * 5 * NP2; w += THREADS) {
      const int l2 = w / (5 * NP2);
      const int rr = w - l2 * 5 * NP2;
      const int v = rr / NP2, q = rr - v * NP2;
      // xi^2 line (i, k): base i + NP^2 k; xi^3 line (i, j): base i + NP j
      const int base = d == 1 ? (q % NP) + NP2 * (q / NP) : q;
      T* line = sF + l2 * 15 * NN + (5 * d + v) * NN + base;
      T rv[NP];
#pragma unroll
      for (int l = 0; l < NP; ++l) rv[l] = line[l * stride];
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        T s = T(0);
#pragma unroll
        for (int l = 0; l < NP; ++l) s += dhat_c<T>(N, a * SM_MAXNP + l) * rv[l];
        line[a * stride] = s;
      }
    }
  }
}

// Exterior state of a weak Dirichlet face (x = x0 or x = x2) at face node vn of element e2:
// the boundary flow at the node's position at the stage time (the moving block shifted by
// the displacement).  pos_ix / pos_f: the element's x index and iz * ny + iy.
template <int N, typename T>
__device__ __forceinline__ void dirichlet_exterior(const MeshDev& m, const StageParams* __restrict__ sp,
                                                   const int blk2, const int pos_ix, const int pos_f, const int vn,
                                                   T (&uout)[5]) {
  constexpr int NP = N + 1, NP2 = NP * NP;
  const T* c = Prec<T>::c(m);
  const int iy = pos_f % m.ny, iz = pos_f / m.ny;
  const T* xi = Prec<T>::x(m.basis);
  const int i = vn % NP, j = (vn / NP) % NP, k = vn / NP2;
  const T hx = c[MC_H + blk2];
  T X[3];
  X[0] = c[MC_X + blk2] + (T)pos_ix * hx + (xi[k] + T(1)) * T(0.5) * hx;
  X[1] = c[MC_X + 2] + (T)iy * c[MC_H + 2] + (xi[i] + T(1)) * T(0.5) * c[MC_H + 2] + (blk2 ? (T)sp->delta : T(0));
  X[2] = c[MC_X + 3] + (T)iz * c[MC_H + 3] + (xi[j] + T(1)) * T(0.5) * c[MC_H + 3];
  boundary_state<T>(m, X, (T)sp->t, uout);
}

// Face fluxes of the CTA's EPB elements (elements e0 ..), one work item per (element, face,
// face node), into sS[EPB][6][5][NP^2] as outward fluxes times the surface element: conforming
// and weak Dirichlet faces by the Riemann solver in canonical orientation (left = minus-side
// element, normal +axis), sliding faces copied from the interface kernel's face fluxes.
// Reads global memory only, so it runs before the CTA's first barrier.
template <int N, typename T, int RIEM, int PHYS>
__device__ __forceinline__ void element_face_fluxes(const MeshDev& m, const StageParams* __restrict__ sp,
                                                    const T* __restrict__ U, const T* __restrict__ Fs,
                                                    const T* __restrict__ Fm, const T* __restrict__ Gr,
                                                    const long long e0, T* sS, const int tid) {
  using C = ElemCfg<N>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN, EPB = C::EPB, THREADS = C::THREADS;
  const T* c = Prec<T>::c(m);
  const T gamma = c[MC_GAMMA];
  for (int w = tid; w < EPB * 6 * NP2; w += THREADS) {
    const int l2 = w / (6 * NP2);
    const int r = w - l2 * 6 * NP2;
    const int fc = r / NP2, ab = r - fc * NP2;
    const long long e2 = e0 + l2;
    if (e2 >= m.E) continue;
    const int blk2 = e2 >= m.Es;
    const int d = fc >> 1, side = fc & 1;
    const int a = ab % NP, b = ab / NP;
    // strides of the face-normal index and of the two in-face indices (a, b)
    const int sn = d == 0 ? 1 : (d == 1 ? NP : NP2);
    const int sab = d == 0 ? NP * ab : (d == 1 ? a + NP2 * b : ab);
    const int vn = sab + (side ? N : 0) * sn;
    // neighbour code and packed position: topology table, or derived from the index
    int nb, pos_ix = 0, pos_f = 0;
    const int* tp = m.topo ? reinterpret_cast<const int*>(m.topo) + 8 * e2 : nullptr;
    if (tp) {
      nb = tp[fc];
    } else {
      const ElemPos p = decode_elem(m, e2);
      long long q = 0;
      const int kind = face_neighbor(m, p, d, side, &q);
      nb = kind == 0 ? (int)q : (kind == 1 ? NB_BOUNDARY : (kind == 2 ? NB_INTERFACE : NB_INTERFACE2));
      pos_ix = p.ix;
      pos_f = p.iz * m.ny + p.iy;
    }
    T Fo[5];
    if (nb == NB_INTERFACE) {
      const int fi = tp ? tp[7] : pos_f;
      const T* src = (blk2 ? Fm : Fs) + (long long)fi * 5 * NP2 + ab;
#pragma unroll
      for (int v = 0; v < 5; ++v) Fo[v] = src[v * NP2];
    } else if (nb == NB_INTERFACE2) {
      // second interface: fluxes of the x-mirrored problem, mirrored back
      const int fi = tp ? tp[7] : pos_f;
      const T* src = reinterpret_cast<const T*>(blk2 ? m.Fm2 : m.Fs2) + (long long)fi * 5 * NP2 + ab;
#pragma unroll
      for (int v = 0; v < 5; ++v) Fo[v] = src[v * NP2];
      Fo[1] = -Fo[1];
    } else {
      T uin[5], uout[5];
      const T* Ui = U + e2 * 5 * NN + vn;
#pragma unroll
      for (int v = 0; v < 5; ++v) uin[v] = Ui[v * NN];
      if (nb >= 0) {
        const T* Un = U + (long long)nb * 5 * NN + sab + (side ? 0 : N) * sn;
#pragma unroll
        for (int v = 0; v < 5; ++v) uout[v] = Un[v * NN];
      } else {
        // weak Dirichlet face (x = x0 or x = x2): node position at the stage time
        if (tp) { pos_ix = tp[6] >> 1; pos_f = tp[7]; }
        dirichlet_exterior<N, T>(m, sp, blk2, pos_ix, pos_f, vn, uout);
      }
      const int ax = d == 0 ? 1 : (d == 1 ? 2 : 0);
      if constexpr (RIEM == 0 && PHYS == 0) {
        // Rusanov along the outward normal: exactly antisymmetric between the neighbours
        T fo[5];
        const T sgn = side ? T(1) : T(-1);
        const T vgn = (d == 0 && blk2) ? sgn * c[MC_VG] : T(0);
        rusanov_outward<T>(uin, uout, ax, sgn, vgn, gamma, fo);
        const T sJ = c[MC_METRIC + 3 * blk2 + d];
#pragma unroll
        for (int v = 0; v < 5; ++v) sS[((l2 * 6 + fc) * 5 + v) * NP2 + ab] = sJ * fo[v];
        continue;
      }
      // canonical orientation: left = minus-side element, normal +axis
      T L[5], R[5], fl[5], fs[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        L[v] = side ? uin[v] : uout[v];
        R[v] = side ? uout[v] : uin[v];
      }
      T Lr[5], Rr[5];
      rotate_to_x(L, ax, Lr);
      rotate_to_x(R, ax, Rr);
      const T vgn = (d == 0 && blk2) ? c[MC_VG] : T(0);
      riemann_axis<T, 0, RIEM>(Lr, Rr, vgn, gamma, fl);
      rotate_from_x(fl, ax, fs);
      if (PHYS) {
        // BR1 viscous face flux: mean of both sides' viscous fluxes along the normal; a
        // weak Dirichlet face pairs the exterior state with the interior gradients
        T gi[15], go[15], fvi[5], fvo[5];
        const T* gp = Gr + e2 * 15 * NN + vn;
        const T* gq = nb >= 0 ? Gr + (long long)nb * 15 * NN + sab + (side ? 0 : N) * sn : gp;
#pragma unroll
        for (int kk = 0; kk < 15; ++kk) { gi[kk] = gp[kk * NN]; go[kk] = gq[kk * NN]; }
        viscous_flux_axis(uin, gi, ax, c, fvi);
        viscous_flux_axis(uout, go, ax, c, fvo);
#pragma unroll
        for (int v = 0; v < 5; ++v) fs[v] -= T(0.5) * (fvi[v] + fvo[v]);
      }
      const T sJ = c[MC_METRIC + 3 * blk2 + d];
      const T sg = side ? sJ : -sJ;
#pragma unroll
      for (int v = 0; v < 5; ++v) Fo[v] = sg * fs[v];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) sS[((l2 * 6 + fc) * 5 + v) * NP2 + ab] = Fo[v];
  }
}

// Surface integral at the element's face nodes, the 1/J scaling and (stage modes) the
// low-storage RK update of node nd of element e, given the node's volume term acc:
//   dU/dt = -(1/J) [ acc + (1/w_0) (outward face flux) ],
//   G = A_k G + dt dU/dt,  U = U + B_k G  (ELEM_STAGE_FIRST: A_k G = 0),
// and the interface node layers of the updated state for the next stage's interface kernel.
template <int N, typename T, int MODE>
__device__ __forceinline__ void element_surface_update(const MeshDev& m, const T* Se, T (&acc)[5], const int nd,
                                                       const long long e, const long long base, const T (&u)[5],
                                                       const T (&g)[5], T* __restrict__ out, T* __restrict__ G,
                                                       const T rkA, const T rkB, const T dt, T* __restrict__ Ts,
                                                       T* __restrict__ Tm) {
  using C = ElemCfg<N>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN;
  const T* c = Prec<T>::c(m);
  const int i = nd % NP, j = (nd / NP) % NP, k = nd / NP2;
  const T iw0 = c[MC_IW0];
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
  const T mInvJ = c[MC_MINVJ + (e >= m.Es)];
  if (MODE == ELEM_RHS) {
#pragma unroll
    for (int v = 0; v < 5; ++v) out[base + v * NN] = acc[v] * mInvJ;
  } else {
    T un[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const T ut = acc[v] * mInvJ;
      const T gn = (MODE == ELEM_STAGE_FIRST) ? dt * ut : rkA * g[v] + dt * ut;
      G[base + v * NN] = gn;
      un[v] = u[v] + rkB * gn;
      out[base + v * NN] = un[v];
    }
    // the interface node layers of the updated state, for the next stage's interface kernel
    const int blk = e >= m.Es;
    if (Ts && k == (blk ? 0 : N)) {
      int ix, f;
      if (m.topo) {
        const int* tp = reinterpret_cast<const int*>(m.topo) + 8 * e;
        ix = tp[6] >> 1;
        f = tp[7];
      } else {
        const ElemPos p = decode_elem(m, e);
        ix = p.ix;
        f = p.iz * m.ny + p.iy;
      }
      if (ix == (blk ? 0 : m.nxs - 1)) {
        T* dst = (blk ? Tm : Ts) + (long long)f * 5 * NP2 + trace_node<T, NP>(i, j);
#pragma unroll
        for (int v = 0; v < 5; ++v) dst[v * NP2] = un[v];
      }
    }
    // the second interface (periodic x): the opposite node layers, x-momentum mirrored
    if (m.Ts2 && k == (blk ? N : 0)) {
      int ix, f;
      if (m.topo) {
        const int* tp = reinterpret_cast<const int*>(m.topo) + 8 * e;
        ix = tp[6] >> 1;
        f = tp[7];
      } else {
        const ElemPos p = decode_elem(m, e);
        ix = p.ix;
        f = p.iz * m.ny + p.iy;
      }
      if (ix == (blk ? m.nxm - 1 : 0)) {
        T* dst = reinterpret_cast<T*>(blk ? m.Tm2 : m.Ts2) + (long long)f * 5 * NP2 + trace_node<T, NP>(i, j);
#pragma unroll
        for (int v = 0; v < 5; ++v) dst[v * NP2] = v == 1 ? -un[v] : un[v];
      }
    }
  }
}

// The work of one CTA: elements e0 .. e0+EPB-1 of one solve.  Shared by the single-solve
// kernel below and the batched persistent kernel.
//
// One barrier per element: before it, every thread computes its node's contravariant
// fluxes into shared memory and one face-node Riemann flux (own and neighbour traces both
// read from the state in global memory, the neighbour codes from the topology table), so
// no thread needs another thread's result until the volume/surface phase after it.
// PHYS 1 (Navier-Stokes) adds the viscous fluxes of the BR1-lifted gradients Gr
// ([E][15][NN], component 5 d + c = d(primitive c)/dx_d): F^c - F^v in the volume and the
// mean of both sides' viscous fluxes on conforming and boundary faces (Sec. 2, 3.1).
template <int N, typename T, int RIEM, int MODE, int PHYS = 0>
__device__ __forceinline__ void element_block(const MeshDev& m, const StageParams* __restrict__ sp,
                                              const T* __restrict__ U, T* __restrict__ out, T* __restrict__ G,
                                              const T* __restrict__ Fs, const T* __restrict__ Fm, const T rkA,
                                              const T rkB, const T dt, const long long e0,
                                              const T* __restrict__ Gr = nullptr, T* __restrict__ Ts = nullptr,
                                              T* __restrict__ Tm = nullptr) {
  using C = ElemCfg<N>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN, EPB = C::EPB, THREADS = C::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // physical fluxes along the axes of xi^1, xi^2, xi^3 (the contravariant fluxes without
  // their constant metric factors), each in node order [v][k][j][i]
  T* sF = reinterpret_cast<T*>(smem_raw);        // [EPB][3][5][NN]
  T* sS = sF + EPB * 15 * NN;                    // [EPB][6][5][NP2] outward face fluxes

  const T* c = Prec<T>::c(m);
  const int tid = threadIdx.x;
  const int le = tid / NN, nd = tid - le * NN;
  const long long e = e0 + le;
  const bool active = e < m.E;
  const long long base = e * 5 * NN + nd;
  const T gamma = c[MC_GAMMA];

  T u[5], g[5];
  if (active) {
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = U[base + v * NN];
    if (MODE == ELEM_STAGE) {
#pragma unroll
      for (int v = 0; v < 5; ++v) g[v] = G[base + v * NN];
    }
    const int blk = e >= m.Es;
    const Prim<T> q = primitives(u, gamma);
    T f[5];
    T* Fe = sF + le * 15 * NN;
    T gn[PHYS ? 15 : 1], fv[5];
    if (PHYS) {
#pragma unroll
      for (int kk = 0; kk < 15; ++kk) gn[kk] = Gr[(e * 15 + kk) * NN + nd];
    }
    axis_flux<T, 1>(u, q, blk ? c[MC_VG] : T(0), f);          // xi^1 -> y (grid velocity)
    if (PHYS) {
      viscous_flux_axis(u, gn, 1, c, fv);
#pragma unroll
      for (int v = 0; v < 5; ++v) f[v] -= fv[v];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) Fe[v * NN + nd] = f[v];
    axis_flux<T, 2>(u, q, T(0), f);                             // xi^2 -> z
    if (PHYS) {
      viscous_flux_axis(u, gn, 2, c, fv);
#pragma unroll
      for (int v = 0; v < 5; ++v) f[v] -= fv[v];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) Fe[(5 + v) * NN + nd] = f[v];
    axis_flux<T, 0>(u, q, T(0), f);                             // xi^3 -> x
    if (PHYS) {
      viscous_flux_axis(u, gn, 0, c, fv);
#pragma unroll
      for (int v = 0; v < 5; ++v) f[v] -= fv[v];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) Fe[(10 + v) * NN + nd] = f[v];
  }

  element_face_fluxes<N, T, RIEM, PHYS>(m, sp, U, Fs, Fm, Gr, e0, sS, tid);

  // ---- volume integral (sum factorisation) + surface integral ----
  T acc[5];
  __syncthreads();
  contract_lines_inplace<N, T>(sF, tid);
  __syncthreads();
  if (!active) return;
  {
    // the metric terms |Ja^d| (constant per block) scale the contracted fluxes
    const int blk = e >= m.Es;
    const T a0 = c[MC_METRIC + 3 * blk], a1 = c[MC_METRIC + 3 * blk + 1], a2 = c[MC_METRIC + 3 * blk + 2];
    const T* Fe = sF + le * 15 * NN + nd;
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] = a0 * Fe[v * NN] + a1 * Fe[(5 + v) * NN] + a2 * Fe[(10 + v) * NN];
  }
  element_surface_update<N, T, MODE>(m, sS + le * 30 * NP2, acc, nd, e, base, u, g, out, G, rkA, rkB, dt, Ts, Tm);
}

template <int N, typename T, int RIEM, int MODE, int PHYS = 0>
__global__ void __launch_bounds__(ElemCfg<N>::THREADS, (sizeof(T) == 4 && PHYS == 0) ? ElemCfg<N>::MINB : 1)
dg_element_kernel(const MeshDev m, const StageParams* __restrict__ sp, const T* __restrict__ U,
                  T* __restrict__ out, T* __restrict__ G, const T* __restrict__ Fs,
                  const T* __restrict__ Fm, const T rkA, const T rkB, const T dt, const T* __restrict__ Gr,
                  T* __restrict__ Ts, T* __restrict__ Tm) {
  element_block<N, T, RIEM, MODE, PHYS>(m, sp, U, out, G, Fs, Fm, rkA, rkB, dt,
                                        (long long)blockIdx.x * ElemCfg<N>::EPB, Gr, Ts, Tm);
}

template <int N, typename T, int RIEM, int MODE, int PHYS = 0>
static cudaError_t launch_elem_t(const ElemArgs& a, cudaStream_t st) {
  using C = ElemCfg<N>;
  const size_t smem = C::template smem_bytes<T>();
  const long long blocks = (a.m.E + C::EPB - 1) / C::EPB;
  if (blocks <= 0) return cudaSuccess;
  dg_element_kernel<N, T, RIEM, MODE, PHYS><<<(unsigned)blocks, C::THREADS, smem, st>>>(
      a.m, a.sp, (const T*)a.U, (T*)a.out, (T*)a.G, (const T*)a.Fs, (const T*)a.Fm, (T)a.rkA, (T)a.rkB, (T)a.dt,
      (const T*)a.Gr, (T*)a.Ts, (T*)a.Tm);
  return cudaGetLastError();
}

// No shared-memory carveout preference: the driver takes the smallest shared-memory
// configuration that holds the resident CTAs, and the rest of the SM's 256 KB stays L1,
// which then holds the element's own and its neighbours' face traces the face fluxes re-read
// (measured on N = 5: 11 % faster than the maximum-shared configuration).
template <int N, typename T, int RIEM, int MODE, int PHYS = 0>
static cudaError_t prepare_elem_t() {
  using C = ElemCfg<N>;
  cudaError_t e = cudaFuncSetAttribute(dg_element_kernel<N, T, RIEM, MODE, PHYS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::template smem_bytes<T>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(dg_element_kernel<N, T, RIEM, MODE, PHYS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutDefault);
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

// BR1 lifting (Bassi and Rebay's first method, Sec. 3.1): the gradients of the primitive
// variables (rho, v1, v2, v3, p) along x, y, z by the same weak DG divergence operator as
// the fluxes, applied to the "flux" Q e_axis with face value the mean of both sides' traces
// (weak Dirichlet faces: the mean with the exterior state; sliding faces: the mortar means
// computed by the interface kernel in lifting mode, Ls / Lm).  Output Gr[e][15][NN] with
// component 5 a + c = d(primitive c)/dx_a.
#pragma once

#include "sm_element.cuh"

template <int N, typename T>
__device__ __forceinline__ void lift_block(const MeshDev& m, const StageParams* __restrict__ sp, const T* __restrict__ U,
                                           T* __restrict__ Gr, const T* __restrict__ Ls, const T* __restrict__ Lm,
                                           const long long e0) {
  using C = ElemCfg<N>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN, EPB = C::EPB, THREADS = C::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sF = reinterpret_cast<T*>(smem_raw);        // [EPB][3][5][NN], the element kernel's line layouts
  T* sS = sF + EPB * 15 * NN;                    // [EPB][6][5][NP2]
  const T* c = Prec<T>::c(m);
  const int tid = threadIdx.x;
  const int le = tid / NN, nd = tid - le * NN;
  const long long e = e0 + le;
  const bool active = e < m.E;
  const T gamma = c[MC_GAMMA];
  const int i = nd % NP, j = (nd / NP) % NP, k = nd / NP2;
  if (active) {
    T u[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = U[e * 5 * NN + v * NN + nd];
    const Prim<T> q = primitives(u, gamma);
    const T Q[5] = {u[0], q.u[0], q.u[1], q.u[2], q.p};
    const int blk = e >= m.Es;
    const T a0 = c[MC_METRIC + 3 * blk], a1 = c[MC_METRIC + 3 * blk + 1], a2 = c[MC_METRIC + 3 * blk + 2];
    T* Fe = sF + le * 15 * NN;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      Fe[v * NN + nd] = a0 * Q[v];
      Fe[(5 + v) * NN + nd] = a1 * Q[v];
      Fe[(10 + v) * NN + nd] = a2 * Q[v];
    }
  }
  for (int w = tid; w < EPB * 6 * NP2; w += THREADS) {
    const int l2 = w / (6 * NP2);
    const int r = w - l2 * 6 * NP2;
    const int fc = r / NP2, ab = r - fc * NP2;
    const long long e2 = e0 + l2;
    if (e2 >= m.E) continue;
    const int blk2 = e2 >= m.Es;
    const int d = fc >> 1, side = fc & 1;
    const int a = ab % NP, b = ab / NP;
    const int sn = d == 0 ? 1 : (d == 1 ? NP : NP2);
    const int sab = d == 0 ? NP * ab : (d == 1 ? a + NP2 * b : ab);
    const int vn = sab + (side ? N : 0) * sn;
    int nb, pos_ix = 0, pos_f = 0;
    const int* tp = m.topo ? reinterpret_cast<const int*>(m.topo) + 8 * e2 : nullptr;
    if (tp) {
      nb = tp[fc];
    } else {
      const ElemPos p = decode_elem(m, e2);
      long long qq = 0;
      const int kind = face_neighbor(m, p, d, side, &qq);
      nb = kind == 0 ? (int)qq : (kind == 1 ? NB_BOUNDARY : NB_INTERFACE);
      pos_ix = p.ix;
      pos_f = p.iz * m.ny + p.iy;
    }
    T Fo[5];
    if (nb == NB_INTERFACE) {
      const int fi = tp ? tp[7] : pos_f;
      const T* src = (blk2 ? Lm : Ls) + (long long)fi * 5 * NP2 + ab;
#pragma unroll
      for (int v = 0; v < 5; ++v) Fo[v] = src[v * NP2];
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
        if (tp) { pos_ix = tp[6] >> 1; pos_f = tp[7]; }
        const int iy = pos_f % m.ny, iz = pos_f / m.ny;
        const T* xi = Prec<T>::x(m.basis);
        const int ii = vn % NP, jj = (vn / NP) % NP, kk = vn / NP2;
        const T hx = c[MC_H + blk2];
        T X[3];
        X[0] = c[MC_X + blk2] + (T)pos_ix * hx + (xi[kk] + T(1)) * T(0.5) * hx;
        X[1] = c[MC_X + 2] + (T)iy * c[MC_H + 2] + (xi[ii] + T(1)) * T(0.5) * c[MC_H + 2] + (blk2 ? (T)sp->delta : T(0));
        X[2] = c[MC_X + 3] + (T)iz * c[MC_H + 3] + (xi[jj] + T(1)) * T(0.5) * c[MC_H + 3];
        boundary_state<T>(m, X, (T)sp->t, uout);
      }
      const Prim<T> qi = primitives(uin, gamma), qo = primitives(uout, gamma);
      const T Qi[5] = {uin[0], qi.u[0], qi.u[1], qi.u[2], qi.p};
      const T Qo[5] = {uout[0], qo.u[0], qo.u[1], qo.u[2], qo.p};
      const T sJ = c[MC_METRIC + 3 * blk2 + d];
      const T sg = side ? sJ : -sJ;
#pragma unroll
      for (int v = 0; v < 5; ++v) Fo[v] = sg * T(0.5) * (Qi[v] + Qo[v]);
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) sS[((l2 * 6 + fc) * 5 + v) * NP2 + ab] = Fo[v];
  }
  __syncthreads();
  contract_lines_inplace<N, T>(sF, tid);
  __syncthreads();
  if (!active) return;
  const T iw0 = c[MC_IW0];
  const T invJ = -c[MC_MINVJ + (e >= m.Es)];
  const T* Fe = sF + le * 15 * NN;
  const T* Se = sS + le * 30 * NP2;
  T* Ge = Gr + e * 15 * NN + nd;
  // xi^1 -> y (axis 1), xi^2 -> z (axis 2), xi^3 -> x (axis 0)
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    T gy = Fe[v * NN + nd];
    T gz = Fe[(5 + v) * NN + nd];
    T gx = Fe[(10 + v) * NN + nd];
    if (i == 0) gy += iw0 * Se[(0 * 5 + v) * NP2 + j + NP * k];
    if (i == N) gy += iw0 * Se[(1 * 5 + v) * NP2 + j + NP * k];
    if (j == 0) gz += iw0 * Se[(2 * 5 + v) * NP2 + i + NP * k];
    if (j == N) gz += iw0 * Se[(3 * 5 + v) * NP2 + i + NP * k];
    if (k == 0) gx += iw0 * Se[(4 * 5 + v) * NP2 + i + NP * j];
    if (k == N) gx += iw0 * Se[(5 * 5 + v) * NP2 + i + NP * j];
    Ge[(0 * 5 + v) * NN] = gx * invJ;
    Ge[(1 * 5 + v) * NN] = gy * invJ;
    Ge[(2 * 5 + v) * NN] = gz * invJ;
  }
}

// Curvilinear kernels: the DGSEM operator of Sec. 3.1 with per-node metric terms
// (Eq. transformed_equation) and the sliding interface of Sec. 3.3 for the rotating
// geometries of the paper's overview figure: the cylindrical interface (rotor inside the
// circle, stator outside; geom 1) and the plane annular interface normal to the axis (rotor
// below, stator above; geom 3), both with a periodic angular sector and slip walls.
//
// Frames.  The state is stored in the global Cartesian frame.  The rotor (block 0 of the
// cylinder) turns rigidly about the z axis by phi(t); its metrics at time t are R(phi)
// times those at t = 0 and its grid velocity omega e_z x X.  The Euler and Navier-Stokes
// fluxes commute with rotations, so a rotor element is evaluated in its own frame: the
// momentum (and the lifted gradients) are turned by -phi on load, the metric terms of
// t = 0 are used as they are, Ja^i . v^g is time-independent, and the residual's momentum
// is turned back by +phi before the Runge-Kutta update.  Stator elements use the identity.
//
// Geometry per node (geo, [E][13][NN]): Ja^i_n (slot 3 i + n), J (slot 9), and
// Ja^i . v^g / |v| of the moving block (slots 10..12, times the grid speed MC_VG).
#pragma once

#include "sm_element.cuh"

// cos, sin of the frame rotation of a block: the rotor of the cylinder turns by phi
template <typename T>
__device__ __forceinline__ void block_frame(const MeshDev& m, const StageParams* sp, int blk, T& c, T& s) {
  if (rotating_geom(m.geom) && blk == 0) {
    c = Prec<T>::rot(sp)[0];
    s = Prec<T>::rot(sp)[1];
  } else {
    c = T(1);
    s = T(0);
  }
}

// the moving block: the plane's block 1 translates, the cylinder's block 0 (rotor) turns
__device__ __forceinline__ bool moving_block(const MeshDev& m, int blk) { return rotating_geom(m.geom) ? blk == 0 : blk == 1; }

// Viscous flux of a state and its gradients dotted with a vector N (all three columns).
template <typename T>
__device__ __forceinline__ void viscous_dot_n(const T U[5], const T g[15], const T N[3], const T* c, T out[5]) {
  T f0[5], f1[5], f2[5];
  viscous_flux_axis(U, g, 0, c, f0);
  viscous_flux_axis(U, g, 1, c, f1);
  viscous_flux_axis(U, g, 2, c, f2);
#pragma unroll
  for (int v = 0; v < 5; ++v) out[v] = N[0] * f0[v] + N[1] * f1[v] + N[2] * f2[v];
}

// Face fluxes of the CTA's EPB curved elements (elements e0 ..), one work item per (element,
// face, face node), in each element's frame, into sS[EPB][6][5][NP^2] as outward fluxes times
// the surface element.  Reads global memory only.
template <int N, typename T, int RIEM, int PHYS>
__device__ __forceinline__ void curved_face_fluxes(const MeshDev& m, const StageParams* __restrict__ sp,
                                                   const T* __restrict__ U, const T* __restrict__ Fs,
                                                   const T* __restrict__ Fm, const T* __restrict__ Gr,
                                                   const long long e0, T* sS, const int tid) {
  using C = ElemCfg<N>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN, EPB = C::EPB, THREADS = C::THREADS;
  const T* c = Prec<T>::c(m);
  const T* geo = reinterpret_cast<const T*>(m.geo);
  const T gamma = c[MC_GAMMA];
  const T vspeed = c[MC_VG];
  for (int w = tid; w < EPB * 6 * NP2; w += THREADS) {
    const int l2 = w / (6 * NP2);
    const int r = w - l2 * 6 * NP2;
    const int fc2 = r / NP2, ab = r - fc2 * NP2;
    const long long e2 = e0 + l2;
    if (e2 >= m.E) continue;
    const int blk2 = e2 >= m.Es;
    const int d = fc2 >> 1, side = fc2 & 1;
    const int a = ab % NP, b = ab / NP;
    const int sn = d == 0 ? 1 : (d == 1 ? NP : NP2);
    const int sab = d == 0 ? NP * ab : (d == 1 ? a + NP2 * b : ab);
    const int vn = sab + (side ? N : 0) * sn;
    T ec, es;
    block_frame<T>(m, sp, blk2, ec, es);
    int nb, pos_ix, pos_f;
    const int* tp = m.topo ? reinterpret_cast<const int*>(m.topo) + 8 * e2 : nullptr;
    if (tp) {
      nb = tp[fc2];
      pos_ix = tp[6] >> 1;
      pos_f = tp[7];
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
      const T* src = (blk2 ? Fm : Fs) + (long long)pos_f * 5 * NP2 + ab;
#pragma unroll
      for (int v = 0; v < 5; ++v) Fo[v] = src[v * NP2];
      rotate_state_z(Fo, ec, -es);
    } else {
      const T* ge = geo + e2 * 13 * NN + vn;
      T Nv[3] = {ge[(3 * d) * NN], ge[(3 * d + 1) * NN], ge[(3 * d + 2) * NN]};
      const T sJ = Prec<T>::sqrt_(Nv[0] * Nv[0] + Nv[1] * Nv[1] + Nv[2] * Nv[2]);
      const T isJ = Prec<T>::rcp(sJ);
      const T nrm[3] = {Nv[0] * isJ, Nv[1] * isJ, Nv[2] * isJ};
      T vgn = (moving_block(m, blk2) ? vspeed : T(0)) * ge[(10 + d) * NN] * isJ;
      const T sg = side ? T(1) : T(-1);
      T uin[5], uout[5];
      const T* Ui = U + e2 * 5 * NN + vn;
#pragma unroll
      for (int v = 0; v < 5; ++v) uin[v] = Ui[v * NN];
      rotate_state_z(uin, ec, -es);
      bool wall = false;
      // periodic sector of the cylinder: the neighbour across theta = y1 (or y0) is the
      // image turned by +Theta (or -Theta)
      T pc = T(1), ps = T(0);
      if (nb >= 0) {
        const T* Un = U + (long long)nb * 5 * NN + sab + (side ? 0 : N) * sn;
#pragma unroll
        for (int v = 0; v < 5; ++v) uout[v] = Un[v * NN];
        rotate_state_z(uout, ec, -es);
        const int iy = pos_f % m.ny;
        if (rotating_geom(m.geom) && d == 0 && ((side && iy == m.ny - 1) || (!side && iy == 0))) {
          pc = c[MC_PCOS];
          ps = side ? c[MC_PSIN] : -c[MC_PSIN];
          rotate_state_z(uout, pc, ps);
        }
      } else if (rotating_geom(m.geom)) {
        // slip wall: interior state with the normal momentum reflected; the wall moves
        // tangentially (zero normal grid velocity)
        wall = true;
        vgn = T(0);
        const T mn = uin[1] * nrm[0] + uin[2] * nrm[1] + uin[3] * nrm[2];
        uout[0] = uin[0];
#pragma unroll
        for (int q3 = 0; q3 < 3; ++q3) uout[1 + q3] = uin[1 + q3] - T(2) * mn * nrm[q3];
        uout[4] = uin[4];
      } else {
        // weak Dirichlet face of the plane box: the flow's state at the node's position
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
      T L[5], Rr[5], f[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        L[v] = side ? uin[v] : uout[v];
        Rr[v] = side ? uout[v] : uin[v];
      }
      riemann_normal<T, RIEM>(L, Rr, nrm, vgn, gamma, f);
#pragma unroll
      for (int v = 0; v < 5; ++v) Fo[v] = sg * sJ * f[v];
      if (PHYS && !wall) {
        // BR1 viscous face flux: mean of both sides' viscous fluxes along the outward N
        T gi[15], go[15], fvi[5], fvo[5];
        const T* gp = Gr + e2 * 15 * NN + vn;
        const T* gq = nb >= 0 ? Gr + (long long)nb * 15 * NN + sab + (side ? 0 : N) * sn : gp;
#pragma unroll
        for (int kk = 0; kk < 15; ++kk) { gi[kk] = gp[kk * NN]; go[kk] = gq[kk * NN]; }
        rotate_grad_z(gi, ec, -es);
        rotate_grad_z(go, ec, -es);
        if (nb >= 0) rotate_grad_z(go, pc, ps);
        const T No[3] = {sg * Nv[0], sg * Nv[1], sg * Nv[2]};
        viscous_dot_n(uin, gi, No, c, fvi);
        viscous_dot_n(uout, go, No, c, fvo);
#pragma unroll
        for (int v = 0; v < 5; ++v) Fo[v] -= T(0.5) * (fvi[v] + fvo[v]);
      }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) sS[((l2 * 6 + fc2) * 5 + v) * NP2 + ab] = Fo[v];
  }

}

// Surface integral, 1/J, the turn back to the global frame (rotor) and the RK update of node
// nd of curved element e, given the node's volume term acc (in the element's frame).
template <int N, typename T, int MODE>
__device__ __forceinline__ void curved_surface_update(const MeshDev& m, const T* Se, T (&acc)[5], const int nd,
                                                      const long long e, const long long base, const T (&u)[5],
                                                      const T (&g)[5], const T fc, const T fs,
                                                      T* __restrict__ out, T* __restrict__ G, const T rkA,
                                                      const T rkB, const T dt) {
  using C = ElemCfg<N>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN;
  const T* c = Prec<T>::c(m);
  const T* geo = reinterpret_cast<const T*>(m.geo);
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
  const T mInvJ = -Prec<T>::rcp(geo[(e * 13 + 9) * NN + nd]);
  T ut[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) ut[v] = acc[v] * mInvJ;
  rotate_state_z(ut, fc, fs);
  if (MODE == ELEM_RHS) {
#pragma unroll
    for (int v = 0; v < 5; ++v) out[base + v * NN] = ut[v];
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const T gn = (MODE == ELEM_STAGE_FIRST) ? dt * ut[v] : rkA * g[v] + dt * ut[v];
      G[base + v * NN] = gn;
      out[base + v * NN] = u[v] + rkB * gn;
    }
  }
}

// One CTA: elements e0 .. e0+EPB-1 (same work split and shared-memory layouts as the
// Cartesian element kernel).  PHYS 1 adds the viscous fluxes of the lifted gradients Gr
// ([E][15][NN] in the global frame, turned into the element's frame on load).
template <int N, typename T, int RIEM, int MODE, int PHYS>
__device__ __forceinline__ void curved_element_block(const MeshDev& m, const StageParams* __restrict__ sp,
                                                     const T* __restrict__ U, T* __restrict__ out,
                                                     T* __restrict__ G, const T* __restrict__ Fs,
                                                     const T* __restrict__ Fm, const T rkA, const T rkB,
                                                     const T dt, const long long e0, const T* __restrict__ Gr) {
  using C = ElemCfg<N>;
  constexpr int NP2 = C::NP2, NN = C::NN, EPB = C::EPB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sF = reinterpret_cast<T*>(smem_raw);        // [EPB][3][5][NN], node order
  T* sS = sF + EPB * 15 * NN;                    // [EPB][6][5][NP2] outward face fluxes
  const T* c = Prec<T>::c(m);
  const T* geo = reinterpret_cast<const T*>(m.geo);
  const int tid = threadIdx.x;
  const int le = tid / NN, nd = tid - le * NN;
  const long long e = e0 + le;
  const bool active = e < m.E;
  const long long base = e * 5 * NN + nd;
  const T gamma = c[MC_GAMMA];
  const T vspeed = c[MC_VG];
  const int blk = active && e >= m.Es;
  T fc, fs;
  block_frame<T>(m, sp, blk, fc, fs);

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
    const Prim<T> q = primitives(ub, gamma);
    T F[3][5];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      F[a][0] = ub[0] * q.u[a];
      F[a][1] = ub[1] * q.u[a] + (a == 0 ? q.p : T(0));
      F[a][2] = ub[2] * q.u[a] + (a == 1 ? q.p : T(0));
      F[a][3] = ub[3] * q.u[a] + (a == 2 ? q.p : T(0));
      F[a][4] = (ub[4] + q.p) * q.u[a];
    }
    if (PHYS) {
      T gn[15], fv[5];
#pragma unroll
      for (int kk = 0; kk < 15; ++kk) gn[kk] = Gr[(e * 15 + kk) * NN + nd];
      rotate_grad_z(gn, fc, -fs);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        viscous_flux_axis(ub, gn, a, c, fv);
#pragma unroll
        for (int v = 0; v < 5; ++v) F[a][v] -= fv[v];
      }
    }
    const T* ge = geo + e * 13 * NN + nd;
    const T vs = moving_block(m, blk) ? vspeed : T(0);
    T* Fe = sF + le * 15 * NN;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T J0 = ge[(3 * d) * NN], J1 = ge[(3 * d + 1) * NN], J2 = ge[(3 * d + 2) * NN];
      const T V = vs * ge[(10 + d) * NN];
#pragma unroll
      for (int v = 0; v < 5; ++v) Fe[(5 * d + v) * NN + nd] = J0 * F[0][v] + J1 * F[1][v] + J2 * F[2][v] - V * ub[v];
    }
  }

  curved_face_fluxes<N, T, RIEM, PHYS>(m, sp, U, Fs, Fm, Gr, e0, sS, tid);

  __syncthreads();
  contract_lines_inplace<N, T>(sF, tid);
  __syncthreads();
  if (!active) return;
  T acc[5];
  {
    const T* Fe = sF + le * 15 * NN + nd;
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] = Fe[v * NN] + Fe[(5 + v) * NN] + Fe[(10 + v) * NN];
  }
  curved_surface_update<N, T, MODE>(m, sS + le * 30 * NP2, acc, nd, e, base, u, g, fc, fs, out, G, rkA, rkB, dt);
}

// Curved sliding interface, one CTA per tile of TF static faces of line iz (Sec. 3.3,
// steps 3-5): both sides' traces staged in shared memory in the rotor's frame (a stator
// face seen through w periodic wraps is turned by w Theta - phi), forward projection along
// the sliding direction, the mortar normal and surface element from the static face's
// Ja^3 projected onto the mortar nodes (grid velocity normal to the interface: zero), the
// mortar values, and the conservative back-projection.  Both outputs are in the global
// frame (static faces turned by +phi, moving faces back by their wrap angle).
// Modes: CV_EULER the Riemann flux; CV_NS adds the BR1 viscous mean of both sides'
// viscous fluxes from the projected states and projected gradients Gr (Sec. 3.2); CV_LIFT
// the lifting values q* N_a (mean of the projected primitive traces), 15 per node.
enum { CV_EULER = 0, CV_NS = 1, CV_LIFT = 2 };

template <int N> struct CurvedIfCfg {
  static constexpr int NP = N + 1, NP2 = NP * NP, TF = 4, THREADS = 128;
  template <typename T, int MODE = CV_EULER> static constexpr size_t smem_bytes() {
    return sizeof(T) * (size_t)(8 * NP2 + 2 * (TF + 1) * 5 * NP2 + (MODE == CV_NS ? 2 * (TF + 1) * 15 * NP2 : 0) +
                                TF * 3 * NP2 + (2 * TF + 1) * (MODE == CV_LIFT ? 15 : 5) * NP2);
  }
};

template <int N, typename T, int RIEM, int MODE = CV_EULER>
__device__ __forceinline__ void curved_interface_tile(const MeshDev& m, const StageParams* __restrict__ sp,
                                                      const T* __restrict__ U, T* __restrict__ Fs,
                                                      T* __restrict__ Fm, const int tile_x, const int iz,
                                                      const T* __restrict__ Gr = nullptr) {
  using C = CurvedIfCfg<N>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = NP * NP * NP, TF = C::TF, THREADS = C::THREADS;
  constexpr int NC = MODE == CV_LIFT ? 15 : 5;   // values per mortar / face node
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sMat = reinterpret_cast<T*>(smem_raw);   // [8][NP2]
  T* sTs = sMat + 8 * NP2;                    // [TF+1][5][NP2]
  T* sTm = sTs + (TF + 1) * 5 * NP2;          // [TF+1][5][NP2]
  T* sGs = sTm + (TF + 1) * 5 * NP2;          // [TF+1][15][NP2] (CV_NS)
  T* sGm = sGs + (MODE == CV_NS ? (TF + 1) * 15 * NP2 : 0);
  T* sN = sGm + (MODE == CV_NS ? (TF + 1) * 15 * NP2 : 0);   // [TF][3][NP2] static face Ja^3
  T* sFm = sN + TF * 3 * NP2;                 // [2TF+1][NC][NP2]
  __shared__ long long s_el[2][TF + 1];
  __shared__ int s_wk[TF + 1];
  const T* geo = reinterpret_cast<const T*>(m.geo);
  const T* c = Prec<T>::c(m);
  const int tid = threadIdx.x;
  const int i0 = tile_x * TF;
  const int ny = m.ny;
  const int TFe = min(TF, ny - i0);
  const long long n = sp->n;
  long long nl = n % ny;
  const int nmod = (int)(nl < 0 ? nl + ny : nl);
  for (int w = tid; w < 8 * NP2; w += THREADS) sMat[w] = Prec<T>::mat(sp, w / NP2)[w % NP2];
  if (tid < 2 * (TFe + 1)) {
    const int side = tid / (TFe + 1), r = tid - side * (TFe + 1);
    int f = side ? i0 - nmod - 1 + r : i0 + r;
    f %= ny;
    if (f < 0) f += ny;
    s_el[side][r] = encode_elem(m, side, side ? 0 : m.nxs - 1, f, iz);
    if (side) {
      // wrap count of the moving face's unwrapped index i0 - n - 1 + r, relative to w0
      const long long a = (long long)i0 - n - 1 + r;
      long long q = a / ny;
      if (a % ny != 0 && a < 0) q -= 1;
      s_wk[r] = (int)(q - sp->w0);
    }
  }
  __syncthreads();
  T rc, rs;
  block_frame<T>(m, sp, 0, rc, rs);
  const T gamma = c[MC_GAMMA];
  for (int w = tid; w < 2 * (TFe + 1) * NP2; w += THREADS) {
    const int side = w >= (TFe + 1) * NP2;
    const int ww = w - side * (TFe + 1) * NP2;
    const int r = ww / NP2, ab = ww - r * NP2;
    const long long e = s_el[side][r];
    const int layer = side ? 0 : NP2 * N;
    T u[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * NN + layer + ab];
    T ac = T(1), as = T(0);
    // the halo static face i0 + TFe = n_par of the last tile is static face 0's periodic
    // image: turned by +Theta, like the moving faces it meets
    const bool image = rotating_geom(m.geom) && !side && i0 + r >= ny;
    if (rotating_geom(m.geom)) {
      if (side) {
        const T* a = Prec<T>::arot(sp, s_wk[r]);
        ac = a[0];
        as = a[1];
      } else {
        ac = rc;
        as = -rs;
      }
      rotate_state_z(u, ac, as);
      if (image) rotate_state_z(u, c[MC_PCOS], c[MC_PSIN]);
    }
    if (MODE == CV_LIFT) {
      const Prim<T> q = primitives(u, gamma);
      u[1] = q.u[0]; u[2] = q.u[1]; u[3] = q.u[2]; u[4] = q.p;
    }
    T* t = (side ? sTm : sTs) + r * 5 * NP2 + ab;
#pragma unroll
    for (int v = 0; v < 5; ++v) t[v * NP2] = u[v];
    if (MODE == CV_NS) {
      T gg[15];
#pragma unroll
      for (int kk = 0; kk < 15; ++kk) gg[kk] = Gr[(e * 15 + kk) * NN + layer + ab];
      rotate_grad_z(gg, ac, as);
      if (image) rotate_grad_z(gg, c[MC_PCOS], c[MC_PSIN]);
      T* tg = (side ? sGm : sGs) + r * 15 * NP2 + ab;
#pragma unroll
      for (int kk = 0; kk < 15; ++kk) tg[kk * NP2] = gg[kk];
    }
    if (!side && r < TFe) {
#pragma unroll
      for (int q = 0; q < 3; ++q) sN[(r * 3 + q) * NP2 + ab] = geo[(e * 13 + 6 + q) * NN + NP2 * N + ab];
    }
  }
  __syncthreads();
  // mortars mi = 2 r + i_sub (r < TFe) and the halo mortar 2 TFe (static face i0+TFe, its
  // normal read from geo directly)
  for (int w = tid; w < (2 * TFe + 1) * NP2; w += THREADS) {
    const int mi = w / NP2, ab = w - mi * NP2;
    const int r = mi >> 1, isub = mi & 1;
    const int j = ab % NP, q = ab / NP;
    const T* Ps = sMat + (isub ? 1 : 0) * NP2 + j * NP;
    const T* Pm = sMat + (isub ? 2 : 3) * NP2 + j * NP;
    const T* ts = sTs + r * 5 * NP2 + q * NP;
    const T* tm = sTm + (r + isub) * 5 * NP2 + q * NP;
    T QL[5], QR[5], Nm[3];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      T al = T(0), ar = T(0);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        al += Ps[i] * ts[v * NP2 + i];
        ar += Pm[i] * tm[v * NP2 + i];
      }
      QL[v] = al;
      QR[v] = ar;
    }
#pragma unroll
    for (int c3 = 0; c3 < 3; ++c3) {
      T an = T(0);
      if (r < TFe) {
#pragma unroll
        for (int i = 0; i < NP; ++i) an += Ps[i] * sN[(r * 3 + c3) * NP2 + q * NP + i];
      } else {
        const T* gn = geo + (s_el[0][r] * 13 + 6 + c3) * NN + NP2 * N + q * NP;
#pragma unroll
        for (int i = 0; i < NP; ++i) an += Ps[i] * gn[i];
      }
      Nm[c3] = an;
    }
    if (rotating_geom(m.geom) && r == TFe && i0 + TFe >= ny) {
      // the halo face is static face 0's image: its normal turned by +Theta
      const T x = c[MC_PCOS] * Nm[0] - c[MC_PSIN] * Nm[1], y = c[MC_PSIN] * Nm[0] + c[MC_PCOS] * Nm[1];
      Nm[0] = x;
      Nm[1] = y;
    }
    if (MODE == CV_LIFT) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int v = 0; v < 5; ++v) sFm[(mi * 15 + a * 5 + v) * NP2 + ab] = T(0.5) * (QL[v] + QR[v]) * Nm[a];
      continue;
    }
    const T sJ = Prec<T>::sqrt_(Nm[0] * Nm[0] + Nm[1] * Nm[1] + Nm[2] * Nm[2]);
    const T isJ = Prec<T>::rcp(sJ);
    const T nrm[3] = {Nm[0] * isJ, Nm[1] * isJ, Nm[2] * isJ};
    T F[5];
    riemann_normal<T, RIEM>(QL, QR, nrm, T(0), gamma, F);
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] *= sJ;
    if (MODE == CV_NS) {
      T GL[15], GR[15], fl[5], fr[5];
      const T* gs = sGs + r * 15 * NP2 + q * NP;
      const T* gm = sGm + (r + isub) * 15 * NP2 + q * NP;
#pragma unroll
      for (int kk = 0; kk < 15; ++kk) {
        T al = T(0), ar = T(0);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          al += Ps[i] * gs[kk * NP2 + i];
          ar += Pm[i] * gm[kk * NP2 + i];
        }
        GL[kk] = al;
        GR[kk] = ar;
      }
      viscous_dot_n(QL, GL, Nm, c, fl);
      viscous_dot_n(QR, GR, Nm, c, fr);
#pragma unroll
      for (int v = 0; v < 5; ++v) F[v] -= T(0.5) * (fl[v] + fr[v]);
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) sFm[(mi * 5 + v) * NP2 + ab] = F[v];
  }
  __syncthreads();
  for (int w = tid; w < 2 * TFe * NP2; w += THREADS) {
    const int side = w >= TFe * NP2;
    const int ww = w - side * TFe * NP2;
    const int r = ww / NP2, ab = ww - r * NP2;
    const int i = ab % NP, q = ab / NP;
    const T* Blo = sMat + (side ? 6 : 4) * NP2 + i * NP;
    const T* Bhi = sMat + (side ? 7 : 5) * NP2 + i * NP;
    const T* flo = sFm + (2 * r + side) * NC * NP2 + q * NP;
    const T* fhi = sFm + (2 * r + 1 + side) * NC * NP2 + q * NP;
    T o[NC];
#pragma unroll
    for (int v = 0; v < NC; ++v) {
      T acc = T(0);
#pragma unroll
      for (int jj = 0; jj < NP; ++jj) acc += Blo[jj] * flo[v * NP2 + jj] + Bhi[jj] * fhi[v * NP2 + jj];
      o[v] = side ? -acc : acc;
    }
    if (rotating_geom(m.geom)) {
      T oc = rc, os = rs;
      if (side) {
        const T* a = Prec<T>::arot(sp, s_wk[r + 1]);
        oc = a[0];
        os = -a[1];
      }
      if constexpr (MODE == CV_LIFT) rotate_grad_z(o, oc, os);
      else rotate_state_z(o, oc, os);
    }
    int f = side ? i0 - nmod + r : i0 + r;
    f %= ny;
    if (f < 0) f += ny;
    T* dst = (side ? Fm : Fs) + (((long long)iz * ny + f) * NC) * NP2 + ab;
#pragma unroll
    for (int v = 0; v < NC; ++v) dst[v * NP2] = o[v];
  }
}

// BR1 lifting with metric terms (Sec. 3.1): for each Cartesian direction a,
//   J d(q)/dx_a = sum_i Dhat_i (Ja^i_a q) + sum_faces q* N_a / w,
// q the primitives (rho, v, p) in the element's frame, q* the mean of both sides' traces
// (slip walls: the mirror state; plane boundaries: the flow's state; the interface: the
// mortar means Ls / Lm, 15 values a * 5 + c per face node in the global frame).  Three
// passes over a share the face values; Gr is written in the global frame.
template <int N, typename T>
__device__ __forceinline__ void curved_lift_block(const MeshDev& m, const StageParams* __restrict__ sp,
                                                  const T* __restrict__ U, T* __restrict__ Gr,
                                                  const T* __restrict__ Ls, const T* __restrict__ Lm,
                                                  const long long e0) {
  using C = ElemCfg<N>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN, EPB = C::EPB, THREADS = C::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sF = reinterpret_cast<T*>(smem_raw);        // [EPB][3][5][NN]
  T* sS = sF + EPB * 15 * NN;                    // [EPB][6][15][NP2] face values q* N_a
  const T* c = Prec<T>::c(m);
  const T* geo = reinterpret_cast<const T*>(m.geo);
  const int tid = threadIdx.x;
  const int le = tid / NN, nd = tid - le * NN;
  const long long e = e0 + le;
  const bool active = e < m.E;
  const T gamma = c[MC_GAMMA];
  const int blk = active && e >= m.Es;
  T fc, fs;
  block_frame<T>(m, sp, blk, fc, fs);
  const int i = nd % NP, j = (nd / NP) % NP, k = nd / NP2;
  T Q[5] = {T(0), T(0), T(0), T(0), T(0)};
  if (active) {
    T u[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = U[e * 5 * NN + v * NN + nd];
    rotate_state_z(u, fc, -fs);
    const Prim<T> q = primitives(u, gamma);
    Q[0] = u[0]; Q[1] = q.u[0]; Q[2] = q.u[1]; Q[3] = q.u[2]; Q[4] = q.p;
  }
  // face values, all three components
  for (int w = tid; w < EPB * 6 * NP2; w += THREADS) {
    const int l2 = w / (6 * NP2);
    const int r = w - l2 * 6 * NP2;
    const int fc2 = r / NP2, ab = r - fc2 * NP2;
    const long long e2 = e0 + l2;
    if (e2 >= m.E) continue;
    const int blk2 = e2 >= m.Es;
    const int d = fc2 >> 1, side = fc2 & 1;
    const int a = ab % NP, b = ab / NP;
    const int sn = d == 0 ? 1 : (d == 1 ? NP : NP2);
    const int sab = d == 0 ? NP * ab : (d == 1 ? a + NP2 * b : ab);
    const int vn = sab + (side ? N : 0) * sn;
    T ec, es;
    block_frame<T>(m, sp, blk2, ec, es);
    int nb, pos_ix, pos_f;
    const int* tp = m.topo ? reinterpret_cast<const int*>(m.topo) + 8 * e2 : nullptr;
    if (tp) {
      nb = tp[fc2];
      pos_ix = tp[6] >> 1;
      pos_f = tp[7];
    } else {
      const ElemPos p = decode_elem(m, e2);
      long long qq = 0;
      const int kind = face_neighbor(m, p, d, side, &qq);
      nb = kind == 0 ? (int)qq : (kind == 1 ? NB_BOUNDARY : NB_INTERFACE);
      pos_ix = p.ix;
      pos_f = p.iz * m.ny + p.iy;
    }
    T L[15];
    if (nb == NB_INTERFACE) {
      const T* src = (blk2 ? Lm : Ls) + (long long)pos_f * 15 * NP2 + ab;
#pragma unroll
      for (int kk = 0; kk < 15; ++kk) L[kk] = src[kk * NP2];
      rotate_grad_z(L, ec, -es);
    } else {
      const T* ge = geo + e2 * 13 * NN + vn;
      const T sg = side ? T(1) : T(-1);
      const T Nv[3] = {sg * ge[(3 * d) * NN], sg * ge[(3 * d + 1) * NN], sg * ge[(3 * d + 2) * NN]};
      T uin[5], uout[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) uin[v] = U[e2 * 5 * NN + v * NN + vn];
      rotate_state_z(uin, ec, -es);
      if (nb >= 0) {
        const T* Un = U + (long long)nb * 5 * NN + sab + (side ? 0 : N) * sn;
#pragma unroll
        for (int v = 0; v < 5; ++v) uout[v] = Un[v * NN];
        rotate_state_z(uout, ec, -es);
        const int iy = pos_f % m.ny;
        if (rotating_geom(m.geom) && d == 0 && ((side && iy == m.ny - 1) || (!side && iy == 0)))
          rotate_state_z(uout, c[MC_PCOS], side ? c[MC_PSIN] : -c[MC_PSIN]);
      } else if (rotating_geom(m.geom)) {
        const T isJ = Prec<T>::rcp(Prec<T>::sqrt_(Nv[0] * Nv[0] + Nv[1] * Nv[1] + Nv[2] * Nv[2]));
        const T nrm[3] = {Nv[0] * isJ, Nv[1] * isJ, Nv[2] * isJ};
        const T mn = uin[1] * nrm[0] + uin[2] * nrm[1] + uin[3] * nrm[2];
        uout[0] = uin[0];
#pragma unroll
        for (int q3 = 0; q3 < 3; ++q3) uout[1 + q3] = uin[1 + q3] - T(2) * mn * nrm[q3];
        uout[4] = uin[4];
      } else {
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
      const T Qm[5] = {T(0.5) * (uin[0] + uout[0]), T(0.5) * (qi.u[0] + qo.u[0]), T(0.5) * (qi.u[1] + qo.u[1]),
                       T(0.5) * (qi.u[2] + qo.u[2]), T(0.5) * (qi.p + qo.p)};
#pragma unroll
      for (int aa = 0; aa < 3; ++aa)
#pragma unroll
        for (int v = 0; v < 5; ++v) L[aa * 5 + v] = Qm[v] * Nv[aa];
    }
#pragma unroll
    for (int kk = 0; kk < 15; ++kk) sS[((l2 * 6 + fc2) * 15 + kk) * NP2 + ab] = L[kk];
  }
  T g[15];
  const T* ge = geo + e * 13 * NN + nd;
  // the three passes stay rolled: unrolled, g lives in registers instead of local memory, but
  // the kernel then takes 54 registers instead of 40, two 512-thread CTAs per SM instead of
  // three, and the cylinder's lifting and interface kernels 1.506 instead of 1.301 ms per stage
#pragma unroll 1
  for (int a = 0; a < 3; ++a) {
    if (active) {
      T* Fe = sF + le * 15 * NN;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T Ja = ge[(3 * d + a) * NN];
#pragma unroll
        for (int v = 0; v < 5; ++v) Fe[(5 * d + v) * NN + nd] = Ja * Q[v];
      }
    }
    __syncthreads();
    contract_lines_inplace<N, T>(sF, tid);
    __syncthreads();
    if (active) {
      const T* Fe = sF + le * 15 * NN;
      const T* Se = sS + le * 6 * 15 * NP2;
      const T iw0 = c[MC_IW0];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        T acc = Fe[v * NN + nd] + Fe[(5 + v) * NN + nd] + Fe[(10 + v) * NN + nd];
        if (i == 0) acc += iw0 * Se[(0 * 15 + a * 5 + v) * NP2 + j + NP * k];
        if (i == N) acc += iw0 * Se[(1 * 15 + a * 5 + v) * NP2 + j + NP * k];
        if (j == 0) acc += iw0 * Se[(2 * 15 + a * 5 + v) * NP2 + i + NP * k];
        if (j == N) acc += iw0 * Se[(3 * 15 + a * 5 + v) * NP2 + i + NP * k];
        if (k == 0) acc += iw0 * Se[(4 * 15 + a * 5 + v) * NP2 + i + NP * j];
        if (k == N) acc += iw0 * Se[(5 * 15 + a * 5 + v) * NP2 + i + NP * j];
        g[a * 5 + v] = acc;
      }
    }
    __syncthreads();
  }
  if (!active) return;
  const T invJ = Prec<T>::rcp(ge[9 * NN]);
#pragma unroll
  for (int kk = 0; kk < 15; ++kk) g[kk] *= invJ;
  rotate_grad_z(g, fc, fs);
#pragma unroll
  for (int kk = 0; kk < 15; ++kk) Gr[(e * 15 + kk) * NN + nd] = g[kk];
}

template <int N> struct CurvedLiftCfg {
  template <typename T> static constexpr size_t smem_bytes() {
    using C = ElemCfg<N>;
    return sizeof(T) * (size_t)(C::EPB * 15 * C::NN + C::EPB * 90 * C::NP2);
  }
};

// Fused sliding-interface kernel (Sec. 3.3, steps 3-5, with the mortar operators of
// Sec. 3.2 and the index relation of Sec. 4.3, Eq. indices).
//
// One CTA owns a tile of TF consecutive static faces (i0 .. i0+TF-1) of one perpendicular
// line i_perp.  It stages in shared memory
//   - the static traces of faces i0 .. i0+TF (one halo face),
//   - the moving traces of faces i0-n-1 .. i0+TF-n-1 (mod n_par),
// computes the 2 TF + 1 mortars (i0+r, i_sub) for r < TF and the halo mortar (i0+TF, 0):
// forward projection of both traces along the sliding direction (perpendicular direction
// is the identity), Riemann flux with the static outward normal +x times the face's
// surface element, then projects back conservatively onto the TF static faces and the TF
// moving faces i0-n .. i0+TF-1-n, each of which finds both of its mortars in the tile.
// Every face is written by exactly one CTA: no atomics.  Face traces are the xi^3 = +1
// layer (static) and xi^3 = -1 layer (moving) of the element, contiguous in the state.
#pragma once

#include "sm_launch.h"

template <int N> struct IfCfg {
  static constexpr int NP = N + 1, NP2 = NP * NP, NN = NP * NP * NP;
#ifdef SM_IF_TF_OVERRIDE
  static constexpr int TF = SM_IF_TF_OVERRIDE;
#else
  static constexpr int TF = N == 1 ? 32 : (N == 2 ? 16 : 8);   // default tile: static faces per CTA
#endif
  static constexpr int THREADS = 256;
  // resident CTAs per SM asked of the register allocator for the FP32 Euler tile
  static constexpr int MINB = 4;
  static constexpr int TF_NS = 4;   // tile of the Navier-Stokes flux mode (gradient traces staged too)
  template <typename T, int TFV = TF, int MODE = 0> static constexpr size_t smem_bytes() {
    // Euler: operators + both sides' projected traces on the 2 TF + 1 mortars; the other
    // modes also stage the face traces (and the gradient traces)
    return MODE == 0 ? sizeof(T) * (size_t)(8 * NP2 + 2 * (2 * TFV + 1) * 5 * NP2)
                     : sizeof(T) * (size_t)(8 * NP2 + 2 * (TFV + 1) * 5 * NP2 +
                                            (MODE == 1 ? 2 * (TFV + 1) * 15 * NP2 : 0) + (2 * TFV + 1) * 5 * NP2);
  }
};

// NP consecutive values of a node row; 8-byte accesses where rows are 8-byte aligned (FP32
// with an even row length: every row offset in the state, the face fluxes and the operator
// tables is then even).
template <int NP, typename T> __device__ __forceinline__ void ld_row(const T* __restrict__ p, T* r) {
  if constexpr (sizeof(T) == 4 && NP % 2 == 0) {
#pragma unroll
    for (int i = 0; i < NP / 2; ++i) {
      const float2 v = reinterpret_cast<const float2*>(p)[i];
      r[2 * i] = v.x;
      r[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NP; ++i) r[i] = p[i];
  }
}
template <int NP, typename T> __device__ __forceinline__ void st_row(T* __restrict__ p, const T* r) {
  if constexpr (sizeof(T) == 4 && NP % 2 == 0) {
#pragma unroll
    for (int i = 0; i < NP / 2; ++i) reinterpret_cast<float2*>(p)[i] = make_float2(r[2 * i], r[2 * i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < NP; ++i) p[i] = r[i];
  }
}

// Euler flux tile, three phases over the tile's 2 TF + 1 mortars:
//   1. one work item per (mortar, side, row q, variable): the face's trace row goes from
//      HBM into registers and is projected along the sliding direction (Sec. 3.2, Eq.
//      projection_domain_mortar) with the side's operator rows, broadcast from shared
//      memory; the projected row is stored in shared memory;
//   2. one work item per mortar node: Riemann flux of the two projected states, times the
//      surface element, in place of the static side's projection;
//   3. one work item per (side, face, row q, variable): the face's two mortar flux rows are
//      projected back (Eq. projection_mortar_domain) and written to the face flux array.
// The traces come from the compact arrays Ts / Tm ([n_perp][n_par][5][(N+1)^2], the face
// fluxes' layout) when given, else from the element node layers of U.
template <int N, typename T, int RIEM, int TF>
__device__ __forceinline__ void interface_tile_euler(const MeshDev& m, const StageParams* __restrict__ sp,
                                                     const T* __restrict__ U, T* __restrict__ Fs,
                                                     T* __restrict__ Fm, const int tile_x, const int iz,
                                                     const T* __restrict__ Ts, const T* __restrict__ Tm) {
  using C = IfCfg<N>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN, THREADS = C::THREADS, NM = 2 * TF + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sMat = reinterpret_cast<T*>(smem_raw);   // [8][NP2]
  T* sQ = sMat + 8 * NP2;                     // [side][NM][5][NP2]; side 0 then holds the mortar fluxes
  __shared__ long long s_base[2][TF + 1];

  const int tid = threadIdx.x;
  const int i0 = tile_x * TF;
  const int ny = m.ny;
  const int TFe = min(TF, ny - i0);
  const int nmort = 2 * TFe + 1;
  long long nl = sp->n % ny;
  const int nmod = (int)(nl < 0 ? nl + ny : nl);

  for (int w = tid; w < 8 * NP2; w += THREADS) {
    const int k = w / NP2, r = w - k * NP2;
    sMat[w] = Prec<T>::mat(sp, k)[r];
  }
  // trace base offsets: static faces i0+r and moving faces i0-n-1+r (mod n_par), r = 0..TFe;
  // in U a static trace is its element's xi^3 = +1 node layer, a moving one the xi^3 = -1 layer
  const bool compact = Ts != nullptr;
  const int vstride = compact ? NP2 : NN;
  if (tid < 2 * (TFe + 1)) {
    const int side = tid / (TFe + 1), r = tid - side * (TFe + 1);
    int f = side ? i0 - nmod - 1 + r : i0 + r;
    f %= ny;
    if (f < 0) f += ny;
    s_base[side][r] = compact ? ((long long)iz * ny + f) * 5 * NP2
                              : encode_elem(m, side, side ? 0 : m.nxs - 1, f, iz) * 5 * NN + (side ? 0 : NP2 * N);
  }
  __syncthreads();

  // 1. projections, one (mortar, side, row q, variable) per work item; mortar mi = 2 r + i_sub
  // meets static face r and moving face r + i_sub
  for (int w = tid; w < nmort * 2 * NP * 5; w += THREADS) {
    const int q = w % NP;
    int rest = w / NP;
    const int v = rest % 5;
    rest /= 5;
    const int side = rest & 1, mi = rest >> 1;
    const int r = mi >> 1, isub = mi & 1;
    T t[NP];
    ld_row<NP>((compact ? (side ? Tm : Ts) : U) + s_base[side][r + side * isub] + v * vstride + q * NP, t);
    // the static lower mortar meets the moving face's upper part and vice versa
    const T* P = sMat + (side ? (isub ? 2 : 3) : (isub ? 1 : 0)) * NP2;
    T o[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      T pr[NP];
      ld_row<NP>(P + j * NP, pr);
      T acc = T(0);
#pragma unroll
      for (int i = 0; i < NP; ++i) acc += pr[i] * t[i];
      o[j] = acc;
    }
    st_row<NP>(sQ + ((side * NM + mi) * 5 + v) * NP2 + q * NP, o);
  }
  __syncthreads();

  // 2. mortar Riemann fluxes, static outward normal +x, times the surface element
  const T sJ = Prec<T>::c(m)[MC_SJ_IF];
  const T gamma = Prec<T>::c(m)[MC_GAMMA];
  for (int w = tid; w < nmort * NP2; w += THREADS) {
    const int mi = w / NP2, ab = w - mi * NP2;
    T* qs = sQ + (mi * 5) * NP2 + ab;
    const T* qm = sQ + ((NM + mi) * 5) * NP2 + ab;
    T QL[5], QR[5], F[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      QL[v] = qs[v * NP2];
      QR[v] = qm[v * NP2];
    }
    riemann_axis<T, 0, RIEM>(QL, QR, T(0), gamma, F);
#pragma unroll
    for (int v = 0; v < 5; ++v) qs[v * NP2] = F[v] * sJ;
  }
  __syncthreads();

  // 3. back-projection, one (side, face, row q, variable) per work item: static face i0+r
  // from mortars (2r, 2r+1); moving face i0-n+r from mortars 2r+1 (its lower part) and 2r+2
  // (its upper part), with the opposite sign
  for (int w = tid; w < 2 * TFe * NP * 5; w += THREADS) {
    const int q = w % NP;
    int rest = w / NP;
    const int v = rest % 5;
    rest /= 5;
    const int side = rest >= TFe;
    const int r = rest - side * TFe;
    T a[NP], b[NP], o[NP];
    ld_row<NP>(sQ + ((2 * r + side) * 5 + v) * NP2 + q * NP, a);
    ld_row<NP>(sQ + ((2 * r + 1 + side) * 5 + v) * NP2 + q * NP, b);
    const T* Blo = sMat + (side ? 6 : 4) * NP2;
    const T* Bhi = sMat + (side ? 7 : 5) * NP2;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      T bl[NP], bh[NP];
      ld_row<NP>(Blo + i * NP, bl);
      ld_row<NP>(Bhi + i * NP, bh);
      T acc = T(0);
#pragma unroll
      for (int jj = 0; jj < NP; ++jj) acc += bl[jj] * a[jj] + bh[jj] * b[jj];
      o[i] = side ? -acc : acc;
    }
    int f = side ? i0 - nmod + r : i0 + r;
    f %= ny;
    if (f < 0) f += ny;
    st_row<NP>((side ? Fm : Fs) + (((long long)iz * ny + f) * 5 + v) * NP2 + q * NP, o);
  }
}

// Interface tile modes: Euler flux, Navier-Stokes flux (BR1 viscous mean of both sides'
// projected gradients on each mortar, Sec. 3.2), lifting (mortar mean of both sides'
// projected primitive traces, the BR1 face value of the gradient computation).
enum { IF_EULER = 0, IF_NS = 1, IF_LIFT = 2 };

// Staged tile (lifting and Navier-Stokes flux): static faces tile_x * TF .. +TF-1 of line iz,
// face traces staged in shared memory, one thread per mortar node.  In IF_LIFT mode Fs / Fm receive
// the lifting face values; IF_NS reads the lifted gradients Gr.
template <int N, typename T, int RIEM, int TF, int MODE>
__device__ __forceinline__ void interface_tile_staged(const MeshDev& m, const StageParams* __restrict__ sp,
                                               const T* __restrict__ U, T* __restrict__ Fs, T* __restrict__ Fm,
                                               const int tile_x, const int iz, const T* __restrict__ Gr = nullptr) {
  using C = IfCfg<N>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN, THREADS = C::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sMat = reinterpret_cast<T*>(smem_raw);          // [8][NP2]
  T* sTs = sMat + 8 * NP2;                           // [TF+1][5][NP2] static traces
  T* sTm = sTs + (TF + 1) * 5 * NP2;                 // [TF+1][5][NP2] moving traces
  T* sGs = sTm + (TF + 1) * 5 * NP2;                 // [TF+1][15][NP2] static gradient traces (IF_NS)
  T* sGm = sGs + (MODE == IF_NS ? (TF + 1) * 15 * NP2 : 0);
  T* sFm = sGm + (MODE == IF_NS ? (TF + 1) * 15 * NP2 : 0);   // [2TF+1][5][NP2] mortar fluxes

  const int tid = threadIdx.x;
  const int i0 = tile_x * TF;
  const int ny = m.ny;
  const int TFe = min(TF, ny - i0);
  long long nl = sp->n % ny;
  const int nmod = (int)(nl < 0 ? nl + ny : nl);

  for (int w = tid; w < 8 * NP2; w += THREADS) {
    const int k = w / NP2, r = w - k * NP2;
    sMat[w] = Prec<T>::mat(sp, k)[r];
  }
  // traces: static faces i0+r (r = 0..TFe) and moving faces i0-n-1+r (r = 0..TFe); the
  // trace of a face is its element's xi^3 = +1 (static) or -1 (moving) node layer, (N+1)^2
  // contiguous values per variable
  __shared__ long long s_base[2][TF + 1];
  if (tid < 2 * (TFe + 1)) {
    const int side = tid / (TFe + 1), r = tid - side * (TFe + 1);
    int f = side ? i0 - nmod - 1 + r : i0 + r;
    f %= ny;
    if (f < 0) f += ny;
    s_base[side][r] = encode_elem(m, side, side ? 0 : m.nxs - 1, f, iz) * 5 * NN + (side ? 0 : NP2 * N);
  }
  __syncthreads();
  const int ntr = (TFe + 1) * 5 * NP2;
  if constexpr (sizeof(T) == 4 && NP2 % 4 == 0) {
    // 16-byte loads: the layer offsets and (N+1)^3 are multiples of 4 values
    constexpr int Q4 = NP2 / 4;
    const int nv = 2 * (TFe + 1) * 5 * Q4;
    for (int w = tid; w < nv; w += THREADS) {
      const int q4 = w % Q4;
      const int rest = w / Q4;
      const int v = rest % 5;
      const int sr = rest / 5;                   // side * (TFe+1) + r
      const int side = sr >= TFe + 1, r = sr - side * (TFe + 1);
      const float4 val = *reinterpret_cast<const float4*>(U + s_base[side][r] + v * NN + 4 * q4);
      *reinterpret_cast<float4*>((side ? sTm : sTs) + (r * 5 + v) * NP2 + 4 * q4) = val;
    }
  } else {
    for (int w = tid; w < 2 * ntr; w += THREADS) {
      const int side = w >= ntr;
      const int ww = w - side * ntr;
      const int r = ww / (5 * NP2);
      const int rem = ww - r * 5 * NP2;
      (side ? sTm : sTs)[ww] = U[s_base[side][r] + rem / NP2 * NN + rem % NP2];
    }
  }
  if (MODE == IF_NS) {
    // gradient traces: the same node layers of the 15 lifted components
    const int ngr = 2 * (TFe + 1) * 15 * NP2;
    for (int w = tid; w < ngr; w += THREADS) {
      const int ab = w % NP2;
      const int rest = w / NP2;
      const int kk = rest % 15;
      const int sr = rest / 15;
      const int side = sr >= TFe + 1, r = sr - side * (TFe + 1);
      const long long eb = s_base[side][r] / (5 * NN);            // element index
      const int layer = side ? 0 : NP2 * N;
      (side ? sGm : sGs)[(r * 15 + kk) * NP2 + ab] = Gr[(eb * 15 + kk) * NN + layer + ab];
    }
  }
  __syncthreads();
  if (MODE == IF_LIFT) {
    // primitive traces (rho, v, p) in place
    const T gam = Prec<T>::c(m)[MC_GAMMA];
    for (int w = tid; w < 2 * (TFe + 1) * NP2; w += THREADS) {
      const int side = w >= (TFe + 1) * NP2;
      const int ww = w - side * (TFe + 1) * NP2;
      const int r = ww / NP2, ab = ww - r * NP2;
      T* t = (side ? sTm : sTs) + r * 5 * NP2 + ab;
      T u[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) u[v] = t[v * NP2];
      const Prim<T> q = primitives(u, gam);
      t[NP2] = q.u[0];
      t[2 * NP2] = q.u[1];
      t[3 * NP2] = q.u[2];
      t[4 * NP2] = q.p;
    }
    __syncthreads();
  }

  // mortars mi = 2 r + i_sub for r < TFe, plus mi = 2 TFe (the halo mortar (i0+TFe, 0))
  const T sJ = Prec<T>::c(m)[MC_SJ_IF];
  const T gamma = Prec<T>::c(m)[MC_GAMMA];
  for (int w = tid; w < (2 * TFe + 1) * NP2; w += THREADS) {
    const int mi = w / NP2, ab = w - mi * NP2;
    const int r = mi >> 1, isub = mi & 1;
    const int j = ab % NP, q = ab / NP;
    // static lower mortar meets the moving face's upper part and vice versa
    const T* Ps = sMat + (isub ? 1 : 0) * NP2 + j * NP;
    const T* Pm = sMat + (isub ? 2 : 3) * NP2 + j * NP;
    const T* ts = sTs + r * 5 * NP2 + q * NP;
    const T* tm = sTm + (r + isub) * 5 * NP2 + q * NP;   // partner i - n + i_sub - 1
    T QL[5], QR[5], F[5];
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
    if (MODE == IF_LIFT) {
#pragma unroll
      for (int v = 0; v < 5; ++v) sFm[(mi * 5 + v) * NP2 + ab] = sJ * T(0.5) * (QL[v] + QR[v]);
      continue;
    }
    riemann_axis<T, 0, RIEM>(QL, QR, T(0), gamma, F);
    if (MODE == IF_NS) {
      T GL[15], GR[15], fvl[5], fvr[5];
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
      viscous_flux_axis(QL, GL, 0, Prec<T>::c(m), fvl);
      viscous_flux_axis(QR, GR, 0, Prec<T>::c(m), fvr);
#pragma unroll
      for (int v = 0; v < 5; ++v) F[v] -= T(0.5) * (fvl[v] + fvr[v]);
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) sFm[(mi * 5 + v) * NP2 + ab] = F[v] * sJ;
  }
  __syncthreads();

  // back-projection: static faces i0+r from mortars (2r, 2r+1); moving faces i0-n+r from
  // mortars (2r+1) [its lower part] and (2r+2) [its upper part], with the opposite sign.
  for (int w = tid; w < 2 * TFe * NP2; w += THREADS) {
    const int side = w >= TFe * NP2;
    const int ww = w - side * TFe * NP2;
    const int r = ww / NP2, ab = ww - r * NP2;
    const int i = ab % NP, q = ab / NP;
    const T* Blo = sMat + (side ? 6 : 4) * NP2 + i * NP;
    const T* Bhi = sMat + (side ? 7 : 5) * NP2 + i * NP;
    const T* flo = sFm + (2 * r + side) * 5 * NP2 + q * NP;
    const T* fhi = sFm + (2 * r + 1 + side) * 5 * NP2 + q * NP;
    int f = side ? i0 - nmod + r : i0 + r;
    f %= ny;
    if (f < 0) f += ny;
    T* dst = (side ? Fm : Fs) + (((long long)iz * ny + f) * 5) * NP2 + ab;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      T acc = T(0);
#pragma unroll
      for (int jj = 0; jj < NP; ++jj) acc += Blo[jj] * flo[v * NP2 + jj] + Bhi[jj] * fhi[v * NP2 + jj];
      dst[v * NP2] = side ? -acc : acc;
    }
  }
}


// One tile of any mode: the Euler flux takes the register-blocked form, lifting and the
// Navier-Stokes flux the staged form.
template <int N, typename T, int RIEM, int TF, int MODE = IF_EULER>
__device__ __forceinline__ void interface_tile(const MeshDev& m, const StageParams* __restrict__ sp,
                                               const T* __restrict__ U, T* __restrict__ Fs, T* __restrict__ Fm,
                                               const int tile_x, const int iz, const T* __restrict__ Gr = nullptr,
                                               const T* __restrict__ Ts = nullptr, const T* __restrict__ Tm = nullptr) {
  if constexpr (MODE == IF_EULER)
    interface_tile_euler<N, T, RIEM, TF>(m, sp, U, Fs, Fm, tile_x, iz, Ts, Tm);
  else
    interface_tile_staged<N, T, RIEM, TF, MODE>(m, sp, U, Fs, Fm, tile_x, iz, Gr);
}

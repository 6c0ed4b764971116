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
  static constexpr int TF = N == 1 ? 32 : (N == 2 ? 16 : 8);   // default tile: static faces per CTA
  static constexpr int THREADS = 256;
  template <typename T, int TFV = TF> static constexpr size_t smem_bytes() {
    return sizeof(T) * (size_t)(8 * NP2 + 2 * (TFV + 1) * 5 * NP2 + (2 * TFV + 1) * 5 * NP2);
  }
};

// One tile: static faces tile_x * TF .. +TF-1 of perpendicular line iz.  Shared by the
// single-solve kernel and the batched persistent kernel.
template <int N, typename T, int RIEM, int TF>
__device__ __forceinline__ void interface_tile(const MeshDev& m, const StageParams* __restrict__ sp,
                                               const T* __restrict__ U, T* __restrict__ Fs, T* __restrict__ Fm,
                                               const int tile_x, const int iz) {
  using C = IfCfg<N>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN, THREADS = C::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sMat = reinterpret_cast<T*>(smem_raw);          // [8][NP2]
  T* sTs = sMat + 8 * NP2;                           // [TF+1][5][NP2] static traces
  T* sTm = sTs + (TF + 1) * 5 * NP2;                 // [TF+1][5][NP2] moving traces
  T* sFm = sTm + (TF + 1) * 5 * NP2;                 // [2TF+1][5][NP2] mortar fluxes

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
  // traces: static faces i0+r (r = 0..TFe) and moving faces i0-n-1+r (r = 0..TFe)
  const int ntr = (TFe + 1) * 5 * NP2;
  for (int w = tid; w < 2 * ntr; w += THREADS) {
    const int side = w >= ntr;
    const int ww = w - side * ntr;
    const int r = ww / (5 * NP2);
    const int rem = ww - r * 5 * NP2;
    const int v = rem / NP2, ab = rem - v * NP2;
    int f = side ? i0 - nmod - 1 + r : i0 + r;
    f %= ny;
    if (f < 0) f += ny;
    const long long e = encode_elem(m, side, side ? 0 : m.nxs - 1, f, iz);
    const T val = U[(e * 5 + v) * NN + (side ? 0 : NP2 * N) + ab];
    (side ? sTm : sTs)[ww] = val;
  }
  __syncthreads();

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
    riemann_axis<T, 0, RIEM>(QL, QR, T(0), gamma, F);
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


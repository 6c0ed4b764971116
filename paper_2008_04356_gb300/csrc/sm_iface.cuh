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
  const int nmod = sp->n_mod;

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

// Register-fused Euler tile (FP32 state, N odd): the three steps of Sec. 3.3 with few
// shared-memory round trips, in persistent CTAs that prefetch the traces of the next two
// tiles with 16-byte cp.async while they compute the current one.  Per tile (TF static faces of one
// perpendicular line plus one halo face per side):
//   A. two threads per (mortar, row q), each for half of the row's NP mortar nodes: both
//      sides' traces of all five variables are projected onto those nodes (Eq.
//      projection_domain_mortar) into registers, as float pairs (static, moving) updated by
//      packed FMAs, and the Riemann flux of each node follows at once, times the surface
//      element;
//   B. two threads per (side, face, row q), each for half of the row's face nodes: the
//      face's two mortar flux rows are projected back (Eq. projection_mortar_domain; pairs
//      (lower, upper mortar) summed at the end) into shared output blocks, which the CTA
//      then copies to the face flux arrays with coalesced 16-byte stores.
// A mortar's arithmetic does not depend on the tile it sits in (the halo mortar is computed
// by both neighbouring tiles with the same operations), so results are independent of TF.
// Lanes of a warp: in A 16 consecutive mortars x the two halves of one row (both halves
// read the same trace values), in B 8 faces x 2 sides x 2 halves of one row; face blocks
// at 4 mod 32 words, mortar blocks at 2 mod 32 and the operator tables 16 apart keep the
// accesses of a warp in distinct banks.
template <int N, int TFV> struct IfFusedCfg {
  static_assert(N % 2 == 1, "the fused interface tile takes odd N (16-byte face blocks)");
  static_assert(TFV % 8 == 0, "the fused interface tile takes TF = 8 k");
  static constexpr int NP = N + 1, NP2 = NP * NP, NN = NP * NP * NP;
  static constexpr int TF = TFV;
  static constexpr int NM = 2 * TF + 1;
  static constexpr int H0 = NP / 2;                              // node halves of a row
  static constexpr int NBA = 2 * TF / 16;                        // 16-mortar blocks (A)
  static constexpr int NBB = TF / 8;                             // 8-face blocks (B)
  static constexpr int ITEMS_A = 32 * NBA * NP + 2 * NP;         // + the halo mortar
  static constexpr int ITEMS_B = 32 * NBB * NP;
  static constexpr int THREADS = ((ITEMS_A + 31) / 32) * 32;
  // resident CTAs per SM asked of the register allocator (about 80 registers a thread)
#ifndef SM_IF_FUSED_REGS
#define SM_IF_FUSED_REGS 80
#endif
  static constexpr int MINB = 65536 / (THREADS * SM_IF_FUSED_REGS) > 0 ? 65536 / (THREADS * SM_IF_FUSED_REGS) : 1;
  static constexpr int TB = 5 * NP2;                             // one face's block (floats)
#ifndef SM_IF_FUSED_PAD
#define SM_IF_FUSED_PAD 1
#endif
  // face block stride: = 4 mod 32 (16-byte rows, conflict-free phase B stores), or unpadded
  static constexpr int FS = SM_IF_FUSED_PAD ? TB + (36 - TB % 32) % 32 : TB;
  static constexpr int MS = TB + (34 - TB % 32) % 32;            // = 2 mod 32
  static constexpr int MR = sm_pair_row(NP);
  static constexpr int MT = sm_pair_stride(NP);
  static constexpr int TBUF = 4 * MT + 2 * (TF + 1) * FS;        // one prefetch buffer (floats)
  static constexpr int SFSZ = ((NM * MS + 3) / 4) * 4;           // mortar fluxes
  static constexpr int OSZ = 2 * TF * FS;                        // output blocks
#ifndef SM_IF_FUSED_NBUF
#define SM_IF_FUSED_NBUF 3
#endif
  static constexpr int NBUF = SM_IF_FUSED_NBUF;                  // trace buffers: NBUF - 1 tiles ahead
  static constexpr size_t smem_floats = (size_t)NBUF * TBUF + SFSZ + OSZ;
  static constexpr size_t smem_bytes = sizeof(float) * smem_floats;
};
// default tile width of the single-solve FP32 launch (the batch autotuner picks 8 or 16)
#ifndef SM_IF_FUSED_TF
#define SM_IF_FUSED_TF 8
#endif
template <int N> struct IfFusedTF { static constexpr int TF = SM_IF_FUSED_TF; };

__device__ __forceinline__ void cp_async_4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory");
}
// Issues the asynchronous copies of one tile into buffer sB: the operator pair tables and the
// traces of static faces i0 + r and moving faces i0 - n - 1 + r (mod n_par), r = 0..TFe,
// from the compact arrays Ts / Tm or, when they are NULL, from the element node layers of U
// (xi^3 = +1 static, xi^3 = -1 moving).
template <int N, int TF>
__device__ __forceinline__ void fused_tile_stage(const MeshDev& m, const StageParams* __restrict__ sp,
                                                 const float* __restrict__ U, const float* __restrict__ Ts,
                                                 const float* __restrict__ Tm, const int tile_x, const int iz,
                                                 float* sB, const int tid) {
  using C = IfFusedCfg<N, TF>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN, THREADS = C::THREADS;
  constexpr int FS = C::FS, MT = C::MT, TB = C::TB;
  const int ny = m.ny;
  const int i0 = tile_x * TF;
  const int TFe = min(TF, ny - i0);
  const int nmod = sp->n_mod;
  for (int w = tid; w < MT; w += THREADS) cp_async_16(sB + 4 * w, sp->pair_f + 4 * w);
  float* sT = sB + 4 * MT;
  const int nslot = 2 * (TFe + 1);
  if (Ts) {
    // compact traces: a face's 5 (N+1)^2 values are contiguous, TB / 4 chunks of 16 bytes;
    // thread = (chunk, slot group)
    constexpr int NC = TB / 4;
    constexpr int G = THREADS / NC;
    if (tid < G * NC) {
      const int c = tid % NC;
      for (int slot = tid / NC; slot < nslot; slot += G) {
        const int side = slot > TFe, r = slot - side * (TFe + 1);
        int f = side ? i0 - nmod - 1 + r : i0 + r;
        f = f < 0 ? f + ny : (f >= ny ? f - ny : f);
        cp_async_16(sT + (side * (TF + 1) + r) * FS + 4 * c, (side ? Tm : Ts) + ((long long)iz * ny + f) * TB + 4 * c);
      }
    }
  } else {
    constexpr int NV = NP2 / 2;
    for (int w = tid; w < nslot * 5 * NV; w += THREADS) {
      const int k = w % NV;
      const int rest = w / NV;
      const int v = rest % 5;
      const int sr = rest / 5;
      const int side = sr >= TFe + 1, r = sr - side * (TFe + 1);
      int f = side ? i0 - nmod - 1 + r : i0 + r;
      f = f < 0 ? f + ny : (f >= ny ? f - ny : f);
      const float* src = U + encode_elem(m, side, side ? 0 : m.nxs - 1, f, iz) * 5 * NN + (side ? 0 : NP2 * N) +
                         (long long)v * NN + 2 * k;
      cp_async_8(sT + (side * (TF + 1) + r) * FS + v * NP2 + 2 * k, src);
    }
  }
}

// Phase A for the NH mortar nodes j0 .. j0+NH-1 of row q of mortar mi.
template <int N, int RIEM, int TF, int NH>
__device__ __forceinline__ void fused_mortar_nodes(const float* sB, float* sF, const int mi, const int q,
                                                   const int j0, const float sJ, const float gamma) {
  using C = IfFusedCfg<N, TF>;
  constexpr int NP = C::NP, NP2 = C::NP2, FS = C::FS, MS = C::MS, MR = C::MR, MT = C::MT;
  const int isub = mi & 1, rs = mi >> 1, rm = rs + isub;
  const float* sT = sB + 4 * MT;
  const float* ts = sT + rs * FS + q * NP;
  const float* tm = sT + (TF + 1 + rm) * FS + q * NP;
  // the static lower mortar meets the moving face's upper part and vice versa
  const float2* PF = reinterpret_cast<const float2*>(sB + isub * MT) + j0;
  float2 acc[5][NH];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int j = 0; j < NH; ++j) acc[v][j] = make_float2(0.f, 0.f);
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    float2 pp[NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) pp[j] = PF[i * MR + j];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const float2 ab = make_float2(ts[v * NP2 + i], tm[v * NP2 + i]);
#pragma unroll
      for (int j = 0; j < NH; ++j) acc[v][j] = __ffma2_rn(pp[j], ab, acc[v][j]);
    }
  }
  float* out = sF + mi * MS + q * NP + j0;
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    float QL[5], QR[5], F[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) { QL[v] = acc[v][j].x; QR[v] = acc[v][j].y; }
    riemann_axis<float, 0, RIEM>(QL, QR, 0.f, gamma, F);
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v * NP2 + j] = F[v] * sJ;
  }
}

// Phase B for the NH face nodes i0n .. i0n+NH-1 of row q of face r on one side, into the
// face's shared output block o (the row's first node).
template <int N, int TF, int NH>
__device__ __forceinline__ void fused_face_nodes(const float* sB, const float* sF, float* o, const int r,
                                                 const int side, const int q, const int i0n) {
  using C = IfFusedCfg<N, TF>;
  constexpr int NP = C::NP, NP2 = C::NP2, MS = C::MS, MR = C::MR, MT = C::MT;
  const float* flo = sF + (2 * r + side) * MS + q * NP;
  const float* fhi = flo + MS;
  const float2* PB = reinterpret_cast<const float2*>(sB + (2 + side) * MT) + i0n;
  float2 acc[5][NH];
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int i = 0; i < NH; ++i) acc[v][i] = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    float2 bb[NH];
#pragma unroll
    for (int i = 0; i < NH; ++i) bb[i] = PB[j * MR + i];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const float2 ab = make_float2(flo[v * NP2 + j], fhi[v * NP2 + j]);
#pragma unroll
      for (int i = 0; i < NH; ++i) acc[v][i] = __ffma2_rn(bb[i], ab, acc[v][i]);
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v)
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      const float x = acc[v][i].x + acc[v][i].y;
      o[v * NP2 + i0n + i] = side ? -x : x;
    }
}

// Phases A and B of one tile whose buffer sB has landed (see fused_tile_stage), into the
// output blocks sO; ends with a barrier, after which sB and sF are free.
template <int N, int RIEM, int TF>
__device__ __forceinline__ void fused_tile_compute(const MeshDev& m, const StageParams* __restrict__ sp,
                                                   float* __restrict__ Fs, float* __restrict__ Fm, const int tile_x,
                                                   const int iz, const float* sB, float* sF, float* sO, const int tid) {
  using C = IfFusedCfg<N, TF>;
  constexpr int NP = C::NP, NP2 = C::NP2, H0 = C::H0, FS = C::FS, TB = C::TB;
  const int ny = m.ny;
  const int i0 = tile_x * TF;
  const int TFe = min(TF, ny - i0);
  const int nme = 2 * TFe + 1;
  const int nmod = sp->n_mod;

  // A. projections of both sides and the mortar Riemann fluxes (static outward normal +x)
  const float sJ = m.cf[MC_SJ_IF];
  const float gamma = m.cf[MC_GAMMA];
  if (tid < C::ITEMS_A) {
    int mi, q, h;
    if (tid < 32 * C::NBA * NP) {
      const int rest = tid >> 5;
      mi = 16 * (rest / NP) + (tid & 15);
      q = rest % NP;
      h = (tid >> 4) & 1;
    } else {
      const int hw = tid - 32 * C::NBA * NP;   // the halo mortar 2 TF
      mi = 2 * TF;
      q = hw % NP;
      h = hw / NP;
    }
    // both halves in one call (H0 = H1): the two half-warps run the same instructions
    if (mi < nme) fused_mortar_nodes<N, RIEM, TF, H0>(sB, sF, mi, q, h * H0, sJ, gamma);
  }
  __syncthreads();

  // B. back-projection: static face i0 + r from mortars (2r, 2r+1); moving face i0 - n + r
  // from mortars 2r+1 (its lower part) and 2r+2 (its upper part), with the opposite sign
  if (tid < C::ITEMS_B) {
    const int rest = tid >> 5;
    const int r = 8 * (rest / NP) + (tid & 7);
    const int q = rest % NP;
    const int side = (tid >> 3) & 1, h = (tid >> 4) & 1;
    if (r < TFe) fused_face_nodes<N, TF, H0>(sB, sF, sO + (side * TF + r) * FS + q * NP, r, side, q, h * H0);
  }
  __syncthreads();
}

// Copies the tile's face flux blocks from sO to the face flux arrays (16-byte stores).
template <int N, int TF>
__device__ __forceinline__ void fused_tile_store(const MeshDev& m, const StageParams* __restrict__ sp,
                                                 float* __restrict__ Fs, float* __restrict__ Fm, const int tile_x,
                                                 const int iz, const float* sO, const int tid) {
  using C = IfFusedCfg<N, TF>;
  constexpr int FS = C::FS, TB = C::TB, THREADS = C::THREADS, NC = TB / 4;
  const int ny = m.ny;
  const int i0 = tile_x * TF;
  const int TFe = min(TF, ny - i0);
  const int nmod = sp->n_mod;
  for (int w = tid; w < 2 * TFe * NC; w += THREADS) {
    const int slot = w / NC, c = w - slot * NC;
    const int side = slot >= TFe, r = slot - side * TFe;
    int f = side ? i0 - nmod + r : i0 + r;
    f = f < 0 ? f + ny : (f >= ny ? f - ny : f);
    const float4 x = *reinterpret_cast<const float4*>(sO + (side * TF + r) * FS + 4 * c);
    *reinterpret_cast<float4*>((side ? Fm : Fs) + ((long long)iz * ny + f) * TB + 4 * c) = x;
  }
}

// Persistent tile pipeline: tiles first, first + stride, ... < total, with the traces of the
// next NBUF - 1 tiles in flight while a tile computes.  stage(item, buffer) issues a tile's
// copies; run(item, buffer) computes it (ending with a barrier) and store(item) writes it.
template <int N, int TF, class Stage, class Run, class Store>
__device__ __forceinline__ void fused_pipeline(const int first, const int stride, const int total, float* sBuf,
                                               Stage stage, Run run, Store store) {
  using C = IfFusedCfg<N, TF>;
  constexpr int NBUF = C::NBUF;
#pragma unroll
  for (int k = 0; k < NBUF - 1; ++k) {
    const int it = first + k * stride;
    if (it < total) stage(it, sBuf + k * C::TBUF);
    cp_async_commit();
  }
  // tile first + k stride sits in buffer k mod NBUF
  int slot = 0;
  for (int t = first; t < total; t += stride) {
    // the buffer of the previous tile (free: its computation ended with a barrier) receives
    // tile t + (NBUF-1) stride; then this tile's group is the oldest of NBUF pending ones
    const int tp = t + (NBUF - 1) * stride;
    if (tp < total) stage(tp, sBuf + (slot == 0 ? NBUF - 1 : slot - 1) * C::TBUF);
    cp_async_commit();
    cp_async_wait<NBUF - 1>();
    __syncthreads();
    run(t, sBuf + slot * C::TBUF);
    store(t);
    slot = slot + 1 == NBUF ? 0 : slot + 1;
  }
  cp_async_wait<0>();
}

// q = t / n, r = t - q n for 0 <= t < 2^24 and n >= 1 from a float estimate (inv = 1 / n),
// corrected by one step either way: cheaper than an integer division by a runtime value.
__device__ __forceinline__ void divmod_small(const int t, const int n, const float inv, int* q, int* r) {
  int qq = __float2int_rz((float)t * inv);
  int rr = t - qq * n;
  if (rr < 0) { --qq; rr += n; }
  else if (rr >= n) { ++qq; rr -= n; }
  *q = qq;
  *r = rr;
}

// The tiles of one solve: (n_par / TF) x n_perp, tile index = tile_x + ntx iz.
template <int N, int RIEM, int TF>
__device__ __forceinline__ void interface_fused_loop(const MeshDev& m, const StageParams* __restrict__ sp,
                                                     const float* __restrict__ U, float* __restrict__ Fs,
                                                     float* __restrict__ Fm, const float* __restrict__ Ts,
                                                     const float* __restrict__ Tm) {
  using C = IfFusedCfg<N, TF>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sBuf = reinterpret_cast<float*>(smem_raw);   // [NBUF][TBUF] trace buffers
  float* sF = sBuf + C::NBUF * C::TBUF;               // [NM][MS] mortar fluxes
  float* sO = sF + C::SFSZ;                           // [2][TF][FS] output blocks
  const int tid = threadIdx.x;
  const int ntx = (m.ny + TF - 1) / TF;
  const float inv = 1.0f / (float)ntx;
  int rx = 0, rz = 0;   // coordinates of the tile being computed
  fused_pipeline<N, TF>(
      blockIdx.x, gridDim.x, ntx * m.nz, sBuf,
      [&](int t, float* dst) {
        int x, z;
        divmod_small(t, ntx, inv, &z, &x);
        fused_tile_stage<N, TF>(m, sp, U, Ts, Tm, x, z, dst, tid);
      },
      [&](int t, const float* sB) {
        divmod_small(t, ntx, inv, &rz, &rx);
        fused_tile_compute<N, RIEM, TF>(m, sp, Fs, Fm, rx, rz, sB, sF, sO, tid);
      },
      [&](int t) { fused_tile_store<N, TF>(m, sp, Fs, Fm, rx, rz, sO, tid); });
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
  const int nmod = sp->n_mod;

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

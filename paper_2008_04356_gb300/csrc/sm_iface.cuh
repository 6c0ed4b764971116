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

// Register-fused Euler tile (FP32 state, N odd) of the batched launch: the three steps of
// Sec. 3.3 with few shared-memory round trips, in persistent CTAs that prefetch the traces
// of the next work item with 16-byte cp.async while they compute the current one.  Per tile
// (TF static faces of one perpendicular line plus one halo face per side):
//   staging: the tile's static faces i0 .. i0+TF and moving faces i0-n-1 .. i0+TF-n-1 are
//      (up to the periodic wrap of the line) contiguous runs of the compact trace arrays,
//      copied as such, with the operator tables;
//   A. one thread per (mortar, row pair, node pair): both sides' traces of all five
//      variables are projected onto two mortar nodes (Eq. projection_domain_mortar) for two
//      rows at once, and the Riemann fluxes of the two nodes follow, times the surface
//      element (mortar_rows);
//   B. one thread per (side, face, row pair, node pair): the face's two mortar flux rows are
//      projected back (Eq. projection_mortar_domain) and stored to the face flux arrays
//      (face_rows).
// The work runs on float pairs over a pair of rows (q, q+1): the compact traces interleave
// the rows of a pair (trace_node) and the operator tables hold every entry duplicated, two
// rows per 16-byte entry, so the operands of the packed multiply-adds (fma.rn.f32x2) of two
// nodes come in 16-byte loads, and the Riemann flux of the two rows is one paired
// evaluation.  A mortar's arithmetic does not depend on the tile it sits in (the halo mortar
// is computed by both neighbouring tiles with the same operations), so results are
// independent of TF and identical to those of the single-solve kernel (warp-owned rows).
#ifndef SM_IF_FUSED_REGS
#define SM_IF_FUSED_REGS 96
#endif
// Each prefetch buffer carries its tile's operator tables (the tiles of a batched launch
// belong to different solves).
template <int N, int TFV> struct IfFusedCfg {
  static_assert(N % 2 == 1, "the fused interface tile takes odd N (rows in pairs)");
  static_assert(TFV % 8 == 0, "the fused interface tile takes TF = 8 k");
  static constexpr int NP = N + 1, NP2 = NP * NP, NN = NP * NP * NP;
  static constexpr int NH = NP / 2;                              // row pairs = node pairs per row
  static constexpr int TF = TFV;
  static constexpr int NM = 2 * TF + 1;
  static constexpr int ITEMS_A = NM * NH * NH;
  static constexpr int ITEMS_B = 2 * TF * NH * NH;
  static constexpr int THREADS = (((ITEMS_A > ITEMS_B ? ITEMS_A : ITEMS_B) + 31) / 32) * 32;
  static constexpr int TB = 5 * NP2;                             // one face's block (floats)
  static constexpr int MS = TB + (36 - TB % 32) % 32;            // mortar flux block stride, 4 mod 32
  static constexpr int TAB = 16 * NP2;                           // duplicated operator tables
  static constexpr int TBUF = 2 * (TF + 1) * TB;                 // one tile's traces (floats)
  static constexpr int SFSZ = ((NM * MS + 3) / 4) * 4;           // mortar fluxes
  static constexpr int NBUF = 2;                                 // the tile and the next one
  static constexpr int NTAB = NBUF;                              // table copies
  // resident CTAs per SM asked of the register allocator
  static constexpr int MINB = 65536 / (THREADS * SM_IF_FUSED_REGS) > 0 ? 65536 / (THREADS * SM_IF_FUSED_REGS) : 1;
  static constexpr size_t smem_floats = (size_t)NTAB * TAB + NBUF * TBUF + SFSZ;
  static constexpr size_t smem_bytes = sizeof(float) * smem_floats;
};

__device__ __forceinline__ void cp_async_4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory");
}

// Copies the 16-byte chunks of cnt consecutive face blocks of a line of ny faces, starting at
// face f0 (0 <= f0 < ny) and wrapping to face 0 at the end of the line, from the compact
// arrays (line base src) into cnt consecutive smem blocks at dst; all threads take part.
template <int TB, int THREADS>
__device__ __forceinline__ void stage_run(float* dst, const float* __restrict__ src, const int f0, const int cnt,
                                          const int ny, const int tid) {
  const int n1 = min(cnt, ny - f0) * (TB / 4), n = cnt * (TB / 4);
  const float* s1 = src + (long long)f0 * TB;
  for (int c = tid; c < n; c += THREADS) cp_async_16(dst + 4 * c, c < n1 ? s1 + 4 * c : src + 4 * (c - n1));
}

// Issues the asynchronous copies of one tile: the duplicated operator tables into sTab (when
// not NULL) and into sT the traces of static faces i0 + r and moving faces i0 - n - 1 + r
// (mod n_par), r = 0..TFe, from the compact arrays Ts / Tm or, when they are NULL, from the
// element node layers of U (xi^3 = +1 static, xi^3 = -1 moving; rows interleaved on the way).
template <int N, int TF>
__device__ __forceinline__ void fused_tile_stage(const MeshDev& m, const StageParams* __restrict__ sp,
                                                 const float* __restrict__ U, const float* __restrict__ Ts,
                                                 const float* __restrict__ Tm, const int tile_x, const int iz,
                                                 float* sTab, float* sT, const int tid) {
  using C = IfFusedCfg<N, TF>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN, THREADS = C::THREADS, TB = C::TB, TAB = C::TAB;
  const int ny = m.ny;
  const int i0 = tile_x * TF;
  const int TFe = min(TF, ny - i0);
  const int nmod = sp->n_mod;
  if (sTab)
    for (int w = tid; w < TAB / 4; w += THREADS) cp_async_16(sTab + 4 * w, sp->pair_f + 4 * w);
  const int fm0 = i0 - nmod - 1 < 0 ? i0 - nmod - 1 + ny : i0 - nmod - 1;
  if (Ts) {
    const long long line = (long long)iz * ny * TB;
    stage_run<TB, THREADS>(sT, Ts + line, i0, TFe + 1, ny, tid);
    stage_run<TB, THREADS>(sT + (TF + 1) * TB, Tm + line, fm0, TFe + 1, ny, tid);
  } else {
    const int nslot = 2 * (TFe + 1);
    for (int w = tid; w < nslot * TB; w += THREADS) {
      const int ab = w % NP2;
      const int rest = w / NP2;
      const int v = rest % 5;
      const int sr = rest / 5;
      const int side = sr >= TFe + 1, r = sr - side * (TFe + 1);
      int f = side ? fm0 + r : i0 + r;
      f = f >= ny ? f - ny : f;
      const float* src = U + encode_elem(m, side, side ? 0 : m.nxs - 1, f, iz) * 5 * NN + (side ? 0 : NP2 * N) +
                         (long long)v * NN + ab;
      cp_async_4(sT + (side * (TF + 1) + r) * TB + v * NP2 + trace_node<float, NP>(ab % NP, ab / NP), src);
    }
  }
}

// Phase A for one mortar (lower part of its static face if isub = 0, upper part if 1), rows
// 2 qp and 2 qp + 1, mortar nodes 2 jp and 2 jp + 1: ts / tm point at the row pair of the
// static / moving face's trace, variables VIN floats apart (rows interleaved, trace_node);
// the mortar fluxes times the surface element go to out (the mortar's row pair, variables
// VOUT floats apart).
template <int N, int RIEM, int VIN, int VOUT>
__device__ __forceinline__ void mortar_rows(const float* sTab, const float* tsp, const float* tmp, float* outp,
                                            const int isub, const int jp, const float sJ, const float gamma) {
  constexpr int NP = N + 1, NH = NP / 2;
  static_assert(VIN % 4 == 0 && VOUT % 4 == 0, "16-byte rows");
  const float4* ts = reinterpret_cast<const float4*>(tsp);
  const float4* tm = reinterpret_cast<const float4*>(tmp);
  // the static lower mortar meets the moving face's upper part and vice versa:
  // tables Ps_isub (slot isub) and Pm_(1-isub) (slot 3 - isub), rows j = 2 jp, 2 jp + 1
  const float4* PT = reinterpret_cast<const float4*>(sTab);
  const float4* ps = PT + (isub * NH + jp) * NP;
  const float4* pm = PT + ((3 - isub) * NH + jp) * NP;
  float2 s0[5], s1[5], m0[5], m1[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) s0[v] = s1[v] = m0[v] = m1[v] = make_float2(0.f, 0.f);
  // static side, then moving side: nodes 2 ih and 2 ih + 1 of both rows per 16-byte load
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const float4* t = side ? tm : ts;
    const float4* P = side ? pm : ps;
    float2* o0 = side ? m0 : s0;
    float2* o1 = side ? m1 : s1;
#pragma unroll
    for (int ih = 0; ih < NH; ++ih) {
      float4 x4[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) x4[v] = t[v * (VIN / 4) + ih];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float4 a = P[2 * ih + h];
        const float2 a0 = make_float2(a.x, a.y), a1 = make_float2(a.z, a.w);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const float2 x = h ? make_float2(x4[v].z, x4[v].w) : make_float2(x4[v].x, x4[v].y);
          o0[v] = fma2(a0, x, o0[v]);
          o1[v] = fma2(a1, x, o1[v]);
        }
      }
    }
  }
  float2 F0[5], F1[5];
  if constexpr (RIEM == 0) {
    // static outward normal +x, no normal grid speed on the interface: both rows at once
    rusanov_outward2(s0, m0, 0, 1.0f, 0.0f, gamma, F0);
    rusanov_outward2(s1, m1, 0, 1.0f, 0.0f, gamma, F1);
  } else {
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      float QL[5], QR[5], f[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const float2 l = h < 2 ? s0[v] : s1[v], r = h < 2 ? m0[v] : m1[v];
        QL[v] = (h & 1) ? l.y : l.x;
        QR[v] = (h & 1) ? r.y : r.x;
      }
      riemann_axis<float, 0, 1>(QL, QR, 0.f, gamma, f);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        float2& o = h < 2 ? F0[v] : F1[v];
        if (h & 1) o.y = f[v];
        else o.x = f[v];
      }
    }
  }
  float4* out = reinterpret_cast<float4*>(outp) + jp;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const float2 g0 = mul2(p2(sJ), F0[v]), g1 = mul2(p2(sJ), F1[v]);
    out[v * (VOUT / 4)] = make_float4(g0.x, g0.y, g1.x, g1.y);
  }
}

// Phase A for mortar mi of a staged tile (layout of fused_tile_stage).
template <int N, int RIEM, int TF>
__device__ __forceinline__ void fused_mortar_rows(const float* sTab, const float* sT, float* sF, const int mi,
                                                  const int qp, const int jp, const float sJ, const float gamma) {
  using C = IfFusedCfg<N, TF>;
  constexpr int NP = C::NP, NP2 = C::NP2, TB = C::TB, MS = C::MS;
  const int isub = mi & 1, rs = mi >> 1, rm = rs + isub;
  mortar_rows<N, RIEM, NP2, NP2>(sTab, sT + rs * TB + qp * 2 * NP, sT + (TF + 1 + rm) * TB + qp * 2 * NP,
                                 sF + mi * MS + qp * 2 * NP, isub, jp, sJ, gamma);
}

// Phase B for one face on one side, rows 2 qp and 2 qp + 1, face nodes 2 ip and 2 ip + 1: the
// face's lower and upper mortar flux rows (flo / fhi: the row pair, variables VIN floats
// apart) projected back and stored to the face flux array at dst (the face's block).
template <int N, int VIN>
__device__ __forceinline__ void face_rows(const float* sTab, const float* flop, const float* fhip,
                                          float* __restrict__ dst, const int side, const int qp, const int ip) {
  constexpr int NP = N + 1, NP2 = NP * NP, NH = NP / 2;
  static_assert(VIN % 4 == 0, "16-byte rows");
  const float4* flo = reinterpret_cast<const float4*>(flop);
  const float4* fhi = reinterpret_cast<const float4*>(fhip);
  // tables B_lo, B_hi of the side (slots 4 + 2 side, 5 + 2 side), rows i = 2 ip, 2 ip + 1
  const float4* PT = reinterpret_cast<const float4*>(sTab);
  const float4* bl = PT + ((4 + 2 * side) * NH + ip) * NP;
  const float4* bh = PT + ((5 + 2 * side) * NH + ip) * NP;
  float2 a0[5], a1[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) a0[v] = a1[v] = make_float2(0.f, 0.f);
  // lower mortar, then upper mortar: nodes 2 jh and 2 jh + 1 of both rows per 16-byte load
#pragma unroll
  for (int part = 0; part < 2; ++part) {
    const float4* f = part ? fhi : flo;
    const float4* B = part ? bh : bl;
#pragma unroll
    for (int jh = 0; jh < NH; ++jh) {
      float4 x4[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) x4[v] = f[v * (VIN / 4) + jh];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float4 l = B[2 * jh + h];
        const float2 l0 = make_float2(l.x, l.y), l1 = make_float2(l.z, l.w);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const float2 x = h ? make_float2(x4[v].z, x4[v].w) : make_float2(x4[v].x, x4[v].y);
          a0[v] = fma2(l0, x, a0[v]);
          a1[v] = fma2(l1, x, a1[v]);
        }
      }
    }
  }
  // rows q = 2 qp (.x) and 2 qp + 1 (.y) of nodes i = 2 ip, 2 ip + 1, outward sign of the side
  const float sg = side ? -1.0f : 1.0f;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    float* d = dst + v * NP2 + 2 * qp * NP + 2 * ip;
    *reinterpret_cast<float2*>(d) = make_float2(sg * a0[v].x, sg * a1[v].x);
    *reinterpret_cast<float2*>(d + NP) = make_float2(sg * a0[v].y, sg * a1[v].y);
  }
}

// Phase B for face r of a staged tile on one side.
template <int N, int TF>
__device__ __forceinline__ void fused_face_rows(const float* sTab, const float* sF, float* __restrict__ dst,
                                                const int r, const int side, const int qp, const int ip) {
  using C = IfFusedCfg<N, TF>;
  constexpr int NP = C::NP, NP2 = C::NP2, MS = C::MS;
  face_rows<N, NP2>(sTab, sF + (2 * r + side) * MS + qp * 2 * NP, sF + (2 * r + 1 + side) * MS + qp * 2 * NP, dst,
                    side, qp, ip);
}

// Phases A and B of one tile whose tables sTab and traces sT have landed (see
// fused_tile_stage), the face fluxes stored to Fs / Fm; one barrier between the phases (the
// caller's next barrier ends the use of sTab, sT and sF).
template <int N, int RIEM, int TF>
__device__ __forceinline__ void fused_tile_compute(const MeshDev& m, const StageParams* __restrict__ sp,
                                                   float* __restrict__ Fs, float* __restrict__ Fm, const int tile_x,
                                                   const int iz, const float* sTab, const float* sT, float* sF,
                                                   const int tid) {
  using C = IfFusedCfg<N, TF>;
  constexpr int NH = C::NH, NM = C::NM, TB = C::TB;
  const int ny = m.ny;
  const int i0 = tile_x * TF;
  const int TFe = min(TF, ny - i0);
  const int nme = 2 * TFe + 1;
  const int nmod = sp->n_mod;

  // A. item = mortar fastest, then node pair, then row pair
  const float sJ = m.cf[MC_SJ_IF];
  const float gamma = m.cf[MC_GAMMA];
  for (int w = tid; w < C::ITEMS_A; w += C::THREADS) {
    const int mi = w % NM;
    const int rest = w / NM;
    const int jp = rest % NH, qp = rest / NH;
    if (mi < nme) fused_mortar_rows<N, RIEM, TF>(sTab, sT, sF, mi, qp, jp, sJ, gamma);
  }
  __syncthreads();

  // B. static face i0 + r from mortars (2r, 2r+1); moving face i0 - n + r from mortars 2r+1
  // (its lower part) and 2r+2 (its upper part), with the opposite sign.  item = face fastest,
  // then side, then node pair, then row pair
  const long long line = (long long)iz * ny;
  for (int w = tid; w < C::ITEMS_B; w += C::THREADS) {
    const int r = w % TF;
    int rest = w / TF;
    const int side = rest & 1;
    rest >>= 1;
    const int ip = rest % NH, qp = rest / NH;
    if (r >= TFe) continue;
    int f = side ? i0 - nmod + r : i0 + r;
    f = f < 0 ? f + ny : (f >= ny ? f - ny : f);
    fused_face_rows<N, TF>(sTab, sF, (side ? Fm : Fs) + (line + f) * TB, r, side, qp, ip);
  }
}

// Persistent tile pipeline: tiles first, first + stride, ... < total, with the next tile's
// copies in flight while a tile computes (two buffers).  stage(item, tables or NULL, traces)
// issues a tile's copies; run(item, tables, traces) computes and stores it.  One barrier per
// tile before the computation: the tile has landed and every thread is done with the
// previous tile, whose buffers the next copies then reuse.
template <int N, int TF, class Stage, class Run>
__device__ __forceinline__ void fused_pipeline(const int first, const int stride, const int total, float* smem,
                                               Stage stage, Run run) {
  using C = IfFusedCfg<N, TF>;
  float* sTab = smem;                        // [NTAB][TAB]
  float* sTr = smem + C::NTAB * C::TAB;      // [NBUF][TBUF]
  if (first < total) stage(first, sTab, sTr);
  cp_async_commit();
  int slot = 0;
  for (int t = first; t < total; t += stride) {
    cp_async_wait<0>();
    __syncthreads();
    const int tn = t + stride;
    if (tn < total) stage(tn, sTab + (slot ^ 1) * C::TAB, sTr + (slot ^ 1) * C::TBUF);
    cp_async_commit();
    run(t, sTab + slot * C::TAB, sTr + slot * C::TBUF);
    slot ^= 1;
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

// Warp-owned rows (FP32, odd N, one solve): the tile's faces split by row pairs, warp w of a
// CTA owning rows 2 w and 2 w + 1 of every face of the CTA's tiles.  The rows of a face are
// independent through projection, Riemann solve and back-projection (the interface slides
// along xi^1 only), so each warp stages its rows of a tile, computes phases A and B and
// stores them with warp-level synchronisation only, and prefetches its rows of the next tile
// meanwhile: no block-wide barrier after the operator tables have landed.  Per warp, in
// shared memory: two trace buffers [side][TF+1 faces][5][2 NP] and the mortar fluxes
// [2 TF + 1][5][2 NP] (stride MSW = 4 mod 32 words).  Same arithmetic per node as the
// staged tile (mortar_rows, face_rows), so the results are bit-identical.
#ifndef SM_IF_WARP_TF
#define SM_IF_WARP_TF 4
#endif
#ifndef SM_IF_WARP_REGS
#define SM_IF_WARP_REGS 168
#endif
template <int N, int TFV> struct IfWarpCfg {
  static_assert(N % 2 == 1, "the warp-owned interface rows take odd N (rows in pairs)");
  static constexpr int NP = N + 1, NP2 = NP * NP, NN = NP * NP * NP;
  static constexpr int NH = NP / 2;                      // row pairs = warps per CTA
  static constexpr int TF = TFV;
  static constexpr int NM = 2 * TF + 1;
  static constexpr int WPB = NH;
  static constexpr int THREADS = 32 * WPB;
  static constexpr int RB = 5 * 2 * NP;                  // one face's row pair, all variables
  static constexpr int TBUFW = 2 * (TF + 1) * RB;        // one buffer of a warp (floats)
  static constexpr int MSW = RB + (36 - RB % 32) % 32;   // mortar flux stride, 4 mod 32
  static constexpr int SFW = ((NM * MSW + 3) / 4) * 4;
  static constexpr int PER_WARP = 2 * TBUFW + SFW;
  static constexpr int TAB = 16 * NP2;
  static constexpr size_t smem_floats = (size_t)TAB + (size_t)WPB * PER_WARP;
  static constexpr size_t smem_bytes = sizeof(float) * smem_floats;
  // resident CTAs per SM asked of the register allocator
  static constexpr int MINB = 65536 / (THREADS * SM_IF_WARP_REGS) > 0 ? 65536 / (THREADS * SM_IF_WARP_REGS) : 1;
};

// Issues the copies of one warp's rows (row pair qp) of tile (tile_x, iz) into buf
// [side][r][v][2 NP]: static faces i0 + r and moving faces i0 - n - 1 + r (mod n_par),
// r = 0..TFe, from the compact arrays (16-byte pieces: a variable's row pair is 2 NP
// contiguous floats) or from the element node layers of U (rows interleaved on the way).
template <int N, int TF>
__device__ __forceinline__ void warp_rows_stage(const MeshDev& m, const int nmod, const float* __restrict__ U,
                                                const float* __restrict__ Ts, const float* __restrict__ Tm,
                                                const int tile_x, const int iz, const int qp, float* buf,
                                                const int lane) {
  using C = IfWarpCfg<N, TF>;
  constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN, TB = 5 * NP2;
  const int ny = m.ny;
  const int i0 = tile_x * TF;
  const int TFe = min(TF, ny - i0);
  const int nf = TFe + 1;
  const int fm0 = i0 - nmod - 1 < 0 ? i0 - nmod - 1 + ny : i0 - nmod - 1;
  if (Ts) {
    constexpr int CH = 2 * NP / 4;                       // 16-byte pieces of a variable's row pair
    const long long line = (long long)iz * ny;
    for (int c = lane; c < 2 * nf * 5 * CH; c += 32) {
      const int ch = c % CH;
      int rest = c / CH;
      const int v = rest % 5;
      rest /= 5;
      const int side = rest >= nf, r = rest - side * nf;
      int f = side ? fm0 + r : i0 + r;
      f = f >= ny ? f - ny : f;
      const float* src = (side ? Tm : Ts) + (line + f) * TB + v * NP2 + qp * 2 * NP + 4 * ch;
      cp_async_16(buf + ((side * (TF + 1) + r) * 5 + v) * 2 * NP + 4 * ch, src);
    }
  } else {
    for (int c = lane; c < 2 * nf * 5 * 2 * NP; c += 32) {
      const int node = c % (2 * NP);                     // i + NP (q & 1): row-major in the layer
      int rest = c / (2 * NP);
      const int v = rest % 5;
      rest /= 5;
      const int side = rest >= nf, r = rest - side * nf;
      int f = side ? fm0 + r : i0 + r;
      f = f >= ny ? f - ny : f;
      const int i = node % NP, q1 = node / NP;
      const float* src = U + encode_elem(m, side, side ? 0 : m.nxs - 1, f, iz) * 5 * NN + (side ? 0 : NP2 * N) +
                         (long long)v * NN + (2 * qp + q1) * NP + i;
      cp_async_4(buf + ((side * (TF + 1) + r) * 5 + v) * 2 * NP + 2 * i + q1, src);
    }
  }
}

template <int N, int RIEM, int TF>
__global__ void __launch_bounds__(IfWarpCfg<N, TF>::THREADS, IfWarpCfg<N, TF>::MINB)
sliding_interface_warp_kernel(const MeshDev m, const StageParams* __restrict__ sp, const float* __restrict__ U,
                              float* __restrict__ Fs, float* __restrict__ Fm, const float* __restrict__ Ts,
                              const float* __restrict__ Tm) {
  using C = IfWarpCfg<N, TF>;
  constexpr int NP = C::NP, NH = C::NH, NM = C::NM, RB = C::RB, MSW = C::MSW, TB = 5 * C::NP2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sTab = reinterpret_cast<float*>(smem_raw);
  const int qp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* wb = sTab + C::TAB + qp * C::PER_WARP;          // [2][TBUFW] traces
  float* sF = wb + 2 * C::TBUFW;                         // [NM][MSW] mortar fluxes
  const int ny = m.ny;
  const int ntx = (ny + TF - 1) / TF;
  const float inv = 1.0f / (float)ntx;
  const int total = ntx * m.nz;
  const int nmod = sp->n_mod;
  const float sJ = m.cf[MC_SJ_IF];
  const float gamma = m.cf[MC_GAMMA];
  for (int w = threadIdx.x; w < C::TAB / 4; w += C::THREADS) cp_async_16(sTab + 4 * w, sp->pair_f + 4 * w);
  int t = blockIdx.x;
  if (t < total) {
    int x, z;
    divmod_small(t, ntx, inv, &z, &x);
    warp_rows_stage<N, TF>(m, nmod, U, Ts, Tm, x, z, qp, wb, lane);
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();                                       // tables and every warp's first rows
  int slot = 0;
  for (; t < total; t += gridDim.x) {
    const int tn = t + gridDim.x;
    if (tn < total) {
      int x, z;
      divmod_small(tn, ntx, inv, &z, &x);
      warp_rows_stage<N, TF>(m, nmod, U, Ts, Tm, x, z, qp, wb + (slot ^ 1) * C::TBUFW, lane);
    }
    cp_async_commit();
    cp_async_wait<1>();                                  // this tile's rows (the next may be in flight)
    __syncwarp();
    int tile_x, iz;
    divmod_small(t, ntx, inv, &iz, &tile_x);
    const int i0 = tile_x * TF;
    const int TFe = min(TF, ny - i0);
    const int nme = 2 * TFe + 1;
    const float* buf = wb + slot * C::TBUFW;
    // A. item = mortar fastest, then node pair
    for (int w = lane; w < NM * NH; w += 32) {
      const int mi = w % NM, jp = w / NM;
      if (mi < nme) {
        const int isub = mi & 1, rs = mi >> 1, rm = rs + isub;
        mortar_rows<N, RIEM, 2 * NP, 2 * NP>(sTab, buf + rs * RB, buf + (TF + 1 + rm) * RB, sF + mi * MSW, isub, jp,
                                             sJ, gamma);
      }
    }
    __syncwarp();
    // B. static face i0 + r from mortars (2r, 2r+1), moving face i0 - n + r from (2r+1, 2r+2);
    // item = face fastest, then side, then node pair
    const long long line = (long long)iz * ny;
    for (int w = lane; w < 2 * TF * NH; w += 32) {
      const int r = w % TF;
      const int rest = w / TF;
      const int side = rest & 1, ip = rest >> 1;
      if (r < TFe) {
        int f = side ? i0 - nmod + r : i0 + r;
        f = f < 0 ? f + ny : (f >= ny ? f - ny : f);
        face_rows<N, 2 * NP>(sTab, sF + (2 * r + side) * MSW, sF + (2 * r + 1 + side) * MSW,
                             (side ? Fm : Fs) + (line + f) * TB, side, qp, ip);
      }
    }
    __syncwarp();                                        // buf and sF free for the next tile
    slot ^= 1;
  }
  cp_async_wait<0>();
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

// Split-form element kernel: the volume integral of the split formulation with Pirozzoli's
// two-point flux (Sec. 3.1, the scheme of all of the paper's computations), the same surface
// integral and low-storage RK update as the weak-form kernel.
//
// Strong form with a two-point volume flux F#, on LGL nodes:
//   J dU/dt|_ijk = -[ sum_l Ds_il F~#1(U_ijk, U_ljk) + sum_l Ds_jl F~#2(U_ijk, U_ilk)
//                     + sum_l Ds_kl F~#3(U_ijk, U_ijl) ] - (1 / w_0) (F* . N sJ) at face nodes,
// with Ds = 2 D - M^-1 B (B = diag(-1, 0, .., 0, 1), M the LGL weights).  The boundary
// correction -F(U)/w of the strong form sits on the diagonal of Ds, and F#(U, U) = F(U).
// On LGL nodes Ds vanishes on the diagonal (D_ii = 0 inside, 2 D_00 = -1/w_0, 2 D_NN = 1/w_N),
// so only pairs i != l enter, and each pair's flux serves both of its nodes:
//   node i gets Ds_il F#(i, l), node l gets Ds_li F#(i, l)  (F# is symmetric).
//
// Two-point flux (reading of the ALE form of Sec. 2): Pirozzoli's split of the convective
// terms rho w phi, phi in {1, v, H}, with the advecting velocity w = v.n - v^g.n taken
// relative to the grid, as products of arithmetic means {{a}} = (a_L + a_R) / 2:
//   F#_rho = {{rho}} {{w}},  F#_rho v = F#_rho {{v}} + {{p}} n,  F#_rho e = F#_rho {{H}} + {{p}} v^g.n,
// H = (rho e + p) / rho; for U_L = U_R it is the ALE flux F.n - (v^g.n) U.  Cartesian
// elements: the contravariant flux of direction xi^d is |Ja^d| F# along the physical axis.
//
// One thread per volume node loads its state and stores the halved primitives
// (rho, v1, v2, v3, p, H) / 2 in shared memory, so that a mean is one addition; the face
// fluxes are computed as in the weak-form kernel.  After a barrier two threads per
// contraction line (direction, line), one per group of conserved variables, hold the
// line's primitives in registers, evaluate the NP (NP - 1) / 2 pair fluxes once and
// accumulate both ends; after a second barrier every node sums its three directions with
// the metric terms and applies the surface integral and the RK update.
//
// Navier-Stokes (PHYS 1; the paper's production scheme, split form with BR1): the advective
// terms take the split form above, the viscous terms keep the weak form of the weak-form
// kernel, and the face flux is the Riemann flux minus the BR1 mean of both sides' viscous
// fluxes, so that the own-flux correction folded into Ds is the advective flux only:
//   J dU/dt = -[ sum_d |Ja^d| sum_l Ds_il F#^d(U_i, U_l) ] + sum_d |Ja^d| sum_l Dhat_il F^v_d(U_l, grad_l)
//             - (1 / w_0) ((F*_adv - {{F^v}}) . N sJ) at face nodes,
// with the lifted gradients of the BR1 lifting kernel.  Every node stores its viscous fluxes
// negated in a third shared array, whose lines are contracted with Dhat beside the split
// lines.
#pragma once

#include "sm_element.cuh"

template <int N> struct SplitCfg {
  using C = ElemCfg<N>;
  static constexpr int NP = C::NP, NP2 = C::NP2, NN = C::NN, EPB = C::EPB, THREADS = C::THREADS;
  static constexpr int LINES = EPB * 3 * NP2;
  // FP32 launch bound: resident CTAs per SM asked of the register allocator (N = 5: 56
  // registers, 5 CTAs of 216 threads; measured 4 % (Roe/HH) to 8 % (Rusanov) faster than 72
  // registers and 4 CTAs)
#ifdef SM_SPLIT_MINB_OVERRIDE
  static constexpr int MINB = SM_SPLIT_MINB_OVERRIDE;
#else
  static constexpr int MINB = N <= 2 ? 2 : (N == 7 ? 1 : (N == 6 ? 2 : (N == 5 ? 5 : 3)));
#endif
  template <typename T, int PHYS = 0> static constexpr size_t smem_bytes() {
    return sizeof(T) * (size_t)(EPB * 6 * NN + EPB * 15 * NN + EPB * 30 * NP2 + (PHYS ? EPB * 15 * NN : 0));
  }
};

// Ds = 2 D - M^-1 B for N = 1..7, [N-1][i*8 + l] (zero diagonal), in constant memory of the
// translation unit that instantiates the split kernels, indexed with compile-time constants.
static __constant__ float c_dsplit_f[7][SM_MAXNP * SM_MAXNP];
static __constant__ double c_dsplit_d[7][SM_MAXNP * SM_MAXNP];

static inline cudaError_t upload_dsplit_here(const float* f, const double* d) {
  cudaError_t e = cudaMemcpyToSymbol(c_dsplit_f, f, sizeof(float) * 7 * SM_MAXNP * SM_MAXNP);
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_dsplit_d, d, sizeof(double) * 7 * SM_MAXNP * SM_MAXNP);
}

template <typename T> __device__ __forceinline__ T dsplit_c(int n, int idx);
template <> __device__ __forceinline__ float dsplit_c<float>(int n, int idx) { return c_dsplit_f[n - 1][idx]; }
template <> __device__ __forceinline__ double dsplit_c<double>(int n, int idx) { return c_dsplit_d[n - 1][idx]; }

// One half of the two-point volume integral of a contraction line: ROLE 0 the mass, normal
// and first tangential momentum components, ROLE 1 the second tangential momentum and the
// energy.  Each half evaluates the parts of the pair fluxes it needs, so a line's two halves
// run on two threads with about half the registers of one thread doing the whole line.
//   sQ [EPB][6][NN]: halved primitives (rho, v1, v2, v3, p, H) / 2 in node order;
//   sV [EPB][3][5][NN]: per direction d, sum_l Ds_al F#(U_a, U_l) (physical momentum order,
//   without the metric factor |Ja^d|).
// Line (l2, d, q): xi^1 (i) lines are contiguous, xi^2 (j) lines have stride NP and xi^3 (k)
// lines stride NP^2.  Velocity slots are read in the order (normal, tangential, tangential)
// of the direction's physical axis, so one code path serves all directions.
template <int N, typename T, int ROLE>
__device__ __forceinline__ void split_line_half(const MeshDev& m, const T* sQ, T* sV, const long long e0,
                                                const int w) {
  constexpr int NP = N + 1, NP2 = NP * NP, NN = NP2 * NP;
  constexpr int NV = ROLE == 0 ? 3 : 2;
  const int l2 = w / (3 * NP2);
  const int r = w - l2 * 3 * NP2;
  const int d = r / NP2, q = r - d * NP2;
  if (e0 + l2 >= m.E) return;
  const int blk = e0 + l2 >= m.Es;
  const int base = d == 0 ? NP * q : (d == 1 ? (q % NP) + NP2 * (q / NP) : q);
  const int stride = d == 0 ? 1 : (d == 1 ? NP : NP2);
  const int ax = d == 0 ? 1 : (d == 1 ? 2 : 0);      // physical axis of xi^{d+1}
  const int sn = 1 + ax, st1 = 1 + (ax + 1) % 3, st2 = 1 + (ax + 2) % 3;
  // grid velocity along the axis: the moving block translates along y = xi^1
  const T vg = (d == 0 && blk) ? Prec<T>::c(m)[MC_VG] : T(0);
  const T* Q = sQ + l2 * 6 * NN + base;
  // ROLE 0 reads (rho, v_n, p, v_t1); ROLE 1 reads (rho, v_n, p, v_t2, H)
  T rh[NP], un[NP], pp[NP], xa[NP], xb[NP];
  const int sa = ROLE == 0 ? st1 : st2;
#pragma unroll
  for (int l = 0; l < NP; ++l) {
    rh[l] = Q[l * stride];
    un[l] = Q[sn * NN + l * stride];
    pp[l] = Q[4 * NN + l * stride];
    xa[l] = Q[sa * NN + l * stride];
    if (ROLE == 1) xb[l] = Q[5 * NN + l * stride];
  }
  T acc[NP][NV];
#pragma unroll
  for (int a = 0; a < NP; ++a)
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[a][v] = T(0);
#pragma unroll
  for (int a = 0; a < NP; ++a) {
#pragma unroll
    for (int l = a + 1; l < NP; ++l) {
      const T nm = un[a] + un[l], pm = pp[a] + pp[l];
      const T fr = (rh[a] + rh[l]) * (nm - vg);
      T f[NV];
      if (ROLE == 0) {
        f[0] = fr;
        f[1] = fr * nm + pm;
        f[2] = fr * (xa[a] + xa[l]);
      } else {
        f[0] = fr * (xa[a] + xa[l]);
        f[1] = fr * (xb[a] + xb[l]) + pm * vg;
      }
      const T dal = dsplit_c<T>(N, a * SM_MAXNP + l), dla = dsplit_c<T>(N, l * SM_MAXNP + a);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        acc[a][v] += dal * f[v];
        acc[l][v] += dla * f[v];
      }
    }
  }
  T* V = sV + (l2 * 3 + d) * 5 * NN + base;
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    if (ROLE == 0) {
      V[a * stride] = acc[a][0];
      V[sn * NN + a * stride] = acc[a][1];
      V[st1 * NN + a * stride] = acc[a][2];
    } else {
      V[st2 * NN + a * stride] = acc[a][0];
      V[4 * NN + a * stride] = acc[a][1];
    }
  }
}

// The two-point volume integral of every contraction line of the CTA's elements: work items
// 0 .. LINES-1 are the first halves of the lines, LINES .. 2 LINES-1 the second halves (the
// two roles meet in at most one warp).
template <int N, typename T>
__device__ __forceinline__ void split_volume_lines(const MeshDev& m, const T* sQ, T* sV, const long long e0,
                                                   const int tid) {
  using C = SplitCfg<N>;
  for (int w = tid; w < 2 * C::LINES; w += C::THREADS) {
    if (w < C::LINES) split_line_half<N, T, 0>(m, sQ, sV, e0, w);
    else split_line_half<N, T, 1>(m, sQ, sV, e0, w - C::LINES);
  }
}

template <int N, typename T, int RIEM, int MODE, int PHYS = 0>
__device__ __forceinline__ void element_block_split(const MeshDev& m, const StageParams* __restrict__ sp,
                                                    const T* __restrict__ U, T* __restrict__ out, T* __restrict__ G,
                                                    const T* __restrict__ Fs, const T* __restrict__ Fm, const T rkA,
                                                    const T rkB, const T dt, const long long e0, T* __restrict__ Ts,
                                                    T* __restrict__ Tm, const T* __restrict__ Gr = nullptr) {
  using C = SplitCfg<N>;
  constexpr int NP2 = C::NP2, NN = C::NN, EPB = C::EPB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sQ = reinterpret_cast<T*>(smem_raw);        // [EPB][6][NN] halved primitives
  T* sV = sQ + EPB * 6 * NN;                     // [EPB][3][5][NN] two-point volume terms
  T* sS = sV + EPB * 15 * NN;                    // [EPB][6][5][NP2] outward face fluxes
  T* sW = sS + EPB * 30 * NP2;                   // PHYS 1: [EPB][3][5][NN] -F^v along the axes of xi^1..3

  const T* c = Prec<T>::c(m);
  const int tid = threadIdx.x;
  const int le = tid / NN, nd = tid - le * NN;
  const long long e = e0 + le;
  const bool active = e < m.E;
  const long long base = e * 5 * NN + nd;

  T u[5], g[5];
  if (active) {
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = U[base + v * NN];
    if (MODE == ELEM_STAGE) {
#pragma unroll
      for (int v = 0; v < 5; ++v) g[v] = G[base + v * NN];
    }
    const Prim<T> q = primitives(u, c[MC_GAMMA]);
    T* Q = sQ + le * 6 * NN + nd;
    Q[0] = T(0.5) * u[0];
    Q[NN] = T(0.5) * q.u[0];
    Q[2 * NN] = T(0.5) * q.u[1];
    Q[3 * NN] = T(0.5) * q.u[2];
    Q[4 * NN] = T(0.5) * q.p;
    Q[5 * NN] = T(0.5) * ((u[4] + q.p) * q.ir);
    if (PHYS) {
      // viscous fluxes of the lifted gradients along the axes of xi^1 (y), xi^2 (z), xi^3 (x)
      T gn[15], fv[5];
#pragma unroll
      for (int kk = 0; kk < 15; ++kk) gn[kk] = Gr[(e * 15 + kk) * NN + nd];
      T* W = sW + le * 15 * NN + nd;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        viscous_flux_axis(u, gn, d == 0 ? 1 : (d == 1 ? 2 : 0), c, fv);
#pragma unroll
        for (int v = 0; v < 5; ++v) W[(5 * d + v) * NN] = -fv[v];
      }
    }
  }

  element_face_fluxes<N, T, RIEM, PHYS>(m, sp, U, Fs, Fm, Gr, e0, sS, tid);

  __syncthreads();
  split_volume_lines<N, T>(m, sQ, sV, e0, tid);
  if (PHYS) contract_lines_inplace<N, T>(sW, tid);
  __syncthreads();
  if (!active) return;
  const int blk = e >= m.Es;
  const T a0 = c[MC_METRIC + 3 * blk], a1 = c[MC_METRIC + 3 * blk + 1], a2 = c[MC_METRIC + 3 * blk + 2];
  T acc[5];
  {
    const T* V = sV + le * 15 * NN + nd;
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] = a0 * V[v * NN] + a1 * V[(5 + v) * NN] + a2 * V[(10 + v) * NN];
    if (PHYS) {
      const T* W = sW + le * 15 * NN + nd;
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] += a0 * W[v * NN] + a1 * W[(5 + v) * NN] + a2 * W[(10 + v) * NN];
    }
  }
  element_surface_update<N, T, MODE>(m, sS + le * 30 * NP2, acc, nd, e, base, u, g, out, G, rkA, rkB, dt, Ts, Tm);
}

template <int N, typename T, int RIEM, int MODE, int PHYS = 0>
__global__ void __launch_bounds__(SplitCfg<N>::THREADS, (sizeof(T) == 4 && PHYS == 0) ? SplitCfg<N>::MINB : 1)
dg_element_split_kernel(const MeshDev m, const StageParams* __restrict__ sp, const T* __restrict__ U,
                        T* __restrict__ out, T* __restrict__ G, const T* __restrict__ Fs,
                        const T* __restrict__ Fm, const T rkA, const T rkB, const T dt, T* __restrict__ Ts,
                        T* __restrict__ Tm, const T* __restrict__ Gr) {
  element_block_split<N, T, RIEM, MODE, PHYS>(m, sp, U, out, G, Fs, Fm, rkA, rkB, dt,
                                              (long long)blockIdx.x * SplitCfg<N>::EPB, Ts, Tm, Gr);
}

template <int N, typename T, int RIEM, int MODE, int PHYS = 0>
static cudaError_t launch_split_t(const ElemArgs& a, cudaStream_t st) {
  using C = SplitCfg<N>;
  const long long blocks = (a.m.E + C::EPB - 1) / C::EPB;
  if (blocks <= 0) return cudaSuccess;
  dg_element_split_kernel<N, T, RIEM, MODE, PHYS><<<(unsigned)blocks, C::THREADS, C::template smem_bytes<T, PHYS>(), st>>>(
      a.m, a.sp, (const T*)a.U, (T*)a.out, (T*)a.G, (const T*)a.Fs, (const T*)a.Fm, (T)a.rkA, (T)a.rkB, (T)a.dt,
      (T*)a.Ts, (T*)a.Tm, (const T*)a.Gr);
  return cudaGetLastError();
}

template <int N, typename T, int RIEM, int MODE, int PHYS = 0>
static cudaError_t prepare_split_t() {
  cudaError_t e = cudaFuncSetAttribute(dg_element_split_kernel<N, T, RIEM, MODE, PHYS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SplitCfg<N>::template smem_bytes<T, PHYS>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(dg_element_split_kernel<N, T, RIEM, MODE, PHYS>,
                              cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutDefault);
}

template <int N, typename T, int PHYS = 0>
static cudaError_t launch_split_n(int riemann, int mode, const ElemArgs& a, cudaStream_t st) {
  if (riemann == 0) {
    if (mode == ELEM_RHS) return launch_split_t<N, T, 0, ELEM_RHS, PHYS>(a, st);
    if (mode == ELEM_STAGE) return launch_split_t<N, T, 0, ELEM_STAGE, PHYS>(a, st);
    return launch_split_t<N, T, 0, ELEM_STAGE_FIRST, PHYS>(a, st);
  }
  if (mode == ELEM_RHS) return launch_split_t<N, T, 1, ELEM_RHS, PHYS>(a, st);
  if (mode == ELEM_STAGE) return launch_split_t<N, T, 1, ELEM_STAGE, PHYS>(a, st);
  return launch_split_t<N, T, 1, ELEM_STAGE_FIRST, PHYS>(a, st);
}

template <int N, typename T, int PHYS = 0>
static cudaError_t prepare_split_n() {
  cudaError_t e = cudaSuccess, r;
  if ((r = prepare_split_t<N, T, 0, ELEM_RHS, PHYS>()) != cudaSuccess) e = r;
  if ((r = prepare_split_t<N, T, 0, ELEM_STAGE, PHYS>()) != cudaSuccess) e = r;
  if ((r = prepare_split_t<N, T, 0, ELEM_STAGE_FIRST, PHYS>()) != cudaSuccess) e = r;
  if ((r = prepare_split_t<N, T, 1, ELEM_RHS, PHYS>()) != cudaSuccess) e = r;
  if ((r = prepare_split_t<N, T, 1, ELEM_STAGE, PHYS>()) != cudaSuccess) e = r;
  if ((r = prepare_split_t<N, T, 1, ELEM_STAGE_FIRST, PHYS>()) != cudaSuccess) e = r;
  return e;
}

#define SM_SPLIT_DISPATCH(T, N, riemann, mode, a, st, PHYS)            \
  switch (N) {                                                         \
    case 1: return launch_split_n<1, T, PHYS>(riemann, mode, a, st);   \
    case 2: return launch_split_n<2, T, PHYS>(riemann, mode, a, st);   \
    case 3: return launch_split_n<3, T, PHYS>(riemann, mode, a, st);   \
    case 4: return launch_split_n<4, T, PHYS>(riemann, mode, a, st);   \
    case 5: return launch_split_n<5, T, PHYS>(riemann, mode, a, st);   \
    case 6: return launch_split_n<6, T, PHYS>(riemann, mode, a, st);   \
    case 7: return launch_split_n<7, T, PHYS>(riemann, mode, a, st);   \
    default: return cudaErrorInvalidValue;                             \
  }

#define SM_SPLIT_PREPARE(T, N, PHYS)                  \
  switch (N) {                                        \
    case 1: return prepare_split_n<1, T, PHYS>();     \
    case 2: return prepare_split_n<2, T, PHYS>();     \
    case 3: return prepare_split_n<3, T, PHYS>();     \
    case 4: return prepare_split_n<4, T, PHYS>();     \
    case 5: return prepare_split_n<5, T, PHYS>();     \
    case 6: return prepare_split_n<6, T, PHYS>();     \
    case 7: return prepare_split_n<7, T, PHYS>();     \
    default: return cudaErrorInvalidValue;            \
  }

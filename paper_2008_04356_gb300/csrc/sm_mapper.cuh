// Interface configuration and mortar operators on the device, in FP64 (Sec. 4.3 and 3.2).
//
// One small kernel per Runge-Kutta stage: stage time t_k = fma(c_k, dt, t), displacement
// Delta = fma(v, t_k, delta0), q = Delta / l, n = floor(q), s = q - n, hanging nodes
// sigma_s = 2 s - 1 (static face) and sigma_m = 1 - 2 s (moving face), then the forward
// operators P (interpolation at the mortar nodes, equal to the L2 projection for equal N)
// and the conservative back operators B = J M^-1 P^T M for both faces.  Every FP64
// operation of the configuration is an explicit round-to-nearest intrinsic, so no
// multiply-add is contracted and the result is bit-identical to any IEEE evaluation of
// the same sequence.
#pragma once

#include "sm_launch.h"


__device__ __forceinline__ void interface_config(double delta, double l, long long* n, double* s) {
  double q = __ddiv_rn(delta, l);
  double fq = floor(q);
  *n = (long long)fq;
  *s = __dsub_rn(q, fq);
}

// ell_i(x) on the LGL nodes by the barycentric formula; exact Kronecker delta at a node.
__device__ __forceinline__ void lagrange_row(int np, const double* xn, const double* lam, double x, double* out) {
  for (int k = 0; k < np; ++k)
    if (x == xn[k]) {
      for (int i = 0; i < np; ++i) out[i] = (i == k) ? 1.0 : 0.0;
      return;
    }
  double den = 0.0;
  for (int k = 0; k < np; ++k) den += lam[k] / (x - xn[k]);
  for (int i = 0; i < np; ++i) out[i] = (lam[i] / (x - xn[i])) / den;
}

// Builds P_lo, P_hi, B_lo, B_hi for hanging node sigma into out[4][np*np] (shared or
// global), cooperatively over the block.  scratch holds 2 np^2 doubles.
__device__ __forceinline__ void build_mortar_ops(int np, const BasisDev* b, double sigma, double* out, double* scratch) {
  const int n2 = np * np;
  const double J[2] = {0.5 * (1.0 + sigma), 0.5 * (1.0 - sigma)};
  // forward: row j of P_part = ell(xi_part(z_j))
  for (int r = threadIdx.x; r < 2 * np; r += blockDim.x) {
    int part = r / np, j = r - part * np;
    double z = b->x[j];
    double xi = part == 0 ? -1.0 + J[0] * (z + 1.0) : sigma + J[1] * (z + 1.0);
    lagrange_row(np, b->x, b->lam, xi, out + part * n2 + j * np);
  }
  __syncthreads();
  // T_part = P_part^T M
  for (int r = threadIdx.x; r < 2 * n2; r += blockDim.x) {
    int part = r / n2, aj = r - part * n2, a = aj / np, j = aj - a * np;
    double acc = 0.0;
    for (int q = 0; q < np; ++q) acc += out[part * n2 + q * np + a] * b->M[q * SM_MAXNP + j];
    scratch[r] = acc;
  }
  __syncthreads();
  // B_part = J_part M^-1 T_part
  for (int r = threadIdx.x; r < 2 * n2; r += blockDim.x) {
    int part = r / n2, ij = r - part * n2, i = ij / np, j = ij - i * np;
    double acc = 0.0;
    for (int a = 0; a < np; ++a) acc += b->Minv[i * SM_MAXNP + a] * scratch[part * n2 + a * np + j];
    out[(2 + part) * n2 + ij] = J[part] * acc;
  }
  __syncthreads();
  // conforming instants: one mortar is the whole face (identity), the other has length 0
  if (sigma == -1.0 || sigma == 1.0) {
    int full = sigma == -1.0 ? 1 : 0;
    for (int r = threadIdx.x; r < n2; r += blockDim.x) {
      double id = (r / np == r % np) ? 1.0 : 0.0;
      out[full * n2 + r] = id;
      out[(2 + full) * n2 + r] = id;
      out[(2 + (1 - full)) * n2 + r] = 0.0;
    }
  }
  __syncthreads();
}

// mode 0: t_k = t_arg.  mode 1: t_k = fma(c_k, dt, *t_dev).  mode 2: as mode 1 and the
// stored time then advances by dt (last stage of a step).  One CTA of 64 threads.
__device__ __forceinline__ void stage_params_body(const MeshDev& m, int np, StageParams* sp, double* t_dev,
                                                  double t_arg, double ck, double dt, int mode) {
  __shared__ double s_ops[4 * SM_MAXNP * SM_MAXNP];
  __shared__ double s_scr[2 * SM_MAXNP * SM_MAXNP];
  __shared__ double s_sig[2];
  if (threadIdx.x == 0) {
    double t = mode == 0 ? t_arg : __fma_rn(ck, dt, *t_dev);
    double delta = __fma_rn(m.v, t, m.delta0);
    long long n;
    double s;
    interface_config(delta, m.hy, &n, &s);
    double two_s = __dmul_rn(2.0, s);
    sp->t = t;
    sp->delta = delta;
    sp->n = n;
    {
      const long long r = n % m.ny;
      sp->n_mod = (int)(r < 0 ? r + m.ny : r);
    }
    sp->s = s;
    sp->sig_s = __dsub_rn(two_s, 1.0);
    sp->sig_m = __dsub_rn(1.0, two_s);
    s_sig[0] = sp->sig_s;
    s_sig[1] = sp->sig_m;
    if (rotating_geom(m.geom)) {
      // the rotor turns by phi = -delta; stator faces seen through w wraps: w Theta - phi
      const double phi = -delta;
      double c0, s0;
      sincos(phi, &s0, &c0);
      sp->rot[0] = c0; sp->rot[1] = s0;
      sp->rot_f[0] = (float)c0; sp->rot_f[1] = (float)s0;
      long long a = -n - 1, q = a / m.ny;
      if (a % m.ny != 0 && a < 0) q -= 1;
      sp->w0 = q;
      for (int k = 0; k < 2; ++k) {
        const double ang = __dsub_rn(__dmul_rn((double)(q + k), m.Theta), phi);
        double ck, sk;
        sincos(ang, &sk, &ck);
        sp->arot[k][0] = ck; sp->arot[k][1] = sk;
        sp->arot_f[k][0] = (float)ck; sp->arot_f[k][1] = (float)sk;
      }
    }
    if (mode == 2) *t_dev = __dadd_rn(*t_dev, dt);
  }
  __syncthreads();
  const int n2 = np * np;
  for (int side = 0; side < 2; ++side) {
    build_mortar_ops(np, m.basis, s_sig[side], s_ops, s_scr);
    // P_lo, P_hi -> slots 2 side + {0,1}; B_lo, B_hi -> 4 + 2 side + {0,1}
    for (int r = threadIdx.x; r < 4 * n2; r += blockDim.x) {
      int k = r / n2, ij = r - k * n2;
      int slot = k < 2 ? 2 * side + k : 4 + 2 * side + (k - 2);
      double v = s_ops[r];
      sp->mat[slot][ij] = v;
      sp->mat_f[slot][ij] = (float)v;
    }
    __syncthreads();
  }
  // the FP32 operators duplicated into float pairs, rows in pairs: [k][h][col][2 rows x 2]
  if (np % 2 == 0) {
    const int nh = np / 2;
    for (int r = threadIdx.x; r < 8 * nh * np; r += blockDim.x) {
      const int col = r % np, kh = r / np, h = kh % nh, k = kh / nh;
      const float v0 = sp->mat_f[k][2 * h * np + col], v1 = sp->mat_f[k][(2 * h + 1) * np + col];
      *reinterpret_cast<float4*>(sp->pair_f + 4 * r) = make_float4(v0, v0, v1, v1);
    }
  }
}


// Launches of the per-stage interface configuration / mortar operator kernel and of the
// batched mapper (bodies in sm_mapper.cuh).
#include "sm_mapper.cuh"

namespace {

__global__ void __launch_bounds__(64) stage_params_kernel(MeshDev m, int np, StageParams* sp, double* t_dev,
                                                          double t_arg, double ck, double dt, int mode) {
  stage_params_body(m, np, sp, t_dev, t_arg, ck, dt, mode);
}

// The five stages of one RK step in one launch: CTA k writes the parameters of stage k into
// sp + k for the stage time fma(c_k, dt, t), t the stored step time; the last CTA to finish
// (counted on ticket, which it resets) advances the stored time by dt, after every CTA has
// read it.
__global__ void __launch_bounds__(64) step_params_kernel(MeshDev m, int np, StageParams* sp, double* t_dev,
                                                         StepCoeffs c, double dt, unsigned* ticket) {
  const int k = blockIdx.x;
  stage_params_body(m, np, sp + k, t_dev, 0.0, c.c[k], dt, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ticket, 1u) == gridDim.x - 1) {
      *t_dev = __dadd_rn(*t_dev, dt);
      *ticket = 0u;
      __threadfence();
    }
  }
}

__global__ void map_batch_kernel(const double* delta, int count, double l, int n_par, long long* n_out,
                                 double* s_out, int* pairs) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= count) return;
  long long n;
  double s;
  interface_config(delta[m], l, &n, &s);
  n_out[m] = n;
  s_out[m] = s;
  if (pairs) {
    long long nm = n % n_par;
    if (nm < 0) nm += n_par;
    for (int i = 0; i < n_par; ++i)
      for (int isub = 0; isub < 2; ++isub) {
        long long it = (long long)i - nm + isub - 1;
        it %= n_par;
        if (it < 0) it += n_par;
        pairs[((long long)m * n_par + i) * 2 + isub] = (int)it;
      }
  }
}

__global__ void __launch_bounds__(64) mortar_ops_kernel(const BasisDev* b, int np, double sigma, double* out) {
  __shared__ double s_ops[4 * SM_MAXNP * SM_MAXNP];
  __shared__ double s_scr[2 * SM_MAXNP * SM_MAXNP];
  build_mortar_ops(np, b, sigma, s_ops, s_scr);
  for (int r = threadIdx.x; r < 4 * np * np; r += blockDim.x) out[r] = s_ops[r];
}

}  // namespace

cudaError_t launch_stage_params(const MeshDev& m, int np, StageParams* sp, double* t_dev, double t_arg,
                                double ck, double dt, int mode, cudaStream_t st) {
  stage_params_kernel<<<1, 64, 0, st>>>(m, np, sp, t_dev, t_arg, ck, dt, mode);
  return cudaGetLastError();
}

cudaError_t launch_step_params(const MeshDev& m, int np, StageParams* sp5, double* t_dev, const double* ck, double dt,
                               unsigned* ticket, cudaStream_t st) {
  StepCoeffs c;
  for (int k = 0; k < 5; ++k) c.c[k] = ck[k];
  step_params_kernel<<<5, 64, 0, st>>>(m, np, sp5, t_dev, c, dt, ticket);
  return cudaGetLastError();
}

cudaError_t launch_map_batch(const double* d_delta, int count, double l, int n_par, long long* d_n, double* d_s,
                             int* d_pairs, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  map_batch_kernel<<<(count + 127) / 128, 128, 0, st>>>(d_delta, count, l, n_par, d_n, d_s, d_pairs);
  return cudaGetLastError();
}

cudaError_t launch_mortar_ops(const BasisDev* b, int np, double sigma, double* d_out, cudaStream_t st) {
  mortar_ops_kernel<<<1, 64, 0, st>>>(b, np, sigma, d_out);
  return cudaGetLastError();
}

// Global FP64 reductions (Sec. 5.3: the global time step is the only
// all-to-all operation of the method): conserved totals, kinetic energy and its
// rate, and the CFL/DFL rates of Eqs. CFLCondition/DFLCondition evaluated per
// reference direction through the metrics.  Per-block partials (deterministic
// order), summed on the host in FP64.
#pragma once
#include "dg_common.cuh"
#include "launch.h"

namespace flexi {

constexpr int RED_T = 256;
constexpr int RED_Q = 9;  // 5 totals, KE, dKE/dt, max conv rate, max visc rate

template <typename real>
__global__ void __launch_bounds__(RED_T) k_reduce(const real* __restrict__ U, const real* __restrict__ Ut,
                                                 const double* __restrict__ wJ, const double* __restrict__ Ja64,
                                                 const double* __restrict__ sJ64, double* __restrict__ partial,
                                                 long long nodes, int n3, Phys<real> ph, double kv_coef) {
  double acc[RED_Q];
#pragma unroll
  for (int q = 0; q < RED_Q; ++q) acc[q] = 0.0;
  for (long long idx = (long long)blockIdx.x * RED_T + threadIdx.x; idx < nodes; idx += (long long)gridDim.x * RED_T) {
    const long long e = idx / n3;
    const int node = idx % n3;
    double u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = (double)U[(e * NV + v) * n3 + node];
    const double w = wJ[idx];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] += w * u[v];
    const double ir = 1.0 / u[0];
    const double vel[3] = {u[1] * ir, u[2] * ir, u[3] * ir};
    const double q2 = vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2];
    acc[5] += w * 0.5 * u[0] * q2;
    if (Ut != nullptr) {
      double ut[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) ut[v] = (double)Ut[(e * NV + v) * n3 + node];
      acc[6] += w * (vel[0] * ut[1] + vel[1] * ut[2] + vel[2] * ut[3] - 0.5 * q2 * ut[0]);
    }
    const double g = (double)ph.gamma;
    const double p = (g - 1.0) * (u[4] - 0.5 * u[0] * q2);
    const double c = sqrt(g * p * ir);
    const double sj = sJ64[idx];
    double lc = 0.0, lv = 0.0;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const double a0 = Ja64[(e * 9 + l * 3 + 0) * n3 + node];
      const double a1 = Ja64[(e * 9 + l * 3 + 1) * n3 + node];
      const double a2 = Ja64[(e * 9 + l * 3 + 2) * n3 + node];
      const double nrm = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
      lc += (fabs(a0 * vel[0] + a1 * vel[1] + a2 * vel[2]) + c * nrm) * sj;
      lv += (nrm * sj) * (nrm * sj);
    }
    lv *= kv_coef * ir;
    acc[7] = fmax(acc[7], lc);
    acc[8] = fmax(acc[8], lv);
  }
  __shared__ double red[RED_Q][RED_T];
#pragma unroll
  for (int q = 0; q < RED_Q; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = RED_T / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int q = 0; q < 7; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
      red[7][threadIdx.x] = fmax(red[7][threadIdx.x], red[7][threadIdx.x + s]);
      red[8][threadIdx.x] = fmax(red[8][threadIdx.x], red[8][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x < RED_Q) partial[(size_t)blockIdx.x * RED_Q + threadIdx.x] = red[threadIdx.x][0];
}

template <typename real>
cudaError_t launch_reduce(const real* U, const real* Ut, const double* wJ, const double* Ja64, const double* sJ64,
                          long long nodes, int n3, const Phys<real>& ph, double kv_coef, double* partial,
                          int nblocks, cudaStream_t st) {
  k_reduce<real><<<nblocks, RED_T, 0, st>>>(U, Ut, wJ, Ja64, sJ64, partial, nodes, n3, ph, kv_coef);
  return cudaGetLastError();
}

}  // namespace flexi

// Allocation-free variant of the global reductions: flexi_reduce_noalloc.
//
// Some callers cannot allocate device memory at the moment they need these
// sums, for example a solver embedded in an application whose memory manager
// owns all device memory, or code that must not call cudaMalloc/cudaFree in
// the middle of a time loop because those calls synchronise the whole device
// with the work other streams are running.  flexi_reduce keeps its partial sums
// in a buffer that flexi_mesh_init allocated for the context; this variant
// keeps them instead in a fixed-size array in the library's own static device
// memory, so the call itself allocates nothing.
//
// The array below is part of the module image: every GPU that loads the
// library holds it (kNoAllocMaxElements * 9 + 9 doubles, about 4.5 MiB) until
// the process exits.  All calls share it and it keeps the values of the last
// call; each call writes every entry it reads.  Calls whose kernels overlap on
// the GPU (two streams, or two host threads on one device) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/flexi.h"
#include "k_reduce.cuh"
#include "launch.h"

namespace flexi {

constexpr int kNoAllocMaxElements = FLEXI_NOALLOC_MAX_ELEMENTS;
constexpr int kQ = 9;  // 5 totals, kinetic energy, dKE/dt, max convective rate, max viscous rate

static __device__ __align__(256) double g_noalloc_scratch[(kNoAllocMaxElements + 1) * kQ];

constexpr int kElemThreads = 512;   // threads per element CTA: one per node, n^3 <= 512 (N <= 7)
constexpr int kFinishThreads = 256;  // threads of the single CTA that sums the element partials

// one CTA of 512 threads per element: FP64 sums over its n^3 <= 512 nodes -> partial[e][q]
template <typename real>
__global__ void k_reduce_elem(const real* __restrict__ U, const real* __restrict__ Ut, const double* __restrict__ wJ,
                              const double* __restrict__ Ja64, const double* __restrict__ sJ64,
                              double* __restrict__ partial, int n3, Phys<real> ph, double kv_coef) {
  __shared__ double red[kQ][kElemThreads];
  const long long e = blockIdx.x;
  const int node = threadIdx.x;
  double acc[kQ];
#pragma unroll
  for (int q = 0; q < kQ; ++q) acc[q] = 0.0;
  if (node < n3) {
    const long long idx = e * n3 + node;
    double u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = (double)U[(e * NV + v) * n3 + node];
    const double w = wJ[idx];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = w * u[v];
    const double ir = 1.0 / u[0];
    const double vel[3] = {u[1] * ir, u[2] * ir, u[3] * ir};
    const double q2 = vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2];
    acc[5] = w * 0.5 * u[0] * q2;
    if (Ut != nullptr) {
      double ut[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) ut[v] = (double)Ut[(e * NV + v) * n3 + node];
      acc[6] = w * (vel[0] * ut[1] + vel[1] * ut[2] + vel[2] * ut[3] - 0.5 * q2 * ut[0]);
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
    acc[7] = lc;
    acc[8] = lv * kv_coef * ir;
  }
#pragma unroll
  for (int q = 0; q < kQ; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = kElemThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int q = 0; q < 7; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
      red[7][threadIdx.x] = fmax(red[7][threadIdx.x], red[7][threadIdx.x + s]);
      red[8][threadIdx.x] = fmax(red[8][threadIdx.x], red[8][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x < kQ) partial[e * kQ + threadIdx.x] = red[threadIdx.x][0];
}

// one CTA: sums the K element partials in a fixed order -> result[q]
__global__ void k_reduce_finish(const double* __restrict__ partial, double* __restrict__ result, int K) {
  __shared__ double red[kQ][kFinishThreads];
  double acc[kQ];
#pragma unroll
  for (int q = 0; q < kQ; ++q) acc[q] = 0.0;
  for (int e = threadIdx.x; e < K; e += kFinishThreads) {
#pragma unroll
    for (int q = 0; q < 7; ++q) acc[q] += partial[(long long)e * kQ + q];
    acc[7] = fmax(acc[7], partial[(long long)e * kQ + 7]);
    acc[8] = fmax(acc[8], partial[(long long)e * kQ + 8]);
  }
#pragma unroll
  for (int q = 0; q < kQ; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = kFinishThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int q = 0; q < 7; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
      red[7][threadIdx.x] = fmax(red[7][threadIdx.x], red[7][threadIdx.x + s]);
      red[8][threadIdx.x] = fmax(red[8][threadIdx.x], red[8][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x < kQ) result[threadIdx.x] = red[threadIdx.x][0];
}


// Device address of the static array, looked up once per device (with that
// device current) by the first call on it.  In host code the array's name
// stands for a host-side shadow, never for the device memory itself.
constexpr int kMaxDevices = 64;
static double* g_scratch_dev[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mu;

static cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_dev[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

template <typename real>
static cudaError_t launch_noalloc(const ReduceInputs& in, const void* U, const void* Ut, const Phys<real>& ph,
                                  double* scratch, cudaStream_t st) {
  // kElemThreads threads per element: nodes beyond n^3 contribute zeros
  k_reduce_elem<real><<<in.K, kElemThreads, 0, st>>>((const real*)U, (const real*)Ut, in.wJ, in.Ja64, in.sJ64, scratch,
                                                in.n3, ph, in.kv_coef);
  k_reduce_finish<<<1, kFinishThreads, 0, st>>>(scratch, scratch + (size_t)kNoAllocMaxElements * kQ, in.K);
  return cudaGetLastError();
}

}  // namespace flexi

using namespace flexi;

extern "C" flexi_status flexi_reduce_noalloc(flexi_ctx* ctx, const void* U, const void* Ut, double cfl, double* out,
                                             void* stream) {
  if (ctx == nullptr || U == nullptr || out == nullptr) return FLEXI_EINVAL;
  ReduceInputs in;
  if (!ctx_reduce_inputs(ctx, &in)) return FLEXI_EINVAL;
  if (in.K > kNoAllocMaxElements) return FLEXI_EINVAL;  // beyond the static array
  if (in.n3 > kElemThreads) return FLEXI_EUNSUPPORTED;   // one thread per node in k_reduce_elem
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != in.device) return FLEXI_EINVAL;  // the context's device only
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return FLEXI_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const cudaError_t e = in.fp64 ? launch_noalloc<double>(in, U, Ut, in.ph64, scratch, st)
                                : launch_noalloc<float>(in, U, Ut, in.ph32, scratch, st);
  if (e != cudaSuccess) return FLEXI_ECUDA;
  double res[kQ];
  unsigned flag = 0;
  if (cudaMemcpyAsync(res, scratch + (size_t)kNoAllocMaxElements * kQ, sizeof(res), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(&flag, in.status, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FLEXI_ECUDA;
  for (int q = 0; q < 7; ++q) out[q] = res[q];
  const double dtc = cfl * 2.0 / ((2.0 * in.N + 1.0) * res[7]);
  const double dtv = res[8] > 0 ? cfl * 4.0 / ((2.0 * in.N + 1.0) * res[8]) : INFINITY;
  out[7] = std::min(dtc, dtv);
  if (flag) {
    if (cudaMemsetAsync(const_cast<unsigned*>(in.status), 0, sizeof(unsigned), st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return FLEXI_ECUDA;
    return FLEXI_ENONPHYSICAL;
  }
  return FLEXI_OK;
}

// Mortar kernels for non-conforming interfaces (Sec. "Non-conforming meshes"),
// one CTA per mortar with the face data in shared memory and the tensor-product
// operators applied one direction at a time.
//
// A big side cut into halves (type 1: along p, type 2: along q) or quarters
// (type 3) is represented by one side per small face ("virtual" side, master =
// the small element, frame = the small element's side frame) and one big side
// (master = the big element).  Per stage:
//   k_mortar_interp<CONS=1>  big side's face state -> slot 1 of its virtual sides:
//                            the solution U (from the stored primitives) is
//                            interpolated with I^a along each cut direction and
//                            converted back to primitives
//   k_mortar_project<0>      BR1 lifting flux of the big element: minus the L2
//                            projection (P^a) of U* n s_hat of its virtual sides
//   k_mortar_interp<CONS=0>  lifted gradients of the big side -> virtual sides
//   k_mortar_project<1>      f* s_hat of the big side: minus the projection of
//                            the virtual sides' fluxes (their normal is the small
//                            element's outward normal)
// Sub-square positions: a (lower/upper half along p) and b (along q); a virtual
// side's orientation code o maps its (p, q) to the sub-square node (p', q'),
// oinv maps back.
#pragma once
#include "dg_common.cuh"
#include "launch.h"

namespace flexi {

// sub-square position of slot pos of a mortar of type typ
__device__ __forceinline__ void mortar_ab(int typ, int pos, int& a, int& b) {
  a = typ == 3 ? (pos & 1) : (typ == 1 ? pos : 0);
  b = typ == 3 ? (pos >> 1) : (typ == 2 ? pos : 0);
}

constexpr int kMortarThreads = 64;

// CTA per mortar: the big side's NC face values (slot 0; converted to U when
// CONS) are staged in shared memory and interpolated to every small side in two
// one-dimensional passes (along p with I^a, then along q with I^b), then written
// to slot 1 of the small side at its own node (p, q) = T_oinv(p', q').
template <typename real, int n, int NC, bool CONS>
__global__ void __launch_bounds__(kMortarThreads) k_mortar_interp(real* __restrict__ F, const int* __restrict__ mbig,
                                                                  const int4* __restrict__ mvirt, int S, int bigBase,
                                                                  int vbase, MortarOps<real> mo, Phys<real> ph) {
  constexpr int n2 = n * n;
  __shared__ real sB[NC * n2];
  __shared__ real sT[NC * n2];
  const int tid = threadIdx.x;
  const int bi = blockIdx.x;
  const int* mb = mbig + bi * 8;
  const int typ = mb[0];
  const real* big = F + (size_t)(bigBase + bi) * NC * n2;
  for (int t = tid; t < n2; t += kMortarThreads) {
    real val[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) val[c] = big[c * n2 + t];
    if constexpr (CONS) {
      real u[NV];
      prim_to_cons(val, u, ph);
#pragma unroll
      for (int c = 0; c < NV; ++c) sB[c * n2 + t] = u[c];
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) sB[c * n2 + t] = val[c];
    }
  }
  __syncthreads();
  for (int pos = 0; pos < 4; ++pos) {
    const int v = mb[1 + pos];
    if (v < 0) continue;  // uniform across the CTA
    int a, b;
    mortar_ab(typ, pos, a, b);
    const int oinv = mvirt[v - vbase].w;
    // pass along p: sT[q][p'] = sum_m I^a[p'][m] sB[q][m]
    for (int t = tid; t < n2; t += kMortarThreads) {
      const int q = t / n, pp = t - q * n;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        real y;
        if (typ & 1) {
          y = real(0);
#pragma unroll
          for (int m = 0; m < n; ++m) y += mo.I[a][pp * n + m] * sB[c * n2 + q * n + m];
        } else {
          y = sB[c * n2 + t];
        }
        sT[c * n2 + t] = y;
      }
    }
    __syncthreads();
    // pass along q and write: sub node (p', q') -> small side node T_oinv(p', q')
    for (int t = tid; t < n2; t += kMortarThreads) {
      const int qq = t / n, pp = t - qq * n;
      real y[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (typ & 2) {
          y[c] = real(0);
#pragma unroll
          for (int m = 0; m < n; ++m) y[c] += mo.I[b][qq * n + m] * sT[c * n2 + m * n + pp];
        } else {
          y[c] = sT[c * n2 + t];
        }
      }
      real* dst = F + ((size_t)(S + v) * NC) * n2 + orient_pq(oinv, n - 1, pp, qq);
      if constexpr (CONS) {
        real W[NV];
        cons_to_prim(y, W, ph);
#pragma unroll
        for (int c = 0; c < NV; ++c) dst[c * n2] = W[c];
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) dst[c * n2] = y[c];
      }
    }
    __syncthreads();
  }
}

// CTA per mortar: minus the L2 projection of the small sides' values onto the big
// side.  KIND 0: BR1 lifting flux U* n s_hat (15 values) from the small sides'
// face states, written to QB; KIND 1: numerical flux f* s_hat (5 values) from Ff,
// written to the big side's Ff.  Each small side's values are gathered into its
// sub-square frame, projected along q (P^b), then along p (P^a) and accumulated.
template <typename real, int n, int KIND>
__global__ void __launch_bounds__(kMortarThreads) k_mortar_project(
    const real* __restrict__ Wf, const real* __restrict__ fgeo, real* __restrict__ Ff, real* __restrict__ QB,
    const int* __restrict__ mbig, const int4* __restrict__ mvirt, int S, int bigBase, int vbase, MortarOps<real> mo) {
  constexpr int n2 = n * n;
  constexpr int NC = KIND == 0 ? 15 : NV;
  constexpr int PT = (n2 + kMortarThreads - 1) / kMortarThreads;  // big nodes per thread
  __shared__ real sV[NC * n2];
  __shared__ real sT[NC * n2];
  const int tid = threadIdx.x;
  const int bi = blockIdx.x;
  const int* mb = mbig + bi * 8;
  const int typ = mb[0];
  real acc[PT][NC];
#pragma unroll
  for (int k = 0; k < PT; ++k)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[k][c] = real(0);
  for (int pos = 0; pos < 4; ++pos) {
    const int v = mb[1 + pos];
    if (v < 0) continue;  // uniform across the CTA
    int a, b;
    mortar_ab(typ, pos, a, b);
    const int oinv = mvirt[v - vbase].w;
    for (int t = tid; t < n2; t += kMortarThreads) {  // gather into the sub-square frame
      const int spq = orient_pq(oinv, n - 1, t % n, t / n);
      if constexpr (KIND == 0) {
        const real* w0 = Wf + ((size_t)v * NV) * n2 + spq;
        const real* w1 = Wf + ((size_t)(S + v) * NV) * n2 + spq;
        const real* g = fgeo + ((size_t)v * 4) * n2 + spq;
        const real sa = g[3 * n2];
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          const real ws = real(0.5) * (w0[c * n2] + w1[c * n2]) * sa;
#pragma unroll
          for (int d = 0; d < 3; ++d) sV[(c * 3 + d) * n2 + t] = ws * g[d * n2];
        }
      } else {
#pragma unroll
        for (int c = 0; c < NV; ++c) sV[c * n2 + t] = Ff[((size_t)v * NV + c) * n2 + spq];
      }
    }
    __syncthreads();
    // along q: sT[j][al] = sum_be P^b[j][be] sV[be][al]
    for (int t = tid; t < n2; t += kMortarThreads) {
      const int j = t / n, al = t - j * n;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        real y;
        if (typ & 2) {
          y = real(0);
#pragma unroll
          for (int m = 0; m < n; ++m) y += mo.P[b][j * n + m] * sV[c * n2 + m * n + al];
        } else {
          y = sV[c * n2 + t];
        }
        sT[c * n2 + t] = y;
      }
    }
    __syncthreads();
    // along p, accumulated per big node (i, j)
#pragma unroll
    for (int k = 0; k < PT; ++k) {
      const int t = tid + k * kMortarThreads;
      if (t < n2) {
        const int j = t / n, i = t - j * n;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          if (typ & 1) {
#pragma unroll
            for (int m = 0; m < n; ++m) acc[k][c] -= mo.P[a][i * n + m] * sT[c * n2 + j * n + m];
          } else {
            acc[k][c] -= sT[c * n2 + t];
          }
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < PT; ++k) {
    const int t = tid + k * kMortarThreads;
    if (t < n2) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if constexpr (KIND == 0)
          QB[((size_t)bi * 15 + c) * n2 + t] = acc[k][c];
        else
          Ff[((size_t)(bigBase + bi) * NV + c) * n2 + t] = acc[k][c];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename real>
cudaError_t launch_mortar_state(const DevMesh& m, const MortarOps<real>& mo, const Phys<real>& ph, cudaStream_t st) {
  if (m.nBig == 0) return cudaSuccess;
  const int4* mv = (const int4*)m.mvirt;
  FLEXI_DISPATCH_N(m.n, (k_mortar_interp<real, NN, NV, true><<<m.nBig, kMortarThreads, 0, st>>>(
                            (real*)m.Wf, m.mbig, mv, m.S, m.Sface, m.vbase, mo, ph)));
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  FLEXI_DISPATCH_N(m.n, (k_mortar_project<real, NN, 0><<<m.nBig, kMortarThreads, 0, st>>>(
                            (const real*)m.Wf, (const real*)m.fgeo, nullptr, (real*)m.QB, m.mbig, mv, m.S, m.Sface,
                            m.vbase, mo)));
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_mortar_grad(const DevMesh& m, const MortarOps<real>& mo, const Phys<real>& ph, cudaStream_t st) {
  if (m.nBig == 0) return cudaSuccess;
  FLEXI_DISPATCH_N(m.n, (k_mortar_interp<real, NN, 15, false><<<m.nBig, kMortarThreads, 0, st>>>(
                            (real*)m.Gf, m.mbig, (const int4*)m.mvirt, m.S, m.Sface, m.vbase, mo, ph)));
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_mortar_flux(const DevMesh& m, const MortarOps<real>& mo, cudaStream_t st) {
  if (m.nBig == 0) return cudaSuccess;
  FLEXI_DISPATCH_N(m.n, (k_mortar_project<real, NN, 1><<<m.nBig, kMortarThreads, 0, st>>>(
                            nullptr, nullptr, (real*)m.Ff, nullptr, m.mbig, (const int4*)m.mvirt, m.S, m.Sface,
                            m.vbase, mo)));
  return cudaGetLastError();
}

}  // namespace flexi

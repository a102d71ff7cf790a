// Mortar kernels for non-conforming interfaces (Sec. "Non-conforming meshes").
//
// A big side cut into halves (type 1: along p, type 2: along q) or quarters
// (type 3) is represented by one side per small face ("virtual" side, master =
// the small element, frame = the small element's side frame) and one big side
// (master = the big element).  Per stage:
//   k_mortar_interp<CONS=1>  big side's face state -> slot 1 of its virtual sides:
//                            the solution U (from the stored primitives) is
//                            interpolated with I^a along each cut direction and
//                            converted back to primitives
//   k_mortar_lift            BR1 lifting flux of the big element: minus the L2
//                            projection (P^a) of U* n s_hat of its virtual sides
//   k_mortar_interp<CONS=0>  lifted gradients of the big side -> virtual sides
//   k_mortar_flux            f* s_hat of the big side: minus the projection of
//                            the virtual sides' fluxes (their normal is the small
//                            element's outward normal)
// Sub-square positions: a (lower/upper half along p) and b (along q); a virtual
// side's orientation code o maps its (p, q) to the sub-square node (p', q'),
// oinv maps back.
#pragma once
#include "dg_common.cuh"
#include "launch.h"

namespace flexi {

// thread per (virtual side, node): values of the big side interpolated to the node
template <typename real, int n, int NC, bool CONS>
__global__ void __launch_bounds__(128) k_mortar_interp(real* __restrict__ F, const int4* __restrict__ mvirt, int S,
                                                       int vbase, int nV, MortarOps<real> mo, Phys<real> ph) {
  constexpr int n2 = n * n;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nV * n2) return;
  const int vi = idx / n2, pq = idx - vi * n2;
  const int4 mv = mvirt[vi];
  const int typ = mv.y & 3, a = (mv.y >> 2) & 1, b = (mv.y >> 3) & 1;
  const int sub = orient_pq(mv.z, n - 1, pq % n, pq / n);
  const int pp = sub % n, qq = sub / n;
  const real* big = F + (size_t)mv.x * NC * n2;  // slot 0: the big element's face values
  real acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = real(0);
  const int q0 = (typ & 2) ? 0 : qq, q1 = (typ & 2) ? n - 1 : qq;
  const int p0 = (typ & 1) ? 0 : pp, p1 = (typ & 1) ? n - 1 : pp;
  for (int m2 = q0; m2 <= q1; ++m2) {
    const real wq = (typ & 2) ? mo.I[b][qq * n + m2] : real(1);
    for (int m1 = p0; m1 <= p1; ++m1) {
      const real w = wq * ((typ & 1) ? mo.I[a][pp * n + m1] : real(1));
      real val[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) val[c] = big[c * n2 + m2 * n + m1];
      if constexpr (CONS) {
        real u[NV];
        prim_to_cons(val, u, ph);
#pragma unroll
        for (int c = 0; c < NV; ++c) acc[c] += w * u[c];
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] += w * val[c];
      }
    }
  }
  real* dst = F + ((size_t)(S + vbase + vi) * NC) * n2 + pq;
  if constexpr (CONS) {
    real W[NV];
    cons_to_prim(acc, W, ph);
#pragma unroll
    for (int c = 0; c < NV; ++c) dst[c * n2] = W[c];
  } else {
#pragma unroll
    for (int c = 0; c < NC; ++c) dst[c * n2] = acc[c];
  }
}

// sub-square position of slot pos of a mortar of type typ
__device__ __forceinline__ void mortar_ab(int typ, int pos, int& a, int& b) {
  a = typ == 3 ? (pos & 1) : (typ == 1 ? pos : 0);
  b = typ == 3 ? (pos >> 1) : (typ == 2 ? pos : 0);
}

// thread per (big side, node (i, j)): minus the L2 projection of NC values per
// virtual-side node produced by `val` (virtual side, its node index, out[NC])
template <typename real, int n, int NC, typename ValFn>
__device__ __forceinline__ void mortar_project(int typ, const int* mb, const int4* __restrict__ mvirt, int vbase,
                                               int i, int j, const MortarOps<real>& mo, ValFn val, real acc[NC]) {
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = real(0);
  for (int pos = 0; pos < 4; ++pos) {
    const int v = mb[1 + pos];
    if (v < 0) continue;
    int a, b;
    mortar_ab(typ, pos, a, b);
    const int oinv = mvirt[v - vbase].w;
    const int be0 = (typ & 2) ? 0 : j, be1 = (typ & 2) ? n - 1 : j;
    const int al0 = (typ & 1) ? 0 : i, al1 = (typ & 1) ? n - 1 : i;
    for (int be = be0; be <= be1; ++be) {
      const real wq = (typ & 2) ? mo.P[b][j * n + be] : real(1);
      for (int al = al0; al <= al1; ++al) {
        const real w = wq * ((typ & 1) ? mo.P[a][i * n + al] : real(1));
        real x[NC];
        val(v, orient_pq(oinv, n - 1, al, be), x);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] -= w * x[c];
      }
    }
  }
}

template <typename real, int n>
__global__ void __launch_bounds__(128) k_mortar_lift(const real* __restrict__ Wf, const real* __restrict__ fgeo,
                                                     const int* __restrict__ mbig, const int4* __restrict__ mvirt,
                                                     real* __restrict__ QB, int S, int vbase, int nBig,
                                                     MortarOps<real> mo) {
  constexpr int n2 = n * n;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nBig * n2) return;
  const int bi = idx / n2, ij = idx - bi * n2;
  const int* mb = mbig + bi * 8;
  real acc[15];
  auto lift_flux = [&](int v, int pq, real x[15]) {
    const real* w0 = Wf + ((size_t)v * NV) * n2 + pq;
    const real* w1 = Wf + ((size_t)(S + v) * NV) * n2 + pq;
    const real* g = fgeo + ((size_t)v * 4) * n2 + pq;
    const real sa = g[3 * n2];
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      const real ws = real(0.5) * (w0[c * n2] + w1[c * n2]) * sa;
#pragma unroll
      for (int d = 0; d < 3; ++d) x[c * 3 + d] = ws * g[d * n2];
    }
  };
  mortar_project<real, n, 15>(mb[0], mb, mvirt, vbase, ij % n, ij / n, mo, lift_flux, acc);
#pragma unroll
  for (int c = 0; c < 15; ++c) QB[((size_t)bi * 15 + c) * n2 + ij] = acc[c];
}

template <typename real, int n>
__global__ void __launch_bounds__(128) k_mortar_flux(real* __restrict__ Ff, const int* __restrict__ mbig,
                                                     const int4* __restrict__ mvirt, int vbase, int bigBase, int nBig,
                                                     MortarOps<real> mo) {
  constexpr int n2 = n * n;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nBig * n2) return;
  const int bi = idx / n2, ij = idx - bi * n2;
  const int* mb = mbig + bi * 8;
  real acc[NV];
  auto flux = [&](int v, int pq, real x[NV]) {
#pragma unroll
    for (int c = 0; c < NV; ++c) x[c] = Ff[((size_t)v * NV + c) * n2 + pq];
  };
  mortar_project<real, n, NV>(mb[0], mb, mvirt, vbase, ij % n, ij / n, mo, flux, acc);
#pragma unroll
  for (int c = 0; c < NV; ++c) Ff[((size_t)(bigBase + bi) * NV + c) * n2 + ij] = acc[c];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename real>
cudaError_t launch_mortar_state(const DevMesh& m, const MortarOps<real>& mo, const Phys<real>& ph, cudaStream_t st) {
  if (m.nBig == 0) return cudaSuccess;
  const int tv = m.nV * m.n * m.n, tb = m.nBig * m.n * m.n;
  const int4* mv = (const int4*)m.mvirt;
  FLEXI_DISPATCH_N(m.n, (k_mortar_interp<real, NN, NV, true><<<(tv + 127) / 128, 128, 0, st>>>(
                            (real*)m.Wf, mv, m.S, m.vbase, m.nV, mo, ph)));
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  FLEXI_DISPATCH_N(m.n, (k_mortar_lift<real, NN><<<(tb + 127) / 128, 128, 0, st>>>(
                            (const real*)m.Wf, (const real*)m.fgeo, m.mbig, mv, (real*)m.QB, m.S, m.vbase, m.nBig,
                            mo)));
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_mortar_grad(const DevMesh& m, const MortarOps<real>& mo, const Phys<real>& ph, cudaStream_t st) {
  if (m.nBig == 0) return cudaSuccess;
  const int tv = m.nV * m.n * m.n;
  FLEXI_DISPATCH_N(m.n, (k_mortar_interp<real, NN, 15, false><<<(tv + 127) / 128, 128, 0, st>>>(
                            (real*)m.Gf, (const int4*)m.mvirt, m.S, m.vbase, m.nV, mo, ph)));
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_mortar_flux(const DevMesh& m, const MortarOps<real>& mo, cudaStream_t st) {
  if (m.nBig == 0) return cudaSuccess;
  const int tb = m.nBig * m.n * m.n;
  FLEXI_DISPATCH_N(m.n, (k_mortar_flux<real, NN><<<(tb + 127) / 128, 128, 0, st>>>(
                            (real*)m.Ff, m.mbig, (const int4*)m.mvirt, m.vbase, m.Sface, m.nBig, mo)));
  return cudaGetLastError();
}

}  // namespace flexi

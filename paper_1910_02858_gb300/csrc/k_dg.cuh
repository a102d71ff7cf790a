// Forward DGSEM kernels (templated on the arithmetic type and on n = N + 1).
//
// Per RK stage (Sec. 5.5 algorithm sequence, re-scheduled for one GPU):
//   k_prolong   element kernel: U -> primitive face states W(U_face) (a1)
//   k_bc        boundary sides: outer state (exact state, outflow or slip wall)
//   (mortar meshes: k_mortar.cuh interpolates and projects around k_lift_vol and k_face)
//   k_lift_vol  element kernel: BR1 lifting (a2, a3, Eq. discreteGradient),
//               gradients to the faces (a4), volume fluxes + contravariant
//               transform (a6) and the D_hat volume integral (a7)
//   k_face      side kernel: Riemann + BR1 viscous flux times s_hat (a5)
//   k_surf      element kernel: surface integral (a8), -1/J scaling (a9), the
//               low-storage RK update (a10) and the face states of the new U
//
// One thread per volume node; NE elements per CTA so that a CTA has >= 64
// threads for small n.  Line sweeps of D_hat read the element's staged fields
// from shared memory; the per-node results stay in registers.
#pragma once
#include <type_traits>

#include "dg_common.cuh"
#include "k_tc.cuh"
#include "launch.h"

namespace flexi {

// shared copy of the 1-D operators: DhatT[n*n], lm, lp, lhm, lhp
template <typename real, int n>
__device__ __forceinline__ void load_ops(real* s, const Ops<real>& ops, int tid, int T) {
  for (int t = tid; t < n * n; t += T) s[t] = ops.DhatT[t];
  for (int t = tid; t < n; t += T) {
    s[n * n + t] = ops.lm[t];
    s[n * n + n + t] = ops.lp[t];
    s[n * n + 2 * n + t] = ops.lhm[t];
    s[n * n + 3 * n + t] = ops.lhp[t];
  }
}

// Three D_hat line sweeps of the 15 staged fields of every element of the CTA:
//   out[el][v][node] = sum_l sum_a Dhat[i_l][a] buf[el][l*5+v][node with index_l = a].
// One thread per line: the line's n values are read once from shared memory and
// D_hat comes from the kernel-parameter bank at compile-time offsets.  The three
// directions accumulate into out one after the other.  With Q != nullptr (the
// lifting of gradient component d) the two face terms of each line,
// l_hat_i(-1) Q[-face] + l_hat_i(+1) Q[+face], are added in the same pass
// (the face node of a line of direction l has (p, q) = the line's free indices).
// Block-wide; ends synced.
template <typename real, int n, bool LGL>
__device__ __forceinline__ void line_sweep3(const real* __restrict__ buf, real* __restrict__ out,
                                            const real* __restrict__ Q, int d, const Ops<real>& ops, int tid) {
  using C = Cfg<n>;
  constexpr int n2 = C::n2, n3p = C::n3p, P = C::P, NE = C::NE, T = C::T;
  constexpr int L = NE * NV * n2;
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const int stride = l == 0 ? 1 : (l == 1 ? P : P * n);
    for (int it = tid; it < L; it += T) {
      const int el = NE == 1 ? 0 : it / (NV * n2);  // it < L: one element per CTA for n >= 4
      const int r = it - el * NV * n2;
      const int v = r / n2, line = r - v * n2;
      const int a0 = line % n, a1 = line / n;  // free indices in increasing direction order
      const int base = l == 0 ? P * line : (l == 1 ? a0 + P * n * a1 : a0 + P * a1);
      const real* src = buf + (el * 15 + l * NV + v) * n3p + base;
      real x[n];
#pragma unroll
      for (int a = 0; a < n; ++a) x[a] = src[a * stride];
      real qm = real(0), qp = real(0);
      if (Q != nullptr) {
        qm = Q[((el * 6 + 2 * l) * 15 + v * 3 + d) * n2 + line];
        qp = Q[((el * 6 + 2 * l + 1) * 15 + v * 3 + d) * n2 + line];
      }
      real* dst = out + (el * NV + v) * n3p + base;
#pragma unroll
      for (int ii = 0; ii < n; ++ii) {
        // on Gauss-Lobatto nodes l_hat(-1) / l_hat(+1) vanish except at the line's ends
        real y = LGL ? (ii == 0 ? ops.lhm[0] * qm : (ii == n - 1 ? ops.lhp[n - 1] * qp : real(0)))
                     : ops.lhm[ii] * qm + ops.lhp[ii] * qp;
#pragma unroll
        for (int a = 0; a < n; ++a) y += ops.DhatT[a * n + ii] * x[a];
        dst[ii * stride] = (l == 0) ? y : dst[ii * stride] + y;
      }
    }
    __syncthreads();
  }
}

// The FP32 CUDA-core lifting sweeps either 5 fields per (gradient component,
// direction) (line_sweep3, nine sweeps) or 15 fields per direction (lift_sweep,
// three sweeps); the 15-field form is taken where it fills the CTA's threads
// better: 3 * passes(5 fields) > passes(15 fields), with passes = ceil(lines / T).
// n = 8: 320 of 512 threads busy in one pass against 960 tasks in two; n = 5, 6, 7
// fill equally (or worse) and keep the 5-field sweeps.
template <int n>
constexpr bool lift15_fills_better() {
  using C = Cfg<n>;
  constexpr int L5 = C::NE * NV * C::n2, T = C::T;
  return 3 * ((L5 + T - 1) / T) > (3 * L5 + T - 1) / T;
}

// One line of lift_sweep (task it = (element, field d*5+v, line)).
template <typename real, int n, bool LGL, int l>
__device__ __forceinline__ void lift_line(const real* __restrict__ buf, real* __restrict__ out,
                                          const real* __restrict__ Q, const Ops<real>& ops, int it) {
  using C = Cfg<n>;
  constexpr int n2 = C::n2, n3p = C::n3p, P = C::P, NE = C::NE;
  constexpr int stride = l == 0 ? 1 : (l == 1 ? P : P * n);
  const int el = NE == 1 ? 0 : it / (15 * n2);
  const int r = it - el * 15 * n2;
  const int c = r / n2, line = r - c * n2;
  const int d = c / NV, v = c - d * NV;
  const int a0 = line % n, a1 = line / n;  // free indices in increasing direction order
  const int base = l == 0 ? P * line : (l == 1 ? a0 + P * n * a1 : a0 + P * a1);
  const real* src = buf + (el * 15 + c) * n3p + base;
  real x[n];
#pragma unroll
  for (int a = 0; a < n; ++a) x[a] = src[a * stride];
  const real qm = Q[((el * 6 + 2 * l) * 15 + v * 3 + d) * n2 + line];
  const real qp = Q[((el * 6 + 2 * l + 1) * 15 + v * 3 + d) * n2 + line];
  real* dst = out + (el * 15 + c) * n3p + base;
#pragma unroll
  for (int ii = 0; ii < n; ++ii) {
    real y = LGL ? (ii == 0 ? ops.lhm[0] * qm : (ii == n - 1 ? ops.lhp[n - 1] * qp : real(0)))
                 : ops.lhm[ii] * qm + ops.lhp[ii] * qp;
#pragma unroll
    for (int a = 0; a < n; ++a) y += ops.DhatT[a * n + ii] * x[a];
    dst[ii * stride] = (l == 0) ? y : dst[ii * stride] + y;
  }
}

// Lifting sweep along one reference direction l for all three gradient components
// at once (FP32 CUDA-core form): buf[el][d*5+v][node] = Ja^l_d W_v is swept with
// D_hat along l into out[el][d*5+v][node] (written for l = 0, accumulated after),
// the face terms l_hat_i(-1) Q[-face] + l_hat_i(+1) Q[+face] of direction l folded
// in.  15 fields x n^2 lines per element keep every thread of the CTA busy, and
// the lifting needs three sweeps instead of nine.  Block-wide; ends synced.
template <typename real, int n, bool LGL, int l>
__device__ __forceinline__ void lift_sweep(const real* __restrict__ buf, real* __restrict__ out,
                                           const real* __restrict__ Q, const Ops<real>& ops, int tid) {
  using C = Cfg<n>;
  constexpr int L = C::NE * 15 * C::n2, T = C::T;
#pragma unroll
  for (int k = 0; k < (L + T - 1) / T; ++k)  // compile-time trip count (a runtime loop spills)
    if (tid + k * T < L) lift_line<real, n, LGL, l>(buf, out, Q, ops, tid + k * T);
  __syncthreads();
}

// Per-node form of line_sweep3's three sweeps (used by the FP64 form, which is bound
// by the FP64 pipe and short of registers for whole lines): the thread of node
// (i,j,k) accumulates sum_a Dhat[i][a] f0(a,j,k) + Dhat[j][a] f1(i,a,k) +
// Dhat[k][a] f2(i,j,a) for the 5 variables, reading the padded staged fields.
template <typename real, int n>
__device__ __forceinline__ void node_sweep3(const real* __restrict__ sD, const real* __restrict__ buf, int i, int j,
                                            int k, real acc[NV]) {
  constexpr int n3p = Cfg<n>::n3p;
#pragma unroll
  for (int a = 0; a < n; ++a) {
    const real d0 = sD[a * n + i], d1 = sD[a * n + j], d2 = sD[a * n + k];
    const int i0 = pidx<n>(a, j, k), i1 = pidx<n>(i, a, k), i2 = pidx<n>(i, j, a);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      acc[v] += d0 * buf[v * n3p + i0];
      acc[v] += d1 * buf[(NV + v) * n3p + i1];
      acc[v] += d2 * buf[(2 * NV + v) * n3p + i2];
    }
  }
}

// Face states of U for all six faces of every element of the CTA, from U staged
// in shared memory with padded lines (sU[el][5][n3p]): one pass per line of
// direction l gives the values on both faces -l and +l (the face node of the
// line has (p, q) = its free indices); W(U_face) goes to the side arrays.
template <typename real, int n, bool LGL>
__device__ __forceinline__ void faces_from_volume(const real* __restrict__ sU, const Ops<real>& ops,
                                                  const int* __restrict__ sES, int e0, int K, int S,
                                                  real* __restrict__ Wf, const Phys<real>& ph,
                                                  unsigned* __restrict__ status, int tid, int T = Cfg<n>::T) {
  using C = Cfg<n>;
  constexpr int n2 = C::n2, n3p = C::n3p, P = C::P;
  if constexpr (sizeof(real) == 8) {
    // FP64 (FP64-pipe bound): one thread per face node keeps more warps on the pipe
    for (int it = tid; it < C::NE * 6 * n2; it += T) {
      const int el = it / (6 * n2);
      const int r = it - el * 6 * n2;
      const int s = r / n2, pq = r - s * n2;
      if (e0 + el >= K) continue;
      const int l = s >> 1, p = pq % n, q = pq / n;
      real Uf[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Uf[v] = real(0);
      if (LGL) {  // the face node is a volume node: a copy
        const int vi = pvol_index<n>(l, (s & 1) ? n - 1 : 0, p, q);
#pragma unroll
        for (int v = 0; v < NV; ++v) Uf[v] = sU[(el * NV + v) * n3p + vi];
      } else {
#pragma unroll
        for (int a = 0; a < n; ++a) {
          const real c = (s & 1) ? ops.lp[a] : ops.lm[a];
          const int vi = pvol_index<n>(l, a, p, q);
#pragma unroll
          for (int v = 0; v < NV; ++v) Uf[v] += c * sU[(el * NV + v) * n3p + vi];
        }
      }
      real W[NV];
      cons_to_prim(Uf, W, ph);
      if (!(W[0] > real(0)) || !(W[4] > real(0))) atomicOr(status, 1u);
      const int es = sES[el * 6 + s];
      const int mpq = orient_pq(es_orient(es), n - 1, p, q);
      real* dst = Wf + ((size_t)(es_slave(es) * S + es_side(es)) * NV) * n2 + mpq;
#pragma unroll
      for (int v = 0; v < NV; ++v) dst[v * n2] = W[v];
    }
    return;
  }
  // items are grouped by direction in runs of n^2 (whole warps for n >= 6): the
  // switch gives each direction compile-time line strides
  auto line_item = [&](auto Lc, int el, int line) {
    constexpr int l = decltype(Lc)::value;
    const int p = line % n, q = line / n;
    constexpr int stride = l == 0 ? 1 : (l == 1 ? P : P * n);
    const int base = l == 0 ? P * line : (l == 1 ? p + P * n * q : p + P * q);
    real Um[NV], Up[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Um[v] = Up[v] = real(0);
    if (LGL) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        Um[v] = sU[(el * NV + v) * n3p + base];
        Up[v] = sU[(el * NV + v) * n3p + base + (n - 1) * stride];
      }
    } else {
#pragma unroll
      for (int a = 0; a < n; ++a) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const real x = sU[(el * NV + v) * n3p + base + a * stride];
          Um[v] += ops.lm[a] * x;
          Up[v] += ops.lp[a] * x;
        }
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      real W[NV], Uh[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Uh[v] = h ? Up[v] : Um[v];
      cons_to_prim(Uh, W, ph);
      if (!(W[0] > real(0)) || !(W[4] > real(0))) atomicOr(status, 1u);
      const int es = sES[el * 6 + 2 * l + h];
      const int mpq = orient_pq(es_orient(es), n - 1, p, q);
      real* dst = Wf + ((size_t)(es_slave(es) * S + es_side(es)) * NV) * n2 + mpq;
#pragma unroll
      for (int v = 0; v < NV; ++v) dst[v * n2] = W[v];
    }
  };
  for (int it = tid; it < C::NE * 3 * n2; it += T) {
    const int el = it / (3 * n2);
    const int r = it - el * 3 * n2;
    const int l = r / n2, line = r - l * n2;
    if (e0 + el >= K) continue;
    if (l == 0)
      line_item(std::integral_constant<int, 0>{}, el, line);
    else if (l == 1)
      line_item(std::integral_constant<int, 1>{}, el, line);
    else
      line_item(std::integral_constant<int, 2>{}, el, line);
  }
}

// ---------------------------------------------------------------------------
// a1: prolongation of U to the faces (primitive face states)
// ---------------------------------------------------------------------------
template <typename real, int n, bool LGL>
__global__ void __launch_bounds__(Cfg<n>::T) k_prolong(const real* __restrict__ U, const int* __restrict__ elemSide,
                                                        real* __restrict__ Wf, int K, int S, Ops<real> ops,
                                                        Phys<real> ph, unsigned* __restrict__ status) {
  using C = Cfg<n>;
  constexpr int n3 = C::n3, n3p = C::n3p;
  __shared__ real sU[C::NE * NV * n3p];
  __shared__ int sES[C::NE * 6];
  const int tid = threadIdx.x;
  const int e0 = blockIdx.x * C::NE;
  for (int t = tid; t < C::NE * 6; t += C::T) sES[t] = (e0 + t / 6 < K) ? elemSide[(size_t)e0 * 6 + t] : 0;
  for (int t = tid; t < C::NE * NV * n3; t += C::T) {
    const int f = t / n3, node = t - f * n3;  // f = el * NV + v
    sU[f * n3p + pidx<n>(node % n, (node / n) % n, node / (n * n))] =
        (e0 + f / NV < K) ? U[(size_t)e0 * NV * n3 + t] : real(1);
  }
  __syncthreads();
  faces_from_volume<real, n, LGL>(sU, ops, sES, e0, K, S, Wf, ph, status, tid);
}

// ---------------------------------------------------------------------------
// boundary sides (weakly imposed through the outer state of the flux): exact state
// at the face nodes (kind 0), the inner state (1, outflow), or the inner state with
// its normal velocity reversed (2, slip wall; the normal is the element's outward one)
// ---------------------------------------------------------------------------
template <typename real, int n>
__global__ void k_bc(const double* __restrict__ xbc, const int* __restrict__ bcKind, const real* __restrict__ fgeo,
                     real* __restrict__ Wf, int S, int nBC, double t, Phys<real> ph) {
  constexpr int n2 = n * n;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nBC * n2) return;
  const int b = idx / n2, pq = idx - b * n2;
  const int kind = bcKind[b];
  real W[NV];
  if (kind == 0) {
    double x[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c] = xbc[((size_t)b * 3 + c) * n2 + pq];
    real U[NV];
    exact_state<real>(ph.bc_exact, x, t, ph, U);
    cons_to_prim(U, W, ph);
  } else {
    const real* src = Wf + ((size_t)b * NV) * n2 + pq;  // slot 0: the element's face state
#pragma unroll
    for (int v = 0; v < NV; ++v) W[v] = src[v * n2];
    if (kind == 2) {
      const real* g = fgeo + ((size_t)b * 4) * n2 + pq;
      const real nx = g[0], ny = g[n2], nz = g[2 * n2];
      const real un = W[1] * nx + W[2] * ny + W[3] * nz;
      W[1] -= real(2) * un * nx;
      W[2] -= real(2) * un * ny;
      W[3] -= real(2) * un * nz;
    }
  }
  real* dst = Wf + ((size_t)(S + b) * NV) * n2 + pq;
#pragma unroll
  for (int v = 0; v < NV; ++v) dst[v * n2] = W[v];
}

// ---------------------------------------------------------------------------
// a2-a4, a6, a7: lifting, gradient prolongation, volume integral
// ---------------------------------------------------------------------------
// BR1 surface terms of the lifting for the NE elements of a CTA: Q = U* n_d s_hat with
// the element's outward normal at every face node ([NE][6][15][n^2], component v*3+d;
// big sides of mortars: the projected lifting flux of their small sides), the
// master-frame node of each face node (sMpq, reused by the gradient prolongation) and,
// with BR2, the jumps (U* - U_e) n s_hat with the element's own face state.
// T threads from tid; no barrier.
template <typename real, int n, int NE, bool BR2>
__device__ __forceinline__ void br1_surface_terms(const real* __restrict__ Wf, const real* __restrict__ fgeo,
                                                  const real* __restrict__ QB, const int* __restrict__ sES,
                                                  real* __restrict__ sQ, int* __restrict__ sMpq,
                                                  real* __restrict__ sJm, int e0, int K, int S, int bigBase, int tid,
                                                  int T) {
  constexpr int n2 = n * n;
  for (int it = tid; it < NE * 6 * n2; it += T) {
    const int el2 = it / (6 * n2);
    const int r = it - el2 * 6 * n2;
    const int s = r / n2, pq = r - s * n2;
    if (e0 + el2 >= K) continue;
    const int es = sES[el2 * 6 + s];
    const int side = es_side(es);
    const int mpq = orient_pq(es_orient(es), n - 1, pq % n, pq / n);
    sMpq[it] = mpq;  // reused by the gradient prolongation
    const real* w0 = Wf + ((size_t)side * NV) * n2 + mpq;
    const real* w1 = Wf + ((size_t)(S + side) * NV) * n2 + mpq;
    const real* g = fgeo + ((size_t)side * 4) * n2 + mpq;
    const real sc = es_slave(es) ? -g[3 * n2] : g[3 * n2];
    const real nd[3] = {g[0] * sc, g[n2] * sc, g[2 * n2] * sc};
    real* Q = sQ + ((el2 * 6 + s) * 15) * n2 + pq;
    if (side >= bigBase) {
      const real* qb = QB + ((size_t)(side - bigBase) * 15) * n2 + mpq;
#pragma unroll
      for (int c = 0; c < 15; ++c) Q[c * n2] = qb[c * n2];
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const real ws = real(0.5) * (w0[v * n2] + w1[v * n2]);
#pragma unroll
        for (int d = 0; d < 3; ++d) Q[(v * 3 + d) * n2] = ws * nd[d];
      }
    }
    if constexpr (BR2) {  // jump (U* - U_e) n s_hat with the element's own face state
      const real* wo = es_slave(es) ? w1 : w0;
      real* Jm = sJm + ((el2 * 6 + s) * 15) * n2 + pq;
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int d = 0; d < 3; ++d) Jm[(v * 3 + d) * n2] = Q[(v * 3 + d) * n2] - wo[v * n2] * nd[d];
    }
  }
}

// Resident CTAs per SM asked of the register allocator, from measurements: FP32
// CUDA-core form two of 512 threads at n = 8 and five of 216 at n = 6 (standard
// form); FP64 an explicit minimum of one, which lets the compiler take more
// registers (about 1 % faster at n = 6 and 8); 0: the compiler's default
// (k_lift_vol without a minimum; an explicit minimum of one halved the occupancy
// of the tensor-core forms).
template <typename real, int n, int SW, int SPLIT, bool BR2>
constexpr int lift_vol_min_blocks() {
  if (sizeof(real) == 8) return 1;
  if (SW != 0) return 0;
  if (Cfg<n>::T == 512) return 2;
  return (Cfg<n>::T == 216 && SPLIT == 0 && !BR2) ? 5 : 0;
}

// SW: 0 line sweeps on the FP32/FP64 pipes; 1 TF32 and 2 BF16 3-term split mma (float only).
// SPLIT (Gauss-Lobatto, SW = 0 only): the split-form volume integral of Sec. 3.3 with the
// kinetic-energy-preserving two-point flux (1) or the entropy-conservative one (2)
// (Eq. semiDiscreteSplit).
template <typename real, int n, int SW, bool LGL, int SPLIT, bool BR2>
__device__ __forceinline__ void lift_vol_body(
    const real* __restrict__ U, const real* __restrict__ Ja, const real* __restrict__ sJ,
    const real* __restrict__ Wf, const real* __restrict__ fgeo, const int* __restrict__ elemSide,
    real* __restrict__ Gf, real* __restrict__ Utv, real* __restrict__ Gvol, int K, int S, int bigBase,
    const real* __restrict__ QB, const Ops<real>& ops, const Phys<real>& ph) {
  using C = Cfg<n>;
  constexpr int n2 = C::n2, n3 = C::n3, NE = C::NE, T = C::T, n3p = C::n3p;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* sbuf = reinterpret_cast<real*>(smem_raw);  // [NE][15][n3p] staged fields (padded lines)
  // FP32 CUDA-core form (not BR2): the lifting may sweep all three gradient components per direction
  constexpr bool kLift15 = SW == 0 && sizeof(real) == 4 && !BR2 && lift15_fills_better<n>();
  constexpr int nout = (sizeof(real) == 8 && SW == 0) ? 0 : NE * (kLift15 ? 15 : NV) * n3p;
  real* sOut = sbuf + NE * 15 * n3p;  // [NE][5 or 15][n3p]  sweep results (not for FP64)
  real* sQ = sOut + nout;                          // [NE][6][15][n2]  (v*3+d)
  real* sO = sQ + NE * 6 * 15 * n2;  // SPLIT, FP64: [NE][3][5][n3p] two-point sums per direction
  real* sJm = sO + ((SPLIT && sizeof(real) == 8) ? NE * 3 * NV * n3p : 0);  // BR2: [NE][6][15][n2] jumps
  real* sSJ = sJm + (BR2 ? NE * 6 * 15 * n2 : 0);                          // BR2: [NE][n3p] 1/J
  real* sOp = sSJ + (BR2 ? NE * n3p : 0);  // DhatT, lm, lp, lhm, lhp (+ DT)
  int* sES = reinterpret_cast<int*>(sOp + n2 + 4 * n + (SPLIT ? n2 : 0));
  int* sSlot = sES + NE * 6;   // [NE][6] side slot (slave * S + side) of each face
  int* sMpq = sSlot + NE * 6;  // [NE][6][n2] master-frame node of each face node
  static_assert(!SPLIT || (LGL && SW == 0), "the split form is built on Gauss-Lobatto nodes with CUDA-core sweeps");
  static_assert(!BR2 || (SW == 0 && !SPLIT), "BR2 face gradients are built for the standard form, CUDA-core sweeps");

  const int tid = threadIdx.x;
  const int el = tid / n3, node = tid - el * n3;
  const int e0 = blockIdx.x * NE;
  const int e = e0 + el;
  const bool valid = e < K;
  const int i = node % n, j = (node / n) % n, k = node / n2;
  const int pn = pidx<n>(i, j, k);

  load_ops<real, n>(sOp, ops, tid, T);
  if constexpr (SPLIT)
    for (int t = tid; t < n2; t += T) sOp[n2 + 4 * n + t] = ops.DT[t];
  for (int t = tid; t < NE * 6; t += T) {
    const int es = (e0 + t / 6 < K) ? elemSide[(size_t)e0 * 6 + t] : 0;
    sES[t] = es;
    sSlot[t] = es_slave(es) * S + es_side(es);
  }

  real Uo[NV], W[NV], jac[9], sj;
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Uo[v] = U[((size_t)e * NV + v) * n3 + node];
#pragma unroll
    for (int c = 0; c < 9; ++c) jac[c] = Ja[((size_t)e * 9 + c) * n3 + node];
    sj = sJ[(size_t)e * n3 + node];
  } else {
    Uo[0] = real(1); Uo[1] = Uo[2] = Uo[3] = real(0); Uo[4] = real(1);
#pragma unroll
    for (int c = 0; c < 9; ++c) jac[c] = real(0);
    sj = real(0);
  }
  cons_to_prim(Uo, W, ph);
  __syncthreads();
  BFrag<SW> bfr;
  if constexpr (SW != 0) bfr = make_bfrag<n, SW>(reinterpret_cast<const float*>(sOp), tid & 31);

  br1_surface_terms<real, n, NE, BR2>(Wf, fgeo, QB, sES, sQ, sMpq, sJm, e0, K, S, bigBase, tid, T);

  real G[15];
  real* myb = sbuf + el * 15 * n3p;
  const real* lhm = sOp + n2 + 2 * n;
  const real* lhp = sOp + n2 + 3 * n;
  const real* Qe = sQ + el * 6 * 15 * n2;
  const int pq0 = j + n * k, pq1 = i + n * k, pq2 = i + n * j;
  if constexpr (kLift15) {
#pragma unroll
    for (int l = 0; l < 3; ++l) {  // the previous sweep ended synced: sbuf is free
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const real a = jac[l * 3 + d];
#pragma unroll
        for (int v = 0; v < NV; ++v) myb[(d * NV + v) * n3p + pn] = a * W[v];
      }
      __syncthreads();
      if (l == 0) lift_sweep<real, n, LGL, 0>(sbuf, sOut, sQ, ops, tid);
      if (l == 1) lift_sweep<real, n, LGL, 1>(sbuf, sOut, sQ, ops, tid);
      if (l == 2) lift_sweep<real, n, LGL, 2>(sbuf, sOut, sQ, ops, tid);
    }
#pragma unroll
    for (int c = 0; c < 15; ++c) G[c] = sOut[(el * 15 + c) * n3p + pn] * sj;
  }
#pragma unroll
  for (int d = 0; d < (kLift15 ? 0 : 3); ++d) {
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const real a = jac[l * 3 + d];
#pragma unroll
      for (int v = 0; v < NV; ++v) myb[(l * NV + v) * n3p + pn] = a * W[v];
    }
    __syncthreads();
    real acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = real(0);
    constexpr bool kLines = (SW == 0 && sizeof(real) == 4);  // FP32: line sweeps with the face terms folded in
    if constexpr (SW == 0 && sizeof(real) == 8) {
      node_sweep3<real, n>(sOp, myb, i, j, k, acc);
    } else {
      if constexpr (SW == 0)
        line_sweep3<real, n, LGL>(sbuf, sOut, sQ, d, ops, tid);
      else
        tc_sweep3<n, NE, SW>(reinterpret_cast<const float*>(sbuf), reinterpret_cast<float*>(sOut), bfr, tid, T);
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = sOut[(el * NV + v) * n3p + pn];
    }
    if constexpr (!kLines && !LGL) {
      const real c0 = lhm[i], c1 = lhp[i], c2 = lhm[j], c3 = lhp[j], c4 = lhm[k], c5 = lhp[k];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int o = (v * 3 + d) * n2;
        real a = acc[v];
        a = dg_fma(c0, Qe[0 * 15 * n2 + o + pq0], a);
        a = dg_fma(c1, Qe[1 * 15 * n2 + o + pq0], a);
        a = dg_fma(c2, Qe[2 * 15 * n2 + o + pq1], a);
        a = dg_fma(c3, Qe[3 * 15 * n2 + o + pq1], a);
        a = dg_fma(c4, Qe[4 * 15 * n2 + o + pq2], a);
        acc[v] = dg_fma(c5, Qe[5 * 15 * n2 + o + pq2], a);
      }
    } else if constexpr (!kLines) {  // Gauss-Lobatto: only nodes on a face receive its term
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int o = (v * 3 + d) * n2;
        if (i == 0) acc[v] += lhm[0] * Qe[0 * 15 * n2 + o + pq0];
        if (i == n - 1) acc[v] += lhp[n - 1] * Qe[1 * 15 * n2 + o + pq0];
        if (j == 0) acc[v] += lhm[0] * Qe[2 * 15 * n2 + o + pq1];
        if (j == n - 1) acc[v] += lhp[n - 1] * Qe[3 * 15 * n2 + o + pq1];
        if (k == 0) acc[v] += lhm[0] * Qe[4 * 15 * n2 + o + pq2];
        if (k == n - 1) acc[v] += lhp[n - 1] * Qe[5 * 15 * n2 + o + pq2];
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) G[d * NV + v] = acc[v] * sj;
  }

  // a4: gradients to the faces (BR2: the broken gradient, G minus every face's
  // lifting r_f = (1/J) l_hat(+-1) (U* - U_e) n s_hat, plus eta r_f on face f below)
  __syncthreads();
  if constexpr (BR2) {
    const real* Je = sJm + el * 6 * 15 * n2;
    const real c0 = lhm[i], c1 = lhp[i], c2 = lhm[j], c3 = lhp[j], c4 = lhm[k], c5 = lhp[k];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int o = (v * 3 + d) * n2;
        real rr;
        if constexpr (LGL) {
          rr = real(0);
          if (i == 0) rr += lhm[0] * Je[0 * 15 * n2 + o + pq0];
          if (i == n - 1) rr += lhp[n - 1] * Je[1 * 15 * n2 + o + pq0];
          if (j == 0) rr += lhm[0] * Je[2 * 15 * n2 + o + pq1];
          if (j == n - 1) rr += lhp[n - 1] * Je[3 * 15 * n2 + o + pq1];
          if (k == 0) rr += lhm[0] * Je[4 * 15 * n2 + o + pq2];
          if (k == n - 1) rr += lhp[n - 1] * Je[5 * 15 * n2 + o + pq2];
        } else {
          rr = c0 * Je[0 * 15 * n2 + o + pq0] + c1 * Je[1 * 15 * n2 + o + pq0] + c2 * Je[2 * 15 * n2 + o + pq1] +
               c3 * Je[3 * 15 * n2 + o + pq1] + c4 * Je[4 * 15 * n2 + o + pq2] + c5 * Je[5 * 15 * n2 + o + pq2];
        }
        myb[(d * NV + v) * n3p + pn] = G[d * NV + v] - sj * rr;
      }
    sSJ[el * n3p + pn] = sj;
  } else {
#pragma unroll
    for (int c = 0; c < 15; ++c) myb[c * n3p + pn] = G[c];
  }
  if (Gvol != nullptr && valid) {
#pragma unroll
    for (int c = 0; c < 15; ++c) Gvol[((size_t)e * 15 + c) * n3 + node] = G[c];
  }
  __syncthreads();
  // BR2: eta times the trace of face s's own lifting at face node (p, q), component c = d*5 + v
  auto br2_own = [&](int el2, int s, int c, int p, int q) -> real {
    const int l = s >> 1;
    const real* sjl = sSJ + el2 * n3p;
    real kap = real(0);
    if (LGL) {
      kap = ((s & 1) ? lhp[n - 1] : lhm[0]) * sjl[pvol_index<n>(l, (s & 1) ? n - 1 : 0, p, q)];
    } else {
#pragma unroll
      for (int a = 0; a < n; ++a)
        kap += ((s & 1) ? ops.lp[a] * lhp[a] : ops.lm[a] * lhm[a]) * sjl[pvol_index<n>(l, a, p, q)];
    }
    const int v = c % NV, d = c / NV;
    return ph.eta_br2 * kap * sJm[((el2 * 6 + s) * 15 + v * 3 + d) * n2 + p + n * q];
  };
  if constexpr (sizeof(real) == 8) {
    // FP64: one thread per (face node, component), more warps on the FP64 pipe
    for (int it = tid; it < NE * 6 * 15 * n2; it += T) {
      const int el2 = it / (6 * 15 * n2);
      int r = it - el2 * 6 * 15 * n2;
      const int s = r / (15 * n2);
      r -= s * 15 * n2;
      const int c = r / n2, pq = r - c * n2;
      if (e0 + el2 >= K) continue;
      const int l = s >> 1, p = pq % n, q = pq / n;
      const real* b = sbuf + (el2 * 15 + c) * n3p;
      real val = real(0);
      if (LGL) {
        val = b[pvol_index<n>(l, (s & 1) ? n - 1 : 0, p, q)];
      } else {
#pragma unroll
        for (int a = 0; a < n; ++a) val += ((s & 1) ? ops.lp[a] : ops.lm[a]) * b[pvol_index<n>(l, a, p, q)];
      }
      if constexpr (BR2) val += br2_own(el2, s, c, p, q);
      const int es = sES[el2 * 6 + s];
      const int mpq = orient_pq(es_orient(es), n - 1, p, q);
      Gf[((size_t)(es_slave(es) * S + es_side(es)) * 15 + c) * n2 + mpq] = val;
    }
  } else if constexpr (NE == 1) {
    // one pass per line of direction l gives the values on both faces -l and +l; the face
    // node of the line has (p, q) = its free indices.  With one element per CTA (n^3
    // threads, n^2 lines) every task of a thread has the same line, tid mod n^2: its two
    // faces' slots and master-frame nodes are read once per direction, and the tasks differ
    // only in the component c = tid / n^2 + k n.
    constexpr int P = C::P;
    const int line = tid % n2, c0 = tid / n2;
    const int p = line % n, q = line / n;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const int stride = l == 0 ? 1 : (l == 1 ? P : P * n);
      const int base = l == 0 ? P * line : (l == 1 ? p + P * n * q : p + P * q);
      real* gm_out = Gf + (size_t)sSlot[2 * l] * 15 * n2 + sMpq[(2 * l) * n2 + line];
      real* gp_out = Gf + (size_t)sSlot[2 * l + 1] * 15 * n2 + sMpq[(2 * l + 1) * n2 + line];
      for (int c = c0; c < 15; c += T / n2) {
        const real* b = sbuf + c * n3p + base;
        real gm = real(0), gp = real(0);
        if (LGL) {
          gm = b[0];
          gp = b[(n - 1) * stride];
        } else {
#pragma unroll
          for (int a = 0; a < n; ++a) {
            const real x = b[a * stride];
            gm += ops.lm[a] * x;
            gp += ops.lp[a] * x;
          }
        }
        if constexpr (BR2) {
          gm += br2_own(0, 2 * l, c, p, q);
          gp += br2_own(0, 2 * l + 1, c, p, q);
        }
        gm_out[c * n2] = gm;
        gp_out[c * n2] = gp;
      }
    }
  } else {
    // one pass per line of direction l gives the values on both faces -l and +l;
    // the face node of the line has (p, q) = its free indices
    constexpr int P = C::P;
#pragma unroll
    for (int l = 0; l < 3; ++l)
    for (int it = tid; it < NE * 15 * n2; it += T) {
      const int el2 = NE == 1 ? 0 : it / (15 * n2);
      const int r = it - el2 * 15 * n2;
      const int c = r / n2, line = r - c * n2;
      if (e0 + el2 >= K) continue;
      const int p = line % n, q = line / n;
      const int stride = l == 0 ? 1 : (l == 1 ? P : P * n);
      const int base = l == 0 ? P * line : (l == 1 ? p + P * n * q : p + P * q);
      const real* b = sbuf + (el2 * 15 + c) * n3p + base;
      real gm = real(0), gp = real(0);
      if (LGL) {
        gm = b[0];
        gp = b[(n - 1) * stride];
      } else {
#pragma unroll
        for (int a = 0; a < n; ++a) {
          const real x = b[a * stride];
          gm += ops.lm[a] * x;
          gp += ops.lp[a] * x;
        }
      }
      if constexpr (BR2) {
        gm += br2_own(el2, 2 * l, c, p, q);
        gp += br2_own(el2, 2 * l + 1, c, p, q);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int f = el2 * 6 + 2 * l + h;
        Gf[((size_t)sSlot[f] * 15 + c) * n2 + sMpq[f * n2 + line]] = h ? gp : gm;
      }
    }
  }
  __syncthreads();

  if constexpr (SPLIT) {
    // Split form (Eq. semiDiscreteSplit).  Viscous part in weak form: D_hat sweeps of
    // -Fcal^{v,l} = -sum_d Ja^l_d F^v_d; on Gauss-Lobatto nodes D_hat = D - M^{-1} B
    // (summation by parts), so this is the strong form -D Fcal^{v,l} plus its face terms.
    real acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = real(0);
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const real nl[3] = {jac[l * 3], jac[l * 3 + 1], jac[l * 3 + 2]};
      real fv[NV];
      visc_normal(W, G, nl, ph, fv);  // linear in its direction argument
#pragma unroll
      for (int v = 0; v < NV; ++v) myb[(l * NV + v) * n3p + pn] = -fv[v];
    }
    __syncthreads();
    if constexpr (sizeof(real) == 8) {
      node_sweep3<real, n>(sOp, myb, i, j, k, acc);
    } else {
      line_sweep3<real, n, true>(sbuf, sOut, nullptr, 0, ops, tid);
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = sOut[(el * NV + v) * n3p + pn];
    }
    __syncthreads();
    // Advective part: 2 sum_a D_{i_l a} Fcal#^l(node, node with index_l = a) with
    // metric terms averaged over the pair.  Staged per node: rho, u, v, w, then
    // p, H = (rho E + p)/rho (kinetic-energy preserving, Pirozzoli) or
    // beta = rho/(2p), |u|^2 (entropy conservative, Chandrashekar), and Ja (9).
#pragma unroll
    for (int c = 0; c < 4; ++c) myb[c * n3p + pn] = W[c];
    const real H = SPLIT == 2 ? W[1] * W[1] + W[2] * W[2] + W[3] * W[3] : (Uo[4] + W[4]) / W[0];
    myb[4 * n3p + pn] = SPLIT == 2 ? real(0.5) * W[0] / W[4] : W[4];
    myb[5 * n3p + pn] = H;
#pragma unroll
    for (int c = 0; c < 9; ++c) myb[(6 + c) * n3p + pn] = jac[c];
    __syncthreads();
    if constexpr (sizeof(real) == 4) {
      // FP32: thread per node, all n pairs of each of its three lines (keeps every
      // thread busy; the FP32 pipes are not the limit)
      const real* sD = sOp + n2 + 4 * n;  // DT[a * n + i] = D[i][a]
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const int il = l == 0 ? i : (l == 1 ? j : k);
        const real J0 = jac[l * 3], J1 = jac[l * 3 + 1], J2 = jac[l * 3 + 2];
        real sm[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) sm[v] = real(0);
#pragma unroll
        for (int a = 0; a < n; ++a) {
          const int pa = l == 0 ? pidx<n>(a, j, k) : (l == 1 ? pidx<n>(i, a, k) : pidx<n>(i, j, a));
          const real* f = myb + pa;
          const real d = sD[a * n + il];
          if constexpr (SPLIT == 2) {
            const real ua[3] = {W[1], W[2], W[3]}, ub[3] = {f[n3p], f[2 * n3p], f[3 * n3p]};
            const real Jm[3] = {real(0.5) * (J0 + f[(6 + 3 * l) * n3p]), real(0.5) * (J1 + f[(7 + 3 * l) * n3p]),
                                real(0.5) * (J2 + f[(8 + 3 * l) * n3p])};
            real F[NV];
            ec_flux(W[0], ua, real(0.5) * W[0] / W[4], H, f[0], ub, f[4 * n3p], f[5 * n3p], Jm, ph, F);
#pragma unroll
            for (int v = 0; v < NV; ++v) sm[v] += real(2) * d * F[v];
          } else {
            const real rs = W[0] + f[0], us = W[1] + f[n3p], vs = W[2] + f[2 * n3p], ws = W[3] + f[3 * n3p];
            const real ps = W[4] + f[4 * n3p], Hs = H + f[5 * n3p];
            const real j0 = J0 + f[(6 + 3 * l) * n3p], j1 = J1 + f[(7 + 3 * l) * n3p],
                       j2 = J2 + f[(8 + 3 * l) * n3p];
            const real m = real(0.125) * rs * (us * j0 + vs * j1 + ws * j2);
            const real dm = d * m, dp = real(0.5) * d * ps;
            sm[0] += real(2) * dm;
            sm[1] += dm * us + dp * j0;
            sm[2] += dm * vs + dp * j1;
            sm[3] += dm * ws + dp * j2;
            sm[4] += dm * Hs;
          }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += sm[v];
      }
    } else {
      // One thread per (direction l, line): F# is symmetric, so every pair (i, a),
      // i < a, of the line is evaluated once and gives D_ia F# to node i and
      // D_ai F# to node a.  Diagonal terms: D_ii = 0 at the interior Gauss-Lobatto
      // nodes (Q + Q^T = B), so only the two end nodes carry 2 D_ii F(U_i).
      // The line's sums go to its own slots of sO[l] (no other thread writes them).
      constexpr int P = C::P;
      const real* sD = sOp + n2 + 4 * n;  // DT[a * n + i] = D[i][a]
      for (int task = tid; task < NE * 3 * n2; task += T) {
        const int el2 = task / (3 * n2);
        const int r = task - el2 * 3 * n2;
        const int l = r / n2, line = r - l * n2;
        const int a0 = line % n, a1 = line / n;
        const int stride = l == 0 ? 1 : (l == 1 ? P : P * n);
        const int base = l == 0 ? P * line : (l == 1 ? a0 + P * n * a1 : a0 + P * a1);
        const real* f = sbuf + el2 * 15 * n3p + base;
        real* o = sO + ((el2 * 3 + l) * NV) * n3p + base;
        const int jo = (6 + 3 * l) * n3p;
#pragma unroll
        for (int ii = 0; ii < n; ++ii)
#pragma unroll
          for (int c = 0; c < NV; ++c) o[c * n3p + ii * stride] = real(0);
        // (the entropy-conservative pair flux is long: keep its loops rolled)
#pragma unroll(SPLIT == 2 ? 1 : n)
        for (int ii = 0; ii < n; ++ii) {
          const real* fi = f + ii * stride;
          const real ri = fi[0], ui = fi[n3p], vi = fi[2 * n3p], wi = fi[3 * n3p], pi = fi[4 * n3p];
          const real Hi = fi[5 * n3p], ji0 = fi[jo], ji1 = fi[jo + n3p], ji2 = fi[jo + 2 * n3p];
          real ai[NV];
#pragma unroll
          for (int c = 0; c < NV; ++c) ai[c] = real(0);
          if (ii == 0 || ii == n - 1) {  // 2 D_ii F#(i, i) = 2 D_ii Fcal^{c,l}(U_i)
            const real dd = real(2) * sD[ii * n + ii];
            if constexpr (SPLIT == 2) {
              const real u3[3] = {ui, vi, wi}, J3[3] = {ji0, ji1, ji2};
              real F[NV];
              ec_flux(ri, u3, pi, Hi, ri, u3, pi, Hi, J3, ph, F);
#pragma unroll
              for (int c = 0; c < NV; ++c) ai[c] = dd * F[c];
            } else {
              const real uc = ui * ji0 + vi * ji1 + wi * ji2;
              const real m = dd * ri * uc;
              ai[0] = m;
              ai[1] = m * ui + dd * pi * ji0;
              ai[2] = m * vi + dd * pi * ji1;
              ai[3] = m * wi + dd * pi * ji2;
              ai[4] = m * Hi;
            }
          }
#pragma unroll(SPLIT == 2 ? 1 : n)
          for (int aa = ii + 1; aa < n; ++aa) {
            const real* fa = f + aa * stride;
            real F0, F1, F2, F3, F4;  // 2 F#(i, a)
            if constexpr (SPLIT == 2) {
              const real u3[3] = {ui, vi, wi}, ua3[3] = {fa[n3p], fa[2 * n3p], fa[3 * n3p]};
              const real Jm[3] = {real(0.5) * (ji0 + fa[jo]), real(0.5) * (ji1 + fa[jo + n3p]),
                                  real(0.5) * (ji2 + fa[jo + 2 * n3p])};
              real F[NV];
              ec_flux(ri, u3, pi, Hi, fa[0], ua3, fa[4 * n3p], fa[5 * n3p], Jm, ph, F);
              F0 = real(2) * F[0]; F1 = real(2) * F[1]; F2 = real(2) * F[2]; F3 = real(2) * F[3]; F4 = real(2) * F[4];
            } else {
              // pair sums (twice the arithmetic means)
              const real rs = ri + fa[0], us = ui + fa[n3p], vs = vi + fa[2 * n3p], ws = wi + fa[3 * n3p];
              const real ps = pi + fa[4 * n3p], Hs = Hi + fa[5 * n3p];
              const real j0 = ji0 + fa[jo], j1 = ji1 + fa[jo + n3p], j2 = ji2 + fa[jo + 2 * n3p];
              const real m = real(0.125) * rs * (us * j0 + vs * j1 + ws * j2);  // {rho} {u . Ja^l}
              const real hp = real(0.5) * ps;
              // 2 F#: mass 2 m; momentum m u_s + (p_s / 2) Ja_s; energy m H_s
              F0 = real(2) * m; F1 = m * us + hp * j0; F2 = m * vs + hp * j1; F3 = m * ws + hp * j2;
              F4 = m * Hs;
            }
            const real dia = sD[aa * n + ii], dai = sD[ii * n + aa];
            ai[0] += dia * F0; ai[1] += dia * F1; ai[2] += dia * F2; ai[3] += dia * F3; ai[4] += dia * F4;
            real* oa = o + aa * stride;
            oa[0] += dai * F0;
            oa[n3p] += dai * F1;
            oa[2 * n3p] += dai * F2;
            oa[3 * n3p] += dai * F3;
            oa[4 * n3p] += dai * F4;
          }
          real* oi = o + ii * stride;
#pragma unroll
          for (int c = 0; c < NV; ++c) oi[c * n3p] += ai[c];
        }
      }
      __syncthreads();
#pragma unroll
      for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += sO[((el * 3 + l) * NV + v) * n3p + pn];
    }
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const int il = l == 0 ? i : (l == 1 ? j : k);
      // face terms of the strong form: -(+-1) l_hat(+-1) Fcal^{c,l} at the line's end nodes
      if (il == 0 || il == n - 1) {
        const real J0 = jac[l * 3], J1 = jac[l * 3 + 1], J2 = jac[l * 3 + 2];
        const real c = il == 0 ? sOp[n2 + 2 * n] : -sOp[n2 + 3 * n + n - 1];
        const real uc = W[1] * J0 + W[2] * J1 + W[3] * J2;
        const real mf = Uo[1] * J0 + Uo[2] * J1 + Uo[3] * J2;
        acc[0] += c * mf;
        acc[1] += c * (Uo[1] * uc + W[4] * J0);
        acc[2] += c * (Uo[2] * uc + W[4] * J1);
        acc[3] += c * (Uo[3] * uc + W[4] * J2);
        acc[4] += c * (uc * (Uo[4] + W[4]));
      }
    }
    if (valid) {
#pragma unroll
      for (int v = 0; v < NV; ++v) Utv[((size_t)e * NV + v) * n3 + node] = acc[v];
    }
    return;
  }
  // a6: contravariant fluxes Fcal^l = sum_d Ja^l_d (F^c_d - F^v_d): in registers for
  // FP32, accumulated in shared memory for FP64 (register budget)
  if constexpr (sizeof(real) == 4) {
    real F[3][NV];
#pragma unroll
    for (int d = 0; d < 3; ++d) flux_total(Uo, W, G, d, ph, F[d]);
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
      for (int v = 0; v < NV; ++v)
        myb[(l * NV + v) * n3p + pn] = jac[l * 3 + 0] * F[0][v] + jac[l * 3 + 1] * F[1][v] + jac[l * 3 + 2] * F[2][v];
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      real F[NV];
      flux_total(Uo, W, G, d, ph, F);
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const real a = jac[l * 3 + d];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          real* dst = &myb[(l * NV + v) * n3p + pn];
          *dst = (d == 0 ? real(0) : *dst) + a * F[v];
        }
      }
    }
  }
  __syncthreads();
  // a7: volume integral
  real acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = real(0);
  if constexpr (SW == 0 && sizeof(real) == 8) {
    node_sweep3<real, n>(sOp, myb, i, j, k, acc);
  } else {
    if constexpr (SW == 0)
      line_sweep3<real, n, LGL>(sbuf, sOut, nullptr, 0, ops, tid);
    else
      tc_sweep3<n, NE, SW>(reinterpret_cast<const float*>(sbuf), reinterpret_cast<float*>(sOut), bfr, tid, T);
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = sOut[(el * NV + v) * n3p + pn];
  }
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Utv[((size_t)e * NV + v) * n3 + node] = acc[v];
  }
}

#define FLEXI_LIFT_VOL_PARAMS                                                                              \
  const real *__restrict__ U, const real *__restrict__ Ja, const real *__restrict__ sJ,                   \
      const real *__restrict__ Wf, const real *__restrict__ fgeo, const int *__restrict__ elemSide,        \
      real *__restrict__ Gf, real *__restrict__ Utv, real *__restrict__ Gvol, int K, int S, int bigBase, \
      const real *__restrict__ QB, Ops<real> ops, Phys<real> ph
#define FLEXI_LIFT_VOL_ARGS U, Ja, sJ, Wf, fgeo, elemSide, Gf, Utv, Gvol, K, S, bigBase, QB, ops, ph

// the kernel at the compiler's default register allocation
template <typename real, int n, int SW, bool LGL, int SPLIT = 0, bool BR2 = false>
__global__ void __launch_bounds__(Cfg<n>::T) k_lift_vol(FLEXI_LIFT_VOL_PARAMS) {
  lift_vol_body<real, n, SW, LGL, SPLIT, BR2>(FLEXI_LIFT_VOL_ARGS);
}

// the same kernel with lift_vol_min_blocks() CTAs per SM (register cap)
template <typename real, int n, int SW, bool LGL, int SPLIT = 0, bool BR2 = false>
__global__ void __launch_bounds__(Cfg<n>::T, lift_vol_min_blocks<real, n, SW, SPLIT, BR2>()) k_lift_vol_mb(FLEXI_LIFT_VOL_PARAMS) {
  lift_vol_body<real, n, SW, LGL, SPLIT, BR2>(FLEXI_LIFT_VOL_ARGS);
}
#undef FLEXI_LIFT_VOL_PARAMS
#undef FLEXI_LIFT_VOL_ARGS

// a2-a4, a6, a7 for small FP64 meshes (fewer elements than SMs, n <= 4; standard form,
// BR1): one element per CTA, spread over three thread groups of n^3 threads.  The lifting
// computes one gradient component per group, the physical fluxes one direction per group,
// the contravariant fluxes and the D_hat volume sweep one reference direction per group
// (their partial sums added at the end), with the fields exchanged through shared memory.
// The arithmetic is that of k_lift_vol; the three groups give the SMs that such meshes
// occupy three times the warps to hide the FP64 pipe's latency.
template <int n, bool LGL>
__global__ void __launch_bounds__(3 * n * n * n) k_lift_vol_g3(
    const double* __restrict__ U, const double* __restrict__ Ja, const double* __restrict__ sJ,
    const double* __restrict__ Wf, const double* __restrict__ fgeo, const int* __restrict__ elemSide,
    double* __restrict__ Gf, double* __restrict__ Utv, double* __restrict__ Gvol, int K, int S, int bigBase,
    const double* __restrict__ QB, Ops<double> ops, Phys<double> ph) {
  using real = double;
  constexpr int n2 = n * n, n3 = n2 * n, T = 3 * n3, n3p = Cfg<n>::n3p;
  __shared__ real sbuf[3 * 15 * n3p];  // three regions of 15 padded fields
  __shared__ real sQ[6 * 15 * n2];     // BR1 surface terms [6][15][n2]
  __shared__ real sOp[n2 + 4 * n];
  __shared__ int sES[6], sSlot[6], sMpq[6 * n2];
  const int tid = threadIdx.x;
  const int g = tid / n3, node = tid - g * n3;
  const int e = blockIdx.x;  // grid = K
  const int i = node % n, j = (node / n) % n, k = node / n2;
  const int pn = pidx<n>(i, j, k);
  load_ops<real, n>(sOp, ops, tid, T);
  if (tid < 6) {
    const int es = elemSide[(size_t)e * 6 + tid];
    sES[tid] = es;
    sSlot[tid] = es_slave(es) * S + es_side(es);
  }
  real Uo[NV], W[NV], jac[9];
#pragma unroll
  for (int v = 0; v < NV; ++v) Uo[v] = U[((size_t)e * NV + v) * n3 + node];
#pragma unroll
  for (int c = 0; c < 9; ++c) jac[c] = Ja[((size_t)e * 9 + c) * n3 + node];
  const real sj = sJ[(size_t)e * n3 + node];
  cons_to_prim(Uo, W, ph);
  __syncthreads();
  br1_surface_terms<real, n, 1, false>(Wf, fgeo, QB, sES, sQ, sMpq, nullptr, e, K, S, bigBase, tid, T);

  // the group's column (Ja^l_g, l = 0..2) and row (Ja^g_d, d = 0..2) of the metric terms,
  // selected by value (a runtime index would put jac in local memory)
  auto pick = [g](real a, real b, real c) { return g == 0 ? a : (g == 1 ? b : c); };
  const real col[3] = {pick(jac[0], jac[1], jac[2]), pick(jac[3], jac[4], jac[5]), pick(jac[6], jac[7], jac[8])};
  const real row[3] = {pick(jac[0], jac[3], jac[6]), pick(jac[1], jac[4], jac[7]), pick(jac[2], jac[5], jac[8])};
  // lifting, gradient component d = g: Ja^l_g W_v staged as field l*5 + v of region g
  real* myb = sbuf + g * 15 * n3p;
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int v = 0; v < NV; ++v) myb[(l * NV + v) * n3p + pn] = col[l] * W[v];
  __syncthreads();
  real acc[NV] = {real(0), real(0), real(0), real(0), real(0)};
  node_sweep3<real, n>(sOp, myb, i, j, k, acc);
  const real* lhm = sOp + n2 + 2 * n;
  const real* lhp = sOp + n2 + 3 * n;
  const int pq0 = j + n * k, pq1 = i + n * k, pq2 = i + n * j;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int o = (v * 3 + g) * n2;
    real a = acc[v];
    if constexpr (LGL) {  // only nodes on a face receive its term
      if (i == 0) a = dg_fma(lhm[0], sQ[0 * 15 * n2 + o + pq0], a);
      if (i == n - 1) a = dg_fma(lhp[n - 1], sQ[1 * 15 * n2 + o + pq0], a);
      if (j == 0) a = dg_fma(lhm[0], sQ[2 * 15 * n2 + o + pq1], a);
      if (j == n - 1) a = dg_fma(lhp[n - 1], sQ[3 * 15 * n2 + o + pq1], a);
      if (k == 0) a = dg_fma(lhm[0], sQ[4 * 15 * n2 + o + pq2], a);
      if (k == n - 1) a = dg_fma(lhp[n - 1], sQ[5 * 15 * n2 + o + pq2], a);
    } else {
      a = dg_fma(lhm[i], sQ[0 * 15 * n2 + o + pq0], a);
      a = dg_fma(lhp[i], sQ[1 * 15 * n2 + o + pq0], a);
      a = dg_fma(lhm[j], sQ[2 * 15 * n2 + o + pq1], a);
      a = dg_fma(lhp[j], sQ[3 * 15 * n2 + o + pq1], a);
      a = dg_fma(lhm[k], sQ[4 * 15 * n2 + o + pq2], a);
      a = dg_fma(lhp[k], sQ[5 * 15 * n2 + o + pq2], a);
    }
    acc[v] = a;
  }
  __syncthreads();  // every region read: region 0 takes the gradients
  real* sG = sbuf;  // [15][n3p], component d*5 + v
#pragma unroll
  for (int v = 0; v < NV; ++v) sG[(g * NV + v) * n3p + pn] = acc[v] * sj;
  __syncthreads();
  real G[15];
#pragma unroll
  for (int c = 0; c < 15; ++c) G[c] = sG[c * n3p + pn];
  if (Gvol != nullptr && g == 0) {
#pragma unroll
    for (int c = 0; c < 15; ++c) Gvol[((size_t)e * 15 + c) * n3 + node] = G[c];
  }
  // a4: gradients to the faces, one thread per (face node, component)
  for (int it = tid; it < 6 * 15 * n2; it += T) {
    const int s = it / (15 * n2);
    const int r = it - s * 15 * n2;
    const int c = r / n2, pq = r - c * n2;
    const int l = s >> 1, p = pq % n, q = pq / n;
    const real* b = sG + c * n3p;
    real val = real(0);
    if (LGL) {
      val = b[pvol_index<n>(l, (s & 1) ? n - 1 : 0, p, q)];
    } else {
#pragma unroll
      for (int a = 0; a < n; ++a) val = dg_fma((s & 1) ? ops.lp[a] : ops.lm[a], b[pvol_index<n>(l, a, p, q)], val);
    }
    Gf[((size_t)sSlot[s] * 15 + c) * n2 + sMpq[s * n2 + pq]] = val;
  }
  // a6: physical flux of direction d = g into region 1, then the contravariant flux of
  // reference direction l = g (sum_d Ja^g_d F_d) into region 2
  real F[NV];
  if (g == 0)  // compile-time directions (flux_total indexes its arrays with d)
    flux_total(Uo, W, G, 0, ph, F);
  else if (g == 1)
    flux_total(Uo, W, G, 1, ph, F);
  else
    flux_total(Uo, W, G, 2, ph, F);
  real* sF = sbuf + 15 * n3p;
  real* sC = sbuf + 2 * 15 * n3p;
#pragma unroll
  for (int v = 0; v < NV; ++v) sF[(g * NV + v) * n3p + pn] = F[v];
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; ++v)
    sC[(g * NV + v) * n3p + pn] = dg_fma(row[2], sF[(2 * NV + v) * n3p + pn],
                                         dg_fma(row[1], sF[(NV + v) * n3p + pn], row[0] * sF[v * n3p + pn]));
  __syncthreads();
  // a7: D_hat sweep along direction l = g; the partial sums go to region 1 (no longer read)
  const int il = g == 0 ? i : (g == 1 ? j : k);
  real sum[NV] = {real(0), real(0), real(0), real(0), real(0)};
#pragma unroll
  for (int a = 0; a < n; ++a) {
    const real dh = sOp[a * n + il];
    const int ia = g == 0 ? pidx<n>(a, j, k) : (g == 1 ? pidx<n>(i, a, k) : pidx<n>(i, j, a));
#pragma unroll
    for (int v = 0; v < NV; ++v) sum[v] = dg_fma(dh, sC[(g * NV + v) * n3p + ia], sum[v]);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) sF[(g * NV + v) * n3p + pn] = sum[v];
  __syncthreads();
  if (g == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
      Utv[((size_t)e * NV + v) * n3 + node] = sF[v * n3p + pn] + sF[(NV + v) * n3p + pn] + sF[(2 * NV + v) * n3p + pn];
  }
}

// Thread-block cluster primitives (sm_90 and later): the CTA's rank in its cluster; a
// barrier over every thread of the cluster whose arrive releases and whose wait acquires
// this CTA's prior shared-memory accesses (split in two where the wait can come later);
// and the generic address of the same shared-memory location in another CTA of the
// cluster (distributed shared memory), readable with ordinary loads.
__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_barrier() {
  cluster_arrive();
  cluster_wait();
}
template <typename T>
__device__ __forceinline__ const T* cluster_peer(const T* p, unsigned rank) {
  unsigned long long a;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(a) : "l"(reinterpret_cast<unsigned long long>(p)), "r"(rank));
  return reinterpret_cast<const T*>(a);
}

// a2-a4, a6, a7 for FP64 meshes with at most half as many elements as SMs (n = 4; standard
// form, BR1).  On such meshes each thread's chain of dependent instructions sets the time,
// not the throughput of any unit (on GB300 an FP64 warp instruction holds its SM
// sub-partition for 64 clocks however few of its lanes are active), so an element's work is
// cut finely.  One cluster of two CTAs per element: CTA r holds the nodes with k in
// [r n/2, (r + 1) n/2), and one warp per pair (g, v) of a direction (or gradient component) g
// and a variable v runs over the CTA's n^3/2 = 32 nodes, 15 warps in all.  Warp (g, v) forms
// the lifting fields Ja^l_g W_v, sweeps them into dW_v/dx_g, evaluates the flux component
// (F_g)_v, then the contravariant flux component of reference direction g and its D_hat
// sweep.  Lines along i and j lie inside a half.  What a half needs of the other one is
// copied from the other CTA's shared memory after a cluster barrier: the lifting fields of
// the third reference direction, the contravariant fluxes of that direction and, on Gauss
// nodes, the gradients that the k faces interpolate.  Each copy fills positions that the
// copying CTA never writes itself, while the other CTA reads only its own positions, and
// every buffer that the other CTA reads stays unchanged until the next cluster barrier.
// The face gradients of a face node come from the half that holds its volume nodes (faces
// +-i and +-j: the half of q, face -k: CTA 0, face +k: CTA 1).  The expressions per node
// are those of k_lift_vol_g3 (cons_to_prim, node_sweep3, flux_total, the same face terms,
// contravariant products and sums in the same order).
template <int n, bool LGL>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(15 * n * n * n / 2) k_lift_vol_c2(
    const double* __restrict__ U, const double* __restrict__ Ja, const double* __restrict__ sJ,
    const double* __restrict__ Wf, const double* __restrict__ fgeo, const int* __restrict__ elemSide,
    double* __restrict__ Gf, double* __restrict__ Utv, double* __restrict__ Gvol, int K, int S, int bigBase,
    const double* __restrict__ QB, Ops<double> ops, Phys<double> ph) {
  static_assert(n * n * n / 2 == 32, "one warp per (g, v) over the 32 nodes of a half element");
  using real = double;
  constexpr int n2 = n * n, n3 = n2 * n, h3 = n3 / 2, hk = n / 2, T = 15 * h3, n3p = Cfg<n>::n3p;
  static_assert(15 * n3p <= 6 * 15 * n2, "the gradients fit the surface-term buffer");
  __shared__ real sbuf[3 * 15 * n3p];  // lifting fields; then fluxes and partial sums (region 1), contravariant fluxes (region 2)
  __shared__ real sQ[6 * 15 * n2];     // BR1 surface terms [6][15][n2]; then the gradients [15][n3p]
  __shared__ real sW[NV * n3p];        // primitive variables of this half's nodes
  __shared__ real sOp[n2 + 4 * n];
  __shared__ int sES[6], sSlot[6], sMpq[6 * n2];
  const int tid = threadIdx.x;
  const unsigned r = cluster_ctarank();
  const int kb = (int)(r ^ 1u) * hk;  // first k of the other half
  const int wp = tid >> 5, ln = tid & 31;
  // (g, v) of warp wp from a table that balances the FP64 warp instructions of the four SM
  // sub-partitions (warp wp runs on sub-partition wp mod 4): one of the three energy-flux
  // warps (v = 4, the longest) on each of sub-partitions 0-2, the primitive variables and
  // no surface terms on sub-partition 3, which has three warps
  //   wp: 0  1  2  3  4  5  6  7  8  9 10 11 12 13 14
  //   g:  0  1  2  1  1  2  0  2  2  0  1  0  0  1  2
  //   v:  4  4  4  1  0  0  0  2  1  1  2  3  2  3  3
  const int g = (int)((0x24128964ull >> (2 * wp)) & 3ull);
  const int v = (int)((0xda689400324ull >> (3 * wp)) & 7ull);  // warp-uniform
  const int e = blockIdx.x >> 1;           // grid = 2 K, clusters of two consecutive CTAs
  const int i = ln % n, j = (ln / n) % n, k = (int)r * hk + ln / n2;
  const int node = i + n * (j + n * k);
  const int pn = pidx<n>(i, j, k);
  load_ops<real, n>(sOp, ops, tid, T);
  if (tid < 6) {
    const int es = elemSide[(size_t)e * 6 + tid];
    sES[tid] = es;
    sSlot[tid] = es_slave(es) * S + es_side(es);
  }
  real Uo[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) Uo[c] = U[((size_t)e * NV + c) * n3 + node];
  real col[3], row[3];  // Ja^l_g (l = 0..2) and Ja^g_d (d = 0..2)
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    col[l] = Ja[((size_t)e * 9 + l * 3 + g) * n3 + node];
    row[l] = Ja[((size_t)e * 9 + g * 3 + l) * n3 + node];
  }
  const real sj = sJ[(size_t)e * n3 + node];
  if ((wp & 3) == 3) {  // the primitive variables as cons_to_prim forms them: warps 3, 7, 11
    const real ir = real(1) / Uo[0];
    const real u = Uo[1] * ir, vv = Uo[2] * ir, w = Uo[3] * ir;
    if (wp == 3) {
      sW[1 * n3p + pn] = u;
      sW[2 * n3p + pn] = vv;
    } else if (wp == 7) {
      sW[0 * n3p + pn] = Uo[0];
      sW[3 * n3p + pn] = w;
    } else {
      sW[4 * n3p + pn] = ph.gm1 * (Uo[4] - real(0.5) * (Uo[1] * u + Uo[2] * vv + Uo[3] * w));
    }
  }
  __syncthreads();
  // BR1 surface terms of the face nodes that this half reads, one thread per (variable,
  // face node) with the expressions of br1_surface_terms: faces 0-3 with q in
  // [r n/2, (r + 1) n/2), then face 4 + r (Gauss-Lobatto: only the nodes on a face read it)
  // or both k faces (Gauss: every node reads both)
  constexpr int nIJq = 4 * (n2 / 2), nKf = LGL ? n2 : 2 * n2, nQ = nIJq + nKf;
  // on the twelve warps of sub-partitions 0-2 (dense index wq = wp - wp / 4)
  const int wq = wp - (wp >> 2);
  for (int it = (wp & 3) == 3 ? NV * nQ : wq * 32 + ln; it < NV * nQ; it += 12 * 32) {
    const int c = it / nQ, f = it - c * nQ;
    int s, pq;
    if (f < nIJq) {
      s = f / (n2 / 2);
      const int m = f - s * (n2 / 2);
      pq = m % n + n * ((int)r * hk + m / n);
    } else {
      const int fk = f - nIJq;
      s = LGL ? 4 + (int)r : 4 + fk / n2;
      pq = fk % n2;
    }
    const int es = sES[s];
    const int side = es_side(es);
    const int mpq = orient_pq(es_orient(es), n - 1, pq % n, pq / n);
    if (c == 0) sMpq[s * n2 + pq] = mpq;
    const real* gq = fgeo + ((size_t)side * 4) * n2 + mpq;
    const real sc = es_slave(es) ? -gq[3 * n2] : gq[3 * n2];
    const real nd[3] = {gq[0] * sc, gq[n2] * sc, gq[2 * n2] * sc};
    real* Q = sQ + (s * 15 + c * 3) * n2 + pq;
    if (side >= bigBase) {
      const real* qb = QB + ((size_t)(side - bigBase) * 15 + c * 3) * n2 + mpq;
#pragma unroll
      for (int d = 0; d < 3; ++d) Q[d * n2] = qb[d * n2];
    } else {
      const real ws = real(0.5) * (Wf[((size_t)side * NV + c) * n2 + mpq] + Wf[((size_t)(S + side) * NV + c) * n2 + mpq]);
#pragma unroll
      for (int d = 0; d < 3; ++d) Q[d * n2] = ws * nd[d];
    }
  }
  real* myb = sbuf + g * 15 * n3p;
  {
    const real Wv = sW[v * n3p + pn];
#pragma unroll
    for (int l = 0; l < 3; ++l) myb[(l * NV + v) * n3p + pn] = col[l] * Wv;
  }
  cluster_barrier();  // both halves' lifting fields staged
  {
    const real* peer = cluster_peer(sbuf, r ^ 1u);
    for (int it = tid; it < 3 * NV * h3; it += T) {
      const int gg = it / (NV * h3), rem = it - gg * NV * h3;
      const int c = rem / h3, m = rem - c * h3;
      const int o = (gg * 15 + 2 * NV + c) * n3p + pidx<n>(m % n, (m / n) % n, kb + m / n2);
      sbuf[o] = peer[o];
    }
  }
  __syncthreads();
  // dW_v/dx_g: the three reference-direction sweeps of node_sweep3, then the face terms
  real acc = real(0);
#pragma unroll
  for (int a = 0; a < n; ++a) {
    const real d0 = sOp[a * n + i], d1 = sOp[a * n + j], d2 = sOp[a * n + k];
    acc += d0 * myb[v * n3p + pidx<n>(a, j, k)];
    acc += d1 * myb[(NV + v) * n3p + pidx<n>(i, a, k)];
    acc += d2 * myb[(2 * NV + v) * n3p + pidx<n>(i, j, a)];
  }
  {
    const real* lhm = sOp + n2 + 2 * n;
    const real* lhp = sOp + n2 + 3 * n;
    const int pq0 = j + n * k, pq1 = i + n * k, pq2 = i + n * j;
    const int o = (v * 3 + g) * n2;
    if constexpr (LGL) {
      if (i == 0) acc = dg_fma(lhm[0], sQ[0 * 15 * n2 + o + pq0], acc);
      if (i == n - 1) acc = dg_fma(lhp[n - 1], sQ[1 * 15 * n2 + o + pq0], acc);
      if (j == 0) acc = dg_fma(lhm[0], sQ[2 * 15 * n2 + o + pq1], acc);
      if (j == n - 1) acc = dg_fma(lhp[n - 1], sQ[3 * 15 * n2 + o + pq1], acc);
      if (k == 0) acc = dg_fma(lhm[0], sQ[4 * 15 * n2 + o + pq2], acc);
      if (k == n - 1) acc = dg_fma(lhp[n - 1], sQ[5 * 15 * n2 + o + pq2], acc);
    } else {
      acc = dg_fma(lhm[i], sQ[0 * 15 * n2 + o + pq0], acc);
      acc = dg_fma(lhp[i], sQ[1 * 15 * n2 + o + pq0], acc);
      acc = dg_fma(lhm[j], sQ[2 * 15 * n2 + o + pq1], acc);
      acc = dg_fma(lhp[j], sQ[3 * 15 * n2 + o + pq1], acc);
      acc = dg_fma(lhm[k], sQ[4 * 15 * n2 + o + pq2], acc);
      acc = dg_fma(lhp[k], sQ[5 * 15 * n2 + o + pq2], acc);
    }
  }
  __syncthreads();  // surface terms read: the buffer takes the gradients
  real* sG = sQ;    // [15][n3p], component d*5 + v
  const real grad = acc * sj;
  sG[(g * NV + v) * n3p + pn] = grad;
  if (Gvol != nullptr) Gvol[((size_t)e * 15 + g * NV + v) * n3 + node] = grad;
  cluster_barrier();  // both halves' gradients; the other CTA has copied its lifting fields
  if constexpr (!LGL) {  // Gauss: the k faces interpolate whole lines along k
    const real* peer = cluster_peer(sG, r ^ 1u);
    for (int it = tid; it < 15 * h3; it += T) {
      const int c = it / h3, m = it - c * h3;
      const int o = c * n3p + pidx<n>(m % n, (m / n) % n, kb + m / n2);
      sG[o] = peer[o];
    }
    __syncthreads();
  }
  // a4: this half's face nodes, one thread per (face node, component): faces 0-3 with
  // q in [r n/2, (r + 1) n/2), then face 4 + r whole
  constexpr int nIJ = 4 * 15 * n2 / 2;
  for (int it = tid; it < nIJ + 15 * n2; it += T) {
    int s, c, p, q;
    if (it < nIJ) {
      s = it / (15 * n2 / 2);
      const int rem = it - s * (15 * n2 / 2);
      c = rem / (n2 / 2);
      const int m = rem - c * (n2 / 2);
      p = m % n;
      q = (int)r * hk + m / n;
    } else {
      s = 4 + (int)r;
      const int rem = it - nIJ;
      c = rem / n2;
      const int pq = rem - c * n2;
      p = pq % n;
      q = pq / n;
    }
    const int l = s >> 1, pq = p + n * q;
    const real* b = sG + c * n3p;
    real val = real(0);
    if (LGL) {
      val = b[pvol_index<n>(l, (s & 1) ? n - 1 : 0, p, q)];
    } else {
#pragma unroll
      for (int a = 0; a < n; ++a) val = dg_fma((s & 1) ? ops.lp[a] : ops.lm[a], b[pvol_index<n>(l, a, p, q)], val);
    }
    Gf[((size_t)sSlot[s] * 15 + c) * n2 + sMpq[s * n2 + pq]] = val;
  }
  // a6: flux component (F_d)_v, d = g, with the expressions of flux_total
  real F;
  {
    real Wn[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) Wn[c] = sW[c * n3p + pn];
    const int d = g;
    const real* Gn = sG + pn;
    const real ud = d == 0 ? Wn[1] : (d == 1 ? Wn[2] : Wn[3]);
    const real p = Wn[4];
    if (v == 0) {
      F = d == 0 ? Uo[1] : (d == 1 ? Uo[2] : Uo[3]);
    } else {
      const real div = Gn[(0 * 5 + 1) * n3p] + Gn[(1 * 5 + 2) * n3p] + Gn[(2 * 5 + 3) * n3p];
      if (v < 4) {
        const int c = v - 1;
        real tau = ph.mu * (Gn[(d * 5 + 1 + c) * n3p] + Gn[(c * 5 + 1 + d) * n3p]);
        if (c == d) tau -= real(2.0 / 3.0) * ph.mu * div;
        const real Uc = v == 1 ? Uo[1] : (v == 2 ? Uo[2] : Uo[3]);
        F = Uc * ud - tau;
        if (c == d) F += p;
      } else {
        real tau[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          tau[c] = ph.mu * (Gn[(d * 5 + 1 + c) * n3p] + Gn[(c * 5 + 1 + d) * n3p]);
          if (c == d) tau[c] -= real(2.0 / 3.0) * ph.mu * div;
        }
        const real ir = real(1) / Wn[0];
        const real dT = (Gn[(d * 5 + 4) * n3p] - p * ir * Gn[(d * 5 + 0) * n3p]) * ir;
        const real fv4 = tau[0] * Wn[1] + tau[1] * Wn[2] + tau[2] * Wn[3] + ph.lam_th * dT;
        F = ud * (Uo[4] + p) - fv4;
      }
    }
  }
  real* sF = sbuf + 15 * n3p;
  real* sC = sbuf + 2 * 15 * n3p;
  sF[(g * NV + v) * n3p + pn] = F;
  __syncthreads();
  // contravariant flux of reference direction g, variable v
  sC[(g * NV + v) * n3p + pn] = dg_fma(row[2], sF[(2 * NV + v) * n3p + pn],
                                       dg_fma(row[1], sF[(NV + v) * n3p + pn], row[0] * sF[v * n3p + pn]));
  cluster_barrier();  // both halves' contravariant fluxes; the other CTA is done with the gradients
  {
    const real* peer = cluster_peer(sC, r ^ 1u);
    for (int it = tid; it < NV * h3; it += T) {
      const int c = it / h3, m = it - c * h3;
      const int o = (2 * NV + c) * n3p + pidx<n>(m % n, (m / n) % n, kb + m / n2);
      sC[o] = peer[o];
    }
  }
  cluster_arrive();  // this CTA's reads of the other one are done (waited for before exit)
  __syncthreads();
  // a7: D_hat sweep of the contravariant flux along direction g
  const int il = g == 0 ? i : (g == 1 ? j : k);
  real sum = real(0);
#pragma unroll
  for (int a = 0; a < n; ++a) {
    const real dh = sOp[a * n + il];
    const int ia = g == 0 ? pidx<n>(a, j, k) : (g == 1 ? pidx<n>(i, a, k) : pidx<n>(i, j, a));
    sum = dg_fma(dh, sC[(g * NV + v) * n3p + ia], sum);
  }
  sF[(g * NV + v) * n3p + pn] = sum;  // region 1: read by no one since the last cluster barrier
  __syncthreads();
  if (g == 0)
    Utv[((size_t)e * NV + v) * n3 + node] = sF[v * n3p + pn] + sF[(NV + v) * n3p + pn] + sF[(2 * NV + v) * n3p + pn];
  cluster_wait();  // the other CTA has finished reading this one's shared memory
}

template <typename real, int n, int SW, bool LGL, int SPLIT, bool BR2>
constexpr auto lift_vol_kernel() {
  if constexpr (lift_vol_min_blocks<real, n, SW, SPLIT, BR2>() > 0)
    return &k_lift_vol_mb<real, n, SW, LGL, SPLIT, BR2>;
  else
    return &k_lift_vol<real, n, SW, LGL, SPLIT, BR2>;
}

template <typename real, int n, int SW, int SPLIT = 0, bool BR2 = false>
constexpr size_t lift_vol_smem() {
  using C = Cfg<n>;
  // the FP64 form sweeps per node and needs no result buffer; the FP32 CUDA-core
  // lifting (not BR2) may sweep 15 fields at once
  constexpr int out = (sizeof(real) == 8 && SW == 0)
                          ? 0
                          : C::NE * ((SW == 0 && !BR2 && lift15_fills_better<n>()) ? 15 : NV) * C::n3p;
  return sizeof(real) * (C::NE * 15 * C::n3p + out + C::NE * 6 * 15 * C::n2 + C::n2 + 4 * n +
                         (SPLIT ? C::n2 : 0) + ((SPLIT && sizeof(real) == 8) ? C::NE * 3 * NV * C::n3p : 0) +
                         (BR2 ? C::NE * 6 * 15 * C::n2 + C::NE * C::n3p : 0)) +
         sizeof(int) * (C::NE * 12 + C::NE * 6 * C::n2);
}

// ---------------------------------------------------------------------------
// a5: numerical flux on every side (master normal)
// ---------------------------------------------------------------------------
// RS: the Riemann solver (FLEXI_RIEMANN_*; 0 serves Roe and smoothed Roe), a template
// parameter so that each kernel holds the registers of its own solver only
template <typename real, int n, int RS>
__global__ void __launch_bounds__(128, sizeof(real) == 4 ? 8 : 1) k_face(const real* __restrict__ Wf, const real* __restrict__ Gf,
                                              const real* __restrict__ fgeo, real* __restrict__ Ff, int S, int nBC,
                                              Phys<real> ph) {
  constexpr int n2 = n * n;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= S * n2) return;
  const int side = idx / n2, pq = idx - side * n2;
  real WL[NV], WR[NV], GL[15], GR[15], nv[3];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    WL[v] = Wf[((size_t)side * NV + v) * n2 + pq];
    WR[v] = Wf[((size_t)(S + side) * NV + v) * n2 + pq];
  }
  const bool bnd = side < nBC;
#pragma unroll
  for (int c = 0; c < 15; ++c) {
    GL[c] = Gf[((size_t)side * 15 + c) * n2 + pq];
    GR[c] = bnd ? GL[c] : Gf[((size_t)(S + side) * 15 + c) * n2 + pq];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) nv[d] = fgeo[((size_t)side * 4 + d) * n2 + pq];
  const real sa = fgeo[((size_t)side * 4 + 3) * n2 + pq];
  real f[NV], fl[NV], fr[NV];
  const real irL = real(1) / WL[0], irR = real(1) / WR[0];  // shared by the Riemann and viscous fluxes
  riemann_kind<RS>(WL, WR, irL, irR, nv, ph, f);
  visc_normal(WL, irL, GL, nv, ph, fl);
  visc_normal(WR, irR, GR, nv, ph, fr);
#pragma unroll
  for (int v = 0; v < NV; ++v) Ff[((size_t)side * NV + v) * n2 + pq] = (f[v] - real(0.5) * (fl[v] + fr[v])) * sa;
}

// The same flux for small meshes (few face nodes per SM): 32 face nodes per CTA of three
// warps, warp 0 computing the Riemann flux, warps 1 and 2 the viscous normal fluxes of
// the two sides, combined through shared memory; for the Roe fluxes a fourth warp takes
// the central part F(W_L).n + F(W_R).n and warp 0 the dissipation only.  Each thread runs
// a part of the dependent FP64 chain of k_face (an FP64 warp instruction holds its SM
// sub-partition for 64 clocks), which is what bounds a mesh that leaves most SMs idle.
template <typename real, int n, int RS>
__global__ void __launch_bounds__(128) k_face3(const real* __restrict__ Wf, const real* __restrict__ Gf,
                                               const real* __restrict__ fgeo, real* __restrict__ Ff, int S,
                                               int nSface, int nBC, Phys<real> ph) {
  constexpr int n2 = n * n;
  constexpr int R = RS == 0 ? 4 : 3;  // warps: Riemann (dissipation), viscous master, viscous slave, (central)
  __shared__ real sf[R][NV][32];
  const int role = threadIdx.x >> 5, lane = threadIdx.x & 31;  // warp-uniform role
  const int idx = blockIdx.x * 32 + lane;
  const bool live = idx < nSface * n2;
  const int side = live ? idx / n2 : 0, pq = live ? idx - side * n2 : 0;
  real nv[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) nv[d] = fgeo[((size_t)side * 4 + d) * n2 + pq];
  const bool bnd = side < nBC;
  real out[NV];
  if (role == 0 || role == 3) {
    real WL[NV], WR[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      WL[v] = Wf[((size_t)side * NV + v) * n2 + pq];
      WR[v] = Wf[((size_t)(S + side) * NV + v) * n2 + pq];
    }
    if constexpr (RS == 0) {
      if (role == 0)
        roe_dissipation(WL, WR, nv, ph, ph.riemann == 2, out);
      else
        roe_central(WL, WR, nv, ph, out);
    } else {
      riemann_kind<RS>(WL, WR, real(1) / WL[0], real(1) / WR[0], nv, ph, out);
    }
  } else {
    // role 1: the master (slot 0) side, role 2: the slave or boundary (slot 1) side,
    // whose gradients on a boundary are the inner ones
    const int slot = role - 1;
    real Wx[NV], Gx[15];
#pragma unroll
    for (int v = 0; v < NV; ++v) Wx[v] = Wf[((size_t)(slot * S + side) * NV + v) * n2 + pq];
    const int gslot = bnd ? 0 : slot;
#pragma unroll
    for (int c = 0; c < 15; ++c) Gx[c] = Gf[((size_t)(gslot * S + side) * 15 + c) * n2 + pq];
    visc_normal(Wx, real(1) / Wx[0], Gx, nv, ph, out);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) sf[role][v][lane] = out[v];
  __syncthreads();
  if (role == 0 && live) {
    const real sa = fgeo[((size_t)side * 4 + 3) * n2 + pq];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const real f = RS == 0 ? real(0.5) * (sf[R - 1][v][lane] - sf[0][v][lane]) : sf[0][v][lane];  // riemann_roe's (S - D) / 2
      Ff[((size_t)side * NV + v) * n2 + pq] = (f - real(0.5) * (sf[1][v][lane] + sf[2][v][lane])) * sa;
    }
  }
}

// ---------------------------------------------------------------------------
// a8-a10: surface integral, -1/J, RK stage update, face states of the new U
// ---------------------------------------------------------------------------
// TM > 1 (small meshes): TM times the threads, the first NE n^3 of them one per node, all
// of them sharing the loops over face nodes (the gather of the face fluxes and the face
// states of the new U), which otherwise take several dependent rounds of global-memory
// latency per thread on a mesh that leaves most SMs idle.
template <typename real, int n, int MODE, bool LGL, int TM = 1>
__global__ void __launch_bounds__(Cfg<n>::T * TM, TM > 1 ? 1 : ((sizeof(real) == 4 && Cfg<n>::T == 512) ? 4 : ((sizeof(real) == 4 && Cfg<n>::T == 216) ? 8 : 2))) k_surf(
    const real* __restrict__ Ff, const int* __restrict__ elemSide, const real* __restrict__ sJ,
    const real* __restrict__ Utv, real* __restrict__ U, real* __restrict__ dU, real* __restrict__ Ut,
    real* __restrict__ Wf, const double* __restrict__ xsol, RkStage<real> rk, double t, SourceParams src, int K,
    int S, Ops<real> ops, Phys<real> ph, unsigned* __restrict__ status) {
  using C = Cfg<n>;
  constexpr int n2 = C::n2, n3 = C::n3, NE = C::NE, T = C::T * TM;
  __shared__ real sF[NE * 6 * NV * n2];
  __shared__ real sU[(MODE == 1) ? NE * NV * C::n3p : 1];
  __shared__ real sOp[n2 + 4 * n];
  __shared__ int sES[NE * 6];
  const int tid = threadIdx.x;
  const bool nodeThread = TM == 1 || tid < C::T;
  const int tn = nodeThread ? tid : 0;
  const int el = tn / n3, node = tn - el * n3;
  const int e0 = blockIdx.x * NE;
  const int e = e0 + el;
  const bool valid = nodeThread && e < K;
  const int i = node % n, j = (node / n) % n, k = node / n2;
  // the node's own global values are requested first, so that their latency
  // overlaps the gather of the face fluxes and the barrier
  real vtv[NV], vU[NV], vdU[NV], sj = real(0);
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const size_t g = ((size_t)e * NV + v) * n3 + node;
      vtv[v] = Utv[g];
      if (MODE == 1) {
        vU[v] = U[g];
        vdU[v] = dU[g];
      }
    }
    sj = sJ[(size_t)e * n3 + node];
  }
  load_ops<real, n>(sOp, ops, tid, T);
  for (int t2 = tid; t2 < NE * 6; t2 += T) sES[t2] = (e0 + t2 / 6 < K) ? elemSide[(size_t)e0 * 6 + t2] : 0;
  __syncthreads();
  for (int it = tid; it < NE * 6 * n2; it += T) {
    const int el2 = it / (6 * n2);
    const int r = it - el2 * 6 * n2;
    const int s = r / n2, pq = r - s * n2;
    if (e0 + el2 >= K) continue;
    const int es = sES[el2 * 6 + s];
    const int mpq = orient_pq(es_orient(es), n - 1, pq % n, pq / n);
    const real* src_f = Ff + ((size_t)es_side(es) * NV) * n2 + mpq;
    const bool slave = es_slave(es);  // the slave side takes -f* s_hat
#pragma unroll
    for (int v = 0; v < NV; ++v) sF[((el2 * 6 + s) * NV + v) * n2 + pq] = dg_neg_if(src_f[v * n2], slave);
  }
  __syncthreads();
  // ut = U_t (MODE 0) or dt U_t (MODE 1: dt folded into the -1/J factor)
  real ut[NV];
  if (valid) {
    const real* lhm = sOp + n2 + 2 * n;
    const real* lhp = sOp + n2 + 3 * n;
    const real c0 = lhm[i], c1 = lhp[i], c2 = lhm[j], c3 = lhp[j], c4 = lhm[k], c5 = lhp[k];
    const int pq0 = j + n * k, pq1 = i + n * k, pq2 = i + n * j;
    const real* Fe = sF + el * 6 * NV * n2;
    const real scale = MODE == 1 ? -(rk.dt * sj) : -sj;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      real s = vtv[v];
      if (LGL) {  // Gauss-Lobatto: only nodes on a face receive its flux
        if (i == 0) s = dg_fma(c0, Fe[(0 * NV + v) * n2 + pq0], s);
        if (i == n - 1) s = dg_fma(c1, Fe[(1 * NV + v) * n2 + pq0], s);
        if (j == 0) s = dg_fma(c2, Fe[(2 * NV + v) * n2 + pq1], s);
        if (j == n - 1) s = dg_fma(c3, Fe[(3 * NV + v) * n2 + pq1], s);
        if (k == 0) s = dg_fma(c4, Fe[(4 * NV + v) * n2 + pq2], s);
        if (k == n - 1) s = dg_fma(c5, Fe[(5 * NV + v) * n2 + pq2], s);
      } else {
        s = dg_fma(c0, Fe[(0 * NV + v) * n2 + pq0], s);
        s = dg_fma(c1, Fe[(1 * NV + v) * n2 + pq0], s);
        s = dg_fma(c2, Fe[(2 * NV + v) * n2 + pq1], s);
        s = dg_fma(c3, Fe[(3 * NV + v) * n2 + pq1], s);
        s = dg_fma(c4, Fe[(4 * NV + v) * n2 + pq2], s);
        s = dg_fma(c5, Fe[(5 * NV + v) * n2 + pq2], s);
      }
      ut[v] = s * scale;
    }
    if (src.on) {
      double x[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) x[c] = xsol[((size_t)e * 3 + c) * n3 + node];
      const real sdt = MODE == 1 ? rk.dt : real(1);
      if constexpr (sizeof(real) == 4) {
        float Sv[NV];
        manufactured_source_f32(x, t, (float)src.gamma, (float)src.mu, (float)src.Pr, Sv);
#pragma unroll
        for (int v = 0; v < NV; ++v) ut[v] = dg_fma(sdt, Sv[v], ut[v]);
      } else {
        double Sv[NV];
        manufactured_source(x, t, src.gamma, src.mu, src.Pr, Sv);
#pragma unroll
        for (int v = 0; v < NV; ++v) ut[v] = dg_fma(sdt, (real)Sv[v], ut[v]);
      }
    }
  }
  if (MODE == 0) {
    if (valid) {
#pragma unroll
      for (int v = 0; v < NV; ++v) Ut[((size_t)e * NV + v) * n3 + node] = ut[v];
    }
    return;
  } else {
    if (valid) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const size_t g = ((size_t)e * NV + v) * n3 + node;
        const real du = dg_fma(rk.A, vdU[v], ut[v]);  // A dU + dt U_t
        const real un = dg_fma(rk.B, du, vU[v]);
        dU[g] = du;
        U[g] = un;
        sU[(el * NV + v) * C::n3p + pidx<n>(i, j, k)] = un;
      }
    } else if (nodeThread) {
#pragma unroll
      for (int v = 0; v < NV; ++v) sU[(el * NV + v) * C::n3p + pidx<n>(i, j, k)] = (v == 0 || v == 4) ? real(1) : real(0);
    }
    if (rk.prolong) {
      __syncthreads();
      faces_from_volume<real, n, LGL>(sU, ops, sES, e0, K, S, Wf, ph, status, tid, T);
    }
  }
}

// a5 and a8-a10 in one kernel for small FP64 meshes (n = 4, fewer elements than SMs, BR1,
// no mortars): each element computes the numerical fluxes of its six sides itself (an inner
// side twice, once by each of its elements), one thread per (warp role of k_face3, face
// node) with k_face3's arithmetic in the master frame of each side, so the fluxes are the
// same values; then the surface integral, -1/J and the RK update with one thread per
// (variable, node) and k_surf's expressions, and the face states of the new U.  On such
// meshes each kernel's chain of dependent instructions, not its work, sets the time, and
// this removes one kernel per stage.  The face states are read from WfIn and the new ones
// written to WfOut, another buffer: a neighbouring element may still read the old states
// of a shared side.
template <int RS, bool LGL>
__global__ void __launch_bounds__(384) k_surf_face(
    const double* __restrict__ WfIn, const double* __restrict__ Gf, const double* __restrict__ fgeo,
    const int* __restrict__ elemSide, const double* __restrict__ sJ, const double* __restrict__ Utv,
    double* __restrict__ U, double* __restrict__ dU, double* __restrict__ WfOut, const double* __restrict__ xsol,
    RkStage<double> rk, double t, SourceParams src, int K, int S, int nBC, Ops<double> ops, Phys<double> ph,
    unsigned* __restrict__ status) {
  using real = double;
  constexpr int n = 4, n2 = n * n, n3 = n2 * n, n3p = Cfg<n>::n3p, T = 384, FN = 6 * n2;
  constexpr int R = RS == 0 ? 4 : 3;  // roles of k_face3
  static_assert(R * FN <= T && NV * n3 <= T, "one thread per (role, face node) and per (variable, node)");
  __shared__ real sf[R][NV][FN];
  __shared__ real sSa[FN];          // s_hat of the face nodes (read with the normals)
  __shared__ real sF[6 * NV * n2];  // [6][5][n2] f* s_hat with the element's sign (k_surf's layout)
  __shared__ real sU[NV * n3p];
  __shared__ real sOp[n2 + 4 * n];
  __shared__ int sES[6];
  const int tid = threadIdx.x;
  const int e = blockIdx.x;  // grid = K
  // the (variable, node) of the update, whose global values are requested first
  const bool upd = tid < NV * n3;
  const int uv = upd ? tid / n3 : 0;  // warp-uniform
  const int node = upd ? tid - uv * n3 : 0;
  const int i = node % n, j = (node / n) % n, k = node / n2;
  const size_t gidx = ((size_t)e * NV + uv) * n3 + node;
  real vtv = real(0), vU = real(0), vdU = real(0), sj = real(0);
  if (upd) {
    vtv = Utv[gidx];
    vU = U[gidx];
    vdU = dU[gidx];
    sj = sJ[(size_t)e * n3 + node];
  }
  load_ops<real, n>(sOp, ops, tid, T);
  if (tid < 6) sES[tid] = elemSide[(size_t)e * 6 + tid];
  __syncthreads();
  // a5: role (warp-uniform: FN is a multiple of 32) and face node of the element
  const int role = tid / FN, fn = tid - role * FN;
  if (role < R) {
    const int s = fn / n2, pq = fn - s * n2;
    const int es = sES[s];
    const int side = es_side(es);
    const int mpq = orient_pq(es_orient(es), n - 1, pq % n, pq / n);
    real nv[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) nv[d] = fgeo[((size_t)side * 4 + d) * n2 + mpq];
    if (role == 0) sSa[fn] = fgeo[((size_t)side * 4 + 3) * n2 + mpq];
    const bool bnd = side < nBC;
    real out[NV];
    if (role == 0 || role == 3) {
      real WL[NV], WR[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        WL[v] = WfIn[((size_t)side * NV + v) * n2 + mpq];
        WR[v] = WfIn[((size_t)(S + side) * NV + v) * n2 + mpq];
      }
      if constexpr (RS == 0) {
        if (role == 0)
          roe_dissipation(WL, WR, nv, ph, ph.riemann == 2, out);
        else
          roe_central(WL, WR, nv, ph, out);
      } else {
        riemann_kind<RS>(WL, WR, real(1) / WL[0], real(1) / WR[0], nv, ph, out);
      }
    } else {
      const int slot = role - 1;  // master, slave or boundary side (inner gradients on a boundary)
      real Wx[NV], Gx[15];
#pragma unroll
      for (int v = 0; v < NV; ++v) Wx[v] = WfIn[((size_t)(slot * S + side) * NV + v) * n2 + mpq];
      const int gslot = bnd ? 0 : slot;
#pragma unroll
      for (int c = 0; c < 15; ++c) Gx[c] = Gf[((size_t)(gslot * S + side) * 15 + c) * n2 + mpq];
      visc_normal(Wx, real(1) / Wx[0], Gx, nv, ph, out);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) sf[role][v][fn] = out[v];
  }
  __syncthreads();
  if (tid < FN) {  // k_face3's combination times s_hat, then the element's sign (k_surf's gather)
    const int s = tid / n2, pq = tid - s * n2;
    const real sa = sSa[tid];
    const bool slave = es_slave(sES[s]);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const real f = RS == 0 ? real(0.5) * (sf[R - 1][v][tid] - sf[0][v][tid]) : sf[0][v][tid];
      sF[(s * NV + v) * n2 + pq] = dg_neg_if((f - real(0.5) * (sf[1][v][tid] + sf[2][v][tid])) * sa, slave);
    }
  }
  __syncthreads();
  // a8-a10 for variable uv at the node, with k_surf's expressions (dt folded into -1/J)
  if (upd) {
    const real* lhm = sOp + n2 + 2 * n;
    const real* lhp = sOp + n2 + 3 * n;
    const int pq0 = j + n * k, pq1 = i + n * k, pq2 = i + n * j;
    real a = vtv;
    if (LGL) {
      if (i == 0) a = dg_fma(lhm[i], sF[(0 * NV + uv) * n2 + pq0], a);
      if (i == n - 1) a = dg_fma(lhp[i], sF[(1 * NV + uv) * n2 + pq0], a);
      if (j == 0) a = dg_fma(lhm[j], sF[(2 * NV + uv) * n2 + pq1], a);
      if (j == n - 1) a = dg_fma(lhp[j], sF[(3 * NV + uv) * n2 + pq1], a);
      if (k == 0) a = dg_fma(lhm[k], sF[(4 * NV + uv) * n2 + pq2], a);
      if (k == n - 1) a = dg_fma(lhp[k], sF[(5 * NV + uv) * n2 + pq2], a);
    } else {
      a = dg_fma(lhm[i], sF[(0 * NV + uv) * n2 + pq0], a);
      a = dg_fma(lhp[i], sF[(1 * NV + uv) * n2 + pq0], a);
      a = dg_fma(lhm[j], sF[(2 * NV + uv) * n2 + pq1], a);
      a = dg_fma(lhp[j], sF[(3 * NV + uv) * n2 + pq1], a);
      a = dg_fma(lhm[k], sF[(4 * NV + uv) * n2 + pq2], a);
      a = dg_fma(lhp[k], sF[(5 * NV + uv) * n2 + pq2], a);
    }
    real ut = a * -(rk.dt * sj);
    if (src.on) {
      double x[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) x[c] = xsol[((size_t)e * 3 + c) * n3 + node];
      double Sv[NV];
      manufactured_source(x, t, src.gamma, src.mu, src.Pr, Sv);
      const double Su = uv == 0 ? Sv[0] : (uv == 1 ? Sv[1] : (uv == 2 ? Sv[2] : (uv == 3 ? Sv[3] : Sv[4])));
      ut = dg_fma(rk.dt, (real)Su, ut);
    }
    const real du = dg_fma(rk.A, vdU, ut);  // A dU + dt U_t
    const real un = dg_fma(rk.B, du, vU);
    dU[gidx] = du;
    U[gidx] = un;
    sU[uv * n3p + pidx<n>(i, j, k)] = un;
  }
  if (rk.prolong) {
    __syncthreads();
    faces_from_volume<real, n, LGL>(sU, ops, sES, e, K, S, WfOut, ph, status, tid, T);
  }
}

// k_surf_face on Gauss-Lobatto nodes with two CTAs per element (meshes with at most half as
// many elements as SMs): CTA r takes the nodes with k in [r n/2, (r + 1) n/2) and the face
// nodes that they lie on (faces 0-3 with q in that range, face 4 + r).  On Gauss-Lobatto
// nodes a node receives the flux and gives the state of a face only where it lies on it,
// so the two halves share nothing.  Warps are role-uniform, two per role over the half's
// 48 face nodes; FP64 warp instructions, which hold an SM sub-partition for 64 clocks
// whatever their active lanes, set the time here, so the twelve warps are placed (warp w on
// sub-partition w mod 4) to give each of the two longest chains, the Riemann dissipation
// (or the whole Riemann flux), a sub-partition of its own, and the central and viscous
// fluxes the other two.  Fluxes, update and face states use the expressions of k_surf_face.
template <int RS>
__global__ void __launch_bounds__(384) k_surf_face2(
    const double* __restrict__ WfIn, const double* __restrict__ Gf, const double* __restrict__ fgeo,
    const int* __restrict__ elemSide, const double* __restrict__ sJ, const double* __restrict__ Utv,
    double* __restrict__ U, double* __restrict__ dU, double* __restrict__ WfOut, const double* __restrict__ xsol,
    RkStage<double> rk, double t, SourceParams src, int K, int S, int nBC, Ops<double> ops, Phys<double> ph,
    unsigned* __restrict__ status) {
  using real = double;
  constexpr int n = 4, n2 = n * n, n3 = n2 * n, n3p = Cfg<n>::n3p, hk = n / 2, h3 = n3 / 2;
  constexpr int R = RS == 0 ? 4 : 3, T = 384;
  constexpr int FIJ = 4 * (n2 / 2), FH = FIJ + n2;  // face nodes of a half: faces 0-3, then face 4 + r
  static_assert(FH <= 64 && NV * h3 <= T, "two warps per role, one thread per (variable, node)");
  __shared__ real sf[R][NV][FH];
  __shared__ real sSa[FH];          // s_hat of the half's face nodes (read with the normals)
  __shared__ real sF[6 * NV * n2];  // k_surf's layout; only this half's face nodes are filled
  __shared__ real sU[NV * n3p];     // only this half's nodes are filled
  __shared__ real sOp[n2 + 4 * n];
  __shared__ int sES[6];
  const int tid = threadIdx.x;
  const int e = blockIdx.x >> 1, r = blockIdx.x & 1;  // grid = 2 K
  // half face node fh -> (side s of the element, face node pq)
  auto face_node = [r](int fh, int& s, int& pq) {
    if (fh < FIJ) {
      s = fh / (n2 / 2);
      const int m = fh - s * (n2 / 2);
      pq = m % n + n * (r * hk + m / n);
    } else {
      s = 4 + r;
      pq = fh - FIJ;
    }
  };
  const bool upd = tid < NV * h3;
  const int uv = upd ? tid / h3 : 0;  // warp-uniform
  const int ln = tid & 31;
  const int i = ln % n, j = (ln / n) % n, k = r * hk + ln / n2;
  const int node = i + n * (j + n * k);
  const size_t gidx = ((size_t)e * NV + uv) * n3 + node;
  real vtv = real(0), vU = real(0), vdU = real(0), sj = real(0);
  if (upd) {
    vtv = Utv[gidx];
    vU = U[gidx];
    vdU = dU[gidx];
    sj = sJ[(size_t)e * n3 + node];
  }
  load_ops<real, n>(sOp, ops, tid, T);
  if (tid < 6) sES[tid] = elemSide[(size_t)e * 6 + tid];
  __syncthreads();
  // a5: roles of warps 0-11, -1 idle: Roe {0, 0, 3, 3, -, -, 1, 1, -, -, 2, 2} (dissipation on
  // sub-partitions 0 and 1, central + viscous on 2 and 3), others {0, 0, 1, 1, -, -, 2, 2, -, ...}
  const int w = tid >> 5;
  int role = -1;
  if (w < 2) role = 0;
  else if (w < 4) role = RS == 0 ? 3 : 1;
  else if (w == 6 || w == 7) role = RS == 0 ? 1 : 2;
  else if ((w == 10 || w == 11) && RS == 0) role = 2;
  const int fh = (w & 1) * 32 + ln;
  if (role >= 0 && fh < FH) {
    int s, pq;
    face_node(fh, s, pq);
    const int es = sES[s];
    const int side = es_side(es);
    const int mpq = orient_pq(es_orient(es), n - 1, pq % n, pq / n);
    real nv[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) nv[d] = fgeo[((size_t)side * 4 + d) * n2 + mpq];
    if (role == 0) sSa[fh] = fgeo[((size_t)side * 4 + 3) * n2 + mpq];
    const bool bnd = side < nBC;
    real out[NV];
    if (role == 0 || role == 3) {
      real WL[NV], WR[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        WL[v] = WfIn[((size_t)side * NV + v) * n2 + mpq];
        WR[v] = WfIn[((size_t)(S + side) * NV + v) * n2 + mpq];
      }
      if constexpr (RS == 0) {
        if (role == 0)
          roe_dissipation(WL, WR, nv, ph, ph.riemann == 2, out);
        else
          roe_central(WL, WR, nv, ph, out);
      } else {
        riemann_kind<RS>(WL, WR, real(1) / WL[0], real(1) / WR[0], nv, ph, out);
      }
    } else {
      const int slot = role - 1;
      real Wx[NV], Gx[15];
#pragma unroll
      for (int v = 0; v < NV; ++v) Wx[v] = WfIn[((size_t)(slot * S + side) * NV + v) * n2 + mpq];
      const int gslot = bnd ? 0 : slot;
#pragma unroll
      for (int c = 0; c < 15; ++c) Gx[c] = Gf[((size_t)(gslot * S + side) * 15 + c) * n2 + mpq];
      visc_normal(Wx, real(1) / Wx[0], Gx, nv, ph, out);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) sf[role][v][fh] = out[v];
  }
  __syncthreads();
  if (tid < FH) {
    int s, pq;
    face_node(tid, s, pq);
    const real sa = sSa[tid];
    const bool slave = es_slave(sES[s]);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const real f = RS == 0 ? real(0.5) * (sf[R - 1][v][tid] - sf[0][v][tid]) : sf[0][v][tid];
      sF[(s * NV + v) * n2 + pq] = dg_neg_if((f - real(0.5) * (sf[1][v][tid] + sf[2][v][tid])) * sa, slave);
    }
  }
  __syncthreads();
  if (upd) {
    const real* lhm = sOp + n2 + 2 * n;
    const real* lhp = sOp + n2 + 3 * n;
    const int pq0 = j + n * k, pq1 = i + n * k, pq2 = i + n * j;
    real a = vtv;
    if (i == 0) a = dg_fma(lhm[i], sF[(0 * NV + uv) * n2 + pq0], a);
    if (i == n - 1) a = dg_fma(lhp[i], sF[(1 * NV + uv) * n2 + pq0], a);
    if (j == 0) a = dg_fma(lhm[j], sF[(2 * NV + uv) * n2 + pq1], a);
    if (j == n - 1) a = dg_fma(lhp[j], sF[(3 * NV + uv) * n2 + pq1], a);
    if (k == 0) a = dg_fma(lhm[k], sF[(4 * NV + uv) * n2 + pq2], a);
    if (k == n - 1) a = dg_fma(lhp[k], sF[(5 * NV + uv) * n2 + pq2], a);
    real ut = a * -(rk.dt * sj);
    if (src.on) {
      double x[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) x[c] = xsol[((size_t)e * 3 + c) * n3 + node];
      double Sv[NV];
      manufactured_source(x, t, src.gamma, src.mu, src.Pr, Sv);
      const double Su = uv == 0 ? Sv[0] : (uv == 1 ? Sv[1] : (uv == 2 ? Sv[2] : (uv == 3 ? Sv[3] : Sv[4])));
      ut = dg_fma(rk.dt, (real)Su, ut);
    }
    const real du = dg_fma(rk.A, vdU, ut);
    const real un = dg_fma(rk.B, du, vU);
    dU[gidx] = du;
    U[gidx] = un;
    sU[uv * n3p + pidx<n>(i, j, k)] = un;
  }
  if (rk.prolong) {
    __syncthreads();
    if (tid < FH) {  // faces_from_volume's Gauss-Lobatto copy for this half's face nodes
      int s, pq;
      face_node(tid, s, pq);
      const int l = s >> 1, p = pq % n, q = pq / n;
      const int vi = pvol_index<n>(l, (s & 1) ? n - 1 : 0, p, q);
      real Uf[NV], W[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Uf[v] = sU[v * n3p + vi];
      cons_to_prim(Uf, W, ph);
      if (!(W[0] > real(0)) || !(W[4] > real(0))) atomicOr(status, 1u);
      const int es = sES[s];
      const int mpq = orient_pq(es_orient(es), n - 1, p, q);
      real* dst = WfOut + ((size_t)(es_slave(es) * S + es_side(es)) * NV) * n2 + mpq;
#pragma unroll
      for (int v = 0; v < NV; ++v) dst[v * n2] = W[v];
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define FLEXI_DISPATCH_N(nval, ...) \
  switch (nval) {                    \
    case 2: { constexpr int NN = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int NN = 3; __VA_ARGS__; } break; \
    case 4: { constexpr int NN = 4; __VA_ARGS__; } break; \
    case 5: { constexpr int NN = 5; __VA_ARGS__; } break; \
    case 6: { constexpr int NN = 6; __VA_ARGS__; } break; \
    case 7: { constexpr int NN = 7; __VA_ARGS__; } break; \
    case 8: { constexpr int NN = 8; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;         \
  }

template <typename real, int n, bool LGL = false>
static cudaError_t prolong_n(const DevMesh& m, const real* U, const Ops<real>& ops, const Phys<real>& ph,
                             cudaStream_t st) {
  using C = Cfg<n>;
  const int grid = (m.K + C::NE - 1) / C::NE;
  k_prolong<real, n, LGL><<<grid, C::T, 0, st>>>(U, m.elemSide, (real*)m.Wf, m.K, m.S, ops, ph, m.status);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_prolong(const DevMesh& m, const real* U, const Ops<real>& ops, const Phys<real>& ph,
                           cudaStream_t st) {
  if (m.lgl) {
    FLEXI_DISPATCH_N(m.n, return prolong_n<real, NN, true>(m, U, ops, ph, st));
  }
  FLEXI_DISPATCH_N(m.n, return prolong_n<real, NN, false>(m, U, ops, ph, st));
  return cudaSuccess;
}

template <typename real>
cudaError_t launch_bc(const DevMesh& m, double t, const Phys<real>& ph, cudaStream_t st) {
  if (m.nBC == 0) return cudaSuccess;
  const int tot = m.nBC * m.n * m.n;
  FLEXI_DISPATCH_N(m.n, (k_bc<real, NN><<<(tot + 127) / 128, 128, 0, st>>>(m.xbc, m.bcKind, (const real*)m.fgeo,
                                                                          (real*)m.Wf, m.S, m.nBC, t, ph)));
  return cudaGetLastError();
}

template <typename real, int n, int SW, bool LGL = false, int SPLIT = 0, bool BR2 = false>
static cudaError_t lift_vol_n(const DevMesh& m, const real* U, const Ops<real>& ops, const Phys<real>& ph,
                              int store_grad, cudaStream_t st) {
  using C = Cfg<n>;
  constexpr size_t smem = lift_vol_smem<real, n, SW, SPLIT, BR2>();
  auto* kernel = lift_vol_kernel<real, n, SW, LGL, SPLIT, BR2>();
  static std::atomic<unsigned long long> attr{0};
  cudaError_t err = ensure_dynamic_smem(kernel, smem, attr);
  if (err != cudaSuccess) return err;
  const int grid = (m.K + C::NE - 1) / C::NE;
  kernel<<<grid, C::T, smem, st>>>(U, (const real*)m.Ja, (const real*)m.sJ,
                                                         (const real*)m.Wf, (const real*)m.fgeo, m.elemSide,
                                                         (real*)m.Gf, (real*)m.Utv,
                                                         store_grad ? (real*)m.Gvol : nullptr, m.K, m.S,
                                                         m.Sface, (const real*)m.QB,
                                                         ops, ph);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_lift_vol(const DevMesh& m, const real* U, const Ops<real>& ops, const Phys<real>& ph,
                            int store_grad, cudaStream_t st) {
  if constexpr (sizeof(real) == 4) {
    if (m.sweep_mode == 1) {
      FLEXI_DISPATCH_N(m.n, return lift_vol_n<real, NN, 1>(m, U, ops, ph, store_grad, st));
    } else if (m.sweep_mode == 2) {
      FLEXI_DISPATCH_N(m.n, return lift_vol_n<real, NN, 2>(m, U, ops, ph, store_grad, st));
    }
  }
  if constexpr (sizeof(real) == 8) {
    // at most half as many elements as SMs at n = 4: two CTAs per element (k_lift_vol_c2)
    if (!m.br2 && m.split == 0 && m.n == 4 && 2 * m.K <= m.nsm) {
      auto* kc2 = m.lgl ? &k_lift_vol_c2<4, true> : &k_lift_vol_c2<4, false>;
      kc2<<<2 * m.K, 15 * 64 / 2, 0, st>>>(U, (const double*)m.Ja, (const double*)m.sJ, (const double*)m.Wf,
                                          (const double*)m.fgeo, m.elemSide, (double*)m.Gf, (double*)m.Utv,
                                          store_grad ? (double*)m.Gvol : nullptr, m.K, m.S, m.Sface,
                                          (const double*)m.QB, ops, ph);
      return cudaGetLastError();
    }
    // fewer elements than SMs at n <= 4: three thread groups per element (k_lift_vol_g3)
    if (!m.br2 && m.split == 0 && m.n <= 4 && m.K < m.nsm) {
#define FLEXI_G3(NN, LG)                                                                                   \
  k_lift_vol_g3<NN, LG><<<m.K, 3 * NN * NN * NN, 0, st>>>(                                                 \
      U, (const double*)m.Ja, (const double*)m.sJ, (const double*)m.Wf, (const double*)m.fgeo, m.elemSide, \
      (double*)m.Gf, (double*)m.Utv, store_grad ? (double*)m.Gvol : nullptr, m.K, m.S, m.Sface,           \
      (const double*)m.QB, ops, ph)
      switch (m.n * 2 + m.lgl) {
        case 4: FLEXI_G3(2, false); break;
        case 5: FLEXI_G3(2, true); break;
        case 6: FLEXI_G3(3, false); break;
        case 7: FLEXI_G3(3, true); break;
        case 8: FLEXI_G3(4, false); break;
        case 9: FLEXI_G3(4, true); break;
        default: return cudaErrorInvalidValue;
      }
#undef FLEXI_G3
      return cudaGetLastError();
    }
  }
  if (m.br2) {
    if (m.lgl) {
      FLEXI_DISPATCH_N(m.n, return lift_vol_n<real, NN, 0, true, 0, true>(m, U, ops, ph, store_grad, st));
    }
    FLEXI_DISPATCH_N(m.n, return lift_vol_n<real, NN, 0, false, 0, true>(m, U, ops, ph, store_grad, st));
  }
  if (m.lgl && m.split == 1) {
    FLEXI_DISPATCH_N(m.n, return lift_vol_n<real, NN, 0, true, 1>(m, U, ops, ph, store_grad, st));
  }
  if (m.lgl && m.split == 2) {
    FLEXI_DISPATCH_N(m.n, return lift_vol_n<real, NN, 0, true, 2>(m, U, ops, ph, store_grad, st));
  }
  if (m.lgl) {
    FLEXI_DISPATCH_N(m.n, return lift_vol_n<real, NN, 0, true>(m, U, ops, ph, store_grad, st));
  }
  FLEXI_DISPATCH_N(m.n, return lift_vol_n<real, NN, 0>(m, U, ops, ph, store_grad, st));
  return cudaSuccess;
}

template <typename real>
cudaError_t launch_face(const DevMesh& m, const Phys<real>& ph, cudaStream_t st) {
  const int tot = m.Sface * m.n * m.n;  // big sides of mortars get their flux by projection
  if (tot == 0) return cudaSuccess;
  // small meshes (128-thread CTAs would leave SMs idle): three warps per 32 face nodes
  if ((tot + 127) / 128 < 2 * m.nsm) {
    const int grid = (tot + 31) / 32;
#define FLEXI_FACE3(RSV)                                                                                    \
  FLEXI_DISPATCH_N(m.n, (k_face3<real, NN, RSV><<<grid, RSV == 0 ? 128 : 96, 0, st>>>((const real*)m.Wf, (const real*)m.Gf, \
                                                                    (const real*)m.fgeo, (real*)m.Ff, m.S, \
                                                                    m.Sface, m.nBC, ph)))
    switch (ph.riemann) {
      case 1: FLEXI_FACE3(1); break;
      case 3: FLEXI_FACE3(3); break;
      case 4: FLEXI_FACE3(4); break;
      default: FLEXI_FACE3(0); break;
    }
#undef FLEXI_FACE3
    return cudaGetLastError();
  }
  const int TB = 128;
  switch (ph.riemann) {
    case 1:
      FLEXI_DISPATCH_N(m.n, (k_face<real, NN, 1><<<(tot + TB - 1) / TB, TB, 0, st>>>(
                                (const real*)m.Wf, (const real*)m.Gf, (const real*)m.fgeo, (real*)m.Ff, m.S, m.nBC, ph)));
      break;
    case 3:
      FLEXI_DISPATCH_N(m.n, (k_face<real, NN, 3><<<(tot + TB - 1) / TB, TB, 0, st>>>(
                                (const real*)m.Wf, (const real*)m.Gf, (const real*)m.fgeo, (real*)m.Ff, m.S, m.nBC, ph)));
      break;
    case 4:
      FLEXI_DISPATCH_N(m.n, (k_face<real, NN, 4><<<(tot + TB - 1) / TB, TB, 0, st>>>(
                                (const real*)m.Wf, (const real*)m.Gf, (const real*)m.fgeo, (real*)m.Ff, m.S, m.nBC, ph)));
      break;
    default:  // Roe (0) and smoothed Roe (2)
      FLEXI_DISPATCH_N(m.n, (k_face<real, NN, 0><<<(tot + TB - 1) / TB, TB, 0, st>>>(
                                (const real*)m.Wf, (const real*)m.Gf, (const real*)m.fgeo, (real*)m.Ff, m.S, m.nBC, ph)));
      break;
  }
  return cudaGetLastError();
}

template <typename real, int n, bool LGL>
static cudaError_t surf_n(const DevMesh& m, int mode, real* U, real* dU, real* Ut, const RkStage<real>& rk, double t,
                          const SourceParams& src, const Ops<real>& ops, const Phys<real>& ph, cudaStream_t st) {
  using C = Cfg<n>;
  const int grid = (m.K + C::NE - 1) / C::NE;
#define FLEXI_SURF(MODEV, TMV)                                                                                    \
  k_surf<real, n, MODEV, LGL, TMV><<<grid, C::T * TMV, 0, st>>>((const real*)m.Ff, m.elemSide, (const real*)m.sJ, \
                                                                 (const real*)m.Utv, U, dU, Ut, (real*)m.Wf, m.xsol, \
                                                                 rk, t, src, m.K, m.S, ops, ph, m.status)
  if constexpr (n <= 4) {
    if (grid < m.nsm) {  // fewer CTAs than SMs: six times the threads for the face loops
      if (mode == 0)
        FLEXI_SURF(0, 6);
      else
        FLEXI_SURF(1, 6);
      return cudaGetLastError();
    }
  }
  if (mode == 0)
    FLEXI_SURF(0, 1);
  else
    FLEXI_SURF(1, 1);
#undef FLEXI_SURF
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_surf(const DevMesh& m, int mode, real* U, real* dU, real* Ut, const RkStage<real>& rk, double t,
                        const SourceParams& src, const Ops<real>& ops, const Phys<real>& ph, cudaStream_t st) {
  if (m.lgl) {
    FLEXI_DISPATCH_N(m.n, return surf_n<real, NN, true>(m, mode, U, dU, Ut, rk, t, src, ops, ph, st));
  }
  FLEXI_DISPATCH_N(m.n, return surf_n<real, NN, false>(m, mode, U, dU, Ut, rk, t, src, ops, ph, st));
  return cudaSuccess;
}

}  // namespace flexi

// Discrete adjoint of the right-hand side: mu = (dL/dU)^T lam, by hand-written
// reverse mode of every step of the forward operator (steps a1..a9 of k_dg.cuh),
// for BR1 or BR2 lifting and the standard or split-form volume integral, on
// periodic meshes, meshes with boundary sides and (BR1) mortar meshes: the
// interpolation of the big side's state and gradients and the projections of the
// lifting and numerical fluxes are linear and are transposed in place
// (k_adj_mortar_interp, k_adj_mortar_project).  Numerical flux: the Roe fluxes have a hand-written
// reverse; HLLC, Rusanov and the entropy-conservative flux are differentiated in
// forward mode (dual numbers, ten tangents per face node).
// Boundary sides: the outer state is a function of the inner one (outflow: the
// same state; slip wall: normal velocity reversed, a reflection; exact state:
// independent of U) and the outer gradient is the inner one, so their adjoints
// flow back to the inner face state and gradient.  Source terms do not depend
// on U and drop out.
//
// Forward recompute (k_prolong, k_bc, k_lift_vol with the volume gradients
// stored), then, in reverse order of the forward data flow:
//   k_adj_lamface  element: lam_vol = -lam/J; its l_hat-weighted face values
//                  (transpose of the surface integral a8/a9)
//   k_adj_face     side: reverse of the numerical flux a5 (Roe + BR1 viscous)
//                  -> adjoints of the face states W_L, W_R and face gradients
//   k_adj_vol      element: reverse of a7 (D_hat^T sweeps), a6 (pointwise flux
//                  VJP), a4 (prolongation^T of the face-gradient adjoints), a3
//                  (lifting: 45 D_hat^T sweeps and the l_hat face projections),
//                  and the primitive map of the volume states
//   k_adj_side     side: BR1 mean (U* = (U_L + U_R)/2), the boundary state's
//                  transpose and the primitive map of the face states
//   k_adj_gather   element: prolongation^T of the face-state adjoints; out =
//                  (accumulate ? out : 0) + scale * mu
#pragma once
#include "dg_common.cuh"
#include "k_dg.cuh"
#include "k_mortar.cuh"
#include "launch.h"

namespace flexi {

// ---------------------------------------------------------------------------
// pointwise reverse-mode building blocks
// ---------------------------------------------------------------------------

// W = prim(U): accumulate lamU += (dW/dU)^T lamW  (expressed with W)
template <typename real>
__device__ __forceinline__ void prim_vjp(const real W[NV], const real lamW[NV], const Phys<real>& ph,
                                         real lamU[NV]) {
  const real ir = real(1) / W[0];
  const real q2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
  real l0 = lamW[0] + lamW[4] * ph.gm1 * real(0.5) * q2;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    l0 -= lamW[1 + c] * W[1 + c] * ir;
    lamU[1 + c] += lamW[1 + c] * ir - lamW[4] * ph.gm1 * W[1 + c];
  }
  lamU[0] += l0;
  lamU[4] += lamW[4] * ph.gm1;
}

// viscous flux reverse: given lamF[d][5] for F^v_d(W, G), accumulate lamW, lamG
template <typename real>
__device__ __forceinline__ void visc_vjp(const real W[NV], const real G[15], const real lamF[3][NV],
                                         const Phys<real>& ph, real lamW[NV], real lamG[15]) {
  const real mu = ph.mu;
  const real div = G[0 * 5 + 1] + G[1 * 5 + 2] + G[2 * 5 + 3];
  const real ir = real(1) / W[0];
  real ldiv = real(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const real* lf = lamF[d];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      real tau = mu * (G[d * 5 + 1 + c] + G[c * 5 + 1 + d]);
      if (c == d) tau -= real(2.0 / 3.0) * mu * div;
      const real ltau = lf[1 + c] + lf[4] * W[1 + c];
      lamW[1 + c] += lf[4] * tau;
      lamG[d * 5 + 1 + c] += mu * ltau;
      lamG[c * 5 + 1 + d] += mu * ltau;
      if (c == d) ldiv -= real(2.0 / 3.0) * mu * ltau;
    }
    // heat flux: lam_th * dT_d, dT_d = (G[d5+4] - (p/rho) G[d5+0]) / rho
    const real ldT = lf[4] * ph.lam_th;
    const real g4 = G[d * 5 + 4], g0 = G[d * 5 + 0];
    lamG[d * 5 + 4] += ldT * ir;
    lamG[d * 5 + 0] -= ldT * W[4] * ir * ir;
    lamW[4] -= ldT * g0 * ir * ir;
    lamW[0] += ldT * (-g4 * ir * ir + real(2) * W[4] * g0 * ir * ir * ir);
  }
  lamG[0 * 5 + 1] += ldiv;
  lamG[1 * 5 + 2] += ldiv;
  lamG[2 * 5 + 3] += ldiv;
}

// convective flux F^c_d(U, W) reverse: lamF[5] -> lamU (direct), lamW
template <typename real>
__device__ __forceinline__ void conv_vjp(const real U[NV], const real W[NV], int d, const real lf[NV], real lamU[NV],
                                         real lamW[NV]) {
  lamU[1 + d] += lf[0];
  real lud = lf[4] * (U[4] + W[4]);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    lamU[1 + c] += lf[1 + c] * W[1 + d];
    lud += lf[1 + c] * U[1 + c];
  }
  lamU[4] += lf[4] * W[1 + d];
  lamW[1 + d] += lud;
  lamW[4] += lf[1 + d] + lf[4] * W[1 + d];
}

template <typename real>
__device__ __forceinline__ void absf_vjp(real x, real del, real idel, bool smooth, real& val, real& dx, real& ddel) {
  const real ax = dg_abs(x);
  if (smooth && ax < del) {  // idel = 1 / del
    const real ih = real(0.5) * idel;
    val = (x * x + del * del) * ih;
    dx = x * idel;
    ddel = (del * del - x * x) * ih * idel;
  } else {
    val = ax;
    dx = x < real(0) ? real(-1) : (x > real(0) ? real(1) : real(0));
    ddel = real(0);
  }
}

// Roe flux reverse: given lamf, accumulate lamWL, lamWR (recomputes the forward)
template <typename real>
__device__ __forceinline__ void roe_vjp(const real WL[NV], const real WR[NV], const real n[3], const Phys<real>& ph,
                                        bool smooth, const real lf[NV], real lWL[NV], real lWR[NV]) {
  const real gm1 = ph.gm1;
  // ---- forward
  const real q2L = WL[1] * WL[1] + WL[2] * WL[2] + WL[3] * WL[3];
  const real q2R = WR[1] * WR[1] + WR[2] * WR[2] + WR[3] * WR[3];
  const real EL = WL[4] * ph.inv_gm1 + real(0.5) * WL[0] * q2L;
  const real ER = WR[4] * ph.inv_gm1 + real(0.5) * WR[0] * q2R;
  const real unL = WL[1] * n[0] + WL[2] * n[1] + WL[3] * n[2];
  const real unR = WR[1] * n[0] + WR[2] * n[1] + WR[3] * n[2];
  // one reciprocal square root per side gives sqrt(rho), 1 / sqrt(rho) and 1 / rho; one more
  // gives c and 1 / c^2 (FP64 divisions and square roots are long dependent sequences)
  const real isL = dg_rsqrt(WL[0]), isR = dg_rsqrt(WR[0]);
  const real sL = WL[0] * isL, sR = WR[0] * isR;
  const real irL = isL * isL, irR = isR * isR;
  const real iws = real(1) / (sL + sR);
  const real HL = (EL + WL[4]) * irL, HR = (ER + WR[4]) * irR;
  real vel[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) vel[k] = (sL * WL[1 + k] + sR * WR[1 + k]) * iws;
  const real H = (sL * HL + sR * HR) * iws;
  const real q2 = vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2];
  const real c2 = gm1 * (H - real(0.5) * q2);
  const real ic = dg_rsqrt(c2);
  const real c = c2 * ic;
  const real ic2 = ic * ic;
  const real rho = sL * sR;
  const real un = vel[0] * n[0] + vel[1] * n[1] + vel[2] * n[2];
  const real dp = WR[4] - WL[4];
  real dv[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) dv[k] = WR[1 + k] - WL[1 + k];
  const real dun = dv[0] * n[0] + dv[1] * n[1] + dv[2] * n[2];
  const real a1 = (dp - rho * c * dun) * real(0.5) * ic2;
  const real a5 = (dp + rho * c * dun) * real(0.5) * ic2;
  const real a2 = (WR[0] - WL[0]) - dp * ic2;
  const real del = real(0.1) * c, idel = real(10) * ic;
  real l1, l2, l5, d1, d2, d5, e1, e2, e5;
  absf_vjp(un - c, del, idel, smooth, l1, d1, e1);
  absf_vjp(un, del, idel, smooth, l2, d2, e2);
  absf_vjp(un + c, del, idel, smooth, l5, d5, e5);
  const real w1 = l1 * a1, w5 = l5 * a5, w2 = l2 * a2, wt = l2 * rho;
  real dvt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) dvt[k] = dv[k] - dun * n[k];
  const real vdvt = vel[0] * dvt[0] + vel[1] * dvt[1] + vel[2] * dvt[2];
  // ---- reverse
  const real h = real(0.5);
  real lw1 = lf[0], lw5 = lf[0], lw2 = lf[0], lwt = real(0);
  real lvel[3] = {0, 0, 0}, lc = 0, lH = 0, lun = 0, lq2 = 0, ldvt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lw1 += lf[1 + k] * (vel[k] - c * n[k]);
    lw5 += lf[1 + k] * (vel[k] + c * n[k]);
    lw2 += lf[1 + k] * vel[k];
    lwt += lf[1 + k] * dvt[k];
    lvel[k] = -h * (lf[1 + k] * (w1 + w5 + w2) + lf[4] * wt * dvt[k]);
    lc += -h * lf[1 + k] * (w5 - w1) * n[k];
    ldvt[k] = -h * (lf[1 + k] * wt + lf[4] * wt * vel[k]);
  }
  lw1 = -h * (lw1 + lf[4] * (H - un * c));
  lw5 = -h * (lw5 + lf[4] * (H + un * c));
  lw2 = -h * (lw2 + lf[4] * real(0.5) * q2);
  lwt = -h * (lwt + lf[4] * vdvt);
  lc += -h * lf[4] * (w5 - w1) * un;
  lH += -h * lf[4] * (w1 + w5);
  lun += -h * lf[4] * (w5 - w1) * c;
  lq2 += -h * lf[4] * w2 * real(0.5);
  // w = l a, wt = l2 rho
  const real la1 = lw1 * l1, la5 = lw5 * l5, la2 = lw2 * l2;
  const real ll1 = lw1 * a1, ll5 = lw5 * a5, ll2 = lw2 * a2 + lwt * rho;
  real lrho = lwt * l2;
  // dvt = dv - dun n
  real ldv[3], ldun = real(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ldv[k] = ldvt[k];
    ldun -= ldvt[k] * n[k];
  }
  // |.| terms (delta = 0.1 c)
  lun += ll1 * d1 + ll2 * d2 + ll5 * d5;
  lc += -ll1 * d1 + ll5 * d5 + real(0.1) * (ll1 * e1 + ll2 * e2 + ll5 * e5);
  // a1, a5, a2
  const real hic2 = h * ic2;
  real ldp = (la1 + la5) * hic2 - la2 * ic2;
  lrho += (-la1 + la5) * hic2 * c * dun;
  lc += (-la1 + la5) * hic2 * rho * dun;
  ldun += (-la1 + la5) * hic2 * rho * c;
  real lic2 = la1 * (dp - rho * c * dun) * h + la5 * (dp + rho * c * dun) * h - la2 * dp;
  const real ldrho = la2;
  // dun = dv . n
#pragma unroll
  for (int k = 0; k < 3; ++k) ldv[k] += ldun * n[k];
  // un = vel . n
#pragma unroll
  for (int k = 0; k < 3; ++k) lvel[k] += lun * n[k];
  // rho = sL sR
  real lsL = lrho * sR, lsR = lrho * sL;
  // ic2 = 1/c2, c = sqrt(c2)
  real lc2 = -lic2 * ic2 * ic2 + lc * h * ic;
  // c2 = gm1 (H - q2/2)
  lH += gm1 * lc2;
  lq2 -= h * gm1 * lc2;
#pragma unroll
  for (int k = 0; k < 3; ++k) lvel[k] += real(2) * vel[k] * lq2;
  // H = (sL HL + sR HR) iws ; vel = (sL uL + sR uR) iws
  real liws = lH * (sL * HL + sR * HR);
  lsL += lH * HL * iws;
  lsR += lH * HR * iws;
  const real lHL = lH * sL * iws, lHR = lH * sR * iws;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    liws += lvel[k] * (sL * WL[1 + k] + sR * WR[1 + k]);
    lsL += lvel[k] * WL[1 + k] * iws;
    lsR += lvel[k] * WR[1 + k] * iws;
    lWL[1 + k] += lvel[k] * sL * iws;
    lWR[1 + k] += lvel[k] * sR * iws;
  }
  lsL -= liws * iws * iws;
  lsR -= liws * iws * iws;
  // dp, dv, drho
  lWR[4] += ldp;
  lWL[4] -= ldp;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lWR[1 + k] += ldv[k];
    lWL[1 + k] -= ldv[k];
  }
  lWR[0] += ldrho;
  lWL[0] -= ldrho;
  // per side: HL = (EL + pL)/rhoL, sL = sqrt(rhoL), FL = euler_normal, EL, unL; irK = 1/rho,
  // isK = 1/sqrt(rho)
  auto side = [&](const real* W, real E, real unK, real HK, real irK, real isK, real lHK, real lsK, real* lW) {
    real lE = lHK * irK;
    lW[4] += lHK * irK;
    lW[0] += -lHK * HK * irK + lsK * h * isK;
    // F = (rho un, rho un u + p n, (E + p) un), weight 1/2
    const real lF0 = h * lf[0], lF4 = h * lf[4];
    real lunK = lF0 * W[0] + lF4 * (E + W[4]);
    lW[0] += lF0 * unK;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const real lFk = h * lf[1 + k];
      lW[0] += lFk * unK * W[1 + k];
      lunK += lFk * W[0] * W[1 + k];
      lW[1 + k] += lFk * W[0] * unK;
      lW[4] += lFk * n[k];
    }
    lW[4] += lF4 * unK;
    lE += lF4 * unK;
    // unK = u . n ; E = p/gm1 + rho q2/2
#pragma unroll
    for (int k = 0; k < 3; ++k) lW[1 + k] += lunK * n[k] + lE * W[0] * W[1 + k];
    lW[4] += lE * ph.inv_gm1;
    lW[0] += lE * real(0.5) * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
  };
  side(WL, EL, unL, HL, irL, isL, lHL, lsL, lWL);
  side(WR, ER, unR, HR, irR, isR, lHR, lsR, lWR);
}

// ---------------------------------------------------------------------------
// reverse of the other numerical fluxes by forward-mode differentiation
// ---------------------------------------------------------------------------
// Dual number x + dx eps (eps^2 = 0): the templated flux functions of
// dg_common.cuh evaluated on Dual<real> give their directional derivative.
template <typename r>
struct Dual {
  r v, d;
  Dual() = default;
  __device__ constexpr Dual(double x) : v(r(x)), d(r(0)) {}
  __device__ constexpr Dual(r x, r dx) : v(x), d(dx) {}
  friend __device__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
  friend __device__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
  friend __device__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
  friend __device__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
  friend __device__ Dual operator/(Dual a, Dual b) {
    const r q = a.v / b.v;
    return Dual(q, (a.d - q * b.d) / b.v);
  }
  __device__ Dual& operator+=(Dual b) { return *this = *this + b; }
  __device__ Dual& operator-=(Dual b) { return *this = *this - b; }
  __device__ Dual& operator*=(Dual b) { return *this = *this * b; }
  friend __device__ bool operator<(Dual a, Dual b) { return a.v < b.v; }
  friend __device__ bool operator>(Dual a, Dual b) { return a.v > b.v; }
  friend __device__ bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
  friend __device__ bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
};

template <typename r>
__device__ __forceinline__ Dual<r> dg_sqrt(Dual<r> x) {
  const r s = dg_sqrt(x.v);
  return Dual<r>(s, x.d / (r(2) * s));
}
template <typename r>
__device__ __forceinline__ Dual<r> dg_rsqrt(Dual<r> x) {  // d(x^-1/2) = -x^-3/2 dx / 2
  const r s = dg_rsqrt(x.v);
  return Dual<r>(s, r(-0.5) * x.d * s * s * s);
}
template <typename r>
__device__ __forceinline__ Dual<r> dg_fma(Dual<r> a, Dual<r> b, Dual<r> c) {
  return a * b + c;
}
template <typename r>
__device__ __forceinline__ Dual<r> dg_log(Dual<r> x) {
  return Dual<r>(dg_log(x.v), x.d / x.v);
}
// min / max: the derivative of the selected argument
template <typename r>
__device__ __forceinline__ Dual<r> fmin(Dual<r> a, Dual<r> b) {
  return b.v < a.v ? b : a;
}
template <typename r>
__device__ __forceinline__ Dual<r> fmax(Dual<r> a, Dual<r> b) {
  return b.v > a.v ? b : a;
}

template <typename r>
__device__ __forceinline__ Phys<Dual<r>> dual_phys(const Phys<r>& p) {
  Phys<Dual<r>> q;
  q.gamma = Dual<r>(p.gamma, r(0));
  q.gm1 = Dual<r>(p.gm1, r(0));
  q.inv_gm1 = Dual<r>(p.inv_gm1, r(0));
  q.mu = Dual<r>(p.mu, r(0));
  q.lam_th = Dual<r>(p.lam_th, r(0));
  q.Ma = Dual<r>(p.Ma, r(0));
  q.eta_br2 = Dual<r>(p.eta_br2, r(0));
  q.riemann = p.riemann;
  q.bc_exact = p.bc_exact;
  return q;
}

// lamWL += (df/dWL)^T lamf, lamWR += (df/dWR)^T lamf for the flux ph.riemann
// (HLLC, Rusanov, entropy-conservative; the Roe fluxes have roe_vjp): one
// dual-number evaluation per input component, each dotted with lamf.  Branches
// (wave-speed min/max, the HLLC star regions) follow the forward evaluation.
template <typename real>
__device__ void riemann_vjp_dual(const real WL[NV], const real WR[NV], const real n[3], const Phys<real>& ph,
                                 const real lf[NV], real lWL[NV], real lWR[NV]) {
  using D = Dual<real>;
  const Phys<D> pd = dual_phys(ph);
  const D nd[3] = {D(n[0], real(0)), D(n[1], real(0)), D(n[2], real(0))};
  real g[2 * NV];
#pragma unroll 1
  for (int j = 0; j < 2 * NV; ++j) {
    D a[NV], b[NV], f[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      a[v] = D(WL[v], j == v ? real(1) : real(0));
      b[v] = D(WR[v], j == NV + v ? real(1) : real(0));
    }
    riemann(a, b, nd, pd, f);
    real s = real(0);
#pragma unroll
    for (int v = 0; v < NV; ++v) s += lf[v] * f[v].d;
    g[j] = s;
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    lWL[v] += g[v];
    lWR[v] += g[NV + v];
  }
}

// Logarithmic mean L(a, b) = (a - b) / (ln a - ln b), its partial dL/da and 1/L, from
// the variable f = (a - b)/(a + b), u = f^2 and F(u) = atanh(f)/f of Ismail and Roe:
// L = (a + b) / (2F), dL/da = (1 - 4 f b F'(u) / (F (a + b))) / (2F), with the series of
// F and F' = dF/du below u = 1e-2 (as in the forward log mean) and otherwise
// F = ln(a/b) / (2f), F' = (1/(1-u) - F) / (2u).
template <typename real>
__device__ __forceinline__ void log_mean_d(real a, real b, real& L, real& dLda, real& iL) {
  const real s = a + b;
  const real is = real(1) / s;
  const real f = (a - b) * is;
  const real u = f * f;
  real F, Fp;
  if (u < real(1e-2)) {
    F = real(1.0 / 15.0);
    F = F * u + real(1.0 / 13.0);
    F = F * u + real(1.0 / 11.0);
    F = F * u + real(1.0 / 9.0);
    F = F * u + real(1.0 / 7.0);
    F = F * u + real(1.0 / 5.0);
    F = F * u + real(1.0 / 3.0);
    F = F * u + real(1);
    Fp = real(7.0 / 15.0);
    Fp = Fp * u + real(6.0 / 13.0);
    Fp = Fp * u + real(5.0 / 11.0);
    Fp = Fp * u + real(4.0 / 9.0);
    Fp = Fp * u + real(3.0 / 7.0);
    Fp = Fp * u + real(2.0 / 5.0);
    Fp = Fp * u + real(1.0 / 3.0);
  } else {
    F = dg_log(a / b) / (real(2) * f);
    Fp = (real(1) / (real(1) - u) - F) / (real(2) * u);
  }
  const real iF = real(1) / F;
  L = real(0.5) * s * iF;
  iL = real(2) * F * is;
  dLda = real(0.5) * iF * (real(1) - real(4) * f * b * Fp * iF * is);
}

// Chandrashekar's pair flux reversed by hand: lamWx += d/dW_x (w . 2F#(W_x, W_a)), F# the
// entropy-conservative two-point flux in the averaged direction Jm = (Jx + Ja)/2.  With
// um = (u_x + u_a)/2, Un = um . Jm, f_rho = L(rho) Un, p~ = (rho_x + rho_a) / (2 (beta_x + beta_a)),
// E' = 1/(2 (gamma-1) L(beta)) - (|u_x|^2 + |u_a|^2)/4:  w . F# = f_rho B + p~ C with
// B = w_0 + w_1..3 . um + w_4 (E' + |um|^2) and C = w_1..3 . Jm + w_4 Un, whose partials reach W_x
// through L(rho), um, |u_x|^2, p~ and beta_x = rho_x / (2 p_x) (given per node with 1/p_x).
// both: W_a is W_x (the diagonal pair), twice the one-sided gradient.
template <typename real>
__device__ __forceinline__ void ec_pair_vjp(const real Wx[NV], real bx, real ipx, real qx, const real Wa[NV],
                                            real ba, const real Jx[3], const real Ja[3], real inv_gm1,
                                            const real w[NV], bool both, real lamWx[NV]) {
  const real Jm[3] = {real(0.5) * (Jx[0] + Ja[0]), real(0.5) * (Jx[1] + Ja[1]), real(0.5) * (Jx[2] + Ja[2])};
  const real um[3] = {real(0.5) * (Wx[1] + Wa[1]), real(0.5) * (Wx[2] + Wa[2]), real(0.5) * (Wx[3] + Wa[3])};
  const real Un = um[0] * Jm[0] + um[1] * Jm[1] + um[2] * Jm[2];
  real Lr, dLr, iLr, Lb, dLb, iLb;
  log_mean_d(Wx[0], Wa[0], Lr, dLr, iLr);
  log_mean_d(bx, ba, Lb, dLb, iLb);
  const real qa = Wa[1] * Wa[1] + Wa[2] * Wa[2] + Wa[3] * Wa[3];
  const real frho = Lr * Un;
  const real ibs = real(1) / (bx + ba);
  const real pt = real(0.5) * (Wx[0] + Wa[0]) * ibs;
  const real Ep = real(0.5) * inv_gm1 * iLb - real(0.25) * (qx + qa);
  const real B = w[0] + w[1] * um[0] + w[2] * um[1] + w[3] * um[2] +
                 w[4] * (Ep + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
  const real C = w[1] * Jm[0] + w[2] * Jm[1] + w[3] * Jm[2] + w[4] * Un;
  const real d_bx = -real(0.5) * inv_gm1 * frho * w[4] * iLb * iLb * dLb - C * pt * ibs;
  const real k = both ? real(4) : real(2);  // 2 F#, and twice that for the diagonal pair
  const real cu = B * Lr, c4 = pt * w[4], fw = frho * w[4];
  lamWx[0] += k * (B * Un * dLr + real(0.5) * C * ibs + real(0.5) * d_bx * ipx);
#pragma unroll
  for (int c = 0; c < 3; ++c)
    lamWx[1 + c] += k * real(0.5) * ((cu + c4) * Jm[c] + frho * w[1 + c] + fw * (real(2) * um[c] - Wx[1 + c]));
  lamWx[4] -= k * d_bx * bx * ipx;
}

// Pirozzoli's pair flux reversed by hand: lamWx += d/dW_x (w . 2F#(W_x, W_a)).  With the
// pair sums rs, s (velocity), ps, Hs and j = Jx + Ja, m = rs (s . j) / 8 and
// w . 2F# = m A + (ps / 2) (w_1..3 . j), A = 2 w_0 + w_1..3 . s + w_4 Hs, so the partials
// are d/drs = A (s . j) / 8, d/ds = A rs j / 8 + m w_1..3, d/dps = (w_1..3 . j) / 2 and
// d/dHs = m w_4, carried to W_x through H_x = gamma/(gamma-1) p/rho + |u|^2/2
// (dH/drho = dHdr, dH/du = u, dH/dp = dHdp, given per node).  both: W_a is W_x (the
// diagonal pair), whose gradient is twice the one-sided one (F# is symmetric).
template <typename real>
__device__ __forceinline__ void kep_pair_vjp(const real Wx[NV], real Hx, real dHdr, real dHdp, const real Wa[NV],
                                             real Ha, const real Jx[3], const real Ja[3], const real w[NV], bool both,
                                             real lamWx[NV]) {
  const real rs = Wx[0] + Wa[0], s0 = Wx[1] + Wa[1], s1 = Wx[2] + Wa[2], s2 = Wx[3] + Wa[3];
  const real j0 = Jx[0] + Ja[0], j1 = Jx[1] + Ja[1], j2 = Jx[2] + Ja[2];
  const real Hs = Hx + Ha;
  const real sj = s0 * j0 + s1 * j1 + s2 * j2;
  const real m = real(0.125) * rs * sj;
  const real A = real(2) * w[0] + w[1] * s0 + w[2] * s1 + w[3] * s2 + w[4] * Hs;
  const real c = real(0.125) * A;
  const real crs = c * rs;
  const real dH = m * w[4];
  const real k = both ? real(2) : real(1);
  lamWx[0] += k * (c * sj + dH * dHdr);
  lamWx[1] += k * (crs * j0 + m * w[1] + dH * Wx[1]);
  lamWx[2] += k * (crs * j1 + m * w[2] + dH * Wx[2]);
  lamWx[3] += k * (crs * j2 + m * w[3] + dH * Wx[3]);
  lamWx[4] += k * (real(0.5) * (w[1] * j0 + w[2] * j1 + w[3] * j2) + dH * dHdp);
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <typename real, int n>
__global__ void __launch_bounds__(Cfg<n>::T) k_adj_lamface(const real* __restrict__ lam, const real* __restrict__ sJ,
                                                            const int* __restrict__ elemSide, real* __restrict__ LF,
                                                            int K, int S, Ops<real> ops) {
  using C = Cfg<n>;
  constexpr int n2 = C::n2, n3 = C::n3, NE = C::NE, T = C::T;
  __shared__ real sL[NE * NV * n3];
  __shared__ real sOp[n2 + 4 * n];
  __shared__ int sES[NE * 6];
  const int tid = threadIdx.x;
  const int e0 = blockIdx.x * NE;
  load_ops<real, n>(sOp, ops, tid, T);
  for (int t = tid; t < NE * 6; t += T) sES[t] = (e0 + t / 6 < K) ? elemSide[(size_t)e0 * 6 + t] : 0;
  for (int t = tid; t < NE * NV * n3; t += T) {
    const int el = t / (NV * n3), r = t - el * NV * n3, node = r % n3;
    const int e = e0 + el;
    sL[t] = e < K ? -lam[(size_t)e * NV * n3 + r] * sJ[(size_t)e * n3 + node] : real(0);
  }
  __syncthreads();
  const real* lhm = sOp + n2 + 2 * n;
  const real* lhp = sOp + n2 + 3 * n;
  for (int it = tid; it < NE * 6 * n2; it += T) {
    const int el = it / (6 * n2);
    const int r = it - el * 6 * n2;
    const int s = r / n2, pq = r - s * n2;
    if (e0 + el >= K) continue;
    const int l = s >> 1;
    const real* lv = (s & 1) ? lhp : lhm;
    const int p = pq % n, q = pq / n;
    real acc[NV] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int a = 0; a < n; ++a) {
      const int vi = vol_index(l, a, p, q, n);
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += lv[a] * sL[(el * NV + v) * n3 + vi];
    }
    const int es = sES[el * 6 + s];
    const int mpq = orient_pq(es_orient(es), n - 1, p, q);
    real* dst = LF + ((size_t)(es_slave(es) * S + es_side(es)) * NV) * n2 + mpq;
#pragma unroll
    for (int v = 0; v < NV; ++v) dst[v * n2] = acc[v];
  }
}

// DUAL: the flux reverse by dual numbers (HLLC, Rusanov, entropy-conservative);
// otherwise the hand-written Roe reverse.
template <typename real, int n, bool DUAL>
__global__ void __launch_bounds__(128) k_adj_face(const real* __restrict__ Wf, const real* __restrict__ Gf,
                                                  const real* __restrict__ fgeo, const real* __restrict__ LF,
                                                  real* __restrict__ LWf, real* __restrict__ LGf, int S, int nBC,
                                                  int nFace, Phys<real> ph) {
  constexpr int n2 = n * n;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= S * n2) return;
  const int side = idx / n2, pq = idx - side * n2;
  if (side >= nFace) {  // big side of a mortar (no numerical flux of its own): start its adjoints at zero
#pragma unroll
    for (int slot = 0; slot < 2; ++slot) {
#pragma unroll
      for (int v = 0; v < NV; ++v) LWf[((size_t)(slot * S + side) * NV + v) * n2 + pq] = real(0);
#pragma unroll
      for (int c = 0; c < 15; ++c) LGf[((size_t)(slot * S + side) * 15 + c) * n2 + pq] = real(0);
    }
    return;
  }
  const bool bnd = side < nBC;  // boundary side: no slave element, outer gradient = inner gradient
  real WL[NV], WR[NV], GL[15], GR[15], nv[3], lf[NV];
  const real sa = fgeo[((size_t)side * 4 + 3) * n2 + pq];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    WL[v] = Wf[((size_t)side * NV + v) * n2 + pq];
    WR[v] = Wf[((size_t)(S + side) * NV + v) * n2 + pq];
    lf[v] = (LF[((size_t)side * NV + v) * n2 + pq] - (bnd ? real(0) : LF[((size_t)(S + side) * NV + v) * n2 + pq])) *
            sa;
  }
#pragma unroll
  for (int c = 0; c < 15; ++c) {
    GL[c] = Gf[((size_t)side * 15 + c) * n2 + pq];
    GR[c] = bnd ? GL[c] : Gf[((size_t)(S + side) * 15 + c) * n2 + pq];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) nv[d] = fgeo[((size_t)side * 4 + d) * n2 + pq];
  real lWL[NV] = {0, 0, 0, 0, 0}, lWR[NV] = {0, 0, 0, 0, 0};
  real lGL[15], lGR[15];
#pragma unroll
  for (int c = 0; c < 15; ++c) lGL[c] = lGR[c] = real(0);
  if constexpr (DUAL)
    riemann_vjp_dual(WL, WR, nv, ph, lf, lWL, lWR);
  else
    roe_vjp(WL, WR, nv, ph, ph.riemann == 2, lf, lWL, lWR);
  real lF[3][NV];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int v = 0; v < NV; ++v) lF[d][v] = -real(0.5) * nv[d] * lf[v];
  visc_vjp(WL, GL, lF, ph, lWL, lGL);
  visc_vjp(WR, GR, lF, ph, lWR, lGR);
  if (bnd) {
#pragma unroll
    for (int c = 0; c < 15; ++c) {
      lGL[c] += lGR[c];
      lGR[c] = real(0);
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    LWf[((size_t)side * NV + v) * n2 + pq] = lWL[v];
    LWf[((size_t)(S + side) * NV + v) * n2 + pq] = lWR[v];
  }
#pragma unroll
  for (int c = 0; c < 15; ++c) {
    LGf[((size_t)side * 15 + c) * n2 + pq] = lGL[c];
    LGf[((size_t)(S + side) * 15 + c) * n2 + pq] = lGR[c];
  }
}

// transposed sweep along direction l at the thread's node: sum_i Dhat[i][a_l] f(node with index_l = i)
template <typename real, int n>
__device__ __forceinline__ real dhatT_line(const real* __restrict__ sD, const real* __restrict__ f, int l, int i, int j,
                                           int k) {
  constexpr int n2 = n * n;
  real s = real(0);
  if (l == 0) {
#pragma unroll
    for (int b = 0; b < n; ++b) s += sD[i * n + b] * f[b + n * j + n2 * k];
  } else if (l == 1) {
#pragma unroll
    for (int b = 0; b < n; ++b) s += sD[j * n + b] * f[i + n * b + n2 * k];
  } else {
#pragma unroll
    for (int b = 0; b < n; ++b) s += sD[k * n + b] * f[i + n * j + n2 * b];
  }
  return s;
}

template <typename real, int n>
constexpr size_t adj_vol_smem(bool br2, bool split) {
  using C = Cfg<n>;
  return sizeof(real) * (C::NE * 15 * C::n3 + C::NE * 6 * 15 * C::n2 + C::n2 + 4 * n +
                         (br2 ? C::NE * C::n3 + C::NE * 6 * NV * C::n2 : 0) +
                         (split ? C::n2 + C::NE * 15 * C::n3 : 0)) +
         sizeof(int) * C::NE * 8;
}

// BR2: the face gradients are the broken gradient G - sum_f r_f plus eta r_s of
// the face's own lifting, r_f = (1/J) l_hat_f Jm_f with the jump
// Jm_f = (U* - W_own) n s_hat; their adjoints reach U* (added to LWs) and the
// element's own face state (added to its slot of LWf, written by k_adj_face).
// SPLIT (Gauss-Lobatto): the reverse of the split-form volume integral: the viscous
// part as in the standard form, the two-point advective sums reversed by hand per
// pair (each node collects d/dW of both ordered pairs it takes part in) and the
// strong-form face terms at the line ends.
template <typename real, int n, bool BR2, int SPLIT>
__global__ void __launch_bounds__(Cfg<n>::T) k_adj_vol(
    const real* __restrict__ U, const real* __restrict__ Ja, const real* __restrict__ sJ, const real* __restrict__ Gvol,
    const real* __restrict__ fgeo, const int* __restrict__ elemSide, const real* __restrict__ lam,
    const real* __restrict__ LGf, real* __restrict__ LWs, real* __restrict__ LWf, real* __restrict__ muv, int K, int S,
    int bigBase, real* __restrict__ LQB, Ops<real> ops, Phys<real> ph) {
  using C = Cfg<n>;
  constexpr int n2 = C::n2, n3 = C::n3, NE = C::NE, T = C::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real* sbuf = reinterpret_cast<real*>(smem_raw);  // [NE][15][n3]
  real* sF = sbuf + NE * 15 * n3;                  // [NE][6][15][n2] face-gradient adjoints
  real* sOp = sF + NE * 6 * 15 * n2;
  real* sSJ = sOp + n2 + 4 * n;                 // BR2: [NE][n3] 1/J
  real* sBr = sSJ + (BR2 ? NE * n3 : 0);        // BR2: [NE][6][5][n2] adjoint of U* from the jumps
  real* sDT = sBr + (BR2 ? NE * 6 * NV * n2 : 0);  // SPLIT: DT[a * n + i] = D[i][a]
  real* sWJ = sDT + (SPLIT ? n2 : 0);              // SPLIT: [NE][15][n3] W (5), Ja (9) and H per node
  int* sES = reinterpret_cast<int*>(sWJ + (SPLIT ? NE * 15 * n3 : 0));
  const int tid = threadIdx.x;
  const int el = tid / n3, node = tid - el * n3;
  const int e0 = blockIdx.x * NE;
  const int e = e0 + el;
  const bool valid = e < K;
  const int i = node % n, j = (node / n) % n, k = node / n2;
  load_ops<real, n>(sOp, ops, tid, T);
  for (int t = tid; t < NE * 6; t += T) sES[t] = (e0 + t / 6 < K) ? elemSide[(size_t)e0 * 6 + t] : 0;
  real Uo[NV], W[NV], jac[9], G[15], sj;
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Uo[v] = U[((size_t)e * NV + v) * n3 + node];
#pragma unroll
    for (int c = 0; c < 9; ++c) jac[c] = Ja[((size_t)e * 9 + c) * n3 + node];
#pragma unroll
    for (int c = 0; c < 15; ++c) G[c] = Gvol[((size_t)e * 15 + c) * n3 + node];
    sj = sJ[(size_t)e * n3 + node];
  } else {
    Uo[0] = real(1); Uo[1] = Uo[2] = Uo[3] = real(0); Uo[4] = real(1);
#pragma unroll
    for (int c = 0; c < 9; ++c) jac[c] = real(0);
#pragma unroll
    for (int c = 0; c < 15; ++c) G[c] = real(0);
    sj = real(0);
  }
  cons_to_prim(Uo, W, ph);
  real* myb = sbuf + el * 15 * n3;
  // lam_vol = -lam / J into the buffer
#pragma unroll
  for (int v = 0; v < NV; ++v) myb[v * n3 + node] = valid ? -lam[((size_t)e * NV + v) * n3 + node] * sj : real(0);
  if constexpr (SPLIT) {
    for (int t = tid; t < n2; t += T) sDT[t] = ops.DT[t];
    real* wj = sWJ + el * 15 * n3 + node;
#pragma unroll
    for (int v = 0; v < NV; ++v) wj[v * n3] = W[v];
#pragma unroll
    for (int c = 0; c < 9; ++c) wj[(NV + c) * n3] = jac[c];
    // kinetic-energy-preserving pairs: total enthalpy H = gamma/(gamma-1) p/rho + |u|^2/2;
    // entropy-conservative pairs: beta = rho / (2 p)
    wj[14 * n3] = SPLIT == 1 ? (ph.inv_gm1 + real(1)) * W[4] / W[0] + real(0.5) * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3])
                             : real(0.5) * W[0] / W[4];
  }
  // face-gradient adjoints of the element's six faces (own slot)
  __syncthreads();
  for (int it = tid; it < NE * 6 * n2; it += T) {
    const int el2 = it / (6 * n2);
    const int r = it - el2 * 6 * n2;
    const int s = r / n2, pq = r - s * n2;
    if (e0 + el2 >= K) continue;
    const int es = sES[el2 * 6 + s];
    const int mpq = orient_pq(es_orient(es), n - 1, pq % n, pq / n);
    const real* src = LGf + ((size_t)(es_slave(es) * S + es_side(es)) * 15) * n2 + mpq;
#pragma unroll
    for (int c = 0; c < 15; ++c) sF[((el2 * 6 + s) * 15 + c) * n2 + pq] = src[c * n2];
  }
  __syncthreads();
  const real* sD = sOp;
  // reverse of a7: lamFl[l][v] = (Dhat^T along l) lam_vol
  real lamU[NV] = {0, 0, 0, 0, 0}, lamW[NV] = {0, 0, 0, 0, 0}, lamG[15];
#pragma unroll
  for (int c = 0; c < 15; ++c) lamG[c] = real(0);
  {
    real lFl[3][NV];
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
      for (int v = 0; v < NV; ++v) lFl[l][v] = dhatT_line<real, n>(sD, myb + v * n3, l, i, j, k);
    // reverse of a6: lam_d = sum_l Ja^l_d lamFl[l]; F_d = F^c_d - F^v_d
    real lvisc[3][NV];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      real ld[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        ld[v] = jac[0 * 3 + d] * lFl[0][v] + jac[1 * 3 + d] * lFl[1][v] + jac[2 * 3 + d] * lFl[2][v];
        lvisc[d][v] = -ld[v];
      }
      if constexpr (!SPLIT) conv_vjp(Uo, W, d, ld, lamU, lamW);
    }
    visc_vjp(W, G, lvisc, ph, lamW, lamG);
  }
  if constexpr (SPLIT) {
    // advective part: sum_l sum_a D_{i_l a} 2F#(x, a) at every node x; node x collects
    // d/dW_x of its own sums (weight D[i_x][a] lam_x) and of its partners' sums in
    // which it appears (weight D[a][i_x] lam_a), in one evaluation per partner
    const real* lv = myb;  // lam_vol [5][n3] of this element
    const real* wj = sWJ + el * 15 * n3;
    // per node: the enthalpy and its partials with respect to rho and p (KEP pairs), or
    // beta, 1/p and |u|^2 (EC pairs)
    const real gg = ph.inv_gm1 + real(1), irx = real(1) / W[0], ipx = real(1) / W[4];
    const real x14 = wj[14 * n3 + node];  // this node's staged H (KEP) or beta (EC)
    const real dHdr = -gg * W[4] * irx * irx, dHdp = gg * irx;
    const real qx = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
#pragma unroll 1
    for (int l = 0; l < 3; ++l) {
      const int ix = l == 0 ? i : (l == 1 ? j : k);
      const real Jx[3] = {jac[l * 3], jac[l * 3 + 1], jac[l * 3 + 2]};
      real lx[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) lx[v] = lv[v * n3 + node];
#pragma unroll 1
      for (int a = 0; a < n; ++a) {
        const int na = l == 0 ? a + n * (j + n * k) : (l == 1 ? i + n * (a + n * k) : i + n * (j + n * a));
        real Wa[NV], w[NV];
        const real Jpa[3] = {wj[(NV + 3 * l) * n3 + na], wj[(NV + 3 * l + 1) * n3 + na],
                             wj[(NV + 3 * l + 2) * n3 + na]};
        const real dxa = sDT[a * n + ix], dax = sDT[ix * n + a];  // D[ix][a], D[a][ix]
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          Wa[v] = wj[v * n3 + na];
          w[v] = a == ix ? dxa * lx[v] : dxa * lx[v] + dax * lv[v * n3 + na];
        }
        if constexpr (SPLIT == 1)
          kep_pair_vjp(W, x14, dHdr, dHdp, Wa, wj[14 * n3 + na], Jx, Jpa, w, a == ix, lamW);
        else
          ec_pair_vjp(W, x14, ipx, qx, Wa, wj[14 * n3 + na], Jx, Jpa, ph.inv_gm1, w, a == ix, lamW);
      }
      // strong-form face terms at the line ends: c Fcal^{c,l}(U_x)
      if (ix == 0 || ix == n - 1) {
        const real c = ix == 0 ? sOp[n2 + 2 * n] : -sOp[n2 + 3 * n + n - 1];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          real lf[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) lf[v] = c * Jx[d] * lx[v];
          conv_vjp(Uo, W, d, lf, lamU, lamW);
        }
      }
    }
  }
  // reverse of a4: face gradients = prolongation of G
  {
    const real* lm = sOp + n2;
    const real* lp = sOp + n2 + n;
    const real* Fe = sF + el * 6 * 15 * n2;
    const int pq0 = j + n * k, pq1 = i + n * k, pq2 = i + n * j;
    const real c0 = lm[i], c1 = lp[i], c2 = lm[j], c3 = lp[j], c4 = lm[k], c5 = lp[k];
    real B[15];
#pragma unroll
    for (int c = 0; c < 15; ++c) {
      B[c] = c0 * Fe[(0 * 15 + c) * n2 + pq0] + c1 * Fe[(1 * 15 + c) * n2 + pq0] +
             c2 * Fe[(2 * 15 + c) * n2 + pq1] + c3 * Fe[(3 * 15 + c) * n2 + pq1] +
             c4 * Fe[(4 * 15 + c) * n2 + pq2] + c5 * Fe[(5 * 15 + c) * n2 + pq2];
      lamG[c] += B[c];
    }
    if constexpr (BR2) {
      // adjoint of the liftings r_f in the broken gradient: (1/J) times the
      // prolongation^T B of the face-gradient adjoints, reduced along each face's lines
      __syncthreads();  // the a7 reverse has read lam_vol from the buffer
#pragma unroll
      for (int c = 0; c < 15; ++c) myb[c * n3 + node] = B[c] * sj;
      sSJ[el * n3 + node] = sj;
      __syncthreads();
      const real* lhm = sOp + n2 + 2 * n;
      const real* lhp = sOp + n2 + 3 * n;
      for (int it = tid; it < NE * 6 * n2; it += T) {
        const int el2 = it / (6 * n2);
        const int r = it - el2 * 6 * n2;
        const int s = r / n2, pq = r - s * n2;
        if (e0 + el2 >= K) continue;
        const int l = s >> 1;
        const real* lv = (s & 1) ? lhp : lhm;  // l_hat(+-1)
        const real* lw = (s & 1) ? lp : lm;    // l(+-1)
        const int p = pq % n, q = pq / n;
        const int es = sES[el2 * 6 + s];
        const int side = es_side(es);
        const int mpq = orient_pq(es_orient(es), n - 1, p, q);
        const real* g = fgeo + ((size_t)side * 4) * n2 + mpq;
        const real sc = es_slave(es) ? -g[3 * n2] : g[3 * n2];
        const real nd[3] = {g[0] * sc, g[n2] * sc, g[2 * n2] * sc};
        const real* b = sbuf + el2 * 15 * n3;
        real kap = real(0);  // trace of the face's own lifting per unit jump
#pragma unroll
        for (int a = 0; a < n; ++a) kap += lw[a] * lv[a] * sSJ[el2 * n3 + vol_index(l, a, p, q, n)];
        const real ek = ph.eta_br2 * kap;
        real* own = LWf + ((size_t)(es_slave(es) * S + side) * NV) * n2 + mpq;
        const bool big = side >= bigBase;  // big side of a mortar: the jump's U* n s_hat is QB
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          real acc = real(0);
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const int c = d * NV + v;
            real lJ = ek * sF[((el2 * 6 + s) * 15 + c) * n2 + pq];
#pragma unroll
            for (int a = 0; a < n; ++a) lJ -= lv[a] * b[c * n3 + vol_index(l, a, p, q, n)];
            acc += nd[d] * lJ;
            if (big) LQB[((size_t)(side - bigBase) * 15 + v * 3 + d) * n2 + mpq] = lJ;  // -> QB
          }
          sBr[((el2 * 6 + s) * NV + v) * n2 + pq] = big ? real(0) : acc;  // -> U* (both sides' mean)
          own[v * n2] -= acc;  // -> the element's own face state
        }
      }
    }
  }
  // reverse of a3: lam_lift = lamG / J ; W receives sum_d sum_l Ja^l_d (Dhat^T_l lam_lift^d)
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 15; ++c) myb[c * n3 + node] = lamG[c] * sj;
  __syncthreads();
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const real a = jac[l * 3 + d];
#pragma unroll
      for (int v = 0; v < NV; ++v) lamW[v] += a * dhatT_line<real, n>(sD, myb + (d * NV + v) * n3, l, i, j, k);
    }
  // lifting surface terms: lamWstar_s[v](pq) = sum_d n_d s_hat sigma sum_a lhat_a lam_lift^d_v(line)
  {
    const real* lhm = sOp + n2 + 2 * n;
    const real* lhp = sOp + n2 + 3 * n;
    for (int it = tid; it < NE * 6 * n2; it += T) {
      const int el2 = it / (6 * n2);
      const int r = it - el2 * 6 * n2;
      const int s = r / n2, pq = r - s * n2;
      if (e0 + el2 >= K) continue;
      const int l = s >> 1;
      const real* lv = (s & 1) ? lhp : lhm;
      const int p = pq % n, q = pq / n;
      const int es = sES[el2 * 6 + s];
      const int side = es_side(es);
      const int mpq = orient_pq(es_orient(es), n - 1, p, q);
      const real* g = fgeo + ((size_t)side * 4) * n2 + mpq;
      const real sc = es_slave(es) ? -g[3 * n2] : g[3 * n2];
      const real nd[3] = {g[0] * sc, g[n2] * sc, g[2 * n2] * sc};
      const real* b = sbuf + el2 * 15 * n3;
      real* dst = LWs + ((size_t)(es_slave(es) * S + side) * NV) * n2 + mpq;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        real acc = real(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          real sdv = real(0);
#pragma unroll
          for (int a = 0; a < n; ++a) sdv += lv[a] * b[(d * NV + v) * n3 + vol_index(l, a, p, q, n)];
          acc += nd[d] * sdv;
        }
        if constexpr (BR2) acc += sBr[((el2 * 6 + s) * NV + v) * n2 + pq];
        dst[v * n2] = side >= bigBase ? real(0) : acc;  // big side: the lifting flux came from QB
      }
      if (side >= bigBase) {  // adjoint of the projected lifting flux QB (component v*3 + d)
        real* lq = LQB + ((size_t)(side - bigBase) * 15) * n2 + mpq;
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            real sdv = real(0);
#pragma unroll
            for (int a = 0; a < n; ++a) sdv += lv[a] * b[(d * NV + v) * n3 + vol_index(l, a, p, q, n)];
            lq[(v * 3 + d) * n2] = BR2 ? lq[(v * 3 + d) * n2] + sdv : sdv;  // BR2: the jump's part first
          }
      }
    }
  }
  // primitive map of the volume state
  prim_vjp(W, lamW, ph, lamU);
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) muv[((size_t)e * NV + v) * n3 + node] = lamU[v];
  }
}

// side: BR1 mean and the primitive map of the face states -> adjoint of U_face.
// Boundary sides: the adjoint of the outer state W_R = B(W_L) (flux and lifting
// mean) is added to the inner one through B^T (exact state: B = 0; outflow:
// B = I; slip wall: the velocity reflection I - 2 n n^T, symmetric); slot 1 is
// cleared (no element gathers it).
template <typename real, int n>
__global__ void __launch_bounds__(128) k_adj_side(const real* __restrict__ Wf, const real* __restrict__ LWs,
                                                  const real* __restrict__ fgeo, const int* __restrict__ bcKind,
                                                  real* __restrict__ LWf, int S, int nBC, int bigBase, Phys<real> ph) {
  constexpr int n2 = n * n;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= S * n2) return;
  const int side = idx / n2, pq = idx - side * n2;
  if (side >= bigBase) {  // big side of a mortar: its state reaches the fluxes through the
    // interpolation (transposed by k_adj_mortar_interp afterwards) and, with BR2, the
    // big element's own jumps (slot 0 of LWf, from k_adj_vol)
    real W[NV], lW[NV], lU[NV] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      W[v] = Wf[((size_t)side * NV + v) * n2 + pq];
      lW[v] = LWf[((size_t)side * NV + v) * n2 + pq];
    }
    prim_vjp(W, lW, ph, lU);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      LWf[((size_t)side * NV + v) * n2 + pq] = lU[v];
      LWf[((size_t)(S + side) * NV + v) * n2 + pq] = real(0);
    }
    return;
  }
  if (side < nBC) {
    real W[NV], lW[NV], lWR[NV], lU[NV] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const size_t g0 = ((size_t)side * NV + v) * n2 + pq, g1 = ((size_t)(S + side) * NV + v) * n2 + pq;
      W[v] = Wf[g0];
      lW[v] = LWf[g0] + real(0.5) * LWs[g0];
      lWR[v] = LWf[g1] + real(0.5) * LWs[g0];
    }
    const int kind = bcKind[side];
    if (kind == 1) {
#pragma unroll
      for (int v = 0; v < NV; ++v) lW[v] += lWR[v];
    } else if (kind == 2) {
      const real* g = fgeo + ((size_t)side * 4) * n2 + pq;
      const real nx = g[0], ny = g[n2], nz = g[2 * n2];
      const real ln = lWR[1] * nx + lWR[2] * ny + lWR[3] * nz;
      lW[0] += lWR[0];
      lW[1] += lWR[1] - real(2) * ln * nx;
      lW[2] += lWR[2] - real(2) * ln * ny;
      lW[3] += lWR[3] - real(2) * ln * nz;
      lW[4] += lWR[4];
    }
    prim_vjp(W, lW, ph, lU);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      LWf[((size_t)side * NV + v) * n2 + pq] = lU[v];
      LWf[((size_t)(S + side) * NV + v) * n2 + pq] = real(0);
    }
    return;
  }
#pragma unroll
  for (int slot = 0; slot < 2; ++slot) {
    real W[NV], lW[NV], lU[NV] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const size_t g0 = ((size_t)side * NV + v) * n2 + pq, g1 = ((size_t)(S + side) * NV + v) * n2 + pq;
      const size_t gs = slot ? g1 : g0;
      W[v] = Wf[gs];
      lW[v] = LWf[gs] + real(0.5) * (LWs[g0] + LWs[g1]);
    }
    prim_vjp(W, lW, ph, lU);
#pragma unroll
    for (int v = 0; v < NV; ++v) LWf[((size_t)(slot * S + side) * NV + v) * n2 + pq] = lU[v];
  }
}

// element: prolongation^T of the face-state adjoints, combine, scale/accumulate
template <typename real, int n>
__global__ void __launch_bounds__(Cfg<n>::T) k_adj_gather(const real* __restrict__ LUf, const int* __restrict__ elemSide,
                                                           const real* __restrict__ muv, real* __restrict__ out,
                                                           real scale, int accumulate, int K, int S, Ops<real> ops) {
  using C = Cfg<n>;
  constexpr int n2 = C::n2, n3 = C::n3, NE = C::NE, T = C::T;
  __shared__ real sF[NE * 6 * NV * n2];
  __shared__ real sOp[n2 + 4 * n];
  __shared__ int sES[NE * 6];
  const int tid = threadIdx.x;
  const int el = tid / n3, node = tid - el * n3;
  const int e0 = blockIdx.x * NE;
  const int e = e0 + el;
  const int i = node % n, j = (node / n) % n, k = node / n2;
  load_ops<real, n>(sOp, ops, tid, T);
  for (int t = tid; t < NE * 6; t += T) sES[t] = (e0 + t / 6 < K) ? elemSide[(size_t)e0 * 6 + t] : 0;
  __syncthreads();
  for (int it = tid; it < NE * 6 * n2; it += T) {
    const int el2 = it / (6 * n2);
    const int r = it - el2 * 6 * n2;
    const int s = r / n2, pq = r - s * n2;
    if (e0 + el2 >= K) continue;
    const int es = sES[el2 * 6 + s];
    const int mpq = orient_pq(es_orient(es), n - 1, pq % n, pq / n);
    const real* src = LUf + ((size_t)(es_slave(es) * S + es_side(es)) * NV) * n2 + mpq;
#pragma unroll
    for (int v = 0; v < NV; ++v) sF[((el2 * 6 + s) * NV + v) * n2 + pq] = src[v * n2];
  }
  __syncthreads();
  if (e >= K) return;
  const real* lm = sOp + n2;
  const real* lp = sOp + n2 + n;
  const real c0 = lm[i], c1 = lp[i], c2 = lm[j], c3 = lp[j], c4 = lm[k], c5 = lp[k];
  const int pq0 = j + n * k, pq1 = i + n * k, pq2 = i + n * j;
  const real* Fe = sF + el * 6 * NV * n2;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const size_t g = ((size_t)e * NV + v) * n3 + node;
    const real m = muv[g] + c0 * Fe[(0 * NV + v) * n2 + pq0] + c1 * Fe[(1 * NV + v) * n2 + pq0] +
                   c2 * Fe[(2 * NV + v) * n2 + pq1] + c3 * Fe[(3 * NV + v) * n2 + pq1] +
                   c4 * Fe[(4 * NV + v) * n2 + pq2] + c5 * Fe[(5 * NV + v) * n2 + pq2];
    out[g] = (accumulate ? out[g] : real(0)) + scale * m;
  }
}

// y = a*y + b*x (elementwise)
template <typename real>
__global__ void k_axpby(real* __restrict__ y, const real* __restrict__ x, real a, real b, size_t count) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < count) y[idx] = a * y[idx] + (x ? b * x[idx] : real(0));
}

// ---------------------------------------------------------------------------
// mortars: transposes of the interpolation and the projections (k_mortar.cuh)
// ---------------------------------------------------------------------------
// Transpose of k_mortar_interp: the adjoints of the virtual sides' slot 1 (NC
// components in each virtual side's frame) are mapped into the sub-square frame,
// multiplied by I^T along q and along p, and summed into the big side's slot 0
// (ACC: added to it, else written).  NC = 15: face gradients; NC = 5: conservative
// face states (the forward interpolates U = cons(W) and converts back, so the
// composition with the big side's primitive state is the identity).
template <typename real, int n, int NC, bool ACC>
__global__ void __launch_bounds__(kMortarThreads) k_adj_mortar_interp(real* __restrict__ L, const int* __restrict__ mbig,
                                                                      const int4* __restrict__ mvirt, int S,
                                                                      int bigBase, int vbase, MortarOps<real> mo) {
  constexpr int n2 = n * n;
  constexpr int PT = (n2 + kMortarThreads - 1) / kMortarThreads;
  __shared__ real sY[NC * n2];
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
    for (int t = tid; t < n2; t += kMortarThreads) {  // sub node (pp, qq) of virtual node T_oinv(pp, qq)
      const real* src = L + ((size_t)(S + v) * NC) * n2 + orient_pq(oinv, n - 1, t % n, t / n);
#pragma unroll
      for (int c = 0; c < NC; ++c) sY[c * n2 + t] = src[c * n2];
    }
    __syncthreads();
    // transpose of the pass along q: sT[m][pp] = sum_qq I^b[qq][m] sY[qq][pp]
    for (int t = tid; t < n2; t += kMortarThreads) {
      const int m = t / n, pp = t - m * n;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        real y;
        if (typ & 2) {
          y = real(0);
#pragma unroll
          for (int qq = 0; qq < n; ++qq) y += mo.I[b][qq * n + m] * sY[c * n2 + qq * n + pp];
        } else {
          y = sY[c * n2 + t];
        }
        sT[c * n2 + t] = y;
      }
    }
    __syncthreads();
    // transpose of the pass along p: big node (m, q) += sum_p' I^a[p'][m] sT[q][p']
#pragma unroll
    for (int k = 0; k < PT; ++k) {
      const int t = tid + k * kMortarThreads;
      if (t < n2) {
        const int q = t / n, m = t - q * n;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          if (typ & 1) {
#pragma unroll
            for (int pp = 0; pp < n; ++pp) acc[k][c] += mo.I[a][pp * n + m] * sT[c * n2 + q * n + pp];
          } else {
            acc[k][c] += sT[c * n2 + t];
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
        real* dst = L + ((size_t)(bigBase + bi) * NC + c) * n2 + t;
        *dst = ACC ? *dst + acc[k][c] : acc[k][c];
      }
    }
  }
}

// Transpose of k_mortar_project: y = (P^a)^T (P^b)^T of the big side's adjoint,
// mapped to each virtual side's own node.  KIND 1 (numerical flux): written to
// slot 1 of the virtual side's LF, so that k_adj_face's slot difference
// LF0 - LF1 applies the projection's minus sign.  KIND 0 (BR1 lifting flux of the
// big element, from LQB): adjoint of U* of the virtual side, -s_hat sum_d n_d
// y_{v*3+d}, written to slot 1 of LWs (k_adj_side adds half of it to each slot).
template <typename real, int n, int KIND>
__global__ void __launch_bounds__(kMortarThreads) k_adj_mortar_project(
    const real* __restrict__ Lbig, real* __restrict__ Lv, const real* __restrict__ fgeo, const int* __restrict__ mbig,
    const int4* __restrict__ mvirt, int S, int bigBase, int vbase, MortarOps<real> mo) {
  constexpr int n2 = n * n;
  constexpr int NC = KIND == 0 ? 15 : NV;
  __shared__ real sB[NC * n2];
  __shared__ real sT[NC * n2];
  const int tid = threadIdx.x;
  const int bi = blockIdx.x;
  const int* mb = mbig + bi * 8;
  const int typ = mb[0];
  const real* src = Lbig + (KIND == 0 ? (size_t)bi * 15 * n2 : (size_t)(bigBase + bi) * NV * n2);
  for (int t = tid; t < NC * n2; t += kMortarThreads) sB[t] = src[t];
  __syncthreads();
  for (int pos = 0; pos < 4; ++pos) {
    const int v = mb[1 + pos];
    if (v < 0) continue;  // uniform across the CTA
    int a, b;
    mortar_ab(typ, pos, a, b);
    const int oinv = mvirt[v - vbase].w;
    // transpose of the pass along p: sT[j][m] = sum_i P^a[i][m] sB[j][i]
    for (int t = tid; t < n2; t += kMortarThreads) {
      const int j = t / n, m = t - j * n;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        real y;
        if (typ & 1) {
          y = real(0);
#pragma unroll
          for (int i = 0; i < n; ++i) y += mo.P[a][i * n + m] * sB[c * n2 + j * n + i];
        } else {
          y = sB[c * n2 + t];
        }
        sT[c * n2 + t] = y;
      }
    }
    __syncthreads();
    // transpose of the pass along q: y[be][m] = sum_j P^b[j][be] sT[j][m], at sub node (m, be)
    for (int t = tid; t < n2; t += kMortarThreads) {
      const int be = t / n, m = t - be * n;
      const int spq = orient_pq(oinv, n - 1, m, be);
      real y[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (typ & 2) {
          y[c] = real(0);
#pragma unroll
          for (int j = 0; j < n; ++j) y[c] += mo.P[b][j * n + be] * sT[c * n2 + j * n + m];
        } else {
          y[c] = sT[c * n2 + t];
        }
      }
      if constexpr (KIND == 1) {
#pragma unroll
        for (int c = 0; c < NV; ++c) Lv[((size_t)(S + v) * NV + c) * n2 + spq] = y[c];
      } else {
        const real* g = fgeo + ((size_t)v * 4) * n2 + spq;
        const real sa = g[3 * n2];
#pragma unroll
        for (int c = 0; c < NV; ++c)
          Lv[((size_t)(S + v) * NV + c) * n2 + spq] =
              -sa * (g[0] * y[c * 3] + g[n2] * y[c * 3 + 1] + g[2 * n2] * y[c * 3 + 2]);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// launcher: forward recompute + reverse sweep
// ---------------------------------------------------------------------------
struct AdjScratch {
  void *LF, *LWf, *LGf, *LWs, *muv, *LQB;
};

inline AdjScratch adj_layout(const DevMesh& m, void* base, size_t rs) {
  const size_t sf5 = 2 * (size_t)m.S * NV * m.n * m.n * rs, sf15 = 2 * (size_t)m.S * 15 * m.n * m.n * rs;
  char* p = (char*)base;
  AdjScratch a;
  a.LF = p; p += sf5;
  a.LWf = p; p += sf5;
  a.LGf = p; p += sf15;
  a.LWs = p; p += sf5;
  a.muv = p; p += (size_t)m.K * NV * m.n * m.n * m.n * rs;
  a.LQB = p;  // [nBig][15][n^2]
  return a;
}

template <typename real, int n, bool BR2, int SPLIT>
static cudaError_t launch_adj_vol(const DevMesh& m, const real* U, const real* lam, const AdjScratch& a,
                                  const Ops<real>& ops, const Phys<real>& ph, int grid, cudaStream_t st) {
  constexpr size_t smem = adj_vol_smem<real, n>(BR2, SPLIT != 0);
  static std::atomic<unsigned long long> attr{0};
  cudaError_t err = ensure_dynamic_smem(k_adj_vol<real, n, BR2, SPLIT>, smem, attr);
  if (err != cudaSuccess) return err;
  k_adj_vol<real, n, BR2, SPLIT><<<grid, Cfg<n>::T, smem, st>>>(
      U, (const real*)m.Ja, (const real*)m.sJ, (const real*)m.Gvol, (const real*)m.fgeo, m.elemSide, lam,
      (const real*)a.LGf, (real*)a.LWs, (real*)a.LWf, (real*)a.muv, m.K, m.S, m.Sface, (real*)a.LQB, ops, ph);
  return cudaGetLastError();
}

template <typename real, int n>
static cudaError_t rhs_adjoint_n(const DevMesh& m, const real* U, const real* lam, real* out, real scale,
                                 int accumulate, const Ops<real>& ops, const MortarOps<real>& mo, const Phys<real>& ph,
                                 void* scratch, double t, cudaStream_t st) {
  using C = Cfg<n>;
  const int grid = (m.K + C::NE - 1) / C::NE;
  const int sgrid = (m.S * n * n + 127) / 128;
  AdjScratch a = adj_layout(m, scratch, sizeof(real));
  const int4* mv = (const int4*)m.mvirt;
  cudaError_t err;
  // forward recompute of face states, face gradients and volume gradients (and,
  // on mortar meshes, the virtual sides' interpolated states and gradients and QB)
  if ((err = prolong_n<real, n>(m, U, ops, ph, st)) != cudaSuccess) return err;
  if ((err = launch_bc<real>(m, t, ph, st)) != cudaSuccess) return err;
  if ((err = launch_mortar_state<real>(m, mo, ph, st)) != cudaSuccess) return err;
  if (m.br2) {
    if ((err = lift_vol_n<real, n, 0, false, 0, true>(m, U, ops, ph, 1, st)) != cudaSuccess) return err;
  } else {
    if ((err = lift_vol_n<real, n, 0>(m, U, ops, ph, 1, st)) != cudaSuccess) return err;
  }
  if ((err = launch_mortar_grad<real>(m, mo, ph, st)) != cudaSuccess) return err;
  k_adj_lamface<real, n><<<grid, C::T, 0, st>>>(lam, (const real*)m.sJ, m.elemSide, (real*)a.LF, m.K, m.S, ops);
  if (m.nBig > 0)  // the big element's flux adjoint to slot 1 of its virtual sides
    k_adj_mortar_project<real, n, 1><<<m.nBig, kMortarThreads, 0, st>>>((const real*)a.LF, (real*)a.LF, nullptr,
                                                                       m.mbig, mv, m.S, m.Sface, m.vbase, mo);
  if (ph.riemann == 0 || ph.riemann == 2)
    k_adj_face<real, n, false><<<sgrid, 128, 0, st>>>((const real*)m.Wf, (const real*)m.Gf, (const real*)m.fgeo,
                                                      (const real*)a.LF, (real*)a.LWf, (real*)a.LGf, m.S, m.nBC,
                                                      m.Sface, ph);
  else
    k_adj_face<real, n, true><<<sgrid, 128, 0, st>>>((const real*)m.Wf, (const real*)m.Gf, (const real*)m.fgeo,
                                                     (const real*)a.LF, (real*)a.LWf, (real*)a.LGf, m.S, m.nBC,
                                                     m.Sface, ph);
  if (m.nBig > 0)  // virtual sides' gradient adjoints (slot 1) to the big element's face gradient
    k_adj_mortar_interp<real, n, 15, false><<<m.nBig, kMortarThreads, 0, st>>>((real*)a.LGf, m.mbig, mv, m.S,
                                                                              m.Sface, m.vbase, mo);
  if (m.br2) {
    if ((err = launch_adj_vol<real, n, true, 0>(m, U, lam, a, ops, ph, grid, st)) != cudaSuccess) return err;
  } else if (m.split == 1) {
    if ((err = launch_adj_vol<real, n, false, 1>(m, U, lam, a, ops, ph, grid, st)) != cudaSuccess) return err;
  } else if (m.split == 2) {
    if ((err = launch_adj_vol<real, n, false, 2>(m, U, lam, a, ops, ph, grid, st)) != cudaSuccess) return err;
  } else {
    if ((err = launch_adj_vol<real, n, false, 0>(m, U, lam, a, ops, ph, grid, st)) != cudaSuccess) return err;
  }
  if (m.nBig > 0)  // adjoint of QB to U* of the virtual sides (slot 1 of LWs)
    k_adj_mortar_project<real, n, 0><<<m.nBig, kMortarThreads, 0, st>>>((const real*)a.LQB, (real*)a.LWs,
                                                                       (const real*)m.fgeo, m.mbig, mv, m.S,
                                                                       m.Sface, m.vbase, mo);
  k_adj_side<real, n><<<sgrid, 128, 0, st>>>((const real*)m.Wf, (const real*)a.LWs, (const real*)m.fgeo, m.bcKind,
                                             (real*)a.LWf, m.S, m.nBC, m.Sface, ph);
  if (m.nBig > 0)  // interpolated states' adjoints (slot 1, conservative) to the big element's face state
    k_adj_mortar_interp<real, n, NV, true><<<m.nBig, kMortarThreads, 0, st>>>((real*)a.LWf, m.mbig, mv, m.S,
                                                                             m.Sface, m.vbase, mo);
  k_adj_gather<real, n><<<grid, C::T, 0, st>>>((const real*)a.LWf, m.elemSide, (const real*)a.muv, out, scale,
                                               accumulate, m.K, m.S, ops);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_rhs_adjoint(const DevMesh& m, const real* U, const real* lam, real* out, real scale, int accumulate,
                               const Ops<real>& ops, const MortarOps<real>& mo, const Phys<real>& ph, void* scratch,
                               double t, cudaStream_t st) {
  FLEXI_DISPATCH_N(m.n, return rhs_adjoint_n<real, NN>(m, U, lam, out, scale, accumulate, ops, mo, ph, scratch, t, st));
  return cudaSuccess;
}

template <typename real>
cudaError_t launch_axpby(real* y, const real* x, real a, real b, size_t count, cudaStream_t st) {
  k_axpby<real><<<(unsigned)((count + 255) / 256), 256, 0, st>>>(y, x, a, b, count);
  return cudaGetLastError();
}

}  // namespace flexi

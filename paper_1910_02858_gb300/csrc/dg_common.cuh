// Shared device definitions of the GB300 DGSEM kernels: 1-D operators, side
// bookkeeping and the pointwise compressible Navier-Stokes physics.
//
// Physics readings (the paper gives the system abstractly, Eq. 3DconsLaw):
//   p = (gamma-1)(rho E - |m|^2/(2 rho));  F^c_d = (m_d, m_d u + p e_d, u_d(rho E + p))
//   tau = mu (grad u + grad u^T - 2/3 div u I);  q = -mu gamma/((gamma-1)Pr) grad(p/rho)
//   F^v_d = (0, tau_.d, tau_.d . u - q_d); lifted variables W = (rho, u, v, w, p).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace flexi {

constexpr int NV = 5;     // conserved / lifted variables
constexpr int MAXN = 8;   // n = N + 1 <= 8

template <typename real>
struct Ops {
  real DhatT[MAXN * MAXN];  // DhatT[a * n + i] = Dhat[i][a]  (Dhat_ij = -(w_j/w_i) D_ji)
  real lm[MAXN], lp[MAXN];  // l_j(-1), l_j(+1)
  real lhm[MAXN], lhp[MAXN];  // l_j(-1)/w_j, l_j(+1)/w_j
  real w[MAXN];
  real DT[MAXN * MAXN];  // DT[a * n + i] = D[i][a]  (strong-form derivative, split form only)
};

// mortar operators (Sec. "Non-conforming meshes"), a = 0 lower / 1 upper half:
// I[a][i * n + m] = l_m((x_i + 2a - 1)/2), P[a][i * n + al] = l_i((x_al + 2a - 1)/2) w_al / w_i
template <typename real>
struct MortarOps {
  real I[2][MAXN * MAXN];
  real P[2][MAXN * MAXN];
};

template <typename real>
struct Phys {
  real gamma, gm1, inv_gm1, mu, lam_th;  // lam_th = mu gamma / ((gamma-1) Pr)
  real Ma;
  real eta_br2;  // BR2 penalty on a face's own lifting
  int riemann;  // 0 Roe, 1 HLLC, 2 Roe with smoothed |lambda|, 3 Rusanov, 4 entropy conservative
  int bc_exact;
};

// Thread-block configuration of the element kernels: one thread per volume
// node, NE elements per CTA (at least 64 threads).  Staged element fields use
// i-lines padded to P = n + 1 entries (n3p per field) to spread shared-memory banks.
template <int n>
struct Cfg {
  static constexpr int n2 = n * n;
  static constexpr int n3 = n * n * n;
  static constexpr int NE = n3 >= 64 ? 1 : (64 + n3 - 1) / n3;
  static constexpr int T = NE * n3;
  static constexpr int P = n + 1;
  static constexpr int n3p = P * n * n;
};

// padded shared-memory offset of node (i, j, k)
template <int n>
__device__ __forceinline__ int pidx(int i, int j, int k) {
  return i + (n + 1) * (j + n * k);
}

// padded offset of face node (p, q) at position a along the face normal direction l
template <int n>
__device__ __forceinline__ int pvol_index(int l, int a, int p, int q) {
  return l == 0 ? pidx<n>(a, p, q) : (l == 1 ? pidx<n>(p, a, q) : pidx<n>(p, q, a));
}

// elemSide packing: (side << 4) | (slave << 3) | orient(local -> master frame)
__host__ __device__ __forceinline__ int es_side(int v) { return v >> 4; }
__host__ __device__ __forceinline__ int es_slave(int v) { return (v >> 3) & 1; }
__host__ __device__ __forceinline__ int es_orient(int v) { return v & 7; }

// (p, q) of this element's side-local frame -> flat index in the neighbour frame
__device__ __forceinline__ int orient_pq(int o, int N, int p, int q) {
  int a = (o & 1) ? q : p;
  int b = (o & 1) ? p : q;
  int pp = (o & 2) ? N - a : a;
  int qq = (o & 4) ? N - b : b;
  return qq * (N + 1) + pp;
}

// volume node of face node (p, q) at position a along the face normal direction l
__device__ __forceinline__ int vol_index(int l, int a, int p, int q, int n) {
  return l == 0 ? a + n * (p + n * q) : (l == 1 ? p + n * (a + n * q) : p + n * (q + n * a));
}

// ---------------------------------------------------------------------------
// pointwise physics
// ---------------------------------------------------------------------------
template <typename real>
__device__ __forceinline__ void cons_to_prim(const real U[NV], real W[NV], const Phys<real>& ph) {
  real ir = real(1) / U[0];
  real u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
  W[0] = U[0];
  W[1] = u;
  W[2] = v;
  W[3] = w;
  W[4] = ph.gm1 * (U[4] - real(0.5) * (U[1] * u + U[2] * v + U[3] * w));
}

template <typename real>
__device__ __forceinline__ void prim_to_cons(const real W[NV], real U[NV], const Phys<real>& ph) {
  U[0] = W[0];
  U[1] = W[0] * W[1];
  U[2] = W[0] * W[2];
  U[3] = W[0] * W[3];
  U[4] = W[4] * ph.inv_gm1 + real(0.5) * (U[1] * W[1] + U[2] * W[2] + U[3] * W[3]);
}

// Navier-Stokes flux F^c_d - F^v_d in physical direction d; G[d*5 + v] = dW_v/dx_d
template <typename real>
__device__ __forceinline__ void flux_total(const real U[NV], const real W[NV], const real G[15], int d,
                                           const Phys<real>& ph, real F[NV]) {
  const real ud = W[1 + d];
  const real p = W[4];
  // viscous stress column d: tau_cd = mu (du_c/dx_d + du_d/dx_c) - 2/3 mu div u delta_cd
  const real div = G[0 * 5 + 1] + G[1 * 5 + 2] + G[2 * 5 + 3];
  real tau[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) tau[c] = ph.mu * (G[d * 5 + 1 + c] + G[c * 5 + 1 + d]);
  tau[d] -= real(2.0 / 3.0) * ph.mu * div;
  const real ir = real(1) / W[0];
  const real dT = (G[d * 5 + 4] - p * ir * G[d * 5 + 0]) * ir;  // d(p/rho)/dx_d
  const real fv4 = tau[0] * W[1] + tau[1] * W[2] + tau[2] * W[3] + ph.lam_th * dT;
  F[0] = U[1 + d];
  F[1] = U[1] * ud - tau[0];
  F[2] = U[2] * ud - tau[1];
  F[3] = U[3] * ud - tau[2];
  F[1 + d] += p;
  F[4] = ud * (U[4] + p) - fv4;
}

// normal viscous flux F^v . n, with ir = 1 / rho of the state
template <typename real>
__device__ __forceinline__ void visc_normal(const real W[NV], const real ir, const real G[15], const real n[3],
                                            const Phys<real>& ph, real f[NV]) {
  const real div = G[0 * 5 + 1] + G[1 * 5 + 2] + G[2 * 5 + 3];
  real tn[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    real s = real(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) s += (G[d * 5 + 1 + c] + G[c * 5 + 1 + d]) * n[d];
    tn[c] = ph.mu * (s - real(2.0 / 3.0) * div * n[c]);
  }
  const real pir = W[4] * ir;
  real dTn = real(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) dTn += (G[d * 5 + 4] - pir * G[d * 5 + 0]) * n[d];
  f[0] = real(0);
  f[1] = tn[0];
  f[2] = tn[1];
  f[3] = tn[2];
  f[4] = tn[0] * W[1] + tn[1] * W[2] + tn[2] * W[3] + ph.lam_th * dTn * ir;
}

template <typename real>
__device__ __forceinline__ void visc_normal(const real W[NV], const real G[15], const real n[3],
                                            const Phys<real>& ph, real f[NV]) {
  visc_normal(W, real(1) / W[0], G, n, ph, f);
}

template <typename real>
__device__ __forceinline__ real dg_sqrt(real x);
template <>
__device__ __forceinline__ double dg_sqrt<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float dg_sqrt<float>(float x) { return sqrtf(x); }

template <typename real>
__device__ __forceinline__ real dg_rsqrt(real x);
template <>
__device__ __forceinline__ double dg_rsqrt<double>(double x) { return rsqrt(x); }
template <>
__device__ __forceinline__ float dg_rsqrt<float>(float x) { return rsqrtf(x); }

template <typename real>
__device__ __forceinline__ real dg_abs(real x) { return x < real(0) ? -x : x; }

// a * b + c in one rounding (one FP64 pipe slot for two flops in the FP64 form;
// a sum written as acc + (a0 b0 + a1 b1) costs a multiply, a fused multiply-add
// and an add instead of two fused multiply-adds)
__device__ __forceinline__ double dg_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float dg_fma(float a, float b, float c) { return fmaf(a, b, c); }

// -x when flag is set, by flipping the sign bit on the integer pipe (no FP64 multiply)
__device__ __forceinline__ double dg_neg_if(double x, bool flag) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)flag << 63));
}
__device__ __forceinline__ float dg_neg_if(float x, bool flag) {
  return __int_as_float(__float_as_int(x) ^ ((int)flag << 31));
}

// Euler normal flux from primitives
template <typename real>
__device__ __forceinline__ void euler_normal(const real W[NV], real E, real un, const real n[3], real F[NV]) {
  const real m = W[0] * un;
  F[0] = m;
  F[1] = m * W[1] + W[4] * n[0];
  F[2] = m * W[2] + W[4] * n[1];
  F[3] = m * W[3] + W[4] * n[2];
  F[4] = (E + W[4]) * un;
}

// HLLC (Toro) with Einfeldt/Davis wave speeds, frame-free form; irL, irR = 1 / rho.
// Roe averages with the weights sqrt(rho_L), sqrt(rho_R) written with their ratio
// r = sqrt(rho_R / rho_L): (a_L + r a_R) / (1 + r) (one square root, one division);
// the star-state factors mK / (S - S*) and p / mK share one division.
template <typename real>
__device__ __forceinline__ void riemann_hllc(const real WL[NV], const real WR[NV], const real irL, const real irR,
                                             const real n[3], const Phys<real>& ph, real f[NV]) {
  const real q2L = WL[1] * WL[1] + WL[2] * WL[2] + WL[3] * WL[3];
  const real q2R = WR[1] * WR[1] + WR[2] * WR[2] + WR[3] * WR[3];
  const real EL = WL[4] * ph.inv_gm1 + real(0.5) * WL[0] * q2L;
  const real ER = WR[4] * ph.inv_gm1 + real(0.5) * WR[0] * q2R;
  const real uL = WL[1] * n[0] + WL[2] * n[1] + WL[3] * n[2];
  const real uR = WR[1] * n[0] + WR[2] * n[1] + WR[3] * n[2];
  const real cL = dg_sqrt(ph.gamma * WL[4] * irL);
  const real cR = dg_sqrt(ph.gamma * WR[4] * irR);
  const real r = dg_sqrt(WR[0] * irL);
  const real iw = real(1) / (real(1) + r);
  const real HL = (EL + WL[4]) * irL, HR = (ER + WR[4]) * irR;
  real vel[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) vel[c] = (WL[1 + c] + r * WR[1 + c]) * iw;
  const real H = (HL + r * HR) * iw;
  const real c = dg_sqrt(ph.gm1 * (H - real(0.5) * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2])));
  const real un = vel[0] * n[0] + vel[1] * n[1] + vel[2] * n[2];
  const real SL = fmin(uL - cL, un - c);
  const real SR = fmax(uR + cR, un + c);
  if (SL >= real(0)) {
    euler_normal(WL, EL, uL, n, f);
    return;
  }
  if (SR <= real(0)) {
    euler_normal(WR, ER, uR, n, f);
    return;
  }
  const real mL = WL[0] * (SL - uL), mR = WR[0] * (SR - uR);
  const real Ss = (WR[4] - WL[4] + mL * uL - mR * uR) / (mL - mR);
  const bool left = Ss >= real(0);
  real W[NV];  // the upwind state, selected by value (a pointer select would force the arrays to memory)
#pragma unroll
  for (int v = 0; v < NV; ++v) W[v] = left ? WL[v] : WR[v];
  const real E = left ? EL : ER;
  const real uK = left ? uL : uR;
  const real S = left ? SL : SR;
  const real mK = left ? mL : mR;
  const real irK = left ? irL : irR;
  euler_normal(W, E, uK, n, f);
  // star state: fac (1, S* n + v_t, E/rho + (S*-u)(S* + p/(rho(S-u)))), fac = mK / (S - S*)
  const real dS = S - Ss;
  const real q = real(1) / (mK * dS);
  const real fac = mK * mK * q;
  const real U0 = W[0];
  f[0] += S * (fac - U0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const real vt = W[1 + c] - uK * n[c];
    f[1 + c] += S * (fac * (vt + Ss * n[c]) - U0 * W[1 + c]);
  }
  const real Estar = fac * (E * irK + (Ss - uK) * (Ss + W[4] * dS * q));
  f[4] += S * (Estar - E);
}

template <typename real>
__device__ __forceinline__ void riemann_hllc(const real WL[NV], const real WR[NV], const real n[3],
                                             const Phys<real>& ph, real f[NV]) {
  riemann_hllc(WL, WR, real(1) / WL[0], real(1) / WR[0], n, ph, f);
}

// Roe flux (5-wave, frame-free); smooth != 0: Harten-type smoothing of |lambda| (below
// delta = 0.1 c, (lambda^2 + delta^2) / (2 delta)).  Written as f = (S - D) / 2: the central
// part S = F(W_L).n + F(W_R).n and the dissipation D = sum_k |lambda_k| alpha_k r_k with
// Roe averages weighted by sqrt(rho) (riemann_roe ignores irL, irR).  The two parts are independent, so
// a kernel with few face nodes per SM computes them in separate warps.
template <typename real>
__device__ __forceinline__ void roe_central(const real WL[NV], const real WR[NV], const real n[3],
                                            const Phys<real>& ph, real S[NV]) {
  const real q2L = WL[1] * WL[1] + WL[2] * WL[2] + WL[3] * WL[3];
  const real q2R = WR[1] * WR[1] + WR[2] * WR[2] + WR[3] * WR[3];
  const real EL = WL[4] * ph.inv_gm1 + real(0.5) * WL[0] * q2L;
  const real ER = WR[4] * ph.inv_gm1 + real(0.5) * WR[0] * q2R;
  const real uL = WL[1] * n[0] + WL[2] * n[1] + WL[3] * n[2];
  const real uR = WR[1] * n[0] + WR[2] * n[1] + WR[3] * n[2];
  real FL[NV], FR[NV];
  euler_normal(WL, EL, uL, n, FL);
  euler_normal(WR, ER, uR, n, FR);
#pragma unroll
  for (int v = 0; v < NV; ++v) S[v] = FL[v] + FR[v];
}

template <typename real>
__device__ __forceinline__ void roe_dissipation(const real WL[NV], const real WR[NV], const real n[3],
                                                const Phys<real>& ph, bool smooth, real D[NV]) {
  const real q2L = WL[1] * WL[1] + WL[2] * WL[2] + WL[3] * WL[3];
  const real q2R = WR[1] * WR[1] + WR[2] * WR[2] + WR[3] * WR[3];
  const real EL = WL[4] * ph.inv_gm1 + real(0.5) * WL[0] * q2L;
  const real ER = WR[4] * ph.inv_gm1 + real(0.5) * WR[0] * q2R;
  // Roe averages (sqrt(rho_L) a_L + sqrt(rho_R) a_R) / (sqrt(rho_L) + sqrt(rho_R)); one
  // reciprocal square root per side gives sqrt(rho) and, for the enthalpy,
  // sqrt(rho) H = (E + p) / sqrt(rho)
  const real isL = dg_rsqrt(WL[0]), isR = dg_rsqrt(WR[0]);
  const real sL = WL[0] * isL, sR = WR[0] * isR;
  const real iw = real(1) / (sL + sR);
  real vel[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) vel[c] = dg_fma(sL, WL[1 + c], sR * WR[1 + c]) * iw;
  const real H = dg_fma(EL + WL[4], isL, (ER + WR[4]) * isR) * iw;
  const real q2 = vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2];
  const real c2 = ph.gm1 * (H - real(0.5) * q2);
  const real ic = dg_rsqrt(c2);  // c = c2 / sqrt(c2) and 1 / c2 from one reciprocal square root
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
  real l1 = dg_abs(un - c), l2 = dg_abs(un), l5 = dg_abs(un + c);
  if (smooth) {
    const real del = real(0.1) * c;
    const real ih = real(5) * ic;  // 1 / (2 del)
    if (l1 < del) l1 = (l1 * l1 + del * del) * ih;
    if (l2 < del) l2 = (l2 * l2 + del * del) * ih;
    if (l5 < del) l5 = (l5 * l5 + del * del) * ih;
  }
  const real w1 = l1 * a1, w5 = l5 * a5, w2 = l2 * a2, wt = l2 * rho;
  real dvt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) dvt[k] = dv[k] - dun * n[k];
  const real vdvt = vel[0] * dvt[0] + vel[1] * dvt[1] + vel[2] * dvt[2];
  D[0] = w1 + w5 + w2;
#pragma unroll
  for (int k = 0; k < 3; ++k)
    D[1 + k] = w1 * (vel[k] - c * n[k]) + w5 * (vel[k] + c * n[k]) + w2 * vel[k] + wt * dvt[k];
  D[4] = w1 * (H - un * c) + w5 * (H + un * c) + w2 * real(0.5) * q2 + wt * vdvt;
}

template <typename real>
__device__ __forceinline__ void riemann_roe(const real WL[NV], const real WR[NV], const real irL, const real irR,
                                            const real n[3], const Phys<real>& ph, bool smooth, real f[NV]) {
  real S[NV], D[NV];
  roe_central(WL, WR, n, ph, S);
  roe_dissipation(WL, WR, n, ph, smooth, D);
#pragma unroll
  for (int v = 0; v < NV; ++v) f[v] = real(0.5) * (S[v] - D[v]);
}

// Rusanov (local Lax-Friedrichs): central flux minus lambda_max/2 times the jump
template <typename real>
__device__ __forceinline__ void riemann_rusanov(const real WL[NV], const real WR[NV], const real n[3],
                                                const Phys<real>& ph, real f[NV]) {
  const real q2L = WL[1] * WL[1] + WL[2] * WL[2] + WL[3] * WL[3];
  const real q2R = WR[1] * WR[1] + WR[2] * WR[2] + WR[3] * WR[3];
  const real EL = WL[4] * ph.inv_gm1 + real(0.5) * WL[0] * q2L;
  const real ER = WR[4] * ph.inv_gm1 + real(0.5) * WR[0] * q2R;
  const real uL = WL[1] * n[0] + WL[2] * n[1] + WL[3] * n[2];
  const real uR = WR[1] * n[0] + WR[2] * n[1] + WR[3] * n[2];
  real FL[NV], FR[NV], UL[NV], UR[NV];
  euler_normal(WL, EL, uL, n, FL);
  euler_normal(WR, ER, uR, n, FR);
  prim_to_cons(WL, UL, ph);
  prim_to_cons(WR, UR, ph);
  const real cL = dg_sqrt(ph.gamma * WL[4] / WL[0]), cR = dg_sqrt(ph.gamma * WR[4] / WR[0]);
  const real lam = fmax(dg_abs(uL) + cL, dg_abs(uR) + cR);
#pragma unroll
  for (int v = 0; v < NV; ++v) f[v] = real(0.5) * (FL[v] + FR[v]) - real(0.5) * lam * (UR[v] - UL[v]);
}

template <typename real>
__device__ __forceinline__ real dg_log(real x);
template <>
__device__ __forceinline__ double dg_log<double>(double x) { return log(x); }
template <>
__device__ __forceinline__ float dg_log<float>(float x) { return logf(x); }

// logarithmic mean (a - b)/(ln a - ln b) of positive a, b (Ismail & Roe form):
// zeta = a/b, f = (zeta - 1)/(zeta + 1), u = f^2; mean = (a + b)/(2 F) with
// F = atanh(f)/f = ln(zeta)/(2 f), or its series sum_k u^k/(2k + 1) to u^7 for u < 1e-2
template <typename real>
__device__ __forceinline__ real log_mean(real a, real b) {
  const real zeta = a / b;
  const real f = (zeta - real(1)) / (zeta + real(1));
  const real u = f * f;
  real F;
  if (u < real(1e-2)) {
    F = real(1.0 / 15.0);
    F = F * u + real(1.0 / 13.0);
    F = F * u + real(1.0 / 11.0);
    F = F * u + real(1.0 / 9.0);
    F = F * u + real(1.0 / 7.0);
    F = F * u + real(1.0 / 5.0);
    F = F * u + real(1.0 / 3.0);
    F = F * u + real(1);
  } else {
    F = dg_log(zeta) / (real(2) * f);
  }
  return (a + b) / (real(2) * F);
}

// Chandrashekar's entropy-conservative two-point flux in the direction Jm (the
// averaged metric row, or the face normal), from the two sides' rho, velocity,
// beta = rho/(2p) and |u|^2:  f_rho = rho_ln {u}.Jm, f_m = f_rho {u} + ({rho}/(2{beta})) Jm,
// f_E = f_rho (1/(2(gamma-1) beta_ln) - {|u|^2}/2) + {u}.f_m
template <typename real>
__device__ __forceinline__ void ec_flux(real ra, const real ua[3], real ba, real qa, real rb, const real ub[3],
                                        real bb, real qb, const real Jm[3], const Phys<real>& ph, real f[NV]) {
  const real um[3] = {real(0.5) * (ua[0] + ub[0]), real(0.5) * (ua[1] + ub[1]), real(0.5) * (ua[2] + ub[2])};
  const real frho = log_mean(ra, rb) * (um[0] * Jm[0] + um[1] * Jm[1] + um[2] * Jm[2]);
  const real ptil = real(0.5) * (ra + rb) / (ba + bb);
  f[0] = frho;
  f[1] = frho * um[0] + ptil * Jm[0];
  f[2] = frho * um[1] + ptil * Jm[1];
  f[3] = frho * um[2] + ptil * Jm[2];
  f[4] = frho * (real(0.5) * ph.inv_gm1 / log_mean(ba, bb) - real(0.25) * (qa + qb)) + um[0] * f[1] + um[1] * f[2] +
         um[2] * f[3];
}

// entropy-conservative surface flux: ec_flux between the face states in the normal n
template <typename real>
__device__ __forceinline__ void riemann_ec(const real WL[NV], const real WR[NV], const real n[3], const Phys<real>& ph,
                                           real f[NV]) {
  const real uL[3] = {WL[1], WL[2], WL[3]}, uR[3] = {WR[1], WR[2], WR[3]};
  ec_flux(WL[0], uL, real(0.5) * WL[0] / WL[4], uL[0] * uL[0] + uL[1] * uL[1] + uL[2] * uL[2], WR[0], uR,
          real(0.5) * WR[0] / WR[4], uR[0] * uR[0] + uR[1] * uR[1] + uR[2] * uR[2], n, ph, f);
}

// numerical flux of a compile-time kind RS (FLEXI_RIEMANN_*: 0 Roe and 2 smoothed Roe
// both take the Roe branch, smoothing from ph), with irL, irR = 1 / rho
template <int RS, typename real>
__device__ __forceinline__ void riemann_kind(const real WL[NV], const real WR[NV], const real irL, const real irR,
                                             const real n[3], const Phys<real>& ph, real f[NV]) {
  if constexpr (RS == 1)
    riemann_hllc(WL, WR, irL, irR, n, ph, f);
  else if constexpr (RS == 3)
    riemann_rusanov(WL, WR, n, ph, f);
  else if constexpr (RS == 4)
    riemann_ec(WL, WR, n, ph, f);
  else
    riemann_roe(WL, WR, irL, irR, n, ph, ph.riemann == 2, f);
}

template <typename real>
__device__ __forceinline__ void riemann(const real WL[NV], const real WR[NV], const real n[3],
                                        const Phys<real>& ph, real f[NV]) {
  if (ph.riemann == 1)
    riemann_hllc(WL, WR, n, ph, f);
  else if (ph.riemann == 3)
    riemann_rusanov(WL, WR, n, ph, f);
  else if (ph.riemann == 4)
    riemann_ec(WL, WR, n, ph, f);
  else
    riemann_roe(WL, WR, real(1) / WL[0], real(1) / WR[0], n, ph, ph.riemann == 2, f);
}

// exact states (Dirichlet data) -- conservative variables at x, time t
template <typename real>
__device__ __forceinline__ void exact_state(int kind, const double x[3], double t, const Phys<real>& ph,
                                            real U[NV]) {
  double W[NV];
  const double g = (double)ph.gamma;
  if (kind == 0) {  // Taylor-Green vortex, V0 = L = rho0 = 1
    double sx, cx, sy, cy, sz, cz;
    sincos(x[0], &sx, &cx);
    sincos(x[1], &sy, &cy);
    sincos(x[2], &sz, &cz);
    const double Ma = (double)ph.Ma;
    W[0] = 1.0;
    W[1] = sx * cy * cz;
    W[2] = -cx * sy * cz;
    W[3] = 0.0;
    W[4] = 1.0 / (g * Ma * Ma) + (cos(2 * x[0]) + cos(2 * x[1])) * (cos(2 * x[2]) + 2.0) / 16.0;
    double Ud[NV];
    Ud[0] = W[0];
    Ud[1] = W[1];
    Ud[2] = W[2];
    Ud[3] = W[3];
    Ud[4] = W[4] / (g - 1.0) + 0.5 * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
    for (int v = 0; v < NV; ++v) U[v] = (real)Ud[v];
  } else if (kind == 1) {  // free stream rho = 1, u = (0.3, 0.2, 0.1), p = 1/gamma
    const double u = 0.3, v = 0.2, w = 0.1, p = 1.0 / g;
    U[0] = (real)1.0;
    U[1] = (real)u;
    U[2] = (real)v;
    U[3] = (real)w;
    U[4] = (real)(p / (g - 1.0) + 0.5 * (u * u + v * v + w * w));
  } else {  // manufactured: rho = 2 + 0.1 sin(pi (x+y+z-2t)), m = (rho,rho,rho), rhoE = rho^2
    const double rho = 2.0 + 0.1 * sin(M_PI * (x[0] + x[1] + x[2] - 2.0 * t));
    U[0] = U[1] = U[2] = U[3] = (real)rho;
    U[4] = (real)(rho * rho);
  }
}

// source term of the manufactured solution (derived by hand from the closed form
// with u = v = w = 1, p = (gamma-1)(rho^2 - 3 rho/2); checked against the oracle's
// automatic differentiation in the tests)
__device__ __forceinline__ void manufactured_source(const double x[3], double t, double gamma, double mu,
                                                    double Pr, double S[NV]) {
  const double A = 0.1, pi = M_PI;
  double s, c;
  sincos(pi * (x[0] + x[1] + x[2] - 2.0 * t), &s, &c);
  const double rho = 2.0 + A * s;
  const double dr = pi * A * c;  // d rho / dx (= dy = dz); d rho/dt = -2 dr
  const double dpx = (gamma - 1.0) * (2.0 * rho - 1.5) * dr;
  S[0] = dr;
  S[1] = S[2] = S[3] = dr + dpx;
  S[4] = 2.0 * rho * dr + 3.0 * dpx + 3.0 * (mu * gamma / Pr) * pi * pi * A * s;
}

// The same source term for the FP32 forms: the phase x + y + z - 2t is formed and
// reduced modulo 2 in FP64 (exact reduction of sin(pi r), cos(pi r) to r in [0, 2)),
// sin(pi r) and cos(pi r) come from sincospif, and the rest is FP32 arithmetic,
// so that the term costs a few FP64 operations per node instead of an FP64 sincos.
__device__ __forceinline__ void manufactured_source_f32(const double x[3], double t, float gamma, float mu,
                                                        float Pr, float S[NV]) {
  const float A = 0.1f, pi = 3.14159265358979323846f;
  const double ph = x[0] + x[1] + x[2] - 2.0 * t;
  const double r = ph - 2.0 * floor(0.5 * ph);
  float s, c;
  sincospif((float)r, &s, &c);
  const float rho = 2.0f + A * s;
  const float dr = pi * A * c;
  const float dpx = (gamma - 1.0f) * (2.0f * rho - 1.5f) * dr;
  S[0] = dr;
  S[1] = S[2] = S[3] = dr + dpx;
  S[4] = 2.0f * rho * dr + 3.0f * dpx + 3.0f * (mu * gamma / Pr) * pi * pi * A * s;
}

}  // namespace flexi

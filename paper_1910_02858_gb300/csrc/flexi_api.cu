// C-ABI layer of libflexi_gb300.so: context, mesh setup (connectivity and
// FP64 geometry precompute), orchestration of the per-stage kernels, the RK
// loop, reductions and kernel timing.  See include/flexi.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/flexi.h"
#include "basis_host.h"
#include "launch.h"

using namespace flexi;

namespace {

// Carpenter & Kennedy (1994) five-stage fourth-order 2N-storage coefficients
// (Williamson form, Sec. 3.4 names the scheme family; the paper prints none).
const double RK_A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double RK_B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};
const double RK_C[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                        2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

enum { KC_LIFTVOL = 0, KC_FACE = 1, KC_SURF = 2, KC_PROLONG = 3, KC_BC = 4, KC_ADJ = 5, KC_RED = 6, KC_OTHER = 7 };

}  // namespace

struct flexi_ctx {
  flexi_params p{};
  int device = -1;  // the CUDA device current at flexi_mesh_init; every call must run with it current
  int K = 0, N = 0, n = 0, n2 = 0, n3 = 0, S = 0, nBC = 0;
  bool fp64 = true;
  size_t rs = 8;
  DevMesh m;
  // FP64 geometry (always) and FP32 copies (FP32 forms)
  double *Ja64 = nullptr, *sJ64 = nullptr, *wJ = nullptr, *xsol = nullptr, *fgeo64 = nullptr, *xbc = nullptr;
  float *Ja32 = nullptr, *sJ32 = nullptr, *fgeo32 = nullptr;
  int* elemSide = nullptr;
  int* bcKind = nullptr;       // device [nBC]
  std::vector<int> bcId;       // host: boundary id of every boundary side
  std::vector<int> bcKindHost;
  unsigned* status = nullptr;
  double* partial = nullptr;
  double* partial_host = nullptr;
  int red_blocks = 0;
  void *Ustate = nullptr, *dUstate = nullptr;
  void* adj_scratch = nullptr;
  Ops<double> ops64{};
  Ops<float> ops32{};
  MortarOps<double> mops64{};
  MortarOps<float> mops32{};
  int nMortar = 0;
  // small FP64 meshes (n = 4, fewer elements than SMs, BR1, no mortars): the face fluxes
  // and the surface/RK kernel of an RK stage run as one kernel (k_surf_face), which reads
  // the face states of one buffer and writes those of the new U into another; m.Wf and the
  // two extra buffers take turns so that every step uses the same pattern (a CUDA graph of
  // one step stays valid)
  bool fused = false;
  void *WfA = nullptr, *WfB = nullptr;
  // CUDA graph of one RK step (flexi_rk_run), keyed by the buffers, dt and stream
  cudaGraphExec_t graph = nullptr;
  const void *gU = nullptr, *gdU = nullptr;
  double gdt = 0.0;
  cudaStream_t gst = nullptr;
  Phys<double> ph64{};
  Phys<float> ph32{};
  SourceParams src{};
  std::vector<void*> allocs;
  size_t dev_bytes = 0;
  // kernel timing
  bool prof = false;
  struct Rec { int cls; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  double ms[8] = {0};
  int64_t cnt[8] = {0};
};

namespace {

flexi_status cuda_status(cudaError_t e) { return e == cudaSuccess ? FLEXI_OK : FLEXI_ECUDA; }

// the calling thread's current device is the one the context's buffers live on
bool on_ctx_device(const flexi_ctx* c) {
  int d = -1;
  return cudaGetDevice(&d) == cudaSuccess && d == c->device;
}

#define CK(expr)                                   \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) return FLEXI_ECUDA;     \
  } while (0)

template <typename T>
flexi_status dalloc(flexi_ctx* c, T** ptr, size_t count) {
  void* p = nullptr;
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if (cudaMalloc(&p, bytes) != cudaSuccess) return FLEXI_ENOMEM;
  if (cudaMemset(p, 0, bytes) != cudaSuccess) return FLEXI_ECUDA;
  c->allocs.push_back(p);
  c->dev_bytes += bytes;
  *ptr = static_cast<T*>(p);
  return FLEXI_OK;
}

struct Prof {
  flexi_ctx* c;
  int cls;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  Prof(flexi_ctx* c_, int cls_, cudaStream_t st_) : c(c_), cls(cls_), st(st_) {
    if (c->prof) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, st);
    }
  }
  ~Prof() {
    if (c->prof) {
      cudaEventRecord(b, st);
      c->pending.push_back({cls, a, b});
    }
  }
};

void drain_profile(flexi_ctx* c) {
  for (auto& r : c->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->ms[r.cls] += ms;
      c->cnt[r.cls] += 1;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  c->pending.clear();
}

template <typename real>
const Ops<real>& ops_of(const flexi_ctx* c);
template <>
const Ops<double>& ops_of<double>(const flexi_ctx* c) { return c->ops64; }
template <>
const Ops<float>& ops_of<float>(const flexi_ctx* c) { return c->ops32; }
template <typename real>
const MortarOps<real>& mo_of(const flexi_ctx* c);
template <>
const MortarOps<double>& mo_of<double>(const flexi_ctx* c) { return c->mops64; }
template <>
const MortarOps<float>& mo_of<float>(const flexi_ctx* c) { return c->mops32; }
template <typename real>
const Phys<real>& ph_of(const flexi_ctx* c);
template <>
const Phys<double>& ph_of<double>(const flexi_ctx* c) { return c->ph64; }
template <>
const Phys<float>& ph_of<float>(const flexi_ctx* c) { return c->ph32; }

// one evaluation of the operator up to (and excluding) the surface kernel
// face = false: without the face fluxes (k_surf_face computes them)
template <typename real>
flexi_status stage_front(flexi_ctx* c, const real* U, double t, bool prolong, int store_grad, cudaStream_t st,
                         bool face = true) {
  const Ops<real>& ops = ops_of<real>(c);
  const Phys<real>& ph = ph_of<real>(c);
  if (prolong) {
    Prof pr(c, KC_PROLONG, st);
    CK(launch_prolong<real>(c->m, U, ops, ph, st));
  }
  if (c->nBC > 0) {
    Prof pr(c, KC_BC, st);
    CK(launch_bc<real>(c->m, t, ph, st));
  }
  if (c->nMortar > 0) {
    Prof pr(c, KC_OTHER, st);
    CK(launch_mortar_state<real>(c->m, mo_of<real>(c), ph, st));
  }
  {
    Prof pr(c, KC_LIFTVOL, st);
    CK(launch_lift_vol<real>(c->m, U, ops, ph, store_grad, st));
  }
  if (c->nMortar > 0) {
    Prof pr(c, KC_OTHER, st);
    CK(launch_mortar_grad<real>(c->m, mo_of<real>(c), ph, st));
  }
  if (face) {
    Prof pr(c, KC_FACE, st);
    CK(launch_face<real>(c->m, ph, st));
  }
  if (c->nMortar > 0) {
    Prof pr(c, KC_OTHER, st);
    CK(launch_mortar_flux<real>(c->m, mo_of<real>(c), st));
  }
  return FLEXI_OK;
}

template <typename real>
flexi_status do_rhs(flexi_ctx* c, const real* U, real* Ut, double t, cudaStream_t st) {
  flexi_status s = stage_front<real>(c, U, t, true, 0, st);
  if (s != FLEXI_OK) return s;
  RkStage<real> rk{real(0), real(0), real(0), 0};
  Prof pr(c, KC_SURF, st);
  CK(launch_surf<real>(c->m, 0, nullptr, nullptr, Ut, rk, t, c->src, ops_of<real>(c), ph_of<real>(c), st));
  return FLEXI_OK;
}

// faces_ready: the face states of U are already in place (written by the last stage of
// the previous step); prolong_last: the last stage also writes the face states of the new
// U for a following step (the same faces_from_volume arithmetic as the prolongation)
// fused stages (c->fused): stage k reads the face states of buffer in(k) and writes those of
// the new U into out(k): C -> B, B -> A, A -> B, B -> A, A -> C with C = m.Wf, so that a
// step starts and ends on m.Wf
template <typename real>
flexi_status do_rk_step_fused(flexi_ctx* c, real* U, real* dU, double t, double dt, real* stages, cudaStream_t st,
                              bool faces_ready, bool prolong_last) {
  if constexpr (sizeof(real) == 8) {
    void* const WfC = c->m.Wf;
    const size_t nU = (size_t)c->K * NV * c->n3;
    flexi_status res = FLEXI_OK;
    for (int k = 0; k < 5 && res == FLEXI_OK; ++k) {
      void* const win = k == 0 ? WfC : ((k & 1) ? c->WfB : c->WfA);
      void* const wout = k == 4 ? WfC : ((k & 1) ? c->WfA : c->WfB);
      const double tk = t + RK_C[k] * dt;
      if (stages != nullptr &&
          cudaMemcpyAsync(stages + k * nU, U, nU * sizeof(real), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        res = FLEXI_ECUDA;
        break;
      }
      c->m.Wf = win;  // prolongation, boundary states and the lifting use the stage's buffer
      res = stage_front<real>(c, U, tk, k == 0 && !faces_ready, 0, st, false);
      if (res != FLEXI_OK) break;
      RkStage<real> rk{(real)RK_A[k], (real)RK_B[k], (real)dt, (k < 4 || prolong_last) ? 1 : 0};
      Prof pr(c, KC_SURF, st);
      if (launch_surf_face(c->m, win, wout, U, dU, rk, tk, c->src, ops_of<real>(c), ph_of<real>(c), st) !=
          cudaSuccess)
        res = FLEXI_ECUDA;
    }
    c->m.Wf = WfC;
    return res;
  } else {
    return FLEXI_EUNSUPPORTED;
  }
}

template <typename real>
flexi_status do_rk_step(flexi_ctx* c, real* U, real* dU, double t, double dt, real* stages, cudaStream_t st,
                        bool faces_ready = false, bool prolong_last = false) {
  if (c->fused) return do_rk_step_fused<real>(c, U, dU, t, dt, stages, st, faces_ready, prolong_last);
  const size_t nU = (size_t)c->K * NV * c->n3;
  for (int k = 0; k < 5; ++k) {
    const double tk = t + RK_C[k] * dt;
    if (stages != nullptr) CK(cudaMemcpyAsync(stages + k * nU, U, nU * sizeof(real), cudaMemcpyDeviceToDevice, st));
    flexi_status s = stage_front<real>(c, U, tk, k == 0 && !faces_ready, 0, st);
    if (s != FLEXI_OK) return s;
    RkStage<real> rk{(real)RK_A[k], (real)RK_B[k], (real)dt, (k < 4 || prolong_last) ? 1 : 0};
    Prof pr(c, KC_SURF, st);
    CK(launch_surf<real>(c->m, 1, U, dU, nullptr, rk, tk, c->src, ops_of<real>(c), ph_of<real>(c), st));
  }
  return FLEXI_OK;
}

template <typename real>
void fill_ops(Ops<real>& o, const std::vector<double>& D, const std::vector<double>& w, const std::vector<double>& lm,
              const std::vector<double>& lp, int n) {
  std::memset(&o, 0, sizeof(o));
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < n; ++a) {
      const double dhat = -(w[a] / w[i]) * D[a * n + i];  // Dhat[i][a] = -(w_a/w_i) D_ai
      o.DhatT[a * n + i] = (real)dhat;
      o.DT[a * n + i] = (real)D[i * n + a];
    }
  for (int i = 0; i < n; ++i) {
    o.lm[i] = (real)lm[i];
    o.lp[i] = (real)lp[i];
    o.lhm[i] = (real)(lm[i] / w[i]);
    o.lhp[i] = (real)(lp[i] / w[i]);
    o.w[i] = (real)w[i];
  }
}

template <typename real>
void fill_phys(Phys<real>& ph, const flexi_params& p) {
  ph.gamma = (real)p.gamma;
  ph.gm1 = (real)(p.gamma - 1.0);
  ph.inv_gm1 = (real)(1.0 / (p.gamma - 1.0));
  ph.mu = (real)p.mu;
  ph.lam_th = (real)(p.mu * p.gamma / ((p.gamma - 1.0) * p.Pr));
  ph.Ma = (real)p.Ma;
  ph.eta_br2 = (real)p.eta_br2;
  ph.riemann = p.riemann;
  ph.bc_exact = p.bc_exact;
}

// orientation code composition helpers (host): T_o(p, q) on an n x n face
void orient_host(int o, int N, int p, int q, int& pp, int& qq) {
  const int a = (o & 1) ? q : p, b = (o & 1) ? p : q;
  pp = (o & 2) ? N - a : a;
  qq = (o & 4) ? N - b : b;
}

bool orient_inverse(int o, int oinv, int N) {
  for (int q = 0; q <= N; ++q)
    for (int p = 0; p <= N; ++p) {
      int p1, q1, p2, q2;
      orient_host(o, N, p, q, p1, q1);
      orient_host(oinv, N, p1, q1, p2, q2);
      if (p2 != p || q2 != q) return false;
    }
  return true;
}

template <typename real>
void fill_mortar_ops(MortarOps<real>& o, const std::vector<double>& x, const std::vector<double>& w, int n) {
  std::memset(&o, 0, sizeof(o));
  for (int a = 0; a < 2; ++a) {
    std::vector<double> eta(n);
    for (int i = 0; i < n; ++i) eta[i] = 0.5 * (x[i] + 2.0 * a - 1.0);
    const std::vector<double> V = host::interp_matrix(x, eta);  // V[i * n + m] = l_m(eta_i)
    for (int i = 0; i < n; ++i)
      for (int m = 0; m < n; ++m) {
        o.I[a][i * n + m] = (real)V[i * n + m];
        o.P[a][i * n + m] = (real)(V[m * n + i] * w[m] / w[i]);  // l_i(eta_m) w_m / w_i
      }
  }
}

flexi_status mesh_init_impl(flexi_ctx* c, const flexi_params* p, int K, const double* coords, const int32_t* conn,
                            int M, const int32_t* mortars, cudaStream_t st) {
  if (cudaGetDevice(&c->device) != cudaSuccess) return FLEXI_ECUDA;
  c->p = *p;
  c->K = K;
  c->N = p->N;
  c->n = p->N + 1;
  c->n2 = c->n * c->n;
  c->n3 = c->n2 * c->n;
  c->fp64 = p->precision == FLEXI_FP64;
  c->rs = c->fp64 ? sizeof(double) : sizeof(float);
  const int N = c->N, n = c->n, n3 = c->n3, n2 = c->n2;
  const int ng = p->Ngeo + 1, ng3 = ng * ng * ng;

  // ---- mortar rows: (big element, big side, type, (small element, side, o) x 4)
  int nMortarSides = 0;
  for (int m = 0; m < M; ++m) {
    const int32_t* r = mortars + 15 * m;
    const int eB = r[0], sB = r[1], typ = r[2];
    if (eB < 0 || eB >= K || sB < 0 || sB > 5 || typ < 1 || typ > 3) return FLEXI_EMESH;
    const int* cb = conn + (eB * 6 + sB) * 3;
    if (cb[0] != FLEXI_CONN_MORTAR || cb[1] != m || cb[2] != -1) return FLEXI_EMESH;
    ++nMortarSides;
    for (int pos = 0; pos < 4; ++pos) {
      const int e2 = r[3 + 3 * pos], s2 = r[4 + 3 * pos], o2 = r[5 + 3 * pos];
      if (typ < 3 && pos >= 2) {
        if (e2 != -1) return FLEXI_EMESH;
        continue;
      }
      if (e2 < 0 || e2 >= K || s2 < 0 || s2 > 5 || o2 < 0 || o2 > 7) return FLEXI_EMESH;
      const int* cs = conn + (e2 * 6 + s2) * 3;
      if (cs[0] != FLEXI_CONN_MORTAR || cs[1] != m || cs[2] != pos) return FLEXI_EMESH;
      ++nMortarSides;
    }
  }

  // ---- sides (Sec. 5.1): boundary sides first, then inner sides (master = smaller
  // (elem, side) key), then one side per small face of a mortar (master = the small
  // element), then the big sides of the mortars
  std::vector<int> es(K * 6, -1);
  std::vector<int> sideMaster;
  std::vector<int> bnd_pairs, inner_pairs;  // (e, s)
  int nMarked = 0;
  for (int e = 0; e < K; ++e)
    for (int s = 0; s < 6; ++s) {
      const int nb = conn[(e * 6 + s) * 3 + 0], ns = conn[(e * 6 + s) * 3 + 1], o = conn[(e * 6 + s) * 3 + 2];
      if (nb == FLEXI_CONN_MORTAR) {
        if (ns < 0 || ns >= M) return FLEXI_EMESH;
        ++nMarked;
        continue;
      }
      if (nb < 0) {
        bnd_pairs.push_back(e * 6 + s);
        continue;
      }
      if (nb >= K || ns < 0 || ns > 5 || o < 0 || o > 7) return FLEXI_EMESH;
      const int bnb = conn[(nb * 6 + ns) * 3 + 0], bns = conn[(nb * 6 + ns) * 3 + 1], bo = conn[(nb * 6 + ns) * 3 + 2];
      if (bnb != e || bns != s || !orient_inverse(o, bo, N)) return FLEXI_EMESH;
      if (e * 6 + s < nb * 6 + ns) inner_pairs.push_back(e * 6 + s);
    }
  if (nMarked != nMortarSides) return FLEXI_EMESH;
  const int nV = nMortarSides - M;
  c->nBC = (int)bnd_pairs.size();
  c->bcId.clear();
  for (int key : bnd_pairs) c->bcId.push_back(-1 - conn[key * 3]);
  c->bcKindHost.assign(c->nBC, FLEXI_BC_EXACT);
  c->nMortar = M;
  c->S = c->nBC + (int)inner_pairs.size() + nV + M;
  sideMaster.resize(2 * c->S);
  int sid = 0;
  for (int key : bnd_pairs) {
    const int e = key / 6, s = key % 6;
    es[key] = (sid << 4);
    sideMaster[2 * sid] = e;
    sideMaster[2 * sid + 1] = s;
    ++sid;
  }
  for (int key : inner_pairs) {
    const int e = key / 6, s = key % 6;
    const int nb = conn[key * 3 + 0], ns = conn[key * 3 + 1];
    es[key] = (sid << 4);
    es[nb * 6 + ns] = (sid << 4) | (1 << 3) | conn[(nb * 6 + ns) * 3 + 2];  // slave: its local -> master frame
    sideMaster[2 * sid] = e;
    sideMaster[2 * sid + 1] = s;
    ++sid;
  }
  const int vbase = sid, bigBase = sid + nV;
  std::vector<int> mvirt((size_t)std::max(nV, 1) * 4, 0), mbig((size_t)std::max(M, 1) * 8, -1);
  for (int m = 0; m < M; ++m) {
    const int32_t* r = mortars + 15 * m;
    const int typ = r[2];
    mbig[m * 8] = typ;
    for (int pos = 0; pos < (typ == 3 ? 4 : 2); ++pos) {
      const int e2 = r[3 + 3 * pos], s2 = r[4 + 3 * pos], o2 = r[5 + 3 * pos];
      int oinv = -1;
      for (int t = 0; t < 8 && oinv < 0; ++t)
        if (orient_inverse(o2, t, N)) oinv = t;
      const int a = typ == 3 ? (pos & 1) : (typ == 1 ? pos : 0);
      const int b = typ == 3 ? (pos >> 1) : (typ == 2 ? pos : 0);
      int* mv = &mvirt[(size_t)(sid - vbase) * 4];
      mv[0] = bigBase + m;
      mv[1] = typ | (a << 2) | (b << 3);
      mv[2] = o2;
      mv[3] = oinv;
      mbig[m * 8 + 1 + pos] = sid;
      if (es[e2 * 6 + s2] != -1) return FLEXI_EMESH;
      es[e2 * 6 + s2] = (sid << 4);
      sideMaster[2 * sid] = e2;
      sideMaster[2 * sid + 1] = s2;
      ++sid;
    }
  }
  for (int m = 0; m < M; ++m) {
    const int eB = mortars[15 * m], sB = mortars[15 * m + 1];
    if (es[eB * 6 + sB] != -1) return FLEXI_EMESH;
    es[eB * 6 + sB] = (sid << 4);
    sideMaster[2 * sid] = eB;
    sideMaster[2 * sid + 1] = sB;
    ++sid;
  }
  for (int v : es)
    if (v < 0) return FLEXI_EMESH;
  const int S = c->S;

  // ---- host operators
  std::vector<double> xs, ws, xl, wl, xg, wg;
  if (p->node_type == FLEXI_NODES_GAUSS) host::gauss(N, xs, ws); else host::lobatto(N, xs, ws);
  host::lobatto(N, xl, wl);
  host::lobatto(p->Ngeo, xg, wg);
  const std::vector<double> Ds = host::diff_matrix(xs), Dl = host::diff_matrix(xl);
  const std::vector<double> Vg2l = host::interp_matrix(xg, xl), Vl2s = host::interp_matrix(xl, xs),
                            Vg2s = host::interp_matrix(xg, xs);
  const std::vector<double> lmv = host::interp_matrix(xs, {-1.0}), lpv = host::interp_matrix(xs, {1.0});
  fill_ops<double>(c->ops64, Ds, ws, lmv, lpv, n);
  fill_ops<float>(c->ops32, Ds, ws, lmv, lpv, n);
  fill_mortar_ops<double>(c->mops64, xs, ws, n);
  fill_mortar_ops<float>(c->mops32, xs, ws, n);
  fill_phys<double>(c->ph64, *p);
  fill_phys<float>(c->ph32, *p);
  c->src.on = p->source;
  c->src.gamma = p->gamma;
  c->src.mu = p->mu;
  c->src.Pr = p->Pr;

  // ---- device buffers that live with the context
  flexi_status s;
#define AL(ptr, cnt) if ((s = dalloc(c, &(ptr), (cnt))) != FLEXI_OK) return s
  AL(c->Ja64, (size_t)K * 9 * n3);
  AL(c->sJ64, (size_t)K * n3);
  AL(c->wJ, (size_t)K * n3);
  AL(c->fgeo64, (size_t)S * 4 * n2);
  AL(c->xbc, (size_t)std::max(c->nBC, 1) * 3 * n2);
  AL(c->bcKind, (size_t)std::max(c->nBC, 1));  // zero: every boundary takes the exact state
  AL(c->elemSide, (size_t)K * 6);
  AL(c->status, 1);
  if (p->source) AL(c->xsol, (size_t)K * 3 * n3);

  // ---- temporary geometry buffers
  std::vector<void*> tmp;
  auto talloc = [&](double** ptr, size_t cnt) -> flexi_status {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(cnt, 1) * sizeof(double)) != cudaSuccess) return FLEXI_ENOMEM;
    tmp.push_back(q);
    *ptr = (double*)q;
    return FLEXI_OK;
  };
  auto free_tmp = [&]() { for (void* q : tmp) cudaFree(q); tmp.clear(); };
  struct Guard { decltype(free_tmp)& f; ~Guard() { f(); } } guard{free_tmp};
  double *X0, *X0r, *A1, *A2, *XL, *dXL[3], *v, *dA, *dB, *JaL, *X, *Xr, *dX[3], *dMat, *wdev;
  int* sideM;
#define TA(ptr, cnt) if ((s = talloc(&(ptr), (cnt))) != FLEXI_OK) return s
  TA(X0, (size_t)K * 3 * ng3);
  TA(X0r, (size_t)K * 3 * ng3);
  TA(A1, (size_t)K * 9 * n3);
  TA(A2, (size_t)K * 9 * n3);
  TA(XL, (size_t)K * 3 * n3);
  for (int l = 0; l < 3; ++l) TA(dXL[l], (size_t)K * 3 * n3);
  TA(v, (size_t)K * 9 * n3);
  TA(dA, (size_t)K * n3);
  TA(dB, (size_t)K * n3);
  TA(JaL, (size_t)K * 9 * n3);
  TA(X, (size_t)K * 3 * n3);
  TA(Xr, (size_t)K * 3 * n3);
  for (int l = 0; l < 3; ++l) TA(dX[l], (size_t)K * 3 * n3);
  TA(dMat, 6 * 64 + 16);
  TA(wdev, 16);
  {
    void* q = nullptr;
    if (cudaMalloc(&q, sizeof(int) * 2 * std::max(S, 1)) != cudaSuccess) return FLEXI_ENOMEM;
    tmp.push_back(q);
    sideM = (int*)q;
  }
  // coordinates: [K][kg][jg][ig][3] -> [K][3][kg][jg][ig], absolute (X0: node positions
  // for boundary states and source terms) and relative to the element's first geometry
  // node (X0r: metric terms and J, which do not change under a translation of the
  // mapping; differentiating absolute coordinates that are large compared with the
  // element's width would cancel digits in every sum)
  {
    std::vector<double> h((size_t)K * 3 * ng3), hr((size_t)K * 3 * ng3);
    for (int e = 0; e < K; ++e)
      for (int node = 0; node < ng3; ++node)
        for (int d = 0; d < 3; ++d) {
          const double x = coords[((size_t)e * ng3 + node) * 3 + d];
          h[((size_t)e * 3 + d) * ng3 + node] = x;
          hr[((size_t)e * 3 + d) * ng3 + node] = x - coords[(size_t)e * ng3 * 3 + d];
        }
    CK(cudaMemcpyAsync(X0, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(X0r, hr.data(), hr.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  // operator matrices on the device: Vg2l, Dl, Vl2s, Vg2s, Ds (each <= 64 entries)
  double* dVg2l = dMat;
  double* dDl = dMat + 64;
  double* dVl2s = dMat + 128;
  double* dVg2s = dMat + 192;
  double* dDs = dMat + 256;
  double* dlm = dMat + 320;
  double* dlp = dMat + 328;
  CK(cudaMemcpy(dVg2l, Vg2l.data(), Vg2l.size() * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dDl, Dl.data(), Dl.size() * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dVl2s, Vl2s.data(), Vl2s.size() * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dVg2s, Vg2s.data(), Vg2s.size() * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dDs, Ds.data(), Ds.size() * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dlm, lmv.data(), n * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dlp, lpv.data(), n * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(wdev, ws.data(), n * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(sideM, sideMaster.data(), sideMaster.size() * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->elemSide, es.data(), es.size() * sizeof(int), cudaMemcpyHostToDevice));

  // interpolate [B][m][m][m] -> [B][n][n][n] with matrix V (n x m)
  auto interp3 = [&](const double* in, double* out, const double* V, int B, int m) -> cudaError_t {
    cudaError_t e;
    if ((e = geom_apply1d(in, A1, V, B, m, m, m, 0, n, st)) != cudaSuccess) return e;
    if ((e = geom_apply1d(A1, A2, V, B, n, m, m, 1, n, st)) != cudaSuccess) return e;
    return geom_apply1d(A2, out, V, B, n, n, m, 2, n, st);
  };
  // curl-form metrics on the degree-N Lobatto points (face metrics of the two
  // elements of a side then agree), interpolated to the solution nodes
  CK(interp3(X0r, XL, dVg2l, 3 * K, ng));
  for (int l = 0; l < 3; ++l) CK(geom_apply1d(XL, dXL[l], dDl, 3 * K, n, n, n, l, n, st));
  CK(geom_metric_products(XL, dXL, v, K, n3, st));
  const size_t blk = (size_t)K * n3;
  for (int nn = 0; nn < 3; ++nn)
    for (int i = 0; i < 3; ++i) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
      CK(geom_apply1d(v + (nn * 3 + i2) * blk, dA, dDl, K, n, n, n, i1, n, st));
      CK(geom_apply1d(v + (nn * 3 + i1) * blk, dB, dDl, K, n, n, n, i2, n, st));
      CK(geom_curl(dA, dB, JaL, K, n3, i, nn, st));
    }
  CK(interp3(JaL, c->Ja64, dVl2s, 9 * K, n));
  // coordinates and Jacobian at the solution nodes
  CK(interp3(X0, X, dVg2s, 3 * K, ng));
  CK(interp3(X0r, Xr, dVg2s, 3 * K, ng));
  for (int l = 0; l < 3; ++l) CK(geom_apply1d(Xr, dX[l], dDs, 3 * K, n, n, n, l, n, st));
  CK(geom_jacobian(dX, c->sJ64, c->wJ, wdev, K, n, c->status, st));
  CK(geom_faces(c->Ja64, X, sideM, dlm, dlp, c->fgeo64, c->xbc, S, c->nBC, n, st));
  if (p->source) CK(cudaMemcpyAsync(c->xsol, X, (size_t)K * 3 * n3 * 8, cudaMemcpyDeviceToDevice, st));
  unsigned bad = 0;
  CK(cudaMemcpyAsync(&bad, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (bad) return FLEXI_EMESH;
  CK(cudaMemset(c->status, 0, sizeof(unsigned)));

  // ---- arithmetic-form copies and scratch
  c->m.K = K; c->m.S = S; c->m.nBC = c->nBC; c->m.N = N; c->m.n = n;
  CK(cudaDeviceGetAttribute(&c->m.nsm, cudaDevAttrMultiProcessorCount, c->device));
  c->m.Sface = S - M;
  c->m.vbase = vbase;
  c->m.nV = nV;
  c->m.nBig = M;
  if (M > 0) {
    int *dmv, *dmb;
    AL(dmv, mvirt.size());
    AL(dmb, mbig.size());
    CK(cudaMemcpy(dmv, mvirt.data(), mvirt.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dmb, mbig.data(), mbig.size() * sizeof(int), cudaMemcpyHostToDevice));
    c->m.mvirt = dmv;
    c->m.mbig = dmb;
    unsigned char* qb;
    AL(qb, (size_t)M * 15 * n2 * c->rs);
    c->m.QB = qb;
  }
  c->m.elemSide = c->elemSide;
  c->m.xbc = c->xbc;
  c->m.bcKind = c->bcKind;
  c->m.xsol = c->xsol;
  c->m.status = c->status;
  c->m.sweep_mode = p->precision == FLEXI_FP32_TF32 ? 1 : (p->precision == FLEXI_FP32_BF16 ? 2 : 0);
  c->m.lgl = p->node_type == FLEXI_NODES_LOBATTO ? 1 : 0;
  c->m.split = p->split_form;
  c->m.br2 = p->lifting == FLEXI_LIFTING_BR2 ? 1 : 0;
  const size_t rs = c->rs;
  if (c->fp64) {
    c->m.Ja = c->Ja64; c->m.sJ = c->sJ64; c->m.fgeo = c->fgeo64;
  } else {
    AL(c->Ja32, (size_t)K * 9 * n3);
    AL(c->sJ32, (size_t)K * n3);
    AL(c->fgeo32, (size_t)S * 4 * n2);
    CK(convert_f64_to_f32(c->Ja64, c->Ja32, (size_t)K * 9 * n3, st));
    CK(convert_f64_to_f32(c->sJ64, c->sJ32, (size_t)K * n3, st));
    CK(convert_f64_to_f32(c->fgeo64, c->fgeo32, (size_t)S * 4 * n2, st));
    c->m.Ja = c->Ja32; c->m.sJ = c->sJ32; c->m.fgeo = c->fgeo32;
  }
  unsigned char *Wf, *Gf, *Ff, *Utv, *Us, *dUs, *Gvol, *adj;
  if (p->adjoint) {  // volume gradients of the forward recompute and the reverse sweep's face data
    AL(Gvol, (size_t)K * 15 * n3 * rs);
    c->m.Gvol = Gvol;
    AL(adj, adjoint_scratch_bytes(c->m, rs));
    c->adj_scratch = adj;
  }
  AL(Wf, 2 * (size_t)S * NV * n2 * rs);
  AL(Gf, 2 * (size_t)S * 15 * n2 * rs);
  AL(Ff, (size_t)S * NV * n2 * rs);
  AL(Utv, (size_t)K * NV * n3 * rs);
  AL(Us, (size_t)K * NV * n3 * rs);
  AL(dUs, (size_t)K * NV * n3 * rs);
  c->m.Wf = Wf; c->m.Gf = Gf; c->m.Ff = Ff; c->m.Utv = Utv;
  c->fused = c->fp64 && !c->m.br2 && c->nMortar == 0 && n == 4 && K < c->m.nsm;
  if (c->fused) {
    unsigned char *WfA, *WfB;
    AL(WfA, 2 * (size_t)S * NV * n2 * rs);
    AL(WfB, 2 * (size_t)S * NV * n2 * rs);
    c->WfA = WfA;
    c->WfB = WfB;
  }
  c->Ustate = Us; c->dUstate = dUs;
  c->red_blocks = std::max(1, std::min(4 * 152, (int)(((size_t)K * n3 + 255) / 256)));
  AL(c->partial, (size_t)c->red_blocks * kReduceQuantities);
  if (cudaMallocHost(&c->partial_host, sizeof(double) * c->red_blocks * kReduceQuantities) != cudaSuccess)
    return FLEXI_ENOMEM;
  CK(cudaStreamSynchronize(st));
#undef AL
#undef TA
  return FLEXI_OK;
}

template <typename real>
flexi_status do_rhs_adjoint(flexi_ctx* c, const real* U, const real* lam, real* out, real scale, int accumulate,
                            double t, cudaStream_t st) {
  Prof pr(c, KC_ADJ, st);
  CK(launch_rhs_adjoint<real>(c->m, U, lam, out, scale, accumulate, ops_of<real>(c), mo_of<real>(c), ph_of<real>(c),
                              c->adj_scratch, t, st));
  return FLEXI_OK;
}

// reverse of one LSERK4(5) step (Williamson 2N form):
//   for k = 5..1: lam_dU += B_k lamU; lamU += dt (dL/dU(U_{k-1}, t + c_k dt))^T lam_dU; lam_dU = A_k lam_dU
template <typename real>
flexi_status do_adjoint_step(flexi_ctx* c, const real* stages, real* lamU, real* lam_dU, double t, double dt,
                             cudaStream_t st) {
  const size_t nU = (size_t)c->K * NV * c->n3;
  for (int k = 4; k >= 0; --k) {
    {
      Prof pr(c, KC_OTHER, st);
      CK(launch_axpby<real>(lam_dU, lamU, real(1), (real)RK_B[k], nU, st));
    }
    flexi_status s = do_rhs_adjoint<real>(c, stages + k * nU, lam_dU, lamU, (real)dt, 1, t + RK_C[k] * dt, st);
    if (s != FLEXI_OK) return s;
    Prof pr(c, KC_OTHER, st);
    CK(launch_axpby<real>(lam_dU, nullptr, (real)RK_A[k], real(0), nU, st));
  }
  return FLEXI_OK;
}

template <typename real>
flexi_status do_reduce(flexi_ctx* c, const void* U, const void* Ut, double cfl, double* out, cudaStream_t st) {
  const double kv = std::max(4.0 / 3.0, c->p.gamma / c->p.Pr) * c->p.mu;
  {
    Prof pr(c, KC_RED, st);
    CK(launch_reduce<real>((const real*)U, (const real*)Ut, c->wJ, c->Ja64, c->sJ64, (long long)c->K * c->n3, c->n3,
                           ph_of<real>(c), kv, c->partial, c->red_blocks, st));
  }
  CK(cudaMemcpyAsync(c->partial_host, c->partial, sizeof(double) * c->red_blocks * kReduceQuantities,
                     cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  double acc[kReduceQuantities] = {0};
  for (int b = 0; b < c->red_blocks; ++b)
    for (int q = 0; q < kReduceQuantities; ++q) {
      const double val = c->partial_host[b * kReduceQuantities + q];
      if (q < 7) acc[q] += val; else acc[q] = std::max(acc[q], val);
    }
  for (int q = 0; q < 7; ++q) out[q] = acc[q];
  const int N = c->N;
  const double dtc = cfl * 2.0 / ((2.0 * N + 1.0) * acc[7]);
  const double dtv = acc[8] > 0 ? cfl * 4.0 / ((2.0 * N + 1.0) * acc[8]) : INFINITY;
  out[7] = std::min(dtc, dtv);
  return FLEXI_OK;
}

}  // namespace

namespace flexi {
bool ctx_reduce_inputs(const flexi_ctx* c, ReduceInputs* r) {
  if (c == nullptr || r == nullptr) return false;
  r->K = c->K;
  r->N = c->N;
  r->device = c->device;
  r->n3 = c->n3;
  r->fp64 = c->fp64 ? 1 : 0;
  r->wJ = c->wJ;
  r->Ja64 = c->Ja64;
  r->sJ64 = c->sJ64;
  r->status = c->status;
  r->kv_coef = std::max(4.0 / 3.0, c->p.gamma / c->p.Pr) * c->p.mu;
  r->ph64 = c->ph64;
  r->ph32 = c->ph32;
  return true;
}

size_t adjoint_scratch_bytes(const DevMesh& m, size_t rs) {
  const size_t n2 = (size_t)m.n * m.n, n3 = n2 * m.n;
  return rs * (4 * 2 * (size_t)m.S * NV * n2 + 2 * (size_t)m.S * 15 * n2 + (size_t)m.K * NV * n3 +
               (size_t)m.nBig * 15 * n2);
}
}  // namespace flexi

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

const char* flexi_strerror(flexi_status s) {
  switch (s) {
    case FLEXI_OK: return "ok";
    case FLEXI_EINVAL: return "invalid argument";
    case FLEXI_ENOMEM: return "out of memory";
    case FLEXI_ECUDA: return "CUDA runtime error";
    case FLEXI_EMESH: return "invalid mesh (connectivity or non-positive Jacobian)";
    case FLEXI_ENONPHYSICAL: return "non-physical state (rho <= 0 or p <= 0) detected";
    case FLEXI_EUNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

void flexi_destroy(flexi_ctx* c) {
  if (c == nullptr) return;
  cudaDeviceSynchronize();
  for (auto& r : c->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (void* p : c->allocs) cudaFree(p);
  if (c->partial_host) cudaFreeHost(c->partial_host);
  delete c;
  (void)cudaGetLastError();  // leave no error of this cleanup behind for the caller's next call
}

flexi_status flexi_mesh_init(flexi_ctx** out, const flexi_params* p, int K, const double* coords,
                             const int32_t* conn, void* stream) {
  return flexi_mesh_init_mortar(out, p, K, coords, conn, 0, nullptr, stream);
}

flexi_status flexi_mesh_init_mortar(flexi_ctx** out, const flexi_params* p, int K, const double* coords,
                                    const int32_t* conn, int M, const int32_t* mortars, void* stream) {
  if (out == nullptr || p == nullptr || coords == nullptr || conn == nullptr || K <= 0) return FLEXI_EINVAL;
  if (M < 0 || (M > 0 && mortars == nullptr)) return FLEXI_EINVAL;
  *out = nullptr;
  if (p->N < 1 || p->N > 7) return p->N > 7 ? FLEXI_EUNSUPPORTED : FLEXI_EINVAL;
  if (p->Ngeo < 1 || p->Ngeo > p->N) return FLEXI_EINVAL;
  if (p->node_type != FLEXI_NODES_GAUSS && p->node_type != FLEXI_NODES_LOBATTO) return FLEXI_EINVAL;
  if (p->riemann < 0 || p->riemann > 4 || p->bc_exact < 0 || p->bc_exact > 2) return FLEXI_EINVAL;
  if (p->precision < FLEXI_FP64 || p->precision > FLEXI_FP32_BF16) return FLEXI_EINVAL;
  if (p->split_form < FLEXI_SPLIT_STANDARD || p->split_form > FLEXI_SPLIT_EC) return FLEXI_EINVAL;
  if (p->adjoint != 0 && p->adjoint != 1) return FLEXI_EINVAL;
  if (p->lifting != FLEXI_LIFTING_BR1 && p->lifting != FLEXI_LIFTING_BR2) return FLEXI_EINVAL;
  if (p->lifting == FLEXI_LIFTING_BR2 && !(p->eta_br2 >= 0.0)) return FLEXI_EINVAL;
  if (p->lifting == FLEXI_LIFTING_BR2 &&
      (p->split_form != FLEXI_SPLIT_STANDARD || (p->precision != FLEXI_FP64 && p->precision != FLEXI_FP32)))
    return FLEXI_EUNSUPPORTED;
  if (p->split_form != FLEXI_SPLIT_STANDARD &&
      (p->node_type != FLEXI_NODES_LOBATTO || (p->precision != FLEXI_FP64 && p->precision != FLEXI_FP32)))
    return FLEXI_EUNSUPPORTED;
  if (!(p->gamma > 1.0) || !(p->Pr > 0.0) || !(p->mu >= 0.0)) return FLEXI_EINVAL;
  if ((long long)K * 6 >= (1LL << 27)) return FLEXI_EUNSUPPORTED;
  flexi_ctx* c = new (std::nothrow) flexi_ctx();
  if (c == nullptr) return FLEXI_ENOMEM;
  const flexi_status s = mesh_init_impl(c, p, K, coords, conn, M, mortars, (cudaStream_t)stream);
  if (s != FLEXI_OK) {
    flexi_destroy(c);
    return s;
  }
  *out = c;
  return FLEXI_OK;
}

flexi_status flexi_set_bc(flexi_ctx* c, int bc_id, int kind) {
  if (c == nullptr || kind < FLEXI_BC_EXACT || kind > FLEXI_BC_SLIP_WALL) return FLEXI_EINVAL;
  if (!on_ctx_device(c)) return FLEXI_EINVAL;
  bool found = false;
  for (int b = 0; b < c->nBC; ++b)
    if (c->bcId[b] == bc_id) {
      c->bcKindHost[b] = kind;
      found = true;
    }
  if (!found) return FLEXI_EINVAL;
  CK(cudaMemcpy(c->bcKind, c->bcKindHost.data(), sizeof(int) * c->nBC, cudaMemcpyHostToDevice));
  return FLEXI_OK;
}

flexi_status flexi_rhs(flexi_ctx* c, const void* U, void* Ut, double t, void* stream) {
  if (c == nullptr || U == nullptr || Ut == nullptr) return FLEXI_EINVAL;
  if (!on_ctx_device(c)) return FLEXI_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  return c->fp64 ? do_rhs<double>(c, (const double*)U, (double*)Ut, t, st)
                 : do_rhs<float>(c, (const float*)U, (float*)Ut, t, st);
}

flexi_status flexi_rk_step(flexi_ctx* c, void* U, void* dU, double t, double dt, void* stream) {
  if (c == nullptr || U == nullptr || dU == nullptr) return FLEXI_EINVAL;
  if (!on_ctx_device(c)) return FLEXI_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  return c->fp64 ? do_rk_step<double>(c, (double*)U, (double*)dU, t, dt, nullptr, st)
                 : do_rk_step<float>(c, (float*)U, (float*)dU, t, dt, nullptr, st);
}

flexi_status flexi_rk_step_stages(flexi_ctx* c, void* U, void* dU, double t, double dt, void* U_stages,
                                  void* stream) {
  if (c == nullptr || U == nullptr || dU == nullptr || U_stages == nullptr) return FLEXI_EINVAL;
  if (!on_ctx_device(c)) return FLEXI_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  return c->fp64 ? do_rk_step<double>(c, (double*)U, (double*)dU, t, dt, (double*)U_stages, st)
                 : do_rk_step<float>(c, (float*)U, (float*)dU, t, dt, (float*)U_stages, st);
}

// every form, flux, lifting, boundary kind and mortar mesh; the FP64 and FP32
// forms (the tensor-core sweeps have no reverse)
static bool adjoint_supported(const flexi_ctx* c) {
  return c->p.adjoint != 0 && (c->p.precision == FLEXI_FP64 || c->p.precision == FLEXI_FP32);
}

flexi_status flexi_adjoint_step(flexi_ctx* c, const void* U_stages, void* lamU, void* lam_dU, double t, double dt,
                                void* stream) {
  if (c == nullptr || U_stages == nullptr || lamU == nullptr || lam_dU == nullptr) return FLEXI_EINVAL;
  if (!on_ctx_device(c)) return FLEXI_EINVAL;
  if (!adjoint_supported(c)) return FLEXI_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  return c->fp64 ? do_adjoint_step<double>(c, (const double*)U_stages, (double*)lamU, (double*)lam_dU, t, dt, st)
                 : do_adjoint_step<float>(c, (const float*)U_stages, (float*)lamU, (float*)lam_dU, t, dt, st);
}

flexi_status flexi_rhs_adjoint(flexi_ctx* c, const void* U, const void* lam, void* out, double t, void* stream) {
  if (c == nullptr || U == nullptr || lam == nullptr || out == nullptr) return FLEXI_EINVAL;
  if (!on_ctx_device(c)) return FLEXI_EINVAL;
  if (!adjoint_supported(c)) return FLEXI_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  return c->fp64 ? do_rhs_adjoint<double>(c, (const double*)U, (const double*)lam, (double*)out, 1.0, 0, t, st)
                 : do_rhs_adjoint<float>(c, (const float*)U, (const float*)lam, (float*)out, 1.0f, 0, t, st);
}

// true when one RK step does not depend on t: no source term and no exact-state
// boundary with a time-dependent state
static bool autonomous(const flexi_ctx* c) {
  if (c->p.source) return false;
  if (c->p.bc_exact != FLEXI_EXACT_MANUFACTURED) return true;
  for (int k : c->bcKindHost)
    if (k == FLEXI_BC_EXACT) return false;
  return true;
}

// one RK step of either precision (see do_rk_step for faces_ready and prolong_last)
static flexi_status rk_step_any(flexi_ctx* c, void* U, void* dU, double t, double dt, cudaStream_t st,
                                bool faces_ready, bool prolong_last) {
  return c->fp64 ? do_rk_step<double>(c, (double*)U, (double*)dU, t, dt, nullptr, st, faces_ready, prolong_last)
                 : do_rk_step<float>(c, (float*)U, (float*)dU, t, dt, nullptr, st, faces_ready, prolong_last);
}

// face states of U (the prolongation that opens a step)
static flexi_status prolong_any(flexi_ctx* c, const void* U, cudaStream_t st) {
  Prof pr(c, KC_PROLONG, st);
  if (c->fp64) {
    CK(launch_prolong<double>(c->m, (const double*)U, ops_of<double>(c), ph_of<double>(c), st));
  } else {
    CK(launch_prolong<float>(c->m, (const float*)U, ops_of<float>(c), ph_of<float>(c), st));
  }
  return FLEXI_OK;
}

flexi_status flexi_rk_run(flexi_ctx* c, void* U, void* dU, int nsteps, double t0, double dt, void* stream) {
  if (c == nullptr || U == nullptr || dU == nullptr || nsteps < 0) return FLEXI_EINVAL;
  if (!on_ctx_device(c)) return FLEXI_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (nsteps == 0) return FLEXI_OK;
  // consecutive steps hand over their face states: the last stage of a step writes those
  // of the next step's U, so only the call's first step prolongs U itself
  const bool use_graph = st != nullptr && !c->prof && autonomous(c) && nsteps > 1;
  if (!use_graph) {
    for (int s = 0; s < nsteps; ++s) {
      const flexi_status r = rk_step_any(c, U, dU, t0 + s * dt, dt, st, s > 0, s + 1 < nsteps);
      if (r != FLEXI_OK) return r;
    }
    return FLEXI_OK;
  }
  int s = 0;
  if (c->graph == nullptr || c->gU != U || c->gdU != dU || c->gdt != dt || c->gst != st) {
    // one eager step (also performs every one-time kernel attribute setting outside a capture)
    {
      const flexi_status r = rk_step_any(c, U, dU, t0, dt, st, false, true);
      if (r != FLEXI_OK) return r;
      s = 1;
    }
    if (c->graph) {
      cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    // the captured step takes its face states from the step before it and leaves the next one's
    const flexi_status r = rk_step_any(c, U, dU, t0, dt, st, true, true);
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    if (r != FLEXI_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      (void)cudaGetLastError();
      return r != FLEXI_OK ? r : FLEXI_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      c->graph = nullptr;
      return FLEXI_ECUDA;
    }
    c->gU = U;
    c->gdU = dU;
    c->gdt = dt;
    c->gst = st;
  } else {
    const flexi_status r = prolong_any(c, U, st);  // the face states of the caller's U
    if (r != FLEXI_OK) return r;
  }
  for (; s < nsteps; ++s) CK(cudaGraphLaunch(c->graph, st));
  return FLEXI_OK;
}

flexi_status flexi_rk_run_host(flexi_ctx* c, void* U_host, int nsteps, double t0, double dt, void* stream) {
  if (c == nullptr || U_host == nullptr || nsteps < 0) return FLEXI_EINVAL;
  if (!on_ctx_device(c)) return FLEXI_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)c->K * NV * c->n3 * c->rs;
  CK(cudaMemcpyAsync(c->Ustate, U_host, bytes, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(c->dUstate, 0, bytes, st));
  for (int s = 0; s < nsteps; ++s) {
    const flexi_status r = rk_step_any(c, c->Ustate, c->dUstate, t0 + s * dt, dt, st, s > 0, s + 1 < nsteps);
    if (r != FLEXI_OK) return r;
  }
  CK(cudaMemcpyAsync(U_host, c->Ustate, bytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return FLEXI_OK;
}

flexi_status flexi_reduce(flexi_ctx* c, const void* U, const void* Ut, double cfl, double* out, void* stream) {
  if (c == nullptr || U == nullptr || out == nullptr) return FLEXI_EINVAL;
  if (!on_ctx_device(c)) return FLEXI_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const flexi_status s = c->fp64 ? do_reduce<double>(c, U, Ut, cfl, out, st) : do_reduce<float>(c, U, Ut, cfl, out, st);
  if (s != FLEXI_OK) return s;
  unsigned flag = 0;
  CK(cudaMemcpy(&flag, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (flag) {
    CK(cudaMemset(c->status, 0, sizeof(unsigned)));
    return FLEXI_ENONPHYSICAL;
  }
  return FLEXI_OK;
}

flexi_status flexi_query(flexi_ctx* c, int what, int64_t* val) {
  if (c == nullptr || val == nullptr) return FLEXI_EINVAL;
  const double n = c->n, f = 3.0 / n;  // unique face nodes per volume node
  const double dof = (double)c->K * c->n3;
  switch (what) {
    case FLEXI_Q_K: *val = c->K; return FLEXI_OK;
    case FLEXI_Q_N: *val = c->N; return FLEXI_OK;
    case FLEXI_Q_NSIDES: *val = c->S; return FLEXI_OK;
    case FLEXI_Q_NBCSIDES: *val = c->nBC; return FLEXI_OK;
    case FLEXI_Q_DOF: *val = (int64_t)dof; return FLEXI_OK;
    case FLEXI_Q_BYTES_PER_STAGE: {
      // minimum-traffic three-kernel schedule, words per DOF: 46 + 117 f
      *val = (int64_t)((46.0 + 117.0 * f) * dof * c->rs);
      return FLEXI_OK;
    }
    case FLEXI_Q_FLOPS_PER_STAGE: {
      // per DOF, FMA = 2: D_hat sweeps 2 (45 + 15) n; Gauss nodes: prolongation of U (5)
      // and of the gradients (15) to 6 faces and the two surface integrals, each 2 * 6 * 20
      // (Gauss-Lobatto: surface terms at face nodes only); contravariant transforms 2 * 90;
      // pointwise fluxes ~100; face fluxes ~300 per face node (f per DOF); RK update 4
      const bool lg = c->p.node_type == FLEXI_NODES_GAUSS;
      const double sweeps = 2.0 * 60.0 * n;
      const double surf = lg ? 2.0 * (6 * 5 + 6 * 15 + 6 * 5 + 6 * 15) : 2.0 * (6 * 5 + 6 * 15) * (1.0 / n) * 2;
      const double transform = 2.0 * 90.0;
      *val = (int64_t)((sweeps + surf + transform + 100.0 + 300.0 * f + 4.0) * dof);
      return FLEXI_OK;
    }
    case FLEXI_Q_STATUS: {
      if (!on_ctx_device(c)) return FLEXI_EINVAL;
      unsigned flag = 0;
      CK(cudaMemcpy(&flag, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
      CK(cudaMemset(c->status, 0, sizeof(unsigned)));
      *val = flag;
      return FLEXI_OK;
    }
    case FLEXI_Q_DEVICE_BYTES: *val = (int64_t)c->dev_bytes; return FLEXI_OK;
    case FLEXI_Q_PRECISION: *val = c->p.precision; return FLEXI_OK;
  }
  return FLEXI_EINVAL;
}

flexi_status flexi_profile(flexi_ctx* c, int enable) {
  if (c == nullptr) return FLEXI_EINVAL;
  c->prof = enable != 0;
  return FLEXI_OK;
}

flexi_status flexi_kernel_times(flexi_ctx* c, double* ms, int64_t* count, int reset) {
  if (c == nullptr) return FLEXI_EINVAL;
  drain_profile(c);
  for (int k = 0; k < 8; ++k) {
    if (ms) ms[k] = c->ms[k];
    if (count) count[k] = c->cnt[k];
    if (reset) {
      c->ms[k] = 0;
      c->cnt[k] = 0;
    }
  }
  return FLEXI_OK;
}

}  // extern "C"

// Internal launcher interface between the C-ABI layer and the kernel
// translation units (one per arithmetic type, compiled in parallel).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "dg_common.cuh"

namespace flexi {

// Raises a kernel's dynamic shared-memory limit to smem bytes once per device
// (the attribute is per device; done holds one bit per device ordinal < 64, and
// larger ordinals set it on every call).  Safe to call from several host threads.
template <typename Kernel>
cudaError_t ensure_dynamic_smem(Kernel* kernel, size_t smem, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (bit != 0 && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err == cudaSuccess && bit != 0) done.fetch_or(bit, std::memory_order_release);
  return err;
}

// Device-resident mesh, geometry and scratch of one context (type-erased).
struct DevMesh {
  int K = 0, S = 0, nBC = 0, N = 0, n = 0;
  int nsm = 1;                 // streaming multiprocessors of the device (launch shapes of small meshes)
  int sweep_mode = 0;          // 0 CUDA-core line sweeps, 1 TF32 and 2 BF16 3-term split mma
  int lgl = 0;                 // 1: Gauss-Lobatto nodes (face terms only at face nodes)
  int split = 0;               // split-form volume integral: 1 kinetic-energy-preserving, 2 entropy-conservative flux
  int br2 = 0;                 // 1: BR2 face gradients for the viscous numerical flux
  const void* Ja = nullptr;    // [K][9][n^3]   Ja^l_d at index l*3+d
  const void* sJ = nullptr;    // [K][n^3]      1/J
  const void* fgeo = nullptr;  // [S][4][n^2]   n_hat (3), s_hat
  const int* elemSide = nullptr;  // [K][6] packed (side<<4 | slave<<3 | orient)
  const double* xbc = nullptr;    // [nBC][3][n^2] face node coordinates of boundary sides
  const int* bcKind = nullptr;    // [nBC] 0 exact state, 1 outflow, 2 slip wall
  const double* xsol = nullptr;   // [K][3][n^3] (only with a source term)
  void* Wf = nullptr;          // [2][S][5][n^2] primitive face states (slot 0 master, 1 slave/boundary)
  void* Gf = nullptr;          // [2][S][15][n^2] lifted gradients on the faces (index d*5+v)
  void* Ff = nullptr;          // [S][5][n^2] numerical flux f* s_hat in the master normal
  void* Utv = nullptr;         // [K][5][n^3] volume-integral part of U_t
  void* Gvol = nullptr;        // [K][15][n^3] volume gradients (adjoint only)
  // mortars: sides are [boundary][inner][virtual small sides][big sides]
  int Sface = 0;               // sides with a numerical flux (all but the big sides)
  int vbase = 0, nV = 0;       // first virtual side and their count
  int nBig = 0;                // big sides, ids Sface .. S-1
  const int* mvirt = nullptr;  // [nV] int4 (big side, type | a<<2 | b<<3, o, oinv)
  const int* mbig = nullptr;   // [nBig][8] (type, virtual side of position 0..3 or -1)
  void* QB = nullptr;          // [nBig][15][n^2] BR1 lifting flux of the big element
  unsigned* status = nullptr;  // device status word (bit 0: non-physical face state)
};

struct SourceParams {
  int on = 0;
  double gamma = 1.4, mu = 0, Pr = 0.72;
};

template <typename real>
struct RkStage {
  real A, B, dt;
  int prolong;  // write face states of the updated U (next stage)
};

template <typename real>
cudaError_t launch_prolong(const DevMesh& m, const real* U, const Ops<real>& ops, const Phys<real>& ph,
                           cudaStream_t st);
template <typename real>
cudaError_t launch_bc(const DevMesh& m, double t, const Phys<real>& ph, cudaStream_t st);
template <typename real>
cudaError_t launch_lift_vol(const DevMesh& m, const real* U, const Ops<real>& ops, const Phys<real>& ph,
                            int store_grad, cudaStream_t st);
template <typename real>
cudaError_t launch_face(const DevMesh& m, const Phys<real>& ph, cudaStream_t st);
// mortars: face states + lifting flux of big sides; gradients; projected fluxes
template <typename real>
cudaError_t launch_mortar_state(const DevMesh& m, const MortarOps<real>& mo, const Phys<real>& ph, cudaStream_t st);
template <typename real>
cudaError_t launch_mortar_grad(const DevMesh& m, const MortarOps<real>& mo, const Phys<real>& ph, cudaStream_t st);
template <typename real>
cudaError_t launch_mortar_flux(const DevMesh& m, const MortarOps<real>& mo, cudaStream_t st);
// mode 0: Ut = L(U); mode 1: RK stage update of U, dU in place
template <typename real>
cudaError_t launch_surf(const DevMesh& m, int mode, real* U, real* dU, real* Ut, const RkStage<real>& rk,
                        double t, const SourceParams& src, const Ops<real>& ops, const Phys<real>& ph,
                        cudaStream_t st);

// a5 and a8-a10 of an RK stage in one kernel (FP64, n = 4, no mortars, BR1; meant for
// meshes with fewer elements than SMs): face states read from WfIn, those of the new U
// written to WfOut when rk.prolong (WfOut != WfIn: other elements still read WfIn)
cudaError_t launch_surf_face(const DevMesh& m, const void* WfIn, void* WfOut, double* U, double* dU,
                             const RkStage<double>& rk, double t, const SourceParams& src, const Ops<double>& ops,
                             const Phys<double>& ph, cudaStream_t st);
// adjoint of the right-hand side: out = (dL/dU)^T lam  (uses Gvol written by
// launch_lift_vol with store_grad = 1); mode 1 accumulates out += scale * result
template <typename real>
cudaError_t launch_rhs_adjoint(const DevMesh& m, const real* U, const real* lam, real* out, real scale,
                               int accumulate, const Ops<real>& ops, const MortarOps<real>& mo,
                               const Phys<real>& ph, void* scratch, double t, cudaStream_t st);
size_t adjoint_scratch_bytes(const DevMesh& m, size_t real_size);
template <typename real>
cudaError_t launch_axpby(real* y, const real* x, real a, real b, size_t count, cudaStream_t st);

// reductions (always FP64 accumulation)
template <typename real>
cudaError_t launch_reduce(const real* U, const real* Ut, const double* wJ, const double* Ja64, const double* sJ64,
                          long long nodes, int n3, const Phys<real>& ph, double kv_coef, double* partial,
                          int nblocks, cudaStream_t st);
constexpr int kReduceQuantities = 9;
}  // namespace flexi
struct flexi_ctx;
namespace flexi {

// read-only view of a context's inputs to the global reductions
struct ReduceInputs {
  int K = 0, N = 0, n3 = 0, fp64 = 1;
  int device = -1;  // the context's CUDA device
  const double *wJ = nullptr, *Ja64 = nullptr, *sJ64 = nullptr;
  const unsigned* status = nullptr;
  double kv_coef = 0;  // max(4/3, gamma/Pr) mu
  Phys<double> ph64{};
  Phys<float> ph32{};
};

bool ctx_reduce_inputs(const flexi_ctx* c, ReduceInputs* r);

// geometry (FP64)
cudaError_t geom_apply1d(const double* in, double* out, const double* M, int B, int ni, int nj, int nk, int l,
                         int nout, cudaStream_t st);
cudaError_t geom_metric_products(const double* XL, const double* const dXL[3], double* v, int K, int n3,
                                 cudaStream_t st);
cudaError_t geom_curl(const double* dA, const double* dB, double* Ja, int K, int n3, int i, int nn,
                      cudaStream_t st);
cudaError_t geom_jacobian(const double* const dX[3], double* sJ, double* wJ, const double* w, int K, int n,
                          unsigned* bad, cudaStream_t st);
cudaError_t geom_faces(const double* Ja, const double* X, const int* sideMaster, const double* lm,
                       const double* lp, double* fgeo, double* xbc, int S, int nBC, int n, cudaStream_t st);
cudaError_t convert_f64_to_f32(const double* in, float* out, size_t count, cudaStream_t st);

}  // namespace flexi

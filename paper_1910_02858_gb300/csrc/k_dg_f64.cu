// Instantiation of the DGSEM kernels for double arithmetic.
#include "k_dg.cuh"
#include "k_mortar.cuh"
#include "k_reduce.cuh"

namespace flexi {
template cudaError_t launch_prolong<double>(const DevMesh&, const double*, const Ops<double>&, const Phys<double>&,
                                          cudaStream_t);
template cudaError_t launch_bc<double>(const DevMesh&, double, const Phys<double>&, cudaStream_t);
template cudaError_t launch_lift_vol<double>(const DevMesh&, const double*, const Ops<double>&, const Phys<double>&, int,
                                           cudaStream_t);
template cudaError_t launch_face<double>(const DevMesh&, const Phys<double>&, cudaStream_t);
template cudaError_t launch_mortar_state<double>(const DevMesh&, const MortarOps<double>&, const Phys<double>&, cudaStream_t);
template cudaError_t launch_mortar_grad<double>(const DevMesh&, const MortarOps<double>&, const Phys<double>&, cudaStream_t);
template cudaError_t launch_mortar_flux<double>(const DevMesh&, const MortarOps<double>&, cudaStream_t);
template cudaError_t launch_surf<double>(const DevMesh&, int, double*, double*, double*, const RkStage<double>&, double,
                                       const SourceParams&, const Ops<double>&, const Phys<double>&, cudaStream_t);
template cudaError_t launch_reduce<double>(const double*, const double*, const double*, const double*, const double*,
                                         long long, int, const Phys<double>&, double, double*, int, cudaStream_t);

cudaError_t launch_surf_face(const DevMesh& m, const void* WfIn, void* WfOut, double* U, double* dU,
                                    const RkStage<double>& rk, double t, const SourceParams& src,
                                    const Ops<double>& ops, const Phys<double>& ph, cudaStream_t st) {
  if (m.n != 4) return cudaErrorInvalidValue;
  if (m.lgl && 2 * m.K <= m.nsm) {  // two CTAs per element
#define FLEXI_SF2(RSV)                                                                                          \
  k_surf_face2<RSV><<<2 * m.K, 384, 0, st>>>(                                                 \
      (const double*)WfIn, (const double*)m.Gf, (const double*)m.fgeo, m.elemSide, (const double*)m.sJ,         \
      (const double*)m.Utv, U, dU, (double*)WfOut, m.xsol, rk, t, src, m.K, m.S, m.nBC, ops, ph, m.status)
    switch (ph.riemann) {
      case 1: FLEXI_SF2(1); break;
      case 3: FLEXI_SF2(3); break;
      case 4: FLEXI_SF2(4); break;
      default: FLEXI_SF2(0); break;
    }
#undef FLEXI_SF2
    return cudaGetLastError();
  }
#define FLEXI_SF(RSV, LG)                                                                                        \
  k_surf_face<RSV, LG><<<m.K, 384, 0, st>>>((const double*)WfIn, (const double*)m.Gf, (const double*)m.fgeo,    \
                                            m.elemSide, (const double*)m.sJ, (const double*)m.Utv, U, dU,       \
                                            (double*)WfOut, m.xsol, rk, t, src, m.K, m.S, m.nBC, ops, ph, m.status)
#define FLEXI_SF_RS(LG)                 \
  switch (ph.riemann) {                 \
    case 1: FLEXI_SF(1, LG); break;     \
    case 3: FLEXI_SF(3, LG); break;     \
    case 4: FLEXI_SF(4, LG); break;     \
    default: FLEXI_SF(0, LG); break;    \
  }
  if (m.lgl) {
    FLEXI_SF_RS(true)
  } else {
    FLEXI_SF_RS(false)
  }
#undef FLEXI_SF_RS
#undef FLEXI_SF
  return cudaGetLastError();
}
}  // namespace flexi

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
}  // namespace flexi

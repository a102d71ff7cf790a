// Instantiation of the DGSEM kernels for float arithmetic.
#include "k_dg.cuh"
#include "k_mortar.cuh"
#include "k_reduce.cuh"

namespace flexi {
template cudaError_t launch_prolong<float>(const DevMesh&, const float*, const Ops<float>&, const Phys<float>&,
                                          cudaStream_t);
template cudaError_t launch_bc<float>(const DevMesh&, double, const Phys<float>&, cudaStream_t);
template cudaError_t launch_lift_vol<float>(const DevMesh&, const float*, const Ops<float>&, const Phys<float>&, int,
                                           cudaStream_t);
template cudaError_t launch_face<float>(const DevMesh&, const Phys<float>&, cudaStream_t);
template cudaError_t launch_mortar_state<float>(const DevMesh&, const MortarOps<float>&, const Phys<float>&, cudaStream_t);
template cudaError_t launch_mortar_grad<float>(const DevMesh&, const MortarOps<float>&, const Phys<float>&, cudaStream_t);
template cudaError_t launch_mortar_flux<float>(const DevMesh&, const MortarOps<float>&, cudaStream_t);
template cudaError_t launch_surf<float>(const DevMesh&, int, float*, float*, float*, const RkStage<float>&, double,
                                       const SourceParams&, const Ops<float>&, const Phys<float>&, cudaStream_t);
template cudaError_t launch_reduce<float>(const float*, const float*, const double*, const double*, const double*,
                                         long long, int, const Phys<float>&, double, double*, int, cudaStream_t);
}  // namespace flexi

// Instantiation of the adjoint kernels for float arithmetic.
#include "k_adj.cuh"

namespace flexi {
template cudaError_t launch_rhs_adjoint<float>(const DevMesh&, const float*, const float*, float*, float, int, const Ops<float>&, const MortarOps<float>&,
                                              const Phys<float>&, void*, double, cudaStream_t);
template cudaError_t launch_axpby<float>(float*, const float*, float, float, size_t, cudaStream_t);
}  // namespace flexi

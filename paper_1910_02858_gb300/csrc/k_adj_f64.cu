// Instantiation of the adjoint kernels for double arithmetic.
#include "k_adj.cuh"

namespace flexi {
template cudaError_t launch_rhs_adjoint<double>(const DevMesh&, const double*, const double*, double*, double, int, const Ops<double>&, const MortarOps<double>&,
                                              const Phys<double>&, void*, double, cudaStream_t);
template cudaError_t launch_axpby<double>(double*, const double*, double, double, size_t, cudaStream_t);
}  // namespace flexi

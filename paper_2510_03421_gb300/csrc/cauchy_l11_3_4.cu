// Cauchy path: the precision ladder's rung kernels for L = 11, 3, 4 limbs.
#include "cauchy_impl.cuh"

namespace perm {
namespace cauchy {

cudaError_t launch_rungs_c(int L, const CauchyArgs& a, int grid, cudaStream_t stream) {
  switch (L) {
    case 11: return launch_rung<11>(a, grid, stream);
    case 3: return launch_rung<3>(a, grid, stream);
    case 4: return launch_rung<4>(a, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cauchy
}  // namespace perm

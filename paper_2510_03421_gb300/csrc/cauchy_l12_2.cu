// Cauchy path: the precision ladder's rung kernels for L = 12, 2 limbs.
#include "cauchy_impl.cuh"

namespace perm {
namespace cauchy {

cudaError_t launch_rungs_b(int L, const CauchyArgs& a, int grid, cudaStream_t stream) {
  switch (L) {
    case 12: return launch_rung<12>(a, grid, stream);
    case 2: return launch_rung<2>(a, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cauchy
}  // namespace perm

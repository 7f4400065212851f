// Cauchy path: the precision ladder's rung kernels for L = 10, 5, 6 limbs.
#include "cauchy_impl.cuh"

namespace perm {
namespace cauchy {

cudaError_t launch_rungs_d(int L, const CauchyArgs& a, int grid, cudaStream_t stream) {
  switch (L) {
    case 10: return launch_rung<10>(a, grid, stream);
    case 5: return launch_rung<5>(a, grid, stream);
    case 6: return launch_rung<6>(a, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cauchy
}  // namespace perm

// Cauchy path: the precision ladder's rung kernels for L = 9, 7, 8 limbs.
#include "cauchy_impl.cuh"

namespace perm {
namespace cauchy {

cudaError_t launch_rungs_e(int L, const CauchyArgs& a, int grid, cudaStream_t stream) {
  switch (L) {
    case 9: return launch_rung<9>(a, grid, stream);
    case 7: return launch_rung<7>(a, grid, stream);
    case 8: return launch_rung<8>(a, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cauchy
}  // namespace perm

// Cauchy path: the precision ladder's rung kernels for L = 16 limbs.
#include "cauchy_impl.cuh"

namespace perm {
namespace cauchy {

cudaError_t launch_rungs_a(int L, const CauchyArgs& a, int grid, cudaStream_t stream) {
  switch (L) {
    case 16: return launch_rung<16>(a, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cauchy
}  // namespace perm

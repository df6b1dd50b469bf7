// Instantiations of the adjoint convolution kernel for radii 1..8.
#include "backward_impl.cuh"

namespace nyf {
cudaError_t bwd_dispatch_a(int Sc, const BwdArgs& a, cudaStream_t st) {
  switch (Sc) {
    case 1: return bwd_launch<1>(a, st);
    case 2: return bwd_launch<2>(a, st);
    case 3: return bwd_launch<3>(a, st);
    case 4: return bwd_launch<4>(a, st);
    case 5: return bwd_launch<5>(a, st);
    case 6: return bwd_launch<6>(a, st);
    case 7: return bwd_launch<7>(a, st);
    case 8: return bwd_launch<8>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace nyf

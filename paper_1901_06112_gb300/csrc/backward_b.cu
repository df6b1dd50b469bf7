// Instantiations of the adjoint convolution kernel for radii 9..16.
#include "backward_impl.cuh"

namespace nyf {
cudaError_t bwd_dispatch_b(int Sc, const BwdArgs& a, cudaStream_t st) {
  switch (Sc) {
    case 9: return bwd_launch<9>(a, st);
    case 10: return bwd_launch<10>(a, st);
    case 11: return bwd_launch<11>(a, st);
    case 12: return bwd_launch<12>(a, st);
    case 13: return bwd_launch<13>(a, st);
    case 14: return bwd_launch<14>(a, st);
    case 15: return bwd_launch<15>(a, st);
    case 16: return bwd_launch<16>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace nyf

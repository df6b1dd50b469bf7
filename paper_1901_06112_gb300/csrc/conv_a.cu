// Instantiations of the fused convolution + combine kernel for radii 1..8.
#include "conv_impl.cuh"

namespace nyf {
cudaError_t conv_dispatch_a(int Sc, const ConvArgs& a, cudaStream_t st) {
  switch (Sc) {
    case 1: return conv_launch<1>(a, st);
    case 2: return conv_launch<2>(a, st);
    case 3: return conv_launch<3>(a, st);
    case 4: return conv_launch<4>(a, st);
    case 5: return conv_launch<5>(a, st);
    case 6: return conv_launch<6>(a, st);
    case 7: return conv_launch<7>(a, st);
    case 8: return conv_launch<8>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace nyf

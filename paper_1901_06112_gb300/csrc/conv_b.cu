// Instantiations of the fused convolution + combine kernel for radii 9..16.
#include "conv_impl.cuh"

namespace nyf {
cudaError_t conv_dispatch_b(int Sc, const ConvArgs& a, cudaStream_t st) {
  switch (Sc) {
    case 9: return conv_launch<9>(a, st);
    case 10: return conv_launch<10>(a, st);
    case 11: return conv_launch<11>(a, st);
    case 12: return conv_launch<12>(a, st);
    case 13: return conv_launch<13>(a, st);
    case 14: return conv_launch<14>(a, st);
    case 15: return conv_launch<15>(a, st);
    case 16: return conv_launch<16>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace nyf

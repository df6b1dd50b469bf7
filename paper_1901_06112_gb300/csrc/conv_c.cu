// Instantiations of the fused convolution + combine kernel for radii 18..32
// (a true radius in between uses the next instantiated one with zero taps).
#include "conv_impl.cuh"

namespace nyf {
cudaError_t conv_dispatch_c(int Sc, const ConvArgs& a, cudaStream_t st) {
  switch (Sc) {
    case 18: return conv_launch<18>(a, st);
    case 20: return conv_launch<20>(a, st);
    case 22: return conv_launch<22>(a, st);
    case 24: return conv_launch<24>(a, st);
    case 28: return conv_launch<28>(a, st);
    case 32: return conv_launch<32>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace nyf

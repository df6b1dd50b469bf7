// Instantiations of the adjoint convolution kernel for radii 18..32 (a true
// radius in between uses the next instantiated one with zero taps), plus the
// geometry helpers of all radius classes.
#include "backward_impl.cuh"

namespace nyf {
cudaError_t bwd_dispatch_c(int Sc, const BwdArgs& a, cudaStream_t st) {
  switch (Sc) {
    case 18: return bwd_launch<18>(a, st);
    case 20: return bwd_launch<20>(a, st);
    case 22: return bwd_launch<22>(a, st);
    case 24: return bwd_launch<24>(a, st);
    case 28: return bwd_launch<28>(a, st);
    case 32: return bwd_launch<32>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

int bwd_chunks(int Sc, int n) {
  const int nq = Sc <= 16 ? 4 : 2;
  return (n + 1 + nq - 1) / nq;
}

int bwd_dphi_slices(int Sc, int n) {
  const int c = bwd_chunks(Sc, n);
  return c > 2 ? c : 1;
}

int64_t bwd_ctas(int Sc, int H, int W, int n) {
  const int tw = Sc <= 24 ? 64 : 32;
  return (int64_t)((W + tw - 1) / tw) * ((H + 31) / 32) * bwd_chunks(Sc, n);
}
}  // namespace nyf

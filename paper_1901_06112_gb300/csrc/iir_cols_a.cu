// Recursive-Gaussian column pass for 3 <= LS <= 31 values per lane
// (one translation unit per range so that the instantiations compile in parallel).
#include "iir_impl.cuh"

namespace nyf {
namespace iir {

cudaError_t dispatch_cols_3_31(int LS, const Args& a, int K, cudaStream_t st) {
  switch (LS) {
    case 3: return launch_cols<3>(a, K, st);
    case 7: return launch_cols<7>(a, K, st);
    case 11: return launch_cols<11>(a, K, st);
    case 15: return launch_cols<15>(a, K, st);
    case 19: return launch_cols<19>(a, K, st);
    case 23: return launch_cols<23>(a, K, st);
    case 27: return launch_cols<27>(a, K, st);
    case 31: return launch_cols<31>(a, K, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace iir
}  // namespace nyf

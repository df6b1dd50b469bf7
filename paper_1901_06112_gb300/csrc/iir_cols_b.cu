// Recursive-Gaussian column pass for 35 <= LS <= 63 values per lane
// (one translation unit per range so that the instantiations compile in parallel).
#include "iir_impl.cuh"

namespace nyf {
namespace iir {

cudaError_t dispatch_cols_35_63(int LS, const Args& a, int K, cudaStream_t st) {
  switch (LS) {
    case 35: return launch_cols<35>(a, K, st);
    case 39: return launch_cols<39>(a, K, st);
    case 43: return launch_cols<43>(a, K, st);
    case 47: return launch_cols<47>(a, K, st);
    case 51: return launch_cols<51>(a, K, st);
    case 55: return launch_cols<55>(a, K, st);
    case 59: return launch_cols<59>(a, K, st);
    case 63: return launch_cols<63>(a, K, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace iir
}  // namespace nyf

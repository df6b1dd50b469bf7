// Recursive-Gaussian row + combine pass for 35 <= LS <= 63 values per lane
// (one translation unit per range so that the instantiations compile in parallel).
#include "iir_impl.cuh"

namespace nyf {
namespace iir {

cudaError_t dispatch_rows_35_63(int LS, const Args& a, int nw, cudaStream_t st) {
  switch (LS) {
    case 35: return launch_rows<35>(a, nw, st);
    case 39: return launch_rows<39>(a, nw, st);
    case 43: return launch_rows<43>(a, nw, st);
    case 47: return launch_rows<47>(a, nw, st);
    case 51: return launch_rows<51>(a, nw, st);
    case 55: return launch_rows<55>(a, nw, st);
    case 59: return launch_rows<59>(a, nw, st);
    case 63: return launch_rows<63>(a, nw, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace iir
}  // namespace nyf

// Recursive-Gaussian row + combine pass for 3 <= LS <= 31 values per lane
// (one translation unit per range so that the instantiations compile in parallel).
#include "iir_impl.cuh"

namespace nyf {
namespace iir {

cudaError_t dispatch_rows_3_31(int LS, const Args& a, int nw, cudaStream_t st) {
  switch (LS) {
    case 3: return launch_rows<3>(a, nw, st);
    case 7: return launch_rows<7>(a, nw, st);
    case 11: return launch_rows<11>(a, nw, st);
    case 15: return launch_rows<15>(a, nw, st);
    case 19: return launch_rows<19>(a, nw, st);
    case 23: return launch_rows<23>(a, nw, st);
    case 27: return launch_rows<27>(a, nw, st);
    case 31: return launch_rows<31>(a, nw, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace iir
}  // namespace nyf

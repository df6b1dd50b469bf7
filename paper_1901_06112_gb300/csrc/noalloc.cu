// nyf_features_static: nyf_features without a caller-provided workspace.
//
// nyf_features needs scratch memory (the device status word, the W_hat factor
// and the FP64 buffers of the eigendecomposition) that normally lives in a
// workspace the caller allocates.  Some callers cannot allocate device memory:
// a plain C host with no device allocator of its own, a plugin whose host owns
// every device allocation, or a latency-critical loop where cudaMalloc would
// synchronise the device.  For them this entry point keeps its scratch in one
// fixed array in device memory (kStaticScratchBytes), which every GPU that
// loads the library holds until the process exits.
//
// The host cannot use the array's symbol as a device address, so the address
// is looked up with cudaGetSymbolAddress once per device, with that device
// current, on the first call made on it (the lookup is cached).  That first
// call should come before any stream capture.  All calls share the array and
// it keeps the last call's contents: the status word is cleared on every call,
// and calls that overlap on the GPU (different streams, or different host
// threads on the same device) race on it.  Because the status word lives in
// the library's array, where no caller can read it, each call copies it, once
// its work is done, to the caller's nullable `status` output.
#include <mutex>

#include "nyf_internal.cuh"

namespace nyf {
namespace {

constexpr size_t kStaticScratchBytes = 256 * 1024;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Device address of g_static_scratch on the current device (looked up once).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace nyf

using namespace nyf;

extern "C" nyf_status nyf_features_static(const float* guide, int64_t N, int rho,
                                          const float* landmarks, int K, float sigma_r,
                                          double eig_rel_tol, int precision, void* phi, int* rank,
                                          double* alphas, int* status, void* stream) {
  // the same argument rules as nyf_features
  if (!guide || !landmarks || !phi || N < 1 || N > ((int64_t)1 << 31) || rho < 1 ||
      !(sigma_r > 0.f) || !isfinite(sigma_r) || !(eig_rel_tol >= 0.0) ||
      (precision != NYF_FP32 && precision != NYF_BF16))
    return NYF_ERR_INVALID_ARG;
  // sizes beyond what the fixed scratch (and the kernels' shared memory) hold
  if (K < 1 || K > NYF_STATIC_MAX_K || rho > NYF_STATIC_MAX_RHO) return NYF_ERR_UNSUPPORTED;
  const size_t off_what = align256(sizeof(DevState));
  const size_t off_eig = off_what + align256(sizeof(float) * NYF_STATIC_MAX_K * NYF_STATIC_MAX_K);
  if (off_eig + eig_scratch_bytes() > kStaticScratchBytes) return NYF_ERR_UNSUPPORTED;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return NYF_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = reinterpret_cast<char*>(base);
  DevState* state = reinterpret_cast<DevState*>(w);
  float* what = reinterpret_cast<float*>(w + off_what);
  if (cudaMemsetAsync(state, 0, sizeof(DevState), st) != cudaSuccess) return NYF_ERR_CUDA;
  if (launch_eig(landmarks, K, rho, sigma_r, eig_rel_tol, what, alphas, rank, state, w + off_eig,
                 st) != cudaSuccess)
    return NYF_ERR_CUDA;
  if (launch_features(guide, N, rho, landmarks, K, sigma_r, what, state, phi,
                      precision == NYF_BF16, st) != cudaSuccess)
    return NYF_ERR_CUDA;
  // the latched device status (NYF_ERR_NUMERIC when no mode was kept and phi was
  // not written) into the caller's own device int
  if (status &&
      cudaMemcpyAsync(status, &state->status, sizeof(int), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return NYF_ERR_CUDA;
  return NYF_OK;
}

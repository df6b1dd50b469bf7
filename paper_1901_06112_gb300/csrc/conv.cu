// Host side of the fused convolution + combine stage: radius selection, the
// split-quantity epilogue (g_hat = zeta / eta when the n + 1 quantities do not
// fit one CTA) and the launch.
#include <math.h>

#include "conv_impl.cuh"

namespace nyf {
namespace {

__global__ void k_divide(const float* __restrict__ zeta, const float* __restrict__ eta, int64_t N,
                         int n, float thr, float* __restrict__ out, DevState* state) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N * n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pix = i / n;
    const float e = eta[pix];
    out[i] = zeta[i] / e;
    if (i % n == 0 && !(e > thr)) atomicAdd(&state->eta_small, 1ull);
  }
}

}  // namespace

cudaError_t conv_tc_dispatch(const ConvArgs& a, cudaStream_t st);
bool conv_tc_supported(int S, int n);

// Smallest compiled radius >= S.
int conv_compiled_radius(int S) {
  if (S <= 16) return S < 1 ? 1 : S;
  static const int big[] = {18, 20, 22, 24, 28, 32};
  for (int v : big)
    if (S <= v) return v;
  return -1;
}

int conv_nq(int Sc) { return Sc <= 24 ? 4 : 2; }

bool conv_split(int S, int n) {
  const int Sc = conv_compiled_radius(S);
  return n + 1 > conv_nq(Sc);
}

cudaError_t launch_conv_combine(const float* f, int H, int W, int n, const void* phi, bool bf16,
                                int tile, int spatial, float sigma_s, int S, DevState* state,
                                float* out, float* eta_out, float* zeta_ws, float* cout,
                                cudaStream_t st) {
  const int Sc = conv_compiled_radius(S);
  if (Sc < 0) return cudaErrorInvalidValue;
  ConvArgs a;
  a.f = f;
  a.H = H;
  a.W = W;
  a.n = n;
  a.N = (int64_t)H * W;
  a.phi = phi;
  a.bf16 = bf16 ? 1 : 0;
  a.state = state;
  a.state_rw = state;
  a.box = spatial == NYF_BOX ? 1 : 0;
  a.inv2s2 = a.box ? 0.f : (float)(1.0 / (2.0 * (double)sigma_s * (double)sigma_s));
  a.S_true = S;
  for (int z = -kMaxTapRadius; z <= kMaxTapRadius; ++z) {
    float g = 0.f;
    if (z >= -S && z <= S)
      g = a.box ? 1.f : (float)exp(-(double)z * z / (2.0 * (double)sigma_s * (double)sigma_s));
    a.taps[kMaxTapRadius + z] = make_float2(g, g);
  }
  double mass = 0.0;   // full-window mass of omega
  for (int z = -S; z <= S; ++z) mass += a.box ? 1.0 : exp(-(double)z * z * a.inv2s2);
  a.eta_thr = (float)(1e-6 * mass * mass);
  // BF16 tensor-core kernel (n <= 3, S <= 16) when asked for; otherwise the FP32 FIR kernel
  const bool mma = tile == NYF_TILE_TENSOR && !bf16 && conv_tc_supported(S, n);
  a.narrow = tile == NYF_TILE_NARROW ? 1 : 0;
  const bool split = mma ? false : n + 1 > conv_nq(Sc);
  a.out = split ? nullptr : out;
  a.zeta = split ? zeta_ws : nullptr;
  a.eta = eta_out;
  a.cout = cout;
  a.k_begin = 0;
  a.k_end = NYF_MAX_K;
  a.c_only = 0;
  cudaError_t e;
  if (mma) e = conv_tc_dispatch(a, st);
  else if (Sc <= 8) e = conv_dispatch_a(Sc, a, st);
  else if (Sc <= 16) e = conv_dispatch_b(Sc, a, st);
  else e = conv_dispatch_c(Sc, a, st);
  if (e != cudaSuccess || !split) return e;
  int64_t g = (a.N * n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_divide<<<(int)g, 256, 0, st>>>(zeta_ws, eta_out, a.N, n, a.eta_thr, out, state);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_conv_recompute(const float* f, int H, int W, int n, const void* phi, bool bf16,
                                  int spatial, float sigma_s, int S, int k_begin, int k_end,
                                  DevState* state, float* cout, cudaStream_t st) {
  const int Sc = conv_compiled_radius(S);
  if (Sc < 0) return cudaErrorInvalidValue;
  ConvArgs a;
  a.f = f;
  a.H = H;
  a.W = W;
  a.n = n;
  a.N = (int64_t)H * W;
  a.phi = phi;
  a.bf16 = bf16 ? 1 : 0;
  a.state = state;
  a.state_rw = state;
  a.box = spatial == NYF_BOX ? 1 : 0;
  a.inv2s2 = a.box ? 0.f : (float)(1.0 / (2.0 * (double)sigma_s * (double)sigma_s));
  a.S_true = S;
  for (int z = -kMaxTapRadius; z <= kMaxTapRadius; ++z) {   // the forward's taps
    float g = 0.f;
    if (z >= -S && z <= S)
      g = a.box ? 1.f : (float)exp(-(double)z * z / (2.0 * (double)sigma_s * (double)sigma_s));
    a.taps[kMaxTapRadius + z] = make_float2(g, g);
  }
  a.eta_thr = 0.f;
  a.narrow = 0;
  a.out = nullptr;
  a.zeta = nullptr;
  a.eta = nullptr;
  a.cout = cout;
  a.k_begin = k_begin;
  a.k_end = k_end;
  a.c_only = 1;
  if (Sc <= 8) return conv_dispatch_a(Sc, a, st);
  if (Sc <= 16) return conv_dispatch_b(Sc, a, st);
  return conv_dispatch_c(Sc, a, st);
}

}  // namespace nyf

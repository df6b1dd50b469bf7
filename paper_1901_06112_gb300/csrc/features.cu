// Per-pixel Nystrom features (Eqs. (11)-(12)).
//
// For pixel x with guide p_x and landmarks mu_m:
//   E_m(x)   = exp(-||p_x - mu_m||^2 / (2 sigma_r^2))       (column x of B, Eq. (11))
//   phi_k(x) = sum_m E_m(x) W_hat[m][k]  =  sqrt(alpha_k) v_k(x)   (Eq. (12))
// Distances are taken as direct FP32 differences (no norm expansion), exp is
// CUDA's expf.  Output planes are planar (plane k at phi + k*N) so that the
// convolution stage reads them coalesced.  The NLM variant forms the
// (2r+1)^2 x n patch guide in shared memory from an image tile (reflect-101
// border) instead of reading a stored guide.
#include "nyf_internal.cuh"

namespace nyf {
namespace {

__device__ inline int reflect101(int i, int n) {
  if (n == 1) return 0;
  const int period = 2 * (n - 1);
  int j = i % period;
  if (j < 0) j += period;
  return j < n ? j : period - j;
}

template <bool BF16>
__device__ inline void store_phi(void* phi, int64_t idx, float v) {
  if (BF16) reinterpret_cast<__nv_bfloat16*>(phi)[idx] = __float2bfloat16_rn(v);
  else reinterpret_cast<float*>(phi)[idx] = v;
}

// Shared tail: E -> phi for one pixel.
template <int KB, bool BF16>
__device__ inline void emit_phi(const float (&e)[KB], int K, int r, const float* Wsm, void* phi,
                                int64_t N, int64_t i) {
  for (int k = 0; k < r; ++k) {
    float acc = 0.f;
#pragma unroll
    for (int m = 0; m < KB; ++m)
      if (m < K) acc = fmaf(e[m], Wsm[m * K + k], acc);
    store_phi<BF16>(phi, (int64_t)k * N + i, acc);
  }
}

// Stored guide (BLF / joint BLF): one pixel per thread.  RB > 0 keeps the
// guide row in registers (rho <= RB); RB == 0 re-reads it (large rho).
template <int KB, int RB, bool BF16>
__global__ void __launch_bounds__(256)
k_features(const float* __restrict__ guide, int64_t N, int rho, const float* __restrict__ lm, int K,
           float inv2s2, const float* __restrict__ what, const DevState* __restrict__ state,
           void* __restrict__ phi) {
  extern __shared__ float sm[];
  float* mu = sm;               // K * rho
  float* Wsm = sm + K * rho;    // K * K
  for (int e = threadIdx.x; e < K * rho; e += blockDim.x) mu[e] = lm[e];
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) Wsm[e] = what[e];
  __syncthreads();
  const int r = state->rank;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float* p = guide + i * rho;
    float x[RB > 0 ? RB : 1];
    if (RB > 0) {
#pragma unroll
      for (int d = 0; d < (RB > 0 ? RB : 1); ++d) x[d] = (d < rho) ? __ldg(p + d) : 0.f;
    }
    float e[KB];
#pragma unroll
    for (int m = 0; m < KB; ++m) {
      float d2 = 0.f;
      if (m < K) {
        const float* c = mu + m * rho;
        if (RB > 0) {
#pragma unroll
          for (int d = 0; d < (RB > 0 ? RB : 1); ++d)
            if (d < rho) {
              const float t = x[d] - c[d];
              d2 = fmaf(t, t, d2);
            }
        } else {
          for (int d = 0; d < rho; ++d) {
            const float t = __ldg(p + d) - c[d];
            d2 = fmaf(t, t, d2);
          }
        }
      }
      e[m] = (m < K) ? expf(-d2 * inv2s2) : 0.f;
    }
    emit_phi<KB, BF16>(e, K, r, Wsm, phi, N, i);
  }
}

// NLM: 16 x 16 pixel tile per CTA; the (16 + 2r)^2 x n image tile (reflect-101
// border) is staged in shared memory and each thread walks its own patch.
constexpr int kNlmTile = 16;

template <int KB, bool BF16>
__global__ void __launch_bounds__(kNlmTile * kNlmTile)
k_features_nlm(const float* __restrict__ f, int H, int W, int n, int r, const float* __restrict__ lm,
               int K, float inv2s2, const float* __restrict__ what,
               const DevState* __restrict__ state, void* __restrict__ phi) {
  extern __shared__ float sm[];
  const int side = 2 * r + 1;
  const int rho = side * side * n;
  const int TS = kNlmTile + 2 * r;
  float* mu = sm;                      // K * rho
  float* Wsm = mu + K * rho;           // K * K
  float* tile = Wsm + K * K;           // TS * TS * n
  const int tid = threadIdx.x;
  const int y0 = blockIdx.y * kNlmTile, x0 = blockIdx.x * kNlmTile;
  for (int e = tid; e < K * rho; e += blockDim.x) mu[e] = lm[e];
  for (int e = tid; e < K * K; e += blockDim.x) Wsm[e] = what[e];
  for (int e = tid; e < TS * TS * n; e += blockDim.x) {
    const int c = e % n, q = e / n;
    const int yy = q / TS, xx = q % TS;
    const int gy = reflect101(y0 - r + yy, H), gx = reflect101(x0 - r + xx, W);
    tile[e] = f[((int64_t)gy * W + gx) * n + c];
  }
  __syncthreads();
  const int ty = tid / kNlmTile, tx = tid % kNlmTile;
  const int y = y0 + ty, x = x0 + tx;
  if (y >= H || x >= W) return;
  float d2[KB];
#pragma unroll
  for (int m = 0; m < KB; ++m) d2[m] = 0.f;
  int j = 0;
  for (int dy = 0; dy < side; ++dy)
    for (int dx = 0; dx < side; ++dx)
      for (int c = 0; c < n; ++c, ++j) {
        const float v = tile[((ty + dy) * TS + (tx + dx)) * n + c];
#pragma unroll
        for (int m = 0; m < KB; ++m)
          if (m < K) {
            const float t = v - mu[m * rho + j];
            d2[m] = fmaf(t, t, d2[m]);
          }
      }
  float e[KB];
#pragma unroll
  for (int m = 0; m < KB; ++m) e[m] = (m < K) ? expf(-d2[m] * inv2s2) : 0.f;
  emit_phi<KB, BF16>(e, K, state->rank, Wsm, phi, (int64_t)H * W, (int64_t)y * W + x);
}

template <int KB, int RB, bool BF16>
cudaError_t features_launch(const float* guide, int64_t N, int rho, const float* lm, int K,
                            float inv2s2, const float* what, const DevState* state, void* phi,
                            cudaStream_t st) {
  const size_t smem = sizeof(float) * ((size_t)K * rho + (size_t)K * K);
  cudaError_t e = cudaFuncSetAttribute(k_features<KB, RB, BF16>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t g = (N + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  k_features<KB, RB, BF16><<<(int)g, 256, smem, st>>>(guide, N, rho, lm, K, inv2s2, what, state, phi);
  count_launches(1);
  return cudaGetLastError();
}

template <int KB, bool BF16>
cudaError_t features_rb(const float* guide, int64_t N, int rho, const float* lm, int K,
                        float inv2s2, const float* what, const DevState* state, void* phi,
                        cudaStream_t st) {
  if (rho <= 4) return features_launch<KB, 4, BF16>(guide, N, rho, lm, K, inv2s2, what, state, phi, st);
  if (rho <= 32) return features_launch<KB, 32, BF16>(guide, N, rho, lm, K, inv2s2, what, state, phi, st);
  return features_launch<KB, 0, BF16>(guide, N, rho, lm, K, inv2s2, what, state, phi, st);
}

template <bool BF16>
cudaError_t features_k(const float* guide, int64_t N, int rho, const float* lm, int K,
                       float inv2s2, const float* what, const DevState* state, void* phi,
                       cudaStream_t st) {
  if (K <= 8) return features_rb<8, BF16>(guide, N, rho, lm, K, inv2s2, what, state, phi, st);
  if (K <= 16) return features_rb<16, BF16>(guide, N, rho, lm, K, inv2s2, what, state, phi, st);
  if (K <= 32) return features_rb<32, BF16>(guide, N, rho, lm, K, inv2s2, what, state, phi, st);
  return features_rb<64, BF16>(guide, N, rho, lm, K, inv2s2, what, state, phi, st);
}

template <int KB, bool BF16>
cudaError_t nlm_launch(const float* f, int H, int W, int n, int r, const float* lm, int K,
                       float inv2s2, const float* what, const DevState* state, void* phi,
                       cudaStream_t st) {
  const int rho = (2 * r + 1) * (2 * r + 1) * n;
  const int TS = kNlmTile + 2 * r;
  const size_t smem = sizeof(float) * ((size_t)K * rho + (size_t)K * K + (size_t)TS * TS * n);
  cudaError_t e = cudaFuncSetAttribute(k_features_nlm<KB, BF16>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((W + kNlmTile - 1) / kNlmTile, (H + kNlmTile - 1) / kNlmTile);
  k_features_nlm<KB, BF16><<<grid, kNlmTile * kNlmTile, smem, st>>>(f, H, W, n, r, lm, K, inv2s2,
                                                                    what, state, phi);
  count_launches(1);
  return cudaGetLastError();
}

template <bool BF16>
cudaError_t nlm_k(const float* f, int H, int W, int n, int r, const float* lm, int K, float inv2s2,
                  const float* what, const DevState* state, void* phi, cudaStream_t st) {
  if (K <= 8) return nlm_launch<8, BF16>(f, H, W, n, r, lm, K, inv2s2, what, state, phi, st);
  if (K <= 16) return nlm_launch<16, BF16>(f, H, W, n, r, lm, K, inv2s2, what, state, phi, st);
  if (K <= 32) return nlm_launch<32, BF16>(f, H, W, n, r, lm, K, inv2s2, what, state, phi, st);
  return nlm_launch<64, BF16>(f, H, W, n, r, lm, K, inv2s2, what, state, phi, st);
}

}  // namespace

cudaError_t launch_features(const float* guide, int64_t N, int rho, const float* landmarks, int K,
                            float sigma_r, const float* what, const DevState* state, void* phi,
                            bool bf16, cudaStream_t st) {
  const float inv2s2 = (float)(1.0 / (2.0 * (double)sigma_r * (double)sigma_r));
  return bf16 ? features_k<true>(guide, N, rho, landmarks, K, inv2s2, what, state, phi, st)
              : features_k<false>(guide, N, rho, landmarks, K, inv2s2, what, state, phi, st);
}

cudaError_t launch_features_nlm(const float* f, int H, int W, int n, int r, const float* landmarks,
                                int K, float sigma_r, const float* what, const DevState* state,
                                void* phi, bool bf16, cudaStream_t st) {
  const float inv2s2 = (float)(1.0 / (2.0 * (double)sigma_r * (double)sigma_r));
  return bf16 ? nlm_k<true>(f, H, W, n, r, landmarks, K, inv2s2, what, state, phi, st)
              : nlm_k<false>(f, H, W, n, r, landmarks, K, inv2s2, what, state, phi, st);
}

size_t features_nlm_smem_bytes(int K, int n, int r) {
  const int rho = (2 * r + 1) * (2 * r + 1) * n;
  const int TS = kNlmTile + 2 * r;
  return sizeof(float) * ((size_t)K * rho + (size_t)K * K + (size_t)TS * TS * n);
}

}  // namespace nyf

// Per-pixel Nystrom features (Eqs. (11)-(12)).
//
// For pixel x with guide p_x and landmarks mu_m:
//   E_m(x)   = exp(-||p_x - mu_m||^2 / (2 sigma_r^2))       (column x of B, Eq. (11))
//   phi_k(x) = sum_m E_m(x) W_hat[m][k]  =  sqrt(alpha_k) v_k(x)   (Eq. (12))
// Distances are taken as direct FP32 differences (no norm expansion), exp is
// CUDA's expf.  Guides of dimension rho >= 16 go to the tensor-core kernel of
// features_tc.cu instead (the contraction over rho is deep enough to be one).
// Output planes are planar (plane k at phi + k*N) so that the convolution
// stage reads them coalesced.  The NLM variant forms the
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

// Shared tail: E -> phi for one pixel.  W_hat sits in shared memory with a
// row stride KP (K rounded up to 4, zero padded) so that four modes' weights
// come in one 16-byte load: one shared load per four FMAs.
__host__ __device__ inline int kpad(int K) { return (K + 3) & ~3; }

template <int KB, bool BF16>
__device__ inline void emit_phi(const float (&e)[KB], int K, int r, const float* Wsm, void* phi,
                                int64_t N, int64_t i) {
  const int KP = kpad(K);
  for (int k = 0; k < r; k += 4) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
    for (int m = 0; m < KB; ++m)
      if (m < K) {
        const float4 w = *reinterpret_cast<const float4*>(Wsm + m * KP + k);
        a0 = fmaf(e[m], w.x, a0);
        a1 = fmaf(e[m], w.y, a1);
        a2 = fmaf(e[m], w.z, a2);
        a3 = fmaf(e[m], w.w, a3);
      }
    store_phi<BF16>(phi, (int64_t)k * N + i, a0);
    if (k + 1 < r) store_phi<BF16>(phi, (int64_t)(k + 1) * N + i, a1);
    if (k + 2 < r) store_phi<BF16>(phi, (int64_t)(k + 2) * N + i, a2);
    if (k + 3 < r) store_phi<BF16>(phi, (int64_t)(k + 3) * N + i, a3);
  }
}

// Two pixels per thread: each 16-byte weight load feeds eight FMAs.
template <int KB, bool BF16>
__device__ inline void emit_phi2(const float (&e0)[KB], const float (&e1)[KB], bool v1, int K,
                                 int r, const float* Wsm, void* phi, int64_t N, int64_t i0,
                                 int64_t i1) {
  const int KP = kpad(K);
  for (int k = 0; k < r; k += 4) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, b0 = 0.f, b1 = 0.f, b2 = 0.f, b3 = 0.f;
#pragma unroll
    for (int m = 0; m < KB; ++m)
      if (m < K) {
        const float4 w = *reinterpret_cast<const float4*>(Wsm + m * KP + k);
        a0 = fmaf(e0[m], w.x, a0);
        a1 = fmaf(e0[m], w.y, a1);
        a2 = fmaf(e0[m], w.z, a2);
        a3 = fmaf(e0[m], w.w, a3);
        b0 = fmaf(e1[m], w.x, b0);
        b1 = fmaf(e1[m], w.y, b1);
        b2 = fmaf(e1[m], w.z, b2);
        b3 = fmaf(e1[m], w.w, b3);
      }
    const float va[4] = {a0, a1, a2, a3}, vb[4] = {b0, b1, b2, b3};
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (k + q < r) {
        store_phi<BF16>(phi, (int64_t)(k + q) * N + i0, va[q]);
        if (v1) store_phi<BF16>(phi, (int64_t)(k + q) * N + i1, vb[q]);
      }
  }
}

// W_hat (K x K, row-major) -> shared memory with row stride kpad(K).
__device__ inline void stage_what(const float* what, int K, float* Wsm) {
  const int KP = kpad(K);
  for (int e = threadIdx.x; e < K * KP; e += blockDim.x) {
    const int m = e / KP, k = e - m * KP;
    Wsm[e] = k < K ? what[m * K + k] : 0.f;
  }
}

// E_m = exp(-||p_i - mu_m||^2 / (2 sigma_r^2)) for one stored guide row.
template <int KB, int RB>
__device__ inline void guide_exp(const float* __restrict__ guide, int64_t i, int rho,
                                 const float* mu, int K, float inv2s2, float (&e)[KB]) {
  const float* p = guide + i * rho;
  float x[RB > 0 ? RB : 1];
  if (RB > 0) {
#pragma unroll
    for (int d = 0; d < (RB > 0 ? RB : 1); ++d) x[d] = (d < rho) ? __ldg(p + d) : 0.f;
  }
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
}

// Stored guide (BLF / joint BLF): two pixels per thread.  RB > 0 keeps the
// guide row in registers (rho <= RB); RB == 0 re-reads it (large rho).
template <int KB, int RB, bool BF16>
__global__ void __launch_bounds__(256)
k_features(const float* __restrict__ guide, int64_t N, int rho, const float* __restrict__ lm, int K,
           float inv2s2, const float* __restrict__ what, const DevState* __restrict__ state,
           void* __restrict__ phi) {
  extern __shared__ float sm[];
  float* Wsm = sm;                      // K * kpad(K), 16-byte aligned
  float* mu = sm + K * kpad(K);         // K * rho
  for (int e = threadIdx.x; e < K * rho; e += blockDim.x) mu[e] = lm[e];
  stage_what(what, K, Wsm);
  __syncthreads();
  const int r = state->planes;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * 2;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x * 2; base < N; base += stride) {
    const int64_t i0 = base + threadIdx.x, i1 = i0 + blockDim.x;
    const bool v0 = i0 < N, v1 = i1 < N;
    float e0[KB], e1[KB];
    guide_exp<KB, RB>(guide, v0 ? i0 : 0, rho, mu, K, inv2s2, e0);
    guide_exp<KB, RB>(guide, v1 ? i1 : 0, rho, mu, K, inv2s2, e1);
    if (v0) emit_phi2<KB, BF16>(e0, e1, v1, K, r, Wsm, phi, N, i0, i1);
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
  float* Wsm = sm;                     // K * kpad(K), 16-byte aligned
  float* mu = Wsm + K * kpad(K);       // K * rho
  float* tile = mu + K * rho;          // TS * TS * n
  const int tid = threadIdx.x;
  const int y0 = blockIdx.y * kNlmTile, x0 = blockIdx.x * kNlmTile;
  for (int e = tid; e < K * rho; e += blockDim.x) mu[e] = lm[e];
  stage_what(what, K, Wsm);
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
  emit_phi<KB, BF16>(e, K, state->planes, Wsm, phi, (int64_t)H * W, (int64_t)y * W + x);
}

template <int KB, int RB, bool BF16>
cudaError_t features_launch(const float* guide, int64_t N, int rho, const float* lm, int K,
                            float inv2s2, const float* what, const DevState* state, void* phi,
                            cudaStream_t st) {
  const size_t smem = sizeof(float) * ((size_t)K * rho + (size_t)K * kpad(K));
  cudaError_t e = cudaFuncSetAttribute(k_features<KB, RB, BF16>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t g = (N + 511) / 512;
  if (g > 152 * 8) g = 152 * 8;
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
  const size_t smem = sizeof(float) * ((size_t)K * rho + (size_t)K * kpad(K) + (size_t)TS * TS * n);
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
  if (rho >= kFeaturesTcMinRho)   // a contraction deep enough for the tensor cores
    return launch_features_tc(guide, N, rho, landmarks, K, sigma_r, what, state, phi, bf16, st);
  const float inv2s2 = (float)(1.0 / (2.0 * (double)sigma_r * (double)sigma_r));
  return bf16 ? features_k<true>(guide, N, rho, landmarks, K, inv2s2, what, state, phi, st)
              : features_k<false>(guide, N, rho, landmarks, K, inv2s2, what, state, phi, st);
}

cudaError_t launch_features_nlm(const float* f, int H, int W, int n, int r, const float* landmarks,
                                int K, float sigma_r, const float* what, const DevState* state,
                                void* phi, bool bf16, cudaStream_t st) {
  if ((2 * r + 1) * (2 * r + 1) * n >= kFeaturesTcMinRho)
    return launch_features_nlm_tc(f, H, W, n, r, landmarks, K, sigma_r, what, state, phi, bf16, st);
  const float inv2s2 = (float)(1.0 / (2.0 * (double)sigma_r * (double)sigma_r));
  return bf16 ? nlm_k<true>(f, H, W, n, r, landmarks, K, inv2s2, what, state, phi, st)
              : nlm_k<false>(f, H, W, n, r, landmarks, K, inv2s2, what, state, phi, st);
}

size_t features_nlm_smem_bytes(int K, int n, int r) {
  const int rho = (2 * r + 1) * (2 * r + 1) * n;
  if (rho >= kFeaturesTcMinRho) return features_tc_smem_bytes(rho, K, n, r);
  const int TS = kNlmTile + 2 * r;
  return sizeof(float) * ((size_t)K * rho + (size_t)K * kpad(K) + (size_t)TS * TS * n);
}

}  // namespace nyf

// Fused spatial convolutions + combine (Eqs. (7), (14), (15); Algorithm 1 loop).
//
// For every kept mode k and every quantity q (the n channels of f, plus the
// constant 1 for the denominator), one CTA computes on its output tile
//     C_kq = omega * (phi_k f_q)     (f_n := 1)
// as a separable FIR (vertical pass into shared memory, then horizontal pass
// into registers) and accumulates zeta_q += phi_k C_kq in registers; eta is
// the q = n accumulator.  Only g_hat = zeta / eta (or zeta and eta when the
// quantities are split over several CTAs) leaves the chip: the K (n+1)
// convolved planes never touch HBM.
//
// Zero padding outside the image is the window clipping of Eq. (1).  The taps
// g(z) = exp(-z^2 / (2 sigma_s^2)) (or 1 for the box) are held in registers;
// the window radius S is a compile-time bound (taps with |z| above the true
// radius are zero) so that the register-blocked FIR loops fully unroll.
#pragma once

#include "nyf_internal.cuh"

namespace nyf {

struct ConvArgs {
  const float* f;
  int H, W, n;
  int64_t N;
  const void* phi;          // K planes of N values
  int bf16;                 // phi element type
  const DevState* state;
  DevState* state_rw;
  float inv2s2;             // 1 / (2 sigma_s^2)
  int S_true;               // true window radius
  int box;                  // box window (taps = 1)
  float eta_thr;            // eta_hat below this counts as "small"
  float* out;               // H x W x n, when all quantities are in one CTA
  float* zeta;              // N x n, when they are split
  float* eta;               // N
};

constexpr int kConvThreads = 256;

template <int S>
struct ConvCfg {
  static constexpr int TH = 32;
  static constexpr int TW = S <= 16 ? 96 : 64;
  static constexpr int RV = 16;
  static constexpr int RH = S <= 16 ? 12 : 8;
  static constexpr int NQ = S <= 24 ? 4 : 2;
  static constexpr int HH = TH + 2 * S;
  static constexpr int HW = TW + 2 * S;
  static constexpr int PS = HW | 1;           // odd row stride: conflict-free column/row walks
  static constexpr int PLANE = HH * PS;
  static constexpr size_t smem = sizeof(float) * ((size_t)(NQ + 1) * PLANE + (size_t)TH * PS);
  static_assert(TH * (TW / RH) == kConvThreads, "one horizontal task per thread");
  static_assert((TH / RV) * HW <= kConvThreads, "at most one vertical task per thread");
};

__device__ __forceinline__ float load_phi(const void* phi, int bf16, int64_t idx) {
  if (bf16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(phi)[idx]);
  return __ldg(reinterpret_cast<const float*>(phi) + idx);
}

template <int S>
__global__ void __launch_bounds__(kConvThreads, 1) k_conv_combine(ConvArgs a) {
  using C = ConvCfg<S>;
  constexpr int T = 2 * S + 1;
  constexpr int TH = C::TH, TW = C::TW, RV = C::RV, RH = C::RH, NQ = C::NQ;
  constexpr int HH = C::HH, HW = C::HW, PS = C::PS, PLANE = C::PLANE;
  extern __shared__ float sm[];
  float* F = sm;                    // NQ image planes (tile + halo)
  float* P = F + NQ * PLANE;        // phi_k (tile + halo)
  float* M = P + PLANE;             // vertical-pass result, TH x HW
  const int tid = threadIdx.x;
  const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;
  const int q0 = blockIdx.z * NQ;
  const int n = a.n;

  float g[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int z = t - S;
    const float zz = (float)(z * z);
    g[t] = (z > a.S_true || -z > a.S_true) ? 0.f : (a.box ? 1.f : expf(-zz * a.inv2s2));
  }

  for (int e = tid; e < NQ * HH * HW; e += kConvThreads) {
    const int qi = e / (HH * HW);
    const int rem = e - qi * (HH * HW);
    const int yy = rem / HW, xx = rem - yy * HW;
    const int c = q0 + qi;
    const int gy = ty0 - S + yy, gx = tx0 - S + xx;
    float v = 0.f;
    if (c < n && gy >= 0 && gy < a.H && gx >= 0 && gx < a.W)
      v = __ldg(a.f + ((int64_t)gy * a.W + gx) * n + c);
    F[qi * PLANE + yy * PS + xx] = v;
  }

  float acc[NQ][RH];
#pragma unroll
  for (int qi = 0; qi < NQ; ++qi)
#pragma unroll
    for (int j = 0; j < RH; ++j) acc[qi][j] = 0.f;

  const int hy = tid / (TW / RH), hx0 = (tid % (TW / RH)) * RH;
  const int vtask = tid;                        // one vertical task per thread (or none)
  const int vx = vtask % HW, vy0 = (vtask / HW) * RV;
  const bool vactive = vtask < (TH / RV) * HW;
  const int r = a.state->rank;

  for (int k = 0; k < r; ++k) {
    __syncthreads();
    const int64_t base = (int64_t)k * a.N;
    for (int e = tid; e < HH * HW; e += kConvThreads) {
      const int yy = e / HW, xx = e - yy * HW;
      const int gy = ty0 - S + yy, gx = tx0 - S + xx;
      float v = 0.f;
      if (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W)
        v = load_phi(a.phi, a.bf16, base + (int64_t)gy * a.W + gx);
      P[yy * PS + xx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int qi = 0; qi < NQ; ++qi) {
      const int q = q0 + qi;
      if (q <= n) {                              // uniform over the block
        const bool den = (q == n);
        const float* Fq = F + qi * PLANE;
        if (vactive) {
          float va[RV];
#pragma unroll
          for (int j = 0; j < RV; ++j) va[j] = 0.f;
#pragma unroll
          for (int i = 0; i < RV + 2 * S; ++i) {
            const int off = (vy0 + i) * PS + vx;
            float v = P[off];
            if (!den) v *= Fq[off];
#pragma unroll
            for (int j = 0; j < RV; ++j) {
              const int t = i - j;
              if (t >= 0 && t < T) va[j] = fmaf(g[t], v, va[j]);
            }
          }
#pragma unroll
          for (int j = 0; j < RV; ++j) M[(vy0 + j) * PS + vx] = va[j];
        }
        __syncthreads();
        float hb[RH];
#pragma unroll
        for (int j = 0; j < RH; ++j) hb[j] = 0.f;
#pragma unroll
        for (int i = 0; i < RH + 2 * S; ++i) {
          const float v = M[hy * PS + hx0 + i];
#pragma unroll
          for (int j = 0; j < RH; ++j) {
            const int t = i - j;
            if (t >= 0 && t < T) hb[j] = fmaf(g[t], v, hb[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < RH; ++j)
          acc[qi][j] = fmaf(P[(hy + S) * PS + hx0 + j + S], hb[j], acc[qi][j]);
        __syncthreads();
      }
    }
  }

  // Epilogue: g_hat = zeta / eta (fused) or zeta, eta to memory (split).
  const int y = ty0 + hy;
  const bool fused = (q0 == 0) && (n + 1 <= NQ);
#pragma unroll
  for (int j = 0; j < RH; ++j) {
    const int x = tx0 + hx0 + j;
    if (y < a.H && x < a.W) {
      const int64_t pix = (int64_t)y * a.W + x;
      if (fused) {
        float eta = 0.f;
#pragma unroll
        for (int qi = 0; qi < NQ; ++qi)
          if (qi == n) eta = acc[qi][j];
#pragma unroll
        for (int qi = 0; qi < NQ; ++qi)
          if (qi < n) a.out[pix * n + qi] = acc[qi][j] / eta;
        a.eta[pix] = eta;
        if (!(eta > a.eta_thr)) atomicAdd(&a.state_rw->eta_small, 1ull);
      } else {
#pragma unroll
        for (int qi = 0; qi < NQ; ++qi) {
          const int q = q0 + qi;
          if (q < n) a.zeta[pix * n + q] = acc[qi][j];
          else if (q == n) a.eta[pix] = acc[qi][j];
        }
      }
    }
  }
}

template <int S>
cudaError_t conv_launch(const ConvArgs& a, cudaStream_t st) {
  using C = ConvCfg<S>;
  cudaError_t e = cudaFuncSetAttribute(k_conv_combine<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.W + C::TW - 1) / C::TW, (a.H + C::TH - 1) / C::TH, (a.n + 1 + C::NQ - 1) / C::NQ);
  k_conv_combine<S><<<grid, kConvThreads, C::smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

// Per-file dispatchers (each instantiates a range of compile-time radii).
cudaError_t conv_dispatch_a(int Sc, const ConvArgs& a, cudaStream_t st);   // 1..8
cudaError_t conv_dispatch_b(int Sc, const ConvArgs& a, cudaStream_t st);   // 9..16
cudaError_t conv_dispatch_c(int Sc, const ConvArgs& a, cudaStream_t st);   // 18..32
bool conv_split(int S, int n);   // true when quantities are split over CTAs

}  // namespace nyf

// Adjoint of the fused convolution + combine stage (backward of Eqs. (14)-(15)).
//
// Forward, per quantity q (q < n: channel f_q; q = n: the constant 1):
//   C_kq = omega * (phi_k f_q),  zeta_q = sum_k phi_k C_kq,  g_hat_c = zeta_c / eta,
//   eta = zeta_n.
// With G = dL/d g_hat:  a_c = G_c / eta (c < n),  a_n = -sum_c G_c g_hat_c / eta, so
// dL/d zeta_q = a_q.  Writing B_kq = omega * (a_q phi_k) (omega is symmetric, so
// the adjoint of the convolution is the convolution itself):
//   dL/d phi_k(x) = sum_q [ a_q(x) C_kq(x) + f_q(x) B_kq(x) ]            (f_n := 1)
//   dL/d f_c(x)  += sum_k phi_k(x) B_kc(x)                     (direct image term)
//   dL/d sigma_s  = sum_x sum_q a_q(x) sum_k phi_k(x) (omega' * (phi_k f_q))(x),
// where omega' = d omega / d sigma_s = g' (x) g + g (x) g' with
// g'(t) = g(t) t^2 / sigma_s^3 (window radius held fixed).
//
// One CTA per (output tile, pair of quantities).  Per mode k the CTA stages
// phi_k (double-buffered, cp.async) and runs, per quantity, one vertical pass
// producing three planes (g on phi f, g' on phi f, g on a phi) and one
// horizontal pass producing C, the sigma_s term and B at its pixels.  dL/dphi_k
// leaves the CTA as one plane per mode (summed with atomics when the
// quantities of a pixel are split over several CTAs), dL/df and the sigma_s
// partial at the end.
#pragma once

#include "conv_impl.cuh"

namespace nyf {

struct BwdArgs {
  const float* f;
  int H, W, n;
  int64_t N;
  const void* phi;
  int bf16;
  const DevState* state;
  const float* eta;       // N, saved by the forward pass
  const float* out;       // g_hat, N x n
  const float* gout;      // dL/d g_hat, N x n
  float inv2s2;           // 1 / (2 sigma_s^2)
  float inv_s3;           // 1 / sigma_s^3
  int S_true;
  int box;
  float* dphi;            // r planes of N
  int atomic_dphi;
  float* df;              // N x n, direct image term
  float* sig_part;        // one sigma_s partial per CTA
};

template <int S>
struct BwdCfg {
  static constexpr int TH = 32;
  static constexpr int TW = S <= 16 ? 64 : (S <= 24 ? 48 : 32);
  static constexpr int RV = S <= 24 ? 16 : 8;
  static constexpr int RH = S <= 16 ? 8 : (S <= 24 ? 6 : 4);
  static constexpr int NQ = S <= 24 ? 2 : 1;
  static constexpr int HH = TH + 2 * S;
  static constexpr int HW = TW + 2 * S;
  static constexpr int PS = HW | 1;
  static constexpr int PLANE = HH * PS;
  static constexpr int VT = (TH / RV) * HW;          // vertical tasks
  static constexpr size_t smem =
      sizeof(float) * ((size_t)(2 * NQ + 2) * PLANE + (size_t)3 * TH * PS);
  static_assert(TH * (TW / RH) == kConvThreads, "one horizontal task per thread");
  static_assert(smem <= 227 * 1024, "shared memory budget");
};

template <int S>
__device__ __forceinline__ void bwd_stage_phi(const BwdArgs& a, float* P, int k, int ty0, int tx0) {
  using C = BwdCfg<S>;
  const int64_t base = (int64_t)k * a.N;
  if (!a.bf16) {
    const float* src = reinterpret_cast<const float*>(a.phi) + base;
    for (int e = threadIdx.x; e < C::HH * C::HW; e += kConvThreads) {
      const int yy = e / C::HW, xx = e - yy * C::HW;
      const int gy = ty0 - S + yy, gx = tx0 - S + xx;
      const bool in = gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
      cp_async4(P + yy * C::PS + xx, in ? src + (int64_t)gy * a.W + gx : src, in);
    }
  } else {
    const __nv_bfloat16* src = reinterpret_cast<const __nv_bfloat16*>(a.phi) + base;
    for (int e = threadIdx.x; e < C::HH * C::HW; e += kConvThreads) {
      const int yy = e / C::HW, xx = e - yy * C::HW;
      const int gy = ty0 - S + yy, gx = tx0 - S + xx;
      float v = 0.f;
      if (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W)
        v = __bfloat162float(src[(int64_t)gy * a.W + gx]);
      P[yy * C::PS + xx] = v;
    }
  }
}

template <int S>
__global__ void __launch_bounds__(kConvThreads, 1) k_conv_bwd(BwdArgs a) {
  using C = BwdCfg<S>;
  constexpr int T = 2 * S + 1;
  constexpr int TH = C::TH, TW = C::TW, RV = C::RV, RH = C::RH, NQ = C::NQ;
  constexpr int HH = C::HH, HW = C::HW, PS = C::PS, PLANE = C::PLANE;
  extern __shared__ float sm[];
  float* F = sm;                    // NQ image planes
  float* Aq = F + NQ * PLANE;       // NQ adjoint planes a_q
  float* PB = Aq + NQ * PLANE;      // two phi planes
  float* Mg = PB + 2 * PLANE;       // vertical passes: g on phi f
  float* Mp = Mg + TH * PS;         //                  g' on phi f
  float* Mb = Mp + TH * PS;         //                  g on a phi
  const int tid = threadIdx.x;
  const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;
  const int q0 = blockIdx.z * NQ;
  const int n = a.n;
  const int r = a.state->planes;

  for (int e = tid; e < NQ * HH * HW; e += kConvThreads) {
    const int qi = e / (HH * HW);
    const int rem = e - qi * (HH * HW);
    const int yy = rem / HW, xx = rem - yy * HW;
    const int c = q0 + qi;
    const int gy = ty0 - S + yy, gx = tx0 - S + xx;
    const bool in = c < n && gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
    cp_async4(F + qi * PLANE + yy * PS + xx, in ? a.f + ((int64_t)gy * a.W + gx) * n + c : a.f, in);
  }
  if (r > 0) bwd_stage_phi<S>(a, PB, 0, ty0, tx0);
  cp_async_commit();
  // a_q on the tile + halo (zero outside the image)
  for (int e = tid; e < NQ * HH * HW; e += kConvThreads) {
    const int qi = e / (HH * HW);
    const int rem = e - qi * (HH * HW);
    const int yy = rem / HW, xx = rem - yy * HW;
    const int q = q0 + qi;
    const int gy = ty0 - S + yy, gx = tx0 - S + xx;
    float v = 0.f;
    if (q <= n && gy >= 0 && gy < a.H && gx >= 0 && gx < a.W) {
      const int64_t pix = (int64_t)gy * a.W + gx;
      const float ie = 1.f / a.eta[pix];
      if (q < n) {
        v = a.gout[pix * n + q] * ie;
      } else {
        float s = 0.f;
        for (int c = 0; c < n; ++c) s = fmaf(a.gout[pix * n + c], a.out[pix * n + c], s);
        v = -s * ie;
      }
    }
    Aq[qi * PLANE + yy * PS + xx] = v;
  }

  // (g, g') tap pairs: one packed FMA updates the g and g' accumulators of an input
  float2 gg[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int z = t - S;
    const float zz = (float)(z * z);
    const bool on = !(z > a.S_true || -z > a.S_true);
    const float gv = on ? (a.box ? 1.f : expf(-zz * a.inv2s2)) : 0.f;
    gg[t] = make_float2(gv, (on && !a.box) ? gv * zz * a.inv_s3 : 0.f);
  }

  float dfa[NQ][RH];
#pragma unroll
  for (int qi = 0; qi < NQ; ++qi)
#pragma unroll
    for (int j = 0; j < RH; ++j) dfa[qi][j] = 0.f;
  float sig = 0.f;

  const int hy = tid / (TW / RH), hx0 = (tid % (TW / RH)) * RH;
  const int y = ty0 + hy;

  for (int k = 0; k < r; ++k) {
    if (k + 1 < r) {
      bwd_stage_phi<S>(a, PB + ((k + 1) & 1) * PLANE, k + 1, ty0, tx0);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* P = PB + (k & 1) * PLANE;
    float dacc[RH];
#pragma unroll
    for (int j = 0; j < RH; ++j) dacc[j] = 0.f;
#pragma unroll
    for (int qi = 0; qi < NQ; ++qi) {
      const int q = q0 + qi;
      if (q <= n) {                              // uniform over the block
        const bool den = (q == n);
        const float* Fq = F + qi * PLANE;
        const float* Aqq = Aq + qi * PLANE;
        for (int task = tid; task < C::VT; task += kConvThreads) {
          const int vx = task % HW, vy0 = (task / HW) * RV;
          float2 vap[RV];            // (g, g') on phi f
          float vb[RV];              // g on a phi
#pragma unroll
          for (int j = 0; j < RV; ++j) {
            vap[j] = make_float2(0.f, 0.f);
            vb[j] = 0.f;
          }
#pragma unroll
          for (int i = 0; i < RV + 2 * S; ++i) {
            const int off = (vy0 + i) * PS + vx;
            const float p = P[off];
            const float h = den ? p : p * Fq[off];
            const float u = p * Aqq[off];
            const float2 hh = make_float2(h, h);
#pragma unroll
            for (int j = 0; j < RV; ++j) {
              const int t = i - j;
              if (t >= 0 && t < T) {
                vap[j] = __ffma2_rn(gg[t], hh, vap[j]);
                vb[j] = fmaf(gg[t].x, u, vb[j]);
              }
            }
          }
#pragma unroll
          for (int j = 0; j < RV; ++j) {
            Mg[(vy0 + j) * PS + vx] = vap[j].x;
            Mp[(vy0 + j) * PS + vx] = vap[j].y;
            Mb[(vy0 + j) * PS + vx] = vb[j];
          }
        }
        __syncthreads();
        float2 ccp[RH];              // (g on Mg, g' on Mg + g on Mp)
        float bb[RH];
#pragma unroll
        for (int j = 0; j < RH; ++j) {
          ccp[j] = make_float2(0.f, 0.f);
          bb[j] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < RH + 2 * S; ++i) {
          const int off = hy * PS + hx0 + i;
          const float mg = Mg[off], mp = Mp[off], mb = Mb[off];
          const float2 mm = make_float2(mg, mg);
#pragma unroll
          for (int j = 0; j < RH; ++j) {
            const int t = i - j;
            if (t >= 0 && t < T) {
              ccp[j] = __ffma2_rn(gg[t], mm, ccp[j]);
              ccp[j].y = fmaf(gg[t].x, mp, ccp[j].y);
              bb[j] = fmaf(gg[t].x, mb, bb[j]);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < RH; ++j) {
          const int ctr = (hy + S) * PS + hx0 + j + S;
          const float p = P[ctr], aq = Aqq[ctr];
          const float fq = den ? 1.f : Fq[ctr];
          dacc[j] = fmaf(aq, ccp[j].x, fmaf(fq, bb[j], dacc[j]));
          if (!den) dfa[qi][j] = fmaf(p, bb[j], dfa[qi][j]);
          sig = fmaf(aq * p, ccp[j].y, sig);
        }
        __syncthreads();
      }
    }
    if (y < a.H) {
      float* dst = a.dphi + (int64_t)k * a.N + (int64_t)y * a.W;
#pragma unroll
      for (int j = 0; j < RH; ++j) {
        const int x = tx0 + hx0 + j;
        if (x < a.W) {
          if (a.atomic_dphi) atomicAdd(dst + x, dacc[j]);
          else dst[x] = dacc[j];
        }
      }
    }
  }
  cp_async_wait<0>();

  if (y < a.H) {
#pragma unroll
    for (int j = 0; j < RH; ++j) {
      const int x = tx0 + hx0 + j;
      if (x < a.W) {
        const int64_t pix = (int64_t)y * a.W + x;
#pragma unroll
        for (int qi = 0; qi < NQ; ++qi)
          if (q0 + qi < n) a.df[pix * n + q0 + qi] = dfa[qi][j];
      }
    }
  }
  // sigma_s partial of this CTA (fixed-order reduction)
  __shared__ float red[kConvThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sig += __shfl_xor_sync(0xffffffffu, sig, o);
  if ((tid & 31) == 0) red[tid >> 5] = sig;
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int w = 0; w < kConvThreads / 32; ++w) s += red[w];
    const int cta = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    a.sig_part[cta] = s;
  }
}

template <int S>
cudaError_t bwd_launch(const BwdArgs& a, cudaStream_t st) {
  using C = BwdCfg<S>;
  cudaError_t e = cudaFuncSetAttribute(k_conv_bwd<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.W + C::TW - 1) / C::TW, (a.H + C::TH - 1) / C::TH, (a.n + 1 + C::NQ - 1) / C::NQ);
  k_conv_bwd<S><<<grid, kConvThreads, C::smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <int S>
dim3 bwd_grid(int H, int W, int n) {
  using C = BwdCfg<S>;
  return dim3((W + C::TW - 1) / C::TW, (H + C::TH - 1) / C::TH, (n + 1 + C::NQ - 1) / C::NQ);
}

cudaError_t bwd_dispatch_a(int Sc, const BwdArgs& a, cudaStream_t st);   // 1..8
cudaError_t bwd_dispatch_b(int Sc, const BwdArgs& a, cudaStream_t st);   // 9..16
cudaError_t bwd_dispatch_c(int Sc, const BwdArgs& a, cudaStream_t st);   // 18..32
int bwd_chunks(int Sc, int n);
int64_t bwd_ctas(int Sc, int H, int W, int n);

}  // namespace nyf

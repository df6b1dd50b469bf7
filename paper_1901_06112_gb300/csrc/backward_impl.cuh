// Adjoint of the fused convolution + combine stage (backward of Eqs. (14)-(15)).
//
// Forward, per quantity q (q < n: channel f_q; q = n: the constant 1):
//   C_kq = omega * (phi_k f_q),  zeta_q = sum_k phi_k C_kq,  g_hat_c = zeta_c / eta,
//   eta = zeta_n.
// With G = dL/d g_hat:  a_c = G_c / eta (c < n),  a_n = -sum_c G_c g_hat_c / eta, so
// dL/d zeta_q = a_q.  Writing u_kq = a_q phi_k and B_kq = omega * u_kq (omega is
// symmetric, so the adjoint of the zero-padded convolution is the convolution
// itself):
//   dL/d phi_k(x) = sum_q [ a_q(x) C_kq(x) + f_q(x) B_kq(x) ]            (f_n := 1)
//   dL/d f_c(x)  += sum_k phi_k(x) B_kc(x)                     (direct image term)
//   dL/d sigma_s  = sum_kq sum_x u_kq(x) (omega' * (phi_k f_q))(x)
//                 = sum_kq sum_x (phi_k f_q)(x) (omega' * u_kq)(x),
// where omega' = d omega / d sigma_s = g' (x) g + g (x) g' with
// g'(t) = g(t) t^2 / sigma_s^3 (window radius held fixed).  The forward pass
// saves C_kq, so the backward convolves only u_kq, with g and g' together:
// vertical pass (g, g') on u, horizontal pass B = g * Mb, B' = g' * Mb + g * Mb'.
//
// One CTA per output tile holds all quantities of its pixels (up to four), so
// dL/dphi_k leaves the CTA as one plane per mode without atomics.  Per mode k
// the CTA stages phi_k once, runs the vertical pass of every quantity in one
// balanced task list, then streams phi_{k+1} in while the horizontal pass and
// the epilogue run.  Lanes of a warp own consecutive rows in the horizontal
// pass (conflict-free shared-memory reads), warps own column segments.  The
// taps come from the launch parameters (constant bank) instead of registers.
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
  const float* adj;       // (n + 1) planes of N: a_q
  const float* cbuf;      // planes C_kq, saved or recomputed: plane (k - k_begin) (n + 1) + q
  int k_begin, k_end;     // modes processed by this launch (k_end capped at the kept planes)
  int accumulate;         // add into df and sig_part (a later chunk of modes) instead of writing
  float inv2s2;           // 1 / (2 sigma_s^2)
  float inv_s3;           // 1 / sigma_s^3
  int S_true;
  int box;
  float* dphi;            // r planes of N
  int atomic_dphi;        // quantities split over several CTAs: accumulate dphi atomically
  float* df;              // N x n, direct image term
  float* sig_part;        // one sigma_s partial per CTA
  float2 taps[2 * kMaxTapRadius + 1];   // (g(z), g'(z)) for z = -S_compiled..S_compiled, zero beyond S
};

constexpr int kBwdThreads = 256;    // 8 warps; the taps live in the launch parameters (constant bank)

template <int S>
struct BwdCfg {
  static constexpr int TH = 32;                                 // = lanes: one row per lane
  static constexpr int TW = S <= 16 ? 64 : (S <= 24 ? 48 : 32);
  static constexpr int RV = 16;
  static constexpr int NQ = S <= 16 ? 4 : 2;                    // quantities per CTA
  static constexpr int RH = TW / (kBwdThreads / 32);            // columns per thread
  static constexpr int HH = TH + 2 * S;
  static constexpr int HW = TW + 2 * S;
  static constexpr int PS = HW | 1;
  static constexpr int PLANE = HH * PS;
  static constexpr int VB = TH / RV;                            // vertical row blocks
  static constexpr int VT = NQ * VB * HW;                       // vertical tasks
  static constexpr size_t smem =
      sizeof(float) * ((size_t)(NQ + 1) * PLANE + (size_t)2 * NQ * TH * PS);
  static_assert(TH == 32 && RH * (kBwdThreads / 32) == TW, "lane = row, warp = segment");
  static_assert(((NQ + 1) * PLANE) % 2 == 0, "float2 alignment of the vertical planes");
  static_assert(smem <= 227 * 1024, "shared memory budget");
};

template <int S>
__device__ __forceinline__ void bwd_stage_phi(const BwdArgs& a, float* P, int k, int ty0, int tx0) {
  using C = BwdCfg<S>;
  const int64_t base = (int64_t)k * a.N;
  if (!a.bf16) {
    const float* src = reinterpret_cast<const float*>(a.phi) + base;
    for (int e = threadIdx.x; e < C::HH * C::HW; e += kBwdThreads) {
      const int yy = e / C::HW, xx = e - yy * C::HW;
      const int gy = ty0 - S + yy, gx = tx0 - S + xx;
      const bool in = gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
      cp_async4(P + yy * C::PS + xx, in ? src + (int64_t)gy * a.W + gx : src, in);
    }
  } else {
    const __nv_bfloat16* src = reinterpret_cast<const __nv_bfloat16*>(a.phi) + base;
    for (int e = threadIdx.x; e < C::HH * C::HW; e += kBwdThreads) {
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
__global__ void __launch_bounds__(kBwdThreads, 1) k_conv_bwd(const __grid_constant__ BwdArgs a) {
  using C = BwdCfg<S>;
  constexpr int T = 2 * S + 1;
  constexpr int TH = C::TH, TW = C::TW, RV = C::RV, RH = C::RH, NQ = C::NQ;
  constexpr int HH = C::HH, HW = C::HW, PS = C::PS, PLANE = C::PLANE;
  extern __shared__ float sm[];
  float* Aq = sm;                                              // NQ adjoint planes
  float* P = Aq + NQ * PLANE;                                  // phi_k
  float2* M = reinterpret_cast<float2*>(P + PLANE);            // NQ x TH x PS: (g, g') on u
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;
  const int q0 = blockIdx.z * NQ;
  const int n = a.n;
  const int nq = min(NQ, n + 1 - q0);                          // quantities of this CTA
  const int kb = a.k_begin;
  const int r = min(a.k_end, a.state->planes);                 // modes kb <= k < r

  // adjoint planes a_q on the tile + halo (zero outside the image), then phi_0
  for (int e = tid; e < NQ * HH * HW; e += kBwdThreads) {
    const int qi = e / (HH * HW);
    const int rem = e - qi * (HH * HW);
    const int yy = rem / HW, xx = rem - yy * HW;
    const int gy = ty0 - S + yy, gx = tx0 - S + xx;
    const bool in = qi < nq && gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
    cp_async4(Aq + qi * PLANE + yy * PS + xx,
              in ? a.adj + (int64_t)(q0 + qi) * a.N + (int64_t)gy * a.W + gx : a.adj, in);
  }
  if (kb < r) bwd_stage_phi<S>(a, P, kb, ty0, tx0);
  cp_async_commit();

  // (g, g') tap pairs from the launch parameters: one packed FMA updates the g
  // and g' sums of an input
  const float2* gg = a.taps + (kMaxTapRadius - S);

  const int hy = lane, hx0 = warp * RH;
  const int y = ty0 + hy;
  const bool yin = y < a.H;
  // image channels at this thread's pixels (f_n := 1 for the denominator)
  float fc[NQ][RH];
#pragma unroll
  for (int qi = 0; qi < NQ; ++qi)
#pragma unroll
    for (int j = 0; j < RH; ++j) {
      const int q = q0 + qi, x = tx0 + hx0 + j;
      fc[qi][j] = q < n ? ((yin && x < a.W) ? a.f[((int64_t)y * a.W + x) * n + q] : 0.f) : 1.f;
    }
  float dfa[NQ][RH];
#pragma unroll
  for (int qi = 0; qi < NQ; ++qi)
#pragma unroll
    for (int j = 0; j < RH; ++j) dfa[qi][j] = 0.f;
  float sig = 0.f;

  for (int k = kb; k < r; ++k) {
    cp_async_wait<0>();
    __syncthreads();                 // phi_k (and the adjoint planes) landed; M is free
    float pc[RH];                    // phi_k at this thread's pixels
#pragma unroll
    for (int j = 0; j < RH; ++j) pc[j] = P[(hy + S) * PS + hx0 + j + S];

    // vertical pass of every quantity: (g, g') on u = a_q phi_k
    for (int task = tid; task < C::VT; task += kBwdThreads) {
      const int qi = task / (C::VB * HW);
      const int rem = task - qi * (C::VB * HW);
      const int vb = rem / HW, vx = rem - vb * HW;
      const int vy0 = vb * RV;
      if (qi < nq) {
        const float* A = Aq + qi * PLANE;
        float2 vm[RV];
#pragma unroll
        for (int j = 0; j < RV; ++j) vm[j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < RV + 2 * S; ++i) {
          const int off = (vy0 + i) * PS + vx;
          const float u = P[off] * A[off];
          const float2 uu = make_float2(u, u);
#pragma unroll
          for (int j = 0; j < RV; ++j) {
            const int t = i - j;
            if (t >= 0 && t < T) vm[j] = __ffma2_rn(gg[t], uu, vm[j]);
          }
        }
        float2* Mq = M + qi * (TH * PS);
#pragma unroll
        for (int j = 0; j < RV; ++j) Mq[(vy0 + j) * PS + vx] = vm[j];
      }
    }
    __syncthreads();                 // M complete; nobody reads P beyond this point
    if (k + 1 < r) {                 // phi_{k+1} streams in under the horizontal pass
      bwd_stage_phi<S>(a, P, k + 1, ty0, tx0);
      cp_async_commit();
    }

    float dacc[RH];
#pragma unroll
    for (int j = 0; j < RH; ++j) dacc[j] = 0.f;
#pragma unroll
    for (int qi = 0; qi < NQ; ++qi) {
      if (qi < nq) {                 // uniform over the block
        const int q = q0 + qi;
        // C_kq at this thread's pixels, saved by the forward pass
        const float* Cp = a.cbuf + ((int64_t)(k - kb) * (n + 1) + q) * a.N + (int64_t)y * a.W + tx0 + hx0;
        float cq[RH];
        if (RH % 4 == 0 && yin && tx0 + hx0 + RH <= a.W &&
            (reinterpret_cast<uintptr_t>(Cp) & 15) == 0) {
#pragma unroll
          for (int m = 0; m < RH / 4; ++m) {
            const float4 v = __ldcs(reinterpret_cast<const float4*>(Cp) + m);
            cq[4 * m] = v.x;
            cq[4 * m + 1] = v.y;
            cq[4 * m + 2] = v.z;
            cq[4 * m + 3] = v.w;
          }
        } else {
#pragma unroll
          for (int j = 0; j < RH; ++j) cq[j] = (yin && tx0 + hx0 + j < a.W) ? __ldcs(Cp + j) : 0.f;
        }
        const float2* Mq = M + qi * (TH * PS) + hy * PS + hx0;
        float2 bp[RH];               // (B, B') at this thread's pixels
#pragma unroll
        for (int j = 0; j < RH; ++j) bp[j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < RH + 2 * S; ++i) {
          const float2 m = Mq[i];
          const float2 mm = make_float2(m.x, m.x);
#pragma unroll
          for (int j = 0; j < RH; ++j) {
            const int t = i - j;
            if (t >= 0 && t < T) {
              bp[j] = __ffma2_rn(gg[t], mm, bp[j]);        // (g Mb, g' Mb)
              bp[j].y = fmaf(gg[t].x, m.y, bp[j].y);        //  + g Mb'
            }
          }
        }
        const float* Ac = Aq + qi * PLANE + (hy + S) * PS + hx0 + S;
#pragma unroll
        for (int j = 0; j < RH; ++j) {
          dacc[j] = fmaf(Ac[j], cq[j], fmaf(fc[qi][j], bp[j].x, dacc[j]));
          dfa[qi][j] = fmaf(pc[j], bp[j].x, dfa[qi][j]);
          sig = fmaf(pc[j] * fc[qi][j], bp[j].y, sig);
        }
      }
    }
    if (yin) {
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

  if (yin) {
#pragma unroll
    for (int j = 0; j < RH; ++j) {
      const int x = tx0 + hx0 + j;
      if (x < a.W) {
        const int64_t pix = (int64_t)y * a.W + x;
#pragma unroll
        for (int qi = 0; qi < NQ; ++qi)
          if (q0 + qi < n) {
            float* d = a.df + pix * n + q0 + qi;
            *d = a.accumulate ? *d + dfa[qi][j] : dfa[qi][j];
          }
      }
    }
  }
  // sigma_s partial of this CTA (fixed-order reduction)
  __shared__ float red[kBwdThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sig += __shfl_xor_sync(0xffffffffu, sig, o);
  if (lane == 0) red[warp] = sig;
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int w = 0; w < kBwdThreads / 32; ++w) s += red[w];
    const int cta = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    a.sig_part[cta] = a.accumulate ? a.sig_part[cta] + s : s;
  }
}

template <int S>
dim3 bwd_grid(int H, int W, int n) {
  using C = BwdCfg<S>;
  return dim3((W + C::TW - 1) / C::TW, (H + C::TH - 1) / C::TH, (n + 1 + C::NQ - 1) / C::NQ);
}

template <int S>
cudaError_t bwd_launch(const BwdArgs& a, cudaStream_t st) {
  using C = BwdCfg<S>;
  cudaError_t e = cudaFuncSetAttribute(k_conv_bwd<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::smem);
  if (e != cudaSuccess) return e;
  k_conv_bwd<S><<<bwd_grid<S>(a.H, a.W, a.n), kBwdThreads, C::smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t bwd_dispatch_a(int Sc, const BwdArgs& a, cudaStream_t st);   // 1..8
cudaError_t bwd_dispatch_b(int Sc, const BwdArgs& a, cudaStream_t st);   // 9..16
cudaError_t bwd_dispatch_c(int Sc, const BwdArgs& a, cudaStream_t st);   // 18..32
int bwd_chunks(int Sc, int n);
int64_t bwd_ctas(int Sc, int H, int W, int n);

}  // namespace nyf

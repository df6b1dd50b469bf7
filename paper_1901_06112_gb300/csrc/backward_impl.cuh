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
// Both taps are even functions of t and g'(0) = 0, so every pass adds the two
// inputs at +t and -t first and multiplies the sum by g(t) and by g'(t): per
// tap pair one addition and two multiply-adds instead of four multiply-adds.
// The quantities are handled in pairs (q, q+1) stored interleaved in shared
// memory, so that each of those operations is one packed FP32x2 instruction
// for two planes.
//
// One CTA per output tile holds all quantities of its pixels (up to four), so
// dL/dphi_k leaves the CTA as one plane per mode without atomics.  Per mode k
// the CTA stages phi_k once, runs the vertical pass of every quantity pair in
// one balanced task list, then streams phi_{k+1} in while the horizontal pass
// and the epilogue run.  Lanes of a warp own consecutive rows in the
// horizontal pass (conflict-free shared-memory reads), warps own column
// segments.  The taps come from the launch parameters (constant bank) instead
// of registers.
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
  int box;
  float* dphi;            // r planes of N
  int atomic_dphi;        // quantities split over two CTAs: accumulate dphi atomically
  float* df;              // N x n, direct image term
  float* sig_part;        // one sigma_s partial per CTA
  // (g(t), g(t)) and (g'(t), g'(t)) for t = 0..S_compiled, zero beyond the true radius
  float2 tg[kMaxTapRadius + 1];
  float2 td[kMaxTapRadius + 1];
  int64_t dphi_slice;     // > 0: the CTAs of quantity slice z write their own plane set at
                          // dphi + z dphi_slice (summed in a fixed order afterwards)
};

constexpr int kBwdThreads = 256;    // 8 warps; the taps live in the launch parameters (constant bank)

template <int S>
struct BwdCfg {
  static constexpr int TH = 32;                                 // = lanes: one row per lane
  static constexpr int TW = S <= 16 ? 64 : (S <= 24 ? 64 : 32);
  static constexpr int RV = 8;                                  // rows per vertical task
  static constexpr int NQ = S <= 16 ? 4 : 2;                    // quantities per CTA
  static constexpr int NP = NQ / 2;                             // quantity pairs
  static constexpr int RH = TW / (kBwdThreads / 32);            // columns per thread
  static constexpr int HH = TH + 2 * S;
  static constexpr int HW = TW + 2 * S;
  static constexpr int PS = HW | 1;     // odd row stride (in elements): conflict-free walks
  static constexpr int PLANE = HH * PS;
  static constexpr int VB = TH / RV;                            // vertical row blocks
  static constexpr int VT = NP * VB * HW;                       // vertical tasks
  // shared memory: NP interleaved adjoint pairs, phi_k, and the vertical
  // outputs (Mb, Mb') as NP interleaved pairs each
  static constexpr size_t smem =
      sizeof(float) * ((size_t)2 * NP * PLANE + (size_t)PLANE + (size_t)4 * NP * TH * PS);
  static_assert(TH == 32 && RH * (kBwdThreads / 32) == TW, "lane = row, warp = segment");
  static_assert(NQ % 2 == 0 && TH % RV == 0, "quantity pairs, whole row blocks");
  static_assert(PLANE % 2 == 0, "float2 alignment of the planes after phi");
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

// R consecutive outputs of a symmetric FIR on a plane pair: og[j] += sum over t of
// g(t) (x[j + S - t] + x[j + S + t]) and, with WITH_D, od[j] += the same with g'(t),
// from inputs x[0 .. R + 2S).  The tap loop is outermost so that the 2R
// accumulator chains interleave.
template <int S, int R, bool WITH_D>
__device__ __forceinline__ void sym_fir(const float2* x, const float2* tg, const float2* td,
                                        float2 (&og)[R], float2 (&od)[R]) {
#pragma unroll
  for (int j = 0; j < R; ++j) og[j] = __ffma2_rn(tg[0], x[j + S], og[j]);
#pragma unroll
  for (int t = 1; t <= S; ++t) {
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const float2 s = __fadd2_rn(x[j + S - t], x[j + S + t]);
      og[j] = __ffma2_rn(tg[t], s, og[j]);
      if (WITH_D) od[j] = __ffma2_rn(td[t], s, od[j]);
    }
  }
}

template <int S, bool SLICES>
__global__ void __launch_bounds__(kBwdThreads, 1) k_conv_bwd(const __grid_constant__ BwdArgs a) {
  using C = BwdCfg<S>;
  constexpr int TH = C::TH, RV = C::RV, RH = C::RH, NQ = C::NQ, NP = C::NP;
  constexpr int HH = C::HH, HW = C::HW, PS = C::PS, PLANE = C::PLANE;
  constexpr bool kEarlyC = S > 16;
  extern __shared__ float sm[];
  float2* A2 = reinterpret_cast<float2*>(sm);                  // NP pairs (a_q, a_q+1)
  float* P = sm + 2 * NP * PLANE;                              // phi_k
  float2* Mg = reinterpret_cast<float2*>(P + PLANE);           // NP x TH x PS: g on u (pairs)
  float2* Md = Mg + NP * TH * PS;                              // NP x TH x PS: g' on u (pairs)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * C::TW;
  const int q0 = blockIdx.z * NQ;
  const int n = a.n;
  const int nq = min(NQ, n + 1 - q0);                          // quantities of this CTA
  const int kb = a.k_begin;
  const int r = min(a.k_end, a.state->planes);                 // modes kb <= k < r

  // adjoint planes a_q on the tile + halo (zero outside the image and for
  // quantities beyond n), interleaved by pairs, then phi_kb
  for (int e = tid; e < NQ * HH * HW; e += kBwdThreads) {
    const int qi = e / (HH * HW);
    const int rem = e - qi * (HH * HW);
    const int yy = rem / HW, xx = rem - yy * HW;
    const int gy = ty0 - S + yy, gx = tx0 - S + xx;
    const bool in = qi < nq && gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
    float* dst = reinterpret_cast<float*>(A2 + (qi >> 1) * PLANE + yy * PS + xx) + (qi & 1);
    cp_async4(dst, in ? a.adj + (int64_t)(q0 + qi) * a.N + (int64_t)gy * a.W + gx : a.adj, in);
  }
  if (kb < r) bwd_stage_phi<S>(a, P, kb, ty0, tx0);
  cp_async_commit();

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
    __syncthreads();                 // phi_k (and the adjoint planes) landed; Mg, Md are free
    float pc[RH];                    // phi_k at this thread's pixels
#pragma unroll
    for (int j = 0; j < RH; ++j) pc[j] = P[(hy + S) * PS + hx0 + j + S];

    // C_kq of quantity qi at this thread's pixels, saved by the forward pass.  The
    // loads are issued well before their use so that their latency hides under a
    // pass: for S <= 16 before the horizontal pass of the pair, for larger radii
    // (fewer quantities per CTA) before the vertical pass.
    float cq[NQ][RH];
    auto load_c = [&](int qi, float (&c)[RH]) {
      const float* Cp =
          a.cbuf + ((int64_t)(k - kb) * (n + 1) + q0 + qi) * a.N + (int64_t)y * a.W + tx0 + hx0;
      const bool have = qi < nq;
      if (RH % 4 == 0 && have && yin && tx0 + hx0 + RH <= a.W &&
          (reinterpret_cast<uintptr_t>(Cp) & 15) == 0) {
#pragma unroll
        for (int m4 = 0; m4 < RH / 4; ++m4) {
          const float4 v = __ldcs(reinterpret_cast<const float4*>(Cp) + m4);
          c[4 * m4] = v.x;
          c[4 * m4 + 1] = v.y;
          c[4 * m4 + 2] = v.z;
          c[4 * m4 + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int j = 0; j < RH; ++j) c[j] = (have && yin && tx0 + hx0 + j < a.W) ? __ldcs(Cp + j) : 0.f;
      }
    };
    if (kEarlyC) {
#pragma unroll
      for (int qi = 0; qi < NQ; ++qi) load_c(qi, cq[qi]);
    }

    // vertical pass of every quantity pair: (g, g') on u = a_q phi_k, RV rows of one column
    for (int task = tid; task < C::VT; task += kBwdThreads) {
      const int qp = task / (C::VB * HW);
      const int rem = task - qp * (C::VB * HW);
      const int vb = rem / HW, vx = rem - vb * HW;
      const int vy0 = vb * RV;
      if (2 * qp < nq) {
        const float2* Aq = A2 + qp * PLANE;
        float2 u[RV + 2 * S];
#pragma unroll
        for (int i = 0; i < RV + 2 * S; ++i) {
          const int off = (vy0 + i) * PS + vx;
          const float p = P[off];
          const float2 av = Aq[off];
          u[i] = make_float2(p * av.x, p * av.y);
        }
        float2* mg = Mg + qp * (TH * PS) + vy0 * PS + vx;
        float2* md = Md + qp * (TH * PS) + vy0 * PS + vx;
        float2 og[RV], od[RV];
#pragma unroll
        for (int j = 0; j < RV; ++j) og[j] = od[j] = make_float2(0.f, 0.f);
        sym_fir<S, RV, true>(u, a.tg, a.td, og, od);
#pragma unroll
        for (int j = 0; j < RV; ++j) {
          mg[j * PS] = og[j];
          md[j * PS] = od[j];
        }
      }
    }
    __syncthreads();                 // Mg, Md complete; nobody reads P beyond this point
    if (k + 1 < r) {                 // phi_{k+1} streams in under the horizontal pass
      bwd_stage_phi<S>(a, P, k + 1, ty0, tx0);
      cp_async_commit();
    }

    float dacc[RH];
#pragma unroll
    for (int j = 0; j < RH; ++j) dacc[j] = 0.f;
#pragma unroll
    for (int qp = 0; qp < NP; ++qp) {
      if (2 * qp < nq) {             // uniform over the block
        if (!kEarlyC) {
          load_c(2 * qp, cq[2 * qp]);
          load_c(2 * qp + 1, cq[2 * qp + 1]);
        }
        // (B, B') of the pair at this thread's pixels: B = g * Mg, B' = g' * Mg + g * Md
        float2 bg[RH], bd[RH];
        {
          const float2* row = Mg + qp * (TH * PS) + hy * PS + hx0;
          float2 m[RH + 2 * S];
#pragma unroll
          for (int i = 0; i < RH + 2 * S; ++i) m[i] = row[i];
#pragma unroll
          for (int j = 0; j < RH; ++j) bg[j] = bd[j] = make_float2(0.f, 0.f);
          sym_fir<S, RH, true>(m, a.tg, a.td, bg, bd);
        }
        {
          const float2* row = Md + qp * (TH * PS) + hy * PS + hx0;
          float2 m[RH + 2 * S];
#pragma unroll
          for (int i = 0; i < RH + 2 * S; ++i) m[i] = row[i];
          sym_fir<S, RH, false>(m, a.tg, a.td, bd, bg);   // bg is not touched
        }
        const float2* Ac = A2 + qp * PLANE + (hy + S) * PS + hx0 + S;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int qi = 2 * qp + h;
          if (qi < nq) {             // uniform over the block
#pragma unroll
            for (int j = 0; j < RH; ++j) {
              const float b = h ? bg[j].y : bg[j].x;
              const float bp = h ? bd[j].y : bd[j].x;
              const float aq = h ? Ac[j].y : Ac[j].x;
              dacc[j] = fmaf(aq, cq[qi][j], fmaf(fc[qi][j], b, dacc[j]));
              dfa[qi][j] = fmaf(pc[j], b, dfa[qi][j]);
              sig = fmaf(pc[j] * fc[qi][j], bp, sig);
            }
          }
        }
      }
    }
    if (yin) {
      float* dst = a.dphi + (int64_t)k * a.N + (int64_t)y * a.W;
      if (SLICES) dst += blockIdx.z * a.dphi_slice;
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

template <int S, bool SLICES>
cudaError_t bwd_launch_v(const BwdArgs& a, cudaStream_t st) {
  using C = BwdCfg<S>;
  cudaError_t e = cudaFuncSetAttribute(k_conv_bwd<S, SLICES>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
  if (e != cudaSuccess) return e;
  k_conv_bwd<S, SLICES><<<bwd_grid<S>(a.H, a.W, a.n), kBwdThreads, C::smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

// the plane-set variant only where quantity slices write their own dL/dphi sets
template <int S>
cudaError_t bwd_launch(const BwdArgs& a, cudaStream_t st) {
  return a.dphi_slice > 0 ? bwd_launch_v<S, true>(a, st) : bwd_launch_v<S, false>(a, st);
}

cudaError_t bwd_dispatch_a(int Sc, const BwdArgs& a, cudaStream_t st);   // 1..8
cudaError_t bwd_dispatch_b(int Sc, const BwdArgs& a, cudaStream_t st);   // 9..16
cudaError_t bwd_dispatch_c(int Sc, const BwdArgs& a, cudaStream_t st);   // 18..32
int bwd_chunks(int Sc, int n);
int64_t bwd_ctas(int Sc, int H, int W, int n);

}  // namespace nyf

// Fused spatial convolutions + combine (Eqs. (7), (14), (15); Algorithm 1 loop).
//
// For every kept mode k and every quantity q (the n channels of f, plus the
// constant 1 for the denominator), one CTA computes on its output tile
//     C_kq = omega * (phi_k f_q)     (f_n := 1)
// as a separable FIR (vertical pass into shared memory, then horizontal pass
// into registers) and accumulates zeta_q += phi_k C_kq in registers; eta is
// the q = n accumulator.  Only g_hat = zeta / eta (or zeta and eta when the
// quantities are split over several CTAs) leaves the chip, plus, when the
// caller will run the backward pass, the K (n+1) convolved planes C_kq
// (written once here instead of being recomputed there).
//
// Zero padding outside the image is the window clipping of Eq. (1).  The taps
// g(z) = exp(-z^2 / (2 sigma_s^2)) come from the launch parameters (constant
// bank); the window radius S is a compile-time bound (taps with |z| above the
// true radius are zero) so that the register-blocked FIR loops fully unroll.
// The box window (the NLM search window) runs as running sums over the true
// radius instead: the first output of a row or column segment sums 2S+1 inputs,
// each next one adds the entering input and subtracts the leaving one.
//
// Per mode k the CTA runs two phases separated by barriers: the vertical pass of
// every quantity pair (one output buffer per pair), then, while phi_{k+1}
// streams into the phi plane, the horizontal pass and combine of every pair.
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
  int narrow;               // FP32 kernel: 32 x 64 tiles instead of 32 x 96 (S <= 16)
  float* cout;              // convolved planes C_kq for the backward pass, or NULL: plane
                            // (k - k_begin) (n + 1) + q for the modes k_begin <= k < k_end
  int k_begin, k_end;       // modes processed (k_end is capped at the kept planes)
  int c_only;               // recompute C only: no combine, nothing else is written
  float2 taps[2 * NYF_MAX_S + 1];   // (g(z), g(z)) for z = -32..32, zero beyond the true radius
};

constexpr int kConvThreads = 256;
constexpr int kMaxTapRadius = NYF_MAX_S;   // tap arrays in launch parameters cover -32..32

// Tile shapes by radius class.  TH x TW output pixels per CTA; the vertical
// pass gives each thread RV rows of one halo column, the horizontal pass RH
// columns of one output row; NQ quantities per CTA, processed in pairs with
// packed FP32x2 FMAs (one instruction, two planes).  Shared memory: NQ image
// planes, the phi plane and one vertical-pass plane pair per quantity pair.
template <int S, bool WIDE = true>
struct ConvCfg {
  static constexpr int TH = 32;
  static constexpr int TW = S <= 16 ? (WIDE ? 96 : 64) : (S <= 24 ? 48 : 64);
  static constexpr int RV = 16;
  static constexpr int RH = S <= 16 ? (WIDE ? 12 : 8) : (S <= 24 ? 6 : 8);
  static constexpr int NQ = S <= 24 ? 4 : 2;
  static constexpr int HH = TH + 2 * S;
  static constexpr int HW = TW + 2 * S;
  static constexpr int PS = HW | 1;           // odd row stride: conflict-free column/row walks
  static constexpr int PLANE = HH * PS;
  // shared memory: NQ image planes, phi_k, and the vertical pass of every quantity pair
  static constexpr size_t smem =
      sizeof(float) * ((size_t)(NQ + 1) * PLANE + (size_t)(NQ / 2) * 2 * TH * PS);
  static_assert(TH * (TW / RH) == kConvThreads, "one horizontal task per thread");
  static_assert((TH / RV) * HW <= kConvThreads, "at most one vertical task per thread and pair");
  static_assert(smem <= 227 * 1024, "shared memory budget");
};

// 4-byte asynchronous global->shared copy; src_size 0 writes a zero (used for
// pixels outside the image, i.e. the zero padding of the window).
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Stage plane k of phi (tile + halo) into P: asynchronous for float32,
// converted through registers for bfloat16.
template <int S, bool WIDE>
__device__ __forceinline__ void stage_phi(const ConvArgs& a, float* P, int k, int ty0, int tx0) {
  using C = ConvCfg<S, WIDE>;
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

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Store RH consecutive values of two planes (v[j].x to ca[j], v[j].y to cb[j]
// unless cb is NULL) for the `valid` leading columns: 16-byte streaming stores
// when the row segment is whole and aligned, else one float at a time.
template <int RH>
__device__ __forceinline__ void store_pair_row(float* ca, float* cb, const float2* v, int valid) {
  const bool vec = (RH % 4 == 0) && valid >= RH &&
                   ((reinterpret_cast<uintptr_t>(ca) | reinterpret_cast<uintptr_t>(cb)) & 15) == 0;
  if (vec) {
#pragma unroll
    for (int m = 0; m < RH / 4; ++m) {
      __stcs(reinterpret_cast<float4*>(ca) + m,
             make_float4(v[4 * m].x, v[4 * m + 1].x, v[4 * m + 2].x, v[4 * m + 3].x));
      if (cb)
        __stcs(reinterpret_cast<float4*>(cb) + m,
               make_float4(v[4 * m].y, v[4 * m + 1].y, v[4 * m + 2].y, v[4 * m + 3].y));
    }
  } else {
#pragma unroll
    for (int j = 0; j < RH; ++j)
      if (j < valid) {
        ca[j] = v[j].x;
        if (cb) cb[j] = v[j].y;
      }
  }
}

template <int S, bool WIDE>
__global__ void __launch_bounds__(kConvThreads, 1) k_conv_combine(const __grid_constant__ ConvArgs a) {
  using C = ConvCfg<S, WIDE>;
  constexpr int T = 2 * S + 1;
  constexpr int TH = C::TH, TW = C::TW, RV = C::RV, RH = C::RH, NQ = C::NQ;
  constexpr int HH = C::HH, HW = C::HW, PS = C::PS, PLANE = C::PLANE;
  constexpr int NP = NQ / 2;        // quantity pairs per CTA
  extern __shared__ float sm[];
  float* F = sm;                    // NQ image planes (tile + halo)
  float* P = F + NQ * PLANE;        // phi_k (tile + halo)
  float2* M = reinterpret_cast<float2*>(P + PLANE);   // NP vertical passes, TH x PS pairs each
  const int tid = threadIdx.x;
  const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;
  const int q0 = blockIdx.z * NQ;
  const int n = a.n;
  const int kb = a.k_begin;
  const int r = min(a.k_end, a.state->planes);   // modes kb <= k < r

  // Image planes of this CTA's quantities (zero outside the image and for the
  // denominator quantity), then phi_kb; both asynchronous.
  for (int e = tid; e < NQ * HH * HW; e += kConvThreads) {
    const int qi = e / (HH * HW);
    const int rem = e - qi * (HH * HW);
    const int yy = rem / HW, xx = rem - yy * HW;
    const int c = q0 + qi;
    const int gy = ty0 - S + yy, gx = tx0 - S + xx;
    const bool in = c < n && gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
    cp_async4(F + qi * PLANE + yy * PS + xx, in ? a.f + ((int64_t)gy * a.W + gx) * n + c : a.f, in);
  }
  if (kb < r) stage_phi<S, WIDE>(a, P, kb, ty0, tx0);
  cp_async_commit();

  const float2* g = a.taps + (kMaxTapRadius - S);   // (g, g) pairs, from the constant bank

  float2 acc[NP][RH];
#pragma unroll
  for (int pi = 0; pi < NP; ++pi)
#pragma unroll
    for (int j = 0; j < RH; ++j) acc[pi][j] = f2(0.f, 0.f);

  const int hy = tid / (TW / RH), hx0 = (tid % (TW / RH)) * RH;
  const int vx = tid % HW, vy0 = (tid / HW) * RV;
  const bool vactive = tid < (TH / RV) * HW;     // one vertical task per thread and pair (or none)

  for (int k = kb; k < r; ++k) {
    cp_async_wait<0>();
    __syncthreads();                 // phi_k (and the image planes) landed; M is free
    float pc[RH];                    // phi_k at this thread's output pixels
#pragma unroll
    for (int j = 0; j < RH; ++j) pc[j] = P[(hy + S) * PS + hx0 + j + S];
    // vertical pass of every quantity pair
#pragma unroll
    for (int pi = 0; pi < NP; ++pi) {
      const int qa = q0 + 2 * pi, qb = qa + 1;
      if (qa <= n && vactive) {      // qa uniform over the block
        // pair member x: image channel qa (or 1 if qa == n); member y: channel
        // qb (1 if qb == n, 0 if qb > n)
        const float* Fa = F + (2 * pi) * PLANE;
        const float* Fb = Fa + PLANE;
        const bool a_den = qa == n, b_den = qb == n, b_none = qb > n;
        float2 va[RV];
        auto vin = [&](int i) {     // (phi f_qa, phi f_qb) at halo row vy0 + i of column vx
          const int off = (vy0 + i) * PS + vx;
          const float p = P[off];
          return f2(a_den ? p : p * Fa[off], b_den ? p : (b_none ? 0.f : p * Fb[off]));
        };
        if (a.box) {
          // box window: running sums over the true radius (2 operations per output
          // after the first; the halo is that of the compiled radius S)
          const int lo = S - a.S_true, T1 = 2 * a.S_true + 1;
          float2 run = f2(0.f, 0.f);
          for (int i = lo; i < lo + T1; ++i) run = __ffma2_rn(f2(1.f, 1.f), vin(i), run);
          va[0] = run;
#pragma unroll
          for (int j = 1; j < RV; ++j) {
            run = __ffma2_rn(f2(1.f, 1.f), vin(j + lo + T1 - 1), run);
            run = __ffma2_rn(f2(-1.f, -1.f), vin(j - 1 + lo), run);
            va[j] = run;
          }
        } else {
#pragma unroll
          for (int j = 0; j < RV; ++j) va[j] = f2(0.f, 0.f);
#pragma unroll
          for (int i = 0; i < RV + 2 * S; ++i) {
            const float2 v = vin(i);
#pragma unroll
            for (int j = 0; j < RV; ++j) {
              const int t = i - j;
              if (t >= 0 && t < T) va[j] = __ffma2_rn(g[t], v, va[j]);
            }
          }
        }
        float2* Mp = M + pi * (TH * PS);
#pragma unroll
        for (int j = 0; j < RV; ++j) Mp[(vy0 + j) * PS + vx] = va[j];
      }
    }
    __syncthreads();                 // M complete; nobody reads P beyond this point
    if (k + 1 < r) {                 // phi_{k+1} streams in under the horizontal pass
      stage_phi<S, WIDE>(a, P, k + 1, ty0, tx0);
      cp_async_commit();
    }
#pragma unroll
    for (int pi = 0; pi < NP; ++pi) {
      const int qa = q0 + 2 * pi, qb = qa + 1;
      if (qa <= n) {                 // uniform over the block
        const bool b_none = qb > n;
        const float2* mr = M + pi * (TH * PS) + hy * PS + hx0;
        float2 hb[RH];
        if (a.box) {                 // running sums along the row
          const int lo = S - a.S_true, T1 = 2 * a.S_true + 1;
          float2 run = f2(0.f, 0.f);
          for (int i = lo; i < lo + T1; ++i) run = __ffma2_rn(f2(1.f, 1.f), mr[i], run);
          hb[0] = run;
#pragma unroll
          for (int j = 1; j < RH; ++j) {
            run = __ffma2_rn(f2(1.f, 1.f), mr[j + lo + T1 - 1], run);
            run = __ffma2_rn(f2(-1.f, -1.f), mr[j - 1 + lo], run);
            hb[j] = run;
          }
        } else {
#pragma unroll
          for (int j = 0; j < RH; ++j) hb[j] = f2(0.f, 0.f);
#pragma unroll
          for (int i = 0; i < RH + 2 * S; ++i) {
            const float2 v = mr[i];
#pragma unroll
            for (int j = 0; j < RH; ++j) {
              const int t = i - j;
              if (t >= 0 && t < T) hb[j] = __ffma2_rn(g[t], v, hb[j]);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < RH; ++j) acc[pi][j] = __ffma2_rn(f2(pc[j], pc[j]), hb[j], acc[pi][j]);
        if (a.cout && ty0 + hy < a.H) {          // keep C_kq for the backward pass
          float* ca = a.cout + ((int64_t)(k - kb) * (n + 1) + qa) * a.N + (int64_t)(ty0 + hy) * a.W + tx0 + hx0;
          store_pair_row<RH>(ca, b_none ? nullptr : ca + a.N, hb, a.W - (tx0 + hx0));
        }
      }
    }
  }
  cp_async_wait<0>();
  if (a.c_only) return;

  // Epilogue: g_hat = zeta / eta (fused) or zeta, eta to memory (split).
  const int y = ty0 + hy;
  const bool fused = (q0 == 0) && (n + 1 <= NQ);
#pragma unroll
  for (int j = 0; j < RH; ++j) {
    const int x = tx0 + hx0 + j;
    if (y < a.H && x < a.W) {
      const int64_t pix = (int64_t)y * a.W + x;
      float v[NQ];
#pragma unroll
      for (int pi = 0; pi < NP; ++pi) {
        v[2 * pi] = acc[pi][j].x;
        v[2 * pi + 1] = acc[pi][j].y;
      }
      if (fused) {
        float eta = 0.f;
#pragma unroll
        for (int qi = 0; qi < NQ; ++qi)
          if (qi == n) eta = v[qi];
#pragma unroll
        for (int qi = 0; qi < NQ; ++qi)
          if (qi < n) a.out[pix * n + qi] = v[qi] / eta;
        a.eta[pix] = eta;
        if (!(eta > a.eta_thr)) atomicAdd(&a.state_rw->eta_small, 1ull);
      } else {
#pragma unroll
        for (int qi = 0; qi < NQ; ++qi) {
          const int q = q0 + qi;
          if (q < n) a.zeta[pix * n + q] = v[qi];
          else if (q == n) a.eta[pix] = v[qi];
        }
      }
    }
  }
}

template <int S>
cudaError_t conv_launch(const ConvArgs& a, cudaStream_t st) {
  // the narrow tile exists for S <= 16 only; it is chosen by conv_tile == NYF_TILE_NARROW
  if (S <= 16 && a.narrow) {
    using C = ConvCfg<S, false>;
    cudaError_t e = cudaFuncSetAttribute(k_conv_combine<S, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.W + C::TW - 1) / C::TW, (a.H + C::TH - 1) / C::TH, (a.n + 1 + C::NQ - 1) / C::NQ);
    k_conv_combine<S, false><<<grid, kConvThreads, C::smem, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
  }
  using C = ConvCfg<S, true>;
  cudaError_t e = cudaFuncSetAttribute(k_conv_combine<S, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.W + C::TW - 1) / C::TW, (a.H + C::TH - 1) / C::TH, (a.n + 1 + C::NQ - 1) / C::NQ);
  k_conv_combine<S, true><<<grid, kConvThreads, C::smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

// Per-file dispatchers (each instantiates a range of compile-time radii).
cudaError_t conv_dispatch_a(int Sc, const ConvArgs& a, cudaStream_t st);   // 1..8
cudaError_t conv_dispatch_b(int Sc, const ConvArgs& a, cudaStream_t st);   // 9..16
cudaError_t conv_dispatch_c(int Sc, const ConvArgs& a, cudaStream_t st);   // 18..32
bool conv_split(int S, int n);   // true when quantities are split over CTAs

}  // namespace nyf

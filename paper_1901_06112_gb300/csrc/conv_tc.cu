// BF16 tensor-core (tcgen05) version of the fused convolution + combine
// (Eqs. (7), (14), (15)), used for the BF16 precision path with n <= 3
// channels and window radius <= 16.
//
// One CTA owns a 32-row x 128-column output tile; TMEM lane x' holds output
// column x = 127 - x' (columns are reversed, see below).  Per mode k and
// quantity q (q < n: channel f_q; q = n: the constant 1) the separable FIR is
// two products on the tensor cores, BF16 operands and FP32 accumulation in
// tensor memory:
//   horizontal  D1 = Gh' Q^T   (128 x HH, K = HW halo columns)
//   vertical    D2 = D1 Gv'^T  (128 x 32, K = HH halo rows)
// with Q = bf16(phi_k f_q) on the tile + halo (HH = 32 + 2 SB rows, HW = 128 +
// 2 SB columns; phi and f staged in FP32, zero outside the image: the window
// clipping of Eq. (1)).  The taps and D1 enter as bf16 hi + lo pairs
// (x = bf16(x) + bf16(x - bf16(x)), lo x lo dropped), which keeps their
// rounding (systematic for the taps) out of the result; D1's pair lives in
// tensor memory as the A operand of the vertical product.  D2 is C_kq
// transposed; zeta_q += phi_k C_kq accumulates in tensor memory with FP32 phi
// and g_hat = zeta / eta leaves at the end.
//
// The band matrices Gh[x][c] = g(c - x - SB) and Gv[y][r] = g(r - y - SB) are
// Toeplitz.  With the output index reversed (x' = 127 - x, y' = 31 - y), the
// 8 x 8 core matrix (i, j) of either one depends only on i + j, so each is
// stored as one strip of core matrices and described with equal leading and
// stride byte offsets (128 B): 4.5 KB instead of 40 KB of shared memory.
//
// Pipeline over the steps t = (k, q): warps 4-7 build Q(t + 1) while the
// tensor core runs the products of step t and warps 0-3 (the TMEM lane
// owners) convert D1 and run the epilogue; one thread issues the MMAs.
#include "conv_impl.cuh"
#include "umma.cuh"

namespace nyf {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTH = 32;          // output rows per tile (columns of D2)
constexpr int kTW = 128;         // output columns per tile (TMEM lanes)
constexpr int kMaxF = 3;         // image channels staged in shared memory
constexpr uint32_t kWait = 1u << 20;   // mbarrier polls before giving up
// TMEM columns: D1 [0, 64), D2 [64, 96), zeta_q [96 + 32 q, ...), A2 hi/lo pairs
constexpr uint32_t kD1 = 0, kD2 = 64, kZeta = 96, kA2H = 224, kA2L = 256, kTmemCols = 512;

template <int SB>
struct TcCfg {
  static constexpr int HH = kTH + 2 * SB;
  static constexpr int HW = kTW + 2 * SB;
  static_assert(HH % 16 == 0 && HW % 16 == 0 && HH <= 64, "MMA shapes");
  static constexpr int PSF = HW + 4;                         // FP32 plane row stride (floats)
  static constexpr int FPLANE = HH * PSF * 4;                // one FP32 halo plane
  static constexpr int QPLANE = HH * HW * 2;                 // one bf16 halo plane, K-major
  static constexpr int STRIP1 = (kTW / 8 + HW / 8) * 128;    // Gh' strip
  static constexpr int STRIP2 = (kTH / 8 + HH / 8) * 128;    // Gv' strip
  static constexpr int OFF_F = 0;
  static constexpr int OFF_P = OFF_F + kMaxF * FPLANE;
  static constexpr int OFF_Q = OFF_P + FPLANE;               // two buffers
  static constexpr int OFF_S1H = OFF_Q + 2 * QPLANE;         // taps = hi + lo
  static constexpr int OFF_S1L = OFF_S1H + STRIP1;
  static constexpr int OFF_S2H = OFF_S1L + STRIP1;
  static constexpr int OFF_S2L = OFF_S2H + STRIP2;
  static constexpr int SMEM = OFF_S2L + STRIP2;
  static_assert(SMEM <= 226 * 1024, "shared memory budget");
};

__device__ __forceinline__ float tap_at(const ConvArgs& a, int z) {
  return (z < -kMaxTapRadius || z > kMaxTapRadius) ? 0.f : a.taps[kMaxTapRadius + z].x;
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Asynchronous copy of the halo of one FP32 plane (element p of the image at
// src[p * stride]) into a row-major shared plane, zero outside the image.
template <int SB>
__device__ __forceinline__ void stage_fp32(float* dst, const float* src, int stride, int ty0,
                                           int tx0, int H, int W, int first, int step) {
  using C = TcCfg<SB>;
  for (int e = first; e < C::HH * C::HW; e += step) {
    const int r = e / C::HW, c = e - r * C::HW;
    const int gy = ty0 - SB + r, gx = tx0 - SB + c;
    const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
    cp_async4(dst + r * C::PSF + c, in ? src + ((int64_t)gy * W + gx) * stride : src, in);
  }
}

// Q = bf16(P * F) (F == nullptr: Q = bf16(P)) into the K-major layout, by the
// `count` threads starting at thread `first`.
template <int SB>
__device__ __forceinline__ void build_q(unsigned char* Q, const float* P, const float* F, int first,
                                        int count) {
  using C = TcCfg<SB>;
  constexpr int CH = C::HW / 8;
  for (int e = (int)threadIdx.x - first; e < C::HH * CH; e += count) {
    const int r = e / CH, c8 = (e - r * CH) * 8;
    const float4* p = reinterpret_cast<const float4*>(P + r * C::PSF + c8);
    float4 u = p[0], w = p[1];
    if (F) {
      const float4* f = reinterpret_cast<const float4*>(F + r * C::PSF + c8);
      const float4 fu = f[0], fw = f[1];
      u.x *= fu.x; u.y *= fu.y; u.z *= fu.z; u.w *= fu.w;
      w.x *= fw.x; w.y *= fw.y; w.z *= fw.z; w.w *= fw.w;
    }
    *reinterpret_cast<uint4*>(Q + umma::kmajor_offset(r, c8, C::HW)) =
        make_uint4(pack2(u.x, u.y), pack2(u.z, u.w), pack2(w.x, w.y), pack2(w.z, w.w));
  }
}

// Named barrier among the 128 builder threads (warps 4-7).
__device__ __forceinline__ void builders_sync() { asm volatile("bar.sync 1, 128;\n" ::: "memory"); }

template <int SB>
__global__ void __launch_bounds__(kTcThreads, 1) k_conv_tc(const __grid_constant__ ConvArgs a) {
  using C = TcCfg<SB>;
  constexpr int HH = C::HH, HW = C::HW;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mbar_h, mbar_v;
  __shared__ uint32_t tslot;
  float* F = reinterpret_cast<float*>(sm + C::OFF_F);
  float* P = reinterpret_cast<float*>(sm + C::OFF_P);
  unsigned char* Q = sm + C::OFF_Q;
  unsigned char* S1H = sm + C::OFF_S1H;
  unsigned char* S1L = sm + C::OFF_S1L;
  unsigned char* S2H = sm + C::OFF_S2H;
  unsigned char* S2L = sm + C::OFF_S2L;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ty0 = blockIdx.y * kTH, tx0 = blockIdx.x * kTW;
  const int n = a.n;
  const int nq = n + 1;                          // all quantities in this CTA (n <= 3)
  const int r = a.state->planes;
  const int T = r * nq;                          // steps (k, q)
  const float* phi = reinterpret_cast<const float*>(a.phi);
  const bool epi = warp < 4;                     // warps 0-3: TMEM lanes 0-127
  const bool bld = !epi;                         // warps 4-7: Q builders

  // image channels and phi_0 (asynchronous), band strips (hi and lo parts)
  for (int c = 0; c < n; ++c)
    stage_fp32<SB>(F + c * (C::FPLANE / 4), a.f + c, n, ty0, tx0, a.H, a.W, tid, kTcThreads);
  if (r > 0) stage_fp32<SB>(P, phi, 1, ty0, tx0, a.H, a.W, tid, kTcThreads);
  cp_async_commit();
  for (int e = tid; e < C::STRIP1 / 2; e += kTcThreads) {
    const int s = e >> 6, a8 = (e >> 3) & 7, b8 = e & 7;
    const float g = tap_at(a, 8 * s + a8 + b8 - (kTW - 1) - SB);
    const __nv_bfloat16 h = __float2bfloat16(g);
    reinterpret_cast<__nv_bfloat16*>(S1H)[e] = h;
    reinterpret_cast<__nv_bfloat16*>(S1L)[e] = __float2bfloat16(g - __bfloat162float(h));
  }
  for (int e = tid; e < C::STRIP2 / 2; e += kTcThreads) {
    const int s = e >> 6, a8 = (e >> 3) & 7, b8 = e & 7;
    const float g = tap_at(a, 8 * s + a8 + b8 - (kTH - 1) - SB);
    const __nv_bfloat16 h = __float2bfloat16(g);
    reinterpret_cast<__nv_bfloat16*>(S2H)[e] = h;
    reinterpret_cast<__nv_bfloat16*>(S2L)[e] = __float2bfloat16(g - __bfloat162float(h));
  }
  if (warp == 0) umma::tmem_alloc(&tslot, kTmemCols);
  if (tid == 0) {
    umma::mbar_init(&mbar_h, 1);
    umma::mbar_init(&mbar_v, 1);
    umma::fence_mbar_init();
  }
  cp_async_wait<0>();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tbase = tslot;
  const uint32_t tlane = (uint32_t)(32 * (warp & 3)) << 16;   // this warp's TMEM lane quarter
  const int xp = 32 * (warp & 3) + lane;                      // TMEM lane of an epilogue thread
  const int xo = tx0 + (kTW - 1) - xp;                        // its output column
  if (epi) {                                                  // zeta = 0
    float z[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) z[i] = 0.f;
    for (int c = 0; c < 4 * kTH; c += 32) umma::tmem_st32(tbase + tlane + kZeta + c, z);
  }
  const uint32_t idesc1 = umma::idesc_bf16(128, HH), idesc2 = umma::idesc_bf16(128, kTH);
  const uint32_t sh1 = umma::smem_u32(S1H), sl1 = umma::smem_u32(S1L);
  const uint32_t sh2 = umma::smem_u32(S2H), sl2 = umma::smem_u32(S2L);
  const uint32_t qaddr = umma::smem_u32(Q);

  auto issue_h = [&](int t) {           // D1 = Gh' Q(t)^T, taps hi + lo
    const uint32_t b = qaddr + (uint32_t)((t & 1) * C::QPLANE);
    for (int ks = 0; ks < HW / 16; ++ks) {
      const uint64_t bd = umma::sdesc(b + 256 * ks, 128, HW * 16);
      umma::mma_bf16(tbase + kD1, umma::sdesc(sh1 + 256 * ks, 128, 128), bd, idesc1, ks > 0);
      umma::mma_bf16(tbase + kD1, umma::sdesc(sl1 + 256 * ks, 128, 128), bd, idesc1, 1);
    }
    umma::commit(&mbar_h);
  };
  auto issue_v = [&]() {                // D2 = (A2H + A2L)(G_hi + G_lo)^T, lo x lo dropped
    for (int ks = 0; ks < HH / 16; ++ks) {
      const uint64_t gh = umma::sdesc(sh2 + 256 * ks, 128, 128);
      umma::mma_bf16_ta(tbase + kD2, tbase + kA2H + 8 * ks, gh, idesc2, ks > 0);
      umma::mma_bf16_ta(tbase + kD2, tbase + kA2H + 8 * ks, umma::sdesc(sl2 + 256 * ks, 128, 128),
                        idesc2, 1);
      umma::mma_bf16_ta(tbase + kD2, tbase + kA2L + 8 * ks, gh, idesc2, 1);
    }
    umma::commit(&mbar_v);
  };

  int ok = 1, stuck_h = 0, stuck_v = 0;
  uint32_t ph_h = 0, ph_v = 0;
  float pc[kTH];                        // phi_k at an epilogue thread's pixels (FP32)
  // prologue: Q(0) by everyone, then the first horizontal product
  if (T > 0) {
    build_q<SB>(Q, P, n > 0 ? F : nullptr, 0, kTcThreads);
    umma::fence_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (tid == 0) issue_h(0);
  }
  int k_loaded = 0;                     // mode whose phi is in P (builders' view)
  for (int t = 0; t < T; ++t) {
    const int k = t / nq, q = t - k * nq;
    // builders: Q(t + 1) into the other buffer (its last reader, the horizontal
    // product of step t - 1, completed before the previous barrier)
    if (bld && t + 1 < T) {
      const int k1 = (t + 1) / nq, q1 = (t + 1) - k1 * nq;
      if (k1 != k_loaded) {             // phi_{k1}: P's last reader was the build of step t
        builders_sync();
        stage_fp32<SB>(P, phi + (int64_t)k1 * a.N, 1, ty0, tx0, a.H, a.W, tid - 128, 128);
        cp_async_commit();
        cp_async_wait<0>();
        builders_sync();
        k_loaded = k1;
      }
      build_q<SB>(Q + ((t + 1) & 1) * C::QPLANE, P, q1 < n ? F + q1 * (C::FPLANE / 4) : nullptr,
                  128, 128);
      umma::fence_async_smem();
    }
    if (epi) {
      if (q == 0) {                     // phi_k at this thread's pixels, FP32, from memory
#pragma unroll
        for (int yp = 0; yp < kTH; ++yp) {
          const int y = ty0 + (kTH - 1) - yp;
          pc[yp] = (y < a.H && xo < a.W) ? __ldg(phi + (int64_t)k * a.N + (int64_t)y * a.W + xo) : 0.f;
        }
      }
      // D1(t) -> A2 hi/lo pairs in TMEM
      if (!umma::mbar_wait(&mbar_h, ph_h, kWait)) { ok = 0; stuck_h = 1; }
      ph_h ^= 1;
      umma::fence_after_sync();
#pragma unroll
      for (int c0 = 0; c0 < HH; c0 += 32) {
        float v[32], hi[16], lo[16];
        umma::tmem_ld32(tbase + tlane + kD1 + c0, v);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * u], v[2 * u + 1]);
          const float2 hf = __bfloat1622float2(h);
          hi[u] = __uint_as_float(*reinterpret_cast<const uint32_t*>(&h));
          lo[u] = __uint_as_float(pack2(v[2 * u] - hf.x, v[2 * u + 1] - hf.y));
        }
        umma::tmem_st16(tbase + tlane + kA2H + c0 / 2, hi);
        umma::tmem_st16(tbase + tlane + kA2L + c0 / 2, lo);
      }
    }
    umma::fence_before_sync();
    if (!__syncthreads_and(ok)) break;  // A2(t) in TMEM, Q(t + 1) in shared memory
    umma::fence_after_sync();
    if (tid == 0) {
      issue_v();
      if (t + 1 < T) issue_h(t + 1);    // D1 was read completely before the barrier
    }
    if (epi) {                          // zeta_q += phi_k C_kq; C_kq to memory if kept
      if (!umma::mbar_wait(&mbar_v, ph_v, kWait)) { ok = 0; stuck_v = 1; }
      ph_v ^= 1;
      umma::fence_after_sync();
      float cv[32], zv[32];
      umma::tmem_ld32(tbase + tlane + kD2, cv);
      umma::tmem_ld32(tbase + tlane + kZeta + 32 * q, zv);
#pragma unroll
      for (int i = 0; i < 32; ++i) zv[i] = fmaf(pc[i], cv[i], zv[i]);
      umma::tmem_st32(tbase + tlane + kZeta + 32 * q, zv);
      if (a.cout && xo < a.W) {
        float* cq = a.cout + ((int64_t)k * (n + 1) + q) * a.N + xo;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int y = ty0 + (kTH - 1) - i;
          if (y < a.H) __stcs(cq + (int64_t)y * a.W, cv[i]);
        }
      }
    }
    umma::fence_before_sync();
    if (!__syncthreads_and(ok)) break;  // D2 read; the vertical product of step t done
    umma::fence_after_sync();
  }
  const int all_ok = __syncthreads_and(ok);

  // g_hat = zeta / eta at this lane's pixels (TMEM loads by whole warps; only
  // the stores depend on the lane)
  if (epi && all_ok && T > 0) {
    float zs[4][32];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < nq) umma::tmem_ld32(tbase + tlane + kZeta + 32 * q, zs[q]);
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int y = ty0 + (kTH - 1) - i;
      if (y < a.H && xo < a.W) {
        const int64_t pix = (int64_t)y * a.W + xo;
        float eta = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q == n) eta = zs[q][i];
#pragma unroll
        for (int q = 0; q < kMaxF; ++q)
          if (q < n) a.out[pix * n + q] = zs[q][i] / eta;
        a.eta[pix] = eta;
        if (!(eta > a.eta_thr)) atomicAdd(&a.state_rw->eta_small, 1ull);
      }
    }
  }
  if (tid == 0 && !all_ok) set_status(a.state_rw, NYF_ERR_TIMEOUT);
  // after a timeout, wait (bounded) for the products that did not report before freeing TMEM
  if (epi && !all_ok) {
    if (stuck_h) umma::mbar_wait(&mbar_h, ph_h ^ 1, kWait);
    if (stuck_v) umma::mbar_wait(&mbar_v, ph_v ^ 1, kWait);
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tbase, kTmemCols);
}

template <int SB>
cudaError_t tc_launch(const ConvArgs& a, cudaStream_t st) {
  using C = TcCfg<SB>;
  cudaError_t e = cudaFuncSetAttribute(k_conv_tc<SB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       C::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid((a.W + kTW - 1) / kTW, (a.H + kTH - 1) / kTH, 1);
  k_conv_tc<SB><<<grid, kTcThreads, C::SMEM, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

// Tensor-core path: n <= 3 channels, window radius <= 16 (else not supported).
bool conv_tc_supported(int S, int n) { return S <= 16 && n <= kMaxF; }

cudaError_t conv_tc_dispatch(const ConvArgs& a, cudaStream_t st) {
  if (a.n > kMaxF || a.bf16) return cudaErrorNotSupported;
  if (a.S_true <= 8) return tc_launch<8>(a, st);
  if (a.S_true <= 16) return tc_launch<16>(a, st);
  return cudaErrorNotSupported;
}

}  // namespace nyf

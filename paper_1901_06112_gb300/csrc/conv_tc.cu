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
// 2 SB columns; phi staged in FP32, f in bf16, zero outside the image: the
// window clipping of Eq. (1)).  The taps and D1 enter as bf16 hi + lo pairs
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
// Warp-specialised pipeline over the steps t = (k, q), every hand-off through
// an mbarrier and a two-slot ring:
//   warps 0-3   build Q(t) in shared memory (and stream phi_{k+1} in),
//   warp  12    issues the horizontal products D1(t) = Gh' Q(t)^T (one thread),
//   warp  13    issues the vertical products D2(t) from A2(t) (one thread),
//   warps 4-7   read D1(t) from tensor memory and write its bf16 pair A2(t),
//   warps 8-11  read D2(t), accumulate zeta and write C_kq if it is kept.
#include "conv_impl.cuh"
#include "umma.cuh"

namespace nyf {
namespace {

constexpr int kTcWarps = 14;
constexpr int kTcThreads = 32 * kTcWarps;
constexpr int kTH = 32;          // output rows per tile (columns of D2)
constexpr int kTW = 128;         // output columns per tile (TMEM lanes)
constexpr int kMaxF = 3;         // image channels staged in shared memory
constexpr uint32_t kWait = 1u << 20;   // mbarrier polls before giving up (each up to 1 us)
// TMEM columns: D1 [0, 64), D2 slots [64, 128), zeta_q [128 + 32 q, 256), A2 (hi 32 +
// lo 32) [256, 320), the horizontal band matrix Gh' as the A operand (hi, lo: HW / 2
// columns each) [320, 320 + HW)
constexpr uint32_t kD1 = 0, kD2 = 64, kZeta = 128, kA2 = 256, kGH = 320, kTmemCols = 512;

template <int SB>
struct TcCfg {
  static constexpr int HH = kTH + 2 * SB;
  static constexpr int HW = kTW + 2 * SB;
  static_assert(HH % 16 == 0 && HW % 16 == 0 && HH <= 64, "MMA shapes");
  static_assert(kGH + HW <= kTmemCols, "tensor memory budget");
  static constexpr int PSF = HW + 4;                         // FP32 phi plane row stride (floats)
  static constexpr int PPLANE = HH * PSF * 4;                // one FP32 phi halo plane
  static constexpr int FSB = HW + 8;                         // bf16 image plane row stride
  static constexpr int FPLANE = HH * FSB * 2;                // one bf16 image halo plane
  static constexpr int QPLANE = HH * HW * 2;                 // one bf16 Q plane, K-major
  static constexpr int STRIP2 = (kTH / 8 + HH / 8) * 128;    // Gv' strip
  static constexpr int OFF_P = 0;                            // two phi buffers
  static constexpr int OFF_F = OFF_P + 2 * PPLANE;
  static constexpr int OFF_Q = OFF_F + kMaxF * FPLANE;       // two Q slots
  static constexpr int OFF_S2H = OFF_Q + 2 * QPLANE;         // vertical taps = hi + lo
  static constexpr int OFF_S2L = OFF_S2H + STRIP2;
  static constexpr int OFF_PC = OFF_S2L + STRIP2;            // phi_k at the tile pixels, [y'][x']
  static constexpr int SMEM = OFF_PC + kTH * kTW * 4;
  static_assert(SMEM <= 225 * 1024, "shared memory budget");
};

// mbarriers of the rings (two slots: slot s = t & 1, use u = t >> 1 completes phase
// u; one slot: step t completes phase t)
struct Bars {
  uint64_t q_full[2], q_empty[2];     // Q slot built / consumed by the horizontal product
  uint64_t d1_full, d1_empty;         // D1 written / read by the converters (one slot)
  uint64_t a2_full, a2_empty;         // A2 written / consumed by the vertical product (one slot)
  uint64_t gh_ready;                  // Gh' written to tensor memory
  uint64_t d2_full[2], d2_empty[2];   // D2 slot written / read by the epilogue
  uint64_t pc_done[2];                // phi buffer's tile pixels copied by the epilogue
  uint64_t phi_ready[2];              // phi_k has landed in buffer k & 1 (builders waited for it)
  uint64_t drain_h, drain_v;          // all products of an issuer complete (end of the kernel)
};

// g(z) from the shared copy of the taps (zero beyond the compiled radius range).
__device__ __forceinline__ float tap_at(const float* taps, int z) {
  return (z < -kMaxTapRadius || z > kMaxTapRadius) ? 0.f : taps[kMaxTapRadius + z];
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(umma::smem_u32(b)) : "memory");
}

// Named barrier among the 128 builder threads (warps 0-3), and the same
// barrier as an AND vote (every builder gets the same result).
__device__ __forceinline__ void builders_sync() { asm volatile("bar.sync 1, 128;\n" ::: "memory"); }
__device__ __forceinline__ bool builders_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, 1, 128, p;\n"
      "selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}

// Asynchronous copy of the halo of phi plane k into a row-major FP32 buffer
// (zero outside the image), by the 128 builders.  With W % 4 == 0 every
// 4-column chunk of a halo row lies wholly inside or outside the image (the
// halo starts at a multiple of 4) and moves as one 16-byte copy.
template <int SB>
__device__ __forceinline__ void stage_phi(float* dst, const float* src, int ty0, int tx0, int H, int W,
                                          int bt) {
  using C = TcCfg<SB>;
  if ((W & 3) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    constexpr int CH = C::HW / 4;
#pragma unroll 4
    for (int e = bt; e < C::HH * CH; e += 128) {
      const int r = e / CH, c4 = (e - r * CH) * 4;
      const int gy = ty0 - SB + r, gx = tx0 - SB + c4;
      const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
      cp_async16(dst + r * C::PSF + c4, in ? src + (int64_t)gy * W + gx : src, in);
    }
  } else {
    for (int e = bt; e < C::HH * C::HW; e += 128) {
      const int r = e / C::HW, c = e - r * C::HW;
      const int gy = ty0 - SB + r, gx = tx0 - SB + c;
      const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
      cp_async4(dst + r * C::PSF + c, in ? src + (int64_t)gy * W + gx : src, in);
    }
  }
}

// Row x' of the horizontal band matrix Gh' (this thread's TMEM lane) as bf16
// hi/lo pairs: element c = g(c - x - SB), x = 127 - x'.
template <int SB>
__device__ __noinline__ void write_gh(const float* taps, uint32_t tlane_base, int xq) {
  constexpr int HW = TcCfg<SB>::HW;
#pragma unroll 1
  for (int c0 = 0; c0 < HW; c0 += 32) {
    float hv[16], lv[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int c = c0 + 2 * i;
      const float g0 = tap_at(taps, c - xq - SB), g1 = tap_at(taps, c + 1 - xq - SB);
      const __nv_bfloat162 h = __floats2bfloat162_rn(g0, g1);
      const float2 hf = __bfloat1622float2(h);
      hv[i] = __uint_as_float(*reinterpret_cast<const uint32_t*>(&h));
      lv[i] = __uint_as_float(pack2(g0 - hf.x, g1 - hf.y));
    }
    umma::tmem_st16x2(tlane_base + kGH + c0 / 2, tlane_base + kGH + HW / 2 + c0 / 2, hv, lv);
  }
}

template <int SB>
__global__ void __launch_bounds__(kTcThreads, 1) k_conv_tc(const __grid_constant__ ConvArgs a) {
  using C = TcCfg<SB>;
  constexpr int HH = C::HH, HW = C::HW;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ Bars bars;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  __shared__ float taps[2 * kMaxTapRadius + 1];
  float* P = reinterpret_cast<float*>(sm + C::OFF_P);
  __nv_bfloat16* F = reinterpret_cast<__nv_bfloat16*>(sm + C::OFF_F);
  unsigned char* Q = sm + C::OFF_Q;
  unsigned char* S2H = sm + C::OFF_S2H;
  unsigned char* S2L = sm + C::OFF_S2L;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ty0 = blockIdx.y * kTH, tx0 = blockIdx.x * kTW;
  const int n = a.n;
  const int nq = n + 1;                          // all quantities in this CTA (n <= 3)
  const int r = a.state->planes;
  const int T = r * nq;                          // steps (k, q)
  const float* phi = reinterpret_cast<const float*>(a.phi);

  // ---- setup: taps, image channels (bf16), phi_0 and phi_1, band strips, barriers, TMEM
  for (int e = tid; e < 2 * kMaxTapRadius + 1; e += kTcThreads) taps[e] = a.taps[e].x;
  __syncthreads();
  for (int e = tid; e < n * HH * HW; e += kTcThreads) {
    const int c = e / (HH * HW), rem = e - c * (HH * HW);
    const int rr = rem / HW, cc = rem - rr * HW;
    const int gy = ty0 - SB + rr, gx = tx0 - SB + cc;
    const float v = (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W)
                        ? __ldg(a.f + ((int64_t)gy * a.W + gx) * n + c) : 0.f;
    F[c * (C::FPLANE / 2) + rr * C::FSB + cc] = __float2bfloat16(v);
  }
  if (warp < 4) {
    for (int kk = 0; kk < 2 && kk < r; ++kk)
      stage_phi<SB>(P + kk * (C::PPLANE / 4), phi + (int64_t)kk * a.N, ty0, tx0, a.H, a.W, tid);
    cp_async_commit();
  }
  for (int e = tid; e < C::STRIP2 / 2; e += kTcThreads) {
    const int s = e >> 6, a8 = (e >> 3) & 7, b8 = e & 7;
    const float g = tap_at(taps, 8 * s + a8 + b8 - (kTH - 1) - SB);
    const __nv_bfloat16 h = __float2bfloat16(g);
    reinterpret_cast<__nv_bfloat16*>(S2H)[e] = h;
    reinterpret_cast<__nv_bfloat16*>(S2L)[e] = __float2bfloat16(g - __bfloat162float(h));
  }
  if (warp == 12) umma::tmem_alloc(&tslot, kTmemCols);
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      umma::mbar_init(&bars.q_full[s], 128);
      umma::mbar_init(&bars.q_empty[s], 1);
      umma::mbar_init(&bars.d2_full[s], 1);
      umma::mbar_init(&bars.d2_empty[s], 128);
      umma::mbar_init(&bars.pc_done[s], 128);
      umma::mbar_init(&bars.phi_ready[s], 1);
    }
    umma::mbar_init(&bars.d1_full, 1);
    umma::mbar_init(&bars.d1_empty, 128);
    umma::mbar_init(&bars.a2_full, 128);
    umma::mbar_init(&bars.a2_empty, 1);
    umma::mbar_init(&bars.gh_ready, 128);
    umma::mbar_init(&bars.drain_h, 1);
    umma::mbar_init(&bars.drain_v, 1);
    umma::fence_mbar_init();
    abort_flag = 0;
  }
  umma::fence_async_smem();             // strips visible to the tensor core
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tbase = tslot;

  if (warp < 4) {
    // ---------------- builders: Q(t) = bf16(phi_k f_q) into slot t & 1
    const int bt = tid;                 // 0..127
    int pbuf = 0;                       // phi buffer of the current mode
    for (int t = 0; t < T; ++t) {
      const int k = t / nq, q = t - k * nq, s = t & 1, u = t >> 1;
      if (q == 0) {                     // phi_k landed (copied at setup or two modes ago)
        // the copy of phi_{k+1} (issued at the end of mode k - 1, for k + 1 >= 2)
        // may stay in flight; everything older must be complete
        if (k >= 1 && k + 1 < r) cp_async_wait<1>();
        else cp_async_wait<0>();
        builders_sync();
        pbuf = k & 1;
        // every builder's copy of phi_k is complete: the epilogue may read the buffer
        if (bt == 0) bar_arrive(&bars.phi_ready[pbuf]);
      }
      bool okw = true;
      if (u > 0) okw = umma::mbar_wait(&bars.q_empty[s], (u - 1) & 1, kWait);
      if (!builders_all(okw && !abort_flag)) {
        abort_flag = 1;
        break;
      }
      const float* Pk = P + pbuf * (C::PPLANE / 4);
      const __nv_bfloat16* Fq = q < n ? F + q * (C::FPLANE / 2) : nullptr;
      unsigned char* Qs = Q + s * C::QPLANE;
      // chunk e: rows 8 g + (e & 7), columns 8 c; consecutive threads take
      // consecutive rows of one core matrix (conflict-free reads and stores)
      constexpr int kChunks = HH * (HW / 8);
#pragma unroll
      for (int j = 0; j < (kChunks + 127) / 128; ++j) {
        const int e = bt + 128 * j;
        if (e >= kChunks) break;
        const int g = e / (8 * (HW / 8)), rem = e - g * (8 * (HW / 8));
        const int rr = 8 * g + (rem & 7), c8 = (rem >> 3) * 8;
        const float4* p = reinterpret_cast<const float4*>(Pk + rr * C::PSF + c8);
        float4 x0 = p[0], x1 = p[1];
        if (Fq) {
          const uint4 fw = *reinterpret_cast<const uint4*>(Fq + rr * C::FSB + c8);
          const float2 f0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&fw.x));
          const float2 f1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&fw.y));
          const float2 f2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&fw.z));
          const float2 f3 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&fw.w));
          x0.x *= f0.x; x0.y *= f0.y; x0.z *= f1.x; x0.w *= f1.y;
          x1.x *= f2.x; x1.y *= f2.y; x1.z *= f3.x; x1.w *= f3.y;
        }
        *reinterpret_cast<uint4*>(Qs + umma::kmajor_offset(rr, c8, HW)) =
            make_uint4(pack2(x0.x, x0.y), pack2(x0.z, x0.w), pack2(x1.x, x1.y), pack2(x1.z, x1.w));
      }
      umma::fence_async_smem();
      bar_arrive(&bars.q_full[s]);
      if (q == nq - 1 && k + 2 < r) {   // phi_{k+2} into the buffer this mode used
        // the epilogue copied its tile pixels, and every builder is done reading it
        const bool okc = umma::mbar_wait(&bars.pc_done[pbuf], (k >> 1) & 1, kWait);
        if (!builders_all(okc && !abort_flag)) {
          abort_flag = 1;
          break;
        }
        stage_phi<SB>(P + pbuf * (C::PPLANE / 4), phi + (int64_t)(k + 2) * a.N, ty0, tx0, a.H, a.W,
                      bt);
        cp_async_commit();
      }
    }
    cp_async_wait<0>();
  } else if (warp >= 12) {
    // ---------------- MMA issuers (one thread each): warp 12 the horizontal
    // products, warp 13 the vertical ones, each as soon as its inputs are ready
    if (lane == 0) {
      const uint32_t idesc1 = umma::idesc_bf16(128, HH), idesc2 = umma::idesc_bf16(128, kTH);
      // descriptors of the K slices: slice ks starts 256 B (16 units of the
      // address field) after slice 0
      const uint64_t dS2H = umma::sdesc(umma::smem_u32(S2H), 128, 128);
      const uint64_t dS2L = umma::sdesc(umma::smem_u32(S2L), 128, 128);
      const uint64_t dQ0 = umma::sdesc(umma::smem_u32(Q), 128, HW * 16);
      bool fine = true;
      if (warp == 12) {
        fine = umma::mbar_wait(&bars.gh_ready, 0, kWait);
        for (int t = 0; fine && t < T; ++t) {   // D1(t) = Gh' Q(t)^T, taps hi + lo, Gh' in TMEM
          const int s = t & 1, u = t >> 1;
          if (!umma::mbar_wait(&bars.q_full[s], u & 1, kWait) ||
              (t > 0 && !umma::mbar_wait(&bars.d1_empty, (t - 1) & 1, kWait)) || abort_flag) {
            fine = false;
            break;
          }
          umma::fence_after_sync();
          const uint32_t d = tbase + kD1;
          uint32_t ah = tbase + kGH, al = ah + HW / 2;
          uint64_t bq = dQ0 + (uint64_t)(s * (C::QPLANE >> 4));
#pragma unroll
          for (int ks = 0; ks < HW / 16; ++ks, ah += 8, al += 8, bq += 16) {
            umma::mma_bf16_ta(d, ah, bq, idesc1, ks > 0);
            umma::mma_bf16_ta(d, al, bq, idesc1, 1);
          }
          umma::commit(&bars.q_empty[s]);
          umma::commit(&bars.d1_full);
        }
        if (!fine) abort_flag = 1;
        umma::commit(&bars.drain_h);       // completes once every product issued above has
        umma::mbar_wait(&bars.drain_h, 0, kWait);
      } else {
        for (int t = 0; t < T; ++t) {      // D2(t) = (A2H + A2L)(G_hi + G_lo)^T, lo x lo dropped
          const int s = t & 1, u = t >> 1;
          if (!umma::mbar_wait(&bars.a2_full, t & 1, kWait) ||
              (u > 0 && !umma::mbar_wait(&bars.d2_empty[s], (u - 1) & 1, kWait)) || abort_flag) {
            fine = false;
            break;
          }
          umma::fence_after_sync();
          const uint32_t d = tbase + kD2 + 32 * s;
          uint32_t ah = tbase + kA2, al = ah + 32;
          uint64_t gh = dS2H, gl = dS2L;
#pragma unroll
          for (int ks = 0; ks < HH / 16; ++ks, ah += 8, al += 8, gh += 16, gl += 16) {
            umma::mma_bf16_ta(d, ah, gh, idesc2, ks > 0);
            umma::mma_bf16_ta(d, ah, gl, idesc2, 1);
            umma::mma_bf16_ta(d, al, gh, idesc2, 1);
          }
          umma::commit(&bars.a2_empty);
          umma::commit(&bars.d2_full[s]);
        }
        if (!fine) abort_flag = 1;
        umma::commit(&bars.drain_v);
        umma::mbar_wait(&bars.drain_v, 0, kWait);
      }
    }
    __syncwarp();
  } else if (warp < 8) {
    // ---------------- converters: Gh' into tensor memory once, then D1(t) -> bf16
    // hi/lo pair A2(t)
    const uint32_t tl = (uint32_t)(32 * (warp & 3)) << 16;
    write_gh<SB>(taps, tbase + tl, (kTW - 1) - (32 * (warp & 3) + lane));
    umma::fence_before_sync();
    bar_arrive(&bars.gh_ready);
    for (int t = 0; t < T; ++t) {
      const int s = t & 1;
      bool okw = umma::mbar_wait(&bars.d1_full, t & 1, kWait);
      if (okw && t > 0) okw = umma::mbar_wait(&bars.a2_empty, (t - 1) & 1, kWait);
      if (!__all_sync(0xffffffffu, okw) || abort_flag) { abort_flag = 1; break; }
      umma::fence_after_sync();
#pragma unroll
      for (int c0 = 0; c0 < HH; c0 += 32) {
        float v[32], hi[16], lo[16];
        umma::tmem_ld32(tbase + tl + kD1 + c0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
          const float2 hf = __bfloat1622float2(h);
          hi[i] = __uint_as_float(*reinterpret_cast<const uint32_t*>(&h));
          lo[i] = __uint_as_float(pack2(v[2 * i] - hf.x, v[2 * i + 1] - hf.y));
        }
        umma::tmem_st16x2(tbase + tl + kA2 + c0 / 2, tbase + tl + kA2 + 32 + c0 / 2, hi, lo);
      }
      umma::fence_before_sync();
      bar_arrive(&bars.d1_empty);
      bar_arrive(&bars.a2_full);
      (void)s;
    }
  } else {
    // ---------------- epilogue: zeta_q += phi_k C_kq, C_kq to memory if kept, g_hat
    const uint32_t tl = (uint32_t)(32 * (warp & 3)) << 16;
    const int xp = 32 * (warp & 3) + lane;
    const int xo = tx0 + (kTW - 1) - xp;          // output column of this lane
    {
      float z[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) z[i] = 0.f;
      for (int c = 0; c < 4 * kTH; c += 32) umma::tmem_st32(tbase + tl + kZeta + c, z);
    }
    float* pcs = reinterpret_cast<float*>(sm + C::OFF_PC);   // this thread owns column xp
    bool fine = true;
    for (int t = 0; t < T; ++t) {
      const int k = t / nq, q = t - k * nq, s = t & 1, u = t >> 1;
      if (q == 0) {                     // phi_k at this lane's pixels (FP32), from the builders'
        // buffer: it holds phi_k once the builders signal phi_ready (their asynchronous
        // copies of it are complete) until they see pc_done for it
        const bool okp = umma::mbar_wait(&bars.phi_ready[k & 1], (k >> 1) & 1, kWait);
        if (!__all_sync(0xffffffffu, okp) || abort_flag) { abort_flag = 1; fine = false; break; }
        const float* src = P + (k & 1) * (C::PPLANE / 4) + (SB + kTH - 1) * C::PSF + SB + (kTW - 1) - xp;
#pragma unroll 8
        for (int yp = 0; yp < kTH; ++yp) pcs[yp * kTW + xp] = src[-yp * C::PSF];
        bar_arrive(&bars.pc_done[k & 1]);
      }
      const bool okw = umma::mbar_wait(&bars.d2_full[s], u & 1, kWait);
      if (!__all_sync(0xffffffffu, okw) || abort_flag) { abort_flag = 1; fine = false; break; }
      umma::fence_after_sync();
      float cv[32], zv[32];
      umma::tmem_ld32x2(tbase + tl + kD2 + 32 * s, tbase + tl + kZeta + 32 * q, cv, zv);
      umma::fence_before_sync();
      bar_arrive(&bars.d2_empty[s]);
#pragma unroll
      for (int i = 0; i < 32; ++i) zv[i] = fmaf(pcs[i * kTW + xp], cv[i], zv[i]);
      umma::tmem_st32(tbase + tl + kZeta + 32 * q, zv);
      if (a.cout && xo < a.W) {
        float* dst = a.cout + ((int64_t)k * (n + 1) + q) * a.N + (int64_t)(ty0 + kTH - 1) * a.W + xo;
        int y = ty0 + kTH - 1;
#pragma unroll
        for (int i = 0; i < 32; ++i, --y, dst -= a.W)
          if (y < a.H) __stcs(dst, cv[i]);
      }
    }
    if (fine && T > 0) {                // g_hat = zeta / eta (TMEM loads by whole warps)
      float eta[32];
      umma::tmem_ld32(tbase + tl + kZeta + 32 * n, eta);
      const int64_t top = (int64_t)(ty0 + kTH - 1) * a.W + xo;   // pixel of row i = 0
      {
        int y = ty0 + kTH - 1;
        float* dst = a.eta + top;
#pragma unroll
        for (int i = 0; i < 32; ++i, --y, dst -= a.W) {
          if (y < a.H && xo < a.W) {
            *dst = eta[i];
            if (!(eta[i] > a.eta_thr)) atomicAdd(&a.state_rw->eta_small, 1ull);
          }
        }
      }
      for (int q = 0; q < n; ++q) {
        float zq[32];
        umma::tmem_ld32(tbase + tl + kZeta + 32 * q, zq);
        int y = ty0 + kTH - 1;
        float* dst = a.out + top * n + q;
#pragma unroll
        for (int i = 0; i < 32; ++i, --y, dst -= (int64_t)a.W * n)
          if (y < a.H && xo < a.W) *dst = zq[i] / eta[i];
      }
    }
  }

  umma::fence_before_sync();
  __syncthreads();
  if (tid == 0 && abort_flag) set_status(a.state_rw, NYF_ERR_TIMEOUT);
  if (warp == 12) umma::tmem_dealloc(tbase, kTmemCols);
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

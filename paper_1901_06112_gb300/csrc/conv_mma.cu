// BF16 tensor-core version of the fused convolution + combine (Eqs. (7),
// (14), (15)), used when the features are stored in bfloat16.
//
// Per output tile (32 x 64 pixels), mode k and quantity q (q < n: channel f_q,
// q = n: the constant 1), the separable FIR is written as two banded Toeplitz
// products on the tensor cores (mma.sync m16n8k16, BF16 in, FP32 accumulate):
//   vertical    M = Gv Q,   Gv[y][y'] = g(y' - y),  Q = bf16(phi_k f_q) on the tile + halo
//   horizontal  O = M Gh,   Gh[x'][x] = g(x' - x)
// and zeta_q += phi_k O in FP32 registers.  Each warp owns 16 output rows and
// one quantity (8 warps = 2 row blocks x 4 quantities).  The taps' fragments
// (Gv as the A operand, Gh as the B operand, one per 8-column offset) are built
// once in registers; Q is built per mode in shared memory and read with
// ldmatrix.trans; the vertical result M stays in registers, its accumulator
// fragments reused directly as the A fragments of the horizontal product.
// Zero padding outside the image is the window clipping of Eq. (1).
#include "conv_impl.cuh"

namespace nyf {
namespace {

constexpr int kMmaThreads = 256;   // 8 warps
constexpr int kTH = 32, kTW = 64;  // output tile
constexpr int kNQ = 4;             // quantities per CTA

template <int SB>
struct MmaCfg {
  static constexpr int HHmax = kTH + 2 * SB;                 // halo rows
  static constexpr int KV = (16 + 2 * SB + 15) / 16;         // vertical k-steps
  static constexpr int QROWS = 16 + 16 * KV;                 // Q rows read by the 2nd row block
  static constexpr int NT = (kTW + 2 * SB + 7) / 8;          // n-tiles of M (8 columns)
  static constexpr int HWP = NT * 8;                         // padded halo width
  static constexpr int NF = (2 * SB + 15) / 8 + 1;           // horizontal tap fragments (offset -8 ..)
  static constexpr int FS = HWP + 2;                         // fp32 plane row stride (even)
  static constexpr int QS = HWP + 8;                         // bf16 Q row stride (conflict-free ldmatrix)
  static constexpr int FROWS = QROWS > HHmax ? QROWS : HHmax;
  static constexpr size_t f_bytes = sizeof(float) * (size_t)kNQ * FROWS * FS;
  static constexpr size_t p_bytes = sizeof(float) * (size_t)2 * FROWS * FS;
  static constexpr size_t q_bytes = sizeof(__nv_bfloat16) * (size_t)kNQ * QROWS * QS;
  static constexpr size_t smem = f_bytes + p_bytes + q_bytes;
  static_assert(smem <= 227 * 1024, "shared memory budget");
  static_assert((QS * 2) % 16 == 0, "ldmatrix rows must be 16-byte aligned");
  static_assert(NT % 2 == 0, "M n-tiles pair up into 16-column k-steps");
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x2_trans(uint32_t& r0, uint32_t& r1, const void* p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(s));
}

// tap g(t) for t in [0, 2S] (box: 1), zero elsewhere
__device__ __forceinline__ float tap(int t, int S, int box, float inv2s2) {
  if (t < 0 || t > 2 * S) return 0.f;
  if (box) return 1.f;
  const float z = (float)(t - S);
  return expf(-z * z * inv2s2);
}

// Stage plane k of phi into P (fp32, row stride FS): asynchronous for float32,
// through registers for bfloat16.
template <int SB>
__device__ __forceinline__ void stage_phi_mma(const ConvArgs& a, float* P, int k, int ty0, int tx0,
                                              int S, int HH, int HW) {
  using C = MmaCfg<SB>;
  const int64_t base = (int64_t)k * a.N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int yy = warp; yy < HH; yy += kMmaThreads / 32) {
    const int gy = ty0 - S + yy;
    const bool rowin = gy >= 0 && gy < a.H;
    for (int xx = lane; xx < HW; xx += 32) {
      const int gx = tx0 - S + xx;
      const bool in = rowin && gx >= 0 && gx < a.W;
      if (!a.bf16) {
        const float* src = reinterpret_cast<const float*>(a.phi) + base;
        cp_async4(P + yy * C::FS + xx, in ? src + (int64_t)gy * a.W + gx : src, in);
      } else {
        const __nv_bfloat16* src = reinterpret_cast<const __nv_bfloat16*>(a.phi) + base;
        P[yy * C::FS + xx] = in ? __bfloat162float(src[(int64_t)gy * a.W + gx]) : 0.f;
      }
    }
  }
}

template <int SB>
__global__ void __launch_bounds__(kMmaThreads, 1) k_conv_combine_mma(ConvArgs a) {
  using C = MmaCfg<SB>;
  extern __shared__ __align__(16) unsigned char raw[];
  float* F = reinterpret_cast<float*>(raw);                              // kNQ planes
  float* PB = reinterpret_cast<float*>(raw + C::f_bytes);                // 2 planes
  __nv_bfloat16* Q = reinterpret_cast<__nv_bfloat16*>(raw + C::f_bytes + C::p_bytes);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int rb = warp & 1, qi = warp >> 1;         // row block, quantity of this warp
  const int S = a.S_true;
  const int HH = kTH + 2 * S, HW = kTW + 2 * S;
  const int ty0 = blockIdx.y * kTH, tx0 = blockIdx.x * kTW;
  const int q0 = blockIdx.z * kNQ;
  const int n = a.n;
  const int r = a.state->planes;

  // image planes (zero outside the image, beyond HH x HW, and for q >= n)
  for (int row = warp; row < kNQ * C::FROWS; row += kMmaThreads / 32) {
    const int qq = row / C::FROWS, yy = row - qq * C::FROWS;
    const int c = q0 + qq;
    const int gy = ty0 - S + yy;
    const bool rowin = c < n && yy < HH && gy >= 0 && gy < a.H;
    float* dst = F + row * C::FS;
    for (int xx = lane; xx < C::FS; xx += 32) {
      const int gx = tx0 - S + xx;
      const bool in = rowin && xx < HW && gx >= 0 && gx < a.W;
      cp_async4(dst + xx, in ? a.f + ((int64_t)gy * a.W + gx) * n + c : a.f, in);
    }
  }
  // phi planes start zero so that padding rows/columns stay zero
  for (int e = tid; e < 2 * C::FROWS * C::FS; e += kMmaThreads) PB[e] = 0.f;
  __syncthreads();
  if (r > 0) stage_phi_mma<SB>(a, PB, 0, ty0, tx0, S, HH, HW);
  cp_async_commit();

  // tap fragments: vertical A (Gv) per k-step, horizontal B (Gh) per offset
  uint32_t Av[C::KV][4];
#pragma unroll
  for (int kv = 0; kv < C::KV; ++kv) {
    // A[row y][col c] = g(16 kv + c - y)
    Av[kv][0] = pack_bf16(tap(16 * kv + 2 * t - g, S, a.box, a.inv2s2),
                          tap(16 * kv + 2 * t + 1 - g, S, a.box, a.inv2s2));
    Av[kv][1] = pack_bf16(tap(16 * kv + 2 * t - g - 8, S, a.box, a.inv2s2),
                          tap(16 * kv + 2 * t + 1 - g - 8, S, a.box, a.inv2s2));
    Av[kv][2] = pack_bf16(tap(16 * kv + 2 * t + 8 - g, S, a.box, a.inv2s2),
                          tap(16 * kv + 2 * t + 9 - g, S, a.box, a.inv2s2));
    Av[kv][3] = pack_bf16(tap(16 * kv + 2 * t + 8 - g - 8, S, a.box, a.inv2s2),
                          tap(16 * kv + 2 * t + 9 - g - 8, S, a.box, a.inv2s2));
  }
  uint32_t Bh[C::NF][2];
#pragma unroll
  for (int j = 0; j < C::NF; ++j) {
    const int d = 8 * j - 8;                         // offset 16 kappa - 8 nb
    // B[k][col] = g(d + k - col), col = g (group id)
    Bh[j][0] = pack_bf16(tap(d + 2 * t - g, S, a.box, a.inv2s2),
                         tap(d + 2 * t + 1 - g, S, a.box, a.inv2s2));
    Bh[j][1] = pack_bf16(tap(d + 2 * t + 8 - g, S, a.box, a.inv2s2),
                         tap(d + 2 * t + 9 - g, S, a.box, a.inv2s2));
  }
  const int kv_need = (16 + 2 * S + 15) / 16;

  float acc[kTW / 8][4];
#pragma unroll
  for (int nb = 0; nb < kTW / 8; ++nb) acc[nb][0] = acc[nb][1] = acc[nb][2] = acc[nb][3] = 0.f;

  const int q = q0 + qi;
  const bool wq = q <= n;                           // this warp has a quantity
  __nv_bfloat16* Qw = Q + qi * C::QROWS * C::QS;

  for (int k = 0; k < r; ++k) {
    if (k + 1 < r) {
      stage_phi_mma<SB>(a, PB + ((k + 1) & 1) * C::FROWS * C::FS, k + 1, ty0, tx0, S, HH, HW);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* P = PB + (k & 1) * C::FROWS * C::FS;
    // Q_q = bf16(phi_k f_q) on rows [0, QROWS) x columns [0, HWP): a warp per
    // row, a lane per column pair
    for (int yy = warp; yy < C::QROWS; yy += kMmaThreads / 32) {
      for (int x2 = 2 * lane; x2 < C::HWP; x2 += 64) {
        const float2 p = *reinterpret_cast<const float2*>(P + yy * C::FS + x2);
#pragma unroll
        for (int qq = 0; qq < kNQ; ++qq) {
          const int c = q0 + qq;
          float2 v = make_float2(0.f, 0.f);
          if (c < n) {
            const float2 fv =
                *reinterpret_cast<const float2*>(F + qq * C::FROWS * C::FS + yy * C::FS + x2);
            v = __fmul2_rn(p, fv);
          } else if (c == n) {
            v = p;
          }
          *reinterpret_cast<uint32_t*>(Q + qq * C::QROWS * C::QS + yy * C::QS + x2) =
              pack_bf16(v.x, v.y);
        }
      }
    }
    __syncthreads();
    if (wq) {
      // vertical: M (16 rows x HWP) = Gv (16 x 16 KV) * Q rows [16 rb, 16 rb + 16 KV)
      float Mv[C::NT][4];
#pragma unroll
      for (int m = 0; m < C::NT; ++m) {
        Mv[m][0] = Mv[m][1] = Mv[m][2] = Mv[m][3] = 0.f;
#pragma unroll
        for (int kv = 0; kv < C::KV; ++kv) {
          if (kv < kv_need) {
            uint32_t b0, b1;
            const __nv_bfloat16* src = Qw + (16 * rb + 16 * kv + (lane & 15)) * C::QS + 8 * m;
            ldmatrix_x2_trans(b0, b1, src);
            mma_bf16(Mv[m], Av[kv], b0, b1);
          }
        }
      }
      // M as bf16 A fragments of the horizontal product (16-column k-steps)
      uint32_t Ma[C::NT / 2][4];
#pragma unroll
      for (int ks = 0; ks < C::NT / 2; ++ks) {
        Ma[ks][0] = pack_bf16(Mv[2 * ks][0], Mv[2 * ks][1]);
        Ma[ks][1] = pack_bf16(Mv[2 * ks][2], Mv[2 * ks][3]);
        Ma[ks][2] = pack_bf16(Mv[2 * ks + 1][0], Mv[2 * ks + 1][1]);
        Ma[ks][3] = pack_bf16(Mv[2 * ks + 1][2], Mv[2 * ks + 1][3]);
      }
      // horizontal: O (16 x 8 per output block nb) = M (16 x HWP) * Gh
#pragma unroll
      for (int nb = 0; nb < kTW / 8; ++nb) {
        float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < C::NT / 2; ++ks) {
          const int d = 16 * ks - 8 * nb;            // offset of this k-step
          if (d >= -8 && d <= 2 * SB + 7) {          // compile-time band
            if (d <= 2 * S + 7) {                    // runtime band
              const int j = (d + 8) / 8;
              mma_bf16(o, Ma[ks], Bh[j][0], Bh[j][1]);
            }
          }
        }
        // combine: rows 16 rb + g (+8), columns 8 nb + 2t (+1); phi at the pixel
        const int y0 = 16 * rb + g + S, x0 = 8 * nb + 2 * t + S;
        acc[nb][0] = fmaf(P[y0 * C::FS + x0], o[0], acc[nb][0]);
        acc[nb][1] = fmaf(P[y0 * C::FS + x0 + 1], o[1], acc[nb][1]);
        acc[nb][2] = fmaf(P[(y0 + 8) * C::FS + x0], o[2], acc[nb][2]);
        acc[nb][3] = fmaf(P[(y0 + 8) * C::FS + x0 + 1], o[3], acc[nb][3]);
        if (a.cout) {                              // keep C_kq for the backward pass
          float* cq = a.cout + ((int64_t)k * (n + 1) + q) * a.N;
          const int gy = ty0 + 16 * rb + g, gx = tx0 + 8 * nb + 2 * t;
          const bool pair = gx + 1 < a.W && (a.W & 1) == 0;   // 8-byte aligned column pair
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (gy + 8 * h < a.H) {
              float* row = cq + (int64_t)(gy + 8 * h) * a.W + gx;
              if (pair) {
                __stcs(reinterpret_cast<float2*>(row), make_float2(o[2 * h], o[2 * h + 1]));
              } else {
                if (gx < a.W) row[0] = o[2 * h];
                if (gx + 1 < a.W) row[1] = o[2 * h + 1];
              }
            }
          }
        }
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();

  // gather the quantities of each pixel through shared memory (reuse F)
  float* Z = F;                                    // kNQ x kTH x kTW
  if (wq) {
#pragma unroll
    for (int nb = 0; nb < kTW / 8; ++nb) {
      const int y = 16 * rb + g, x = 8 * nb + 2 * t;
      float* z = Z + qi * kTH * kTW;
      z[y * kTW + x] = acc[nb][0];
      z[y * kTW + x + 1] = acc[nb][1];
      z[(y + 8) * kTW + x] = acc[nb][2];
      z[(y + 8) * kTW + x + 1] = acc[nb][3];
    }
  }
  __syncthreads();
  const bool fused = (q0 == 0) && (n + 1 <= kNQ);
  for (int e = tid; e < kTH * kTW; e += kMmaThreads) {
    const int y = e / kTW, x = e - y * kTW;
    const int gy = ty0 + y, gx = tx0 + x;
    if (gy < a.H && gx < a.W) {
      const int64_t pix = (int64_t)gy * a.W + gx;
      if (fused) {
        const float eta = Z[n * kTH * kTW + e];
        for (int c = 0; c < n; ++c) a.out[pix * n + c] = Z[c * kTH * kTW + e] / eta;
        a.eta[pix] = eta;
        if (!(eta > a.eta_thr)) atomicAdd(&a.state_rw->eta_small, 1ull);
      } else {
        for (int qq = 0; qq < kNQ; ++qq) {
          const int c = q0 + qq;
          if (c < n) a.zeta[pix * n + c] = Z[qq * kTH * kTW + e];
          else if (c == n) a.eta[pix] = Z[qq * kTH * kTW + e];
        }
      }
    }
  }
}

template <int SB>
cudaError_t mma_launch(const ConvArgs& a, cudaStream_t st) {
  using C = MmaCfg<SB>;
  cudaError_t e = cudaFuncSetAttribute(k_conv_combine_mma<SB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.W + kTW - 1) / kTW, (a.H + kTH - 1) / kTH, (a.n + 1 + kNQ - 1) / kNQ);
  k_conv_combine_mma<SB><<<grid, kMmaThreads, C::smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

// Tensor-core path for window radii up to 16; returns cudaErrorNotSupported otherwise.
cudaError_t conv_mma_dispatch(const ConvArgs& a, cudaStream_t st) {
  if (a.S_true <= 8) return mma_launch<8>(a, st);
  if (a.S_true <= 16) return mma_launch<16>(a, st);
  return cudaErrorNotSupported;
}

bool conv_mma_split(int n) { return n + 1 > kNQ; }

}  // namespace nyf

// Per-pixel Nystrom features on the fifth-generation tensor cores (tcgen05),
// for guides of dimension rho >= 16 (hyperspectral pixels, NLM patches, PCA
// coordinates): Eqs. (11)-(12) as two contractions,
//   X   = P~ M~^T              (N x rho . rho x K: the cross term of the distances)
//   D   = ||p~||^2 + ||mu~||^2 - 2 X,   E = exp(-D / (2 sigma_r^2))   (Eq. (11))
//   Phi = E W_hat               (N x K . K x K, Eq. (12) with the symmetric factor)
// where p~ = p - c and mu~ = mu - c are centred on the mean c of the
// landmarks (distances do not change; the norms, and with them the
// cancellation in D, shrink).
//
// Precision.  The method's exponent exp(-D / 2 sigma_r^2) turns an absolute
// error in D into a relative error of E that is D's error over 2 sigma_r^2;
// for the 512 x 512 x 31 hyperspectral workload 2 sigma_r^2 = 0.045 against
// squared norms of order 1, so D needs close to FP32 accuracy.  Every FP32
// operand x is therefore split exactly into three bfloat16 terms
//   x = x1 + x2 + x3,  x1 = bf16(x), x2 = bf16(x - x1), x3 = x - x1 - x2,
// and each contraction sums the six products whose weight is at least
// 2^-16 of the leading one (x1 y1, x1 y2, x2 y1, x1 y3, x2 y2, x3 y1; the
// three dropped ones weigh 2^-24 and less), accumulated in FP32 in tensor
// memory.  The norms are FP32 sums on the CUDA cores, and D is formed with an
// exact two-sum of the norms followed by one fused multiply-add.
//
// One CTA of four warps owns a tile of 128 pixels (tensor-memory lane t =
// pixel t of the tile) and walks the tiles of the image (persistent grid):
//   1. each thread loads its pixel's guide row (a stored row, or its NLM patch
//      from a shared-memory image tile), centres it, accumulates ||p~||^2 and
//      writes the three bf16 terms into the K-major A operand;
//   2. one thread issues the six products of X into tensor memory;
//   3. each thread reads its row of X, forms D and E, and writes E's three
//      terms into the A operand of the second product (the same shared memory);
//   4. one thread issues the six products of Phi into tensor memory;
//   5. each thread reads its row of Phi and stores the planes (plane k at
//      phi + k N), 32 consecutive pixels per warp store.
// The landmarks' and W_hat's bf16 terms stay in shared memory for the whole
// kernel.  Every wait is bounded: a timeout latches NYF_ERR_TIMEOUT, and the
// kernel waits (bounded) for its own products before freeing tensor memory.
#include "nyf_internal.cuh"
#include "split_bf16.cuh"
#include "umma.cuh"

namespace nyf {
namespace {

using splitbf::issue_split_gemm;
using splitbf::put8;

constexpr int kFtThreads = 128;
constexpr int kFtRows = 128;                 // pixels per tile (MMA M, tensor-memory lanes)
constexpr uint32_t kFtWait = 1u << 20;       // mbarrier polls before giving up (each up to 1 us)
constexpr uint32_t kD1Col = 0, kD2Col = 64, kFtTmemCols = 128;
constexpr int kNlmTY = 8, kNlmTX = 16;       // NLM tile: 8 rows x 16 columns of pixels

__host__ __device__ inline int pad16(int v) { return (v + 15) & ~15; }

// Shared-memory layout (byte offsets) of one CTA.
struct FtLayout {
  int rp, kp;                  // rho and K rounded up to 16
  int a, b1, b2, c, bn, tile, poff, total;
};

__host__ __device__ inline FtLayout ft_layout(int rho, int K, int tile_floats) {
  FtLayout L;
  L.rp = pad16(rho);
  L.kp = pad16(K);
  const int a1 = 3 * kFtRows * L.rp * 2, a2 = 3 * kFtRows * L.kp * 2;
  int o = 0;
  L.a = o;
  o += a1 > a2 ? a1 : a2;                    // P~ terms, then E terms (after X is read)
  L.b1 = o;
  o += 3 * L.kp * L.rp * 2;                  // landmark terms (N x K-dim = kp x rp)
  L.b2 = o;
  o += 3 * L.kp * L.kp * 2;                  // W_hat terms (kp x kp)
  L.c = o;
  o += 4 * L.rp;                             // centre c
  L.bn = o;
  o += 4 * L.kp;                             // ||mu~_m||^2
  L.tile = o;
  o += 4 * tile_floats;                      // NLM image tile
  L.poff = o;
  o += tile_floats > 0 ? 4 * L.rp : 0;       // NLM: tile offset of each patch component
  L.total = (o + 127) & ~127;
  return L;
}

__device__ __forceinline__ int reflect101(int i, int n) {
  if (n == 1) return 0;
  const int period = 2 * (n - 1);
  int j = i % period;
  if (j < 0) j += period;
  return j < n ? j : period - j;
}

struct FtArgs {
  const float* guide;      // N x rho rows (stored guide), or NULL for NLM patches
  const float* f;          // NLM: H x W x n image
  int H, W, n, r;          // NLM geometry (patch radius r)
  int64_t N;
  int rho, K;
  const float* lm;         // K x rho landmarks
  const float* what;       // K x K W_hat (row-major, symmetric)
  float inv2s2;
  const DevState* state;
  DevState* state_rw;
  void* phi;
  int bf16;
};

template <bool NLM>
__global__ void __launch_bounds__(kFtThreads, 1) k_features_tc(const __grid_constant__ FtArgs a) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t mbar, drain;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int rho = a.rho, K = a.K;
  const int side = 2 * a.r + 1;
  const int TSY = kNlmTY + 2 * a.r, TSX = kNlmTX + 2 * a.r;
  const FtLayout L = ft_layout(rho, K, NLM ? TSY * TSX * a.n : 0);
  const int rp = L.rp, kp = L.kp;
  unsigned char* A = sm + L.a;
  unsigned char* B1 = sm + L.b1;
  unsigned char* B2 = sm + L.b2;
  float* cen = reinterpret_cast<float*>(sm + L.c);
  float* bnorm = reinterpret_cast<float*>(sm + L.bn);
  float* tile = reinterpret_cast<float*>(sm + L.tile);
  int* poff = reinterpret_cast<int*>(sm + L.poff);
  if (NLM)   // component j = (dy side + dx) n + c sits at tile offset (dy TSX + dx) n + c
    for (int d = tid; d < rho; d += kFtThreads) {
      const int c = d % a.n, q = d / a.n;
      const int dy = q / side, dx = q - dy * side;
      poff[d] = (dy * TSX + dx) * a.n + c;
    }
  const int a1_term = kFtRows * rp * 2, a2_term = kFtRows * kp * 2;
  const int b1_term = kp * rp * 2, b2_term = kp * kp * 2;

  // centre c = mean of the landmarks (fixed order: every CTA gets the same c)
  for (int d = tid; d < rp; d += kFtThreads) {
    float s = 0.f;
    if (d < rho)
      for (int m = 0; m < K; ++m) s += a.lm[m * rho + d];
    cen[d] = d < rho ? s / (float)K : 0.f;
  }
  __syncthreads();
  // landmark terms (rows m < kp; zero rows beyond K) and ||mu~||^2
  for (int m = tid; m < kp; m += kFtThreads) {
    float nrm = 0.f;
    for (int d0 = 0; d0 < rp; d0 += 8) {
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int d = d0 + i;
        v[i] = (m < K && d < rho) ? a.lm[m * rho + d] - cen[d] : 0.f;
        nrm = fmaf(v[i], v[i], nrm);
      }
      put8(B1, b1_term, m, d0, rp, v);
    }
    bnorm[m] = nrm;
  }
  // W_hat terms: B2[n][k] = W_hat[k][n] (W_hat is symmetric, so the row is read directly)
  for (int nrow = tid; nrow < kp; nrow += kFtThreads)
    for (int k0 = 0; k0 < kp; k0 += 8) {
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = k0 + i;
        v[i] = (nrow < K && k < K) ? a.what[k * K + nrow] : 0.f;
      }
      put8(B2, b2_term, nrow, k0, kp, v);
    }
  if (warp == 0) umma::tmem_alloc(&tslot, kFtTmemCols);
  if (tid == 0) {
    umma::mbar_init(&mbar, 1);
    umma::mbar_init(&drain, 1);
    umma::fence_mbar_init();
    abort_flag = 0;
  }
  umma::fence_async_smem();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tbase = tslot;
  const uint32_t lane_base = tbase + ((uint32_t)(32 * warp) << 16);
  const uint32_t a_s = umma::smem_u32(A), b1_s = umma::smem_u32(B1), b2_s = umma::smem_u32(B2);
  const uint32_t id1 = umma::idesc_bf16(128, kp), id2 = umma::idesc_bf16(128, kp);
  const int planes = a.state->planes;
  const float inv2s2 = a.inv2s2;
  uint32_t phase = 0;
  bool ok = true;

  int64_t ntiles;
  int tiles_x = 1;
  if (NLM) {
    tiles_x = (a.W + kNlmTX - 1) / kNlmTX;
    ntiles = (int64_t)tiles_x * ((a.H + kNlmTY - 1) / kNlmTY);
  } else {
    ntiles = (a.N + kFtRows - 1) / kFtRows;
  }
  for (int64_t t = blockIdx.x; t < ntiles && ok && planes > 0; t += gridDim.x) {
    // ---- 1. guide rows -> centred bf16 terms of the A operand, ||p~||^2
    int64_t pix = -1;
    float anorm = 0.f;
    if (NLM) {
      const int ty0 = (int)(t / tiles_x) * kNlmTY, tx0 = (int)(t % tiles_x) * kNlmTX;
      for (int e = tid; e < TSY * TSX * a.n; e += kFtThreads) {
        const int c = e % a.n, q = e / a.n;
        const int yy = q / TSX, xx = q - yy * TSX;
        const int gy = reflect101(ty0 - a.r + yy, a.H), gx = reflect101(tx0 - a.r + xx, a.W);
        tile[e] = a.f[((int64_t)gy * a.W + gx) * a.n + c];
      }
      __syncthreads();
      const int ty = tid / kNlmTX, tx = tid % kNlmTX;
      if (ty0 + ty < a.H && tx0 + tx < a.W) pix = (int64_t)(ty0 + ty) * a.W + tx0 + tx;
      // the patch components, read from the tile through the offset table
      const float* tp = tile + (ty * TSX + tx) * a.n;
      for (int d0 = 0; d0 < rp; d0 += 8) {
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int d = d0 + i;
          float x = 0.f;
          if (pix >= 0 && d < rho) x = tp[poff[d]] - cen[d];
          v[i] = x;
          anorm = fmaf(x, x, anorm);
        }
        put8(A, a1_term, tid, d0, rp, v);
      }
    } else {
      const int64_t i = t * kFtRows + tid;
      if (i < a.N) pix = i;
      const float* p = a.guide + (pix >= 0 ? pix : 0) * (int64_t)rho;
      for (int d0 = 0; d0 < rp; d0 += 8) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int d = d0 + k;
          const float x = (pix >= 0 && d < rho) ? __ldg(p + d) - cen[d] : 0.f;
          v[k] = x;
          anorm = fmaf(x, x, anorm);
        }
        put8(A, a1_term, tid, d0, rp, v);
      }
    }
    umma::fence_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    // ---- 2. X = P~ M~^T
    if (tid == 0) {
      issue_split_gemm(tbase + kD1Col, a_s, a1_term, b1_s, b1_term, rp, id1);
      umma::commit(&mbar);
    }
    ok = __all_sync(0xffffffffu, umma::mbar_wait(&mbar, phase, kFtWait));
    phase ^= 1;
    umma::fence_after_sync();
    if (!ok) {
      atomicExch(&abort_flag, 1);
    } else {
      // ---- 3. D, E = exp(-D / 2 sigma_r^2), E's terms into the A operand
      for (int c0 = 0; c0 < kp; c0 += 16) {
        float x[16];
        umma::tmem_ld16(lane_base + kD1Col + c0, x);
        for (int j0 = 0; j0 < 16; j0 += 8) {
          float v[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int m = c0 + j0 + i;
            float e = 0.f;
            if (m < K) {
              const float s = anorm + bnorm[m];          // two-sum of the norms
              const float bb = s - anorm;
              const float err = (anorm - (s - bb)) + (bnorm[m] - bb);
              const float dd = fmaf(-2.f, x[j0 + i], s) + err;
              e = expf(-dd * inv2s2);
            }
            v[i] = e;
          }
          put8(A, a2_term, tid, c0 + j0, kp, v);
        }
      }
    }
    umma::fence_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (abort_flag) {
      ok = false;
      break;
    }
    // ---- 4. Phi = E W_hat
    if (tid == 0) {
      issue_split_gemm(tbase + kD2Col, a_s, a2_term, b2_s, b2_term, kp, id2);
      umma::commit(&mbar);
    }
    ok = __all_sync(0xffffffffu, umma::mbar_wait(&mbar, phase, kFtWait));
    phase ^= 1;
    umma::fence_after_sync();
    if (!ok) {
      atomicExch(&abort_flag, 1);
    } else {
      // ---- 5. the planes of this tile (every thread takes part in the loads)
      for (int c0 = 0; c0 < kp; c0 += 16) {
        float v[16];
        umma::tmem_ld16(lane_base + kD2Col + c0, v);
        if (pix >= 0) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int k = c0 + i;
            if (k < planes) {
              if (a.bf16)
                reinterpret_cast<__nv_bfloat16*>(a.phi)[(int64_t)k * a.N + pix] = __float2bfloat16_rn(v[i]);
              else
                reinterpret_cast<float*>(a.phi)[(int64_t)k * a.N + pix] = v[i];
            }
          }
        }
      }
    }
    umma::fence_before_sync();
    __syncthreads();     // A, the tile and tensor memory are free for the next tile
    umma::fence_after_sync();
    if (abort_flag) ok = false;
  }
  // drain: every product this CTA issued has completed before tensor memory is freed
  if (tid == 0) {
    umma::commit(&drain);
    if (!umma::mbar_wait(&drain, 0, kFtWait)) atomicExch(&abort_flag, 1);
    if (abort_flag) set_status(a.state_rw, NYF_ERR_TIMEOUT);
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (warp == 0) umma::tmem_dealloc(tbase, kFtTmemCols);
}

// Shared memory is requested at no less than this, so that at most three CTAs
// (3 x 128 tensor-memory columns) share an SM.
constexpr int kFtMinSmem = 60 * 1024;

template <bool NLM>
cudaError_t ft_launch(const FtArgs& a, int tile_floats, int64_t ntiles, cudaStream_t st) {
  const FtLayout L = ft_layout(a.rho, a.K, tile_floats);
  const int smem = L.total > kFtMinSmem ? L.total : kFtMinSmem;
  cudaError_t e = cudaFuncSetAttribute(k_features_tc<NLM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int per_sm = (227 * 1024) / (smem + 1024);
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 3) per_sm = 3;
  int64_t g = 152 * (int64_t)per_sm;
  if (g > ntiles) g = ntiles;
  if (g < 1) g = 1;
  k_features_tc<NLM><<<(int)g, kFtThreads, smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

size_t features_tc_smem_bytes(int rho, int K, int n, int r) {
  const int tile = r > 0 ? (kNlmTY + 2 * r) * (kNlmTX + 2 * r) * n : 0;
  return (size_t)ft_layout(rho, K, tile).total;
}

cudaError_t launch_features_tc(const float* guide, int64_t N, int rho, const float* landmarks,
                               int K, float sigma_r, const float* what, const DevState* state,
                               void* phi, bool bf16, cudaStream_t st) {
  FtArgs a{};
  a.guide = guide;
  a.N = N;
  a.rho = rho;
  a.K = K;
  a.lm = landmarks;
  a.what = what;
  a.inv2s2 = (float)(1.0 / (2.0 * (double)sigma_r * (double)sigma_r));
  a.state = state;
  a.state_rw = const_cast<DevState*>(state);
  a.phi = phi;
  a.bf16 = bf16 ? 1 : 0;
  return ft_launch<false>(a, 0, (N + kFtRows - 1) / kFtRows, st);
}

cudaError_t launch_features_nlm_tc(const float* f, int H, int W, int n, int r,
                                   const float* landmarks, int K, float sigma_r, const float* what,
                                   const DevState* state, void* phi, bool bf16, cudaStream_t st) {
  FtArgs a{};
  a.f = f;
  a.H = H;
  a.W = W;
  a.n = n;
  a.r = r;
  a.N = (int64_t)H * W;
  a.rho = (2 * r + 1) * (2 * r + 1) * n;
  a.K = K;
  a.lm = landmarks;
  a.what = what;
  a.inv2s2 = (float)(1.0 / (2.0 * (double)sigma_r * (double)sigma_r));
  a.state = state;
  a.state_rw = const_cast<DevState*>(state);
  a.phi = phi;
  a.bf16 = bf16 ? 1 : 0;
  const int64_t ntiles = (int64_t)((W + kNlmTX - 1) / kNlmTX) * ((H + kNlmTY - 1) / kNlmTY);
  return ft_launch<true>(a, (kNlmTY + 2 * r) * (kNlmTX + 2 * r) * n, ntiles, st);
}

}  // namespace nyf

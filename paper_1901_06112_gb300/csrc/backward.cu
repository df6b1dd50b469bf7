// Backward of the features and the landmark-kernel factor (adjoint of
// Eqs. (9)-(12)), and the host launcher of the whole backward pass.
//
// With E_im = exp(-D_im / (2 sigma_r^2)), D_im = ||p_i - mu_m||^2 and
// Phi = E W_hat (W_hat = W_r Lambda_r^{-1/2} W_r^T, the symmetric factor, so
// W_hat W_hat^T is the truncated inverse of A):
//   dE_im = sum_k dPhi_ik W_hat[m][k]
//   dp_i  = sum_m (-E_im dE_im / (2 sigma_r^2)) 2 (p_i - mu_m)
//   dsigma_r (through E) = sum_im dE_im E_im D_im / sigma_r^3
// The filter depends on W_hat only through M = W_hat W_hat^T = A^+ (it sees
// Phi Phi^T), so with G_W = E^T dPhi:  dL/dA = -1/2 W_hat (W_hat^T G_W) W_hat^T
// (exact for full rank; for a truncated rank the rotation of the kept subspace
// is not differentiated), and
//   dsigma_r (through A) = sum_ij dL/dA_ij A_ij ||mu_i - mu_j||^2 / sigma_r^3.
// Landmarks are held fixed.  All cross-block sums run in a fixed order in FP64.
#include <math.h>

#include "backward_impl.cuh"

namespace nyf {
namespace {

constexpr int kFbThreads = 256;
constexpr int kFbBlocks = 456;      // features-backward CTAs (3 per SM), at most
// CTAs of the features backward for N pixels: one round of kFbThreads pixels per CTA
// at least (a small image does not pay for 456 partials); fixed by N, so every sum
// keeps its order for a given image size
inline int fb_blocks(int64_t N) {
  const int64_t b = (N + kFbThreads - 1) / kFbThreads;
  return (int)(b < 1 ? 1 : (b < kFbBlocks ? b : kFbBlocks));
}

__host__ __device__ inline int kpad4(int K) { return (K + 3) & ~3; }

// Rows of Es / Ds (one per pixel, KB floats) are written and read as 16-byte
// chunks; chunk c of row `row` sits at chunk position c ^ (row mod min(8, KB/4)),
// so a warp's 16-byte stores of the same chunk of 32 consecutive rows fall in
// distinct banks (an unswizzled row stride of KB floats puts them all in one).
template <int KB>
__device__ __forceinline__ int chunk_at(int row, int c) {
  constexpr int CH = KB / 4, MASK = (CH < 8 ? CH : 8) - 1;
  return c ^ (row & MASK);
}

template <int KB, int RB>
__global__ void __launch_bounds__(kFbThreads, (KB <= 32 && RB != 32) ? 3 : 1)
k_features_bwd(const float* __restrict__ guide, int64_t N, int rho, const float* __restrict__ lm,
               int K, float inv2s2r, const float* __restrict__ what,
               const DevState* __restrict__ state, const float* __restrict__ dphi,
               float* __restrict__ dguide, int add_into, float* __restrict__ gw_part,
               float* __restrict__ sr_part) {
  extern __shared__ __align__(16) float sm[];
  const int KP = kpad4(K);
  float* Wsm = sm;                          // K x KP
  float* mu = Wsm + K * KP;                 // K x rho
  float* Es = mu + ((K * rho + 3) & ~3);    // kFbThreads x KB
  float* Ds = Es + kFbThreads * KB;         // kFbThreads x KB
  // RB == 0 (rho > 32): this thread's guide row and its dL/dp accumulate in shared
  // memory (row stride rho | 1: odd, so a warp's rows fall in distinct banks).
  // RB < 0 (that does not fit): the row is read from global memory and dL/dp
  // accumulated there, one landmark at a time.
  const int RS = rho | 1;
  float* Xs = Ds + kFbThreads * KB;         // kFbThreads x RS (RB == 0 only)
  float* Ps = Xs + kFbThreads * RS;         // kFbThreads x RS (RB == 0 only)
  const int tid = threadIdx.x;
  const int r = state->planes;
  for (int e = tid; e < K * KP; e += blockDim.x) {
    const int m = e / KP, k = e - m * KP;
    Wsm[e] = k < K ? what[m * K + k] : 0.f;
  }
  for (int e = tid; e < K * rho; e += blockDim.x) mu[e] = lm[e];
  // this thread's 4 x 4 block of G_W = E^T dPhi: block (m0, k0) = (4 (blk / rb4), 4 (blk % rb4));
  // with fewer blocks than threads, group g of the threads takes the pixels px = g mod G
  // of each round (G groups, combined in a fixed order at the end)
  // (the block grid is that of KB, so the pixel stride G is a compile-time constant;
  // rows of Es beyond K and of Ds beyond the kept modes are zero)
  constexpr int nb4 = KB / 4, nblk4 = nb4 * nb4;
  constexpr int G = kFbThreads / nblk4 > 0 ? kFbThreads / nblk4 : 1;
  const int grp = tid / nblk4, blk = tid - grp * nblk4;
  const bool own = grp < G;
  const int m0 = 4 * (blk / nb4), k0 = 4 * (blk % nb4);
  float gw[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) gw[q] = 0.f;
  float srp = 0.f;
  __syncthreads();

  for (int64_t base = (int64_t)blockIdx.x * kFbThreads; base < N;
       base += (int64_t)gridDim.x * kFbThreads) {
    const int64_t i = base + tid;
    const bool valid = i < N;
    const float* p = guide + (valid ? i : 0) * rho;
    constexpr int RX = RB > 0 ? RB : 1;
    float x[RX], dp[RX];
#pragma unroll
    for (int d = 0; d < RX; ++d) {
      x[d] = (RB > 0 && d < rho) ? __ldg(p + d) : 0.f;
      dp[d] = 0.f;
    }
    float* xs = Xs + tid * RS;
    float* ps = Ps + tid * RS;
    if (RB == 0)
      for (int d = 0; d < rho; ++d) {
        xs[d] = __ldg(p + d);
        ps[d] = 0.f;
      }
    float g[KB];                                   // dPhi of this pixel
#pragma unroll
    for (int k = 0; k < KB; ++k) g[k] = (valid && k < r) ? dphi[(int64_t)k * N + i] : 0.f;
    // one landmark at a time: E_m, dE_m = sum_k dPhi_k W_hat[m][k], then its terms;
    // E goes to this thread's row of Es four landmarks at a time
    for (int m4 = 0; m4 < K; m4 += 4) {
      float e4[4];
#pragma unroll
      for (int mq = 0; mq < 4; ++mq) {
        const int m = m4 + mq;
        e4[mq] = 0.f;
        if (m >= K) continue;
        const float* c = mu + m * rho;
        float d2 = 0.f;
        if (RB > 0) {
#pragma unroll
          for (int d = 0; d < RX; ++d)
            if (d < rho) {
              const float t = x[d] - c[d];
              d2 = fmaf(t, t, d2);
            }
        } else if (RB == 0) {
          for (int d = 0; d < rho; ++d) {
            const float t = xs[d] - c[d];
            d2 = fmaf(t, t, d2);
          }
        } else {
          for (int d = 0; d < rho; ++d) {
            const float t = __ldg(p + d) - c[d];
            d2 = fmaf(t, t, d2);
          }
        }
        const float e = valid ? expf(-d2 * inv2s2r) : 0.f;
        float de0 = 0.f, de1 = 0.f;
#pragma unroll
        for (int k = 0; k < KB; k += 4) {
          if (k < r) {
            const float4 w = *reinterpret_cast<const float4*>(Wsm + m * KP + k);
            de0 = fmaf(g[k], w.x, de0);
            de1 = fmaf(g[k + 1], w.y, de1);
            de0 = fmaf(g[k + 2], w.z, de0);
            de1 = fmaf(g[k + 3], w.w, de1);
          }
        }
        const float de = de0 + de1;
        srp = fmaf(de * e, d2, srp);
        const float dDm = -e * de * inv2s2r;
        if (RB > 0) {
#pragma unroll
          for (int d = 0; d < RX; ++d)
            if (d < rho) dp[d] = fmaf(dDm, 2.f * (x[d] - c[d]), dp[d]);
        } else if (RB == 0) {
          for (int d = 0; d < rho; ++d) ps[d] = fmaf(dDm, 2.f * (xs[d] - c[d]), ps[d]);
        } else if (valid) {
          float* dst = dguide + i * rho;
          for (int d = 0; d < rho; ++d) {
            const float v = dDm * 2.f * (__ldg(p + d) - c[d]);
            dst[d] = (m == 0 && !add_into) ? v : dst[d] + v;
          }
        }
        e4[mq] = e;
      }
      *reinterpret_cast<float4*>(Es + tid * KB + 4 * chunk_at<KB>(tid, m4 >> 2)) =
          make_float4(e4[0], e4[1], e4[2], e4[3]);
    }
    for (int c4 = (K + 3) >> 2; c4 < KB / 4; ++c4)
      *reinterpret_cast<float4*>(Es + tid * KB + 4 * chunk_at<KB>(tid, c4)) =
          make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
      float* dst = dguide + i * rho;
      if (RB > 0) {
#pragma unroll
        for (int d = 0; d < RX; ++d)
          if (d < rho) dst[d] = add_into ? dst[d] + dp[d] : dp[d];
      } else if (RB == 0) {
        for (int d = 0; d < rho; ++d) dst[d] = add_into ? dst[d] + ps[d] : ps[d];
      }
    }
#pragma unroll
    for (int c4 = 0; c4 < KB / 4; ++c4)
      *reinterpret_cast<float4*>(Ds + tid * KB + 4 * chunk_at<KB>(tid, c4)) =
          make_float4(g[4 * c4], g[4 * c4 + 1], g[4 * c4 + 2], g[4 * c4 + 3]);
    __syncthreads();
    // G_W += E^T dPhi over this round's pixels: two 16-byte loads per 16 FMAs
    if (own) {
#pragma unroll 4
      for (int px = grp; px < kFbThreads; px += G) {
        const float4 ev = *reinterpret_cast<const float4*>(Es + px * KB + 4 * chunk_at<KB>(px, m0 >> 2));
        const float4 dv = *reinterpret_cast<const float4*>(Ds + px * KB + 4 * chunk_at<KB>(px, k0 >> 2));
        const float e4[4] = {ev.x, ev.y, ev.z, ev.w}, d4[4] = {dv.x, dv.y, dv.z, dv.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) gw[a * 4 + c] = fmaf(e4[a], d4[c], gw[a * 4 + c]);
      }
    }
    __syncthreads();
  }
  // block partials: G_W (K x K, entries k >= r stay zero) and the sigma_r term.  The
  // groups' sums go through shared memory (the Es region, free now) and are added in
  // group order.
  float* gp = gw_part + (int64_t)blockIdx.x * K * K;
  for (int e = tid; e < K * K; e += blockDim.x) gp[e] = 0.f;
  float* gs = Es;   // G x nblk4 x 16 <= 16 kFbThreads floats: Es and Ds (2 KB kFbThreads), both free now
  if (own) {
#pragma unroll
    for (int q = 0; q < 16; ++q) gs[(grp * nblk4 + blk) * 16 + q] = gw[q];
  }
  __syncthreads();
  if (own && grp == 0) {
    for (int q = 0; q < 16; ++q) {
      float t = 0.f;
      for (int g2 = 0; g2 < G; ++g2) t += gs[(g2 * nblk4 + blk) * 16 + q];
      const int m = m0 + q / 4, k = k0 + q % 4;
      if (m < K && k < r) gp[m * K + k] = t;
    }
  }
  __shared__ float red[kFbThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) srp += __shfl_xor_sync(0xffffffffu, srp, o);
  if ((tid & 31) == 0) red[tid >> 5] = srp;
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int w = 0; w < kFbThreads / 32; ++w) s += red[w];
    sr_part[blockIdx.x] = s;
  }
}

// Z = (W_hat W_hat^T) X W_hat with X_ij = A_ij ||mu_i - mu_j||^2, one CTA per row
// i.  With dL/dA = -1/2 W_hat W_hat^T G_W W_hat^T, the sigma_r term through A is
//   sum_ij dL/dA_ij A_ij ||mu_i - mu_j||^2 / sigma_r^3 = -1/2 <G_W, Z> / sigma_r^3,
// so Z (which does not depend on the incoming gradient) replaces three K^3
// products after the reduction of G_W by one dot product per row.
__global__ void __launch_bounds__(kMaxK)
k_tail_ad2(int K, int rho, const float* __restrict__ lm, const double* __restrict__ A64,
           double* __restrict__ AD2) {
  // (A o D2)[a][t] = A(a, t) ||mu_a - mu_t||^2, one row per CTA (FP64)
  const int a = blockIdx.x, t = threadIdx.x;
  if (t < K) {
    double d2 = 0.0;
    for (int d = 0; d < rho; ++d) {
      const double u = (double)lm[a * rho + d] - (double)lm[t * rho + d];
      d2 += u * u;
    }
    AD2[a * K + t] = A64[a * K + t] * d2;
  }
}

__global__ void __launch_bounds__(kMaxK)
k_tail_z(int K, const float* __restrict__ what, const double* __restrict__ AD2,
         const DevState* __restrict__ state, double* __restrict__ Z) {
  __shared__ double Mrow[kMaxK], MX[kMaxK];
  const int i = blockIdx.x, t = threadIdx.x;
  const int r = state->planes;
  if (t < K) {
    double s = 0.0;
    for (int k = 0; k < r; ++k) s += (double)what[i * K + k] * (double)what[t * K + k];
    Mrow[t] = s;
  }
  __syncthreads();
  if (t < K) {
    double s = 0.0;
    for (int a = 0; a < K; ++a) s += Mrow[a] * AD2[a * K + t];
    MX[t] = s;
  }
  __syncthreads();
  if (t < K) {
    double s = 0.0;
    if (t < r)
      for (int b = 0; b < K; ++b) s += MX[b] * (double)what[b * K + t];
    Z[i * K + t] = s;
  }
}

// G_W[m][k] = sum over blocks (FP64, fixed order: thread (g, k) sums blocks
// g, g + G, ..., then the G group sums are added in order); one CTA per row m.
// Also rowdot[m] = sum_k G_W[m][k] Z[m][k].
__global__ void __launch_bounds__(256)
k_gw_reduce(const float* __restrict__ part, int nblk, int K, const double* __restrict__ Z,
            double* __restrict__ gw, double* __restrict__ rowdot) {
  __shared__ double red[256];
  __shared__ double prod[kMaxK];
  const int m = blockIdx.x, tid = threadIdx.x;
  const int G = 256 / K, g = tid / K, k = tid - g * K;
  double s = 0.0;
  if (g < G) {
    const float* src = part + (int64_t)m * K + k;
    const int64_t step = (int64_t)K * K;
#pragma unroll 4
    for (int b = g; b < nblk; b += G) s += (double)src[b * step];
  }
  red[tid] = s;
  __syncthreads();
  if (tid < K) {
    double t = 0.0;
    for (int q = 0; q < G; ++q) t += red[q * K + tid];
    gw[m * K + tid] = t;
    prod[tid] = t * Z[m * K + tid];
  }
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < K; ++q) t += prod[q];
    rowdot[m] = t;
  }
}

// FP64 sum of `cnt` partials, fixed order (strided per thread, then a tree).
template <typename T>
__device__ double block_sum_fixed(const T* __restrict__ v, int64_t cnt, double* red) {
  const int tid = threadIdx.x;
  double s = 0.0;
  for (int64_t i = tid; i < cnt; i += blockDim.x) s += (double)v[i];
  red[tid] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (tid < o) red[tid] += red[tid + o];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// dsigma_r (through E and through A) and dsigma_s.
__global__ void __launch_bounds__(256)
k_bwd_tail(int K, float sigma_r, const double* __restrict__ rowdot,
           const float* __restrict__ sr_part, int n_sr, const float* __restrict__ ss_part,
           int64_t n_ss, DevState* state, float* __restrict__ grad_sigma) {
  __shared__ double red[256];
  const double s3 = (double)sigma_r * sigma_r * sigma_r;
  const double through_A = -0.5 * block_sum_fixed(rowdot, K, red) / s3;
  const double through_E = block_sum_fixed(sr_part, n_sr, red) / s3;
  const double dss = block_sum_fixed(ss_part, n_ss, red);
  if (threadIdx.x == 0) {
    const float dsr = (float)(through_A + through_E);
    grad_sigma[0] = dsr;
    grad_sigma[1] = (float)dss;
    state->grad_sigma[0] = dsr;
    state->grad_sigma[1] = (float)dss;
  }
}

// dL/d zeta_q as planes: a_c = G_c / eta (c < n), a_n = -sum_c G_c g_hat_c / eta.
// dL/dphi of modes [k0, k1) (capped at the kept planes) from the quantity slices'
// partial plane sets: the sets 1 .. slices-1 are added to set 0 in slice order, so
// the result does not depend on the order in which the slices' CTAs ran.
__global__ void k_dphi_slices(float* __restrict__ dphi, int slices, int64_t slice, int64_t N,
                              int k0, int k1, const DevState* __restrict__ state) {
  const int ke = min(k1, state->planes);
  const int64_t total = (int64_t)(ke - k0) * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t idx = (int64_t)k0 * N + e;
    float v = dphi[idx];
    for (int z = 1; z < slices; ++z) v += dphi[z * slice + idx];
    dphi[idx] = v;
  }
}

__global__ void k_adjoint(const float* __restrict__ gout, const float* __restrict__ out,
                          const float* __restrict__ eta, int64_t N, int n, float* __restrict__ adj) {
  for (int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pix < N;
       pix += (int64_t)gridDim.x * blockDim.x) {
    const float ie = 1.f / eta[pix];
    float s = 0.f;
    for (int c = 0; c < n; ++c) {
      const float g = gout[pix * n + c];
      adj[(int64_t)c * N + pix] = g * ie;
      s = fmaf(g, out[pix * n + c], s);
    }
    adj[(int64_t)n * N + pix] = -s * ie;
  }
}

template <int KB, int RB>
cudaError_t fb_launch(const float* guide, int64_t N, int rho, const float* lm, int K, float inv2s2r,
                      const float* what, const DevState* state, const float* dphi, float* dguide,
                      int add_into, float* gw_part, float* sr_part, cudaStream_t st) {
  const size_t smem = sizeof(float) * ((size_t)K * kpad4(K) + (size_t)((K * rho + 3) & ~3) +
                                       (size_t)2 * kFbThreads * KB +
                                       (RB == 0 ? (size_t)2 * kFbThreads * (rho | 1) : 0));
  cudaError_t e = cudaFuncSetAttribute(k_features_bwd<KB, RB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_features_bwd<KB, RB><<<fb_blocks(N), kFbThreads, smem, st>>>(guide, N, rho, lm, K, inv2s2r, what,
                                                             state, dphi, dguide, add_into,
                                                             gw_part, sr_part);
  count_launches(1);
  return cudaGetLastError();
}

template <int KB>
cudaError_t fb_rb(const float* guide, int64_t N, int rho, const float* lm, int K, float inv2s2r,
                  const float* what, const DevState* state, const float* dphi, float* dguide,
                  int add_into, float* gw_part, float* sr_part, cudaStream_t st) {
  if (rho <= 4)
    return fb_launch<KB, 4>(guide, N, rho, lm, K, inv2s2r, what, state, dphi, dguide, add_into,
                            gw_part, sr_part, st);
  if (rho <= 32)
    return fb_launch<KB, 32>(guide, N, rho, lm, K, inv2s2r, what, state, dphi, dguide, add_into,
                             gw_part, sr_part, st);
  const size_t rows = sizeof(float) * ((size_t)K * kpad4(K) + (size_t)((K * rho + 3) & ~3) +
                                       (size_t)2 * kFbThreads * KB + (size_t)2 * kFbThreads * (rho | 1));
  if (rows <= 227 * 1024)
    return fb_launch<KB, 0>(guide, N, rho, lm, K, inv2s2r, what, state, dphi, dguide, add_into,
                            gw_part, sr_part, st);
  return fb_launch<KB, -1>(guide, N, rho, lm, K, inv2s2r, what, state, dphi, dguide, add_into,
                           gw_part, sr_part, st);
}

}  // namespace

size_t backward_gpart_floats(int K) {
  return (size_t)kFbBlocks * K * K + kFbBlocks;
}

size_t backward_spart_floats(int H, int W, int n) {
  return (size_t)((W + 31) / 32) * ((H + 31) / 32) * (n + 1);
}

const double* eig_A64(const void* scratch);

cudaError_t launch_bwd_conv(const float* f, int H, int W, int n, int K, int spatial, float sigma_s,
                            int S, const void* phi, bool bf16, const float* eta, const float* out,
                            const float* grad_out, const float* cbuf, float* adj, float* grad_f,
                            float* dphi, float* spart, const DevState* state, cudaStream_t st,
                            int k_begin, int k_end) {
  const int Sc = conv_compiled_radius(S);
  if (Sc < 0) return cudaErrorInvalidValue;
  const int64_t N = (int64_t)H * W;
  const bool first = k_begin == 0;    // the first chunk of modes forms the adjoint planes
  if (first) {
    int64_t g = (N + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    k_adjoint<<<(int)g, 256, 0, st>>>(grad_out, out, eta, N, n, adj);
    count_launches(1);
  }
  const int chunks = bwd_chunks(Sc, n);
  const int slices = bwd_dphi_slices(Sc, n);
  cudaError_t e;
  if (chunks > 1 && slices == 1 && first) {
    e = cudaMemsetAsync(dphi, 0, sizeof(float) * (size_t)K * N, st);
    if (e != cudaSuccess) return e;
  }
  BwdArgs a;
  a.f = f;
  a.H = H;
  a.W = W;
  a.n = n;
  a.N = N;
  a.phi = phi;
  a.bf16 = bf16 ? 1 : 0;
  a.state = state;
  a.adj = adj;
  a.cbuf = cbuf;
  a.box = spatial == NYF_BOX ? 1 : 0;
  // taps of the window and their sigma_s derivative, g'(t) = g(t) t^2 / sigma_s^3, for
  // t >= 0 (both even in t), zero beyond the true radius (the compiled radius Sc may be larger)
  for (int t = 0; t <= kMaxTapRadius; ++t) {
    float g = 0.f, gd = 0.f;
    if (t <= S) {
      if (a.box) {
        g = 1.f;
      } else {
        const double s = (double)sigma_s, e = exp(-(double)t * t / (2.0 * s * s));
        g = (float)e;
        gd = (float)(e * t * t / (s * s * s));
      }
    }
    a.tg[t] = make_float2(g, g);
    a.td[t] = make_float2(gd, gd);
  }
  a.k_begin = k_begin;
  a.k_end = k_end;
  a.accumulate = first ? 0 : 1;
  a.dphi = dphi;
  // two slices: atomic adds onto zero (commutative, so still one result); more:
  // a plane set per slice, summed in slice order below
  a.atomic_dphi = (chunks > 1 && slices == 1) ? 1 : 0;
  a.dphi_slice = slices > 1 ? (int64_t)K * N : 0;
  a.df = grad_f;
  a.sig_part = spart;
  e = Sc <= 8 ? bwd_dispatch_a(Sc, a, st) : (Sc <= 16 ? bwd_dispatch_b(Sc, a, st) : bwd_dispatch_c(Sc, a, st));
  if (e != cudaSuccess || slices == 1) return e;
  int64_t g = ((int64_t)(k_end - k_begin) * N + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  k_dphi_slices<<<(int)g, 256, 0, st>>>(dphi, slices, (int64_t)K * N, N, k_begin, k_end, state);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_bwd_features(const float* f, const float* guide, int H, int W, int n, int rho,
                                const float* landmarks, int K, float sigma_r, int S,
                                const float* what, const float* dphi, float* grad_f,
                                float* grad_guide, float* gpart, const float* spart, double* gw,
                                const void* eig_scratch, float* grad_sigma, DevState* state,
                                cudaStream_t st) {
  const int Sc = conv_compiled_radius(S);
  if (Sc < 0) return cudaErrorInvalidValue;
  const int64_t N = (int64_t)H * W;
  // the guide gradient goes into grad_f when the guide is the image
  const bool tied = guide == f;
  float* dguide = tied ? grad_f : grad_guide;
  const int add_into = tied ? 1 : 0;
  const float inv2s2r = (float)(1.0 / (2.0 * (double)sigma_r * sigma_r));
  float* gw_part = gpart;
  float* sr_part = gpart + (size_t)kFbBlocks * K * K;
  double* Z = gw + (size_t)K * K;
  double* rowdot = Z + (size_t)K * K;
  double* AD2 = rowdot + K;
  k_tail_ad2<<<K, kMaxK, 0, st>>>(K, rho, landmarks, eig_A64(eig_scratch), AD2);
  k_tail_z<<<K, kMaxK, 0, st>>>(K, what, AD2, state, Z);
  count_launches(2);
  cudaError_t e;
  if (K <= 8) e = fb_rb<8>(guide, N, rho, landmarks, K, inv2s2r, what, state, dphi, dguide, add_into, gw_part, sr_part, st);
  else if (K <= 16) e = fb_rb<16>(guide, N, rho, landmarks, K, inv2s2r, what, state, dphi, dguide, add_into, gw_part, sr_part, st);
  else if (K <= 32) e = fb_rb<32>(guide, N, rho, landmarks, K, inv2s2r, what, state, dphi, dguide, add_into, gw_part, sr_part, st);
  else e = fb_rb<64>(guide, N, rho, landmarks, K, inv2s2r, what, state, dphi, dguide, add_into, gw_part, sr_part, st);
  if (e != cudaSuccess) return e;
  k_gw_reduce<<<K, 256, 0, st>>>(gw_part, fb_blocks(N), K, Z, gw, rowdot);
  count_launches(1);
  const int64_t n_ss = bwd_ctas(Sc, H, W, n);
  k_bwd_tail<<<1, 256, 0, st>>>(K, sigma_r, rowdot, sr_part, fb_blocks(N), spart, n_ss, state,
                                grad_sigma);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace nyf

// PCA-NLM (Sec. IV, after Tasdizen's principal-neighbourhood NLM): the NLM
// guide p(x), the colour patch of radius r around x (reflect-101 border,
// components ordered (dy, dx, c)), is replaced by its coordinates in the q
// leading principal directions of the image's patches:
//     m = (1/N) sum_x p(x),   C = (1/N) sum_x (p(x) - m)(p(x) - m)^T = U diag(lambda) U^T,
//     p~(x) = U_q^T (p(x) - m).
// Kernels:
//   k_channel_sums  per-channel FP64 partial sums (the shift s: patches are
//                   accumulated as p(x) - s so that C = G/N - m' m'^T does not
//                   cancel digits);
//   k_patch_gram    persistent CTAs over 16 x 16 pixel tiles; each thread owns
//                   up to four 4 x 4 blocks of the upper triangle of the Gram
//                   matrix sum (p - s)(p - s)^T (FP32 within a CTA, one partial
//                   per CTA);
//   k_gram_reduce   FP64 sum of the partials, the covariance and the mean;
//   k_jacobi_pca    one CTA: cyclic Jacobi with round-robin ordering on the
//                   rho x rho covariance in FP32 (shared memory), eigenvalues
//                   sorted descending, the q leading eigenvectors;
//   k_pca_project   p~(x) for every pixel (16 x 16 tiles, one thread per pixel).
#include <math.h>

#include "nyf_internal.cuh"

namespace nyf {
namespace {

constexpr int kTile = 16;
constexpr int kGramThreads = 256;
constexpr int kGramCtas = 2 * 152;
constexpr int kBpt = 4;                 // Gram blocks per thread
constexpr int kSumCtas = 152;
constexpr int kJacobiThreads = 512;
constexpr int kJacobiSweeps = 20;
constexpr uint32_t kStatusJacobi = NYF_ERR_TIMEOUT;

__device__ inline int reflect101(int i, int n) {
  if (n == 1) return 0;
  const int period = 2 * (n - 1);
  int j = i % period;
  if (j < 0) j += period;
  return j < n ? j : period - j;
}

// ---- per-channel sums (FP64), one partial per CTA and channel
__global__ void k_channel_sums(const float* __restrict__ f, int64_t N, int n, double* __restrict__ part) {
  __shared__ double red[256];
  for (int c = 0; c < n; ++c) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
      s += (double)f[i * n + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x * n + c] = red[0];
    __syncthreads();
  }
}

__global__ void k_shift(const double* __restrict__ part, int nparts, int n, int64_t N, float* __restrict__ shift) {
  const int c = threadIdx.x;
  if (c >= n) return;
  double s = 0.0;
  for (int b = 0; b < nparts; ++b) s += part[b * n + c];
  shift[c] = (float)(s / (double)N);
}

// ---- Gram partials of the shifted patches
// rp = rho rounded up to a multiple of 4; nb = rp / 4 blocks per side; the
// upper triangle (bi <= bj) has nb (nb + 1) / 2 blocks, thread t owns blocks
// t, t + 256, ... (at most kBpt).  part layout per CTA: [block][4][4] then rp sums.
__global__ void __launch_bounds__(kGramThreads, 2) k_patch_gram(const float* __restrict__ f, int H, int W, int n,
                                                             int r, int rho, const float* __restrict__ shift,
                                                             float* __restrict__ part) {
  extern __shared__ float sm[];
  const int side = 2 * r + 1;
  const int TS = kTile + 2 * r;
  const int rp = (rho + 3) & ~3, nb = rp / 4, nblk = nb * (nb + 1) / 2;
  // TS * TS * n tile, then TS * TS * n zeros: a padding component reads
  // pb[zero_off] with pb inside the tile, which lands inside the zeros
  float* tile = sm;
  const int zero_off = TS * TS * n;
  const int tid = threadIdx.x;
  // component offsets of this thread's blocks (relative to a pixel's base)
  int offi[kBpt][4], offj[kBpt][4];
  bool own[kBpt];
#pragma unroll
  for (int s = 0; s < kBpt; ++s) {
    const int b = tid + s * kGramThreads;
    own[s] = b < nblk;
    int bi = 0, rem = own[s] ? b : 0;
    while (rem >= nb - bi) {                    // row bi of the triangle holds nb - bi blocks
      rem -= nb - bi;
      ++bi;
    }
    const int bj = bi + rem;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int ci = 4 * bi + e, cj = 4 * bj + e;
      offi[s][e] = ci < rho ? ((ci / n) / side * TS + (ci / n) % side) * n + ci % n : zero_off;
      offj[s][e] = cj < rho ? ((cj / n) / side * TS + (cj / n) % side) * n + cj % n : zero_off;
    }
  }
  const int offs = tid < rho ? ((tid / n) / side * TS + (tid / n) % side) * n + tid % n : zero_off;
  float acc[kBpt][16];
#pragma unroll
  for (int s = 0; s < kBpt; ++s)
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[s][e] = 0.f;
  float psum = 0.f;
  for (int e = tid; e < zero_off; e += kGramThreads) tile[zero_off + e] = 0.f;
  const int tx_n = (W + kTile - 1) / kTile, ty_n = (H + kTile - 1) / kTile;
  for (int t = blockIdx.x; t < tx_n * ty_n; t += gridDim.x) {
    const int y0 = (t / tx_n) * kTile, x0 = (t % tx_n) * kTile;
    __syncthreads();
    for (int e = tid; e < TS * TS * n; e += kGramThreads) {
      const int c = e % n, q = e / n;
      const int yy = q / TS, xx = q % TS;
      const int gy = reflect101(y0 - r + yy, H), gx = reflect101(x0 - r + xx, W);
      tile[e] = f[((int64_t)gy * W + gx) * n + c] - shift[c];
    }
    __syncthreads();
    const int ny = min(kTile, H - y0), nx = min(kTile, W - x0);
    for (int py = 0; py < ny; ++py)
      for (int px = 0; px < nx; ++px) {
        const float* pb = tile + (py * TS + px) * n;
        psum += tid < rp ? pb[offs] : 0.f;
#pragma unroll
        for (int s = 0; s < kBpt; ++s)
          if (own[s]) {
            float a[4], b[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              a[e] = pb[offi[s][e]];
              b[e] = pb[offj[s][e]];
            }
#pragma unroll
            for (int e = 0; e < 4; ++e)
#pragma unroll
              for (int g = 0; g < 4; ++g) acc[s][e * 4 + g] = fmaf(a[e], b[g], acc[s][e * 4 + g]);
          }
      }
  }
  float* out = part + (size_t)blockIdx.x * ((size_t)nblk * 16 + rp);
#pragma unroll
  for (int s = 0; s < kBpt; ++s)
    if (own[s])
#pragma unroll
      for (int e = 0; e < 16; ++e) out[(size_t)(tid + s * kGramThreads) * 16 + e] = acc[s][e];
  if (tid < rp) out[(size_t)nblk * 16 + tid] = psum;
}

// ---- FP64 reduction: covariance C (rp x rp float, padding zero) and the mean
__global__ void k_gram_reduce(const float* __restrict__ part, int nparts, int rho, int64_t N,
                              const float* __restrict__ shift, int n, float* __restrict__ C,
                              float* __restrict__ mean) {
  const int rp = (rho + 3) & ~3, nb = rp / 4, nblk = nb * (nb + 1) / 2;
  const size_t stride = (size_t)nblk * 16 + rp;
  const int i = blockIdx.x;                      // row of C
  __shared__ double msh[160];
  for (int k = threadIdx.x; k < rp; k += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += (double)part[b * stride + (size_t)nblk * 16 + k];
    msh[k] = k < rho ? s / (double)N : 0.0;
  }
  __syncthreads();
  const int bi_row = i / 4, ei = i % 4;
  for (int j = threadIdx.x; j < rp; j += blockDim.x) {
    const int a = min(i, j), b = max(i, j);
    const int ba = a / 4, bb = b / 4;
    const int blk = ba * nb - ba * (ba - 1) / 2 + (bb - ba);
    const int e = (a == i ? ei : j % 4) * 4 + (a == i ? j % 4 : ei);
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += (double)part[p * stride + (size_t)blk * 16 + e];
    const double cij = (i < rho && j < rho) ? s / (double)N - msh[i] * msh[j] : 0.0;
    C[(size_t)i * rp + j] = (float)cij;
  }
  (void)bi_row;
  if (i < rho && threadIdx.x == 0) mean[i] = (float)(msh[i] + (double)shift[i % n]);
}

// ---- one-CTA Jacobi on the rp x rp covariance (FP32), then sort and basis
__global__ void __launch_bounds__(kJacobiThreads) k_jacobi_pca(const float* __restrict__ C, int rho, int q,
                                                               float* __restrict__ eigvals,
                                                               float* __restrict__ basis,
                                                               DevState* state) {
  extern __shared__ float smj[];
  const int rp = (rho + 3) & ~3;                 // even
  const int ld = rp + 1;
  float* A = smj;                                // rp x ld
  float* V = A + rp * ld;                        // rp x ld
  float* cs = V + rp * ld;                       // rp / 2 cosines
  float* sn = cs + rp / 2;                       // rp / 2 sines
  int* top = reinterpret_cast<int*>(sn + rp / 2);
  int* bot = top + rp / 2;
  int* order = bot + rp / 2;                     // rp
  __shared__ float red[kJacobiThreads / 32];
  __shared__ int done;
  const int tid = threadIdx.x, m = rp / 2;
  const int warp = tid >> 5, lane = tid & 31, nwarp = blockDim.x >> 5;
  for (int e = tid; e < rp * rp; e += blockDim.x) {
    const int i = e / rp, j = e % rp;
    A[i * ld + j] = C[e];
    V[i * ld + j] = i == j ? 1.f : 0.f;
  }
  __syncthreads();
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    // off-diagonal and total squared norms
    float off = 0.f, tot = 0.f;
    for (int e = tid; e < rp * rp; e += blockDim.x) {
      const int i = e / rp, j = e % rp;
      const float a = A[i * ld + j];
      tot += a * a;
      if (i != j) off += a * a;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if ((tid & 31) == 0) red[tid >> 5] = off;
    __syncthreads();
    if (tid == 0) {
      float so = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) so += red[w];
      red[0] = so;
    }
    __syncthreads();
    const float offs = red[0];
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = tot;
    __syncthreads();
    if (tid == 0) {
      float st = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) st += red[w];
      done = offs <= 1e-13f * st;
      if (sweep == kJacobiSweeps - 1 && !done) atomicCAS(&state->status, 0, (int)kStatusJacobi);
    }
    __syncthreads();
    if (done) break;
    for (int step = 0; step < rp - 1; ++step) {
      // circle-method pairing in closed form: index rp - 1 meets `step`, and
      // (step + k, step - k) mod (rp - 1) for k = 1 .. m - 1
      for (int k = tid; k < m; k += blockDim.x) {
        const int a0 = k == 0 ? step : (step + k) % (rp - 1);
        const int b0 = k == 0 ? rp - 1 : (step - k + rp - 1) % (rp - 1);
        const int p = min(a0, b0), qq = max(a0, b0);
        top[k] = p;
        bot[k] = qq;
        const float apq = A[p * ld + qq];
        float c = 1.f, s = 0.f;
        if (fabsf(apq) > 1e-30f) {
          const float tau = (A[qq * ld + qq] - A[p * ld + p]) / (2.f * apq);
          const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
          c = rsqrtf(1.f + t * t);
          s = t * c;
        }
        cs[k] = c;
        sn[k] = s;
      }
      __syncthreads();
      for (int k = warp; k < m; k += nwarp) {               // rows p, q of A
        const int p = top[k], qq = bot[k];
        const float c = cs[k], s = sn[k];
        for (int j = lane; j < rp; j += 32) {
          const float a = A[p * ld + j], b = A[qq * ld + j];
          A[p * ld + j] = c * a - s * b;
          A[qq * ld + j] = s * a + c * b;
        }
      }
      __syncthreads();
      for (int k = warp; k < m; k += nwarp) {               // columns p, q of A and V
        const int p = top[k], qq = bot[k];
        const float c = cs[k], s = sn[k];
        for (int i = lane; i < rp; i += 32) {
          const float a = A[i * ld + p], b = A[i * ld + qq];
          A[i * ld + p] = c * a - s * b;
          A[i * ld + qq] = s * a + c * b;
          const float va = V[i * ld + p], vb = V[i * ld + qq];
          V[i * ld + p] = c * va - s * vb;
          V[i * ld + qq] = s * va + c * vb;
        }
      }
      __syncthreads();
    }
  }
  // eigenvalues as Rayleigh quotients v_i^T C v_i / v_i^T v_i on the unrotated
  // covariance: the diagonal the rotations leave, and the norms of the
  // accumulated FP32 columns, carry their rounding (~1e-5 of lambda_max at
  // rho = 147); C V (FP32, into A's storage) and the quotients (FP64 sums) are
  // accurate to ~1e-6.
  for (int a = warp; a < rp; a += nwarp)
    for (int i = lane; i < rp; i += 32) {
      float s = 0.f;
      for (int b = 0; b < rp; ++b) s = fmaf(C[(size_t)a * rp + b], V[b * ld + i], s);
      A[a * ld + i] = s;
    }
  __syncthreads();
  float* lam = cs;                               // rp floats (cs and sn are contiguous)
  for (int i = tid; i < rp; i += blockDim.x) {   // v^T C v / v^T v: the FP32 columns drift off unit norm
    double l = 0.0, nn = 0.0;
    for (int a = 0; a < rp; ++a) {
      const double va = (double)V[a * ld + i];
      l += va * (double)A[a * ld + i];
      nn += va * va;
    }
    lam[i] = (float)(nn > 0.0 ? l / nn : 0.0);
  }
  __syncthreads();
  // rank of each real eigenvalue (descending, ties by index); padding ranks last
  for (int i = tid; i < rp; i += blockDim.x) {
    int rank = 0;
    const float li = i < rho ? lam[i] : -INFINITY;
    for (int j = 0; j < rp; ++j) {
      const float lj = j < rho ? lam[j] : -INFINITY;
      rank += (lj > li) || (lj == li && j < i);
    }
    order[rank] = i;
  }
  __syncthreads();
  for (int k = tid; k < rho; k += blockDim.x) eigvals[k] = lam[order[k]];
  for (int e = tid; e < rho * q; e += blockDim.x) {
    const int i = e / q, j = e % q;
    basis[e] = V[i * ld + order[j]];
  }
}

// ---- the q output columns re-orthonormalised in FP64 by classical Gram-Schmidt
// applied twice (CGS2): the FP32 rotations leave them orthonormal only to
// ~1e-4.  All dot products of one column are taken at once (a warp per earlier
// column), so a column costs four barriers.
__global__ void k_orthonormalize(float* __restrict__ basis, int rho, int q) {
  __shared__ double v[160];
  __shared__ double d[32];
  __shared__ double red[8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarp = blockDim.x >> 5;
  for (int j = 0; j < q; ++j) {
    for (int i = tid; i < rho; i += blockDim.x) v[i] = (double)basis[i * q + j];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int k = warp; k < j; k += nwarp) {          // d_k = u_k . v
        double s = 0.0;
        for (int i = lane; i < rho; i += 32) s += v[i] * (double)basis[i * q + k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) d[k] = s;
      }
      __syncthreads();
      for (int i = tid; i < rho; i += blockDim.x) {     // v -= sum_k d_k u_k
        double t = v[i];
        for (int k = 0; k < j; ++k) t -= d[k] * (double)basis[i * q + k];
        v[i] = t;
      }
      __syncthreads();
    }
    double nn = 0.0;
    for (int i = tid; i < rho; i += blockDim.x) nn += v[i] * v[i];
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    if (lane == 0) red[warp] = nn;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < nwarp; ++w) tot += red[w];
    const double inv = tot > 0.0 ? 1.0 / sqrt(tot) : 0.0;
    for (int i = tid; i < rho; i += blockDim.x) basis[i * q + j] = (float)(v[i] * inv);
    __syncthreads();
  }
}

// ---- p~(x) = U_q^T (p(x) - m), one thread per pixel of a 16 x 16 tile
template <int QB>
__global__ void __launch_bounds__(kTile * kTile) k_pca_project(const float* __restrict__ f, int H, int W, int n,
                                                               int r, int q, const float* __restrict__ mean,
                                                               const float* __restrict__ basis,
                                                               float* __restrict__ guide) {
  extern __shared__ float smp[];
  const int side = 2 * r + 1;
  const int rho = side * side * n;
  const int TS = kTile + 2 * r;
  float* U = smp;                                 // rho x QB (zero beyond q)
  float* mu = U + rho * QB;                       // rho
  float* tile = mu + rho;                         // TS * TS * n
  const int tid = threadIdx.x;
  const int y0 = blockIdx.y * kTile, x0 = blockIdx.x * kTile;
  for (int e = tid; e < rho * QB; e += blockDim.x) {
    const int i = e / QB, j = e % QB;
    U[e] = j < q ? basis[i * q + j] : 0.f;
  }
  for (int e = tid; e < rho; e += blockDim.x) mu[e] = mean[e];
  for (int e = tid; e < TS * TS * n; e += blockDim.x) {
    const int c = e % n, qq = e / n;
    const int yy = qq / TS, xx = qq % TS;
    const int gy = reflect101(y0 - r + yy, H), gx = reflect101(x0 - r + xx, W);
    tile[e] = f[((int64_t)gy * W + gx) * n + c];
  }
  __syncthreads();
  const int ty = tid / kTile, tx = tid % kTile;
  const int y = y0 + ty, x = x0 + tx;
  if (y >= H || x >= W) return;
  float acc[QB];
#pragma unroll
  for (int j = 0; j < QB; ++j) acc[j] = 0.f;
  int i = 0;
  for (int dy = 0; dy < side; ++dy)
    for (int dx = 0; dx < side; ++dx)
      for (int c = 0; c < n; ++c, ++i) {
        const float v = tile[((ty + dy) * TS + (tx + dx)) * n + c] - mu[i];
        const float4* u4 = reinterpret_cast<const float4*>(U + i * QB);
#pragma unroll
        for (int j4 = 0; j4 < QB / 4; ++j4) {
          const float4 u = u4[j4];
          acc[4 * j4 + 0] = fmaf(v, u.x, acc[4 * j4 + 0]);
          acc[4 * j4 + 1] = fmaf(v, u.y, acc[4 * j4 + 1]);
          acc[4 * j4 + 2] = fmaf(v, u.z, acc[4 * j4 + 2]);
          acc[4 * j4 + 3] = fmaf(v, u.w, acc[4 * j4 + 3]);
        }
      }
  float* g = guide + ((int64_t)y * W + x) * q;
#pragma unroll
  for (int j = 0; j < QB; ++j)
    if (j < q) g[j] = acc[j];
}

template <int QB>
cudaError_t project_launch(const float* f, int H, int W, int n, int r, int q, const float* mean,
                           const float* basis, float* guide, cudaStream_t st) {
  const int rho = (2 * r + 1) * (2 * r + 1) * n;
  const int TS = kTile + 2 * r;
  const size_t smem = sizeof(float) * ((size_t)rho * QB + rho + (size_t)TS * TS * n);
  cudaError_t e = cudaFuncSetAttribute(k_pca_project<QB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((W + kTile - 1) / kTile, (H + kTile - 1) / kTile);
  k_pca_project<QB><<<grid, kTile * kTile, smem, st>>>(f, H, W, n, r, q, mean, basis, guide);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

// Scratch of the moments + eigendecomposition (bytes, 256-aligned pieces).
size_t pca_scratch_bytes(int n, int r) {
  const int rho = (2 * r + 1) * (2 * r + 1) * n;
  const int rp = (rho + 3) & ~3, nb = rp / 4, nblk = nb * (nb + 1) / 2;
  auto a256 = [](size_t v) { return (v + 255) & ~(size_t)255; };
  return a256(sizeof(double) * kSumCtas * n) + a256(sizeof(float) * 64) +
         a256(sizeof(float) * kGramCtas * ((size_t)nblk * 16 + rp)) + a256(sizeof(float) * (size_t)rp * rp);
}

size_t pca_jacobi_smem(int rho) {
  const int rp = (rho + 3) & ~3;
  return sizeof(float) * (2 * (size_t)rp * (rp + 1) + rp) + sizeof(int) * (size_t)(rp + rp);
}

cudaError_t launch_patch_pca(const float* f, int H, int W, int n, int r, int q, void* scratch,
                             float* mean, float* basis, float* eigvals, DevState* state,
                             cudaStream_t st) {
  const int rho = (2 * r + 1) * (2 * r + 1) * n;
  const int rp = (rho + 3) & ~3, nb = rp / 4, nblk = nb * (nb + 1) / 2;
  if (rho > 160 || q < 1 || q > rho) return cudaErrorInvalidValue;
  auto a256 = [](size_t v) { return (v + 255) & ~(size_t)255; };
  char* w = reinterpret_cast<char*>(scratch);
  double* csum = reinterpret_cast<double*>(w);
  w += a256(sizeof(double) * kSumCtas * n);
  float* shift = reinterpret_cast<float*>(w);
  w += a256(sizeof(float) * 64);
  float* part = reinterpret_cast<float*>(w);
  w += a256(sizeof(float) * kGramCtas * ((size_t)nblk * 16 + rp));
  float* C = reinterpret_cast<float*>(w);
  const int64_t N = (int64_t)H * W;
  k_channel_sums<<<kSumCtas, 256, 0, st>>>(f, N, n, csum);
  k_shift<<<1, 64, 0, st>>>(csum, kSumCtas, n, N, shift);
  const int TS = kTile + 2 * r;
  const size_t gsm = sizeof(float) * 2 * (size_t)TS * TS * n;
  cudaError_t e = cudaFuncSetAttribute(k_patch_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
  if (e != cudaSuccess) return e;
  k_patch_gram<<<kGramCtas, kGramThreads, gsm, st>>>(f, H, W, n, r, rho, shift, part);
  k_gram_reduce<<<rp, 128, 0, st>>>(part, kGramCtas, rho, N, shift, n, C, mean);
  const size_t jsm = pca_jacobi_smem(rho);
  e = cudaFuncSetAttribute(k_jacobi_pca, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jsm);
  if (e != cudaSuccess) return e;
  k_jacobi_pca<<<1, kJacobiThreads, jsm, st>>>(C, rho, q, eigvals, basis, state);
  k_orthonormalize<<<1, 256, 0, st>>>(basis, rho, q);
  count_launches(6);
  return cudaGetLastError();
}

cudaError_t launch_pca_project(const float* f, int H, int W, int n, int r, int q, const float* mean,
                               const float* basis, float* guide, cudaStream_t st) {
  if (q <= 8) return project_launch<8>(f, H, W, n, r, q, mean, basis, guide, st);
  if (q <= 16) return project_launch<16>(f, H, W, n, r, q, mean, basis, guide, st);
  if (q <= 32) return project_launch<32>(f, H, W, n, r, q, mean, basis, guide, st);
  return cudaErrorInvalidValue;
}

}  // namespace nyf

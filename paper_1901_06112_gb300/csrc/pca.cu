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
//   k_eig_pca       one CTA: Householder tridiagonalisation, bisection for every
//                   eigenvalue and inverse iteration for the q leading
//                   eigenvectors, in FP32 (shared memory);
//   k_orthonormalize the q columns re-orthonormalised in FP64;
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

// ---- one-CTA symmetric eigensolver for the rho x rho covariance (FP32):
//   1. Householder tridiagonalisation T = Q^T C Q (reflector k kept in the
//      zeroed column k of A; warps over rows, lanes along rows);
//   2. every eigenvalue of T by bisection on Sturm counts (one thread each;
//      the count is the number of negative pivots of the LDL^T factorisation
//      of T - x I);
//   3. the q leading eigenvectors of T by inverse iteration (4 steps from a
//      fixed start vector; tridiagonal Gaussian elimination with partial
//      pivoting on lane 0 of warp 0), each step reorthogonalised against the
//      earlier vectors whose eigenvalues lie within 1e-3 ||T|| (a cluster);
//   4. back-transformation u = Q x through the reflectors (a warp per vector).
// Every loop has a fixed trip count.
constexpr int kPcaSweeps = 20;

__device__ __forceinline__ float block_sum_f(float x, float* red, int tid) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((tid & 31) == 0) red[tid >> 5] = x;
  __syncthreads();
  float s = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;
}

__device__ __forceinline__ int pca_player(int pos, int step, int Kp) {
  return pos == 0 ? 0 : 1 + (pos - 1 + step) % (Kp - 1);
}

// ---- eigendecomposition of the rho x rho covariance (rho <= 160): parallel cyclic
// Jacobi in FP32 on one CTA.  Round-robin ("circle") ordering: at step s position
// 0 holds index 0 and position i > 0 index 1 + (i - 1 + s) mod (Kp - 1); position
// i meets position Kp - 1 - i, so the Kp / 2 rotations of a step act on disjoint
// index pairs and A' = J^T A J splits into independent 2 x 2 blocks (pair u, pair
// v) -> R_u^T [A]_uv R_v.  Each thread owns a fixed set of blocks and of V's
// column pairs per step, loads a chunk of them before storing it (no other thread
// touches them), and two barriers separate the steps.  Entries below FP32
// resolution of their diagonal are not rotated.  Eigenvalues are the final
// diagonal (descending), eigenvectors the columns of V; the q leading columns go
// to `basis` (re-orthonormalised in FP64 afterwards).
__global__ void __launch_bounds__(kJacobiThreads) k_eig_pca(const float* __restrict__ C, int rho, int q,
                                                            float* __restrict__ eigvals,
                                                            float* __restrict__ basis, DevState* state) {
  extern __shared__ float smj[];
  const int n = rho, rp = (rho + 3) & ~3, ld = n | 1;
  const int Kp = (n + 1) & ~1, half = Kp / 2;
  float* A = smj;                                // n x ld
  float* V = A + n * ld;                         // n x ld
  float* pc = V + n * ld;                        // rotation cosines (half)
  float* ps = pc + 80;                           // sines
  int* pp = reinterpret_cast<int*>(ps + 80);     // pair members p <= q (q = p: none)
  int* pq = pp + 80;
  int* ord = pq + 80;                            // eigenvalue order, descending (n)
  __shared__ float red[kJacobiThreads / 32];
  const int tid = threadIdx.x;
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    A[i * ld + j] = C[(size_t)i * rp + j];
    V[i * ld + j] = i == j ? 1.f : 0.f;
  }
  __syncthreads();
  const float diag2 = block_sum_f(tid < n ? A[tid * ld + tid] * A[tid * ld + tid] : 0.f, red, tid);
  float prev = INFINITY;
  int sweeps = 0;
  for (; sweeps < kPcaSweeps; ++sweeps) {
    float off = 0.f;
    for (int e = tid; e < n * n; e += blockDim.x) {
      const int i = e / n, j = e - i * n;
      if (i < j) off += A[i * ld + j] * A[i * ld + j];
    }
    off = block_sum_f(off, red, tid);
    if (off <= 1e-14f * diag2 || off == 0.f) break;
    if (off <= 1e-9f * diag2 && off > 0.25f * prev) break;   // FP32 noise floor reached
    prev = off;
    for (int step = 0; step < Kp - 1; ++step) {
      if (tid < half) {
        int a = pca_player(tid, step, Kp), b = pca_player(Kp - 1 - tid, step, Kp);
        if (a > b) { const int t = a; a = b; b = t; }
        float c = 1.f, sn = 0.f;
        if (b < n) {
          const float apq = A[a * ld + b], app = A[a * ld + a], aqq = A[b * ld + b];
          if (fabsf(apq) > 1e-30f * (fabsf(app) + fabsf(aqq)) && fabsf(apq) > 1e-36f) {
            const float theta = (aqq - app) / (2.f * apq);
            const float t = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(1.f + theta * theta));
            c = rsqrtf(1.f + t * t);
            sn = t * c;
          }
        } else {
          b = a;                                   // odd n: the dummy partner
        }
        pp[tid] = a;
        pq[tid] = b;
        pc[tid] = c;
        ps[tid] = sn;
      }
      __syncthreads();
      // 2 x 2 blocks of A, in chunks of 4 (loads of a chunk first, then its stores)
      for (int base = tid; base < half * half; base += 4 * kJacobiThreads) {
        float la[4][4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          const int e = base + o * kJacobiThreads;
          if (e < half * half) {
            const int u = e / half, v = e - u * half;
            const int pu = pp[u], qu = pq[u], pv = pp[v], qv = pq[v];
            la[o][0] = A[pu * ld + pv];
            la[o][1] = A[pu * ld + qv];
            la[o][2] = A[qu * ld + pv];
            la[o][3] = A[qu * ld + qv];
          }
        }
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          const int e = base + o * kJacobiThreads;
          if (e < half * half) {
            const int u = e / half, v = e - u * half;
            const int pu = pp[u], qu = pq[u], pv = pp[v], qv = pq[v];
            const float cu = pc[u], su = ps[u], cv = pc[v], sv = ps[v];
            const float r00 = cu * la[o][0] - su * la[o][2], r01 = cu * la[o][1] - su * la[o][3];
            const float r10 = su * la[o][0] + cu * la[o][2], r11 = su * la[o][1] + cu * la[o][3];
            const float n00 = cv * r00 - sv * r01, n01 = sv * r00 + cv * r01;
            const float n10 = cv * r10 - sv * r11, n11 = sv * r10 + cv * r11;
            if (pu == qu && pv == qv) {
              A[pu * ld + pv] = n00;
            } else if (pu == qu) {
              A[pu * ld + pv] = n00;
              A[pu * ld + qv] = n01;
            } else if (pv == qv) {
              A[pu * ld + pv] = n00;
              A[qu * ld + pv] = n10;
            } else {
              A[pu * ld + pv] = n00;
              A[qu * ld + qv] = n11;
              if (u == v) {                        // the annihilated pair
                A[pu * ld + qv] = 0.f;
                A[qu * ld + pv] = 0.f;
              } else {
                A[pu * ld + qv] = n01;
                A[qu * ld + pv] = n10;
              }
            }
          }
        }
      }
      // V <- V J: column pairs, in chunks of 8
      for (int base = tid; base < n * half; base += 8 * kJacobiThreads) {
        float lv[8][2];
#pragma unroll
        for (int o = 0; o < 8; ++o) {
          const int e = base + o * kJacobiThreads;
          if (e < n * half) {
            const int i = e / half, v = e - i * half;
            lv[o][0] = V[i * ld + pp[v]];
            lv[o][1] = V[i * ld + pq[v]];
          }
        }
#pragma unroll
        for (int o = 0; o < 8; ++o) {
          const int e = base + o * kJacobiThreads;
          if (e < n * half) {
            const int i = e / half, v = e - i * half;
            const int pv = pp[v], qv = pq[v];
            if (pv != qv) {
              V[i * ld + pv] = pc[v] * lv[o][0] - ps[v] * lv[o][1];
              V[i * ld + qv] = ps[v] * lv[o][0] + pc[v] * lv[o][1];
            }
          }
        }
      }
      __syncthreads();
    }
  }
  if (tid == 0 && sweeps == kPcaSweeps) set_status(state, NYF_ERR_TIMEOUT);
  // descending order of the diagonal (a permutation whatever the values: NaN last)
  if (tid < n) {
    const float x = A[tid * ld + tid];
    const float v = isnan(x) ? -INFINITY : x;
    int rk = 0;
    for (int j = 0; j < n; ++j) {
      const float y = A[j * ld + j];
      const float w = isnan(y) ? -INFINITY : y;
      rk += (w > v) || (w == v && j < tid);
    }
    ord[rk] = tid;
    if (!isfinite(x)) set_status(state, NYF_ERR_NUMERIC);
  }
  __syncthreads();
  for (int k = tid; k < rho; k += blockDim.x) eigvals[k] = A[ord[k] * ld + ord[k]];
  for (int e3 = tid; e3 < rho * q; e3 += blockDim.x) {
    const int i = e3 / q, j = e3 % q;
    basis[e3] = V[i * ld + ord[j]];
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
  const int ld = rho | 1;
  return sizeof(float) * (2 * (size_t)rho * ld + 4 * 80 + (size_t)rho);
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
  e = cudaFuncSetAttribute(k_eig_pca, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jsm);
  if (e != cudaSuccess) return e;
  k_eig_pca<<<1, kJacobiThreads, jsm, st>>>(C, rho, q, eigvals, basis, state);
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

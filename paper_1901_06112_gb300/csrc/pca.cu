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
//                   eigenvectors (all q at once, a warp per vector, with
//                   Gram-Schmidt inside clusters of close eigenvalues), in FP32
//                   (shared memory);
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
constexpr int kBisectIters = 64;
constexpr int kInvIters = 4;

__device__ __forceinline__ float block_sum_f(float x, float* red, int tid) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((tid & 31) == 0) red[tid >> 5] = x;
  __syncthreads();
  float s = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;
}

// Number of eigenvalues of the tridiagonal (d, e2 = e^2) strictly below x.
__device__ int sturm_count(const float* d, const float* e2, int n, float x, float pivmin) {
  int c = 0;
  float q = 1.f;
  for (int k = 0; k < n; ++k) {
    q = (d[k] - x) - (k > 0 ? __fdividef(e2[k - 1], q) : 0.f);   // |q| >= pivmin, a normal number
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

// Solves (T - shift I) y = x in place for the symmetric tridiagonal T (diagonal
// d, off-diagonal e, n rows) by Gaussian elimination with partial pivoting, one
// thread.  The row being eliminated is carried in registers (diagonal a,
// superdiagonal b; its next entry is always zero), so each step's dependency
// chain is a few arithmetic operations; U (pivot, first and second
// superdiagonal) goes to ua, u1, u2.  Zero pivots are replaced by `tiny`.
__device__ void tri_solve(const float* d, const float* e, int n, float shift, float tiny,
                          float* x, float* ua, float* u1, float* u2) {
  float a = d[0] - shift, b = n > 1 ? e[0] : 0.f;
  float xk = x[0];
  for (int k = 0; k < n - 1; ++k) {
    const float sub = e[k];
    const float an = d[k + 1] - shift;
    const float bn = k + 1 < n - 1 ? e[k + 1] : 0.f;
    const float xn = x[k + 1];
    if (fabsf(a) >= fabsf(sub)) {            // pivot: the carried row
      if (a == 0.f) a = tiny;
      const float m = __fdividef(sub, a);    // |m| <= 1, a normal
      ua[k] = a;
      u1[k] = b;
      u2[k] = 0.f;
      x[k] = xk;
      a = an - m * b;
      b = bn;
      xk = xn - m * xk;
    } else {                                 // pivot: the next row (|sub| > |a|)
      const float m = __fdividef(a, sub);
      ua[k] = sub;
      u1[k] = an;
      u2[k] = bn;
      x[k] = xn;
      a = b - m * an;
      b = -m * bn;
      xk = xk - m * xn;
    }
  }
  ua[n - 1] = a != 0.f ? a : tiny;
  u1[n - 1] = 0.f;
  u2[n - 1] = 0.f;
  x[n - 1] = xk;
  float x1 = 0.f, x2 = 0.f;                  // x[k + 1], x[k + 2]
  for (int k = n - 1; k >= 0; --k) {
    const float s = (x[k] - u1[k] * x1 - u2[k] * x2) / ua[k];
    x[k] = s;
    x2 = x1;
    x1 = s;
  }
}

__global__ void __launch_bounds__(kJacobiThreads) k_eig_pca(const float* __restrict__ C, int rho, int q,
                                                            float* __restrict__ eigvals,
                                                            float* __restrict__ basis, DevState* state) {
  extern __shared__ float smj[];
  const int n = rho, rp = (rho + 3) & ~3, ld = n | 1;
  float* A = smj;                                // n x ld
  float* X = A + n * ld;                         // q columns of n (eigenvectors of T, then of C)
  float* d = X + n * q;
  float* e = d + n;
  float* e2 = e + n;
  float* beta = e2 + n;
  float* lam = beta + n;                         // ascending
  float* vv = lam + n;                           // reflector / work vector
  float* pw = vv + n;                            // p, then w
  float* gwork = pw + n;                         // per warp: U factors of its solves (3 n)
  __shared__ float red[kJacobiThreads / 32];
  __shared__ float coef[32];                     // Gram-Schmidt coefficients (q <= 32)
  __shared__ float bounds[3];                    // lo, hi, ||T||
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarp = blockDim.x >> 5;
  (void)state;                                   // fixed trip counts: no status to latch
  for (int i = warp; i < n; i += nwarp)
    for (int j = lane; j < n; j += 32) A[i * ld + j] = C[(size_t)i * rp + j];
  __syncthreads();
  // ---- 1. tridiagonalisation
  for (int k = 0; k < n - 2; ++k) {
    float ss = 0.f;
    for (int i = k + 1 + tid; i < n; i += blockDim.x) ss += A[i * ld + k] * A[i * ld + k];
    const float sig = sqrtf(block_sum_f(ss, red, tid));
    const float x0 = A[(k + 1) * ld + k];
    if (!(sig > 0.f)) {                          // column already reduced (uniform)
      if (tid == 0) {
        e[k] = 0.f;
        beta[k] = 0.f;
      }
      __syncthreads();
      continue;
    }
    const float alpha = x0 >= 0.f ? -sig : sig;
    const float b = 1.f / (sig * (sig + fabsf(x0)));
    for (int i = k + 1 + tid; i < n; i += blockDim.x) vv[i] = i == k + 1 ? x0 - alpha : A[i * ld + k];
    __syncthreads();
    for (int i = k + 1 + warp; i < n; i += nwarp) {       // p = b B v
      float t = 0.f;
      for (int j = k + 1 + lane; j < n; j += 32) t = fmaf(A[i * ld + j], vv[j], t);
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) pw[i] = b * t;
    }
    __syncthreads();
    float vp = 0.f;
    for (int i = k + 1 + tid; i < n; i += blockDim.x) vp += vv[i] * pw[i];
    const float K = 0.5f * b * block_sum_f(vp, red, tid);
    for (int i = k + 1 + tid; i < n; i += blockDim.x) pw[i] -= K * vv[i];   // w
    __syncthreads();
    for (int i = k + 1 + warp; i < n; i += nwarp)            // B -= v w^T + w v^T
      for (int j = k + 1 + lane; j < n; j += 32)
        A[i * ld + j] -= vv[i] * pw[j] + pw[i] * vv[j];
    for (int i = k + 1 + tid; i < n; i += blockDim.x) A[i * ld + k] = vv[i];   // keep the reflector
    if (tid == 0) {
      e[k] = alpha;
      beta[k] = b;
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) e[n - 2] = A[(n - 1) * ld + (n - 2)];
    e[n - 1] = 0.f;
  }
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) {
    d[i] = A[i * ld + i];
    e2[i] = e[i] * e[i];
  }
  __syncthreads();
  if (tid == 0) {                                // Gershgorin interval and ||T||
    float lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < n; ++i) {
      const float rad = fabsf(e[i]) + (i > 0 ? fabsf(e[i - 1]) : 0.f);
      lo = fminf(lo, d[i] - rad);
      hi = fmaxf(hi, d[i] + rad);
    }
    bounds[0] = lo;
    bounds[1] = hi;
    bounds[2] = fmaxf(fabsf(lo), fabsf(hi));
  }
  __syncthreads();
  const float tnorm = bounds[2];
  const float eps = 1.1920929e-7f;
  const float pivmin = fmaxf(1e-30f, 1e-2f * eps * eps * tnorm * tnorm);
  // ---- 2. bisection: thread i finds the i-th smallest eigenvalue
  for (int i = tid; i < n; i += blockDim.x) {
    float a = bounds[0], b = bounds[1];
    for (int it = 0; it < kBisectIters; ++it) {
      const float mid = 0.5f * (a + b);
      if (!(mid > a && mid < b)) break;
      if (sturm_count(d, e2, n, mid, pivmin) <= i) a = mid;
      else b = mid;
      if (b - a <= 2.f * eps * fmaxf(fabsf(a), fabsf(b)) + pivmin) break;
    }
    lam[i] = 0.5f * (a + b);
  }
  __syncthreads();
  // ---- 3. inverse iteration for the q largest eigenvalues, all vectors at once: each
  // iteration solves (T - lam_j I) y_j = x_j for every j (a warp per vector, its lane 0
  // solving), then, in order of j, orthogonalises y_j against the y_i (i < j) whose
  // eigenvalues lie within ortol of lam_j (classical Gram-Schmidt) and normalises it
  {
    const float tiny = eps * tnorm, ortol = 1e-3f * tnorm;
    float* wa = gwork + warp * 3 * n;            // this warp's U factors
    for (int e3 = tid; e3 < q * n; e3 += blockDim.x) {
      const int j = e3 / n, i = e3 - j * n;
      X[e3] = (float)((37 * (i + 1) + 11 * j) % 97) / 97.f - 0.5f;
    }
    __syncthreads();
    for (int it = 0; it < kInvIters; ++it) {
      for (int j = warp; j < q; j += nwarp)
        if (lane == 0) tri_solve(d, e, n, lam[n - 1 - j], tiny, X + j * n, wa, wa + n, wa + 2 * n);
      __syncthreads();
      for (int j = 0; j < q; ++j) {
        float* xj = X + j * n;
        const float lj = lam[n - 1 - j];
        bool any = false;                          // uniform: an earlier vector of its cluster
        for (int i2 = 0; i2 < j; ++i2) any |= fabsf(lam[n - 1 - i2] - lj) < ortol;
        if (any) {
          for (int i2 = warp; i2 < j; i2 += nwarp) {
            float dt = 0.f;
            if (fabsf(lam[n - 1 - i2] - lj) < ortol) {
              const float* xi = X + i2 * n;
              for (int i = lane; i < n; i += 32) dt = fmaf(xi[i], xj[i], dt);
              for (int o = 16; o > 0; o >>= 1) dt += __shfl_xor_sync(0xffffffffu, dt, o);
            }
            if (lane == 0) coef[i2] = dt;
          }
          __syncthreads();
          for (int c = tid; c < n; c += blockDim.x) {
            float v = xj[c];
            for (int i2 = 0; i2 < j; ++i2) v = fmaf(-coef[i2], X[i2 * n + c], v);
            xj[c] = v;
          }
          __syncthreads();
        }
        float nn = 0.f;
        for (int c = tid; c < n; c += blockDim.x) nn = fmaf(xj[c], xj[c], nn);
        nn = block_sum_f(nn, red, tid);
        const float inv = nn > 0.f ? rsqrtf(nn) : 0.f;
        for (int c = tid; c < n; c += blockDim.x) xj[c] *= inv;
        __syncthreads();
      }
    }
  }
  // ---- 4. u_j = H_0 H_1 ... H_{n-3} x_j, a warp per vector
  for (int j = warp; j < q; j += nwarp) {
    float* x = X + j * n;
    for (int k = n - 3; k >= 0; --k) {
      const float bk = beta[k];
      if (bk == 0.f) continue;
      float dt = 0.f;
      for (int i = k + 1 + lane; i < n; i += 32) dt += A[i * ld + k] * x[i];
      for (int o = 16; o > 0; o >>= 1) dt += __shfl_xor_sync(0xffffffffu, dt, o);
      for (int i = k + 1 + lane; i < n; i += 32) x[i] -= bk * dt * A[i * ld + k];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int k = tid; k < rho; k += blockDim.x) eigvals[k] = lam[n - 1 - k];
  for (int e3 = tid; e3 < rho * q; e3 += blockDim.x) {
    const int i = e3 / q, j = e3 % q;
    basis[e3] = X[j * n + i];
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
  return sizeof(float) * ((size_t)rho * ld + (size_t)rho * 32 + 9 * (size_t)rho +
                          3 * (size_t)rho * (kJacobiThreads / 32));
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

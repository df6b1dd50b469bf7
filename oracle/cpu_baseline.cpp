// CPU baseline (test and benchmark infrastructure, not the oracle and not the
// product): the forward Nystrom bilateral filter of Algorithm 1 in FP32 C++
// with OpenMP, the same algorithm as the GPU path, for timing on the host's
// cores beside the GPU.  Only bench.py's CPU-baseline leg and its CPU test load
// it.  It shares no code with the CUDA path.
//
// Steps (Sec. III, Algorithm 1):
//   1. k-means landmarks (Sec. III): initial rows = the first K distinct values of
//      SplitMix64(seed) mod N (Steele, Lea & Flood 2014), `iters` Lloyd iterations
//      (assignment in FP32, ties to the lowest index; centroid sums in FP64; an empty
//      cluster keeps its centroid) -- unless landmarks are given;
//   2. A(i, j) = kappa(mu_i, mu_j) (Eq. (9)) in FP64, eigenpairs by cyclic Jacobi in
//      FP64 (Eq. (10)), modes with alpha_k > tau alpha_max kept, and the symmetric
//      factor W = W_r Lambda_r^(-1/2) W_r^T;
//   3. phi_j(x) = sum_m kappa(p(x), mu_m) W(m, j) (Eqs. (11)-(12)) in FP32;
//   4. per mode, the zero-padded separable FIR of phi_j f_c and phi_j (Eq. (7),
//      omega(z) = exp(-|z|^2 / 2 sigma_s^2) on |z|_inf <= S), accumulated into
//      zeta and eta (Eqs. (14)-(15)); g_hat = zeta / eta.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

uint64_t mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// output t (t >= 1) of the SplitMix64 stream whose state starts at `seed`
uint64_t splitmix(uint64_t seed, uint64_t t) { return mix(seed + t * 0x9E3779B97F4A7C15ull); }

void kmeans(const float* X, int64_t N, int d, int K, int iters, uint64_t seed, float* mu) {
  std::vector<int64_t> init;
  for (uint64_t t = 1; (int)init.size() < K && t < 1000000; ++t) {
    const int64_t i = (int64_t)(splitmix(seed, t) % (uint64_t)N);
    if (std::find(init.begin(), init.end(), i) == init.end()) init.push_back(i);
  }
  for (int k = 0; k < K; ++k)
    for (int c = 0; c < d; ++c) mu[k * d + c] = X[init[k] * d + c];
  std::vector<int> lab(N);
  for (int it = 0; it < iters; ++it) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
      int best = 0;
      float bd = INFINITY;
      for (int k = 0; k < K; ++k) {
        float s = 0.f;
        for (int c = 0; c < d; ++c) {
          const float t = X[i * d + c] - mu[k * d + c];
          s += t * t;
        }
        if (s < bd) {
          bd = s;
          best = k;
        }
      }
      lab[i] = best;
    }
    std::vector<double> sum((size_t)K * d, 0.0);
    std::vector<int64_t> cnt(K, 0);
    for (int64_t i = 0; i < N; ++i) {
      cnt[lab[i]]++;
      for (int c = 0; c < d; ++c) sum[(size_t)lab[i] * d + c] += X[i * d + c];
    }
    for (int k = 0; k < K; ++k)
      if (cnt[k] > 0)
        for (int c = 0; c < d; ++c) mu[k * d + c] = (float)(sum[(size_t)k * d + c] / cnt[k]);
  }
}

// Cyclic Jacobi on the symmetric K x K matrix A (row-major, overwritten); V = eigenvectors
// (columns), eigenvalues on A's diagonal.
void jacobi(std::vector<double>& A, std::vector<double>& V, int K) {
  V.assign((size_t)K * K, 0.0);
  for (int i = 0; i < K; ++i) V[(size_t)i * K + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < K; ++i)
      for (int j = i + 1; j < K; ++j) off += A[(size_t)i * K + j] * A[(size_t)i * K + j];
    if (off < 1e-30) break;
    for (int p = 0; p < K; ++p)
      for (int q = p + 1; q < K; ++q) {
        const double apq = A[(size_t)p * K + q];
        if (fabs(apq) < 1e-300) continue;
        const double app = A[(size_t)p * K + p], aqq = A[(size_t)q * K + q];
        const double th = (aqq - app) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < K; ++k) {      // columns p, q
          const double akp = A[(size_t)k * K + p], akq = A[(size_t)k * K + q];
          A[(size_t)k * K + p] = c * akp - s * akq;
          A[(size_t)k * K + q] = s * akp + c * akq;
        }
        for (int k = 0; k < K; ++k) {      // rows p, q
          const double apk = A[(size_t)p * K + k], aqk = A[(size_t)q * K + k];
          A[(size_t)p * K + k] = c * apk - s * aqk;
          A[(size_t)q * K + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < K; ++k) {
          const double vkp = V[(size_t)k * K + p], vkq = V[(size_t)k * K + q];
          V[(size_t)k * K + p] = c * vkp - s * vkq;
          V[(size_t)k * K + q] = s * vkp + c * vkq;
        }
      }
  }
}

}  // namespace

// Zero-padded separable FIR of one H x W plane: vertical into tmp, horizontal into dst.
static void fir2(const float* src, float* tmp, float* dst, int H, int W, const float* g, int S) {
  for (int y = 0; y < H; ++y) {
    float* t = tmp + (size_t)y * W;
    for (int x = 0; x < W; ++x) t[x] = 0.f;
    const int z0 = std::max(-S, y - (H - 1)), z1 = std::min(S, y);
    for (int z = z0; z <= z1; ++z) {                 // tmp[y] += g(z) src[y - z]
      const float w = g[z + S];
      const float* s = src + (size_t)(y - z) * W;
      for (int x = 0; x < W; ++x) t[x] += w * s[x];
    }
  }
  for (int y = 0; y < H; ++y) {
    const float* t = tmp + (size_t)y * W;
    float* d = dst + (size_t)y * W;
    for (int x = 0; x < W; ++x) {
      float s = 0.f;
      const int z0 = std::max(-S, x - (W - 1)), z1 = std::min(S, x);
      for (int z = z0; z <= z1; ++z) s += g[z + S] * t[x - z];
      d[x] = s;
    }
  }
}

extern "C" int nyf_cpu_blf(const float* f, int H, int W, int n, float sigma_s, float sigma_r, int K,
                           int iters, uint64_t seed, double tau, const float* landmarks, float* out,
                           int threads) {
  if (!f || !out || H < 1 || W < 1 || n < 1 || K < 1 || K > 64 || !(sigma_r > 0.f) ||
      !(sigma_s > 0.f))
    return 1;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#endif
  const int64_t N = (int64_t)H * W;
  std::vector<float> mu((size_t)K * n);
  if (landmarks) memcpy(mu.data(), landmarks, sizeof(float) * K * n);
  else kmeans(f, N, n, K, iters, seed, mu.data());
  // Eqs. (9)-(10): A, eigenpairs, kept modes, symmetric factor
  const double i2 = 1.0 / (2.0 * (double)sigma_r * sigma_r);
  std::vector<double> A((size_t)K * K), V;
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < K; ++j) {
      double s = 0.0;
      for (int c = 0; c < n; ++c) {
        const double t = (double)mu[i * n + c] - mu[j * n + c];
        s += t * t;
      }
      A[(size_t)i * K + j] = exp(-s * i2);
    }
  jacobi(A, V, K);
  double amax = 0.0;
  for (int k = 0; k < K; ++k) amax = std::max(amax, A[(size_t)k * K + k]);
  std::vector<double> Whd((size_t)K * K, 0.0);
  int r = 0;
  for (int k = 0; k < K; ++k) {
    const double a = A[(size_t)k * K + k];
    if (!(a > tau * amax)) continue;
    ++r;
    for (int i = 0; i < K; ++i)
      for (int j = 0; j < K; ++j)
        Whd[(size_t)i * K + j] += V[(size_t)i * K + k] * V[(size_t)j * K + k] / sqrt(a);
  }
  if (r == 0) return 4;
  std::vector<float> Wh(Whd.begin(), Whd.end());
  // Eqs. (11)-(12): phi planar, K planes of N
  const float i2f = (float)i2;
  std::vector<float> phi((size_t)K * N);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    float e[64];
    for (int m = 0; m < K; ++m) {
      float s = 0.f;
      for (int c = 0; c < n; ++c) {
        const float t = f[i * n + c] - mu[m * n + c];
        s += t * t;
      }
      e[m] = expf(-s * i2f);
    }
    for (int j = 0; j < K; ++j) {
      float s = 0.f;
      for (int m = 0; m < K; ++m) s += e[m] * Wh[(size_t)m * K + j];
      phi[(size_t)j * N + i] = s;
    }
  }
  // Eq. (7) and Eqs. (14)-(15): K (n + 1) separable convolutions and the combine
  const int S = (int)ceil(3.0 * sigma_s);
  std::vector<float> g(2 * S + 1);
  for (int z = -S; z <= S; ++z) g[z + S] = (float)exp(-(double)z * z / (2.0 * sigma_s * sigma_s));
  std::vector<float> zeta((size_t)N * n, 0.f), eta(N, 0.f);
  const int nq = n + 1;
#pragma omp parallel
  {
    std::vector<float> src(N), tmp(N), cv(N);
    std::vector<float> zl((size_t)N * n, 0.f), el(N, 0.f);
#pragma omp for schedule(dynamic)
    for (int t = 0; t < K * nq; ++t) {
      const int k = t / nq, q = t % nq;
      const float* ph = phi.data() + (size_t)k * N;
      for (int64_t i = 0; i < N; ++i) src[i] = q < n ? ph[i] * f[i * n + q] : ph[i];
      fir2(src.data(), tmp.data(), cv.data(), H, W, g.data(), S);
      if (q < n)
        for (int64_t i = 0; i < N; ++i) zl[i * n + q] += ph[i] * cv[i];
      else
        for (int64_t i = 0; i < N; ++i) el[i] += ph[i] * cv[i];
    }
#pragma omp critical
    {
      for (size_t i = 0; i < zl.size(); ++i) zeta[i] += zl[i];
      for (int64_t i = 0; i < N; ++i) eta[i] += el[i];
    }
  }
  for (int64_t i = 0; i < N; ++i)
    for (int c = 0; c < n; ++c) out[i * n + c] = zeta[i * n + c] / eta[i];
  return 0;
}

// Number of threads OpenMP gives a parallel region (1 without OpenMP).
extern "C" int nyf_cpu_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Landmark kernel A (Eq. (9)) and its eigendecomposition (Eq. (10)) in FP64.
//
// One CTA per landmark set.  A(i, j) = exp(-||mu_i - mu_j||^2 / (2 sigma_r^2))
// is built in FP64 from the float32 landmarks and diagonalised by the parallel
// cyclic Jacobi method (round-robin ordering: K/2 disjoint rotations per step,
// K-1 steps per sweep), which is accurate to a few units of FP64 rounding
// relative to ||A||.  The eigenvalues are sorted descending, modes with
// alpha_k > tau * alpha_max are kept, and the factor
//     W_hat[m][k] = w_mk / sqrt(alpha_k)      (k < r; zero for k >= r)
// is written in float32, so that phi_k(x) = sum_m kappa(p_x, mu_m) W_hat[m][k]
// equals sqrt(alpha_k) v_k(x) of Eq. (12).  Each eigenvector's sign is fixed so
// that its entry of largest magnitude (first such entry on ties) is positive.
#include <math.h>

#include "nyf_internal.cuh"

namespace nyf {
namespace {

constexpr int kEigThreads = 256;
constexpr int kMaxSweeps = 40;

struct EigSmem {
  double A[kMaxK][kMaxK + 1];
  double V[kMaxK][kMaxK + 1];
  double c[kMaxK / 2], s[kMaxK / 2];
  int p[kMaxK / 2], q[kMaxK / 2];
  int ring[kMaxK];
  int order[kMaxK];
  double red[kEigThreads];
};

__device__ double block_sum(double v, double* red) {
  const int tid = threadIdx.x;
  red[tid] = v;
  __syncthreads();
  for (int o = kEigThreads / 2; o > 0; o >>= 1) {
    if (tid < o) red[tid] += red[tid + o];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kEigThreads)
k_eig(const float* __restrict__ lm, int K, int rho, float sigma_r, double tau,
      float* __restrict__ what, double* __restrict__ alphas_out, int* __restrict__ rank_out,
      DevState* state) {
  extern __shared__ __align__(16) unsigned char raw[];
  EigSmem& sm = *reinterpret_cast<EigSmem*>(raw);
  const int tid = threadIdx.x;
  const int Kp = (K + 1) & ~1;            // even number of players; index K is a dummy if K is odd
  const int half = Kp / 2;
  const double inv2s2 = 1.0 / (2.0 * (double)sigma_r * (double)sigma_r);

  // A(i, j) = kappa(mu_i, mu_j), Eq. (9); V = I.
  double nonfinite = 0.0;
  for (int e = tid; e < K * K; e += kEigThreads) {
    const int i = e / K, j = e - i * K;
    double d2 = 0.0;
    for (int d = 0; d < rho; ++d) {
      const double t = (double)lm[i * rho + d] - (double)lm[j * rho + d];
      d2 = fma(t, t, d2);
    }
    const double a = exp(-d2 * inv2s2);
    if (!isfinite(a)) nonfinite += 1.0;
    sm.A[i][j] = a;
    sm.V[i][j] = (i == j) ? 1.0 : 0.0;
  }
  if (tid < Kp) sm.ring[tid] = tid;
  __syncthreads();
  const double bad = block_sum(nonfinite, sm.red);
  const double diag2 = block_sum(tid < K ? sm.A[tid][tid] * sm.A[tid][tid] : 0.0, sm.red);

  if (bad == 0.0) {
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
      double off = 0.0;
      for (int e = tid; e < K * K; e += kEigThreads) {
        const int i = e / K, j = e - i * K;
        if (i < j) off += sm.A[i][j] * sm.A[i][j];
      }
      off = block_sum(off, sm.red);
      if (off <= 1e-30 * diag2 || off == 0.0) break;
      for (int step = 0; step < Kp - 1; ++step) {
        // Rotation of each pair, classical Jacobi (Golub & Van Loan, sym.schur2).
        if (tid < half) {
          int a = sm.ring[tid], b = sm.ring[Kp - 1 - tid];
          if (a > b) { const int t = a; a = b; b = t; }
          double c = 1.0, s = 0.0;
          if (b < K) {
            const double apq = sm.A[a][b];
            if (apq != 0.0) {
              const double theta = (sm.A[b][b] - sm.A[a][a]) / (2.0 * apq);
              const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
              c = 1.0 / sqrt(1.0 + t * t);
              s = t * c;
            }
          }
          sm.p[tid] = a;
          sm.q[tid] = b;
          sm.c[tid] = c;
          sm.s[tid] = s;
        }
        __syncthreads();
        // Rows p, q <- J^T A.
        for (int e = tid; e < half * K; e += kEigThreads) {
          const int pr = e / K, j = e - pr * K;
          const int a = sm.p[pr], b = sm.q[pr];
          if (b < K) {
            const double c = sm.c[pr], s = sm.s[pr];
            const double x = sm.A[a][j], y = sm.A[b][j];
            sm.A[a][j] = c * x - s * y;
            sm.A[b][j] = s * x + c * y;
          }
        }
        __syncthreads();
        // Columns p, q <- A J, and V <- V J.
        for (int e = tid; e < half * K; e += kEigThreads) {
          const int pr = e / K, i = e - pr * K;
          const int a = sm.p[pr], b = sm.q[pr];
          if (b < K) {
            const double c = sm.c[pr], s = sm.s[pr];
            const double x = sm.A[i][a], y = sm.A[i][b];
            sm.A[i][a] = c * x - s * y;
            sm.A[i][b] = s * x + c * y;
            const double u = sm.V[i][a], v = sm.V[i][b];
            sm.V[i][a] = c * u - s * v;
            sm.V[i][b] = s * u + c * v;
          }
        }
        __syncthreads();
        if (tid < half && sm.q[tid] < K && sm.s[tid] != 0.0) {
          sm.A[sm.p[tid]][sm.q[tid]] = 0.0;
          sm.A[sm.q[tid]][sm.p[tid]] = 0.0;
        }
        // Next round-robin pairing: player 0 stays, the others rotate by one.
        if (tid == 0) {
          const int last = sm.ring[Kp - 1];
          for (int t = Kp - 1; t > 1; --t) sm.ring[t] = sm.ring[t - 1];
          sm.ring[1] = last;
        }
        __syncthreads();
      }
    }
  }

  // Sort descending (stable selection), truncate, write factors.
  if (tid == 0) {
    for (int k = 0; k < K; ++k) sm.order[k] = k;
    for (int k = 0; k < K; ++k) {
      int best = k;
      for (int j = k + 1; j < K; ++j)
        if (sm.A[sm.order[j]][sm.order[j]] > sm.A[sm.order[best]][sm.order[best]]) best = j;
      const int t = sm.order[k];
      sm.order[k] = sm.order[best];
      sm.order[best] = t;
    }
    const double amax = sm.A[sm.order[0]][sm.order[0]];
    int r = 0;
    if (bad == 0.0 && amax > 0.0 && isfinite(amax))
      while (r < K && sm.A[sm.order[r]][sm.order[r]] > tau * amax) ++r;
    for (int k = 0; k < K; ++k) {
      const double a = sm.A[sm.order[k]][sm.order[k]];
      state->alpha[k] = a;
      if (alphas_out) alphas_out[k] = a;
    }
    state->rank = r;
    if (rank_out) *rank_out = r;
    if (r == 0) set_status(state, NYF_ERR_NUMERIC);
    sm.red[0] = (double)r;
  }
  __syncthreads();
  const int r = (int)sm.red[0];
  for (int e = tid; e < K * K; e += kEigThreads) {
    const int m = e / K, k = e - m * K;
    float w = 0.f;
    if (k < r) {
      const int col = sm.order[k];
      // sign convention: the entry of largest magnitude is positive
      int arg = 0;
      double best = -1.0;
      for (int i = 0; i < K; ++i) {
        const double v = fabs(sm.V[i][col]);
        if (v > best) { best = v; arg = i; }
      }
      const double sgn = sm.V[arg][col] < 0.0 ? -1.0 : 1.0;
      w = (float)(sgn * sm.V[m][col] / sqrt(sm.A[col][col]));
    }
    what[m * K + k] = w;
  }
}

}  // namespace

cudaError_t launch_eig(const float* landmarks, int K, int rho, float sigma_r, double tau,
                       float* what, double* alphas_out, int* rank_out, DevState* state,
                       cudaStream_t st) {
  const size_t smem = sizeof(EigSmem);
  cudaError_t e = cudaFuncSetAttribute(k_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_eig<<<1, kEigThreads, smem, st>>>(landmarks, K, rho, sigma_r, tau, what, alphas_out, rank_out,
                                      state);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace nyf

// Landmark kernel A (Eq. (9)) and its eigendecomposition (Eq. (10)), FP64 accurate.
//
// GB300 executes FP64 at about 1/64 of its FP32 rate, so an FP64 Jacobi
// sweep on one SM costs as much as the whole filter.  The decomposition is
// therefore computed in parts:
//   1. k_a64      (K CTAs)  A(i, j) = exp(-||mu_i - mu_j||^2 / (2 sigma_r^2)) in FP64;
//   2. k_jacobi32 (1 CTA)   parallel cyclic Jacobi on float(A) in FP32
//                           (round-robin ordering, K/2 rotations per step);
//   3. three iterations of the refinement of Ogita & Aishima ("Iterative
//      refinement for symmetric eigenvalue decomposition", Japan J. Indust.
//      Appl. Math. 35, 2018), all in FP64, each product spread over K CTAs
//      (one column per CTA):
//         R = I - X^T X,  S = X^T A X,  lam_i = S_ii / (1 - R_ii),
//         E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i)  if |lam_i - lam_j| > delta,
//                R_ij / 2 otherwise,   X <- X + X E,
//         delta = 2 (||S - diag(lam)|| + ||A|| ||R||)   (Frobenius norms);
//      each iteration squares the error of the FP32 start;
//      then S = X^T A X once more and a thresholded FP64 Jacobi "polish" on S
//      (one warp) that resolves clusters of nearly equal eigenvalues, which
//      the first-order refinement only orthonormalises;
//   4. k_finalize (1 CTA)   sort descending, keep alpha_k > tau * alpha_max;
//      k_wsym (K CTAs)      the symmetric factor W_hat = W_r Lambda_r^{-1/2} W_r^T
//                           in float32 (see k_finalize).
// phi_j(x) = sum_m kappa(p_x, mu_m) W_hat[m][j], j < K, then satisfies
// sum_j phi_j(x) phi_j(y) = sum_{k<r} alpha_k v_k(x) v_k(y) with v_k of Eq. (12).
#include <math.h>

#include "nyf_internal.cuh"

namespace nyf {
namespace {

constexpr int kJacThreads = 512;
constexpr int kMaxSweeps32 = 16;
constexpr int kRefineIters = 3;

// FP64 scratch of the decomposition (inside the workspace).
struct EigBuf {
  double A[kMaxK * kMaxK];
  double X[2][kMaxK * kMaxK];   // X[m*K + i] = component m of eigenvector i
  double Y[kMaxK * kMaxK];
  double S[kMaxK * kMaxK];
  double R[kMaxK * kMaxK];
  double lam[kMaxK];
  double cnA[kMaxK], cnS[kMaxK], cnR[kMaxK];   // per-column squared norms
  int order[kMaxK];                            // eigenvalue order, descending
  int rank;
  int bad;
};

// Arguments of one decomposition.  The kernels take them through a policy P:
// EigOne (one problem per launch) or EigMany (a batch, problem = blockIdx.y), so
// every problem of a batch runs exactly the code and order of a single launch.
struct EigJob {
  const float* lm;
  double inv2s2;
  EigBuf* b;
  double* alphas;   // nullable
  int* rank;        // nullable
  DevState* state;
  float* what;
};
struct EigOne {
  EigJob j;
  __device__ __forceinline__ const EigJob& get() const { return j; }
};
struct EigMany {
  EigJob j[kBatchMax];
  __device__ __forceinline__ const EigJob& get() const { return j[blockIdx.y]; }
};

template <class P>
__global__ void k_eig_reset(const __grid_constant__ P p) {
  if (threadIdx.x == 0) p.get().b->bad = 0;
}

// ---- 1. A in FP64, one column per CTA
template <class P>
__global__ void k_a64(const __grid_constant__ P p, int K, int rho) {
  const float* __restrict__ lm = p.get().lm;
  const double inv2s2 = p.get().inv2s2;
  EigBuf* b = p.get().b;
  const int j = blockIdx.x, i = threadIdx.x;
  __shared__ double red[kMaxK];
  double a = 0.0;
  if (i < K) {
    double d2 = 0.0;
    for (int d = 0; d < rho; ++d) {
      const double t = (double)lm[i * rho + d] - (double)lm[j * rho + d];
      d2 = fma(t, t, d2);
    }
    a = exp(-d2 * inv2s2);
    b->A[i * K + j] = a;
  }
  red[i] = (i < K) ? a * a : 0.0;
  __syncthreads();
  if (i == 0) {
    double s = 0.0;
    bool bad = false;
    for (int q = 0; q < K; ++q) {
      s += red[q];
      bad |= !isfinite(red[q]);
    }
    b->cnA[j] = s;
    if (bad) b->bad = 1;
  }
}

// ---- 2. FP32 parallel cyclic Jacobi on float(A)
//
// Round-robin ("circle") ordering: at step s player 0 stays and position i > 0
// holds player 1 + (i - 1 + s) mod (Kp - 1); position i meets position Kp-1-i.
// The K/2 rotations of a step act on disjoint index pairs, so A' = J^T A J
// splits into independent 2 x 2 blocks: block (pair a, pair b) becomes
// R_a^T [A]_ab R_b and depends on nothing else.  One pass over A (and one over
// V) per step, two barriers per step.
struct Jac32 {
  float A[kMaxK][kMaxK + 1];
  float V[kMaxK][kMaxK + 1];
  float c[kMaxK / 2], s[kMaxK / 2];
  int p[kMaxK / 2], q[kMaxK / 2];
  float red[kJacThreads];
};

__device__ float block_sum_f(float v, float* red) {
  const int tid = threadIdx.x;
  red[tid] = v;
  __syncthreads();
  for (int o = kJacThreads / 2; o > 0; o >>= 1) {
    if (tid < o) red[tid] += red[tid + o];
    __syncthreads();
  }
  const float r = red[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ int rr_player(int pos, int step, int Kp) {
  return pos == 0 ? 0 : 1 + (pos - 1 + step) % (Kp - 1);
}

template <class P>
__global__ void __launch_bounds__(kJacThreads, 1) k_jacobi32(const __grid_constant__ P p, int K) {
  EigBuf* b = p.get().b;
  extern __shared__ __align__(16) unsigned char raw[];
  Jac32& sm = *reinterpret_cast<Jac32*>(raw);
  const int tid = threadIdx.x;
  const int Kp = (K + 1) & ~1;
  const int half = Kp / 2;
  for (int e = tid; e < K * K; e += kJacThreads) {
    const int i = e / K, j = e - i * K;
    sm.A[i][j] = (float)b->A[i * K + j];
    sm.V[i][j] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  const float diag2 = block_sum_f(tid < K ? sm.A[tid][tid] * sm.A[tid][tid] : 0.f, sm.red);
  float prev = INFINITY;
  // this thread's 2 x 2 blocks (pair u, pair v) of A and (row i, pair v) entries of V:
  // fixed for the whole kernel, so the steps carry no integer divisions
  constexpr int kMaxBlocks = (kMaxK / 2) * (kMaxK / 2) / kJacThreads;
  constexpr int kMaxCols = kMaxK * (kMaxK / 2) / kJacThreads;
  int bu[kMaxBlocks], bv[kMaxBlocks], ci[kMaxCols], cv[kMaxCols];
#pragma unroll
  for (int m = 0; m < kMaxBlocks; ++m) {
    const int e = tid + m * kJacThreads;
    bu[m] = e < half * half ? e / half : -1;
    bv[m] = e - (e / half) * half;
  }
#pragma unroll
  for (int m = 0; m < kMaxCols; ++m) {
    const int e = tid + m * kJacThreads;
    ci[m] = e < K * half ? e / half : -1;
    cv[m] = e - (e / half) * half;
  }
  if (b->bad == 0) {
    for (int sweep = 0; sweep < kMaxSweeps32; ++sweep) {
      float off = 0.f;
      for (int e = tid; e < K * K; e += kJacThreads) {
        const int i = e / K, j = e - i * K;
        if (i < j) off += sm.A[i][j] * sm.A[i][j];
      }
      off = block_sum_f(off, sm.red);
      // stop at convergence, or once FP32 rounding noise stops the decrease
      // (only near the noise floor: early sweeps can decrease slowly)
      if (off <= 1e-14f * diag2 || off == 0.f) break;
      if (off <= 1e-9f * diag2 && off > 0.25f * prev) break;
      prev = off;
      for (int step = 0; step < Kp - 1; ++step) {
        if (tid < half) {        // rotation of pair tid (Golub & Van Loan, sym.schur2)
          int a = rr_player(tid, step, Kp), bb = rr_player(Kp - 1 - tid, step, Kp);
          if (a > bb) { const int t = a; a = bb; bb = t; }
          float c = 1.f, s = 0.f;
          if (bb < K) {
            const float apq = sm.A[a][bb], app = sm.A[a][a], aqq = sm.A[bb][bb];
            // entries below FP32 resolution of the diagonal (subnormal ones included) are
            // not rotated, so that theta stays finite
            if (fabsf(apq) > 1e-30f * (fabsf(app) + fabsf(aqq)) && fabsf(apq) > 1e-36f) {
              // fast divisions: |2 a_pq| is a normal number here, and an infinite theta
              // gives t = 0 (no rotation); the FP64 refinement makes the start exact
              const float theta = __fdividef(aqq - app, 2.f * apq);
              const float t = (theta >= 0.f ? 1.f : -1.f) *
                              __fdividef(1.f, fabsf(theta) + sqrtf(1.f + theta * theta));
              c = rsqrtf(1.f + t * t);
              s = t * c;
            }
          } else {
            bb = a;              // dummy partner: identity on a single index
          }
          sm.p[tid] = a;
          sm.q[tid] = bb;
          sm.c[tid] = c;
          sm.s[tid] = s;
        }
        __syncthreads();
        // 2 x 2 blocks of A (rows of pair u, columns of pair v) and the columns of V
        // of pair v.  Distinct blocks touch distinct entries, so every thread first
        // loads all of its blocks, then writes them: one shared-memory latency per
        // step instead of one per block.
#pragma unroll
        for (int m = 0; m < kMaxBlocks; ++m) {
          if (bu[m] >= 0) {
            const int u = bu[m], v = bv[m];
            const int pu = sm.p[u], qu = sm.q[u], pv = sm.p[v], qv = sm.q[v];
            const float cu = sm.c[u], su = sm.s[u], cv = sm.c[v], sv = sm.s[v];
            const float a00 = sm.A[pu][pv], a01 = sm.A[pu][qv];
            const float a10 = sm.A[qu][pv], a11 = sm.A[qu][qv];
            const float r00 = cu * a00 - su * a10, r01 = cu * a01 - su * a11;
            const float r10 = su * a00 + cu * a10, r11 = su * a01 + cu * a11;
            const float n00 = cv * r00 - sv * r01, n01 = sv * r00 + cv * r01;
            const float n10 = cv * r10 - sv * r11, n11 = sv * r10 + cv * r11;
            if (pu == qu && pv == qv) {
              sm.A[pu][pv] = n00;
            } else if (pu == qu) {
              sm.A[pu][pv] = n00;
              sm.A[pu][qv] = n01;
            } else if (pv == qv) {
              sm.A[pu][pv] = n00;
              sm.A[qu][pv] = n10;
            } else {
              sm.A[pu][pv] = n00;
              sm.A[pu][qv] = n01;
              sm.A[qu][pv] = n10;
              sm.A[qu][qv] = n11;
              if (u == v) sm.A[pu][qv] = sm.A[qu][pv] = 0.f;
            }
          }
        }
#pragma unroll
        for (int m = 0; m < kMaxCols; ++m) {
          if (ci[m] >= 0) {
            const int i = ci[m], v = cv[m];
            const int pv = sm.p[v], qv = sm.q[v];
            if (pv != qv) {
              const float cvv = sm.c[v], sv = sm.s[v];
              const float x = sm.V[i][pv], y = sm.V[i][qv];
              sm.V[i][pv] = cvv * x - sv * y;
              sm.V[i][qv] = sv * x + cvv * y;
            }
          }
        }
        __syncthreads();
      }
    }
  }
  for (int e = tid; e < K * K; e += kJacThreads) {
    const int m = e / K, i = e - m * K;
    b->X[0][e] = (double)sm.V[m][i];
  }
}

// ---- 3a. Y = A X (column j per CTA)
template <class P>
__global__ void k_oa_y(const __grid_constant__ P p, int K, int src) {
  EigBuf* b = p.get().b;
  const int j = blockIdx.x, i = threadIdx.x;
  __shared__ double xj[kMaxK];
  if (i < K) xj[i] = b->X[src][i * K + j];
  __syncthreads();
  if (i < K) {
    double s = 0.0;
    for (int m = 0; m < K; ++m) s = fma(b->A[i * K + m], xj[m], s);
    b->Y[i * K + j] = s;
  }
}

// ---- 3b. S = X^T Y, R = I - X^T X (column j per CTA) and their column norms
template <class P>
__global__ void k_oa_sr(const __grid_constant__ P p, int K, int src) {
  EigBuf* b = p.get().b;
  const int j = blockIdx.x, i = threadIdx.x;
  __shared__ double xj[kMaxK], yj[kMaxK], rs[kMaxK], rr[kMaxK];
  const double* X = b->X[src];
  if (i < K) {
    xj[i] = X[i * K + j];
    yj[i] = b->Y[i * K + j];
  }
  __syncthreads();
  double s = 0.0, r = 0.0;
  if (i < K) {
    double xx = 0.0;
    for (int m = 0; m < K; ++m) {
      const double xmi = X[m * K + i];
      s = fma(xmi, yj[m], s);
      xx = fma(xmi, xj[m], xx);
    }
    r = (i == j ? 1.0 : 0.0) - xx;
    b->S[i * K + j] = s;
    b->R[i * K + j] = r;
  }
  rs[i] = (i < K && i != j) ? s * s : 0.0;
  rr[i] = (i < K) ? r * r : 0.0;
  __syncthreads();
  if (i == 0) {
    double a = 0.0, c = 0.0;
    for (int q = 0; q < K; ++q) {
      a += rs[q];
      c += rr[q];
    }
    b->cnS[j] = a;
    b->cnR[j] = c;
  }
}

// ---- 3c. lam, E[:, j] and X_new[:, j] = X[:, j] + X E[:, j]
template <class P>
__global__ void k_oa_update(const __grid_constant__ P p, int K, int src, int orth_only) {
  EigBuf* b = p.get().b;
  const int j = blockIdx.x, i = threadIdx.x;
  __shared__ double lam[kMaxK], ej[kMaxK], cS[kMaxK], cR[kMaxK], cA[kMaxK];
  __shared__ double delta;
  if (i < K) {
    lam[i] = b->S[i * K + i] / (1.0 - b->R[i * K + i]);
    cS[i] = b->cnS[i];
    cR[i] = b->cnR[i];
    cA[i] = b->cnA[i];
  }
  __syncthreads();
  if (i == 0) {
    double nS = 0.0, nR = 0.0, nA = 0.0;
    for (int q = 0; q < K; ++q) {
      nS += cS[q];
      nR += cR[q];
      nA += cA[q];
    }
    delta = 2.0 * (sqrt(nS) + sqrt(nA) * sqrt(nR));
  }
  __syncthreads();
  if (i < K) {
    const double r = b->R[i * K + j];
    double e;
    if (i == j || orth_only) {
      e = 0.5 * r;
    } else {
      const double gap = lam[j] - lam[i];
      const double num = b->S[i * K + j] + lam[j] * r;
      // first-order update only where it is small; near-degenerate pairs are
      // orthonormalised here and resolved by the final polish
      e = (fabs(gap) > delta && fabs(num) <= 1e-4 * fabs(gap)) ? num / gap : 0.5 * r;
    }
    ej[i] = e;
    if (j == 0 && !orth_only) b->lam[i] = lam[i];
  }
  __syncthreads();
  if (i < K) {
    const double* X = b->X[src];
    double s = X[i * K + j];
    for (int m = 0; m < K; ++m) s = fma(X[i * K + m], ej[m], s);
    b->X[src ^ 1][i * K + j] = s;
  }
}

// ---- 3d. Polish: thresholded FP64 Jacobi on S = X^T A X.  After the refinement
// S is diagonal to FP64 rounding except inside clusters of nearly equal
// eigenvalues, so only a few pairs rotate; each rotation is applied to S and
// to the columns of X.  One warp; pairs are scanned in cyclic row order and a
// pair rotates when |S_pq| > 4 eps sqrt(|S_pp S_qq|) (the negligibility test of
// Demmel & Veselic).  Writes the eigenvalues to lam.
template <class P>
__global__ void k_polish(const __grid_constant__ P p, int K, int src) {
  EigBuf* b = p.get().b;
  extern __shared__ double ps[];
  double* Sm = ps;                     // K x (K + 1)
  double* Xm = ps + K * (K + 1);       // K x (K + 1)
  const int lane = threadIdx.x;
  const int ld = K + 1;
  for (int e = lane; e < K * K; e += 32) {
    const int i = e / K, j = e - i * K;
    Sm[i * ld + j] = 0.5 * (b->S[i * K + j] + b->S[j * K + i]);
    Xm[i * ld + j] = b->X[src][i * K + j];
  }
  __syncwarp();
  const double eps4 = 4.0 * 2.220446049250313e-16;
  const int npairs = K * (K - 1) / 2;
  for (int sweep = 0; sweep < 12; ++sweep) {
    int rotated = 0;
    for (int base = 0; base < npairs; base += 32) {
      const int t = base + lane;
      int p = 0, q = 0;
      bool flag = false;
      if (t < npairs) {                      // t -> (p, q), p < q, row-major order
        int rem = t;
        p = 0;
        while (rem >= K - 1 - p) { rem -= K - 1 - p; ++p; }
        q = p + 1 + rem;
        const double spq = Sm[p * ld + q];
        flag = fabs(spq) > eps4 * sqrt(fabs(Sm[p * ld + p] * Sm[q * ld + q])) && spq != 0.0;
      }
      unsigned m = __ballot_sync(0xffffffffu, flag);
      while (m) {
        const int src_lane = __ffs(m) - 1;
        m &= m - 1;
        const int pp = __shfl_sync(0xffffffffu, p, src_lane);
        const int qq = __shfl_sync(0xffffffffu, q, src_lane);
        const double apq = Sm[pp * ld + qq];
        if (apq == 0.0) continue;            // uniform: every lane reads the same value
        const double theta = (Sm[qq * ld + qq] - Sm[pp * ld + pp]) / (2.0 * apq);
        const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
        const double c = 1.0 / sqrt(1.0 + tt * tt), s = tt * c;
        __syncwarp();
        for (int j = lane; j < K; j += 32) {     // rows p, q
          const double x = Sm[pp * ld + j], y = Sm[qq * ld + j];
          Sm[pp * ld + j] = c * x - s * y;
          Sm[qq * ld + j] = s * x + c * y;
        }
        __syncwarp();
        for (int i = lane; i < K; i += 32) {     // columns p, q of S and X
          const double x = Sm[i * ld + pp], y = Sm[i * ld + qq];
          Sm[i * ld + pp] = c * x - s * y;
          Sm[i * ld + qq] = s * x + c * y;
          const double u = Xm[i * ld + pp], v = Xm[i * ld + qq];
          Xm[i * ld + pp] = c * u - s * v;
          Xm[i * ld + qq] = s * u + c * v;
        }
        __syncwarp();
        if (lane == 0) Sm[pp * ld + qq] = Sm[qq * ld + pp] = 0.0;
        __syncwarp();
        rotated = 1;
      }
    }
    if (!rotated) break;
  }
  __syncwarp();
  for (int e = lane; e < K * K; e += 32) {
    const int i = e / K, j = e - i * K;
    b->X[src][i * K + j] = Xm[i * ld + j];
  }
  for (int i = lane; i < K; i += 32) b->lam[i] = Sm[i * ld + i];
}

// ---- 4. sort and truncate (1 CTA), then the symmetric factor (K CTAs).
//
// Any W_hat with W_hat W_hat^T = A_r^+ gives the same K-hat = E A_r^+ E^T and
// hence the same filter.  The library uses the symmetric one,
//     W_hat = W_r Lambda_r^{-1/2} W_r^T = A_r^{-1/2},
// which is unique (no eigenvector sign or rotation freedom) and the closest
// factor to the identity: with well-separated landmarks A is near I and each
// feature stays close to one landmark's kernel column, so the sum over modes
// in Eqs. (14)-(15) does not cancel large terms (it does with the eigenvector
// factor, whose rounding then dominates the result in low precision).
template <class P>
__global__ void k_finalize(const __grid_constant__ P p, int K, double tau) {
  EigBuf* b = p.get().b;
  double* __restrict__ alphas_out = p.get().alphas;
  int* __restrict__ rank_out = p.get().rank;
  DevState* state = p.get().state;
  __shared__ double lam[kMaxK];
  const int tid = threadIdx.x;
  if (tid < K) lam[tid] = b->lam[tid];
  __syncthreads();
  if (tid < K) {   // stable descending rank of each eigenvalue; NaN ranks last, so the
                   // ranks are a permutation whatever the values (order[] indexes memory)
    const double v = isnan(lam[tid]) ? -INFINITY : lam[tid];
    int rk = 0;
    for (int q = 0; q < K; ++q) {
      const double w = isnan(lam[q]) ? -INFINITY : lam[q];
      rk += (w > v) || (w == v && q < tid);
    }
    b->order[rk] = tid;
    if (!isfinite(lam[tid])) b->bad = 1;
  }
  __syncthreads();
  if (tid == 0) {
    const double amax = lam[b->order[0]];
    int r = 0;
    if (b->bad == 0 && amax > 0.0 && isfinite(amax))
      while (r < K && lam[b->order[r]] > tau * amax) ++r;
    b->rank = r;
    state->rank = r;
    state->planes = r > 0 ? K : 0;
    if (rank_out) *rank_out = r;
    if (r == 0) set_status(state, NYF_ERR_NUMERIC);
  }
  if (tid < K) {
    const double a = lam[b->order[tid]];
    state->alpha[tid] = a;
    if (alphas_out) alphas_out[tid] = a;
  }
}

// W_hat[m][j] = sum_{k < r} w_m,k w_j,k / sqrt(alpha_k)  (FP64, one column per CTA)
template <class P>
__global__ void k_wsym(const __grid_constant__ P p, int K, int src) {
  const EigBuf* b = p.get().b;
  float* __restrict__ what = p.get().what;
  const int j = blockIdx.x, m = threadIdx.x;
  __shared__ double cj[kMaxK];
  const double* X = b->X[src];
  const int r = b->rank;
  if (m < r) {
    const int col = b->order[m];
    cj[m] = X[j * K + col] / sqrt(b->lam[col]);
  }
  __syncthreads();
  if (m < K) {
    double s = 0.0;
    for (int k = 0; k < r; ++k) s = fma(X[m * K + b->order[k]], cj[k], s);
    what[m * K + j] = (float)s;
  }
}

}  // namespace

size_t eig_scratch_bytes() { return sizeof(EigBuf); }

const double* eig_A64(const void* scratch) { return reinterpret_cast<const EigBuf*>(scratch)->A; }

namespace {

// The sequence of launches of the decomposition for `count` problems (grid.y).
template <class P>
cudaError_t eig_run(const P& p, int count, int K, int rho, double tau, cudaStream_t st) {
  const dim3 one(1, count), cols(K, count);
  k_eig_reset<P><<<one, 32, 0, st>>>(p);
  k_a64<P><<<cols, kMaxK, 0, st>>>(p, K, rho);
  count_launches(2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(Jac32);
  e = cudaFuncSetAttribute(k_jacobi32<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_jacobi32<P><<<one, kJacThreads, smem, st>>>(p, K);
  count_launches(1);
  int src = 0;
  for (int it = 0; it < kRefineIters; ++it) {
    k_oa_y<P><<<cols, kMaxK, 0, st>>>(p, K, src);
    k_oa_sr<P><<<cols, kMaxK, 0, st>>>(p, K, src);
    k_oa_update<P><<<cols, kMaxK, 0, st>>>(p, K, src, 0);
    count_launches(3);
    src ^= 1;
  }
  // orthonormalise once more (X <- X (I + R / 2), second-order accurate), then
  // S = X^T A X for the polish
  k_oa_y<P><<<cols, kMaxK, 0, st>>>(p, K, src);
  k_oa_sr<P><<<cols, kMaxK, 0, st>>>(p, K, src);
  k_oa_update<P><<<cols, kMaxK, 0, st>>>(p, K, src, 1);
  src ^= 1;
  k_oa_y<P><<<cols, kMaxK, 0, st>>>(p, K, src);
  k_oa_sr<P><<<cols, kMaxK, 0, st>>>(p, K, src);
  count_launches(5);
  const size_t psmem = sizeof(double) * 2 * K * (K + 1);
  e = cudaFuncSetAttribute(k_polish<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
  if (e != cudaSuccess) return e;
  k_polish<P><<<one, 32, psmem, st>>>(p, K, src);
  k_finalize<P><<<one, kMaxK, 0, st>>>(p, K, tau);
  k_wsym<P><<<cols, kMaxK, 0, st>>>(p, K, src);
  count_launches(3);
  return cudaGetLastError();
}

EigJob make_job(const float* landmarks, float sigma_r, float* what, double* alphas_out,
                int* rank_out, DevState* state, void* scratch) {
  EigJob j;
  j.lm = landmarks;
  j.inv2s2 = 1.0 / (2.0 * (double)sigma_r * (double)sigma_r);
  j.b = reinterpret_cast<EigBuf*>(scratch);
  j.alphas = alphas_out;
  j.rank = rank_out;
  j.state = state;
  j.what = what;
  return j;
}

}  // namespace

cudaError_t launch_eig(const float* landmarks, int K, int rho, float sigma_r, double tau,
                       float* what, double* alphas_out, int* rank_out, DevState* state,
                       void* scratch, cudaStream_t st) {
  EigOne p;
  p.j = make_job(landmarks, sigma_r, what, alphas_out, rank_out, state, scratch);
  return eig_run(p, 1, K, rho, tau, st);
}

cudaError_t launch_eig_batched(const EigItem* items, int count, int K, int rho, double tau,
                               cudaStream_t st) {
  for (int b0 = 0; b0 < count; b0 += kBatchMax) {
    const int m = count - b0 < kBatchMax ? count - b0 : kBatchMax;
    EigMany p;
    for (int i = 0; i < m; ++i) {
      const EigItem& it = items[b0 + i];
      p.j[i] = make_job(it.landmarks, it.sigma_r, it.what, nullptr, nullptr, it.state, it.scratch);
    }
    for (int i = m; i < kBatchMax; ++i) p.j[i] = p.j[0];
    cudaError_t e = eig_run(p, m, K, rho, tau, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace nyf

// k-means landmark selection (Sec. III; Algorithm 1, clustering step) and the
// NLM subsample gather.
//
// One Lloyd iteration = k_assign (nearest centroid of every row, ties to the
// lowest index, plus per-block partial sums of the members of each cluster)
// followed by k_update (one CTA per cluster sums the partials in FP64 and moves
// the centroid to the mean; an empty cluster keeps its centroid).  Every
// reduction runs in a fixed order, so the result is bitwise reproducible.
#include "nyf_internal.cuh"

namespace nyf {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ inline float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

constexpr int assign_threads(int RB) { return RB > 0 ? 256 : 128; }
constexpr int assign_ppt(int RB) { return RB == 0 ? 1 : (RB <= 8 ? 4 : (RB <= 16 ? 2 : 1)); }
constexpr int assign_rb(int rho) { return rho <= 4 ? 4 : (rho <= 8 ? 8 : (rho <= 16 ? 16 : (rho <= 32 ? 32 : 0))); }

// BLF subsample: stratum t of the row order gives row
// lo + SplitMix64(seed ^ kSampleStream, t + 1) mod (hi - lo); it is copied to X.
__global__ void k_sample_rows(const float* __restrict__ G, int64_t N, int rho, int64_t Ns,
                              uint64_t seed, int64_t* __restrict__ idx, float* __restrict__ X) {
  const int64_t total = Ns * rho;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / rho;
    const int j = (int)(e - t * rho);
    const int64_t lo = (int64_t)(((unsigned __int128)t * N) / Ns);
    const int64_t hi = (int64_t)(((unsigned __int128)(t + 1) * N) / Ns);
    const int64_t row = lo + (int64_t)(splitmix64(seed ^ kSampleStream, (uint64_t)t + 1) %
                                       (uint64_t)(hi - lo));
    if (j == 0) idx[t] = row;
    X[e] = G[row * rho + j];
  }
}

// Centroids are stored with row stride 4 (float4, zero padded) when rho <= 4.
__host__ __device__ constexpr int mu_stride(int rho) { return rho <= 4 ? 4 : rho; }

// Rows of rho <= 4 also keep the negated centroids as duplicated pairs
// (-mu_jd, -mu_jd), d < 4, for the packed distance loop.
__host__ __device__ constexpr size_t neg_pairs_offset(int K, int rho, int warps) {
  return ((size_t)K * mu_stride(rho) + (size_t)warps * K * (rho + 1) + 3) & ~(size_t)3;
}

size_t assign_smem(int K, int rho) {
  const int warps = assign_threads(rho <= 32 ? 1 : 0) / 32;
  const size_t pairs = rho <= 4 ? (size_t)K * 8 : 0;
  return sizeof(float) * (neg_pairs_offset(K, rho, warps) + pairs);
}

int kmeans_grid(int64_t N, int rho) {
  const int rb = assign_rb(rho);
  const int64_t t = (int64_t)assign_threads(rb) * assign_ppt(rb);
  const int64_t g = (N + t - 1) / t;
  return (int)(g < kKmeansBlocks ? (g < 1 ? 1 : g) : kKmeansBlocks);
}

__device__ inline int reflect101(int i, int n) {
  if (n == 1) return 0;
  const int period = 2 * (n - 1);
  int j = i % period;
  if (j < 0) j += period;
  return j < n ? j : period - j;
}

// Arguments of one clustering problem.  The kernels take them through a policy
// P: KmOne (one problem per launch) or KmMany (a batch; the assignment pass maps
// its flat block index to (problem, block) through the prefix sums `first`, the
// other kernels take the problem from blockIdx.y), so every problem of a batch
// runs exactly the code, grid partition and reduction order of a single launch.
struct KmJob {
  const float* X;
  int64_t N;
  float* cent;
  int32_t* labels;          // nullable
  float* part;
  float* qpart;
  double* qerr_out;         // nullable
  const int64_t* init_idx;  // nullable
  int64_t* idx_out;
  DevState* state;
  uint64_t seed;
  int grid;                 // blocks of this problem's assignment pass
};
struct KmOne {
  KmJob j;
  __device__ __forceinline__ const KmJob& get() const { return j; }
  __device__ __forceinline__ const KmJob& job_for_block(int& blk) const {
    blk = blockIdx.x;
    return j;
  }
};
struct KmMany {
  int count;
  int first[kBatchMax + 1];
  KmJob j[kBatchMax];
  __device__ __forceinline__ const KmJob& get() const { return j[blockIdx.y]; }
  __device__ __forceinline__ const KmJob& job_for_block(int& blk) const {
    const int x = blockIdx.x;
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (first[mid] <= x) lo = mid;
      else hi = mid - 1;
    }
    blk = x - first[lo];
    return j[lo];
  }
};

// Initial centroids: rows init_idx[j] of X, or the first K distinct values of
// SplitMix64(seed) mod N (bounded number of draws).
template <class P>
__global__ void k_draw_init(const __grid_constant__ P p, int rho, int K) {
  const KmJob& J = p.get();
  const float* __restrict__ X = J.X;
  const int64_t N = J.N;
  const uint64_t seed = J.seed;
  const int64_t* __restrict__ init_idx = J.init_idx;
  int64_t* __restrict__ idx_out = J.idx_out;
  float* __restrict__ cent = J.cent;
  DevState* state = J.state;
  __shared__ int64_t idx[kMaxK];
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    if (init_idx) {
      for (int j = 0; j < K; ++j) {
        int64_t v = init_idx[j];
        if (v < 0 || v >= N) { ok = 0; v = 0; }
        idx[j] = v;
      }
      if (!ok) set_status(state, NYF_ERR_INVALID_ARG);
    } else {
      int cnt = 0;
      const uint64_t max_draws = 64ull * (uint64_t)K + 4096ull;
      for (uint64_t t = 1; t <= max_draws && cnt < K; ++t) {
        const int64_t c = (int64_t)(splitmix64(seed, t) % (uint64_t)N);
        bool dup = false;
        for (int q = 0; q < cnt; ++q) dup |= (idx[q] == c);
        if (!dup) idx[cnt++] = c;
      }
      if (cnt < K) {
        ok = 0;
        for (int q = cnt; q < K; ++q) idx[q] = 0;
        set_status(state, NYF_ERR_TIMEOUT);
      }
    }
    for (int j = 0; j < K; ++j) idx_out[j] = idx[j];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < K * rho; e += blockDim.x) {
    const int j = e / rho, d = e - j * rho;
    cent[e] = X[idx[j] * rho + d];
  }
}

template <int R, int PPT, int RX>
__device__ __forceinline__ void unpack_rows(const float* buf, float (&x)[PPT][RX]) {
#pragma unroll
  for (int q = 0; q < PPT; ++q)
#pragma unroll
    for (int d = 0; d < RX; ++d) x[q][d] = d < R ? buf[q * R + d] : 0.f;
}

// Nearest centroid of the PPT rows in x (R <= 4 coordinates; mu: centroids with
// row stride 4; nmu2: (-mu_jd, -mu_jd) pairs, 8 floats per centroid).  Rows are
// evaluated two at a time in packed FP32x2: t = x + (-mu), dist = sum of t^2 in
// coordinate order.  The running minimum is kept as a key, the distance's bit
// pattern (non-negative, so ordered like the value) with its six low mantissa
// bits replaced by j: one integer minimum per row and centroid, ties (and
// distances equal to within 2^-17 relative) to the lowest index.  The chosen
// centroid's distance is then formed again, exactly as in the loop.
template <int R, int PPT>
__device__ __forceinline__ void nearest_small(const float (&x)[PPT][4], const float* mu,
                                              const float* nmu2, int K, int (&best)[PPT],
                                              float (&bd)[PPT]) {
  static_assert(PPT % 2 == 0 && R >= 1 && R <= 4, "row pairs, at most 4 coordinates");
  static_assert(kMaxK <= 64, "the centroid index fits the six low bits of a key");
  unsigned key[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) key[q] = 0xffffffffu;
#pragma unroll 4
  for (int j = 0; j < K; ++j) {
    const float4 n01 = *reinterpret_cast<const float4*>(nmu2 + 8 * j);
    const float4 n23 = *reinterpret_cast<const float4*>(nmu2 + 8 * j + 4);
    const float2 nc[4] = {make_float2(n01.x, n01.y), make_float2(n01.z, n01.w),
                          make_float2(n23.x, n23.y), make_float2(n23.z, n23.w)};
#pragma unroll
    for (int pr = 0; pr < PPT / 2; ++pr) {
      float2 t = __fadd2_rn(make_float2(x[2 * pr][0], x[2 * pr + 1][0]), nc[0]);
      float2 dist = __fmul2_rn(t, t);
#pragma unroll
      for (int d = 1; d < R; ++d) {
        t = __fadd2_rn(make_float2(x[2 * pr][d], x[2 * pr + 1][d]), nc[d]);
        dist = __ffma2_rn(t, t, dist);
      }
      key[2 * pr] = min(key[2 * pr], (__float_as_uint(dist.x) & ~63u) | (unsigned)j);
      key[2 * pr + 1] = min(key[2 * pr + 1], (__float_as_uint(dist.y) & ~63u) | (unsigned)j);
    }
  }
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    best[q] = (int)(key[q] & 63u);
    const float* c = mu + 4 * best[q];
    float t = x[q][0] + (-c[0]);
    float dist = t * t;
#pragma unroll
    for (int d = 1; d < R; ++d) {
      t = x[q][d] + (-c[d]);
      dist = fmaf(t, t, dist);
    }
    bd[q] = dist;
  }
}

// Assignment pass.  RB > 0: each thread holds PPT consecutive rows in
// registers (rho <= RB), so one centroid load from shared memory serves PPT
// distance evaluations, evaluated two rows at a time with packed FP32x2
// arithmetic (x - c as x + (-c), then the same fused multiply-adds as one row
// at a time, so the distances are bitwise those of the scalar form).  Rows of a
// thread that share a label are summed in the thread first (image rows are
// spatially coherent), then every label present in the warp is reduced across
// the lanes once.  RB == 0: rows are re-read from global memory (large rho,
// used for small row counts).
// part[b][j][0..rho) = sum of the members of cluster j seen by block b,
// part[b][j][rho] = their count; qpart[b] = sum of their squared distances.
// Every sum runs in an order fixed by the data layout, so results are bitwise
// reproducible.
template <class P, int RB, int THREADS, int PPT>
__global__ void __launch_bounds__(THREADS)
k_assign(const __grid_constant__ P p, int rho, int K, int accumulate) {
  int blk;
  const KmJob& J = p.job_for_block(blk);
  const int nblk = J.grid;
  const float* __restrict__ X = J.X;
  const int64_t N = J.N;
  const float* __restrict__ cent = J.cent;
  int32_t* __restrict__ labels = J.labels;
  float* __restrict__ part = J.part;
  float* __restrict__ qpart = J.qpart;
  extern __shared__ __align__(16) float sm[];
  constexpr int kWarps = THREADS / 32;
  constexpr int RX = RB > 0 ? RB : 1;
  const int ms = mu_stride(rho);
  float* mu = sm;                       // K * ms
  float* acc = sm + K * ms;             // kWarps * K * (rho + 1)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int stride = rho + 1;
  for (int e = tid; e < K * ms; e += blockDim.x) {
    const int j = e / ms, d = e - j * ms;
    mu[e] = d < rho ? cent[j * rho + d] : 0.f;
  }
  float* nmu2 = sm + neg_pairs_offset(K, rho, kWarps);   // rho <= 4 only
  if (RB == 4)
    for (int e = tid; e < K * 4; e += blockDim.x) {
      const int j = e / 4, d = e - j * 4;
      const float v = d < rho ? -cent[j * rho + d] : 0.f;
      nmu2[8 * j + 2 * d] = v;
      nmu2[8 * j + 2 * d + 1] = v;
    }
  if (accumulate)
    for (int e = tid; e < kWarps * K * stride; e += blockDim.x) acc[e] = 0.f;
  __syncthreads();

  float qsum = 0.f;
  if (RB > 0) {
    for (int64_t base = (int64_t)blk * THREADS * PPT; base < N;
         base += (int64_t)nblk * THREADS * PPT) {
      const int64_t i0 = base + (int64_t)tid * PPT;       // this thread's first row
      float x[PPT][RX];
      bool valid[PPT];
      int best[PPT];
      float bd[PPT];
      const float* xi = X + (i0 < N ? i0 : 0) * rho;
      const bool vec = RB == 4 && i0 + PPT <= N && (PPT * rho) % 4 == 0 &&
                       (reinterpret_cast<uintptr_t>(xi) & 15) == 0;
      if (vec) {                                          // PPT rows = rho float4 loads
        float buf[PPT * RX];
#pragma unroll
        for (int v = 0; v < RX; ++v) {
          if (v < rho) {
            const float4 w = __ldg(reinterpret_cast<const float4*>(xi) + v);
            buf[4 * v] = w.x;
            buf[4 * v + 1] = w.y;
            buf[4 * v + 2] = w.z;
            buf[4 * v + 3] = w.w;
          }
        }
        switch (rho) {                                    // row q, coordinate d = buf[q rho + d]
          case 1: unpack_rows<1, PPT, RX>(buf, x); break;
          case 2: unpack_rows<2, PPT, RX>(buf, x); break;
          case 3: unpack_rows<3, PPT, RX>(buf, x); break;
          default: unpack_rows<4, PPT, RX>(buf, x); break;
        }
      } else {
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
          const bool ok = i0 + q < N;
          const float* r = X + (ok ? i0 + q : 0) * rho;
#pragma unroll
          for (int d = 0; d < RX; ++d) x[q][d] = (ok && d < rho) ? __ldg(r + d) : 0.f;
        }
      }
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        valid[q] = i0 + q < N;
        best[q] = 0;
        bd[q] = __int_as_float(0x7f800000);
      }
      if constexpr (RB == 4 && PPT % 2 == 0) {
        const float (&x4)[PPT][4] = reinterpret_cast<const float (&)[PPT][4]>(x);
        switch (rho) {
          case 1: nearest_small<1, PPT>(x4, mu, nmu2, K, best, bd); break;
          case 2: nearest_small<2, PPT>(x4, mu, nmu2, K, best, bd); break;
          case 3: nearest_small<3, PPT>(x4, mu, nmu2, K, best, bd); break;
          default: nearest_small<4, PPT>(x4, mu, nmu2, K, best, bd); break;
        }
      } else {
#pragma unroll 4
      for (int j = 0; j < K; ++j) {
        const float* m = mu + j * ms;
        float c[RX];
        if (RB == 4) {
          const float4 c4 = *reinterpret_cast<const float4*>(m);
          c[0] = c4.x;
          c[RX > 1 ? 1 : 0] = c4.y;
          c[RX > 2 ? 2 : 0] = c4.z;
          c[RX > 3 ? 3 : 0] = c4.w;
        } else {
#pragma unroll
          for (int d = 0; d < RX; ++d) c[d] = d < rho ? m[d] : 0.f;
        }
        if (PPT >= 2) {
          float2 nc[RX];
#pragma unroll
          for (int d = 0; d < RX; ++d) nc[d] = make_float2(-c[d], -c[d]);
#pragma unroll
          for (int pr = 0; pr < PPT / 2; ++pr) {
            float2 t = __fadd2_rn(make_float2(x[2 * pr][0], x[2 * pr + 1][0]), nc[0]);
            float2 dist = __fmul2_rn(t, t);
#pragma unroll
            for (int d = 1; d < RX; ++d) {
              t = __fadd2_rn(make_float2(x[2 * pr][d], x[2 * pr + 1][d]), nc[d]);
              dist = __ffma2_rn(t, t, dist);
            }
            // strict: ties keep the lowest index
            if (dist.x < bd[2 * pr]) { bd[2 * pr] = dist.x; best[2 * pr] = j; }
            if (dist.y < bd[2 * pr + 1]) { bd[2 * pr + 1] = dist.y; best[2 * pr + 1] = j; }
          }
        } else {
          float dist = 0.f;
#pragma unroll
          for (int d = 0; d < RX; ++d) {
            const float t = x[0][d] - c[d];
            dist = fmaf(t, t, dist);
          }
          if (dist < bd[0]) { bd[0] = dist; best[0] = j; }
        }
      }
      }
#pragma unroll
      for (int q = 0; q < PPT; ++q)
        if (valid[q]) {
          qsum += bd[q];
          if (labels) labels[i0 + q] = best[q];
        }
      if (accumulate) {
        // merge this thread's rows by label (fixed order), then one warp
        // reduction per label present in the warp
        int cnt[PPT];
        bool live[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
          cnt[q] = 1;
          live[q] = valid[q];
        }
#pragma unroll
        for (int q = 1; q < PPT; ++q)
#pragma unroll
          for (int p = 0; p < q; ++p)
            if (live[p] && live[q] && best[p] == best[q]) {
#pragma unroll
              for (int d = 0; d < RX; ++d) x[p][d] += x[q][d];
              cnt[p] += cnt[q];
              live[q] = false;
            }
        for (int guard = 0; guard < 32 * PPT; ++guard) {
          int my = K;
#pragma unroll
          for (int q = PPT - 1; q >= 0; --q)
            if (live[q]) my = best[q];
          const unsigned any = __ballot_sync(kFull, my < K);
          if (!any) break;
          const int L = __shfl_sync(kFull, my, __ffs(any) - 1);
          float v[RX];
          int c = 0;
#pragma unroll
          for (int d = 0; d < RX; ++d) v[d] = 0.f;
#pragma unroll
          for (int q = 0; q < PPT; ++q)
            if (live[q] && best[q] == L) {
#pragma unroll
              for (int d = 0; d < RX; ++d) v[d] = x[q][d];
              c = cnt[q];
              live[q] = false;
            }
          float* a = acc + (warp * K + L) * stride;
#pragma unroll
          for (int d = 0; d < RX; ++d) {
            if (d < rho) {
              const float s = warp_sum(v[d]);
              if (lane == 0) a[d] += s;
            }
          }
          const unsigned total = __reduce_add_sync(kFull, (unsigned)c);
          if (lane == 0) a[rho] += (float)total;
        }
      }
    }
  } else {
    for (int64_t base = (int64_t)blk * THREADS; base < N; base += (int64_t)nblk * THREADS) {
      const int64_t i = base + tid;
      const bool valid = i < N;
      const float* xi = X + (valid ? i : 0) * rho;
      int best = 0;
      float bd = __int_as_float(0x7f800000);
      for (int j = 0; j < K; ++j) {
        const float* m = mu + j * ms;
        float dist = 0.f;
        for (int d = 0; d < rho; ++d) {
          const float t = __ldg(xi + d) - m[d];
          dist = fmaf(t, t, dist);
        }
        if (dist < bd) { bd = dist; best = j; }
      }
      if (valid) {
        qsum += bd;
        if (labels) labels[i] = best;
      }
      if (accumulate) {
        unsigned todo = __ballot_sync(kFull, valid);
        while (todo) {
          const int leader = __ffs(todo) - 1;
          const int L = __shfl_sync(kFull, best, leader);
          const bool mine = valid && best == L;
          const unsigned grp = __ballot_sync(kFull, mine);
          float* a = acc + (warp * K + L) * stride;
          for (int d = 0; d < rho; ++d) {
            const float v = warp_sum(mine ? __ldg(xi + d) : 0.f);
            if (lane == 0) a[d] += v;
          }
          if (lane == 0) a[rho] += (float)__popc(grp);
          todo &= ~grp;
        }
      }
    }
  }
  __syncthreads();
  if (accumulate) {
    for (int e = tid; e < K * stride; e += blockDim.x) {
      float s = 0.f;
      for (int w = 0; w < kWarps; ++w) s += acc[w * K * stride + e];
      part[(int64_t)blk * K * stride + e] = s;
    }
  }
  __shared__ float qs[kWarps];
  qsum = warp_sum(qsum);
  if (lane == 0) qs[warp] = qsum;
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int w = 0; w < kWarps; ++w) s += qs[w];
    qpart[blk] = s;
  }
}

// One CTA per cluster j: FP64 sums of the block partials in a fixed order, then
// the centroid moves to the mean of its members (kept if it has none).  The
// rho + 1 sums run side by side: thread (g, d) sums partials b = g, g + G, ...
// of coordinate d (d = rho is the count), then thread d adds the G group sums
// in order.
template <class P>
__global__ void __launch_bounds__(256) k_update(const __grid_constant__ P p, int rho, int K) {
  const KmJob& J = p.get();
  const float* __restrict__ part = J.part;
  const int nblk = J.grid;
  float* __restrict__ cent = J.cent;
  __shared__ double red[256];
  __shared__ double sum[kMaxRho + 1];
  const int j = blockIdx.x, tid = threadIdx.x, stride = rho + 1;
  const int G = 256 / stride;
  const int g = tid / stride, d = tid - g * stride;
  double s = 0.0;
  if (g < G) {
    const float* src = part + (int64_t)j * stride + d;
    const int64_t step = (int64_t)K * stride;
#pragma unroll 4
    for (int b = g; b < nblk; b += G) s += (double)src[b * step];
  }
  red[tid] = s;
  __syncthreads();
  if (tid < stride) {
    double t = 0.0;
    for (int q = 0; q < G; ++q) t += red[q * stride + tid];
    sum[tid] = t;
  }
  __syncthreads();
  if (tid < rho && sum[rho] > 0.0) cent[j * rho + tid] = (float)(sum[tid] / sum[rho]);
}

// Strip processing: the FP64 sums of the block partials without the division
// (sums[j][d], d < rho; sums[j][rho] = the count), one CTA per cluster, in the
// fixed order of k_update, so that partial sums of several strips can be added
// (all-reduced) before the centroids move.
__global__ void __launch_bounds__(256)
k_sums(const float* __restrict__ part, int nblk, int rho, int K, double* __restrict__ sums) {
  __shared__ double red[256];
  const int j = blockIdx.x, tid = threadIdx.x, stride = rho + 1;
  const int G = 256 / stride;
  const int g = tid / stride, d = tid - g * stride;
  double s = 0.0;
  if (g < G) {
    const float* src = part + (int64_t)j * stride + d;
    const int64_t step = (int64_t)K * stride;
    for (int b = g; b < nblk; b += G) s += (double)src[b * step];
  }
  red[tid] = s;
  __syncthreads();
  if (tid < stride) {
    double t = 0.0;
    for (int q = 0; q < G; ++q) t += red[q * stride + tid];
    sums[j * stride + tid] = t;
  }
}

// Centroid j = sums[j][0..rho) / sums[j][rho]; kept if the count is zero.
__global__ void k_apply_sums(const double* __restrict__ sums, int K, int rho, float* __restrict__ cent) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * rho; e += gridDim.x * blockDim.x) {
    const int j = e / rho, d = e - j * rho;
    const double c = sums[j * (rho + 1) + rho];
    if (c > 0.0) cent[e] = (float)(sums[j * (rho + 1) + d] / c);
  }
}

// out[j] = row idx[j] - row0 of X (N rows) when it lies in this strip, else zeros.
__global__ void k_gather_rows(const float* __restrict__ X, int64_t N, int rho, int64_t row0,
                              const int64_t* __restrict__ idx, int K, float* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * rho; e += gridDim.x * blockDim.x) {
    const int j = e / rho, d = e - j * rho;
    const int64_t r = idx[j] - row0;
    out[e] = (r >= 0 && r < N) ? X[r * rho + d] : 0.f;
  }
}

// Quantisation error e = sum of the block partials (FP64, fixed order).
template <class P>
__global__ void k_qerr(const __grid_constant__ P p) {
  const KmJob& J = p.get();
  const float* __restrict__ qpart = J.qpart;
  const int nblk = J.grid;
  double* __restrict__ out = J.qerr_out;
  DevState* state = J.state;
  __shared__ double red[256];
  const int tid = threadIdx.x;
  double s = 0.0;
  for (int b = tid; b < nblk; b += 256) s += (double)qpart[b];
  red[tid] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o) red[tid] += red[tid + o];
    __syncthreads();
  }
  if (tid == 0) {
    state->qerr = red[0];
    if (out) *out = red[0];
  }
}

// NLM subsample: stratum t of the row-major pixel order gives pixel
// lo + SplitMix64(seed ^ kSampleStream, t + 1) mod (hi - lo); its patch vector
// (reflect-101 border, order (dy, dx, c)) becomes row t of X.
__global__ void k_nlm_sample(const float* __restrict__ f, int H, int W, int n, int r, int64_t Ns,
                             uint64_t seed, int64_t* __restrict__ idx, float* __restrict__ X) {
  const int side = 2 * r + 1;
  const int rho = side * side * n;
  const int64_t N = (int64_t)H * W;
  const int64_t total = Ns * rho;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / rho;
    const int j = (int)(e - t * rho);
    const int64_t lo = (int64_t)(((unsigned __int128)t * N) / Ns);
    const int64_t hi = (int64_t)(((unsigned __int128)(t + 1) * N) / Ns);
    const int64_t pix = lo + (int64_t)(splitmix64(seed ^ kSampleStream, (uint64_t)t + 1) %
                                       (uint64_t)(hi - lo));
    if (j == 0) idx[t] = pix;
    const int c = j % n;
    const int q = j / n;
    const int dy = q / side - r, dx = q % side - r;
    const int y = (int)(pix / W), x = (int)(pix % W);
    X[e] = f[((int64_t)reflect101(y + dy, H) * W + reflect101(x + dx, W)) * n + c];
  }
}

template <class P, int RB>
cudaError_t assign_launch(const P& p, int grid, int rho, int K, int accumulate, cudaStream_t st) {
  constexpr int T = assign_threads(RB);
  constexpr int PPT = assign_ppt(RB);
  const size_t smem = assign_smem(K, rho);
  cudaError_t e = cudaFuncSetAttribute(k_assign<P, RB, T, PPT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_assign<P, RB, T, PPT><<<grid, T, smem, st>>>(p, rho, K, accumulate);
  count_launches(1);
  return cudaGetLastError();
}

// grid: total blocks of the launch (the sum of the problems' grids for KmMany)
template <class P>
cudaError_t assign_dispatch(const P& p, int grid, int rho, int K, int accumulate, cudaStream_t st) {
  if (rho <= 4) return assign_launch<P, 4>(p, grid, rho, K, accumulate, st);
  if (rho <= 8) return assign_launch<P, 8>(p, grid, rho, K, accumulate, st);
  if (rho <= 16) return assign_launch<P, 16>(p, grid, rho, K, accumulate, st);
  if (rho <= 32) return assign_launch<P, 32>(p, grid, rho, K, accumulate, st);
  return assign_launch<P, 0>(p, grid, rho, K, accumulate, st);
}

KmJob make_job(const float* X, int64_t N, int rho, float* cent, int32_t* labels, float* part,
               float* qpart, double* qerr_out, DevState* state) {
  KmJob j;
  j.X = X;
  j.N = N;
  j.cent = cent;
  j.labels = labels;
  j.part = part;
  j.qpart = qpart;
  j.qerr_out = qerr_out;
  j.init_idx = nullptr;
  j.idx_out = nullptr;
  j.state = state;
  j.seed = 0;
  j.grid = kmeans_grid(N, rho);
  return j;
}

}  // namespace

size_t kmeans_smem_bytes(int K, int rho) { return assign_smem(K, rho); }

cudaError_t launch_draw_init(const float* X, int64_t N, int rho, int K, uint64_t seed,
                             const int64_t* init_idx, int64_t* idx_out, float* centroids,
                             DevState* state, cudaStream_t st) {
  KmOne p;
  p.j = make_job(X, N, rho, centroids, nullptr, nullptr, nullptr, nullptr, state);
  p.j.seed = seed;
  p.j.init_idx = init_idx;
  p.j.idx_out = idx_out;
  k_draw_init<KmOne><<<1, 256, 0, st>>>(p, rho, K);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_kmeans(const float* X, int64_t N, int rho, int K, int iters, float* centroids,
                          int32_t* labels, double* qerr_out, float* part, float* qpart,
                          DevState* state, cudaStream_t st) {
  KmOne p;
  p.j = make_job(X, N, rho, centroids, nullptr, part, qpart, qerr_out, state);
  if (assign_tc_supported(rho, K)) {   // rows deep enough for the tensor cores
    const int grid = assign_tc_grid(N);
    p.j.grid = grid;
    for (int it = 0; it < iters; ++it) {
      cudaError_t e = launch_assign_tc(grid, X, N, rho, K, centroids, nullptr, part, qpart, 1,
                                       state, st);
      if (e != cudaSuccess) return e;
      k_update<KmOne><<<K, 256, 0, st>>>(p, rho, K);
      count_launches(1);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    cudaError_t e = launch_assign_tc(grid, X, N, rho, K, centroids, labels, part, qpart, 0, state, st);
    if (e != cudaSuccess) return e;
    k_qerr<KmOne><<<1, 256, 0, st>>>(p);
    count_launches(1);
    return cudaGetLastError();
  }
  const int grid = kmeans_grid(N, rho);
  p.j.grid = grid;
  for (int it = 0; it < iters; ++it) {
    cudaError_t e = assign_dispatch(p, grid, rho, K, 1, st);
    if (e != cudaSuccess) return e;
    k_update<KmOne><<<K, 256, 0, st>>>(p, rho, K);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  p.j.labels = labels;
  cudaError_t e = assign_dispatch(p, grid, rho, K, 0, st);
  if (e != cudaSuccess) return e;
  k_qerr<KmOne><<<1, 256, 0, st>>>(p);
  count_launches(1);
  return cudaGetLastError();
}

bool kmeans_batchable(int rho, int K) { return !assign_tc_supported(rho, K); }

cudaError_t launch_kmeans_batched(const KmItem* items, int count, int rho, int K, int iters,
                                  cudaStream_t st) {
  if (!kmeans_batchable(rho, K)) return cudaErrorInvalidValue;
  for (int b0 = 0; b0 < count; b0 += kBatchMax) {
    const int m = count - b0 < kBatchMax ? count - b0 : kBatchMax;
    KmMany p;
    p.count = m;
    int total = 0;
    for (int i = 0; i < kBatchMax; ++i) {
      const KmItem& it = items[b0 + (i < m ? i : 0)];
      p.j[i] = make_job(it.X, it.N, rho, it.cent, nullptr, it.part, it.qpart, nullptr, it.state);
      p.j[i].seed = it.seed;
      p.j[i].idx_out = it.idx_out;
      if (i < m) {
        p.first[i] = total;
        total += p.j[i].grid;
      }
    }
    p.first[m] = total;
    const dim3 one(1, m), clusters(K, m);
    k_draw_init<KmMany><<<one, 256, 0, st>>>(p, rho, K);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int it = 0; it < iters; ++it) {
      if ((e = assign_dispatch(p, total, rho, K, 1, st)) != cudaSuccess) return e;
      k_update<KmMany><<<clusters, 256, 0, st>>>(p, rho, K);
      count_launches(1);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = assign_dispatch(p, total, rho, K, 0, st)) != cudaSuccess) return e;
    k_qerr<KmMany><<<one, 256, 0, st>>>(p);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_kmeans_partials(const float* X, int64_t N, int rho, int K, const float* cent,
                                   double* sums, double* qerr, float* part, float* qpart,
                                   DevState* state, cudaStream_t st) {
  cudaError_t e;
  KmOne p;
  p.j = make_job(X, N, rho, const_cast<float*>(cent), nullptr, part, qpart, qerr, state);
  int grid;
  if (assign_tc_supported(rho, K)) {
    grid = assign_tc_grid(N);
    e = launch_assign_tc(grid, X, N, rho, K, cent, nullptr, part, qpart, 1, state, st);
  } else {
    grid = kmeans_grid(N, rho);
    e = assign_dispatch(p, grid, rho, K, 1, st);
  }
  if (e != cudaSuccess) return e;
  p.j.grid = grid;
  k_sums<<<K, 256, 0, st>>>(part, grid, rho, K, sums);
  k_qerr<KmOne><<<1, 256, 0, st>>>(p);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_apply_sums(const double* sums, int K, int rho, float* cent, cudaStream_t st) {
  k_apply_sums<<<(K * rho + 255) / 256, 256, 0, st>>>(sums, K, rho, cent);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const float* X, int64_t N, int rho, int64_t row0, const int64_t* idx,
                               int K, float* out, cudaStream_t st) {
  k_gather_rows<<<(K * rho + 255) / 256, 256, 0, st>>>(X, N, rho, row0, idx, K, out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_sample_rows(const float* guide, int64_t N, int rho, int64_t Ns, uint64_t seed,
                               int64_t* idx, float* X, cudaStream_t st) {
  int64_t grid = (Ns * rho + 255) / 256;
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  k_sample_rows<<<(int)grid, 256, 0, st>>>(guide, N, rho, Ns, seed, idx, X);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_nlm_sample(const float* f, int H, int W, int n, int r, int64_t Ns, uint64_t seed,
                              int64_t* idx, float* X, cudaStream_t st) {
  const int rho = (2 * r + 1) * (2 * r + 1) * n;
  const int64_t total = Ns * rho;
  int grid = (int)((total + 255) / 256);
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  k_nlm_sample<<<grid, 256, 0, st>>>(f, H, W, n, r, Ns, seed, idx, X);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace nyf

// k-means assignment on the fifth-generation tensor cores (tcgen05), for rows of
// dimension 16 <= rho <= 80 (hyperspectral pixels, NLM patch samples, PCA
// coordinates): the assignment step of Lloyd's algorithm (Sec. III, Algorithm 1's
// clustering), with the per-cluster sums of the update step, as two products.
//
//   X~ = X - c, M~ = mu - c   (c = mean of the centroids; distances do not change)
//   D  = ||x~||^2 + ||mu~||^2 - 2 X~ M~^T              (128 rows x K per tile)
//   label(i) = argmin_j D(i, j)   (ties to the lowest j),  e += min_j D(i, j)
//   S  += L^T [X | 1]                                  (K x (rho + 1) per CTA)
// L is the tile's one-hot label matrix (exact in bfloat16).  X~ M~^T and S use the
// exact three-term bfloat16 split of the FP32 operands (split_bf16.cuh): six
// products for the distances, three for the sums (L is exact), FP32 accumulation
// in tensor memory.  S accumulates in tensor memory over every tile a CTA takes,
// in a fixed tile order, so the partial sums are bitwise reproducible; column rho
// of S counts the members.  The CTA writes S and its error sum in the layout of
// the CUDA-core assignment pass (part[b][j][0..rho], qpart[b]), which the update
// pass reduces in FP64.
//
// One CTA of four warps owns a tile of 128 rows (tensor-memory lane t = row t):
//   1. each thread loads its row, writes the centred row's terms (A operand of the
//      distances) and the raw row's terms transposed (B operand of the sums, one
//      column per row, with a 1 in row rho for the count);
//   2. one thread issues the distance products;
//   3. each thread reads its distances, takes the nearest centroid and writes the
//      one in its column of L^T;
//   4. one thread issues the sum products, accumulating into S;
//   5. each thread clears its one once the products completed.
// Every wait is bounded: a timeout latches NYF_ERR_TIMEOUT, and the kernel waits
// (bounded) for its own products before freeing tensor memory.
#include "nyf_internal.cuh"
#include "split_bf16.cuh"
#include "umma.cuh"

namespace nyf {
namespace {

using splitbf::issue_split_gemm;
using splitbf::put8;
using splitbf::split3;

constexpr int kKtThreads = 128;
constexpr int kKtRows = 128;
constexpr uint32_t kKtWait = 1u << 20;
constexpr uint32_t kDCol = 0, kSCol = 64, kKtTmemCols = 256;
constexpr int kKtMaxRho = 80;

__host__ __device__ inline int kt_pad16(int v) { return (v + 15) & ~15; }

struct KtLayout {
  int rp, kp, np;            // rho, K and rho + 1 rounded up to 16
  int a1, b1, a2, b2, c, bn, total;
};

__host__ __device__ inline KtLayout kt_layout(int rho, int K) {
  KtLayout L;
  L.rp = kt_pad16(rho);
  L.kp = kt_pad16(K);
  L.np = kt_pad16(rho + 1);
  int o = 0;
  L.a1 = o;
  o += 3 * kKtRows * L.rp * 2;          // centred rows, three terms ([row][d])
  L.b1 = o;
  o += 3 * L.kp * L.rp * 2;             // centred centroids, three terms ([j][d])
  L.a2 = o;
  o += kKtRows * kKtRows * 2;           // L^T, one-hot ([j][row], rows j >= K zero)
  L.b2 = o;
  o += 3 * L.np * kKtRows * 2;          // [X | 1]^T, three terms ([d][row])
  L.c = o;
  o += 4 * L.rp;
  L.bn = o;
  o += 4 * L.kp;
  L.total = (o + 127) & ~127;
  return L;
}

// Element (r, k) of a K-major operand with a K-dim of kdim, one bfloat16.
__device__ __forceinline__ __nv_bfloat16* at_kmajor(unsigned char* base, int r, int k, int kdim) {
  return reinterpret_cast<__nv_bfloat16*>(base + umma::kmajor_offset(r, k, kdim));
}

// The three products of D (+)= A B^T with A exact (one term) and B in three terms.
__device__ __forceinline__ void issue_exact_a_gemm(uint32_t d_tmem, uint32_t a0, uint32_t b0,
                                                   int b_term, int kdim, uint32_t idesc,
                                                   uint32_t acc) {
  const uint32_t sbo = (uint32_t)kdim * 16;
#pragma unroll
  for (int j = 2; j >= 0; --j)
    for (int ks = 0; ks < kdim / 16; ++ks) {
      umma::mma_bf16(d_tmem, umma::sdesc(a0 + ks * 256, 128, sbo),
                     umma::sdesc(b0 + j * b_term + ks * 256, 128, sbo), idesc, acc);
      acc = 1;
    }
}

__global__ void __launch_bounds__(kKtThreads, 1)
k_assign_tc(const float* __restrict__ X, int64_t N, int rho, int K, const float* __restrict__ cent,
            int32_t* __restrict__ labels, float* __restrict__ part, float* __restrict__ qpart,
            int accumulate, DevState* __restrict__ state) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t mbar, drain;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  __shared__ float qs[kKtThreads / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const KtLayout L = kt_layout(rho, K);
  const int rp = L.rp, kp = L.kp, np = L.np;
  unsigned char* A1 = sm + L.a1;
  unsigned char* B1 = sm + L.b1;
  unsigned char* A2 = sm + L.a2;
  unsigned char* B2 = sm + L.b2;
  float* cen = reinterpret_cast<float*>(sm + L.c);
  float* bnorm = reinterpret_cast<float*>(sm + L.bn);
  const int a1_term = kKtRows * rp * 2, b1_term = kp * rp * 2, b2_term = np * kKtRows * 2;

  for (int d = tid; d < rp; d += kKtThreads) {       // centre: mean of the centroids
    float s = 0.f;
    if (d < rho)
      for (int j = 0; j < K; ++j) s += cent[j * rho + d];
    cen[d] = d < rho ? s / (float)K : 0.f;
  }
  // L^T and [X | 1]^T start at zero (rows j >= K of L^T and d > rho of B2 stay zero)
  for (int e = tid; e < kKtRows * kKtRows / 8; e += kKtThreads)
    reinterpret_cast<uint4*>(A2)[e] = make_uint4(0u, 0u, 0u, 0u);
  for (int e = tid; e < 3 * np * kKtRows / 8; e += kKtThreads)
    reinterpret_cast<uint4*>(B2)[e] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (int j = tid; j < kp; j += kKtThreads) {        // centroid terms and ||mu~||^2
    float nrm = 0.f;
    for (int d0 = 0; d0 < rp; d0 += 8) {
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int d = d0 + i;
        v[i] = (j < K && d < rho) ? cent[j * rho + d] - cen[d] : 0.f;
        nrm = fmaf(v[i], v[i], nrm);
      }
      put8(B1, b1_term, j, d0, rp, v);
    }
    bnorm[j] = nrm;
  }
  if (warp == 0) umma::tmem_alloc(&tslot, kKtTmemCols);
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
  const uint32_t a1_s = umma::smem_u32(A1), b1_s = umma::smem_u32(B1);
  const uint32_t a2_s = umma::smem_u32(A2), b2_s = umma::smem_u32(B2);
  const uint32_t id_d = umma::idesc_bf16(128, kp), id_s = umma::idesc_bf16(128, np);
  uint32_t phase = 0, s_acc = 0;
  float qsum = 0.f;
  bool ok = true;
  const int64_t ntiles = (N + kKtRows - 1) / kKtRows;

  for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
    // ---- 1. this thread's row: centred terms ([row][d]) and raw terms transposed ([d][row])
    const int64_t i = t * kKtRows + tid;
    const bool valid = i < N;
    const float* x = X + (valid ? i : 0) * (int64_t)rho;
    float anorm = 0.f;
    for (int d0 = 0; d0 < rp; d0 += 8) {
      float v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int d = d0 + k;
        const float raw = (valid && d < rho) ? __ldg(x + d) : 0.f;
        v[k] = (valid && d < rho) ? raw - cen[d] : 0.f;
        anorm = fmaf(v[k], v[k], anorm);
        if (accumulate && d < rho) {
          __nv_bfloat16 r1, r2, r3;
          split3(raw, r1, r2, r3);
          *at_kmajor(B2, d, tid, kKtRows) = r1;
          *at_kmajor(B2 + b2_term, d, tid, kKtRows) = r2;
          *at_kmajor(B2 + 2 * b2_term, d, tid, kKtRows) = r3;
        }
      }
      put8(A1, a1_term, tid, d0, rp, v);
    }
    if (accumulate) *at_kmajor(B2, rho, tid, kKtRows) = __float2bfloat16_rn(valid ? 1.f : 0.f);
    umma::fence_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    // ---- 2. the distances' cross term
    if (tid == 0) {
      issue_split_gemm(tbase + kDCol, a1_s, a1_term, b1_s, b1_term, rp, id_d);
      umma::commit(&mbar);
    }
    ok = __all_sync(0xffffffffu, umma::mbar_wait(&mbar, phase, kKtWait));
    phase ^= 1;
    umma::fence_after_sync();
    int best = 0;
    if (!ok) {
      atomicExch(&abort_flag, 1);
    } else {
      // ---- 3. nearest centroid (ties to the lowest index) and its one in L^T
      float bd = __int_as_float(0x7f800000);
      for (int c0 = 0; c0 < kp; c0 += 16) {
        float xv[16];
        umma::tmem_ld16(lane_base + kDCol + c0, xv);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int j = c0 + q;
          if (j < K) {
            const float s = anorm + bnorm[j];               // two-sum of the norms
            const float bb = s - anorm;
            const float err = (anorm - (s - bb)) + (bnorm[j] - bb);
            const float dd = fmaf(-2.f, xv[q], s) + err;
            if (dd < bd) {
              bd = dd;
              best = j;
            }
          }
        }
      }
      if (valid) {
        qsum += fmaxf(bd, 0.f);
        if (labels) labels[i] = best;
        if (accumulate) *at_kmajor(A2, best, tid, kKtRows) = __float2bfloat16_rn(1.f);
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
    if (accumulate) {
      // ---- 4. S += L^T [X | 1]
      if (tid == 0) {
        issue_exact_a_gemm(tbase + kSCol, a2_s, b2_s, b2_term, kKtRows, id_s, s_acc);
        umma::commit(&mbar);
      }
      s_acc = 1;
      ok = __all_sync(0xffffffffu, umma::mbar_wait(&mbar, phase, kKtWait));
      phase ^= 1;
      umma::fence_after_sync();
      if (!ok) atomicExch(&abort_flag, 1);
      // ---- 5. clear this thread's one (the products that read it have completed)
      else if (valid) *at_kmajor(A2, best, tid, kKtRows) = __float2bfloat16_rn(0.f);
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (abort_flag) ok = false;
  }
  // the CTA's partial sums (row j of S = cluster j) and its error sum
  if (ok && accumulate) {
    const int j = tid;                          // lane t of tensor memory = cluster t
    for (int c0 = 0; c0 < np; c0 += 16) {
      float v[16];
      umma::tmem_ld16(lane_base + kSCol + c0, v);
      if (j < K) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int d = c0 + q;
          if (d <= rho) part[((int64_t)blockIdx.x * K + j) * (rho + 1) + d] = v[q];
        }
      }
    }
  }
  float w = qsum;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  if (lane == 0) qs[warp] = w;
  // drain: every product this CTA issued has completed before tensor memory is freed
  if (tid == 0) {
    umma::commit(&drain);
    if (!umma::mbar_wait(&drain, 0, kKtWait)) atomicExch(&abort_flag, 1);
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (tid == 0) {
    qpart[blockIdx.x] = (qs[0] + qs[1]) + (qs[2] + qs[3]);
    if (abort_flag) set_status(state, NYF_ERR_TIMEOUT);
  }
  if (warp == 0) umma::tmem_dealloc(tbase, kKtTmemCols);
}

}  // namespace

bool assign_tc_supported(int rho, int K) { return rho >= 16 && rho <= kKtMaxRho && K <= kMaxK; }

// Grid of the tensor-core assignment for N rows (at most kKmeansBlocks partial slots).
int assign_tc_grid(int64_t N) {
  int64_t g = (N + kKtRows - 1) / kKtRows;
  if (g > 2 * 152) g = 2 * 152;
  if (g > kKmeansBlocks) g = kKmeansBlocks;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_assign_tc(int grid, const float* X, int64_t N, int rho, int K,
                             const float* cent, int32_t* labels, float* part, float* qpart,
                             int accumulate, DevState* state, cudaStream_t st) {
  const KtLayout L = kt_layout(rho, K);
  // no less than 76 KB, so that at most two CTAs (2 x 256 tensor-memory columns) share an SM
  const int smem = L.total > 76 * 1024 ? L.total : 76 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_assign_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_assign_tc<<<grid, kKtThreads, smem, st>>>(X, N, rho, K, cent, labels, part, qpart, accumulate,
                                               state);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace nyf

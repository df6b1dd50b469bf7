// Self-test of the tcgen05 building blocks (umma.cuh): one CTA computes
// D = A B^T for M = 128, N in {16, ..., 256}, K in {16, ..., 128} from operands
// generated in the kernel (small integers over powers of two, exact in
// bfloat16), with the accumulator in tensor memory.  The caller compares D with
// the same product computed on the host.  The paper has no counterpart; this
// checks the tensor-core plumbing the BF16 convolutions build on.
#include "nyf_internal.cuh"
#include "umma.cuh"

namespace nyf {
namespace {

constexpr uint32_t kWaitLimit = 1u << 22;   // mbarrier polls before giving up

__host__ __device__ inline float st_a(int m, int k) { return (float)(((m * 3 + k * 5) % 17) - 8) * 0.125f; }
__host__ __device__ inline float st_b(int n, int k) { return (float)(((n * 7 + k * 3) % 13) - 6) * 0.25f; }

// a_in_tmem: A is written into tensor memory (row m = lane m, bf16 pairs per
// 32-bit column) instead of shared memory.
__global__ void __launch_bounds__(128, 1) k_umma_selftest(float* __restrict__ D, int N, int K,
                                                         int a_in_tmem, int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int M = 128;
  unsigned char* A = sm;                       // M x K, K-major core matrices
  unsigned char* B = sm + M * K * 2;           // N x K
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < M * K; e += blockDim.x) {
    const int m = e / K, k = e - m * K;
    *reinterpret_cast<__nv_bfloat16*>(A + umma::kmajor_offset(m, k, K)) = __float2bfloat16(st_a(m, k));
  }
  for (int e = tid; e < N * K; e += blockDim.x) {
    const int n = e / K, k = e - n * K;
    *reinterpret_cast<__nv_bfloat16*>(B + umma::kmajor_offset(n, k, K)) = __float2bfloat16(st_b(n, k));
  }
  umma::fence_async_smem();
  uint32_t ncols = 32;
  while ((int)ncols < N + (a_in_tmem ? K / 2 : 0)) ncols <<= 1;
  if (warp == 0) umma::tmem_alloc(&tmem_slot, ncols);
  if (tid == 0) {
    umma::mbar_init(&mbar, 1);
    umma::fence_mbar_init();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tbase = tmem_slot;
  const uint32_t acol = (uint32_t)N;                 // A's columns follow D's when in TMEM
  if (a_in_tmem) {                                   // row m = 32 warp + lane, pairs of K
    const int m = 32 * warp + lane;
    for (int c0 = 0; c0 < K / 2; c0 += 32) {
      float v[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int kk = 2 * (c0 + i);
        __nv_bfloat162 h = __floats2bfloat162_rn(kk < K ? st_a(m, kk) : 0.f, kk + 1 < K ? st_a(m, kk + 1) : 0.f);
        v[i] = __uint_as_float(*reinterpret_cast<uint32_t*>(&h));
      }
      umma::tmem_st32(tbase + ((uint32_t)(32 * warp) << 16) + acol + c0, v);
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
  }
  if (tid == 0) {
    const uint32_t a0 = umma::smem_u32(A), b0 = umma::smem_u32(B);
    const uint32_t sbo = (uint32_t)K * 16;
    for (int ks = 0; ks < K / 16; ++ks) {
      if (a_in_tmem)
        umma::mma_bf16_ta(tbase, tbase + acol + 8 * ks, umma::sdesc(b0 + ks * 256, 128, sbo),
                          umma::idesc_bf16(M, N), ks > 0 ? 1u : 0u);
      else
        umma::mma_bf16(tbase, umma::sdesc(a0 + ks * 256, 128, sbo), umma::sdesc(b0 + ks * 256, 128, sbo),
                       umma::idesc_bf16(M, N), ks > 0 ? 1u : 0u);
    }
    umma::commit(&mbar);
  }
  const bool ok = __all_sync(0xffffffffu, umma::mbar_wait(&mbar, 0, kWaitLimit));   // warp-uniform
  umma::fence_after_sync();
  if (!ok && lane == 0) atomicExch(status, 1);
  if (ok) {
    for (int c0 = 0; c0 < N; c0 += 32) {
      float v[32];
      umma::tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
      const int m = 32 * warp + lane;
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (c0 + i < N) D[m * N + c0 + i] = v[i];
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tbase, ncols);
}

// Bounded-wait self-test: an mbarrier that nothing ever arrives on, waited for
// with `limit` polls (each at most ~1 us).  The wait gives up, the kernel
// latches NYF_ERR_TIMEOUT into *status and returns; nothing traps or hangs.
__global__ void k_wait_timeout_selftest(uint32_t limit, int* __restrict__ status) {
  __shared__ uint64_t mbar;
  if (threadIdx.x == 0) {
    umma::mbar_init(&mbar, 1);
    umma::fence_mbar_init();
  }
  __syncthreads();
  const bool ok = __all_sync(0xffffffffu, umma::mbar_wait(&mbar, 0, limit));
  if (!ok && threadIdx.x == 0) atomicCAS(status, 0, (int)NYF_ERR_TIMEOUT);
}

}  // namespace
}  // namespace nyf

using namespace nyf;

extern "C" nyf_status nyf_selftest_wait_timeout(int limit, int* status, void* stream) {
  if (!status || limit < 1 || limit > 4096) return NYF_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return NYF_ERR_CUDA;
  k_wait_timeout_selftest<<<1, 32, 0, st>>>((uint32_t)limit, status);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? NYF_OK : NYF_ERR_CUDA;
}

extern "C" nyf_status nyf_selftest_umma(float* D, int N, int K, int a_in_tmem, int* status,
                                        void* stream) {
  if (!D || !status || N < 16 || N > 256 || (N & 15) || K < 16 || K > 128 || (K & 15) ||
      (a_in_tmem && N + K / 2 > 512))
    return NYF_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t smem = (size_t)(128 + N) * K * 2;
  if (cudaFuncSetAttribute(k_umma_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return NYF_ERR_CUDA;
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return NYF_ERR_CUDA;
  k_umma_selftest<<<1, 128, smem, st>>>(D, N, K, a_in_tmem, status);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? NYF_OK : NYF_ERR_CUDA;
}

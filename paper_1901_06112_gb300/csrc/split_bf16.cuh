// Exact three-term bfloat16 splits of FP32 operands and the split products
// that the tensor-core kernels (features_tc.cu, kmeans_tc.cu) use to reach
// FP32 accuracy on the BF16 tcgen05 path: x = x1 + x2 + x3 with every term in
// bfloat16 (exact for FP32 x, bfloat16 having FP32's exponent range), and the
// six products x_i y_j of weight >= 2^-16 of the leading one summed in FP32.
#pragma once

#include "nyf_internal.cuh"
#include "umma.cuh"

namespace nyf {
namespace splitbf {

// x = x1 + x2 + x3 with each term in bfloat16 (exact for FP32 x).
__device__ __forceinline__ void split3(float x, __nv_bfloat16& x1, __nv_bfloat16& x2,
                                       __nv_bfloat16& x3) {
  x1 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(x1);
  x2 = __float2bfloat16_rn(r1);
  x3 = __float2bfloat16_rn(r1 - __bfloat162float(x2));
}

// Writes eight consecutive K-dim values of one row as the three terms' core-matrix rows.
__device__ __forceinline__ void put8(unsigned char* base, int term_bytes, int row, int k0, int kdim,
                                     const float (&v)[8]) {
  __align__(16) __nv_bfloat16 t1[8], t2[8], t3[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) split3(v[i], t1[i], t2[i], t3[i]);
  const uint32_t off = umma::kmajor_offset(row, k0, kdim);
  *reinterpret_cast<uint4*>(base + off) = *reinterpret_cast<const uint4*>(t1);
  *reinterpret_cast<uint4*>(base + term_bytes + off) = *reinterpret_cast<const uint4*>(t2);
  *reinterpret_cast<uint4*>(base + 2 * term_bytes + off) = *reinterpret_cast<const uint4*>(t3);
}

// The six split products of D (+)= A B^T over a K-dim of kdim, smallest first.
__device__ __forceinline__ void issue_split_gemm(uint32_t d_tmem, uint32_t a0, int a_term,
                                                 uint32_t b0, int b_term, int kdim, uint32_t idesc) {
  const int ia[6] = {2, 1, 0, 1, 0, 0};
  const int ib[6] = {0, 1, 2, 0, 1, 0};
  const uint32_t sbo = (uint32_t)kdim * 16;
  uint32_t acc = 0;
#pragma unroll
  for (int p = 0; p < 6; ++p)
    for (int ks = 0; ks < kdim / 16; ++ks) {
      umma::mma_bf16(d_tmem, umma::sdesc(a0 + ia[p] * a_term + ks * 256, 128, sbo),
                     umma::sdesc(b0 + ib[p] * b_term + ks * 256, 128, sbo), idesc, acc);
      acc = 1;
    }
}

}  // namespace splitbf
}  // namespace nyf

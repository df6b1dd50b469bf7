// Device side of the recursive O(1) Gaussian (Young & van Vliet 1995) used for
// the spatial convolutions of Eqs. (14)-(15) when omega is a Gaussian (the
// filter of the paper's experiments, Sec. IV).
//
// Each line (a column, then a row) is filtered by the causal recursion
//     w[i] = B x[i] + c1 w[i-1] + c2 w[i-2] + c3 w[i-3]
// and the same recursion run backwards on w, on the line extended by zeros
// (the window clipping of Eq. (1)).  It is evaluated in difference form, with
// state (w[i], d1 = w[i] - w[i-1], d2 = w[i-1] - w[i-2]):
//     dl = B x[i] - B w[i-2] + g1 d1 - e2 d2,   w[i] = w[i-1] + dl,
// (e1 = c2 + c3, e2 = c3, g1 = -(e1 + B)): the same filter, but B stays an FP32
// number of its own instead of 1 - (c1 + c2 + c3) of rounded coefficients,
// which for sigma_s >> 1 (poles near z = 1, B small) is about 100x more
// accurate in FP32.
//
// A warp filters one line padded with zeros to 32 LS values: lane l holds
// [l LS, (l + 1) LS) in registers (LS odd: conflict-free shared-memory walks).
// Each lane runs the recursion from a zero state; the true incoming state of
// every segment follows from an inclusive scan over the lanes of the local end
// states (state_out = T^LS state_in + local_end, T the homogeneous step, its
// powers T^{LS 2^d} precomputed), and the continuation of that state is added.
// The padding is part of the zero-padded line, so the causal pass simply runs
// on through it; at the padded end a 3 x 3 map Rm gives the state the
// anticausal pass starts from (the causal recursion continued through the rest
// of the infinite zero padding, then run back).  The anticausal pass repeats
// the scheme with a suffix scan.
#pragma once

#include "nyf_internal.cuh"

namespace nyf {
namespace iir {

constexpr int kColWarps = 4;          // column pairs per CTA of the column pass
constexpr int kUnroll = 8;            // rows staged per thread per batch (2 loads each in flight)

// One line direction: coefficients and the lane-scan matrices, all in the
// difference basis (value, first difference, previous first difference).
struct Line {
  float B, nB, g1, ne2;  // B, -B, g1 = -(e1 + B), -e2
  int LS;               // values per lane; the padded line has 32 LS
  int len;              // true line length
  int pad0, pad1;
  float P[5][9];        // T^{LS 2^d}, d = 0..4, row-major
  float Rm[9];          // anticausal state at 32 LS from the causal state at 32 LS - 1
};

struct Args {
  const float* f;       // H x W x n
  const float* phi;     // K planes of H x W
  float* Y;             // K (n + 1) planes of H x W: vertically filtered phi_k f_c, phi_k
  float* out;           // H x W x n, or nullptr (zeta to the workspace, divided afterwards)
  float* eta;           // H x W
  float* zeta;          // H x W x n when out == nullptr
  const DevState* state;
  DevState* state_rw;
  int H, W, n;
  int64_t N;
  float eta_thr;
  Line col, row;
};

// Two lines are filtered per lane with paired FP32 arithmetic (FFMA2): x and y
// of every float2 belong to two independent lines with the same coefficients.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ float2 shfl_up2(float2 v, int off) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, off), __shfl_up_sync(0xffffffffu, v.y, off));
}
__device__ __forceinline__ float2 shfl_down2(float2 v, int off) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, off), __shfl_down_sync(0xffffffffu, v.y, off));
}

// acc += M x for both lines (M: 3 x 3 row-major)
__device__ __forceinline__ void mat3_acc2(float2& a0, float2& a1, float2& a2, const float* M, float2 x0,
                                          float2 x1, float2 x2) {
  a0 = fma2(f2(M[0]), x0, fma2(f2(M[1]), x1, fma2(f2(M[2]), x2, a0)));
  a1 = fma2(f2(M[3]), x0, fma2(f2(M[4]), x1, fma2(f2(M[5]), x2, a1)));
  a2 = fma2(f2(M[6]), x0, fma2(f2(M[7]), x1, fma2(f2(M[8]), x2, a2)));
}

// Coefficients of one direction as pairs.
struct Coef2 {
  float2 B, nB, g1, ne2;
  __device__ __forceinline__ explicit Coef2(const Line& c) : B(f2(c.B)), nB(f2(c.nB)), g1(f2(c.g1)), ne2(f2(c.ne2)) {}
};

// One step with input x: (w1, w2) = (w[i-1], w[i-2]), (d1, d2) = (w[i-1] - w[i-2],
// w[i-2] - w[i-3]); returns w[i] and shifts.  The chain from one step to the
// next is the single FMA with g1.
__device__ __forceinline__ float2 step_in(float2 x, float2& w1, float2& w2, float2& d1, float2& d2,
                                          const Coef2& c) {
  const float2 pre = fma2(c.B, x, fma2(c.nB, w2, mul2(c.ne2, d2)));
  const float2 dl = fma2(c.g1, d1, pre);
  const float2 w = add2(w1, dl);
  w2 = w1;
  w1 = w;
  d2 = d1;
  d1 = dl;
  return w;
}

// The same step with zero input: the continuation of an incoming state.
__device__ __forceinline__ float2 step_free(float2& w1, float2& w2, float2& d1, float2& d2, const Coef2& c) {
  const float2 pre = fma2(c.nB, w2, mul2(c.ne2, d2));
  const float2 dl = fma2(c.g1, d1, pre);
  const float2 w = add2(w1, dl);
  w2 = w1;
  w1 = w;
  d2 = d1;
  d1 = dl;
  return w;
}

// Filters in place the two padded lines the warp holds (lane l: v = values
// [l LS, (l + 1) LS) of both lines).
template <int LS>
__device__ __forceinline__ void filter_lines(float2 (&v)[LS], int lane, const Line& line) {
  const Coef2 c(line);
  const float2 z = f2(0.f);
  float2 w1 = z, w2 = z, d1 = z, d2 = z;
#pragma unroll
  for (int j = 0; j < LS; ++j) v[j] = step_in(v[j], w1, w2, d1, d2, c);
  const float2 e0 = w1, e1 = d1, e2 = d2;
  float2 p0 = e0, p1 = e1, p2 = e2;         // inclusive prefix of the end states
#pragma unroll
  for (int d = 0; d < 5; ++d) {
    const int off = 1 << d;
    const float2 q0 = shfl_up2(p0, off), q1 = shfl_up2(p1, off), q2 = shfl_up2(p2, off);
    if (lane >= off) mat3_acc2(p0, p1, p2, line.P[d], q0, q1, q2);
  }
  float2 h0 = shfl_up2(p0, 1), h1 = shfl_up2(p1, 1), h2 = shfl_up2(p2, 1);
  if (lane == 0) h0 = h1 = h2 = z;
  w1 = h0;
  w2 = sub2(h0, h1);
  d1 = h1;
  d2 = h2;
#pragma unroll
  for (int j = 0; j < LS; ++j) v[j] = add2(v[j], step_free(w1, w2, d1, d2, c));
  // lane 31: true causal state at the padded end -> anticausal state entering there
  float2 r0 = z, r1 = z, r2 = z;
  if (lane == 31) mat3_acc2(r0, r1, r2, line.Rm, add2(e0, w1), add2(e1, d1), add2(e2, d2));
  w1 = w2 = d1 = d2 = z;
#pragma unroll
  for (int j = LS - 1; j >= 0; --j) v[j] = step_in(v[j], w1, w2, d1, d2, c);
  float2 g0 = w1, g1 = d1, g2 = d2;         // suffix of the start states
  if (lane == 31) mat3_acc2(g0, g1, g2, line.P[0], r0, r1, r2);
#pragma unroll
  for (int d = 0; d < 5; ++d) {
    const int off = 1 << d;
    const float2 q0 = shfl_down2(g0, off), q1 = shfl_down2(g1, off), q2 = shfl_down2(g2, off);
    if (lane + off < 32) mat3_acc2(g0, g1, g2, line.P[d], q0, q1, q2);
  }
  float2 k0 = shfl_down2(g0, 1), k1 = shfl_down2(g1, 1), k2 = shfl_down2(g2, 1);
  if (lane == 31) {
    k0 = r0;
    k1 = r1;
    k2 = r2;
  }
  w1 = k0;
  w2 = sub2(k0, k1);
  d1 = k1;
  d2 = k2;
#pragma unroll
  for (int j = LS - 1; j >= 0; --j) v[j] = add2(v[j], step_free(w1, w2, d1, d2, c));
}

// ---- column pass: Y_kc = omega_v * (phi_k f_c), Y_kn = omega_v * phi_k.
// One CTA per (8-column strip, k); warp w filters columns x0 + 2w, x0 + 2w + 1
// (a float2 per row).  Thread t stages column t & 7 of rows t >> 3, + 16, ...
// into a tile of 32 LS rows (zero below H) with a 10-float pitch: the float2
// column walks of the 32 lanes (rows LS apart, LS odd) are conflict-free.
// Small CTAs (4 warps, 45 KB at H = 1080) let four of them share an SM, so that
// one CTA's staging overlaps another's filtering.
template <int LS>
__global__ void __launch_bounds__(kColWarps * 32, LS <= 47 ? 4 : 2) k_cols(const __grid_constant__ Args a) {
  const int k = blockIdx.y;
  if (k >= a.state->planes) return;
  extern __shared__ __align__(16) float sm_cols[];
  constexpr int PT = 2 * kColWarps + 2;
  constexpr int HP = 32 * LS;              // padded column length
  constexpr int RS = kColWarps * 32 / (2 * kColWarps); // rows one pass of the threads covers
  float* tile = sm_cols;
  const int H = a.H, W = a.W, n = a.n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tx = threadIdx.x & (2 * kColWarps - 1), ty = threadIdx.x / (2 * kColWarps);
  const int x = blockIdx.x * (2 * kColWarps) + tx;
  const bool xin = x < W;
  const float* php = a.phi + (int64_t)k * a.N + x;
  for (int c = 0; c <= n; ++c) {
    const float* fp = a.f + (int64_t)x * n + c;
    const int64_t fstride = (int64_t)W * n;
    for (int r0 = ty; r0 < HP; r0 += RS * kUnroll) {
      float pv[kUnroll], fv[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int r = r0 + u * RS;
        const bool in = xin && r < H;
        pv[u] = in ? __ldg(php + (int64_t)r * W) : 0.f;
        fv[u] = (in && c < n) ? __ldg(fp + (int64_t)r * fstride) : 1.f;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int r = r0 + u * RS;
        if (r < HP) tile[r * PT + tx] = pv[u] * fv[u];
      }
    }
    __syncthreads();
    float2 v[LS];
    float2* col = reinterpret_cast<float2*>(tile + lane * LS * PT + 2 * warp);
#pragma unroll
    for (int j = 0; j < LS; ++j) v[j] = col[j * (PT / 2)];
    filter_lines<LS>(v, lane, a.col);
#pragma unroll
    for (int j = 0; j < LS; ++j) col[j * (PT / 2)] = v[j];
    __syncthreads();
    float* Yp = a.Y + ((int64_t)k * (n + 1) + c) * a.N + x;
    if (xin)
      for (int r = ty; r < H; r += RS) Yp[(int64_t)r * W] = tile[r * PT + tx];
    __syncthreads();
  }
}

__device__ __forceinline__ void cp16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Copy W floats from src to dst (all threads of the CTA).
__device__ __forceinline__ void stage_row(float* dst, const float* src, int W, bool vec) {
  if (vec) {
    for (int e = threadIdx.x * 4; e < W; e += blockDim.x * 4) cp16(dst + e, src + e);
  } else {
    for (int e = threadIdx.x; e < W; e += blockDim.x) cp4(dst + e, src + e);
  }
}

// ---- row pass + combine: one CTA per row y, warp w filters quantity c0 + w
// (c < n: a channel of zeta, c == n: eta) for the planes k, k + 1 together and
// accumulates phi_k (omega * .) + phi_k+1 (omega * .) in registers.  The rows of
// Y are staged once (released as soon as they are in registers, then the next
// pair is fetched during the filtering); the rows of phi, needed after the
// filtering, have two stages.  Row padding [W, 32 LS) is zeroed once.
template <int LS>
__global__ void __launch_bounds__(LS <= 31 ? 512 : 256) k_rows(const __grid_constant__ Args a) {
  extern __shared__ __align__(16) float sm_rows[];
  constexpr int pitch = 32 * LS;            // padded row length (a multiple of 32)
  const int y = blockIdx.x;
  const int W = a.W, n = a.n, planes = a.state->planes;
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* ybuf = sm_rows;                    // 2 nw rows: Y_k,c0+w and Y_k+1,c0+w
  float* pbuf = sm_rows + 2 * nw * pitch;   // 2 stages x 2 rows: phi_k, phi_k+1
  const int base = lane * LS;
  const bool vec = (W & 3) == 0;
  const int64_t row0 = (int64_t)y * W;
  const bool fused = a.out != nullptr;
  const int nrows = 2 * nw + 4;
  for (int i = threadIdx.x; i < nrows * (pitch - W); i += blockDim.x) {
    const int r = i / (pitch - W);
    sm_rows[r * pitch + W + (i - r * (pitch - W))] = 0.f;
  }
  for (int c0 = 0; c0 <= n; c0 += nw) {
    const int c = c0 + warp;
    const int nact = min(nw, n + 1 - c0);
    float acc[LS];
#pragma unroll
    for (int j = 0; j < LS; ++j) acc[j] = 0.f;
    // stage pair p (planes 2p, 2p + 1): Y rows into ybuf, phi rows into pbuf stage p & 1
    auto issue = [&](int p) {
      const int k0 = 2 * p;
      const int nk = min(2, planes - k0);
      for (int t = 0; t < nk; ++t) {
        stage_row(pbuf + ((p & 1) * 2 + t) * pitch, a.phi + (int64_t)(k0 + t) * a.N + row0, W, vec);
        for (int q = 0; q < nact; ++q)
          stage_row(ybuf + (2 * q + t) * pitch,
                    a.Y + ((int64_t)(k0 + t) * (n + 1) + c0 + q) * a.N + row0, W, vec);
      }
      cp_commit();
    };
    const int pairs = (planes + 1) >> 1;
    if (pairs > 0) issue(0);
    for (int p = 0; p < pairs; ++p) {
      const bool two = 2 * p + 1 < planes;
      cp_wait_all();
      __syncthreads();
      float2 v[LS];
      if (warp < nact) {
        const float* ya = ybuf + 2 * warp * pitch + base;
        const float* yb = ya + pitch;
#pragma unroll
        for (int j = 0; j < LS; ++j) v[j] = make_float2(ya[j], two ? yb[j] : 0.f);
      }
      __syncthreads();
      if (p + 1 < pairs) issue(p + 1);
      if (warp < nact) {
        filter_lines<LS>(v, lane, a.row);
        const float* pa = pbuf + (p & 1) * 2 * pitch + base;
        const float* pb = pa + pitch;
#pragma unroll
        for (int j = 0; j < LS; ++j) acc[j] = fmaf(pa[j], v[j].x, two ? fmaf(pb[j], v[j].y, acc[j]) : acc[j]);
      }
    }
    __syncthreads();
    if (warp < nact && c == n) {            // eta
      unsigned small = 0;
#pragma unroll
      for (int j = 0; j < LS; ++j)
        if (base + j < W) {
          a.eta[row0 + base + j] = acc[j];
          if (fused) sm_rows[base + j] = acc[j];
          small += !(acc[j] > a.eta_thr);
        }
      small = __reduce_add_sync(0xffffffffu, small);
      if (lane == 0 && small) atomicAdd(&a.state_rw->eta_small, (unsigned long long)small);
    }
    if (fused) {                            // one round: every quantity is in this CTA
      __syncthreads();
      float* ost = sm_rows + pitch;         // W x n interleaved output row
      if (warp < n) {
#pragma unroll
        for (int j = 0; j < LS; ++j)
          if (base + j < W) ost[(base + j) * n + c] = acc[j] / sm_rows[base + j];
      }
      __syncthreads();
      float* dst = a.out + row0 * n;
      for (int i = threadIdx.x; i < W * n; i += blockDim.x) dst[i] = ost[i];
    } else if (warp < nact && c < n) {
#pragma unroll
      for (int j = 0; j < LS; ++j)
        if (base + j < W) a.zeta[(row0 + base + j) * n + c] = acc[j];
    }
    __syncthreads();
  }
}

// Launchers, instantiated for LS = 3, 7, ..., 63 in the iir_*.cu units.
template <int LS>
cudaError_t launch_cols(const Args& a, int K, cudaStream_t st) {
  const size_t smem = sizeof(float) * (size_t)(32 * LS) * (2 * kColWarps + 2);
  cudaError_t e = cudaFuncSetAttribute(k_cols<LS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)ceil_div(a.W, 2 * kColWarps), (unsigned)K);
  k_cols<LS><<<grid, kColWarps * 32, smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

// Shared memory of the row pass: 2 nw Y rows and 2 x 2 phi rows of 32 LS floats.
constexpr size_t rows_smem(int LS, int nw) { return sizeof(float) * (size_t)(2 * nw + 4) * (32 * LS); }

template <int LS>
cudaError_t launch_rows(const Args& a, int nw, cudaStream_t st) {
  const size_t smem = rows_smem(LS, nw);
  cudaError_t e = cudaFuncSetAttribute(k_rows<LS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_rows<LS><<<a.H, nw * 32, smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

// Largest number of quantity warps per CTA of the row pass (register budget).
constexpr int row_warps_max(int LS) { return LS <= 31 ? 16 : 8; }

cudaError_t dispatch_cols_3_31(int LS, const Args& a, int K, cudaStream_t st);
cudaError_t dispatch_cols_35_63(int LS, const Args& a, int K, cudaStream_t st);
cudaError_t dispatch_rows_3_31(int LS, const Args& a, int nw, cudaStream_t st);
cudaError_t dispatch_rows_35_63(int LS, const Args& a, int nw, cudaStream_t st);

}  // namespace iir
}  // namespace nyf

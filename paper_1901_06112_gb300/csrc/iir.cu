// Recursive O(1) Gaussian (Young & van Vliet 1995) for the spatial convolutions
// of Eqs. (14)-(15): the filter the paper's experiments use for a Gaussian omega
// (Sec. IV) and one of the O(1)-per-pixel methods Sec. III names for the
// (n + 1) K convolutions.  Cost per pixel and plane is independent of sigma_s.
//
// Each line (a column, then a row) is filtered by the causal recursion
//     w[i] = B x[i] + c1 w[i-1] + c2 w[i-2] + c3 w[i-3]
// followed by the same recursion run backwards on w.  It is evaluated in
// difference form, with state (w[i], d1 = w[i] - w[i-1], d2 = w[i-1] - w[i-2]):
//     dl = B (x[i] - w[i-2]) + g1 d1 - e2 d2,  w[i] = w[i-1] + dl,
// (e1 = c2 + c3, e2 = c3, g1 = -(e1 + B)), which is the same filter; for
// sigma_s >> 1 the poles approach z = 1 and B = 1 - c1 - c2 - c3 becomes
// small, and this form keeps B as its own FP32 number instead of a difference
// of rounded coefficients (about 100x less FP32 error at sigma_s = 20).  The line is zero-padded
// on both sides (the window clipping of Eq. (1)): the causal pass starts from a
// zero state, and the anticausal pass starts from the state the causal pass
// reaches after running on into the zero padding, a 3 x 3 map Rm of the causal
// end state computed on the host in FP64.
//
// A warp filters one line: lane l holds the odd-length segment
// [l Ls, (l + 1) Ls) in registers.  Each lane runs the recursion on its segment
// from a zero state; the true incoming state of every segment follows from an
// inclusive scan over the lanes of the segments' end states (state_out =
// M^Ls state_in + local_end, M the companion matrix of the recursion, its powers
// M^{Ls 2^d} precomputed); the homogeneous continuation of that state is then
// added to the segment.  The anticausal pass does the same with a suffix scan.
//
// k_iir_cols: one warp per column of an 8-column strip staged in shared memory
// (input phi_k f_c formed on the fly), writing the vertically filtered planes
// Y_kc.  k_iir_rows: one CTA per image row, one warp per quantity c (the n
// channels of zeta and eta), rows of Y_kc and phi_k double-buffered with
// cp.async; zeta_c = sum_k phi_k (omega * (phi_k f_c)) accumulates in
// registers and g_hat = zeta / eta is written in the same kernel.
#include <math.h>

#include <algorithm>

#include "nyf_internal.cuh"

namespace nyf {
namespace {

constexpr int kColWarps = 8;          // columns per CTA of the column pass

// One line direction: recursion coefficients and the lane-scan matrices, all in
// the difference basis (value, first difference, previous first difference).
struct IirLine {
  float B, nB, g1, ne2;  // B, -B, g1 = -(e1 + B), -e2
  int Ls;               // segment length (odd)
  int len;              // line length
  int last;             // last lane holding data: (len - 1) / Ls
  int pad;
  float P[5][9];        // T^{Ls 2^d}, d = 0..4, row-major; T the homogeneous step
  float Plast[9];       // T^{len - last Ls}
  float Rm[9];          // anticausal state entering at len from the causal state at len - 1
};

struct IirArgs {
  const float* f;       // H x W x n
  const float* phi;     // K planes of H x W
  float* Y;             // K (n + 1) planes of H x W: vertically filtered phi_k f_c, phi_k
  float* out;           // H x W x n, or nullptr (zeta to zeta_ws, divided afterwards)
  float* eta;           // H x W
  float* zeta;          // H x W x n when out == nullptr
  const DevState* state;
  DevState* state_rw;
  int H, W, n;
  int64_t N;
  float eta_thr;
  IirLine col, row;
};

// acc += M x (3 x 3, row-major)
__device__ __forceinline__ void mat3_acc(float& a0, float& a1, float& a2, const float* M, float x0,
                                         float x1, float x2) {
  a0 = fmaf(M[0], x0, fmaf(M[1], x1, fmaf(M[2], x2, a0)));
  a1 = fmaf(M[3], x0, fmaf(M[4], x1, fmaf(M[5], x2, a1)));
  a2 = fmaf(M[6], x0, fmaf(M[7], x1, fmaf(M[8], x2, a2)));
}

// One step of the recursion in difference form: (w1, w2) = (w[i-1], w[i-2]),
// (d1, d2) = (w[i-1] - w[i-2], w[i-2] - w[i-3]); returns w[i] and shifts.
__device__ __forceinline__ float iir_step(float x, float& w1, float& w2, float& d1, float& d2,
                                          const IirLine& c) {
  const float pre = fmaf(c.B, x - w2, c.ne2 * d2);
  const float dl = fmaf(c.g1, d1, pre);
  const float w = w1 + dl;
  w2 = w1;
  w1 = w;
  d2 = d1;
  d1 = dl;
  return w;
}

// The same step with zero input (the continuation of an incoming state).
__device__ __forceinline__ float iir_free(float& w1, float& w2, float& d1, float& d2, const IirLine& c) {
  const float pre = fmaf(c.nB, w2, c.ne2 * d2);
  const float dl = fmaf(c.g1, d1, pre);
  const float w = w1 + dl;
  w2 = w1;
  w1 = w;
  d2 = d1;
  d1 = dl;
  return w;
}

// Filters the line held by the warp in place: lane `lane` holds v[0..len) (len
// may be <= 0 past the end of the line), lanes 0..last - 1 hold Ls values each.
// States are (w, d1, d2); w2 = w - d1 is carried alongside.
template <int LS>
__device__ __forceinline__ void iir_line(float (&v)[LS], int len, int lane, const IirLine& c) {
  const unsigned all = 0xffffffffu;
  // causal pass from a zero state
  float w1 = 0.f, w2 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
  for (int j = 0; j < LS; ++j)
    if (j < len) v[j] = iir_step(v[j], w1, w2, d1, d2, c);
  const float e0 = w1, e1 = d1, e2 = d2;
  // inclusive prefix over lanes of the local end states
  float p0 = e0, p1 = e1, p2 = e2;
#pragma unroll
  for (int d = 0; d < 5; ++d) {
    const int off = 1 << d;
    const float q0 = __shfl_up_sync(all, p0, off);
    const float q1 = __shfl_up_sync(all, p1, off);
    const float q2 = __shfl_up_sync(all, p2, off);
    if (lane >= off) mat3_acc(p0, p1, p2, c.P[d], q0, q1, q2);
  }
  float h0 = __shfl_up_sync(all, p0, 1), h1 = __shfl_up_sync(all, p1, 1), h2 = __shfl_up_sync(all, p2, 1);
  if (lane == 0) h0 = h1 = h2 = 0.f;
  // add the continuation of the incoming state
  float hw1 = h0, hw2 = h0 - h1, hd1 = h1, hd2 = h2;
#pragma unroll
  for (int j = 0; j < LS; ++j)
    if (j < len) v[j] += iir_free(hw1, hw2, hd1, hd2, c);
  // true causal end state of the line on the last lane, mapped through the zero padding
  float r0 = 0.f, r1 = 0.f, r2 = 0.f;
  if (lane == c.last) mat3_acc(r0, r1, r2, c.Rm, e0 + hw1, e1 + hd1, e2 + hd2);
  // anticausal pass from a zero state at each segment's end
  w1 = w2 = d1 = d2 = 0.f;
#pragma unroll
  for (int j = LS - 1; j >= 0; --j)
    if (j < len) v[j] = iir_step(v[j], w1, w2, d1, d2, c);
  // suffix over lanes of the local start states; the last lane's includes the boundary
  float g0 = w1, g1 = d1, g2 = d2;
  if (lane == c.last) mat3_acc(g0, g1, g2, c.Plast, r0, r1, r2);
#pragma unroll
  for (int d = 0; d < 5; ++d) {
    const int off = 1 << d;
    const float q0 = __shfl_down_sync(all, g0, off);
    const float q1 = __shfl_down_sync(all, g1, off);
    const float q2 = __shfl_down_sync(all, g2, off);
    if (lane + off < 32) mat3_acc(g0, g1, g2, c.P[d], q0, q1, q2);
  }
  float k0 = __shfl_down_sync(all, g0, 1), k1 = __shfl_down_sync(all, g1, 1), k2 = __shfl_down_sync(all, g2, 1);
  if (lane == c.last) {
    k0 = r0;
    k1 = r1;
    k2 = r2;
  }
  hw1 = k0;
  hw2 = k0 - k1;
  hd1 = k1;
  hd2 = k2;
#pragma unroll
  for (int j = LS - 1; j >= 0; --j)
    if (j < len) v[j] += iir_free(hw1, hw2, hd1, hd2, c);
}

// ---- column pass: Y_kc = omega_v * (phi_k f_c), Y_kn = omega_v * phi_k
template <int LS>
__global__ void __launch_bounds__(kColWarps * 32) k_iir_cols(const __grid_constant__ IirArgs a) {
  const int k = blockIdx.y;
  if (k >= a.state->planes) return;
  extern __shared__ float tile[];          // H rows x (kColWarps + 1): odd pitch
  constexpr int PT = kColWarps + 1;
  const int H = a.H, W = a.W, n = a.n;
  const int x0 = blockIdx.x * kColWarps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Ls = a.col.Ls, base = lane * Ls, len = min(Ls, H - base);
  const float* phik = a.phi + (int64_t)k * a.N;
  for (int c = 0; c <= n; ++c) {
    for (int i = threadIdx.x; i < H * kColWarps; i += blockDim.x) {
      const int r = i / kColWarps, cc = i - r * kColWarps, x = x0 + cc;
      float v = 0.f;
      if (x < W) {
        const int64_t p = (int64_t)r * W + x;
        v = phik[p];
        if (c < n) v *= a.f[p * n + c];
      }
      tile[r * PT + cc] = v;
    }
    __syncthreads();
    float v[LS];
#pragma unroll
    for (int j = 0; j < LS; ++j) v[j] = j < len ? tile[(base + j) * PT + warp] : 0.f;
    iir_line<LS>(v, len, lane, a.col);
#pragma unroll
    for (int j = 0; j < LS; ++j)
      if (j < len) tile[(base + j) * PT + warp] = v[j];
    __syncthreads();
    float* Yp = a.Y + ((int64_t)k * (n + 1) + c) * a.N;
    for (int i = threadIdx.x; i < H * kColWarps; i += blockDim.x) {
      const int r = i / kColWarps, cc = i - r * kColWarps, x = x0 + cc;
      if (x < W) Yp[(int64_t)r * W + x] = tile[r * PT + cc];
    }
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
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Stage the row of phi_k (dst row 0) and the rows of Y_k,c0..c0+nq-1 (dst rows
// 1..nq) starting at element row0 of their planes; all threads take part.
__device__ __forceinline__ void stage_rows(float* dst, int pitch, const float* phik, const float* ykc0,
                                           int64_t plane, int nq, int64_t row0, int W, bool vec) {
  const int rows = nq + 1;
  if (vec) {
    const int q = W >> 2;
    for (int i = threadIdx.x; i < rows * q; i += blockDim.x) {
      const int r = i / q, e = (i - r * q) << 2;
      const float* src = (r == 0 ? phik : ykc0 + (int64_t)(r - 1) * plane) + row0 + e;
      cp16(dst + r * pitch + e, src);
    }
  } else {
    for (int i = threadIdx.x; i < rows * W; i += blockDim.x) {
      const int r = i / W, e = i - r * W;
      const float* src = (r == 0 ? phik : ykc0 + (int64_t)(r - 1) * plane) + row0 + e;
      cp4(dst + r * pitch + e, src);
    }
  }
}

// ---- row pass + combine: one CTA per row y, warp w filters quantity c0 + w
template <int LS>
__global__ void __launch_bounds__(LS <= 31 ? 512 : 256) k_iir_rows(const __grid_constant__ IirArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int y = blockIdx.x;
  const int W = a.W, n = a.n, planes = a.state->planes;
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pitch = (W + 3) & ~3;
  const int stage_floats = (nw + 1) * pitch;           // phi row + one Y row per warp
  const int Ls = a.row.Ls, base = lane * Ls, len = min(Ls, W - base);
  const bool vec = (W & 3) == 0;
  const int64_t row0 = (int64_t)y * W;
  const bool fused = a.out != nullptr;
  for (int c0 = 0; c0 <= n; c0 += nw) {
    const int c = c0 + warp;
    const int nact = min(nw, n + 1 - c0);
    float acc[LS];
#pragma unroll
    for (int j = 0; j < LS; ++j) acc[j] = 0.f;
    auto issue = [&](int k, int s) {
      stage_rows(sm + s * stage_floats, pitch, a.phi + (int64_t)k * a.N,
                 a.Y + ((int64_t)k * (n + 1) + c0) * a.N, a.N, nact, row0, W, vec);
    };
    if (planes > 0) issue(0, 0);
    cp_commit();
    for (int k = 0; k < planes; ++k) {
      if (k + 1 < planes) issue(k + 1, (k + 1) & 1);
      cp_commit();
      cp_wait1();
      __syncthreads();
      if (warp < nact) {
        const float* P = sm + (k & 1) * stage_floats;
        const float* Yr = P + (1 + warp) * pitch;
        float v[LS];
#pragma unroll
        for (int j = 0; j < LS; ++j) v[j] = j < len ? Yr[base + j] : 0.f;
        iir_line<LS>(v, len, lane, a.row);
#pragma unroll
        for (int j = 0; j < LS; ++j)
          if (j < len) acc[j] = fmaf(P[base + j], v[j], acc[j]);
      }
      __syncthreads();
    }
    if (warp < nact && c == n) {            // eta
      unsigned small = 0;
#pragma unroll
      for (int j = 0; j < LS; ++j)
        if (j < len) {
          a.eta[row0 + base + j] = acc[j];
          if (fused) sm[base + j] = acc[j];
          small += !(acc[j] > a.eta_thr);
        }
      small = __reduce_add_sync(0xffffffffu, small);
      if (lane == 0 && small) atomicAdd(&a.state_rw->eta_small, (unsigned long long)small);
    }
    if (fused) {                            // one round: every quantity is in this CTA
      __syncthreads();
      float* ost = sm + pitch;              // W x n interleaved output row
      if (warp < n) {
#pragma unroll
        for (int j = 0; j < LS; ++j)
          if (j < len) ost[(base + j) * n + c] = acc[j] / sm[base + j];
      }
      __syncthreads();
      float* dst = a.out + row0 * n;
      for (int i = threadIdx.x; i < W * n; i += blockDim.x) dst[i] = ost[i];
    } else if (warp < nact && c < n) {
#pragma unroll
      for (int j = 0; j < LS; ++j)
        if (j < len) a.zeta[(row0 + base + j) * n + c] = acc[j];
    }
    __syncthreads();
  }
}

__global__ void k_iir_divide(const float* __restrict__ zeta, const float* __restrict__ eta, int64_t N,
                             int n, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N * n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = zeta[i] / eta[i / n];
}

// ---- host: coefficients (FP64) and scan matrices
struct Coef64 {
  double B, c1, c2, c3;
};

// Young & van Vliet's coefficients for standard deviation s >= 0.5.
Coef64 yvv(double s) {
  const double q = s >= 2.5 ? 0.98711 * s - 0.96330 : 3.97156 - 4.14554 * sqrt(1.0 - 0.26891 * s);
  const double q2 = q * q, q3 = q2 * q;
  const double b0 = 1.57825 + 2.44413 * q + 1.4281 * q2 + 0.422205 * q3;
  const double b1 = 2.44413 * q + 2.85619 * q2 + 1.26661 * q3;
  const double b2 = -(1.4281 * q2 + 1.26661 * q3);
  const double b3 = 0.422205 * q3;
  Coef64 k;
  k.c1 = b1 / b0;
  k.c2 = b2 / b0;
  k.c3 = b3 / b0;
  k.B = 1.0 - (b1 + b2 + b3) / b0;
  return k;
}

void mat3_mul(const double* a, const double* b, double* c) {
  double t[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) t[i * 3 + j] = a[i * 3] * b[j] + a[i * 3 + 1] * b[3 + j] + a[i * 3 + 2] * b[6 + j];
  for (int i = 0; i < 9; ++i) c[i] = t[i];
}

void mat3_pow(const double* M, long long e, double* out) {
  double base[9], r[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  for (int i = 0; i < 9; ++i) base[i] = M[i];
  while (e > 0) {
    if (e & 1) mat3_mul(r, base, r);
    mat3_mul(base, base, base);
    e >>= 1;
  }
  for (int i = 0; i < 9; ++i) out[i] = r[i];
}

// Rm: the anticausal pass over the zero padding after the line,
//   y[L + i] = B sum_{m >= 0} a[m] w[L + i + m],  i = 0, 1, 2,
// with w the causal recursion continued through zeros from the end state and a
// the impulse response of the anticausal recursion; summed forwards until the
// continued state has decayed below 1e-20 of its start.
void right_boundary(const Coef64& k, double* Rm) {
  for (int i = 0; i < 3; ++i) {
    double w1 = i == 0, w2 = i == 1, w3 = i == 2;   // (w[L-1], w[L-2], w[L-3])
    double a0 = 1.0, a1 = 0.0, a2 = 0.0;            // a[t], a[t-1], a[t-2]
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (long long t = 0; t < 400000000LL; ++t) {
      const double w = k.c1 * w1 + k.c2 * w2 + k.c3 * w3;   // w[L + t]
      w3 = w2;
      w2 = w1;
      w1 = w;
      s0 += a0 * w;
      s1 += a1 * w;
      s2 += a2 * w;
      const double an = k.c1 * a0 + k.c2 * a1 + k.c3 * a2;
      a2 = a1;
      a1 = a0;
      a0 = an;
      if (fabs(w1) + fabs(w2) + fabs(w3) < 1e-20) break;
    }
    Rm[0 * 3 + i] = k.B * s0;
    Rm[1 * 3 + i] = k.B * s1;
    Rm[2 * 3 + i] = k.B * s2;
  }
}

int segment_length(int len) {
  int Ls = (len + 31) / 32;
  return Ls | 1;
}

int lanes_template(int Ls) { return Ls <= 15 ? 15 : Ls <= 31 ? 31 : Ls <= 47 ? 47 : Ls <= 63 ? 63 : -1; }

IirLine make_line(double sigma, int len) {
  const Coef64 k = yvv(sigma);
  IirLine L;
  // FP32 parameters of the difference form; every matrix below is computed in
  // FP64 from these rounded values, so the scans match the recursion that runs
  L.B = (float)k.B;
  L.nB = -L.B;
  L.g1 = (float)(-(k.c2 + k.c3) - k.B);
  L.ne2 = (float)(-k.c3);
  const double B = L.B, e1 = -((double)L.g1 + B), e2 = -(double)L.ne2;
  const Coef64 kf{B, 1.0 - B - e1, e1 - e2, e2};            // the same filter, classic form
  L.len = len;
  L.Ls = segment_length(len);
  L.last = (len - 1) / L.Ls;
  L.pad = 0;
  const double T[9] = {1.0 - B, -e1, -e2, -B, -e1, -e2, 0.0, 1.0, 0.0};
  double m[9];
  for (int d = 0; d < 5; ++d) {
    mat3_pow(T, (long long)L.Ls << d, m);
    for (int i = 0; i < 9; ++i) L.P[d][i] = (float)m[i];
  }
  mat3_pow(T, len - L.last * L.Ls, m);
  for (int i = 0; i < 9; ++i) L.Plast[i] = (float)m[i];
  // boundary map in the classic basis (values at i, i+1, i+2), then S Rm S^-1
  // with S (a, b, c) = (a, a - b, b - c)
  double Rc[9], t[9];
  right_boundary(kf, Rc);
  const double S[9] = {1, 0, 0, 1, -1, 0, 0, 1, -1};
  const double Si[9] = {1, 0, 0, 1, -1, 0, 1, -1, -1};
  mat3_mul(Rc, Si, t);
  mat3_mul(S, t, m);
  for (int i = 0; i < 9; ++i) L.Rm[i] = (float)m[i];
  return L;
}

template <int LSC>
cudaError_t launch_cols(const IirArgs& a, int K, cudaStream_t st) {
  const size_t smem = sizeof(float) * (size_t)a.H * (kColWarps + 1);
  cudaError_t e = cudaFuncSetAttribute(k_iir_cols<LSC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)ceil_div(a.W, kColWarps), (unsigned)K);
  k_iir_cols<LSC><<<grid, kColWarps * 32, smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <int LSR>
cudaError_t launch_rows(const IirArgs& a, int nw, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_iir_rows<LSR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_iir_rows<LSR><<<a.H, nw * 32, smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

// Largest number of quantity warps per CTA of the row pass for segment template LS.
int row_warps_max(int LS) { return LS <= 31 ? 16 : 8; }

}  // namespace

bool iir_supported(int H, int W, int n) {
  (void)n;
  return lanes_template(segment_length(H)) > 0 && lanes_template(segment_length(W)) > 0;
}

size_t iir_workspace_floats(int64_t N, int K, int n) { return (size_t)K * (n + 1) * (size_t)N; }

cudaError_t launch_iir_combine(const float* f, int H, int W, int n, const float* phi, int K,
                               float sigma_s, DevState* state, float* out, float* eta_out,
                               float* zeta_ws, float* ybuf, cudaStream_t st) {
  const int lsc = lanes_template(segment_length(H)), lsr = lanes_template(segment_length(W));
  if (lsc < 0 || lsr < 0) return cudaErrorInvalidValue;
  IirArgs a;
  a.f = f;
  a.phi = phi;
  a.Y = ybuf;
  a.eta = eta_out;
  a.zeta = zeta_ws;
  a.state = state;
  a.state_rw = state;
  a.H = H;
  a.W = W;
  a.n = n;
  a.N = (int64_t)H * W;
  a.eta_thr = 1e-6f;                       // the recursive filter has unit DC gain: sum omega = 1
  a.col = make_line(sigma_s, H);
  a.row = make_line(sigma_s, W);
  const int pitch = (W + 3) & ~3;
  int nw = std::min(n + 1, row_warps_max(lsr));
  while (nw > 1 && sizeof(float) * 2 * (size_t)(nw + 1) * pitch > 200 * 1024) --nw;
  const size_t row_smem = sizeof(float) * 2 * (size_t)(nw + 1) * pitch;
  if (row_smem > 227 * 1024) return cudaErrorInvalidValue;
  const bool fused = nw >= n + 1;
  a.out = fused ? out : nullptr;
  cudaError_t e;
  switch (lsc) {
    case 15: e = launch_cols<15>(a, K, st); break;
    case 31: e = launch_cols<31>(a, K, st); break;
    case 47: e = launch_cols<47>(a, K, st); break;
    default: e = launch_cols<63>(a, K, st); break;
  }
  if (e != cudaSuccess) return e;
  switch (lsr) {
    case 15: e = launch_rows<15>(a, nw, row_smem, st); break;
    case 31: e = launch_rows<31>(a, nw, row_smem, st); break;
    case 47: e = launch_rows<47>(a, nw, row_smem, st); break;
    default: e = launch_rows<63>(a, nw, row_smem, st); break;
  }
  if (e != cudaSuccess || fused) return e;
  int64_t g = (a.N * n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_iir_divide<<<(int)g, 256, 0, st>>>(zeta_ws, eta_out, a.N, n, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace nyf

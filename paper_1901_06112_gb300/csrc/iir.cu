// Host side of the recursive O(1) Gaussian (Young & van Vliet 1995) for the
// spatial convolutions of Eqs. (14)-(15) (Sec. IV): coefficients and scan
// matrices in FP64, the workspace shape and the launches (the kernels and the
// scheme are described in iir_impl.cuh).
#include <math.h>

#include <algorithm>

#include "iir_impl.cuh"

namespace nyf {
namespace {

using iir::Args;
using iir::Line;

__global__ void k_iir_divide(const float* __restrict__ zeta, const float* __restrict__ eta, int64_t N,
                             int n, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N * n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = zeta[i] / eta[i / n];
}

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

// Anticausal pass over the zero padding after position L - 1 (classic basis):
//   y[L + i] = B sum_{m >= 0} a[m] w[L + i + m],  i = 0, 1, 2,
// with w the causal recursion continued through zeros from (w[L-1], w[L-2],
// w[L-3]) and a the impulse response of the anticausal recursion; summed
// forwards until the continued state has decayed below 1e-20 of its start.
void right_boundary(const Coef64& k, double* Rm) {
  for (int i = 0; i < 3; ++i) {
    double w1 = i == 0, w2 = i == 1, w3 = i == 2;
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

// Values per lane for a line of `len`: the smallest LS = 4 j + 3 with 32 LS >= len.
int lane_values(int len) {
  int LS = 3;
  while (32 * LS < len) LS += 4;
  return LS <= 63 ? LS : -1;
}

Line make_line(double sigma, int len) {
  const Coef64 k = yvv(sigma);
  Line L;
  // FP32 parameters of the difference form; every matrix below is computed in
  // FP64 from these rounded values, so the scans match the recursion that runs
  L.B = (float)k.B;
  L.nB = -L.B;
  L.g1 = (float)(-(k.c2 + k.c3) - k.B);
  L.ne2 = (float)(-k.c3);
  const double B = L.B, e1 = -((double)L.g1 + B), e2 = -(double)L.ne2;
  const Coef64 kf{B, 1.0 - B - e1, e1 - e2, e2};            // the same filter, classic form
  L.len = len;
  L.LS = lane_values(len);
  L.pad0 = L.pad1 = 0;
  const double T[9] = {1.0 - B, -e1, -e2, -B, -e1, -e2, 0.0, 1.0, 0.0};
  double m[9];
  for (int d = 0; d < 5; ++d) {
    mat3_pow(T, (long long)L.LS << d, m);
    for (int i = 0; i < 9; ++i) L.P[d][i] = (float)m[i];
  }
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

}  // namespace

}  // namespace nyf

// Diagnostic: the host-computed parameters of one line direction (no GPU work).
extern "C" nyf_status nyf_iir_line_params(double sigma_s, int len, float* out, int out_len) {
  using namespace nyf;
  if (!out || out_len < 60 || !(sigma_s >= 0.5) || !(sigma_s <= 1e4) || len < 1) return NYF_ERR_INVALID_ARG;
  if (lane_values(len) < 0) return NYF_ERR_UNSUPPORTED;
  const Line L = make_line(sigma_s, len);
  out[0] = L.B;
  out[1] = L.nB;
  out[2] = L.g1;
  out[3] = L.ne2;
  out[4] = (float)L.LS;
  out[5] = (float)L.len;
  for (int d = 0; d < 5; ++d)
    for (int i = 0; i < 9; ++i) out[6 + 9 * d + i] = L.P[d][i];
  for (int i = 0; i < 9; ++i) out[51 + i] = L.Rm[i];
  return NYF_OK;
}

namespace nyf {

bool iir_supported(int H, int W, int n) {
  (void)n;
  return lane_values(H) > 0 && lane_values(W) > 0;
}

cudaError_t launch_iir_combine(const float* f, int H, int W, int n, const float* phi, int K,
                               float sigma_s, DevState* state, float* out, float* eta_out,
                               float* zeta_ws, float* ybuf, cudaStream_t st) {
  if (!iir_supported(H, W, n)) return cudaErrorInvalidValue;
  Args a;
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
  const int lsr = a.row.LS;
  int nw = std::min(n + 1, iir::row_warps_max(lsr));
  while (nw > 1 && iir::rows_smem(lsr, nw) > 200 * 1024) --nw;
  if (iir::rows_smem(lsr, nw) > 227 * 1024) return cudaErrorInvalidValue;
  const bool fused = nw >= n + 1;
  a.out = fused ? out : nullptr;
  cudaError_t e = a.col.LS <= 31 ? iir::dispatch_cols_3_31(a.col.LS, a, K, st)
                                 : iir::dispatch_cols_35_63(a.col.LS, a, K, st);
  if (e != cudaSuccess) return e;
  e = lsr <= 31 ? iir::dispatch_rows_3_31(lsr, a, nw, st) : iir::dispatch_rows_35_63(lsr, a, nw, st);
  if (e != cudaSuccess || fused) return e;
  int64_t g = (a.N * n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_iir_divide<<<(int)g, 256, 0, st>>>(zeta_ws, eta_out, a.N, n, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace nyf

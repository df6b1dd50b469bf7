// The C ABI of libnyf (include/nyf.h): argument checks, workspace layout and
// the order of the stages of Algorithm 1.  Everything is enqueued on the
// caller's stream; nothing here allocates device memory or synchronises
// (except nyf_get_stats).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "nyf_internal.cuh"

namespace nyf {

static std::atomic<long long> g_launches{0};
void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

WsLayout ws_layout(const WsShape& s) {
  WsLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  const size_t K = (size_t)s.K, rho = (size_t)s.rho, N = (size_t)s.N, Ns = (size_t)s.Ns;
  L.state = take(sizeof(DevState));
  L.landmarks = take(sizeof(float) * K * rho);
  L.what = take(sizeof(float) * K * K);
  L.eig = take(eig_scratch_bytes());
  L.init_idx = take(sizeof(int64_t) * K);
  L.km_part = take(sizeof(float) * (size_t)kKmeansBlocks * K * (rho + 1));
  L.km_qpart = take(sizeof(float) * (size_t)kKmeansBlocks);
  const bool gather = s.gather || Ns < N;
  L.sample_idx = take(sizeof(int64_t) * (gather ? Ns : 0));
  L.sample_x = take(sizeof(float) * (gather ? Ns * rho : 0));
  L.phi = take((s.bf16 ? 2 : 4) * K * N);
  L.eta = take(sizeof(float) * N);
  L.zeta = take(sizeof(float) * N * (size_t)s.n);
  // backward only: dL/dphi, reduction partials, G_W / Z / row dots, the adjoint
  // planes a_q and the forward's convolved planes C_kq
  const size_t nq1 = (size_t)s.n + 1;
  L.dphi = take(s.bwd ? sizeof(float) * K * N * (size_t)(s.dphi_slices > 1 ? s.dphi_slices : 1) : 0);
  L.gpart = take(s.bwd ? sizeof(float) * backward_gpart_floats(s.K) : 0);
  L.spart = take(s.bwd ? sizeof(float) * backward_spart_floats(s.H, s.W, s.n) : 0);
  L.gw = take(s.bwd ? sizeof(double) * (3 * K * K + K) : 0);   // G_W, Z, row dots, A o D2
  L.adj = take(s.bwd ? sizeof(float) * nq1 * N : 0);
  const size_t kc = s.recompute ? std::min(K, (size_t)kRecomputeModes) : K;
  L.cbuf = take(s.bwd ? sizeof(float) * kc * nq1 * N : 0);
  L.ybuf = take(s.iir ? sizeof(float) * K * nq1 * N : 0);
  L.total = o;
  return L;
}

}  // namespace nyf

using namespace nyf;

namespace {

// ---- per-stage CUDA-event timing (instrumentation only)
constexpr int kStages = 7;
std::atomic<int> g_timing{0};
std::mutex g_timing_mu;
bool g_events_ready = false;
cudaEvent_t g_ev[kStages][2];
int g_ran[kStages];

struct Stage {
  cudaStream_t st;
  int id;
  bool on;
  Stage(cudaStream_t s, int i, bool timed = true)
      : st(s), id(i), on(timed && g_timing.load() != 0 && g_events_ready) {
    if (on) cudaEventRecord(g_ev[id][0], st);
  }
  ~Stage() {
    if (on) {
      cudaEventRecord(g_ev[id][1], st);
      g_ran[id] = 1;
    }
  }
};

void timing_begin(int first, int last) {
  if (!g_timing.load() || !g_events_ready) return;
  for (int i = first; i <= last; ++i) g_ran[i] = 0;
}

int window_radius(const nyf_params* p) {
  if (p->S > 0) return p->S;
  return (int)ceil(3.0 * (double)p->sigma_s);
}

int64_t subsample_rows(int64_t N, float frac) {
  int64_t v = (int64_t)floor((double)frac * (double)N + 0.5);
  if (v < 1) v = 1;
  if (v > N) v = N;
  return v;
}

int resolve_tile(const nyf_params* p) {
  if (p->conv_tile == NYF_TILE_AUTO)
    return p->precision == NYF_BF16 ? NYF_TILE_TENSOR : NYF_TILE_WIDE;
  return p->conv_tile;
}

nyf_status check_params(const nyf_params* p, int n) {
  if (!p) return NYF_ERR_INVALID_ARG;
  if (!(p->sigma_r > 0.f) || !isfinite(p->sigma_r)) return NYF_ERR_INVALID_ARG;
  if (p->K < 1 || p->K > NYF_MAX_K) return NYF_ERR_INVALID_ARG;
  if (p->kmeans_iters < 0) return NYF_ERR_INVALID_ARG;
  if (!(p->eig_rel_tol >= 0.0) || !isfinite(p->eig_rel_tol)) return NYF_ERR_INVALID_ARG;
  if (p->precision != NYF_FP32 && p->precision != NYF_BF16) return NYF_ERR_INVALID_ARG;
  if (p->spatial != NYF_GAUSSIAN && p->spatial != NYF_BOX && p->spatial != NYF_GAUSSIAN_IIR)
    return NYF_ERR_INVALID_ARG;
  if (p->spatial == NYF_GAUSSIAN && (!(p->sigma_s > 0.f) || !isfinite(p->sigma_s)))
    return NYF_ERR_INVALID_ARG;
  if (p->spatial == NYF_GAUSSIAN_IIR) {
    if (!(p->sigma_s >= 0.5f) || !isfinite(p->sigma_s)) return NYF_ERR_INVALID_ARG;
    if (p->sigma_s > 1e4f || p->precision != NYF_FP32 || p->save_for_backward)
      return NYF_ERR_UNSUPPORTED;
  }
  if (p->spatial == NYF_BOX && p->S <= 0 && (!(p->sigma_s > 0.f) || !isfinite(p->sigma_s)))
    return NYF_ERR_INVALID_ARG;
  if (!(p->sample_frac > 0.f) || p->sample_frac > 1.f) return NYF_ERR_INVALID_ARG;
  if (n < 1 || n > NYF_MAX_CHANNELS) return NYF_ERR_INVALID_ARG;
  if (p->patch_radius < 0) return NYF_ERR_INVALID_ARG;
  if (p->conv_tile < NYF_TILE_AUTO || p->conv_tile > NYF_TILE_TENSOR) return NYF_ERR_INVALID_ARG;
  if (p->save_for_backward < NYF_SAVE_NONE || p->save_for_backward > NYF_SAVE_RECOMPUTE)
    return NYF_ERR_INVALID_ARG;
  if (p->spatial == NYF_GAUSSIAN_IIR) return NYF_OK;   // no window radius
  const int S = window_radius(p);
  if (S < 1) return NYF_ERR_INVALID_ARG;
  if (S > NYF_MAX_S) return NYF_ERR_UNSUPPORTED;
  return NYF_OK;
}

bool ws_ok(const void* ws, size_t have, size_t need) {
  return ws && (reinterpret_cast<uintptr_t>(ws) & 255) == 0 && have >= need;
}

#define NYF_TRY(expr)                                   \
  do {                                                  \
    cudaError_t _e = (expr);                            \
    if (_e != cudaSuccess) return NYF_ERR_CUDA;         \
  } while (0)

bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3) == 0; }

int nlm_rho(int n, int r) { return (2 * r + 1) * (2 * r + 1) * n; }

// Shared argument checks of the filter entry points.
nyf_status check_filter(const float* f, int H, int W, int n, int rho, const nyf_params* p,
                        const float* out) {
  nyf_status s = check_params(p, n);
  if (s != NYF_OK) return s;
  if (!f || !out || !aligned4(f) || !aligned4(out)) return NYF_ERR_INVALID_ARG;
  if (H < 1 || W < 1 || (int64_t)H * W > ((int64_t)1 << 31)) return NYF_ERR_INVALID_ARG;
  if (rho < 1 || rho > NYF_MAX_RHO) return NYF_ERR_INVALID_ARG;
  if (kmeans_smem_bytes(p->K, rho) > 227 * 1024) return NYF_ERR_UNSUPPORTED;
  if (p->spatial == NYF_GAUSSIAN_IIR && !iir_supported(H, W, n)) return NYF_ERR_UNSUPPORTED;
  return NYF_OK;
}

WsShape shape_for(int H, int W, int n, int rho, const nyf_params* p) {
  WsShape s;
  s.H = H;
  s.W = W;
  s.N = (int64_t)H * W;
  s.n = n;
  s.rho = rho;
  s.K = p->K;
  s.Ns = subsample_rows(s.N, p->sample_frac);
  s.bf16 = false;   // the filters keep phi in float32 (see nyf_params.precision)
  s.gather = p->patch_radius > 0;
  s.bwd = p->save_for_backward != NYF_SAVE_NONE && p->patch_radius == 0;
  s.recompute = p->save_for_backward == NYF_SAVE_RECOMPUTE;
  s.iir = p->spatial == NYF_GAUSSIAN_IIR;
  const int Sc = conv_compiled_radius(window_radius(p));
  s.dphi_slices = (s.bwd && Sc > 0) ? bwd_dphi_slices(Sc, n) : 1;
  return s;
}

// Spatial convolutions + combine (Eqs. (14)-(15)): the recursive Gaussian or the FIR window.
cudaError_t spatial_combine(const float* f, int H, int W, int n, const nyf_params* p, int tile,
                            char* w, const WsLayout& L, float* out, float* cout, cudaStream_t st) {
  DevState* state = reinterpret_cast<DevState*>(w + L.state);
  if (p->spatial == NYF_GAUSSIAN_IIR)
    return launch_iir_combine(f, H, W, n, reinterpret_cast<const float*>(w + L.phi), p->K,
                              p->sigma_s, state, out, reinterpret_cast<float*>(w + L.eta),
                              reinterpret_cast<float*>(w + L.zeta),
                              reinterpret_cast<float*>(w + L.ybuf), st);
  return launch_conv_combine(f, H, W, n, w + L.phi, false, tile, p->spatial, p->sigma_s,
                             window_radius(p), state, out, reinterpret_cast<float*>(w + L.eta),
                             reinterpret_cast<float*>(w + L.zeta), cout, st);
}

// Landmarks into ws: copied, or k-means on the rows X (N x rho).
nyf_status stage_landmarks(const float* X_full, int64_t N, int rho, const nyf_params* p,
                           const float* landmarks, char* w, const WsLayout& L, bool nlm,
                           const float* f, int H, int W, int n, cudaStream_t st) {
  DevState* state = reinterpret_cast<DevState*>(w + L.state);
  float* lm = reinterpret_cast<float*>(w + L.landmarks);
  if (landmarks) {
    NYF_TRY(cudaMemcpyAsync(lm, landmarks, sizeof(float) * p->K * rho, cudaMemcpyDeviceToDevice, st));
    return NYF_OK;
  }
  const int64_t Ns = subsample_rows(N, p->sample_frac);
  if (p->K > Ns) return NYF_ERR_INVALID_ARG;
  const float* X = X_full;
  if (nlm) {
    NYF_TRY(launch_nlm_sample(f, H, W, n, p->patch_radius, Ns, p->seed,
                              reinterpret_cast<int64_t*>(w + L.sample_idx),
                              reinterpret_cast<float*>(w + L.sample_x), st));
    X = reinterpret_cast<const float*>(w + L.sample_x);
  } else if (Ns < N) {
    NYF_TRY(launch_sample_rows(X_full, N, rho, Ns, p->seed,
                               reinterpret_cast<int64_t*>(w + L.sample_idx),
                               reinterpret_cast<float*>(w + L.sample_x), st));
    X = reinterpret_cast<const float*>(w + L.sample_x);
  }
  NYF_TRY(launch_draw_init(X, Ns, rho, p->K, p->seed, nullptr,
                           reinterpret_cast<int64_t*>(w + L.init_idx), lm, state, st));
  NYF_TRY(launch_kmeans(X, Ns, rho, p->K, p->kmeans_iters, lm, nullptr, nullptr,
                        reinterpret_cast<float*>(w + L.km_part),
                        reinterpret_cast<float*>(w + L.km_qpart), state, st));
  return NYF_OK;
}

}  // namespace

namespace {

// Forward of one image in parts, so that the batched path can run the
// landmark and eigendecomposition steps of all its images in shared launches:
// fwd_prepare (checks, no launch), fwd_reset, the landmarks (stage_landmarks),
// launch_eig, then fwd_finish (features and the convolutions + combine).
struct FwdCtx {
  const float* f;
  const float* guide;
  int H, W, n, rho;
  const nyf_params* p;
  float* out;
  char* w;
  WsLayout L;
  DevState* state;
  int64_t N;
};

nyf_status fwd_prepare(const float* f, const float* guide, int H, int W, int n, int rho,
                       const nyf_params* p, float* out, void* ws, size_t ws_bytes, FwdCtx* c) {
  if (!p || p->patch_radius != 0) return NYF_ERR_INVALID_ARG;
  if (!guide) {
    if (rho != n) return NYF_ERR_INVALID_ARG;
    guide = f;
  }
  nyf_status s = check_filter(f, H, W, n, rho, p, out);
  if (s != NYF_OK) return s;
  if (!aligned4(guide)) return NYF_ERR_INVALID_ARG;
  c->L = ws_layout(shape_for(H, W, n, rho, p));
  if (!ws_ok(ws, ws_bytes, c->L.total)) return NYF_ERR_WORKSPACE;
  c->f = f;
  c->guide = guide;
  c->H = H;
  c->W = W;
  c->n = n;
  c->rho = rho;
  c->p = p;
  c->out = out;
  c->w = reinterpret_cast<char*>(ws);
  c->state = reinterpret_cast<DevState*>(c->w + c->L.state);
  c->N = (int64_t)H * W;
  return NYF_OK;
}

nyf_status fwd_reset(const FwdCtx& c, const int* pre_status, cudaStream_t st) {
  NYF_TRY(cudaMemsetAsync(c.state, 0, sizeof(DevState), st));
  if (pre_status)   // status of work done for this call before the filter (PCA guide)
    NYF_TRY(cudaMemcpyAsync(&c.state->status, pre_status, sizeof(int), cudaMemcpyDeviceToDevice, st));
  return NYF_OK;
}

nyf_status fwd_finish(const FwdCtx& c, cudaStream_t st, bool timed) {
  const nyf_params* p = c.p;
  const float* lm = reinterpret_cast<const float*>(c.w + c.L.landmarks);
  const float* what = reinterpret_cast<const float*>(c.w + c.L.what);
  void* phi = c.w + c.L.phi;
  {
    Stage t(st, 2, timed);
    NYF_TRY(launch_features(c.guide, c.N, c.rho, lm, p->K, p->sigma_r, what, c.state, phi, false, st));
  }
  {
    Stage t(st, 3, timed);
    NYF_TRY(spatial_combine(c.f, c.H, c.W, c.n, p, resolve_tile(p), c.w, c.L, c.out,
                            p->save_for_backward == NYF_SAVE_PLANES
                                ? reinterpret_cast<float*>(c.w + c.L.cbuf) : nullptr, st));
  }
  return NYF_OK;
}

nyf_status blf_impl(const float* f, const float* guide, int H, int W, int n, int rho,
                    const nyf_params* p, const float* landmarks, float* out, void* ws,
                    size_t ws_bytes, void* stream, bool timed, const int* pre_status = nullptr) {
  FwdCtx c;
  nyf_status s = fwd_prepare(f, guide, H, W, n, rho, p, out, ws, ws_bytes, &c);
  if (s != NYF_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if ((s = fwd_reset(c, pre_status, st)) != NYF_OK) return s;
  if (timed) timing_begin(0, 3);
  {
    Stage t(st, 0, timed);
    s = stage_landmarks(c.guide, c.N, rho, p, landmarks, c.w, c.L, false, f, H, W, n, st);
  }
  if (s != NYF_OK) return s;
  {
    Stage t(st, 1, timed);
    NYF_TRY(launch_eig(reinterpret_cast<const float*>(c.w + c.L.landmarks), p->K, rho, p->sigma_r,
                       p->eig_rel_tol, reinterpret_cast<float*>(c.w + c.L.what), nullptr, nullptr,
                       c.state, c.w + c.L.eig, st));
  }
  return fwd_finish(c, st, timed);
}

nyf_status blf_backward_impl(const float* f, const float* guide, int H, int W, int n, int rho,
                             const nyf_params* p, const float* out, const float* grad_out,
                             float* grad_f, float* grad_guide, float* grad_sigma, void* ws,
                             size_t ws_bytes, void* stream, bool timed) {
  if (!p || p->patch_radius != 0 || !p->save_for_backward) return NYF_ERR_INVALID_ARG;
  const bool tied = guide == nullptr || guide == f;
  if (tied) {
    if (rho != n) return NYF_ERR_INVALID_ARG;
    guide = f;
  }
  nyf_status s = check_filter(f, H, W, n, rho, p, out);
  if (s != NYF_OK) return s;
  if (!grad_out || !grad_f || !grad_sigma || !aligned4(grad_out) || !aligned4(grad_f) ||
      !aligned4(grad_sigma) || (!tied && (!grad_guide || !aligned4(grad_guide))))
    return NYF_ERR_INVALID_ARG;
  const WsLayout L = ws_layout(shape_for(H, W, n, rho, p));
  if (!ws_ok(ws, ws_bytes, L.total)) return NYF_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = reinterpret_cast<char*>(ws);
  DevState* state = reinterpret_cast<DevState*>(w + L.state);
  const int tile = resolve_tile(p);
  const int S = window_radius(p);
  float* dphi = reinterpret_cast<float*>(w + L.dphi);
  float* spart = reinterpret_cast<float*>(w + L.spart);
  if (timed) timing_begin(4, 6);
  {
    Stage t(st, 4, timed);
    float* cbuf = reinterpret_cast<float*>(w + L.cbuf);
    // NYF_SAVE_PLANES: one pass over the saved planes.  NYF_SAVE_RECOMPUTE: chunks of
    // kRecomputeModes modes, each convolved again (C_kq) and then taken through the adjoint.
    const int chunk = p->save_for_backward == NYF_SAVE_RECOMPUTE ? kRecomputeModes : p->K;
    for (int k0 = 0; k0 < p->K; k0 += chunk) {
      if (p->save_for_backward == NYF_SAVE_RECOMPUTE)
        NYF_TRY(launch_conv_recompute(f, H, W, n, w + L.phi, false, p->spatial, p->sigma_s, S, k0,
                                      k0 + chunk, state, cbuf, st));
      NYF_TRY(launch_bwd_conv(f, H, W, n, p->K, p->spatial, p->sigma_s, S, w + L.phi, false,
                              reinterpret_cast<const float*>(w + L.eta), out, grad_out, cbuf,
                              reinterpret_cast<float*>(w + L.adj), grad_f, dphi, spart, state, st,
                              k0, k0 + chunk));
    }
  }
  {
    Stage t(st, 5, timed);
    NYF_TRY(launch_bwd_features(f, guide, H, W, n, rho, reinterpret_cast<const float*>(w + L.landmarks),
                                p->K, p->sigma_r, S, reinterpret_cast<const float*>(w + L.what),
                                dphi, grad_f, tied ? nullptr : grad_guide,
                                reinterpret_cast<float*>(w + L.gpart), spart,
                                reinterpret_cast<double*>(w + L.gw), w + L.eig, grad_sigma, state,
                                st));
  }
  return NYF_OK;
}

// ---- batched filtering: images spread over a pool of internal streams, forked
// from and joined back to the caller's stream with events (capturable).
constexpr int kPool = 8;
constexpr int kMaxDevices = 64;
struct StreamPool {
  bool ready = false;
  cudaStream_t s[kPool];
  cudaEvent_t fork;
  cudaEvent_t join[kPool];
};
StreamPool g_pools[kMaxDevices];
std::mutex g_pool_mu;

cudaError_t device_pool(StreamPool** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  StreamPool& P = g_pools[dev];
  if (!P.ready) {
    for (int i = 0; i < kPool; ++i) {
      if ((e = cudaStreamCreateWithFlags(&P.s[i], cudaStreamNonBlocking)) != cudaSuccess) return e;
      if ((e = cudaEventCreateWithFlags(&P.join[i], cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    if ((e = cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
    P.ready = true;
  }
  *out = &P;
  return cudaSuccess;
}

nyf_params item_params(const nyf_params* p, const nyf_batch_item& it) {
  nyf_params q = *p;
  q.sigma_s = it.sigma_s;
  q.sigma_r = it.sigma_r;
  if (it.conv_tile != NYF_TILE_AUTO) q.conv_tile = it.conv_tile;
  return q;
}

// Workspace offset of every image (256-byte aligned slices) and the total.
bool batch_layout(const nyf_batch_item* items, int B, int n, const nyf_params* p, size_t* offs,
                  size_t* total) {
  size_t o = 0;
  for (int b = 0; b < B; ++b) {
    const nyf_params q = item_params(p, items[b]);
    const size_t sz = nyf_workspace_size(items[b].H, items[b].W, n, n, &q);
    if (sz == 0) return false;
    if (offs) offs[b] = o;
    o = (o + sz + 255) & ~(size_t)255;
  }
  *total = o;
  return true;
}

// Longest-processing-time assignment of images to pool streams.
void assign_streams(const nyf_batch_item* items, int B, int* stream_of) {
  long long load[kPool] = {0};
  std::vector<int> order(B);
  for (int b = 0; b < B; ++b) order[b] = b;
  std::sort(order.begin(), order.end(), [&](int a, int c) {
    return (long long)items[a].H * items[a].W > (long long)items[c].H * items[c].W;
  });
  for (int b : order) {
    int best = 0;
    for (int i = 1; i < kPool; ++i)
      if (load[i] < load[best]) best = i;
    stream_of[b] = best;
    load[best] += (long long)items[b].H * items[b].W;
  }
}

// pre(offs, total, caller): work on the caller's stream before the fork (the
// stage-batched steps); per_image(b, params, ws, bytes, stream): image b on its pool stream.
template <typename Pre, typename Fn>
nyf_status run_batched(const nyf_batch_item* items, int B, int n, const nyf_params* p, void* ws,
                       size_t ws_bytes, void* stream, Pre&& pre, Fn&& per_image) {
  if (!items || B < 1 || !p) return NYF_ERR_INVALID_ARG;
  std::vector<size_t> offs(B);
  size_t total = 0;
  if (!batch_layout(items, B, n, p, offs.data(), &total)) return NYF_ERR_INVALID_ARG;
  if (!ws_ok(ws, ws_bytes, total)) return NYF_ERR_WORKSPACE;
  for (int b = 0; b < B; ++b)
    if (items[b].offset < 0 || items[b].H < 1 || items[b].W < 1) return NYF_ERR_INVALID_ARG;
  StreamPool* P = nullptr;
  if (device_pool(&P) != cudaSuccess) return NYF_ERR_CUDA;
  cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
  nyf_status status = pre(offs, total, caller);
  if (status != NYF_OK) return status;
  std::vector<int> sof(B);
  assign_streams(items, B, sof.data());
  bool used[kPool] = {false};
  for (int b = 0; b < B; ++b) used[sof[b]] = true;
  NYF_TRY(cudaEventRecord(P->fork, caller));
  for (int i = 0; i < kPool; ++i)
    if (used[i]) NYF_TRY(cudaStreamWaitEvent(P->s[i], P->fork, 0));
  for (int b = 0; b < B && status == NYF_OK; ++b) {
    const nyf_params q = item_params(p, items[b]);
    status = per_image(b, q, reinterpret_cast<char*>(ws) + offs[b], total - offs[b], P->s[sof[b]]);
  }
  // join every used stream back even after an error, so the caller's stream stays ordered
  for (int i = 0; i < kPool; ++i)
    if (used[i]) {
      if (cudaEventRecord(P->join[i], P->s[i]) != cudaSuccess) return NYF_ERR_CUDA;
      if (cudaStreamWaitEvent(caller, P->join[i], 0) != cudaSuccess) return NYF_ERR_CUDA;
    }
  return status;
}

template <typename Fn>
nyf_status run_batched(const nyf_batch_item* items, int B, int n, const nyf_params* p, void* ws,
                       size_t ws_bytes, void* stream, Fn&& per_image) {
  return run_batched(items, B, n, p, ws, ws_bytes, stream,
                     [](const std::vector<size_t>&, size_t, cudaStream_t) { return NYF_OK; },
                     per_image);
}

// Whether the batched forward runs its landmark and eigendecomposition steps as
// stage-batched launches (every image's k-means on the CUDA-core assignment
// pass over all of its rows, or landmarks given; a FIR or recursive window).
bool staged_forward(const nyf_params* p, int n, const float* landmarks) {
  return p->sample_frac >= 1.f && (landmarks || kmeans_batchable(n, p->K));
}

// Stage-batched forward: per image the checks and state reset, then the
// landmarks of all images (k-means batch or copies), the eigendecompositions of
// all images, then features + convolutions per image on the stream pool.  Every
// image runs the kernels and reduction orders of nyf_filter_blf, so the results
// are bitwise those of per-image calls.
nyf_status blf_batched_forward(const float* f, const nyf_batch_item* items, int B, int n,
                               const nyf_params* p, const float* landmarks, float* out, void* ws,
                               size_t ws_bytes, void* stream) {
  const int64_t lm_stride = (int64_t)p->K * n;
  std::vector<nyf_params> qs(B);
  std::vector<FwdCtx> ctx(B);
  auto pre = [&](const std::vector<size_t>& offs, size_t total, cudaStream_t st) -> nyf_status {
    for (int b = 0; b < B; ++b) {
      const nyf_batch_item& it = items[b];
      qs[b] = item_params(p, it);
      nyf_status s = fwd_prepare(f + it.offset, nullptr, it.H, it.W, n, n, &qs[b], out + it.offset,
                                 reinterpret_cast<char*>(ws) + offs[b], total - offs[b], &ctx[b]);
      if (s != NYF_OK) return s;
      if (p->K > ctx[b].N) return NYF_ERR_INVALID_ARG;
    }
    for (int b = 0; b < B; ++b) {
      nyf_status s = fwd_reset(ctx[b], nullptr, st);
      if (s != NYF_OK) return s;
    }
    if (landmarks) {
      for (int b = 0; b < B; ++b)
        NYF_TRY(cudaMemcpyAsync(ctx[b].w + ctx[b].L.landmarks, landmarks + b * lm_stride,
                                sizeof(float) * lm_stride, cudaMemcpyDeviceToDevice, st));
    } else {
      std::vector<KmItem> km(B);
      for (int b = 0; b < B; ++b) {
        const FwdCtx& c = ctx[b];
        km[b].X = c.guide;
        km[b].N = c.N;
        km[b].seed = qs[b].seed;
        km[b].cent = reinterpret_cast<float*>(c.w + c.L.landmarks);
        km[b].part = reinterpret_cast<float*>(c.w + c.L.km_part);
        km[b].qpart = reinterpret_cast<float*>(c.w + c.L.km_qpart);
        km[b].idx_out = reinterpret_cast<int64_t*>(c.w + c.L.init_idx);
        km[b].state = c.state;
      }
      NYF_TRY(launch_kmeans_batched(km.data(), B, n, p->K, p->kmeans_iters, st));
    }
    std::vector<EigItem> eg(B);
    for (int b = 0; b < B; ++b) {
      const FwdCtx& c = ctx[b];
      eg[b].landmarks = reinterpret_cast<const float*>(c.w + c.L.landmarks);
      eg[b].sigma_r = qs[b].sigma_r;
      eg[b].what = reinterpret_cast<float*>(c.w + c.L.what);
      eg[b].state = c.state;
      eg[b].scratch = c.w + c.L.eig;
    }
    NYF_TRY(launch_eig_batched(eg.data(), B, p->K, n, p->eig_rel_tol, st));
    return NYF_OK;
  };
  return run_batched(items, B, n, p, ws, ws_bytes, stream, pre,
                     [&](int b, const nyf_params&, void*, size_t, cudaStream_t s) {
                       return fwd_finish(ctx[b], s, false);
                     });
}

// ---- PCA-NLM: the joint-filter layout for a q-dimensional guide, then the
// guide, the PCA outputs, a device state for the eigendecomposition and its scratch.
struct PcaLayout {
  WsLayout blf;
  size_t guide, mean, basis, eig, state, scratch, total;
};

PcaLayout pca_layout(int H, int W, int n, int q, const nyf_params* p) {
  nyf_params p2 = *p;
  p2.patch_radius = 0;
  PcaLayout L;
  L.blf = ws_layout(shape_for(H, W, n, q, &p2));
  const int rho = nlm_rho(n, p->patch_radius);
  size_t o = L.blf.total;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.guide = take(sizeof(float) * (size_t)H * W * q);
  L.mean = take(sizeof(float) * rho);
  L.basis = take(sizeof(float) * (size_t)rho * q);
  L.eig = take(sizeof(float) * rho);
  L.state = take(sizeof(DevState));
  L.scratch = take(pca_scratch_bytes(n, p->patch_radius));
  L.total = o;
  return L;
}

nyf_status check_pca(int H, int W, int n, int r, int q) {
  if (H < 1 || W < 1 || n < 1 || r < 1) return NYF_ERR_INVALID_ARG;
  const int rho = nlm_rho(n, r);
  if (rho > 160 || q < 1 || q > rho || q > 32) return NYF_ERR_INVALID_ARG;
  if ((int64_t)H * W > ((int64_t)1 << 31)) return NYF_ERR_INVALID_ARG;
  if (pca_jacobi_smem(rho) > 227 * 1024) return NYF_ERR_UNSUPPORTED;
  return NYF_OK;
}

}  // namespace

extern "C" {

int nyf_version(void) { return 102; }

void nyf_set_timing(int enable) {
  std::lock_guard<std::mutex> lk(g_timing_mu);
  if (enable && !g_events_ready) {
    for (int i = 0; i < kStages; ++i) {
      cudaEventCreate(&g_ev[i][0]);
      cudaEventCreate(&g_ev[i][1]);
      g_ran[i] = 0;
    }
    g_events_ready = true;
  }
  g_timing.store(enable ? 1 : 0);
}

int nyf_get_timing(float* ms, int max_stages) {
  if (!ms || max_stages < 1) return 0;
  const int n = max_stages < kStages ? max_stages : kStages;
  for (int i = 0; i < n; ++i) {
    ms[i] = -1.f;
    if (g_events_ready && g_ran[i]) {
      float t = -1.f;
      if (cudaEventSynchronize(g_ev[i][1]) == cudaSuccess &&
          cudaEventElapsedTime(&t, g_ev[i][0], g_ev[i][1]) == cudaSuccess)
        ms[i] = t;
    }
  }
  return n;
}

long long nyf_launch_count(void) { return g_launches.load(); }

const char* nyf_status_string(nyf_status s) {
  switch (s) {
    case NYF_OK: return "ok";
    case NYF_ERR_INVALID_ARG: return "invalid argument";
    case NYF_ERR_UNSUPPORTED: return "unsupported configuration";
    case NYF_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case NYF_ERR_NUMERIC: return "numeric failure (no eigenvalue kept or non-finite data)";
    case NYF_ERR_CUDA: return "CUDA launch or copy failed";
    case NYF_ERR_TIMEOUT: return "bounded device loop reached its limit";
  }
  return "unknown status";
}

size_t nyf_workspace_size(int H, int W, int n, int rho, const nyf_params* p) {
  if (!p || H < 1 || W < 1 || n < 1 || p->K < 1 || p->K > NYF_MAX_K) return 0;
  if (p->patch_radius > 0) rho = nlm_rho(n, p->patch_radius);
  if (rho < 1 || rho > NYF_MAX_RHO) return 0;
  if (!(p->sample_frac > 0.f) || p->sample_frac > 1.f) return 0;
  return ws_layout(shape_for(H, W, n, rho, p)).total;
}

nyf_status nyf_kmeans(const float* X, int64_t N, int rho, int K, int iters, uint64_t seed,
                      const int64_t* init_idx, float* centroids, int32_t* labels, double* qerr,
                      void* ws, size_t ws_bytes, void* stream) {
  if (!X || !centroids || N < 1 || N > ((int64_t)1 << 31) || rho < 1 || rho > NYF_MAX_RHO ||
      K < 1 || K > NYF_MAX_K || K > N || iters < 0)
    return NYF_ERR_INVALID_ARG;
  if (kmeans_smem_bytes(K, rho) > 227 * 1024) return NYF_ERR_UNSUPPORTED;
  WsShape s{(int)N, 1, N, 1, rho, K, N, false, false, false, false};
  const WsLayout L = ws_layout(s);
  if (!ws_ok(ws, ws_bytes, L.km_qpart + sizeof(float) * kKmeansBlocks)) return NYF_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = reinterpret_cast<char*>(ws);
  DevState* state = reinterpret_cast<DevState*>(w + L.state);
  NYF_TRY(cudaMemsetAsync(state, 0, sizeof(DevState), st));
  NYF_TRY(launch_draw_init(X, N, rho, K, seed, init_idx, reinterpret_cast<int64_t*>(w + L.init_idx),
                           centroids, state, st));
  NYF_TRY(launch_kmeans(X, N, rho, K, iters, centroids, labels, qerr,
                        reinterpret_cast<float*>(w + L.km_part),
                        reinterpret_cast<float*>(w + L.km_qpart), state, st));
  return NYF_OK;
}

nyf_status nyf_kmeans_partials(const float* X, int64_t N, int rho, int K, const float* centroids,
                               double* sums, double* qerr, void* ws, size_t ws_bytes, void* stream) {
  if (!X || !centroids || !sums || !qerr || N < 1 || N > ((int64_t)1 << 31) || rho < 1 ||
      rho > NYF_MAX_RHO || K < 1 || K > NYF_MAX_K)
    return NYF_ERR_INVALID_ARG;
  if (kmeans_smem_bytes(K, rho) > 227 * 1024) return NYF_ERR_UNSUPPORTED;
  WsShape s{(int)N, 1, N, 1, rho, K, N, false, false, false, false};
  const WsLayout L = ws_layout(s);
  if (!ws_ok(ws, ws_bytes, L.km_qpart + sizeof(float) * kKmeansBlocks)) return NYF_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = reinterpret_cast<char*>(ws);
  DevState* state = reinterpret_cast<DevState*>(w + L.state);
  NYF_TRY(cudaMemsetAsync(state, 0, sizeof(DevState), st));
  NYF_TRY(launch_kmeans_partials(X, N, rho, K, centroids, sums, qerr,
                                 reinterpret_cast<float*>(w + L.km_part),
                                 reinterpret_cast<float*>(w + L.km_qpart), state, st));
  return NYF_OK;
}

nyf_status nyf_kmeans_apply_sums(const double* sums, int K, int rho, float* centroids, void* stream) {
  if (!sums || !centroids || K < 1 || K > NYF_MAX_K || rho < 1 || rho > NYF_MAX_RHO)
    return NYF_ERR_INVALID_ARG;
  NYF_TRY(launch_apply_sums(sums, K, rho, centroids, reinterpret_cast<cudaStream_t>(stream)));
  return NYF_OK;
}

nyf_status nyf_gather_rows(const float* X, int64_t N, int rho, int64_t row0, const int64_t* idx,
                           int K, float* out, void* stream) {
  if (!X || !idx || !out || N < 1 || rho < 1 || K < 1 || K > NYF_MAX_K || row0 < 0)
    return NYF_ERR_INVALID_ARG;
  NYF_TRY(launch_gather_rows(X, N, rho, row0, idx, K, out, reinterpret_cast<cudaStream_t>(stream)));
  return NYF_OK;
}

int nyf_draw_indices(uint64_t seed, int64_t N, int K, int64_t* out) {
  if (!out || N < 1 || K < 1 || K > NYF_MAX_K || K > N) return 0;
  int cnt = 0;
  const uint64_t max_draws = 64ull * (uint64_t)K + 4096ull;   // as the device draw
  for (uint64_t t = 1; t <= max_draws && cnt < K; ++t) {
    const int64_t c = (int64_t)(splitmix64(seed, t) % (uint64_t)N);
    bool dup = false;
    for (int q = 0; q < cnt; ++q) dup |= out[q] == c;
    if (!dup) out[cnt++] = c;
  }
  return cnt;
}

nyf_status nyf_features(const float* guide, int64_t N, int rho, const float* landmarks, int K,
                        float sigma_r, double eig_rel_tol, int precision, void* phi, int* rank,
                        double* alphas, void* ws, size_t ws_bytes, void* stream) {
  if (!guide || !landmarks || !phi || N < 1 || N > ((int64_t)1 << 31) || rho < 1 ||
      rho > NYF_MAX_RHO || K < 1 || K > NYF_MAX_K || !(sigma_r > 0.f) || !isfinite(sigma_r) ||
      !(eig_rel_tol >= 0.0) || (precision != NYF_FP32 && precision != NYF_BF16))
    return NYF_ERR_INVALID_ARG;
  if (sizeof(float) * ((size_t)K * rho + (size_t)K * K) > 227 * 1024) return NYF_ERR_UNSUPPORTED;
  WsShape s{(int)N, 1, N, 1, rho, K, N, precision == NYF_BF16, false, false, false};
  const WsLayout L = ws_layout(s);
  if (!ws_ok(ws, ws_bytes, L.eig + eig_scratch_bytes())) return NYF_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = reinterpret_cast<char*>(ws);
  DevState* state = reinterpret_cast<DevState*>(w + L.state);
  float* what = reinterpret_cast<float*>(w + L.what);
  NYF_TRY(cudaMemsetAsync(state, 0, sizeof(DevState), st));
  NYF_TRY(launch_eig(landmarks, K, rho, sigma_r, eig_rel_tol, what, alphas, rank, state, w + L.eig,
                     st));
  NYF_TRY(launch_features(guide, N, rho, landmarks, K, sigma_r, what, state, phi,
                          precision == NYF_BF16, st));
  return NYF_OK;
}

nyf_status nyf_filter_blf(const float* f, const float* guide, int H, int W, int n, int rho,
                          const nyf_params* p, const float* landmarks, float* out, void* ws,
                          size_t ws_bytes, void* stream) {
  return blf_impl(f, guide, H, W, n, rho, p, landmarks, out, ws, ws_bytes, stream, true);
}

nyf_status nyf_filter_nlm(const float* f, int H, int W, int n, const nyf_params* p,
                          const float* landmarks, float* out, void* ws, size_t ws_bytes,
                          void* stream) {
  if (!p || p->patch_radius < 0 || p->patch_radius > 8) return NYF_ERR_INVALID_ARG;
  const int rho = nlm_rho(n, p->patch_radius);
  nyf_status s = check_filter(f, H, W, n, rho, p, out);
  if (s != NYF_OK) return s;
  if (features_nlm_smem_bytes(p->K, n, p->patch_radius) > 227 * 1024) return NYF_ERR_UNSUPPORTED;
  const WsLayout L = ws_layout(shape_for(H, W, n, rho, p));
  if (!ws_ok(ws, ws_bytes, L.total)) return NYF_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = reinterpret_cast<char*>(ws);
  DevState* state = reinterpret_cast<DevState*>(w + L.state);
  const int tile = resolve_tile(p);
  NYF_TRY(cudaMemsetAsync(state, 0, sizeof(DevState), st));
  // The patch guide is never stored: k-means always clusters a gathered
  // subsample of patch vectors (all pixels when sample_frac == 1).
  const int64_t N = (int64_t)H * W;
  timing_begin(0, 3);
  {
    Stage t(st, 0);
    s = stage_landmarks(nullptr, N, rho, p, landmarks, w, L, true, f, H, W, n, st);
  }
  if (s != NYF_OK) return s;
  const float* lm = reinterpret_cast<const float*>(w + L.landmarks);
  float* what = reinterpret_cast<float*>(w + L.what);
  void* phi = w + L.phi;
  {
    Stage t(st, 1);
    NYF_TRY(launch_eig(lm, p->K, rho, p->sigma_r, p->eig_rel_tol, what, nullptr, nullptr, state,
                       w + L.eig, st));
  }
  {
    Stage t(st, 2);
    NYF_TRY(launch_features_nlm(f, H, W, n, p->patch_radius, lm, p->K, p->sigma_r, what, state,
                                phi, false, st));
  }
  {
    Stage t(st, 3);
    NYF_TRY(spatial_combine(f, H, W, n, p, tile, w, L, out, nullptr, st));
  }
  return NYF_OK;
}

nyf_status nyf_filter_blf_backward(const float* f, const float* guide, int H, int W, int n,
                                   int rho, const nyf_params* p, const float* out,
                                   const float* grad_out, float* grad_f, float* grad_guide,
                                   float* grad_sigma, void* ws, size_t ws_bytes, void* stream) {
  return blf_backward_impl(f, guide, H, W, n, rho, p, out, grad_out, grad_f, grad_guide, grad_sigma,
                           ws, ws_bytes, stream, true);
}

nyf_status nyf_get_stats(const void* ws, nyf_stats* out, void* stream) {
  if (!ws || !out) return NYF_ERR_INVALID_ARG;
  DevState h;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&h, ws, sizeof(DevState), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return NYF_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return NYF_ERR_CUDA;
  memset(out, 0, sizeof(*out));
  out->status = h.status;
  out->rank = h.rank;
  out->qerr = h.qerr;
  out->alpha_max = h.alpha[0];
  out->alpha_min_kept = h.rank > 0 ? h.alpha[h.rank - 1] : 0.0;
  out->eta_small = (long long)h.eta_small;
  out->grad_sigma_r = h.grad_sigma[0];
  out->grad_sigma_s = h.grad_sigma[1];
  return NYF_OK;
}

size_t nyf_batched_workspace_size(const nyf_batch_item* items, int B, int n,
                                  const nyf_params* p) {
  if (!items || B < 1 || !p) return 0;
  size_t total = 0;
  return batch_layout(items, B, n, p, nullptr, &total) ? total : 0;
}

size_t nyf_patch_pca_workspace_size(int n, int r) {
  if (n < 1 || r < 1 || nlm_rho(n, r) > 160) return 0;
  return align256(sizeof(DevState)) + pca_scratch_bytes(n, r);
}

nyf_status nyf_patch_pca(const float* f, int H, int W, int n, int r, int q, float* mean,
                         float* basis, float* eigvals, void* ws, size_t ws_bytes, void* stream) {
  nyf_status s = check_pca(H, W, n, r, q);
  if (s != NYF_OK) return s;
  if (!f || !mean || !basis || !eigvals || !aligned4(f)) return NYF_ERR_INVALID_ARG;
  if (!ws_ok(ws, ws_bytes, nyf_patch_pca_workspace_size(n, r))) return NYF_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = reinterpret_cast<char*>(ws);
  DevState* state = reinterpret_cast<DevState*>(w);
  NYF_TRY(cudaMemsetAsync(state, 0, sizeof(DevState), st));
  NYF_TRY(launch_patch_pca(f, H, W, n, r, q, w + align256(sizeof(DevState)), mean, basis, eigvals,
                           state, st));
  return NYF_OK;
}

nyf_status nyf_pca_project(const float* f, int H, int W, int n, int r, int q, const float* mean,
                           const float* basis, float* guide, void* stream) {
  nyf_status s = check_pca(H, W, n, r, q);
  if (s != NYF_OK) return s;
  if (!f || !mean || !basis || !guide || !aligned4(f)) return NYF_ERR_INVALID_ARG;
  NYF_TRY(launch_pca_project(f, H, W, n, r, q, mean, basis, guide,
                             reinterpret_cast<cudaStream_t>(stream)));
  return NYF_OK;
}

size_t nyf_pca_nlm_workspace_size(int H, int W, int n, int q, const nyf_params* p) {
  if (!p || check_pca(H, W, n, p->patch_radius, q) != NYF_OK || p->K < 1 || p->K > NYF_MAX_K)
    return 0;
  if (!(p->sample_frac > 0.f) || p->sample_frac > 1.f) return 0;
  return pca_layout(H, W, n, q, p).total;
}

nyf_status nyf_filter_pca_nlm(const float* f, int H, int W, int n, int q, const nyf_params* p,
                              const float* mean, const float* basis, const float* landmarks,
                              float* out, void* ws, size_t ws_bytes, void* stream) {
  if (!p || p->save_for_backward) return NYF_ERR_INVALID_ARG;
  nyf_status s = check_pca(H, W, n, p->patch_radius, q);
  if (s != NYF_OK) return s;
  if ((mean == nullptr) != (basis == nullptr)) return NYF_ERR_INVALID_ARG;
  nyf_params p2 = *p;
  p2.patch_radius = 0;
  s = check_filter(f, H, W, n, q, &p2, out);
  if (s != NYF_OK) return s;
  const PcaLayout L = pca_layout(H, W, n, q, p);
  if (!ws_ok(ws, ws_bytes, L.total)) return NYF_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = reinterpret_cast<char*>(ws);
  const int r = p->patch_radius;
  const int* pre = nullptr;
  if (!basis) {
    DevState* ps = reinterpret_cast<DevState*>(w + L.state);
    NYF_TRY(cudaMemsetAsync(ps, 0, sizeof(DevState), st));
    mean = reinterpret_cast<float*>(w + L.mean);
    basis = reinterpret_cast<float*>(w + L.basis);
    NYF_TRY(launch_patch_pca(f, H, W, n, r, q, w + L.scratch, reinterpret_cast<float*>(w + L.mean),
                             reinterpret_cast<float*>(w + L.basis), reinterpret_cast<float*>(w + L.eig),
                             ps, st));
    pre = &ps->status;
  }
  float* guide = reinterpret_cast<float*>(w + L.guide);
  NYF_TRY(launch_pca_project(f, H, W, n, r, q, mean, basis, guide, st));
  return blf_impl(f, guide, H, W, n, q, &p2, landmarks, out, ws, L.blf.total, stream, true, pre);
}

nyf_status nyf_filter_blf_batched(const float* f, const nyf_batch_item* items, int B, int n,
                                  const nyf_params* p, const float* landmarks, float* out, void* ws,
                                  size_t ws_bytes, void* stream) {
  if (!f || !out || !p || (landmarks && !aligned4(landmarks))) return NYF_ERR_INVALID_ARG;
  if (staged_forward(p, n, landmarks))
    return blf_batched_forward(f, items, B, n, p, landmarks, out, ws, ws_bytes, stream);
  const int64_t lm_stride = (int64_t)p->K * n;
  return run_batched(items, B, n, p, ws, ws_bytes, stream,
                     [&](int b, const nyf_params& q, void* wsb, size_t wsn, cudaStream_t s) {
                       const nyf_batch_item& it = items[b];
                       return blf_impl(f + it.offset, nullptr, it.H, it.W, n, n, &q,
                                       landmarks ? landmarks + b * lm_stride : nullptr,
                                       out + it.offset, wsb, wsn, s, false);
                     });
}

nyf_status nyf_filter_blf_batched_backward(const float* f, const nyf_batch_item* items, int B,
                                           int n, const nyf_params* p, const float* out,
                                           const float* grad_out, float* grad_f,
                                           float* grad_sigma, void* ws, size_t ws_bytes,
                                           void* stream) {
  if (!f || !out || !grad_out || !grad_f || !grad_sigma) return NYF_ERR_INVALID_ARG;
  return run_batched(items, B, n, p, ws, ws_bytes, stream,
                     [&](int b, const nyf_params& q, void* wsb, size_t wsn, cudaStream_t s) {
                       const nyf_batch_item& it = items[b];
                       return blf_backward_impl(f + it.offset, nullptr, it.H, it.W, n, n, &q,
                                                out + it.offset, grad_out + it.offset,
                                                grad_f + it.offset, nullptr, grad_sigma + 2 * b,
                                                wsb, wsn, s, false);
                     });
}

nyf_status nyf_batched_stats(const void* ws, const nyf_batch_item* items, int B, int n,
                             const nyf_params* p, int b, nyf_stats* out, void* stream) {
  if (!ws || !items || b < 0 || b >= B) return NYF_ERR_INVALID_ARG;
  std::vector<size_t> offs(B);
  size_t total = 0;
  if (!batch_layout(items, B, n, p, offs.data(), &total)) return NYF_ERR_INVALID_ARG;
  return nyf_get_stats(reinterpret_cast<const char*>(ws) + offs[b], out, stream);
}

}  // extern "C"

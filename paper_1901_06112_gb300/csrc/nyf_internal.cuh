// Internal declarations shared by the libnyf translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/nyf.h"

namespace nyf {

constexpr int kMaxK = NYF_MAX_K;
constexpr int kMaxRho = NYF_MAX_RHO;
constexpr int kMaxS = NYF_MAX_S;
constexpr int kMaxChannels = NYF_MAX_CHANNELS;
constexpr int kKmeansBlocks = 608;       // 4 x 152 SMs: partial-sum slots of the assign pass
constexpr int kKmeansThreads = 256;

// Device-side state at the start of every workspace.
struct DevState {
  int status;                 // sticky nyf_status
  int rank;                   // kept modes r
  int planes;                 // feature planes (K when r > 0, else 0)
  int pad0;
  unsigned long long eta_small;
  double qerr;
  double alpha[kMaxK];        // eigenvalues of A, descending
  float grad_sigma[2];
  int pad[2];
};

// Byte offsets of every region of a workspace (all 256-byte aligned).
struct WsLayout {
  size_t state, landmarks, what, eig, init_idx, km_part, km_qpart, sample_idx, sample_x, phi,
      eta, zeta, dphi, gpart, spart, gw, adj, cbuf, ybuf, total;
};

// Problem geometry used to size a workspace.
struct WsShape {
  int H, W;         // image size (H * W == N for images; N x 1 for row sets)
  int64_t N;        // pixels (rows of the guide)
  int n;            // image channels
  int rho;          // guide dimension
  int K;            // landmarks
  int64_t Ns;       // rows k-means clusters
  bool bf16;        // features stored as bfloat16
  bool gather;      // k-means rows are gathered (subsample or NLM patches)
  bool bwd;         // regions of the backward pass (saved convolutions, adjoints, partials)
  bool iir;         // recursive-Gaussian planes (omega_v * (phi_k f_c), K (n + 1) planes)
  bool recompute;   // backward recomputes C_kq: room for kRecomputeModes modes' planes only
  int dphi_slices;  // backward: dL/dphi as this many partial plane sets (1: one set)
};

WsLayout ws_layout(const WsShape& s);

__host__ __device__ inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Sticky error latch: the first error wins.
__device__ inline void set_status(DevState* st, int code) { atomicCAS(&st->status, 0, code); }

// ---- SplitMix64 (Steele, Lea & Flood 2014): output t of the stream seeded with s.
__host__ __device__ inline uint64_t splitmix64(uint64_t seed, uint64_t t) {
  uint64_t z = seed + t * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
constexpr uint64_t kSampleStream = 0xA5A5A5A5A5A5A5A5ull;

// Host-side count of kernel launches (nyf_launch_count).
void count_launches(int k);

// ---- launchers (one per kernel family); all enqueue on `st` and return a cudaError_t.
cudaError_t launch_draw_init(const float* X, int64_t N, int rho, int K, uint64_t seed,
                             const int64_t* init_idx, int64_t* idx_out, float* centroids,
                             DevState* state, cudaStream_t st);
cudaError_t launch_kmeans(const float* X, int64_t N, int rho, int K, int iters, float* centroids,
                          int32_t* labels, double* qerr_out, float* part, float* qpart,
                          DevState* state, cudaStream_t st);
cudaError_t launch_sample_rows(const float* guide, int64_t N, int rho, int64_t Ns, uint64_t seed,
                               int64_t* idx, float* X, cudaStream_t st);
size_t kmeans_smem_bytes(int K, int rho);
// Strip processing: one assignment pass's FP64 partial sums and error, the
// centroid update from (all-reduced) sums, and the gather of drawn rows.
cudaError_t launch_kmeans_partials(const float* X, int64_t N, int rho, int K, const float* cent,
                                   double* sums, double* qerr, float* part, float* qpart,
                                   DevState* state, cudaStream_t st);
cudaError_t launch_apply_sums(const double* sums, int K, int rho, float* cent, cudaStream_t st);
cudaError_t launch_gather_rows(const float* X, int64_t N, int rho, int64_t row0, const int64_t* idx,
                               int K, float* out, cudaStream_t st);
// Tensor-core (tcgen05) assignment pass for rows of dimension 16..80 (kmeans_tc.cu).
bool assign_tc_supported(int rho, int K);
int assign_tc_grid(int64_t N);
cudaError_t launch_assign_tc(int grid, const float* X, int64_t N, int rho, int K,
                             const float* cent, int32_t* labels, float* part, float* qpart,
                             int accumulate, DevState* state, cudaStream_t st);
cudaError_t launch_nlm_sample(const float* f, int H, int W, int n, int r, int64_t Ns, uint64_t seed,
                              int64_t* idx, float* X, cudaStream_t st);
cudaError_t launch_eig(const float* landmarks, int K, int rho, float sigma_r, double tau,
                       float* what, double* alphas_out, int* rank_out, DevState* state,
                       void* scratch, cudaStream_t st);
size_t eig_scratch_bytes();
// Stage-batched launches: one launch per step for a batch of independent
// problems (the images of nyf_filter_blf_batched), problem b reading and
// writing only its own buffers.  Each problem runs the code and reduction
// order of a single-problem launch, so the results are bitwise those of
// per-problem calls.  Batches above kBatchMax problems go in slices.
constexpr int kBatchMax = 64;
struct EigItem {
  const float* landmarks;
  float sigma_r;
  float* what;
  DevState* state;
  void* scratch;
};
// k-means of a batch (Algorithm 1, clustering step, per problem): the initial
// draw, `iters` Lloyd iterations and the final error pass, one launch per step.
// Only for rows on the CUDA-core assignment pass (kmeans_batchable).
struct KmItem {
  const float* X;
  int64_t N;
  uint64_t seed;
  float* cent;
  float* part;
  float* qpart;
  int64_t* idx_out;
  DevState* state;
};
bool kmeans_batchable(int rho, int K);
cudaError_t launch_kmeans_batched(const KmItem* items, int count, int rho, int K, int iters,
                                  cudaStream_t st);
cudaError_t launch_eig_batched(const EigItem* items, int count, int K, int rho, double tau,
                               cudaStream_t st);
cudaError_t launch_features(const float* guide, int64_t N, int rho, const float* landmarks, int K,
                            float sigma_r, const float* what, const DevState* state, void* phi,
                            bool bf16, cudaStream_t st);
cudaError_t launch_features_nlm(const float* f, int H, int W, int n, int r, const float* landmarks,
                                int K, float sigma_r, const float* what, const DevState* state,
                                void* phi, bool bf16, cudaStream_t st);
size_t features_nlm_smem_bytes(int K, int n, int r);
// Tensor-core (tcgen05) features for guides of dimension rho >= kFeaturesTcMinRho.
constexpr int kFeaturesTcMinRho = 16;
cudaError_t launch_features_tc(const float* guide, int64_t N, int rho, const float* landmarks,
                               int K, float sigma_r, const float* what, const DevState* state,
                               void* phi, bool bf16, cudaStream_t st);
cudaError_t launch_features_nlm_tc(const float* f, int H, int W, int n, int r,
                                   const float* landmarks, int K, float sigma_r, const float* what,
                                   const DevState* state, void* phi, bool bf16, cudaStream_t st);
size_t features_tc_smem_bytes(int rho, int K, int n, int r);
cudaError_t launch_conv_combine(const float* f, int H, int W, int n, const void* phi, bool bf16,
                                int tile, int spatial, float sigma_s, int S, DevState* state,
                                float* out, float* eta_out, float* zeta_ws, float* cout,
                                cudaStream_t st);
int conv_compiled_radius(int S);
// Partial dL/dphi plane sets of the adjoint convolution for compiled radius Sc and
// n channels: one per quantity slice when more than two CTAs share a tile (summed
// in a fixed order afterwards), else 1 (direct writes, or two commutative adds).
int bwd_dphi_slices(int Sc, int n);
bool iir_supported(int H, int W, int n);
cudaError_t launch_iir_combine(const float* f, int H, int W, int n, const float* phi, int K,
                               float sigma_s, DevState* state, float* out, float* eta_out,
                               float* zeta_ws, float* ybuf, cudaStream_t st);
bool conv_split(int S, int n);
// Adjoint convolutions of the modes k_begin <= k < k_end; cbuf holds their planes
// C_kq (plane (k - k_begin) (n + 1) + q).  The chunk with k_begin == 0 also forms the
// adjoint planes; later chunks add into grad_f and the sigma_s partials.
cudaError_t launch_bwd_conv(const float* f, int H, int W, int n, int K, int spatial, float sigma_s,
                            int S, const void* phi, bool bf16, const float* eta, const float* out,
                            const float* grad_out, const float* cbuf, float* adj, float* grad_f,
                            float* dphi, float* spart, const DevState* state, cudaStream_t st,
                            int k_begin, int k_end);
// C_kq = omega * (phi_k f_q) of the modes k_begin <= k < k_end into cout (plane
// (k - k_begin) (n + 1) + q), with the forward's FP32 kernel and nothing else written.
cudaError_t launch_conv_recompute(const float* f, int H, int W, int n, const void* phi, bool bf16,
                                  int spatial, float sigma_s, int S, int k_begin, int k_end,
                                  DevState* state, float* cout, cudaStream_t st);
constexpr int kRecomputeModes = NYF_RECOMPUTE_MODES;   // modes whose planes the recompute backward keeps at once
cudaError_t launch_bwd_features(const float* f, const float* guide, int H, int W, int n, int rho,
                                const float* landmarks, int K, float sigma_r, int S,
                                const float* what, const float* dphi, float* grad_f,
                                float* grad_guide, float* gpart, const float* spart, double* gw,
                                const void* eig_scratch, float* grad_sigma, DevState* state,
                                cudaStream_t st);
size_t pca_scratch_bytes(int n, int r);
size_t pca_jacobi_smem(int rho);
cudaError_t launch_patch_pca(const float* f, int H, int W, int n, int r, int q, void* scratch,
                             float* mean, float* basis, float* eigvals, DevState* state,
                             cudaStream_t st);
cudaError_t launch_pca_project(const float* f, int H, int W, int n, int r, int q, const float* mean,
                               const float* basis, float* guide, cudaStream_t st);
size_t backward_gpart_floats(int K);
size_t backward_spart_floats(int H, int W, int n);
const double* eig_A64(const void* scratch);

}  // namespace nyf

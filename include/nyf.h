/*
 * nyf.h -- C ABI of libnyf, the GB300 (sm_103a) Nystrom kernel filter.
 *
 * Method: P. Nair and K. N. Chaudhury, "Fast High-Dimensional Kernel
 * Filtering", arXiv 1901.06112.  The exact filter is Eq. (1); the fast filter
 * is Algorithm 1, i.e. Eqs. (9)-(12) for the Nystrom factors and
 * Eqs. (14)-(15) for the output, with k-means landmarks (Sec. III).
 *
 * Conventions shared by every entry point
 *  - Images are HWC float32, row-major, contiguous: element (y, x, c) of an
 *    H x W x C image is at index (y * W + x) * C + c.  A "guide" is an
 *    H x W x rho image (the paper's p : Omega -> R^rho).
 *  - All data pointers are DEVICE pointers owned by the caller unless stated
 *    otherwise.  The library never allocates device memory: scratch space is
 *    the caller's workspace `ws` of at least nyf_workspace_size() bytes,
 *    256-byte aligned.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call only enqueues work on it; none synchronises, except
 *    nyf_get_stats.
 *  - Argument errors are detected on the host before anything is enqueued and
 *    returned at once.  Errors found on the device while the work runs (no
 *    eigenvalue kept, a draw that did not finish) are latched into a sticky
 *    status word inside `ws` and read back with nyf_get_stats.
 *  - Range kernel kappa(t, s) = exp(-||t - s||^2 / (2 sigma_r^2)) (sigma_r is
 *    the paper's theta, Sec. IV setup).  Spatial kernel omega(z) =
 *    exp(-||z||^2 / (2 sigma_s^2)) on the window ||z||_inf <= S (S defaults to
 *    ceil(3 sigma_s), Sec. IV setup) or a box of ones; the window is clipped
 *    to the image (zero padding).  NYF_GAUSSIAN_IIR replaces the window by
 *    the recursive Gaussian of Young & van Vliet (1995), the O(1) filter the
 *    paper's experiments use (Sec. IV): a third-order causal recursion and
 *    the same recursion run backwards, along columns and then rows, applied
 *    to the zero-padded image (unit DC gain, no truncation radius).
 *  - Eq. (12) divides by the eigenvalues alpha_k of A; only modes with
 *    alpha_k > eig_rel_tol * alpha_max are used (their number is the rank r).
 */
#ifndef NYF_H
#define NYF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NYF_MAX_K 64        /* largest number of landmarks m0 */
#define NYF_MAX_RHO 160     /* largest guide dimension rho */
#define NYF_MAX_S 32        /* largest window radius S */
#define NYF_MAX_CHANNELS 64 /* largest number of image channels n */

typedef enum {
  NYF_OK = 0,
  NYF_ERR_INVALID_ARG = 1, /* a size, pointer or parameter is out of range */
  NYF_ERR_UNSUPPORTED = 2, /* valid but outside what this build implements */
  NYF_ERR_WORKSPACE = 3,   /* ws is NULL, misaligned or smaller than required */
  NYF_ERR_NUMERIC = 4,     /* device: no eigenvalue kept (rank 0) or non-finite data */
  NYF_ERR_CUDA = 5,        /* a CUDA launch or copy failed */
  NYF_ERR_TIMEOUT = 6      /* device: a bounded loop reached its limit */
} nyf_status;

typedef enum { NYF_FP32 = 0, NYF_BF16 = 1 } nyf_precision;
/* NYF_GAUSSIAN_IIR: forward only, NYF_FP32 only (the separable passes keep a
 * K (n+1)-plane float32 intermediate in the workspace), 0.5 <= sigma_s <= 1e4,
 * H and W <= 2016 (NYF_ERR_UNSUPPORTED otherwise); S and conv_tile are ignored. */
typedef enum { NYF_GAUSSIAN = 0, NYF_BOX = 1, NYF_GAUSSIAN_IIR = 2 } nyf_spatial;

/* Convolution kernel variant (nyf_params.conv_tile).  AUTO: tensor cores for
 * NYF_BF16, wide FP32 tiles otherwise.  WIDE / NARROW: FP32 FIR kernel with
 * 32 x 96 / 32 x 64 output tiles (radius <= 16; larger radii have one tile
 * shape).  TENSOR: BF16 tensor-core kernel (radius <= 16, else WIDE).  The
 * autotuner (paper_1901_06112_gb300.tune) picks one per radius by timing. */
typedef enum { NYF_TILE_AUTO = 0, NYF_TILE_WIDE = 1, NYF_TILE_NARROW = 2, NYF_TILE_TENSOR = 3 } nyf_tile;

/* Filter parameters (Sec. IV setup; Algorithm 1's m0 is K). */
typedef struct {
  float sigma_s;      /* spatial Gaussian std; unused for NYF_BOX unless S <= 0 */
  float sigma_r;      /* range Gaussian std (theta), > 0 */
  int K;              /* number of landmarks m0, 1..NYF_MAX_K */
  int kmeans_iters;   /* Lloyd iterations, >= 0 (0: landmarks = the drawn pixels) */
  uint64_t seed;      /* SplitMix64 seed of the initial-landmark and subsample draws */
  double eig_rel_tol; /* tau: modes with alpha_k > tau * alpha_max are kept, >= 0 */
  int precision;      /* nyf_precision.  Filters: NYF_BF16 runs the convolutions (window
                         radius <= 16) on the BF16 tensor cores -- operands phi f and
                         the vertical-pass result rounded to bfloat16, FP32
                         accumulation; the features stay float32 in the workspace
                         (bfloat16 storage of phi alone costs up to 4e-3 relative
                         error when landmarks are sparse relative to sigma_r).
                         nyf_features: storage type of phi. */
  int spatial;        /* nyf_spatial */
  int S;              /* window radius; <= 0 means ceil(3 sigma_s) */
  int patch_radius;   /* NLM: guide = (2r+1)^2 x n patch, reflect-101 border */
  float sample_frac;  /* fraction of pixels k-means clusters, (0, 1] */
  int conv_tile;      /* nyf_tile: convolution kernel variant */
  int save_for_backward; /* nyf_save: what nyf_filter_blf keeps in the workspace for
                            nyf_filter_blf_backward.  NYF_SAVE_NONE: forward-only
                            workspace.  NYF_SAVE_PLANES: the K (n+1) convolved planes
                            C_kq = omega * (phi_k f_q) (the workspace grows by
                            K (n+1) H W floats plus the backward scratch).
                            NYF_SAVE_RECOMPUTE: the features and eta only; the backward
                            convolves C_kq again, NYF_RECOMPUTE_MODES modes at a time,
                            so the planes take min(K, NYF_RECOMPUTE_MODES) (n+1) H W
                            floats (the backward costs about the forward's
                            convolutions more).  Other values: NYF_ERR_INVALID_ARG. */
} nyf_params;

/* nyf_params.save_for_backward */
typedef enum { NYF_SAVE_NONE = 0, NYF_SAVE_PLANES = 1, NYF_SAVE_RECOMPUTE = 2 } nyf_save;
#define NYF_RECOMPUTE_MODES 4

/* Device-side results of the last call on a workspace (nyf_get_stats). */
typedef struct {
  int status;              /* sticky nyf_status of the work run on this workspace */
  int rank;                /* kept modes r */
  double qerr;             /* k-means quantisation error e for the final landmarks (Sec. III) */
  double alpha_max;        /* largest eigenvalue of A */
  double alpha_min_kept;   /* smallest kept eigenvalue */
  long long eta_small;     /* pixels with eta_hat <= 1e-6 * sum(omega) (Eq. (15)) */
  float grad_sigma_r;      /* last backward: dL/d sigma_r */
  float grad_sigma_s;      /* last backward: dL/d sigma_s */
} nyf_stats;

/* Bytes of workspace that the filter calls need for an H x W image with n
 * channels and guide dimension rho (rho is ignored for NLM, whose guide
 * dimension is n (2r+1)^2).  The same workspace serves nyf_kmeans and
 * nyf_features on N = H * W rows.  Returns 0 if the arguments are invalid. */
size_t nyf_workspace_size(int H, int W, int n, int rho, const nyf_params* params);

/* k-means landmark selection (Sec. III "we partition R into m0 disjoint sets
 * using k-means"; Algorithm 1, clustering step).
 *   X         N x rho rows to cluster (device, read only)
 *   init_idx  K distinct row indices of the initial centroids (device int64),
 *             or NULL: drawn on the device as the first K distinct values of
 *             SplitMix64(seed) output mod N
 *   centroids K x rho output (device)
 *   labels    N int32 output for the final centroids, or NULL
 *   qerr      1 double output: quantisation error e for the final centroids, or NULL
 * Each iteration assigns every row to its nearest centroid (ties to the
 * lowest index) and moves each centroid to the mean of its members (an empty
 * cluster keeps its centroid).  Reductions run in a fixed order, so results
 * are bitwise reproducible. */
nyf_status nyf_kmeans(const float* X, int64_t N, int rho, int K, int iters, uint64_t seed,
                      const int64_t* init_idx, float* centroids, int32_t* labels, double* qerr,
                      void* ws, size_t ws_bytes, void* stream);

/* ---- Strip processing: an image cut into horizontal strips (one per GPU, or
 * one at a time on one GPU), each filtered with an S-row halo, with k-means
 * run over all strips by exchanging per-cluster sums (Sec. III clustering:
 * the Lloyd update is a mean, so it only needs the strips' sums and counts).
 *
 * nyf_draw_indices (host only, no GPU work): the k-means initial rows of an
 * image of N rows, the first K distinct values of SplitMix64(seed) output mod N
 * (the same draw as nyf_kmeans with init_idx == NULL), into out[0..K) (host
 * int64).  Returns the number drawn (K, or fewer if the draw limit of 64 K +
 * 4096 outputs was reached; 0 for invalid arguments). */
int nyf_draw_indices(uint64_t seed, int64_t N, int K, int64_t* out);

/* out (K x rho, device) = row idx[j] - row0 of X (N x rho, device) when
 * 0 <= idx[j] - row0 < N, else zeros: a strip's share of the initial centroids
 * (the strips' shares add up to the rows of the whole image).  idx: K device
 * int64 (whole-image row numbers); row0: the strip's first row number. */
nyf_status nyf_gather_rows(const float* X, int64_t N, int rho, int64_t row0, const int64_t* idx,
                           int K, float* out, void* stream);

/* One assignment pass of Lloyd's algorithm over the N x rho rows X against the
 * K x rho centroids (nearest centroid, ties to the lowest index):
 *   sums  K x (rho + 1) doubles (device, out): sums[j (rho + 1) + d] = the sum of
 *         coordinate d over the rows assigned to j, sums[j (rho + 1) + rho] = their count
 *   qerr  1 double (device, out): the sum of the rows' squared distances to their centroid.
 * Sums are formed in a fixed order (bitwise reproducible).  ws as for nyf_kmeans. */
nyf_status nyf_kmeans_partials(const float* X, int64_t N, int rho, int K, const float* centroids,
                               double* sums, double* qerr, void* ws, size_t ws_bytes, void* stream);

/* The update step from (all-reduced) sums: centroid j = sums[j][0..rho) / sums[j][rho],
 * unchanged when the count is zero. */
nyf_status nyf_kmeans_apply_sums(const double* sums, int K, int rho, float* centroids, void* stream);

/* Nystrom per-pixel features (Eqs. (9)-(12)).  For landmarks mu (K x rho):
 * A(i,j) = kappa(mu_i, mu_j) is decomposed to FP64 accuracy (Eq. (10)),
 * modes with alpha_k > eig_rel_tol * alpha_max are kept (r of them), and for
 * every row p_x of `guide` (N x rho)
 *     phi_j(x) = sum_m kappa(p_x, mu_m) W[m][j],   j < K,
 * with the symmetric factor W = W_r Lambda_r^{-1/2} W_r^T (= A_r^{-1/2}), so
 * that sum_j phi_j(x) phi_j(y) = K-hat(x, y) = sum_{k<r} alpha_k v_k(x) v_k(y)
 * with v_k of Eq. (12).  The symmetric factor is unique (no eigenvector sign
 * or rotation freedom) and keeps the features well conditioned.
 *   phi     output, K planes of N values (plane j at phi + j * N), float32
 *           (NYF_FP32) or bfloat16 (NYF_BF16)
 *   rank    1 int output (device): r, or NULL
 *   alphas  K doubles output (device): all eigenvalues of A, descending, or NULL */
nyf_status nyf_features(const float* guide, int64_t N, int rho, const float* landmarks, int K,
                        float sigma_r, double eig_rel_tol, int precision, void* phi, int* rank,
                        double* alphas, void* ws, size_t ws_bytes, void* stream);

/* nyf_features for callers that cannot allocate device memory (a plain C host
 * without a device allocator, a plugin whose host owns all device memory, a
 * latency-critical loop where cudaMalloc would synchronise the device).  The
 * paper has no counterpart: this is a deployment variant of nyf_features.
 * Same arguments, argument checks and results as nyf_features, without
 * ws/ws_bytes: its scratch (status word, W_hat factor, FP64 eigendecomposition
 * buffers) is a fixed 256 KiB array in device memory that every GPU loading the
 * library holds until the process exits.  The first call on a device looks up
 * that array's address (cudaGetSymbolAddress, with the device current) and
 * caches it; make that first call before any stream capture.  All calls share
 * the array and it keeps the last call's contents, so calls that overlap on the
 * GPU race.
 *   status  1 int output (device), or NULL: written, stream-ordered after the
 *           call's work, with the status the device latched -- NYF_OK, or
 *           NYF_ERR_NUMERIC when no eigenvalue was kept (rank 0), in which case
 *           phi was NOT written.  The latched word lives in the library's own
 *           array, so this output is the only way to see a device-side error.
 * Returns NYF_ERR_UNSUPPORTED for K > NYF_STATIC_MAX_K or
 * rho > NYF_STATIC_MAX_RHO, NYF_ERR_CUDA if the address lookup fails.
 * Allocates nothing. */
#define NYF_STATIC_MAX_K 64
#define NYF_STATIC_MAX_RHO 160
nyf_status nyf_features_static(const float* guide, int64_t N, int rho, const float* landmarks,
                               int K, float sigma_r, double eig_rel_tol, int precision, void* phi,
                               int* rank, double* alphas, int* status, void* stream);

/* Nystrom bilateral filter, Algorithm 1 with output Eqs. (14)-(15).
 *   f          H x W x n image (device)
 *   guide      H x W x rho guide (joint BLF), or NULL: guide = f (rho must equal n)
 *   landmarks  K x rho landmarks (device), or NULL: k-means on every pixel
 *              of the guide (params->kmeans_iters, params->seed)
 *   out        H x W x n output g_hat = zeta / eta (device); pixels where
 *              eta_hat <= 0 are not clamped (Eq. (15) can vanish)
 * The workspace keeps the landmarks, factors, features and eta, and with
 * params->save_for_backward the convolved planes C_kq, for
 * nyf_filter_blf_backward. */
nyf_status nyf_filter_blf(const float* f, const float* guide, int H, int W, int n, int rho,
                          const nyf_params* params, const float* landmarks, float* out,
                          void* ws, size_t ws_bytes, void* stream);

/* Nystrom nonlocal means: guide p(x) = the (2r+1) x (2r+1) x n patch around x
 * (Sec. II; Sec. IV "Color NLM", rho = n (2r+1)^2), reflect-101 border,
 * components ordered (dy, dx, c); box window of radius params->S.
 * k-means runs on round(sample_frac * N) pixels, one drawn per stratum of the
 * row-major pixel order with SplitMix64(seed ^ 0xA5A5A5A5A5A5A5A5).
 *   landmarks  K x rho patch landmarks (device) or NULL (k-means). */
nyf_status nyf_filter_nlm(const float* f, int H, int W, int n, const nyf_params* params,
                          const float* landmarks, float* out, void* ws, size_t ws_bytes,
                          void* stream);

/* Diagnostic for NYF_GAUSSIAN_IIR (host only, no GPU work): the parameters one
 * line direction of length len uses, as computed on the host in FP64 and rounded
 * to FP32.  out[0..3] = B, -B, g1, -e2 of the difference form
 *   dl = B x[i] - B w[i-2] + g1 d1 - e2 d2,  w[i] = w[i-1] + dl
 * (d1 = w[i-1] - w[i-2], d2 = w[i-2] - w[i-3]); out[4] = LS, values per lane of
 * the line padded with zeros to 32 LS; out[5] = len; out[6 + 9 d .. ] = the 3 x 3
 * matrix T^(LS 2^d), d = 0..4 (row-major, basis (w, d1, d2), T the step with zero
 * input); out[51..59] = Rm, the anticausal state entering at the padded end from
 * the causal state at its last value.  out_len >= 60. */
nyf_status nyf_iir_line_params(double sigma_s, int len, float* out, int out_len);

/* ---- PCA-NLM (Sec. IV: the paper's NLM experiments use principal-neighbourhood
 * NLM).  The patch guide p(x) of nyf_filter_nlm (rho = n (2r+1)^2 <= 160, r =
 * params->patch_radius >= 1) is replaced by its coordinates in the q leading
 * principal directions of the image's patches:
 *     m = (1/N) sum_x p(x),  C = (1/N) sum_x (p(x) - m)(p(x) - m)^T = U diag(lambda) U^T,
 *     guide p~(x) = U_q^T (p(x) - m),   1 <= q <= min(rho, 32).
 * The leading eigenvectors are unique only up to sign and rotations within
 * groups of equal eigenvalues; the filter depends on U_q only through the
 * subspace it spans. */

/* Mean patch, all rho eigenvalues of C (descending) and the q leading
 * eigenvectors.  Covariance accumulated in FP32 per CTA from patches shifted by
 * the channel means, reduced in FP64; eigendecomposition in FP32 on one CTA:
 * Householder tridiagonalisation, every eigenvalue by bisection on Sturm
 * counts, the q leading eigenvectors by inverse iteration (reorthogonalised
 * within clusters of close eigenvalues) and back-transformation, then the q
 * columns re-orthonormalised in FP64.  Every loop has a fixed trip count.
 *   mean     rho floats (device, out)
 *   basis    rho x q floats, row-major: basis[i * q + j] = component i of
 *            eigenvector j (device, out)
 *   eigvals  rho floats (device, out)
 *   ws       at least nyf_patch_pca_workspace_size(n, r) bytes, 256-B aligned.
 * NYF_ERR_INVALID_ARG for r < 1, rho > 160, q outside [1, min(rho, 32)]. */
size_t nyf_patch_pca_workspace_size(int n, int r);
nyf_status nyf_patch_pca(const float* f, int H, int W, int n, int r, int q, float* mean,
                         float* basis, float* eigvals, void* ws, size_t ws_bytes, void* stream);

/* guide (H x W x q, device, out) = U_q^T (p(x) - m) with the given mean and basis
 * (layouts as for nyf_patch_pca).  No workspace. */
nyf_status nyf_pca_project(const float* f, int H, int W, int n, int r, int q, const float* mean,
                           const float* basis, float* guide, void* stream);

/* PCA-NLM through Algorithm 1: the PCA guide (from mean and basis when both are
 * given, else from the image's own moments), then the joint filter of
 * nyf_filter_blf with that guide (rho = q): k-means on round(sample_frac * N)
 * guide rows (landmarks == NULL) or the given q-dimensional landmarks, and
 * params->spatial / S as for the other filters (the paper: a box, S = 10).
 * params->save_for_backward must be 0 and precision FP32 or BF16 as for
 * nyf_filter_blf.  ws: nyf_pca_nlm_workspace_size bytes. */
size_t nyf_pca_nlm_workspace_size(int H, int W, int n, int q, const nyf_params* params);
nyf_status nyf_filter_pca_nlm(const float* f, int H, int W, int n, int q, const nyf_params* params,
                              const float* mean, const float* basis, const float* landmarks,
                              float* out, void* ws, size_t ws_bytes, void* stream);

/* Adjoint of nyf_filter_blf (the paper has no gradients; derived from
 * Eqs. (9)-(15)).  Must follow the nyf_filter_blf call that produced `out`
 * on the same workspace, with the same f, guide and params, and
 * params->save_for_backward NYF_SAVE_PLANES or NYF_SAVE_RECOMPUTE (else
 * NYF_ERR_INVALID_ARG).  With NYF_SAVE_RECOMPUTE the convolved planes are
 * formed again, in FP32, a few modes at a time.  Landmarks are
 * held fixed; the window radius S is held at its forward value; the kept
 * modes are held fixed.  Given grad_out = dL/d g_hat (H x W x n):
 *   grad_f      H x W x n output dL/df; if guide was NULL this is the total
 *               derivative (image and guide are the same tensor)
 *   grad_guide  H x W x rho output dL/dp for a joint guide, or NULL
 *   grad_sigma  2 floats output (device): dL/d sigma_r, dL/d sigma_s
 *               (dL/d sigma_s is 0 for the box window). */
nyf_status nyf_filter_blf_backward(const float* f, const float* guide, int H, int W, int n,
                                   int rho, const nyf_params* params, const float* out,
                                   const float* grad_out, float* grad_f, float* grad_guide,
                                   float* grad_sigma, void* ws, size_t ws_bytes, void* stream);

/* Self-test of the fifth-generation tensor-core path the BF16 convolutions use
 * (the paper has no counterpart): one CTA computes D = A B^T, M = 128,
 * N in {16, 32, ..., 256}, K in {16, 32, ..., 128}, from operands the kernel
 * generates, A[m][k] = (((3m + 5k) mod 17) - 8) / 8 and
 * B[n][k] = (((7n + 3k) mod 13) - 6) / 4 (exact in bfloat16), with tcgen05.mma
 * accumulating in tensor memory.
 *   D          128 x N float32 output (device, row-major)
 *   a_in_tmem  0: A in shared memory; 1: A in tensor memory (bf16 pairs per column)
 *   status     1 int output (device): 0, or 1 if the MMA completion wait timed out
 * Returns NYF_ERR_INVALID_ARG for other sizes. */
nyf_status nyf_selftest_umma(float* D, int N, int K, int a_in_tmem, int* status, void* stream);

/* Self-test of the bounded device waits every waiting kernel uses (the paper
 * has no counterpart): one warp waits for an mbarrier phase that nothing
 * completes, gives up after `limit` polls (1..4096, each at most ~1 us) and
 * latches NYF_ERR_TIMEOUT into *status (device int, zeroed first).  Nothing
 * traps or hangs; the context stays usable. */
nyf_status nyf_selftest_wait_timeout(int limit, int* status, void* stream);

/* ---- Batched filtering of images of uneven sizes (one workload, one call).
 * Image b of the batch is the H_b x W_b x n HWC block starting at element
 * items[b].offset of the packed buffers f / out / grad_out / grad_f (device);
 * items is a host array read during the call.  Each image uses its own
 * sigma_s, sigma_r (and conv_tile unless NYF_TILE_AUTO) and the shared
 * fields of *params; landmarks come from k-means per image.  The steps that
 * are small per image run as one launch per step for the whole batch, on
 * `stream`: the k-means of every image (when its rows take the CUDA-core
 * assignment pass, i.e. n outside 16..80, and params->sample_frac >= 1) or
 * the copies of given landmarks, then the eigendecompositions.  The rest
 * (features, convolutions, and the k-means of the other cases) runs per
 * image on a small pool of internal streams of the current device, forked
 * from and joined back to `stream` with events, so the whole call can be
 * captured into a CUDA graph and replayed.  Every image's result is bitwise
 * that of the per-image call with the same arguments.  The pool (streams and events) is
 * created by the first batched call made on a device, so make that first call
 * outside any stream capture (stream creation is not allowed while a capture
 * is in progress).  Do not issue batched calls on the same device from several
 * host threads at once (they share the pool). */
typedef struct {
  int64_t offset;   /* first element of image b in the packed buffers */
  int H, W;
  float sigma_s, sigma_r;
  int conv_tile;    /* nyf_tile for this image, or NYF_TILE_AUTO for params->conv_tile */
  int reserved;
} nyf_batch_item;

/* Workspace bytes for the batch (per-image slices), 0 if invalid. */
size_t nyf_batched_workspace_size(const nyf_batch_item* items, int B, int n,
                                  const nyf_params* params);

/* Forward of every image (as nyf_filter_blf with guide = image).
 *   landmarks  B x K x n floats (device; image b's K x n landmarks start at
 *              landmarks + b K n), or NULL: k-means per image
 *              (params->kmeans_iters, params->seed) as nyf_filter_blf does. */
nyf_status nyf_filter_blf_batched(const float* f, const nyf_batch_item* items, int B, int n,
                                  const nyf_params* params, const float* landmarks, float* out,
                                  void* ws, size_t ws_bytes, void* stream);

/* Backward of every image (as nyf_filter_blf_backward), after the batched
 * forward on the same workspace.  grad_sigma: 2 B floats (device),
 * [dL/d sigma_r, dL/d sigma_s] per image. */
nyf_status nyf_filter_blf_batched_backward(const float* f, const nyf_batch_item* items, int B,
                                           int n, const nyf_params* params, const float* out,
                                           const float* grad_out, float* grad_f,
                                           float* grad_sigma, void* ws, size_t ws_bytes,
                                           void* stream);

/* nyf_get_stats of image b of a batch. */
nyf_status nyf_batched_stats(const void* ws, const nyf_batch_item* items, int B, int n,
                             const nyf_params* params, int b, nyf_stats* out, void* stream);

/* Copies the device-side results of the last call on `ws` to *out.  This is
 * the one call that synchronises `stream`. */
nyf_status nyf_get_stats(const void* ws, nyf_stats* out, void* stream);

/* Per-stage timing (instrumentation for measurement, off by default).  While
 * enabled, each filter call records CUDA events on its stream around its
 * stages: 0 landmarks (subsample + k-means), 1 eigendecomposition,
 * 2 features, 3 convolution + combine, 4 backward convolutions,
 * 5 backward features, 6 backward landmark-kernel term.  nyf_get_timing
 * synchronises on the events of the last instrumented call and writes the
 * elapsed milliseconds of up to `max_stages` stages (-1 for a stage that did
 * not run); it returns the number of stages written.  Not for use while a
 * stream is being captured into a CUDA graph. */
void nyf_set_timing(int enable);
int nyf_get_timing(float* ms, int max_stages);

/* Number of kernels this process has launched through libnyf so far. */
long long nyf_launch_count(void);

/* Static description of a status code. */
const char* nyf_status_string(nyf_status s);

/* ABI version (major * 100 + minor). */
int nyf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NYF_H */

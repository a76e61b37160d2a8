/*
 * vb.h -- C ABI of libvb: the sparse self-tuning variable-bandwidth (VB) kernel
 * build of Davis & Giannakis, "Graph-theoretic algorithms for Kolmogorov
 * operators" (arXiv 2104.15124), on one NVIDIA GB300 (sm_103a).
 *
 * The library turns n samples x^(i) in R^m (Sec. 2, problem statement) into
 * the sparse symmetric matrix L-hat that approximates the Kolmogorov operator
 * L_{psi,c} (Eq. symmetric discrete Kolmogorov operator), following the four
 * steps of Sec. 4: exact kNN and the bandwidth b (Eq. bandwidth parameter),
 * the self-tuned density kernel and density estimate psi (Sec. 2.1, 2.3), the
 * self-tuned operator kernel and its normalisations (Sec. 2.2), the CSR of
 * L-hat, and the sparse matrix-vector product consumed by eigen-solvers.
 *
 * Conventions shared by every entry point
 *   - Return value: VB_OK (0) or a negative vb_status.  Argument and launch
 *     errors are returned synchronously; errors found on the device (a zero
 *     bandwidth, a non-finite coordinate, an over-full row) are recorded in the
 *     context's device report and read with vb_report_read().
 *   - Every pointer argument is a DEVICE pointer owned by the caller unless
 *     stated otherwise; arrays are dense and contiguous.  The library never
 *     allocates, frees or keeps caller memory.  Scratch memory comes from a
 *     caller-provided workspace of at least the size returned by the matching
 *     vb_*_workspace() call (256-byte aligned base).
 *   - All work is enqueued asynchronously on the context's CUDA stream.  No
 *     call synchronises the host except vb_report_read() and vb_solve().
 *   - Indices: int32 for points and columns, int64 for row offsets.
 *     Limits: 2 <= n < 2^31 - 1, 1 <= m <= 128, 1 <= k <= n - 1,
 *     k + margin <= 256.
 *   - Sizes whose value is data-dependent (the number of stored entries nnz)
 *     stay on the device; callers size CSR outputs for the worst case
 *     n * (2k + 1) and read nnz from the device.
 */
#ifndef VB_H
#define VB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t vb_status;
#define VB_OK                 0
#define VB_ERR_ARG           -1   /* invalid argument (sizes, NULL, limits) */
#define VB_ERR_CUDA          -2   /* a CUDA runtime call or launch failed */
#define VB_ERR_WORKSPACE     -3   /* workspace smaller than required */
#define VB_ERR_DEGENERATE    -4   /* b_i = 0 (more than k_bw copies of a point) or non-finite input */
#define VB_ERR_EPS_BOUNDARY  -5   /* tuned epsilon sits at an end of its grid (reported as a warning) */
#define VB_ERR_NOT_CONVERGED -6   /* eigen-solver did not reach its tolerance */
#define VB_ERR_TIMEOUT       -7   /* a bounded device-side wait ran out */
#define VB_ERR_BOUNDS        -8   /* an index fell outside its array (debug checks) */
#define VB_ERR_UNSUPPORTED   -9   /* valid request outside what this build handles */

/* Human-readable name of a status code (static string). */
const char* vb_status_string(vb_status s);

/* ------------------------------------------------------------------ context */

typedef struct vb_ctx vb_ctx;

/* Creates a context bound to CUDA device `device` and stream `stream`
 * (a cudaStream_t; NULL = legacy default stream).  Allocates one 256-byte
 * device report block and a pinned host mirror, freed by vb_destroy(). */
vb_status vb_create(vb_ctx** ctx, int32_t device, void* stream);
vb_status vb_destroy(vb_ctx* ctx);
/* Rebinds the context to another stream of the same device. */
vb_status vb_set_stream(vb_ctx* ctx, void* stream);

/* Device-side report of the work enqueued since the last reset. */
typedef struct {
    int32_t error;              /* first device-detected vb_status, 0 if none */
    int32_t warnings;           /* bit 0: density epsilon at a grid end; bit 1: operator epsilon at a grid end */
    int64_t knn_fallback_rows;  /* kNN rows whose FP32 candidate list failed the FP64 certificate */
    int64_t knn_candidates;     /* (query, candidate) distances evaluated by the tiled search */
    int64_t union_big_rows;     /* rows of the symmetric union longer than the warp path's limit */
    int64_t knn_heap_levels;    /* heap levels walked by the kNN selection (inserts and final sort) */
    int64_t knn_tiles_staged;   /* candidate tiles staged in shared memory by the kNN search */
    int64_t knn_insert_rounds;  /* per-query insertion rounds executed by the kNN search */
    int64_t knn_retry_tiles;    /* query tiles the radius-first search handed back to the exact search */
    int64_t knn_rows_short;     /* rows with fewer than k candidates kept (radius too small) */
    int64_t knn_rows_long_run;  /* rows whose FP32/16-bit ties or error band exceeded the exact-order buffer */
    int64_t knn_rows_uncertified; /* rows whose k-th FP64 distance did not clear the certificate bound */
    int64_t knn_retry_candidates; /* the part of knn_candidates evaluated by the exact FP32 pass over handed-back tiles */
    int64_t knn_redo_tiles;     /* query tiles the 16-bit radius-first search searched again at twice the radius */
} vb_report;

/* Waits for the context's stream and copies the device report to *out. */
vb_status vb_report_read(vb_ctx* ctx, vb_report* out);
/* Clears the device report (asynchronous, on the context's stream). */
vb_status vb_report_reset(vb_ctx* ctx);

/* Measurement hooks (not part of the paper's method).  When enabled, every
 * stage below is bracketed by CUDA events on the context's stream, and the
 * host counts the kernel launches it enqueues. */
#define VB_STAGE_KNN_ORDER       0   /* bounding box, Morton keys, radix sort, gather, tile and super-tile boxes */
#define VB_STAGE_KNN_TILE        1   /* first search pass (FP32 or 16-bit tiles), FP64 rescoring and certificate */
#define VB_STAGE_KNN_FALLBACK    2   /* exact FP64 selection of uncertified rows */
#define VB_STAGE_GRAPH           3   /* symmetric union CSR */
#define VB_STAGE_BANDWIDTH       4
#define VB_STAGE_SWEEP_DENSITY   5
#define VB_STAGE_DENSITY         6
#define VB_STAGE_CENTRE          7
#define VB_STAGE_SWEEP_OPERATOR  8
#define VB_STAGE_OPERATOR        9   /* q and D passes */
#define VB_STAGE_LHAT           10   /* L-hat CSR values */
#define VB_STAGE_KNN_RADIUS     11   /* per-point search radius (learned model or caller's radii) */
#define VB_STAGE_KNN_RETRY      12   /* exact FP32 search of the query tiles the first pass handed back */
#define VB_NUM_STAGES           13
vb_status vb_profile_enable(vb_ctx* ctx, int32_t on);
/* Synchronises the stream; ms[s] = duration of stage s in its most recent run
 * since the last read (negative when it did not run); *launches = kernels
 * enqueued since profiling was enabled.  Either output may be NULL. */
vb_status vb_profile_read(vb_ctx* ctx, float* ms, int64_t* launches);

/* --------------------------------------------------------------- kNN (a1-a5)
 * Exact k nearest neighbours (Sec. 2.1: I(x, r) is the r-th closest sample,
 * I(x^(i), 0) = i, so the point itself is excluded).  Distances are the
 * canonical FP64 squared distances
 *     d2 = ((s_0 + s_1) + s_2) + ...,  s_r = (x_ir - x_jr)^2  (RN, no FMA),
 * and neighbours are ordered by (d2, j): distance first, then smaller index.
 * The search stages the points in a Morton order (of the coordinates when
 * m <= 4, of the projections on the cloud's 5 leading principal axes when
 * m > 4), prunes 64-point tiles by bounding boxes (in the FP32 search of a cloud
 * of more than 1,024 tiles, boxes of 64-tile super-tiles first; in the pipelined
 * 16-bit search, also balls about the box centres) and keeps the k + margin
 * nearest FP32 (or 16-bit) candidates per row;
 * an FP64 rescoring with a proven FP32 error bound certifies every row, and
 * rows that fail it are recomputed by an exact FP64 radix selection.  The
 * output is therefore exact, identical to a brute-force FP64 search. */

#define VB_PREC_FP32 0      /* FP32 ALU distances */
#define VB_PREC_BF16 1      /* BF16 tensor-core distance tiles (tcgen05.mma, FP32 accumulation) with FP64 rescoring
                               (the staged kernel, operands recentred on every query tile) */
#define VB_PREC_FP16 2      /* the same with FP16 tiles (11-bit significand: an 8x narrower error band) */
#define VB_PRUNE_NONE    0  /* visit every candidate tile (brute force) */
#define VB_PRUNE_EXACT   1  /* skip tiles whose box distance exceeds the running k+margin-th distance */
#define VB_PRUNE_LEARNED 2  /* radius-first search: every query's heap starts full of sentinels at its radius
                               guess, so tiles and candidates outside it are pruned from the start and no seed
                               tiles are needed; tiles with a row that finds fewer than k points inside its
                               radius, or fails the certificate, are redone by the exact search, so the output
                               stays exact */
/* Kernel of the 16-bit search.  STAGED: one CTA converts and stages one candidate
 * tile per step, then MMA, then selection.  PIPELINED: every 64-point tile is
 * converted once into its MMA operand image; a producer warp stages the images by
 * bulk copies (TMA) into a shared-memory ring, an MMA warp feeds four tensor-memory
 * accumulator buffers, and four warps select, all overlapped. */
#define VB_KEYS_COMPACT 0
#define VB_KEYS_FULL    1
#define VB_CURVE_AUTO    0
#define VB_CURVE_MORTON  1
#define VB_TC_AUTO      0
#define VB_TC_STAGED    1
#define VB_TC_PIPELINED 2

typedef struct vb_mlp vb_mlp;

typedef struct {
    int32_t k;               /* neighbours per point */
    int32_t margin;          /* extra FP32 candidates kept for the certificate (exact search) */
    int32_t precision;       /* VB_PREC_* */
    int32_t prune;           /* VB_PRUNE_* */
    const float* radius;     /* VB_PRUNE_LEARNED without a model: per point (original order) guess of the
                                distance to its k-th neighbour, n floats on the device */
    const vb_mlp* mlp;       /* VB_PRUNE_LEARNED: learned radius model (NULL = use `radius`) */
    float radius_inflate;    /* factor applied to every radius guess (0 = 1.5) */
    float radius_log_shift;  /* added to the model's predicted log radius, e.g. ln(n_train / n) / d */
    const float* cloud_log_shift;  /* batched build with a model: device array of B shifts added per
                                      cloud, e.g. ln(n_train / n_b) / d (NULL = none) */
    int32_t seed_tiles;      /* exact FP32 search: neighbouring tiles on each side of a query tile that are
                                searched before any pruning (0 = enough to fill every heap) */
    int32_t tc_variant;      /* 16-bit tiles: VB_TC_AUTO (FP16: pipelined when its shared memory fits, else
                                staged; BF16: staged), VB_TC_STAGED or VB_TC_PIPELINED (VB_ERR_UNSUPPORTED
                                when k + margin and m leave no room for two ring slots).  The pipelined
                                kernel centres its operands on the whole cloud, not on each query tile,
                                so its 16-bit error band is wider: exact either way, but with BF16 many
                                rows go back to the FP32 search */
    int32_t heap_keys;       /* m <= 16: VB_KEYS_COMPACT (default: 32-bit heap keys, half the shared memory;
                                in the FP32 search, tiles that need more than 255 candidate-tile visits or
                                fail the certificate are redone with full keys, and so are the tiles a
                                radius-first or 16-bit first pass hands back) or VB_KEYS_FULL (64-bit keys
                                only; always when m > 16).  The staged 16-bit search keeps compact keys at
                                m <= 16 except with VB_KEYS_FULL at m <= 4 */
    float* dbg_d2;           /* diagnostic (NULL = off), 16-bit searches: n x (k + margin) device floats; row i
                                receives the 16-bit tile distances of the candidates its search kept, ascending,
                                before the FP64 rescoring (the kernel's own tile arithmetic; with compact keys
                                the lower edge of the key's bucket, 2^-10 relative below the distance) */
    int32_t* dbg_idx;        /* with dbg_d2: n x (k + margin) device int32, the original index of each of those
                                candidates (-1 for an unused slot) */
    int32_t curve;           /* spatial order of the search's tiles at 2 <= m <= 4: VB_CURVE_AUTO (default, the
                                Hilbert curve) or VB_CURVE_MORTON; m = 1 and m > 4 (principal-axis keys) always
                                take the Morton interleave.  The lists are exact either way */
} vb_knn_params;

/* Launch-shape autotuner (a16).  Times vb_knn on the caller's input for every
 * candidate shape -- heap depth k + margin with margin in {2, 4, 8, 16, 32} and
 * seed_tiles in {1, 2, 3} for the FP32 search, margin in {4, 8, 16, 32} and the kernel
 * (tc_variant staged or pipelined) for 16-bit tiles --
 * with CUDA events on the context's stream (synchronising), and writes the
 * fastest into *best (a copy of *p with margin, seed_tiles and tc_variant set) and its time
 * into *best_ms.  Results are cached for the process by (m, k, precision, prune,
 * floor(log2 n)); a cached key returns at once without running anything (then
 * *best_ms = 0).  nbr / nbr_d2 / ws as for vb_knn, sized for k; every result is
 * exact, so the outputs hold the neighbour lists afterwards.  cloud_ptr_dev / B
 * describe a batch as in vb_build_batch (NULL / 1 for one cloud); the cache key
 * then uses the mean cloud size. */
vb_status vb_knn_autotune(vb_ctx* ctx, const float* x, int64_t n, int32_t m, const int64_t* cloud_ptr_dev,
                          int32_t B, const vb_knn_params* p, int32_t* nbr, double* nbr_d2, void* ws,
                          size_t ws_bytes, vb_knn_params* best, float* best_ms);

/* Workspace bytes vb_knn() needs for n points in R^m. */
size_t vb_knn_workspace(int64_t n, int32_t m, const vb_knn_params* p);

/* x: n x m FP32 row-major.  nbr: n x k int32, nbr_d2: n x k FP64 (row i holds
 * the neighbours of point i in rank order). */
vb_status vb_knn(vb_ctx* ctx, const float* x, int64_t n, int32_t m, const vb_knn_params* p,
                 int32_t* nbr, double* nbr_d2, void* ws, size_t ws_bytes);

/* ---------------------------------------------------- learned radius (a7)
 * A small network in_dim -> 64 -> 64 -> 1 (GELU, erf form) predicts the log of
 * a point's distance to its k-th neighbour from its coordinates; with
 * VB_PRUNE_LEARNED and knn.mlp set, exp(prediction + radius_log_shift) *
 * radius_inflate is each point's radius guess.  Parameters live on the
 * device: FP32 master weights, a BF16 copy used by the forward passes, Adam
 * moments.  Inputs and targets are standardised with host-side constants.
 * Parameter layout (vb_mlp_param_count floats): W1 [64][in_dim], b1 [64],
 * W2 [64][64], b2 [64], w3 [64], b3 [1]. */
#define VB_MLP_HIDDEN 64
#define VB_MLP_MAX_IN 16
struct vb_mlp {
    int32_t in_dim;                     /* 1 .. VB_MLP_MAX_IN (the first in_dim coordinates are used) */
    float* master;                      /* device FP32 parameters */
    uint16_t* weights;                  /* device BF16 parameters (round-to-nearest copy of master) */
    float* adam_m;                      /* device Adam moments, same size */
    float* adam_v;
    float in_mean[VB_MLP_MAX_IN];       /* input standardisation: (x - mean) / scale */
    float in_scale[VB_MLP_MAX_IN];
    float out_mean, out_scale;          /* prediction = out_mean + out_scale * network output */
    int64_t step;                       /* Adam steps taken */
};
int64_t vb_mlp_param_count(int32_t in_dim);
/* Sets the standardisation constants of mlp from the training data: in_mean / in_scale the mean and
 * sample standard deviation (n - 1) of each of the first in_dim columns of x [n][ld], out_mean /
 * out_scale those of y [n] (scales floored at 1e-12); FP64 sums in a fixed order.  ws: at least
 * 8 * 2 (VB_MLP_MAX_IN + 1) bytes of device memory.  Synchronises the host (the constants are host fields). */
vb_status vb_mlp_standardise(vb_ctx* ctx, vb_mlp* mlp, const float* x, int32_t ld, const float* y, int64_t n,
                             void* ws, size_t ws_bytes);
/* He-normal initialisation of master (counter-based generator from seed), zero moments, BF16 copy. */
vb_status vb_mlp_init(vb_ctx* ctx, vb_mlp* mlp, uint64_t seed);
size_t vb_mlp_workspace(int32_t in_dim, int64_t batch);
/* One epoch of Adam (lr, beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared error of the
 * standardised target over x [n][ld] (first in_dim columns used) and y [n] (raw log radii), in
 * minibatches of `batch` consecutive rows, starting from a block chosen by seed.
 * loss_dev (optional, device FP32): mean squared error of the epoch's last minibatch. */
vb_status vb_mlp_train_epoch(vb_ctx* ctx, vb_mlp* mlp, const float* x, int32_t ld, const float* y, int64_t n,
                             int32_t batch, float lr, uint64_t seed, float* loss_dev, void* ws, size_t ws_bytes);
/* Full-batch gradient of the loss (mean over n of (net(x) - y_std)^2) at the BF16 weights, FP32
 * arithmetic, deterministic; grad: vb_mlp_param_count FP32 on the device; loss_dev: 1 FP32. */
vb_status vb_mlp_gradient(vb_ctx* ctx, const vb_mlp* mlp, const float* x, int32_t ld, const float* y, int64_t n,
                          float* grad, float* loss_dev, void* ws, size_t ws_bytes);
/* y[i] = predicted log radius of row i of x [n][ld] (BF16 weights, FP32 arithmetic). */
vb_status vb_mlp_predict(vb_ctx* ctx, const vb_mlp* mlp, const float* x, int32_t ld, int64_t n, float* y);
/* The same prediction on the tensor cores, as the radius-first kNN search evaluates it: 128 rows per
 * step, each layer one chain of tcgen05.mma (BF16 x BF16, FP32 accumulation in tensor memory), so the
 * inputs and hidden activations are rounded to BF16 (relative 2^-9) where vb_mlp_predict keeps FP32. */
vb_status vb_mlp_predict_tc(vb_ctx* ctx, const vb_mlp* mlp, const float* x, int32_t ld, int64_t n, float* y);

/* ------------------------------------------------- symmetric pattern (a6)
 * The sparsity pattern of the kernel matrices: the diagonal (Algorithm 1
 * starts its inner loop at j = i) united with every kNN pair in both
 * directions (K^ij = K^ji, Algorithm 1).  Rows are sorted by column; ed2
 * holds every stored entry's squared distance rounded to FP32 (0 on the
 * diagonal), bitwise symmetric. */

typedef struct {
    int64_t n;
    const int64_t* row_ptr;  /* n + 1 */
    const int32_t* col;      /* nnz */
    const float* ed2;        /* nnz */
} vb_graph;

size_t vb_graph_workspace(int64_t n, int32_t k);

/* nbr / nbr_d2 as written by vb_knn(): exact lists in (d2, index) order (the
 * construction decides whether a pair is mutual by comparing it with the other
 * point's k-th entry, which is only valid for such lists).  row_ptr: n + 1 int64;
 * col, ed2: cap entries, cap >= n * (2k + 1); nnz_dev: one int64 receiving nnz.
 * VB_ERR_UNSUPPORTED (reported) when a point lies in more than 8192 other lists
 * beyond its own neighbours. */
vb_status vb_graph_build(vb_ctx* ctx, int64_t n, int32_t k, const int32_t* nbr, const double* nbr_d2,
                         int64_t* row_ptr, int32_t* col, float* ed2, int64_t cap, int64_t* nnz_dev,
                         void* ws, size_t ws_bytes);

/* --------------------------------------------------------- bandwidth (a8)
 * Eq. (bandwidth parameter): b_i^2 = sum_{r=1}^{k_bw} d2(i, I(i, r)), summed in
 * rank order in FP64; b = sqrt(b^2).  nbr_d2: n x k with k_bw <= k.  A zero
 * b_i records VB_ERR_DEGENERATE in the report. */
vb_status vb_bandwidth(vb_ctx* ctx, int64_t n, int32_t k, int32_t k_bw, const double* nbr_d2, double* b);

/* -------------------------------------------------- epsilon sweep (a9, a11)
 * Sec. 2.3, Eq. (bandwidth sensitivity): with eps^2 = 2^xi on the grid
 * xi_g = xi_c + xi_lo + g * dxi (g = 0 .. G-1, G <= 64),
 *     chi_g  = sum_{(i,j) in E} exp(-ed2_ij / (scale * 2^xi_g * rho_i * rho_j)),
 *     chi'_g = (ln chi_{g+1} - ln chi_g) / (dxi ln 2),
 * g* = the first maximiser of chi', eps2 = 2^xi_{g*}, dim_est = 2 chi'_{g*}.
 * scale = 1 with rho = b gives the density sweep (K_eps); scale = 4 with
 * rho = P = psi^beta the operator sweep (K_{eps,beta}, rho = 2 psi^beta in
 * Algorithm 1).  xi_c_dev: optional device FP64 grid offset (NULL = 0).
 * Outputs (device FP64): eps2_dev[1], chi_dev[G], dim_est_dev[1].
 * warn_bit (1 or 2) is set in the report when g* is an end of the grid. */
size_t vb_epsilon_tune_workspace(int64_t n);
vb_status vb_epsilon_tune(vb_ctx* ctx, const vb_graph* g, const double* rho, double scale,
                          const double* xi_c_dev, double xi_lo, double xi_hi, double dxi, int32_t warn_bit,
                          double* eps2_dev, double* chi_dev, double* dim_est_dev, void* ws, size_t ws_bytes);

/* ---------------------------------------------------------- density (a10)
 * Eq. (density estimation): psi = W^-1 K_eps 1 with
 * K_eps^ij = exp(-ed2_ij / (eps^2 b_i b_j)), W_ii = n (pi eps^2 b_i^2)^(d/2);
 * P_i = psi_i^beta (Sec. 2.2).  eps2_dev: device FP64 scalar. */
size_t vb_density_workspace(int64_t n);
vb_status vb_density(vb_ctx* ctx, const vb_graph* g, const double* b, const double* eps2_dev, double d,
                     double beta, double* psi, double* P, void* ws, size_t ws_bytes);

/* Operator-sweep centre (the paper leaves the grid of the operator sweep
 * unstated; this library centres it):
 *     xi_c = round(4 log2(sum_E' ed2/(4 P_i P_j) / sum_E' ed2/(b_i b_j))) / 4,
 * E' = off-diagonal entries.  Writes one FP64 to xi_c_dev. */
size_t vb_operator_centre_workspace(int64_t n);
vb_status vb_operator_centre(vb_ctx* ctx, const vb_graph* g, const double* b, const double* P,
                             double* xi_c_dev, void* ws, size_t ws_bytes);

/* ------------------------------------------- operator and L-hat (a12-a13)
 * Sec. 2.2 in order: K_{eps,beta}^ij = exp(-ed2/(4 eps^2 P_i P_j)),
 * q_i = psi_i^(-beta d) sum_j K^ij, K~^ij = K^ij / (q_i q_j)^alpha with
 * alpha = (2 - c + (d + 2) beta) / 2 (from c = 2 - 2 alpha + d beta + 2 beta),
 * D_i = sum_j K~^ij, S_i = P_i D_i^(1/2), and the CSR values of
 *     L-hat = eps^-2 (S^-1 K~ S^-1 - P^-2)   (Eq. symmetric discrete Kolmogorov operator)
 * written as L-hat_ij = K~^ij / (eps^2 S_i S_j) off the diagonal and
 * L-hat_ii = -sum_{j != i} K~^ij / (eps^2 S_i^2) on it (the same value,
 * since S P^-2 S = D, without cancellation).  val is bitwise symmetric.
 * val: nnz FP32 in the graph's order; q, D, S: n FP64. */
typedef struct {
    double c;      /* Kolmogorov operator parameter */
    double beta;   /* variable-bandwidth exponent (the paper's examples use -1/4) */
    double d;      /* intrinsic dimension */
} vb_op_params;

size_t vb_kernel_csr_workspace(int64_t n);
vb_status vb_kernel_csr(vb_ctx* ctx, const vb_graph* g, const double* psi, const double* P,
                        const vb_op_params* op, const double* eps2_op_dev, float* val, double* q, double* D,
                        double* S, void* ws, size_t ws_bytes);

/* ------------------------------------------------------------- SpMV (a14)
 * y = alpha * A x + beta * y for the CSR matrix (g, val), one warp per row.
 * VB_SPMV_PLAIN uses every stored value.  VB_SPMV_LAPLACIAN applies L-hat in
 * difference form, y_i = alpha * sum_{j != i} val_ij S_j (x_j/S_j - x_i/S_i)
 * + beta y_i, which equals L-hat x because L-hat (S 1) = 0, and keeps the
 * accuracy of smooth vectors: the differences x_j/S_j - x_i/S_i are taken in
 * FP64 and the diagonal is not read.  S: n FP64, used in Laplacian mode only,
 * which also needs a workspace of vb_spmv_workspace(n) bytes (plain mode
 * accepts ws = NULL).  x, y: n FP32 (x and y must not alias). */
#define VB_SPMV_PLAIN     0
#define VB_SPMV_LAPLACIAN 1
size_t vb_spmv_workspace(int64_t n);
vb_status vb_spmv(vb_ctx* ctx, const vb_graph* g, const float* val, const double* S, int32_t mode,
                  float alpha, const float* x, float beta, float* y, void* ws, size_t ws_bytes);

/* Difference-form SpMV that allocates nothing and takes no workspace.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory, such as code that records an eigen-solver loop
 * into a CUDA graph (cudaMalloc is not allowed during stream capture) or a
 * host runtime that only lends this library buffers it already owns.  It
 * computes what vb_spmv() computes in VB_SPMV_LAPLACIAN mode, on the given
 * stream (a cudaStream_t; NULL = legacy default stream) of the current device.
 *   - Scratch: one static device array inside libvb, sized for
 *     VB_NOALLOC_MAX_N rows at 12 bytes per row (about 12.6 MB); every GPU
 *     that loads the library holds it until the process exits.
 *   - The first call on each device resolves the array's device address
 *     (cudaGetSymbolAddress, with that device current) and caches it; make
 *     that first call before any stream capture.  The cache is never
 *     refreshed: after cudaDeviceReset() (or any teardown of the device's
 *     primary context) the cached address is stale, so do not call this
 *     entry point in a process that has reset the device.
 *   - All calls share the one array and it keeps the last call's contents.
 *     Nothing in it has to start at zero (each call overwrites every row it
 *     reads), but calls whose work can overlap on the GPU (several streams,
 *     several host threads) race on it: the caller must serialise them.
 *   - g->n > VB_NOALLOC_MAX_N returns VB_ERR_UNSUPPORTED; use vb_spmv(). */
#define VB_NOALLOC_MAX_N 1048576
vb_status vb_spmv_laplacian_noalloc(void* stream, const vb_graph* g, const float* val, const double* S,
                                    float alpha, const float* x, float beta, float* y);

/* ------------------------------------ eigenpairs and spectral solve (boundary)
 * Sec. 2.2 and Sec. 4 step 3: the ell + 1 largest eigenvalues
 * 0 ~ lambda_0 > lambda_1 >= ... of L (those of L-hat, Eq. symmetric discrete
 * Kolmogorov operator) and the eigenvectors phi_j = S^-1 phi-hat_j, normalised
 * so that <phi_i, phi_j>_S = delta_ij with <f, g>_S = f^T S^2 g / n (Eq. inner
 * product), i.e. phi-hat_i^T phi-hat_j = n delta_ij.  Sec. 3.1 (Eqs. LS
 * minimiser and f_LS), when g_rhs and f are given: f = sum_{j=1..ell}
 * (<phi_j, g>_S / lambda_j) phi_j, lambda_0 excluded.
 * Method: block Chebyshev-filtered subspace iteration on L in the coordinates
 * z = S^-1 x, where (L z)_i = sum_{j != i} w_ij (z_j - z_i) with
 * w_ij = L-hat_ij S_j / S_i, so FP32 differences keep smooth vectors exact;
 * Rayleigh-Ritz in FP64 on the host.  Synchronises the host.
 * val, S: from vb_kernel_csr (cap = capacity of val); evals: ell + 1 FP64
 * (device); phi: (ell + 1) x n FP32 (device, eigenvector j contiguous) or
 * NULL; g_rhs, f: n FP32 (device) or NULL; iters: host int32 or NULL.
 * Returns VB_ERR_NOT_CONVERGED (outputs still written) when max_iter ran out. */
typedef struct {
    int32_t ell;        /* nonzero eigenpairs wanted (ell + 1 are computed), ell >= 1 */
    int32_t block;      /* subspace size, multiple of 32, <= 128 (0 = max(2 (ell + 1), ell + 17) rounded up to
                           a multiple of 32, capped at 128 while ell <= 111) */
    int32_t degree;     /* Chebyshev filter degree per iteration (0 = 30) */
    int32_t max_iter;   /* outer iterations (0 = 60) */
    double tol;         /* stop once the wanted Ritz values move by < tol * max |lambda_j| twice (0 = 1e-7) */
    uint64_t seed;      /* initial block */
} vb_solve_params;

size_t vb_solve_workspace(int64_t n, int64_t cap, const vb_solve_params* p);
vb_status vb_solve(vb_ctx* ctx, const vb_graph* g, int64_t cap, const float* val, const double* S,
                   const vb_solve_params* p, double* evals, float* phi, const float* g_rhs, float* f,
                   int32_t* iters, void* ws, size_t ws_bytes);

/* ------------------------------------------- gradients in the eigenbasis
 * Sec. 3.2 (Lemma Carre du Champ identity, Eqs. C_ijk and gradient of u): the
 * derivatives of a function u along every coordinate, from ell + 1 eigenpairs
 * of L (as written by vb_solve),
 *     du/dx_s = sum_{l,j,k=0..ell} u_j v_k (C_ljk / 2)(lambda_l - lambda_j - lambda_k) phi_l,
 * C_ljk = <phi_l, phi_j * phi_k>_S, u_j = <u, phi_j>_S, v_k = <x_s, phi_k>_S and
 * <f, g>_S = f^T S^2 g / n.  Computed without forming C: the sums over j and k
 * reduce exactly to projections of the products (sum_j u_j phi_j)(sum_k v_k phi_k)
 * and their lambda-weighted companions, O(ell n) per coordinate; FP32 products,
 * FP64 sums across 1024-sample chunks, reproducible run to run.
 * evals: ell + 1 FP64 (device); phi: (ell + 1) x n FP32 (device, eigenvector j
 * contiguous, phi_j = S^-1 phi-hat_j); S: n FP64 (device, from vb_kernel_csr);
 * u: n FP32 (device); x: n x m FP32 row-major (device, the samples, so that
 * v = x_s); grad: n x m FP32 row-major (device): grad[i m + s] = du/dx_s at x_i.
 * 1 <= m <= 128, 0 <= ell <= 1023; workspace from vb_gradient_workspace(). */
size_t vb_gradient_workspace(int64_t n, int32_t ell, int32_t m);
vb_status vb_gradient(vb_ctx* ctx, int64_t n, int32_t ell, const double* evals, const float* phi, const double* S,
                      const float* u, const float* x, int32_t m, float* grad, void* ws, size_t ws_bytes);

/* Diagnostic: one tensor-core tile (tcgen05.mma, kind::f16), d [128][N] = a [128][K] b [N][K]^T
 * with a and b rounded to BF16 and FP32 accumulation in tensor memory; K a multiple of 16 up
 * to 128, N a multiple of 32 up to 128; FP32 row-major device arrays.  The BF16 distance tiles
 * of the kNN search are built from the same primitives. */
vb_status vb_tc_dot_tile(vb_ctx* ctx, const float* a, const float* b, int32_t K, int32_t N, float* d);

/* ------------------------------------------------- the whole build (a0-a13)
 * One call for Sec. 4 steps 1-3 up to L-hat: kNN, pattern, bandwidth,
 * density sweep, density, operator-sweep centre, operator sweep, L-hat.
 * Every array is a caller-owned device buffer. */
typedef struct {
    vb_knn_params knn;
    int32_t k_bw;         /* neighbours in b (<= knn.k; 0 = knn.k) */
    vb_op_params op;
    double xi_lo, xi_hi, dxi;   /* sweep grid (the paper's parameterisation eps^2 = 2^xi) */
    int32_t pin_eps;      /* 1 = skip both sweeps and use *eps2_den / *eps2_op as given */
} vb_build_params;

typedef struct {
    int32_t* nbr;      double* nbr_d2;             /* n x k */
    double* b;                                     /* n */
    int64_t* row_ptr;  int32_t* col; float* ed2;   /* n + 1, cap, cap */
    int64_t cap;       int64_t* nnz;               /* cap >= n (2k + 1); nnz: 1 */
    double* eps2_den;  double* chi_den; double* dim_den;   /* 1, G, 1 */
    double* psi;       double* P;                  /* n, n */
    double* xi_c;                                  /* 1 */
    double* eps2_op;   double* chi_op;  double* dim_op;    /* 1, G, 1 */
    float* val;                                    /* cap */
    double* q;         double* D;       double* S; /* n, n, n */
} vb_build_out;

size_t vb_build_workspace(int64_t n, int32_t m, const vb_build_params* p);
vb_status vb_build(vb_ctx* ctx, const float* x, int64_t n, int32_t m, const vb_build_params* p,
                   const vb_build_out* out, void* ws, size_t ws_bytes);

/* ------------------------------------------------- batched build (a16)
 * B independent point clouds in one build: cloud b is the rows
 * [cloud_ptr[b], cloud_ptr[b + 1]) of x, and every step of vb_build is applied
 * to each cloud on its own (Sec. 4 steps 1-3 per cloud: neighbours only within
 * the cloud, its own n_b in the density, its own bandwidth sweeps).  Each stage
 * is one launch over all clouds: the kNN sorts by (cloud, Morton key) and each
 * query tile searches only the tiles of its clouds; every reduction is
 * segmented per cloud with a fixed order, so a cloud's results do not depend on
 * the other clouds beyond rounding order of its own sums.  No host
 * synchronisation happens inside, so the call can be recorded in a CUDA graph.
 *   cloud_ptr_host: B + 1 host int64 (read during the call for validation: 0 =
 *     cloud_ptr[0] < ... < cloud_ptr[B] = n, every n_b >= knn.k + 1);
 *   cloud_ptr_dev: the same values on the device (used by the kernels; it must
 *     stay valid until the work completes).
 * Outputs as in vb_build over all n points; the CSR is block-diagonal with global
 * column indices; eps2_den, dim_den, xi_c, eps2_op, dim_op hold B values and
 * chi_den, chi_op B x G (row b = cloud b).  With pin_eps, eps2_den / eps2_op
 * hold the B pinned values.  VB_ERR_ARG for an invalid cloud_ptr. */
size_t vb_build_batch_workspace(int64_t n, int32_t m, int32_t B, const vb_build_params* p);
vb_status vb_build_batch(vb_ctx* ctx, const float* x, int64_t n, int32_t m, const int64_t* cloud_ptr_host,
                         const int64_t* cloud_ptr_dev, int32_t B, const vb_build_params* p,
                         const vb_build_out* out, void* ws, size_t ws_bytes);

/* ------------------------------------------ the delta_tol radius pattern (Algorithm 1, Sec. 4)
 * The paper's own sparsity: an entry of a kernel matrix K^ij = exp(-d2_ij / (eps^2 rho_i rho_j))
 * is kept only where it exceeds delta_tol (Algorithm 1; Sec. 4 finds the candidates with a k-d
 * tree inside the critical radius R^2 = -eps^2 b_max^2 log(delta_tol)).  The test is evaluated
 * as t_ij < tau with t_ij = d2_ij / (eps^2 (rho_i rho_j)) (the product rho_i rho_j first, so the
 * pattern is symmetric bit for bit) and tau = -log(delta_tol) in FP64; d2 is the canonical FP64
 * squared distance of vb_knn; the diagonal is kept (t = 0).  The search runs on the kNN
 * search's Morton-ordered 64-point tiles and skips a tile pair when the gap of the two boxes
 * with the largest rho of each tile already fails the test (the critical radius per tile
 * pair); the pairs that remain are tested one by one, so the pattern is exact.
 *   x: n x m FP32 (device); rho: n FP64 (device, b for the density kernel, 2 psi^beta for the
 *   operator kernel); row_ptr: n + 1 int64; col: cap int32; d2: cap FP64 (rows sorted by
 *   column); nnz_dev: one int64.  A pattern with more than cap entries records
 *   VB_ERR_WORKSPACE in the report and leaves col and d2 unwritten; a row of more than 2048
 *   entries records VB_ERR_UNSUPPORTED and stays unsorted.  1 <= m <= 128. */
size_t vb_radius_workspace(int64_t n, int32_t m);
vb_status vb_radius_pattern(vb_ctx* ctx, const float* x, int64_t n, int32_t m, const double* rho, double eps2,
                            double delta_tol, int64_t* row_ptr, int32_t* col, double* d2, int64_t cap,
                            int64_t* nnz_dev, void* ws, size_t ws_bytes);
/* Eq. (bandwidth sensitivity) with the delta_tol pattern of every grid point: on the grid
 * xi_g = xi_lo + g dxi (G <= 64 points), chi_g = sum over the pairs (i, j) with
 * t_ij / 2^xi_g < tau of exp(-t_ij / 2^xi_g), t_ij = d2_ij / (scale (rho_i rho_j)), every
 * pair of the cloud considered (the diagonal adds n); then, as in vb_epsilon_tune, the first
 * maximiser g* of chi' gives eps2 = 2^xi_{g*} and dim_est = 2 chi'_{g*}.  FP64 sums in a fixed
 * order.  chi_dev: G FP64; eps2_dev, dim_est_dev: one FP64 each (device). */
vb_status vb_radius_sweep(vb_ctx* ctx, const float* x, int64_t n, int32_t m, const double* rho, double scale,
                          double xi_lo, double xi_hi, double dxi, double delta_tol, double* chi_dev, double* eps2_dev,
                          double* dim_est_dev, void* ws, size_t ws_bytes);

/* ------------------------------------------ particle evolution (Sec. 6)
 * One explicit step of the evolution of a time-dependent density (Sec. 6, Eq. SDE and
 * Eq. discrete sample evolution): the samples x of psi(.; t) move by
 *     x_next = x + dt (u - grad f) + sqrt(dt) sigma W,
 * where f solves the Kolmogorov problem L_{1,psi} f = g on the current samples (Eq.
 * advection-diffusion-Laplace): the whole build of vb_build with c = 1, the spectral solve
 * of vb_solve with ell eigenpairs (the constant mode dropped), and grad f by vb_gradient.
 * The source is centred on the samples, g - mean(g), the sample mean standing for the
 * expectation under psi(.; t).  The Gaussian draws W are inputs (the caller draws them), so
 * a step is a deterministic function of its arguments.  Synchronises the host (vb_solve).
 *   x, W, x_next: n x m FP32 row-major (device); u: n x m FP32 (device) or NULL (u = 0);
 *   sigma: m x m FP32 row-major (device); g: n FP32 (device);
 *   out: the build's caller-owned buffers, as for vb_build (p->build.op.c must be 1);
 *   f: n FP32 (device), the solution; grad: n x m FP32 (device), grad f at the samples.
 * Returns VB_ERR_NOT_CONVERGED (outputs still written) when the eigen-solver ran out of
 * iterations. */
typedef struct {
    vb_build_params build;   /* the operator of every step (op.c = 1: L_{1,psi}) */
    vb_solve_params solve;   /* eigenpairs of the spectral solve */
    double dt;               /* step length, > 0 */
} vb_evolve_params;

size_t vb_evolve_workspace(int64_t n, int32_t m, const vb_evolve_params* p);
vb_status vb_evolve_step(vb_ctx* ctx, const float* x, int64_t n, int32_t m, const vb_evolve_params* p,
                         const float* u, const float* sigma, const float* W, const float* g,
                         const vb_build_out* out, float* f, float* grad, float* x_next, void* ws, size_t ws_bytes);

#ifdef __cplusplus
}
#endif
#endif /* VB_H */

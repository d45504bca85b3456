/*
 * hyde.h -- C ABI of the GB300 HyRes library (libhyde.so).
 *
 * HyRes is the automatic, parameter-free, low-rank, wavelet-based Gaussian
 * denoiser for hyperspectral images packaged by HyDe (arXiv 2204.06979,
 * Sec. 2.1). This library runs its data-parallel path on one GPU:
 *
 *   Gram matrix -> per-band noise level by multiple regression -> whitening
 *   -> eigendecomposition (spectral subspace) -> rank-r_max projection ->
 *   per-component 2D db2 DWT -> SURE table over (rank, lambda) -> selection
 *   -> soft threshold + inverse DWT -> back-projection and un-whitening.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Cubes are band-major (BSQ): float[p][H][W], C-contiguous, in DEVICE
 *   memory. A pixel is one (y, x); n = H * W. The library reads the cube as
 *   the n x p matrix Y whose rows are pixels and columns are bands.
 * - Every pointer argument is device memory owned by the caller unless the
 *   comment says otherwise. The library never allocates or frees memory;
 *   scratch space is a caller-provided workspace whose size comes from the
 *   matching *_workspace_size query. Workspaces must be 256-byte aligned and
 *   must not be shared by calls that can run concurrently.
 * - Work is enqueued asynchronously on the given stream (0 = the legacy
 *   default stream); no entry point synchronises the host or reads device
 *   memory back. Results are valid once the stream has reached them.
 * - Argument errors detectable on the host return a status immediately and
 *   enqueue nothing. Errors only the device can see (NaN/Inf input, a Gram
 *   matrix that is not positive definite, a non-positive noise level) are
 *   written to a status word (hyde_hyres_info.status, or the status output of
 *   the stage call); the host reads it after synchronising.
 * - Sizes: 2 <= p <= 256 bands for the Gram and noise stages; the
 *   eigensolver and noise solve hold a p x p float matrix in one SM's shared
 *   memory, which bounds p (about 208 at r_max = 20, see hyde_workspace_size).
 *   1 <= levels <= 10; the padded sides H_p, W_p (H, W rounded up to
 *   multiples of 2^levels) need H_p - H <= H - 1 and W_p - W <= W - 1 (the
 *   reflection must stay inside the image).
 */
#ifndef HYDE_H
#define HYDE_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HYDE_OK = 0,
    HYDE_ERR_INVALID_ARG = 1,   /* null pointer, bad enum, misaligned buffer */
    HYDE_ERR_SHAPE = 2,         /* sizes outside the supported range        */
    HYDE_ERR_NUMERIC = 3,       /* NaN/Inf, non-SPD Gram, sigma <= 0        */
    HYDE_ERR_NOT_CONVERGED = 4, /* eigensolver iteration limit               */
    HYDE_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up        */
    HYDE_ERR_CUDA = 6,          /* a CUDA runtime call or launch failed      */
    HYDE_ERR_WORKSPACE = 7      /* workspace missing or too small            */
} hyde_status;

typedef enum {
    HYDE_PREC_FP32 = 0,    /* FP32-accurate arithmetic: the whole-path calls
                              take the Gram matrix as in HYDE_PREC_TF32X3
                              when its conditions hold (p a multiple of 4,
                              p <= 160, cube 16-byte aligned) and as FP32
                              SIMT products otherwise; every other stage in
                              FP32 SIMT. hyde_gram with this value is always
                              the SIMT kernel                                 */
    HYDE_PREC_TF32X3 = 1,  /* Gram matrix on the tensor cores, FP32-accurate:
                              each float is split into tf32 hi (rounded) +
                              lo = y - hi and y_a y_b is taken as
                              hi hi + hi lo + lo hi (tcgen05.mma kind::tf32,
                              TMEM windows of 64 pixels added into FP32
                              registers, double across SMs); needs p a
                              multiple of 4 and <= 160 and a 16-byte aligned
                              cube (HYDE_ERR_SHAPE / INVALID_ARG otherwise);
                              the other stages as in HYDE_PREC_FP32          */
    HYDE_PREC_BF16X3 = 2,  /* Gram matrix on the tensor cores: each float is
                              split into bf16 hi + lo and y_a y_b is taken as
                              hi hi + hi lo + lo hi (tcgen05.mma, FP32
                              accumulation in TMEM, double across SMs); the
                              other stages as in HYDE_PREC_FP32             */
    HYDE_PREC_BF16X3_ALL = 3 /* as HYDE_PREC_BF16X3, and the projection and
                              back-projection also as split-BF16 products on
                              the tensor cores (both are HBM-bound at ~10
                              flop/B, where the FP32 forms measure faster)   */
} hyde_precision;

/* How the SURE selection (Sec. 2.1, "parameter-free") assigns thresholds.
 * The paper leaves open whether the kept components share one threshold. */
typedef enum {
    HYDE_LAMBDA_SHARED = 0,        /* one lambda_{k*} for every kept component:
                                      (r*, k*) = argmin over the (r, k) table */
    HYDE_LAMBDA_PER_COMPONENT = 1, /* component i thresholded at its own
                                      lambda_{k_i}, k_i = argmin_k S_i(lambda_k)
                                      (first minimum); r* = argmin_r U(r) with
                                      U(r) = sum_{i<=r} S_i(lambda_{k_i})
                                             + sum_{r<i<=r_max} S_i(inf)
                                      (first minimum)                         */
    HYDE_LAMBDA_PER_LEVEL = 2      /* the detail bands of level l of component
                                      i thresholded at their own lambda_{k_il},
                                      k_il = argmin_k S_il(lambda_k), S_il the
                                      SURE of that group alone (the final LL
                                      band joins group L when threshold_ll);
                                      S*_i = (kept coefficients) + sum_l
                                      S_il(lambda_{k_il}) replaces S_i above.
                                      Needs 256 * levels * n_lambda bytes of
                                      shared memory <= 200 KiB                */
} hyde_lambda_mode;

/* Parameters of one HyRes run. */
typedef struct {
    int wavelet;    /* number of vanishing moments of the Daubechies filter;
                       2 (db2) is the only supported value                  */
    int levels;     /* DWT levels L, 1..10                                  */
    int r_max;      /* largest rank tried, 1..min(p, 32)                    */
    int n_lambda;   /* K threshold candidates, 2..256; 64 is the default    */
    int precision;  /* hyde_precision                                       */
    int lambda_mode;/* hyde_lambda_mode; HYDE_LAMBDA_SHARED is the default,
                       and the only mode of the scaled (differentiation)
                       entry points                                         */
    int threshold_ll;/* 0 (default): the final LL band is kept as is and
                       each of its coefficients adds 1 to SURE; 1: it is
                       soft-thresholded (at the component's threshold) and
                       counted in SURE like the detail bands. The paper
                       leaves this open; 0 only for the scaled entry points */
    int reserved;   /* must be zero                                         */
} hyde_hyres_params;

/* Outcome of one HyRes run, written by the device into caller memory. */
typedef struct {
    int status;        /* hyde_status seen on the device (HYDE_OK if none)   */
    int rank;          /* selected rank r*, 1..r_max                          */
    int lambda_index;  /* selected candidate k*, 0..K-1                       */
    int reserved;
    double lambda;     /* selected threshold lambda_{k*} (whitened units)     */
    double sure_min;   /* minimum total SURE                                  */
    double sure_gap;   /* (runner-up - minimum) / |minimum|                   */
} hyde_hyres_info;

/* Byte offsets of the intermediates hyde_hyres_denoise leaves in its
 * workspace (for inspection after the stream has finished). */
typedef struct {
    size_t total;      /* workspace bytes needed                            */
    size_t R;          /* double[p][p]   Gram matrix Y^T Y                  */
    size_t sigma;      /* double[p]      per-band noise std                  */
    size_t evals;      /* double[r_max]  leading eigenvalues of D^-1 R D^-1  */
    size_t V;          /* double[p][r_max] eigenvectors, row b = band b      */
    size_t coef;       /* float[r_max][H_p][W_p] wavelet coefficients        */
    size_t sure;       /* double[r_max][K] SURE of thresholding component i
                          (HYDE_LAMBDA_PER_LEVEL: double[r_max][levels][K],
                          S_il of each level group)                          */
    size_t sure_inf;   /* double[r_max]  SURE of dropping component i        */
    size_t sure_total; /* double[r_max][K] total SURE of rank r=i+1, lambda_k
                          (not written with HYDE_LAMBDA_PER_LEVEL)           */
    size_t status;     /* int            device status word                  */
    size_t lam_comp;   /* float[r_max][levels] threshold that each component's
                          detail bands of each level were soft-thresholded at
                          (HYDE_LAMBDA_PER_COMPONENT: row i < r* holds
                          lambda_{k_i} in every column; HYDE_LAMBDA_PER_LEVEL:
                          lambda_{k_il}; the other rows 0; not written with
                          HYDE_LAMBDA_SHARED)                                */
} hyde_ws_layout;

/* Human-readable name of a status code (static storage). */
const char* hyde_status_string(hyde_status s);

/* Library version as major*10000 + minor*100 + patch. */
int hyde_version(void);

/* ------------------------------------------------------------------ Gram
 * R = Y^T Y, the uncentred p x p Gram (covariance) matrix of the n x p
 * pixel-by-band matrix; the spectral statistics of the low-rank model
 * (Sec. 2.1, "low-rank"). Y is float[p][n] band-major (ld = n); R is
 * double[p][p] row-major, full symmetric. Per-block float partial sums are
 * combined in double. precision: HYDE_PREC_FP32 (FP32 FMA), HYDE_PREC_TF32X3
 * (split-TF32 products on the tensor cores, FP32-accurate; p a multiple of 4,
 * p <= 160, Y 16-byte aligned) or HYDE_PREC_BF16X3 (split-BF16 products on
 * the tensor cores).
 */
hyde_status hyde_gram_workspace_size(int p, long long n, int precision,
                                     size_t* bytes);
hyde_status hyde_gram(const float* Y, int p, long long n, int precision,
                      double* R, void* ws, size_t ws_bytes,
                      cudaStream_t stream);

/* Allocation-free Gram matrix, for callers that cannot allocate device
 * memory: code running where cudaMalloc is unavailable or forbidden (inside
 * a memory-budgeted host framework that owns every allocation, a real-time
 * loop that must not allocate) and that therefore cannot supply the
 * workspace hyde_gram needs. The paper has no counterpart; this is an
 * interface convenience. Same inputs and output as hyde_gram with
 * precision HYDE_PREC_FP32; the float partial sums go to one fixed
 * 16 MiB array in device global memory (hyde_gram_noalloc_scratch_bytes)
 * that every GPU loading the library holds until the process exits. The
 * grid is capped so the partials fit (fewer blocks for large p, never
 * fewer than one); p > 256 is rejected with HYDE_ERR_SHAPE. Every call
 * looks up the array's device address on the current device
 * (cudaGetSymbolAddress, no allocation), so the address stays right after
 * the caller resets the device; the first call on a device also loads the
 * library's device code there, so make that first call before any stream
 * capture. All
 * calls share the one array: calls that can overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Calls no cudaMalloc, cudaFree or allocating library routine.
 */
size_t hyde_gram_noalloc_scratch_bytes(void);
hyde_status hyde_gram_noalloc(const float* Y, int p, long long n, double* R,
                              cudaStream_t stream);

/* ------------------------------------------------------------ noise level
 * Per-band noise standard deviation by multiple regression of each band on
 * all other bands (least squares, no intercept): sigma_b^2 is the residual
 * sum of squares over n, i.e. 1 / (n [R^-1]_bb) (the HySime-style estimator
 * of Sec. 2.1). Y is float[p][H][W]; sigma is double[p]. The inverse is
 * formed in float by Gauss-Jordan on the diagonally scaled matrix and its
 * diagonal is corrected by one double-precision Newton step. status (device
 * int, may be NULL) receives HYDE_ERR_NUMERIC if R is not positive definite
 * or a sigma_b^2 is not positive.
 */
hyde_status hyde_noise_est_workspace_size(int p, int H, int W, size_t* bytes);
hyde_status hyde_noise_est(const float* Y, int p, int H, int W, double* sigma,
                           int* status, void* ws, size_t ws_bytes,
                           cudaStream_t stream);

/* ----------------------------------------------------------------- HySime
 * Signal-subspace identification (Sec. 2.1: the subspace step the paper
 * ships for FastHyDe and runs on GPUs; Bioucas-Dias and Nascimento, 2008).
 * The noise is each band's least-squares residual on all the other bands
 * (as in hyde_noise_est); R_y, R_n and R_x are the data, noise and signal
 * correlation matrices (uncentred, over n); the subspace holds the
 * eigenvectors e of R_x with delta = -e^T R_y e + 2 e^T R_n e < 0. Only
 * the Gram matrix touches the data: with Q = (Y^T Y)^-1 and D = diag(Q),
 * R_n = D^-1 Q D^-1 / n and R_x = (Y^T Y - 2 D^-1 + D^-1 Q D^-1) / n.
 * Y: float[p][n] band-major device, 2 <= p <= 256, n >= p. r_max: the
 * candidates, the leading eigenvectors of R_x, 1..min(p, 32) (the published
 * method ranks all p; eigenvectors past the leading ones carry the least
 * signal). Outputs (device): *k; idx int[r_max], the kept candidates in
 * ascending delta, then -1; E double[p][r_max], the candidates (column c,
 * descending eigenvalue; row b = band b); delta, evals double[r_max].
 * status: device int the caller zeroes (HYDE_ERR_NUMERIC for a singular or
 * non-finite matrix, or a refined inverse with a diagonal entry that is not
 * positive). Workspace: hyde_hysime_workspace_size.
 * When k == r_max < p every candidate lowered the error: the subspace may
 * be larger than the candidates cover, and k is then only a lower bound
 * (call again with a larger r_max, at most 32).
 */
hyde_status hyde_hysime_workspace_size(int p, long long n, int r_max,
                                       size_t* bytes);
hyde_status hyde_hysime(const float* Y, int p, long long n, int r_max, int* k,
                        int* idx, double* E, double* delta, double* evals,
                        int* status, void* ws, size_t ws_bytes,
                        cudaStream_t stream);

/* ----------------------------------------------------------- eigenvectors
 * Leading r eigenpairs of a symmetric positive semi-definite p x p matrix A
 * (double, row-major): the spectral subspace of the low-rank model
 * (Sec. 2.1). evals (double[r]) are in descending order; V is double[p][r]
 * (column i = eigenvector i); the entry of largest magnitude of each
 * eigenvector is positive. In float: Householder tridiagonalisation in one
 * thread block; then one block per eigenpair (multisection for the
 * eigenvalue, twisted-factorisation eigenvector, back-transformation); then
 * Cholesky QR (twice) of the r vectors in descending order (Gram-Schmidt
 * in exact arithmetic). status as above.
 * 2 <= p <= 256 (about 208 at r = 32, shared-memory bound), 1 <= r <=
 * min(p, 32); ws: hyde_eig_workspace_size bytes (the reflectors and the
 * unnormalised vectors travel between the kernels there).
 */
hyde_status hyde_eig_workspace_size(int p, int r, size_t* bytes);
hyde_status hyde_eig_sym_top(const double* A, int p, int r, double* evals,
                             double* V, int* status, void* ws, size_t ws_bytes,
                             cudaStream_t stream);

/* -------------------------------------------------------------------- DWT
 * L-level separable 2D periodic db2 analysis of a batch of images.
 * in: float[batch][H][W]; each image is first extended at the bottom and
 * right to H_p x W_p by whole-sample symmetric reflection
 * (x[M + j] = x[M - 2 - j]). coef: float[batch][H_p][W_p] in Mallat layout
 * (LL of the last level top-left; at each level the row-detail band is right
 * of LL, the column-detail band below it, the diagonal band diagonally).
 * One level: a_k = sum_m h_m x[(2k+m) mod M], d_k = sum_m g_m x[(2k+m) mod M]
 * along rows, then along columns, g_m = (-1)^m h_{3-m}.
 * hyde_idwt2 is the exact transpose (the inverse of the periodic transform)
 * followed by cropping to H x W. wavelet must be 2. These two calls have no
 * status word, so their tiles are gathered with cp.async only; inside the
 * HyRes path the interior tiles of each analysis level are TMA copies.
 */
hyde_status hyde_dwt_workspace_size(int batch, int H, int W, int levels,
                                    size_t* bytes);
hyde_status hyde_dwt2(const float* in, float* coef, int batch, int H, int W,
                      int wavelet, int levels, void* ws, size_t ws_bytes,
                      cudaStream_t stream);
hyde_status hyde_idwt2(const float* coef, float* out, int batch, int H, int W,
                       int wavelet, int levels, void* ws, size_t ws_bytes,
                       cudaStream_t stream);

/* --------------------------------------------------------------- SURE
 * Stein's unbiased risk estimate of soft-thresholding each coefficient image
 * (unit noise variance), on the candidate grid
 * lambda_k = k sqrt(2 ln N) / (K - 1), k = 0..K-1, N = H_p W_p:
 *   S[i][k] = N - 2 #{detail : |c| <= lambda_k}
 *             + sum_detail min(c^2, lambda_k^2)
 * (the LL band of the last level is kept and contributes 1 per coefficient),
 * and S_inf[i] = sum_all c^2 - N (the risk of dropping image i).
 * coef: float[batch][H_p][W_p] Mallat layout; S: double[batch][K];
 * S_inf: double[batch]. Counts are exact integers; sums of squares are
 * accumulated in float per thread and in double across blocks.
 */
hyde_status hyde_sure_workspace_size(int batch, int K, size_t* bytes);
hyde_status hyde_sure_table(const float* coef, int batch, int Hp, int Wp,
                            int levels, int K, double* S, double* S_inf,
                            void* ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------- whole HyRes
 * Denoise Y (float[p][H][W]) into X (float[p][H][W]; may not alias Y).
 * Rank r* in 1..r_max and threshold lambda_{k*} minimise the total SURE
 *   T(r, k) = sum_{i<=r} S_i(lambda_k) + sum_{r<i<=r_max} S_i(inf)
 * (ties: smallest r, then smallest k). info (device) receives the choice
 * and the device status; NULL is allowed. With lambda_mode
 * HYDE_LAMBDA_PER_COMPONENT each kept component i gets its own lambda_{k_i}
 * (see hyde_lambda_mode); info then holds r*, k_0 and lambda_{k_0} of the
 * first component, sure_min = U(r*) and sure_gap from the runner-up rank,
 * and the workspace's lam_comp table holds every component's threshold.
 * HYDE_LAMBDA_PER_LEVEL likewise, with k_00 (component 1, level 1) in info
 * and one threshold per (component, level) in lam_comp.
 * With threshold_ll = 1 the sums and counts of S run over all N
 * coefficients and the final LL band is thresholded as well.
 */
hyde_status hyde_workspace_size(int p, int H, int W,
                                const hyde_hyres_params* params,
                                size_t* bytes);
hyde_status hyde_workspace_layout(int p, int H, int W,
                                  const hyde_hyres_params* params,
                                  hyde_ws_layout* layout);
hyde_status hyde_hyres_denoise(const float* Y, float* X, int p, int H, int W,
                               const hyde_hyres_params* params,
                               hyde_hyres_info* info, void* ws,
                               size_t ws_bytes, cudaStream_t stream);

/* A stream of cubes in host memory: denoises count cubes Y_host[s] ->
 * X_host[s] (float[p][H][W] each, page-locked for the copies to overlap),
 * copying cube s+1 in and cube s-1 out while cube s is denoised. The copies
 * run on h2d and d2h (one cudaMemcpyAsync per cube and direction), the
 * denoise of every cube on `stream`, in order, with the one workspace ws
 * (as for hyde_hyres_denoise). dev: four device cubes owned by the caller,
 * input buffers dev[0], dev[1] and output buffers dev[2], dev[3], used in
 * turn; info_dev: two device info records; info_host: count page-locked
 * records that receive each cube's hyde_hyres_info, or NULL. events: seven
 * caller-created events (copy-in done, denoise done, copy-out done for each
 * buffer pair, and one fork event); a buffer is refilled only after the
 * work that read it has completed. The call forks the copy streams from
 * `stream` and joins them back to it: work queued on `stream` before the
 * call precedes all of it, and everything the call enqueues, copies
 * included, precedes later work on `stream`. Asynchronous; X_host[s] may
 * repeat when the caller does not read it in between. Returns the status
 * codes of hyde_hyres_denoise, or HYDE_ERR_CUDA if a copy or an event call
 * fails. (Sec. 2.1's HyRes per cube; the overlap is this library's.) */
hyde_status hyde_hyres_denoise_host(const float* const* Y_host, float* const* X_host,
                                    hyde_hyres_info* info_host, int count, int p, int H,
                                    int W, const hyde_hyres_params* params,
                                    float* const* dev, hyde_hyres_info* info_dev, void* ws,
                                    size_t ws_bytes, cudaStream_t stream, cudaStream_t h2d,
                                    cudaStream_t d2h, cudaEvent_t* events);

/* Stage boundaries of hyde_hyres_denoise_timed, in enqueue order. */
#define HYDE_N_STAGES 8   /* gram, noise, eig+weights, projection, DWT,
                             SURE+selection, threshold+IDWT, back-projection */

/* Same as hyde_hyres_denoise, and records events[0] before the first stage
 * and events[s+1] after stage s (HYDE_N_STAGES + 1 events created by the
 * caller) on the stream, so the caller can time each stage with
 * cudaEventElapsedTime after synchronising. For measurement only. */
hyde_status hyde_hyres_denoise_timed(const float* Y, float* X, int p, int H,
                                     int W, const hyde_hyres_params* params,
                                     hyde_hyres_info* info, void* ws,
                                     size_t ws_bytes, cudaStream_t stream,
                                     cudaEvent_t* events);

/* ------------------------------------------------- differentiation form
 * HyRes with learnable threshold scales: the paper's package makes several
 * conventional methods differentiable with autograd and puts a trainable
 * HyRes step in front of a DNN (Sec. 2.1, Sec. 2.2). The rank r* and base
 * threshold lambda* are chosen by SURE at scale = 1 and held fixed (no
 * gradient through the selection); the detail coefficients of component i
 * at level l are soft-thresholded at lambda* * scale[i][l].
 * scale: float[r_max][levels] device (row i = component i, rows >= r*
 * unused). Otherwise identical to hyde_hyres_denoise, including the
 * workspace, which the backward then reads. params must have lambda_mode
 * HYDE_LAMBDA_SHARED and threshold_ll 0 (HYDE_ERR_INVALID_ARG otherwise,
 * before any device work): the scales multiply one shared lambda* on the
 * detail bands. The same holds for the backward and its workspace query.
 */
hyde_status hyde_hyres_denoise_scaled(const float* Y, float* X, int p, int H,
                                      int W, const hyde_hyres_params* params,
                                      const float* scale, hyde_hyres_info* info,
                                      void* ws, size_t ws_bytes,
                                      cudaStream_t stream);

/* Gradient with respect to the scales, by the hand-written adjoint. fws is
 * the workspace of the preceding hyde_hyres_denoise(_scaled) call on the same
 * Y and params (read only: weights, rank, lambda*); bws is a separate scratch
 * (hyde_backward_workspace_size). The forward wavelet coefficients are
 * recomputed from Y, not stored.
 *   loss = 0: dX (float[p][H][W] device) is dL/dX_hat;
 *             dscale[i][l] = lambda* sum dC (-sign C) [|C| > lambda_il] over the
 *             level-l detail coefficients of component i, dC = DWT of the
 *             zero-embedded V^T D dX (the inverse DWT is orthogonal).
 *   loss = 1: the SURE of the kept components with per-level thresholds,
 *             sum_i [N - sum_l (2 #{|c| <= lambda_il} - sum min(c^2, lambda_il^2))],
 *             is written to *sure_value (device double, may be NULL) and
 *             dscale[i][l] = lambda* 2 lambda_il #{|c| > lambda_il} (the count
 *             term is piecewise constant; dX is ignored).
 * dscale: float[r_max][levels] device; rows >= r* are zero.
 */
hyde_status hyde_backward_workspace_size(int p, int H, int W,
                                         const hyde_hyres_params* params,
                                         size_t* bytes);
hyde_status hyde_hyres_backward(const float* Y, const float* dX, int p, int H,
                                int W, const hyde_hyres_params* params,
                                const float* scale, int loss, float* dscale,
                                double* sure_value, const void* fws,
                                size_t fws_bytes, void* bws, size_t bws_bytes,
                                cudaStream_t stream);

/* ------------------------------------------------------ several cubes at once
 * Denoises count independent cubes (Y[k] -> X[k], device pointers in host
 * arrays; each cube as hyde_hyres_denoise with the same shape and params)
 * over `slots` workspaces (1..16; ws[s], each hyde_workspace_size bytes,
 * 256-byte aligned): cube k runs on slot_streams[k % slots] with ws[k % slots],
 * so the cubes of different slots overlap on the GPU. Per cube, a third of
 * the work is single-block (the noise inverse and the eigensolver) and leaves
 * most SMs idle; another cube's bandwidth-bound stages fill them. The slot
 * streams are forked from `stream` (events[0]) and joined back to it
 * (events[1 + s]): work enqueued on `stream` afterwards sees every X[k].
 * info: device array of count records, or NULL. Cubes of the same slot run
 * in order on its stream. Asynchronous; no host synchronisation. On a
 * 349 x 1905 x 144 cube four slots measured fastest of one to four (0.54 ms
 * per cube against 0.88 ms one at a time). (No counterpart in the paper.)
 */
hyde_status hyde_hyres_denoise_many(const float* const* Y, float* const* X, int count, int p,
                                    int H, int W, const hyde_hyres_params* params,
                                    hyde_hyres_info* info, void* const* ws, size_t ws_bytes,
                                    int slots, cudaStream_t stream,
                                    const cudaStream_t* slot_streams, const cudaEvent_t* events);

/* ----------------------------------------------------------------- FORPDN
 * First-order spectral roughness penalty denoising (Sec. 2.1: a full-rank,
 * wavelet-based method for additive Gaussian noise; the paper states no
 * more). Reading: every band image is padded (whole-sample symmetric) and
 * transformed by the L-level periodic db2 DWT; the coefficient positions
 * form L + 1 groups (group 0 the final LL band, group l the detail positions
 * of level l); in group g every position's spectrum c (its p band
 * coefficients) becomes (I + lam_g D^T D)^-1 c, D the first difference
 * along the bands; lam_g is the first minimiser over the grid lam_0 = 0,
 * lam_m = 10^(-3 + 7 (m - 1) / (n_lambda - 2)) of Stein's unbiased risk
 * estimate under independent band noise of variance sigma_b^2 (the
 * regression noise estimate of the HyRes stage); the inverse DWT, cropped,
 * is written to X.
 * Y, X: float[p][H][W], device, may not alias. 2 <= p <= 256, H W >= p,
 * 1 <= levels <= 10 (sides padded as for hyde_hyres_denoise),
 * 2 <= n_lambda <= 256. info (device int[levels + 2], or NULL): info[0] the
 * status seen on the device (HYDE_OK if none), info[1 + g] the chosen grid
 * index of group g. sure (device double[levels + 1][n_lambda], or NULL):
 * the SURE table. ws: hyde_forpdn_workspace_size bytes, 256-byte aligned.
 * Asynchronous on stream; no host synchronisation.
 */
hyde_status hyde_forpdn_workspace_size(int p, int H, int W, int levels, int n_lambda,
                                       size_t* bytes);
hyde_status hyde_forpdn(const float* Y, float* X, int p, int H, int W, int levels,
                        int n_lambda, int* info, double* sure, void* ws, size_t ws_bytes,
                        cudaStream_t stream);

/* ------------------------------------------------------------------ WSRRR
 * Wavelet-based sparse reduced-rank regression (Sec. 2.1: a low-rank,
 * wavelet-based method for Gaussian noise that also extracts features; the
 * paper states no more). Reading: on the whitened cube Yw (the bands
 * divided by the HyRes noise estimate, padded by whole-sample symmetric
 * extension, one row per padded pixel) the model Yw ~ W2 B V^T (W2 the
 * orthogonal L-level db2 synthesis of r component images, B their wavelet
 * coefficients, V^T V = I) and the objective
 * 1/2 ||Yw - W2 B V^T||^2 + lambda |B without the final LL band|_1,
 * decreased by cyclic descent from HyRes's basis, rank r* and threshold
 * lambda*: iters times B <- soft(W2^T Yw V, lambda) (the HyRes projection,
 * analysis and thresholded synthesis), V <- polar(Yw^T W2 B) (orthogonal
 * Procrustes, in double); then a last B-step. X = sigma_b (W2 B V^T),
 * cropped; iters = 0 gives HyRes's estimate.
 * params as for hyde_hyres_denoise with lambda_mode HYDE_LAMBDA_SHARED,
 * threshold_ll 0, precision HYDE_PREC_FP32 or HYDE_PREC_TF32X3, r_max <= 32;
 * 0 <= iters <= 1000. info: HyRes's choice (r*, lambda index) and the
 * device status. features (device float[r_max][H_p][W_p], or NULL): the
 * final component images W2 B on the padded domain (rows >= r* zero).
 * ws: hyde_wsrrr_workspace_size bytes, 256-byte aligned. Asynchronous.
 */
hyde_status hyde_wsrrr_workspace_size(int p, int H, int W, const hyde_hyres_params* params,
                                      size_t* bytes);
hyde_status hyde_wsrrr(const float* Y, float* X, int p, int H, int W,
                       const hyde_hyres_params* params, int iters, hyde_hyres_info* info,
                       float* features, void* ws, size_t ws_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------- HyMiNoR
 * Mixed Gaussian and sparse noise reduction built on HyRes (Sec. 2.1: after
 * HyRes removes the Gaussian noise, an l1-l1 problem solved by a modified
 * split-Bregman iteration removes the remaining sparse noise). The paper
 * states neither; this library's reading: G = HyRes(Y) (params as for
 * hyde_hyres_denoise, info receives its choice); per band image the problem
 *   min_x ||G/s - x||_1 + lam (||Dx x||_1 + ||Dy x||_1),  s = max |G|,
 * Dx, Dy periodic forward differences along rows and columns; split Bregman
 * on A = G/s - x, Bx = Dx x, By = Dy x with penalty mu (thresholds 1/mu and
 * lam/mu), from x = G/s and zero splitting variables, the x-subproblem
 * (5 x - sum of the 4 neighbours = rhs) solved by two Jacobi sweeps from
 * the current x, `iters` iterations; X = s x. Defaults in the binding:
 * lam = 1, mu = 10, iters = 50. Y, X: float[p][H][W] device, X may not
 * alias Y. lam >= 0, mu > 0 (HYDE_ERR_INVALID_ARG otherwise), 1 <= iters
 * <= 100000. Workspace: hyde_hyminor_workspace_size (the HyRes workspace
 * plus nine cube-sized float buffers: G and two sets of iteration state).
 */
hyde_status hyde_hyminor_workspace_size(int p, int H, int W,
                                        const hyde_hyres_params* params,
                                        size_t* bytes);
hyde_status hyde_hyminor(const float* Y, float* X, int p, int H, int W,
                         const hyde_hyres_params* params, float lam, float mu,
                         int iters, hyde_hyres_info* info, void* ws,
                         size_t ws_bytes, cudaStream_t stream);

/* ------------------------------------------------------- sliding windows
 * Batched form: the scene Y (float[p][H][W]) is cut into windows, each
 * denoised with its own noise levels, subspace, rank and threshold, and X
 * takes every pixel from the window whose core holds it. The paper denoises
 * images too large for one pass by slicing them into tiles and reassembling
 * the results (Sec. 2.2.2). win (HOST memory) lists the windows; the cores
 * must tile the scene (not checked: pixels outside every core are left
 * untouched in X). info (device, may be NULL) receives one record per
 * window. Windows go round-robin to n_slots slots; slot s works on
 * streams[s] (caller-created) with its own part of ws
 * (hyde_windows_workspace_size). events holds n_slots + 1 caller-created
 * events used to fork the slot streams from `stream` and join them back, so
 * the call behaves as one operation on `stream` and can be captured into a
 * single CUDA graph.
 */
typedef struct {
    int y0, x0, h, w;       /* window in scene pixels                       */
    int cy0, cx0, ch, cw;   /* its core (inside the window)                 */
} hyde_window;

hyde_status hyde_windows_workspace_size(int p, int H, int W,
                                        const hyde_window* win, int n_win,
                                        const hyde_hyres_params* params,
                                        int n_slots, size_t* bytes);
hyde_status hyde_hyres_denoise_windows(const float* Y, float* X, int p, int H,
                                       int W, const hyde_window* win,
                                       int n_win,
                                       const hyde_hyres_params* params,
                                       hyde_hyres_info* info, void* ws,
                                       size_t ws_bytes,
                                       const cudaStream_t* streams,
                                       int n_slots, cudaEvent_t* events,
                                       cudaStream_t stream);

/* ----------------------------------------------- batched sliding windows
 * The same form with one launch per stage over all windows (Sec. 2.2.2:
 * the tiles of a large scene, each denoised on its own by HyRes, Sec. 2.1):
 * the Gram matrices of all windows on the tensor cores (split-BF16, the
 * windows read in place from the scene), a one-block Gauss-Jordan and
 * eigensolver per window, the projection, the DWT, SURE and its selection,
 * the thresholded inverse DWT and the back-projection of the cores, each a
 * single launch over every window (12 kernels per group of windows; the
 * windows form two groups, each run on its own stream, so 24 for a scene).
 *
 * Differences from hyde_hyres_denoise on the window's cube: the Gram matrices
 * come from a four-term split-BF16 product on the tensor cores (every
 * product term exact, an unbiased 2^-18 split residual; FP32-accurate like
 * the split-TF32 kernel), sigma from the float Gauss-Jordan inverse without
 * the FP64 Newton step (that step is p^3 double FMAs per window; its effect
 * on a window's output is ~1e-5 relative at p = 200), and only the
 * shared-lambda mode with the LL band kept (lambda_mode HYDE_LAMBDA_SHARED,
 * threshold_ll 0) with precision HYDE_PREC_FP32 or HYDE_PREC_TF32X3 (the
 * same path) is accepted.
 *
 * A plan holds the window table and the layout of the workspace. Create it
 * once per table (host only; copies win), query its workspace size, and run
 * it any number of times; every call first copies the plan's tables (held in
 * page-locked host memory) into the workspace on `stream`, so a call can be
 * captured into a CUDA graph and replayed while the plan lives. Limits:
 * 1 <= p <= 208, W a multiple of 4, every window's x0 a multiple of 4 and
 * its padded sides (multiples of 2^levels) shorter than twice its sides,
 * at most 65535 windows; HYDE_ERR_SHAPE otherwise (hyde_hyres_denoise_windows
 * takes any table). Y (16-byte aligned) and X: float[p][H][W] device, X may
 * not alias Y; info (device, may be NULL): one record per window.
 */
typedef struct hyde_windows_plan_s* hyde_windows_plan;

hyde_status hyde_windows_plan_create(int p, int H, int W, const hyde_window* win,
                                     int n_win, const hyde_hyres_params* params,
                                     hyde_windows_plan* plan);
hyde_status hyde_windows_plan_workspace_size(hyde_windows_plan plan, size_t* bytes);
/* Kernels one hyde_hyres_denoise_windows_batched call launches (-1 if NULL). */
int hyde_windows_plan_kernel_launches(hyde_windows_plan plan);
hyde_status hyde_windows_plan_destroy(hyde_windows_plan plan);
/* Byte offsets of intermediates a batched call leaves in its workspace, for
 * inspection after the stream has finished: R double[n_win][p][p] (each
 * window's Gram matrix), sigma double[n_win][p], V double[n_win][p][r_max]. */
typedef struct {
    size_t R;
    size_t sigma;
    size_t V;
} hyde_windows_ws_layout;
hyde_status hyde_windows_plan_layout(hyde_windows_plan plan, hyde_windows_ws_layout* out);
/* Tuning of the batched form: the projection tile (padded pixels per block, a
 * multiple of 256 up to 4096) and the weight of the window Gram's second band
 * role when it splits the CTAs between its two roles (p > 128; > 0, up to
 * 16). The defaults, 256 and 1.6, measured best on the 2048 x 2048 x 200
 * scene. hyde_windows_plan_autotune times every candidate (tiles 256, 512,
 * 1024 x weights 1.2, 1.6, 2.0) on the caller's scene with
 * hyde_hyres_denoise_windows_batched (an untimed call, then the median of
 * three), keeps the fastest and reports its time in *best_ms (may be NULL);
 * it synchronizes `stream` and may not run while the stream is being
 * captured. Change the tuning only while no call of the plan is in flight,
 * and capture graphs again afterwards: a captured call keeps the grid sizes
 * of the tuning it was captured with. HYDE_ERR_INVALID_ARG for values out of
 * range. (No counterpart in the paper.) */
hyde_status hyde_windows_plan_set_tuning(hyde_windows_plan plan, int proj_tile,
                                         double gram_role_weight);
hyde_status hyde_windows_plan_get_tuning(hyde_windows_plan plan, int* proj_tile,
                                         double* gram_role_weight);
hyde_status hyde_windows_plan_autotune(hyde_windows_plan plan, const float* Y, float* X,
                                       void* ws, size_t ws_bytes, cudaStream_t stream,
                                       float* best_ms);
hyde_status hyde_hyres_denoise_windows_batched(const float* Y, float* X,
                                               hyde_windows_plan plan,
                                               hyde_hyres_info* info, void* ws,
                                               size_t ws_bytes, cudaStream_t stream);

/* Caps, for the calling host thread, the SM count that the launchers size
 * their grids from (0 removes the cap); returns the previous cap. For many
 * small pipelines on concurrent streams: multi-block kernels sized for
 * every SM keep the one-block kernels of the other streams from finding a
 * free SM. A workspace sized without the cap stays large enough. */
int hyde_set_grid_sm_cap(int sms);

/* Sets, for the calling host thread, the time limit of the bounded
 * mbarrier waits in the main loop of the tensor-core Gram kernels (0
 * restores the default of one second); returns the previous setting. When a
 * wait runs out the kernel stops its loop, writes HYDE_ERR_TIMEOUT to the
 * status word of the call (hyde_hyres_info.status for the whole path),
 * waits at most one second more for its own tensor-core work in flight,
 * frees its tensor memory and returns; its Gram output is then zero and the
 * CUDA context stays usable. The same limit bounds the waits for the TMA
 * copies of the wavelet analysis inside the HyRes, WSRRR and FORPDN calls:
 * a block whose copy runs out writes HYDE_ERR_TIMEOUT, lets its copies in
 * flight land (at most one second) and stops, leaving its tiles of the
 * coefficients unwritten. Meant for testing those paths: the default suits
 * every supported size. (No counterpart in the paper.) */
unsigned long long hyde_set_wait_limit_ns(unsigned long long ns);

/* Number of kernels one hyde_hyres_denoise call launches on a p x H x W
 * cube: 12 + 2 * (DWT launches), a DWT launch per level, except that the
 * coarse levels run fused in one launch (20 at 349 x 1905, 5 levels). The
 * memsets are not counted: one clears the workspace header, and the SIMT
 * and split-BF16 Gram clear R before their reduction (the split-TF32 Gram
 * writes R whole). -1 for bad params or shapes. */
int hyde_hyres_kernel_launches(int p, int H, int W, const hyde_hyres_params* params);

#ifdef __cplusplus
}
#endif

#endif /* HYDE_H */

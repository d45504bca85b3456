// Internal declarations shared by the libhyde translation units.
// Every kernel of the HyRes path (arXiv 2204.06979, Sec. 2.1) is launched
// through one of the host launchers declared here; the extern "C" layer in
// abi.cu validates arguments, carves the caller's workspace and calls them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>
#include <vector>

#include "../../include/hyde.h"

namespace hyde {

// ---------------------------------------------------------------- limits
constexpr int kMaxBandsGram = 256;   // p bound of the Gram kernel (8x8 tiles)
constexpr int kMaxRank = 32;         // r_max bound (one warp per eigenpair)
constexpr int kMaxLambda = 256;      // K bound of the SURE table
constexpr int kMaxLevels = 10;
constexpr size_t kAlign = 256;       // workspace carve alignment

// ------------------------------------------------------- db2 filter taps
// Daubechies' orthonormal scaling filter with two vanishing moments, from its
// closed form h = (1+r3, 3+r3, 3-r3, 1-r3) / (4 r2); wavelet filter
// g_m = (-1)^m h_{3-m}.
constexpr double kR3 = 1.7320508075688772935274463;
constexpr double kR2 = 1.4142135623730950488016887;
constexpr float kH0 = (float)((1.0 + kR3) / (4.0 * kR2));
constexpr float kH1 = (float)((3.0 + kR3) / (4.0 * kR2));
constexpr float kH2 = (float)((3.0 - kR3) / (4.0 * kR2));
constexpr float kH3 = (float)((1.0 - kR3) / (4.0 * kR2));
constexpr float kG0 = kH3;
constexpr float kG1 = -kH2;
constexpr float kG2 = kH1;
constexpr float kG3 = -kH0;

// ---------------------------------------------------------------- helpers
__host__ __device__ inline size_t align_up(size_t x, size_t a) {
    return (x + a - 1) / a * a;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Two FP32 FMAs in one instruction (c0 += a0 b0, c1 += a1 b1, each rounded
// once): halves the issue slots of the FMA-heavy loops.
__device__ __forceinline__ void fma_f32x2(float& c0, float& c1, float a0, float a1, float b0,
                                          float b1) {
    asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%0, %1};\n\t"
        "fma.rn.f32x2 rc, ra, rb, rc;\n\t"
        "mov.b64 {%0, %1}, rc;\n\t}"
        : "+f"(c0), "+f"(c1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// double -> float from the IEEE-754 bit fields on the integer pipes (FP64
// arithmetic and conversions run at a small fraction of the FP32 rate on
// this part): sign, exponent rebased from 1023 to 127, the top 23 of the 52
// mantissa bits rounded to nearest (ties away from zero; a carry into the
// exponent is the correct result). Values below the float normal range give
// a signed zero, values above it (and inf, NaN) give inf.
__device__ __forceinline__ float d2f_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    unsigned bits = ((unsigned)e << 23) + m + ((lo >> 28) & 1u);
    if (e <= 0) bits = 0u;
    if (e >= 255 || bits >= 0x7f800000u) bits = 0x7f800000u;
    return __int_as_float((int)(sign | bits));
}

__device__ __forceinline__ void set_status(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// ------------------------------------------- programmatic dependent launch
// Every kernel is launched with programmatic stream serialisation: its blocks
// may be scheduled while the previous kernel on the stream is still running,
// which hides the launch and ramp-up between the dependent kernels of the
// path. Each kernel therefore begins with pdl_wait(), which returns once the
// previous grid has completed and its writes are visible (at once when there
// is none), before it touches global memory; pdl_trigger() then lets the next
// kernel's blocks be scheduled. Because the trigger comes after the wait, at
// most one grid waits behind a running one, and that running grid has every
// block resident, so the waiting blocks cannot hold resources it needs.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launches from one host thread use the attribute unless a PdlOff guard is
// alive on that thread: the sliding-window form runs dozens of small
// pipelines on concurrent streams, where blocks resident ahead of their
// predecessor take SM room from the other streams' running kernels.
extern thread_local bool tl_pdl;
struct PdlOff {
    bool prev;
    PdlOff() : prev(tl_pdl) { tl_pdl = false; }
    ~PdlOff() { tl_pdl = prev; }
};

// Grids are sized from device_sm_count(); while an SmCap guard is alive on a
// host thread that count is capped, which the sliding-window form uses so
// that each window's multi-block kernels leave SMs free for the one-block
// kernels of the other windows.
extern thread_local int tl_sm_cap;

// Time limit of the bounded mbarrier waits in the main loop of the
// tensor-core Gram kernel, for kernels launched from this host thread
// (0: the default, one second). A shorter limit exists to exercise the
// timeout path; see hyde_set_wait_limit_ns.
extern thread_local unsigned long long tl_wait_ns;
inline unsigned long long wait_limit_ns() { return tl_wait_ns ? tl_wait_ns : 1000000000ull; }

struct SmCap {
    int prev;
    explicit SmCap(int cap) : prev(tl_sm_cap) { tl_sm_cap = cap; }
    ~SmCap() { tl_sm_cap = prev; }
};

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args&&... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = tl_pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Number of SMs of the current device (cached per device).
int device_sm_count();

// Sets the dynamic shared-memory limit of a kernel once per device.
cudaError_t ensure_smem_limit(const void* func, int bytes);

inline hyde_status cuda_status(cudaError_t e) {
    return e == cudaSuccess ? HYDE_OK : HYDE_ERR_CUDA;
}

// ----------------------------------------------------------------- Gram
struct GramPlan {
    int mode;        // 0: 8x8 tiles, FFMA; 1: 8x4 tiles, paired FP32 FMA (f32x2)
    int PT;          // 8-band tile rows
    int ntiles;      // upper-triangle tiles
    int threads;     // threads per block
    int blocks;      // blocks in the grid
    size_t smem;     // dynamic shared memory per block
    size_t partial_bytes;
};
hyde_status gram_plan(int p, long long n, GramPlan* plan);
hyde_status launch_gram(const float* Y, int p, long long n, const GramPlan& plan,
                        float* partials, double* R, int* status,
                        cudaStream_t s);

// Split-BF16 (hi*hi + hi*lo + lo*hi) Gram on the tensor cores (tcgen05.mma,
// accumulators in TMEM); per-SM float partials p x p, summed in double.
hyde_status gram_tc_partial_bytes(int p, size_t* bytes);
// Split-TF32 (hi*hi + hi*lo + lo*hi) Gram on the tensor cores, FP32-accurate:
// TMA loads, TMEM windows of 64 pixels drained into FP32 registers. Needs p a
// multiple of 4, 4 <= p <= 160 and Y 16-byte aligned; partials as for
// launch_gram_tc (gram_tc_partial_bytes).
bool gram_tf32_shape_ok(int p, long long n);
bool gram_tf32_supported(const float* Y, int p, long long n);
hyde_status launch_gram_tf32(const float* Y, int p, long long n, float* partials, double* R,
                             int* status, cudaStream_t s);
hyde_status launch_gram_tc(const float* Y, int p, long long n, float* partials, double* R,
                           int* status, cudaStream_t s);

// ------------------------------------------------------- small dense LA
size_t noise_ws_bytes(int p);
hyde_status launch_noise_from_gram(const double* R, int p, long long n,
                                   double* sigma, void* ws, int* status,
                                   cudaStream_t s);
// Q = R^-1 (double[p][p], column b refined in double by one Newton step
// from the float Gauss-Jordan inverse; ws as for launch_noise_from_gram).
hyde_status launch_inverse_from_gram(const double* R, int p, void* ws, double* Q, int* status,
                                     cudaStream_t s);
size_t eig_smem_bytes(int p, int r);   // largest dynamic smem of the three eig kernels
size_t eig_ws_bytes(int p, int r);     // workspace of launch_eig_top (16-byte aligned)
size_t noise_smem_bytes(int p);   // dynamic smem of the Gauss-Jordan kernel (0 = registers)
// Leading r eigenpairs (descending) of A, whitened on load by wsig (NULL: no
// whitening): evals double[r], V double[p][r]; ws holds eig_ws_bytes(p, r).
hyde_status launch_eig_top(const double* A, const double* wsig, int p,
                           int r, double* evals, double* V, void* ws, int* status,
                           cudaStream_t s);
// P[b][i] = V[b][i] / sigma_b and Q[b][i] = V[b][i] * sigma_b (float,
// row stride ldw, zero for i >= r)
hyde_status launch_weights(const double* V, const double* sigma, int p, int r,
                           int ldw, float* P, float* Q, cudaStream_t s);

// ------------------------------------------------- projection / back
// zero_pad: the padding is zero (the transpose of cropping) instead of the
// symmetric reflection of the image
hyde_status launch_project_pad(const float* Y, int p, int H, int W,
                               const float* P, int r, int ldw, float* Zp,
                               int Hp, int Wp, cudaStream_t s, bool zero_pad = false);
hyde_status launch_backproject(const float* Zh, long long n, const float* Q,
                               int p, int r_max, int ldw, const int* rank,
                               float* X, cudaStream_t s);
// Split-BF16 tcgen05 versions (precision form): the same contractions with
// the pixels on the MMA's M. Supported for p <= 256 and r_max <= 32.
bool project_tc_supported(int p, int r_max);
hyde_status launch_project_pad_tc(const float* Y, int p, int H, int W, const float* P, int r,
                                  int ldw, float* Zp, int Hp, int Wp, int* status,
                                  cudaStream_t s);
hyde_status launch_backproject_tc(const float* Zh, long long n, const float* Q, int p, int ldw,
                                  const int* rank, float* X, int* status, cudaStream_t s);

// ------------------------------------------------------------------ DWT
// Source of the first analysis level: the image is read at (y, x) of the
// padded domain through whole-sample symmetric reflection at hv, wv.
// Padded sides for an L-level transform: multiples of 2^L that whole-sample
// symmetric extension can reach (at most H - 1 rows and W - 1 columns
// added); false for unsupported shapes.
inline bool padded_dims(int H, int W, int levels, int* Hp, int* Wp) {
    if (levels < 1 || levels > kMaxLevels || H < 1 || W < 1) return false;
    const int q = 1 << levels;
    const long long hp = ((long long)H + q - 1) / q * q, wp = ((long long)W + q - 1) / q * q;
    if (hp > (1 << 30) || wp > (1 << 30)) return false;
    if (hp - H > H - 1 || wp - W > W - 1) return false;
    *Hp = (int)hp;
    *Wp = (int)wp;
    return true;
}

struct DwtSrc {
    const float* ptr;
    long long bstride;
    int ld;
    int hv, wv;
};
size_t dwt_scratch_floats(int Hp, int Wp);
// kernel launches of launch_dwt2 / launch_idwt2 on a padded Hp x Wp image (aligned buffers)
int dwt_launches(int Hp, int Wp, int levels);   // per image, both ping-pong halves
// status (may be NULL): receives HYDE_ERR_TIMEOUT if a TMA copy of an
// interior tile does not complete within the wait limit; without it every
// tile is gathered with cp.async.
hyde_status launch_dwt2(const DwtSrc& src, float* coef, int batch, int Hp,
                        int Wp, int levels, float* scratch, cudaStream_t s,
                        int* status = nullptr);
// Synthesis with optional soft threshold of detail coefficients at *lam
// (times scale[image * scale_ld + level - 1] when scale != NULL) and an
// optional rank limit (*rank images are processed; NULL = all). ll_thr: the
// final LL band is thresholded too, at the last level's threshold.
hyde_status launch_idwt2(const float* coef, float* out, int batch, int Hp,
                         int Wp, int H, int W, int levels, float* scratch,
                         const double* lam, const int* rank, cudaStream_t s,
                         const float* scale = nullptr, int scale_ld = 0,
                         bool ll_thr = false);

// ------------------------------------------------------------------ WSRRR
// M (double [p][ldm]) = Yw^T Xr over the padded pixels (Yw = the cube read
// through the symmetric extension, divided by sigma_b; Xr = the first
// *rank_dev of the RM padded component images); partials: nblocks x p x RM
// floats (wsrrr_cross_partial_bytes).
hyde_status launch_wsrrr_cross(const float* Y, int p, int H, int W, const float* Xr, int RM,
                               int Hp, int Wp, const int* rank_dev, const double* sigma,
                               float* partials, int nblocks, double* M, int ldm, int* status,
                               cudaStream_t s);
size_t wsrrr_cross_partial_bytes(int p, int RM, int nblocks);
// V[:, :r] (double [p][ldv]) = the orthonormal polar factor of M[:, :r],
// r = *rank_dev <= 32, in double.
hyde_status launch_wsrrr_polar(const double* M, int p, int ldm, const int* rank_dev, double* V,
                               int ldv, int* status, cudaStream_t s);

// ------------------------------------------------- differentiation form
// acc[i][l] (double, zeroed by the caller) += per-(component, level) sums over
// the detail coefficients of components i < *rank:
//   mode 0: dC * (-sign C) * [|C| > lam_il]         (needs dC)
//   mode 1: 2 lam_il [|C| > lam_il]; sure_acc += -2 [|C| <= lam_il] + min(C^2, lam_il^2)
// with lam_il = *lam * scale[i * scale_ld + l - 1].
hyde_status launch_scale_grad(const float* C, const float* dC, int r_max, int Hp, int Wp,
                              int levels, const int* rank, const double* lam,
                              const float* scale, int scale_ld, int mode, double* acc,
                              double* sure_acc, cudaStream_t s);
// dscale[i][l] = (float)(lam * acc[i][l]) for i < rank, 0 otherwise; in mode 1
// *sure_value = rank * N + sure_acc.
hyde_status launch_scale_grad_finish(const double* acc, int r_max, int levels,
                                     const int* rank, const double* lam, float* dscale,
                                     int dscale_ld, int mode, long long N,
                                     const double* sure_acc, double* sure_value,
                                     cudaStream_t s);

// ------------------------------------------------------- sliding windows
hyde_status launch_gather_window(const float* Y, int H, int W, int y0, int x0, int h, int w,
                                 int p, float* out, cudaStream_t s);
hyde_status launch_scatter_core(const float* cube, int h, int w, int y0, int x0, int cy0,
                                int cx0, int ch, int cw, int p, int H, int W, float* X,
                                cudaStream_t s);

// ------------------------------------------- batched sliding windows
// One window of a batched call as its kernels see it (a device table). The
// window's r_max component images (padded Hp x Wp) start at float offset
// `img` of the component and coefficient buffers, its DWT scratch at `scr`.
struct WinDesc {
    int y0, x0, h, w;         // window in scene pixels
    int cy0, cx0, ch, cw;     // its core, in scene pixels
    int Hp, Wp;               // padded component images
    int sh, pad_;             // SURE fixed-point unit 2^-sh
    long long img;
    long long scr;
    double delta;             // SURE grid step sqrt(2 ln N) / (K - 1), N = Hp Wp
};

// Floats of DWT scratch per component image of N = Hp Wp values (the LL
// bands of two consecutive levels, rounded to 16 bytes).
__host__ __device__ inline long long win_scratch_stride(long long N) {
    return (N / 4 + N / 16 + 3) & ~3LL;
}

// Pieces of the window Gram matrices: CTA g of the tensor-core kernel takes
// pieces[pbeg[g] .. pbeg[g + 1]) = (window, first chunk, end chunk, partial
// slot); window w's partials are slots wslot0[w] .. wslot0[w + 1] (role 0,
// rows < 128) and wslot1 (role 1, bands >= 128, p > 128 only).
struct WinGramLayout {
    int G0, G1, nslot0, nslot1;
    size_t part0_floats, part1_floats;
    std::vector<int4> pieces;
    std::vector<int> pbeg, wslot0, wslot1;
};
// geo[w] = (y0, x0, h, w); every x0 must be a multiple of 4
bool win_gram_supported(int p, int W, const float* Y);
hyde_status win_gram_layout(int p, const int4* geo, int n_win, int sms, double w1x,
                            WinGramLayout* L);
hyde_status launch_win_gram(const float* Y, int p, int H, int W, const int4* pieces,
                            const int* pbeg, const int4* geo, const int* wslot0,
                            const int* wslot1, int n_win, int G0, int G1, float* part0,
                            float* part1, double* R, int* status, cudaStream_t s);
// Noise levels of every window from its Gram matrix (R [n_win][p][p]): the
// float Gauss-Jordan inverse of the scaled matrix, sigma_b^2 = S_b^2 /
// (n_w [As^-1]_bb); scratch Ainv float [n_win][p][p], S double [n_win][p].
hyde_status launch_win_noise(const double* R, int p, int n_win, const WinDesc* desc,
                             double* sigma, float* Ainv, double* S, int* status,
                             cudaStream_t s);
// Leading eigenpairs of every window's whitened Gram matrix (strides: one
// window's R, sigma, eigensolver workspace, evals, V, status).
hyde_status launch_eig_top_batched(const double* A, const double* wsig, int p, int r,
                                   double* evals, double* V, void* ws, size_t ws_stride,
                                   int* status, int n_win, cudaStream_t s);
hyde_status launch_weights_batched(const double* V, const double* sigma, int p, int r, int ldw,
                                   float* P, float* Q, int n_win, cudaStream_t s);
// The stages after the weights (windows_batched.cu): projection into the
// padded component images, DWT, SURE tables and selection, thresholded
// inverse DWT, back-projection of the cores into X.
// tstart[w] .. tstart[w + 1]: window w's tiles of `tile` padded pixels
// (projection; a multiple of 256, tuned by the batched plan) or kWinBackTile
// core pixels (back-projection), n_tiles in all. Measured on the 2048 x 2048
// x 200 scene (whole call): projection tiles of 1024 / 512 / 256 pixels
// 8.81 / 8.71 / 8.61 ms; back-projection tiles of 512 / 1024 / 2048 core
// pixels 8.71 / 8.71 / 8.73 ms.
constexpr int kWinBackTile = 1024;
hyde_status launch_win_project(const float* Y, int p, int H, int W, const WinDesc* desc,
                               const int* tstart, int n_win, int n_tiles, int tile,
                               const float* P, int r, int ldw, float* Zp, cudaStream_t s);
// DWT of every kept component with the SURE histogram rows formed on the way
hyde_status launch_win_dwt(const float* Zp, float* coef, float* scratch, const WinDesc* desc,
                           int n_win, int r, int levels, int K, unsigned int* counts,
                           double* sums, double* sum_all, cudaStream_t s);
hyde_status launch_win_sure(const WinDesc* desc, int n_win, int r, int levels, int K,
                            const unsigned int* counts, const double* sums,
                            const double* sum_all, int* rank, double* lam, hyde_hyres_info* info,
                            const int* status, const int* gstatus, cudaStream_t s);
hyde_status launch_win_idwt(const float* coef, float* Zh, float* scratch, const WinDesc* desc,
                            int n_win, int r, int levels, const int* rank, const double* lam,
                            cudaStream_t s);
hyde_status launch_win_backproject(const float* Zh, const WinDesc* desc, const int* tstart,
                                   int n_win, int n_tiles, const float* Q, int p, int ldw,
                                   const int* rank, int H, int W, float* X, cudaStream_t s);

// ----------------------------------------------------------------- SURE
struct SureBufs {
    unsigned int* counts;   // [batch][K]
    double* sums;           // [batch][K]
    double* sum_all;        // [batch]
    unsigned int* done;     // blocks finished (selection kernel); cleared with the rest
    long long* sint;        // [2][batch][K] integer prefix rows (selection kernel)
};
size_t sure_accum_bytes(int batch, int K);
// all_coef: every coefficient is binned (the final LL band too)
hyde_status launch_sure_hist(const float* coef, int batch, int Hp, int Wp,
                             int levels, int K, double delta,
                             const SureBufs& b, cudaStream_t s,
                             bool all_coef = false);
// Builds S, S_inf (and, when T != NULL, the (rank, lambda) table plus the
// selection written to info/rank_out/lam_out). With lam_comp != NULL (and T
// != NULL) the selection takes one threshold per component instead: the
// rank comes from the per-component minima, *lam_out = 1 and
// lam_comp[i][l] (float[batch][levels]) holds component i's threshold.
hyde_status launch_sure_select(const SureBufs& b, int batch, int K, long long N,
                               long long N_det, double delta, double* S,
                               double* S_inf, double* T,
                               hyde_hyres_info* info, int* rank_out,
                               double* lam_out, const int* status,
                               cudaStream_t s, float* lam_comp = nullptr,
                               int levels = 0);

// Per-level thresholds: histograms per (component, level group) ([batch][levels][K],
// the final LL band in the last group when all_coef), then per group the SURE
// table S[batch][levels][K] and its first minimum, the rank, and
// lam_comp[i][l] (float[batch][levels]); *lam_out = 1.
hyde_status launch_sure_hist_levels(const float* coef, int batch, int Hp, int Wp, int levels,
                                    int K, double delta, bool all_coef, const SureBufs& b,
                                    cudaStream_t s);
hyde_status launch_sure_select_levels(const SureBufs& b, int batch, int levels, int K, int Hp,
                                      int Wp, bool all_coef, long long N, double delta,
                                      double* S, double* S_inf, hyde_hyres_info* info,
                                      int* rank_out, double* lam_out, const int* status,
                                      float* lam_comp, cudaStream_t s);

}  // namespace hyde

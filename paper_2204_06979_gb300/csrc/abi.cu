// extern "C" entry points of libhyde (declared in include/hyde.h): argument
// checks, workspace carving and the launch sequence of the HyRes path
// (arXiv 2204.06979, Sec. 2.1). No entry point allocates, frees or
// synchronises; everything is enqueued on the caller's stream.
#include <math.h>
#include <string.h>

#include "hyde_internal.cuh"

namespace hyde {

thread_local bool tl_pdl = true;
thread_local int tl_sm_cap = 0;
thread_local unsigned long long tl_wait_ns = 0;

int device_sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    static int cache[64] = {0};
    int v = 0;
    if (dev >= 0 && dev < 64 && cache[dev] > 0) {
        v = cache[dev];
    } else {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        if (dev >= 0 && dev < 64) cache[dev] = v;
    }
    return tl_sm_cap > 0 && tl_sm_cap < v ? tl_sm_cap : v;
}

cudaError_t ensure_smem_limit(const void* func, int bytes) {
    // Without the opt-in a block gets 48 KiB of static and dynamic shared
    // memory together. Every kernel launched through here keeps its static
    // shared memory under 8 KiB (the most, the SURE selection, 3.2 KiB), so
    // up to 40 KiB of dynamic memory needs no attribute.
    if (bytes <= 40 * 1024) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return e;
    // dynamic + static shared memory may not exceed the opt-in limit
    const int room = optin - (int)fa.sharedSizeBytes;
    if (bytes > room) return cudaErrorInvalidValue;
    // the largest value is always safe to set; concurrent callers agree on it
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, room);
}

namespace {

inline bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

inline int rank_pad(int r) { return (r + 3) / 4 * 4; }   // weights row stride: r rounded up to 4

bool padded(int H, int W, int levels, int* Hp, int* Wp) { return padded_dims(H, W, levels, Hp, Wp); }

// Bump allocator over the caller's workspace (offsets only).
struct Carver {
    size_t off = 0;
    size_t take(size_t bytes) {
        size_t o = off;
        off += align_up(bytes, kAlign);
        return o;
    }
};

struct HyresLayout {
    int Hp, Wp, RM, K;
    long long N, n;
    GramPlan gram;
    hyde_ws_layout pub;
    size_t rank_dev, lam_dev, counts, sums, sum_all, done, sint, P, Q, noise, eig, partials, zp,
        scratch;
    size_t zero_begin, zero_end;
};

hyde_status hyres_layout(int p, int H, int W, const hyde_hyres_params* pr, HyresLayout* L) {
    if (!pr) return HYDE_ERR_INVALID_ARG;
    if (pr->wavelet != 2) return HYDE_ERR_INVALID_ARG;
    if (pr->precision != HYDE_PREC_FP32 && pr->precision != HYDE_PREC_BF16X3 &&
        pr->precision != HYDE_PREC_BF16X3_ALL && pr->precision != HYDE_PREC_TF32X3)
        return HYDE_ERR_INVALID_ARG;
    if (pr->lambda_mode != HYDE_LAMBDA_SHARED && pr->lambda_mode != HYDE_LAMBDA_PER_COMPONENT &&
        pr->lambda_mode != HYDE_LAMBDA_PER_LEVEL)
        return HYDE_ERR_INVALID_ARG;
    if (pr->threshold_ll != 0 && pr->threshold_ll != 1) return HYDE_ERR_INVALID_ARG;
    if (pr->reserved) return HYDE_ERR_INVALID_ARG;
    if (p < 2 || p > kMaxBandsGram) return HYDE_ERR_SHAPE;
    if (pr->r_max < 1 || pr->r_max > kMaxRank || pr->r_max > p) return HYDE_ERR_SHAPE;
    if (pr->n_lambda < 2 || pr->n_lambda > kMaxLambda) return HYDE_ERR_SHAPE;
    int Hp, Wp;
    if (!padded(H, W, pr->levels, &Hp, &Wp)) return HYDE_ERR_SHAPE;
    const long long n = (long long)H * W;
    if (n < p) return HYDE_ERR_SHAPE;
    if (eig_smem_bytes(p, pr->r_max) > 227 * 1024) return HYDE_ERR_SHAPE;
    if (noise_smem_bytes(p) > 227 * 1024) return HYDE_ERR_SHAPE;
    // per-level thresholds: one SURE histogram per (component, level), held in
    // shared memory as [level][bin][32 lanes] x (count, sum)
    const int G = pr->lambda_mode == HYDE_LAMBDA_PER_LEVEL ? pr->levels : 1;
    if (G > 1 && (size_t)2 * G * pr->n_lambda * 32 * sizeof(unsigned int) > 200 * 1024)
        return HYDE_ERR_SHAPE;
    HyresLayout l;
    l.Hp = Hp; l.Wp = Wp; l.RM = rank_pad(pr->r_max); l.K = pr->n_lambda;
    l.N = (long long)Hp * Wp; l.n = n;
    hyde_status st = gram_plan(p, n, &l.gram);
    if (st != HYDE_OK) return st;
    if (pr->precision == HYDE_PREC_TF32X3 && !gram_tf32_shape_ok(p, n)) return HYDE_ERR_SHAPE;
    if (pr->precision != HYDE_PREC_FP32) {   // split-BF16 or split-TF32 Gram on the tensor cores
        size_t tcb = 0;
        st = gram_tc_partial_bytes(p, &tcb);
        if (st != HYDE_OK) return st;
        l.gram.partial_bytes = tcb;
    } else if (gram_tf32_shape_ok(p, n)) {
        // the FP32 path takes the split-TF32 Gram when the cube is 16-byte
        // aligned (known only at the call) and the SIMT kernel otherwise:
        // room for either's partials
        size_t tcb = 0;
        st = gram_tc_partial_bytes(p, &tcb);
        if (st != HYDE_OK) return st;
        if (tcb > l.gram.partial_bytes) l.gram.partial_bytes = tcb;
    }
    const int r = pr->r_max, K = pr->n_lambda;
    Carver c;
    memset(&l.pub, 0, sizeof(l.pub));
    // zero-initialised block first: status, rank, lambda, SURE accumulators
    l.zero_begin = c.off;
    l.pub.status = c.take(sizeof(int));
    l.rank_dev = c.take(sizeof(int));
    l.lam_dev = c.take(sizeof(double));
    l.counts = c.take((size_t)r * G * K * sizeof(unsigned int));
    l.sums = c.take((size_t)r * G * K * sizeof(double));
    l.sum_all = c.take((size_t)r * sizeof(double));
    l.done = c.take(sizeof(unsigned int));
    l.zero_end = c.off;
    l.pub.R = c.take((size_t)p * p * sizeof(double));
    l.pub.sigma = c.take((size_t)p * sizeof(double));
    l.pub.evals = c.take((size_t)r * sizeof(double));
    l.pub.V = c.take((size_t)p * r * sizeof(double));
    l.pub.sure = c.take((size_t)r * G * K * sizeof(double));
    l.pub.sure_inf = c.take((size_t)r * sizeof(double));
    l.pub.sure_total = c.take((size_t)r * K * sizeof(double));
    l.pub.lam_comp = c.take((size_t)r * pr->levels * sizeof(float));
    l.sint = c.take((size_t)2 * r * G * K * sizeof(long long));
    l.P = c.take((size_t)p * l.RM * sizeof(float));
    l.Q = c.take((size_t)p * l.RM * sizeof(float));
    l.noise = c.take(noise_ws_bytes(p));
    l.eig = c.take(eig_ws_bytes(p, r));
    l.partials = c.take(l.gram.partial_bytes);
    l.zp = c.take((size_t)r * l.N * sizeof(float));
    l.pub.coef = c.take((size_t)r * l.N * sizeof(float));
    l.scratch = c.take((size_t)r * dwt_scratch_floats(Hp, Wp) * sizeof(float));
    l.pub.total = c.off;
    *L = l;
    return HYDE_OK;
}

template <typename T>
inline T* at(void* ws, size_t off) {
    return reinterpret_cast<T*>(reinterpret_cast<char*>(ws) + off);
}

}  // namespace
}  // namespace hyde

using namespace hyde;

extern "C" {

const char* hyde_status_string(hyde_status s) {
    switch (s) {
        case HYDE_OK: return "ok";
        case HYDE_ERR_INVALID_ARG: return "invalid argument";
        case HYDE_ERR_SHAPE: return "unsupported shape";
        case HYDE_ERR_NUMERIC: return "numerical failure (NaN/Inf input or non-SPD Gram matrix)";
        case HYDE_ERR_NOT_CONVERGED: return "eigensolver did not converge";
        case HYDE_ERR_TIMEOUT: return "bounded device wait gave up";
        case HYDE_ERR_CUDA: return "CUDA runtime error";
        case HYDE_ERR_WORKSPACE: return "workspace missing or too small";
    }
    return "unknown status";
}

int hyde_version(void) { return 100; }

// ------------------------------------------------------------------ Gram
hyde_status hyde_gram_workspace_size(int p, long long n, int precision, size_t* bytes) {
    if (!bytes) return HYDE_ERR_INVALID_ARG;
    if (precision == HYDE_PREC_BF16X3 || precision == HYDE_PREC_TF32X3) {
        if (n < 1) return HYDE_ERR_SHAPE;
        if (precision == HYDE_PREC_TF32X3 && !gram_tf32_shape_ok(p, n)) return HYDE_ERR_SHAPE;
        size_t b = 0;
        hyde_status st = gram_tc_partial_bytes(p, &b);
        if (st != HYDE_OK) return st;
        *bytes = align_up(b, kAlign);
        return HYDE_OK;
    }
    if (precision != HYDE_PREC_FP32) return HYDE_ERR_INVALID_ARG;
    GramPlan g;
    hyde_status st = gram_plan(p, n, &g);
    if (st != HYDE_OK) return st;
    *bytes = align_up(g.partial_bytes, kAlign);
    return HYDE_OK;
}

hyde_status hyde_gram(const float* Y, int p, long long n, int precision, double* R, void* ws,
                      size_t ws_bytes, cudaStream_t stream) {
    if (!Y || !R) return HYDE_ERR_INVALID_ARG;
    size_t need = 0;
    hyde_status st = hyde_gram_workspace_size(p, n, precision, &need);
    if (st != HYDE_OK) return st;
    if (!ws || !aligned(ws, kAlign) || ws_bytes < need) return HYDE_ERR_WORKSPACE;
    if (precision == HYDE_PREC_BF16X3)
        return launch_gram_tc(Y, p, n, reinterpret_cast<float*>(ws), R, nullptr, stream);
    if (precision == HYDE_PREC_TF32X3) {
        if (!aligned(Y, 16)) return HYDE_ERR_INVALID_ARG;
        return launch_gram_tf32(Y, p, n, reinterpret_cast<float*>(ws), R, nullptr, stream);
    }
    GramPlan g;
    gram_plan(p, n, &g);
    return launch_gram(Y, p, n, g, reinterpret_cast<float*>(ws), R, nullptr, stream);
}

// ------------------------------------------------------------ noise level
hyde_status hyde_noise_est_workspace_size(int p, int H, int W, size_t* bytes) {
    if (!bytes) return HYDE_ERR_INVALID_ARG;
    if (p < 2 || H < 1 || W < 1) return HYDE_ERR_SHAPE;
    long long n = (long long)H * W;
    if (n < p) return HYDE_ERR_SHAPE;
    GramPlan g;
    hyde_status st = gram_plan(p, n, &g);
    if (st != HYDE_OK) return st;
    *bytes = align_up(g.partial_bytes, kAlign) + align_up((size_t)p * p * sizeof(double), kAlign) +
             noise_ws_bytes(p);
    return HYDE_OK;
}

hyde_status hyde_noise_est(const float* Y, int p, int H, int W, double* sigma, int* status,
                           void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (!Y || !sigma) return HYDE_ERR_INVALID_ARG;
    size_t need = 0;
    hyde_status st = hyde_noise_est_workspace_size(p, H, W, &need);
    if (st != HYDE_OK) return st;
    if (noise_smem_bytes(p) > 227 * 1024) return HYDE_ERR_SHAPE;
    if (!ws || !aligned(ws, kAlign) || ws_bytes < need) return HYDE_ERR_WORKSPACE;
    long long n = (long long)H * W;
    GramPlan g;
    gram_plan(p, n, &g);
    char* w = reinterpret_cast<char*>(ws);
    float* partials = reinterpret_cast<float*>(w);
    double* R = reinterpret_cast<double*>(w + align_up(g.partial_bytes, kAlign));
    void* nws = w + align_up(g.partial_bytes, kAlign) + align_up((size_t)p * p * sizeof(double), kAlign);
    st = launch_gram(Y, p, n, g, partials, R, status, stream);
    if (st != HYDE_OK) return st;
    return launch_noise_from_gram(R, p, n, sigma, nws, status, stream);
}

// ----------------------------------------------------------- eigenvectors
hyde_status hyde_eig_workspace_size(int p, int r, size_t* bytes) {
    if (!bytes) return HYDE_ERR_INVALID_ARG;
    if (p < 2 || r < 1 || r > p || r > kMaxRank || p > kMaxBandsGram) return HYDE_ERR_SHAPE;
    if (eig_smem_bytes(p, r) > 227 * 1024) return HYDE_ERR_SHAPE;
    *bytes = align_up(eig_ws_bytes(p, r), kAlign);
    return HYDE_OK;
}

hyde_status hyde_eig_sym_top(const double* A, int p, int r, double* evals, double* V,
                             int* status, void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (!A || !evals || !V) return HYDE_ERR_INVALID_ARG;
    size_t need = 0;
    hyde_status st = hyde_eig_workspace_size(p, r, &need);
    if (st != HYDE_OK) return st;
    if (!ws || !aligned(ws, kAlign) || ws_bytes < need) return HYDE_ERR_WORKSPACE;
    return launch_eig_top(A, nullptr, p, r, evals, V, ws, status, stream);
}

// -------------------------------------------------------------------- DWT
hyde_status hyde_dwt_workspace_size(int batch, int H, int W, int levels, size_t* bytes) {
    if (!bytes) return HYDE_ERR_INVALID_ARG;
    int Hp, Wp;
    if (batch < 1 || batch > 65535 || !padded(H, W, levels, &Hp, &Wp)) return HYDE_ERR_SHAPE;
    *bytes = align_up((size_t)batch * dwt_scratch_floats(Hp, Wp) * sizeof(float), kAlign);
    return HYDE_OK;
}

static hyde_status dwt_common(const void* a, const void* b, int batch, int H, int W, int wavelet,
                              int levels, void* ws, size_t ws_bytes, int* Hp, int* Wp) {
    if (!a || !b || wavelet != 2) return HYDE_ERR_INVALID_ARG;
    size_t need = 0;
    hyde_status st = hyde_dwt_workspace_size(batch, H, W, levels, &need);
    if (st != HYDE_OK) return st;
    padded(H, W, levels, Hp, Wp);
    if (levels > 1 && (!ws || !aligned(ws, kAlign) || ws_bytes < need)) return HYDE_ERR_WORKSPACE;
    return HYDE_OK;
}

hyde_status hyde_dwt2(const float* in, float* coef, int batch, int H, int W, int wavelet,
                      int levels, void* ws, size_t ws_bytes, cudaStream_t stream) {
    int Hp, Wp;
    hyde_status st = dwt_common(in, coef, batch, H, W, wavelet, levels, ws, ws_bytes, &Hp, &Wp);
    if (st != HYDE_OK) return st;
    DwtSrc src{in, (long long)H * W, W, H, W};
    return launch_dwt2(src, coef, batch, Hp, Wp, levels, reinterpret_cast<float*>(ws), stream);
}

hyde_status hyde_idwt2(const float* coef, float* out, int batch, int H, int W, int wavelet,
                       int levels, void* ws, size_t ws_bytes, cudaStream_t stream) {
    int Hp, Wp;
    hyde_status st = dwt_common(coef, out, batch, H, W, wavelet, levels, ws, ws_bytes, &Hp, &Wp);
    if (st != HYDE_OK) return st;
    return launch_idwt2(coef, out, batch, Hp, Wp, H, W, levels, reinterpret_cast<float*>(ws),
                        nullptr, nullptr, stream);
}

// ------------------------------------------------------------------- SURE
hyde_status hyde_sure_workspace_size(int batch, int K, size_t* bytes) {
    if (!bytes) return HYDE_ERR_INVALID_ARG;
    if (batch < 1 || batch > 65535 || K < 2 || K > kMaxLambda) return HYDE_ERR_SHAPE;
    *bytes = sure_accum_bytes(batch, K);
    return HYDE_OK;
}

hyde_status hyde_sure_table(const float* coef, int batch, int Hp, int Wp, int levels, int K,
                            double* S, double* S_inf, void* ws, size_t ws_bytes,
                            cudaStream_t stream) {
    if (!coef || !S || !S_inf) return HYDE_ERR_INVALID_ARG;
    size_t need = 0;
    hyde_status st = hyde_sure_workspace_size(batch, K, &need);
    if (st != HYDE_OK) return st;
    if (levels < 1 || levels > kMaxLevels || Hp < 2 || Wp < 2 || (Hp % (1 << levels)) ||
        (Wp % (1 << levels)))
        return HYDE_ERR_SHAPE;
    if (!ws || !aligned(ws, kAlign) || ws_bytes < need) return HYDE_ERR_WORKSPACE;
    char* w = reinterpret_cast<char*>(ws);
    SureBufs b;
    b.counts = reinterpret_cast<unsigned int*>(w);
    b.sums = reinterpret_cast<double*>(w + align_up((size_t)batch * K * sizeof(unsigned int), kAlign));
    b.sum_all = reinterpret_cast<double*>(reinterpret_cast<char*>(b.sums) +
                                          align_up((size_t)batch * K * sizeof(double), kAlign));
    b.done = nullptr;   // the table-only path has no selection
    b.sint = nullptr;
    if (cudaMemsetAsync(ws, 0, need, stream) != cudaSuccess) return HYDE_ERR_CUDA;
    const long long N = (long long)Hp * Wp;
    const long long N_det = N - (long long)(Hp >> levels) * (Wp >> levels);
    const double delta = sqrt(2.0 * log((double)N)) / (K - 1);
    st = launch_sure_hist(coef, batch, Hp, Wp, levels, K, delta, b, stream);
    if (st != HYDE_OK) return st;
    return launch_sure_select(b, batch, K, N, N_det, delta, S, S_inf, nullptr, nullptr, nullptr,
                              nullptr, nullptr, stream);
}

// ---------------------------------------------------------- whole HyRes
hyde_status hyde_workspace_size(int p, int H, int W, const hyde_hyres_params* params,
                                size_t* bytes) {
    if (!bytes) return HYDE_ERR_INVALID_ARG;
    HyresLayout L;
    hyde_status st = hyres_layout(p, H, W, params, &L);
    if (st != HYDE_OK) return st;
    *bytes = L.pub.total;
    return HYDE_OK;
}

hyde_status hyde_workspace_layout(int p, int H, int W, const hyde_hyres_params* params,
                                  hyde_ws_layout* layout) {
    if (!layout) return HYDE_ERR_INVALID_ARG;
    HyresLayout L;
    hyde_status st = hyres_layout(p, H, W, params, &L);
    if (st != HYDE_OK) return st;
    *layout = L.pub;
    return HYDE_OK;
}

static hyde_status hyres_enqueue(const float* Y, float* X, int p, int H, int W,
                                 const hyde_hyres_params* params, hyde_hyres_info* info,
                                 void* ws, size_t ws_bytes, cudaStream_t stream,
                                 cudaEvent_t* ev, const float* scale = nullptr) {
    if (!Y || !X || Y == X) return HYDE_ERR_INVALID_ARG;
    // the scaled forms multiply one shared lambda by their detail-level scales
    const bool per_comp = params && params->lambda_mode == HYDE_LAMBDA_PER_COMPONENT;
    const bool per_level = params && params->lambda_mode == HYDE_LAMBDA_PER_LEVEL;
    const bool all_coef = params && params->threshold_ll == 1;
    if ((per_comp || per_level || all_coef) && scale) return HYDE_ERR_INVALID_ARG;
    HyresLayout L;
    hyde_status st = hyres_layout(p, H, W, params, &L);
    if (st != HYDE_OK) return st;
    if (!ws || !aligned(ws, kAlign) || ws_bytes < L.pub.total) return HYDE_ERR_WORKSPACE;
    const int r = params->r_max, K = params->n_lambda, lev = params->levels;
    int* status = at<int>(ws, L.pub.status);
    int* rank_dev = at<int>(ws, L.rank_dev);
    double* lam_dev = at<double>(ws, L.lam_dev);
    double* R = at<double>(ws, L.pub.R);
    double* sigma = at<double>(ws, L.pub.sigma);
    double* evals = at<double>(ws, L.pub.evals);
    double* V = at<double>(ws, L.pub.V);
    float* P = at<float>(ws, L.P);
    float* Q = at<float>(ws, L.Q);
    float* zp = at<float>(ws, L.zp);
    float* coef = at<float>(ws, L.pub.coef);
    float* scratch = at<float>(ws, L.scratch);
    SureBufs sb{at<unsigned int>(ws, L.counts), at<double>(ws, L.sums), at<double>(ws, L.sum_all),
                at<unsigned int>(ws, L.done), at<long long>(ws, L.sint)};
    int mark = 0;
    auto stage = [&]() -> hyde_status {
        if (!ev) return HYDE_OK;
        return cuda_status(cudaEventRecord(ev[mark++], stream));
    };
#define HYDE_TRY(x) do { hyde_status s_ = (x); if (s_ != HYDE_OK) return s_; } while (0)
    HYDE_TRY(stage());
    if (cudaMemsetAsync(at<char>(ws, L.zero_begin), 0, L.zero_end - L.zero_begin, stream) !=
        cudaSuccess)
        return HYDE_ERR_CUDA;
    // 1. Gram matrix: split-TF32 on the tensor cores (FP32-accurate; the FP32
    // path's choice whenever the shape and alignment allow), split-BF16, or
    // float SIMT
    if (params->precision == HYDE_PREC_TF32X3 ||
        (params->precision == HYDE_PREC_FP32 && gram_tf32_supported(Y, p, L.n)))
        HYDE_TRY(launch_gram_tf32(Y, p, L.n, at<float>(ws, L.partials), R, status, stream));
    else if (params->precision != HYDE_PREC_FP32)
        HYDE_TRY(launch_gram_tc(Y, p, L.n, at<float>(ws, L.partials), R, status, stream));
    else
        HYDE_TRY(launch_gram(Y, p, L.n, L.gram, at<float>(ws, L.partials), R, status, stream));
    HYDE_TRY(stage());
    // 2. noise level by regression
    HYDE_TRY(launch_noise_from_gram(R, p, L.n, sigma, at<void>(ws, L.noise), status, stream));
    HYDE_TRY(stage());
    // 3-4. whitened Gram matrix, leading eigenpairs, float weights
    HYDE_TRY(launch_eig_top(R, sigma, p, r, evals, V, at<void>(ws, L.eig), status, stream));
    HYDE_TRY(launch_weights(V, sigma, p, r, L.RM, P, Q, stream));
    HYDE_TRY(stage());
    // 5. projection into padded component images
    const bool tc_proj =
        params->precision == HYDE_PREC_BF16X3_ALL && project_tc_supported(p, r);
    if (tc_proj)
        HYDE_TRY(launch_project_pad_tc(Y, p, H, W, P, r, L.RM, zp, L.Hp, L.Wp, status, stream));
    else
        HYDE_TRY(launch_project_pad(Y, p, H, W, P, r, L.RM, zp, L.Hp, L.Wp, stream));
    HYDE_TRY(stage());
    // 6. wavelet analysis
    DwtSrc src{zp, L.N, L.Wp, L.Hp, L.Wp};
    HYDE_TRY(launch_dwt2(src, coef, r, L.Hp, L.Wp, lev, scratch, stream, status));
    HYDE_TRY(stage());
    // 7-8. SURE table and (rank, lambda) selection
    const long long N_det =
        all_coef ? L.N : L.N - (long long)(L.Hp >> lev) * (L.Wp >> lev);
    const double delta = sqrt(2.0 * log((double)L.N)) / (K - 1);
    float* lam_comp = (per_comp || per_level) ? at<float>(ws, L.pub.lam_comp) : nullptr;
    if (per_level) {
        HYDE_TRY(launch_sure_hist_levels(coef, r, L.Hp, L.Wp, lev, K, delta, all_coef, sb,
                                         stream));
        HYDE_TRY(launch_sure_select_levels(sb, r, lev, K, L.Hp, L.Wp, all_coef, L.N, delta,
                                           at<double>(ws, L.pub.sure),
                                           at<double>(ws, L.pub.sure_inf), info, rank_dev,
                                           lam_dev, status, lam_comp, stream));
    } else {
        HYDE_TRY(launch_sure_hist(coef, r, L.Hp, L.Wp, lev, K, delta, sb, stream, all_coef));
        HYDE_TRY(launch_sure_select(sb, r, K, L.N, N_det, delta, at<double>(ws, L.pub.sure),
                                    at<double>(ws, L.pub.sure_inf),
                                    at<double>(ws, L.pub.sure_total), info, rank_dev, lam_dev,
                                    status, stream, lam_comp, lev));
    }
    HYDE_TRY(stage());
    // 9. soft threshold + inverse DWT of the kept components (into zp, H x W);
    // per-component and per-level thresholds are lam_comp[i][l] times *lam_dev = 1
    HYDE_TRY(launch_idwt2(coef, zp, r, L.Hp, L.Wp, H, W, lev, scratch, lam_dev, rank_dev, stream,
                          lam_comp ? lam_comp : scale, lev, all_coef));
    HYDE_TRY(stage());
    // 10. back-projection and un-whitening
    if (tc_proj)
        HYDE_TRY(launch_backproject_tc(zp, L.n, Q, p, L.RM, rank_dev, X, status, stream));
    else
        HYDE_TRY(launch_backproject(zp, L.n, Q, p, r, L.RM, rank_dev, X, stream));
    HYDE_TRY(stage());
#undef HYDE_TRY
    return HYDE_OK;
}

hyde_status hyde_hyres_denoise(const float* Y, float* X, int p, int H, int W,
                               const hyde_hyres_params* params, hyde_hyres_info* info, void* ws,
                               size_t ws_bytes, cudaStream_t stream) {
    return hyres_enqueue(Y, X, p, H, W, params, info, ws, ws_bytes, stream, nullptr);
}

// ------------------------------------------------------- several cubes at once
hyde_status hyde_hyres_denoise_many(const float* const* Y, float* const* X, int count, int p,
                                    int H, int W, const hyde_hyres_params* params,
                                    hyde_hyres_info* info, void* const* ws, size_t ws_bytes,
                                    int slots, cudaStream_t stream,
                                    const cudaStream_t* slot_streams, const cudaEvent_t* events) {
    if (!Y || !X || !ws || !slot_streams || !events || !params) return HYDE_ERR_INVALID_ARG;
    if (count < 1 || slots < 1 || slots > 16) return HYDE_ERR_INVALID_ARG;
    for (int k = 0; k < count; ++k)
        if (!Y[k] || !X[k] || Y[k] == X[k]) return HYDE_ERR_INVALID_ARG;
    for (int s = 0; s < slots; ++s)
        if (!ws[s] || !slot_streams[s] || !events[1 + s]) return HYDE_ERR_INVALID_ARG;
    if (!events[0]) return HYDE_ERR_INVALID_ARG;
    const int used = count < slots ? count : slots;
    // fork the slot streams from the caller's stream
    if (cudaEventRecord(events[0], stream) != cudaSuccess) return HYDE_ERR_CUDA;
    for (int s = 0; s < used; ++s)
        if (cudaStreamWaitEvent(slot_streams[s], events[0], 0) != cudaSuccess) return HYDE_ERR_CUDA;
    for (int k = 0; k < count; ++k) {
        const int s = k % slots;
        const hyde_status st = hyres_enqueue(Y[k], X[k], p, H, W, params, info ? info + k : nullptr,
                                             ws[s], ws_bytes, slot_streams[s], nullptr);
        if (st != HYDE_OK) return st;
    }
    // join them back
    for (int s = 0; s < used; ++s) {
        if (cudaEventRecord(events[1 + s], slot_streams[s]) != cudaSuccess) return HYDE_ERR_CUDA;
        if (cudaStreamWaitEvent(stream, events[1 + s], 0) != cudaSuccess) return HYDE_ERR_CUDA;
    }
    return HYDE_OK;
}

// ------------------------------------------------------------------ WSRRR
static hyde_status wsrrr_check(const hyde_hyres_params* params) {
    if (!params) return HYDE_ERR_INVALID_ARG;
    if (params->lambda_mode != HYDE_LAMBDA_SHARED || params->threshold_ll != 0)
        return HYDE_ERR_INVALID_ARG;
    if (params->precision != HYDE_PREC_FP32 && params->precision != HYDE_PREC_TF32X3)
        return HYDE_ERR_INVALID_ARG;
    if (params->r_max > 32) return HYDE_ERR_SHAPE;
    return HYDE_OK;
}

struct WsrrrExtra {
    size_t hy, M, partials, total;
    int nblocks;
};

static hyde_status wsrrr_layout(int p, int H, int W, const hyde_hyres_params* params,
                                HyresLayout* L, WsrrrExtra* E) {
    hyde_status st = wsrrr_check(params);
    if (st != HYDE_OK) return st;
    st = hyres_layout(p, H, W, params, L);
    if (st != HYDE_OK) return st;
    const int sms = device_sm_count();
    if (sms <= 0) return HYDE_ERR_CUDA;
    E->nblocks = 2 * sms;
    Carver c;
    E->hy = c.take(L->pub.total);
    E->M = c.take((size_t)p * params->r_max * sizeof(double));
    E->partials = c.take(wsrrr_cross_partial_bytes(p, params->r_max, E->nblocks));
    E->total = c.off;
    return HYDE_OK;
}

hyde_status hyde_wsrrr_workspace_size(int p, int H, int W, const hyde_hyres_params* params,
                                      size_t* bytes) {
    if (!bytes) return HYDE_ERR_INVALID_ARG;
    HyresLayout L;
    WsrrrExtra E;
    const hyde_status st = wsrrr_layout(p, H, W, params, &L, &E);
    if (st != HYDE_OK) return st;
    *bytes = E.total;
    return HYDE_OK;
}

hyde_status hyde_wsrrr(const float* Y, float* X, int p, int H, int W,
                       const hyde_hyres_params* params, int iters, hyde_hyres_info* info,
                       float* features, void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (!Y || !X || Y == X) return HYDE_ERR_INVALID_ARG;
    if (iters < 0 || iters > 1000) return HYDE_ERR_SHAPE;
    HyresLayout L;
    WsrrrExtra E;
    hyde_status st = wsrrr_layout(p, H, W, params, &L, &E);
    if (st != HYDE_OK) return st;
    if (!ws || !aligned(ws, kAlign) || ws_bytes < E.total) return HYDE_ERR_WORKSPACE;
    void* hws = at<void>(ws, E.hy);
    // HyRes: noise estimate, subspace, rank r* and threshold lambda*
    st = hyres_enqueue(Y, X, p, H, W, params, info, hws, L.pub.total, stream, nullptr);
    if (st != HYDE_OK) return st;
    if (iters == 0 && !features) return HYDE_OK;
    const int r = params->r_max, lev = params->levels;
    int* status = at<int>(hws, L.pub.status);
    int* rank_dev = at<int>(hws, L.rank_dev);
    double* lam_dev = at<double>(hws, L.lam_dev);
    double* sigma = at<double>(hws, L.pub.sigma);
    double* V = at<double>(hws, L.pub.V);
    float* P = at<float>(hws, L.P);
    float* Q = at<float>(hws, L.Q);
    float* zp = at<float>(hws, L.zp);
    float* coef = at<float>(hws, L.pub.coef);
    float* scratch = at<float>(hws, L.scratch);
    double* M = at<double>(ws, E.M);
    const DwtSrc src{zp, L.N, L.Wp, L.Hp, L.Wp};
#define HYDE_TRY(x) do { hyde_status s_ = (x); if (s_ != HYDE_OK) return s_; } while (0)
    // B-step: coefficients of the projected whitened cube, thresholded
    auto bstep = [&]() -> hyde_status {
        HYDE_TRY(launch_weights(V, sigma, p, r, L.RM, P, Q, stream));
        HYDE_TRY(launch_project_pad(Y, p, H, W, P, r, L.RM, zp, L.Hp, L.Wp, stream));
        return launch_dwt2(src, coef, r, L.Hp, L.Wp, lev, scratch, stream, status);
    };
    for (int it = 0; it < iters; ++it) {
        HYDE_TRY(bstep());
        // component images W2 B on the padded domain (no crop)
        HYDE_TRY(launch_idwt2(coef, zp, r, L.Hp, L.Wp, L.Hp, L.Wp, lev, scratch, lam_dev,
                              rank_dev, stream));
        // V-step: the orthogonal Procrustes basis of Yw^T W2 B
        HYDE_TRY(launch_wsrrr_cross(Y, p, H, W, zp, r, L.Hp, L.Wp, rank_dev, sigma,
                                    at<float>(ws, E.partials), E.nblocks, M, r, status, stream));
        HYDE_TRY(launch_wsrrr_polar(M, p, r, rank_dev, V, r, status, stream));
    }
    HYDE_TRY(bstep());
    if (features) {
        if (cudaMemsetAsync(features, 0, (size_t)r * L.N * sizeof(float), stream) != cudaSuccess)
            return HYDE_ERR_CUDA;
        HYDE_TRY(launch_idwt2(coef, features, r, L.Hp, L.Wp, L.Hp, L.Wp, lev, scratch, lam_dev,
                              rank_dev, stream));
    }
    HYDE_TRY(launch_idwt2(coef, zp, r, L.Hp, L.Wp, H, W, lev, scratch, lam_dev, rank_dev, stream));
    HYDE_TRY(launch_backproject(zp, L.n, Q, p, r, L.RM, rank_dev, X, stream));
#undef HYDE_TRY
    return cuda_status(cudaGetLastError());
}

hyde_status hyde_hyres_denoise_host(const float* const* Y_host, float* const* X_host,
                                    hyde_hyres_info* info_host, int count, int p, int H,
                                    int W, const hyde_hyres_params* params,
                                    float* const* dev, hyde_hyres_info* info_dev, void* ws,
                                    size_t ws_bytes, cudaStream_t stream, cudaStream_t h2d,
                                    cudaStream_t d2h, cudaEvent_t* events) {
    if (!Y_host || !X_host || !dev || !info_dev || !events || count < 1 || !params)
        return HYDE_ERR_INVALID_ARG;
    for (int q = 0; q < 4; ++q)
        if (!dev[q]) return HYDE_ERR_INVALID_ARG;
    for (int q = 0; q < 7; ++q)
        if (!events[q]) return HYDE_ERR_INVALID_ARG;
    for (int s = 0; s < count; ++s)
        if (!Y_host[s] || !X_host[s]) return HYDE_ERR_INVALID_ARG;
    HyresLayout L;
    hyde_status st = hyres_layout(p, H, W, params, &L);
    if (st != HYDE_OK) return st;
    const size_t bytes = (size_t)p * H * W * sizeof(float);
    cudaEvent_t* in_done = events;          // per input buffer
    cudaEvent_t* comp_done = events + 2;    // per buffer pair
    cudaEvent_t* out_done = events + 4;     // per output buffer
#define HYDE_CU(x) do { if ((x) != cudaSuccess) return HYDE_ERR_CUDA; } while (0)
    // fork: the copies follow what is already queued on `stream`
    HYDE_CU(cudaEventRecord(events[6], stream));
    HYDE_CU(cudaStreamWaitEvent(h2d, events[6], 0));
    HYDE_CU(cudaStreamWaitEvent(d2h, events[6], 0));
    for (int s = 0; s < count; ++s) {
        const int b = s & 1;
        float* Yd = dev[b];
        float* Xd = dev[2 + b];
        // copy in once the denoise of cube s - 2 has read the buffer
        if (s >= 2) HYDE_CU(cudaStreamWaitEvent(h2d, comp_done[b], 0));
        HYDE_CU(cudaMemcpyAsync(Yd, Y_host[s], bytes, cudaMemcpyHostToDevice, h2d));
        HYDE_CU(cudaEventRecord(in_done[b], h2d));
        // denoise once the input is in and cube s - 2's output is out
        HYDE_CU(cudaStreamWaitEvent(stream, in_done[b], 0));
        if (s >= 2) HYDE_CU(cudaStreamWaitEvent(stream, out_done[b], 0));
        st = hyres_enqueue(Yd, Xd, p, H, W, params, info_dev + b, ws, ws_bytes, stream, nullptr);
        if (st != HYDE_OK) return st;
        HYDE_CU(cudaEventRecord(comp_done[b], stream));
        // copy out
        HYDE_CU(cudaStreamWaitEvent(d2h, comp_done[b], 0));
        HYDE_CU(cudaMemcpyAsync(X_host[s], Xd, bytes, cudaMemcpyDeviceToHost, d2h));
        if (info_host)
            HYDE_CU(cudaMemcpyAsync(info_host + s, info_dev + b, sizeof(hyde_hyres_info),
                                    cudaMemcpyDeviceToHost, d2h));
        HYDE_CU(cudaEventRecord(out_done[b], d2h));
    }
    // join: the last copy-out ends the d2h stream's work; the h2d stream's
    // last copy was already waited for by the last denoise
    HYDE_CU(cudaStreamWaitEvent(stream, out_done[(count - 1) & 1], 0));
#undef HYDE_CU
    return HYDE_OK;
}

hyde_status hyde_hyres_denoise_timed(const float* Y, float* X, int p, int H, int W,
                                     const hyde_hyres_params* params, hyde_hyres_info* info,
                                     void* ws, size_t ws_bytes, cudaStream_t stream,
                                     cudaEvent_t* events) {
    if (!events) return HYDE_ERR_INVALID_ARG;
    return hyres_enqueue(Y, X, p, H, W, params, info, ws, ws_bytes, stream, events);
}

hyde_status hyde_hyres_denoise_scaled(const float* Y, float* X, int p, int H, int W,
                                      const hyde_hyres_params* params, const float* scale,
                                      hyde_hyres_info* info, void* ws, size_t ws_bytes,
                                      cudaStream_t stream) {
    if (!scale) return HYDE_ERR_INVALID_ARG;
    return hyres_enqueue(Y, X, p, H, W, params, info, ws, ws_bytes, stream, nullptr, scale);
}

// Backward workspace: recomputed coefficients C, their adjoint dC, one padded
// image buffer, the DWT scratch, and the (component, level) accumulators.
struct BackLayout {
    size_t C, dC, zp, scratch, acc, sure_acc, total;
};

static hyde_status back_layout(const HyresLayout& L, int r, int levels, BackLayout* B) {
    Carver c;
    BackLayout b;
    b.acc = c.take((size_t)r * levels * sizeof(double));
    b.sure_acc = c.take(sizeof(double));
    b.C = c.take((size_t)r * L.N * sizeof(float));
    b.dC = c.take((size_t)r * L.N * sizeof(float));
    b.zp = c.take((size_t)r * L.N * sizeof(float));
    b.scratch = c.take((size_t)r * dwt_scratch_floats(L.Hp, L.Wp) * sizeof(float));
    b.total = c.off;
    *B = b;
    return HYDE_OK;
}

hyde_status hyde_backward_workspace_size(int p, int H, int W, const hyde_hyres_params* params,
                                         size_t* bytes) {
    if (!bytes) return HYDE_ERR_INVALID_ARG;
    if (params && (params->lambda_mode != HYDE_LAMBDA_SHARED || params->threshold_ll != 0))
        return HYDE_ERR_INVALID_ARG;
    HyresLayout L;
    hyde_status st = hyres_layout(p, H, W, params, &L);
    if (st != HYDE_OK) return st;
    BackLayout B;
    back_layout(L, params->r_max, params->levels, &B);
    *bytes = B.total;
    return HYDE_OK;
}

hyde_status hyde_hyres_backward(const float* Y, const float* dX, int p, int H, int W,
                                const hyde_hyres_params* params, const float* scale, int loss,
                                float* dscale, double* sure_value, const void* fws,
                                size_t fws_bytes, void* bws, size_t bws_bytes,
                                cudaStream_t stream) {
    if (!Y || !scale || !dscale || (loss != 0 && loss != 1)) return HYDE_ERR_INVALID_ARG;
    if (loss == 0 && !dX) return HYDE_ERR_INVALID_ARG;
    if (params && (params->lambda_mode != HYDE_LAMBDA_SHARED || params->threshold_ll != 0))
        return HYDE_ERR_INVALID_ARG;
    HyresLayout L;
    hyde_status st = hyres_layout(p, H, W, params, &L);
    if (st != HYDE_OK) return st;
    BackLayout B;
    back_layout(L, params->r_max, params->levels, &B);
    if (!fws || !aligned(fws, kAlign) || fws_bytes < L.pub.total) return HYDE_ERR_WORKSPACE;
    if (!bws || !aligned(bws, kAlign) || bws_bytes < B.total) return HYDE_ERR_WORKSPACE;
    void* f = const_cast<void*>(fws);
    const int r = params->r_max, lev = params->levels;
    const float* P = at<float>(f, L.P);
    const float* Q = at<float>(f, L.Q);
    const int* rank_dev = at<int>(f, L.rank_dev);
    const double* lam_dev = at<double>(f, L.lam_dev);
    float* C = at<float>(bws, B.C);
    float* dC = at<float>(bws, B.dC);
    float* zp = at<float>(bws, B.zp);
    float* scratch = at<float>(bws, B.scratch);
    double* acc = at<double>(bws, B.acc);
    double* sacc = at<double>(bws, B.sure_acc);
#define HYDE_TRY(x) do { hyde_status s_ = (x); if (s_ != HYDE_OK) return s_; } while (0)
    if (cudaMemsetAsync(bws, 0, B.C, stream) != cudaSuccess) return HYDE_ERR_CUDA;
    // recompute the forward coefficients C = DWT(pad(Y P))
    HYDE_TRY(launch_project_pad(Y, p, H, W, P, r, L.RM, zp, L.Hp, L.Wp, stream));
    DwtSrc src{zp, L.N, L.Wp, L.Hp, L.Wp};
    HYDE_TRY(launch_dwt2(src, C, r, L.Hp, L.Wp, lev, scratch, stream));
    if (loss == 0) {
        // adjoint of back-projection, crop and inverse DWT: dC = DWT(zero-embed(Q^T dX))
        HYDE_TRY(launch_project_pad(dX, p, H, W, Q, r, L.RM, zp, L.Hp, L.Wp, stream, true));
        HYDE_TRY(launch_dwt2(src, dC, r, L.Hp, L.Wp, lev, scratch, stream));
    }
    HYDE_TRY(launch_scale_grad(C, loss == 0 ? dC : nullptr, r, L.Hp, L.Wp, lev, rank_dev, lam_dev,
                               scale, lev, loss, acc, sacc, stream));
    HYDE_TRY(launch_scale_grad_finish(acc, r, lev, rank_dev, lam_dev, dscale, lev, loss, L.N,
                                      sacc, sure_value, stream));
#undef HYDE_TRY
    return HYDE_OK;
}

// ------------------------------------------------------- sliding windows
// SMs a window's multi-block kernels are sized for. The one-block kernels
// (Gauss-Jordan, eigensolver, each with most of an SM's shared memory) carry
// most of the window form's GPU time; grids sized for all SMs leave them no
// free SM. Measured on the 2048 x 2048 x 200 scene (512 windows, 64 slots):
// 46.0 ms per scene uncapped, 41.0 at 38 SMs, 37.5 at 10, 37.8 at 6, 41.6
// at 4, 58.3 at 2.
constexpr int kWindowSmCap = 10;
static int window_sm_cap() { return kWindowSmCap; }

static hyde_status window_valid(const hyde_window& wn, int H, int W) {
    if (wn.h < 1 || wn.w < 1 || wn.y0 < 0 || wn.x0 < 0 || wn.y0 + wn.h > H || wn.x0 + wn.w > W)
        return HYDE_ERR_SHAPE;
    if (wn.ch < 1 || wn.cw < 1 || wn.cy0 < wn.y0 || wn.cx0 < wn.x0 ||
        wn.cy0 + wn.ch > wn.y0 + wn.h || wn.cx0 + wn.cw > wn.x0 + wn.w)
        return HYDE_ERR_SHAPE;
    return HYDE_OK;
}

struct SlotLayout {
    size_t cube_in, cube_out, hyres, stride;
};

static hyde_status slot_layout(int p, const hyde_window* win, int n_win,
                               const hyde_hyres_params* params, SlotLayout* S) {
    size_t max_cube = 0, max_ws = 0;
    for (int k = 0; k < n_win; ++k) {
        HyresLayout L;
        hyde_status st = hyres_layout(p, win[k].h, win[k].w, params, &L);
        if (st != HYDE_OK) return st;
        if (L.pub.total > max_ws) max_ws = L.pub.total;
        const size_t cube = (size_t)p * win[k].h * win[k].w * sizeof(float);
        if (cube > max_cube) max_cube = cube;
    }
    Carver c;
    SlotLayout s;
    s.cube_in = c.take(max_cube);
    s.cube_out = c.take(max_cube);
    s.hyres = c.take(max_ws);
    s.stride = c.off;
    *S = s;
    return HYDE_OK;
}

hyde_status hyde_windows_workspace_size(int p, int H, int W, const hyde_window* win, int n_win,
                                        const hyde_hyres_params* params, int n_slots,
                                        size_t* bytes) {
    if (!win || !bytes || n_win < 1 || n_slots < 1) return HYDE_ERR_INVALID_ARG;
    const SmCap sm_cap(window_sm_cap());
    for (int k = 0; k < n_win; ++k) {
        hyde_status st = window_valid(win[k], H, W);
        if (st != HYDE_OK) return st;
    }
    SlotLayout S;
    hyde_status st = slot_layout(p, win, n_win, params, &S);
    if (st != HYDE_OK) return st;
    const int slots = n_slots < n_win ? n_slots : n_win;
    *bytes = S.stride * (size_t)slots;
    return HYDE_OK;
}

hyde_status hyde_hyres_denoise_windows(const float* Y, float* X, int p, int H, int W,
                                       const hyde_window* win, int n_win,
                                       const hyde_hyres_params* params,
                                       hyde_hyres_info* info, void* ws, size_t ws_bytes,
                                       const cudaStream_t* streams, int n_slots,
                                       cudaEvent_t* events, cudaStream_t stream) {
    if (!Y || !X || Y == X || !win || !streams || !events || n_win < 1 || n_slots < 1)
        return HYDE_ERR_INVALID_ARG;
    const SmCap sm_cap(window_sm_cap());   // also around the workspace query below
    size_t need = 0;
    hyde_status st = hyde_windows_workspace_size(p, H, W, win, n_win, params, n_slots, &need);
    if (st != HYDE_OK) return st;
    if (!ws || !aligned(ws, kAlign) || ws_bytes < need) return HYDE_ERR_WORKSPACE;
    SlotLayout S;
    slot_layout(p, win, n_win, params, &S);
    const int slots = n_slots < n_win ? n_slots : n_win;
    const PdlOff plain_launches;   // concurrent slot streams: ordinary stream order
    // fork: every slot stream waits for the work already on the caller's stream
    if (cudaEventRecord(events[slots], stream) != cudaSuccess) return HYDE_ERR_CUDA;
    for (int s = 0; s < slots; ++s)
        if (cudaStreamWaitEvent(streams[s], events[slots], 0) != cudaSuccess) return HYDE_ERR_CUDA;
    for (int k = 0; k < n_win; ++k) {
        const int s = k % slots;
        cudaStream_t ss = streams[s];
        char* base = reinterpret_cast<char*>(ws) + S.stride * (size_t)s;
        float* cin = reinterpret_cast<float*>(base + S.cube_in);
        float* cout = reinterpret_cast<float*>(base + S.cube_out);
        void* hws = base + S.hyres;
        const hyde_window& wn = win[k];
        st = launch_gather_window(Y, H, W, wn.y0, wn.x0, wn.h, wn.w, p, cin, ss);
        if (st != HYDE_OK) return st;
        st = hyres_enqueue(cin, cout, p, wn.h, wn.w, params, info ? info + k : nullptr, hws,
                           S.stride - S.hyres, ss, nullptr);
        if (st != HYDE_OK) return st;
        st = launch_scatter_core(cout, wn.h, wn.w, wn.y0, wn.x0, wn.cy0, wn.cx0, wn.ch, wn.cw, p,
                                 H, W, X, ss);
        if (st != HYDE_OK) return st;
    }
    // join
    for (int s = 0; s < slots; ++s) {
        if (cudaEventRecord(events[s], streams[s]) != cudaSuccess) return HYDE_ERR_CUDA;
        if (cudaStreamWaitEvent(stream, events[s], 0) != cudaSuccess) return HYDE_ERR_CUDA;
    }
    return HYDE_OK;
}

int hyde_set_grid_sm_cap(int sms) {
    const int prev = tl_sm_cap;
    tl_sm_cap = sms > 0 ? sms : 0;
    return prev;
}

unsigned long long hyde_set_wait_limit_ns(unsigned long long ns) {
    const unsigned long long prev = tl_wait_ns;
    tl_wait_ns = ns;
    return prev;
}

int hyde_hyres_kernel_launches(int p, int H, int W, const hyde_hyres_params* params) {
    if (!params || params->levels < 1 || params->levels > kMaxLevels || p < 1) return -1;
    if (params->lambda_mode != HYDE_LAMBDA_SHARED &&
        params->lambda_mode != HYDE_LAMBDA_PER_COMPONENT &&
        params->lambda_mode != HYDE_LAMBDA_PER_LEVEL)
        return -1;
    if (params->threshold_ll != 0 && params->threshold_ll != 1) return -1;
    int Hp, Wp;
    if (!padded(H, W, params->levels, &Hp, &Wp)) return -1;
    // gram 2, noise 2, eig 3 (tridiagonalisation, eigenpairs, orthonormalisation),
    // weights 1, projection 1, DWT, SURE 2, IDWT, back 1 (the workspace carve
    // keeps the DWT buffers 16-byte aligned, so the coarse levels always run
    // fused where the shape allows)
    return 12 + 2 * dwt_launches(Hp, Wp, params->levels);
}

}  // extern "C"

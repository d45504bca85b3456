// Plan and entry point of the batched sliding-window form (arXiv 2204.06979:
// the tiles of a large scene each denoised by HyRes, Sec. 2.2.2 and 2.1).
//
// The plan turns the host window table into device tables (one WinDesc per
// window, the Gram pieces, the tile tables of the projections) and a
// workspace layout. It keeps the tables in page-locked host memory; each call
// copies them into the workspace on the caller's stream and then launches
// every stage once per group of windows. The windows form two groups, each
// run on its own stream (the caller's and one the plan owns, forked and
// joined with events): the one-block-per-window stages of one group (the
// Gauss-Jordan inverse, the tridiagonalisation, the eigenpairs, all bound by
// the latency of one SM) then share the SMs with the bandwidth- and
// tensor-bound stages of the other. A call is one capturable sequence of 24
// kernels whatever the number of windows.
#include <math.h>
#include <string.h>

#include <vector>

#include "hyde_internal.cuh"

using namespace hyde;

#ifndef HYDE_WIN_GROUPS
#define HYDE_WIN_GROUPS 2
#endif
namespace {
constexpr int kGroups = HYDE_WIN_GROUPS;
static_assert(kGroups >= 1, "at least one window group");
constexpr int kSideSlots = kGroups > 1 ? kGroups - 1 : 1;
}

struct WinGroup {
    int w0, n;                       // windows [w0, w0 + n)
    int G0, G1, proj_tiles, back_tiles;
    size_t pieces, pbeg, wslot0, wslot1, tproj, tback;   // table offsets
    size_t part0, part1;             // its Gram partials
};

struct hyde_windows_plan_s {
    int p, H, W, n_win, r, L, K, RM, ngroups, sms;
    int proj_tile;           // tuned: projection tile (padded pixels)
    double w1x;              // tuned: weight of the Gram's second band role
    std::vector<int4> geo_v;             // (y0, x0, h, w) per window
    std::vector<long long> npad;         // padded pixels per window
    std::vector<int> tback_v;            // back-projection tile prefix
    WinGroup g[kGroups];
    void* host;              // page-locked copy of the tables
    size_t tables;           // their bytes (the head of the workspace)
    cudaStream_t side[kSideSlots];       // the streams of groups 1, 2, ...
    cudaEvent_t fork, join[kSideSlots];
    // workspace offsets
    size_t desc, geo;
    size_t status, R, sigma, Ainv, S, eig, eig_stride, evals, V, P, Q;
    size_t zp, coef, scr, counts, sums, sum_all, rank, lam, total;
};

namespace {

struct Carve {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off += align_up(bytes, kAlign);
        return o;
    }
};

hyde_status window_ok(const hyde_window& wn, int H, int W) {
    if (wn.h < 1 || wn.w < 1 || wn.y0 < 0 || wn.x0 < 0 || wn.y0 + wn.h > H || wn.x0 + wn.w > W)
        return HYDE_ERR_SHAPE;
    if (wn.ch < 1 || wn.cw < 1 || wn.cy0 < wn.y0 || wn.cx0 < wn.x0 ||
        wn.cy0 + wn.ch > wn.y0 + wn.h || wn.cx0 + wn.cw > wn.x0 + wn.w)
        return HYDE_ERR_SHAPE;
    return HYDE_OK;
}

// Fixed-point unit 2^-sh of the window SURE histogram: rn(c^2 2^sh) < 2^22
// for every binned coefficient (|c| <= (K - 1) delta, with margin), and one
// lane column (N / 32 values in a block over N coefficients) below 2^32.
bool sure_shift(long long N, int K, double delta, int* sh_out) {
    const float inv_delta = (float)(1.0 / delta);
    const double q = (K - 1) / (double)inv_delta;
    const double c2max = q * q * 1.001 + 1e-300;
    const double per_col = (double)((N + 31) / 32);
    for (int sh = 16; sh >= 0; --sh) {
        const double sc = ldexp(1.0, sh);
        if (c2max * sc >= 4194304.0) continue;
        const double qmax = floor(c2max * sc) + 1.0;
        if (qmax * per_col < 4294967295.0) {
            *sh_out = sh;
            return true;
        }
    }
    return false;
}

template <typename T>
T* at(void* base, size_t off) {
    return reinterpret_cast<T*>(reinterpret_cast<char*>(base) + off);
}

}  // namespace

// The tables that depend on the tuned parameters (the Gram pieces and CTA
// split of each group, the projection tile tables), written into the plan's
// page-locked copy. The workspace is carved for every setting at once.
static hyde_status fill_tables(hyde_windows_plan_s* P, int tile, double w1x) {
    if (tile < 256 || tile > 4096 || (tile % 256) != 0 || !(w1x > 0.0) || w1x > 16.0)
        return HYDE_ERR_INVALID_ARG;
    for (int gi = 0; gi < P->ngroups; ++gi) {
        WinGroup& g = P->g[gi];
        WinGramLayout G;
        const hyde_status st = win_gram_layout(P->p, P->geo_v.data() + g.w0, g.n, P->sms, w1x, &G);
        if (st != HYDE_OK) return st;
        // the carve holds at most sms + n pieces per role and sms + 1 CTA starts
        if (G.pieces.size() > (size_t)2 * (P->sms + g.n) || G.pbeg.size() > (size_t)P->sms + 1)
            return HYDE_ERR_SHAPE;
        g.G0 = G.G0;
        g.G1 = G.G1;
        std::vector<int> tp(g.n + 1, 0), tb(g.n + 1, 0);
        for (int k = 0; k < g.n; ++k) {
            tp[k + 1] = tp[k] + (int)((P->npad[g.w0 + k] + tile - 1) / tile);
            tb[k + 1] = P->tback_v[g.w0 + k + 1] - P->tback_v[g.w0];
        }
        g.proj_tiles = tp[g.n];
        g.back_tiles = tb[g.n];
        memset(at<char>(P->host, g.pieces), 0, (size_t)2 * (P->sms + g.n) * sizeof(int4));
        if (!G.pieces.empty())
            memcpy(at<char>(P->host, g.pieces), G.pieces.data(), G.pieces.size() * sizeof(int4));
        memcpy(at<char>(P->host, g.pbeg), G.pbeg.data(), G.pbeg.size() * sizeof(int));
        memcpy(at<char>(P->host, g.wslot0), G.wslot0.data(), (g.n + 1) * sizeof(int));
        memcpy(at<char>(P->host, g.wslot1), G.wslot1.data(), (g.n + 1) * sizeof(int));
        memcpy(at<char>(P->host, g.tproj), tp.data(), (g.n + 1) * sizeof(int));
        memcpy(at<char>(P->host, g.tback), tb.data(), (g.n + 1) * sizeof(int));
    }
    P->proj_tile = tile;
    P->w1x = w1x;
    return HYDE_OK;
}

extern "C" {

hyde_status hyde_windows_plan_create(int p, int H, int W, const hyde_window* win, int n_win,
                                     const hyde_hyres_params* params, hyde_windows_plan* out) {
    if (!win || !params || !out || n_win < 1) return HYDE_ERR_INVALID_ARG;
    *out = nullptr;
    if (params->wavelet != 2 || params->levels < 1 || params->levels > kMaxLevels ||
        params->r_max < 1 || params->r_max > kMaxRank || params->r_max > p ||
        params->n_lambda < 2 || params->n_lambda > 256)
        return HYDE_ERR_INVALID_ARG;
    if ((params->precision != HYDE_PREC_FP32 && params->precision != HYDE_PREC_TF32X3) ||
        params->lambda_mode != HYDE_LAMBDA_SHARED || params->threshold_ll != 0)
        return HYDE_ERR_INVALID_ARG;
    if (n_win > 65535 || p < 1 || p > 208 || H < 1 || W < 1 || (W % 4) != 0)
        return HYDE_ERR_SHAPE;
    const int r = params->r_max, L = params->levels, K = params->n_lambda;
    std::vector<WinDesc> D(n_win);
    std::vector<int4> geo(n_win);
    std::vector<int> tback(n_win + 1, 0);
    long long img = 0, scr = 0;
    for (int k = 0; k < n_win; ++k) {
        const hyde_window& wn = win[k];
        hyde_status st = window_ok(wn, H, W);
        if (st != HYDE_OK) return st;
        int Hp, Wp;
        if ((wn.x0 % 4) != 0 || !padded_dims(wn.h, wn.w, L, &Hp, &Wp)) return HYDE_ERR_SHAPE;
        const long long N = (long long)Hp * Wp;
        if (N > (1LL << 30)) return HYDE_ERR_SHAPE;
        WinDesc d = {};
        d.y0 = wn.y0; d.x0 = wn.x0; d.h = wn.h; d.w = wn.w;
        d.cy0 = wn.cy0; d.cx0 = wn.cx0; d.ch = wn.ch; d.cw = wn.cw;
        d.Hp = Hp; d.Wp = Wp;
        d.img = img;
        d.scr = scr;
        d.delta = sqrt(2.0 * log((double)N)) / (K - 1);
        if (!sure_shift(N, K, d.delta, &d.sh)) return HYDE_ERR_SHAPE;
        img += (long long)align_up((size_t)(r * N), 64);
        scr += (long long)align_up((size_t)(r * win_scratch_stride(N)), 64);
        D[k] = d;
        geo[k] = make_int4(wn.y0, wn.x0, wn.h, wn.w);
        tback[k + 1] =
            tback[k] + (int)(((long long)wn.ch * wn.cw + kWinBackTile - 1) / kWinBackTile);
    }
    const int sms = device_sm_count();
    if (sms <= 0) return HYDE_ERR_CUDA;
    const int ngroups = n_win >= kGroups ? kGroups : 1;
    // groups of consecutive windows with about equal pixel counts
    int wb[kGroups + 1] = {0};
    {
        long long tot = 0;
        for (int k = 0; k < n_win; ++k) tot += (long long)win[k].h * win[k].w;
        long long acc = 0;
        int gi = 1;
        for (int k = 0; k < n_win && gi < ngroups; ++k) {
            acc += (long long)win[k].h * win[k].w;
            if (acc * ngroups >= tot * gi && k + 1 < n_win) wb[gi++] = k + 1;
        }
        for (; gi < ngroups; ++gi) wb[gi] = wb[gi - 1] + 1;
        wb[ngroups] = n_win;
    }

    hyde_windows_plan_s* P = new hyde_windows_plan_s();
    P->p = p; P->H = H; P->W = W; P->n_win = n_win; P->r = r; P->L = L; P->K = K;
    P->RM = (r + 3) / 4 * 4;
    P->ngroups = ngroups;
    P->sms = sms;
    P->geo_v = geo;
    P->npad.resize(n_win);
    for (int k = 0; k < n_win; ++k) P->npad[k] = (long long)D[k].Hp * D[k].Wp;
    P->tback_v = tback;
    const size_t n = (size_t)n_win, pp = (size_t)p * p;
    const size_t rows0 = (size_t)(p < 128 ? p : 128), rows1 = (size_t)(p > 128 ? p - 128 : 0);
    Carve c;
    P->desc = c.take(n * sizeof(WinDesc));
    P->geo = c.take(n * sizeof(int4));
    for (int gi = 0; gi < ngroups; ++gi) {
        WinGroup& g = P->g[gi];
        g.w0 = wb[gi];
        g.n = wb[gi + 1] - wb[gi];
        g.pieces = c.take((size_t)2 * (sms + g.n) * sizeof(int4));
        g.pbeg = c.take((size_t)(sms + 1) * sizeof(int));
        g.wslot0 = c.take((g.n + 1) * sizeof(int));
        g.wslot1 = c.take((g.n + 1) * sizeof(int));
        g.tproj = c.take((g.n + 1) * sizeof(int));
        g.tback = c.take((g.n + 1) * sizeof(int));
    }
    P->tables = c.off;
    P->status = c.take((n + 1) * sizeof(int));
    P->R = c.take(n * pp * sizeof(double));
    P->sigma = c.take(n * p * sizeof(double));
    P->Ainv = c.take(n * pp * sizeof(float));
    P->S = c.take(n * p * sizeof(double));
    P->eig_stride = align_up(eig_ws_bytes(p, r), kAlign);
    P->eig = c.take(n * P->eig_stride);
    P->evals = c.take(n * r * sizeof(double));
    P->V = c.take(n * p * r * sizeof(double));
    P->P = c.take(n * p * P->RM * sizeof(float));
    P->Q = c.take(n * p * P->RM * sizeof(float));
    P->zp = c.take((size_t)img * sizeof(float));
    P->coef = c.take((size_t)img * sizeof(float));
    P->scr = c.take((size_t)(scr > 0 ? scr : 4) * sizeof(float));
    P->counts = c.take(n * r * K * sizeof(unsigned int));
    P->sums = c.take(n * r * K * sizeof(double));
    P->sum_all = c.take(n * r * sizeof(double));
    P->rank = c.take(n * sizeof(int));
    P->lam = c.take(n * sizeof(double));
    for (int gi = 0; gi < ngroups; ++gi) {
        // a role's pieces: at most one per CTA plus one per window boundary
        const size_t slots = (size_t)sms + P->g[gi].n;
        P->g[gi].part0 = c.take((slots * rows0 * p > 0 ? slots * rows0 * p : 4) * sizeof(float));
        P->g[gi].part1 = c.take((slots * rows1 * rows1 > 0 ? slots * rows1 * rows1 : 4) * sizeof(float));
    }
    P->total = c.off;

    if (cudaMallocHost(&P->host, P->tables) != cudaSuccess) {
        P->host = nullptr;
        hyde_windows_plan_destroy(P);
        return HYDE_ERR_CUDA;
    }
    bool made = cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int gi = 0; made && gi + 1 < kGroups; ++gi)
        made = cudaStreamCreateWithFlags(&P->side[gi], cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreateWithFlags(&P->join[gi], cudaEventDisableTiming) == cudaSuccess;
    if (!made) {
        hyde_windows_plan_destroy(P);
        return HYDE_ERR_CUDA;
    }
    memset(P->host, 0, P->tables);
    memcpy(at<char>(P->host, P->desc), D.data(), n * sizeof(WinDesc));
    memcpy(at<char>(P->host, P->geo), geo.data(), n * sizeof(int4));
    // defaults: the settings measured best on the 2048 x 2048 x 200 scene
    const hyde_status st = fill_tables(P, 256, 1.6);
    if (st != HYDE_OK) {
        hyde_windows_plan_destroy(P);
        return st;
    }
    *out = P;
    return HYDE_OK;
}

hyde_status hyde_windows_plan_workspace_size(hyde_windows_plan plan, size_t* bytes) {
    if (!plan || !bytes) return HYDE_ERR_INVALID_ARG;
    *bytes = plan->total;
    return HYDE_OK;
}

int hyde_windows_plan_kernel_launches(hyde_windows_plan plan) {
    // per group: Gram 2, noise 1, eigensolver 3, weights 1, projection 1,
    // DWT with the SURE histogram 1, SURE selection 1, inverse DWT 1,
    // back-projection 1
    return plan ? 12 * plan->ngroups : -1;
}

hyde_status hyde_windows_plan_set_tuning(hyde_windows_plan plan, int proj_tile,
                                         double gram_role_weight) {
    if (!plan) return HYDE_ERR_INVALID_ARG;
    return fill_tables(plan, proj_tile, gram_role_weight);
}

hyde_status hyde_windows_plan_get_tuning(hyde_windows_plan plan, int* proj_tile,
                                         double* gram_role_weight) {
    if (!plan || !proj_tile || !gram_role_weight) return HYDE_ERR_INVALID_ARG;
    *proj_tile = plan->proj_tile;
    *gram_role_weight = plan->w1x;
    return HYDE_OK;
}

hyde_status hyde_windows_plan_layout(hyde_windows_plan plan, hyde_windows_ws_layout* out) {
    if (!plan || !out) return HYDE_ERR_INVALID_ARG;
    out->R = plan->R;
    out->sigma = plan->sigma;
    out->V = plan->V;
    return HYDE_OK;
}

hyde_status hyde_windows_plan_destroy(hyde_windows_plan plan) {
    if (!plan) return HYDE_ERR_INVALID_ARG;
    if (plan->host) cudaFreeHost(plan->host);
    for (int gi = 0; gi + 1 < kGroups; ++gi) {
        if (plan->side[gi]) cudaStreamDestroy(plan->side[gi]);
        if (plan->join[gi]) cudaEventDestroy(plan->join[gi]);
    }
    if (plan->fork) cudaEventDestroy(plan->fork);
    delete plan;
    return HYDE_OK;
}

// One group's stages on stream s: per-window arrays from the group's first
// window on, its own Gram pieces, partials and tile tables.
static hyde_status enqueue_group(const hyde_windows_plan_s* P, const WinGroup& g, const float* Y,
                                 float* X, hyde_hyres_info* info, void* ws, cudaStream_t s) {
    const int p = P->p, n = g.n, r = P->r, w0 = g.w0;
    const size_t pp = (size_t)p * p;
    const WinDesc* desc = at<WinDesc>(ws, P->desc) + w0;
    int* status = at<int>(ws, P->status) + w0;
    int* gstatus = at<int>(ws, P->status) + P->n_win;
    float* zp = at<float>(ws, P->zp);
    float* coef = at<float>(ws, P->coef);
    float* scr = at<float>(ws, P->scr);
    int* rank = at<int>(ws, P->rank) + w0;
    double* lam = at<double>(ws, P->lam) + w0;
    double* R = at<double>(ws, P->R) + w0 * pp;
    double* sigma = at<double>(ws, P->sigma) + (size_t)w0 * p;
    double* V = at<double>(ws, P->V) + (size_t)w0 * p * r;
    float* Pw = at<float>(ws, P->P) + (size_t)w0 * p * P->RM;
    float* Qw = at<float>(ws, P->Q) + (size_t)w0 * p * P->RM;
#define HYDE_TRY(x) do { hyde_status s_ = (x); if (s_ != HYDE_OK) return s_; } while (0)
    HYDE_TRY(launch_win_gram(Y, p, P->H, P->W, at<int4>(ws, g.pieces), at<int>(ws, g.pbeg),
                             at<int4>(ws, P->geo) + w0, at<int>(ws, g.wslot0),
                             at<int>(ws, g.wslot1), n, g.G0, g.G1, at<float>(ws, g.part0),
                             at<float>(ws, g.part1), R, gstatus, s));
    HYDE_TRY(launch_win_noise(R, p, n, desc, sigma, at<float>(ws, P->Ainv) + w0 * pp,
                              at<double>(ws, P->S) + (size_t)w0 * p, status, s));
    HYDE_TRY(launch_eig_top_batched(R, sigma, p, r, at<double>(ws, P->evals) + (size_t)w0 * r, V,
                                    at<char>(ws, P->eig) + (size_t)w0 * P->eig_stride,
                                    P->eig_stride, status, n, s));
    HYDE_TRY(launch_weights_batched(V, sigma, p, r, P->RM, Pw, Qw, n, s));
    HYDE_TRY(launch_win_project(Y, p, P->H, P->W, desc, at<int>(ws, g.tproj), n, g.proj_tiles,
                                P->proj_tile, Pw, r, P->RM, zp, s));
    unsigned int* counts = at<unsigned int>(ws, P->counts) + (size_t)w0 * r * P->K;
    double* sums = at<double>(ws, P->sums) + (size_t)w0 * r * P->K;
    double* sum_all = at<double>(ws, P->sum_all) + (size_t)w0 * r;
    HYDE_TRY(launch_win_dwt(zp, coef, scr, desc, n, r, P->L, P->K, counts, sums, sum_all, s));
    HYDE_TRY(launch_win_sure(desc, n, r, P->L, P->K, counts, sums, sum_all, rank, lam,
                             info ? info + w0 : nullptr, status, gstatus, s));
    HYDE_TRY(launch_win_idwt(coef, zp, scr, desc, n, r, P->L, rank, lam, s));
    HYDE_TRY(launch_win_backproject(zp, desc, at<int>(ws, g.tback), n, g.back_tiles, Qw, p,
                                    P->RM, rank, P->H, P->W, X, s));
#undef HYDE_TRY
    return HYDE_OK;
}

hyde_status hyde_hyres_denoise_windows_batched(const float* Y, float* X, hyde_windows_plan P,
                                               hyde_hyres_info* info, void* ws,
                                               size_t ws_bytes, cudaStream_t s) {
    if (!Y || !X || Y == X || !P) return HYDE_ERR_INVALID_ARG;
    if (((uintptr_t)Y % 16) != 0 || ((uintptr_t)X % 4) != 0) return HYDE_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws % kAlign) != 0 || ws_bytes < P->total) return HYDE_ERR_WORKSPACE;
    int* status = at<int>(ws, P->status);
    if (cudaMemcpyAsync(ws, P->host, P->tables, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(status, 0, (size_t)(P->n_win + 1) * sizeof(int), s) != cudaSuccess)
        return HYDE_ERR_CUDA;
    if (P->ngroups == 1) return enqueue_group(P, P->g[0], Y, X, info, ws, s);
    // groups 1, 2, ... on the plan's streams, forked from and joined back to s
    if (cudaEventRecord(P->fork, s) != cudaSuccess) return HYDE_ERR_CUDA;
    for (int gi = 1; gi < P->ngroups; ++gi)
        if (cudaStreamWaitEvent(P->side[gi - 1], P->fork, 0) != cudaSuccess) return HYDE_ERR_CUDA;
    hyde_status st = enqueue_group(P, P->g[0], Y, X, info, ws, s);
    for (int gi = 1; gi < P->ngroups; ++gi) {
        const hyde_status sg = enqueue_group(P, P->g[gi], Y, X, info, ws, P->side[gi - 1]);
        if (st == HYDE_OK) st = sg;
        if (cudaEventRecord(P->join[gi - 1], P->side[gi - 1]) != cudaSuccess ||
            cudaStreamWaitEvent(s, P->join[gi - 1], 0) != cudaSuccess)
            return HYDE_ERR_CUDA;
    }
    return st;
}

// Times every candidate setting on the caller's scene (one untimed call,
// then the median of three, CUDA events on `stream`) and keeps the fastest.
hyde_status hyde_windows_plan_autotune(hyde_windows_plan P, const float* Y, float* X, void* ws,
                                       size_t ws_bytes, cudaStream_t stream, float* best_ms) {
    if (!P) return HYDE_ERR_INVALID_ARG;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return HYDE_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return HYDE_ERR_INVALID_ARG;
    static const int kTiles[] = {256, 512, 1024};
    static const double kWeights[] = {1.2, 1.6, 2.0};
    const int nw = P->p > 128 ? 3 : 1;   // the weight only splits two band roles
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return HYDE_ERR_CUDA;
    }
    const int tile0 = P->proj_tile;
    const double w0 = P->w1x;
    int best_tile = tile0;
    double best_w = w0;
    float best = -1.f;
    hyde_status st = HYDE_OK;
    for (int ti = 0; ti < 3 && st == HYDE_OK; ++ti) {
        for (int wi = 0; wi < nw && st == HYDE_OK; ++wi) {
            const double w = nw == 1 ? w0 : kWeights[wi];
            // the previous setting's calls have finished: its tables may change
            if (cudaStreamSynchronize(stream) != cudaSuccess) { st = HYDE_ERR_CUDA; break; }
            st = fill_tables(P, kTiles[ti], w);
            if (st != HYDE_OK) break;
            float ms[3];
            for (int it = 0; it < 4 && st == HYDE_OK; ++it) {
                if (it > 0 && cudaEventRecord(e0, stream) != cudaSuccess) st = HYDE_ERR_CUDA;
                if (st == HYDE_OK)
                    st = hyde_hyres_denoise_windows_batched(Y, X, P, nullptr, ws, ws_bytes, stream);
                if (st == HYDE_OK && it > 0) {
                    if (cudaEventRecord(e1, stream) != cudaSuccess ||
                        cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms[it - 1], e0, e1) != cudaSuccess)
                        st = HYDE_ERR_CUDA;
                }
            }
            if (st != HYDE_OK) break;
            float a = ms[0], b = ms[1], c = ms[2];   // median of three
            const float med = a > b ? (b > c ? b : (a > c ? c : a)) : (a > c ? a : (b > c ? c : b));
            if (best < 0.f || med < best) {
                best = med;
                best_tile = kTiles[ti];
                best_w = w;
            }
        }
    }
    cudaStreamSynchronize(stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const hyde_status st2 = fill_tables(P, st == HYDE_OK ? best_tile : tile0,
                                        st == HYDE_OK ? best_w : w0);
    if (st != HYDE_OK) return st;
    if (best_ms) *best_ms = best;
    return st2;
}

}  // extern "C"

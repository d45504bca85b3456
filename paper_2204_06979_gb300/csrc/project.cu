// Rank-r_max projection onto the whitened spectral subspace and the
// back-projection with un-whitening (the low-rank model of HyRes, arXiv
// 2204.06979 Sec. 2.1):
//   Z_i(pixel) = sum_b Y_b(pixel) P[b][i],  P = D^-1 V   (D = diag(sigma))
//   X_b(pixel) = sum_{i < r*} Q[b][i] Zh_i(pixel),  Q = D V
// Both are skinny contractions (<= 32 outputs or inputs per pixel) at about
// the FP32/HBM balance point, so they stay on the FP32 pipes, with weights in
// shared memory read as broadcast float4 and the cube streamed band by band
// with coalesced accesses. The projection takes two pixels per thread (one
// weight load feeds eight FMAs), keeps two groups of 8 bands x 2 pixels of
// loads in flight per thread and writes straight into the padded H_p x W_p
// component images (whole-sample symmetric reflection at the bottom/right),
// so the DWT never sees an unpadded image; its two pixels per thread share
// each weight in one fma.rn.f32x2. The back-projection (one pixel per thread)
// unrolls to ceil(r*/4)*4 terms, r* read on the device; two pixels per thread
// there (paired FMAs, half the weight loads) measured slower, 113 against
// 109 us at C1: the extra registers cost a third of the resident warps.
#include "hyde_internal.cuh"

namespace hyde {
namespace {

constexpr int kThreads = 128;
constexpr int kBandGroup = 8;
constexpr int kPix = 2;   // pixels per thread: each broadcast weight feeds kPix FMAs
// The back-projection is bound by its stores (one per band and pixel):
// one pixel per thread and 256-thread blocks keep more warps resident.
constexpr int kBpThreads = 256;

// Source address of padded pixel pix (whole-sample reflection at the bottom
// and right edges); false for a padding pixel that is zero-filled instead.
__device__ __forceinline__ bool padded_source(long long pix, int H, int W, int Wp,
                                              int zero_pad, long long& src) {
    // 32-bit division when the padded image is below 2^31 pixels
    int y, x;
    if (pix < 0x7fffffffLL) {
        const int pi = (int)pix;
        y = pi / Wp;
        x = pi - y * Wp;
    } else {
        y = (int)(pix / Wp);
        x = (int)(pix - (long long)y * Wp);
    }
    if (zero_pad && (y >= H || x >= W)) { src = 0; return false; }
    if (y >= H) y = 2 * H - 2 - y;
    if (x >= W) x = 2 * W - 2 - x;
    src = (long long)y * W + x;
    return true;
}

// The two pixels of a thread share each weight: one paired FMA per component.
static_assert(kPix == 2, "the projection pairs its two pixels in fma.rn.f32x2");
template <int RM>
__device__ __forceinline__ void project_fma(float (&acc)[kPix][RM], const float (&v)[kPix],
                                            const float4* __restrict__ w4) {
#pragma unroll
    for (int q = 0; q < RM / 4; ++q) {
        const float4 w = w4[q];
        fma_f32x2(acc[0][4 * q + 0], acc[1][4 * q + 0], v[0], v[1], w.x, w.x);
        fma_f32x2(acc[0][4 * q + 1], acc[1][4 * q + 1], v[0], v[1], w.y, w.y);
        fma_f32x2(acc[0][4 * q + 2], acc[1][4 * q + 2], v[0], v[1], w.z, w.z);
        fma_f32x2(acc[0][4 * q + 3], acc[1][4 * q + 3], v[0], v[1], w.w, w.w);
    }
}

// Each thread projects kPix pixels (pix and pix + kThreads of its block's
// tile); the loads of band group g+1 are issued before the FMAs of group g.
template <int RM>
__global__ void __launch_bounds__(kThreads)
project_pad_kernel(const float* __restrict__ Y, int p, int H, int W,
                   const float* __restrict__ P, int r, float* __restrict__ Zp, int Hp,
                   int Wp, int zero_pad) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float4 Ps4[];   // p * RM / 4
    float* Ps = reinterpret_cast<float*>(Ps4);
    for (int e = threadIdx.x; e < p * RM; e += kThreads) Ps[e] = P[e];
    __syncthreads();
    const long long N = (long long)Hp * Wp, n = (long long)H * W;
    const long long tile = (long long)kThreads * kPix;
    for (long long base = (long long)blockIdx.x * tile; base < N;
         base += (long long)gridDim.x * tile) {
        long long src[kPix];
        bool live[kPix], data[kPix];
#pragma unroll
        for (int u = 0; u < kPix; ++u) {
            const long long pix = base + threadIdx.x + (long long)u * kThreads;
            live[u] = pix < N;
            data[u] = live[u] && padded_source(pix, H, W, Wp, zero_pad, src[u]);
            if (!data[u]) src[u] = 0;           // a valid address; the result is dropped
        }
        float acc[kPix][RM];
#pragma unroll
        for (int u = 0; u < kPix; ++u)
#pragma unroll
            for (int i = 0; i < RM; ++i) acc[u][i] = 0.f;
        const int pg = p - p % kBandGroup;      // bands in whole groups
        float v[kBandGroup][kPix];
        if (pg > 0) {
#pragma unroll
            for (int g = 0; g < kBandGroup; ++g)
#pragma unroll
                for (int u = 0; u < kPix; ++u) v[g][u] = __ldg(Y + (long long)g * n + src[u]);
        }
        for (int b = 0; b < pg; b += kBandGroup) {
            float nv[kBandGroup][kPix];
            const int bn = b + kBandGroup < pg ? b + kBandGroup : b;   // last group: reload
#pragma unroll
            for (int g = 0; g < kBandGroup; ++g)
#pragma unroll
                for (int u = 0; u < kPix; ++u)
                    nv[g][u] = __ldg(Y + (long long)(bn + g) * n + src[u]);
#pragma unroll
            for (int g = 0; g < kBandGroup; ++g)
                project_fma<RM>(acc, v[g], Ps4 + (b + g) * (RM / 4));
#pragma unroll
            for (int g = 0; g < kBandGroup; ++g)
#pragma unroll
                for (int u = 0; u < kPix; ++u) v[g][u] = nv[g][u];
        }
        for (int b = pg; b < p; ++b) {
            float vt[kPix];
#pragma unroll
            for (int u = 0; u < kPix; ++u) vt[u] = __ldg(Y + (long long)b * n + src[u]);
            project_fma<RM>(acc, vt, Ps4 + b * (RM / 4));
        }
#pragma unroll
        for (int u = 0; u < kPix; ++u) {
            if (!live[u]) continue;
            const long long pix = base + threadIdx.x + (long long)u * kThreads;
#pragma unroll
            for (int i = 0; i < RM; ++i)
                if (i < r) Zp[(long long)i * N + pix] = data[u] ? acc[u][i] : 0.f;
        }
    }
}

// X_b = sum_{i < R} Q[b][i] z_i for two pixels at once (component images of
// N pixels, pixel z0 written to X0 + b bs, z1 to X1 + b bs): every weight
// read from shared memory feeds both, in one paired FMA. The window form
// takes pixels c and c + kBpThreads of a tile, so that each store is
// coalesced; there one pixel per thread took 1.15 ms on the 2048 x 2048 x 200
// scene (short-scoreboard stalls on the weights leading) and two 0.79 ms. On
// the one-cube path (backproject_kernel, 349 x 1905 x 144) the same pairing
// measured 116 against 110 us, so that kernel keeps one pixel per thread.
template <int R, int RM>
__device__ __forceinline__ void backproject_pair(const float* __restrict__ Zh, int N, int z0,
                                                     int z1, bool two,
                                                     const float4* __restrict__ Qs4, int p, int r,
                                                     long long bs, float* __restrict__ X0,
                                                     float* __restrict__ X1) {
    float za[R], zb[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        za[i] = (i < r) ? __ldg(Zh + (long long)i * N + z0) : 0.f;
        zb[i] = (i < r && two) ? __ldg(Zh + (long long)i * N + z1) : 0.f;
    }
    for (int b = 0; b < p; ++b) {
        const float4* w4 = Qs4 + b * (RM / 4);
        float xa = 0.f, xb = 0.f;
#pragma unroll
        for (int q = 0; q < R / 4; ++q) {
            const float4 w = w4[q];
            fma_f32x2(xa, xb, za[4 * q + 0], zb[4 * q + 0], w.x, w.x);
            fma_f32x2(xa, xb, za[4 * q + 1], zb[4 * q + 1], w.y, w.y);
            fma_f32x2(xa, xb, za[4 * q + 2], zb[4 * q + 2], w.z, w.z);
            fma_f32x2(xa, xb, za[4 * q + 3], zb[4 * q + 3], w.w, w.w);
        }
        X0[(long long)b * bs] = xa;
        if (two) X1[(long long)b * bs] = xb;
    }
}

// X_b = sum_{i < R} Q[b][i] z_i for one pixel, R a multiple of 4 >= r*.
template <int R, int RM>
__device__ __forceinline__ void backproject_pixel(const float* __restrict__ Zh, long long n,
                                                  const float4* __restrict__ Qs4, int p, int r,
                                                  long long pix, float* __restrict__ X) {
    float z[R];
#pragma unroll
    for (int i = 0; i < R; ++i) z[i] = (i < r) ? __ldg(Zh + (long long)i * n + pix) : 0.f;
    for (int b = 0; b < p; ++b) {
        const float4* w4 = Qs4 + b * (RM / 4);
        float x = 0.f;
#pragma unroll
        for (int q = 0; q < R / 4; ++q) {
            const float4 w = w4[q];
            x = fmaf(z[4 * q + 0], w.x, x);
            x = fmaf(z[4 * q + 1], w.y, x);
            x = fmaf(z[4 * q + 2], w.z, x);
            x = fmaf(z[4 * q + 3], w.w, x);
        }
        X[(long long)b * n + pix] = x;
    }
}

template <int RM>
__global__ void __launch_bounds__(kBpThreads)
backproject_kernel(const float* __restrict__ Zh, long long n, const float* __restrict__ Q,
                   int p, const int* __restrict__ rank, float* __restrict__ X) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float4 Qs4[];
    float* Qs = reinterpret_cast<float*>(Qs4);
    for (int e = threadIdx.x; e < p * RM; e += kBpThreads) Qs[e] = Q[e];
    __syncthreads();
    const int r = min(*rank, RM);
    const int groups = (r + 3) / 4;
    for (long long pix = (long long)blockIdx.x * kBpThreads + threadIdx.x; pix < n;
         pix += (long long)gridDim.x * kBpThreads) {
        switch (groups) {
#define HYDE_BP_CASE(G) \
    case G: if (4 * G <= RM) backproject_pixel<4 * G, RM>(Zh, n, Qs4, p, r, pix, X); break;
            HYDE_BP_CASE(1) HYDE_BP_CASE(2) HYDE_BP_CASE(3) HYDE_BP_CASE(4)
            HYDE_BP_CASE(5) HYDE_BP_CASE(6) HYDE_BP_CASE(7) HYDE_BP_CASE(8)
#undef HYDE_BP_CASE
            default: break;
        }
    }
}

// --------------------------------------------------------------------------
// Batched sliding windows: one block per tile of one window (the window of
// tile t is found by bisection of the tile table), the window's weights in
// shared memory, the window read in place from the scene (row stride W, band
// stride H W).
// --------------------------------------------------------------------------
__device__ __forceinline__ int window_of_tile(const int* __restrict__ tstart, int n_win, int t) {
    int lo = 0, hi = n_win;   // tstart[lo] <= t < tstart[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(tstart + mid) <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Padded component images of a window: Zp[img + i Hp Wp + y Wp + x] for
// i < r, with whole-sample reflection of the window at its bottom and right.
template <int RM>
__global__ void __launch_bounds__(kThreads)
win_project_kernel(const float* __restrict__ Y, int p, int H, int W,
                   const WinDesc* __restrict__ desc, const int* __restrict__ tstart, int n_win,
                   int tile, const float* __restrict__ P, int r, float* __restrict__ Zp) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float4 Ps4[];
    float* Ps = reinterpret_cast<float*>(Ps4);
    const int t = blockIdx.x;
    const int wi = window_of_tile(tstart, n_win, t);
    const WinDesc d = desc[wi];
    const float* Pw = P + (long long)wi * p * RM;
    for (int e = threadIdx.x; e < p * RM; e += kThreads) Ps[e] = Pw[e];
    __syncthreads();
    const int N = d.Hp * d.Wp;
    const long long bs = (long long)H * W;
    const float* Yw = Y + (long long)d.y0 * W + d.x0;
    float* Zw = Zp + d.img;
    const int t0 = (t - __ldg(tstart + wi)) * tile;
    const int t1 = min(t0 + tile, N);
    for (int base = t0; base < t1; base += kThreads * kPix) {
        int src[kPix];
        bool live[kPix];
#pragma unroll
        for (int u = 0; u < kPix; ++u) {
            const int pix = base + threadIdx.x + u * kThreads;
            live[u] = pix < t1;
            int y = live[u] ? pix / d.Wp : 0;
            int x = live[u] ? pix - y * d.Wp : 0;
            if (y >= d.h) y = 2 * d.h - 2 - y;
            if (x >= d.w) x = 2 * d.w - 2 - x;
            src[u] = y * W + x;
        }
        float acc[kPix][RM];
#pragma unroll
        for (int u = 0; u < kPix; ++u)
#pragma unroll
            for (int i = 0; i < RM; ++i) acc[u][i] = 0.f;
        // the loads of band group g + 1 are issued before the FMAs of group g
        const int pg = p - p % kBandGroup;
        float v[kBandGroup][kPix];
        if (pg > 0) {
#pragma unroll
            for (int g = 0; g < kBandGroup; ++g)
#pragma unroll
                for (int u = 0; u < kPix; ++u) v[g][u] = __ldg(Yw + (long long)g * bs + src[u]);
        }
        for (int b0 = 0; b0 < pg; b0 += kBandGroup) {
            float nv[kBandGroup][kPix];
            const int bn = b0 + kBandGroup < pg ? b0 + kBandGroup : b0;   // last group: reload
#pragma unroll
            for (int g = 0; g < kBandGroup; ++g)
#pragma unroll
                for (int u = 0; u < kPix; ++u)
                    nv[g][u] = __ldg(Yw + (long long)(bn + g) * bs + src[u]);
#pragma unroll
            for (int g = 0; g < kBandGroup; ++g)
                project_fma<RM>(acc, v[g], Ps4 + (b0 + g) * (RM / 4));
#pragma unroll
            for (int g = 0; g < kBandGroup; ++g)
#pragma unroll
                for (int u = 0; u < kPix; ++u) v[g][u] = nv[g][u];
        }
        for (int b = pg; b < p; ++b) {
            float vt[kPix];
#pragma unroll
            for (int u = 0; u < kPix; ++u) vt[u] = __ldg(Yw + (long long)b * bs + src[u]);
            project_fma<RM>(acc, vt, Ps4 + b * (RM / 4));
        }
#pragma unroll
        for (int u = 0; u < kPix; ++u) {
            if (!live[u]) continue;
            const int pix = base + threadIdx.x + u * kThreads;
#pragma unroll
            for (int i = 0; i < RM; ++i)
                if (i < r) Zw[(long long)i * N + pix] = acc[u][i];
        }
    }
}

template <int RM>
__global__ void __launch_bounds__(kBpThreads)
win_backproject_kernel(const float* __restrict__ Zh, const WinDesc* __restrict__ desc,
                       const int* __restrict__ tstart, int n_win, const float* __restrict__ Q,
                       int p, const int* __restrict__ rank, int H, int W,
                       float* __restrict__ X) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float4 Qs4[];
    float* Qs = reinterpret_cast<float*>(Qs4);
    const int t = blockIdx.x;
    const int wi = window_of_tile(tstart, n_win, t);
    const WinDesc d = desc[wi];
    const float* Qw = Q + (long long)wi * p * RM;
    for (int e = threadIdx.x; e < p * RM; e += kBpThreads) Qs[e] = Qw[e];
    __syncthreads();
    const int r = min(rank[wi], RM);
    const int groups = (r + 3) / 4;
    const int N = d.Hp * d.Wp, n = d.ch * d.cw;
    const long long bs = (long long)H * W;
    const float* Zw = Zh + d.img;
    const int t0 = (t - __ldg(tstart + wi)) * kWinBackTile;
    const int t1 = min(t0 + kWinBackTile, n);
    for (int c = t0 + threadIdx.x; c < t1; c += 2 * kBpThreads) {
        const int c1 = c + kBpThreads;
        const bool two = c1 < t1;
        const int y0 = c / d.cw, x0 = c - y0 * d.cw;
        const int y1 = two ? c1 / d.cw : y0, x1 = two ? c1 - y1 * d.cw : x0;
        const int z0 = (d.cy0 - d.y0 + y0) * d.Wp + (d.cx0 - d.x0 + x0);
        const int z1 = (d.cy0 - d.y0 + y1) * d.Wp + (d.cx0 - d.x0 + x1);
        float* X0 = X + (long long)(d.cy0 + y0) * W + (d.cx0 + x0);
        float* X1 = X + (long long)(d.cy0 + y1) * W + (d.cx0 + x1);
        switch (groups) {
#define HYDE_WBP_CASE(G)                                                                          \
    case G:                                                                                       \
        if (4 * G <= RM)                                                                          \
            backproject_pair<4 * G, RM>(Zw, N, z0, z1, two, Qs4, p, r, bs, X0, X1);               \
        break;
            HYDE_WBP_CASE(1) HYDE_WBP_CASE(2) HYDE_WBP_CASE(3) HYDE_WBP_CASE(4)
            HYDE_WBP_CASE(5) HYDE_WBP_CASE(6) HYDE_WBP_CASE(7) HYDE_WBP_CASE(8)
#undef HYDE_WBP_CASE
            default: break;
        }
    }
}

// Grid of a grid-stride kernel: the blocks that fit on the device at once
// (occupancy of this kernel at this shared-memory size), fewer if the work
// has fewer tiles; small tiles (256 pixels) keep the last wave short.
int resident_grid(const void* func, int threads, size_t smem, long long tiles) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, smem) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    long long cap = (long long)device_sm_count() * per_sm;
    if (tiles < cap) cap = tiles;
    return cap < 1 ? 1 : (int)cap;
}

}  // namespace

hyde_status launch_project_pad(const float* Y, int p, int H, int W, const float* P, int r,
                               int ldw, float* Zp, int Hp, int Wp, cudaStream_t s,
                               bool zero_pad) {
    const long long N = (long long)Hp * Wp;
    const long long tiles = (N + kThreads * kPix - 1) / (kThreads * kPix);
    const size_t smem = (size_t)p * ldw * sizeof(float);
    if (smem > 227 * 1024) return HYDE_ERR_SHAPE;
    switch (ldw) {
#define HYDE_PROJ(RMV)                                                                         \
    case RMV:                                                                                  \
        if (ensure_smem_limit((const void*)project_pad_kernel<RMV>, (int)smem) != cudaSuccess) \
            return HYDE_ERR_CUDA;                                                              \
        launch_pdl(project_pad_kernel<RMV>,                                                    \
                   resident_grid((const void*)project_pad_kernel<RMV>, kThreads, smem, tiles), \
                   kThreads, smem, s, Y, p, H, W, P, r, Zp, Hp, Wp, zero_pad ? 1 : 0);          \
        break;
        HYDE_PROJ(4) HYDE_PROJ(8) HYDE_PROJ(12) HYDE_PROJ(16)
        HYDE_PROJ(20) HYDE_PROJ(24) HYDE_PROJ(28) HYDE_PROJ(32)
#undef HYDE_PROJ
        default: return HYDE_ERR_INVALID_ARG;
    }
    return cuda_status(cudaGetLastError());
}

hyde_status launch_backproject(const float* Zh, long long n, const float* Q, int p, int r_max,
                               int ldw, const int* rank, float* X, cudaStream_t s) {
    (void)r_max;
    const long long tiles = (n + kBpThreads - 1) / kBpThreads;
    const size_t smem = (size_t)p * ldw * sizeof(float);
    if (smem > 227 * 1024) return HYDE_ERR_SHAPE;
    switch (ldw) {
#define HYDE_BACK(RMV)                                                                         \
    case RMV:                                                                                  \
        if (ensure_smem_limit((const void*)backproject_kernel<RMV>, (int)smem) != cudaSuccess) \
            return HYDE_ERR_CUDA;                                                              \
        launch_pdl(backproject_kernel<RMV>,                                                    \
                   resident_grid((const void*)backproject_kernel<RMV>, kBpThreads, smem, tiles), \
                   kBpThreads, smem, s, Zh, n, Q, p, rank, X);                                  \
        break;
        HYDE_BACK(4) HYDE_BACK(8) HYDE_BACK(12) HYDE_BACK(16)
        HYDE_BACK(20) HYDE_BACK(24) HYDE_BACK(28) HYDE_BACK(32)
#undef HYDE_BACK
        default: return HYDE_ERR_INVALID_ARG;
    }
    return cuda_status(cudaGetLastError());
}

hyde_status launch_win_project(const float* Y, int p, int H, int W, const WinDesc* desc,
                               const int* tstart, int n_win, int n_tiles, int tile,
                               const float* P, int r, int ldw, float* Zp, cudaStream_t s) {
    const size_t smem = (size_t)p * ldw * sizeof(float);
    if (smem > 227 * 1024 || n_tiles < 1 || tile < 256 || (tile % 256) != 0) return HYDE_ERR_SHAPE;
    switch (ldw) {
#define HYDE_WPROJ(RMV)                                                                         \
    case RMV:                                                                                   \
        if (ensure_smem_limit((const void*)win_project_kernel<RMV>, (int)smem) != cudaSuccess)  \
            return HYDE_ERR_CUDA;                                                               \
        launch_pdl(win_project_kernel<RMV>, n_tiles, kThreads, smem, s, Y, p, H, W, desc, tstart, \
                   n_win, tile, P, r, Zp);                                                      \
        break;
        HYDE_WPROJ(4) HYDE_WPROJ(8) HYDE_WPROJ(12) HYDE_WPROJ(16)
        HYDE_WPROJ(20) HYDE_WPROJ(24) HYDE_WPROJ(28) HYDE_WPROJ(32)
#undef HYDE_WPROJ
        default: return HYDE_ERR_INVALID_ARG;
    }
    return cuda_status(cudaGetLastError());
}

hyde_status launch_win_backproject(const float* Zh, const WinDesc* desc, const int* tstart,
                                   int n_win, int n_tiles, const float* Q, int p, int ldw,
                                   const int* rank, int H, int W, float* X, cudaStream_t s) {
    const size_t smem = (size_t)p * ldw * sizeof(float);
    if (smem > 227 * 1024 || n_tiles < 1) return HYDE_ERR_SHAPE;
    switch (ldw) {
#define HYDE_WBACK(RMV)                                                                         \
    case RMV:                                                                                   \
        if (ensure_smem_limit((const void*)win_backproject_kernel<RMV>, (int)smem) !=           \
            cudaSuccess)                                                                        \
            return HYDE_ERR_CUDA;                                                               \
        launch_pdl(win_backproject_kernel<RMV>, n_tiles, kBpThreads, smem, s, Zh, desc, tstart, \
                   n_win, Q, p, rank, H, W, X);                                                 \
        break;
        HYDE_WBACK(4) HYDE_WBACK(8) HYDE_WBACK(12) HYDE_WBACK(16)
        HYDE_WBACK(20) HYDE_WBACK(24) HYDE_WBACK(28) HYDE_WBACK(32)
#undef HYDE_WBACK
        default: return HYDE_ERR_INVALID_ARG;
    }
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

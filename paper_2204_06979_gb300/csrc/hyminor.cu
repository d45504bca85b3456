// HyMiNoR (arXiv 2204.06979, Sec. 2.1): HyRes removes the Gaussian noise,
// then an l1-l1 problem removes the remaining sparse noise by a modified
// split-Bregman iteration. The paper states neither; the reading built here:
// per band image, min_x ||h - x||_1 + lam (||Dx x||_1 + ||Dy x||_1) on the
// HyRes output (Dx, Dy periodic forward differences: anisotropic total
// variation), split Bregman on A = h - x, Bx = Dx x, By = Dy x with penalty
// mu, the x-subproblem (5 x - neighbours = rhs) by two Jacobi sweeps from
// the current x. The problem is posed on h = G / max|G|; the iteration is
// positively homogeneous, so it runs on G itself with the thresholds 1/mu
// and lam/mu scaled by s = max|G|.
//
// State per voxel: x and, in place of (A, bA), (Bx, bx), (By, by), the
// sums t = h - x + bA, ux = Dx x + bx, uy = Dy x + by of the last step, from
// which A = shrink(t), bA = clip(t) (and likewise for ux, uy) follow:
// shrink(v, tau) + clip(v, tau) = v. One iteration is then one stencil
// kernel per 32 x 32 tile of a band image:
//   rhs = h - t + 2 clip(t, tA) + (wx(i, j-1) - wx(i, j)) + (wy(i-1, j) - wy(i, j)),
//         w = u - 2 clip(u, tB)  (= shrink(u) - clip(u));
//   x1 = (rhs + 4 neighbours of x) / 5;  x2 = (rhs + 4 neighbours of x1) / 5;
//   t' = h - x2 + clip(t, tA);  ux' = x2(i, j+1) - x2 + clip(ux, tB);
//   uy' = x2(i+1, j) - x2 + clip(uy, tB);
// with a halo of three pixels (wrapped periodically) recomputed in shared
// memory. Reads and writes ping-pong between two state sets (neighbouring
// tiles read the old halo). HBM-bound: ~41 bytes per voxel per iteration.
#include "hyde_internal.cuh"

namespace hyde {
namespace {

constexpr int kTs = 32;                 // tile side
constexpr int kTvThreads = 256;

__device__ __forceinline__ float clipf(float v, float t) { return fminf(fmaxf(v, -t), t); }
__device__ __forceinline__ int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Largest |G| over the cube into *smax (float bits, non-negative, cleared
// beforehand).
__global__ void maxabs_kernel(const float* __restrict__ G, long long total, unsigned int* smax) {
    pdl_wait();
    pdl_trigger();
    float m = 0.f;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(__ldg(G + e)));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 8));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    if ((threadIdx.x & 31) == 0) atomicMax(smax, __float_as_uint(m));
}

struct TvState {
    const float* x;
    const float* t;
    const float* ux;
    const float* uy;
};
struct TvOut {
    float* x;
    float* t;
    float* ux;
    float* uy;
};

// One split-Bregman iteration on tile (blockIdx.x, blockIdx.y) of band
// blockIdx.z (32 x 8 threads: threadIdx.x runs along the image rows).
// first: the state is x = h and t = ux = uy = 0 (not read).
__device__ __forceinline__ int wrap_near(int i, int n) {
    // the halo reaches at most three pixels past an edge; tiny images wrap
    // more than once
    if (i >= 0 && i < n) return i;
    return wrap(i, n);
}

__global__ void __launch_bounds__(kTvThreads)
tvl1_iter_kernel(const float* __restrict__ h, TvState in, TvOut out, int H, int W,
                 const unsigned int* __restrict__ smax, float inv_mu, float lam_inv_mu,
                 int first) {
    pdl_wait();
    pdl_trigger();
    constexpr int N0 = kTs + 5, N1 = kTs + 3, N2 = kTs + 1;
    __shared__ float s_x0[N0][N0 + 1];        // x at (y0-2+r, x0-2+c)
    __shared__ float s_wx[N1][kTs + 5];       // wx at (y0-1+r, x0-2+c)
    __shared__ float s_wy[kTs + 4][N1 + 1];   // wy at (y0-2+r, x0-1+c)
    __shared__ float s_rhs[N1][N1 + 1];       // rhs at (y0-1+r, x0-1+c)
    __shared__ float s_x1[N1][N1 + 1];        // x1 at (y0-1+r, x0-1+c)
    __shared__ float s_x2[N2][N2 + 1];        // x2 at (y0+r, x0+c)
    __shared__ int s_col[N0];                 // wrapped columns x0-2 .. x0+kTs+2
    __shared__ int s_row[N0];                 // wrapped rows y0-2 .. y0+kTs+2 (times W)
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int y0 = blockIdx.y * kTs, x0 = blockIdx.x * kTs;
    const long long off = (long long)blockIdx.z * H * W;
    const float s = __uint_as_float(*smax);
    const float tA = s * inv_mu, tB = s * lam_inv_mu;
    const float* hb = h + off;
    const float* xb = (first ? h : in.x) + off;
    const float* tb = in.t + off;
    const float* uxb = in.ux + off;
    const float* uyb = in.uy + off;
    const int lin = ty * 32 + tx;
    for (int i = lin; i < N0; i += kTvThreads) {
        s_col[i] = wrap_near(x0 - 2 + i, W);
        s_row[i] = wrap_near(y0 - 2 + i, H) * W;
    }
    __syncthreads();

    for (int r = ty; r < N0; r += 8) {
        const float* row = xb + s_row[r];
        for (int c = tx; c < N0; c += 32) s_x0[r][c] = __ldg(row + s_col[c]);
    }
    for (int r = ty; r < N1; r += 8) {           // wx rows y0-1.., columns x0-2..
        const int gr = s_row[r + 1];
        for (int c = tx; c < kTs + 4; c += 32) {
            float w = 0.f;
            if (!first) {
                const float u = __ldg(uxb + gr + s_col[c]);
                w = u - 2.0f * clipf(u, tB);
            }
            s_wx[r][c] = w;
        }
    }
    for (int r = ty; r < kTs + 4; r += 8) {      // wy rows y0-2.., columns x0-1..
        const int gr = s_row[r];
        for (int c = tx; c < N1; c += 32) {
            float w = 0.f;
            if (!first) {
                const float u = __ldg(uyb + gr + s_col[c + 1]);
                w = u - 2.0f * clipf(u, tB);
            }
            s_wy[r][c] = w;
        }
    }
    __syncthreads();
    // right-hand side and the first Jacobi sweep on the (kTs + 3)^2 region
    for (int r = ty; r < N1; r += 8) {
        const int gr = s_row[r + 1];
        for (int c = tx; c < N1; c += 32) {
            const int g = gr + s_col[c + 1];
            const float tv = first ? 0.f : __ldg(tb + g);
            const float rhs = __ldg(hb + g) - tv + 2.0f * clipf(tv, tA) +
                              (s_wx[r][c] - s_wx[r][c + 1]) + (s_wy[r][c] - s_wy[r + 1][c]);
            s_rhs[r][c] = rhs;
            const float nb =
                s_x0[r][c + 1] + s_x0[r + 2][c + 1] + s_x0[r + 1][c] + s_x0[r + 1][c + 2];
            s_x1[r][c] = (rhs + nb) * 0.2f;
        }
    }
    __syncthreads();
    // second sweep on the (kTs + 1)^2 region
    for (int r = ty; r < N2; r += 8) {
        for (int c = tx; c < N2; c += 32) {
            const float nb =
                s_x1[r][c + 1] + s_x1[r + 2][c + 1] + s_x1[r + 1][c] + s_x1[r + 1][c + 2];
            s_x2[r][c] = (s_rhs[r + 1][c + 1] + nb) * 0.2f;
        }
    }
    __syncthreads();
    // the tile's new state (coalesced rows of 32)
    const int gx = x0 + tx;
    if (gx >= W) return;
    for (int r = ty; r < kTs; r += 8) {
        const int gy = y0 + r;
        if (gy >= H) break;
        const long long g = off + (long long)gy * W + gx;
        const float x2 = s_x2[r][tx];
        float tv = 0.f, uxv = 0.f, uyv = 0.f;
        if (!first) {
            tv = __ldg(in.t + g);
            uxv = __ldg(in.ux + g);
            uyv = __ldg(in.uy + g);
        }
        out.x[g] = x2;
        out.t[g] = __ldg(h + g) - x2 + clipf(tv, tA);
        out.ux[g] = (s_x2[r][tx + 1] - x2) + clipf(uxv, tB);
        out.uy[g] = (s_x2[r + 1][tx] - x2) + clipf(uyv, tB);
    }
}

struct HmLayout {
    size_t hyres, smax, G, state[2][4], total;
};

hyde_status hm_layout(int p, int H, int W, const hyde_hyres_params* params, HmLayout* L) {
    size_t hy = 0;
    hyde_status st = hyde_workspace_size(p, H, W, params, &hy);
    if (st != HYDE_OK) return st;
    const size_t cube = align_up((size_t)p * H * W * sizeof(float), kAlign);
    HmLayout l;
    size_t off = 0;
    l.hyres = off;  off += align_up(hy, kAlign);
    l.smax = off;   off += kAlign;
    l.G = off;      off += cube;
    for (int k = 0; k < 2; ++k)
        for (int a = 0; a < 4; ++a) { l.state[k][a] = off; off += cube; }
    l.total = off;
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

extern "C" hyde_status hyde_hyminor_workspace_size(int p, int H, int W,
                                                   const hyde_hyres_params* params,
                                                   size_t* bytes) {
    if (!bytes) return HYDE_ERR_INVALID_ARG;
    HmLayout L;
    hyde_status st = hm_layout(p, H, W, params, &L);
    if (st != HYDE_OK) return st;
    *bytes = L.total;
    return HYDE_OK;
}

extern "C" hyde_status hyde_hyminor(const float* Y, float* X, int p, int H, int W,
                                    const hyde_hyres_params* params, float lam, float mu,
                                    int iters, hyde_hyres_info* info, void* ws,
                                    size_t ws_bytes, cudaStream_t stream) {
    if (!Y || !X || !params) return HYDE_ERR_INVALID_ARG;
    if (!(lam >= 0.f) || !(mu > 0.f) || !isfinite(lam) || !isfinite(mu)) return HYDE_ERR_INVALID_ARG;
    if (iters < 1 || iters > 100000) return HYDE_ERR_SHAPE;
    if ((long long)H * W > 0x7fffffffLL) return HYDE_ERR_SHAPE;   // one band image in int
    HmLayout L;
    hyde_status st = hm_layout(p, H, W, params, &L);
    if (st != HYDE_OK) return st;
    if (!ws || ((uintptr_t)ws % kAlign) != 0 || ws_bytes < L.total) return HYDE_ERR_WORKSPACE;
    float* G = at<float>(ws, L.G);
    unsigned int* smax = at<unsigned int>(ws, L.smax);
    size_t hy = 0;
    hyde_workspace_size(p, H, W, params, &hy);
    // 1. the Gaussian stage
    st = hyde_hyres_denoise(Y, G, p, H, W, params, info, at<void>(ws, L.hyres), hy, stream);
    if (st != HYDE_OK) return st;
    // 2. s = max |G|
    if (cudaMemsetAsync(smax, 0, sizeof(unsigned int), stream) != cudaSuccess) return HYDE_ERR_CUDA;
    const long long total = (long long)p * H * W;
    const int sms = device_sm_count();
    if (sms <= 0) return HYDE_ERR_CUDA;
    launch_pdl(maxabs_kernel, 4 * sms, 256, 0, stream, (const float*)G, total, smax);
    // 3-4. split Bregman, ping-pong between the two state sets; the last
    // iteration writes x into X
    const dim3 grid((unsigned)((W + kTs - 1) / kTs), (unsigned)((H + kTs - 1) / kTs), (unsigned)p);
    for (int k = 0; k < iters; ++k) {
        const int src = k & 1, dst = src ^ 1;
        TvState in{at<float>(ws, L.state[src][0]), at<float>(ws, L.state[src][1]),
                   at<float>(ws, L.state[src][2]), at<float>(ws, L.state[src][3])};
        TvOut out{k == iters - 1 ? X : at<float>(ws, L.state[dst][0]),
                  at<float>(ws, L.state[dst][1]), at<float>(ws, L.state[dst][2]),
                  at<float>(ws, L.state[dst][3])};
        launch_pdl(tvl1_iter_kernel, grid, dim3(32, kTvThreads / 32), 0, stream, (const float*)G,
                   in, out, H, W,
                   (const unsigned int*)smax, 1.0f / mu, lam / mu, k == 0 ? 1 : 0);
    }
    return cuda_status(cudaGetLastError());
}

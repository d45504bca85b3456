// Rank-r_max projection onto the whitened spectral subspace and the
// back-projection with un-whitening (the low-rank model of HyRes, arXiv
// 2204.06979 Sec. 2.1):
//   Z_i(pixel) = sum_b Y_b(pixel) P[b][i],  P = D^-1 V   (D = diag(sigma))
//   X_b(pixel) = sum_{i < r*} Q[b][i] Zh_i(pixel),  Q = D V
// Both are skinny contractions (<= 32 outputs or inputs per pixel) at about
// the FP32/HBM balance point, so they stay on the FP32 pipes: one thread per
// pixel, weights in shared memory read as broadcast float4, the cube streamed
// band by band with coalesced accesses. The projection keeps 8 bands of loads
// in flight per thread and writes straight into the padded H_p x W_p
// component images (whole-sample symmetric reflection at the bottom/right),
// so the DWT never sees an unpadded image. The back-projection unrolls to
// ceil(r*/4)*4 terms, r* read on the device.
#include "hyde_internal.cuh"

namespace hyde {
namespace {

constexpr int kThreads = 256;
constexpr int kBandGroup = 8;

template <int RM>
__global__ void __launch_bounds__(kThreads)
project_pad_kernel(const float* __restrict__ Y, int p, int H, int W,
                   const float* __restrict__ P, int r, float* __restrict__ Zp, int Hp,
                   int Wp, int zero_pad) {
    extern __shared__ float4 Ps4[];   // p * RM / 4
    float* Ps = reinterpret_cast<float*>(Ps4);
    for (int e = threadIdx.x; e < p * RM; e += kThreads) Ps[e] = P[e];
    __syncthreads();
    const long long N = (long long)Hp * Wp, n = (long long)H * W;
    for (long long pix = (long long)blockIdx.x * kThreads + threadIdx.x; pix < N;
         pix += (long long)gridDim.x * kThreads) {
        int y = (int)(pix / Wp), x = (int)(pix - (long long)(pix / Wp) * Wp);
        if (zero_pad && (y >= H || x >= W)) {
#pragma unroll
            for (int i = 0; i < RM; ++i)
                if (i < r) Zp[(long long)i * N + pix] = 0.f;
            continue;
        }
        if (y >= H) y = 2 * H - 2 - y;
        if (x >= W) x = 2 * W - 2 - x;
        const float* yp = Y + (long long)y * W + x;
        float acc[RM];
#pragma unroll
        for (int i = 0; i < RM; ++i) acc[i] = 0.f;
        int b = 0;
        for (; b + kBandGroup <= p; b += kBandGroup) {
            float v[kBandGroup];
#pragma unroll
            for (int u = 0; u < kBandGroup; ++u) v[u] = __ldg(yp + (long long)(b + u) * n);
#pragma unroll
            for (int u = 0; u < kBandGroup; ++u) {
                const float4* w4 = Ps4 + (b + u) * (RM / 4);
#pragma unroll
                for (int q = 0; q < RM / 4; ++q) {
                    const float4 w = w4[q];
                    acc[4 * q + 0] = fmaf(v[u], w.x, acc[4 * q + 0]);
                    acc[4 * q + 1] = fmaf(v[u], w.y, acc[4 * q + 1]);
                    acc[4 * q + 2] = fmaf(v[u], w.z, acc[4 * q + 2]);
                    acc[4 * q + 3] = fmaf(v[u], w.w, acc[4 * q + 3]);
                }
            }
        }
        for (; b < p; ++b) {
            const float v = __ldg(yp + (long long)b * n);
            const float4* w4 = Ps4 + b * (RM / 4);
#pragma unroll
            for (int q = 0; q < RM / 4; ++q) {
                const float4 w = w4[q];
                acc[4 * q + 0] = fmaf(v, w.x, acc[4 * q + 0]);
                acc[4 * q + 1] = fmaf(v, w.y, acc[4 * q + 1]);
                acc[4 * q + 2] = fmaf(v, w.z, acc[4 * q + 2]);
                acc[4 * q + 3] = fmaf(v, w.w, acc[4 * q + 3]);
            }
        }
#pragma unroll
        for (int i = 0; i < RM; ++i)
            if (i < r) Zp[(long long)i * N + pix] = acc[i];
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
__global__ void __launch_bounds__(kThreads)
backproject_kernel(const float* __restrict__ Zh, long long n, const float* __restrict__ Q,
                   int p, const int* __restrict__ rank, float* __restrict__ X) {
    extern __shared__ float4 Qs4[];
    float* Qs = reinterpret_cast<float*>(Qs4);
    for (int e = threadIdx.x; e < p * RM; e += kThreads) Qs[e] = Q[e];
    __syncthreads();
    const int r = min(*rank, RM);
    const int groups = (r + 3) / 4;
    for (long long pix = (long long)blockIdx.x * kThreads + threadIdx.x; pix < n;
         pix += (long long)gridDim.x * kThreads) {
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

int grid_for(long long items, int per_block, int blocks_per_sm) {
    int sms = device_sm_count();
    long long need = (items + per_block - 1) / per_block;
    long long cap = (long long)sms * blocks_per_sm;
    if (need > cap) need = cap;
    if (need < 1) need = 1;
    return (int)need;
}

}  // namespace

hyde_status launch_project_pad(const float* Y, int p, int H, int W, const float* P, int r,
                               int ldw, float* Zp, int Hp, int Wp, cudaStream_t s,
                               bool zero_pad) {
    const long long N = (long long)Hp * Wp;
    const int grid = grid_for(N, kThreads, 8);
    const size_t smem = (size_t)p * ldw * sizeof(float);
    if (smem > 227 * 1024) return HYDE_ERR_SHAPE;
    switch (ldw) {
#define HYDE_PROJ(RMV)                                                                         \
    case RMV:                                                                                  \
        if (ensure_smem_limit((const void*)project_pad_kernel<RMV>, (int)smem) != cudaSuccess) \
            return HYDE_ERR_CUDA;                                                              \
        project_pad_kernel<RMV><<<grid, kThreads, smem, s>>>(Y, p, H, W, P, r, Zp, Hp, Wp, \
                                                             zero_pad ? 1 : 0);                 \
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
    const int grid = grid_for(n, kThreads, 8);
    const size_t smem = (size_t)p * ldw * sizeof(float);
    if (smem > 227 * 1024) return HYDE_ERR_SHAPE;
    switch (ldw) {
#define HYDE_BACK(RMV)                                                                         \
    case RMV:                                                                                  \
        if (ensure_smem_limit((const void*)backproject_kernel<RMV>, (int)smem) != cudaSuccess) \
            return HYDE_ERR_CUDA;                                                              \
        backproject_kernel<RMV><<<grid, kThreads, smem, s>>>(Zh, n, Q, p, rank, X);            \
        break;
        HYDE_BACK(4) HYDE_BACK(8) HYDE_BACK(12) HYDE_BACK(16)
        HYDE_BACK(20) HYDE_BACK(24) HYDE_BACK(28) HYDE_BACK(32)
#undef HYDE_BACK
        default: return HYDE_ERR_INVALID_ARG;
    }
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

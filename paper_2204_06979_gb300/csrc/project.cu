// Rank-r_max projection onto the whitened spectral subspace and the
// back-projection with un-whitening (the low-rank model of HyRes, arXiv
// 2204.06979 Sec. 2.1):
//   Z_i(pixel) = sum_b Y_b(pixel) P[b][i],  P = D^-1 V   (D = diag(sigma))
//   X_b(pixel) = sum_{i < r*} Q[b][i] Zh_i(pixel),  Q = D V
// Both are skinny contractions (r_max <= 32 outputs or inputs per pixel):
// one thread per pixel (two pixels per thread for ILP), the weights in shared
// memory read as broadcast float4, the cube streamed band by band with
// coalesced loads/stores. The projection writes straight into the padded
// H_p x W_p component images (whole-sample symmetric reflection at the
// bottom/right), so the DWT never sees an unpadded image.
#include "hyde_internal.cuh"

namespace hyde {
namespace {

constexpr int kThreads = 256;

template <int RM>
__global__ void __launch_bounds__(kThreads)
project_pad_kernel(const float* __restrict__ Y, int p, int H, int W,
                   const float* __restrict__ P, int r, float* __restrict__ Zp, int Hp,
                   int Wp) {
    extern __shared__ float4 Ps4[];   // p * RM / 4
    float* Ps = reinterpret_cast<float*>(Ps4);
    for (int e = threadIdx.x; e < p * RM; e += kThreads) Ps[e] = P[e];
    __syncthreads();
    const long long N = (long long)Hp * Wp, n = (long long)H * W;
    const long long step = 2LL * kThreads * gridDim.x;
    for (long long base = 2LL * kThreads * blockIdx.x; base < N; base += step) {
        long long pix[2];
        long long src[2];
        bool ok[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            pix[u] = base + threadIdx.x + u * kThreads;
            ok[u] = pix[u] < N;
            const long long q = ok[u] ? pix[u] : 0;
            int y = (int)(q / Wp), x = (int)(q - (long long)(q / Wp) * Wp);
            if (y >= H) y = 2 * H - 2 - y;
            if (x >= W) x = 2 * W - 2 - x;
            src[u] = (long long)y * W + x;
        }
        float acc[2][RM];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int i = 0; i < RM; ++i) acc[u][i] = 0.f;
        const float* yb = Y;
        for (int b = 0; b < p; ++b, yb += n) {
            const float v0 = __ldg(yb + src[0]);
            const float v1 = __ldg(yb + src[1]);
            const float4* w4 = Ps4 + b * (RM / 4);
#pragma unroll
            for (int q = 0; q < RM / 4; ++q) {
                const float4 w = w4[q];
                acc[0][4 * q + 0] = fmaf(v0, w.x, acc[0][4 * q + 0]);
                acc[0][4 * q + 1] = fmaf(v0, w.y, acc[0][4 * q + 1]);
                acc[0][4 * q + 2] = fmaf(v0, w.z, acc[0][4 * q + 2]);
                acc[0][4 * q + 3] = fmaf(v0, w.w, acc[0][4 * q + 3]);
                acc[1][4 * q + 0] = fmaf(v1, w.x, acc[1][4 * q + 0]);
                acc[1][4 * q + 1] = fmaf(v1, w.y, acc[1][4 * q + 1]);
                acc[1][4 * q + 2] = fmaf(v1, w.z, acc[1][4 * q + 2]);
                acc[1][4 * q + 3] = fmaf(v1, w.w, acc[1][4 * q + 3]);
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (!ok[u]) continue;
#pragma unroll
            for (int i = 0; i < RM; ++i)
                if (i < r) Zp[(long long)i * N + pix[u]] = acc[u][i];
        }
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
    const int r = *rank;
    const long long step = 2LL * kThreads * gridDim.x;
    for (long long base = 2LL * kThreads * blockIdx.x; base < n; base += step) {
        const long long p0 = base + threadIdx.x, p1 = p0 + kThreads;
        const bool ok0 = p0 < n, ok1 = p1 < n;
        float z0[RM], z1[RM];
#pragma unroll
        for (int i = 0; i < RM; ++i) {
            z0[i] = (ok0 && i < r) ? __ldg(Zh + (long long)i * n + p0) : 0.f;
            z1[i] = (ok1 && i < r) ? __ldg(Zh + (long long)i * n + p1) : 0.f;
        }
        for (int b = 0; b < p; ++b) {
            const float4* w4 = Qs4 + b * (RM / 4);
            float x0 = 0.f, x1 = 0.f;
#pragma unroll
            for (int q = 0; q < RM / 4; ++q) {
                const float4 w = w4[q];
                x0 = fmaf(z0[4 * q + 0], w.x, x0);
                x0 = fmaf(z0[4 * q + 1], w.y, x0);
                x0 = fmaf(z0[4 * q + 2], w.z, x0);
                x0 = fmaf(z0[4 * q + 3], w.w, x0);
                x1 = fmaf(z1[4 * q + 0], w.x, x1);
                x1 = fmaf(z1[4 * q + 1], w.y, x1);
                x1 = fmaf(z1[4 * q + 2], w.z, x1);
                x1 = fmaf(z1[4 * q + 3], w.w, x1);
            }
            if (ok0) X[(long long)b * n + p0] = x0;
            if (ok1) X[(long long)b * n + p1] = x1;
        }
    }
}

int grid_for(long long items, int per_block) {
    int sms = device_sm_count();
    long long need = (items + per_block - 1) / per_block;
    long long cap = (long long)sms * 8;
    if (need > cap) need = cap;
    if (need < 1) need = 1;
    return (int)need;
}

}  // namespace

hyde_status launch_project_pad(const float* Y, int p, int H, int W, const float* P, int r,
                               int ldw, float* Zp, int Hp, int Wp, cudaStream_t s) {
    const long long N = (long long)Hp * Wp;
    const int grid = grid_for(N, 2 * kThreads);
    const size_t smem = (size_t)p * ldw * sizeof(float);
    if (smem > 227 * 1024) return HYDE_ERR_SHAPE;
    switch (ldw) {
#define HYDE_PROJ(RMV)                                                                       \
    case RMV:                                                                                \
        if (ensure_smem_limit((const void*)project_pad_kernel<RMV>, (int)smem) != cudaSuccess) \
            return HYDE_ERR_CUDA;                                                            \
        project_pad_kernel<RMV><<<grid, kThreads, smem, s>>>(Y, p, H, W, P, r, Zp, Hp, Wp); \
        break;
        HYDE_PROJ(8)
        HYDE_PROJ(16)
        HYDE_PROJ(24)
        HYDE_PROJ(32)
#undef HYDE_PROJ
        default: return HYDE_ERR_INVALID_ARG;
    }
    return cuda_status(cudaGetLastError());
}

hyde_status launch_backproject(const float* Zh, long long n, const float* Q, int p, int r_max,
                               int ldw, const int* rank, float* X, cudaStream_t s) {
    (void)r_max;
    const int grid = grid_for(n, 2 * kThreads);
    const size_t smem = (size_t)p * ldw * sizeof(float);
    if (smem > 227 * 1024) return HYDE_ERR_SHAPE;
    switch (ldw) {
#define HYDE_BACK(RMV)                                                                      \
    case RMV:                                                                               \
        if (ensure_smem_limit((const void*)backproject_kernel<RMV>, (int)smem) != cudaSuccess) \
            return HYDE_ERR_CUDA;                                                           \
        backproject_kernel<RMV><<<grid, kThreads, smem, s>>>(Zh, n, Q, p, rank, X);         \
        break;
        HYDE_BACK(8)
        HYDE_BACK(16)
        HYDE_BACK(24)
        HYDE_BACK(32)
#undef HYDE_BACK
        default: return HYDE_ERR_INVALID_ARG;
    }
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

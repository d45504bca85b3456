// Differentiation form of HyRes: gradients with respect to per-(component,
// level) threshold scales s[i][l], with lambda_il = lambda* s[i][l] and the
// rank r* and base threshold lambda* chosen by SURE at s = 1 and held fixed.
// The paper's package makes conventional methods differentiable with autograd
// and trains a HyRes step in front of a DNN (arXiv 2204.06979, Sec. 2.1,
// Sec. 2.2); this file holds the reduction at the end of the hand-written
// adjoint:
//   loss given dL/dX:  dL/ds_il = lambda* sum_{level l, comp i} dC (-sign C) [|C| > lambda_il]
//   SURE loss:         dL/ds_il = lambda* sum 2 lambda_il [|C| > lambda_il]
//                      (the count term of SURE is piecewise constant in s)
// where C are the forward wavelet coefficients (recomputed, not stored) and
// dC = DWT(zero-embedded Q^T dL/dX) is the adjoint of the inverse transform
// (the DWT is orthogonal, so the inverse transform's transpose is the DWT).
#include "hyde_internal.cuh"

namespace hyde {
namespace {

constexpr int kThreads = 256;

// level (1..L) of Mallat position (y, x); 0 for the final LL band
__device__ __forceinline__ int level_of(int y, int x, int Hp, int Wp, int L) {
#pragma unroll 1
    for (int l = 1; l <= L; ++l)
        if (y >= (Hp >> l) || x >= (Wp >> l)) return l;
    return 0;
}

__global__ void __launch_bounds__(kThreads)
scale_grad_kernel(const float* __restrict__ C, const float* __restrict__ dC, int Hp, int Wp,
                  int L, const int* __restrict__ rank, const double* __restrict__ lam,
                  const float* __restrict__ scale, int scale_ld, int mode, int rows_per_block,
                  double* __restrict__ acc, double* __restrict__ sure_acc) {
    pdl_wait();
    pdl_trigger();
    __shared__ float s_lam[kMaxLevels];
    __shared__ float s_part[kMaxLevels][kThreads];   // private column per thread
    const int i = blockIdx.y;
    if (i >= *rank) return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid < L) s_lam[tid] = (float)(*lam) * scale[(long long)i * scale_ld + tid];
    for (int l = 0; l < L; ++l) s_part[l][tid] = 0.f;
    __syncthreads();
    const long long N = (long long)Hp * Wp;
    const float* Ci = C + (long long)i * N;
    const float* Di = dC ? dC + (long long)i * N : nullptr;
    const int y0 = blockIdx.x * rows_per_block, y1 = min(y0 + rows_per_block, Hp);
    float sval = 0.f;
    for (int y = y0 + wid; y < y1; y += kThreads / 32) {
        for (int x = lane; x < Wp; x += 32) {
            const int l = level_of(y, x, Hp, Wp, L);
            if (l == 0) continue;
            const float c = Ci[(long long)y * Wp + x];
            const float lv = s_lam[l - 1];
            const bool kept = fabsf(c) > lv;
            if (mode == 0) {
                if (kept) {
                    const float g = Di[(long long)y * Wp + x];
                    s_part[l - 1][tid] += (c > 0.f) ? -g : (c < 0.f ? g : 0.f);
                }
            } else {
                if (kept) {
                    s_part[l - 1][tid] += 2.f * lv;
                    sval += lv * lv;
                } else {
                    sval += c * c - 2.f;
                }
            }
        }
    }
    if (mode == 1) {
        sval = warp_sum(sval);
        if (lane == 0) atomicAdd(sure_acc, (double)sval);
    }
    __syncthreads();
    for (int l = wid; l < L; l += kThreads / 32) {
        float v = 0.f;
        for (int q = lane; q < kThreads; q += 32) v += s_part[l][q];
        v = warp_sum(v);
        if (lane == 0 && v != 0.f) atomicAdd(&acc[(long long)i * L + l], (double)v);
    }
}

__global__ void scale_grad_finish_kernel(const double* __restrict__ acc, int r_max, int L,
                                         const int* __restrict__ rank,
                                         const double* __restrict__ lam,
                                         float* __restrict__ dscale, int ld, int mode,
                                         long long N, const double* __restrict__ sure_acc,
                                         double* __restrict__ sure_value) {
    pdl_wait();
    pdl_trigger();
    const int r = *rank;
    for (int e = threadIdx.x; e < r_max * L; e += blockDim.x) {
        const int i = e / L, l = e % L;
        dscale[(long long)i * ld + l] = i < r ? (float)((*lam) * acc[e]) : 0.f;
    }
    if (mode == 1 && threadIdx.x == 0 && sure_value)
        *sure_value = (double)r * (double)N + *sure_acc;
}

}  // namespace

hyde_status launch_scale_grad(const float* C, const float* dC, int r_max, int Hp, int Wp,
                              int levels, const int* rank, const double* lam,
                              const float* scale, int scale_ld, int mode, double* acc,
                              double* sure_acc, cudaStream_t s) {
    if (levels < 1 || levels > kMaxLevels) return HYDE_ERR_SHAPE;
    const int sms = device_sm_count();
    if (sms <= 0) return HYDE_ERR_CUDA;
    int per = (4 * sms + r_max - 1) / r_max;
    if (per > Hp) per = Hp;
    if (per < 1) per = 1;
    const int rows = (Hp + per - 1) / per;
    per = (Hp + rows - 1) / rows;
    dim3 grid(per, r_max);
    launch_pdl(scale_grad_kernel, grid, kThreads, 0, s, C, dC, Hp, Wp, levels, rank, lam, scale,
               scale_ld, mode, rows, acc, sure_acc);
    return cuda_status(cudaGetLastError());
}

hyde_status launch_scale_grad_finish(const double* acc, int r_max, int levels, const int* rank,
                                     const double* lam, float* dscale, int dscale_ld, int mode,
                                     long long N, const double* sure_acc, double* sure_value,
                                     cudaStream_t s) {
    launch_pdl(scale_grad_finish_kernel, 1, 256, 0, s, acc, r_max, levels, rank, lam, dscale,
               dscale_ld, mode, N, sure_acc, sure_value);
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

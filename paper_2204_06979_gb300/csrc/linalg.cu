// Small dense linear algebra of the HyRes path (arXiv 2204.06979, Sec. 2.1):
//
//  * noise level by multiple regression: sigma_b^2 = 1 / (n [R^-1]_bb), the
//    residual power of regressing band b on all other bands (the Schur
//    complement of the normal equations);
//  * the float projection / back-projection weights V/sigma and V*sigma.
// (The eigensolver of the whitened Gram matrix is in eig.cu.)
//
// GB300 runs FP64 at 1/64 of its FP32 rate, so the O(p^3) work is done in
// FP32 inside one thread block and FP64 is used where it buys accuracy
// cheaply: the diagonal of the inverse gets one Newton correction in double,
// spread over p blocks.
//
// The p-step Gauss-Jordan recurrence is latency- and issue-bound on one SM,
// so for p <= 200 the matrix lives in registers: a G x G thread grid where
// thread (ty, tx) owns the T x T tile of rows ty*T.. and columns tx*T.. . A
// step then costs T^2 FMAs per thread plus one barrier; the pivot row and
// column are published through small double-buffered shared vectors. Larger
// p falls back to a kernel that keeps the matrix in shared memory.
#include <float.h>

#include "hyde_internal.cuh"


namespace hyde {
namespace {

constexpr int kLA = 1024;     // threads of the single-block kernels

// --------------------------------------------------------------------------
// Noise level, part 1: Gauss-Jordan inverse (no pivoting: the matrix is SPD)
// of As = S^-1 R S^-1, S = sqrt(diag R), in float; writes As^-1 and S.
// Pivots of the unit-diagonal matrix are Schur complements >= its smallest
// eigenvalue; below ~16 ulp the float inverse is meaningless (exactly
// collinear bands give ~1 ulp), which is reported as HYDE_ERR_NUMERIC.
// --------------------------------------------------------------------------
constexpr float kPivotFloor = 2e-6f;

// The G x G threads form a grid over the matrix: thread (ty, tx) owns the
// T x T tile of rows ty T.. and columns tx T.. in registers. A step costs T^2
// FMAs and 2T shared loads per thread plus one barrier; the pivot row and
// column are published through double-buffered shared vectors. G = 16 (256
// threads, up to 13 x 13 tiles: p <= 208) keeps the per-thread work of a step
// high and the number of warps that repeat the pivot arithmetic low.
template <int T, int G>
__device__ __forceinline__ void noise_gj_reg_body(const double* __restrict__ R, int p,
                                                  float* __restrict__ Ainv,
                                                  double* __restrict__ S, int* status) {
    pdl_wait();
    pdl_trigger();
    __shared__ float s_inv[G * T];
    __shared__ float s_row[2][G * T];
    __shared__ float s_col[2][G * T];
    const int t = threadIdx.x, tx = t % G, ty = t / G;
    const int r0 = ty * T, c0 = tx * T;
    for (int i = t; i < G * T; i += G * G) {
        float inv = 0.f;
        if (i < p) {
            const double d = R[(long long)i * p + i];
            if (!(d > 0.0) || !isfinite(d)) set_status(status, HYDE_ERR_NUMERIC);
            const double sd = d > 0.0 ? sqrt(d) : 1.0;
            S[i] = sd;
            inv = (float)(1.0 / sd);
        }
        s_inv[i] = inv;
    }
    __syncthreads();
    float a[T][T];
#pragma unroll
    for (int ii = 0; ii < T; ++ii) {
        const int i = r0 + ii;
#pragma unroll
        for (int jj = 0; jj < T; ++jj) {
            const int j = c0 + jj;
            float v = (i == j) ? 1.f : 0.f;      // identity on the padding
            if (i < p && j < p) v = (float)R[(long long)i * p + j] * s_inv[i] * s_inv[j];
            a[ii][jj] = v;
        }
    }
    // Steps k = kt T + ko with ko unrolled: the pivot row and column of the
    // register tile are compile-time indices (no runtime selection).
    for (int kt = 0; kt * T < p; ++kt) {
#pragma unroll
        for (int ko = 0; ko < T; ++ko) {
            const int k = kt * T + ko;
            if (k < p) {
                const int buf = k & 1;
                if (ty == kt) {
#pragma unroll
                    for (int jj = 0; jj < T; ++jj) s_row[buf][c0 + jj] = a[ko][jj];
                }
                if (tx == kt) {
#pragma unroll
                    for (int ii = 0; ii < T; ++ii) s_col[buf][r0 + ii] = a[ii][ko];
                }
                __syncthreads();   // one barrier per step: the vectors are double-buffered
                const float pk = s_col[buf][k];
                if (t == 0 && !(pk > kPivotFloor)) set_status(status, HYDE_ERR_NUMERIC);
                // ~1 ulp reciprocal: the FP64 Newton step on the diagonal follows
                const float piv = __fdividef(1.0f, pk);
                float rk[T], ck[T];
#pragma unroll
                for (int q = 0; q < T; ++q) {
                    rk[q] = s_row[buf][c0 + q];
                    ck[q] = s_col[buf][r0 + q] * piv;
                }
#pragma unroll
                for (int ii = 0; ii < T; ++ii)
#pragma unroll
                    for (int jj = 0; jj < T; ++jj) a[ii][jj] = fmaf(-ck[ii], rk[jj], a[ii][jj]);
                if (ty == kt) {   // row k: a_kj * piv
#pragma unroll
                    for (int jj = 0; jj < T; ++jj) a[ko][jj] = rk[jj] * piv;
                }
                if (tx == kt) {   // column k: -a_ik * piv, and the pivot itself
#pragma unroll
                    for (int ii = 0; ii < T; ++ii) a[ii][ko] = (ty == kt && ii == ko) ? piv : -ck[ii];
                }
            }
        }
    }
#pragma unroll
    for (int ii = 0; ii < T; ++ii) {
        const int i = r0 + ii;
#pragma unroll
        for (int jj = 0; jj < T; ++jj) {
            const int j = c0 + jj;
            if (i < p && j < p) Ainv[(long long)i * p + j] = a[ii][jj];
        }
    }
}

template <int T, int G>
__global__ void __launch_bounds__(G * G, 1)
noise_gj_reg_kernel(const double* __restrict__ R, int p, float* __restrict__ Ainv,
                    double* __restrict__ S, int* status) {
    noise_gj_reg_body<T, G>(R, p, Ainv, S, status);
}


// Shared-memory Gauss-Jordan for p > 208 (same arithmetic, matrix in smem).
__global__ void __launch_bounds__(kLA, 1)
noise_gj_smem_kernel(const double* __restrict__ R, int p, float* __restrict__ Ainv,
                     double* __restrict__ S, int* status) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float sm[];
    float* A = sm;                  // p * p
    float* colk = A + p * p;        // p
    float* rowk = colk + p;         // p   (first holds 1 / S in float)
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int i = t; i < p; i += blockDim.x) {
        double d = R[(long long)i * p + i];
        if (!(d > 0.0) || !isfinite(d)) set_status(status, HYDE_ERR_NUMERIC);
        const double sd = d > 0.0 ? sqrt(d) : 1.0;
        S[i] = sd;
        rowk[i] = (float)(1.0 / sd);
    }
    __syncthreads();
    for (int i = wid; i < p; i += 32) {
        const float si = rowk[i];
        for (int j = lane; j < p; j += 32)
            A[i * p + j] = (float)R[(long long)i * p + j] * si * rowk[j];
    }
    __syncthreads();
    for (int k = 0; k < p; ++k) {
        for (int i = t; i < p; i += blockDim.x) {
            colk[i] = A[i * p + k];
            rowk[i] = A[k * p + i];
        }
        __syncthreads();
        const float pk = colk[k];
        if (t == 0 && !(pk > kPivotFloor)) set_status(status, HYDE_ERR_NUMERIC);
        const float piv = 1.0f / pk;
        for (int i = wid; i < p; i += 32) {
            const float ci = -colk[i] * piv;
            for (int j = lane; j < p; j += 32) {
                float v;
                if (i == k) v = (j == k) ? piv : rowk[j] * piv;
                else if (j == k) v = ci;
                else v = fmaf(ci, rowk[j], A[i * p + j]);
                A[i * p + j] = v;
            }
        }
        __syncthreads();
    }
    for (int e = t; e < p * p; e += blockDim.x) Ainv[e] = A[e];
}

// --------------------------------------------------------------------------
// Noise level, part 2 (block b): x = column b of X0 = S^-1 As^-1 S^-1 (the
// float inverse of R), d_b = 2 x_b - x^T R x (one Newton step X0(2I - R X0)
// for the diagonal, in double), sigma_b = sqrt(1 / (n d_b)).
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
noise_refine_kernel(const double* __restrict__ R, const float* __restrict__ Ainv,
                    const double* __restrict__ S, int p, long long n,
                    double* __restrict__ sigma, int* status) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ double xs[];   // p
    __shared__ double red[8];
    const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    const double sb = S[b];
    for (int i = t; i < p; i += blockDim.x)
        xs[i] = (double)Ainv[(long long)i * p + b] / (S[i] * sb);
    __syncthreads();
    // x^T R x = sum_i x_i sum_j R_ij x_j: each lane keeps its own share of
    // the double sum (rows w + 8m, columns lane + 32q); one warp sum at the end.
    // Rows go in groups of kRefRows whose loads are all issued before the
    // first FMA, so the warp waits on L2 once per group, not once per row.
    constexpr int kRefRows = 4;
    double part = 0.0;
    for (int i0 = w; i0 < p; i0 += 8 * kRefRows) {
        double rv[kRefRows][8];
#pragma unroll
        for (int m = 0; m < kRefRows; ++m) {
            const int i = i0 + 8 * m;
            const double* Ri = R + (long long)(i < p ? i : 0) * p;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int j = lane + 32 * q;
                rv[m][q] = (i < p && j < p) ? __ldg(Ri + j) : 0.0;
            }
        }
#pragma unroll
        for (int m = 0; m < kRefRows; ++m) {
            const int i = i0 + 8 * m;
            if (i >= p) break;
            const double* Ri = R + (long long)i * p;
            double u = 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int j = lane + 32 * q;
                if (j < p) u = fma(rv[m][q], xs[j], u);
            }
            for (int j = lane + 256; j < p; j += 32) u = fma(__ldg(Ri + j), xs[j], u);
            part = fma(xs[i], u, part);
        }
    }
    part = warp_sum_d(part);
    if (lane == 0) red[w] = part;
    __syncthreads();
    if (t == 0) {
        double q = 0.0;
        for (int i = 0; i < 8; ++i) q += red[i];
        double d = 2.0 * xs[b] - q;
        double s2 = 1.0 / ((double)n * d);
        if (!(d > 0.0) || !isfinite(s2) || !(s2 > 0.0)) {
            set_status(status, HYDE_ERR_NUMERIC);
            s2 = 1.0;
        }
        sigma[b] = sqrt(s2);
    }
}

__global__ void weights_kernel(const double* __restrict__ V, const double* __restrict__ sigma,
                               int p, int r, int ldw, float* __restrict__ P,
                               float* __restrict__ Q) {
    pdl_wait();
    pdl_trigger();
    // window blockIdx.y of a batched call (one window: gridDim.y = 1)
    const int wi = blockIdx.y;
    V += (long long)wi * p * r;
    sigma += (long long)wi * p;
    P += (long long)wi * p * ldw;
    Q += (long long)wi * p * ldw;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p * ldw;
         e += gridDim.x * blockDim.x) {
        int b = e / ldw, i = e % ldw;
        double v = i < r ? V[(long long)b * r + i] : 0.0;
        P[e] = (float)(v / sigma[b]);
        Q[e] = (float)(v * sigma[b]);
    }
}

// --------------------------------------------------------------------------
// Noise levels of the windows of a batched sliding-window call, one window
// per block: the register Gauss-Jordan inverse of the window's scaled Gram
// matrix, then sigma_b = S_b / sqrt(n_w [As^-1]_bb) (n_w the window's
// pixels) straight from the float inverse. The FP64 Newton step of the
// one-cube path costs p^3 double FMAs per window, which over hundreds of
// windows would take longer than the whole batched call; without it sigma
// carries the float inverse's error (~1e-5 relative at p = 200).
// --------------------------------------------------------------------------
template <int T, int G>
__global__ void __launch_bounds__(G * G, 1)
win_noise_kernel(const double* __restrict__ R, int p, const WinDesc* __restrict__ desc,
                 double* __restrict__ sigma, float* __restrict__ Ainv, double* __restrict__ S,
                 int* status) {
    const int w = blockIdx.x;
    const long long pp = (long long)p * p;
    float* Aw = Ainv + w * pp;
    double* Sw = S + (long long)w * p;
    noise_gj_reg_body<T, G>(R + w * pp, p, Aw, Sw, status + w);
    __syncthreads();   // the block's global writes of Aw and Sw are visible to it
    const double n = (double)desc[w].h * (double)desc[w].w;
    for (int b = threadIdx.x; b < p; b += G * G) {
        const double a = (double)Aw[(long long)b * p + b];
        double s2 = Sw[b] * Sw[b] / (n * a);
        if (!(a > 0.0) || !isfinite(s2) || !(s2 > 0.0)) {
            set_status(status + w, HYDE_ERR_NUMERIC);
            s2 = 1.0;
        }
        sigma[(long long)w * p + b] = sqrt(s2);
    }
}

// --------------------------------------------------------------------------
// Full inverse (block b): column b of Q = R^-1 in double from the float
// inverse X0 = S^-1 As^-1 S^-1 by one Newton step X0 (2I - R X0): with
// x = column b of X0 and u = R x, q_b = 2 x - X0 u. One warp per row, lanes
// over the columns, double sums.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
inverse_refine_kernel(const double* __restrict__ R, const float* __restrict__ Ainv,
                      const double* __restrict__ S, int p, double* __restrict__ Q,
                      int* status) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ double xs[];   // x [p], u [p], 1/S [p]
    double* us = xs + p;
    double* is = xs + 2 * p;
    const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    constexpr int nw = 256 / 32;
    for (int i = t; i < p; i += blockDim.x) is[i] = 1.0 / S[i];
    __syncthreads();
    for (int i = t; i < p; i += blockDim.x)
        xs[i] = (double)Ainv[(long long)i * p + b] * is[i] * is[b];
    __syncthreads();
    for (int i = w; i < p; i += nw) {
        double acc = 0.0;
        for (int j = lane; j < p; j += 32) acc = fma(__ldg(R + (long long)i * p + j), xs[j], acc);
        acc = warp_sum_d(acc);
        if (lane == 0) us[i] = acc;
    }
    __syncthreads();
    for (int i = w; i < p; i += nw) {
        double acc = 0.0;
        for (int j = lane; j < p; j += 32)
            acc = fma((double)Ainv[(long long)i * p + j] * is[j], us[j], acc);
        acc = warp_sum_d(acc) * is[i];
        if (lane == 0) {
            const double v = 2.0 * xs[i] - acc;
            if (!isfinite(v)) set_status(status, HYDE_ERR_NUMERIC);
            Q[(long long)i * p + b] = v;
        }
    }
}


}  // namespace

size_t noise_ws_bytes(int p) {
    return align_up((size_t)p * p * sizeof(float), kAlign) +
           align_up((size_t)p * sizeof(double), kAlign);
}

// A 16 x 16 thread grid with T x T register tiles covers p <= 16 T; T <= 13
// (p <= 208) stays in registers without spilling (244 at T = 13, one block
// of 256 threads). A 20 x 20 grid of 10 x 10 tiles measured 259 against
// 217 us at p = 200 (it spills at 400 threads). Larger p use the
// shared-memory kernel.
constexpr int kGjRegMax = 208;

size_t noise_smem_bytes(int p) {
    return p <= kGjRegMax ? 0 : ((size_t)p * p + 2 * p) * sizeof(float);
}

// The float inverse of the scaled Gram matrix into ws (Ainv, then the
// scales S): a register-tile Gauss-Jordan kernel for p <= 208, the
// shared-memory kernel above.
static hyde_status launch_gj_inverse(const double* R, int p, void* ws, int* status,
                                     cudaStream_t s) {
    float* Ainv = reinterpret_cast<float*>(ws);
    double* Sd = reinterpret_cast<double*>(reinterpret_cast<char*>(ws) +
                                           align_up((size_t)p * p * sizeof(float), kAlign));
    const int T16 = (p + 15) / 16;
    if (p <= kGjRegMax) {
        switch (T16) {
#define HYDE_GJ16(TV) \
    case TV: launch_pdl(noise_gj_reg_kernel<TV, 16>, 1, 256, 0, s, R, p, Ainv, Sd, status); \
        break;
            HYDE_GJ16(1) HYDE_GJ16(2) HYDE_GJ16(3) HYDE_GJ16(4) HYDE_GJ16(5)
            HYDE_GJ16(6) HYDE_GJ16(7) HYDE_GJ16(8) HYDE_GJ16(9) HYDE_GJ16(10)
            HYDE_GJ16(11) HYDE_GJ16(12) HYDE_GJ16(13)
#undef HYDE_GJ16
            default: return HYDE_ERR_SHAPE;
        }
    } else {
        size_t smem = noise_smem_bytes(p);
        if (ensure_smem_limit((const void*)noise_gj_smem_kernel, (int)smem) != cudaSuccess)
            return HYDE_ERR_SHAPE;
        launch_pdl(noise_gj_smem_kernel, 1, kLA, smem, s, R, p, Ainv, Sd, status);
    }
    return HYDE_OK;
}

hyde_status launch_noise_from_gram(const double* R, int p, long long n, double* sigma,
                                   void* ws, int* status, cudaStream_t s) {
    const float* Ainv = reinterpret_cast<const float*>(ws);
    const double* Sd = reinterpret_cast<const double*>(
        reinterpret_cast<const char*>(ws) + align_up((size_t)p * p * sizeof(float), kAlign));
    hyde_status st = launch_gj_inverse(R, p, ws, status, s);
    if (st != HYDE_OK) return st;
    launch_pdl(noise_refine_kernel, p, 256, p * sizeof(double), s, R, Ainv, Sd, p, n, sigma,
               status);
    return cuda_status(cudaGetLastError());
}

hyde_status launch_inverse_from_gram(const double* R, int p, void* ws, double* Q, int* status,
                                     cudaStream_t s) {
    const float* Ainv = reinterpret_cast<const float*>(ws);
    const double* Sd = reinterpret_cast<const double*>(
        reinterpret_cast<const char*>(ws) + align_up((size_t)p * p * sizeof(float), kAlign));
    hyde_status st = launch_gj_inverse(R, p, ws, status, s);
    if (st != HYDE_OK) return st;
    launch_pdl(inverse_refine_kernel, p, 256, 3 * p * sizeof(double), s, R, Ainv, Sd, p, Q,
               status);
    return cuda_status(cudaGetLastError());
}

hyde_status launch_win_noise(const double* R, int p, int n_win, const WinDesc* desc,
                             double* sigma, float* Ainv, double* S, int* status,
                             cudaStream_t s) {
    if (p < 1 || p > kGjRegMax || n_win < 1) return HYDE_ERR_SHAPE;
    switch ((p + 15) / 16) {
#define HYDE_WGJ(TV)                                                                            \
    case TV:                                                                                    \
        launch_pdl(win_noise_kernel<TV, 16>, n_win, 256, 0, s, R, p, desc, sigma, Ainv, S,      \
                   status);                                                                     \
        break;
        HYDE_WGJ(1) HYDE_WGJ(2) HYDE_WGJ(3) HYDE_WGJ(4) HYDE_WGJ(5)
        HYDE_WGJ(6) HYDE_WGJ(7) HYDE_WGJ(8) HYDE_WGJ(9) HYDE_WGJ(10)
        HYDE_WGJ(11) HYDE_WGJ(12) HYDE_WGJ(13)
#undef HYDE_WGJ
        default: return HYDE_ERR_SHAPE;
    }
    return cuda_status(cudaGetLastError());
}

hyde_status launch_weights_batched(const double* V, const double* sigma, int p, int r, int ldw,
                                   float* P, float* Q, int n_win, cudaStream_t s) {
    int tot = p * ldw;
    launch_pdl(weights_kernel, dim3((tot + 255) / 256, n_win), 256, 0, s, V, sigma, p, r, ldw,
               P, Q);
    return cuda_status(cudaGetLastError());
}

hyde_status launch_weights(const double* V, const double* sigma, int p, int r, int ldw,
                           float* P, float* Q, cudaStream_t s) {
    int tot = p * ldw;
    launch_pdl(weights_kernel, (tot + 255) / 256, 256, 0, s, V, sigma, p, r, ldw, P, Q);
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

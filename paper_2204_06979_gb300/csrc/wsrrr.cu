// WSRRR, wavelet-based sparse reduced-rank regression (arXiv 2204.06979
// Sec. 2.1: a low-rank, wavelet-based method for Gaussian noise that also
// extracts features; the paper states nothing more). Reading: on the
// whitened cube Yw (padded, one row per padded pixel) the model
// Yw ~ W2 B V^T, W2 the orthogonal DWT synthesis of r component images, B
// their wavelet coefficients, V^T V = I; the objective
// 1/2 ||Yw - W2 B V^T||^2 + lam |B_detail|_1 is decreased by cyclic descent
// from HyRes's subspace, rank and threshold: B <- soft(W2^T Yw V, lam) (the
// HyRes projection, DWT and thresholded inverse DWT), then V <- polar(M),
// M = Yw^T W2 B (orthogonal Procrustes). This file holds the two kernels
// the HyRes path lacks:
//  * wsrrr_cross_kernel: float partial sums of M over ranges of padded
//    pixels, the cube read through the whole-sample symmetric extension
//    (one thread per band, the component values broadcast from shared
//    memory); wsrrr_cross_reduce_kernel sums them in double and divides
//    row b by sigma_b;
//  * wsrrr_polar_kernel (one block, double): G = M^T M, its Cholesky factor
//    L (M = Q1 L^T), Q1 by triangular solves, the polar factor U of L^T by
//    the scaled Newton iteration X <- (g X + X^-T / g) / 2 (Gauss-Jordan
//    inverses with partial pivoting; stops once an update is below 1e-12 of
//    X, at most 40 iterations), V = Q1 U.
#include <float.h>

#include "hyde_internal.cuh"

namespace hyde {
namespace {

constexpr int kCrossPix = 32;        // padded pixels per chunk (one row segment)
constexpr int kCrossThreads = 256;
constexpr int kPolarThreads = 256;
constexpr int kMaxR = 32;

__device__ __forceinline__ int reflect_idx(int i, int n) {
    // whole-sample symmetric extension past the end: x[n + j] = x[n - 2 - j]
    return i < n ? i : 2 * n - 2 - i;
}

__device__ __forceinline__ void cp4(float* dst, const float* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 4 : 0));
}

// acc[i] += sum_k a[k] B[i][k] for the first RC components (B rows of 32
// pixels, read as float4 broadcasts; rows past the rank hold stale values
// whose sums are discarded).
template <int RC>
__device__ __forceinline__ void cross_acc(const float* __restrict__ a, const float* __restrict__ B,
                                          float (&acc)[kMaxR]) {
#pragma unroll 2
    for (int k = 0; k < kCrossPix; k += 4) {
        const float a0 = a[k], a1 = a[k + 1], a2 = a[k + 2], a3 = a[k + 3];
#pragma unroll
        for (int i = 0; i < RC; ++i) {
            const float4 bv = *reinterpret_cast<const float4*>(B + i * kCrossPix + k);
            acc[i] = fmaf(a0, bv.x, acc[i]);
            acc[i] = fmaf(a1, bv.y, acc[i]);
            acc[i] = fmaf(a2, bv.z, acc[i]);
            acc[i] = fmaf(a3, bv.w, acc[i]);
        }
    }
}

// Block: chunks [c0, c1) of the padded image (a chunk is up to 32 pixels of
// one padded row); stage = band rows [p][33] and component rows [RM][32].
// Thread b < p accumulates M[b][0..RM) over the block's pixels.
__global__ void __launch_bounds__(kCrossThreads)
wsrrr_cross_kernel(const float* __restrict__ Y, int p, int H, int W, const float* __restrict__ X,
                   int RM, int Hp, int Wp, long long nchunks, const int* __restrict__ rank_dev,
                   float* __restrict__ partials) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float csm[];
    // float4-aligned rows of B; rows reserved up to RM rounded to 4, the
    // widest that cross_acc reads
    const int sa = (p * (kCrossPix + 1) + 3) & ~3, sb = ((RM + 3) & ~3) * kCrossPix;
    const int t = threadIdx.x, lane = t & 31, wrp = t >> 5, nw = kCrossThreads / 32;
    const int r = min(*rank_dev, RM);
    const long long cpr = (Wp + kCrossPix - 1) / kCrossPix;
    const long long c0 = (long long)blockIdx.x * nchunks / gridDim.x;
    const long long c1 = (long long)(blockIdx.x + 1) * nchunks / gridDim.x;
    const long long plane = (long long)H * W, pplane = (long long)Hp * Wp;
    auto issue = [&](long long c, int st) {
        float* A = csm + st * (sa + sb);
        float* B = A + sa;
        const int y = (int)(c / cpr), x = (int)(c - (long long)y * cpr) * kCrossPix + lane;
        const bool ok = x < Wp;
        const int ys = reflect_idx(y, H), xs = ok ? reflect_idx(x, W) : 0;
        const float* src = Y + (long long)ys * W + xs;
        for (int b = wrp; b < p; b += nw) cp4(A + b * (kCrossPix + 1) + lane, src + b * plane, ok);
        const float* xsrc = X + (long long)y * Wp + (ok ? x : 0);
        for (int i = wrp; i < r; i += nw) cp4(B + i * kCrossPix + lane, xsrc + i * pplane, ok);
        asm volatile("cp.async.commit_group;\n");
    };
    float acc[kMaxR];
#pragma unroll
    for (int i = 0; i < kMaxR; ++i) acc[i] = 0.f;
    if (c0 < c1) issue(c0, 0);
    for (long long c = c0; c < c1; ++c) {
        const int st = (int)(c - c0) & 1;
        if (c + 1 < c1) {
            issue(c + 1, st ^ 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        const float* A = csm + st * (sa + sb);
        const float* B = A + sa;
        if (t < p) {
            const float* arow = A + t * (kCrossPix + 1);
            switch ((r + 3) >> 2) {
                case 1: cross_acc<4>(arow, B, acc); break;
                case 2: cross_acc<8>(arow, B, acc); break;
                case 3: cross_acc<12>(arow, B, acc); break;
                case 4: cross_acc<16>(arow, B, acc); break;
                case 5: cross_acc<20>(arow, B, acc); break;
                case 6: cross_acc<24>(arow, B, acc); break;
                case 7: cross_acc<28>(arow, B, acc); break;
                default: cross_acc<32>(arow, B, acc); break;
            }
        }
        __syncthreads();   // the stage is refilled by the next iteration's copy
    }
    if (t < p) {
        float* out = partials + ((long long)blockIdx.x * p + t) * RM;
#pragma unroll
        for (int i = 0; i < kMaxR; ++i)
            if (i < RM) out[i] = i < r ? acc[i] : 0.f;
    }
}

// M[b][i] (double [p][ldm]) = sum over blocks of the partials / sigma_b, in
// block order; one thread per (b, i < RM).
__global__ void wsrrr_cross_reduce_kernel(const float* __restrict__ partials, int nblocks, int p,
                                          int RM, const double* __restrict__ sigma, int ldm,
                                          double* __restrict__ M, int* status) {
    pdl_wait();
    pdl_trigger();
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= p * RM) return;
    const int b = idx / RM, i = idx - b * RM;
    double s = 0.0;
    for (int k = 0; k < nblocks; ++k) s += (double)__ldg(partials + (long long)k * p * RM + idx);
    s /= sigma[b];
    if (!isfinite(s)) set_status(status, HYDE_ERR_NUMERIC);
    if (i < ldm) M[(long long)b * ldm + i] = s;
}

// Inverse of the r x r matrix A (shared, row stride kMaxR + 1) into Inv by
// Gauss-Jordan elimination with partial pivoting, in one warp (lane i holds
// row i of the current step). A is overwritten. Returns false if a pivot is
// zero.
__device__ bool gj_inverse_warp(double (*A)[kMaxR + 1], double (*Inv)[kMaxR + 1], int r,
                                int lane) {
    for (int j = 0; j < r; ++j)
        if (lane < r) Inv[lane][j] = lane == j ? 1.0 : 0.0;
    __syncwarp();
    bool ok = true;
    for (int k = 0; k < r; ++k) {
        double best = lane >= k && lane < r ? fabs(A[lane][k]) : -1.0;
        int bi = lane;
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (!(best > 0.0)) ok = false;
        if (bi != k) {   // swap rows k and bi, lanes over columns
            for (int j = lane; j < r; j += 32) {
                const double a = A[k][j], b = A[bi][j];
                A[k][j] = b; A[bi][j] = a;
                const double c = Inv[k][j], d = Inv[bi][j];
                Inv[k][j] = d; Inv[bi][j] = c;
            }
        }
        __syncwarp();
        const double piv = A[k][k];
        const double ip = piv != 0.0 ? 1.0 / piv : 0.0;
        __syncwarp();
        for (int j = lane; j < r; j += 32) { A[k][j] *= ip; Inv[k][j] *= ip; }
        __syncwarp();
        if (lane < r && lane != k) {
            const double f = A[lane][k];
            for (int j = 0; j < r; ++j) {
                A[lane][j] = fma(-f, A[k][j], A[lane][j]);
                Inv[lane][j] = fma(-f, Inv[k][j], Inv[lane][j]);
            }
        }
        __syncwarp();
    }
    return ok;
}

// V (double [p][ldv], columns < r) = polar(M[:, :r]) with r = *rank_dev: see
// the file comment. One block.
__global__ void __launch_bounds__(kPolarThreads)
wsrrr_polar_kernel(const double* __restrict__ M, int p, int ldm, const int* __restrict__ rank_dev,
                   double* __restrict__ V, int ldv, int* status) {
    pdl_wait();
    pdl_trigger();
    __shared__ double Gm[kMaxR][kMaxR + 1];   // M^T M, then its Cholesky factor L (lower)
    __shared__ double X[kMaxR][kMaxR + 1];    // Newton iterate, starting at L^T
    __shared__ double A[kMaxR][kMaxR + 1];    // copy of X for the elimination
    __shared__ double Xi[kMaxR][kMaxR + 1];   // X^-1
    __shared__ double s_red[kPolarThreads / 32];
    __shared__ double s_nx, s_ni;
    __shared__ int s_stop;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int r = min(min(*rank_dev, kMaxR), ldm);
    if (r < 1) return;
    // G = M^T M, lower triangle
    const int npair = r * (r + 1) / 2;
    for (int q = t; q < npair; q += kPolarThreads) {
        int i = 0, rem = q;
        while (rem > i) { rem -= i + 1; ++i; }
        const int j = rem;
        double s = 0.0;
        for (int b = 0; b < p; ++b) s = fma(M[(long long)b * ldm + i], M[(long long)b * ldm + j], s);
        Gm[i][j] = s;
    }
    __syncthreads();
    // right-looking Cholesky in warp 0
    if (wid == 0) {
        const double gdiag = lane < r ? Gm[lane][lane] : 0.0;
        for (int k = 0; k < r; ++k) {
            const double v = Gm[k][k];
            const double floor_ = 1e-26 * __shfl_sync(0xffffffffu, gdiag, k);
            if (lane == 0 && !(v > floor_)) set_status(status, HYDE_ERR_NUMERIC);
            const double lkk = sqrt(v > floor_ ? v : (floor_ > 0.0 ? floor_ : 1e-300));
            const double inv = 1.0 / lkk;
            __syncwarp();
            double l = 0.0;
            if (lane > k && lane < r) {
                l = Gm[lane][k] * inv;
                Gm[lane][k] = l;
            }
            if (lane == k) Gm[k][k] = lkk;
            __syncwarp();
            if (lane > k && lane < r)
                for (int j = k + 1; j <= lane; ++j) Gm[lane][j] = fma(-l, Gm[j][k], Gm[lane][j]);
            __syncwarp();
        }
    }
    __syncthreads();
    for (int e = t; e < r * r; e += kPolarThreads) {
        const int i = e / r, j = e - i * r;
        X[i][j] = j >= i ? Gm[j][i] : 0.0;
    }
    if (t == 0) s_stop = 0;
    __syncthreads();
    // scaled Newton iteration for the polar factor of L^T
    for (int it = 0; it < 40; ++it) {
        for (int e = t; e < r * r; e += kPolarThreads) {
            const int i = e / r, j = e - i * r;
            A[i][j] = X[i][j];
        }
        __syncthreads();
        if (wid == 0 && !gj_inverse_warp(A, Xi, r, lane) && lane == 0)
            set_status(status, HYDE_ERR_NUMERIC);
        __syncthreads();
        // Frobenius norms of X and X^-1
        double sx = 0.0, si = 0.0;
        for (int e = t; e < r * r; e += kPolarThreads) {
            const int i = e / r, j = e - i * r;
            sx = fma(X[i][j], X[i][j], sx);
            si = fma(Xi[i][j], Xi[i][j], si);
        }
        sx = warp_sum_d(sx);
        if (lane == 0) s_red[wid] = sx;
        __syncthreads();
        if (t == 0) {
            double a = 0.0;
            for (int w = 0; w < kPolarThreads / 32; ++w) a += s_red[w];
            s_nx = a;
        }
        __syncthreads();
        si = warp_sum_d(si);
        if (lane == 0) s_red[wid] = si;
        __syncthreads();
        if (t == 0) {
            double a = 0.0;
            for (int w = 0; w < kPolarThreads / 32; ++w) a += s_red[w];
            s_ni = a;
        }
        __syncthreads();
        const double g = sqrt(sqrt(s_ni / s_nx));      // (|X^-1|_F / |X|_F)^(1/2)
        const double ginv = 1.0 / g;
        double dd = 0.0, nn = 0.0;
        for (int e = t; e < r * r; e += kPolarThreads) {
            const int i = e / r, j = e - i * r;
            const double xn = 0.5 * (g * X[i][j] + Xi[j][i] * ginv);
            const double d = xn - X[i][j];
            dd = fma(d, d, dd);
            nn = fma(xn, xn, nn);
            A[i][j] = xn;
        }
        dd = warp_sum_d(dd);
        nn = warp_sum_d(nn);
        __syncthreads();
        if (lane == 0) { s_red[wid] = dd; }
        __syncthreads();
        if (t == 0) {
            double a = 0.0;
            for (int w = 0; w < kPolarThreads / 32; ++w) a += s_red[w];
            s_nx = a;
        }
        __syncthreads();
        if (lane == 0) s_red[wid] = nn;
        __syncthreads();
        if (t == 0) {
            double a = 0.0;
            for (int w = 0; w < kPolarThreads / 32; ++w) a += s_red[w];
            s_stop = s_nx <= 1e-24 * a ? 1 : 0;   // |update| <= 1e-12 |X|: quadratic convergence
        }
        for (int e = t; e < r * r; e += kPolarThreads) {
            const int i = e / r, j = e - i * r;
            X[i][j] = A[i][j];
        }
        __syncthreads();
        if (s_stop) break;
    }
    // V = Q1 U with Q1 = M L^-T (row b: forward substitution with L)
    __shared__ double s_dinv[kMaxR];
    for (int i = t; i < r; i += kPolarThreads) s_dinv[i] = 1.0 / Gm[i][i];
    __syncthreads();
    for (int b = t; b < p; b += kPolarThreads) {
        double q[kMaxR];
        for (int i = 0; i < r; ++i) {
            double v = M[(long long)b * ldm + i];
            for (int j = 0; j < i; ++j) v = fma(-q[j], Gm[i][j], v);
            q[i] = v * s_dinv[i];
        }
        for (int j = 0; j < r; ++j) {
            double v = 0.0;
            for (int i = 0; i < r; ++i) v = fma(q[i], X[i][j], v);
            V[(long long)b * ldv + j] = v;
        }
    }
}

}  // namespace

hyde_status launch_wsrrr_cross(const float* Y, int p, int H, int W, const float* Xr, int RM,
                               int Hp, int Wp, const int* rank_dev, const double* sigma,
                               float* partials, int nblocks, double* M, int ldm, int* status,
                               cudaStream_t s) {
    if (RM > kMaxR || p > 256) return HYDE_ERR_SHAPE;
    const long long nchunks = (long long)Hp * ((Wp + kCrossPix - 1) / kCrossPix);
    const size_t smem = 2 * ((size_t)((p * (kCrossPix + 1) + 3) & ~3) +
                             (size_t)((RM + 3) & ~3) * kCrossPix) * sizeof(float);
    if (ensure_smem_limit((const void*)wsrrr_cross_kernel, (int)smem) != cudaSuccess)
        return HYDE_ERR_CUDA;
    launch_pdl(wsrrr_cross_kernel, nblocks, kCrossThreads, smem, s, Y, p, H, W, Xr, RM, Hp, Wp,
               nchunks, rank_dev, partials);
    launch_pdl(wsrrr_cross_reduce_kernel, (p * RM + 255) / 256, 256, 0, s,
               (const float*)partials, nblocks, p, RM, sigma, ldm, M, status);
    return cuda_status(cudaGetLastError());
}

hyde_status launch_wsrrr_polar(const double* M, int p, int ldm, const int* rank_dev, double* V,
                               int ldv, int* status, cudaStream_t s) {
    if (ldm > kMaxR) return HYDE_ERR_SHAPE;
    launch_pdl(wsrrr_polar_kernel, 1, kPolarThreads, 0, s, M, p, ldm, rank_dev, V, ldv, status);
    return cuda_status(cudaGetLastError());
}

size_t wsrrr_cross_partial_bytes(int p, int RM, int nblocks) {
    return (size_t)nblocks * p * RM * sizeof(float);
}

}  // namespace hyde

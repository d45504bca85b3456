// Small dense linear algebra of the HyRes path (arXiv 2204.06979, Sec. 2.1):
//
//  * noise level by multiple regression: sigma_b^2 = 1 / (n [R^-1]_bb), the
//    residual power of regressing band b on all other bands (the Schur
//    complement of the normal equations);
//  * leading eigenpairs of the whitened Gram matrix D^-1 R D^-1 (the spectral
//    subspace of the low-rank model);
//  * the float projection / back-projection weights V/sigma and V*sigma.
//
// GB300 runs FP64 at 1/64 of its FP32 rate, so the O(p^3) work is done in
// FP32 inside one thread block and FP64 is used where it buys accuracy
// cheaply: the diagonal of the inverse gets one Newton correction in double,
// spread over p blocks.
//
// The p-step recurrences (Gauss-Jordan, Householder) are latency- and
// issue-bound on one SM, so for p <= 192 the matrix lives in registers: the
// 1024 threads form a 32 x 32 grid and thread (w, l) owns the T x T tile of
// rows w*T.. and columns l*T.. (T = ceil(p/32)). A step then costs T^2 FMAs
// per thread plus one to three barriers; the row and column of the current
// step are published through small double-buffered shared vectors. Larger p
// falls back to kernels that keep the matrix in shared memory.
#include <float.h>

#include "hyde_internal.cuh"

#ifndef HYDE_EIG_WARPS
#define HYDE_EIG_WARPS 16
#endif

namespace hyde {
namespace {

constexpr int kLA = 1024;     // threads of the single-block kernels
constexpr int kEigWarps = HYDE_EIG_WARPS;   // warps of the tridiagonalisation

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
// threads, up to 10 x 10 tiles) keeps the per-thread work of a step high and
// the number of warps that repeat the pivot arithmetic low; G = 20 covers
// p <= 200.
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


// Shared-memory Gauss-Jordan for p > 192 (same arithmetic, matrix in smem).
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

// --------------------------------------------------------------------------
// Leading r eigenpairs of a symmetric p x p matrix (one block, 1024 threads),
// optionally whitened on load (A_ij / (wsig_i wsig_j)) and scaled by
// 1 / max |diag|.
// 1. Householder tridiagonalisation in float (A = Q T Q^T); the reflectors
//    v_k (v_k[0] = 1) are kept for step 5.
// 2. Eigenvalues of T by multisection: one warp per wanted eigenvalue, each
//    lane counts eigenvalues below one of 32 points (Sturm sequence).
// 3. Eigenvectors of T from a twisted factorisation at each eigenvalue.
// 4. Classical Gram-Schmidt, twice, over the r vectors (orthogonality inside
//    clusters of close eigenvalues).
// 5. Back-transformation by the reflectors (one warp per vector), sign rule
//    (largest-magnitude entry positive), write-out in double.
// --------------------------------------------------------------------------
struct EigTail {
    float* d; float* e; float* e2; float* tau; float* lam; float* X; float* Dp; float* Dm;
    float* dots;
};

// Barrier among warps 0..NW-1 only (named barrier 1); the other warps of the
// block do not take part and wait at the next __syncthreads.
template <int NW>
__device__ __forceinline__ void bar_sync_warps() {
    if (NW == 32) __syncthreads();
    else asm volatile("bar.sync 1, %0;" ::"n"(NW * 32) : "memory");
}

// Warp sums of NB <= 32 per-lane values at once (reduce-scatter): the
// values are padded to G = 1, 2, 4, ..., 32 slots; each butterfly level with G > 1 slots
// left sends half of them to the partner lane and keeps the other half, so
// sum a is complete after ~G + 4 shuffles instead of 5 NB. Returns the total
// of value `a` (set on return) in every lane; lanes with the same a form
// groups of 32/G consecutive lanes.
__host__ __device__ constexpr int rows_groups(int nb) {
    return nb <= 1 ? 1 : nb <= 2 ? 2 : nb <= 4 ? 4 : nb <= 8 ? 8 : nb <= 16 ? 16 : 32;
}

template <int NB>
__device__ __forceinline__ float rows_reduce_scatter(const float (&s)[NB], int lane, int& a) {
    constexpr int G = rows_groups(NB);
    float x[G];
#pragma unroll
    for (int q = 0; q < G; ++q) x[q] = q < NB ? s[q] : 0.f;
    int idx = 0, off = 16;
#pragma unroll
    for (int half = G / 2; half >= 1; half >>= 1) {
        const bool hi = (lane & off) != 0;
#pragma unroll
        for (int q = 0; q < half; ++q) {
            const float send = hi ? x[q] : x[q + half];
            const float keep = hi ? x[q + half] : x[q];
            x[q] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
        if (hi) idx += half;
        off >>= 1;
    }
    float v = x[0];
    for (; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    a = idx;
    return v;
}

__device__ __forceinline__ int sturm_count(const float* d, const float* e2, int p,
                                           float x, float pivmin) {
    float q = d[0] - x;
    int c = q < 0.f;
    for (int i = 1; i < p; ++i) {
        if (fabsf(q) < pivmin) q = -pivmin;
        q = (d[i] - x) - __fdividef(e2[i - 1], q);
        c += q < 0.f;
    }
    return c;
}

// Stages 2-5 on the tridiagonal (d, e) in shared memory; all 1024 threads.
template <int NBV>
__device__ __forceinline__ void eig_tail_stages234(const EigTail& S, int p, int r, int* status) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int i = t; i < p; i += blockDim.x) {
        S.e2[i] = S.e[i] * S.e[i];
        if (!isfinite(S.d[i]) || !isfinite(S.e[i])) set_status(status, HYDE_ERR_NUMERIC);
    }
    __syncthreads();

    __shared__ float s_lo, s_hi, s_pivmin;
    if (wid == 0) {
        float lo = FLT_MAX, hi = -FLT_MAX, emax = 0.f;
        for (int i = lane; i < p; i += 32) {
            float rad = fabsf(S.e[i]) + (i > 0 ? fabsf(S.e[i - 1]) : 0.f);
            lo = fminf(lo, S.d[i] - rad);
            hi = fmaxf(hi, S.d[i] + rad);
            emax = fmaxf(emax, S.e2[i]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        }
        if (lane == 0) {
            float w = hi - lo;
            s_lo = lo - 1e-6f * fmaxf(w, 1e-30f);
            s_hi = hi + 1e-6f * fmaxf(w, 1e-30f);
            s_pivmin = FLT_MIN * fmaxf(1.f, emax);
        }
    }
    __syncthreads();

    // 2. multisection, warp j finds the (j+1)-th largest eigenvalue
    if (wid < r) {
        const int target = p - 1 - wid;       // ascending index
        float lo = s_lo, hi = s_hi;
        for (int it = 0; it < 16; ++it) {
            const float x = lo + (hi - lo) * (float)(lane + 1) / 33.0f;
            const int c = sturm_count(S.d, S.e2, p, x, s_pivmin);
            const unsigned below = __ballot_sync(0xffffffffu, c <= target);
            const int nle = __popc(below);
            const float xl = __shfl_sync(0xffffffffu, x, nle > 0 ? nle - 1 : 0);
            const float xh = __shfl_sync(0xffffffffu, x, nle < 32 ? nle : 31);
            const float nlo = nle > 0 ? xl : lo;
            const float nhi = nle < 32 ? xh : hi;
            if (!(nlo < nhi) || (nhi - nlo) >= (hi - lo)) break;
            lo = nlo; hi = nhi;
            if (hi - lo <= 2.f * FLT_EPSILON * fmaxf(fabsf(lo), fabsf(hi))) break;
        }
        if (lane == 0) S.lam[wid] = 0.5f * (lo + hi);
    }
    __syncthreads();

    // 3. twisted factorisation eigenvector of T for each eigenvalue
    if (wid < r) {
        const float lam = S.lam[wid];
        float* Dp = S.Dp + wid * p;
        float* Dm = S.Dm + wid * p;
        float* z = S.X + wid * p;
        const float pm = s_pivmin;
        // the two factorisations run in lockstep in lanes 0 (L D L^T from the
        // top) and 1 (U D U^T from the bottom): one instruction stream, no
        // divergent branches
        if (lane < 2) {
            const bool fwd = lane == 0;
            float* D = fwd ? Dp : Dm;
            int i = fwd ? 0 : p - 1;
            const int step = fwd ? 1 : -1;
            float q = S.d[i] - lam;
            if (fabsf(q) < pm) q = -pm;
            D[i] = q;
            for (int s2 = 1; s2 < p; ++s2) {
                i += step;
                const float e2 = S.e2[fwd ? i - 1 : i];
                q = (S.d[i] - lam) - __fdividef(e2, q);
                if (fabsf(q) < pm) q = -pm;
                D[i] = q;
            }
        }
        __syncwarp();
        // twist index: minimum |gamma_i|, gamma_i = Dp_i + Dm_i - (d_i - lam)
        float best = FLT_MAX;
        int bi = 0;
        for (int i = lane; i < p; i += 32) {
            float g = fabsf(Dp[i] + Dm[i] - (S.d[i] - lam));
            if (g < best) { best = g; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            float ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob < best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        const int kt = bi;
        // z from the twist outwards, lane 0 upwards (rows kt-1..0, from L D L^T)
        // and lane 1 downwards (rows kt+1..p-1, from U D U^T), in lockstep
        if (lane < 2) {
            const bool up = lane == 0;
            const int len = up ? kt : p - 1 - kt;
            const int steps = max(kt, p - 1 - kt);
            if (up) z[kt] = 1.0f;
            int i = kt;
            float zz = 1.0f;
            for (int s2 = 0; s2 < steps; ++s2) {
                if (s2 < len) {
                    i += up ? -1 : 1;
                    const float num = S.e[up ? i : i - 1];
                    const float den = up ? Dp[i] : Dm[i];
                    zz = -__fdividef(num, den) * zz;
                    z[i] = zz;
                }
            }
        }
        __syncwarp();
        float ss = 0.f;
        for (int i = lane; i < p; i += 32) ss = fmaf(z[i], z[i], ss);
        ss = warp_sum(ss);
        const float inv = ss > 0.f ? rsqrtf(ss) : 0.f;
        for (int i = lane; i < p; i += 32) z[i] *= inv;
    }
    __syncthreads();

    // 4. classical Gram-Schmidt, two passes, in descending order
    for (int j = 1; j < r; ++j) {
        float* zj = S.X + j * p;
        for (int pass = 0; pass < 2; ++pass) {
            if (wid < j) {
                const float* zi = S.X + wid * p;
                float dt = 0.f;
                for (int i = lane; i < p; i += 32) dt = fmaf(zi[i], zj[i], dt);
                dt = warp_sum(dt);
                if (lane == 0) S.dots[wid] = dt;
            }
            __syncthreads();
            for (int i = t; i < p; i += blockDim.x) {
                float acc = zj[i];
                for (int q = 0; q < j; ++q) acc = fmaf(-S.dots[q], S.X[q * p + i], acc);
                zj[i] = acc;
            }
            __syncthreads();
        }
        if (wid == 0) {
            float ss = 0.f;
            for (int i = lane; i < p; i += 32) ss = fmaf(zj[i], zj[i], ss);
            ss = warp_sum(ss);
            const float inv = ss > 0.f ? rsqrtf(ss) : 0.f;
            for (int i = lane; i < p; i += 32) zj[i] *= inv;
        }
        __syncthreads();
    }
}

// Scalars of Householder reflector kr from column kr of A (row-major, leading
// dimension lda): alpha = A[kr+1][kr], ss = sum of squares below it. The
// reflector is v = e_{kr+1} + sc * (A[kr+2..][kr]), H = I - tau v v^T, and it
// maps the column onto beta e_{kr+1}. ss == 0 gives the identity (tau = 0).
__device__ __forceinline__ void hh_scalars(const float* A, int lda, int kr, float ss,
                                           float& tau, float& sc, float& beta) {
    const float alpha = A[(kr + 1) * lda + kr];
    tau = 0.f; beta = alpha; sc = 0.f;
    if (ss > 0.f) {
        const float nrm = sqrtf(fmaf(alpha, alpha, ss));
        beta = alpha >= 0.f ? -nrm : nrm;
        tau = __fdividef(beta - alpha, beta);
        sc = __fdividef(1.0f, alpha - beta);
    }
}

// The same scalars from alpha and ss given directly.
__device__ __forceinline__ void hh_scalars_of(float alpha, float ss, float& tau, float& sc,
                                              float& beta) {
    tau = 0.f; beta = alpha; sc = 0.f;
    if (ss > 0.f) {
        const float nrm = sqrtf(fmaf(alpha, alpha, ss));
        beta = alpha >= 0.f ? -nrm : nrm;
        tau = __fdividef(beta - alpha, beta);
        sc = __fdividef(1.0f, alpha - beta);
    }
}

// Entry i of reflector kr (see hh_scalars).
__device__ __forceinline__ float hh_coef(const float* A, int lda, int p, int kr, float sc, int i) {
    return i == kr + 1 ? 1.0f : ((i > kr + 1 && i < p) ? A[i * lda + kr] * sc : 0.f);
}

// --------------------------------------------------------------------------
// Eigensolver with the matrix in shared memory and the per-step vectors in
// registers (one block, 1024 threads; NB = ceil(p/32) column chunks per
// lane). Warp w owns rows i = w (mod 32) of the trailing matrix, lane l owns
// columns j = l + 32b, and caches v_j and w_j of those columns in registers,
// so a matrix element costs one load and one FMA in the matvec and one
// load, two FMAs and one store in the rank-2 update; K = tau/2 v^T p is one
// warp shuffle-sum per warp. The back-transformation keeps each eigenvector
// in registers (lane l holds entries l + 32b).
// --------------------------------------------------------------------------
template <int NB, int NW>
__global__ void __launch_bounds__(kLA, 1)
eig_fast_kernel(const double* __restrict__ Ain, const double* __restrict__ wsig, int p, int r,
                double* __restrict__ evals, double* __restrict__ V, int* status) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float sm[];
    const int lda = p + 1;
    float* q = sm;
    float* A = q;    q += p * lda;
    float* tauv = q; q += p;
    float* dv = q;   q += p;
    float* ev = q;   q += p;
    float* e2v = q;  q += p;
    float* vf = q;   q += p;     // reflector buffer 0, full length
    float* pvv = q;  q += 2 * p; // p = tau A v, then reflector buffer 1
    float* red = q;  q += 64;
    float* lamv = q; q += 32;
    float* dots = q; q += 32;
    float* X = q;    q += p * r;
    float* Dp = q;   q += p * r;
    float* Dm = q;   q += p * r;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;

    // Whitening weights 1/sigma and the largest whitened diagonal entry in
    // float over all threads, the matrix converted on the integer pipes: no
    // FP64 arithmetic on this one SM.
    __shared__ float s_scale;
    __shared__ int s_mx;
    float* iw = vf;
    if (t == 0) s_mx = 0;
    __syncthreads();
    for (int i = t; i < p; i += blockDim.x) {
        const float w = wsig ? 1.0f / d2f_bits(wsig[i]) : 1.0f;
        iw[i] = w;
        const float a = d2f_bits(Ain[(long long)i * p + i]) * w * w;
        if (!isfinite(a)) set_status(status, HYDE_ERR_NUMERIC);
        atomicMax(&s_mx, __float_as_int(fabsf(a)));   // non-negative floats order as ints
    }
    __syncthreads();
    if (t == 0) {
        const float mx = __int_as_float(s_mx);
        s_scale = mx > 0.f && isfinite(mx) ? 1.0f / mx : 1.0f;
    }
    __syncthreads();
    const float scale = s_scale;
    for (int i = wid; i < p; i += 32) {
        const float si = iw[i] * scale;
        for (int j = lane; j < p; j += 32)
            A[i * lda + j] = d2f_bits(Ain[(long long)i * p + j]) * si * iw[j];
    }
    __syncthreads();

    // Fused steps. Reflector k is kept as (column k of A, scale sc_k):
    // v_k[i] = 1 at i = k+1, A[i][k] sc_k beyond. Per step: K = tau/2 v^T p
    // in every warp from p in shared memory; the owner lanes update column
    // k+1 and sum the squares of its entries below k+2; after one barrier
    // every warp forms reflector k+1's scalars itself; then one sweep over
    // the trailing matrix applies update k and accumulates p' = A' v_{k+1} of
    // step k+1 from the new values (row sums by a reduce-scatter). Two
    // barriers per step, one read and one write of each trailing element.
    float* const scv = vf;           // reflector scales (vf is free after the load)
    float* const cvec = e2v;         // updated column k+1 (e2v is filled by the tail)
    constexpr int NA = (32 * NB + NW - 1) / NW;   // trailing rows per warp
    if (wid < NW) {
    // prologue: reflector 0 (scalars in every warp) and p_0 = tau_0 A v_0
    float tau_k = 0.f, sc_k = 0.f;
    float vreg[NB];
    if (p >= 3) {
        float ss = 0.f;
        for (int i = 2 + lane; i < p; i += 32) { const float x = A[i * lda]; ss = fmaf(x, x, ss); }
        ss = warp_sum(ss);
        float beta;
        hh_scalars(A, lda, 0, ss, tau_k, sc_k, beta);
        if (t == 0) { tauv[0] = tau_k; scv[0] = sc_k; dv[0] = A[0]; ev[0] = beta; }
#pragma unroll
        for (int b = 0; b < NB; ++b) vreg[b] = hh_coef(A, lda, p, 0, sc_k, lane + 32 * b);
        const int i0 = 1 + ((wid - 1) & (NW - 1));
        float sacc[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const int i = i0 + NW * a;
            sacc[a] = 0.f;
            if (i < p) {
                const float* row = A + i * lda;
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const int j = lane + 32 * b;
                    if (j < p) sacc[a] = fmaf(row[j], vreg[b], sacc[a]);
                }
            }
        }
        int a_own;
        const float tot = rows_reduce_scatter<NA>(sacc, lane, a_own);
        const int i = i0 + NW * a_own;
        if (a_own < NA && (lane & (32 / rows_groups(NA) - 1)) == 0 && i < p) pvv[i] = tot * tau_k;
    }
    bar_sync_warps<NW>();
    for (int k = 0; k + 2 < p; ++k) {
        const float* pc = pvv + (k & 1) * p;
        float* pn = pvv + ((k + 1) & 1) * p;
        const bool has_next = k + 4 <= p;
        // K = tau/2 v^T p and w = p - K v (v_k, p_k nonzero on rows > k)
        float pj[NB];
        float kp = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = lane + 32 * b;
            pj[b] = (j > k && j < p) ? pc[j] : 0.f;
            kp = fmaf(vreg[b], pj[b], kp);
        }
        const float K = 0.5f * tau_k * warp_sum(kp);
        float wreg[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) wreg[b] = fmaf(-K, vreg[b], pj[b]);
        const int i0 = k + 1 + ((wid - (k + 1)) & (NW - 1));
        // column k+1 by warp 0 alone (lane l: rows k+1+l+32b), written to
        // cvec (A keeps the old values: the sweep updates the column in
        // place), and the sum of squares below row k+2 for reflector k+1
        const int jn = k + 1;
        if (wid == 0) {
            const float wjn = pc[jn] - K;          // v_k[jn] = 1
            float ssp = 0.f;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int i = jn + lane + 32 * b;
                if (i < p) {
                    const float vi = hh_coef(A, lda, p, k, sc_k, i);
                    const float x = fmaf(-vi, wjn, A[i * lda + jn] - fmaf(-K, vi, pc[i]));
                    cvec[i] = x;
                    if (i >= k + 3) ssp = fmaf(x, x, ssp);
                }
            }
            ssp = warp_sum(ssp);
            if (lane == 0) red[32] = ssp;
        }
        bar_sync_warps<NW>();
        float tau_n = 0.f, sc_n = 0.f;
        float vn[NB];
        if (has_next) {
            float beta;
            hh_scalars_of(cvec[k + 2], red[32], tau_n, sc_n, beta);
            if (t == 0) {
                tauv[k + 1] = tau_n; scv[k + 1] = sc_n;
                dv[k + 1] = cvec[k + 1]; ev[k + 1] = beta;
            }
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int j = lane + 32 * b;
                vn[b] = j == k + 2 ? 1.0f : ((j > k + 2 && j < p) ? cvec[j] * sc_n : 0.f);
            }
        } else {
#pragma unroll
            for (int b = 0; b < NB; ++b) vn[b] = 0.f;
        }
        // fused sweep: update k on rows > k+1, columns > k+1; accumulate p' rows
        // Columns j <= k have v = w = 0 and are rewritten unchanged; column
        // k+1 gets the same value warp 0 put in cvec; only the last column
        // block can reach past p (p > 32 (NB - 1)).
        float sacc[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const int i = i0 + NW * a;
            sacc[a] = 0.f;
            if (i > k + 1 && i < p) {
                float* row = A + i * lda;
                const float vi = row[k] * sc_k, wi = fmaf(-K, vi, pc[i]);
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const int j = lane + 32 * b;
                    if (b < NB - 1 || j < p) {
                        const float x = fmaf(-vi, wreg[b], fmaf(-wi, vreg[b], row[j]));
                        row[j] = x;
                        sacc[a] = fmaf(x, vn[b], sacc[a]);
                    }
                }
            }
        }
        if (has_next) {
            int a_own;
            const float tot = rows_reduce_scatter<NA>(sacc, lane, a_own);
            const int i = i0 + NW * a_own;
            if (a_own < NA && (lane & (32 / rows_groups(NA) - 1)) == 0 && i > k + 1 && i < p)
                pn[i] = tot * tau_n;
        }
        tau_k = tau_n;
        sc_k = sc_n;
#pragma unroll
        for (int b = 0; b < NB; ++b) vreg[b] = vn[b];
        bar_sync_warps<NW>();
    }
    }   // wid < NW
    __syncthreads();
    // reflector k as an explicit vector in column k: 0 above row k+1, 1 at
    // k+1, x * scale below (the back-transformation then reads it directly)
    for (int i = wid; i < p; i += 32) {
        for (int k = lane; k < p - 2; k += 32) {
            float* a = A + i * lda + k;
            *a = i <= k ? 0.f : (i == k + 1 ? 1.0f : *a * scv[k]);
        }
    }
    __syncthreads();
    // cpair[k] = v_{k-1} . v_k (k >= 1) for the paired back-transformation;
    // the reflector scales are no longer needed, so their array holds it
    float* const cpair = vf;
    for (int k = 1 + wid; k <= p - 3; k += 32) {
        float s2 = 0.f;
        for (int i = k + lane; i < p; i += 32) s2 = fmaf(A[i * lda + k - 1], A[i * lda + k], s2);
        s2 = warp_sum(s2);
        if (lane == 0) cpair[k] = s2;
    }
    if (t == 0) {
        // with p >= 3 the last step left column p-2 in cvec (row p-2 of A is
        // not updated by the sweep); A[p-1][p-1] is current
        if (p >= 3) {
            dv[p - 2] = cvec[p - 2];
            ev[p - 2] = cvec[p - 1];
            tauv[p - 2] = 0.f;
        } else if (p == 2) {
            dv[0] = A[0];
            ev[0] = A[lda];
            tauv[0] = 0.f;
        }
        dv[p - 1] = A[(p - 1) * lda + (p - 1)];
        ev[p - 1] = 0.f;
    }
    __syncthreads();
    EigTail tail{dv, ev, e2v, tauv, lamv, X, Dp, Dm, dots};
    eig_tail_stages234<NB>(tail, p, r, status);
    // 5. back-transformation with the vector in registers, one warp per vector
    if (wid < r) {
        float x[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int i = lane + 32 * b;
            x[b] = i < p ? X[wid * p + i] : 0.f;
        }
        // Reflectors k (column k of A, explicit) in pairs (k, k-1): both dot
        // products come from one pass and two interleaved warp sums;
        // H_{k-1} H_k x = x - d_a v_k - d_b v_{k-1} with d_a = tau_k v_k.x and
        // d_b = tau_{k-1} (v_{k-1}.x - d_a v_{k-1}.v_k) (cpair[k]). The next
        // pair's columns are loaded while this pair's sums run.
        auto load_col = [&](int k, float (&c)[NB]) {
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int i = lane + 32 * b;
                c[b] = (b < NB - 1 || i < p) ? A[i * lda + k] : 0.f;
            }
        };
        float ca[NB], cb[NB];
        int k = p - 3;
        if (k >= 1) { load_col(k, ca); load_col(k - 1, cb); }
        for (; k >= 1; k -= 2) {
            float va[NB], vb[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) { va[b] = ca[b]; vb[b] = cb[b]; }
            const float ta = tauv[k], tb = tauv[k - 1], cab = cpair[k];
            if (k >= 3) { load_col(k - 2, ca); load_col(k - 3, cb); }
            float sa = 0.f, sb = 0.f;
#pragma unroll
            for (int b = 0; b < NB; ++b) { sa = fmaf(va[b], x[b], sa); sb = fmaf(vb[b], x[b], sb); }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sa += __shfl_xor_sync(0xffffffffu, sa, o);
                sb += __shfl_xor_sync(0xffffffffu, sb, o);
            }
            const float da = ta * sa;
            const float db = tb * fmaf(-da, cab, sb);
#pragma unroll
            for (int b = 0; b < NB; ++b) x[b] = fmaf(-db, vb[b], fmaf(-da, va[b], x[b]));
        }
        if (k == 0) {   // an odd count leaves reflector 0
            float v0[NB];
            load_col(0, v0);
            float s0 = 0.f;
#pragma unroll
            for (int b = 0; b < NB; ++b) s0 = fmaf(v0[b], x[b], s0);
            const float d0 = tauv[0] * warp_sum(s0);
#pragma unroll
            for (int b = 0; b < NB; ++b) x[b] = fmaf(-d0, v0[b], x[b]);
        }
        float best = -1.f;
        int bi = 0;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int i = lane + 32 * b;
            if (i < p && fabsf(x[b]) > best) { best = fabsf(x[b]); bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            float ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        const int owner = bi & 31;
        float xb = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (b == (bi >> 5)) xb = x[b];
        xb = __shfl_sync(0xffffffffu, xb, owner);
        const float sg = xb < 0.f ? -1.f : 1.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int i = lane + 32 * b;
            if (i < p) V[(long long)i * r + wid] = (double)(sg * x[b]);
        }
        if (lane == 0) evals[wid] = (double)(lamv[wid] / scale);
    }
}

__global__ void weights_kernel(const double* __restrict__ V, const double* __restrict__ sigma,
                               int p, int r, int ldw, float* __restrict__ P,
                               float* __restrict__ Q) {
    pdl_wait();
    pdl_trigger();
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p * ldw;
         e += gridDim.x * blockDim.x) {
        int b = e / ldw, i = e % ldw;
        double v = i < r ? V[(long long)b * r + i] : 0.0;
        P[e] = (float)(v / sigma[b]);
        Q[e] = (float)(v * sigma[b]);
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

size_t eig_fast_bytes(int p, int r) {
    return ((size_t)p * (p + 1) + 7 * (size_t)p + 64 + 32 + 32 + 3 * (size_t)p * r) *
           sizeof(float);
}

}  // namespace

size_t noise_ws_bytes(int p) {
    return align_up((size_t)p * p * sizeof(float), kAlign) +
           align_up((size_t)p * sizeof(double), kAlign);
}

// A 20 x 20 thread grid with 10 x 10 register tiles (400 threads) covers
// p <= 200; larger p use the shared-memory kernel.
constexpr int kGj20Max = 200;

size_t noise_smem_bytes(int p) {
    return p <= kGj20Max ? 0 : ((size_t)p * p + 2 * p) * sizeof(float);
}

// The float inverse of the scaled Gram matrix into ws (Ainv, then the
// scales S): a register-tile Gauss-Jordan kernel for p <= 200, the
// shared-memory kernel above.
static hyde_status launch_gj_inverse(const double* R, int p, void* ws, int* status,
                                     cudaStream_t s) {
    float* Ainv = reinterpret_cast<float*>(ws);
    double* Sd = reinterpret_cast<double*>(reinterpret_cast<char*>(ws) +
                                           align_up((size_t)p * p * sizeof(float), kAlign));
    const int T16 = (p + 15) / 16;
    if (T16 <= 10) {
        switch (T16) {
#define HYDE_GJ16(TV) \
    case TV: launch_pdl(noise_gj_reg_kernel<TV, 16>, 1, 256, 0, s, R, p, Ainv, Sd, status); \
        break;
            HYDE_GJ16(1) HYDE_GJ16(2) HYDE_GJ16(3) HYDE_GJ16(4) HYDE_GJ16(5)
            HYDE_GJ16(6) HYDE_GJ16(7) HYDE_GJ16(8) HYDE_GJ16(9) HYDE_GJ16(10)
#undef HYDE_GJ16
            default: return HYDE_ERR_SHAPE;
        }
    } else if (p <= kGj20Max) {
        // 400 threads take registers in whole 4-warp groups (512 threads' worth), so the
        // 10 x 10 tile gets 128 registers and spills a little: still far ahead of the
        // shared-memory kernel
        launch_pdl(noise_gj_reg_kernel<10, 20>, 1, 400, 0, s, R, p, Ainv, Sd, status);
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

size_t eig_smem_bytes(int p, int r) { return eig_fast_bytes(p, r); }

hyde_status launch_eig_top(const double* A, const double* wsig, int p, int r, double* evals,
                           double* V, int* status, cudaStream_t s) {
    if (r > 32 || r < 1 || r > p || p > 256) return HYDE_ERR_SHAPE;
    const size_t smem = eig_fast_bytes(p, r);
    if (smem > 227 * 1024) return HYDE_ERR_SHAPE;
    const int NB = (p + 31) / 32;
    switch (NB) {
#define HYDE_EIG(NBV)                                                                          \
    case NBV:                                                                                  \
        if (ensure_smem_limit((const void*)eig_fast_kernel<NBV, kEigWarps>, (int)smem) !=      \
            cudaSuccess)    \
            return HYDE_ERR_SHAPE;                                                             \
        launch_pdl(eig_fast_kernel<NBV, kEigWarps>, 1, kLA, smem, s, A, wsig, p, r, evals, V, \
                   status);                                                                   \
        break;
        HYDE_EIG(1) HYDE_EIG(2) HYDE_EIG(3) HYDE_EIG(4)
        HYDE_EIG(5) HYDE_EIG(6) HYDE_EIG(7) HYDE_EIG(8)
#undef HYDE_EIG
        default: return HYDE_ERR_SHAPE;
    }
    return cuda_status(cudaGetLastError());
}

hyde_status launch_weights(const double* V, const double* sigma, int p, int r, int ldw,
                           float* P, float* Q, cudaStream_t s) {
    int tot = p * ldw;
    launch_pdl(weights_kernel, (tot + 255) / 256, 256, 0, s, V, sigma, p, r, ldw, P, Q);
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

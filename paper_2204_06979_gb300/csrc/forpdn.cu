// FORPDN, first-order spectral roughness penalty denoising (arXiv 2204.06979
// Sec. 2.1: a full-rank, wavelet-based method for additive Gaussian noise;
// the paper states nothing more). The reading built here: every band image
// is padded and transformed by the L-level periodic db2 DWT; the coefficient
// positions form L + 1 groups (the detail positions of each level and the
// final LL band); per group, every position's spectrum c (its p band
// coefficients) is replaced by (I + lam D^T D)^-1 c, D the first difference
// along the bands, with lam the first minimiser over a grid of Stein's
// unbiased risk estimate under independent band noise of variance sigma_b^2
// (the regression noise estimate of the HyRes stage); the inverse DWT gives
// the estimate.
//
// D^T D is diagonalised by the orthonormal DCT-II basis U (eigenvalues
// mu_k = 4 sin^2(pi k / 2p)), so with E_k = u_k^T G u_k (G the group's
// Gram matrix of spectra) and A_k = sum_b sigma_b^2 U_bk^2
//   SURE(lam) = sum_k [(lam mu_k / (1 + lam mu_k))^2 E_k + 2 N A_k / (1 + lam mu_k)]
//               - N sum_b sigma_b^2.
// Kernels:
//  * forpdn_gram_kernel: float partial Gram matrices of the groups' spectra
//    (8 x 8 tiles per thread over 32-position chunks of the groups' rows, a
//    cp.async pipeline into swizzled shared rows, as in the Gram of the
//    cube); forpdn_gram_reduce_kernel sums them in double in a fixed order;
//  * forpdn_energy_kernel: E_k per group and A_k, one block per (group, k),
//    in double;
//  * forpdn_select_kernel: the SURE table, its first minimum and the
//    tridiagonal factors of I + lam D^T D per group;
//  * forpdn_smooth_kernel: the tridiagonal solve for every position, in
//    place (Thomas algorithm: I + lam D^T D is symmetric and diagonally
//    dominant), forward values in shared memory.
// The noise estimate, the DWT and the inverse DWT are the HyRes kernels.
#include <float.h>

#include "hyde_internal.cuh"

namespace hyde {

// Groups of Mallat positions: 0 = the final LL band (rows < Hp >> L, columns
// < Wp >> L), l = 1..L the detail positions of level l, two rectangles each
// (rows < h_l, columns in [w_l, 2 w_l); rows in [h_l, 2 h_l), columns <
// 2 w_l; h_l = Hp >> l, w_l = Wp >> l).
struct FpRect {
    int y0, x0, h, w;
};
struct FpGeom {
    int ngroups;               // L + 1
    int nrect[kMaxLevels + 1];
    FpRect rect[kMaxLevels + 1][2];
    long long chunks[kMaxLevels + 1];        // 32-position chunks of each group
    int block0[kMaxLevels + 2];              // first block of each group (prefix)
};

namespace {

constexpr int FKC = 32;         // positions per chunk
constexpr int FSTAGES = 3;
constexpr int kFpMaxThreads = 544;
constexpr int kSmoothThreads = 64;
constexpr int kEnergyThreads = 128;

__host__ __device__ inline FpRect make_rect(int y0, int x0, int h, int w) {
    FpRect r;
    r.y0 = y0; r.x0 = x0; r.h = h; r.w = w;
    return r;
}

__device__ __forceinline__ void fp_tile_of(int t, int PT, int& ti, int& tj) {
    int row = 0, rem = t, len = PT;
    while (rem >= len) { rem -= len; ++row; --len; }
    ti = row;
    tj = row + rem;
}

__device__ __forceinline__ void fp_cp_async4(float* dst, const float* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n));
}

// Chunk c of group g -> (row y, first column x, columns left in the row).
__device__ __forceinline__ void fp_chunk(const FpGeom& G, int g, long long c, int& y, int& x,
                                         int& left) {
    const FpRect& r0 = G.rect[g][0];
    const long long cpr0 = (r0.w + FKC - 1) / FKC;
    const long long n0 = cpr0 * r0.h;
    const FpRect& r = c < n0 ? r0 : G.rect[g][1];
    const long long cc = c < n0 ? c : c - n0;
    const long long cpr = (r.w + FKC - 1) / FKC;
    const int row = (int)(cc / cpr), col = (int)(cc - (long long)row * cpr) * FKC;
    y = r.y0 + row;
    x = r.x0 + col;
    left = r.w - col;
}

// Partial Gram matrices of the groups' spectra. Block -> group by the prefix
// table; each block of a group takes an even share of its chunks. Tiles and
// shared layout as in the Gram of the cube: band b is one 128-byte row of 8
// float4 (32 positions), float4 column q stored at q ^ ((b >> 3) & 7).
template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
forpdn_gram_kernel(const float* __restrict__ C, int p, int Wp, long long plane, FpGeom G, int PT,
                   int ntiles, float* __restrict__ partials) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float4 fsm4[];
    const int p8 = PT * 8;
    const int t = threadIdx.x, T = blockDim.x;
    int g = 0;
    while (g + 1 < G.ngroups && (int)blockIdx.x >= G.block0[g + 1]) ++g;
    const int nb = G.block0[g + 1] - G.block0[g], bi = (int)blockIdx.x - G.block0[g];
    for (int i = t; i < (p8 - p) * 8 * FSTAGES; i += T) {
        const int st = i / ((p8 - p) * 8), o = i % ((p8 - p) * 8);
        fsm4[st * p8 * 8 + p * 8 + o] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const long long nch = G.chunks[g];
    const long long c0 = (long long)bi * nch / nb, c1 = (long long)(bi + 1) * nch / nb;
    const int lane = t & 31, wrp = t >> 5, nw = T >> 5;
    const int kq = lane >> 2, kr = lane & 3;
    auto issue = [&](long long c, int st) {
        float* d = reinterpret_cast<float*>(fsm4 + st * p8 * 8);
        int y, x, left;
        fp_chunk(G, g, c, y, x, left);
        const bool ok = lane < left;
        const float* src = C + (long long)y * Wp + x + (ok ? lane : 0) + (long long)wrp * plane;
        for (int b = wrp; b < p; b += nw, src += (long long)nw * plane)
            fp_cp_async4(d + b * 32 + ((kq ^ ((b >> 3) & 7)) << 2) + kr, src, ok);
    };
    const bool active = t < ntiles;
    int ti = 0, tj = 0;
    if (active) fp_tile_of(t, PT, ti, tj);
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll
    for (int s = 0; s < FSTAGES - 1; ++s) {
        if (c0 + s < c1) issue(c0 + s, s);
        asm volatile("cp.async.commit_group;\n");
    }
    for (long long c = c0; c < c1; ++c) {
        asm volatile("cp.async.wait_group %0;\n" ::"n"(FSTAGES - 2));
        __syncthreads();
        const long long nxt = c + FSTAGES - 1;
        if (nxt < c1) issue(nxt, (int)(nxt - c0) % FSTAGES);
        asm volatile("cp.async.commit_group;\n");
        if (active) {
            const float4* B = fsm4 + ((int)(c - c0) % FSTAGES) * p8 * 8;
            const float4* Ba = B + 64 * ti;
            const float4* Bb = B + 64 * tj;
            const int xa = ti & 7, xb = tj & 7;
#pragma unroll 1
            for (int q = 0; q < 8; ++q) {
                const int qa = q ^ xa, qb = q ^ xb;
                float4 a[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = Ba[8 * i + qa];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 bv = Bb[8 * j + qb];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        acc[i][j] = fmaf(a[i].x, bv.x, acc[i][j]);
                        acc[i][j] = fmaf(a[i].y, bv.y, acc[i][j]);
                        acc[i][j] = fmaf(a[i].z, bv.z, acc[i][j]);
                        acc[i][j] = fmaf(a[i].w, bv.w, acc[i][j]);
                    }
                }
            }
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (active) {
        float4* out = reinterpret_cast<float4*>(partials + ((long long)blockIdx.x * ntiles + t) * 64);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            out[2 * i] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            out[2 * i + 1] = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
        }
    }
}

// Gg[g][i][j] (double, both triangles) = the sum of group g's block partials
// in block order: one thread per (group, tile element).
__global__ void forpdn_gram_reduce_kernel(const float* __restrict__ partials, FpGeom G, int p,
                                          int PT, int ntiles, double* __restrict__ Gg,
                                          int* status) {
    pdl_wait();
    pdl_trigger();
    const int g = blockIdx.y;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)ntiles * 64) return;
    const long long stride = (long long)ntiles * 64;
    double s = 0.0;
    for (int b = G.block0[g]; b < G.block0[g + 1]; ++b) s += (double)__ldg(partials + b * stride + idx);
    const int t = (int)(idx / 64), e = (int)(idx % 64);
    int ti, tj;
    fp_tile_of(t, PT, ti, tj);
    const int i = 8 * ti + e / 8, j = 8 * tj + e % 8;
    if (i < p && j < p && i <= j) {
        if (!isfinite(s)) set_status(status, HYDE_ERR_NUMERIC);
        double* Gm = Gg + (long long)g * p * p;
        Gm[(long long)i * p + j] = s;
        Gm[(long long)j * p + i] = s;
    }
}

// Entry b of the orthonormal DCT-II basis vector k: the eigenvectors of
// D^T D (first-difference operator, free ends).
__device__ __forceinline__ double fp_dct(int b, int k, int p) {
    return k == 0 ? sqrt(1.0 / p) : sqrt(2.0 / p) * cospi((double)(2 * b + 1) * k / (2.0 * p));
}

// Block (k, g): E[g][k] = u_k^T G_g u_k for g < ngroups, and for
// g = ngroups the noise weights A_k = sum_b sigma_b^2 U_bk^2. Double; G_g is
// read by columns (coalesced; it is symmetric).
__global__ void __launch_bounds__(kEnergyThreads)
forpdn_energy_kernel(const double* __restrict__ Gg, const double* __restrict__ sigma, int p,
                     int ngroups, double* __restrict__ E) {
    pdl_wait();
    pdl_trigger();
    __shared__ double u[256];
    __shared__ double red[kEnergyThreads / 32];
    const int k = blockIdx.x, g = blockIdx.y, t = threadIdx.x;
    for (int b = t; b < p; b += kEnergyThreads) u[b] = fp_dct(b, k, p);
    __syncthreads();
    double acc = 0.0;
    if (g < ngroups) {
        const double* Gm = Gg + (long long)g * p * p;
        for (int a = t; a < p; a += kEnergyThreads) {
            double w = 0.0;
            for (int b = 0; b < p; ++b) w = fma(Gm[(long long)b * p + a], u[b], w);
            acc = fma(u[a], w, acc);
        }
    } else {
        for (int b = t; b < p; b += kEnergyThreads) acc = fma(sigma[b] * sigma[b], u[b] * u[b], acc);
    }
    acc = warp_sum_d(acc);
    if ((t & 31) == 0) red[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < kEnergyThreads / 32; ++w) s += red[w];
        E[(long long)g * p + k] = s;
    }
}

// Block g: the SURE table of group g over the grid lam_0 = 0,
// lam_m = 10^(-3 + 7 (m - 1) / (K - 2)), its first minimum, and the factors
// of the tridiagonal I + lam D^T D at it (diagonal 1 + lam deg_b, deg = 1 at
// the ends and 2 inside; off-diagonal -lam): m_0 = a_0,
// m_b = a_b - lam^2 / m_{b-1}, stored as inv_b = 1 / m_b and
// cp_b = -lam / m_b. Four threads share a grid point (k split four ways,
// fixed combination order); each term's factors are formed in float (their
// relative error, ~1e-7, is far below the table's use) and accumulated in
// double. The factorisation runs in double (for large lam the system's
// condition number, ~1 + 4 lam, amplifies float rounding in the pivots),
// with reciprocals from a float seed and two Newton-Raphson steps
// r <- r (2 - x r) (each squares the relative error, ~6e-8 -> ~4e-15 ->
// double rounding) in place of double divisions.
constexpr int kSelParts = 4;

__device__ __forceinline__ double rcp_newton(double x) {
    double r = (double)(1.0f / (float)x);
    r = r * fma(-x, r, 2.0);
    r = r * fma(-x, r, 2.0);
    return r;
}

__global__ void __launch_bounds__(256)
forpdn_select_kernel(const double* __restrict__ E, const double* __restrict__ sigma, int p,
                     int K, FpGeom G, double* __restrict__ sure, int* __restrict__ kidx,
                     float* __restrict__ tables, int* status, int* info) {
    pdl_wait();
    pdl_trigger();
    __shared__ float mu[256];
    __shared__ double Ek[256], Ak[256];
    __shared__ double S[256];
    __shared__ double part[256];
    __shared__ double s_sig2;
    const int g = blockIdx.x, t = threadIdx.x, ng = G.ngroups;
    for (int k = t; k < p; k += blockDim.x) {
        const double sn = sinpi((double)k / (2.0 * p));
        mu[k] = (float)(4.0 * sn * sn);
        Ek[k] = E[(long long)g * p + k];
        Ak[k] = E[(long long)ng * p + k];
    }
    if (t < 32) {
        double s2 = 0.0;
        for (int b = t; b < p; b += 32) s2 = fma(sigma[b], sigma[b], s2);
        s2 = warp_sum_d(s2);
        if (t == 0) s_sig2 = s2;
    }
    __syncthreads();
    double npos = 0.0;
    for (int r = 0; r < G.nrect[g]; ++r) npos += (double)G.rect[g][r].h * G.rect[g][r].w;
    for (int m0 = 0; m0 < K; m0 += 256 / kSelParts) {
        const int m = m0 + t / kSelParts, part_id = t % kSelParts;
        double s = 0.0;
        if (m < K) {
            const float lam = m == 0 ? 0.f
                                     : (float)exp10(-3.0 + 7.0 * (m - 1) / (double)(K > 2 ? K - 2 : 1));
            for (int k = part_id; k < p; k += kSelParts) {
                const float den = fmaf(lam, mu[k], 1.0f);
                const float iden = 1.0f / den;
                const float f = lam * mu[k] * iden;
                s = fma((double)(f * f), Ek[k], s);
                s = fma(2.0 * npos * (double)iden, Ak[k], s);
            }
        }
        part[t] = s;
        __syncthreads();
        if (part_id == 0 && m < K) {
            const double tot = ((part[t] + part[t + 1]) + (part[t + 2] + part[t + 3])) - npos * s_sig2;
            S[m] = tot;
            if (!isfinite(tot)) set_status(status, HYDE_ERR_NUMERIC);
            sure[(long long)g * K + m] = tot;
        }
        __syncthreads();
    }
    if (t == 0) {
        int best = 0;
        for (int m = 1; m < K; ++m)
            if (S[m] < S[best]) best = m;
        kidx[g] = best;
        if (info) info[1 + g] = best;
        const double lam = best == 0 ? 0.0
                                     : exp10(-3.0 + 7.0 * (best - 1) / (double)(K > 2 ? K - 2 : 1));
        float* inv = tables + (long long)g * (2 * p + 1);
        float* cpv = inv + p;
        double imprev = 1.0;
        for (int b = 0; b < p; ++b) {
            const double deg = p == 1 ? 0.0 : ((b == 0 || b == p - 1) ? 1.0 : 2.0);
            const double a = fma(lam, deg, 1.0);
            const double m = b == 0 ? a : fma(-lam * lam, imprev, a);
            const double im = rcp_newton(m);
            inv[b] = (float)im;
            cpv[b] = (float)(-lam * im);
            imprev = im;
        }
        inv[2 * p] = (float)lam;
    }
}

// A block of kSmoothThreads consecutive Mallat positions: their spectra
// (p band rows of kSmoothThreads floats) are copied into shared memory with
// 16-byte cp.async; one thread per position finds its group and solves the
// tridiagonal system there (forward values d_b = (c_b + lam d_{b-1}) / m_b,
// then x_b = d_b - cp_b x_{b+1}, in place); the block writes the rows back
// with 16-byte stores. The plane Hp Wp and the block's first position are
// multiples of 4, so every 16-byte piece is wholly inside or outside.
__global__ void __launch_bounds__(kSmoothThreads)
forpdn_smooth_kernel(float* __restrict__ C, int p, int Hp, int Wp, int levels,
                     const float* __restrict__ tables) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float fsm[];
    const int ng = levels + 1;
    const int ntab = (ng * (2 * p + 1) + 3) & ~3;
    float* tab = fsm;                          // [ng][2 p + 1]
    float* dsm = fsm + ntab;                   // [p][kSmoothThreads], 16-byte aligned
    const int t = threadIdx.x;
    const long long plane = (long long)Hp * Wp;
    const long long q0 = (long long)blockIdx.x * kSmoothThreads;
    constexpr int Q4 = kSmoothThreads / 4;
    for (int e = t; e < p * Q4; e += kSmoothThreads) {
        const int b = e / Q4, k4 = e - b * Q4;
        const long long q = q0 + 4 * k4;
        const bool ok = q < plane;
        const unsigned d = (unsigned)__cvta_generic_to_shared(dsm + b * kSmoothThreads + 4 * k4);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d),
                     "l"(C + (long long)b * plane + (ok ? q : 0)), "r"(ok ? 16 : 0));
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    for (int i = t; i < ng * (2 * p + 1); i += kSmoothThreads) tab[i] = tables[i];
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const long long q = q0 + t;
    if (q < plane) {
        const int y = (int)(q / Wp), x = (int)(q - (long long)y * Wp);
        int ly = 0, lx = 0;
        for (int j = 1; j <= levels; ++j) {
            if (y < (Hp >> j)) ly = j;
            if (x < (Wp >> j)) lx = j;
        }
        const int m = ly < lx ? ly : lx;
        const int g = m == levels ? 0 : m + 1;
        const float* inv = tab + g * (2 * p + 1);
        const float* cpv = inv + p;
        const float lam = inv[2 * p];
        float d = 0.f;
        for (int b = 0; b < p; ++b) {
            d = fmaf(lam, d, dsm[b * kSmoothThreads + t]) * inv[b];
            dsm[b * kSmoothThreads + t] = d;
        }
        float xv = d;
        for (int b = p - 2; b >= 0; --b) {
            xv = fmaf(-cpv[b], xv, dsm[b * kSmoothThreads + t]);
            dsm[b * kSmoothThreads + t] = xv;
        }
    }
    __syncthreads();
    for (int e = t; e < p * Q4; e += kSmoothThreads) {
        const int b = e / Q4, k4 = e - b * Q4;
        const long long qq = q0 + 4 * k4;
        if (qq < plane)
            *reinterpret_cast<float4*>(C + (long long)b * plane + qq) =
                *reinterpret_cast<const float4*>(dsm + b * kSmoothThreads + 4 * k4);
    }
}

}  // namespace

namespace {

struct FpLayout {
    int Hp, Wp, K, PT, ntiles, threads, blocks;
    long long n, N;
    GramPlan gram;
    FpGeom geom;
    size_t smem_gram, smem_smooth;
    size_t status, R, sigma, noise, partials, coef, scratch, gpart, Gg, E, sure, kidx, tables,
        total;
};

template <typename T>
inline T* fp_at(void* ws, size_t off) {
    return reinterpret_cast<T*>(reinterpret_cast<char*>(ws) + off);
}

hyde_status fp_layout(int p, int H, int W, int levels, int K, FpLayout* out) {
    if (p < 2 || p > kMaxBandsGram) return HYDE_ERR_SHAPE;
    if (K < 2 || K > 256) return HYDE_ERR_SHAPE;
    FpLayout L;
    if (!padded_dims(H, W, levels, &L.Hp, &L.Wp)) return HYDE_ERR_SHAPE;
    L.n = (long long)H * W;
    L.N = (long long)L.Hp * L.Wp;
    if (L.n < p) return HYDE_ERR_SHAPE;
    if (noise_smem_bytes(p) > 227 * 1024) return HYDE_ERR_SHAPE;
    hyde_status st = gram_plan(p, L.n, &L.gram);
    if (st != HYDE_OK) return st;
    if (gram_tf32_shape_ok(p, L.n)) {   // room for the split-TF32 Gram's partials too
        size_t tcb = 0;
        st = gram_tc_partial_bytes(p, &tcb);
        if (st != HYDE_OK) return st;
        if (tcb > L.gram.partial_bytes) L.gram.partial_bytes = tcb;
    }
    L.K = K;
    // groups and their rectangles of Mallat positions
    FpGeom& G = L.geom;
    memset(&G, 0, sizeof(G));
    G.ngroups = levels + 1;
    G.nrect[0] = 1;
    G.rect[0][0] = make_rect(0, 0, L.Hp >> levels, L.Wp >> levels);
    for (int l = 1; l <= levels; ++l) {
        const int h = L.Hp >> l, w = L.Wp >> l;
        G.nrect[l] = 2;
        G.rect[l][0] = make_rect(0, w, h, w);
        G.rect[l][1] = make_rect(h, 0, h, 2 * w);
    }
    long long total = 0;
    for (int g = 0; g < G.ngroups; ++g) {
        long long c = 0;
        for (int r = 0; r < G.nrect[g]; ++r)
            c += (long long)G.rect[g][r].h * ((G.rect[g][r].w + FKC - 1) / FKC);
        G.chunks[g] = c;
        total += c;
    }
    // blocks in proportion to the groups' chunks, at least one each
    const int sms = device_sm_count();
    if (sms <= 0) return HYDE_ERR_CUDA;
    const long long target = 2LL * sms;
    G.block0[0] = 0;
    for (int g = 0; g < G.ngroups; ++g) {
        long long b = (target * G.chunks[g] + total - 1) / total;
        if (b < 1) b = 1;
        if (b > G.chunks[g]) b = G.chunks[g] > 0 ? G.chunks[g] : 1;
        G.block0[g + 1] = G.block0[g] + (int)b;
    }
    L.blocks = G.block0[G.ngroups];
    L.PT = (p + 7) / 8;
    L.ntiles = L.PT * (L.PT + 1) / 2;
    L.threads = (L.ntiles < 128 ? 128 : (L.ntiles + 31) / 32 * 32);
    if (L.threads > kFpMaxThreads) return HYDE_ERR_SHAPE;
    L.smem_gram = (size_t)FSTAGES * L.PT * 8 * FKC * sizeof(float);
    L.smem_smooth = ((size_t)((G.ngroups * (2 * p + 1) + 3) & ~3) + (size_t)p * kSmoothThreads) *
                    sizeof(float);
    if (L.smem_gram > 227 * 1024 || L.smem_smooth > 227 * 1024) return HYDE_ERR_SHAPE;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(bytes, kAlign);
        return o;
    };
    L.status = take(sizeof(int));
    L.R = take((size_t)p * p * sizeof(double));
    L.sigma = take((size_t)p * sizeof(double));
    L.noise = take(noise_ws_bytes(p));
    L.partials = take(L.gram.partial_bytes);
    L.coef = take((size_t)p * L.N * sizeof(float));
    L.scratch = take((size_t)p * dwt_scratch_floats(L.Hp, L.Wp) * sizeof(float));
    L.gpart = take((size_t)L.blocks * L.ntiles * 64 * sizeof(float));
    L.Gg = take((size_t)G.ngroups * p * p * sizeof(double));
    L.E = take((size_t)(G.ngroups + 1) * p * sizeof(double));
    L.sure = take((size_t)G.ngroups * K * sizeof(double));
    L.kidx = take((size_t)G.ngroups * sizeof(int));
    L.tables = take((size_t)G.ngroups * (2 * p + 1) * sizeof(float));
    L.total = off;
    *out = L;
    return HYDE_OK;
}

}  // namespace
}  // namespace hyde

using namespace hyde;

extern "C" hyde_status hyde_forpdn_workspace_size(int p, int H, int W, int levels, int n_lambda,
                                                  size_t* bytes) {
    if (!bytes) return HYDE_ERR_INVALID_ARG;
    FpLayout L;
    const hyde_status st = fp_layout(p, H, W, levels, n_lambda, &L);
    if (st != HYDE_OK) return st;
    *bytes = L.total;
    return HYDE_OK;
}

extern "C" hyde_status hyde_forpdn(const float* Y, float* X, int p, int H, int W, int levels,
                                   int n_lambda, int* info, double* sure, void* ws,
                                   size_t ws_bytes, cudaStream_t stream) {
    if (!Y || !X) return HYDE_ERR_INVALID_ARG;
    FpLayout L;
    hyde_status st = fp_layout(p, H, W, levels, n_lambda, &L);
    if (st != HYDE_OK) return st;
    if (!ws || ((uintptr_t)ws % kAlign) != 0 || ws_bytes < L.total) return HYDE_ERR_WORKSPACE;
    const FpGeom& G = L.geom;
    int* status = info ? info : fp_at<int>(ws, L.status);
    if (cudaMemsetAsync(status, 0, info ? (size_t)(G.ngroups + 1) * sizeof(int) : sizeof(int),
                        stream) != cudaSuccess)
        return HYDE_ERR_CUDA;
    double* R = fp_at<double>(ws, L.R);
    double* sigma = fp_at<double>(ws, L.sigma);
    float* coef = fp_at<float>(ws, L.coef);
    float* scratch = fp_at<float>(ws, L.scratch);
    // 1. noise level by regression from the Gram matrix (the HyRes stage)
    if (gram_tf32_supported(Y, p, L.n))
        st = launch_gram_tf32(Y, p, L.n, fp_at<float>(ws, L.partials), R, status, stream);
    else
        st = launch_gram(Y, p, L.n, L.gram, fp_at<float>(ws, L.partials), R, status, stream);
    if (st != HYDE_OK) return st;
    st = launch_noise_from_gram(R, p, L.n, sigma, fp_at<void>(ws, L.noise), status, stream);
    if (st != HYDE_OK) return st;
    // 2. DWT of every band, read through the symmetric extension
    const DwtSrc src{Y, L.n, W, H, W};
    st = launch_dwt2(src, coef, p, L.Hp, L.Wp, levels, scratch, stream, status);
    if (st != HYDE_OK) return st;
    // 3. Gram matrices of the groups' spectra
    float* gpart = fp_at<float>(ws, L.gpart);
    double* Gg = fp_at<double>(ws, L.Gg);
    auto gram_go = [&](auto kernel) -> hyde_status {
        if (ensure_smem_limit((const void*)kernel, (int)L.smem_gram) != cudaSuccess)
            return HYDE_ERR_CUDA;
        launch_pdl(kernel, L.blocks, L.threads, L.smem_gram, stream, (const float*)coef, p, L.Wp,
                   L.N, G, L.PT, L.ntiles, gpart);
        return HYDE_OK;
    };
    st = L.threads <= 256 ? gram_go(forpdn_gram_kernel<256>) : gram_go(forpdn_gram_kernel<kFpMaxThreads>);
    if (st != HYDE_OK) return st;
    launch_pdl(forpdn_gram_reduce_kernel, dim3((unsigned)((L.ntiles * 64 + 255) / 256), G.ngroups),
               dim3(256), 0, stream, (const float*)gpart, G, p, L.PT, L.ntiles, Gg, status);
    // 4. DCT energies and noise weights, 5. SURE and the factors
    double* E = fp_at<double>(ws, L.E);
    launch_pdl(forpdn_energy_kernel, dim3((unsigned)p, G.ngroups + 1), dim3(kEnergyThreads), 0,
               stream, (const double*)Gg, (const double*)sigma, p, G.ngroups, E);
    float* tables = fp_at<float>(ws, L.tables);
    launch_pdl(forpdn_select_kernel, G.ngroups, 256, 0, stream, (const double*)E,
               (const double*)sigma, p, L.K, G, sure ? sure : fp_at<double>(ws, L.sure),
               fp_at<int>(ws, L.kidx), tables, status, info);
    // 6. the spectral smoothing in place, 7. inverse DWT with the crop
    if (ensure_smem_limit((const void*)forpdn_smooth_kernel, (int)L.smem_smooth) != cudaSuccess)
        return HYDE_ERR_CUDA;
    launch_pdl(forpdn_smooth_kernel, (unsigned)((L.N + kSmoothThreads - 1) / kSmoothThreads),
               kSmoothThreads, L.smem_smooth, stream, coef, p, L.Hp, L.Wp, levels,
               (const float*)tables);
    st = launch_idwt2(coef, X, p, L.Hp, L.Wp, H, W, levels, scratch, nullptr, nullptr, stream);
    if (st != HYDE_OK) return st;
    return cuda_status(cudaGetLastError());
}

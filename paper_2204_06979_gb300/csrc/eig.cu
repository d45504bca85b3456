// Leading r eigenpairs of the whitened Gram matrix, the spectral subspace of
// the low-rank model (arXiv 2204.06979, Sec. 2.1 "low-rank"): three kernels.
//
//  1. Tridiagonalisation (one block): the matrix, optionally whitened on load
//     (A_ij / (wsig_i wsig_j)) and scaled by 1 / max |diag|, is reduced to
//     tridiagonal form T = Q^T A Q by Householder reflectors in float.
//     eig_tridiag_reg_kernel (p <= 160, 512 threads) keeps the trailing
//     matrix in registers, eig_tridiag_kernel (larger p, 1024 threads) in
//     shared memory. Both write T (d, e), the reflectors as explicit vectors
//     (row k = v_k) and tau_k to the workspace.
//  2. eig_pair_kernel (one block of 256 threads per wanted eigenpair, r
//     blocks on r SMs): the eigenvalue by multisection (every thread counts
//     the eigenvalues of T below one of 256 points, Sturm sequence; a few
//     rounds reach float resolution), the eigenvector of T from a twisted
//     factorisation at it (one warp), and its back-transformation by the
//     reflectors in blocks of eight (compact WY form, built by the other
//     warps meanwhile).
//  3. eig_orth_kernel (one block): Cholesky QR, twice, of the r vectors in
//     descending order (Gram-Schmidt in that order; orthogonality inside
//     clusters of close eigenvalues), the sign rule (largest-magnitude entry
//     positive), and the write-out in double.
// The p-step Householder recurrence is the only part bound to one SM; the
// per-eigenpair work runs on r SMs at once.
#include <float.h>

#include "hyde_internal.cuh"

#ifndef HYDE_EIG_WARPS
#define HYDE_EIG_WARPS 16
#endif

namespace hyde {
namespace {

constexpr int kLA = 1024;                   // threads of the tridiagonalisation block
constexpr int kEigWarps = HYDE_EIG_WARPS;   // warps of the Householder sweep
constexpr int kPairThreads = 256;           // threads per eigenpair block
constexpr int kMaxWyBlocks = 32;            // blocks of 8 reflectors, p <= 258

// Workspace of the three kernels (floats): reflectors [p][p] (row k = v_k,
// k < p - 2), tau, d, e (p each), the scale, the eigenvalues of
// the scaled T (32), and the back-transformed vectors X [r][p].
struct EigWs {
    float* refl;
    float* tau;
    float* d;
    float* e;
    float* scale;
    float* lam;
    float* X;
};

__host__ __device__ inline EigWs eig_ws_carve(float* base, int p) {
    EigWs w;
    float* q = base;
    w.refl = q;  q += (size_t)p * p;
    w.tau = q;   q += p;
    w.d = q;     q += p;
    w.e = q;     q += p;
    w.scale = q; q += 4;
    w.lam = q;   q += 32;
    w.X = q;
    return w;
}

// Window blockIdx.y of a batched call: every workspace pointer moves by the
// window's stride (floats); one-window launches have gridDim.y = 1.
__device__ __forceinline__ EigWs eig_ws_window(EigWs w, long long off) {
    w.refl += off; w.tau += off; w.d += off; w.e += off;
    w.scale += off; w.lam += off; w.X += off;
    return w;
}

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

// Number of eigenvalues of the tridiagonal T (diagonal d, squared
// off-diagonal e2) below x, from the signs of the characteristic
// polynomials of its leading blocks, P_0 = 1, P_1 = d_0 - x,
// P_{i+1} = (d_i - x) P_i - e_{i-1}^2 P_{i-1} (Sturm's theorem: the sign
// changes of P_0 .. P_p number the eigenvalues below x; a zero P_i takes the
// sign opposite to P_{i-1}, as a zero pivot of the LDL^T form counts as
// negative). One FMA per step on the dependent path (the
// product e^2 P_{i-1} is known a step ahead); every second step both
// values are scaled by a power of two so that the larger is in [1, 2),
// which keeps the signs and prevents overflow and underflow.
__device__ __forceinline__ int sturm_count_poly(const float* d, const float* e2, int p, float x) {
    float Pm = 1.0f, P = d[0] - x;
    bool s = !(P > 0.f);
    int c = s;
#pragma unroll 8
    for (int i = 1; i < p; ++i) {
        const float t = e2[i - 1] * Pm;
        const float Pn = fmaf(d[i] - x, P, -t);
        const bool sn = Pn < 0.f || (Pn == 0.f && !s);
        c += sn != s;
        s = sn;
        Pm = P;
        P = Pn;
        if (i & 1) {
            const float m = fmaxf(fabsf(P), fabsf(Pm));
            const int ex = min((__float_as_int(m) >> 23) & 255, 254);
            const float sc = __int_as_float((254 - ex) << 23);
            P *= sc;
            Pm *= sc;
        }
    }
    return c;
}

// Scalars of the Householder reflector that maps (alpha, x) onto beta e_0
// (ss = |x|^2): v = e_0 + sc x, H = I - tau v v^T. ss == 0 gives the identity
// (tau = 0).
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

// The same scalars with one reciprocal square root and one reciprocal on the
// dependent path: with n = |(alpha, x)|, beta = -sign(alpha) n,
// tau = 1 + |alpha| / n and sc = sign(alpha) / (|alpha| + n). Tiny norms
// (below FLT_MIN, where the approximate rsqrt flushes) take hh_scalars_of.
__device__ __forceinline__ void hh_scalars_fast(float alpha, float ss, float& tau, float& sc,
                                                float& beta) {
    const float s2 = fmaf(alpha, alpha, ss);
    if (!(ss > 0.f) || s2 < FLT_MIN) {
        hh_scalars_of(alpha, ss, tau, sc, beta);
        return;
    }
    const float rn = rsqrtf(s2);
    const float nrm = s2 * rn;
    const float aa = fabsf(alpha);
    const float sg = alpha >= 0.f ? 1.0f : -1.0f;
    beta = -sg * nrm;
    tau = fmaf(aa, rn, 1.0f);
    sc = __fdividef(sg, aa + nrm);
}

// One sweep of the fused step (see eig_tridiag_kernel) over the column chunks
// b >= B0: row i (> k+1) of this warp gets update k on its columns > k+1
// (column k+1 is read but not stored) and sacc collects the row's product
// with v_{k+1}. The chunk range is a compile-time bound so that the loads of
// a row issue together.
template <int NB, int NA, int NW, int B0>
__device__ __forceinline__ void tri_sweep_from(float* A, int lda, int p, int k, int i0, int lane,
                                               const float (&vreg)[NB], const float (&wreg)[NB],
                                               const float (&vn)[NB], float sc_k, float K,
                                               const float* pc, float (&sacc)[NA]) {
    const int jn = k + 1;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const int i = i0 + NW * a;
        sacc[a] = 0.f;
        if (i > k + 1 && i < p) {
            float* row = A + i * lda;
            const float vi = A[k * lda + i] * sc_k, wi = fmaf(-K, vi, pc[i]);
#pragma unroll
            for (int b = B0; b < NB; ++b) {
                const int j = lane + 32 * b;
                if (b < NB - 1 || j < p) {
                    const float x = fmaf(-vi, wreg[b], fmaf(-wi, vreg[b], row[j]));
                    if (j > jn) row[j] = x;
                    sacc[a] = fmaf(x, vn[b], sacc[a]);
                }
            }
        }
    }
}

// Dispatch on the first live chunk b0 = (k + 2) / 32 (chunks left of it hold
// only columns <= k+1, which update k leaves unchanged).
template <int NB, int NA, int NW, int B0 = 0>
__device__ __forceinline__ void tri_sweep(int b0, float* A, int lda, int p, int k, int i0, int lane,
                                          const float (&vreg)[NB], const float (&wreg)[NB],
                                          const float (&vn)[NB], float sc_k, float K,
                                          const float* pc, float (&sacc)[NA]) {
    if constexpr (B0 < NB - 1) {
        if (b0 > B0) {
            tri_sweep<NB, NA, NW, B0 + 1>(b0, A, lda, p, k, i0, lane, vreg, wreg, vn, sc_k, K, pc,
                                          sacc);
            return;
        }
    }
    tri_sweep_from<NB, NA, NW, B0>(A, lda, p, k, i0, lane, vreg, wreg, vn, sc_k, K, pc, sacc);
}

// --------------------------------------------------------------------------
// 1. Householder tridiagonalisation with the matrix in shared memory and the
// per-step vectors in registers (NB = ceil(p/32) column chunks per lane).
// Warp w owns rows i = w (mod NW) of the trailing matrix, lane l owns columns
// j = l + 32b, and caches v_j and w_j of those columns in registers, so a
// matrix element costs one load and one FMA in the matvec and one load, two
// FMAs and one store in the rank-2 update; K = tau/2 v^T p is one warp
// shuffle-sum per warp.
// --------------------------------------------------------------------------
template <int NB, int NW>
__global__ void __launch_bounds__(kLA, 1)
eig_tridiag_kernel(const double* __restrict__ Ain, const double* __restrict__ wsig, int p,
                   EigWs G, int* status, long long wst) {
    pdl_wait();
    pdl_trigger();
    if (blockIdx.y) {
        const int wi = blockIdx.y;
        Ain += (long long)wi * p * p;
        if (wsig) wsig += (long long)wi * p;
        G = eig_ws_window(G, wi * wst);
        if (status) status += wi;
    }
    extern __shared__ float sm[];
    const int lda = p + 1;
    float* q = sm;
    float* A = q;    q += p * lda;
    float* tauv = q; q += p;
    float* dv = q;   q += p;
    float* ev = q;   q += p;
    float* vf = q;   q += p;     // whitening weights, then reflector scales
    float* pvv = q;  q += 2 * p; // p = tau A v of this step and the next
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
    const int nwarps = (int)(blockDim.x >> 5);
    for (int i = wid; i < p; i += nwarps) {
        const float si = iw[i] * scale;
        for (int j = lane; j < p; j += 32)
            A[i * lda + j] = d2f_bits(Ain[(long long)i * p + j]) * si * iw[j];
    }
    __syncthreads();

    // Fused steps, one barrier each. Reflector k is kept as (row k of A,
    // scale sc_k): v_k[i] = 1 at i = k+1, A[k][i] sc_k beyond (row 0 is
    // column 0 of the symmetric input). Per step, every warp redundantly:
    // K = tau/2 v^T p from p in shared memory, w = p - K v on its lanes'
    // columns, the updated column k+1 (x_j = A[j][k+1] - w_j - v_j w_{k+1} on
    // its lanes) and its sum of squares, so reflector k+1's scalars and v_{k+1}
    // need no barrier; warp 0 stores x into row k+1 (the reflector's home);
    // then one sweep over the warp's rows applies update k to columns > k+1
    // and accumulates p' = A' v_{k+1} (row sums by a reduce-scatter). Column
    // k+1 itself is never stored by the sweep (the other warps read it in
    // the same step), and column chunks left of k+2 are skipped.
    float* const scv = vf;           // reflector scales (vf is free after the load)
    constexpr int NA = (32 * NB + NW - 1) / NW;   // trailing rows per warp
    if (wid < NW) {
    // prologue: reflector 0 (scalars in every warp) and p_0 = tau_0 A v_0
    float tau_k = 0.f, sc_k = 0.f;
    float vreg[NB];
    if (p >= 3) {
        // reflector 0 from row 0 (where the sweep reads it; the whitened
        // matrix is symmetric only to rounding)
        float ss = 0.f;
        for (int i = 2 + lane; i < p; i += 32) { const float x = A[i]; ss = fmaf(x, x, ss); }
        ss = warp_sum(ss);
        float beta;
        hh_scalars_of(A[1], ss, tau_k, sc_k, beta);
        if (t == 0) { tauv[0] = tau_k; scv[0] = sc_k; dv[0] = A[0]; ev[0] = beta; }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = lane + 32 * b;
            vreg[b] = j == 1 ? 1.0f : ((j > 1 && j < p) ? A[j] * sc_k : 0.f);
        }
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
        const int jn = k + 1;
        // the loads of this step that do not depend on K, issued together
        // (indices clamped into the matrix; masked below)
        const float pjn = pc[jn];
        float pjr[NB], colr[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = lane + 32 * b;
            const int jc = j < p ? j : p - 1;
            pjr[b] = pc[jc];
            colr[b] = A[jc * lda + jn];
        }
        // K = tau/2 v^T p and w = p - K v (v_k, p_k nonzero on rows > k)
        float pj[NB];
        float kp = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = lane + 32 * b;
            pj[b] = (j > k && j < p) ? pjr[b] : 0.f;
            kp = fmaf(vreg[b], pj[b], kp);
        }
        const float K = 0.5f * tau_k * warp_sum(kp);
        float wreg[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) wreg[b] = fmaf(-K, vreg[b], pj[b]);
        // column k+1 after update k on this warp's lanes (v_k[jn] = 1)
        const float wjn = pjn - K;
        float xj[NB];
        float ss = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = lane + 32 * b;
            const float x = fmaf(-vreg[b], wjn, colr[b] - wreg[b]);
            xj[b] = (j >= jn && j < p) ? x : 0.f;
            ss = fmaf(j >= k + 3 ? xj[b] : 0.f, xj[b], ss);
        }
        ss = warp_sum(ss);
        float xd = 0.f, xa = 0.f;                // x_{k+1} (diagonal) and x_{k+2} (alpha)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (b == (jn >> 5)) xd = xj[b];
            if (b == ((k + 2) >> 5)) xa = xj[b];
        }
        xd = __shfl_sync(0xffffffffu, xd, jn & 31);
        xa = __shfl_sync(0xffffffffu, xa, (k + 2) & 31);
        float tau_n = 0.f, sc_n = 0.f;
        float vn[NB];
        if (has_next) {
            float beta;
            hh_scalars_fast(xa, ss, tau_n, sc_n, beta);
            if (t == 0) {
                tauv[k + 1] = tau_n; scv[k + 1] = sc_n;
                dv[k + 1] = xd; ev[k + 1] = beta;
            }
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int j = lane + 32 * b;
                vn[b] = j == k + 2 ? 1.0f : ((j > k + 2 && j < p) ? xj[b] * sc_n : 0.f);
            }
            if (wid == 0) {
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const int j = lane + 32 * b;
                    if (j >= k + 3 && j < p) A[jn * lda + j] = xj[b];
                }
            }
        } else {
            // last step (k = p - 3): T's last off-diagonal is x_{p-1}
            if (t == 0) {
                tauv[k + 1] = 0.f; scv[k + 1] = 0.f;
                dv[k + 1] = xd; ev[k + 1] = xa;
            }
#pragma unroll
            for (int b = 0; b < NB; ++b) vn[b] = 0.f;
        }
        // fused sweep: update k on rows > k+1, columns > k+1; accumulate p' rows
        const int i0 = k + 1 + ((wid - (k + 1)) & (NW - 1));
        float sacc[NA];
        tri_sweep<NB, NA, NW>((k + 2) >> 5, A, lda, p, k, i0, lane, vreg, wreg, vn, sc_k, K, pc,
                              sacc);
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
    // reflector k as an explicit vector in row k: 0 up to k, 1 at k+1,
    // x * scale beyond (the back-transformation then reads it directly)
    for (int k = wid; k < p - 2; k += nwarps) {
        const float sck = scv[k];
        for (int i = lane; i < p; i += 32) {
            float* a = A + k * lda + i;
            *a = i <= k ? 0.f : (i == k + 1 ? 1.0f : *a * sck);
        }
    }
    __syncthreads();
    if (t == 0) {
        // p >= 3: the last step wrote d[p-2] and e[p-2]; A[p-1][p-1] is current
        if (p == 2) {
            dv[0] = A[0];
            ev[0] = A[lda];
            tauv[0] = 0.f;
        }
        dv[p - 1] = A[(p - 1) * lda + (p - 1)];
        ev[p - 1] = 0.f;
    }
    __syncthreads();
    // write-out: T, the reflectors as rows (row k of A, already explicit),
    // tau and the scale
    for (int k = wid; k < p - 2; k += nwarps)
        for (int i = lane; i < p; i += 32) G.refl[(size_t)k * p + i] = A[k * lda + i];
    for (int i = t; i < p; i += blockDim.x) {
        G.d[i] = dv[i];
        G.e[i] = ev[i];
        G.tau[i] = tauv[i];
    }
    if (t == 0) G.scale[0] = scale;
}

// --------------------------------------------------------------------------
// 1'. The same reduction with the trailing matrix in registers, for
// p <= 32 NB, NB <= kRegMaxNB (512 threads, up to 128 registers each). Warp
// w keeps rows i = w + 16 a (a < 2 NB) of A, lane l columns l + 32 b, so the
// sweep of a step is register arithmetic only: shared memory carries the
// vectors, one published row per step and the reflectors. At the end of
// step k the owner of row k+2 publishes it (updated) for step k+1, whose
// column k+2 is that row by symmetry; warp 0 stores each reflector's raw
// entries as a row of `refl`. One barrier per step.
// --------------------------------------------------------------------------
constexpr int kRegThreads = 512;
constexpr int kRegMaxNB = 5;

// Rows a >= A0 of this warp (i = wid + 16 a), column chunks b >= A0 / 2:
// update k and the row sums with v_{k+1}, without branches (a row that is
// not in the trailing block gets v_i = w_i = 0 and contributes 0). Rows below
// slot A0 = (k + 2) / 16 and chunks below (k + 2) / 32 lie left of or above
// the trailing block in every warp.
template <int NB, int NA, int A0>
__device__ __forceinline__ void tri_sweep_reg_from(float (&M)[NA][NB], const float* refl_k,
                                                   int p, int k, int wid,
                                                   const float (&vreg)[NB], const float (&wreg)[NB],
                                                   const float (&vn)[NB], float sc_k, float K,
                                                   const float* pc, float (&sacc)[NA]) {
    constexpr int B0 = A0 / 2;
#pragma unroll
    for (int a = 0; a < NA; ++a) sacc[a] = 0.f;
    float vi[NA], wi[NA];
#pragma unroll
    for (int a = A0; a < NA; ++a) {
        const int i = wid + 16 * a;
        const bool act = i > k + 1 && i < p;
        const int ic = act ? i : k + 2;
        const float v = refl_k[ic] * sc_k, pi = pc[ic];
        vi[a] = act ? v : 0.f;
        wi[a] = act ? fmaf(-K, v, pi) : 0.f;
    }
#pragma unroll
    for (int a = A0; a < NA; ++a) {
        float s = 0.f;
#pragma unroll
        for (int b = B0; b < NB; ++b) {
            const float x = fmaf(-vi[a], wreg[b], fmaf(-wi[a], vreg[b], M[a][b]));
            M[a][b] = x;
            s = fmaf(x, vn[b], s);
        }
        const int i = wid + 16 * a;
        sacc[a] = (i > k + 1 && i < p) ? s : 0.f;
    }
}

template <int NB, int NA, int A0 = 0>
__device__ __forceinline__ void tri_sweep_reg(int a0, float (&M)[NA][NB], const float* refl_k,
                                              int p, int k, int wid,
                                              const float (&vreg)[NB], const float (&wreg)[NB],
                                              const float (&vn)[NB], float sc_k, float K,
                                              const float* pc, float (&sacc)[NA]) {
    if constexpr (A0 < NA - 1) {
        if (a0 > A0) {
            tri_sweep_reg<NB, NA, A0 + 1>(a0, M, refl_k, p, k, wid, vreg, wreg, vn, sc_k, K, pc,
                                          sacc);
            return;
        }
    }
    tri_sweep_reg_from<NB, NA, A0>(M, refl_k, p, k, wid, vreg, wreg, vn, sc_k, K, pc, sacc);
}

// Row i = wid + 16 a of M into dst[0..p) (compile-time a; the owner warp
// only).
template <int NB, int NA>
__device__ __forceinline__ void publish_row(const float (&M)[NA][NB], int a_pub, int lane, int p,
                                            float* dst) {
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        if (a == a_pub) {
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int j = lane + 32 * b;
                if (j < p) dst[j] = M[a][b];
            }
        }
    }
}

// Entry i of the explicit reflector k from its raw row (see the kernel).
__device__ __forceinline__ float refl_entry(const float* refl, int p, const float* scv, int k,
                                            int i) {
    return i <= k ? 0.f : (i == k + 1 ? 1.0f : refl[k * p + i] * scv[k]);
}

template <int NB>
__global__ void __launch_bounds__(kRegThreads, 1)
eig_tridiag_reg_kernel(const double* __restrict__ Ain, const double* __restrict__ wsig, int p,
                       EigWs G, int* status, long long wst) {
    pdl_wait();
    pdl_trigger();
    if (blockIdx.y) {
        const int wi = blockIdx.y;
        Ain += (long long)wi * p * p;
        if (wsig) wsig += (long long)wi * p;
        G = eig_ws_window(G, wi * wst);
        if (status) status += wi;
    }
    constexpr int NA = 2 * NB;                 // rows per warp: i = wid + 16 a < 32 NB
    extern __shared__ float sm[];
    float* q = sm;
    float* refl = q;  q += p * p;              // row k: raw entries of reflector k
    float* rowb = q;  q += 2 * p;              // the published row, by step parity
    float* pvv = q;   q += 2 * p;              // p = tau A v, by step parity
    float* tauv = q;  q += p;
    float* dv = q;    q += p;
    float* ev = q;    q += p;
    float* scv = q;   q += p;                  // reflector scales
    float* iw = q;    q += p;                  // whitening weights
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int i = t; i < p; i += kRegThreads) { tauv[i] = 0.f; dv[i] = 0.f; ev[i] = 0.f; scv[i] = 0.f; }

    __shared__ float s_scale;
    __shared__ int s_mx;
    if (t == 0) s_mx = 0;
    __syncthreads();
    for (int i = t; i < p; i += kRegThreads) {
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
    float M[NA][NB];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const int i = wid + 16 * a;
        const float si = i < p ? iw[i] * scale : 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = lane + 32 * b;
            M[a][b] = (i < p && j < p) ? d2f_bits(Ain[(long long)i * p + j]) * si * iw[j] : 0.f;
        }
    }
    // row 0 is column 0 (reflector 0's source); row 1 is step 0's column 1
    if (wid == 0) publish_row<NB, NA>(M, 0, lane, p, refl);
    if (wid == 1) publish_row<NB, NA>(M, 0, lane, p, rowb);
    __syncthreads();

    float tau_k = 0.f, sc_k = 0.f;
    float vreg[NB];
    if (p >= 3) {
        float ss = 0.f;
        for (int i = 2 + lane; i < p; i += 32) { const float x = refl[i]; ss = fmaf(x, x, ss); }
        ss = warp_sum(ss);
        float beta;
        hh_scalars_of(refl[1], ss, tau_k, sc_k, beta);
        if (t == 0) { tauv[0] = tau_k; scv[0] = sc_k; dv[0] = refl[0]; ev[0] = beta; }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = lane + 32 * b;
            vreg[b] = j == 1 ? 1.0f : ((j > 1 && j < p) ? refl[j] * sc_k : 0.f);
        }
        float sacc[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            sacc[a] = 0.f;
#pragma unroll
            for (int b = 0; b < NB; ++b) sacc[a] = fmaf(M[a][b], vreg[b], sacc[a]);
        }
        int a_own;
        const float tot = rows_reduce_scatter<NA>(sacc, lane, a_own);
        const int i = wid + 16 * a_own;
        if (a_own < NA && (lane & (32 / rows_groups(NA) - 1)) == 0 && i >= 1 && i < p)
            pvv[i] = tot * tau_k;
    }
    __syncthreads();
    for (int k = 0; k + 2 < p; ++k) {
        const float* pc = pvv + (k & 1) * p;
        float* pn = pvv + ((k + 1) & 1) * p;
        const float* rb = rowb + (k & 1) * p;       // row k+1 of A after update k-1
        const bool has_next = k + 4 <= p;
        const int jn = k + 1;
        const float pjn = pc[jn];
        // x_{k+1} and x_{k+2} from the same inputs and operations as their
        // owner lanes use below (v_k[k+1] = 1, v_k[k+2] from reflector k's row)
        const float cjn = rb[jn], c2 = rb[k + 2], p2 = pc[k + 2];
        const float v2 = refl[k * p + k + 2] * sc_k;
        float pjr[NB], colr[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = lane + 32 * b;
            const int jc = j < p ? j : p - 1;
            pjr[b] = pc[jc];
            colr[b] = rb[jc];
        }
        // K = tau/2 v^T p and w = p - K v (v_k, p_k nonzero on rows > k)
        float pj[NB];
        float kp = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = lane + 32 * b;
            pj[b] = (j > k && j < p) ? pjr[b] : 0.f;
            kp = fmaf(vreg[b], pj[b], kp);
        }
        const float K = 0.5f * tau_k * warp_sum(kp);
        float wreg[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) wreg[b] = fmaf(-K, vreg[b], pj[b]);
        // row (= column) k+1 after update k on this warp's lanes (v_k[jn] = 1)
        const float wjn = pjn - K;
        float xj[NB];
        float ss = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = lane + 32 * b;
            const float x = fmaf(-vreg[b], wjn, colr[b] - wreg[b]);
            xj[b] = (j >= jn && j < p) ? x : 0.f;
            ss = fmaf(j >= k + 3 ? xj[b] : 0.f, xj[b], ss);
        }
        ss = warp_sum(ss);
        // x_{k+1} (diagonal) and x_{k+2} (alpha), bitwise as in their lanes
        const float xd = fmaf(-1.0f, wjn, cjn - fmaf(-K, 1.0f, pjn));
        const float xa = fmaf(-v2, wjn, c2 - fmaf(-K, v2, p2));
        float tau_n = 0.f, sc_n = 0.f;
        float vn[NB];
        if (has_next) {
            float beta;
            hh_scalars_fast(xa, ss, tau_n, sc_n, beta);
            if (t == 0) {
                tauv[k + 1] = tau_n; scv[k + 1] = sc_n;
                dv[k + 1] = xd; ev[k + 1] = beta;
            }
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int j = lane + 32 * b;
                vn[b] = j == k + 2 ? 1.0f : ((j > k + 2 && j < p) ? xj[b] * sc_n : 0.f);
            }
            if (wid == 0) {
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const int j = lane + 32 * b;
                    if (j >= k + 2 && j < p) refl[jn * p + j] = xj[b];
                }
            }
        } else {
            // last step (k = p - 3): T's last off-diagonal is x_{p-1}
            if (t == 0) {
                tauv[k + 1] = 0.f; scv[k + 1] = 0.f;
                dv[k + 1] = xd; ev[k + 1] = xa;
            }
#pragma unroll
            for (int b = 0; b < NB; ++b) vn[b] = 0.f;
        }
        // sweep: update k on this warp's rows > k+1 (registers), p' row sums
        float sacc[NA];
        tri_sweep_reg<NB, NA>((k + 2) >> 4, M, refl + k * p, p, k, wid, vreg, wreg, vn, sc_k, K,
                              pc, sacc);
        // row k+2, now current, for the next step's column
        if (wid == ((k + 2) & 15)) publish_row<NB, NA>(M, (k + 2) >> 4, lane, p,
                                                       rowb + ((k + 1) & 1) * p);
        if (has_next) {
            int a_own;
            const float tot = rows_reduce_scatter<NA>(sacc, lane, a_own);
            const int i = wid + 16 * a_own;
            if (a_own < NA && (lane & (32 / rows_groups(NA) - 1)) == 0 && i > k + 1 && i < p)
                pn[i] = tot * tau_n;
        }
        tau_k = tau_n;
        sc_k = sc_n;
#pragma unroll
        for (int b = 0; b < NB; ++b) vreg[b] = vn[b];
        __syncthreads();
    }
    // the last diagonal entry: its owner publishes row p-1 (the row buffers
    // are free once the loop has ended)
    if (wid == ((p - 1) & 15)) publish_row<NB, NA>(M, (p - 1) >> 4, lane, p, rowb);
    __syncthreads();
    if (t == 0) {
        dv[p - 1] = rowb[p - 1];
        if (p == 2) {
            dv[0] = refl[0];
            ev[0] = refl[1];
            tauv[0] = 0.f;
        }
        ev[p - 1] = 0.f;
    }
    __syncthreads();
    // write-out: T, the explicit reflectors as rows, tau and the scale
    for (int k = wid; k < p - 2; k += 16)
        for (int i = lane; i < p; i += 32) G.refl[(size_t)k * p + i] = refl_entry(refl, p, scv, k, i);
    for (int i = t; i < p; i += kRegThreads) {
        G.d[i] = dv[i];
        G.e[i] = ev[i];
        G.tau[i] = tauv[i];
    }
    if (t == 0) G.scale[0] = scale;
}

size_t eig_tridiag_reg_bytes(int p) { return ((size_t)p * p + 9 * (size_t)p) * sizeof(float); }

// --------------------------------------------------------------------------
// 2. One eigenpair per block: multisection, twisted factorisation and
// back-transformation of eigenpair c (c = 0: the largest eigenvalue).
// --------------------------------------------------------------------------
template <int NB>
__global__ void __launch_bounds__(kPairThreads)
eig_pair_kernel(EigWs G, int p, int* status, long long wst) {
    pdl_wait();
    pdl_trigger();
    if (blockIdx.y) {
        G = eig_ws_window(G, blockIdx.y * wst);
        if (status) status += blockIdx.y;
    }
    extern __shared__ float sm[];
    float* d = sm;
    float* e = d + p;
    float* e2 = e + p;
    float* tau = e2 + p;
    float* Dp = tau + p;
    float* Dm = Dp + p;
    float* z = Dm + p;
    float* refl = z + 2 * p;      // [p - 2][p] at 8 p floats: 16-byte aligned for cp.async
    __shared__ float s_lo, s_hi, s_pivmin;
    const int c = blockIdx.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int i = t; i < p; i += kPairThreads) {
        const float di = G.d[i], ei = G.e[i];
        d[i] = di;
        e[i] = ei;
        e2[i] = ei * ei;
        tau[i] = G.tau[i];
        if (!isfinite(di) || !isfinite(ei)) set_status(status, HYDE_ERR_NUMERIC);
    }
    // the reflectors, for the back-transformation at the end: asynchronous
    // 16-byte copies (p - 2 rows of p floats) that land while the
    // multisection runs
    {
        const int nv = (p - 2) * p;
        for (int i = t; i < nv / 4; i += kPairThreads)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                             (uint32_t)__cvta_generic_to_shared(refl + 4 * i)),
                         "l"(G.refl + 4 * i));
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        for (int i = (nv / 4) * 4 + t; i < nv; i += kPairThreads) refl[i] = G.refl[i];
    }
    __syncthreads();
    if (wid == 0) {
        float lo = FLT_MAX, hi = -FLT_MAX, emax = 0.f;
        for (int i = lane; i < p; i += 32) {
            const float rad = fabsf(e[i]) + (i > 0 ? fabsf(e[i - 1]) : 0.f);
            lo = fminf(lo, d[i] - rad);
            hi = fmaxf(hi, d[i] + rad);
            emax = fmaxf(emax, e2[i]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        }
        if (lane == 0) {
            const float w = hi - lo;
            s_lo = lo - 1e-6f * fmaxf(w, 1e-30f);
            s_hi = hi + 1e-6f * fmaxf(w, 1e-30f);
            s_pivmin = FLT_MIN * fmaxf(1.f, emax);
        }
    }
    __syncthreads();
    // multisection: point t of kPairThreads splits [lo, hi]; the count of
    // points with at most `target` eigenvalues below them brackets the
    // (target+1)-th smallest eigenvalue between two neighbouring points
    const int target = p - 1 - c;
    const float pivmin = s_pivmin;
    float lo = s_lo, hi = s_hi;
    for (int it = 0; it < 8; ++it) {
        const float x = lo + (hi - lo) * (float)(t + 1) / (float)(kPairThreads + 1);
        const int below = sturm_count_poly(d, e2, p, x) <= target;
        const int nle = __syncthreads_count(below);
        const float xl = lo + (hi - lo) * (float)nle / (float)(kPairThreads + 1);
        const float xh = lo + (hi - lo) * (float)(nle + 1) / (float)(kPairThreads + 1);
        const float nlo = nle > 0 ? xl : lo;
        const float nhi = nle < kPairThreads ? xh : hi;
        if (!(nlo < nhi) || (nhi - nlo) >= (hi - lo)) break;
        lo = nlo;
        hi = nhi;
        if (hi - lo <= 2.f * FLT_EPSILON * fmaxf(fabsf(lo), fabsf(hi))) break;
    }
    const float lam = 0.5f * (lo + hi);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();   // every thread's reflector copies are visible
    // Warps 1..7 build the compact WY factors of the back-transformation
    // while warp 0 computes the eigenvector of T: block b of reflectors
    // k0 = 8 b .. k0 + 7 (k < p - 2; the rest are identities) gives
    // H_k0 ... H_k0+7 = I - V T V^T with T upper triangular, T_qq = tau_q and
    // column q above the diagonal -tau_q T[0:q, 0:q] (V[:, 0:q]^T v_q).
    __shared__ __align__(16) float Tm[kMaxWyBlocks][8][8];
    const int nblk = (p - 2 + 7) / 8;
    if (wid != 0) {
        for (int blk = wid - 1; blk < nblk; blk += kPairThreads / 32 - 1) {
            const int k0 = 8 * blk;
            float vq[8][NB];
#pragma unroll
            for (int q = 0; q < 8; ++q)
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const int i = lane + 32 * b;
                    vq[q][b] = (k0 + q < p - 2 && i < p) ? refl[(k0 + q) * p + i] : 0.f;
                }
            float W[8][8];   // W[a][q] = v_a . v_q, a < q
#pragma unroll
            for (int q = 1; q < 8; ++q)
#pragma unroll
                for (int a = 0; a < q; ++a) {
                    float d0 = 0.f;
#pragma unroll
                    for (int b = 0; b < NB; ++b) d0 = fmaf(vq[a][b], vq[q][b], d0);
                    W[a][q] = d0;
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int q = 1; q < 8; ++q)
#pragma unroll
                    for (int a = 0; a < q; ++a) W[a][q] += __shfl_xor_sync(0xffffffffu, W[a][q], o);
            float T[8][8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float tq = k0 + q < p - 2 ? tau[k0 + q] : 0.f;
#pragma unroll
                for (int a = 0; a < 8; ++a) T[a][q] = 0.f;
                T[q][q] = tq;
#pragma unroll
                for (int a = 0; a < q; ++a) {
                    float acc = 0.f;
#pragma unroll
                    for (int m = a; m < q; ++m) acc = fmaf(T[a][m], W[m][q], acc);
                    T[a][q] = -tq * acc;
                }
            }
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (lane == ((8 * a + q) & 31)) Tm[blk][a][q] = T[a][q];
        }
        asm volatile("bar.arrive 2, %0;" ::"n"(kPairThreads) : "memory");
        return;
    }
    // twisted factorisation at lam: L D L^T from the top in lane 0, U D U^T
    // from the bottom in lane 1, in lockstep
    if (lane < 2) {
        const bool fwd = lane == 0;
        float* D = fwd ? Dp : Dm;
        int i = fwd ? 0 : p - 1;
        const int step = fwd ? 1 : -1;
        float qv = d[i] - lam;
        if (fabsf(qv) < pivmin) qv = -pivmin;
        D[i] = qv;
#pragma unroll 4
        for (int s2 = 1; s2 < p; ++s2) {
            i += step;
            const float ee = e2[fwd ? i - 1 : i];
            qv = (d[i] - lam) - __fdividef(ee, qv);
            if (fabsf(qv) < pivmin) qv = -pivmin;
            D[i] = qv;
        }
    }
    __syncwarp();
    // twist index: minimum |gamma_i|, gamma_i = Dp_i + Dm_i - (d_i - lam)
    float best = FLT_MAX;
    int bi = 0;
    for (int i = lane; i < p; i += 32) {
        const float g = fabsf(Dp[i] + Dm[i] - (d[i] - lam));
        if (g < best) { best = g; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob < best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    const int kt = bi;
    // z from the twist outwards: the ratios z_i / z_{i+1} = -e_i / Dp_i above
    // the twist and z_i / z_{i-1} = -e_{i-1} / Dm_i below it, all lanes at
    // once (into e2, free now), then the running products, lane 0 upwards
    // (rows kt-1..0) and lane 1 downwards (rows kt+1..p-1) in lockstep
    for (int i = lane; i < p; i += 32)
        e2[i] = i < kt ? -__fdividef(e[i], Dp[i]) : (i > kt ? -__fdividef(e[i - 1], Dm[i]) : 1.0f);
    __syncwarp();
    if (lane < 2) {
        const bool up = lane == 0;
        const int len = up ? kt : p - 1 - kt;
        const int steps = max(kt, p - 1 - kt);
        if (up) z[kt] = 1.0f;
        int i = kt;
        float zz = 1.0f;
#pragma unroll 8
        for (int s2 = 0; s2 < steps; ++s2) {
            if (s2 < len) {
                i += up ? -1 : 1;
                zz *= e2[i];
                z[i] = zz;
            }
        }
    }
    __syncwarp();
    // back-transformation x = H_0 .. H_{p-3} z with the vector in registers,
    // block by block from the last: x <- x - V (T (V^T x))
    float x[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int i = lane + 32 * b;
        x[b] = i < p ? z[i] : 0.f;
    }
    asm volatile("bar.sync 2, %0;" ::"n"(kPairThreads) : "memory");   // the T blocks
    for (int blk = nblk - 1; blk >= 0; --blk) {
        const int k0 = 8 * blk;
        float vq[8][NB];
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int i = lane + 32 * b;
                vq[q][b] = (k0 + q < p - 2 && i < p) ? refl[(k0 + q) * p + i] : 0.f;
            }
        float y[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            y[q] = 0.f;
#pragma unroll
            for (int b = 0; b < NB; ++b) y[q] = fmaf(vq[q][b], x[b], y[q]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 8; ++q) y[q] += __shfl_xor_sync(0xffffffffu, y[q], o);
        float u[8];
#pragma unroll
        for (int a2 = 0; a2 < 8; ++a2) {
            float acc = 0.f;
#pragma unroll
            for (int q = a2; q < 8; ++q) acc = fmaf(Tm[blk][a2][q], y[q], acc);
            u[a2] = acc;
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            float xv = x[b];
#pragma unroll
            for (int q = 0; q < 8; ++q) xv = fmaf(-u[q], vq[q][b], xv);
            x[b] = xv;
        }
    }
    // normalised (the twisted vector has z[kt] = 1)
    float ss = 0.f;
#pragma unroll
    for (int b = 0; b < NB; ++b) ss = fmaf(x[b], x[b], ss);
    ss = warp_sum(ss);
    const float inv = ss > 0.f ? rsqrtf(ss) : 0.f;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int i = lane + 32 * b;
        if (i < p) G.X[(size_t)c * p + i] = x[b] * inv;
    }
    if (lane == 0) G.lam[c] = lam;
}

// --------------------------------------------------------------------------
// 2b. All r eigenpairs of a window in one block (the batched window form,
// one block per window): the eigenvalues by multisection, eight points per
// eigenvalue and round (four eigenvalues per warp; with 33 points per
// eigenvalue and four Sturm chains interleaved per lane the multisection took
// 711k of the kernel's ~1M cycles per window), then warp w takes eigenpairs
// c = w, w + 8, ... (at most four): the eigenvectors of T by the twisted
// factorisation as in eig_pair_kernel, and the back-transformation by the
// same compact-WY blocks, built once per window by all warps and applied by
// each warp to its vectors together (one load of a reflector block for all
// of them). The reflectors are read through L2.
// --------------------------------------------------------------------------
constexpr int kAllThreads = 256, kAllWarps = kAllThreads / 32, kMaxPerWarp = 4;

size_t eig_pairs_all_bytes(int p, int r) {
    return ((size_t)4 * p + (size_t)3 * kAllWarps * p + (size_t)r * p) * sizeof(float);
}

#ifndef HYDE_EIG_ALL_MINB
#define HYDE_EIG_ALL_MINB 2
#endif
template <int NB>
__global__ void __launch_bounds__(kAllThreads, HYDE_EIG_ALL_MINB)
eig_pairs_all_kernel(EigWs G, int p, int r, int* status, long long wst) {
    pdl_wait();
    pdl_trigger();
    G = eig_ws_window(G, blockIdx.x * wst);
    if (status) status += blockIdx.x;
    extern __shared__ float sm[];
    float* d = sm;
    float* e = d + p;
    float* e2 = e + p;
    float* tau = e2 + p;
    float* wsc = tau + p;                       // per warp: Dp, Dm, ratios (p each)
    float* Z = wsc + 3 * kAllWarps * p;         // [r][p] eigenvectors of T
    __shared__ float s_lo, s_hi, s_pivmin;
    __shared__ __align__(16) float Tm[kMaxWyBlocks][8][8];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int i = t; i < p; i += kAllThreads) {
        const float di = G.d[i], ei = G.e[i];
        d[i] = di;
        e[i] = ei;
        e2[i] = ei * ei;
        tau[i] = G.tau[i];
        if (!isfinite(di) || !isfinite(ei)) set_status(status, HYDE_ERR_NUMERIC);
    }
    __syncthreads();
    if (wid == 0) {
        float lo = FLT_MAX, hi = -FLT_MAX, emax = 0.f;
        for (int i = lane; i < p; i += 32) {
            const float rad = fabsf(e[i]) + (i > 0 ? fabsf(e[i - 1]) : 0.f);
            lo = fminf(lo, d[i] - rad);
            hi = fmaxf(hi, d[i] + rad);
            emax = fmaxf(emax, e2[i]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        }
        if (lane == 0) {
            const float w = hi - lo;
            s_lo = lo - 1e-6f * fmaxf(w, 1e-30f);
            s_hi = hi + 1e-6f * fmaxf(w, 1e-30f);
            s_pivmin = FLT_MIN * fmaxf(1.f, emax);
        }
    }
    __syncthreads();
    const float pivmin = s_pivmin;
    // multisection: eigenvalue slot c = 4 wid + (lane / 8) (the (p - c)-th
    // smallest) is searched by the eight lanes of its octet, lane j counting
    // at point j + 1 of 9 of the slot's interval; each round keeps the one of
    // nine sub-intervals that holds it. One Sturm count per lane and round.
    __shared__ float s_lam[kAllWarps * 4];
    {
        const int c = 4 * wid + (lane >> 3), j = lane & 7;
        const int target = p - 1 - c;
        float lo = s_lo, hi = s_hi;
        bool act = c < r;
        for (int it = 0; it < 48; ++it) {   // 48 rounds of 9x exceed float resolution
            const float x = lo + (hi - lo) * (float)(j + 1) / 9.f;
            const int cnt = sturm_count_poly(d, e2, p, x);
            const unsigned bal = __ballot_sync(0xffffffffu, cnt <= target);
            const int nle = __popc((bal >> (lane & ~7)) & 0xffu);
            if (act) {
                const float xl = lo + (hi - lo) * (float)nle / 9.f;
                const float xh = lo + (hi - lo) * (float)(nle + 1) / 9.f;
                const float nlo = nle > 0 ? xl : lo;
                const float nhi = nle < 8 ? xh : hi;
                if (!(nlo < nhi) || (nhi - nlo) >= (hi - lo)) {
                    act = false;
                } else {
                    lo = nlo;
                    hi = nhi;
                    if (hi - lo <= 2.f * FLT_EPSILON * fmaxf(fabsf(lo), fabsf(hi))) act = false;
                }
            }
            if (!__any_sync(0xffffffffu, act)) break;
        }
        if (j == 0) s_lam[c] = 0.5f * (lo + hi);
    }
    __syncthreads();
    // eigenvectors of T by the twisted factorisation, one at a time per warp
    float* Dp = wsc + 3 * wid * p;
    float* Dm = Dp + p;
    float* rat = Dm + p;
#pragma unroll
    for (int k = 0; k < kMaxPerWarp; ++k) {
        const int c = wid + kAllWarps * k;
        if (c >= r) continue;   // warp-uniform
        const float lam = s_lam[c];
        if (lane < 2) {
            const bool fwd = lane == 0;
            float* D = fwd ? Dp : Dm;
            int i = fwd ? 0 : p - 1;
            const int step = fwd ? 1 : -1;
            float qv = d[i] - lam;
            if (fabsf(qv) < pivmin) qv = -pivmin;
            D[i] = qv;
            for (int s2 = 1; s2 < p; ++s2) {
                i += step;
                const float ee = e2[fwd ? i - 1 : i];
                qv = (d[i] - lam) - __fdividef(ee, qv);
                if (fabsf(qv) < pivmin) qv = -pivmin;
                D[i] = qv;
            }
        }
        __syncwarp();
        float best = FLT_MAX;
        int bi = 0;
        for (int i = lane; i < p; i += 32) {
            const float g = fabsf(Dp[i] + Dm[i] - (d[i] - lam));
            if (g < best) { best = g; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob < best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        const int kt = bi;
        for (int i = lane; i < p; i += 32)
            rat[i] = i < kt ? -__fdividef(e[i], Dp[i]) : (i > kt ? -__fdividef(e[i - 1], Dm[i]) : 1.0f);
        __syncwarp();
        float* z = Z + (size_t)c * p;
        if (lane < 2) {
            const bool up = lane == 0;
            const int len = up ? kt : p - 1 - kt;
            if (up) z[kt] = 1.0f;
            int i = kt;
            float zz = 1.0f;
            for (int s2 = 0; s2 < len; ++s2) {
                i += up ? -1 : 1;
                zz *= rat[i];
                z[i] = zz;
            }
        }
        __syncwarp();
    }
    // compact WY factors of the reflector blocks, by all warps
    const int nblk = (p - 2 + 7) / 8;
    for (int blk = wid; blk < nblk; blk += kAllWarps) {
        const int k0 = 8 * blk;
        float vq[8][NB];
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int i = lane + 32 * b;
                vq[q][b] = (k0 + q < p - 2 && i < p) ? __ldg(G.refl + (k0 + q) * p + i) : 0.f;
            }
        float W[8][8];
#pragma unroll
        for (int q = 1; q < 8; ++q)
#pragma unroll
            for (int a = 0; a < q; ++a) {
                float d0 = 0.f;
#pragma unroll
                for (int b = 0; b < NB; ++b) d0 = fmaf(vq[a][b], vq[q][b], d0);
                W[a][q] = d0;
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 1; q < 8; ++q)
#pragma unroll
                for (int a = 0; a < q; ++a) W[a][q] += __shfl_xor_sync(0xffffffffu, W[a][q], o);
        float T[8][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float tq = k0 + q < p - 2 ? tau[k0 + q] : 0.f;
#pragma unroll
            for (int a = 0; a < 8; ++a) T[a][q] = 0.f;
            T[q][q] = tq;
#pragma unroll
            for (int a = 0; a < q; ++a) {
                float acc = 0.f;
#pragma unroll
                for (int m = a; m < q; ++m) acc = fmaf(T[a][m], W[m][q], acc);
                T[a][q] = -tq * acc;
            }
        }
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (lane == ((8 * a + q) & 31)) Tm[blk][a][q] = T[a][q];
    }
    __syncthreads();   // every T block, every z
    // back-transformation of the warp's vectors: x <- x - V (T (V^T x))
    const int nv = r > wid ? (r - wid + kAllWarps - 1) / kAllWarps : 0;
    float x[kMaxPerWarp][NB];
#pragma unroll
    for (int k = 0; k < kMaxPerWarp; ++k)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int i = lane + 32 * b;
            x[k][b] = (k < nv && i < p) ? Z[(size_t)(wid + kAllWarps * k) * p + i] : 0.f;
        }
    if (nv > 0) {
        for (int blk = nblk - 1; blk >= 0; --blk) {
            const int k0 = 8 * blk;
            float vq[8][NB];
#pragma unroll
            for (int q = 0; q < 8; ++q)
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const int i = lane + 32 * b;
                    vq[q][b] = (k0 + q < p - 2 && i < p) ? __ldg(G.refl + (k0 + q) * p + i) : 0.f;
                }
#pragma unroll
            for (int k = 0; k < kMaxPerWarp; ++k) {
                if (k >= nv) break;   // warp-uniform
                float y[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    y[q] = 0.f;
#pragma unroll
                    for (int b = 0; b < NB; ++b) y[q] = fmaf(vq[q][b], x[k][b], y[q]);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int q = 0; q < 8; ++q) y[q] += __shfl_xor_sync(0xffffffffu, y[q], o);
                float u[8];
#pragma unroll
                for (int a2 = 0; a2 < 8; ++a2) {
                    float acc = 0.f;
#pragma unroll
                    for (int q = a2; q < 8; ++q) acc = fmaf(Tm[blk][a2][q], y[q], acc);
                    u[a2] = acc;
                }
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    float xv = x[k][b];
#pragma unroll
                    for (int q = 0; q < 8; ++q) xv = fmaf(-u[q], vq[q][b], xv);
                    x[k][b] = xv;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kMaxPerWarp; ++k) {
        if (k >= nv) break;
        const int c = wid + kAllWarps * k;
        float ss = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) ss = fmaf(x[k][b], x[k][b], ss);
        ss = warp_sum(ss);
        const float inv = ss > 0.f ? rsqrtf(ss) : 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int i = lane + 32 * b;
            if (i < p) G.X[(size_t)c * p + i] = x[k][b] * inv;
        }
        if (lane == 0) G.lam[c] = s_lam[c];
    }
}

// --------------------------------------------------------------------------
// 3. Orthonormalisation of the r vectors (rows of X, descending eigenvalue)
// by Cholesky QR, twice: G = X X^T, G = L L^T, X <- L^-1 X. In exact
// arithmetic this is Gram-Schmidt in the same order (row i becomes a
// combination of rows 0..i); the second pass removes the first pass's
// rounding (vectors of well-separated eigenvalues are orthogonal to ~u
// already, those of close ones to ~u / gap). A pivot that is not positive
// (two vectors equal to rounding) is floored at 1e-12 G_kk. Then the sign
// rule and the write-out in double. One thread per entry of G (the rows of
// X padded to an odd stride, so that one column's entries sit in distinct
// banks), a right-looking Cholesky factorisation in warp 0 (lane i updates
// row i), and the triangular solve with one thread per column of X. The
// loops stay rolled: the kernel runs once per call, and straight-line code
// of this size would be fetched rather than executed.
// --------------------------------------------------------------------------
constexpr int kOrthThreads = 512;

__global__ void __launch_bounds__(kOrthThreads, 1)
eig_orth_kernel(EigWs G, int p, int r, double* __restrict__ evals, double* __restrict__ V,
                long long wst) {
    pdl_wait();
    pdl_trigger();
    if (blockIdx.y) {
        const int wi = blockIdx.y;
        G = eig_ws_window(G, wi * wst);
        evals += (long long)wi * r;
        V += (long long)wi * p * r;
    }
    extern __shared__ float sm[];
    const int ldx = p | 1;
    float* X = sm;                // [r][ldx]
    __shared__ float Gm[32][33];  // X X^T (lower triangle), then L; 1 / L_kk in Dinv
    __shared__ float Dinv[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int i = t; i < r * p; i += kOrthThreads) {
        const int c = i / p, e = i - c * p;
        X[c * ldx + e] = G.X[i];
    }
    __syncthreads();
    const int npair = r * (r + 1) / 2;
    for (int pass = 0; pass < 2; ++pass) {
        // G = X X^T, lower triangle: thread q takes entry (i, j), j <= i
        for (int q = t; q < npair; q += kOrthThreads) {
            int i = 0, rem = q;
            while (rem > i) { rem -= i + 1; ++i; }
            const int j = rem;
            const float* xi = X + i * ldx;
            const float* xj = X + j * ldx;
            float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
            int e = 0;
            for (; e + 4 <= p; e += 4) {
                d0 = fmaf(xi[e], xj[e], d0);
                d1 = fmaf(xi[e + 1], xj[e + 1], d1);
                d2 = fmaf(xi[e + 2], xj[e + 2], d2);
                d3 = fmaf(xi[e + 3], xj[e + 3], d3);
            }
            for (; e < p; ++e) d0 = fmaf(xi[e], xj[e], d0);
            Gm[i][j] = (d0 + d1) + (d2 + d3);
        }
        __syncthreads();
        // right-looking Cholesky in warp 0: step k scales column k and lane
        // i > k subtracts L_ik L_jk from row i, columns k < j <= i
        if (wid == 0) {
            const float gdiag = lane < r ? Gm[lane][lane] : 0.f;
            for (int k = 0; k < r; ++k) {
                const float v = Gm[k][k];
                const float floor_ = 1e-12f * __shfl_sync(0xffffffffu, gdiag, k);
                const float lkk = sqrtf(v > floor_ ? v : (floor_ > 0.f ? floor_ : 1e-30f));
                const float inv = 1.0f / lkk;
                __syncwarp();
                float l = 0.f;
                if (lane > k && lane < r) {
                    l = Gm[lane][k] * inv;
                    Gm[lane][k] = l;
                }
                if (lane == k) { Gm[k][k] = lkk; Dinv[k] = inv; }
                __syncwarp();
                if (lane > k && lane < r)
                    for (int j = k + 1; j <= lane; ++j) Gm[lane][j] = fmaf(-l, Gm[j][k], Gm[lane][j]);
                __syncwarp();
            }
        }
        __syncthreads();
        // X <- L^-1 X: thread e solves column e (forward substitution)
        for (int e = t; e < p; e += kOrthThreads) {
            for (int i = 0; i < r; ++i) {
                float v = X[i * ldx + e];
                for (int m = 0; m < i; ++m) v = fmaf(-Gm[i][m], X[m * ldx + e], v);
                X[i * ldx + e] = v * Dinv[i];
            }
        }
        __syncthreads();
    }
    // sign rule (largest-magnitude entry positive; first such index), one
    // warp per vector
    const float scale = G.scale[0];
    for (int c = wid; c < r; c += kOrthThreads / 32) {
        const float* xc = X + c * ldx;
        float best = -1.f;
        int bi = 0;
        for (int i = lane; i < p; i += 32)
            if (fabsf(xc[i]) > best) { best = fabsf(xc[i]); bi = i; }
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        const float sg = xc[bi] < 0.f ? -1.f : 1.f;
        for (int i = lane; i < p; i += 32) V[(size_t)i * r + c] = (double)(sg * xc[i]);
        if (lane == 0) evals[c] = (double)(G.lam[c] / scale);
    }
}

size_t eig_tridiag_bytes(int p) { return ((size_t)p * (p + 1) + 6 * (size_t)p) * sizeof(float); }
size_t eig_pair_bytes(int p) { return ((size_t)8 * p + (size_t)(p - 2 > 0 ? p - 2 : 0) * p) * sizeof(float); }

}  // namespace

size_t eig_ws_bytes(int p, int r) {
    return ((size_t)p * p + 3 * (size_t)p + 4 + 32 + (size_t)r * p) * sizeof(float) + 16;
}

// The tridiagonalisation: the register form for p <= 32 kRegMaxNB, the
// shared-memory form above.
template <int NB>
hyde_status launch_tridiag(const double* A, const double* wsig, int p, EigWs G, int* status,
                           int n_win, long long wst, cudaStream_t s) {
    if constexpr (NB <= kRegMaxNB) {
        const size_t sr = eig_tridiag_reg_bytes(p);
        if (ensure_smem_limit((const void*)eig_tridiag_reg_kernel<NB>, (int)sr) != cudaSuccess)
            return HYDE_ERR_SHAPE;
        launch_pdl(eig_tridiag_reg_kernel<NB>, dim3(1, n_win), kRegThreads, sr, s, A, wsig, p, G,
                   status, wst);
    } else {
        const size_t st = eig_tridiag_bytes(p);
        if (ensure_smem_limit((const void*)eig_tridiag_kernel<NB, kEigWarps>, (int)st) !=
            cudaSuccess)
            return HYDE_ERR_SHAPE;
        // only the kEigWarps sweep warps work after the load: many windows at
        // once launch just those, so that the block leaves half the SM's
        // registers to other kernels' blocks
        launch_pdl(eig_tridiag_kernel<NB, kEigWarps>, dim3(1, n_win), n_win > 1 ? 32 * kEigWarps : kLA,
                   st, s, A, wsig, p, G, status, wst);
    }
    return HYDE_OK;
}

size_t eig_smem_bytes(int p, int r) {
    const size_t a0 = eig_tridiag_bytes(p), a1 = eig_tridiag_reg_bytes(p);
    const size_t a = a0 > a1 ? a0 : a1, b = eig_pair_bytes(p), c = (size_t)r * (p | 1) * sizeof(float);
    return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

// n_win windows (block row y = window): window w reads A + w p^2, wsig + w p,
// the workspace at ws + w ws_stride bytes and writes evals + w r, V + w p r,
// status + w.
static hyde_status eig_top(const double* A, const double* wsig, int p, int r, double* evals,
                           double* V, void* ws, size_t ws_stride, int* status, int n_win,
                           cudaStream_t s) {
    if (r > 32 || r < 1 || r > p || p > 256 || p < 2 || !ws || n_win < 1 || n_win > 65535)
        return HYDE_ERR_SHAPE;
    if (eig_smem_bytes(p, r) > 227 * 1024) return HYDE_ERR_SHAPE;
    if (n_win > 1 && (ws_stride % 16) != 0) return HYDE_ERR_SHAPE;
    const long long wst = (long long)(ws_stride / sizeof(float));
    const EigWs G = eig_ws_carve(reinterpret_cast<float*>(ws), p);
    const size_t sp = eig_pair_bytes(p), so = (size_t)r * (p | 1) * sizeof(float);
    const int NB = (p + 31) / 32;
    switch (NB) {
#define HYDE_EIG(NBV)                                                                              \
    case NBV:                                                                                      \
        if (launch_tridiag<NBV>(A, wsig, p, G, status, n_win, wst, s) != HYDE_OK)                 \
            return HYDE_ERR_SHAPE;                                                                 \
        if (n_win == 1) {                                                                          \
            if (ensure_smem_limit((const void*)eig_pair_kernel<NBV>, (int)sp) != cudaSuccess)      \
                return HYDE_ERR_SHAPE;                                                             \
            launch_pdl(eig_pair_kernel<NBV>, dim3(r, 1), kPairThreads, sp, s, G, p, status, wst);  \
        } else {                                                                                   \
            const size_t sa = eig_pairs_all_bytes(p, r);                                           \
            if (ensure_smem_limit((const void*)eig_pairs_all_kernel<NBV>, (int)sa) != cudaSuccess) \
                return HYDE_ERR_SHAPE;                                                             \
            launch_pdl(eig_pairs_all_kernel<NBV>, n_win, kAllThreads, sa, s, G, p, r, status, wst); \
        }                                                                                          \
        break;
        HYDE_EIG(1) HYDE_EIG(2) HYDE_EIG(3) HYDE_EIG(4)
        HYDE_EIG(5) HYDE_EIG(6) HYDE_EIG(7) HYDE_EIG(8)
#undef HYDE_EIG
        default: return HYDE_ERR_SHAPE;
    }
    if (ensure_smem_limit((const void*)eig_orth_kernel, (int)so) != cudaSuccess)
        return HYDE_ERR_SHAPE;
    launch_pdl(eig_orth_kernel, dim3(1, n_win), kOrthThreads, so, s, G, p, r, evals, V, wst);
    return cuda_status(cudaGetLastError());
}

hyde_status launch_eig_top(const double* A, const double* wsig, int p, int r, double* evals,
                           double* V, void* ws, int* status, cudaStream_t s) {
    return eig_top(A, wsig, p, r, evals, V, ws, 0, status, 1, s);
}

hyde_status launch_eig_top_batched(const double* A, const double* wsig, int p, int r,
                                   double* evals, double* V, void* ws, size_t ws_stride,
                                   int* status, int n_win, cudaStream_t s) {
    return eig_top(A, wsig, p, r, evals, V, ws, ws_stride, status, n_win, s);
}

}  // namespace hyde

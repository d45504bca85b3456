// Leading r eigenpairs of the whitened Gram matrix, the spectral subspace of
// the low-rank model (arXiv 2204.06979, Sec. 2.1 "low-rank"): three kernels.
//
//  1. eig_tridiag_kernel (one block, 1024 threads): the matrix, optionally
//     whitened on load (A_ij / (wsig_i wsig_j)) and scaled by 1 / max |diag|,
//     is reduced to tridiagonal form T = Q^T A Q by Householder reflectors in
//     float, with the matrix in shared memory. Writes T (d, e), the
//     reflectors as explicit vectors (row k = v_k), tau_k and the products
//     v_{k-1} . v_k to the workspace.
//  2. eig_pair_kernel (one block of 256 threads per wanted eigenpair, r
//     blocks on r SMs): the eigenvalue by multisection (every thread counts
//     the eigenvalues of T below one of 256 points, Sturm sequence; a few
//     rounds reach float resolution), the eigenvector of T from a twisted
//     factorisation at it, and its back-transformation by the reflectors
//     (read into shared memory), one warp.
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

// Workspace of the three kernels (floats): reflectors [p][p] (row k = v_k,
// k < p - 2), tau, v_{k-1}.v_k, d, e (p each), the scale, the eigenvalues of
// the scaled T (32), and the back-transformed vectors X [r][p].
struct EigWs {
    float* refl;
    float* tau;
    float* cpair;
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
    w.cpair = q; q += p;
    w.d = q;     q += p;
    w.e = q;     q += p;
    w.scale = q; q += 4;
    w.lam = q;   q += 32;
    w.X = q;
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

__device__ __forceinline__ int sturm_count(const float* d, const float* e2, int p,
                                           float x, float pivmin) {
    float q = d[0] - x;
    int c = q < 0.f;
    // unrolled so that the shared-memory loads of later steps issue ahead of
    // the dependent chain through q
#pragma unroll 8
    for (int i = 1; i < p; ++i) {
        if (fabsf(q) < pivmin) q = -pivmin;
        q = (d[i] - x) - __fdividef(e2[i - 1], q);
        c += q < 0.f;
    }
    return c;
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
                   EigWs G, int* status) {
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
    // write-out: T, the reflectors as rows (column k of A, already explicit),
    // tau, v_{k-1}.v_k and the scale
    for (int k = wid; k < p - 2; k += 32)
        for (int i = lane; i < p; i += 32) G.refl[(size_t)k * p + i] = A[i * lda + k];
    for (int i = t; i < p; i += blockDim.x) {
        G.d[i] = dv[i];
        G.e[i] = ev[i];
        G.tau[i] = tauv[i];
        G.cpair[i] = (i >= 1 && i <= p - 3) ? cpair[i] : 0.f;
    }
    if (t == 0) G.scale[0] = scale;
}

// --------------------------------------------------------------------------
// 2. One eigenpair per block: multisection, twisted factorisation and
// back-transformation of eigenpair c (c = 0: the largest eigenvalue).
// --------------------------------------------------------------------------
template <int NB>
__global__ void __launch_bounds__(kPairThreads)
eig_pair_kernel(EigWs G, int p, int* status) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float sm[];
    float* d = sm;
    float* e = d + p;
    float* e2 = e + p;
    float* tau = e2 + p;
    float* cpair = tau + p;
    float* Dp = cpair + p;
    float* Dm = Dp + p;
    float* z = Dm + p;
    float* refl = z + p;          // [p - 2][p]
    __shared__ float s_lo, s_hi, s_pivmin;
    const int c = blockIdx.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int i = t; i < p; i += kPairThreads) {
        const float di = G.d[i], ei = G.e[i];
        d[i] = di;
        e[i] = ei;
        e2[i] = ei * ei;
        tau[i] = G.tau[i];
        cpair[i] = G.cpair[i];
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
        const int below = sturm_count(d, e2, p, x, pivmin) <= target;
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
    if (wid != 0) return;
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
    // z from the twist outwards: lane 0 upwards (rows kt-1..0), lane 1
    // downwards (rows kt+1..p-1), in lockstep
    if (lane < 2) {
        const bool up = lane == 0;
        const int len = up ? kt : p - 1 - kt;
        const int steps = max(kt, p - 1 - kt);
        if (up) z[kt] = 1.0f;
        int i = kt;
        float zz = 1.0f;
#pragma unroll 4
        for (int s2 = 0; s2 < steps; ++s2) {
            if (s2 < len) {
                i += up ? -1 : 1;
                const float num = e[up ? i : i - 1];
                const float den = up ? Dp[i] : Dm[i];
                zz = -__fdividef(num, den) * zz;
                z[i] = zz;
            }
        }
    }
    __syncwarp();
    // back-transformation x = H_0 .. H_{p-3} z with the vector in registers;
    // reflectors in pairs (k, k-1): both dot products in one pass,
    // H_{k-1} H_k x = x - d_a v_k - d_b v_{k-1} with d_a = tau_k v_k.x and
    // d_b = tau_{k-1} (v_{k-1}.x - d_a v_{k-1}.v_k)
    float x[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int i = lane + 32 * b;
        x[b] = i < p ? z[i] : 0.f;
    }
    auto load_v = [&](int k, float (&cv)[NB]) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int i = lane + 32 * b;
            cv[b] = i < p ? refl[k * p + i] : 0.f;
        }
    };
    int k = p - 3;
    for (; k >= 1; k -= 2) {
        float va[NB], vb[NB];
        load_v(k, va);
        load_v(k - 1, vb);
        const float ta = tau[k], tb = tau[k - 1], cab = cpair[k];
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
        load_v(0, v0);
        float s0 = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) s0 = fmaf(v0[b], x[b], s0);
        const float d0 = tau[0] * warp_sum(s0);
#pragma unroll
        for (int b = 0; b < NB; ++b) x[b] = fmaf(-d0, v0[b], x[b]);
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
// 3. Orthonormalisation of the r vectors (rows of X, descending eigenvalue)
// by Cholesky QR, twice: G = X X^T, G = L L^T, X <- L^-1 X. In exact
// arithmetic this is Gram-Schmidt in the same order (row i becomes a
// combination of rows 0..i); the second pass removes the first pass's
// rounding (vectors of well-separated eigenvalues are orthogonal to ~u
// already, those of close ones to ~u / gap). A pivot that is not positive
// (two vectors equal to rounding) is floored at 1e-12 G_kk. Then the sign rule and
// the write-out in double.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(kLA, 1)
eig_orth_kernel(EigWs G, int p, int r, double* __restrict__ evals, double* __restrict__ V) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float sm[];
    float* X = sm;                // [r][p]
    __shared__ float Gm[32][33];  // X X^T, then L (lower triangle)
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    constexpr int nw = kLA / 32;
    for (int i = t; i < r * p; i += kLA) X[i] = G.X[i];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        // upper triangle of X X^T, one warp per entry
        for (int e = wid; e < r * r; e += nw) {
            const int i = e / r, j = e - i * r;
            if (j < i) continue;
            const float* xi = X + i * p;
            const float* xj = X + j * p;
            float dt = 0.f;
            for (int k = lane; k < p; k += 32) dt = fmaf(xi[k], xj[k], dt);
            dt = warp_sum(dt);
            if (lane == 0) Gm[i][j] = dt;
        }
        __syncthreads();
        // Cholesky by warp 0: column k at step k, lane i holds row i
        if (wid == 0) {
            for (int k = 0; k < r; ++k) {
                float lkk = 0.f;
                if (lane == k) {
                    float v = Gm[k][k];
                    for (int m = 0; m < k; ++m) v = fmaf(-Gm[k][m], Gm[k][m], v);
                    const float floor_ = 1e-12f * Gm[k][k];
                    lkk = sqrtf(v > floor_ ? v : (floor_ > 0.f ? floor_ : 1e-30f));
                    Gm[k][k] = lkk;
                }
                lkk = __shfl_sync(0xffffffffu, lkk, k);
                if (lane > k && lane < r) {
                    float v = Gm[k][lane];                       // G[k][i], i = lane
                    for (int m = 0; m < k; ++m) v = fmaf(-Gm[lane][m], Gm[k][m], v);
                    Gm[lane][k] = v / lkk;                       // L[i][k]
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // X <- L^-1 X, one column of X per thread (forward substitution; the
        // solved entries are read back from shared memory)
        for (int e = t; e < p; e += kLA) {
            for (int i = 0; i < r; ++i) {
                float v = X[i * p + e];
                for (int m = 0; m < i; ++m) v = fmaf(-Gm[i][m], X[m * p + e], v);
                X[i * p + e] = v / Gm[i][i];
            }
        }
        __syncthreads();
    }
    // sign rule (largest-magnitude entry positive; first such index), one
    // warp per vector
    const float scale = G.scale[0];
    for (int c = wid; c < r; c += nw) {
        const float* xc = X + c * p;
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

size_t eig_tridiag_bytes(int p) { return ((size_t)p * (p + 1) + 7 * (size_t)p + 64) * sizeof(float); }
size_t eig_pair_bytes(int p) { return ((size_t)8 * p + (size_t)(p - 2 > 0 ? p - 2 : 0) * p) * sizeof(float); }

}  // namespace

size_t eig_ws_bytes(int p, int r) {
    return ((size_t)p * p + 4 * (size_t)p + 4 + 32 + (size_t)r * p) * sizeof(float) + 16;
}

size_t eig_smem_bytes(int p, int r) {
    const size_t a = eig_tridiag_bytes(p), b = eig_pair_bytes(p), c = (size_t)r * p * sizeof(float);
    return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

hyde_status launch_eig_top(const double* A, const double* wsig, int p, int r, double* evals,
                           double* V, void* ws, int* status, cudaStream_t s) {
    if (r > 32 || r < 1 || r > p || p > 256 || p < 2 || !ws) return HYDE_ERR_SHAPE;
    if (eig_smem_bytes(p, r) > 227 * 1024) return HYDE_ERR_SHAPE;
    const EigWs G = eig_ws_carve(reinterpret_cast<float*>(ws), p);
    const size_t st = eig_tridiag_bytes(p), sp = eig_pair_bytes(p), so = (size_t)r * p * sizeof(float);
    const int NB = (p + 31) / 32;
    switch (NB) {
#define HYDE_EIG(NBV)                                                                              \
    case NBV:                                                                                      \
        if (ensure_smem_limit((const void*)eig_tridiag_kernel<NBV, kEigWarps>, (int)st) !=        \
                cudaSuccess ||                                                                     \
            ensure_smem_limit((const void*)eig_pair_kernel<NBV>, (int)sp) != cudaSuccess)          \
            return HYDE_ERR_SHAPE;                                                                 \
        launch_pdl(eig_tridiag_kernel<NBV, kEigWarps>, 1, kLA, st, s, A, wsig, p, G, status);     \
        launch_pdl(eig_pair_kernel<NBV>, r, kPairThreads, sp, s, G, p, status);                   \
        break;
        HYDE_EIG(1) HYDE_EIG(2) HYDE_EIG(3) HYDE_EIG(4)
        HYDE_EIG(5) HYDE_EIG(6) HYDE_EIG(7) HYDE_EIG(8)
#undef HYDE_EIG
        default: return HYDE_ERR_SHAPE;
    }
    if (ensure_smem_limit((const void*)eig_orth_kernel, (int)so) != cudaSuccess)
        return HYDE_ERR_SHAPE;
    launch_pdl(eig_orth_kernel, 1, kLA, so, s, G, p, r, evals, V);
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

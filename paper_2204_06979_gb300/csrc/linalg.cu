// Small dense linear algebra of the HyRes path (arXiv 2204.06979, Sec. 2.1):
//
//  * noise level by multiple regression: sigma_b^2 = 1 / (n [R^-1]_bb), the
//    residual power of regressing band b on all other bands (the Schur
//    complement of the normal equations);
//  * leading eigenpairs of the whitened Gram matrix D^-1 R D^-1 (the spectral
//    subspace of the low-rank model);
//  * the float projection / back-projection weights V/sigma and V*sigma.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so the O(p^3) work is
// done in FP32 inside one thread block (the p x p matrix lives in shared
// memory) and FP64 is used where it buys accuracy cheaply: the diagonal of the
// inverse gets one Newton correction in double, spread over p blocks.
#include <float.h>

#include "hyde_internal.cuh"

namespace hyde {
namespace {

constexpr int kLA = 1024;   // threads of the single-block kernels

// --------------------------------------------------------------------------
// Noise level, part 1: Gauss-Jordan inverse (no pivoting: the matrix is SPD)
// of As = S^-1 R S^-1, S = sqrt(diag R), in float. Writes As^-1 (p x p) and
// S (double[p]).
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(kLA, 1)
noise_gj_kernel(const double* __restrict__ R, int p, float* __restrict__ Ainv,
                double* __restrict__ S, int* status) {
    extern __shared__ float sm[];
    float* A = sm;                  // p * p
    float* colk = A + p * p;        // p
    float* rowk = colk + p;         // p   (first holds 1 / S in float)
    const int t = threadIdx.x;
    const int lane0 = t & 31, wid0 = t >> 5;
    // FP64 is slow on this part: p square roots in double, the p^2 scaling in float
    for (int i = t; i < p; i += blockDim.x) {
        double d = R[(long long)i * p + i];
        if (!(d > 0.0) || !isfinite(d)) set_status(status, HYDE_ERR_NUMERIC);
        const double s = d > 0.0 ? sqrt(d) : 1.0;
        S[i] = s;
        rowk[i] = (float)(1.0 / s);
    }
    __syncthreads();
    for (int i = wid0; i < p; i += 32) {
        const float si = rowk[i];
        for (int j = lane0; j < p; j += 32)
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
        // pivots of the unit-diagonal matrix are Schur complements >= its
        // smallest eigenvalue; below ~16 ulp the float inverse is meaningless
        // (exactly collinear bands give ~1 ulp)
        if (t == 0 && !(pk > 2e-6f)) set_status(status, HYDE_ERR_NUMERIC);
        const float piv = 1.0f / pk;
        const int lane = t & 31, wid = t >> 5;
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
    extern __shared__ double xs[];   // p
    __shared__ double red[8];
    const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int i = t; i < p; i += blockDim.x)
        xs[i] = (double)Ainv[(long long)i * p + b] / (S[i] * S[b]);
    __syncthreads();
    double part = 0.0;
    for (int i = w; i < p; i += 8) {
        double u = 0.0;
        for (int j = lane; j < p; j += 32) u = fma(R[(long long)i * p + j], xs[j], u);
        u = warp_sum_d(u);
        part = fma(xs[i], u, part);   // identical in all lanes
    }
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
// optionally whitened on load: A_ij / (wsig_i wsig_j).
// 1. Householder tridiagonalisation in float (A = Q T Q^T, reflectors kept
//    below the diagonal).
// 2. Eigenvalues of T by multisection: one warp per wanted eigenvalue, each
//    lane counts eigenvalues below one of 32 points (Sturm sequence).
// 3. Eigenvectors of T from a twisted factorisation at each eigenvalue.
// 4. Classical Gram-Schmidt, twice, over the r vectors (orthogonality inside
//    clusters of close eigenvalues).
// 5. Back-transformation by the reflectors (one warp per vector).
// --------------------------------------------------------------------------
struct EigSmem {
    float* A; float* tau; float* d; float* e; float* e2; float* v; float* pv;
    float* red; float* lam; float* X; float* Dp; float* Dm; float* dots;
    int lda;
};

__device__ inline EigSmem eig_carve(float* base, int p, int r) {
    EigSmem m;
    m.lda = p + 1;
    float* q = base;
    m.A = q;   q += p * m.lda;
    m.tau = q; q += p;
    m.d = q;   q += p;
    m.e = q;   q += p;
    m.e2 = q;  q += p;
    m.v = q;   q += p;
    m.pv = q;  q += p;
    m.red = q; q += 64;
    m.lam = q; q += 32;
    m.dots = q; q += 32;
    m.X = q;   q += p * r;
    m.Dp = q;  q += p * r;
    m.Dm = q;  q += p * r;
    return m;
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

__global__ void __launch_bounds__(kLA, 1)
eig_top_kernel(const double* __restrict__ Ain, const double* __restrict__ wsig,
               int p, int r, double* __restrict__ evals, double* __restrict__ V,
               int* status) {
    extern __shared__ float sm[];
    EigSmem S = eig_carve(sm, p, r);
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int lda = S.lda;

    // ---- load (optionally whitened) matrix, scaled by 1 / max |diag|;
    // FP64 only for the p diagonal entries, the p^2 scaling in float
    __shared__ float s_scale;
    float* iw = S.v;   // 1 / wsig (float), reused as the Householder vector later
    if (t < 32) {
        double mx = 0.0;
        for (int i = lane; i < p; i += 32) {
            double a = Ain[(long long)i * p + i];
            double w = wsig ? 1.0 / wsig[i] : 1.0;
            iw[i] = (float)w;
            a *= w * w;
            if (!isfinite(a)) set_status(status, HYDE_ERR_NUMERIC);
            mx = fmax(mx, fabs(a));
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) s_scale = mx > 0.0 ? (float)(1.0 / mx) : 1.0f;
    }
    __syncthreads();
    const float scale = s_scale;
    for (int i = wid; i < p; i += 32) {
        const float si = iw[i] * scale;
        for (int j = lane; j < p; j += 32)
            S.A[i * lda + j] = (float)Ain[(long long)i * p + j] * si * iw[j];
    }
    __syncthreads();

    // ---- 1. Householder tridiagonalisation
    for (int k = 0; k + 2 < p; ++k) {
        const int m = p - k - 1;
        float* col = S.A + (k + 1) * lda + k;   // col[i * lda] = A[k+1+i][k]
        if (wid == 0) {
            float ss = 0.f;
            for (int i = 1 + lane; i < m; i += 32) { float x = col[i * lda]; ss = fmaf(x, x, ss); }
            ss = warp_sum(ss);
            const float alpha = col[0];
            __syncwarp();   // every lane has read col[] before lane 0 rewrites it
            float tau = 0.f, beta = alpha, sc = 0.f;
            if (ss > 0.f) {
                const float nrm = sqrtf(fmaf(alpha, alpha, ss));
                beta = alpha >= 0.f ? -nrm : nrm;
                tau = (beta - alpha) / beta;
                sc = 1.0f / (alpha - beta);
            }
            for (int i = lane; i < m; i += 32) {
                float vi = (i == 0) ? 1.0f : col[i * lda] * sc;
                if (ss == 0.f) vi = (i == 0) ? 1.0f : 0.f;
                S.v[i] = vi;
                col[i * lda] = vi;       // reflector kept for step 5
            }
            if (lane == 0) { S.tau[k] = tau; S.d[k] = S.A[k * lda + k]; S.e[k] = beta; }
        }
        __syncthreads();
        const float tau = S.tau[k];
        if (tau != 0.f) {
            // p = tau * A22 v, one warp per row; K partials per warp
            float kpart = 0.f;
            for (int i = wid; i < m; i += 32) {
                const float* row = S.A + (k + 1 + i) * lda + (k + 1);
                float u = 0.f;
                for (int j = lane; j < m; j += 32) u = fmaf(row[j], S.v[j], u);
                u = warp_sum(u) * tau;
                if (lane == 0) S.pv[i] = u;
                kpart = fmaf(u, S.v[i], kpart);
            }
            if (lane == 0) S.red[wid] = kpart;
            __syncthreads();
            float K = 0.f;
#pragma unroll
            for (int w = 0; w < 32; ++w) K += S.red[w];
            K *= 0.5f * tau;
            // A22 -= v w^T + w v^T, w = p - K v
            for (int i = wid; i < m; i += 32) {
                float* row = S.A + (k + 1 + i) * lda + (k + 1);
                const float vi = S.v[i], wi = fmaf(-K, vi, S.pv[i]);
                for (int j = lane; j < m; j += 32) {
                    const float vj = S.v[j], wj = fmaf(-K, vj, S.pv[j]);
                    row[j] = fmaf(-vi, wj, fmaf(-wi, vj, row[j]));
                }
            }
        }
        __syncthreads();
    }
    if (t == 0) {
        if (p >= 2) {
            S.d[p - 2] = S.A[(p - 2) * lda + (p - 2)];
            S.e[p - 2] = S.A[(p - 1) * lda + (p - 2)];
            S.tau[p - 2] = 0.f;
        }
        S.d[p - 1] = S.A[(p - 1) * lda + (p - 1)];
        S.e[p - 1] = 0.f;
    }
    __syncthreads();
    for (int i = t; i < p; i += blockDim.x) {
        S.e2[i] = S.e[i] * S.e[i];
        if (!isfinite(S.d[i]) || !isfinite(S.e[i])) set_status(status, HYDE_ERR_NUMERIC);
    }
    __syncthreads();

    // ---- Gershgorin interval and pivot guard (warp 0)
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

    // ---- 2. multisection, warp j finds the (j+1)-th largest eigenvalue
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

    // ---- 3. twisted factorisation eigenvector of T for each eigenvalue
    if (wid < r) {
        const float lam = S.lam[wid];
        float* Dp = S.Dp + wid * p;
        float* Dm = S.Dm + wid * p;
        float* z = S.X + wid * p;
        const float pm = s_pivmin;
        if (lane == 0) {
            float q = S.d[0] - lam;
            if (fabsf(q) < pm) q = -pm;
            Dp[0] = q;
            for (int i = 1; i < p; ++i) {
                q = (S.d[i] - lam) - S.e2[i - 1] / q;
                if (fabsf(q) < pm) q = -pm;
                Dp[i] = q;
            }
        } else if (lane == 1) {
            float q = S.d[p - 1] - lam;
            if (fabsf(q) < pm) q = -pm;
            Dm[p - 1] = q;
            for (int i = p - 2; i >= 0; --i) {
                q = (S.d[i] - lam) - S.e2[i] / q;
                if (fabsf(q) < pm) q = -pm;
                Dm[i] = q;
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
        if (lane == 0) {
            z[kt] = 1.0f;
            float zz = 1.0f;
            for (int i = kt - 1; i >= 0; --i) { zz = -(S.e[i] / Dp[i]) * zz; z[i] = zz; }
        } else if (lane == 1) {
            float zz = 1.0f;
            for (int i = kt + 1; i < p; ++i) { zz = -(S.e[i - 1] / Dm[i]) * zz; z[i] = zz; }
        }
        __syncwarp();
        float ss = 0.f;
        for (int i = lane; i < p; i += 32) ss = fmaf(z[i], z[i], ss);
        ss = warp_sum(ss);
        const float inv = ss > 0.f ? rsqrtf(ss) : 0.f;
        for (int i = lane; i < p; i += 32) z[i] *= inv;
    }
    __syncthreads();

    // ---- 4. classical Gram-Schmidt, two passes, in descending order
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

    // ---- 5. back-transformation x <- H_0 ... H_{p-3} x, one warp per vector
    if (wid < r) {
        float* x = S.X + wid * p;
        for (int k = p - 3; k >= 0; --k) {
            const float tau = S.tau[k];
            if (tau == 0.f) continue;
            const int m = p - k - 1;
            const float* col = S.A + (k + 1) * lda + k;
            float dt = 0.f;
            for (int i = lane; i < m; i += 32) dt = fmaf(col[i * lda], x[k + 1 + i], dt);
            dt = warp_sum(dt) * tau;
            for (int i = lane; i < m; i += 32) x[k + 1 + i] = fmaf(-dt, col[i * lda], x[k + 1 + i]);
            __syncwarp();
        }
        // sign: entry of largest magnitude positive (smallest index on ties)
        float best = -1.f;
        int bi = 0;
        for (int i = lane; i < p; i += 32) {
            float a = fabsf(x[i]);
            if (a > best) { best = a; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            float ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        const float sg = x[bi] < 0.f ? -1.f : 1.f;
        for (int i = lane; i < p; i += 32) V[(long long)i * r + wid] = (double)(sg * x[i]);
        if (lane == 0) evals[wid] = (double)S.lam[wid] / (double)scale;
    }
}

__global__ void weights_kernel(const double* __restrict__ V, const double* __restrict__ sigma,
                               int p, int r, int ldw, float* __restrict__ P,
                               float* __restrict__ Q) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p * ldw;
         e += gridDim.x * blockDim.x) {
        int b = e / ldw, i = e % ldw;
        double v = i < r ? V[(long long)b * r + i] : 0.0;
        P[e] = (float)(v / sigma[b]);
        Q[e] = (float)(v * sigma[b]);
    }
}

}  // namespace

size_t noise_ws_bytes(int p) {
    return align_up((size_t)p * p * sizeof(float), kAlign) +
           align_up((size_t)p * sizeof(double), kAlign);
}

hyde_status launch_noise_from_gram(const double* R, int p, long long n, double* sigma,
                                   void* ws, int* status, cudaStream_t s) {
    float* Ainv = reinterpret_cast<float*>(ws);
    double* Sd = reinterpret_cast<double*>(reinterpret_cast<char*>(ws) +
                                           align_up((size_t)p * p * sizeof(float), kAlign));
    size_t smem = ((size_t)p * p + 2 * p) * sizeof(float);
    if (smem > 227 * 1024) return HYDE_ERR_SHAPE;
    if (ensure_smem_limit((const void*)noise_gj_kernel, (int)smem) != cudaSuccess)
        return HYDE_ERR_CUDA;
    noise_gj_kernel<<<1, kLA, smem, s>>>(R, p, Ainv, Sd, status);
    noise_refine_kernel<<<p, 256, p * sizeof(double), s>>>(R, Ainv, Sd, p, n, sigma, status);
    return cuda_status(cudaGetLastError());
}

size_t eig_smem_bytes(int p, int r) {
    return ((size_t)p * (p + 1) + 6 * (size_t)p + 64 + 32 + 32 + 3 * (size_t)p * r) *
           sizeof(float);
}

hyde_status launch_eig_top(const double* A, const double* wsig, int p, int r,
                           double* evals, double* V, int* status, cudaStream_t s) {
    size_t smem = eig_smem_bytes(p, r);
    if (smem > 227 * 1024 || r > 32 || r < 1 || r > p) return HYDE_ERR_SHAPE;
    if (ensure_smem_limit((const void*)eig_top_kernel, (int)smem) != cudaSuccess)
        return HYDE_ERR_CUDA;
    eig_top_kernel<<<1, kLA, smem, s>>>(A, wsig, p, r, evals, V, status);
    return cuda_status(cudaGetLastError());
}

hyde_status launch_weights(const double* V, const double* sigma, int p, int r, int ldw,
                           float* P, float* Q, cudaStream_t s) {
    int tot = p * ldw;
    weights_kernel<<<(tot + 255) / 256, 256, 0, s>>>(V, sigma, p, r, ldw, P, Q);
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

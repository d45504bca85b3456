// HySime signal-subspace identification (arXiv 2204.06979, Sec. 2.1: the
// subspace step of FastHyDe, run on GPUs). Its published definition: the
// noise is each band's least-squares residual on all the other bands; with
// R_y, R_n and R_x the data, noise and signal correlation matrices, the
// subspace keeps the eigenvectors e of R_x whose inclusion lowers the
// projection error, delta = -e^T R_y e + 2 e^T R_n e < 0.
//
// Everything after the Gram matrix R = Y^T Y is p x p work. With Q = R^-1 the
// residual of band b is Y q_b / q_bb, so with D = diag(Q):
//   R_n = D^-1 Q D^-1 / n,   Y^T W = D^-1,
//   R_x = (R - 2 D^-1 + D^-1 Q D^-1) / n,   R_y = R / n,
// and no pass over the data beyond the Gram matrix is needed. Q is the float
// Gauss-Jordan inverse of the noise estimator refined in double by one Newton
// step per column; the eigensolver is the one of the HyRes path (unit
// weights); one block per candidate eigenvector forms its delta, and the
// last block ranks them.
#include <cstdint>

#include "hyde_internal.cuh"

namespace hyde {
namespace {

// R_n and R_x from R and Q (Q symmetrised), one element per thread. The
// diagonal of the inverse of a positive definite matrix is positive; a
// refined inverse whose diagonal is not (a singular or badly conditioned
// Gram matrix) is reported as HYDE_ERR_NUMERIC.
__global__ void __launch_bounds__(256)
hysime_form_kernel(const double* __restrict__ R, const double* __restrict__ Q, int p,
                   double inv_n, double* __restrict__ Rn, double* __restrict__ Rx,
                   int* status) {
    pdl_wait();
    pdl_trigger();
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)p * p) return;
    const int i = (int)(e / p), j = (int)(e - (long long)i * p);
    const double qs = 0.5 * (Q[(long long)i * p + j] + Q[(long long)j * p + i]);
    const double qii = Q[(long long)i * p + i], qjj = Q[(long long)j * p + j];
    if (i == j && !(qii > 0.0 && isfinite(qii))) set_status(status, HYDE_ERR_NUMERIC);
    const double di = 1.0 / qii, dj = 1.0 / qjj;
    const double rn = di * qs * dj;
    Rn[e] = rn * inv_n;
    Rx[e] = (R[e] - (i == j ? 2.0 * di : 0.0) + rn) * inv_n;
}

constexpr int kHsThreads = 256;

// Block c: delta_c = -e^T R e / n + 2 e^T R_n e for column c of E (double
// [p][r], row b = band b); the last block to finish ranks the candidates by
// (delta, index) and writes the kept ones (delta < 0) first.
__global__ void __launch_bounds__(kHsThreads)
hysime_delta_kernel(const double* __restrict__ R, const double* __restrict__ Rn,
                    const double* __restrict__ E, int p, int r, double inv_n,
                    double* delta, unsigned int* done, int* k_out, int* idx_out, int* status) {
    pdl_wait();
    pdl_trigger();
    __shared__ double red_y[kHsThreads / 32], red_n[kHsThreads / 32];
    __shared__ int s_last;
    const int c = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    constexpr int nw = kHsThreads / 32;
    double py = 0.0, pn = 0.0;
    for (int i = w; i < p; i += nw) {
        double ay = 0.0, an = 0.0;
        for (int j = lane; j < p; j += 32) {
            const double ej = E[(long long)j * r + c];
            ay = fma(R[(long long)i * p + j], ej, ay);
            an = fma(Rn[(long long)i * p + j], ej, an);
        }
        ay = warp_sum_d(ay);
        an = warp_sum_d(an);
        const double ei = E[(long long)i * r + c];
        py = fma(ei, ay, py);
        pn = fma(ei, an, pn);
    }
    if (lane == 0) { red_y[w] = py; red_n[w] = pn; }
    __syncthreads();
    if (t == 0) {
        double sy = 0.0, sn = 0.0;
        for (int q = 0; q < nw; ++q) { sy += red_y[q]; sn += red_n[q]; }
        const double d = -sy * inv_n + 2.0 * sn;
        if (!isfinite(d)) set_status(status, HYDE_ERR_NUMERIC);
        delta[c] = d;
    }
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = atomicAdd(done, 1u) == (unsigned)gridDim.x - 1u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    bool kept = false;
    if (t < r) {
        const double dt = __ldcg(delta + t);
        int rank = 0;
        for (int j = 0; j < r; ++j) {
            const double dj = __ldcg(delta + j);
            rank += (dj < dt) || (dj == dt && j < t);
        }
        kept = dt < 0.0;
        if (kept) idx_out[rank] = t;   // the negative deltas take ranks 0..k-1
    }
    const int k = __syncthreads_count(kept);
    for (int q = k + t; q < r; q += kHsThreads) idx_out[q] = -1;
    if (t == 0) *k_out = k;
}

struct HysimeLayout {
    GramPlan gram;
    size_t done, partials, R, noise, Q, Rn, Rx, eig, total;
};

hyde_status hysime_layout(int p, long long n, int r, HysimeLayout* L) {
    if (p < 2 || p > kMaxBandsGram || n < p) return HYDE_ERR_SHAPE;
    if (r < 1 || r > p || r > kMaxRank) return HYDE_ERR_SHAPE;
    if (eig_smem_bytes(p, r) > 227 * 1024 || noise_smem_bytes(p) > 227 * 1024)
        return HYDE_ERR_SHAPE;
    HysimeLayout l;
    hyde_status st = gram_plan(p, n, &l.gram);
    if (st != HYDE_OK) return st;
    const size_t pp = (size_t)p * p * sizeof(double);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, kAlign);
        return o;
    };
    l.done = take(sizeof(unsigned int));
    l.partials = take(l.gram.partial_bytes);
    l.R = take(pp);
    l.noise = take(noise_ws_bytes(p));
    l.Q = take(pp);
    l.Rn = take(pp);
    l.Rx = take(pp);
    l.eig = take(eig_ws_bytes(p, r));
    l.total = off;
    *L = l;
    return HYDE_OK;
}

inline bool ws_aligned(const void* q) { return ((uintptr_t)q % kAlign) == 0; }

template <typename T>
inline T* at(void* ws, size_t off) {
    return reinterpret_cast<T*>(reinterpret_cast<char*>(ws) + off);
}

}  // namespace
}  // namespace hyde

using namespace hyde;

extern "C" hyde_status hyde_hysime_workspace_size(int p, long long n, int r_max,
                                                  size_t* bytes) {
    if (!bytes) return HYDE_ERR_INVALID_ARG;
    HysimeLayout L;
    hyde_status st = hysime_layout(p, n, r_max, &L);
    if (st != HYDE_OK) return st;
    *bytes = L.total;
    return HYDE_OK;
}

extern "C" hyde_status hyde_hysime(const float* Y, int p, long long n, int r_max, int* k,
                                   int* idx, double* E, double* delta, double* evals,
                                   int* status, void* ws, size_t ws_bytes,
                                   cudaStream_t stream) {
    if (!Y || !k || !idx || !E || !delta || !evals) return HYDE_ERR_INVALID_ARG;
    HysimeLayout L;
    hyde_status st = hysime_layout(p, n, r_max, &L);
    if (st != HYDE_OK) return st;
    if (!ws || !ws_aligned(ws) || ws_bytes < L.total) return HYDE_ERR_WORKSPACE;
    if (cudaMemsetAsync(at<char>(ws, L.done), 0, sizeof(unsigned int), stream) != cudaSuccess)
        return HYDE_ERR_CUDA;
    double* R = at<double>(ws, L.R);
    double* Q = at<double>(ws, L.Q);
    double* Rn = at<double>(ws, L.Rn);
    double* Rx = at<double>(ws, L.Rx);
    const double inv_n = 1.0 / (double)n;
    st = launch_gram(Y, p, n, L.gram, at<float>(ws, L.partials), R, status, stream);
    if (st != HYDE_OK) return st;
    st = launch_inverse_from_gram(R, p, at<void>(ws, L.noise), Q, status, stream);
    if (st != HYDE_OK) return st;
    const long long pp = (long long)p * p;
    launch_pdl(hysime_form_kernel, (unsigned)((pp + 255) / 256), 256, 0, stream, R, Q, p, inv_n,
               Rn, Rx, status);
    st = launch_eig_top(Rx, nullptr, p, r_max, evals, E, at<void>(ws, L.eig), status, stream);
    if (st != HYDE_OK) return st;
    launch_pdl(hysime_delta_kernel, r_max, kHsThreads, 0, stream, R, Rn, E, p, r_max, inv_n,
               delta, at<unsigned int>(ws, L.done), k, idx, status);
    return cuda_status(cudaGetLastError());
}

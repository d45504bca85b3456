// Stein's unbiased risk estimate (SURE) of soft-thresholding whitened wavelet
// coefficients, for every component and every threshold candidate, and the
// choice of (rank, lambda) that minimises the total risk: what makes HyRes
// "parameter-free" (arXiv 2204.06979, Sec. 2.1).
//
// For unit-variance noise, soft-thresholding the detail coefficients of
// component i at lambda (keeping LL) has risk
//   S_i(lambda) = N - 2 #{detail: |c| <= lambda} + sum_detail min(c^2, lambda^2),
// and dropping the component has risk S_i(inf) = sum_all c^2 - N.
// On the uniform grid lambda_k = k * delta both counts and clipped sums come
// from one histogram pass: bin k collects the coefficients with
// lambda_{k-1} < |c| <= lambda_k (bin 0: c == 0), so prefix sums give
//   #{|c| <= lambda_k} and sum_{|c| <= lambda_k} c^2
// and coefficients above lambda_{K-1} contribute lambda_k^2 each.
#include <float.h>

#include "hyde_internal.cuh"

namespace hyde {
namespace {

// Every thread owns a private column of the block's histogram (layout
// [bin][thread], so a thread's updates never conflict with another's and
// need no atomics): 16-bit counts (the launcher bounds the values a thread
// sees below 2^16) and float sums, 6 bytes per bin and thread, so that a
// 256-thread block fits in 96 KB. The block reduces the columns and adds them
// to the global table with one atomic per bin. Each lane keeps eight float4
// loads in flight.
constexpr int kHistUnroll = 8;

__global__ void __launch_bounds__(256)
sure_hist_kernel(const float* __restrict__ coef, int Hp, int Wp, int hl, int wl, int K,
                 float inv_delta, int rows_per_block, unsigned int* __restrict__ counts,
                 double* __restrict__ sums, double* __restrict__ sum_all) {
    extern __shared__ unsigned char smraw[];
    const int T = blockDim.x, tid = threadIdx.x;
    float* hs = reinterpret_cast<float*>(smraw);                         // [K][T]
    unsigned short* hc = reinterpret_cast<unsigned short*>(hs + (size_t)K * T);   // [K][T]
    const int i = blockIdx.y;
    const int lane = tid & 31, wid = tid >> 5, nw = T >> 5;
    for (int e = tid; e < K * T; e += T) { hc[e] = 0; hs[e] = 0.f; }
    __syncthreads();
    const int y0 = blockIdx.x * rows_per_block;
    const int y1 = min(y0 + rows_per_block, Hp);
    const float* base = coef + (long long)i * Hp * Wp;
    float all = 0.f;
    // bin ceil(|c| / delta) by one float-to-int conversion rounding up; the
    // value is clamped below 2^24 so the conversion is exact and cannot wrap
    auto one = [&](float c, bool in_ll) {
        const float c2 = c * c;
        all += c2;
        if (in_ll) return;
        const int k = __float2int_ru(fminf(fabsf(c) * inv_delta, 16777216.f));
        if (k < K) {
            hc[k * T + tid] += 1;
            hs[k * T + tid] += c2;
        }
    };
    if ((Wp & 3) == 0) {
        const int W4 = Wp >> 2;
        for (int y = y0 + wid; y < y1; y += nw) {
            const float4* row = reinterpret_cast<const float4*>(base + (long long)y * Wp);
            const bool yll = y < hl;
            for (int x40 = lane; x40 < W4; x40 += 32 * kHistUnroll) {
                float4 v[kHistUnroll];
#pragma unroll
                for (int u = 0; u < kHistUnroll; ++u) {
                    const int x4 = x40 + 32 * u;
                    v[u] = x4 < W4 ? __ldg(row + x4) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < kHistUnroll; ++u) {
                    const int x4 = x40 + 32 * u;
                    if (x4 < W4) {
                        if (yll) {   // rows holding the final LL band
                            const int x = x4 * 4;
                            one(v[u].x, x < wl);
                            one(v[u].y, x + 1 < wl);
                            one(v[u].z, x + 2 < wl);
                            one(v[u].w, x + 3 < wl);
                        } else {
                            one(v[u].x, false);
                            one(v[u].y, false);
                            one(v[u].z, false);
                            one(v[u].w, false);
                        }
                    }
                }
            }
        }
    } else {
        for (int y = y0 + wid; y < y1; y += nw) {
            const float* row = base + (long long)y * Wp;
            const bool yll = y < hl;
            for (int x = lane; x < Wp; x += 32) one(__ldg(row + x), yll && x < wl);
        }
    }
    all = warp_sum(all);
    if (lane == 0 && all != 0.f) atomicAdd(&sum_all[i], (double)all);
    __syncthreads();
    for (int k = wid; k < K; k += nw) {
        unsigned int c = 0;
        float sacc = 0.f;
        for (int q = lane; q < T; q += 32) { c += hc[k * T + q]; sacc += hs[k * T + q]; }
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
        }
        if (lane == 0 && c) {
            atomicAdd(&counts[(long long)i * K + k], c);
            atomicAdd(&sums[(long long)i * K + k], (double)sacc);
        }
    }
}

// S[i][k] and S_inf[i]: one warp per component; the prefix sums over the
// bins are warp scans (K/32 chunks of shuffles), not a K-long serial chain.
__global__ void __launch_bounds__(256)
sure_table_kernel(const unsigned int* __restrict__ counts, const double* __restrict__ sums,
                  const double* __restrict__ sum_all, int batch, int K, long long N,
                  long long N_det, double delta, double* __restrict__ S,
                  double* __restrict__ S_inf) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= batch) return;
    double ccarry = 0.0, scarry = 0.0;
    for (int k0 = 0; k0 < K; k0 += 32) {
        const int k = k0 + lane;
        double c = k < K ? (double)counts[(long long)i * K + k] : 0.0;
        double q = k < K ? sums[(long long)i * K + k] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double c2 = __shfl_up_sync(0xffffffffu, c, o);
            const double q2 = __shfl_up_sync(0xffffffffu, q, o);
            if (lane >= o) { c += c2; q += q2; }
        }
        const double cle = c + ccarry, sle = q + scarry;
        if (k < K) {
            const double lam = k * delta;
            S[(long long)i * K + k] = (double)N - 2.0 * cle + sle + lam * lam * ((double)N_det - cle);
        }
        ccarry = __shfl_sync(0xffffffffu, cle, 31);
        scarry = __shfl_sync(0xffffffffu, sle, 31);
    }
    if (lane == 0) S_inf[i] = sum_all[i] - (double)N;
}

// Table and choice over the grid: block i (one warp of work) forms
// S_i(lambda_k) by warp scans over the bins and S_inf[i], so the FP64 work is
// spread over `batch` SMs (FP64 runs at a small fraction of the FP32 rate on
// this part); the last block to finish (a counter in the zeroed workspace)
// forms T(r, k) = sum_{i<=r} S_i(lambda_k) + sum_{i>r} S_inf[i] with one
// thread per column k walking r upwards (a sequential prefix: fewer FP64
// instructions than scans), keeps each column's first minimum and runner-up,
// and reduces them: the first minimum in row-major (rank, lambda) order and
// the relative gap to the runner-up.
__global__ void __launch_bounds__(256)
sure_select_kernel(const unsigned int* __restrict__ counts, const double* __restrict__ sums,
                   const double* __restrict__ sum_all, int batch, int K, long long N,
                   long long N_det, double delta, double* __restrict__ S,
                   double* __restrict__ S_inf, double* __restrict__ T, unsigned int* done,
                   hyde_hyres_info* info, int* rank_out, double* lam_out, const int* status) {
    __shared__ double tail[kMaxRank];
    __shared__ double wm1[8], wm2[8];
    __shared__ int wi1[8];
    __shared__ int s_last;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    const int i = blockIdx.x;
    if (wid == 0) {
        double ccarry = 0.0, scarry = 0.0;
        for (int k0 = 0; k0 < K; k0 += 32) {
            const int k = k0 + lane;
            double c = k < K ? (double)counts[(long long)i * K + k] : 0.0;
            double q = k < K ? sums[(long long)i * K + k] : 0.0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double c2 = __shfl_up_sync(0xffffffffu, c, o);
                const double q2 = __shfl_up_sync(0xffffffffu, q, o);
                if (lane >= o) { c += c2; q += q2; }
            }
            const double cle = c + ccarry, sle = q + scarry;
            if (k < K) {
                const double lam = k * delta;
                S[(long long)i * K + k] =
                    (double)N - 2.0 * cle + sle + lam * lam * ((double)N_det - cle);
            }
            ccarry = __shfl_sync(0xffffffffu, cle, 31);
            scarry = __shfl_sync(0xffffffffu, sle, 31);
        }
        if (lane == 0) S_inf[i] = sum_all[i] - (double)N;
    }
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = atomicAdd(done, 1u) == (unsigned)gridDim.x - 1u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // every block's S row, copied once with coalesced loads (L2, not L1)
    extern __shared__ double Ssh[];   // [batch][K]
    for (int e = t; e < batch * K; e += blockDim.x) Ssh[e] = __ldcg(S + e);
    if (t == 0) {   // tail[r] = sum_{i > r} S_inf[i]
        double acc = 0.0;
        for (int r = batch - 1; r >= 0; --r) {
            tail[r] = acc;
            acc += __ldcg(S_inf + r);
        }
    }
    __syncthreads();
    double m1 = DBL_MAX, m2 = DBL_MAX;
    int i1 = 0x7fffffff;
    for (int k = t; k < K; k += blockDim.x) {
        double head = 0.0;
        for (int r = 0; r < batch; ++r) {
            head += Ssh[r * K + k];
            const double v = head + tail[r];
            if (T) T[(long long)r * K + k] = v;
            const int e = r * K + k;
            if (v < m1 || (v == m1 && e < i1)) { m2 = fmin(m2, m1); m1 = v; i1 = e; }
            else m2 = fmin(m2, v);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double om1 = __shfl_xor_sync(0xffffffffu, m1, o);
        const double om2 = __shfl_xor_sync(0xffffffffu, m2, o);
        const int oi1 = __shfl_xor_sync(0xffffffffu, i1, o);
        if (om1 < m1 || (om1 == m1 && oi1 < i1)) { m2 = fmin(m1, om2); m1 = om1; i1 = oi1; }
        else m2 = fmin(m2, om1);
    }
    if (lane == 0) { wm1[wid] = m1; wm2[wid] = m2; wi1[wid] = i1; }
    __syncthreads();
    if (t == 0) {
        m1 = wm1[0]; m2 = wm2[0]; i1 = wi1[0];
        for (int q = 1; q < nw; ++q) {
            if (wm1[q] < m1 || (wm1[q] == m1 && wi1[q] < i1)) {
                m2 = fmin(m1, wm2[q]); m1 = wm1[q]; i1 = wi1[q];
            } else {
                m2 = fmin(m2, wm1[q]);
            }
        }
        const int tot = batch * K;
        const int r = i1 / K, k = i1 % K;
        if (rank_out) *rank_out = r + 1;
        if (lam_out) *lam_out = k * delta;
        if (info) {
            info->status = status ? *status : 0;
            info->rank = r + 1;
            info->lambda_index = k;
            info->reserved = 0;
            info->lambda = k * delta;
            info->sure_min = m1;
            info->sure_gap = (tot > 1) ? (m2 - m1) / fmax(fabs(m1), 1e-300) : 0.0;
        }
    }
}

}  // namespace

size_t sure_accum_bytes(int batch, int K) {
    return align_up((size_t)batch * K * sizeof(unsigned int), kAlign) +
           align_up((size_t)batch * K * sizeof(double), kAlign) +
           align_up((size_t)batch * sizeof(double), kAlign);
}

hyde_status launch_sure_hist(const float* coef, int batch, int Hp, int Wp, int levels, int K,
                             double delta, const SureBufs& b, cudaStream_t s) {
    int sms = device_sm_count();
    if (sms <= 0) return HYDE_ERR_CUDA;
    // threads per block: the private histograms (6 bytes per bin and thread)
    // stay within 96 KB so that two blocks share an SM
    int threads = (int)((96 * 1024) / (6 * (size_t)K)) / 32 * 32;
    if (threads > 256) threads = 256;
    if (threads < 32) threads = 32;
    int per_comp = (4 * sms + batch - 1) / batch;
    // a thread must see fewer than 2^16 values (16-bit bin counts)
    const long long per_thread_cap = 60000;
    const long long min_blocks = ((long long)Hp * Wp + per_thread_cap * threads - 1) /
                                 (per_thread_cap * threads);
    if (per_comp < min_blocks) per_comp = (int)min_blocks;
    if (per_comp > Hp) per_comp = Hp;
    if (per_comp < 1) per_comp = 1;
    int rows = (Hp + per_comp - 1) / per_comp;
    per_comp = (Hp + rows - 1) / rows;
    if ((long long)rows * Wp > per_thread_cap * threads) return HYDE_ERR_SHAPE;
    size_t smem = (size_t)K * threads * 6;
    if (ensure_smem_limit((const void*)sure_hist_kernel, (int)smem) != cudaSuccess)
        return HYDE_ERR_CUDA;
    dim3 grid(per_comp, batch);
    sure_hist_kernel<<<grid, threads, smem, s>>>(coef, Hp, Wp, Hp >> levels, Wp >> levels, K,
                                                 (float)(1.0 / delta), rows, b.counts, b.sums,
                                                 b.sum_all);
    return cuda_status(cudaGetLastError());
}

hyde_status launch_sure_select(const SureBufs& b, int batch, int K, long long N,
                               long long N_det, double delta, double* S, double* S_inf,
                               double* T, hyde_hyres_info* info, int* rank_out,
                               double* lam_out, const int* status, cudaStream_t s) {
    if (T == nullptr) {   // the tables only
        sure_table_kernel<<<(batch + 7) / 8, 256, 0, s>>>(b.counts, b.sums, b.sum_all, batch, K,
                                                           N, N_det, delta, S, S_inf);
    } else {
        if (batch > kMaxRank || b.done == nullptr) return HYDE_ERR_SHAPE;
        int threads = (K + 31) / 32 * 32;
        if (threads > 256) threads = 256;
        const size_t smem = (size_t)batch * K * sizeof(double);
        if (ensure_smem_limit((const void*)sure_select_kernel, (int)smem) != cudaSuccess)
            return HYDE_ERR_CUDA;
        sure_select_kernel<<<batch, threads, smem, s>>>(b.counts, b.sums, b.sum_all, batch, K, N,
                                                     N_det, delta, S, S_inf, T, b.done, info,
                                                     rank_out, lam_out, status);
    }
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

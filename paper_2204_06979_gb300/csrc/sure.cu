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

#include <cmath>

#include "hyde_internal.cuh"

namespace hyde {
namespace {

// The block's histogram has one column per lane index, [bin][lane], shared by
// all of its warps through shared-memory atomics whose result is unused (no
// thread waits on a read-modify-write, and lane l of every warp hits bank l):
// 32-bit counts and 32-bit fixed-point sums of c^2 in units of 2^-s. The
// launcher picks s and the rows per block so that no column can overflow.
// Integer sums make the table independent of the order of the additions; the
// block adds its columns to the global table with one atomic per bin, as
// doubles holding exact multiples of 2^-s.
//
// Both integers come from one FMA onto 1.5 * 2^23, where the float spacing
// is 1: rounded upwards it gives ceil(|c| / delta), rounded to nearest
// rn(c^2 * 2^s), in the low mantissa bits (exact below 2^22; larger |c|,
// inf and NaN give bit patterns above every bin).
constexpr int kHistThreads = 256;
constexpr int kHistUnroll = 4;
constexpr float kMagic = 12582912.f;   // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;

__global__ void __launch_bounds__(kHistThreads)
sure_hist_kernel(const float* __restrict__ coef, int Hp, int Wp, int hl, int wl, int K,
                 float inv_delta, float qscale, double inv_qscale, int rows_per_block,
                 unsigned int* __restrict__ counts, double* __restrict__ sums,
                 double* __restrict__ sum_all) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ unsigned int hsm[];   // counts [K][32], then sums [K][32]
    __shared__ double wall[kHistThreads / 32];
    unsigned int* hc = hsm;
    unsigned int* hq = hsm + K * 32;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int nw = kHistThreads / 32;
    for (int e = tid; e < 2 * K * 32; e += kHistThreads) hsm[e] = 0u;
    __syncthreads();
    const int i = blockIdx.y;
    const int y0 = blockIdx.x * rows_per_block;
    const int y1 = min(y0 + rows_per_block, Hp);
    const float* base = coef + (long long)i * Hp * Wp;
    float all = 0.f;
    auto one = [&](float c, bool in_ll) {
        const float c2 = c * c;
        all += c2;
        if (in_ll) return;
        const unsigned k =
            (unsigned)(__float_as_int(__fmaf_ru(fabsf(c), inv_delta, kMagic)) - kMagicBits);
        if (k < (unsigned)K) {
            const unsigned q = (unsigned)(__float_as_int(fmaf(c2, qscale, kMagic)) - kMagicBits);
            atomicAdd(hc + k * 32 + lane, 1u);
            atomicAdd(hq + k * 32 + lane, q);
        }
    };
    if (y0 < y1) {
        if ((Wp & 3) == 0) {
            // the block's rows as one run of float4s
            const int W4 = Wp >> 2;
            const float4* b4 = reinterpret_cast<const float4*>(base) + (long long)y0 * W4;
            const int nf = (y1 - y0) * W4;
            const bool has_ll = y0 < hl;   // only the first rows hold the final LL band
            for (int f = tid; f < nf; f += kHistThreads * kHistUnroll) {
                float4 v[kHistUnroll];
#pragma unroll
                for (int u = 0; u < kHistUnroll; ++u) {
                    const int fu = f + u * kHistThreads;
                    v[u] = fu < nf ? __ldg(b4 + fu) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < kHistUnroll; ++u) {
                    const int fu = f + u * kHistThreads;
                    if (fu >= nf) continue;
                    if (has_ll) {
                        const int yy = fu / W4;
                        const int x = (fu - yy * W4) * 4;
                        const bool yll = y0 + yy < hl;
                        one(v[u].x, yll && x < wl);
                        one(v[u].y, yll && x + 1 < wl);
                        one(v[u].z, yll && x + 2 < wl);
                        one(v[u].w, yll && x + 3 < wl);
                    } else {
                        one(v[u].x, false);
                        one(v[u].y, false);
                        one(v[u].z, false);
                        one(v[u].w, false);
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
    }
    all = warp_sum(all);
    if (lane == 0) wall[wid] = (double)all;
    __syncthreads();
    for (int k = wid; k < K; k += nw) {
        unsigned int c = hc[k * 32 + lane];
        unsigned long long q = hq[k * 32 + lane];
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            q += __shfl_xor_sync(0xffffffffu, q, o);
        }
        if (lane == 0 && c) {
            atomicAdd(&counts[(long long)i * K + k], c);
            atomicAdd(&sums[(long long)i * K + k], (double)q * inv_qscale);
        }
    }
    if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < nw; ++w) tot += wall[w];
        if (tot != 0.0) atomicAdd(&sum_all[i], tot);
    }
}

// Per-level thresholds: the same binning with one histogram per (component,
// group), group g = level g + 1 (the detail bands of that level; the final LL
// band joins the last group when all_coef, else it is not binned). In the
// Mallat layout the level of position (y, x) is min(ly, lx), ly the largest
// l <= L with y < Hp >> (l - 1) (likewise lx), and the LL band has ly = lx = L.
// A warp takes whole rows (ly once per row), its lanes four columns each per
// step (coalesced scalar loads, four in flight); the shared histogram is
// [group][bin][lane], the overflow bound the same as the detail-only kernel's
// with ceil(Wp / 32) values per lane column and row.
constexpr int kLevCols = 4;

__global__ void __launch_bounds__(kHistThreads)
sure_hist_level_kernel(const float* __restrict__ coef, int Hp, int Wp, int levels, int all_coef,
                       int K, float inv_delta, float qscale, double inv_qscale,
                       int rows_per_block, unsigned int* __restrict__ counts,
                       double* __restrict__ sums, double* __restrict__ sum_all) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ unsigned int hsm[];   // counts [G][K][32], then sums [G][K][32]
    __shared__ double wall[kHistThreads / 32];
    const int G = levels, GK = levels * K;
    unsigned int* hc = hsm;
    unsigned int* hq = hsm + GK * 32;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int nw = kHistThreads / 32;
    for (int e = tid; e < 2 * GK * 32; e += kHistThreads) hsm[e] = 0u;
    __syncthreads();
    const int i = blockIdx.y;
    const int y0 = blockIdx.x * rows_per_block;
    const int y1 = min(y0 + rows_per_block, Hp);
    const int hll = Hp >> levels, wll = Wp >> levels;
    const float* base = coef + (long long)i * Hp * Wp;
    float all = 0.f;
    for (int y = y0 + wid; y < y1; y += nw) {
        int ly = 1;
        for (int j = 1; j < G; ++j) ly += y < (Hp >> j);
        const bool yll = y < hll;
        const float* row = base + (long long)y * Wp;
        for (int x0 = 0; x0 < Wp; x0 += 32 * kLevCols) {
            float v[kLevCols];
#pragma unroll
            for (int u = 0; u < kLevCols; ++u) {
                const int x = x0 + 32 * u + lane;
                v[u] = x < Wp ? __ldg(row + x) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kLevCols; ++u) {
                const int x = x0 + 32 * u + lane;
                if (x >= Wp) continue;
                const float c = v[u];
                const float c2 = c * c;
                all += c2;
                if (yll && x < wll && !all_coef) continue;
                int lx = 1;
                for (int j = 1; j < G; ++j) lx += x < (Wp >> j);
                const int g = min(ly, lx) - 1;
                const unsigned k = (unsigned)(__float_as_int(__fmaf_ru(fabsf(c), inv_delta,
                                                                       kMagic)) - kMagicBits);
                if (k < (unsigned)K) {
                    const unsigned q =
                        (unsigned)(__float_as_int(fmaf(c2, qscale, kMagic)) - kMagicBits);
                    atomicAdd(hc + (g * K + (int)k) * 32 + lane, 1u);
                    atomicAdd(hq + (g * K + (int)k) * 32 + lane, q);
                }
            }
        }
    }
    all = warp_sum(all);
    if (lane == 0) wall[wid] = (double)all;
    __syncthreads();
    for (int e = wid; e < GK; e += nw) {
        unsigned int c = hc[e * 32 + lane];
        unsigned long long q = hq[e * 32 + lane];
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            q += __shfl_xor_sync(0xffffffffu, q, o);
        }
        if (lane == 0 && c) {
            atomicAdd(&counts[(long long)i * GK + e], c);
            atomicAdd(&sums[(long long)i * GK + e], (double)q * inv_qscale);
        }
    }
    if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < nw; ++w) tot += wall[w];
        if (tot != 0.0) atomicAdd(&sum_all[i], tot);
    }
}

// S[i][k] and S_inf[i]: one warp per component; the prefix sums over the
// bins are warp scans (K/32 chunks of shuffles), not a K-long serial chain.
__global__ void __launch_bounds__(256)
sure_table_kernel(const unsigned int* __restrict__ counts, const double* __restrict__ sums,
                  const double* __restrict__ sum_all, int batch, int K, long long N,
                  long long N_det, double delta, double* __restrict__ S,
                  double* __restrict__ S_inf) {
    pdl_wait();
    pdl_trigger();
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

// Table and choice over the grid. FP64 runs at a small fraction of the FP32
// rate on this part and a dependent FP64 instruction costs many cycles, so
// the counts and clipped sums are prefixed as integers: the histogram sums
// are exact multiples of 2^-16 (the fixed-point unit of the histogram, or a
// coarser power of two), so with c the count and q the sum in units of
// 2^-16, both cumulated over the bins up to k,
//   A_ik = (N - 2 c) 2^16 + q,   B_ik = N_det - c   (64-bit integers)
// give S_i(lambda_k) = A_ik 2^-16 + lambda_k^2 B_ik exactly but for the final
// rounding. Block i forms row i of A and B (block-wide integer scans) and of
// S, and S_inf[i]; the last block to finish (a counter in the zeroed
// workspace) prefixes A and B over the components, which gives
//   T(r, k) = sum_{i<=r} S_i(lambda_k) + sum_{i>r} S_inf[i]
//           = PA_rk 2^-16 + lambda_k^2 PB_rk + sum_{i>r} S_inf[i],
// forms every T with a few FP64 operations spread over the block, and finds
// the first minimum in row-major (rank, lambda) order and the runner-up on
// order-preserving integer keys.
//
// Per-component thresholds (one lambda per kept component): before the
// prefix, one warp per component takes the first minimum of row i of S (the
// same FP64 expression as the table), k_i; then
//   U(r) = sum_{i<=r} S_i(lambda_{k_i}) + sum_{i>r} S_inf[i]
// is accumulated over r in FP64 by one thread (at most 32 terms) and its
// first minimum gives the rank. The thresholds go to lam_comp[i][level] for
// the inverse transform, which multiplies them by *lam_out = 1.
constexpr int kSelThreads = 256;

__device__ __forceinline__ long long ord_key(double v) {
    const long long bits = __double_as_longlong(v);
    return bits >= 0 ? bits : bits ^ 0x7fffffffffffffffLL;
}
__device__ __forceinline__ double key_value(long long k) {
    return __longlong_as_double(k >= 0 ? k : k ^ 0x7fffffffffffffffLL);
}

// inclusive block scan of (c, q) over threads 0..blockDim-1 (kSelThreads)
__device__ __forceinline__ void block_scan2(long long& c, long long& q, long long* wc,
                                            long long* wq) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long c2 = __shfl_up_sync(0xffffffffu, c, o);
        const long long q2 = __shfl_up_sync(0xffffffffu, q, o);
        if (lane >= o) { c += c2; q += q2; }
    }
    if (lane == 31) { wc[wid] = c; wq[wid] = q; }
    __syncthreads();
    long long oc = 0, oq = 0;
    for (int w = 0; w < wid; ++w) { oc += wc[w]; oq += wq[w]; }
    c += oc;
    q += oq;
}

__device__ __forceinline__ void keep_min2(long long kv, int e, long long& m1, long long& m2,
                                          int& i1) {
    if (kv < m1 || (kv == m1 && e < i1)) {
        m2 = min(m2, m1);
        m1 = kv;
        i1 = e;
    } else {
        m2 = min(m2, kv);
    }
}

__global__ void __launch_bounds__(kSelThreads)
sure_select_kernel(const unsigned int* __restrict__ counts, const double* __restrict__ sums,
                   const double* __restrict__ sum_all, int batch, int K, long long N,
                   long long N_det, double delta, double* __restrict__ S,
                   double* __restrict__ S_inf, double* __restrict__ T, long long* sint,
                   unsigned int* done, hyde_hyres_info* info, int* rank_out, double* lam_out,
                   const int* status, float* lam_comp, int levels) {
    pdl_wait();
    pdl_trigger();
    __shared__ long long wc[kSelThreads / 32], wq[kSelThreads / 32];
    __shared__ double tail[kMaxRank], sinf[kMaxRank];
    __shared__ double cmin[kMaxRank];   // per-component minimum S_i(lambda_{k_i})
    __shared__ int ck[kMaxRank];        // its k_i
    __shared__ int s_rank;
    __shared__ double lam2[kMaxLambda];
    __shared__ long long wm1[kSelThreads / 32], wm2[kSelThreads / 32];
    __shared__ int wi1[kSelThreads / 32];
    __shared__ int s_last;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    constexpr int nw = kSelThreads / 32;
    const int i = blockIdx.x;
    long long* A = sint;                       // [batch][K]
    long long* B = sint + (long long)batch * K;
    {   // row i: integer scans over the bins (K <= kSelThreads)
        long long c = 0, q = 0;
        if (t < K) {
            c = counts[(long long)i * K + t];
            q = (long long)(sums[(long long)i * K + t] * 65536.0);   // exact
        }
        block_scan2(c, q, wc, wq);
        if (t < K) {
            const long long a = (N - 2 * c) * 65536LL + q, bb = N_det - c;
            A[(long long)i * K + t] = a;
            B[(long long)i * K + t] = bb;
            const double lam = t * delta;
            S[(long long)i * K + t] = fma(lam * lam, (double)bb, (double)a * (1.0 / 65536.0));
        }
        if (t == 0) S_inf[i] = sum_all[i] - (double)N;
    }
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = atomicAdd(done, 1u) == (unsigned)gridDim.x - 1u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // every block's rows of A and B (L2, not L1), prefixed over the components in place
    extern __shared__ long long Psh[];   // PA [batch][K], then PB [batch][K]
    long long* PA = Psh;
    long long* PB = Psh + batch * K;
    for (int e = t; e < batch * K; e += kSelThreads) {
        PA[e] = __ldcg(A + e);
        PB[e] = __ldcg(B + e);
    }
    if (t < batch) sinf[t] = __ldcg(S_inf + t);
    for (int k = t; k < K; k += kSelThreads) {
        const double lam = k * delta;
        lam2[k] = lam * lam;
    }
    __syncthreads();
    if (lam_comp) {   // per-component first minimum over the rows of S (not yet prefixed)
        for (int i = wid; i < batch; i += nw) {
            long long m = 0x7fffffffffffffffLL;
            int kb = 0x7fffffff;
            for (int k = lane; k < K; k += 32) {   // ascending k: strict < keeps the first
                const long long kv = ord_key(fma(lam2[k], (double)PB[i * K + k],
                                                 (double)PA[i * K + k] * (1.0 / 65536.0)));
                if (kv < m) { m = kv; kb = k; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const long long om = __shfl_xor_sync(0xffffffffu, m, o);
                const int ok = __shfl_xor_sync(0xffffffffu, kb, o);
                if (om < m || (om == m && ok < kb)) { m = om; kb = ok; }
            }
            if (lane == 0) { cmin[i] = key_value(m); ck[i] = kb; }
        }
        __syncthreads();
    }
    if (t < batch) {   // tail[r] = sum_{i > r} S_inf[i], added from i = batch - 1 down
        double acc = 0.0;
        for (int r = batch - 1; r > t; --r) acc += sinf[r];
        tail[t] = acc;
    }
    for (int k = t; k < K; k += kSelThreads) {
        long long pa = 0, pb = 0;
        for (int r = 0; r < batch; ++r) {
            pa += PA[r * K + k];
            pb += PB[r * K + k];
            PA[r * K + k] = pa;
            PB[r * K + k] = pb;
        }
    }
    __syncthreads();
    long long m1 = 0x7fffffffffffffffLL, m2 = 0x7fffffffffffffffLL;
    int i1 = 0x7fffffff;
    for (int e = t; e < batch * K; e += kSelThreads) {
        const int r = e / K, k = e - r * K;
        const double v =
            fma(lam2[k], (double)PB[e], (double)PA[e] * (1.0 / 65536.0)) + tail[r];
        if (T) T[e] = v;
        keep_min2(ord_key(v), e, m1, m2, i1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long om1 = __shfl_xor_sync(0xffffffffu, m1, o);
        const long long om2 = __shfl_xor_sync(0xffffffffu, m2, o);
        const int oi1 = __shfl_xor_sync(0xffffffffu, i1, o);
        if (om1 < m1 || (om1 == m1 && oi1 < i1)) { m2 = min(m1, om2); m1 = om1; i1 = oi1; }
        else m2 = min(m2, om1);
    }
    if (lane == 0) { wm1[wid] = m1; wm2[wid] = m2; wi1[wid] = i1; }
    __syncthreads();
    if (t == 0) {
        m1 = wm1[0]; m2 = wm2[0]; i1 = wi1[0];
        for (int q = 1; q < nw; ++q) {
            if (wm1[q] < m1 || (wm1[q] == m1 && wi1[q] < i1)) {
                m2 = min(m1, wm2[q]); m1 = wm1[q]; i1 = wi1[q];
            } else {
                m2 = min(m2, wm1[q]);
            }
        }
        const int tot = batch * K;
        int r = i1 / K, k = i1 % K;
        double v1 = key_value(m1), v2 = key_value(m2), scale = k * delta;
        int cand = tot;
        if (lam_comp) {   // U(r): first minimum over r and the runner-up
            double acc = 0.0, u1 = 0.0, u2 = 0.0;
            int rb = 0;
            for (int q = 0; q < batch; ++q) {
                acc += cmin[q];
                const double u = acc + tail[q];
                if (q == 0) { u1 = u; u2 = u; }
                else if (u < u1) { u2 = (q == 1) ? u1 : fmin(u2, u1); u1 = u; rb = q; }
                else u2 = (q == 1) ? u : fmin(u2, u);
            }
            r = rb;
            k = ck[0];
            v1 = u1;
            v2 = u2;
            scale = 1.0;
            cand = batch;
        }
        s_rank = r;
        if (rank_out) *rank_out = r + 1;
        if (lam_out) *lam_out = scale;
        if (info) {
            info->status = status ? *status : 0;
            info->rank = r + 1;
            info->lambda_index = k;
            info->reserved = 0;
            info->lambda = k * delta;
            info->sure_min = v1;
            info->sure_gap = (cand > 1) ? (v2 - v1) / fmax(fabs(v1), 1e-300) : 0.0;
        }
    }
    if (lam_comp) {   // thresholds of the kept components, 0 for the dropped ones
        __syncthreads();
        const int rk = s_rank;
        for (int e = t; e < batch * levels; e += kSelThreads) {
            const int i = e / levels;
            lam_comp[e] = i <= rk ? (float)(ck[i] * delta) : 0.f;
        }
    }
}

// Per-level selection. Block (i, g) scans row (i, g) of the histogram into
// the group's SURE, S_ig(lambda_k) = A 2^-16 + lambda_k^2 B with
//   A = (N_g - 2 c) 2^16 + q,   B = N_g - c,
// N_g the group's size (3 (Hp >> l)(Wp >> l) detail coefficients of level
// l = g + 1, plus the LL band in the last group when all_coef), and keeps its
// first minimum over k (key and index in sint). The last block to finish adds
// each component's group minima to the count of kept coefficients, forms
//   U(r) = sum_{i<=r} S*_i + sum_{i>r} S_inf[i]
// and writes the rank, the thresholds lam_comp[i][g] and the info record.
__global__ void __launch_bounds__(kSelThreads)
sure_select_level_kernel(const unsigned int* __restrict__ counts,
                         const double* __restrict__ sums, const double* __restrict__ sum_all,
                         int batch, int G, int K, int Hp, int Wp, int all_coef, long long N,
                         double delta, double* __restrict__ S, double* __restrict__ S_inf,
                         long long* sint, unsigned int* done, hyde_hyres_info* info,
                         int* rank_out, double* lam_out, const int* status, float* lam_comp) {
    pdl_wait();
    pdl_trigger();
    __shared__ long long wc[kSelThreads / 32], wq[kSelThreads / 32];
    __shared__ long long wk[kSelThreads / 32];
    __shared__ int wi[kSelThreads / 32];
    __shared__ double comp[kMaxRank], tail[kMaxRank], sinf[kMaxRank];
    __shared__ int s_last, s_rank;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    constexpr int nw = kSelThreads / 32;
    const int row = blockIdx.x, i = row / G, g = row - i * G;
    const int rows = batch * G;
    long long Ng = 3LL * (Hp >> (g + 1)) * (Wp >> (g + 1));
    if (all_coef && g == G - 1) Ng += (long long)(Hp >> G) * (Wp >> G);
    {
        long long c = 0, q = 0;
        if (t < K) {
            c = counts[(long long)row * K + t];
            q = (long long)(sums[(long long)row * K + t] * 65536.0);   // exact
        }
        block_scan2(c, q, wc, wq);
        long long key = 0x7fffffffffffffffLL;
        int kb = 0x7fffffff;
        if (t < K) {
            const long long a = (Ng - 2 * c) * 65536LL + q, bb = Ng - c;
            const double lam = t * delta;
            const double v = fma(lam * lam, (double)bb, (double)a * (1.0 / 65536.0));
            S[(long long)row * K + t] = v;
            key = ord_key(v);
            kb = t;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const long long ok = __shfl_xor_sync(0xffffffffu, key, o);
            const int oi = __shfl_xor_sync(0xffffffffu, kb, o);
            if (ok < key || (ok == key && oi < kb)) { key = ok; kb = oi; }
        }
        if (lane == 0) { wk[wid] = key; wi[wid] = kb; }
        __syncthreads();
        if (t == 0) {
            for (int w = 1; w < nw; ++w)
                if (wk[w] < key || (wk[w] == key && wi[w] < kb)) { key = wk[w]; kb = wi[w]; }
            sint[row] = key;
            sint[rows + row] = kb;
            if (g == 0) S_inf[i] = sum_all[i] - (double)N;
        }
    }
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = atomicAdd(done, 1u) == (unsigned)gridDim.x - 1u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const double n_kept = all_coef ? 0.0 : (double)((long long)(Hp >> G) * (Wp >> G));
    if (t < batch) {
        double acc = n_kept;
        for (int q = 0; q < G; ++q) acc += key_value(__ldcg(sint + t * G + q));
        comp[t] = acc;
        sinf[t] = __ldcg(S_inf + t);
    }
    __syncthreads();
    if (t < batch) {
        double acc = 0.0;
        for (int r = batch - 1; r > t; --r) acc += sinf[r];
        tail[t] = acc;
    }
    __syncthreads();
    if (t == 0) {
        double acc = 0.0, u1 = 0.0, u2 = 0.0;
        int rb = 0;
        for (int q = 0; q < batch; ++q) {
            acc += comp[q];
            const double u = acc + tail[q];
            if (q == 0) { u1 = u; u2 = u; }
            else if (u < u1) { u2 = (q == 1) ? u1 : fmin(u2, u1); u1 = u; rb = q; }
            else u2 = (q == 1) ? u : fmin(u2, u);
        }
        s_rank = rb;
        const int k0 = (int)__ldcg(sint + rows);
        if (rank_out) *rank_out = rb + 1;
        if (lam_out) *lam_out = 1.0;
        if (info) {
            info->status = status ? *status : 0;
            info->rank = rb + 1;
            info->lambda_index = k0;
            info->reserved = 0;
            info->lambda = k0 * delta;
            info->sure_min = u1;
            info->sure_gap = batch > 1 ? (u2 - u1) / fmax(fabs(u1), 1e-300) : 0.0;
        }
    }
    __syncthreads();
    const int rk = s_rank;
    for (int e = t; e < rows; e += kSelThreads) {
        const int ci = e / G;
        lam_comp[e] = ci <= rk ? (float)(__ldcg(sint + rows + e) * delta) : 0.f;
    }
}

}  // namespace

size_t sure_accum_bytes(int batch, int K) {
    return align_up((size_t)batch * K * sizeof(unsigned int), kAlign) +
           align_up((size_t)batch * K * sizeof(double), kAlign) +
           align_up((size_t)batch * sizeof(double), kAlign);
}

hyde_status launch_sure_hist(const float* coef, int batch, int Hp, int Wp, int levels, int K,
                             double delta, const SureBufs& b, cudaStream_t s, bool all_coef) {
    const int sms = device_sm_count();
    if (sms <= 0) return HYDE_ERR_CUDA;
    if (K < 1 || !(delta > 0.0)) return HYDE_ERR_INVALID_ARG;
    const size_t smem = (size_t)2 * K * 32 * sizeof(unsigned int);
    if (smem > 200 * 1024) return HYDE_ERR_SHAPE;
    const float inv_delta = (float)(1.0 / delta);
    // largest c^2 that lands in a bin below K (ceil(|c| * inv_delta) <= K - 1), with margin
    const double q = (K - 1) / (double)inv_delta;
    const double c2max = q * q * 1.001 + 1e-300;
    // fixed-point unit 2^-s: rn(c^2 * 2^s) must stay below 2^22 (the FMA trick)
    int sh = 16;
    while (sh > 0 && c2max * std::ldexp(1.0, sh) >= 4194304.0) --sh;
    if (c2max * std::ldexp(1.0, sh) >= 4194304.0) return HYDE_ERR_SHAPE;
    const double qmax = std::floor(c2max * std::ldexp(1.0, sh)) + 1.0;
    // values one lane column can receive per row, and the rows that keep its sum below 2^32
    const double per_row = 4.0 * (double)(((long long)Wp + 127) / 128);
    const long long rows_cap = (long long)(4294967295.0 / (qmax * per_row));
    if (rows_cap < 1) return HYDE_ERR_SHAPE;
    // about eight 256-thread blocks per SM
    int per_comp = (8 * sms + batch - 1) / batch;
    if (per_comp > Hp) per_comp = Hp;
    if (per_comp < 1) per_comp = 1;
    long long rows = (Hp + per_comp - 1) / per_comp;
    if (rows > rows_cap) rows = rows_cap;
    per_comp = (int)((Hp + rows - 1) / rows);
    if (ensure_smem_limit((const void*)sure_hist_kernel, (int)smem) != cudaSuccess)
        return HYDE_ERR_CUDA;
    dim3 grid(per_comp, batch);
    // an empty excluded band (0 x 0) bins every coefficient
    const int hl = all_coef ? 0 : Hp >> levels, wl = all_coef ? 0 : Wp >> levels;
    launch_pdl(sure_hist_kernel, grid, kHistThreads, smem, s, coef, Hp, Wp, hl, wl, K, inv_delta,
               (float)std::ldexp(1.0, sh), std::ldexp(1.0, -sh), (int)rows, b.counts, b.sums,
               b.sum_all);
    return cuda_status(cudaGetLastError());
}

hyde_status launch_sure_hist_levels(const float* coef, int batch, int Hp, int Wp, int levels,
                                    int K, double delta, bool all_coef, const SureBufs& b,
                                    cudaStream_t s) {
    const int sms = device_sm_count();
    if (sms <= 0) return HYDE_ERR_CUDA;
    if (K < 1 || !(delta > 0.0) || levels < 1 || levels > kMaxLevels)
        return HYDE_ERR_INVALID_ARG;
    const size_t smem = (size_t)2 * levels * K * 32 * sizeof(unsigned int);
    if (smem > 200 * 1024) return HYDE_ERR_SHAPE;
    const float inv_delta = (float)(1.0 / delta);
    const double q = (K - 1) / (double)inv_delta;
    const double c2max = q * q * 1.001 + 1e-300;
    int sh = 16;
    while (sh > 0 && c2max * std::ldexp(1.0, sh) >= 4194304.0) --sh;
    if (c2max * std::ldexp(1.0, sh) >= 4194304.0) return HYDE_ERR_SHAPE;
    const double qmax = std::floor(c2max * std::ldexp(1.0, sh)) + 1.0;
    // values one lane column can receive per row, and the rows that keep its sum below 2^32
    const double per_row = (double)(((long long)Wp + 31) / 32);
    const long long rows_cap = (long long)(4294967295.0 / (qmax * per_row));
    if (rows_cap < 1) return HYDE_ERR_SHAPE;
    int per_comp = (8 * sms + batch - 1) / batch;
    if (per_comp > Hp) per_comp = Hp;
    if (per_comp < 1) per_comp = 1;
    long long rows = (Hp + per_comp - 1) / per_comp;
    if (rows > rows_cap) rows = rows_cap;
    per_comp = (int)((Hp + rows - 1) / rows);
    if (ensure_smem_limit((const void*)sure_hist_level_kernel, (int)smem) != cudaSuccess)
        return HYDE_ERR_CUDA;
    launch_pdl(sure_hist_level_kernel, dim3(per_comp, batch), kHistThreads, smem, s, coef, Hp,
               Wp, levels, all_coef ? 1 : 0, K, inv_delta, (float)std::ldexp(1.0, sh),
               std::ldexp(1.0, -sh), (int)rows, b.counts, b.sums, b.sum_all);
    return cuda_status(cudaGetLastError());
}

hyde_status launch_sure_select_levels(const SureBufs& b, int batch, int levels, int K, int Hp,
                                      int Wp, bool all_coef, long long N, double delta,
                                      double* S, double* S_inf, hyde_hyres_info* info,
                                      int* rank_out, double* lam_out, const int* status,
                                      float* lam_comp, cudaStream_t s) {
    if (batch > kMaxRank || K > kSelThreads || levels < 1 || levels > kMaxLevels ||
        b.done == nullptr || b.sint == nullptr || lam_comp == nullptr)
        return HYDE_ERR_SHAPE;
    launch_pdl(sure_select_level_kernel, batch * levels, kSelThreads, 0, s, b.counts, b.sums,
               b.sum_all, batch, levels, K, Hp, Wp, all_coef ? 1 : 0, N, delta, S, S_inf,
               b.sint, b.done, info, rank_out, lam_out, status, lam_comp);
    return cuda_status(cudaGetLastError());
}

hyde_status launch_sure_select(const SureBufs& b, int batch, int K, long long N,
                               long long N_det, double delta, double* S, double* S_inf,
                               double* T, hyde_hyres_info* info, int* rank_out,
                               double* lam_out, const int* status, cudaStream_t s,
                               float* lam_comp, int levels) {
    if (T == nullptr) {   // the tables only
        launch_pdl(sure_table_kernel, (batch + 7) / 8, 256, 0, s, b.counts, b.sums, b.sum_all,
                   batch, K, N, N_det, delta, S, S_inf);
    } else {
        if (batch > kMaxRank || K > kSelThreads || b.done == nullptr || b.sint == nullptr)
            return HYDE_ERR_SHAPE;
        if (lam_comp && levels < 1) return HYDE_ERR_INVALID_ARG;
        const size_t smem = (size_t)2 * batch * K * sizeof(long long);
        if (ensure_smem_limit((const void*)sure_select_kernel, (int)smem) != cudaSuccess)
            return HYDE_ERR_CUDA;
        launch_pdl(sure_select_kernel, batch, kSelThreads, smem, s, b.counts, b.sums,
                   b.sum_all, batch, K, N, N_det, delta, S, S_inf, T, b.sint, b.done, info,
                   rank_out, lam_out, status, lam_comp, levels);
    }
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

// Wavelet-domain stages of the batched sliding-window form (arXiv
// 2204.06979: HyRes, Sec. 2.1, on every tile of a scene denoised in tiles,
// Sec. 2.2.2): every kernel here covers all windows of the call in one
// launch, one block per (component, window).
//
//  * win_dwt_kernel: the L-level periodic db2 analysis of one padded
//    component image, level after level inside the block (the LL band of a
//    level goes to the block's scratch in global memory, read back through L2
//    by the next level after a barrier);
//    the detail coefficients go straight into the component's SURE
//    histogram on the grid lambda_k = k delta (counts and 2^-sh fixed-point
//    sums of c^2 per bin, exact integers, so the table does not depend on the
//    order of the additions), written as row i of the window's table;
//  * win_sure_select_kernel (one block per window): the integer-prefixed
//    tables, T(r, k) = sum_{i<=r} S_i(lambda_k) + sum_{i>r} S_inf[i], the
//    first minimum in row-major (r, k) order and the runner-up;
//  * win_idwt_kernel: soft threshold at the window's lambda* and the
//    L-level synthesis of each kept component into its padded image.
// The arithmetic of each stage is that of the one-cube kernels (dwt.cu,
// sure.cu); what differs is the mapping to blocks.
#include <cmath>

#include "hyde_internal.cuh"

namespace hyde {
namespace {

constexpr int kWdThreads = 256;

__device__ __forceinline__ float softf(float c, float lam) {
    return copysignf(fmaxf(fabsf(c) - lam, 0.f), c);
}

// SURE histogram: bin k collects the detail coefficients with
// (k - 1) delta < |c| <= k delta (bin 0: c = 0); the bin and rn(c^2 2^sh)
// each come from one FMA onto 1.5 * 2^23 (exact below 2^22), into a
// [bin][lane] shared histogram (lane l of every warp hits bank l). The plan
// picks sh so that no lane column can overflow 32 bits.
constexpr float kMagic = 12582912.f;   // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;

// Analysis of component i of window w: levels 1..L. Level l reads its input
// (h x w, the padded image at l = 1, else LL_{l-1} from scratch) and writes
// the three detail bands to their Mallat positions of the coefficient image
// (row stride Wp) and LL_l to scratch (half A for odd l, B for even l) or,
// at l = L, into the coefficient image. Every detail coefficient goes into
// the component's SURE histogram as it is formed (the final LL band only
// into the sum of squares), so the coefficients are not read again for SURE
// (a separate histogram kernel over the 512-window scene took 0.33 ms).
__global__ void __launch_bounds__(kWdThreads)
win_dwt_kernel(const float* __restrict__ Zp, float* __restrict__ coef,
               float* __restrict__ scratch, const WinDesc* __restrict__ desc, int levels,
               int r, int K, unsigned int* __restrict__ counts, double* __restrict__ sums,
               double* __restrict__ sum_all) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ unsigned int whsm[];   // counts [K][32], then sums [K][32]
    __shared__ double wall[kWdThreads / 32];
    unsigned int* hc = whsm;
    unsigned int* hq = whsm + K * 32;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int e = tid; e < 2 * K * 32; e += kWdThreads) whsm[e] = 0u;
    const int i = blockIdx.x, wi = blockIdx.y;
    const WinDesc d = desc[wi];
    const float inv_delta = (float)(1.0 / d.delta);
    const float qscale = ldexpf(1.0f, d.sh);
    float all = 0.f;
    auto bin = [&](float c) {
        const float c2 = c * c;
        all += c2;
        const unsigned k =
            (unsigned)(__float_as_int(__fmaf_ru(fabsf(c), inv_delta, kMagic)) - kMagicBits);
        if (k < (unsigned)K) {
            const unsigned q = (unsigned)(__float_as_int(fmaf(c2, qscale, kMagic)) - kMagicBits);
            atomicAdd(hc + k * 32 + lane, 1u);
            atomicAdd(hq + k * 32 + lane, q);
        }
    };
    __syncthreads();
    const int N = d.Hp * d.Wp;
    const float* img = Zp + d.img + (long long)i * N;
    float* C = coef + d.img + (long long)i * N;
    float* A = scratch + d.scr + (long long)i * win_scratch_stride(N);
    float* B = A + N / 4;
    for (int l = 1; l <= levels; ++l) {
        const int h = d.Hp >> (l - 1), w = d.Wp >> (l - 1), hh = h >> 1, wh = w >> 1;
        const float* in = l == 1 ? img : ((l & 1) ? B : A);
        float* ll = l == levels ? C : ((l & 1) ? A : B);
        const int ll_ld = l == levels ? d.Wp : wh;
        for (int e = threadIdx.x; e < hh * wh; e += kWdThreads) {
            const int J = e / wh, Kc = e - J * wh;
            const int x0 = 2 * Kc, x2 = (2 * Kc + 2 >= w) ? 2 * Kc + 2 - w : 2 * Kc + 2;
            float a[4], dd[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                int y = 2 * J + m;
                if (y >= h) y -= h;
                const float* row = in + (long long)y * w;
                float2 u, v;
                if (l == 1) {   // written by the previous kernel
                    u = __ldg(reinterpret_cast<const float2*>(row + x0));
                    v = __ldg(reinterpret_cast<const float2*>(row + x2));
                } else {        // written by this block: through L2, not L1
                    u = __ldcg(reinterpret_cast<const float2*>(row + x0));
                    v = __ldcg(reinterpret_cast<const float2*>(row + x2));
                }
                a[m] = kH0 * u.x + kH1 * u.y + kH2 * v.x + kH3 * v.y;
                dd[m] = kG0 * u.x + kG1 * u.y + kG2 * v.x + kG3 * v.y;
            }
            float* pt = C + (long long)J * d.Wp;
            float* pb = C + (long long)(hh + J) * d.Wp;
            const float hl = kH0 * dd[0] + kH1 * dd[1] + kH2 * dd[2] + kH3 * dd[3];   // row detail
            const float lh = kG0 * a[0] + kG1 * a[1] + kG2 * a[2] + kG3 * a[3];       // column detail
            const float hhv = kG0 * dd[0] + kG1 * dd[1] + kG2 * dd[2] + kG3 * dd[3];
            const float llv = kH0 * a[0] + kH1 * a[1] + kH2 * a[2] + kH3 * a[3];
            pt[wh + Kc] = hl;
            pb[Kc] = lh;
            pb[wh + Kc] = hhv;
            ll[(long long)J * ll_ld + Kc] = llv;
            bin(hl);
            bin(lh);
            bin(hhv);
            if (l == levels) all += llv * llv;   // kept, not binned
        }
        __syncthreads();
    }
    all = warp_sum(all);
    if (lane == 0) wall[wid] = (double)all;
    __syncthreads();
    const double inv_q = ldexp(1.0, -d.sh);
    const long long row = ((long long)wi * r + i) * K;
    for (int k = wid; k < K; k += kWdThreads / 32) {
        unsigned int c = hc[k * 32 + lane];
        unsigned long long q = hq[k * 32 + lane];
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            q += __shfl_xor_sync(0xffffffffu, q, o);
        }
        if (lane == 0) {
            counts[row + k] = c;
            sums[row + k] = (double)q * inv_q;
        }
    }
    if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < kWdThreads / 32; ++w) tot += wall[w];
        sum_all[(long long)wi * r + i] = tot;
    }
}


__device__ __forceinline__ long long ord_key(double v) {
    const long long bits = __double_as_longlong(v);
    return bits >= 0 ? bits : bits ^ 0x7fffffffffffffffLL;
}
__device__ __forceinline__ double key_value(long long k) {
    return __longlong_as_double(k >= 0 ? k : k ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ void keep_first_min2(long long kv, int e, long long& m1, long long& m2,
                                                int& i1) {
    if (kv < m1 || (kv == m1 && e < i1)) {
        m2 = min(m2, m1);
        m1 = kv;
        i1 = e;
    } else {
        m2 = min(m2, kv);
    }
}

// Selection for window w (one block, K <= 256 threads, thread t = bin t).
// With c and q the count and the sum (units of 2^-16) cumulated over the
// bins up to k, A = (N - 2c) 2^16 + q and B = N_det - c are exact 64-bit
// integers, S_i(lambda_k) = A 2^-16 + lambda_k^2 B; their prefixes over the
// components give T(r, k) = PA 2^-16 + lambda_k^2 PB + sum_{i>r} S_inf[i].
__global__ void __launch_bounds__(kWdThreads)
win_sure_select_kernel(const unsigned int* __restrict__ counts, const double* __restrict__ sums,
                       const double* __restrict__ sum_all, const WinDesc* __restrict__ desc,
                       int r, int levels, int K, int* __restrict__ rank_out,
                       double* __restrict__ lam_out, hyde_hyres_info* __restrict__ info,
                       const int* __restrict__ status, const int* __restrict__ gstatus) {
    pdl_wait();
    pdl_trigger();
    __shared__ long long wc[kWdThreads / 32], wq[kWdThreads / 32];
    __shared__ double sinf[kMaxRank], tail[kMaxRank];
    __shared__ long long wm1[kWdThreads / 32], wm2[kWdThreads / 32];
    __shared__ int wi1[kWdThreads / 32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int wi = blockIdx.x;
    const WinDesc d = desc[wi];
    const long long N = (long long)d.Hp * d.Wp;
    const long long N_det = N - (long long)(d.Hp >> levels) * (d.Wp >> levels);
    const double delta = d.delta;
    if (t < r) sinf[t] = sum_all[(long long)wi * r + t] - (double)N;
    __syncthreads();
    if (t < r) {   // tail[t] = sum_{i > t} S_inf[i], added from i = r - 1 down
        double acc = 0.0;
        for (int q = r - 1; q > t; --q) acc += sinf[q];
        tail[t] = acc;
    }
    const double lam = t * delta, lam2 = lam * lam;
    long long PA = 0, PB = 0;
    long long m1 = 0x7fffffffffffffffLL, m2 = 0x7fffffffffffffffLL;
    int i1 = 0x7fffffff;
    for (int i = 0; i < r; ++i) {
        const long long row = ((long long)wi * r + i) * K;
        long long c = 0, q = 0;
        if (t < K) {
            c = counts[row + t];
            q = (long long)(sums[row + t] * 65536.0);   // exact
        }
        // inclusive block scan of (c, q) over the bins
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long c2 = __shfl_up_sync(0xffffffffu, c, o);
            const long long q2 = __shfl_up_sync(0xffffffffu, q, o);
            if (lane >= o) { c += c2; q += q2; }
        }
        __syncthreads();   // the previous row's warp totals have been read
        if (lane == 31) { wc[wid] = c; wq[wid] = q; }
        __syncthreads();
        for (int w = 0; w < wid; ++w) { c += wc[w]; q += wq[w]; }
        if (t < K) {
            PA += (N - 2 * c) * 65536LL + q;
            PB += N_det - c;
            const double v = fma(lam2, (double)PB, (double)PA * (1.0 / 65536.0)) + tail[i];
            keep_first_min2(ord_key(v), i * K + t, m1, m2, i1);
        }
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
        for (int q = 1; q < kWdThreads / 32; ++q) {
            if (wm1[q] < m1 || (wm1[q] == m1 && wi1[q] < i1)) {
                m2 = min(m1, wm2[q]); m1 = wm1[q]; i1 = wi1[q];
            } else {
                m2 = min(m2, wm1[q]);
            }
        }
        const int rr = i1 / K, k = i1 % K;
        const double v1 = key_value(m1), v2 = key_value(m2);
        rank_out[wi] = rr + 1;
        lam_out[wi] = k * delta;
        if (info) {
            const int st = status[wi] ? status[wi] : *gstatus;
            hyde_hyres_info& o = info[wi];
            o.status = st;
            o.rank = rr + 1;
            o.lambda_index = k;
            o.reserved = 0;
            o.lambda = k * delta;
            o.sure_min = v1;
            o.sure_gap = (r * K > 1) ? (v2 - v1) / fmax(fabs(v1), 1e-300) : 0.0;
        }
    }
}

// Synthesis of component i < r*_w of window w, levels L..1, the detail
// coefficients soft-thresholded at lambda*_w on load. Thread (j, k) of a
// level reads rows j and j - 1, columns k and k - 1 (mod the band size) of
// the four bands and writes output pixels 2j, 2j + 1 x 2k, 2k + 1: columns
// first (even and odd output rows), then rows.
__global__ void __launch_bounds__(kWdThreads)
win_idwt_kernel(const float* __restrict__ coef, float* __restrict__ Zh,
                float* __restrict__ scratch, const WinDesc* __restrict__ desc, int levels,
                const int* __restrict__ rank, const double* __restrict__ lam) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x, wi = blockIdx.y;
    if (i >= rank[wi]) return;
    const WinDesc d = desc[wi];
    const float lv = (float)lam[wi];
    const int N = d.Hp * d.Wp;
    const float* C = coef + d.img + (long long)i * N;
    float* A = scratch + d.scr + (long long)i * win_scratch_stride(N);
    float* B = A + N / 4;
    for (int l = levels; l >= 1; --l) {
        const int h = d.Hp >> (l - 1), w = d.Wp >> (l - 1), hh = h >> 1, wh = w >> 1;
        // LL_l: the coefficient image at l = L, else level l + 1's output
        const float* L = l == levels ? C : (((l + 1) & 1) ? B : A);
        const int lld = l == levels ? d.Wp : wh;
        float* O = l == 1 ? Zh + d.img + (long long)i * N : ((l & 1) ? B : A);
        const int old = l == 1 ? d.Wp : w;
        // the finest level writes only the 2 x 2 output blocks that meet the
        // core (the back-projection reads nothing else); coarser levels all
        const int jlo = l == 1 ? (d.cy0 - d.y0) >> 1 : 0;
        const int klo = l == 1 ? (d.cx0 - d.x0) >> 1 : 0;
        const int jn = l == 1 ? ((d.cy0 - d.y0 + d.ch + 1) >> 1) - jlo : hh;
        const int kn = l == 1 ? ((d.cx0 - d.x0 + d.cw + 1) >> 1) - klo : wh;
        for (int e = threadIdx.x; e < jn * kn; e += kWdThreads) {
            const int j = jlo + e / kn, k = klo + (e - (e / kn) * kn);
            const int jm = j == 0 ? hh - 1 : j - 1, km = k == 0 ? wh - 1 : k - 1;
            auto ll = [&](int y, int x) {
                return l == levels ? __ldg(L + (long long)y * lld + x)
                                   : __ldcg(L + (long long)y * lld + x);
            };
            auto hl = [&](int y, int x) { return softf(__ldg(C + (long long)y * d.Wp + wh + x), lv); };
            auto lh = [&](int y, int x) {
                return softf(__ldg(C + (long long)(hh + y) * d.Wp + x), lv);
            };
            auto hhb = [&](int y, int x) {
                return softf(__ldg(C + (long long)(hh + y) * d.Wp + wh + x), lv);
            };
            float le[2], lo[2], he[2], ho[2];   // [0]: column k, [1]: column k - 1
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int c = q == 0 ? k : km;
                const float a0 = ll(j, c), a1 = ll(jm, c);
                const float b0 = lh(j, c), b1 = lh(jm, c);
                const float c0 = hl(j, c), c1 = hl(jm, c);
                const float d0 = hhb(j, c), d1 = hhb(jm, c);
                le[q] = kH0 * a0 + kG0 * b0 + kH2 * a1 + kG2 * b1;
                lo[q] = kH1 * a0 + kG1 * b0 + kH3 * a1 + kG3 * b1;
                he[q] = kH0 * c0 + kG0 * d0 + kH2 * c1 + kG2 * d1;
                ho[q] = kH1 * c0 + kG1 * d0 + kH3 * c1 + kG3 * d1;
            }
            float* r0 = O + (long long)(2 * j) * old + 2 * k;
            float* r1 = r0 + old;
            r0[0] = kH0 * le[0] + kG0 * he[0] + kH2 * le[1] + kG2 * he[1];
            r0[1] = kH1 * le[0] + kG1 * he[0] + kH3 * le[1] + kG3 * he[1];
            r1[0] = kH0 * lo[0] + kG0 * ho[0] + kH2 * lo[1] + kG2 * ho[1];
            r1[1] = kH1 * lo[0] + kG1 * ho[0] + kH3 * lo[1] + kG3 * ho[1];
        }
        __syncthreads();
    }
}

}  // namespace

hyde_status launch_win_dwt(const float* Zp, float* coef, float* scratch, const WinDesc* desc,
                           int n_win, int r, int levels, int K, unsigned int* counts,
                           double* sums, double* sum_all, cudaStream_t s) {
    if (n_win < 1 || n_win > 65535 || r < 1 || levels < 1 || K < 2 || K > kWdThreads)
        return HYDE_ERR_SHAPE;
    const size_t smem = (size_t)2 * K * 32 * sizeof(unsigned int);
    if (ensure_smem_limit((const void*)win_dwt_kernel, (int)smem) != cudaSuccess)
        return HYDE_ERR_CUDA;
    launch_pdl(win_dwt_kernel, dim3(r, n_win), kWdThreads, smem, s, Zp, coef, scratch, desc,
               levels, r, K, counts, sums, sum_all);
    return cuda_status(cudaGetLastError());
}

hyde_status launch_win_sure(const WinDesc* desc, int n_win, int r, int levels, int K,
                            const unsigned int* counts, const double* sums,
                            const double* sum_all, int* rank, double* lam, hyde_hyres_info* info,
                            const int* status, const int* gstatus, cudaStream_t s) {
    if (n_win < 1 || n_win > 65535 || r < 1 || r > kMaxRank || K < 2 || K > kWdThreads)
        return HYDE_ERR_SHAPE;
    launch_pdl(win_sure_select_kernel, n_win, kWdThreads, 0, s, counts, sums, sum_all, desc, r,
               levels, K, rank, lam, info, status, gstatus);
    return cuda_status(cudaGetLastError());
}

hyde_status launch_win_idwt(const float* coef, float* Zh, float* scratch, const WinDesc* desc,
                            int n_win, int r, int levels, const int* rank, const double* lam,
                            cudaStream_t s) {
    if (n_win < 1 || n_win > 65535 || r < 1 || levels < 1) return HYDE_ERR_SHAPE;
    launch_pdl(win_idwt_kernel, dim3(r, n_win), kWdThreads, 0, s, coef, Zh, scratch, desc,
               levels, rank, lam);
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

// Separable periodic db2 wavelet transform of a batch of images (the spatial
// sparsifying basis of HyRes, "wavelet-based", arXiv 2204.06979 Sec. 2.1),
// and its transpose with the soft threshold fused into the coefficient load.
//
// One level of analysis on an h x w image:
//   rows:    a_k = sum_m h_m x[(2k+m) mod w],  d_k = sum_m g_m x[(2k+m) mod w]
//   columns: the same filters along y on both row outputs,
// giving LL (top-left), the row-detail band (top-right), the column-detail
// band (bottom-left) and the diagonal band. LL is recursed on.
//
// Every analysis level runs as a persistent pipeline (tiles of 16 x 64
// coefficients per band, the next tile streamed into shared memory while the
// current one is filtered: one TMA copy for an interior tile, cp.async
// through the halo; float4 filter passes); the first level of an unpadded
// image reads through the symmetric extension.
// Synthesis levels use one tile per block (16 x 32 coefficients) or the
// register form below. Details go straight to their Mallat position in the
// coefficient image; LL goes to a compact ping-pong buffer (or, at the last
// level, into the coefficient image), so no level reads what another block
// of the same launch writes. (A pipelined synthesis with the same structure
// as the analysis measured slower on the 20 x 352 x 1920 components: its
// blocks hold too few tiles to hide the first load.)
#include <cuda.h>
#include <string.h>

#include "hyde_internal.cuh"
#include "tc_common.cuh"
#include "tmap.cuh"

namespace hyde {
namespace {

constexpr int TH = 16, TW = 32;            // coefficient tile per subband
constexpr int kThreads = 256;

// v in [0, m + tile) -> v mod m, with the division only for tiny images
__device__ __forceinline__ int wrap(int v, int m) {
    if (v < m) return v;
    v -= m;
    return v < m ? v : v % m;
}

// --------------------------------------------------------------------------
// Analysis level as a persistent pipeline: block (g, image) walks tiles
// g, g + G, ... of one image, 16 x 64 coefficients per subband each, from a
// 34 x 132 input tile (rows and columns past the valid hv x wv source are
// read through the whole-sample symmetric extension).
// The next tile streams into the other half of a double buffer while the
// current one is filtered: the row pass reads 10 inputs and writes 4 outputs
// per thread as float4, the column pass forms the four subbands of 4
// coefficients per thread and stores them as float4 rows.
// Interior tiles (the whole 34 x 132 box inside the valid source) are one
// TMA copy (a 3D tensor map over width, height and image; x = 2 tx0 is a
// multiple of 128 floats), completed on the buffer's mbarrier. Tiles that
// meet the halo (periodic wrap of the padded image, symmetric extension of
// an unpadded one) are gathered with cp.async instead: 16-byte copies where
// the row is 16-byte aligned and the chunk stays inside the valid width,
// 4-byte copies through the wrap and the reflection elsewhere.
// --------------------------------------------------------------------------
constexpr int FTH = 16, FTW = 64;           // coefficients per subband per tile
constexpr int FIH = 2 * FTH + 2;            // input rows
constexpr int FIW = 2 * FTW + 4;            // input columns (2 FTW + 2 used, multiple of 4)
constexpr int FIBUF = 4512;                 // buffer stride in floats (FIH FIW rounded to 128 B)
constexpr int kFThreads = 256;
constexpr uint32_t kTileBytes = FIH * FIW * sizeof(float);
static_assert(FIBUF >= FIH * FIW && (FIBUF * sizeof(float)) % 128 == 0, "buffer stride");
static_assert((FIW * sizeof(float)) % 16 == 0 && FIW <= 256 && FIH <= 256, "TMA box");

__device__ __forceinline__ void cpa16(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cpa4(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__global__ void __launch_bounds__(kFThreads)
dwt_level_pipe_kernel(const __grid_constant__ CUtensorMap tmap, int use_tma,
                      unsigned long long wait_ns, int* __restrict__ status,
                      const float* __restrict__ src, long long src_bs, int src_ld, int hv,
                      int wv, int h, int w, float* __restrict__ coef, long long coef_bs,
                      int coef_ld, float* __restrict__ ll, long long ll_bs, int ll_ld) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float4 fsm4[];
    __shared__ __align__(8) uint64_t full[2];          // TMA completion, one per buffer
    // the TMA destination wants 128-byte alignment: round the dynamic base up
    const uint32_t base_s = smem_u32(fsm4);
    float* inb = reinterpret_cast<float*>(reinterpret_cast<char*>(fsm4) +
                                          (((base_s + 127u) & ~127u) - base_s));   // [2][FIBUF]
    float* ra = inb + 2 * FIBUF;                      // [FIH][FTW]
    float* rd = ra + FIH * FTW;                       // [FIH][FTW]
    const int tid = threadIdx.x;
    if (use_tma && tid == 0) {
        mbar_init(smem_u32(&full[0]), 1);
        mbar_init(smem_u32(&full[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap))
                     : "memory");
    }
    __syncthreads();
    const int b = blockIdx.y, G = gridDim.x;
    const int hh = h >> 1, wh = w >> 1;
    const int tiles_x = (wh + FTW - 1) / FTW, tiles_y = (hh + FTH - 1) / FTH;
    const int ntiles = tiles_x * tiles_y;
    const float* S = src + (long long)b * src_bs;
    float* CB = coef + (long long)b * coef_bs;
    float* LB = ll + (long long)b * ll_bs;
    const bool vin = (src_ld & 3) == 0 && ((reinterpret_cast<uintptr_t>(S) & 15) == 0);
    const bool vout = (wh & 3) == 0 && (coef_ld & 3) == 0 && (ll_ld & 3) == 0 &&
                      ((reinterpret_cast<uintptr_t>(CB) & 15) == 0) &&
                      ((reinterpret_cast<uintptr_t>(LB) & 15) == 0);

    // tma_pend bit j: the tile in buffer j is a TMA copy not yet waited for;
    // phase bit j: the parity that buffer j's barrier completes next
    unsigned tma_pend = 0, phase = 0;
    auto load_tile = [&](int t, int buf) {
        const int ty0 = (t / tiles_x) * FTH, tx0 = (t % tiles_x) * FTW;
        float* in = inb + buf * FIBUF;
        if (use_tma && 2 * tx0 + FIW <= wv && 2 * ty0 + FIH <= hv) {
            if (tid == 0) {
                // the buffer's last generic reads finished before the block
                // barrier that precedes this call; order them before the copy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const uint32_t bar = smem_u32(&full[buf]);
                mbar_arrive_expect_tx(bar, kTileBytes);
                tma_load_3d(smem_u32(in), &tmap, 2 * tx0, 2 * ty0, b, bar);
            }
            tma_pend |= 1u << buf;
            return;
        }
        for (int e = tid; e < FIH * (FIW / 4); e += kFThreads) {
            const int r = e / (FIW / 4), cq = e - r * (FIW / 4);
            int y = wrap(2 * ty0 + r, h);
            if (y >= hv) y = 2 * hv - 2 - y;   // symmetric extension of an unpadded source
            const float* row = S + (long long)y * src_ld;
            const int x0 = 2 * tx0 + 4 * cq;
            float* d = in + r * FIW + 4 * cq;
            if (vin && x0 + 3 < wv) {
                cpa16(d, row + x0);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    int x = wrap(x0 + u, w);
                    if (x >= wv) x = 2 * wv - 2 - x;
                    cpa4(d + u, row + x);
                }
            }
        }
    };

    int t = blockIdx.x;
    if (t < ntiles) load_tile(t, 0);
    cpa_commit();
    for (int it = 0; t < ntiles; ++it, t += G) {
        const int buf = it & 1;
        if (t + G < ntiles) load_tile(t + G, buf ^ 1);
        cpa_commit();
        cpa_wait<1>();
        int late = 0;
        if (tma_pend & (1u << buf)) {
            late = !mbar_wait_bounded(smem_u32(&full[buf]), (phase >> buf) & 1u, wait_ns);
            tma_pend &= ~(1u << buf);
            phase ^= 1u << buf;
        }
        // tile t landed; the previous column pass is done
        if (__syncthreads_or(late)) {
            // a copy did not complete in time: report it, let the copies
            // still in flight land (bounded by the default limit, whatever
            // the configured one, so that none outlives the block), and stop
            if (tid == 0) {
                set_status(status, HYDE_ERR_TIMEOUT);
                if (late)   // this buffer's copy, whose phase was already passed on
                    mbar_wait_bounded(smem_u32(&full[buf]), ((phase >> buf) & 1u) ^ 1u, kWaitNs);
                if (tma_pend & (1u << (buf ^ 1)))
                    mbar_wait_bounded(smem_u32(&full[buf ^ 1]), (phase >> (buf ^ 1)) & 1u,
                                      kWaitNs);
            }
            cpa_wait<0>();
            return;
        }
        const float* in = inb + buf * FIBUF;
        for (int e = tid; e < FIH * (FTW / 4); e += kFThreads) {
            const int r = e / (FTW / 4), kq = e - r * (FTW / 4);
            const float* ir = in + r * FIW + 8 * kq;
            const float4 v0 = *reinterpret_cast<const float4*>(ir);
            const float4 v1 = *reinterpret_cast<const float4*>(ir + 4);
            const float2 v2 = *reinterpret_cast<const float2*>(ir + 8);
            const float x[10] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y};
            float a[4], d[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = kH0 * x[2 * u] + kH1 * x[2 * u + 1] + kH2 * x[2 * u + 2] + kH3 * x[2 * u + 3];
                d[u] = kG0 * x[2 * u] + kG1 * x[2 * u + 1] + kG2 * x[2 * u + 2] + kG3 * x[2 * u + 3];
            }
            *reinterpret_cast<float4*>(ra + r * FTW + 4 * kq) = make_float4(a[0], a[1], a[2], a[3]);
            *reinterpret_cast<float4*>(rd + r * FTW + 4 * kq) = make_float4(d[0], d[1], d[2], d[3]);
        }
        __syncthreads();   // row outputs complete; buffer `buf` may be refilled
        const int ty0 = (t / tiles_x) * FTH, tx0 = (t % tiles_x) * FTW;
        const int j = tid / (FTW / 4), kq = tid - j * (FTW / 4);
        const int J = ty0 + j, Kc = tx0 + 4 * kq;
        if (J < hh && Kc < wh) {
            float4 A[4], D[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                A[m] = *reinterpret_cast<const float4*>(ra + (2 * j + m) * FTW + 4 * kq);
                D[m] = *reinterpret_cast<const float4*>(rd + (2 * j + m) * FTW + 4 * kq);
            }
            auto comb = [](const float4 (&V)[4], float c0, float c1, float c2, float c3) {
                return make_float4(c0 * V[0].x + c1 * V[1].x + c2 * V[2].x + c3 * V[3].x,
                                   c0 * V[0].y + c1 * V[1].y + c2 * V[2].y + c3 * V[3].y,
                                   c0 * V[0].z + c1 * V[1].z + c2 * V[2].z + c3 * V[3].z,
                                   c0 * V[0].w + c1 * V[1].w + c2 * V[2].w + c3 * V[3].w);
            };
            const float4 LL = comb(A, kH0, kH1, kH2, kH3);
            const float4 LH = comb(A, kG0, kG1, kG2, kG3);   // column detail
            const float4 HL = comb(D, kH0, kH1, kH2, kH3);   // row detail
            const float4 HH = comb(D, kG0, kG1, kG2, kG3);
            float* pLL = LB + (long long)J * ll_ld + Kc;
            float* pHL = CB + (long long)J * coef_ld + wh + Kc;
            float* pLH = CB + (long long)(hh + J) * coef_ld + Kc;
            float* pHH = CB + (long long)(hh + J) * coef_ld + wh + Kc;
            if (vout) {
                *reinterpret_cast<float4*>(pLL) = LL;
                *reinterpret_cast<float4*>(pHL) = HL;
                *reinterpret_cast<float4*>(pLH) = LH;
                *reinterpret_cast<float4*>(pHH) = HH;
            } else {
                const float ll4[4] = {LL.x, LL.y, LL.z, LL.w}, hl4[4] = {HL.x, HL.y, HL.z, HL.w};
                const float lh4[4] = {LH.x, LH.y, LH.z, LH.w}, hh4[4] = {HH.x, HH.y, HH.z, HH.w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (Kc + q < wh) {
                        pLL[q] = ll4[q];
                        pHL[q] = hl4[q];
                        pLH[q] = lh4[q];
                        pHH[q] = hh4[q];
                    }
            }
        }
    }
    cpa_wait<0>();
}

__device__ __forceinline__ float soft(float c, float lam) {
    return copysignf(fmaxf(fabsf(c) - lam, 0.f), c);
}

// Synthesis of one level: coefficients of an (h/2 x w/2) x 4 layout -> an
// h x w image, written only where y < ho and x < wo (crop at the last level).
// Output rows 2j and 2j+1 draw on coefficient rows j and j-1 (mod h/2):
//   x[2j]   = h0 a_j + g0 d_j + h2 a_{j-1} + g2 d_{j-1}
//   x[2j+1] = h1 a_j + g1 d_j + h3 a_{j-1} + g3 d_{j-1}
__global__ void __launch_bounds__(kThreads)
idwt_level_kernel(const float* __restrict__ llsrc, long long ll_bs, int ll_ld,
                  const float* __restrict__ coef, long long coef_bs, int coef_ld, int h,
                  int w, const double* __restrict__ lam, const float* __restrict__ scale,
                  int scale_ld, int lev, const int* __restrict__ rank,
                  float* __restrict__ out, long long out_bs, int out_ld, int ho, int wo,
                  int llt) {
    pdl_wait();
    pdl_trigger();
    __shared__ float sLL[TH + 1][TW + 2], sLH[TH + 1][TW + 2];
    __shared__ float sHL[TH + 1][TW + 2], sHH[TH + 1][TW + 2];
    __shared__ float tl[2 * TH][TW + 2], th[2 * TH][TW + 2];
    const int b = blockIdx.z;
    if (rank && b >= *rank) return;
    // threshold of this level's detail bands: lambda (* scale[image][level])
    float lv = lam ? (float)(*lam) : 0.f;
    if (lam && scale) lv *= scale[(long long)b * scale_ld + (lev - 1)];
    const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;
    const int hh = h >> 1, wh = w >> 1;
    const float* L = llsrc + (long long)b * ll_bs;
    const float* C = coef + (long long)b * coef_bs;
    constexpr int kLoadSteps = ((TH + 1) * (TW + 1) + kThreads - 1) / kThreads;
#pragma unroll
    for (int q = 0; q < kLoadSteps; ++q) {
        const int e = threadIdx.x + q * kThreads;
        if (e >= (TH + 1) * (TW + 1)) break;
        const int j = e / (TW + 1), k = e % (TW + 1);
        const int J = ty0 + j == 0 ? hh - 1 : wrap(ty0 + j - 1, hh);
        const int K = tx0 + k == 0 ? wh - 1 : wrap(tx0 + k - 1, wh);
        const float ll = L[(long long)J * ll_ld + K];
        sLL[j][k] = llt ? soft(ll, lv) : ll;
        const float hl = C[(long long)J * coef_ld + wh + K];
        const float lh = C[(long long)(hh + J) * coef_ld + K];
        const float hhv = C[(long long)(hh + J) * coef_ld + wh + K];
        sHL[j][k] = soft(hl, lv);
        sLH[j][k] = soft(lh, lv);
        sHH[j][k] = soft(hhv, lv);
    }
    __syncthreads();
    // columns: local output row y (0..2TH-1) from coefficient rows y/2 (+1 in smem)
    for (int e = threadIdx.x; e < 2 * TH * (TW + 1); e += kThreads) {
        const int y = e / (TW + 1), k = e % (TW + 1);
        const int j = (y >> 1) + 1;
        float l, hgh;
        if ((y & 1) == 0) {
            l = kH0 * sLL[j][k] + kG0 * sLH[j][k] + kH2 * sLL[j - 1][k] + kG2 * sLH[j - 1][k];
            hgh = kH0 * sHL[j][k] + kG0 * sHH[j][k] + kH2 * sHL[j - 1][k] + kG2 * sHH[j - 1][k];
        } else {
            l = kH1 * sLL[j][k] + kG1 * sLH[j][k] + kH3 * sLL[j - 1][k] + kG3 * sLH[j - 1][k];
            hgh = kH1 * sHL[j][k] + kG1 * sHH[j][k] + kH3 * sHL[j - 1][k] + kG3 * sHH[j - 1][k];
        }
        tl[y][k] = l;
        th[y][k] = hgh;
    }
    __syncthreads();
    float* O = out + (long long)b * out_bs;
    for (int e = threadIdx.x; e < 2 * TH * 2 * TW; e += kThreads) {
        const int y = e / (2 * TW), x = e % (2 * TW);
        const int Y = 2 * ty0 + y, X = 2 * tx0 + x;
        if (Y >= ho || X >= wo) continue;
        const int k = (x >> 1) + 1;
        float v;
        if ((x & 1) == 0)
            v = kH0 * tl[y][k] + kG0 * th[y][k] + kH2 * tl[y][k - 1] + kG2 * th[y][k - 1];
        else
            v = kH1 * tl[y][k] + kG1 * th[y][k] + kH3 * tl[y][k - 1] + kG3 * th[y][k - 1];
        O[(long long)Y * out_ld + X] = v;
    }
}

// --------------------------------------------------------------------------
// Synthesis of one level, register form: lane l of a warp owns coefficient
// columns k0 = 128 s + 4 l .. k0 + 3 of a 128-column strip s and walks
// kSynRows coefficient rows down it, keeping the previous row's four bands in
// registers, so every coefficient is loaded once (float4, soft threshold on
// load) and column k0 - 1 comes from the left lane by a shuffle (lane 0
// loads it). Per coefficient row j the lane forms output rows 2j and 2j + 1
// at columns 2 k0 .. 2 k0 + 7. Output rows that are 16-byte aligned take
// float4 stores; otherwise (the cropped last level, row length W) the two
// rows go through a per-warp shared buffer so that each store instruction
// writes 32 consecutive floats.
// --------------------------------------------------------------------------
constexpr int kSynRows = 4;
constexpr int kSynThreads = 256;
constexpr int kSynWarps = kSynThreads / 32;

__device__ __forceinline__ float4 soft4(float4 v, float lam) {
    return make_float4(soft(v.x, lam), soft(v.y, lam), soft(v.z, lam), soft(v.w, lam));
}

// One (strip, run) unit of the register-form synthesis for the calling warp.
// L is the LL band (global memory when LLG, else shared memory), C the
// component's coefficient image; st0/st1 the warp's staging rows (used when
// !vout). llt: the LL band is soft-thresholded at lv too (the final LL band
// in the variant that thresholds every coefficient).
template <bool LLG, int ROWS>
__device__ __forceinline__ void syn_unit(const float* L, int ll_ld, const float* __restrict__ C,
                                         int coef_ld, int hh, int wh, float lv, bool llt,
                                         int strip,
                                         int run, float* O, int out_ld, int ho, int wo,
                                         bool vout, float4* st0, float4* st1, int lane) {
    const int k0 = strip * 128 + 4 * lane;
    const bool active = k0 < wh;        // wh is a multiple of 4: the lane's 4 columns exist
    const int kc = active ? k0 : 0;
    const int km1 = (strip == 0 ? wh : strip * 128) - 1;
    auto ldl4 = [&](long long off) {
        return LLG ? __ldg(reinterpret_cast<const float4*>(L + off))
                   : *reinterpret_cast<const float4*>(L + off);
    };
    auto ldl1 = [&](long long off) { return LLG ? __ldg(L + off) : L[off]; };
    // bands in the order LL, LH (column detail), HL (row detail), HH
    auto load_row = [&](int J, float4 (&v)[4], float (&left)[4]) {
        const long long rl = (long long)J * ll_ld, rt = (long long)J * coef_ld,
                        rb = (long long)(hh + J) * coef_ld;
        v[0] = ldl4(rl + kc);
        if (llt) v[0] = soft4(v[0], lv);
        v[1] = soft4(__ldg(reinterpret_cast<const float4*>(C + rb + kc)), lv);
        v[2] = soft4(__ldg(reinterpret_cast<const float4*>(C + rt + wh + kc)), lv);
        v[3] = soft4(__ldg(reinterpret_cast<const float4*>(C + rb + wh + kc)), lv);
        float e0 = 0.f, e1 = 0.f, e2 = 0.f, e3 = 0.f;
        if (lane == 0) {
            e0 = ldl1(rl + km1);
            if (llt) e0 = soft(e0, lv);
            e1 = soft(__ldg(C + rb + km1), lv);
            e2 = soft(__ldg(C + rt + wh + km1), lv);
            e3 = soft(__ldg(C + rb + wh + km1), lv);
        }
        left[0] = __shfl_up_sync(0xffffffffu, v[0].w, 1);
        left[1] = __shfl_up_sync(0xffffffffu, v[1].w, 1);
        left[2] = __shfl_up_sync(0xffffffffu, v[2].w, 1);
        left[3] = __shfl_up_sync(0xffffffffu, v[3].w, 1);
        if (lane == 0) { left[0] = e0; left[1] = e1; left[2] = e2; left[3] = e3; }
    };
    const int j0 = run * ROWS;
    float4 pv[4];
    float pl[4];
    load_row(j0 == 0 ? hh - 1 : j0 - 1, pv, pl);
    const int X0 = 2 * k0;
#pragma unroll
    for (int s = 0; s < ROWS; ++s) {
        const int j = j0 + s;
        if (j >= hh) break;   // warp-uniform
        float4 cv[4];
        float cl[4];
        load_row(j, cv, cl);
        // column pass on the five columns k0 - 1 .. k0 + 3
        float le[5], lo[5], he[5], hq[5];
        auto col = [&](int c, float cLL, float cLH, float cHL, float cHH, float pLL, float pLH,
                       float pHL, float pHH) {
            le[c] = kH0 * cLL + kG0 * cLH + kH2 * pLL + kG2 * pLH;
            lo[c] = kH1 * cLL + kG1 * cLH + kH3 * pLL + kG3 * pLH;
            he[c] = kH0 * cHL + kG0 * cHH + kH2 * pHL + kG2 * pHH;
            hq[c] = kH1 * cHL + kG1 * cHH + kH3 * pHL + kG3 * pHH;
        };
        col(0, cl[0], cl[1], cl[2], cl[3], pl[0], pl[1], pl[2], pl[3]);
        col(1, cv[0].x, cv[1].x, cv[2].x, cv[3].x, pv[0].x, pv[1].x, pv[2].x, pv[3].x);
        col(2, cv[0].y, cv[1].y, cv[2].y, cv[3].y, pv[0].y, pv[1].y, pv[2].y, pv[3].y);
        col(3, cv[0].z, cv[1].z, cv[2].z, cv[3].z, pv[0].z, pv[1].z, pv[2].z, pv[3].z);
        col(4, cv[0].w, cv[1].w, cv[2].w, cv[3].w, pv[0].w, pv[1].w, pv[2].w, pv[3].w);
        // row pass: outputs 2k and 2k + 1 for k = k0 .. k0 + 3 (column index c = k - k0 + 1)
        float oe[8], oo[8];
#pragma unroll
        for (int c = 1; c <= 4; ++c) {
            oe[2 * c - 2] = kH0 * le[c] + kG0 * he[c] + kH2 * le[c - 1] + kG2 * he[c - 1];
            oe[2 * c - 1] = kH1 * le[c] + kG1 * he[c] + kH3 * le[c - 1] + kG3 * he[c - 1];
            oo[2 * c - 2] = kH0 * lo[c] + kG0 * hq[c] + kH2 * lo[c - 1] + kG2 * hq[c - 1];
            oo[2 * c - 1] = kH1 * lo[c] + kG1 * hq[c] + kH3 * lo[c - 1] + kG3 * hq[c - 1];
        }
        const int Y = 2 * j;
        if (vout) {
            if (active) {
                float* r0 = O + (long long)Y * out_ld + X0;
                float* r1 = r0 + out_ld;
                *reinterpret_cast<float4*>(r0) = make_float4(oe[0], oe[1], oe[2], oe[3]);
                *reinterpret_cast<float4*>(r0 + 4) = make_float4(oe[4], oe[5], oe[6], oe[7]);
                *reinterpret_cast<float4*>(r1) = make_float4(oo[0], oo[1], oo[2], oo[3]);
                *reinterpret_cast<float4*>(r1 + 4) = make_float4(oo[4], oo[5], oo[6], oo[7]);
            }
        } else {
            st0[2 * lane] = make_float4(oe[0], oe[1], oe[2], oe[3]);
            st0[2 * lane + 1] = make_float4(oe[4], oe[5], oe[6], oe[7]);
            st1[2 * lane] = make_float4(oo[0], oo[1], oo[2], oo[3]);
            st1[2 * lane + 1] = make_float4(oo[4], oo[5], oo[6], oo[7]);
            __syncwarp();
            const float* f0 = reinterpret_cast<const float*>(st0);
            const float* f1 = reinterpret_cast<const float*>(st1);
            const int xs = 256 * strip;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int X = xs + 32 * q + lane;
                if (X < wo) {
                    if (Y < ho) O[(long long)Y * out_ld + X] = f0[32 * q + lane];
                    if (Y + 1 < ho) O[(long long)(Y + 1) * out_ld + X] = f1[32 * q + lane];
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) { pv[q] = cv[q]; pl[q] = cl[q]; }
    }
}

__global__ void __launch_bounds__(kSynThreads)
idwt_level_vec_kernel(const float* __restrict__ llsrc, long long ll_bs, int ll_ld,
                      const float* __restrict__ coef, long long coef_bs, int coef_ld, int h,
                      int w, const double* __restrict__ lam, const float* __restrict__ scale,
                      int scale_ld, int lev, const int* __restrict__ rank,
                      float* __restrict__ out, long long out_bs, int out_ld, int ho, int wo,
                      int vout, int llt) {
    pdl_wait();
    pdl_trigger();
    __shared__ float4 stage4[kSynWarps][2][64];   // two output rows of 256 floats per warp
    const int b = blockIdx.y;
    if (rank && b >= *rank) return;
    float lv = lam ? (float)(*lam) : 0.f;
    if (lam && scale) lv *= scale[(long long)b * scale_ld + (lev - 1)];
    const int hh = h >> 1, wh = w >> 1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nstrips = (wh + 127) >> 7;
    const int nruns = (hh + kSynRows - 1) / kSynRows;
    const int u = blockIdx.x * kSynWarps + wid;
    if (u >= nstrips * nruns) return;   // whole warp
    syn_unit<true, kSynRows>(llsrc + (long long)b * ll_bs, ll_ld,
                             coef + (long long)b * coef_bs, coef_ld, hh, wh, lv, llt != 0,
                             u % nstrips,
                             u / nstrips, out + (long long)b * out_bs, out_ld, ho, wo, vout != 0,
                             stage4[wid][0], stage4[wid][1], lane);
}

// --------------------------------------------------------------------------
// The coarse levels in one block per component. Below a few tens of
// thousands of coefficients a level is all launch and ramp: one launch per
// level leaves most SMs idle while each of its blocks waits on its first
// load. These kernels run levels lo..hi of one component in one block (1024
// threads for the analysis, 768 for the synthesis), the intermediate LL bands
// in shared memory.
// --------------------------------------------------------------------------
constexpr int kTailThreads = 1024;
constexpr int kTailSynThreads = 768;   // 24 warps: the synthesis unit needs ~73 registers
// The tail starts at the first level with at most this many input values
// (analysis) or output values (synthesis) per component: below it a level on
// one SM costs less than a launch of its own (at C1, levels 4-5: the level-3
// input, 42k values, took 13.7 us on one SM against 4.5 us as its own launch).
constexpr int kTailMaxFloats = 12288;

// Analysis, levels lo..hi: the input LL_{lo-1} (h0 x w0) is loaded once; each
// thread forms the four subbands of one coefficient, consecutive lanes taking
// consecutive columns (float2 shared loads, no bank conflicts), the row filter
// recomputed for each of its 4 input rows (no row-pass buffer).
__global__ void __launch_bounds__(kTailThreads, 1)
dwt_tail_kernel(const float* __restrict__ src, long long src_bs, int src_ld, int Hp, int Wp,
                int lo, int hi, float* __restrict__ coef, long long coef_bs, int coef_ld) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float4 tail4[];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int h0 = Hp >> (lo - 1), w0 = Wp >> (lo - 1);
    float* A = reinterpret_cast<float*>(tail4);   // h0 x w0
    float* B = A + h0 * w0;                        // h0/2 x w0/2
    const float* S = src + (long long)b * src_bs;
    const int w4 = w0 >> 2;
    for (int e = tid; e < h0 * w4; e += kTailThreads) {
        const int y = e / w4, x4 = e - y * w4;
        reinterpret_cast<float4*>(A)[e] =
            __ldg(reinterpret_cast<const float4*>(S + (long long)y * src_ld) + x4);
    }
    __syncthreads();
    float* CB = coef + (long long)b * coef_bs;
    for (int l = lo; l <= hi; ++l) {
        const int h = Hp >> (l - 1), w = Wp >> (l - 1), hh = h >> 1, wh = w >> 1;
        const float* in = ((l - lo) & 1) ? B : A;
        float* ob = ((l - lo) & 1) ? A : B;
        for (int e = tid; e < hh * wh; e += kTailThreads) {
            const int J = e / wh, K = e - J * wh;
            const int x0 = 2 * K, x2 = (2 * K + 2 >= w) ? 2 * K + 2 - w : 2 * K + 2;
            float a[4], d[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                int y = 2 * J + m;
                if (y >= h) y -= h;
                const float* row = in + y * w;
                const float2 u = *reinterpret_cast<const float2*>(row + x0);
                const float2 v = *reinterpret_cast<const float2*>(row + x2);
                a[m] = kH0 * u.x + kH1 * u.y + kH2 * v.x + kH3 * v.y;
                d[m] = kG0 * u.x + kG1 * u.y + kG2 * v.x + kG3 * v.y;
            }
            const float LL = kH0 * a[0] + kH1 * a[1] + kH2 * a[2] + kH3 * a[3];
            const float LH = kG0 * a[0] + kG1 * a[1] + kG2 * a[2] + kG3 * a[3];
            const float HL = kH0 * d[0] + kH1 * d[1] + kH2 * d[2] + kH3 * d[3];
            const float HH = kG0 * d[0] + kG1 * d[1] + kG2 * d[2] + kG3 * d[3];
            float* pt = CB + (long long)J * coef_ld;
            float* pb = CB + (long long)(hh + J) * coef_ld;
            pt[wh + K] = HL;
            pb[K] = LH;
            pb[wh + K] = HH;
            if (l == hi) pt[K] = LL;
            else ob[J * wh + K] = LL;
        }
        __syncthreads();
    }
}

// Synthesis, levels hi..lo: the LL band of level l > lo goes to shared memory
// (level lo+1 into A, then alternating), level lo writes LL_{lo-1} to `out`
// (row stride Wp >> (lo-1), 16-byte aligned rows). Warps take the (strip,
// run) units of a level in turn, one coefficient row each.
__global__ void __launch_bounds__(kTailSynThreads, 1)
idwt_tail_kernel(const float* __restrict__ coef, long long coef_bs, int coef_ld, int Hp, int Wp,
                 int lo, int hi, const double* __restrict__ lam, const float* __restrict__ scale,
                 int scale_ld, const int* __restrict__ rank, float* __restrict__ out,
                 long long out_bs, int llt) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float4 tail4[];
    const int b = blockIdx.x;
    if (rank && b >= *rank) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float* A = reinterpret_cast<float*>(tail4);          // (Hp >> lo) x (Wp >> lo)
    float* B = A + (Hp >> lo) * (Wp >> lo);               // a quarter of A
    const float* C = coef + (long long)b * coef_bs;
    const float lam0 = lam ? (float)(*lam) : 0.f;
    for (int l = hi; l >= lo; --l) {
        const int h = Hp >> (l - 1), w = Wp >> (l - 1), hh = h >> 1, wh = w >> 1;
        float lv = lam0;
        if (lam && scale) lv *= scale[(long long)b * scale_ld + (l - 1)];
        float* O = (l == lo) ? out + (long long)b * out_bs : (((l - lo) & 1) ? A : B);
        const int nstrips = (wh + 127) >> 7;
        const int units = nstrips * hh;   // one coefficient row per unit: more warps busy
        for (int u = wid; u < units; u += kTailSynThreads / 32) {
            if (l == hi)
                syn_unit<true, 1>(C, coef_ld, C, coef_ld, hh, wh, lv, llt != 0, u % nstrips,
                                  u / nstrips, O, w, h, w, true, nullptr, nullptr, lane);
            else
                syn_unit<false, 1>(((l + 1 - lo) & 1) ? A : B, wh, C, coef_ld, hh, wh, lv,
                                false, u % nstrips, u / nstrips, O, w, h, w, true, nullptr, nullptr,
                                lane);
        }
        __syncthreads();
    }
}

}  // namespace

size_t dwt_scratch_floats(int Hp, int Wp) {
    size_t N = (size_t)Hp * Wp;
    return N / 4 + N / 16;
}

// LL of level j (1-based, size (Hp>>j) x (Wp>>j)) lives in half A (odd j)
// or half B (even j) of the per-image scratch.
static inline float* ll_buf(float* scratch, int batch, int Hp, int Wp, int j,
                            long long* bs) {
    size_t N = (size_t)Hp * Wp;
    if (j & 1) { *bs = (long long)(N / 4); return scratch; }
    *bs = (long long)(N / 16);
    return scratch + (size_t)batch * (N / 4);
}

// First level of the fused coarse tail: the smallest lo >= 2 whose level-lo
// input (analysis) / output (synthesis), (Hp >> (lo-1)) x (Wp >> (lo-1)),
// has at most kTailMaxFloats values, provided every tail level keeps its
// half-width a multiple of 4 (float4 rows); levels + 1 when there is none.
static int tail_first_level(int Hp, int Wp, int levels) {
    if (levels < 2 || (Wp & 3) != 0 || ((Wp >> levels) & 3) != 0) return levels + 1;
    for (int lo = 2; lo <= levels; ++lo)
        if ((long long)(Hp >> (lo - 1)) * (Wp >> (lo - 1)) <= kTailMaxFloats) return lo;
    return levels + 1;
}

int dwt_launches(int Hp, int Wp, int levels) {
    const int lo = tail_first_level(Hp, Wp, levels);
    return lo <= levels ? lo : levels;   // lo - 1 single levels and the fused tail
}

static inline bool aligned16(const void* p) {
    return (reinterpret_cast<uintptr_t>(p) & 15) == 0;
}

// Tensor map of the TMA copies of the interior tiles of one analysis level:
// the source as width x height x image (floats), box FIW x FIH x 1. False
// (cp.async for every tile) where the layout does not allow it: a base or a
// row or image stride not a multiple of 16 bytes, a source smaller than the
// box, or no encoder in the driver.
static bool dwt_tmap(const float* sp, long long sbs, int sld, int hv, int wv, int batch,
                     CUtensorMap* tm) {
    if ((reinterpret_cast<uintptr_t>(sp) & 15) != 0 || (sld & 3) != 0 || (sbs & 3) != 0 ||
        wv < FIW || hv < FIH || sld < wv || sbs < (long long)sld * hv)
        return false;
    EncodeTiledFn enc = encode_tiled_fn();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)wv, (cuuint64_t)hv, (cuuint64_t)batch};
    const cuuint64_t strides[2] = {(cuuint64_t)sld * sizeof(float),
                                   (cuuint64_t)sbs * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)FIW, (cuuint32_t)FIH, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(sp), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

hyde_status launch_dwt2(const DwtSrc& src, float* coef, int batch, int Hp, int Wp,
                        int levels, float* scratch, cudaStream_t s, int* status) {
    const long long cbs = (long long)Hp * Wp;
    const size_t pipe_smem = (size_t)(2 * FIBUF + 2 * FIH * FTW) * sizeof(float) + 128;
    if (ensure_smem_limit((const void*)dwt_level_pipe_kernel, (int)pipe_smem) != cudaSuccess)
        return HYDE_ERR_CUDA;
    const int sms = device_sm_count();
    if (sms <= 0) return HYDE_ERR_CUDA;
    int pipe_per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pipe_per_sm, dwt_level_pipe_kernel,
                                                      kFThreads, pipe_smem) != cudaSuccess ||
        pipe_per_sm < 1)
        pipe_per_sm = 1;
    int lo = tail_first_level(Hp, Wp, levels);
    if (lo <= levels) {
        long long bs;
        const float* tin = ll_buf(scratch, batch, Hp, Wp, lo - 1, &bs);
        if (!aligned16(tin) || !aligned16(coef) || (bs & 3) != 0 || (cbs & 3) != 0)
            lo = levels + 1;
    }
    for (int lev = 1; lev <= levels && lev < lo; ++lev) {
        const int h = Hp >> (lev - 1), w = Wp >> (lev - 1);
        const float* sp;
        long long sbs;
        int sld, hv, wv;
        if (lev == 1) {
            sp = src.ptr; sbs = src.bstride; sld = src.ld; hv = src.hv; wv = src.wv;
        } else {
            sp = ll_buf(scratch, batch, Hp, Wp, lev - 1, &sbs);
            sld = w; hv = h; wv = w;
        }
        float* lp;
        long long lbs;
        int lld;
        if (lev == levels) { lp = coef; lbs = cbs; lld = Wp; }
        else { lp = ll_buf(scratch, batch, Hp, Wp, lev, &lbs); lld = w / 2; }
        // the pipelined kernel, a few tiles per block; an unpadded source
        // (level 1 of hyde_dwt2) is read through the symmetric extension
        const int ntiles = ((w / 2 + FTW - 1) / FTW) * ((h / 2 + FTH - 1) / FTH);
        int G = (pipe_per_sm * sms + batch - 1) / batch;
        if (G > ntiles) G = ntiles;
        if (G < 1) G = 1;
        // TMA copies for the interior tiles only where a timeout can be
        // reported (the caller passed a status word)
        CUtensorMap tm;
        memset(&tm, 0, sizeof(tm));
        const int use_tma = status && dwt_tmap(sp, sbs, sld, hv, wv, batch, &tm) ? 1 : 0;
        launch_pdl(dwt_level_pipe_kernel, dim3(G, batch), kFThreads, pipe_smem, s, tm, use_tma,
                   wait_limit_ns(), status, sp, sbs, sld, hv, wv, h, w, coef, cbs, Wp, lp, lbs,
                   lld);
    }
    if (lo <= levels) {
        long long bs;
        const float* tin = ll_buf(scratch, batch, Hp, Wp, lo - 1, &bs);
        const size_t smem =
            (size_t)(Hp >> (lo - 1)) * (Wp >> (lo - 1)) * 5 / 4 * sizeof(float);
        if (ensure_smem_limit((const void*)dwt_tail_kernel, (int)smem) != cudaSuccess)
            return HYDE_ERR_CUDA;
        launch_pdl(dwt_tail_kernel, batch, kTailThreads, smem, s, tin, bs, Wp >> (lo - 1), Hp,
                   Wp, lo, levels, coef, cbs, Wp);
    }
    return cuda_status(cudaGetLastError());
}

hyde_status launch_idwt2(const float* coef, float* out, int batch, int Hp, int Wp, int H,
                         int W, int levels, float* scratch, const double* lam,
                         const int* rank, cudaStream_t s, const float* scale, int scale_ld,
                         bool ll_thr) {
    const long long cbs = (long long)Hp * Wp;
    int lo = tail_first_level(Hp, Wp, levels);
    if (lo <= levels) {
        long long bs;
        float* tout = ll_buf(scratch, batch, Hp, Wp, lo - 1, &bs);
        if (!aligned16(tout) || !aligned16(coef) || (bs & 3) != 0 || (cbs & 3) != 0) {
            lo = levels + 1;
        } else {
            const size_t smem = (size_t)(Hp >> lo) * (Wp >> lo) * 5 / 4 * sizeof(float);
            if (ensure_smem_limit((const void*)idwt_tail_kernel, (int)smem) != cudaSuccess)
                return HYDE_ERR_CUDA;
            launch_pdl(idwt_tail_kernel, batch, kTailSynThreads, smem, s, coef, cbs, Wp, Hp, Wp, lo,
                       levels, lam, scale, scale_ld, rank, tout, bs, ll_thr ? 1 : 0);
        }
    }
    for (int lev = (lo <= levels ? lo - 1 : levels); lev >= 1; --lev) {
        const int h = Hp >> (lev - 1), w = Wp >> (lev - 1);
        const float* lp;
        long long lbs;
        int lld;
        if (lev == levels) { lp = coef; lbs = cbs; lld = Wp; }
        else {
            lp = ll_buf(scratch, batch, Hp, Wp, lev, &lbs);
            lld = w / 2;
        }
        float* op;
        long long obs;
        int old, ho, wo;
        if (lev == 1) { op = out; obs = (long long)H * W; old = W; ho = H; wo = W; }
        else {
            op = ll_buf(scratch, batch, Hp, Wp, lev - 1, &obs);
            old = w; ho = h; wo = w;
        }
        const int wh = w / 2, hh = h / 2;
        const bool vin = (Wp & 3) == 0 && (wh & 3) == 0 && (lld & 3) == 0 && (lbs & 3) == 0 &&
                         (cbs & 3) == 0 && (reinterpret_cast<uintptr_t>(lp) & 15) == 0 &&
                         (reinterpret_cast<uintptr_t>(coef) & 15) == 0;
        if (vin) {
            // every output row inside the crop; float4 stores when rows are 16-byte aligned
            const bool vout = (old & 3) == 0 && (obs & 3) == 0 && ho == h && wo == w &&
                              (reinterpret_cast<uintptr_t>(op) & 15) == 0;
            const long long units =
                (long long)((wh + 127) / 128) * ((hh + kSynRows - 1) / kSynRows);
            const dim3 vgrid((unsigned)((units + kSynWarps - 1) / kSynWarps), batch);
            launch_pdl(idwt_level_vec_kernel, vgrid, kSynThreads, 0, s, lp, lbs, lld, coef, cbs,
                       Wp, h, w, lam, scale, scale_ld, lev, rank, op, obs, old, ho, wo,
                       vout ? 1 : 0, (ll_thr && lev == levels) ? 1 : 0);
            continue;
        }
        dim3 grid((w / 2 + TW - 1) / TW, (h / 2 + TH - 1) / TH, batch);
        launch_pdl(idwt_level_kernel, grid, kThreads, 0, s, lp, lbs, lld, coef, cbs, Wp, h, w,
                   lam, scale, scale_ld, lev, rank, op, obs, old, ho, wo,
                   (ll_thr && lev == levels) ? 1 : 0);
    }
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

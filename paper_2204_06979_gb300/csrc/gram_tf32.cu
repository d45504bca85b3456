// Gram matrix R = Y^T Y on the 5th-generation tensor cores with split-TF32
// compensated products (the spectral statistics of the low-rank model, arXiv
// 2204.06979 Sec. 2.1; the paper runs HyRes in FP32, Sec. 3). FP32-accurate:
// used by the FP32 path and by the TF32 precision mode.
//
// Every float y is split into hi = tf32(y) (rounded to nearest) and
// lo = y - hi (exact in float; the tensor core reads its leading 11 bits,
// a relative error of 2^-22 of y). The product y_a y_b is taken as
// hi_a hi_b + hi_a lo_b + lo_a hi_b; the dropped lo_a lo_b is ~2^-24 y_a y_b.
// Tiles: bands [0, 128) against all Np bands (Np = p rounded to 16; one MMA
// of N = Np per product), and for p > 128 the corner [Np - 128, Np) against
// [128, Np) (N = Np - 128). Each MMA reads its whole A operand (128 rows)
// from shared memory, so few wide MMAs keep the operand traffic low.
//
// Data path, one CTA per SM over a contiguous range of 32-pixel chunks:
//  * a TMA warp loads each chunk into a ring of raw stages. Y is [p][n] with
//    n arbitrary, so a tensor map over rows of stride n would break the
//    16-byte stride rule; the map views Y as [p/4][4n] (stride 16n bytes)
//    and band b = 4r + j is row r at column offset j n. The x coordinate of a
//    box must be a multiple of 4 floats, so band class j is loaded from
//    x0 - s_j, s_j = (j n) mod 4, in a 36-pixel box;
//  * four converter warps read the raw boxes at the offset s_j, round hi,
//    form lo and store both into the 128-byte-swizzled K-major tiles the
//    UMMA descriptors expect (bands as rows, 32 pixels per 128-byte row);
//  * one thread issues tcgen05.mma kind::tf32 into TMEM accumulators that
//    are double buffered over windows of two chunks (64 pixels);
//  * eight drain warps add each finished window into FP32 registers
//    (tcgen05.ld), so that no TMEM accumulator sums more than 24 tensor-core
//    additions (the tensor cores' FP32 accumulation loses ~2^-25 relative per
//    addition, which over the ~4.4k pixels of a CTA would exceed FP32
//    accuracy).
// Each CTA writes its float partial; a second kernel sums the partials in
// double in a fixed order.
//
// Every mbarrier wait is bounded in time: a timeout sets HYDE_ERR_TIMEOUT and
// every role winds down, waiting (bounded) for its own TMA loads and MMAs in
// flight before the CTA frees its TMEM and exits.
#include <cuda.h>

#include "hyde_internal.cuh"
#include "tc_common.cuh"
#include "tmap.cuh"

namespace hyde {
namespace {

constexpr int kK = 32;              // pixels per chunk: one 128-byte row of fp32
constexpr int kKBox = kK + 4;       // pixels per TMA box (room for the shift s_j)
constexpr int kOpStages = 2;
constexpr int kMaxRaw = 8;
#ifndef HYDE_TF32_WIN
#define HYDE_TF32_WIN 2
#endif
constexpr int kWin = HYDE_TF32_WIN; // chunks per TMEM accumulation window
// Warpgroups 0-1: the TMA warp, the MMA warp and six converter warps;
// warpgroups 2-3: the eight drain warps, which keep up to 96 FP32 sums each.
// Launched with 128 registers per thread, warpgroups 0-1 release down to 64
// and 2-3 take up to 192 (setmaxnreg), adding up to the launch's 65536.
constexpr int kTmaWarp = 0, kMmaWarp = 1, kCvtWarp0 = 2, kCvtWarps = 6;
constexpr int kDrainWarp0 = kCvtWarp0 + kCvtWarps, kDrainWarps = 8;
constexpr int kT32Threads = (kDrainWarp0 + kDrainWarps) * 32;
constexpr int kLaunchRegs = 128, kLowRegs = 64, kHighRegs = 192;
static_assert(kT32Threads == 512, "four warpgroups");
static_assert(256 * kLowRegs + 256 * kHighRegs == kT32Threads * kLaunchRegs,
              "the register split must add up to the launch allocation");
constexpr int kMaxP = 160;          // bands of the tensor-core Gram

struct T32Plan {
    int p, Np, NT, NC, rows, q4;
    int raw_stages;
    uint32_t box_bytes, raw_stage_bytes, op_bytes;
    int colT, buf_cols, tmem_cols;
    size_t smem;
    unsigned long long wait_ns;
};

__device__ __forceinline__ float tf32_rn(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// NT: columns of the top tile (all bands rounded to 16, or 32/64/128 for
// p <= 128); NC: columns of the corner tile (0 if p <= 128); H0: columns the
// first half of the drain warps accumulates (the second half takes the rest
// of the top tile and the corner, H0 as well).
template <int NT, int NC, int H0>
__global__ void __launch_bounds__(kT32Threads, 1)
gram_tf32_kernel(const __grid_constant__ CUtensorMap tmap, long long n, T32Plan P,
                 float* __restrict__ partials, int* status) {
    pdl_wait();
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t raw_full[kMaxRaw], raw_empty[kMaxRaw];
    __shared__ uint64_t op_full[kOpStages], op_empty[kOpStages];
    __shared__ uint64_t acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t s0 = smem_u32(smem_raw);
    const uint32_t base = (s0 + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - s0);
    // op stage o: hi tile at base + 2 o op_bytes, lo tile op_bytes after it;
    // then the raw stages
    const uint32_t op_area = 2u * kOpStages * P.op_bytes;
    const uint32_t rawb = base + op_area;
    volatile int* abort_v = &abort_s;
    const int RS = P.raw_stages;

    for (uint32_t e = tid; e < op_area / 16; e += kT32Threads)   // rows >= p stay zero
        reinterpret_cast<uint4*>(gbase)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int q = 0; q < RS; ++q) {
            mbar_init(smem_u32(&raw_full[q]), 1);
            mbar_init(smem_u32(&raw_empty[q]), kCvtWarps * 32);
        }
        for (int q = 0; q < kOpStages; ++q) {
            mbar_init(smem_u32(&op_full[q]), kCvtWarps * 32);
            mbar_init(smem_u32(&op_empty[q]), 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(smem_u32(&acc_full[q]), 1);
            mbar_init(smem_u32(&acc_empty[q]), kDrainWarps * 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_s)),
                     "r"((uint32_t)P.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    const long long nchunks = (n + kK - 1) / kK;
    const long long c0 = (long long)blockIdx.x * nchunks / gridDim.x;
    const long long c1 = (long long)(blockIdx.x + 1) * nchunks / gridDim.x;
    const long long iters = c1 > c0 ? c1 - c0 : 0;
    const long long nwin = (iters + kWin - 1) / kWin;

    if (warp < kDrainWarp0) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(kLowRegs));
    if (warp == kTmaWarp) {
        // ------------------------------------------------------ TMA loads
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap))
                         : "memory");
            long long issued = 0;
            for (long long it = 0; it < iters; ++it) {
                if (*abort_v) break;
                const int s = (int)(it % RS);
                if (it >= RS && !mbar_wait_bounded(smem_u32(&raw_empty[s]),
                                                   (uint32_t)((it / RS - 1) & 1), P.wait_ns)) {
                    *abort_v = 1;
                    break;
                }
                const uint32_t bar = smem_u32(&raw_full[s]);
                mbar_arrive_expect_tx(bar, 4u * (uint32_t)(P.q4 * kKBox * 4));
                const int x0 = (int)((c0 + it) * kK);
                const uint32_t dst = rawb + (uint32_t)s * P.raw_stage_bytes;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    tma_load_2d(dst + (uint32_t)j * P.box_bytes, &tmap,
                                j * (int)n + x0 - (int)((j * n) & 3), 0, bar);
                issued = it + 1;
            }
            // every issued load must have landed before the CTA moves on
            const long long first = issued > RS ? issued - RS : 0;
            for (long long it = first; it < issued; ++it)
                if (!mbar_wait_bounded(smem_u32(&raw_full[(int)(it % RS)]),
                                       (uint32_t)((it / RS) & 1), kWaitNs))
                    *abort_v = 1;
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------ MMA issue (1 thread)
        if (lane == 0) {
            const uint32_t idT = idesc_tf32(128, NT);
            const uint32_t idC = idesc_tf32(128, NC > 0 ? NC : 16);
            const uint32_t bo = 128u * 128u;                       // row 128 of a tile
            const uint32_t co = (uint32_t)(P.Np - 128) * 128u;     // row Np - 128
            const uint32_t colT = (uint32_t)P.colT;
            long long issued = 0;
            for (long long it = 0; it < iters; ++it) {
                if (*abort_v) break;
                const int o = (int)(it % kOpStages);
                const long long w = it / kWin;
                const bool first = (it % kWin) == 0;
                const bool last = (it % kWin) == kWin - 1 || it == iters - 1;
                const int b = (int)(w & 1);
                if (!mbar_wait_bounded(smem_u32(&op_full[o]), (uint32_t)((it / kOpStages) & 1),
                                       P.wait_ns)) {
                    *abort_v = 1;
                    break;
                }
                if (first && w >= 2 &&
                    !mbar_wait_bounded(smem_u32(&acc_empty[b]), (uint32_t)((w / 2 - 1) & 1),
                                       P.wait_ns)) {
                    *abort_v = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t hi = base + (uint32_t)o * 2u * P.op_bytes, lo = hi + P.op_bytes;
                const uint32_t d = tmem + (uint32_t)b * (uint32_t)P.buf_cols;
#pragma unroll
                for (int kk = 0; kk < kK / 8; ++kk) {
                    const uint32_t ko = (uint32_t)kk * 32u;   // 8 tf32 along K
                    const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
                    // bands [0,128) x [0,NT): hi hi + hi lo + lo hi
                    umma_tf32(d + colT, sw128_desc(hi + ko), sw128_desc(hi + ko), idT, acc);
                    umma_tf32(d + colT, sw128_desc(hi + ko), sw128_desc(lo + ko), idT, 1u);
                    umma_tf32(d + colT, sw128_desc(lo + ko), sw128_desc(hi + ko), idT, 1u);
                    if (NC > 0) {
                        // bands [Np-128,Np) x [128,Np)
                        umma_tf32(d, sw128_desc(hi + co + ko), sw128_desc(hi + bo + ko), idC, acc);
                        umma_tf32(d, sw128_desc(hi + co + ko), sw128_desc(lo + bo + ko), idC, 1u);
                        umma_tf32(d, sw128_desc(lo + co + ko), sw128_desc(hi + bo + ko), idC, 1u);
                    }
                }
                umma_commit(smem_u32(&op_empty[o]));
                if (last) umma_commit(smem_u32(&acc_full[b]));
                issued = it + 1;
            }
            // MMAs complete in order: the last commit covers every one issued
            if (issued > 0 &&
                !mbar_wait_bounded(smem_u32(&op_empty[(int)((issued - 1) % kOpStages)]),
                                   (uint32_t)(((issued - 1) / kOpStages) & 1),
                                   P.wait_ns > kWaitNs ? P.wait_ns : kWaitNs))
                *abort_v = 1;
        }
    } else {
        // ------------------------------------------------ split into hi and lo
        const int ct = tid - kCvtWarp0 * 32;
        for (long long it = 0; it < iters; ++it) {
            if (*abort_v) break;
            const int s = (int)(it % RS), o = (int)(it % kOpStages);
            if (!mbar_wait_bounded(smem_u32(&raw_full[s]), (uint32_t)((it / RS) & 1), P.wait_ns)) {
                *abort_v = 1;
                break;
            }
            if (it >= kOpStages &&
                !mbar_wait_bounded(smem_u32(&op_empty[o]), (uint32_t)((it / kOpStages - 1) & 1),
                                   P.wait_ns)) {
                *abort_v = 1;
                break;
            }
            const long long x0 = (c0 + it) * kK;
            const int valid = (int)(n - x0 < kK ? n - x0 : kK);
            const uint8_t* raw = gbase + (op_area + (uint32_t)s * P.raw_stage_bytes);
            uint8_t* hi_t = gbase + (uint32_t)o * 2u * P.op_bytes;
            uint8_t* lo_t = hi_t + P.op_bytes;
            for (int g = ct; g < P.p * 8; g += kCvtWarps * 32) {
                const int b = g >> 3, k4 = g & 7, j = b & 3, r = b >> 2;
                const float* src = reinterpret_cast<const float*>(raw + (uint32_t)j * P.box_bytes) +
                                   r * kKBox + (int)((j * n) & 3) + 4 * k4;
                float v[4], h[4], l[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    v[e] = (4 * k4 + e < valid) ? src[e] : 0.f;
                    h[e] = tf32_rn(v[e]);
                    l[e] = v[e] - h[e];
                }
                const uint32_t off = (uint32_t)b * 128u + ((uint32_t)(k4 ^ (b & 7)) << 4);
                *reinterpret_cast<float4*>(hi_t + off) = make_float4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<float4*>(lo_t + off) = make_float4(l[0], l[1], l[2], l[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(&op_full[o]));
            mbar_arrive(smem_u32(&raw_empty[s]));
        }
    }
    } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(kHighRegs));
    // ---------------------------------------------- drain warps (and output)
    // A drain thread owns TMEM lane `row` and H0 columns in blocks of 16:
    // half 0 the top tile's columns [0, H0); half 1 the top tile's columns
    // [H0, NT), then the corner's [0, NC). Block k maps to TMEM column tcol(k)
    // and to the partial's (band, column) (orow(k), ocol(k)).
    const int dw = warp - kDrainWarp0;
    const int quad = warp & 3, half = dw >> 2;
    const int row = 32 * quad + lane;                     // TMEM lane
    const uint32_t lane_addr = (uint32_t)(32 * quad) << 16;
    constexpr int T1 = NT - H0;                           // top columns of half 1
    auto tcol = [&](int k) -> int {
        return half == 0 ? P.colT + 16 * k : (16 * k < T1 ? P.colT + H0 + 16 * k : 16 * k - T1);
    };
    float acc[H0];
#pragma unroll
    for (int c = 0; c < H0; ++c) acc[c] = 0.f;
    for (long long w = 0; w < nwin; ++w) {
        if (*abort_v) break;
        const int b = (int)(w & 1);
        if (!mbar_wait_bounded(smem_u32(&acc_full[b]), (uint32_t)((w / 2) & 1), P.wait_ns)) {
            *abort_v = 1;
            break;
        }
        __syncwarp();
        tc_fence_after();
        const uint32_t t0 = tmem + lane_addr + (uint32_t)b * (uint32_t)P.buf_cols;
#pragma unroll
        for (int k = 0; k < H0 / 16; ++k) {
            uint32_t r[16];
            tmem_ld16_nowait(t0 + (uint32_t)tcol(k), r);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 16; ++e) acc[16 * k + e] += __uint_as_float(r[e]);
        }
        tc_fence_before();
        mbar_arrive(smem_u32(&acc_empty[b]));
    }
    // the partial (a CTA without chunks writes zeros); overwritten with zeros
    // below if any role gave up
    const int p = P.p;
    float* out = partials + (long long)blockIdx.x * p * p;
    // top tile: lane = band (< 128); corner: lane -> band Np - 128 + lane
#pragma unroll
    for (int k = 0; k < H0 / 16; ++k) {
        const bool corner = half == 1 && 16 * k >= T1;
        const int orow = corner ? P.Np - 128 + row : row;
        const int ocol = half == 0 ? 16 * k : (corner ? 128 + 16 * k - T1 : H0 + 16 * k);
        if (orow < p && (!corner || orow >= 128)) {
#pragma unroll
            for (int e = 0; e < 16; ++e)
                if (ocol + e < p) out[(long long)orow * p + ocol + e] = acc[16 * k + e];
        }
    }
    }
    tc_fence_before();
    __syncthreads();
    if (abort_s) {
        if (tid == 0) set_status(status, HYDE_ERR_TIMEOUT);
        const int p = P.p;
        float* out = partials + (long long)blockIdx.x * p * p;
        for (int e = tid; e < p * p; e += kT32Threads) out[e] = 0.f;
    }
    // the reduction may start once every CTA has written its partial
    pdl_trigger();
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)P.tmem_cols));
    }
}

// R[i][j] = R[j][i] = sum over CTAs of partial[i][j] (i <= j) in double, in
// a fixed order: a block takes 32 consecutive elements, warp w sums the
// partials of CTAs w, w + 8, ... (coalesced rows of 32 floats), and thread
// t < 32 adds the eight warp sums in warp order. Entries of the lower
// triangle of a CTA's partial are not read.
constexpr int kRedWarps = 8;

__global__ void __launch_bounds__(kRedWarps * 32)
gram_tf32_reduce_kernel(const float* __restrict__ partials, int nblocks, int p,
                        double* __restrict__ R, int* status) {
    pdl_wait();
    pdl_trigger();
    __shared__ double part[kRedWarps][32];
    const long long tot = (long long)p * p;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long e = (long long)blockIdx.x * 32 + lane;
    double s0 = 0.0, s1 = 0.0;
    if (e < tot) {
        int b = w;
        for (; b + kRedWarps < nblocks; b += 2 * kRedWarps) {
            s0 += (double)__ldg(partials + (long long)b * tot + e);
            s1 += (double)__ldg(partials + (long long)(b + kRedWarps) * tot + e);
        }
        if (b < nblocks) s0 += (double)__ldg(partials + (long long)b * tot + e);
    }
    part[w][lane] = s0 + s1;
    __syncthreads();
    if (w == 0 && e < tot) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < kRedWarps; ++q) s += part[q][lane];
        const int i = (int)(e / p), j = (int)(e - (long long)i * p);
        if (j >= i) {
            if (!isfinite(s)) set_status(status, HYDE_ERR_NUMERIC);
            R[(long long)i * p + j] = s;
            R[(long long)j * p + i] = s;
        }
    }
}

bool t32_plan(int p, long long n, T32Plan* out) {
    if (p < 4 || p > kMaxP || (p & 3) != 0 || n < 1 || 4 * n > 0x7fffffffLL) return false;
    T32Plan P = {};
    P.p = p;
    P.Np = (p + 15) / 16 * 16;
    P.NT = P.Np > 128 ? P.Np : (p <= 32 ? 32 : p <= 64 ? 64 : 128);
    P.NC = P.Np > 128 ? P.Np - 128 : 0;
    P.rows = P.Np > 128 ? P.Np : 128;
    P.q4 = p / 4;
    P.box_bytes = (uint32_t)align_up((size_t)P.q4 * kKBox * 4, 128);
    P.raw_stage_bytes = 4u * P.box_bytes;
    P.op_bytes = (uint32_t)P.rows * 128u;
    // TMEM per buffer: the corner at column 0 (32 columns reserved), the top
    // tile after it; rounded to 32 columns
    P.colT = P.NC > 0 ? 32 : 0;
    P.buf_cols = (int)align_up((size_t)(P.colT + P.NT), 32);
    const int need = 2 * P.buf_cols;
    if (need > 512) return false;
    P.tmem_cols = need <= 32 ? 32 : need <= 64 ? 64 : need <= 128 ? 128 : need <= 256 ? 256 : 512;
    const size_t room = 227 * 1024 - 1024 - 512;   // alignment slack, static shared memory
    const size_t op_area = 2u * kOpStages * P.op_bytes;
    if (op_area + 2 * P.raw_stage_bytes > room) return false;
    const int rs = (int)((room - op_area) / P.raw_stage_bytes);
    P.raw_stages = rs > kMaxRaw ? kMaxRaw : rs;
    P.smem = 1024 + op_area + (size_t)P.raw_stages * P.raw_stage_bytes;
    *out = P;
    return true;
}

}  // namespace

// cuTensorMapEncodeTiled from the driver through the runtime (no link
// against the driver library); looked up once.
EncodeTiledFn encode_tiled_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    }
    return fn;
}

bool gram_tf32_shape_ok(int p, long long n) {
    T32Plan P;
    return t32_plan(p, n, &P);
}

bool gram_tf32_supported(const float* Y, int p, long long n) {
    T32Plan P;
    return ((uintptr_t)Y % 16) == 0 && t32_plan(p, n, &P) && encode_tiled_fn() != nullptr;
}

hyde_status launch_gram_tf32(const float* Y, int p, long long n, float* partials, double* R,
                             int* status, cudaStream_t s) {
    T32Plan P;
    if (((uintptr_t)Y % 16) != 0 || !t32_plan(p, n, &P)) return HYDE_ERR_SHAPE;
    EncodeTiledFn enc = encode_tiled_fn();
    if (!enc) return HYDE_ERR_CUDA;
    P.wait_ns = wait_limit_ns();
    CUtensorMap tmap;
    const cuuint64_t dims[2] = {(cuuint64_t)(4 * n), (cuuint64_t)P.q4};
    const cuuint64_t strides[1] = {(cuuint64_t)(16 * n)};
    const cuuint32_t box[2] = {(cuuint32_t)kKBox, (cuuint32_t)P.q4};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(Y), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return HYDE_ERR_CUDA;
    const int sms = device_sm_count();
    if (sms <= 0) return HYDE_ERR_CUDA;
    const long long nchunks = (n + kK - 1) / kK;
    const int blocks = (int)(nchunks < sms ? nchunks : sms);
    auto go = [&](auto kernel) -> hyde_status {
        if (ensure_smem_limit((const void*)kernel, (int)P.smem) != cudaSuccess)
            return HYDE_ERR_CUDA;
        // the setmaxnreg split assumes exactly kLaunchRegs registers per thread at launch
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, (const void*)kernel) != cudaSuccess ||
            fa.numRegs != kLaunchRegs)
            return HYDE_ERR_CUDA;
        launch_pdl(kernel, blocks, kT32Threads, P.smem, s, tmap, n, P, partials, status);
        return HYDE_OK;
    };
    hyde_status st;
    switch (P.NT) {
        case 32: st = go(gram_tf32_kernel<32, 0, 16>); break;
        case 64: st = go(gram_tf32_kernel<64, 0, 32>); break;
        case 128: st = go(gram_tf32_kernel<128, 0, 64>); break;
        case 144: st = go(gram_tf32_kernel<144, 16, 80>); break;
        case 160: st = go(gram_tf32_kernel<160, 32, 96>); break;
        default: return HYDE_ERR_SHAPE;
    }
    if (st != HYDE_OK) return st;
    const long long tot = (long long)p * p;
    launch_pdl(gram_tf32_reduce_kernel, (unsigned)((tot + 31) / 32), kRedWarps * 32, 0, s,
               partials, blocks, p, R, status);
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

// Gram matrix R = Y^T Y on the 5th-generation tensor cores (precision form of
// HyRes, arXiv 2204.06979 Sec. 2.1 "low-rank"; the paper runs in FP32 and
// compares against FP64 references, Sec. 3).
//
// Split-BF16 compensated product: every float y is split into
// hi = bf16(y) and lo = bf16(y - hi); y_a y_b is taken as
// hi_a hi_b + hi_a lo_b + lo_a hi_b (the lo*lo term, ~2^-18 relative, is
// dropped), three tcgen05.mma kind::f16 (BF16 x BF16 -> FP32) per K step with
// the accumulator in TMEM.
//
// One CTA per SM walks a contiguous range of 64-pixel chunks through a ring
// of shared-memory stages. Eight producer warps load the chunk (a warp reads
// 64 consecutive pixels of a band), split it and store hi and lo into the
// 128-byte-swizzled K-major layout the UMMA shared-memory descriptors
// expect, then arrive on the stage's "full" mbarrier; a ninth warp waits on
// it, issues the chunk's MMAs and commits them to the stage's "empty"
// mbarrier, which the producers wait on before refilling the stage. Rows of the
// accumulator: bands [0, 128) (M-tile 0, all N = Np columns) and, for
// p > 128, bands [Np - 128, Np) against columns [128, Np) (M-tile 1). Each
// CTA writes its float partial; a second kernel sums them in double.
//
// Every wait on an mbarrier is bounded in time (a status flag is set and the
// kernel winds down: it waits, again bounded, for its MMAs in flight and
// frees its TMEM).
#include <cuda_bf16.h>

#include "hyde_internal.cuh"
#include "tc_common.cuh"

namespace hyde {
namespace {

constexpr int kTcMaxStages = 4;
constexpr int kChunk = 64;                      // pixels per chunk = one 128 B row of bf16

struct TcPlan {
    int Np;        // rows in shared memory (p rounded up to 16, at least 128)
    int nmt;       // M tiles (1 or 2)
    int m1_row0;   // first band of M-tile 1
    int n1;        // columns of M-tile 1 (bands [128, Np))
    int d1_col;    // TMEM column of M-tile 1
    int tmem_cols; // allocated TMEM columns
    int stages;    // shared-memory stages (<= kTcMaxStages)
    size_t stage_bytes, smem;
    unsigned long long wait_ns;   // limit of the main-loop mbarrier waits
};

// Producer warps 0..7 convert; warp 8 issues the MMAs. Each producer thread
// owns band rows b = warp + 8q (q < RPW) and the pixel pair (2 lane,
// 2 lane + 1) of every chunk, double-buffered in registers: chunk it + 2 is
// loaded while chunk it is split and stored. All of a thread's rows share
// b & 7 = warp, so in the 128-byte-swizzled layout row b sits at
// q * 1024 + (a per-thread offset).
constexpr int kProducerWarps = 8;
constexpr int kTcThreadsWs = (kProducerWarps + 1) * 32;

template <int RPW>
struct ChunkRegs {
    float v[RPW][2];
};

template <int RPW>
__device__ __forceinline__ void load_chunk(ChunkRegs<RPW>& R, const float* __restrict__ yb,
                                           long long bstride, int p, long long n,
                                           long long pix, int warp) {
    const bool full = pix + 1 < n;     // both pixels of the pair inside the cube
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
        float v0 = 0.f, v1 = 0.f;
        if (warp + kProducerWarps * q < p) {
            const float* yr = yb + q * bstride;
            if (full) {
                v0 = __ldg(yr);
                v1 = __ldg(yr + 1);
            } else if (pix < n) {
                v0 = __ldg(yr);
            }
        }
        R.v[q][0] = v0;
        R.v[q][1] = v1;
    }
}

template <int RPW>
__device__ __forceinline__ void store_chunk(const ChunkRegs<RPW>& R, uint8_t* st, uint32_t half,
                                            uint32_t toff, int p, int warp) {
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
        if (warp + kProducerWarps * q < p) {
            uint32_t hi, lo;
            split_pair(R.v[q][0], R.v[q][1], hi, lo);
            *reinterpret_cast<uint32_t*>(st + q * 1024 + toff) = hi;
            *reinterpret_cast<uint32_t*>(st + half + q * 1024 + toff) = lo;
        }
    }
}

template <int RPW>
__global__ void __launch_bounds__(kTcThreadsWs, 1)
gram_tc_kernel(const float* __restrict__ Y, int p, long long n, TcPlan P,
               long long chunks_per_cta, float* __restrict__ partials, int* status) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[kTcMaxStages], empty_bar[kTcMaxStages];
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // 1024-byte aligned stage area (the swizzle atoms must not straddle)
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    const uint32_t half = (uint32_t)P.Np * 128u;   // hi tile, then lo tile
    volatile int* abort_v = &abort_s;

    // zero every stage once: rows p..Np-1 stay zero
    const int S = P.stages;
    for (size_t e = tid; e < (size_t)S * P.stage_bytes / 16; e += kTcThreadsWs)
        reinterpret_cast<uint4*>(gbase)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(smem_u32(&full_bar[q]), kProducerWarps * 32);
            mbar_init(smem_u32(&empty_bar[q]), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
    }
    if (warp == kProducerWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_s)),
                     "r"((uint32_t)P.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // the zeroed stages are read by the tensor cores (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    const long long nchunks = (n + kChunk - 1) / kChunk;
    // even split: block b takes chunks [b N / G, (b + 1) N / G)
    const long long c0 = (long long)blockIdx.x * nchunks / gridDim.x;
    const long long c1 = (long long)(blockIdx.x + 1) * nchunks / gridDim.x;
    (void)chunks_per_cta;
    const long long iters = c1 > c0 ? c1 - c0 : 0;

    if (warp < kProducerWarps) {
        // ---------------- producers
        const uint32_t toff = (uint32_t)(warp * 128 + (((lane >> 2) ^ warp) << 4) +
                                         ((lane & 3) << 2));
        const long long bstride = (long long)kProducerWarps * n;
        const float* yw = Y + (long long)warp * n + 2 * lane;
        ChunkRegs<RPW> ra, rb;
        if (iters > 0) load_chunk(ra, yw + c0 * kChunk, bstride, p, n, c0 * kChunk + 2 * lane, warp);
        if (iters > 1)
            load_chunk(rb, yw + (c0 + 1) * kChunk, bstride, p, n, (c0 + 1) * kChunk + 2 * lane,
                       warp);
        for (long long it = 0; it < iters; ++it) {
            const int s = (int)(it % S);
            if (it >= S) {
                // the MMAs that last read this stage (iteration it - S) are done
                const uint32_t par = (uint32_t)((it / S - 1) & 1);
                if (!mbar_wait_bounded(smem_u32(&empty_bar[s]), par, P.wait_ns)) *abort_v = 1;
            }
            if (*abort_v) break;
            uint8_t* st = gbase + (size_t)s * P.stage_bytes;
            const long long cn = c0 + it + 2;
            if ((it & 1) == 0) {
                store_chunk(ra, st, half, toff, p, warp);
                if (it + 2 < iters) load_chunk(ra, yw + cn * kChunk, bstride, p, n, cn * kChunk + 2 * lane, warp);
            } else {
                store_chunk(rb, st, half, toff, p, warp);
                if (it + 2 < iters) load_chunk(rb, yw + cn * kChunk, bstride, p, n, cn * kChunk + 2 * lane, warp);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(&full_bar[s]));
        }
    } else if (lane == 0) {
        // ---------------- MMA issuer (one thread)
        const uint32_t id0 = idesc_bf16(128, P.Np);
        const uint32_t id1 = idesc_bf16(128, P.n1 > 0 ? P.n1 : 16);
        long long issued = 0;
        for (long long it = 0; it < iters; ++it) {
            const int s = (int)(it % S);
            if (!mbar_wait_bounded(smem_u32(&full_bar[s]), (uint32_t)((it / S) & 1), P.wait_ns)) {
                *abort_v = 1;
                break;
            }
            if (*abort_v) break;
            tc_fence_after();
            const uint32_t hi0 = base + (uint32_t)s * (uint32_t)P.stage_bytes, lo0 = hi0 + half;
#pragma unroll
            for (int kk = 0; kk < kChunk / 16; ++kk) {
                const uint32_t ko = (uint32_t)kk * 32u;   // 16 bf16 along K
                const uint32_t acc0 = (it > 0 || kk > 0) ? 1u : 0u;
                // M-tile 0: bands [0,128) x all Np columns
                umma_bf16(tmem, sw128_desc(hi0 + ko), sw128_desc(hi0 + ko), id0, acc0);
                umma_bf16(tmem, sw128_desc(hi0 + ko), sw128_desc(lo0 + ko), id0, 1u);
                umma_bf16(tmem, sw128_desc(lo0 + ko), sw128_desc(hi0 + ko), id0, 1u);
                if (P.nmt == 2) {
                    // M-tile 1: bands [Np-128, Np) x columns [128, Np)
                    const uint32_t ao = (uint32_t)P.m1_row0 * 128u, bo = 128u * 128u;
                    const uint32_t d1 = tmem + (uint32_t)P.d1_col;
                    umma_bf16(d1, sw128_desc(hi0 + ao + ko), sw128_desc(hi0 + bo + ko), id1, acc0);
                    umma_bf16(d1, sw128_desc(hi0 + ao + ko), sw128_desc(lo0 + bo + ko), id1, 1u);
                    umma_bf16(d1, sw128_desc(lo0 + ao + ko), sw128_desc(hi0 + bo + ko), id1, 1u);
                }
            }
            umma_commit(smem_u32(&empty_bar[s]));
            issued = it + 1;
        }
        // MMAs complete in order: the last commit covers all of them (bounded,
        // never by less than one second, however short the main-loop limit)
        if (issued > 0) {
            const long long last = issued - 1;
            if (!mbar_wait_bounded(smem_u32(&empty_bar[(int)(last % S)]),
                                   (uint32_t)((last / S) & 1),
                                   P.wait_ns > kWaitNs ? P.wait_ns : kWaitNs))
                *abort_v = 1;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const bool ok = iters > 0 && !abort_s;
    if (abort_s && tid == 0) set_status(status, HYDE_ERR_TIMEOUT);

    // epilogue: warp w % 4 reads TMEM lanes 32 (w % 4) .. + 31
    float* out = partials + (long long)blockIdx.x * p * p;
    const int quad = warp & 3;
    const uint32_t lane_addr = (uint32_t)(32 * quad) << 16;
    if (warp < 4) {
        const int row = 32 * quad + lane;           // band of M-tile 0
        for (int j = 0; j < P.Np; j += 8) {
            float v[8];
            if (ok) tmem_ld8(tmem + lane_addr + (uint32_t)j, v);
            else for (int q = 0; q < 8; ++q) v[q] = 0.f;
            if (row < p)
                for (int q = 0; q < 8; ++q)
                    if (j + q < p) out[(long long)row * p + j + q] = v[q];
        }
    } else if (warp < 8 && P.nmt == 2) {
        const int row = P.m1_row0 + 32 * quad + lane;   // band of M-tile 1
        for (int j = 0; j < P.n1; j += 8) {
            float v[8];
            if (ok) tmem_ld8(tmem + lane_addr + (uint32_t)(P.d1_col + j), v);
            else for (int q = 0; q < 8; ++q) v[q] = 0.f;
            if (row >= 128 && row < p)
                for (int q = 0; q < 8; ++q)
                    if (128 + j + q < p) out[(long long)row * p + 128 + j + q] = v[q];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kProducerWarps) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)P.tmem_cols));
    }
}

// R[i][j] = R[j][i] = sum over CTAs of the partial (i <= j): rows < 128 come
// from M-tile 0, rows >= 128 (then j >= 128) from M-tile 1. Thread (e, y)
// sums the partials of CTAs [16 y, 16 y + 16) for element e (coalesced over
// e, independent loads) and adds the segment total with a double atomic to R,
// which is cleared beforehand.
constexpr int kTcReduceSeg = 16;

__global__ void gram_tc_reduce_kernel(const float* __restrict__ partials, int nblocks, int p,
                                      double* __restrict__ R, int* status) {
    pdl_wait();
    pdl_trigger();
    const long long tot = (long long)p * p;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= tot) return;
    const int i = (int)(e / p), j = (int)(e % p);
    if (j < i) return;
    const int b0 = blockIdx.y * kTcReduceSeg, b1 = min(b0 + kTcReduceSeg, nblocks);
    double s = 0.0;
#pragma unroll 4
    for (int b = b0; b < b1; ++b) s += (double)__ldg(partials + (long long)b * tot + e);
    if (!isfinite(s)) set_status(status, HYDE_ERR_NUMERIC);
    atomicAdd(&R[(long long)i * p + j], s);
    if (i != j) atomicAdd(&R[(long long)j * p + i], s);
}

TcPlan tc_plan(int p) {
    TcPlan P;
    int np16 = (p + 15) / 16 * 16;
    P.Np = np16 < 128 ? 128 : np16;
    P.nmt = P.Np > 128 ? 2 : 1;
    P.m1_row0 = P.Np - 128;
    P.n1 = P.nmt == 2 ? P.Np - 128 : 0;
    P.d1_col = (P.Np + 31) / 32 * 32;
    const int cols = P.d1_col + P.n1;
    P.tmem_cols = cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : cols <= 256 ? 256 : 512;
    P.stage_bytes = (size_t)P.Np * 128 * 2;
    const size_t room = 227 * 1024 - 1024 - 256;   // alignment slack, static smem
    P.stages = (int)(room / P.stage_bytes);
    if (P.stages > kTcMaxStages) P.stages = kTcMaxStages;
    P.smem = (size_t)P.stages * P.stage_bytes + 1024;
    return P;
}

}  // namespace

hyde_status gram_tc_partial_bytes(int p, size_t* bytes) {
    if (p < 1 || p > kMaxBandsGram) return HYDE_ERR_SHAPE;
    const int sms = device_sm_count();
    if (sms <= 0) return HYDE_ERR_CUDA;
    *bytes = (size_t)sms * p * p * sizeof(float);
    return HYDE_OK;
}

hyde_status launch_gram_tc(const float* Y, int p, long long n, float* partials, double* R,
                           int* status, cudaStream_t s) {
    if (p < 1 || p > kMaxBandsGram || n < 1) return HYDE_ERR_SHAPE;
    TcPlan P = tc_plan(p);
    P.wait_ns = wait_limit_ns();
    if (P.stages < 2 || P.smem > 227 * 1024 || P.tmem_cols > 512) return HYDE_ERR_SHAPE;
    const int sms = device_sm_count();
    if (sms <= 0) return HYDE_ERR_CUDA;
    const long long nchunks = (n + kChunk - 1) / kChunk;
    const int blocks = sms;
    const long long per = (nchunks + blocks - 1) / blocks;
    const int rpw = (p + kProducerWarps - 1) / kProducerWarps;   // band rows per producer warp
    switch ((rpw + 7) / 8) {
#define HYDE_TC(G)                                                                            \
    case G:                                                                                   \
        if (ensure_smem_limit((const void*)gram_tc_kernel<8 * G>, (int)P.smem) != cudaSuccess) \
            return HYDE_ERR_CUDA;                                                             \
        launch_pdl(gram_tc_kernel<8 * G>, blocks, kTcThreadsWs, P.smem, s, Y, p, n, P, per,   \
                   partials, status);                                                         \
        break;
        HYDE_TC(1) HYDE_TC(2) HYDE_TC(3) HYDE_TC(4)
#undef HYDE_TC
        default: return HYDE_ERR_SHAPE;
    }
    if (cudaMemsetAsync(R, 0, (size_t)p * p * sizeof(double), s) != cudaSuccess)
        return HYDE_ERR_CUDA;
    dim3 rgrid((unsigned)((p * p + 255) / 256), (blocks + kTcReduceSeg - 1) / kTcReduceSeg);
    launch_pdl(gram_tc_reduce_kernel, rgrid, 256, 0, s, partials, blocks, p, R, status);
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

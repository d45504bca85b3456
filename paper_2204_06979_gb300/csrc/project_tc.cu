// Projection and back-projection of the precision form on the tcgen05 tensor
// cores (HyRes low-rank model, arXiv 2204.06979 Sec. 2.1):
//   Z_i(pixel) = sum_b Y_b(pixel) P[b][i],     P = D^-1 V
//   X_b(pixel) = sum_{i < r*} Q[b][i] Zh_i(pixel),  Q = D V
// as GEMMs with the pixels on M (128 per tile), split-BF16 compensated
// products (hi hi + hi lo + lo hi, FP32 accumulation in TMEM) like the Gram
// matrix of this form.
//
// Both kernels are persistent (one CTA per SM) and warp-specialised:
//  * producer warps load the FP32 operand of a 128-pixel tile, split it into
//    BF16 hi and lo and store them in the 128-byte-swizzled K-major layout
//    (row = pixel, K along bands or components; a thread packs the two K
//    neighbours of its pixel into one 32-bit word), then arrive on the
//    stage's "full" mbarrier;
//  * one thread issues the MMAs of a stage and commits them to the stage's
//    "empty" mbarrier, and after a tile's last stage to the "tmem_full"
//    mbarrier of one of two TMEM accumulators;
//  * epilogue warps (one per TMEM lane quadrant, or two for the wide
//    back-projection) read the accumulator with tcgen05.ld, release it on
//    "tmem_empty" and write the result with coalesced stores (thread =
//    pixel).
// The weights (P or Q) are split and laid out once per CTA. Every mbarrier
// wait is bounded (1 s): on a timeout the kernel records HYDE_ERR_TIMEOUT,
// stops, waits (bounded) for the MMAs it issued and frees its TMEM.
#include "hyde_internal.cuh"
#include "tc_common.cuh"

namespace hyde {
namespace {

constexpr int kTileM = 128;                 // pixels per tile (MMA M)
constexpr int kProdWarps = 8;               // producer warps (256 threads)
constexpr int kMmaWarp = kProdWarps;        // warp 8 issues the MMAs
constexpr int kEpiWarp0 = kProdWarps + 1;   // first epilogue warp
constexpr uint32_t kKBlockBytes = kTileM * 128;   // 128 rows x 128 B: 64 bf16 of K

// byte offset of the packed K pair (k, k+1), k even, of row `row` in a
// 128-byte-swizzled K-major tile (8-row atoms of 1024 B)
__device__ __forceinline__ uint32_t sw128_pair_offset(int row, int k) {
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 3) ^ (row & 7)) & 7) << 4) +
                      ((k & 7) << 1));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}
__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Source pixel of padded pixel pix (reflection at the bottom/right edges);
// false where the padding is zero or pix is past the end.
__device__ __forceinline__ bool pad_src(long long pix, long long N, int H, int W, int Wp,
                                        int zero_pad, long long& src) {
    src = 0;
    if (pix >= N) return false;
    const int pi = (int)pix;               // N < 2^31 (checked by the launcher)
    int y = pi / Wp, x = pi - y * Wp;
    if (zero_pad && (y >= H || x >= W)) return false;
    if (y >= H) y = 2 * H - 2 - y;
    if (x >= W) x = 2 * W - 2 - x;
    src = (long long)y * W + x;
    return true;
}

// Split weights W[kk][n] (float, row stride ldw; kk < k_valid, n < n_valid,
// zero elsewhere) into hi and lo tiles with rows n (N of the MMA) and K along
// kk: rows x 128 B per 64-wide K block, K blocks of `rows` rows back to back.
__device__ void build_weight_tiles(const float* __restrict__ W, int ldw, int k_valid,
                                   int n_valid, int rows, int kblocks, uint8_t* hi,
                                   uint8_t* lo, int tid, int nthreads) {
    const int pairs = rows * kblocks * 32;   // 32 K pairs per row and K block
    for (int e = tid; e < pairs; e += nthreads) {
        const int kb = e / (rows * 32);
        const int rem = e - kb * rows * 32;
        const int n = rem / 32, kp = rem % 32;
        const int k = kb * 64 + 2 * kp;
        const float a = (n < n_valid && k < k_valid) ? W[(long long)k * ldw + n] : 0.f;
        const float b = (n < n_valid && k + 1 < k_valid) ? W[(long long)(k + 1) * ldw + n] : 0.f;
        uint32_t h, l;
        split_pair(a, b, h, l);
        const uint32_t off = (uint32_t)kb * (uint32_t)rows * 128u + sw128_pair_offset(n, 2 * kp);
        *reinterpret_cast<uint32_t*>(hi + off) = h;
        *reinterpret_cast<uint32_t*>(lo + off) = l;
    }
}

// ---------------------------------------------------------------- projection
constexpr int kPjN = 32;        // components (MMA N); r_max <= 32
constexpr int kPjStages = 5;    // (tile, K block) stages of 32 KB
constexpr int kPjEpiWarps = 4;
constexpr int kPjThreads = (kProdWarps + 1 + kPjEpiWarps) * 32;
constexpr int kPjSlots = 16;    // (row, K pair) slots per producer thread and stage

// Producer thread mapping of one 128-row x 64-K stage: warp w covers the
// 8-row atoms w and w + 8, lane l row (l & 7) of the atom and K pairs
// 4 j + (l >> 3), j < 8. The 32 lanes of a store then hit one 16-byte chunk
// position per row (8 rows) and four words within it: 32 distinct banks.
struct PjRegs {
    float v[kPjSlots][2];
};

// element offsets (32 bit: p * n < 2^31) of band pair (b, b + 1) at pixel src
__device__ __forceinline__ void pj_load(PjRegs& R, const float* __restrict__ Y, unsigned n, int p,
                                        int kb, int pq, const unsigned (&src)[2],
                                        const bool (&data)[2]) {
#pragma unroll
    for (int a = 0; a < 2; ++a) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int b = kb * 64 + 2 * (4 * j + pq);
            const unsigned off = (unsigned)b * n + src[a];
            R.v[a * 8 + j][0] = (data[a] && b < p) ? __ldg(Y + off) : 0.f;
            R.v[a * 8 + j][1] = (data[a] && b + 1 < p) ? __ldg(Y + off + n) : 0.f;
        }
    }
}

__device__ __forceinline__ void pj_store(const PjRegs& R, uint8_t* hi, uint8_t* lo, int warp,
                                         int rr, int pq) {
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int row = 8 * (warp + 8 * a) + rr;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t h, l;
            split_pair(R.v[a * 8 + j][0], R.v[a * 8 + j][1], h, l);
            const uint32_t off = sw128_pair_offset(row, 2 * (4 * j + pq));
            *reinterpret_cast<uint32_t*>(hi + off) = h;
            *reinterpret_cast<uint32_t*>(lo + off) = l;
        }
    }
}

__global__ void __launch_bounds__(kPjThreads, 1)
project_tc_kernel(const float* __restrict__ Y, int p, int H, int W, const float* __restrict__ P,
                  int r, int ldw, float* __restrict__ Zp, int Hp, int Wp, int zero_pad,
                  int* status) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[kPjStages], empty_bar[kPjStages];
    __shared__ uint64_t tfull_bar[2], tempty_bar[2];
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;
    volatile int* abort_v = &abort_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);

    const int KB = (p + 63) / 64;                       // K blocks of 64 bands
    const int ks_last = ((p - 64 * (KB - 1)) + 15) / 16; // K steps of the last block
    const uint32_t wtile = (uint32_t)kPjN * 128u;       // one K block of weights
    uint8_t* Bhi = gbase;
    uint8_t* Blo = gbase + KB * wtile;
    const uint32_t stage0 = 2u * KB * wtile;            // multiple of 1024
    const uint32_t stage_bytes = 2u * kKBlockBytes;     // hi, then lo

    if (tid == 0) {
        for (int q = 0; q < kPjStages; ++q) {
            mbar_init(smem_u32(&full_bar[q]), kProdWarps * 32);
            mbar_init(smem_u32(&empty_bar[q]), 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(smem_u32(&tfull_bar[q]), 1);
            mbar_init(smem_u32(&tempty_bar[q]), kPjEpiWarps * 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_s)),
                     "r"(64u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    build_weight_tiles(P, ldw, p, r, kPjN, KB, Bhi, Blo, tid, kPjThreads);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    const long long N = (long long)Hp * Wp, n = (long long)H * W;
    const long long tiles = (N + kTileM - 1) / kTileM;
    const long long t0 = (long long)blockIdx.x * tiles / gridDim.x;
    const long long t1 = (long long)(blockIdx.x + 1) * tiles / gridDim.x;
    const long long ntile = t1 - t0;
    const long long nstage = ntile * KB;

    if (warp < kProdWarps) {
        // ---- producers (mapping above)
        const int rr = lane & 7, pq = lane >> 3;
        PjRegs ra, rb;
        // source pixels of the tile being loaded (the same for its K blocks)
        unsigned src[2] = {0u, 0u};
        bool data[2] = {false, false};
        auto prep = [&](long long u, PjRegs& R) {
            const int kb = (int)(u % KB);
            if (kb == 0) {
                const long long tl = t0 + u / KB;
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    long long sp;
                    data[a] = pad_src(tl * kTileM + 8 * (warp + 8 * a) + rr, N, H, W, Wp,
                                      zero_pad, sp);
                    src[a] = (unsigned)sp;
                }
            }
            pj_load(R, Y, (unsigned)n, p, kb, pq, src, data);
        };
        if (nstage > 0) prep(0, ra);
        if (nstage > 1) prep(1, rb);
        for (long long u = 0; u < nstage; ++u) {
            const int s = (int)(u % kPjStages);
            if (u >= kPjStages &&
                !mbar_wait_bounded(smem_u32(&empty_bar[s]), (uint32_t)((u / kPjStages - 1) & 1)))
                *abort_v = 1;
            if (*abort_v) break;
            uint8_t* hi = gbase + stage0 + (uint32_t)s * stage_bytes;
            if ((u & 1) == 0) {
                pj_store(ra, hi, hi + kKBlockBytes, warp, rr, pq);
                if (u + 2 < nstage) prep(u + 2, ra);
            } else {
                pj_store(rb, hi, hi + kKBlockBytes, warp, rr, pq);
                if (u + 2 < nstage) prep(u + 2, rb);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(&full_bar[s]));
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            // ---- MMA issuer
            const uint32_t idesc = idesc_bf16(kTileM, kPjN);
            long long issued = 0;
            for (long long u = 0; u < nstage; ++u) {
                const long long tl = u / KB;
                const int kb = (int)(u % KB), s = (int)(u % kPjStages);
                const int buf = (int)(tl & 1);
                if (kb == 0 && tl >= 2 &&
                    !mbar_wait_bounded(smem_u32(&tempty_bar[buf]), (uint32_t)((tl / 2 - 1) & 1))) {
                    *abort_v = 1;
                    break;
                }
                if (!mbar_wait_bounded(smem_u32(&full_bar[s]), (uint32_t)((u / kPjStages) & 1))) {
                    *abort_v = 1;
                    break;
                }
                if (*abort_v) break;
                tc_fence_after();
                const uint32_t ahi = base + stage0 + (uint32_t)s * stage_bytes;
                const uint32_t alo = ahi + kKBlockBytes;
                const uint32_t bhi = base + (uint32_t)kb * wtile, blo = bhi + KB * wtile;
                const uint32_t d = tmem + (uint32_t)(buf * kPjN);
                const int ks_n = kb == KB - 1 ? ks_last : 4;
                for (int ks = 0; ks < ks_n; ++ks) {
                    const uint32_t ko = (uint32_t)ks * 32u;
                    const uint32_t acc = (kb > 0 || ks > 0) ? 1u : 0u;
                    umma_bf16(d, sw128_desc(ahi + ko), sw128_desc(bhi + ko), idesc, acc);
                    umma_bf16(d, sw128_desc(ahi + ko), sw128_desc(blo + ko), idesc, 1u);
                    umma_bf16(d, sw128_desc(alo + ko), sw128_desc(bhi + ko), idesc, 1u);
                }
                umma_commit(smem_u32(&empty_bar[s]));
                if (kb == KB - 1) umma_commit(smem_u32(&tfull_bar[buf]));
                issued = u + 1;
            }
            // the MMAs complete in order: wait for the last commit (bounded)
            if (issued > 0) {
                const long long last = issued - 1;
                if (!mbar_wait_bounded(smem_u32(&empty_bar[(int)(last % kPjStages)]),
                                       (uint32_t)((last / kPjStages) & 1)))
                    *abort_v = 1;
            }
        }
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (pixels)
        const int quad = warp & 3;
        const int m = 32 * quad + lane;
        const uint32_t lane_addr = (uint32_t)(32 * quad) << 16;
        for (long long tl = 0; tl < ntile; ++tl) {
            const int buf = (int)(tl & 1);
            if (!mbar_wait_bounded(smem_u32(&tfull_bar[buf]), (uint32_t)((tl / 2) & 1))) {
                *abort_v = 1;
                break;
            }
            if (*abort_v) break;
            tc_fence_after();
            float v[kPjN];
            tmem_ld16(tmem + lane_addr + (uint32_t)(buf * kPjN), v);
            tmem_ld16(tmem + lane_addr + (uint32_t)(buf * kPjN + 16), v + 16);
            tmem_wait_ld();
            tc_fence_before();
            mbar_arrive(smem_u32(&tempty_bar[buf]));
            const long long pix = (t0 + tl) * kTileM + m;
            if (pix < N) {
                unsigned off = (unsigned)pix;
#pragma unroll
                for (int i = 0; i < kPjN; ++i, off += (unsigned)N)
                    if (i < r) Zp[off] = v[i];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (abort_s && tid == 0) set_status(status, HYDE_ERR_TIMEOUT);
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64u));
    }
}

// ----------------------------------------------------------- back-projection
constexpr int kBpK = 32;          // components (MMA K, two steps of 16)
constexpr int kBpStages = 3;      // tiles of 32 KB (hi + lo, one 64-wide K block)
constexpr int kBpEpiWarps = 8;    // two per TMEM lane quadrant (column halves)
constexpr int kBpThreads = (kProdWarps + 1 + kBpEpiWarps) * 32;
constexpr int kBpSlots = 8;       // (row, K pair) slots per producer thread: K = 32
constexpr uint32_t kBpAccCols = 256;   // TMEM columns per accumulator (N <= 256)

// Producer mapping for a 128-row x 32-K tile (16 K pairs): warp w covers the
// 8-row atoms w and w + 8, lane l row (l & 7) and K pairs 4 j + (l >> 3),
// j < 4 (conflict-free stores as in the projection).
struct BpRegs {
    float v[kBpSlots][2];
};

__device__ __forceinline__ void bp_load(BpRegs& R, const float* __restrict__ Zh, unsigned n, int r,
                                        int warp, int rr, int pq, long long tile) {
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const long long pix = tile * kTileM + 8 * (warp + 8 * a) + rr;
        const bool live = pix < (long long)n;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = 2 * (4 * j + pq);
            const unsigned off = (unsigned)i * n + (unsigned)pix;
            R.v[a * 4 + j][0] = (live && i < r) ? __ldg(Zh + off) : 0.f;
            R.v[a * 4 + j][1] = (live && i + 1 < r) ? __ldg(Zh + off + n) : 0.f;
        }
    }
}

__device__ __forceinline__ void bp_store(const BpRegs& R, uint8_t* hi, uint8_t* lo, int warp,
                                         int rr, int pq) {
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int row = 8 * (warp + 8 * a) + rr;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t h, l;
            split_pair(R.v[a * 4 + j][0], R.v[a * 4 + j][1], h, l);
            const uint32_t off = sw128_pair_offset(row, 2 * (4 * j + pq));
            *reinterpret_cast<uint32_t*>(hi + off) = h;
            *reinterpret_cast<uint32_t*>(lo + off) = l;
        }
    }
}

__global__ void __launch_bounds__(kBpThreads, 1)
backproject_tc_kernel(const float* __restrict__ Zh, long long n, const float* __restrict__ Q,
                      int p, int ldw, const int* __restrict__ rank, float* __restrict__ X,
                      int* status) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[kBpStages], empty_bar[kBpStages];
    __shared__ uint64_t tfull_bar[2], tempty_bar[2];
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;
    volatile int* abort_v = &abort_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);

    const int r = min(*rank, min(ldw, kBpK));
    const int Np = (p + 15) / 16 * 16;               // MMA N (bands)
    const int Nrows = (Np + 7) / 8 * 8;              // weight rows (8-row atoms)
    const uint32_t wtile = (uint32_t)Nrows * 128u;
    uint8_t* Bhi = gbase;
    uint8_t* Blo = gbase + wtile;
    const uint32_t stage0 = (2u * wtile + 1023u) & ~1023u;
    const uint32_t stage_bytes = 2u * kKBlockBytes;
    const int ks_n = (r + 15) / 16;                   // 1 or 2 K steps

    if (tid == 0) {
        for (int q = 0; q < kBpStages; ++q) {
            mbar_init(smem_u32(&full_bar[q]), kProdWarps * 32);
            mbar_init(smem_u32(&empty_bar[q]), 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(smem_u32(&tfull_bar[q]), 1);
            mbar_init(smem_u32(&tempty_bar[q]), kBpEpiWarps * 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_s)),
                     "r"(2u * kBpAccCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // weights Q[b][i]: rows = bands (N), K = components; transpose of the
    // projection's layout, so W[k][n] = Q[n][k] is read with ldw swapped
    {
        const int pairs = Nrows * 32;
        for (int e = tid; e < pairs; e += kBpThreads) {
            const int nn = e / 32, kp = e % 32;
            const int k = 2 * kp;
            const float a = (nn < p && k < r) ? Q[(long long)nn * ldw + k] : 0.f;
            const float b = (nn < p && k + 1 < r) ? Q[(long long)nn * ldw + k + 1] : 0.f;
            uint32_t h, l;
            split_pair(a, b, h, l);
            const uint32_t off = sw128_pair_offset(nn, k);
            *reinterpret_cast<uint32_t*>(Bhi + off) = h;
            *reinterpret_cast<uint32_t*>(Blo + off) = l;
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    const long long tiles = (n + kTileM - 1) / kTileM;
    const long long t0 = (long long)blockIdx.x * tiles / gridDim.x;
    const long long t1 = (long long)(blockIdx.x + 1) * tiles / gridDim.x;
    const long long ntile = t1 - t0;

    if (warp < kProdWarps) {
        const int rr = lane & 7, pq = lane >> 3;
        const unsigned nu = (unsigned)n;
        BpRegs ra, rb;
        if (ntile > 0) bp_load(ra, Zh, nu, r, warp, rr, pq, t0);
        if (ntile > 1) bp_load(rb, Zh, nu, r, warp, rr, pq, t0 + 1);
        for (long long u = 0; u < ntile; ++u) {
            const int s = (int)(u % kBpStages);
            if (u >= kBpStages &&
                !mbar_wait_bounded(smem_u32(&empty_bar[s]), (uint32_t)((u / kBpStages - 1) & 1)))
                *abort_v = 1;
            if (*abort_v) break;
            uint8_t* hi = gbase + stage0 + (uint32_t)s * stage_bytes;
            if ((u & 1) == 0) {
                bp_store(ra, hi, hi + kKBlockBytes, warp, rr, pq);
                if (u + 2 < ntile) bp_load(ra, Zh, nu, r, warp, rr, pq, t0 + u + 2);
            } else {
                bp_store(rb, hi, hi + kKBlockBytes, warp, rr, pq);
                if (u + 2 < ntile) bp_load(rb, Zh, nu, r, warp, rr, pq, t0 + u + 2);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(&full_bar[s]));
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(kTileM, Np);
            long long issued = 0;
            for (long long u = 0; u < ntile; ++u) {
                const int s = (int)(u % kBpStages), buf = (int)(u & 1);
                if (u >= 2 &&
                    !mbar_wait_bounded(smem_u32(&tempty_bar[buf]), (uint32_t)((u / 2 - 1) & 1))) {
                    *abort_v = 1;
                    break;
                }
                if (!mbar_wait_bounded(smem_u32(&full_bar[s]), (uint32_t)((u / kBpStages) & 1))) {
                    *abort_v = 1;
                    break;
                }
                if (*abort_v) break;
                tc_fence_after();
                const uint32_t ahi = base + stage0 + (uint32_t)s * stage_bytes;
                const uint32_t alo = ahi + kKBlockBytes;
                const uint32_t bhi = base, blo = base + wtile;
                const uint32_t d = tmem + (uint32_t)buf * kBpAccCols;
                for (int ks = 0; ks < ks_n; ++ks) {
                    const uint32_t ko = (uint32_t)ks * 32u;
                    const uint32_t acc = ks > 0 ? 1u : 0u;
                    umma_bf16(d, sw128_desc(ahi + ko), sw128_desc(bhi + ko), idesc, acc);
                    umma_bf16(d, sw128_desc(ahi + ko), sw128_desc(blo + ko), idesc, 1u);
                    umma_bf16(d, sw128_desc(alo + ko), sw128_desc(bhi + ko), idesc, 1u);
                }
                umma_commit(smem_u32(&empty_bar[s]));
                umma_commit(smem_u32(&tfull_bar[buf]));
                issued = u + 1;
            }
            if (issued > 0) {
                const long long last = issued - 1;
                if (!mbar_wait_bounded(smem_u32(&empty_bar[(int)(last % kBpStages)]),
                                       (uint32_t)((last / kBpStages) & 1)))
                    *abort_v = 1;
            }
        }
    } else {
        // epilogue: warp w: lane quadrant w % 4, column half (w - first) / 4
        const int e = warp - kEpiWarp0;
        const int quad = warp & 3, half = e >> 2;
        const int m = 32 * quad + lane;
        const uint32_t lane_addr = (uint32_t)(32 * quad) << 16;
        const int c_begin = half * (Np / 32) * 16;                 // multiple of 16
        const int c_end = half == 0 ? c_begin + (Np / 32) * 16 : Np;
        for (long long u = 0; u < ntile; ++u) {
            const int buf = (int)(u & 1);
            if (!mbar_wait_bounded(smem_u32(&tfull_bar[buf]), (uint32_t)((u / 2) & 1))) {
                *abort_v = 1;
                break;
            }
            if (*abort_v) break;
            tc_fence_after();
            const long long pix = (t0 + u) * kTileM + m;
            const unsigned nu = (unsigned)n;
            for (int c = c_begin; c < c_end; c += 16) {
                float v[16];
                tmem_ld16(tmem + lane_addr + (uint32_t)buf * kBpAccCols + (uint32_t)c, v);
                tmem_wait_ld();
                if (pix < n) {
                    unsigned off = (unsigned)c * nu + (unsigned)pix;
                    if (c + 16 <= p) {
#pragma unroll
                        for (int q = 0; q < 16; ++q, off += nu) X[off] = v[q];
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q, off += nu)
                            if (c + q < p) X[off] = v[q];
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&tempty_bar[buf]));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (abort_s && tid == 0) set_status(status, HYDE_ERR_TIMEOUT);
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(2u * kBpAccCols));
    }
}

size_t project_tc_smem(int p) {
    const int KB = (p + 63) / 64;
    return 1024 + 2 * (size_t)KB * kPjN * 128 + (size_t)kPjStages * 2 * kKBlockBytes;
}
size_t backproject_tc_smem(int p) {
    const int Nrows = ((p + 15) / 16 * 16 + 7) / 8 * 8;
    const size_t w = ((2 * (size_t)Nrows * 128) + 1023) / 1024 * 1024;
    return 1024 + w + (size_t)kBpStages * 2 * kKBlockBytes;
}

}  // namespace

bool project_tc_supported(int p, int r_max) {
    return p >= 1 && p <= kMaxBandsGram && r_max >= 1 && r_max <= kPjN &&
           project_tc_smem(p) <= 227 * 1024 && backproject_tc_smem(p) <= 227 * 1024;
}

// the kernels index with 32-bit element offsets
static bool offsets_fit(long long elems) { return elems > 0 && elems < (1LL << 31); }

hyde_status launch_project_pad_tc(const float* Y, int p, int H, int W, const float* P, int r,
                                  int ldw, float* Zp, int Hp, int Wp, int* status,
                                  cudaStream_t s) {
    if (!project_tc_supported(p, r)) return HYDE_ERR_SHAPE;
    if (!offsets_fit((long long)p * H * W) || !offsets_fit((long long)kPjN * Hp * Wp))
        return HYDE_ERR_SHAPE;
    const size_t smem = project_tc_smem(p);
    if (ensure_smem_limit((const void*)project_tc_kernel, (int)smem) != cudaSuccess)
        return HYDE_ERR_CUDA;
    const long long tiles = ((long long)Hp * Wp + kTileM - 1) / kTileM;
    long long grid = device_sm_count();
    if (grid <= 0) return HYDE_ERR_CUDA;
    if (grid > tiles) grid = tiles;
    launch_pdl(project_tc_kernel, (int)grid, kPjThreads, smem, s, Y, p, H, W, P, r, ldw, Zp, Hp,
               Wp, 0, status);
    return cuda_status(cudaGetLastError());
}

hyde_status launch_backproject_tc(const float* Zh, long long n, const float* Q, int p, int ldw,
                                  const int* rank, float* X, int* status, cudaStream_t s) {
    if (!project_tc_supported(p, ldw > kBpK ? kBpK : ldw)) return HYDE_ERR_SHAPE;
    if (!offsets_fit((long long)(p > kBpK ? p : kBpK) * n)) return HYDE_ERR_SHAPE;
    const size_t smem = backproject_tc_smem(p);
    if (ensure_smem_limit((const void*)backproject_tc_kernel, (int)smem) != cudaSuccess)
        return HYDE_ERR_CUDA;
    const long long tiles = (n + kTileM - 1) / kTileM;
    long long grid = device_sm_count();
    if (grid <= 0) return HYDE_ERR_CUDA;
    if (grid > tiles) grid = tiles;
    launch_pdl(backproject_tc_kernel, (int)grid, kBpThreads, smem, s, Zh, n, Q, p, ldw, rank, X,
               status);
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

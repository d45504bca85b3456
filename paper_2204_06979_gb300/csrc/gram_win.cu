// Gram matrices R_w = Y_w^T Y_w of every window of a batched sliding-window
// call on the 5th-generation tensor cores (the spectral statistics of HyRes,
// arXiv 2204.06979 Sec. 2.1, for each tile of a scene that is denoised in
// tiles, Sec. 2.2.2), with a four-term split-BF16 product: y = hi + lo + e,
// hi = bf16_rn(y), lo = bf16_rn(y - hi), |e| <= 2^-18 |y| (unbiased), and
// y_a y_b ~ hi hi + hi lo + lo hi + lo lo, every term exact in FP32, on
// kind::f16 MMAs (K = 16 per instruction) into TMEM windows of one 64-pixel
// chunk, each window drained into FP32 registers. The per-instruction cost
// of the MMAs, not their arithmetic, bounds this kernel at these shapes:
// split-TF32 (three products at K = 8) issues 50 % more instructions per
// pixel and drops the lo lo term.
//
// The data path:
//  * the windows are read in place from the scene Y [p][H][W] through one
//    3D tensor map (x, y, band); a chunk is a 32 x 2 pixel block of one
//    window, a box {32, 2, bands} that lands as [band][64 floats];
//  * six converter warps split each chunk into the hi and lo tiles in the
//    128-byte-swizzled K-major layout (one 128-byte row of 64 bf16 per
//    band), pixels outside the window set to zero;
//  * the bands split into two roles so that the accumulators of one CTA fit
//    its registers for p up to 208: role 0 computes rows [0, 128) of R
//    against all bands (one MMA of N = round16(p) per product), role 1 the
//    Gram matrix of the bands [128, p) (rows [128, p) against columns
//    [128, p)). The two roles are CTAs of the same launch;
//  * the chunks of all windows, window after window, form one sequence per
//    role that is cut into equal contiguous ranges, one per CTA. A CTA's
//    range crosses a few window boundaries; each (window, range) piece ends
//    with the drain warps writing their FP32 sums to the piece's own partial,
//    and a second kernel adds a window's partials in double in piece order.
// Measured on the 2048 x 2048 x 200 scene (512 windows): split-TF32 with two
// converter warps 5.6 ms (the converters busy ~2.7k of ~3.6k cycles per
// 32-pixel chunk), with six converter warps 3.9 ms (the MMA issue ~115-140
// cycles per instruction, whatever N).
// Every mbarrier wait is bounded in time; a timeout sets HYDE_ERR_TIMEOUT and
// every role winds down (waiting, bounded, for its own copies and MMAs in
// flight) before the CTA frees its TMEM.
#include <algorithm>
#include <vector>

#include "hyde_internal.cuh"
#include "tc_common.cuh"
#include "tmap.cuh"

namespace hyde {
namespace {

constexpr int kK = 64;                 // pixels per chunk: one 128-byte row of bf16
constexpr int kCx = 32, kCy = 2;       // chunk: 32 x 2 pixels of one window
constexpr int kOpStages = 2;
constexpr int kMaxRaw = 8;
constexpr int kWin = 1;                // chunks per TMEM accumulation window (64 pixels)
// Warp roles: warpgroups 0-1 hold the TMA warp, the MMA warp and six
// converter warps, warpgroups 2-3 the eight drain warps. The drain warps
// keep up to 112 FP32 sums each; the block is launched with 128 registers
// per thread, then warpgroups 0-1 release down to kLowRegs and 2-3 take up
// to kHighRegs (setmaxnreg), which adds up to the launch's 65536 exactly.
constexpr int kTmaWarp = 0, kMmaWarp = 1, kCvtWarp0 = 2, kCvtWarps = 6;
constexpr int kDrainWarp0 = kCvtWarp0 + kCvtWarps, kDrainWarps = 8;
constexpr int kWgThreads = (kDrainWarp0 + kDrainWarps) * 32;
constexpr int kLaunchRegs = 128, kLowRegs = 64, kHighRegs = 192;
static_assert(kWgThreads == 512, "four warpgroups");
static_assert(256 * kLowRegs + 256 * kHighRegs == kWgThreads * kLaunchRegs,
              "the register split must add up to the launch allocation");
constexpr int kMaxP = 208;

struct WgRole {
    int band0, nb;        // bands [band0, band0 + nb) are loaded
    int rows;             // rows of an operand tile (>= 128, >= the MMA's N)
    int raw_stages;
    uint32_t raw_stage_bytes, op_bytes;
    int buf_cols, tmem_cols;
    int out_rows, out_cols;   // a piece's partial: out_rows x out_cols floats
};

struct WgParams {
    WgRole role[2];
    int G0;                   // CTAs [0, G0) take role 0, the rest role 1
    unsigned long long wait_ns;
};

// One CTA of role `R` (NT = the MMA's N). Pieces pbeg[g] .. pbeg[g + 1] - 1
// of `pieces` (x: window, y, z: chunk range, w: partial slot); geo[window] =
// (y0, x0, h, w) in scene pixels.
template <int NT>
__device__ __forceinline__ void win_gram_role(const CUtensorMap* tmap, const int4* __restrict__ pieces,
                                              int q0, int q1, const int4* __restrict__ geo,
                                              const WgRole& P, unsigned long long wait_ns,
                                              float* __restrict__ partials, int* status,
                                              uint8_t* smem_raw) {
    constexpr int NB16 = NT / 16;
    constexpr int KB = (NB16 + 1) / 2;   // column blocks of a drain group
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
    // then the raw stages ([band][64 floats], as TMA writes them)
    const uint32_t op_area = 2u * kOpStages * P.op_bytes;
    const uint32_t rawb = base + op_area;
    const uint32_t all_area = op_area + (uint32_t)P.raw_stages * P.raw_stage_bytes;
    volatile int* abort_v = &abort_s;
    const int RS = P.raw_stages;

    for (uint32_t e = tid; e < all_area / 16; e += kWgThreads)   // rows >= nb stay zero
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

    if (warp < kDrainWarp0) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(kLowRegs));
    if (warp == kTmaWarp) {
        // ------------------------------------------------------ TMA loads
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmap))
                         : "memory");
            const uint32_t bytes = (uint32_t)P.nb * (uint32_t)(kK * 4);
            long long it = 0, issued = 0;
            bool stop = false;
            for (int q = q0; q < q1 && !stop; ++q) {
                const int4 pc = pieces[q];
                const int4 g = geo[pc.x];
                const int nx = (g.w + kCx - 1) / kCx;
                for (int c = pc.y; c < pc.z; ++c, ++it) {
                    if (*abort_v) { stop = true; break; }
                    const int s = (int)(it % RS);
                    if (it >= RS && !mbar_wait_bounded(smem_u32(&raw_empty[s]),
                                                       (uint32_t)((it / RS - 1) & 1), wait_ns)) {
                        *abort_v = 1;
                        stop = true;
                        break;
                    }
                    const uint32_t bar = smem_u32(&raw_full[s]);
                    mbar_arrive_expect_tx(bar, bytes);
                    const int cy = c / nx, cx = c - cy * nx;
                    tma_load_3d(rawb + (uint32_t)s * P.raw_stage_bytes, tmap, g.y + kCx * cx,
                                g.x + kCy * cy, P.band0, bar);   // x0 + 32 cx: 16-byte aligned
                    issued = it + 1;
                }
            }
            // every issued load must have landed before the CTA moves on
            const long long first = issued > RS ? issued - RS : 0;
            for (long long i = first; i < issued; ++i)
                if (!mbar_wait_bounded(smem_u32(&raw_full[(int)(i % RS)]),
                                       (uint32_t)((i / RS) & 1), kWaitNs))
                    *abort_v = 1;
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------ MMA issue (1 thread)
        if (lane == 0) {
            const uint32_t idT = idesc_bf16(128, NT);
            long long it = 0, issued = 0, wg = 0;
            bool stop = false;
            for (int q = q0; q < q1 && !stop; ++q) {
                const int4 pc = pieces[q];
                const int len = pc.z - pc.y;
                for (int j = 0; j < len; ++j, ++it) {
                    if (*abort_v) { stop = true; break; }
                    const int o = (int)(it % kOpStages);
                    const bool first = (j % kWin) == 0;
                    const bool last = (j % kWin) == kWin - 1 || j == len - 1;
                    const int b = (int)(wg & 1);
                    if (!mbar_wait_bounded(smem_u32(&op_full[o]),
                                           (uint32_t)((it / kOpStages) & 1), wait_ns)) {
                        *abort_v = 1;
                        stop = true;
                        break;
                    }
                    if (first && wg >= 2 &&
                        !mbar_wait_bounded(smem_u32(&acc_empty[b]), (uint32_t)((wg / 2 - 1) & 1),
                                           wait_ns)) {
                        *abort_v = 1;
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t hi = base + (uint32_t)o * 2u * P.op_bytes, lo = hi + P.op_bytes;
                    const uint32_t d = tmem + (uint32_t)b * (uint32_t)P.buf_cols;
#pragma unroll
                    for (int kk = 0; kk < kK / 16; ++kk) {
                        const uint32_t ko = (uint32_t)kk * 32u;   // 16 bf16 along K
                        const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
                        umma_bf16(d, sw128_desc(hi + ko), sw128_desc(hi + ko), idT, acc);
                        umma_bf16(d, sw128_desc(hi + ko), sw128_desc(lo + ko), idT, 1u);
                        umma_bf16(d, sw128_desc(lo + ko), sw128_desc(hi + ko), idT, 1u);
                        umma_bf16(d, sw128_desc(lo + ko), sw128_desc(lo + ko), idT, 1u);
                    }
                    umma_commit(smem_u32(&op_empty[o]));
                    if (last) {
                        umma_commit(smem_u32(&acc_full[b]));
                        ++wg;
                    }
                    issued = it + 1;
                }
            }
            // MMAs complete in order: the last commit covers every one issued
            if (issued > 0 &&
                !mbar_wait_bounded(smem_u32(&op_empty[(int)((issued - 1) % kOpStages)]),
                                   (uint32_t)(((issued - 1) / kOpStages) & 1),
                                   wait_ns > kWaitNs ? wait_ns : kWaitNs))
                *abort_v = 1;
        }
    } else {
        // ------------------------------------ split into hi and lo, mask the window
        const int ct = tid - kCvtWarp0 * 32;
        long long it = 0;
        bool stop = false;
        for (int q = q0; q < q1 && !stop; ++q) {
            const int4 pc = pieces[q];
            const int4 g = geo[pc.x];
            const int nx = (g.w + kCx - 1) / kCx;
            for (int c = pc.y; c < pc.z; ++c, ++it) {
                if (*abort_v) { stop = true; break; }
                const int s = (int)(it % RS), o = (int)(it % kOpStages);
                if (!mbar_wait_bounded(smem_u32(&raw_full[s]), (uint32_t)((it / RS) & 1),
                                       wait_ns)) {
                    *abort_v = 1;
                    stop = true;
                    break;
                }
                if (it >= kOpStages &&
                    !mbar_wait_bounded(smem_u32(&op_empty[o]),
                                       (uint32_t)((it / kOpStages - 1) & 1), wait_ns)) {
                    *abort_v = 1;
                    stop = true;
                    break;
                }
                const int cy = c / nx, cx = c - cy * nx;
                const int rv = min(kCy, g.z - kCy * cy), cv = min(kCx, g.w - kCx * cx);
                const float* raw = reinterpret_cast<const float*>(
                    gbase + (op_area + (uint32_t)s * P.raw_stage_bytes));
                uint8_t* hi_t = gbase + (uint32_t)o * 2u * P.op_bytes;
                uint8_t* lo_t = hi_t + P.op_bytes;
                // item (b, k8): pixels 8 k8 .. 8 k8 + 7 of band b (window row
                // k8 / 4, columns 8 (k8 % 4) ..), one 16-byte chunk of the
                // swizzled bf16 row in each tile; pixels outside the window
                // are zero. The 32-byte stride of the reads costs bank
                // conflicts (22.9M of 42M shared wavefronts in a capture), but
                // one float4 per lane with 8-byte stores measured slower
                // (1.38 against 1.33 ms per window group).
                constexpr int kStep = kCvtWarps * 32, kU = 2;
                const int nit = P.nb * 8;
                for (int g0 = ct; g0 < nit; g0 += kU * kStep) {
                    float4 va[kU], vb[kU];
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        const int gi = g0 + u * kStep;
                        const float* src = raw + (gi < nit ? gi : 0) * 8;
                        va[u] = *reinterpret_cast<const float4*>(src);
                        vb[u] = *reinterpret_cast<const float4*>(src + 4);
                    }
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        const int gi = g0 + u * kStep;
                        if (gi >= nit) break;
                        const int b = gi >> 3, k8 = gi & 7;
                        const int row = k8 >> 2, col0 = (k8 & 3) * 8;
                        float v[8] = {va[u].x, va[u].y, va[u].z, va[u].w,
                                      vb[u].x, vb[u].y, vb[u].z, vb[u].w};
                        if (row >= rv || col0 + 8 > cv) {
#pragma unroll
                            for (int e = 0; e < 8; ++e)
                                if (row >= rv || col0 + e >= cv) v[e] = 0.f;
                        }
                        uint32_t h[4], l[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) split_pair(v[2 * e], v[2 * e + 1], h[e], l[e]);
                        const uint32_t off = (uint32_t)b * 128u + ((uint32_t)(k8 ^ (b & 7)) << 4);
                        *reinterpret_cast<uint4*>(hi_t + off) = make_uint4(h[0], h[1], h[2], h[3]);
                        *reinterpret_cast<uint4*>(lo_t + off) = make_uint4(l[0], l[1], l[2], l[3]);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(smem_u32(&op_full[o]));
                mbar_arrive(smem_u32(&raw_empty[s]));
            }
        }
    }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(kHighRegs));
        // ---------------------------------------------------- drain warps
        // Drain group grp (warps 8-11 or 12-15) owns TMEM lane `row` (the
        // band band0 + row) and the column blocks grp, grp + 2, ...; at the
        // end of a piece it writes its sums to the piece's partial.
        const int dw = warp - kDrainWarp0, grp = dw >> 2;
        const int quad = warp & 3;
        const int row = 32 * quad + lane;
        const uint32_t lane_addr = (uint32_t)(32 * quad) << 16;
        float acc[16 * KB];
#pragma unroll
        for (int c = 0; c < 16 * KB; ++c) acc[c] = 0.f;
        long long wg = 0;
        bool stop = false;
        for (int q = q0; q < q1 && !stop; ++q) {
            const int4 pc = pieces[q];
            const int len = pc.z - pc.y;
            const int nw = (len + kWin - 1) / kWin;
            for (int j = 0; j < nw; ++j, ++wg) {
                if (*abort_v) { stop = true; break; }
                const int b = (int)(wg & 1);
                if (!mbar_wait_bounded(smem_u32(&acc_full[b]), (uint32_t)((wg / 2) & 1),
                                       wait_ns)) {
                    *abort_v = 1;
                    stop = true;
                    break;
                }
                __syncwarp();
                tc_fence_after();
                const uint32_t t0 = tmem + lane_addr + (uint32_t)b * (uint32_t)P.buf_cols;
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    const int cb = grp + 2 * k;
                    if (cb < NB16) {
                        uint32_t r[16];
                        tmem_ld16_nowait(t0 + (uint32_t)(16 * cb), r);
                        tmem_wait_ld();
#pragma unroll
                        for (int e = 0; e < 16; ++e) acc[16 * k + e] += __uint_as_float(r[e]);
                    }
                }
                tc_fence_before();
                mbar_arrive(smem_u32(&acc_empty[b]));
            }
            if (stop) break;
            // the piece is complete: write its partial, start the next from zero
            float* out = partials + (long long)pc.w * P.out_rows * P.out_cols;
            if (row < P.out_rows) {
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    const int cb = grp + 2 * k;
                    if (cb < NB16) {
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int col = 16 * cb + e;
                            if (col < P.out_cols) out[(long long)row * P.out_cols + col] = acc[16 * k + e];
                        }
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 16 * KB; ++c) acc[c] = 0.f;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (abort_s && tid == 0) set_status(status, HYDE_ERR_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)P.tmem_cols));
    }
}

// CTAs [0, G0) run role 0 (N = NT0), the others role 1 (N = NT0 - 128).
template <int NT0>
__global__ void __launch_bounds__(kWgThreads, 1)
win_gram_kernel(const __grid_constant__ CUtensorMap tmap0, const __grid_constant__ CUtensorMap tmap1,
                const int4* __restrict__ pieces, const int* __restrict__ pbeg,
                const int4* __restrict__ geo, WgParams W, float* __restrict__ part0,
                float* __restrict__ part1, int* status) {
    pdl_wait();
    extern __shared__ uint8_t smem_raw[];
    const int g = blockIdx.x;
    const int q0 = pbeg[g], q1 = pbeg[g + 1];
    if (g < W.G0) {
        win_gram_role<NT0>(&tmap0, pieces, q0, q1, geo, W.role[0], W.wait_ns, part0, status,
                           smem_raw);
    } else {
        if constexpr (NT0 > 128)
            win_gram_role<NT0 - 128>(&tmap1, pieces, q0, q1, geo, W.role[1], W.wait_ns, part1,
                                     status, smem_raw);
    }
    pdl_trigger();
}

// R_w[i][j] = R_w[j][i] (j >= i) = sum of the window's partials in piece
// order, in double: rows i < 128 from role 0's partials (p columns), rows
// i >= 128 from role 1's (p - 128 columns). Block (x, w): rows 8x .. 8x + 7
// of window w, one warp per row.
__global__ void __launch_bounds__(256)
win_gram_reduce_kernel(const float* __restrict__ part0, const float* __restrict__ part1,
                       const int* __restrict__ wslot0, const int* __restrict__ wslot1, int p,
                       double* __restrict__ R, int* status) {
    pdl_wait();
    pdl_trigger();
    const int w = blockIdx.y, lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= p) return;
    double* Rw = R + (long long)w * p * p;
    const bool top = i < 128;
    const int s0 = top ? wslot0[w] : wslot1[w], s1 = top ? wslot0[w + 1] : wslot1[w + 1];
    const float* part = top ? part0 : part1;
    const int cols = top ? p : p - 128, r = top ? i : i - 128, c0 = top ? 0 : 128;
    const long long psz = (long long)(top ? (p < 128 ? p : 128) : p - 128) * cols;
    for (int j = i + lane; j < p; j += 32) {
        double s = 0.0;
        for (int q = s0; q < s1; ++q) s += (double)__ldg(part + q * psz + (long long)r * cols + (j - c0));
        if (!isfinite(s)) set_status(status, HYDE_ERR_NUMERIC);
        Rw[(long long)i * p + j] = s;
        Rw[(long long)j * p + i] = s;
    }
}

bool role_plan(int p, int band0, int nb, int NT, WgRole* r, size_t* smem) {
    WgRole R = {};
    R.band0 = band0;
    R.nb = nb;
    R.rows = NT > 128 ? NT : 128;
    R.op_bytes = (uint32_t)R.rows * 128u;   // one bf16 tile: rows x 64 pixels, swizzled
    R.raw_stage_bytes = (uint32_t)align_up((size_t)nb * kK * 4, 1024);
    R.buf_cols = (int)align_up((size_t)NT, 32);
    const int need = 2 * R.buf_cols;
    if (need > 512) return false;
    R.tmem_cols = need <= 32 ? 32 : need <= 64 ? 64 : need <= 128 ? 128 : need <= 256 ? 256 : 512;
    R.out_rows = nb < 128 ? nb : 128;
    R.out_cols = band0 == 0 ? p : nb;
    const size_t room = 227 * 1024 - 1024 - 1024;   // alignment slack, static shared memory
    const size_t op_area = 2u * kOpStages * R.op_bytes;
    if (op_area + 2 * R.raw_stage_bytes > room) return false;
    const int rs = (int)((room - op_area) / R.raw_stage_bytes);
    R.raw_stages = rs > kMaxRaw ? kMaxRaw : rs;
    *smem = 1024 + op_area + (size_t)R.raw_stages * R.raw_stage_bytes;
    *r = R;
    return true;
}

int nt0_of(int p) {
    if (p <= 32) return 32;
    if (p <= 64) return 64;
    if (p <= 128) return 128;
    return (p + 15) / 16 * 16;
}

}  // namespace

bool win_gram_supported(int p, int W, const float* Y) {
    return p >= 1 && p <= kMaxP && (W % 4) == 0 && ((uintptr_t)Y % 16) == 0 &&
           encode_tiled_fn() != nullptr;
}

// Host plan of the pieces: the chunks of all windows (window by window, each
// window's 32 x 2 blocks row by row) cut into G0 equal ranges for role 0 and
// G1 for role 1. CTAs go to the roles in proportion to their work per chunk
// (bands loaded + the MMA's N), role 1's weighted by w1x: its MMAs
// (N = p - 128) cost nearly as much per instruction as role 0's, so it
// needs more CTAs than its arithmetic (the batched plan tunes w1x; 1.6 on
// the 2048 x 2048 x 200 scene: 2.57 ms against 2.88 at 1.2 and 2.91 at 2.2).
hyde_status win_gram_layout(int p, const int4* geo, int n_win, int sms, double w1x,
                            WinGramLayout* L) {
    if (p < 1 || p > kMaxP || n_win < 1 || sms < 1) return HYDE_ERR_SHAPE;
    for (int w = 0; w < n_win; ++w)
        if (geo[w].z < 1 || geo[w].w < 1 || (geo[w].y % 4) != 0) return HYDE_ERR_SHAPE;
    const bool two = p > 128;
    if (!(w1x > 0.0)) return HYDE_ERR_INVALID_ARG;
    const double w0 = (double)p + nt0_of(p),
                 w1 = two ? w1x * ((double)(p - 128) + (nt0_of(p) - 128)) : 0.0;
    int G0 = two ? (int)(sms * w0 / (w0 + w1) + 0.5) : sms;
    if (G0 < 1) G0 = 1;
    if (two && G0 > sms - 1) G0 = sms - 1;
    const int G1 = two ? sms - G0 : 0;
    std::vector<long long> start(n_win + 1, 0);
    for (int w = 0; w < n_win; ++w) {
        const long long nc = (long long)((geo[w].z + kCy - 1) / kCy) * ((geo[w].w + kCx - 1) / kCx);
        start[w + 1] = start[w] + nc;
    }
    const long long tot = start[n_win];
    L->pieces.clear();
    L->pbeg.assign(G0 + G1 + 1, 0);
    L->wslot0.assign(n_win + 1, 0);
    L->wslot1.assign(n_win + 1, 0);
    int slots[2] = {0, 0};
    for (int role = 0; role < (two ? 2 : 1); ++role) {
        const int G = role == 0 ? G0 : G1, goff = role == 0 ? 0 : G0;
        std::vector<int>& ws = role == 0 ? L->wslot0 : L->wslot1;
        std::vector<int> first_slot(n_win, -1), count(n_win, 0);
        for (int g = 0; g < G; ++g) {
            L->pbeg[goff + g] = (int)L->pieces.size();
            const long long a = tot * g / G, b = tot * (g + 1) / G;
            // windows overlapping [a, b)
            int w = (int)(std::upper_bound(start.begin(), start.end(), a) - start.begin()) - 1;
            for (; w < n_win && start[w] < b; ++w) {
                const long long lo = a > start[w] ? a : start[w];
                const long long hi = b < start[w + 1] ? b : start[w + 1];
                if (hi <= lo) continue;
                const int slot = slots[role]++;
                if (first_slot[w] < 0) first_slot[w] = slot;
                ++count[w];
                L->pieces.push_back(make_int4(w, (int)(lo - start[w]), (int)(hi - start[w]), slot));
            }
        }
        // a window's pieces are consecutive slots
        for (int w = 0; w < n_win; ++w) ws[w + 1] = ws[w] + count[w];
        for (int w = 0; w < n_win; ++w)
            if (count[w] > 0 && first_slot[w] != ws[w]) return HYDE_ERR_SHAPE;
    }
    L->pbeg[G0 + G1] = (int)L->pieces.size();
    L->G0 = G0;
    L->G1 = G1;
    L->nslot0 = slots[0];
    L->nslot1 = slots[1];
    L->part0_floats = (size_t)slots[0] * (p < 128 ? p : 128) * p;
    L->part1_floats = two ? (size_t)slots[1] * (p - 128) * (p - 128) : 0;
    return HYDE_OK;
}

hyde_status launch_win_gram(const float* Y, int p, int H, int W, const int4* pieces,
                            const int* pbeg, const int4* geo, const int* wslot0,
                            const int* wslot1, int n_win, int G0, int G1, float* part0,
                            float* part1, double* R, int* status, cudaStream_t s) {
    if (!win_gram_supported(p, W, Y)) return HYDE_ERR_SHAPE;
    EncodeTiledFn enc = encode_tiled_fn();
    const int NT0 = nt0_of(p);
    const bool two = p > 128;
    WgParams Wp = {};
    size_t sm0 = 0, sm1 = 0;
    if (!role_plan(p, 0, p, NT0, &Wp.role[0], &sm0)) return HYDE_ERR_SHAPE;
    if (two && !role_plan(p, 128, p - 128, NT0 - 128, &Wp.role[1], &sm1)) return HYDE_ERR_SHAPE;
    Wp.G0 = G0;
    Wp.wait_ns = wait_limit_ns();
    const size_t smem = sm0 > sm1 ? sm0 : sm1;
    CUtensorMap tm[2];
    for (int r = 0; r < (two ? 2 : 1); ++r) {
        const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)p};
        const cuuint64_t strides[2] = {(cuuint64_t)W * 4, (cuuint64_t)H * W * 4};
        const cuuint32_t box[3] = {(cuuint32_t)kCx, (cuuint32_t)kCy, (cuuint32_t)Wp.role[r].nb};
        const cuuint32_t estr[3] = {1, 1, 1};
        if (enc(&tm[r], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(Y), dims, strides,
                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return HYDE_ERR_CUDA;
    }
    if (!two) tm[1] = tm[0];
    auto go = [&](auto kernel) -> hyde_status {
        if (ensure_smem_limit((const void*)kernel, (int)smem) != cudaSuccess) return HYDE_ERR_CUDA;
        // the setmaxnreg split assumes exactly kLaunchRegs registers per thread at launch
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, (const void*)kernel) != cudaSuccess ||
            fa.numRegs != kLaunchRegs)
            return HYDE_ERR_CUDA;
        launch_pdl(kernel, G0 + G1, kWgThreads, smem, s, tm[0], tm[1], pieces, pbeg, geo, Wp,
                   part0, part1, status);
        return HYDE_OK;
    };
    hyde_status st;
    switch (NT0) {
        case 32: st = go(win_gram_kernel<32>); break;
        case 64: st = go(win_gram_kernel<64>); break;
        case 128: st = go(win_gram_kernel<128>); break;
        case 144: st = go(win_gram_kernel<144>); break;
        case 160: st = go(win_gram_kernel<160>); break;
        case 176: st = go(win_gram_kernel<176>); break;
        case 192: st = go(win_gram_kernel<192>); break;
        case 208: st = go(win_gram_kernel<208>); break;
        default: return HYDE_ERR_SHAPE;
    }
    if (st != HYDE_OK) return st;
    launch_pdl(win_gram_reduce_kernel, dim3((p + 7) / 8, n_win), 256, 0, s, part0, part1, wslot0,
               wslot1, p, R, status);
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

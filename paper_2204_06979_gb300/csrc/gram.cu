// Gram matrix R = Y^T Y of the n x p pixel-by-band matrix (the spectral
// statistics of HyRes's low-rank model, arXiv 2204.06979 Sec. 2.1).
//
// Plain FP32 SIMT design. The symmetric p x p result is cut into 8 x 8 tiles;
// one thread owns one tile of the upper triangle (PT(PT+1)/2 tiles for
// PT = ceil(p/8)), so each thread does 64 FMAs per pixel from 16 float4
// shared-memory loads. A block walks a contiguous range of 32-pixel chunks
// through a 3-stage cp.async pipeline (each warp copies a fixed set of
// bands, one band's 32 consecutive pixels per copy instruction) into a
// swizzled shared buffer, so that the 8 rows a thread reads are spread over
// all 32 banks. Each block writes its float
// partial; a second kernel sums the partials in double and mirrors the
// triangle.

#include "hyde_internal.cuh"

namespace hyde {
namespace {

constexpr int KC = 32;        // pixels per chunk
constexpr int KC84 = 64;      // pixels per chunk of the 8 x 4 kernel (one barrier each);
                              // the copy below fills it as two 32-pixel halves
static_assert(KC84 == 64, "gram_partial84_kernel copies a chunk as two 32-pixel halves");
constexpr int STAGES = 3;     // cp.async pipeline depth
constexpr int kGramMaxThreads = 544;

__device__ __forceinline__ void tile_of(int t, int PT, int& ti, int& tj) {
    // row-major enumeration of the upper triangle: row ti holds PT - ti tiles
    int row = 0, rem = t, len = PT;
    while (rem >= len) { rem -= len; ++row; --len; }
    ti = row;
    tj = row + rem;
}

// Shared layout: band b occupies one 128-byte row of 8 float4 (32 pixels);
// logical float4 column q is stored at q ^ ((b >> 3) & 7).

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? 4 : 0;   // zero-fill outside the cube
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Rows of Y are only 4-byte aligned when n is odd, so the copies are 4-byte
// cp.async (a warp still covers one band's 32 consecutive pixels: 128 B).
template <int MAXT>
__global__ void __launch_bounds__(MAXT, (MAXT <= 256 ? 2 : 1))
gram_partial_kernel(const float* __restrict__ Y, int p, long long n, int PT,
                    int ntiles, long long chunks_per_block,
                    float* __restrict__ partials) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float4 sm4[];
    const int p8 = PT * 8;
    const int t = threadIdx.x;
    const int T = blockDim.x;

    // padded bands p..p8-1 stay zero in every stage
    for (int i = t; i < (p8 - p) * 8 * STAGES; i += T) {
        const int st = i / ((p8 - p) * 8), o = i % ((p8 - p) * 8);
        sm4[st * p8 * 8 + p * 8 + o] = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    const long long nchunks = (n + KC - 1) / KC;
    // even split: block b takes chunks [b N / G, (b + 1) N / G)
    const long long c0 = (long long)blockIdx.x * nchunks / gridDim.x;
    const long long c1 = (long long)(blockIdx.x + 1) * nchunks / gridDim.x;
    (void)chunks_per_block;

    // Copy of one chunk: warp w copies bands w, w + nw, ...; lane k copies
    // pixel k of each (128 contiguous bytes per band), so the source pointer
    // just advances by nw bands and the destination offset needs the band's
    // swizzle only.
    const int lane = t & 31, wrp = t >> 5, nw = T >> 5;
    const int kq = lane >> 2, kr = lane & 3;
    const long long bstride = (long long)nw * n;
    auto issue = [&](long long c, int st) {
        float* d = reinterpret_cast<float*>(sm4 + st * p8 * 8);
        const long long pix = c * KC + lane;
        const bool ok = pix < n;
        const float* src = Y + (long long)wrp * n + (ok ? pix : 0);
        for (int b = wrp; b < p; b += nw, src += bstride)
            cp_async4(d + b * 32 + ((kq ^ ((b >> 3) & 7)) << 2) + kr, src, ok);
    };

    const bool active = t < ntiles;
    int ti = 0, tj = 0;
    if (active) tile_of(t, PT, ti, tj);

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (c0 + s < c1) issue(c0 + s, s);
        cp_async_commit();
    }
    for (long long c = c0; c < c1; ++c) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();   // chunk c visible to all; stage (c-1)%STAGES is free
        const long long nxt = c + STAGES - 1;
        if (nxt < c1) issue(nxt, (int)(nxt - c0) % STAGES);
        cp_async_commit();
        if (active) {
            // rows 8ti.. and 8tj.. of the stage; logical float4 column q sits
            // at q ^ (ti & 7) and q ^ (tj & 7) respectively
            const float4* B = sm4 + ((int)(c - c0) % STAGES) * p8 * 8;
            const float4* Ba = B + 64 * ti;
            const float4* Bb = B + 64 * tj;
            const int xa = ti & 7, xb = tj & 7;
#pragma unroll 1
            for (int q = 0; q < 8; ++q) {
                const int qa = q ^ xa, qb = q ^ xb;
                float4 a[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = Ba[8 * i + qa];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 bv = Bb[8 * j + qb];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        acc[i][j] = fmaf(a[i].x, bv.x, acc[i][j]);
                        acc[i][j] = fmaf(a[i].y, bv.y, acc[i][j]);
                        acc[i][j] = fmaf(a[i].z, bv.z, acc[i][j]);
                        acc[i][j] = fmaf(a[i].w, bv.w, acc[i][j]);
                    }
                }
            }
        }
    }
    cp_async_wait<0>();

    if (active) {
        float4* out = reinterpret_cast<float4*>(
            partials + ((long long)blockIdx.x * ntiles + t) * 64);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            out[2 * i] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            out[2 * i + 1] = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
        }
    }
}

// Variant with 8 x 4 tiles (rows 8ti.., columns 4tj.., tj >= 2ti: PT (PT+1)
// tiles) and paired FP32 FMAs: fma.rn.f32x2 updates an (even pixel, odd
// pixel) accumulator pair of one (i, j) from the (x, y) or (z, w) halves of
// the float4 operands, so 128 FMAs of four pixels take 64 instructions. The
// stage rows are swizzled by (b >> 2) & 7 so that the 4-row B tiles of a
// warp's lanes fall on different float4 columns.

__device__ __forceinline__ void tile84_of(int t, int PT, int& ti, int& tj) {
    // row ti holds the 2 PT - 2 ti tiles tj = 2 ti .. 2 PT - 1
    int row = 0, rem = t, len = 2 * PT;
    while (rem >= len) { rem -= len; ++row; len -= 2; }
    ti = row;
    tj = 2 * row + rem;
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
gram_partial84_kernel(const float* __restrict__ Y, int p, long long n, int PT, int ntiles,
                      float* __restrict__ partials) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ float4 sm4[];
    const int p8 = PT * 8;
    const int t = threadIdx.x;
    const int T = blockDim.x;
    constexpr int RQ = KC84 / 4;   // float4 per stage row
    for (int i = t; i < (p8 - p) * RQ * STAGES; i += T) {
        const int st = i / ((p8 - p) * RQ), o = i % ((p8 - p) * RQ);
        sm4[st * p8 * RQ + p * RQ + o] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const long long nchunks = (n + KC84 - 1) / KC84;
    const long long c0 = (long long)blockIdx.x * nchunks / gridDim.x;
    const long long c1 = (long long)(blockIdx.x + 1) * nchunks / gridDim.x;
    const int lane = t & 31, wrp = t >> 5, nw = T >> 5;
    const int kq = lane >> 2, kr = lane & 3;
    const long long bstride = (long long)nw * n;
    // a warp copies 32 + 32 consecutive pixels of each of its bands; float4
    // column kq of a row is stored at kq ^ ((b >> 2) & 7) (the XOR keeps each
    // half of the row in place)
    auto issue = [&](long long c, int st) {
        float* d = reinterpret_cast<float*>(sm4 + st * p8 * RQ);
        const long long pix = c * KC84 + lane;
        const bool ok0 = pix < n, ok1 = pix + 32 < n;
        const float* src0 = Y + (long long)wrp * n + (ok0 ? pix : 0);
        const float* src1 = Y + (long long)wrp * n + (ok1 ? pix + 32 : 0);
        for (int b = wrp; b < p; b += nw, src0 += bstride, src1 += bstride) {
            float* row = d + b * KC84 + (((kq ^ ((b >> 2) & 7))) << 2) + kr;
            cp_async4(row, src0, ok0);
            cp_async4(row + 32, src1, ok1);
        }
    };
    const bool active = t < ntiles;
    int ti = 0, tj = 0;
    if (active) tile84_of(t, PT, ti, tj);
    float ae[8][4], ao[8][4];   // even / odd pixel accumulators
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ae[i][j] = ao[i][j] = 0.f;
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (c0 + s < c1) issue(c0 + s, s);
        cp_async_commit();
    }
    for (long long c = c0; c < c1; ++c) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        const long long nxt = c + STAGES - 1;
        if (nxt < c1) issue(nxt, (int)(nxt - c0) % STAGES);
        cp_async_commit();
        if (active) {
            const float4* B = sm4 + ((int)(c - c0) % STAGES) * p8 * RQ;
            const float4* Ba = B + 8 * RQ * ti;   // rows 8ti .. 8ti+7
            const float4* Bb = B + 4 * RQ * tj;   // rows 4tj .. 4tj+3
            const int xa0 = (2 * ti) & 7, xa1 = (2 * ti + 1) & 7, xb = tj & 7;
#pragma unroll 2
            for (int q = 0; q < RQ; ++q) {
                float4 a[8], b[4];
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = Ba[RQ * i + (q ^ (i < 4 ? xa0 : xa1))];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = Bb[RQ * j + (q ^ xb)];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        fma_f32x2(ae[i][j], ao[i][j], a[i].x, a[i].y, b[j].x, b[j].y);
                        fma_f32x2(ae[i][j], ao[i][j], a[i].z, a[i].w, b[j].z, b[j].w);
                    }
            }
        }
    }
    cp_async_wait<0>();
    if (active) {
        float4* out = reinterpret_cast<float4*>(partials + ((long long)blockIdx.x * ntiles + t) * 32);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            out[i] = make_float4(ae[i][0] + ao[i][0], ae[i][1] + ao[i][1], ae[i][2] + ao[i][2],
                                 ae[i][3] + ao[i][3]);
    }
}

// Block partials -> R in double. Each thread sums one element over a segment
// of kReduceSeg blocks (independent loads, double accumulation) and adds the
// segment total to R with a double atomic; R is cleared beforehand.
constexpr int kReduceSeg = 16;

__global__ void gram_reduce_kernel(const float* __restrict__ partials, int nblocks,
                                   int p, int PT, int ntiles, int mode, double* __restrict__ R,
                                   int* status) {
    pdl_wait();
    pdl_trigger();
    const int te = mode == 0 ? 64 : 32;   // elements per tile
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)ntiles * te) return;
    const int b0 = blockIdx.y * kReduceSeg;
    const int b1 = min(b0 + kReduceSeg, nblocks);
    if (b0 >= b1) return;
    const long long stride = (long long)ntiles * te;
    double s = 0.0;
#pragma unroll 4
    for (int b = b0; b < b1; ++b) s += (double)__ldg(partials + (long long)b * stride + idx);
    const int t = (int)(idx / te), e = (int)(idx % te);
    int ti, tj, i, j;
    if (mode == 0) {
        tile_of(t, PT, ti, tj);
        i = 8 * ti + e / 8;
        j = 8 * tj + e % 8;
    } else {
        tile84_of(t, PT, ti, tj);
        i = 8 * ti + e / 4;
        j = 4 * tj + e % 4;
    }
    // tiles on the diagonal hold both (i, j) and (j, i): take i <= j only
    if (i < p && j < p && i <= j) {
        if (!isfinite(s)) set_status(status, HYDE_ERR_NUMERIC);
        atomicAdd(&R[(long long)i * p + j], s);
        if (i != j) atomicAdd(&R[(long long)j * p + i], s);
    }
}

}  // namespace

template <int MAXT>
static hyde_status plan_for(GramPlan& g, long long n) {
    cudaError_t e = ensure_smem_limit((const void*)gram_partial_kernel<MAXT>, (int)g.smem);
    if (e != cudaSuccess) return HYDE_ERR_CUDA;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gram_partial_kernel<MAXT>,
                                                      g.threads, g.smem);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    int sms = device_sm_count();
    if (sms <= 0) return HYDE_ERR_CUDA;
    long long nchunks = (n + KC - 1) / KC;
    long long blocks = (long long)sms * per_sm;
    if (blocks > nchunks) blocks = nchunks;
    g.blocks = (int)blocks;
    return HYDE_OK;
}

template <int MAXT>
static hyde_status plan_for84(GramPlan& g, long long n) {
    cudaError_t e = ensure_smem_limit((const void*)gram_partial84_kernel<MAXT>, (int)g.smem);
    if (e != cudaSuccess) return HYDE_ERR_CUDA;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gram_partial84_kernel<MAXT>,
                                                      g.threads, g.smem);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    int sms = device_sm_count();
    if (sms <= 0) return HYDE_ERR_CUDA;
    long long nchunks = (n + KC84 - 1) / KC84;
    long long blocks = (long long)sms * per_sm;
    if (blocks > nchunks) blocks = nchunks;
    g.blocks = (int)blocks;
    return HYDE_OK;
}

hyde_status gram_plan(int p, long long n, GramPlan* plan) {
    if (p < 1 || p > kMaxBandsGram || n < 1) return HYDE_ERR_SHAPE;
    GramPlan g;
    g.PT = (p + 7) / 8;
    g.smem = (size_t)STAGES * g.PT * 8 * KC * sizeof(float);
    hyde_status st;
    if (g.PT * (g.PT + 1) <= 384) {
        // 8 x 4 tiles with paired FMAs, one block of up to 384 threads per SM
        g.mode = 1;
        g.smem = (size_t)STAGES * g.PT * 8 * KC84 * sizeof(float);
        g.ntiles = g.PT * (g.PT + 1);
        g.threads = (g.ntiles + 31) / 32 * 32;
        st = plan_for84<384>(g, n);
    } else {
        g.mode = 0;
        g.ntiles = g.PT * (g.PT + 1) / 2;
        g.threads = (g.ntiles + 31) / 32 * 32;
        if (g.threads > kGramMaxThreads) return HYDE_ERR_SHAPE;
        st = g.threads <= 256   ? plan_for<256>(g, n)
             : g.threads <= 384 ? plan_for<384>(g, n)
                                : plan_for<kGramMaxThreads>(g, n);
    }
    if (st != HYDE_OK) return st;
    g.partial_bytes = (size_t)g.blocks * g.ntiles * (g.mode == 0 ? 64 : 32) * sizeof(float);
    *plan = g;
    return HYDE_OK;
}

hyde_status launch_gram(const float* Y, int p, long long n, const GramPlan& g,
                        float* partials, double* R, int* status, cudaStream_t s) {
    long long nchunks = (n + KC - 1) / KC;
    long long per = (nchunks + g.blocks - 1) / g.blocks;
    if (g.mode == 1)
        launch_pdl(gram_partial84_kernel<384>, g.blocks, g.threads, g.smem, s, Y, p, n, g.PT,
                   g.ntiles, partials);
    else if (g.threads <= 256)
        launch_pdl(gram_partial_kernel<256>, g.blocks, g.threads, g.smem, s, Y, p, n, g.PT,
                   g.ntiles, per, partials);
    else if (g.threads <= 384)
        launch_pdl(gram_partial_kernel<384>, g.blocks, g.threads, g.smem, s, Y, p, n, g.PT,
                   g.ntiles, per, partials);
    else
        launch_pdl(gram_partial_kernel<kGramMaxThreads>, g.blocks, g.threads, g.smem, s, Y, p, n,
                   g.PT, g.ntiles, per, partials);
    long long tot = (long long)g.ntiles * (g.mode == 0 ? 64 : 32);
    if (cudaMemsetAsync(R, 0, (size_t)p * p * sizeof(double), s) != cudaSuccess)
        return HYDE_ERR_CUDA;
    dim3 rgrid((unsigned)((tot + 255) / 256), (g.blocks + kReduceSeg - 1) / kReduceSeg);
    launch_pdl(gram_reduce_kernel, rgrid, 256, 0, s, partials, g.blocks, p, g.PT, g.ntiles,
               g.mode, R, status);
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

// --------------------------------------------------------------------------
// Allocation-free variant of hyde_gram.
//
// The float partial sums of the Gram kernel live in a fixed array in device
// global memory, reserved when the module is loaded onto a GPU and held by
// every GPU that loads the library until the process exits. Host code cannot
// use the array's name as a device pointer (it names a host-side shadow), so
// its device address is looked up with the caller's device current. The
// lookup is repeated on every call (it allocates nothing and is cheap once
// the module is loaded): a cached address would go stale when the caller
// resets the device and the module is loaded again elsewhere.
// --------------------------------------------------------------------------
namespace hyde {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;   // 16 MiB

static __device__ __align__(256) unsigned char g_gram_scratch[kNoAllocScratchBytes];

hyde_status gram_scratch_for_current_device(float** out) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_gram_scratch) != cudaSuccess || !addr)
        return HYDE_ERR_CUDA;
    *out = reinterpret_cast<float*>(addr);
    return HYDE_OK;
}

}  // namespace
}  // namespace hyde

extern "C" size_t hyde_gram_noalloc_scratch_bytes(void) { return hyde::kNoAllocScratchBytes; }

extern "C" hyde_status hyde_gram_noalloc(const float* Y, int p, long long n, double* R,
                                         cudaStream_t stream) {
    using namespace hyde;
    if (!Y || !R) return HYDE_ERR_INVALID_ARG;
    GramPlan g;
    hyde_status st = gram_plan(p, n, &g);
    if (st != HYDE_OK) return st;
    // each block writes one partial per tile element; use as many blocks as
    // the fixed scratch holds (never more than the occupancy-sized grid)
    const size_t per_block = (size_t)g.ntiles * (g.mode == 0 ? 64 : 32) * sizeof(float);
    const size_t max_blocks = kNoAllocScratchBytes / per_block;
    if (max_blocks < 1) return HYDE_ERR_SHAPE;
    if ((size_t)g.blocks > max_blocks) g.blocks = (int)max_blocks;
    g.partial_bytes = (size_t)g.blocks * per_block;
    float* scratch = nullptr;
    st = gram_scratch_for_current_device(&scratch);
    if (st != HYDE_OK) return st;
    // every block overwrites its whole partial slot, so nothing needs clearing
    return launch_gram(Y, p, n, g, scratch, R, nullptr, stream);
}


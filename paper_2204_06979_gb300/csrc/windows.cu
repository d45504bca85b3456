// Batched (sliding-window) HyRes: a scene too large or too varied for one
// global model is cut into windows, each denoised on its own (own noise
// levels, subspace, rank and threshold) and reassembled; the paper slices
// large images into tiles and denoises each tile (arXiv 2204.06979,
// Sec. 2.2.2). Each window's output is taken only over its core, so every
// scene pixel has exactly one source.
//
// Windows are spread round-robin over a pool of slots; a slot owns a stream
// (the caller's), a workspace slice and two contiguous window cubes. On its
// stream a window is gathered into the slot's input cube, denoised by the
// single-cube pipeline, and its core scattered into the scene. Slots run
// concurrently; the whole call can be captured into one CUDA graph.
#include "hyde_internal.cuh"

namespace hyde {
namespace {

// scene [p][H][W] -> cube [p][h][w] of the window at (y0, x0)
__global__ void gather_window_kernel(const float* __restrict__ Y, int H, int W, int y0, int x0,
                                     int h, int w, int p, float* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    const long long n = (long long)h * w, tot = n * p;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / n);
        const long long r = e - (long long)b * n;
        const int yy = (int)(r / w), xx = (int)(r - (long long)yy * w);
        out[e] = __ldg(Y + ((long long)b * H + (y0 + yy)) * W + (x0 + xx));
    }
}

// core (cy0, cx0, ch, cw) of the window cube -> scene
__global__ void scatter_core_kernel(const float* __restrict__ cube, int h, int w, int y0, int x0,
                                    int cy0, int cx0, int ch, int cw, int p, int H, int W,
                                    float* __restrict__ X) {
    pdl_wait();
    pdl_trigger();
    const long long n = (long long)ch * cw, tot = n * p;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / n);
        const long long r = e - (long long)b * n;
        const int yy = (int)(r / cw), xx = (int)(r - (long long)yy * cw);
        const int sy = cy0 + yy, sx = cx0 + xx;
        X[((long long)b * H + sy) * W + sx] =
            cube[((long long)b * h + (sy - y0)) * w + (sx - x0)];
    }
}

}  // namespace

hyde_status launch_gather_window(const float* Y, int H, int W, int y0, int x0, int h, int w,
                                 int p, float* out, cudaStream_t s) {
    const long long tot = (long long)h * w * p;
    const int sms = device_sm_count();
    long long blocks = (tot + 255) / 256;
    if (blocks > 8LL * sms) blocks = 8LL * sms;
    launch_pdl(gather_window_kernel, (unsigned)blocks, 256, 0, s, Y, H, W, y0, x0, h, w, p, out);
    return cuda_status(cudaGetLastError());
}

hyde_status launch_scatter_core(const float* cube, int h, int w, int y0, int x0, int cy0,
                                int cx0, int ch, int cw, int p, int H, int W, float* X,
                                cudaStream_t s) {
    const long long tot = (long long)ch * cw * p;
    const int sms = device_sm_count();
    long long blocks = (tot + 255) / 256;
    if (blocks > 8LL * sms) blocks = 8LL * sms;
    launch_pdl(scatter_core_kernel, (unsigned)blocks, 256, 0, s, cube, h, w, y0, x0, cy0, cx0, ch,
               cw, p, H, W, X);
    return cuda_status(cudaGetLastError());
}

}  // namespace hyde

// kern_image.cu -- cross-pixel warm start of image scans.  A row-major
// width x height image is inverted in two passes: the coarse pixels (every
// `stride`-th column of every `stride`-th row) with the full search, then
// every other pixel with a prior built from its coarse neighbours: a box in
// the normalised cube spanning their winners (widened by a margin) and the
// winners themselves as seed particles.  This follows the paper's
// observation that tighter search bounds cut the number of swarm
// generations (Sec. 4.1) and its aim of real-time imaging (Sec. 1, 5).
#include "afm_device.cuh"
#include "afm_launch.h"

namespace afm {

namespace {

__host__ __device__ __forceinline__ int ceil_div(int a, int b) { return (a + b - 1) / b; }

}  // namespace

void image_counts(int width, int height, int stride, int* n_coarse, int* n_fine) {
    const int nc = ceil_div(width, stride) * ceil_div(height, stride);
    *n_coarse = nc;
    *n_fine = width * height - nc;
}

// One thread per pixel: its index in the coarse or the fine list, by
// counting (rows in order, columns in order within a row).
__global__ void image_plan_kernel(int width, int height, int stride, int* __restrict__ coarse,
                                  int* __restrict__ fine) {
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= width * height) return;
    const int i = pix % width, j = pix / width;
    const int ncx = ceil_div(width, stride);
    const bool crow = j % stride == 0;
    if (crow && i % stride == 0) {
        coarse[(j / stride) * ncx + i / stride] = pix;
        return;
    }
    // coarse pixels before this one: full coarse rows above, then coarse
    // columns to the left in this row
    const int rows_above = ceil_div(j, stride);
    const int left = crow ? ceil_div(i, stride) : 0;
    fine[pix - rows_above * ncx - left] = pix;
}

// One thread per fine pixel: the box and seeds from the coarse neighbours'
// winners (the result records of the coarse pass).
__global__ void image_prior_kernel(int width, int height, int stride, int D, float margin,
                                   const afm_result* __restrict__ res, const int* __restrict__ fine,
                                   int n_fine, float* __restrict__ box_lo,
                                   float* __restrict__ box_hi, float* __restrict__ seeds) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_fine) return;
    const int pix = fine[f];
    const int i = pix % width, j = pix / width;
    const int ncx = ceil_div(width, stride), ncy = ceil_div(height, stride);
    const int cx0 = i / stride, cy0 = j / stride;
    const int cx1 = min(cx0 + 1, ncx - 1), cy1 = min(cy0 + 1, ncy - 1);
    const int nb[4] = {(cy0 * stride) * width + cx0 * stride, (cy0 * stride) * width + cx1 * stride,
                       (cy1 * stride) * width + cx0 * stride, (cy1 * stride) * width + cx1 * stride};
    for (int d = 0; d < D; ++d) {
        float lo = 1.f, hi = 0.f;
        for (int k = 0; k < 4; ++k) {
            const float x = (float)res[nb[k]].x[d];
            seeds[((size_t)f * 4 + k) * D + d] = x;
            lo = fminf(lo, x);
            hi = fmaxf(hi, x);
        }
        lo = fmaxf(lo - margin, 0.f);
        hi = fminf(hi + margin, 1.f);
        box_lo[(size_t)f * D + d] = lo;
        box_hi[(size_t)f * D + d] = hi;
    }
}

cudaError_t launch_image_plan(int width, int height, int stride, int* coarse, int* fine,
                              cudaStream_t st) {
    const int n = width * height, threads = 256;
    image_plan_kernel<<<(n + threads - 1) / threads, threads, 0, st>>>(width, height, stride, coarse,
                                                                       fine);
    return cudaGetLastError();
}

cudaError_t launch_image_prior(int width, int height, int stride, int D, float margin,
                               const afm_result* res, const int* fine, int n_fine, float* box_lo,
                               float* box_hi, float* seeds, cudaStream_t st) {
    const int threads = 128;
    image_prior_kernel<<<(n_fine + threads - 1) / threads, threads, 0, st>>>(
        width, height, stride, D, margin, res, fine, n_fine, box_lo, box_hi, seeds);
    return cudaGetLastError();
}

}  // namespace afm

// ihist_window.cuh -- sliding-window histogram search over a resident
// integral histogram, the use arXiv 1711.01919 builds the integral for
// (Sec. 1: detection and tracking compare the histogram of every candidate
// window with a target histogram).
//
// Window (i, j) covers rows i*stride .. i*stride+win_h-1 and columns
// j*stride .. j*stride+win_w-1; its histogram comes from Eq. 2 (four
// lookups per bin, whatever the window's area) and its score is the
// histogram intersection sum_b min(h_b, target_b) (Swain and Ballard),
// an exact integer no larger than the window's area.
#pragma once

#include "ihist_device.cuh"

namespace ihist {

// Best window so far as one 64-bit word: score in the high half, and the
// complement of the window index in the low half, so that atomicMax keeps
// the highest score and, among equal scores, the lowest index.
__device__ __forceinline__ unsigned long long pack_best(uint32_t score, long long wi) {
  return ((unsigned long long)score << 32) | (unsigned long long)(0xffffffffu - (uint32_t)wi);
}

// Reduce a warp's (score, index) pairs and fold the winner into *best.
__device__ __forceinline__ void fold_best(unsigned long long *best, unsigned long long v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(kFull, v, d);
    v = o > v ? o : v;
  }
  if ((threadIdx.x & 31) == 0 && v != 0ull) atomicMax(best, v);
}

__device__ __forceinline__ uint32_t window_count(const uint32_t *__restrict__ hist, size_t at_y1x1,
                                                 size_t at_y0x1, size_t at_y1x0, size_t at_y0x0, bool top,
                                                 bool left) {
  uint32_t v = __ldg(hist + at_y1x1);
  if (top) v -= __ldg(hist + at_y0x1);
  if (left) v -= __ldg(hist + at_y1x0);
  if (top && left) v += __ldg(hist + at_y0x0);
  return v;
}

// Bin-major H[b][y][x]: one thread per window, bins in a loop.  Neighbouring
// lanes hold neighbouring windows of a grid row, so each corner load of a
// warp touches stride*4-byte spaced words of one row of one plane.
template <bool BEST>
__global__ void __launch_bounds__(256) window_kernel_bin_major(
    const uint32_t *__restrict__ hist, int H, int W, int B, const uint32_t *__restrict__ target, int win_h,
    int win_w, int stride, int ny, int nx, uint32_t *__restrict__ scores, unsigned long long *best) {
  extern __shared__ uint32_t s_target[];
  for (int b = threadIdx.x; b < B; b += blockDim.x) s_target[b] = target[b];
  __syncthreads();
  const size_t plane = (size_t)H * (size_t)W;
  const long long total = (long long)ny * nx;
  unsigned long long mine = 0ull;  // this thread's best (score, index), 0 = none
  for (long long wi = (long long)blockIdx.x * blockDim.x + threadIdx.x; wi < total;
       wi += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(wi / nx), j = (int)(wi - (long long)i * nx);
    const int y0 = i * stride, x0 = j * stride, y1 = y0 + win_h - 1, x1 = x0 + win_w - 1;
    const bool top = y0 > 0, left = x0 > 0;
    // offsets inside one plane; corners at index -1 are never read
    const size_t o11 = (size_t)y1 * W + x1;
    const size_t o01 = top ? (size_t)(y0 - 1) * W + x1 : 0;
    const size_t o10 = left ? (size_t)y1 * W + (x0 - 1) : 0;
    const size_t o00 = (top && left) ? (size_t)(y0 - 1) * W + (x0 - 1) : 0;
    uint32_t score = 0u;
    // the unroll depth that keeps enough corner loads in flight differs
    // between the two variants (measured: 40 us for both on 1080p x 64)
    if constexpr (BEST) {
#pragma unroll 16
      for (int b = 0; b < B; ++b) {
        const size_t p = (size_t)b * plane;
        score += min(window_count(hist, p + o11, p + o01, p + o10, p + o00, top, left), s_target[b]);
      }
    } else {
      for (int b = 0; b < B; ++b) {
        const size_t p = (size_t)b * plane;
        score += min(window_count(hist, p + o11, p + o01, p + o10, p + o00, top, left), s_target[b]);
      }
    }
    if (!BEST || scores) scores[wi] = score;
    if (BEST) {
      const unsigned long long v = pack_best(score, wi);
      mine = v > mine ? v : mine;
    }
  }
  if (BEST) fold_best(best, mine);
}

// Pixel-major H[y][x][b]: one warp per window, lanes over bins, so each
// corner is one contiguous B-word vector; a warp reduction sums the bins.
template <bool BEST>
__global__ void __launch_bounds__(256) window_kernel_pixel_major(
    const uint32_t *__restrict__ hist, int H, int W, int B, const uint32_t *__restrict__ target, int win_h,
    int win_w, int stride, int ny, int nx, uint32_t *__restrict__ scores, unsigned long long *best) {
  extern __shared__ uint32_t s_target[];
  for (int b = threadIdx.x; b < B; b += blockDim.x) s_target[b] = target[b];
  __syncthreads();
  const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  const long long total = (long long)ny * nx;
  unsigned long long mine = 0ull;  // lane 0: this warp's best (score, index)
  for (long long wi = (long long)blockIdx.x * warps + (threadIdx.x >> 5); wi < total;
       wi += (long long)gridDim.x * warps) {
    const int i = (int)(wi / nx), j = (int)(wi - (long long)i * nx);
    const int y0 = i * stride, x0 = j * stride, y1 = y0 + win_h - 1, x1 = x0 + win_w - 1;
    const bool top = y0 > 0, left = x0 > 0;
    const size_t o11 = ((size_t)y1 * W + x1) * B;
    const size_t o01 = top ? ((size_t)(y0 - 1) * W + x1) * B : 0;
    const size_t o10 = left ? ((size_t)y1 * W + (x0 - 1)) * B : 0;
    const size_t o00 = (top && left) ? ((size_t)(y0 - 1) * W + (x0 - 1)) * B : 0;
    uint32_t score = 0u;
    for (int b = lane; b < B; b += 32)
      score += min(window_count(hist, o11 + b, o01 + b, o10 + b, o00 + b, top, left), s_target[b]);
    score = __reduce_add_sync(kFull, score);
    if (lane == 0 && (!BEST || scores)) scores[wi] = score;
    if (BEST) {
      const unsigned long long v = pack_best(score, wi);
      mine = v > mine ? v : mine;
    }
  }
  if (BEST && lane == 0 && mine != 0ull) atomicMax(best, mine);
}

}  // namespace ihist

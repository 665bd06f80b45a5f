// ihist_query.cuh -- region histograms by Eq. 2 of arXiv 1711.01919:
//   h(R, b) = H[y1][x1] - H[y0-1][x1] - H[y1][x0-1] + H[y0-1][x0-1]
// for inclusive rectangles, terms at index -1 being zero.  Four lookups per
// (rectangle, bin), independent of the rectangle's area (the O(1) query of
// Sec. 1).  Evaluated in uint32 modular arithmetic: the true count lies in
// [0, area], so wrap-around in the intermediate sums cancels exactly.
#pragma once

#include "ihist_device.cuh"

namespace ihist {

// One thread per (rectangle, bin) pair p = r * B + b, grid-stride.  Output
// row r of [n][B] is written by B consecutive threads (coalesced).  The
// rectangle's four ints are re-read by its B threads and served by L1.  In
// the quad-major layout the four threads of a quad read one 16-byte word per
// corner (one DRAM sector for four bins).
template <int LAYOUT>
__global__ void __launch_bounds__(256) query_kernel(const uint32_t *__restrict__ hist, int H,
                                                     int W, int B,
                                                     const int32_t *__restrict__ rects,
                                                     unsigned int total,
                                                     uint32_t *__restrict__ out, Ctrl *ctrl) {
  // Launched with programmatic stream serialization: the histogram is read
  // only once the grid before (normally the scan that wrote it) completed.
  // The grids that let this one start early are the library's own, which
  // never write rectangles, so each thread's first rectangle is read before
  // that wait.
  const size_t plane = (size_t)H * (size_t)W;
  const unsigned int stride = gridDim.x * blockDim.x;
  unsigned int p = blockIdx.x * blockDim.x + threadIdx.x;
  int x0 = 0, y0 = 0, x1 = -1, y1 = -1;
  auto load_rect = [&](unsigned int pp) {
    const size_t r4 = 4 * (size_t)(pp / (unsigned)B);
    x0 = __ldg(rects + r4 + 0);
    y0 = __ldg(rects + r4 + 1);
    x1 = __ldg(rects + r4 + 2);
    y1 = __ldg(rects + r4 + 3);
  };
  if (p < total) load_rect(p);
  griddep_wait_and_release();
  for (; p < total; p += stride) {
    if (p != blockIdx.x * blockDim.x + threadIdx.x) load_rect(p);
    const unsigned int r = p / (unsigned)B;
    const int b = (int)(p - r * (unsigned)B);
    const bool ok = (0 <= x0) & (x0 <= x1) & (x1 < W) & (0 <= y0) & (y0 <= y1) & (y1 < H);
    uint32_t v = 0u;
    if (ok) {
      // element offset of H at (row y, column x) for this bin
      auto at = [&](int y, int x) -> size_t {
        return LAYOUT == 0   ? (size_t)b * plane + (size_t)y * W + x
               : LAYOUT == 1 ? ((size_t)y * W + x) * (size_t)B + b
                             : ((size_t)(b >> 2) * plane + (size_t)y * W + x) * 4 + (b & 3);
      };
      v = __ldg(hist + at(y1, x1));
      if (y0 > 0) v -= __ldg(hist + at(y0 - 1, x1));
      if (x0 > 0) v -= __ldg(hist + at(y1, x0 - 1));
      if (x0 > 0 && y0 > 0) v += __ldg(hist + at(y0 - 1, x0 - 1));
    } else if (b == 0) {
      latch_status(ctrl, kStatusBadRect);
    }
    out[p] = v;
  }
}

// Queries over every frame of a batch in one launch: frame f has n
// rectangles at rects + 4*n*f and its rows at out + n * bins_end[f-1].
// Thread p covers (frame, rect, bin); the frame is found by binary search
// over bins_end (prefix sums of the frames' bin counts, times n).  The
// per-frame descriptors are read with coherent loads, once per use.
template <typename Desc>
__global__ void __launch_bounds__(256) query_batch_kernel(const Desc *frames,
                                                           const unsigned int *bins_end,
                                                           int nframes, const int32_t *__restrict__ rects,
                                                           unsigned int n, unsigned long long total,
                                                           uint32_t *__restrict__ out, Ctrl *ctrl) {
  for (unsigned long long p = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; p < total;
       p += (unsigned long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = nframes - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((unsigned long long)ld_relaxed_u32(bins_end + mid) * n > p) hi = mid; else lo = mid + 1;
    }
    const int fi = lo;
    const unsigned long long base = fi > 0 ? (unsigned long long)ld_relaxed_u32(bins_end + fi - 1) * n : 0ull;
    const Desc *f = frames + fi;
    const int B = (int)ld_relaxed_u32(&f->B), H = (int)ld_relaxed_u32(&f->H);
    const int W = (int)ld_relaxed_u32(&f->W), layout = (int)ld_relaxed_u32(&f->layout);
    const uint32_t *hist = reinterpret_cast<const uint32_t *>(ld_relaxed_u64(&f->out));
    if (B <= 0 || p < base) {  // a descriptor that cannot be right: never dereference it
      latch_status(ctrl, kStatusBadRect);
      continue;
    }
    const unsigned long long local = p - base;
    const unsigned int r = (unsigned int)(local / (unsigned)B);
    const int b = (int)(local - (unsigned long long)r * (unsigned)B);
    if (r >= n) {
      latch_status(ctrl, kStatusBadRect);
      continue;
    }
    const int32_t *rc = rects + 4 * ((size_t)fi * n + r);
    const int x0 = __ldg(rc + 0), y0 = __ldg(rc + 1), x1 = __ldg(rc + 2), y1 = __ldg(rc + 3);
    const bool ok = (0 <= x0) & (x0 <= x1) & (x1 < W) & (0 <= y0) & (y0 <= y1) & (y1 < H);
    uint32_t v = 0u;
    if (ok) {
      const size_t plane = (size_t)H * (size_t)W;
      auto at = [&](int y, int x) -> size_t {
        return layout == 0   ? (size_t)b * plane + (size_t)y * W + x
               : layout == 1 ? ((size_t)y * W + x) * (size_t)B + b
                             : ((size_t)(b >> 2) * plane + (size_t)y * W + x) * 4 + (b & 3);
      };
      v = __ldg(hist + at(y1, x1));
      if (y0 > 0) v -= __ldg(hist + at(y0 - 1, x1));
      if (x0 > 0) v -= __ldg(hist + at(y1, x0 - 1));
      if (x0 > 0 && y0 > 0) v += __ldg(hist + at(y0 - 1, x0 - 1));
    } else if (b == 0) {
      latch_status(ctrl, kStatusBadRect);
    }
    out[p] = v;
  }
}

}  // namespace ihist

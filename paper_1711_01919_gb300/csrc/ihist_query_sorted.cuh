// ihist_query_sorted.cuh -- Eq. 2 region histograms for large rectangle
// batches on a bin-major H, with the corner lookups put in row order first.
//
// Eq. 2 reads four words of H per (rectangle, bin).  In the bin-major layout
// a bin plane is h x w words, so the lookups of random rectangles land on
// random DRAM lines: each 4-byte corner costs a whole line fetch (one
// thread per (rectangle, bin) runs at the random-gather rate of the GPU).
// Here the corners of all rectangles are first bucketed by their row (a
// counting sort), then read bucket after bucket: the corners of one row of
// one plane are read at about the same time, so every line of H they touch
// comes from DRAM once and serves all of them from L2.  The rectangles
// share their corners' row order across bins, so the sort is paid once per
// batch:
//
//   1. corner_count     per valid rectangle, its (up to) four corners (the
//                       index -1 terms of Eq. 2 are skipped): cnt[y] += 1
//   2. row_offsets      exclusive scan of cnt over the h rows (one CTA)
//   3. corner_scatter   corner -> position off[y] + (a decrement of cnt[y],
//                       which leaves cnt at zero for the next batch):
//                       pts[pos] = (y, x), slot[r][corner] = pos
//   4. corner_gather    per group of nb bins: val[pos][j] = H[b0 + j][y][x]
//   5. corner_combine   out[r][b0 + j] = val[s0][j] - val[s1][j] - val[s2][j]
//                       + val[s3][j] (absent corners read as 0), uint32
//                       modular arithmetic as in Eq. 2
//
// Corners within a row bucket come in atomic order, which changes the
// positions but not the result: each output word is the same four terms.
#pragma once

#include "ihist_device.cuh"

namespace ihist {

// Rectangle r's four corner slots: 0 = (y1, x1) +, 1 = (y0-1, x1) -,
// 2 = (y1, x0-1) -, 3 = (y0-1, x0-1) +.  Slot s is present when its row and
// column indices are >= 0; a rectangle out of range has none.
__device__ __forceinline__ bool rect_ok(const int32_t *rects, unsigned int r, int H, int W, int &x0, int &y0,
                                        int &x1, int &y1) {
  const int32_t *p = rects + 4 * (size_t)r;  // 4-byte aligned rows: four scalar loads
  x0 = __ldg(p);
  y0 = __ldg(p + 1);
  x1 = __ldg(p + 2);
  y1 = __ldg(p + 3);
  return (0 <= x0) & (x0 <= x1) & (x1 < W) & (0 <= y0) & (y0 <= y1) & (y1 < H);
}

__device__ __forceinline__ bool corner_of(int s, int x0, int y0, int x1, int y1, int &y, int &x) {
  y = (s & 1) ? y0 - 1 : y1;
  x = (s & 2) ? x0 - 1 : x1;
  return y >= 0 && x >= 0;
}

// 1. row counts of the present corners (bad rectangles latch the status)
__global__ void __launch_bounds__(256) corner_count_kernel(const int32_t *__restrict__ rects, unsigned int n, int H,
                                                           int W, unsigned int *cnt, Ctrl *ctrl) {
  for (unsigned int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    int x0, y0, x1, y1;
    if (!rect_ok(rects, r, H, W, x0, y0, x1, y1)) {
      latch_status(ctrl, kStatusBadRect);
      continue;
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      int y, x;
      if (corner_of(s, x0, y0, x1, y1, y, x)) atomicAdd(cnt + y, 1u);
    }
  }
}

// 2. off[y] = sum of cnt[0..y), off[H] = the number of corners; one CTA of
// 1024 threads, each scanning a contiguous run of rows.
__global__ void __launch_bounds__(1024) row_offsets_kernel(const unsigned int *__restrict__ cnt, int H,
                                                           unsigned int *off) {
  __shared__ unsigned int s_part[1024];
  const int t = threadIdx.x;
  const int per = (H + 1023) / 1024;
  const int y0 = min(H, t * per), y1 = min(H, y0 + per);
  unsigned int sum = 0u;
  for (int y = y0; y < y1; ++y) sum += cnt[y];
  s_part[t] = sum;
  __syncthreads();
  // inclusive scan of the 1024 partial sums (Hillis-Steele in shared memory)
  for (int d = 1; d < 1024; d <<= 1) {
    const unsigned int v = t >= d ? s_part[t - d] : 0u;
    __syncthreads();
    s_part[t] += v;
    __syncthreads();
  }
  unsigned int run = s_part[t] - sum;
  for (int y = y0; y < y1; ++y) {
    off[y] = run;
    run += cnt[y];
  }
  if (t == 1023) off[H] = s_part[1023];
}

// 3. each present corner takes the next free position of its row bucket;
// absent corners (and all corners of a bad rectangle) get slot 0xffffffff.
__global__ void __launch_bounds__(256) corner_scatter_kernel(const int32_t *__restrict__ rects, unsigned int n, int H,
                                                             int W, unsigned int *cnt,
                                                             const unsigned int *__restrict__ off,
                                                             uint32_t *__restrict__ pts, uint4 *__restrict__ slot) {
  for (unsigned int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    int x0, y0, x1, y1;
    uint32_t sl[4] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu};
    if (rect_ok(rects, r, H, W, x0, y0, x1, y1)) {
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        int y, x;
        if (corner_of(s, x0, y0, x1, y1, y, x)) {
          const unsigned int pos = off[y] + atomicSub(cnt + y, 1u) - 1u;
          pts[pos] = ((uint32_t)y << 16) | (uint32_t)x;
          sl[s] = pos;
        }
      }
    }
    slot[r] = make_uint4(sl[0], sl[1], sl[2], sl[3]);
  }
}

// 4. one thread per corner position (row order): the nb words of bins
// b0 .. b0+nb-1 at that pixel, val[pos][0..nb).  NB is the compile-time
// group width (the last group may hold fewer bins, nb <= NB).
template <int NB>
__global__ void __launch_bounds__(256) corner_gather_kernel(const uint32_t *__restrict__ hist, int H, int W, int b0,
                                                            int nb, const uint32_t *__restrict__ pts,
                                                            const unsigned int *__restrict__ off,
                                                            uint32_t *__restrict__ val) {
  const unsigned int total = off[H];
  const size_t plane = (size_t)H * (size_t)W;
  for (unsigned int pos = blockIdx.x * blockDim.x + threadIdx.x; pos < total; pos += gridDim.x * blockDim.x) {
    const uint32_t pt = pts[pos];
    const uint32_t *src = hist + (size_t)b0 * plane + (size_t)(pt >> 16) * W + (pt & 0xffffu);
    uint32_t v[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) v[j] = j < nb ? __ldg(src + (size_t)j * plane) : 0u;
    uint32_t *dst = val + (size_t)pos * NB;
#pragma unroll
    for (int j = 0; j < NB; j += 4) *reinterpret_cast<uint4 *>(dst + j) = make_uint4(v[j], v[j + 1], v[j + 2], v[j + 3]);
  }
}

// 5. out[r][b0 + j] by Eq. 2 from the gathered corners: NB consecutive
// threads per rectangle (one per bin of the group), so the four val rows
// and the output piece are each read or written as whole sectors.
template <int NB>
__global__ void __launch_bounds__(256) corner_combine_kernel(const uint4 *__restrict__ slot, unsigned int n, int B,
                                                             int b0, int nb, const uint32_t *__restrict__ val,
                                                             uint32_t *__restrict__ out) {
  const unsigned long long total = (unsigned long long)n * NB;
  for (unsigned long long p = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; p < total;
       p += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned int r = (unsigned int)(p / NB);
    const int j = (int)(p % NB);
    if (j >= nb) continue;
    const uint4 s = __ldg(slot + r);
    uint32_t v = 0u;
    if (s.x != 0xffffffffu) v = __ldg(val + (size_t)s.x * NB + j);  // a rectangle with no (y1, x1) is out of range
    if (s.y != 0xffffffffu) v -= __ldg(val + (size_t)s.y * NB + j);
    if (s.z != 0xffffffffu) v -= __ldg(val + (size_t)s.z * NB + j);
    if (s.w != 0xffffffffu) v += __ldg(val + (size_t)s.w * NB + j);
    out[(size_t)r * B + b0 + j] = v;
  }
}

}  // namespace ihist

// ihist_scan.cuh -- the fused integral-histogram kernel.
//
// Computes, for one frame, H[b][y][x] = #{x' <= x, y' <= y : Q(I[y'][x']) = b}
// (Eq. 1 of arXiv 1711.01919), the result Algorithm 1 builds with its
// recurrence, in one pass over the frame:
//
//   * a1 quantise: q = floor(v * B / 256) in registers; the paper's one-hot
//     initialisation tensor (Alg. 2-4, step 1) is never materialised.
//   * a2 row scan: per bin and row, a running count across the columns --
//     4 columns per lane, then a warp shuffle scan over 128 columns with four
//     bins packed in the bytes of one register, then a per-row carry from
//     the chunks to the left.
//   * a3 column scan: per-lane register accumulators walk down the rows.
//   * a4 carries between bands: decoupled look-back.  The paper's WF-TiS
//     (Sec. 3.5) launches one kernel per tile anti-diagonal (Eq. 6) and saves
//     each tile's last column in an extra array; here a CTA publishes its
//     band's column counts (an aggregate that depends on its own pixels
//     only) before it waits for anything, then looks back over the bands
//     above until it meets a published inclusive prefix row.
//   * a5 store: each output word is written once, 128-bit streaming stores.
//
// Work item = (band k of R rows, bin group g of G bins).  The CTA's warps
// split the frame width: warp w owns 128-column chunks [w*m, w*m + m).  The
// horizontal carry between warps comes from a counting pass (per-row bin
// totals of each warp's columns, reduced with one redux.sync per 4 bins)
// and an exclusive scan over warps in shared memory.  The vertical carry
// between bands is the look-back, per (band, group, chunk).
#pragma once

#include "ihist_device.cuh"

namespace ihist {

// One frame as the kernel sees it.  Offsets of the carry buffers are in
// units of "chunk items": ci = (item * nchunks + chunk), item = k*ngroups + g.
struct FrameDesc {
  const uint8_t *in;
  long long pitch;      // bytes between rows of in
  uint32_t *out;
  int H, W, B, layout;  // layout: 0 bin-major, 1 pixel-major
  int R, nbands, ngroups, nchunks, m;
  int fault_skip_band;  // -1 off
  unsigned int nitems;  // nbands * ngroups
  unsigned int pad0;
  uint32_t *agg_cnt;    // [ci][128 cols][G/4] words: packed column counts (bytes)
  uint32_t *agg_left;   // [ci][G]: band count left of the chunk
  uint32_t *incl;       // [ci][G][128]: H on the band's last row
  uint32_t *flags;      // [ci]
};

// Bit offset 8*q of the pixel's bin relative to the CTA's first bin
// (gbase = 8 * g * G); an invalid column gets an offset that no sub-group
// can match (shl_clamp gives 0).
__device__ __forceinline__ uint32_t bin_offset(uint32_t v, uint32_t nbins, uint32_t gbase) {
  return (((v * nbins) >> 8) << 3) - gbase;
}

constexpr uint32_t kNoBin = 0x80000000u;

// Four consecutive pixels of one row starting at column x (x % 4 == 0).
template <bool VEC>
__device__ __forceinline__ void load_offsets(const uint8_t *__restrict__ row, int x, int W,
                                             uint32_t nbins, uint32_t gbase, uint32_t u[4]) {
  if (VEC) {
    // VEC: row start 4-byte aligned and W % 4 == 0, so a lane is all-in or all-out.
    if (x < W) {
      const uint32_t px = __ldg(reinterpret_cast<const unsigned int *>(row + x));
#pragma unroll
      for (int i = 0; i < 4; ++i) u[i] = bin_offset(__byte_perm(px, 0u, 0x4440u + i), nbins, gbase);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) u[i] = kNoBin;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      u[i] = (x + i < W) ? bin_offset(__ldg(row + x + i), nbins, gbase) : kNoBin;
  }
}

// Exclusive/inclusive scan helpers on 4 columns x one 32-bit value per lane.
// Returns the inclusive prefix of v[0..3] over the 128-column chunk.
__device__ __forceinline__ void chunk_scan32(uint32_t v[4], int lane) {
  v[1] += v[0];
  v[2] += v[1];
  v[3] += v[2];
  const uint32_t t = warp_scan_incl(v[3], lane);
  const uint32_t ex = t - v[3];
  v[0] += ex;
  v[1] += ex;
  v[2] += ex;
  v[3] = t;
}

// ---------------------------------------------------------------------------
// One work item: band k, bin group g.  smem layout (32-bit words):
//   s_row [NW][R][G]   per-warp per-row bin totals, then row carries
//   s_ctot[nchunks][G] per-chunk band totals, then their exclusive prefix
template <int G, int MMAX, bool VEC>
__device__ __forceinline__ void process_item(const FrameDesc &f, unsigned int it, uint32_t epoch,
                                             Ctrl *ctrl, unsigned long long timeout_ns,
                                             uint32_t *s_row, uint32_t *s_ctot) {
  constexpr int GQ = G / 4;
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int NW = blockDim.x >> 5;
  const int k = (int)(it / (unsigned)f.ngroups);
  const int g = (int)(it % (unsigned)f.ngroups);
  const int y0 = k * f.R;
  const int nrows = min(f.R, f.H - y0);
  const uint32_t nbins = (uint32_t)f.B;
  const uint32_t gbase = 8u * (uint32_t)(g * G);
  const int c_begin = w * f.m;
  const int my_m = max(0, min(f.m, f.nchunks - c_begin));  // warp-uniform
  const bool publish = (k != f.fault_skip_band);
  const unsigned int ci0 = it * (unsigned)f.nchunks;        // chunk-item of chunk 0

  // ---- counting pass: column counts (bytes) and per-row segment totals ----
  uint32_t colcnt[MMAX][GQ][4];
#pragma unroll
  for (int cc = 0; cc < MMAX; ++cc)
#pragma unroll
    for (int q = 0; q < GQ; ++q)
#pragma unroll
      for (int i = 0; i < 4; ++i) colcnt[cc][q][i] = 0u;

  for (int yl = 0; yl < nrows; ++yl) {
    const uint8_t *row = f.in + (long long)(y0 + yl) * f.pitch;
    uint32_t rs[GQ];
#pragma unroll
    for (int q = 0; q < GQ; ++q) rs[q] = 0u;
#pragma unroll
    for (int cc = 0; cc < MMAX; ++cc) {
      if (cc < my_m) {
        uint32_t u[4];
        load_offsets<VEC>(row, (c_begin + cc) * kChunk + 4 * lane, f.W, nbins, gbase, u);
#pragma unroll
        for (int q = 0; q < GQ; ++q)
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint32_t ind = shl_clamp(1u, u[i] - 32u * q);
            colcnt[cc][q][i] += ind;
            rs[q] += ind;
          }
      }
    }
    uint32_t *dst = s_row + ((size_t)w * f.R + yl) * G;
    if (my_m > 0) {
#pragma unroll
      for (int q = 0; q < GQ; ++q) {
        uint32_t t0, t1, t2, t3;
        if (MMAX == 1) {
          // one chunk: each byte sums at most 4 x 32 = 128
          const uint32_t t = __reduce_add_sync(kFull, rs[q]);
          t0 = t & 0xffu; t1 = (t >> 8) & 0xffu; t2 = (t >> 16) & 0xffu; t3 = t >> 24;
        } else {
          const uint32_t lo = __reduce_add_sync(kFull, __byte_perm(rs[q], 0u, 0x4140u));
          const uint32_t hi = __reduce_add_sync(kFull, __byte_perm(rs[q], 0u, 0x4342u));
          t0 = lo & 0xffffu; t1 = lo >> 16; t2 = hi & 0xffffu; t3 = hi >> 16;
        }
        if (lane == 0) *reinterpret_cast<uint4 *>(dst + 4 * q) = make_uint4(t0, t1, t2, t3);
      }
    } else if (lane == 0) {
#pragma unroll
      for (int q = 0; q < GQ; ++q) *reinterpret_cast<uint4 *>(dst + 4 * q) = make_uint4(0, 0, 0, 0);
    }
  }

  // per-chunk band totals and the column-count aggregate of each chunk
#pragma unroll
  for (int cc = 0; cc < MMAX; ++cc) {
    if (cc < my_m) {
      const int c = c_begin + cc;
#pragma unroll
      for (int q = 0; q < GQ; ++q) {
        uint32_t lo = 0u, hi = 0u;  // 16-bit lanes, each at most 4R <= 1020
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          lo += __byte_perm(colcnt[cc][q][i], 0u, 0x4140u);
          hi += __byte_perm(colcnt[cc][q][i], 0u, 0x4342u);
        }
        lo = __reduce_add_sync(kFull, lo);  // at most 128R <= 32640 per lane
        hi = __reduce_add_sync(kFull, hi);
        if (lane == 0)
          *reinterpret_cast<uint4 *>(s_ctot + (size_t)c * G + 4 * q) =
              make_uint4(lo & 0xffffu, lo >> 16, hi & 0xffffu, hi >> 16);
      }
      // aggregate: this band's column counts, [128 cols][GQ] words
      uint32_t *dst = f.agg_cnt + ((size_t)(ci0 + c) * kChunk + 4 * lane) * GQ;
#pragma unroll
      for (int j = 0; j < GQ; ++j) {
        // words 4j..4j+3 of this lane's 4*GQ words: col (4j+t)/GQ, group (4j+t)%GQ
        uint32_t wv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) wv[t] = colcnt[cc][(4 * j + t) % GQ][(4 * j + t) / GQ];
        *reinterpret_cast<uint4 *>(dst + 4 * j) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
      }
    }
  }
  __syncthreads();

  // ---- horizontal carries: exclusive scans over warps and over chunks ----
  for (int e = threadIdx.x; e < nrows * G; e += blockDim.x) {
    uint32_t run = 0u;
    for (int ww = 0; ww < NW; ++ww) {
      uint32_t *p = s_row + (size_t)ww * f.R * G + e;
      const uint32_t v = *p;
      *p = run;
      run += v;
    }
  }
  for (int b = threadIdx.x; b < G; b += blockDim.x) {
    uint32_t run = 0u;
    for (int c = 0; c < f.nchunks; ++c) {
      uint32_t *p = s_ctot + (size_t)c * G + b;
      const uint32_t v = *p;
      *p = run;
      run += v;
    }
  }
  __syncthreads();

  // ---- publish aggregates (all chunks first: they depend on no one) ----
  for (int cc = 0; cc < my_m; ++cc) {
    const int c = c_begin + cc;
    if (lane < G) f.agg_left[(size_t)(ci0 + c) * G + lane] = s_ctot[(size_t)c * G + lane];
    __threadfence();
    __syncwarp();
    if (publish && lane == 0) st_release_gpu(f.flags + ci0 + c, (epoch << 2) | kStateAgg);
  }

  // ---- per chunk: look-back, publish inclusive row, emit ----
  for (int cc = 0; cc < my_m; ++cc) {
    const int c = c_begin + cc;
    const unsigned int ci = ci0 + c;
    const int x = c * kChunk + 4 * lane;

    uint32_t acc[G][4];   // becomes the running H of this lane's 4 columns
    uint32_t left[G];     // band-count sums left of the chunk, from aggregates
    uint32_t s16[GQ][4][2];
#pragma unroll
    for (int b = 0; b < G; ++b) {
      left[b] = 0u;
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[b][i] = 0u;
    }
#pragma unroll
    for (int q = 0; q < GQ; ++q)
#pragma unroll
      for (int i = 0; i < 4; ++i) s16[q][i][0] = s16[q][i][1] = 0u;

    bool poisoned = false;
    bool summed = false;
    for (int j = k - 1; j >= 0; --j) {
      const unsigned int cj = ((unsigned)j * f.ngroups + g) * (unsigned)f.nchunks + c;
      const uint32_t st = wait_flag(f.flags + cj, epoch, ctrl, timeout_ns);
      if (st == kStatePoison) {
        poisoned = true;
        break;
      }
      if (st == kStateIncl) {
#pragma unroll
        for (int b = 0; b < G; ++b) {
          const uint4 v = ld_relaxed_v4(f.incl + ((size_t)cj * G + b) * kChunk + 4 * lane);
          acc[b][0] = v.x; acc[b][1] = v.y; acc[b][2] = v.z; acc[b][3] = v.w;
        }
        break;
      }
      // aggregate: add the band's column counts (16-bit lanes, at most H)
      const uint32_t *src = f.agg_cnt + ((size_t)cj * kChunk + 4 * lane) * GQ;
#pragma unroll
      for (int jj = 0; jj < GQ; ++jj) {
        const uint4 v = ld_relaxed_v4(src + 4 * jj);
        const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int q = (4 * jj + t) % GQ, i = (4 * jj + t) / GQ;
          s16[q][i][0] += __byte_perm(wv[t], 0u, 0x4140u);
          s16[q][i][1] += __byte_perm(wv[t], 0u, 0x4342u);
        }
      }
#pragma unroll
      for (int b4 = 0; b4 < GQ; ++b4) {
        const uint4 v = ld_relaxed_v4(f.agg_left + (size_t)cj * G + 4 * b4);
        left[4 * b4 + 0] += v.x; left[4 * b4 + 1] += v.y;
        left[4 * b4 + 2] += v.z; left[4 * b4 + 3] += v.w;
      }
      summed = true;
    }
    poisoned = __any_sync(kFull, poisoned);

    if (!poisoned) {
      // top = incl row found + sum over the aggregates passed (Eq. 1 split
      // into the part left of the chunk and a prefix across the chunk)
      if (summed) {
#pragma unroll
        for (int b = 0; b < G; ++b) {
          const int q = b >> 2, h = (b >> 1) & 1, sh = (b & 1) * 16;
          uint32_t v[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) v[i] = (s16[q][i][h] >> sh) & 0xffffu;
          chunk_scan32(v, lane);
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[b][i] += v[i] + left[b];
        }
      }
      // inclusive row of this band = top + own aggregate, published for the bands below
      const uint32_t *own = f.agg_cnt + ((size_t)ci * kChunk + 4 * lane) * GQ;
      uint32_t ow[4 * GQ];
#pragma unroll
      for (int jj = 0; jj < GQ; ++jj) {
        const uint4 v = *reinterpret_cast<const uint4 *>(own + 4 * jj);
        ow[4 * jj + 0] = v.x; ow[4 * jj + 1] = v.y; ow[4 * jj + 2] = v.z; ow[4 * jj + 3] = v.w;
      }
#pragma unroll
      for (int b = 0; b < G; ++b) {
        const int q = b >> 2, bb = b & 3;
        uint32_t v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = __byte_perm(ow[i * GQ + q], 0u, 0x4440u + bb);
        chunk_scan32(v, lane);
        const uint32_t lown = s_ctot[(size_t)c * G + b];
        if (publish)
          *reinterpret_cast<uint4 *>(f.incl + ((size_t)ci * G + b) * kChunk + 4 * lane) =
              make_uint4(acc[b][0] + v[0] + lown, acc[b][1] + v[1] + lown,
                         acc[b][2] + v[2] + lown, acc[b][3] + v[3] + lown);
      }
      __threadfence();
      __syncwarp();
      if (publish && lane == 0) st_release_gpu(f.flags + ci, (epoch << 2) | kStateIncl);

      // ---- emit the band's rows of this chunk ----
      uint32_t *rowc = s_row + (size_t)w * f.R * G;
      const uint8_t *row = f.in + (long long)y0 * f.pitch;
      uint32_t un[4];
      load_offsets<VEC>(row, x, f.W, nbins, gbase, un);
      for (int yl = 0; yl < nrows; ++yl) {
        uint32_t u[4] = {un[0], un[1], un[2], un[3]};
        if (yl + 1 < nrows)
          load_offsets<VEC>(row + (long long)(yl + 1) * f.pitch, x, f.W, nbins, gbase, un);
        uint32_t rc[G];
#pragma unroll
        for (int b4 = 0; b4 < GQ; ++b4) {
          const uint4 v = *reinterpret_cast<const uint4 *>(rowc + (size_t)yl * G + 4 * b4);
          rc[4 * b4 + 0] = v.x; rc[4 * b4 + 1] = v.y; rc[4 * b4 + 2] = v.z; rc[4 * b4 + 3] = v.w;
        }
#pragma unroll
        for (int q = 0; q < GQ; ++q) {
          uint32_t p[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) p[i] = shl_clamp(1u, u[i] - 32u * q);
          p[1] += p[0];
          p[2] += p[1];
          p[3] += p[2];
          const uint32_t t = warp_scan_incl(p[3], lane);   // bytes <= 128
          const uint32_t ex = t - p[3];
          const uint32_t tot = __shfl_sync(kFull, t, 31);  // row total of the chunk
          p[0] += ex;
          p[1] += ex;
          p[2] += ex;
          p[3] = t;
#pragma unroll
          for (int bb = 0; bb < 4; ++bb) {
            const int b = 4 * q + bb;
            const uint32_t sel = 0x4440u + bb;
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[b][i] += __byte_perm(p[i], 0u, sel) + rc[b];
            rc[b] += __byte_perm(tot, 0u, sel);
          }
        }
        // store the row: bin-major H[b][y][x..x+3] or pixel-major H[y][x+i][b]
        const int y = y0 + yl;
        if (f.layout == 0) {
#pragma unroll
          for (int b = 0; b < G; ++b) {
            const int bg = g * G + b;
            if (bg < f.B) {
              uint32_t *o = f.out + ((size_t)bg * f.H + y) * f.W + x;
              if (VEC) {
                if (x < f.W) st_stream_v4(o, acc[b][0], acc[b][1], acc[b][2], acc[b][3]);
              } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                  if (x + i < f.W) st_stream(o + i, acc[b][i]);
              }
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if (x + i < f.W) {
              uint32_t *o = f.out + ((size_t)y * f.W + x + i) * f.B + g * G;
              if (VEC && (f.B % G == 0)) {
#pragma unroll
                for (int b4 = 0; b4 < GQ; ++b4)
                  st_stream_v4(o + 4 * b4, acc[4 * b4][i], acc[4 * b4 + 1][i], acc[4 * b4 + 2][i],
                               acc[4 * b4 + 3][i]);
              } else {
#pragma unroll
                for (int b = 0; b < G; ++b)
                  if (g * G + b < f.B) st_stream(o + b, acc[b][i]);
              }
            }
          }
        }
        __syncwarp();
        if (lane == 0) {
#pragma unroll
          for (int b4 = 0; b4 < GQ; ++b4)
            *reinterpret_cast<uint4 *>(rowc + (size_t)yl * G + 4 * b4) =
                make_uint4(rc[4 * b4], rc[4 * b4 + 1], rc[4 * b4 + 2], rc[4 * b4 + 3]);
        }
      }
    } else {
      if (publish && lane == 0) st_release_gpu(f.flags + ci, (epoch << 2) | kStatePoison);
    }
  }
}

// Persistent scan kernel over the work items of one frame.  CTAs draw
// tickets in increasing (band, group) order, so every band a CTA waits on
// belongs to a CTA that is already running; the last CTA to finish resets
// the ticket and advances the epoch, so launches need no host-side reset
// and can be captured in a CUDA graph.
template <int G, int MMAX, bool VEC>
__global__ void __launch_bounds__(512) scan_kernel(FrameDesc f, Ctrl *ctrl,
                                                    unsigned long long timeout_ns) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned int s_item, s_epoch;
  uint32_t *s_row = smem;
  uint32_t *s_ctot = smem + (size_t)(blockDim.x >> 5) * f.R * G;
  if (threadIdx.x == 0) s_epoch = *(volatile unsigned int *)&ctrl->epoch & 0x3fffffffu;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&ctrl->ticket, 1u);
    __syncthreads();
    const unsigned int it = s_item;
    const uint32_t epoch = s_epoch;
    __syncthreads();
    if (it >= f.nitems) break;
    process_item<G, MMAX, VEC>(f, it, epoch, ctrl, timeout_ns, s_row, s_ctot);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int d = atomicAdd(&ctrl->done, 1u);
    if (d == gridDim.x - 1) {
      ctrl->ticket = 0u;
      ctrl->done = 0u;
      __threadfence();
      atomicAdd(&ctrl->epoch, 1u);
    }
  }
}

}  // namespace ihist

// ihist_scan.cuh -- the fused integral-histogram kernel.
//
// Computes, for one frame, H[b][y][x] = #{x' <= x, y' <= y : Q(I[y'][x']) = b}
// (Eq. 1 of arXiv 1711.01919), the result Algorithm 1 builds with its
// recurrence, in one pass over the frame:
//
//   * a1 quantise: q = floor(v * B / 256) in registers (or, for other bin
//     structures, a 256-entry value -> bin table in shared memory); the
//     paper's one-hot initialisation tensor (Alg. 2-4, step 1) is never
//     materialised.
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
// Work item = (band k of R rows, bin group g of G bins, width segment s).
// The CTA's warps split the segment: warp w owns 128-column chunks
// [s*cps + w*m, s*cps + w*m + m) (cps = chunks per segment; one segment
// spans the whole width unless the frame is wider than a CTA's warps can
// cover).  Each
// warp stages its chunk's R x 128-byte input tile in shared memory (a TMA
// tensor copy when the frame is 16-byte aligned, else plain loads) and reads
// it once to count and once to emit.  The horizontal carry between warps
// comes from the counting pass (per-row bin totals of each warp's columns,
// one redux.sync per 4 bins) and an exclusive scan over warps in shared
// memory.  Between width segments of a band, each segment publishes its
// per-row bin totals right after counting (they depend on its own pixels
// only) and a segment adds those of every segment to its left: no chain, so
// the horizontal carry costs one wait for data that is already published
// when the segments run side by side.  The vertical carry between bands is
// the look-back, per (band, group, chunk).
#pragma once

#include <cuda.h>

#include "ihist_device.cuh"

namespace ihist {

// One frame as the kernel sees it.  Offsets of the carry buffers are in
// units of "chunk items": ci = ((k * ngroups + g) * nchunks + chunk) for band
// k, bin group g.  A work item is (band k, set of gpc bin groups).
struct FrameDesc {
  const uint8_t *in;
  long long pitch;      // bytes between rows of in
  uint32_t *out;
  const uint32_t *lut;  // table kernels: 8 * bin of each intensity, or kNoBin (no bin)
  int H, W, B, layout;  // layout: 0 bin-major, 1 pixel-major
  int qmul;             // uniform bins: q = (v * qmul) >> 8; qmul = B, or 256 when
                        // the input already holds bin indices
  int late_wait;        // scan_kernel: 1 = wait for the previous grid only before the
                        // first store; 0 = right after taking the first work item
  int R, nbands, ngroups, nchunks, m;
  int wpg;              // warps per bin group: ceil(nchunks / m)
  int gpc;              // bin groups per CTA (warp w serves group w / wpg)
  int ngsets;           // ceil(ngroups / gpc)
  int fault_skip_band;  // -1 off
  unsigned int nitems;  // nbands * ngsets
  uint32_t *agg_cnt;    // [ci][128 cols][G/4] words: packed column counts (bytes)
  uint32_t *agg_left;   // [ci][G]: band count left of the chunk
  uint32_t *incl;       // [ci][G][128]: H on the band's last row
  uint32_t *flags;      // [ci]
  int nsegs;            // width segments per band (1: one CTA spans the width)
  int cps;              // chunks per segment (wpg * m)
  uint32_t *hagg;       // [(k * ngroups + g) * nsegs + s][R * G + G]: a segment's per-row bin
                        // totals, then its band totals per bin (nsegs > 1 only)
  uint32_t *hflags;     // [(k * ngroups + g) * nsegs + s] (nsegs > 1 only)
};

// Dynamic shared memory of one CTA, carved from a 128-byte aligned base.
struct SmemLayout {
  uint32_t tile_off, row_off, ctot_off, bar_off, stage_off, bytes;
};

// Pixel-major rows go through a per-warp staging area when a bin group has
// at least 8 bins (see emit_pixel_major_staged).
__host__ __device__ inline bool pm_staged(int layout, int G) { return layout == 1 && G >= 8; }

__host__ __device__ inline SmemLayout smem_layout(int NW, int R, int G, int nchunks, bool stage = false) {
  SmemLayout L;
  uint32_t off = 0;
  L.tile_off = off;  // [NW][R][128] bytes
  off += (uint32_t)NW * (uint32_t)R * kChunk;
  off = (off + 15u) & ~15u;
  L.row_off = off;  // [NW][R][G] u32
  off += (uint32_t)NW * (uint32_t)R * (uint32_t)G * 4u;
  L.ctot_off = off;  // [groups per CTA][nchunks][G] u32 (nchunks passed as gpc * nchunks)
  off += (uint32_t)nchunks * (uint32_t)G * 4u;
  off = (off + 7u) & ~7u;
  L.bar_off = off;  // [NW] mbarriers
  off += (uint32_t)NW * 8u;
  off = (off + 15u) & ~15u;
  L.stage_off = off;  // [NW][128 px][G] u32 staging of pixel-major rows
  if (stage) off += (uint32_t)NW * kChunk * (uint32_t)G * 4u;
  L.bytes = off + 128u;  // + base alignment slack
  return L;
}

constexpr uint32_t kNoBin = 0x80000000u;

// a1: bit offset 8*q of a pixel's bin relative to the CTA's first bin
// (gbase = 8 * g * G).  Offsets of bins outside the CTA's group, of values
// in no bin and of columns past the frame are large or wrap around, so no
// 4-bin sub-group matches them (shl_clamp gives 0).
template <bool LUT>
struct Binner {
  uint32_t qmul;        // uniform: q = (v * qmul) >> 8
  const uint32_t *lut;  // table: 8 * bin of each intensity (shared memory)
  __device__ __forceinline__ uint32_t operator()(uint32_t v, uint32_t gbase) const {
    if constexpr (LUT)
      return lut[v] - gbase;
    else
      return (((v * qmul) >> 8) << 3) - gbase;
  }
};

// Inclusive prefix of v[0..3] (this lane's 4 columns) over the 128-column chunk.
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

// Bin offsets of this lane's 4 pixels in tile row yl (columns x .. x+3).
template <bool LUT>
__device__ __forceinline__ void tile_offsets(const uint8_t *tile, int yl, int lane, int x, int W,
                                             const Binner<LUT> &bin, uint32_t gbase, uint32_t u[4]) {
  const uint32_t px = *reinterpret_cast<const uint32_t *>(tile + yl * kChunk + 4 * lane);
#pragma unroll
  for (int i = 0; i < 4; ++i)
    u[i] = (x + i < W) ? bin(__byte_perm(px, 0u, 0x4440u + i), gbase) : kNoBin;
}

// Stage rows y0 .. y0+nrows-1, columns c*128 .. c*128+127 of the frame into
// this warp's tile.  TMA: one lane issues a tensor copy and the warp waits
// on the tile's mbarrier (bounded).  Otherwise: each lane copies its 4 bytes
// of every row with plain loads.  Columns past W are don't-care (masked by
// the x < W tests).  Returns false if the wait timed out.
template <bool TMA>
__device__ __forceinline__ bool stage_tile(const FrameDesc &f, const CUtensorMap *tmap, uint8_t *tile,
                                           uint64_t *bar, uint32_t &phase, int y0, int nrows, int c,
                                           int lane, unsigned long long timeout_ns) {
  if (TMA) {
    __syncwarp();  // every lane is done reading the previous tile
    if (lane == 0) {
      fence_proxy_async_smem();
      tma_load_2d(tmap, tile, bar, c * kChunk, y0, (uint32_t)f.R * kChunk);
    }
    const bool ok = mbar_wait(bar, phase, timeout_ns);
    phase ^= 1u;
    return __all_sync(kFull, ok);
  } else {
    __syncwarp();
    const int x = c * kChunk + 4 * lane;
    const bool aligned = ((reinterpret_cast<uintptr_t>(f.in) | (uintptr_t)f.pitch) & 3u) == 0;
#pragma unroll 4
    for (int yl = 0; yl < nrows; ++yl) {
      const uint8_t *src = f.in + (long long)(y0 + yl) * f.pitch + x;
      uint32_t v = 0u;
      if (aligned && x + 3 < f.W) {
        v = __ldg(reinterpret_cast<const unsigned int *>(src));
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (x + i < f.W) v |= (uint32_t)__ldg(src + i) << (8 * i);
      }
      *reinterpret_cast<uint32_t *>(tile + yl * kChunk + 4 * lane) = v;
    }
    __syncwarp();
    return true;
  }
}

// ---------------------------------------------------------------------------
// One work item: band k, bin group g.
// Slot of pixel p's quad r (4 bins) in a warp's staging area of
// [G/4 quads][128 pixels] 16-byte slots.  The XOR swizzle makes both the
// writes (lane -> its 4 pixels) and the reads (G/4 lanes per pixel) hit 8
// distinct 16-byte bank groups per quarter warp.
template <int GQ>
__device__ __forceinline__ int stage_slot(int r, int p) {
  constexpr int kShift = GQ >= 4 ? 1 : GQ == 2 ? 2 : 3;
  return r * kChunk + (p & ~7) + ((p ^ ((p >> 3) & 3) ^ (r << kShift)) & 7);
}

// Pixel-major store of one row of a warp's 128-pixel chunk through shared
// memory.  A pixel's record is B words; this CTA owns G of them.  Stored
// straight from registers, each warp store would put 16 bytes into each of
// 32 pixels' records; staged, G/4 consecutive lanes write one pixel's G
// contiguous words, so a warp store covers 32/(G/4) records in full pieces.
template <int G, bool VEC>
__device__ __forceinline__ void emit_pixel_major_staged(const FrameDesc &f, uint4 *stage, const uint32_t (&acc)[G][4],
                                                        int lane, int cbase, int y, int g, Ctrl *ctrl) {
  const uint32_t *out_end = f.out + (size_t)f.H * f.W * f.B;
  (void)out_end;
  (void)ctrl;
  constexpr int GQ = G / 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int r = 0; r < GQ; ++r)
      stage[stage_slot<GQ>(r, 4 * lane + i)] =
          make_uint4(acc[4 * r][i], acc[4 * r + 1][i], acc[4 * r + 2][i], acc[4 * r + 3][i]);
  __syncwarp();
  constexpr int PPI = 32 / GQ;  // pixels per warp store
  const int k = lane / GQ, r = lane % GQ;
  const bool full = VEC && (f.B & 3) == 0 && g * G + 4 * r + 4 <= f.B;
#pragma unroll 4
  for (int s = 0; s < kChunk / PPI; ++s) {
    const int p = s * PPI + k;
    const int x = cbase + p;
    if (x < f.W) {
      const uint4 v = stage[stage_slot<GQ>(r, p)];
      uint32_t *o = f.out + ((size_t)y * f.W + x) * f.B + g * G + 4 * r;
      if (full) {
        if (IHIST_GUARD(ctrl, o >= f.out && o + 4 <= out_end)) st_stream_v4(o, v.x, v.y, v.z, v.w);
      } else {
        const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int bb = 0; bb < 4; ++bb)
          if (g * G + 4 * r + bb < f.B && IHIST_GUARD(ctrl, o + bb >= f.out && o + bb < out_end))
            st_stream(o + bb, vv[bb]);
      }
    }
  }
  __syncwarp();  // the next row may overwrite the staging area
}

// Pixel-major rows when one CTA owns every bin of its pixels (gpc groups of
// G bins covering B, with B / 4 a power of two): the gpc warps that hold
// the same 128 columns, one per bin group, put their counts into one shared
// area of whole pixel records (B words each), then store the row's records
// together as one contiguous run of H, so each warp store writes 512
// contiguous bytes.  A record is kept as U = B / 4 16-byte units, unit j of
// pixel p at p * U + (j ^ ((p / 4) mod U)): eight consecutive lanes hit
// eight distinct 16-byte bank groups when writing (lane -> its 4 pixels)
// and when reading (consecutive units).  Two named barriers per row (id
// bar_id, the gpc warps) order the writes before the reads and the reads
// before the next row's writes.
template <int G, bool VEC>
__device__ __forceinline__ void emit_pixel_major_record(const FrameDesc &f, uint4 *rec, const uint32_t (&acc)[G][4],
                                                        int lane, int lg, int cbase, int y, int bar_id, int nthr,
                                                        Ctrl *ctrl) {
  const uint32_t *out_end = f.out + (size_t)f.H * f.W * f.B;
  (void)out_end;
  (void)ctrl;
  constexpr int GQ = G / 4;
  const int U = f.B >> 2;
  const int um = U - 1;
  const int lu = __ffs(U) - 1;
#pragma unroll
  for (int r = 0; r < GQ; ++r) {
    const int j = lg * GQ + r;
    if (j < U) {
      const int js = j ^ (lane & um);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        rec[(4 * lane + i) * U + js] = make_uint4(acc[4 * r][i], acc[4 * r + 1][i], acc[4 * r + 2][i], acc[4 * r + 3][i]);
    }
  }
  named_bar_sync(bar_id, nthr);
  const int nu = min(kChunk, f.W - cbase) << lu;
  uint32_t *o0 = f.out + ((size_t)y * f.W + cbase) * f.B;
  for (int u = lg * 32 + lane; u < nu; u += nthr) {
    const int p = u >> lu, j = u & um;
    const uint4 v = rec[p * U + (j ^ ((p >> 2) & um))];
    uint32_t *o = o0 + 4 * u;
    if (IHIST_GUARD(ctrl, o >= f.out && o + 4 <= out_end)) {
      if (VEC) {
        st_stream_v4(o, v.x, v.y, v.z, v.w);
      } else {
        st_stream(o, v.x);
        st_stream(o + 1, v.y);
        st_stream(o + 2, v.z);
        st_stream(o + 3, v.w);
      }
    }
  }
  named_bar_sync(bar_id, nthr);
}

// Bin counts whose pixel records the whole-record path can hold: B / 4
// 16-byte units, a power of two.
__host__ __device__ inline bool pm_record_bins(int B) {
  const int U = B >> 2;
  return (B & 3) == 0 && U > 0 && (U & (U - 1)) == 0;
}

// Whether a pixel-major frame takes the whole-record path above (uniform
// over the CTA: it depends only on the frame and the tiling).
template <int G>
__host__ __device__ inline bool pm_record(int layout, int B, int gpc, int ngroups) {
  return layout == 1 && G >= 8 && gpc > 1 && gpc == ngroups && gpc * G >= B && pm_record_bins(B);
}

template <int G, int MMAX, bool TMA, bool VEC, bool LUT, bool WINDOW>
__device__ __forceinline__ void process_item(const FrameDesc &f, const CUtensorMap *tmap,
                                             unsigned int it, uint32_t epoch, Ctrl *ctrl,
                                             unsigned long long timeout_ns, uint8_t *s_tiles,
                                             uint32_t *s_row, uint32_t *s_ctot, uint64_t *s_bar,
                                             const uint32_t *s_lut, uint4 *s_stage, uint32_t &phase,
                                             bool &dep_pending) {
  constexpr int GQ = G / 4;
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int nsegs = f.nsegs > 1 ? f.nsegs : 1;
  const int seg = (int)(it % (unsigned)nsegs);
  const unsigned int kg = it / (unsigned)nsegs;
  const int k = (int)(kg / (unsigned)f.ngsets);
  const int gs = (int)(kg % (unsigned)f.ngsets);
  // checked builds: the item must lie inside the frame (uniform over the CTA)
  if (!IHIST_GUARD(ctrl, k < f.nbands && gs < f.ngsets)) return;
  const int cseg0 = nsegs > 1 ? seg * f.cps : 0;                        // first chunk of the segment
  const int nchs = nsegs > 1 ? min(f.cps, f.nchunks - cseg0) : f.nchunks;  // chunks of the segment
  const int lg = w / f.wpg;  // local bin group of this warp
  const int wg = w % f.wpg;  // warp slot within the group
  const int g = gs * f.gpc + lg;
  const bool gvalid = (lg < f.gpc) && (g < f.ngroups);
  const int y0 = k * f.R;
  const int nrows = min(f.R, f.H - y0);
  const Binner<LUT> bin{(uint32_t)f.qmul, s_lut};
  const uint32_t gbase = 8u * (uint32_t)(g * G);
  const int c_begin = cseg0 + wg * f.m;
  const int my_m = gvalid ? max(0, min(f.m, cseg0 + nchs - c_begin)) : 0;  // warp-uniform
  const bool publish = (k != f.fault_skip_band);
  const unsigned int ci0 = ((unsigned)k * f.ngroups + g) * (unsigned)f.nchunks;  // chunk 0
  const unsigned int nci = (unsigned)f.nbands * f.ngroups * f.nchunks;  // carry slots of the frame
  const uint32_t *out_end = f.out + (size_t)f.H * f.W * f.B;           // end of the frame's H
  (void)nci;
  (void)out_end;
  // band totals per chunk of the segment, indexed by chunk - cseg0
  uint32_t *my_ctot = s_ctot + (size_t)(gvalid ? lg : 0) * nchs * G - (size_t)cseg0 * G;
  uint8_t *tile = s_tiles + (size_t)w * f.R * kChunk;
  uint64_t *bar = s_bar + w;
  uint32_t *myrow = s_row + (size_t)w * f.R * G;
  bool stage_ok = true;
  int staged = -1;  // chunk currently held in this warp's tile

  // ---- counting pass: column counts (bytes) and per-row segment totals ----
  uint32_t colcnt[MMAX][GQ][4];
#pragma unroll
  for (int cc = 0; cc < MMAX; ++cc)
#pragma unroll
    for (int q = 0; q < GQ; ++q)
#pragma unroll
      for (int i = 0; i < 4; ++i) colcnt[cc][q][i] = 0u;

  if (my_m == 0) {
    for (int e = lane; e < nrows * G; e += 32) myrow[e] = 0u;
  }
#pragma unroll
  for (int cc = 0; cc < MMAX; ++cc) {
    if (cc < my_m) {
      const int c = c_begin + cc;
      const int x = c * kChunk + 4 * lane;
      stage_ok &= stage_tile<TMA>(f, tmap, tile, bar, phase, y0, nrows, c, lane, timeout_ns);
      staged = c;
#pragma unroll 4
      for (int yl = 0; yl < nrows; ++yl) {
        uint32_t u[4];
        tile_offsets(tile, yl, lane, x, f.W, bin, gbase, u);
#pragma unroll
        for (int q = 0; q < GQ; ++q) {
          uint32_t rs = 0u;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint32_t ind = shl_clamp(1u, u[i] - 32u * q);
            colcnt[cc][q][i] += ind;
            rs += ind;
          }
          // row total of this chunk, four bins in bytes (each at most 128)
          const uint32_t t = __reduce_add_sync(kFull, rs);
          if (lane == 0) {
            uint4 *d = reinterpret_cast<uint4 *>(myrow + (size_t)yl * G + 4 * q);
            uint4 v = make_uint4(t & 0xffu, (t >> 8) & 0xffu, (t >> 16) & 0xffu, t >> 24);
            if (cc > 0) {
              const uint4 o = *d;
              v.x += o.x;
              v.y += o.y;
              v.z += o.z;
              v.w += o.w;
            }
            *d = v;
          }
        }
      }
    }
  }

  // the previous grid on the stream must be complete before the first
  // store to the carries or the output
  if (dep_pending) {
    griddep_wait_and_release();
    dep_pending = false;
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
          *reinterpret_cast<uint4 *>(my_ctot + (size_t)c * G + 4 * q) =
              make_uint4(lo & 0xffffu, lo >> 16, hi & 0xffffu, hi >> 16);
      }
      // aggregate: this band's column counts, [128 cols][GQ] words
      uint32_t *dst = f.agg_cnt + ((size_t)(ci0 + c) * kChunk + 4 * lane) * GQ;
      if (!IHIST_GUARD(ctrl, ci0 + c < nci)) continue;
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

  // ---- horizontal carries: exclusive scans over the warps of each bin
  // group (row carries) and over chunks (band counts left of each chunk) ----
  const int ngl = min(f.gpc, f.ngroups - gs * f.gpc);  // bin groups in this item
  // a segment's own totals, for the segments to its right
  const bool seg_pub = nsegs > 1 && seg < nsegs - 1 && publish;
  const size_t hstride = (size_t)f.R * G + G;                       // words per segment record
  const unsigned int hbase = ((unsigned)k * f.ngroups + gs * f.gpc) * (unsigned)nsegs;  // group lg: + lg * nsegs
  for (int e = threadIdx.x; e < ngl * nrows * G; e += blockDim.x) {
    const int l = e / (nrows * G), r = e - l * (nrows * G);
    uint32_t run = 0u;
    for (int ww = 0; ww < f.wpg; ++ww) {
      uint32_t *p = s_row + (size_t)(l * f.wpg + ww) * f.R * G + r;
      const uint32_t v = *p;
      *p = run;
      run += v;
    }
    if (seg_pub) f.hagg[(size_t)(hbase + l * nsegs + seg) * hstride + r] = run;
  }
  for (int e = threadIdx.x; e < ngl * G; e += blockDim.x) {
    const int l = e / G, b = e - l * G;
    uint32_t run = 0u;
    for (int c = 0; c < nchs; ++c) {
      uint32_t *p = s_ctot + ((size_t)l * nchs + c) * G + b;
      const uint32_t v = *p;
      *p = run;
      run += v;
    }
    if (seg_pub) f.hagg[(size_t)(hbase + l * nsegs + seg) * hstride + (size_t)f.R * G + b] = run;
  }
  if (nsegs > 1) {
    // publish this segment's totals (poisoned if any warp's staging failed),
    // then add the totals of every segment to the left
    if (seg_pub) __threadfence();
    const bool bad = __syncthreads_or(!stage_ok);
    if (seg_pub && threadIdx.x < ngl)
      st_release_gpu(f.hflags + hbase + threadIdx.x * nsegs + seg, (epoch << 2) | (bad ? kStatePoison : kStateAgg));
    bool hpoison = bad;
    for (int l = 0; l < ngl && !hpoison; ++l)
      for (int j = 0; j < seg && !hpoison; ++j)
        if (wait_flag(f.hflags + hbase + l * nsegs + j, epoch, ctrl, timeout_ns) == kStatePoison) hpoison = true;
    hpoison = __syncthreads_or(hpoison);
    if (hpoison) {
      stage_ok = false;  // publish poison below and emit nothing
    } else if (seg > 0) {
      for (int e = threadIdx.x; e < ngl * nrows * G; e += blockDim.x) {
        const int l = e / (nrows * G), r = e - l * (nrows * G);
        uint32_t left = 0u;
        for (int j = 0; j < seg; ++j) left += ld_relaxed_u32(f.hagg + (size_t)(hbase + l * nsegs + j) * hstride + r);
        for (int ww = 0; ww < f.wpg; ++ww) s_row[(size_t)(l * f.wpg + ww) * f.R * G + r] += left;
      }
      for (int e = threadIdx.x; e < ngl * G; e += blockDim.x) {
        const int l = e / G, b = e - l * G;
        uint32_t left = 0u;
        for (int j = 0; j < seg; ++j)
          left += ld_relaxed_u32(f.hagg + (size_t)(hbase + l * nsegs + j) * hstride + (size_t)f.R * G + b);
        for (int c = 0; c < nchs; ++c) s_ctot[((size_t)l * nchs + c) * G + b] += left;
      }
    }
  }
  __syncthreads();

  // ---- publish aggregates (all chunks first: they depend on no one) ----
  for (int cc = 0; cc < my_m; ++cc) {
    const int c = c_begin + cc;
    if (!IHIST_GUARD(ctrl, ci0 + c < nci)) continue;
    if (lane < G) f.agg_left[(size_t)(ci0 + c) * G + lane] = my_ctot[(size_t)c * G + lane];
    __threadfence();
    __syncwarp();
    if (publish && lane == 0)
      st_release_gpu(f.flags + ci0 + c, (epoch << 2) | (stage_ok ? kStateAgg : kStatePoison));
  }

  // ---- per chunk: look-back, publish inclusive row, emit ----
  // Whole-record pixel-major rows: the warps of every bin group holding the
  // same columns (same wg, same chunks, same rows) meet at named barrier
  // 1 + wg, so each of them runs the same barrier sequence per chunk: one
  // vote before the rows (taken on every path) and two per row.
  const bool record = s_stage != nullptr && pm_record<G>(f.layout, f.B, f.gpc, f.ngroups);
  const int rec_bar = 1 + wg, rec_thr = 32 * f.gpc;
  for (int cc = 0; cc < my_m; ++cc) {
    const int c = c_begin + cc;
    const unsigned int ci = ci0 + c;
    const int x = c * kChunk + 4 * lane;
    const bool ci_ok = IHIST_GUARD(ctrl, ci < nci);
    if (!ci_ok && !record) continue;

    uint32_t left[G];  // band-count sums left of the chunk, from aggregates
    uint32_t s16[GQ][4][2];
#pragma unroll
    for (int b = 0; b < G; ++b) left[b] = 0u;
#pragma unroll
    for (int q = 0; q < GQ; ++q)
#pragma unroll
      for (int i = 0; i < 4; ++i) s16[q][i][0] = s16[q][i][1] = 0u;

    bool poisoned = !stage_ok || !ci_ok;
    bool summed = false;
    int incl_at = -1;  // band whose inclusive row ends the look-back
    // Look back over the bands above.  The band just above has usually
    // published its inclusive row already, so the first pass watches that
    // one band with every lane (one flag); if it holds only its aggregate,
    // later passes watch 32 bands at a time: lane l acquires band j - l's
    // flag, the nearest inclusive row (or poison) ends the walk, and the
    // aggregates before it are added with independent loads.  A frame whose
    // bands all run at once (less than one wave) thus resolves its carries
    // in a few round trips instead of one per band.
    int j = k - 1;
    int wn = 1;  // bands watched in this pass
    while (WINDOW && j >= 0 && !poisoned) {
      const int jb = j - (wn > 1 ? lane : 0);  // the band this lane watches
      const unsigned int cjl = ((unsigned)(jb >= 0 ? jb : 0) * f.ngroups + g) * (unsigned)f.nchunks + c;
      if (!IHIST_GUARD(ctrl, cjl < nci)) {
        poisoned = true;
        break;
      }
      unsigned long long t0 = 0;
      unsigned int backoff = 32;
      uint32_t st = kStateIncl;  // past band 0: an inclusive row of zeros
      int first = -1;            // lane of the nearest inclusive row or poison; wn: none in this pass
      for (;;) {
        if (jb >= 0) {
          const uint32_t fl = ld_acquire_gpu(f.flags + cjl);
          st = ((fl >> 2) == epoch) ? (fl & 3u) : 0u;
        }
        const unsigned int stop = __ballot_sync(kFull, st == kStateIncl || st == kStatePoison);
        const unsigned int ready = __ballot_sync(kFull, st != 0u);
        first = stop ? min(__ffs(stop) - 1, wn) : wn;
        const unsigned int need = first >= 32 ? kFull : ((1u << first) - 1u);
        if ((ready & need) == need) break;  // every band before the stop has published
        const unsigned long long now = __shfl_sync(kFull, global_ns(), 0);
        if (t0 == 0) {
          t0 = now;
        } else if (now - t0 > timeout_ns) {
          if (lane == 0) {
            latch_status(ctrl, kStatusTimeout);
            atomicAdd(&ctrl->timeouts, 1u);
          }
          first = -1;
          break;
        }
        __nanosleep(backoff);
        if (backoff < 1024) backoff <<= 1;
      }
      if (first < 0) {
        poisoned = true;
        break;
      }
      __syncwarp();  // orders every lane's reads below after the acquiring lanes' flag loads
      for (int l = 0; l < first; ++l) {
        // aggregate of band j - l: its column counts (16-bit lanes, at most
        // H) and its counts left of the chunk
        const unsigned int cj = ((unsigned)(j - l) * f.ngroups + g) * (unsigned)f.nchunks + c;
        const uint32_t *src = f.agg_cnt + ((size_t)cj * kChunk + 4 * lane) * GQ;
#pragma unroll
        for (int jj = 0; jj < GQ; ++jj) {
          const uint4 v = ld_relaxed_v4(src + 4 * jj);
          const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int q = (4 * jj + t) % GQ, ii = (4 * jj + t) / GQ;
            s16[q][ii][0] += __byte_perm(wv[t], 0u, 0x4140u);
            s16[q][ii][1] += __byte_perm(wv[t], 0u, 0x4342u);
          }
        }
#pragma unroll
        for (int b4 = 0; b4 < GQ; ++b4) {
          const uint4 v = ld_relaxed_v4(f.agg_left + (size_t)cj * G + 4 * b4);
          left[4 * b4 + 0] += v.x;
          left[4 * b4 + 1] += v.y;
          left[4 * b4 + 2] += v.z;
          left[4 * b4 + 3] += v.w;
        }
        summed = true;
      }
      if (first < wn) {
        const uint32_t sf = __shfl_sync(kFull, st, first);
        if (sf == kStatePoison)
          poisoned = true;
        else if (j - first >= 0)
          incl_at = j - first;
        break;
      }
      j -= wn;
      wn = 32;
    }
    // Batched launches: many waves, so the band above has nearly always
    // published its inclusive row; walk one band at a time (less code in
    // the loop that every item runs: the window measured 4% slower there).
    for (j = k - 1; !WINDOW && j >= 0 && !poisoned; --j) {
      const unsigned int cj = ((unsigned)j * f.ngroups + g) * (unsigned)f.nchunks + c;
      if (!IHIST_GUARD(ctrl, cj < nci)) {
        poisoned = true;
        break;
      }
      const uint32_t st = wait_flag(f.flags + cj, epoch, ctrl, timeout_ns);
      if (st == kStatePoison) {
        poisoned = true;
        break;
      }
      if (st == kStateIncl) {
        incl_at = j;
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
          const int q = (4 * jj + t) % GQ, ii = (4 * jj + t) / GQ;
          s16[q][ii][0] += __byte_perm(wv[t], 0u, 0x4140u);
          s16[q][ii][1] += __byte_perm(wv[t], 0u, 0x4342u);
        }
      }
#pragma unroll
      for (int b4 = 0; b4 < GQ; ++b4) {
        const uint4 v = ld_relaxed_v4(f.agg_left + (size_t)cj * G + 4 * b4);
        left[4 * b4 + 0] += v.x;
        left[4 * b4 + 1] += v.y;
        left[4 * b4 + 2] += v.z;
        left[4 * b4 + 3] += v.w;
      }
      summed = true;
    }
    poisoned = __any_sync(kFull, poisoned);

    if (!poisoned) {
      // top = inclusive row found + the aggregates passed (Eq. 1 split into
      // the count left of the chunk and a prefix across the chunk)
      uint32_t acc[G][4];  // becomes the running H of this lane's 4 columns
      // bin by bin, so each bin's aggregate sums are dead once its row is in
      // acc (fewer registers live at once than loading the whole row first)
      const unsigned int cji = ((unsigned)(incl_at >= 0 ? incl_at : 0) * f.ngroups + g) * (unsigned)f.nchunks + c;
#pragma unroll
      for (int b = 0; b < G; ++b) {
        if (incl_at >= 0) {
          const uint4 v = ld_relaxed_v4(f.incl + ((size_t)cji * G + b) * kChunk + 4 * lane);
          acc[b][0] = v.x;
          acc[b][1] = v.y;
          acc[b][2] = v.z;
          acc[b][3] = v.w;
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[b][i] = 0u;
        }
        if (summed) {
          const int q = b >> 2, h = (b >> 1) & 1, sh = (b & 1) * 16;
          uint32_t v[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) v[i] = (s16[q][i][h] >> sh) & 0xffffu;
          chunk_scan32(v, lane);
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[b][i] += v[i] + left[b];
        }
      }
      // inclusive row of this band = top + own aggregate, for the bands below
      // (own column counts read one 4-bin quad at a time)
      const uint32_t *own = f.agg_cnt + ((size_t)ci * kChunk + 4 * lane) * GQ;
#pragma unroll
      for (int q = 0; q < GQ; ++q) {
        uint32_t ow[4];  // bins 4q..4q+3 of this lane's 4 columns: word i*GQ + q
#pragma unroll
        for (int i = 0; i < 4; ++i) ow[i] = own[i * GQ + q];
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) {
          const int b = 4 * q + bb;
          uint32_t v[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) v[i] = __byte_perm(ow[i], 0u, 0x4440u + bb);
          chunk_scan32(v, lane);
          const uint32_t lown = my_ctot[(size_t)c * G + b];
          if (publish)
            *reinterpret_cast<uint4 *>(f.incl + ((size_t)ci * G + b) * kChunk + 4 * lane) =
                make_uint4(acc[b][0] + v[0] + lown, acc[b][1] + v[1] + lown,
                           acc[b][2] + v[2] + lown, acc[b][3] + v[3] + lown);
        }
      }
      __threadfence();
      __syncwarp();
      if (publish && lane == 0) st_release_gpu(f.flags + ci, (epoch << 2) | kStateIncl);

      // ---- emit the band's rows of this chunk ----
      bool emit_ok = true;
      if (staged != c) {
        emit_ok = stage_tile<TMA>(f, tmap, tile, bar, phase, y0, nrows, c, lane, timeout_ns);
        if (emit_ok)
          staged = c;
        else if (lane == 0)
          latch_status(ctrl, kStatusTimeout);
      }
      if (record) emit_ok = named_bar_and(rec_bar, rec_thr, emit_ok);
      if (!emit_ok) continue;
      const size_t plane = (size_t)f.H * (size_t)f.W;
      const bool last_chunk = (cc == my_m - 1);  // its row carries are not needed again
      for (int yl = 0; yl < nrows; ++yl) {
        uint32_t u[4];
        tile_offsets(tile, yl, lane, x, f.W, bin, gbase, u);
        uint32_t *rcp = myrow + (size_t)yl * G;
#pragma unroll
        for (int q = 0; q < GQ; ++q) {
          uint4 rc = *reinterpret_cast<const uint4 *>(rcp + 4 * q);
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
          const uint32_t rcv[4] = {rc.x, rc.y, rc.z, rc.w};
#pragma unroll
          for (int bb = 0; bb < 4; ++bb) {
            const uint32_t sel = 0x4440u + bb;
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[4 * q + bb][i] += __byte_perm(p[i], 0u, sel) + rcv[bb];
          }
          if (!last_chunk) {
            rc.x += __byte_perm(tot, 0u, 0x4440u);
            rc.y += __byte_perm(tot, 0u, 0x4441u);
            rc.z += __byte_perm(tot, 0u, 0x4442u);
            rc.w += __byte_perm(tot, 0u, 0x4443u);
            __syncwarp();
            if (lane == 0) *reinterpret_cast<uint4 *>(rcp + 4 * q) = rc;
          }
        }
        // store the row: bin-major H[b][y][x..x+3] or pixel-major H[y][x+i][b]
        const int y = y0 + yl;
        if (f.layout == 0) {
          uint32_t *o = f.out + ((size_t)(g * G) * f.H + y) * f.W + x;
#pragma unroll
          for (int b = 0; b < G; ++b, o += plane) {
            if (g * G + b < f.B) {
              if (VEC) {
                if (x < f.W && IHIST_GUARD(ctrl, o >= f.out && o + 4 <= out_end))
                  st_stream_v4(o, acc[b][0], acc[b][1], acc[b][2], acc[b][3]);
              } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                  if (x + i < f.W && IHIST_GUARD(ctrl, o + i >= f.out && o + i < out_end))
                    st_stream(o + i, acc[b][i]);
              }
            }
          }
        } else if (f.layout == 2) {
          // quad-major H[b/4][y][x][b%4]: a pixel's four counts of a quad in
          // one 16-byte word, so a warp's row of a quad is 2 KB contiguous.
          // Two pixels per 32-byte store, so every store fills whole DRAM
          // sectors (16-byte stores at a 64-byte stride left half-written
          // sectors: 8.2 ms against 5.2 for 64 1080p frames).
          const bool v8 = VEC && ((reinterpret_cast<uintptr_t>(f.out) & 31u) == 0);
#pragma unroll
          for (int q = 0; q < GQ; ++q) {
            const int b0 = g * G + 4 * q;
            if (b0 < f.B) {  // B is a multiple of 4: the whole quad exists
              uint32_t *o = f.out + (((size_t)(b0 >> 2) * f.H + y) * f.W + x) * 4;
#pragma unroll
              for (int j = 0; j < 2; ++j) {
                const uint4 p0 = make_uint4(acc[4 * q][2 * j], acc[4 * q + 1][2 * j], acc[4 * q + 2][2 * j],
                                            acc[4 * q + 3][2 * j]);
                const uint4 p1 = make_uint4(acc[4 * q][2 * j + 1], acc[4 * q + 1][2 * j + 1],
                                            acc[4 * q + 2][2 * j + 1], acc[4 * q + 3][2 * j + 1]);
                uint32_t *oj = o + 8 * j;
                if (v8 && x + 2 * j + 1 < f.W) {  // VEC: w % 4 == 0, so oj is 32-byte aligned
                  if (IHIST_GUARD(ctrl, oj >= f.out && oj + 8 <= out_end &&
                                            (reinterpret_cast<uintptr_t>(oj) & 31u) == 0))
                    st_stream_v8(oj, p0, p1);
                } else {
#pragma unroll
                  for (int k = 0; k < 2; ++k) {
                    const uint4 v = k ? p1 : p0;
                    uint32_t *ok = oj + 4 * k;
                    if (x + 2 * j + k < f.W && IHIST_GUARD(ctrl, ok >= f.out && ok + 4 <= out_end)) {
                      if (VEC) {
                        st_stream_v4(ok, v.x, v.y, v.z, v.w);
                      } else {
                        st_stream(ok, v.x);
                        st_stream(ok + 1, v.y);
                        st_stream(ok + 2, v.z);
                        st_stream(ok + 3, v.w);
                      }
                    }
                  }
                }
              }
            }
          }
        } else if (G >= 8 && s_stage != nullptr) {
          if (record)
            emit_pixel_major_record<G, VEC>(f, s_stage + (size_t)wg * (kChunk * G / 4) * f.gpc, acc, lane, lg,
                                            c * kChunk, y, rec_bar, rec_thr, ctrl);
          else
            emit_pixel_major_staged<G, VEC>(f, s_stage + (size_t)w * (kChunk * G / 4), acc, lane, c * kChunk, y, g,
                                            ctrl);
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if (x + i < f.W) {
              uint32_t *o = f.out + ((size_t)y * f.W + x + i) * f.B + g * G;
#pragma unroll
              for (int b4 = 0; b4 < GQ; ++b4) {
                if (VEC && (f.B & 3) == 0 && g * G + 4 * b4 + 4 <= f.B) {
                  if (IHIST_GUARD(ctrl, o + 4 * b4 >= f.out && o + 4 * b4 + 4 <= out_end))
                    st_stream_v4(o + 4 * b4, acc[4 * b4][i], acc[4 * b4 + 1][i], acc[4 * b4 + 2][i],
                                 acc[4 * b4 + 3][i]);
                } else {
#pragma unroll
                  for (int bb = 0; bb < 4; ++bb)
                    if (g * G + 4 * b4 + bb < f.B &&
                        IHIST_GUARD(ctrl, o + 4 * b4 + bb >= f.out && o + 4 * b4 + bb < out_end))
                      st_stream(o + 4 * b4 + bb, acc[4 * b4 + bb][i]);
                }
              }
            }
          }
        }
      }
    } else {
      if (ci_ok && publish && lane == 0) st_release_gpu(f.flags + ci, (epoch << 2) | kStatePoison);
      if (!stage_ok && lane == 0) latch_status(ctrl, kStatusTimeout);
      if (record) (void)named_bar_and(rec_bar, rec_thr, false);  // the vote the rows would take
    }
  }
}

// Persistent scan kernel over the work items of one frame.  CTAs draw
// tickets in increasing (band, group) order, so every band a CTA waits on
// belongs to a CTA that is already running; the last CTA to finish resets
// the ticket and advances the epoch, so launches need no host-side reset
// and can be captured in a CUDA graph.
template <int G, int MMAX, bool TMA, bool VEC, bool LUT>
__global__ void __launch_bounds__(512, (G <= 8 ? 2 : 1))
    scan_kernel(FrameDesc f, const __grid_constant__ CUtensorMap tmap, Ctrl *ctrl,
                unsigned long long timeout_ns) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ unsigned int s_item, s_epoch;
  __shared__ uint32_t s_lut[LUT ? 256 : 1];
  const int NW = blockDim.x >> 5;
  const bool stage = pm_staged(f.layout, G);
  const int ncl = f.nsegs > 1 ? min(f.nchunks, f.cps) : f.nchunks;  // chunks of one CTA group
  const SmemLayout L = smem_layout(NW, f.R, G, ncl * f.gpc, stage);
  uint8_t *base = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint4 *s_stage = stage ? reinterpret_cast<uint4 *>(base + L.stage_off) : nullptr;
  uint8_t *s_tiles = base + L.tile_off;
  uint32_t *s_row = reinterpret_cast<uint32_t *>(base + L.row_off);
  uint32_t *s_ctot = reinterpret_cast<uint32_t *>(base + L.ctot_off);
  uint64_t *s_bar = reinterpret_cast<uint64_t *>(base + L.bar_off);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (TMA && lane == 0) mbar_init(s_bar + w, 1);
  if (threadIdx.x == 0) s_epoch = *(volatile unsigned int *)&ctrl->epoch & 0x3fffffffu;
  if (LUT)
    for (int i = threadIdx.x; i < 256; i += blockDim.x) s_lut[i] = __ldg(f.lut + i);
  if (TMA) mbar_init_fence();
  uint32_t phase = 0;
  bool dep_pending = true;  // griddepcontrol.wait not yet done by this thread
  // A grid of one CTA per item (frames below one wave): the first draws
  // take every ticket, so no CTA draws a second one.
  const bool one_each = gridDim.x >= f.nitems;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&ctrl->ticket, 1u);
    __syncthreads();
    const unsigned int it = s_item;
    const uint32_t epoch = s_epoch;
    __syncthreads();
    if (it >= f.nitems) break;
    // Programmatic dependent launch: by default nothing of the frame is read
    // before the grid the launch depends on has completed; with late_wait
    // the first band is staged and counted first (the caller guarantees
    // that grid does not write the frame).
    if (dep_pending && f.late_wait == 0) {
      griddep_wait_and_release();
      dep_pending = false;
    }
    process_item<G, MMAX, TMA, VEC, LUT, true>(f, &tmap, it, epoch, ctrl, timeout_ns, s_tiles, s_row, s_ctot,
                                         s_bar, s_lut, s_stage, phase, dep_pending);
    __syncthreads();
    if (one_each) break;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int d = atomicAdd(&ctrl->done, 1u);
    if (d == gridDim.x - 1) {
      ctrl->ticket = 0u;
      ctrl->done = 0u;
      __threadfence();
      atomicAdd(&ctrl->epoch, 2u);
    }
  }
}

// Batched persistent kernel: one launch over the work items of many frames
// of uneven size (Sec. 4.4's image sequences, as one work-list).  Tickets
// run frame by frame and band-major within a frame, so a CTA only waits on
// bands of its own frame that a running CTA holds.  Per-frame descriptors
// and TMA tensor maps live in device memory; shared memory is sized for the
// largest frame (R_max rows, nchunk_gpc_max chunk x group columns).  LUT:
// every frame bins through its own value -> bin table (FrameDesc::lut),
// copied into shared memory whenever the CTA moves to another frame.
template <int G, int MMAX, bool TMA, bool VEC, bool LUT>
__global__ void __launch_bounds__(512, (G <= 8 ? 2 : 1))
    batch_kernel(const FrameDesc *frames, const CUtensorMap *__restrict__ tmaps,
                 const unsigned int *item_end, int nframes, int R_max,
                 int nchunk_gpc_max, int stage, Ctrl *ctrl, unsigned long long timeout_ns) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ unsigned int s_item, s_epoch;
  __shared__ int s_frame;
  __shared__ __align__(16) FrameDesc s_f;
  __shared__ uint32_t s_lut[LUT ? 256 : 1];
  const int NW = blockDim.x >> 5;
  const SmemLayout L = smem_layout(NW, R_max, G, nchunk_gpc_max, stage != 0);
  uint8_t *base = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint8_t *s_tiles = base + L.tile_off;
  uint32_t *s_row = reinterpret_cast<uint32_t *>(base + L.row_off);
  uint32_t *s_ctot = reinterpret_cast<uint32_t *>(base + L.ctot_off);
  uint64_t *s_bar = reinterpret_cast<uint64_t *>(base + L.bar_off);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (TMA && lane == 0) mbar_init(s_bar + w, 1);
  if (threadIdx.x == 0) s_epoch = *(volatile unsigned int *)&ctrl->epoch & 0x3fffffffu;
  if (TMA) mbar_init_fence();
  const unsigned int total = ld_relaxed_u32(item_end + nframes - 1);
  uint32_t phase = 0;
  bool dep_pending = true;  // griddepcontrol.wait not yet done by this thread
  int lut_frame = -1;       // frame whose table s_lut holds
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned int t = atomicAdd(&ctrl->ticket, 1u);
      s_item = t;
      int lo = 0, hi = nframes - 1;  // first frame whose item range ends after t
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ld_relaxed_u32(item_end + mid) > t) hi = mid; else lo = mid + 1;
      }
      s_frame = lo;
    }
    __syncthreads();
    const unsigned int t = s_item;
    const int fi = s_frame;
    const uint32_t epoch = s_epoch;
    if (t < total) {
      // descriptors are read with coherent loads (never a stale cached line)
      constexpr int kWords = (int)(sizeof(FrameDesc) / sizeof(uint32_t));
      const uint32_t *src = reinterpret_cast<const uint32_t *>(frames + fi);
      for (int i = threadIdx.x; i < kWords; i += blockDim.x)
        reinterpret_cast<uint32_t *>(&s_f)[i] = ld_relaxed_u32(src + i);
      if (LUT && fi != lut_frame) {
        const uint32_t *lut = reinterpret_cast<const uint32_t *>(ld_relaxed_u64(&frames[fi].lut));
        const bool ok = IHIST_GUARD(ctrl, lut != nullptr);
        for (int i = threadIdx.x; i < 256; i += blockDim.x) s_lut[i] = ok ? ld_relaxed_u32(lut + i) : kNoBin;
      }
    }
    __syncthreads();
    if (t >= total) break;
    lut_frame = fi;
    const unsigned int it = t - (fi > 0 ? ld_relaxed_u32(item_end + fi - 1) : 0u);
    uint4 *s_stage = (stage != 0 && pm_staged(s_f.layout, G)) ? reinterpret_cast<uint4 *>(base + L.stage_off)
                                                               : nullptr;
    process_item<G, MMAX, TMA, VEC, LUT, false>(s_f, tmaps + fi, it, epoch, ctrl, timeout_ns, s_tiles, s_row,
                                         s_ctot, s_bar, LUT ? s_lut : nullptr, s_stage, phase, dep_pending);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int d = atomicAdd(&ctrl->done, 1u);
    if (d == gridDim.x - 1) {
      ctrl->ticket = 0u;
      ctrl->done = 0u;
      __threadfence();
      atomicAdd(&ctrl->epoch, 2u);
    }
  }
}

}  // namespace ihist

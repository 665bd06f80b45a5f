// ihist_mappings.cu -- the paper's own GPU mappings of the integral
// histogram (arXiv 1711.01919, Sec. 3.3-3.5), rebuilt on this GPU as
// comparison kernels for the ablation of the fused look-back design:
//
//   CW-STS (Sec. 3.3, Alg. 3): one-hot initialisation of the b x h x w
//          tensor, one horizontal scan launch over every row of every bin,
//          a 3-D transpose, the same row scan over the transposed rows, and
//          a transpose back to [b][h][w].
//   CW-TiS (Sec. 3.4, Alg. 4): one-hot initialisation, then a horizontal
//          pass strip by strip (one launch per vertical strip of tile
//          width, each tile scanning its rows from the last column of the
//          strip to its left) and a vertical pass strip by strip (one launch
//          per horizontal strip).
//   WF-TiS (Sec. 3.5, Alg. 5, Eq. 6): one-hot initialisation, then one
//          launch per anti-diagonal of tiles; each tile does its 2-D scan in
//          shared memory and adds the final last column of the tile to its
//          left, the final last row of the tile above and their corner.
//
// They compute exactly the H of Eq. 1 (bin-major), but with the paper's
// passes over global memory and its launch counts; they are measured, not
// tuned.  Tiles are 32 x 32 words.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ihist.h"

namespace {

constexpr int kT = 32;  // tile edge

// Step 1 of Alg. 2-5: Q[b][y][x] = 1 if the pixel falls in bin b.
__global__ void onehot_kernel(const uint8_t *__restrict__ in, long long pitch, int H, int W, int B,
                              uint32_t *__restrict__ q) {
  const long long plane = (long long)H * W;
  const long long total = plane * B;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / plane);
    const long long p = e - (long long)b * plane;
    const int y = (int)(p / W), x = (int)(p - (long long)y * W);
    const uint32_t v = in[(long long)y * pitch + x];
    q[e] = ((v * (uint32_t)B) >> 8) == (uint32_t)b ? 1u : 0u;
  }
}

// Inclusive scan of `rows` rows of `len` words in place, one block per row:
// each thread scans a contiguous run, then a block scan of the run totals.
__global__ void __launch_bounds__(256) row_scan_kernel(uint32_t *__restrict__ a, long long rows, int len) {
  __shared__ uint32_t s_tot[256];
  const int t = threadIdx.x;
  const int per = (len + blockDim.x - 1) / blockDim.x;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    uint32_t *row = a + r * len;
    const int lo = min(len, t * per), hi = min(len, lo + per);
    uint32_t run = 0u;
    for (int i = lo; i < hi; ++i) run += row[i];
    s_tot[t] = run;
    __syncthreads();
    for (int d = 1; d < (int)blockDim.x; d <<= 1) {  // Hillis-Steele scan of the run totals
      const uint32_t v = t >= d ? s_tot[t - d] : 0u;
      __syncthreads();
      s_tot[t] += v;
      __syncthreads();
    }
    uint32_t acc = t > 0 ? s_tot[t - 1] : 0u;
    for (int i = lo; i < hi; ++i) {
      acc += row[i];
      row[i] = acc;
    }
    __syncthreads();
  }
}

// [b][h][w] -> [b][w][h] through 32 x 33 shared tiles.
__global__ void transpose_kernel(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst, int H, int W) {
  __shared__ uint32_t tile[kT][kT + 1];
  const int b = blockIdx.z;
  const uint32_t *s = src + (size_t)b * H * W;
  uint32_t *d = dst + (size_t)b * H * W;
  const int x0 = blockIdx.x * kT, y0 = blockIdx.y * kT;
  for (int j = threadIdx.y; j < kT; j += blockDim.y) {
    const int y = y0 + j, x = x0 + threadIdx.x;
    if (y < H && x < W) tile[j][threadIdx.x] = s[(size_t)y * W + x];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < kT; j += blockDim.y) {
    const int x = x0 + j, y = y0 + threadIdx.x;  // output row x, column y
    if (x < W && y < H) d[(size_t)x * H + y] = tile[threadIdx.x][j];
  }
}

// CW-TiS horizontal pass over one vertical strip (columns sx .. sx+31):
// each block scans the rows of one 32 x 32 tile of one bin, starting from
// the (already final) last column of the strip to the left.
__global__ void tis_hstrip_kernel(uint32_t *__restrict__ a, int H, int W, int sx) {
  __shared__ uint32_t tile[kT][kT + 1];
  const int b = blockIdx.z, y0 = blockIdx.y * kT;
  uint32_t *p = a + (size_t)b * H * W;
  for (int j = threadIdx.y; j < kT; j += blockDim.y) {
    const int y = y0 + j, x = sx + threadIdx.x;
    tile[j][threadIdx.x] = (y < H && x < W) ? p[(size_t)y * W + x] : 0u;
  }
  __syncthreads();
  if (threadIdx.y == 0) {  // one thread per row of the tile
    const int y = y0 + threadIdx.x;
    if (y < H) {
      uint32_t run = sx > 0 ? p[(size_t)y * W + sx - 1] : 0u;
      for (int i = 0; i < kT; ++i) {
        run += tile[threadIdx.x][i];
        tile[threadIdx.x][i] = run;
      }
    }
  }
  __syncthreads();
  for (int j = threadIdx.y; j < kT; j += blockDim.y) {
    const int y = y0 + j, x = sx + threadIdx.x;
    if (y < H && x < W) p[(size_t)y * W + x] = tile[j][threadIdx.x];
  }
}

// CW-TiS vertical pass over one horizontal strip (rows sy .. sy+31).
__global__ void tis_vstrip_kernel(uint32_t *__restrict__ a, int H, int W, int sy) {
  __shared__ uint32_t tile[kT][kT + 1];
  const int b = blockIdx.z, x0 = blockIdx.x * kT;
  uint32_t *p = a + (size_t)b * H * W;
  for (int j = threadIdx.y; j < kT; j += blockDim.y) {
    const int y = sy + j, x = x0 + threadIdx.x;
    tile[j][threadIdx.x] = (y < H && x < W) ? p[(size_t)y * W + x] : 0u;
  }
  __syncthreads();
  if (threadIdx.y == 0) {  // one thread per column of the tile
    const int x = x0 + threadIdx.x;
    if (x < W) {
      uint32_t run = sy > 0 ? p[(size_t)(sy - 1) * W + x] : 0u;
      for (int i = 0; i < kT; ++i) {
        run += tile[i][threadIdx.x];
        tile[i][threadIdx.x] = run;
      }
    }
  }
  __syncthreads();
  for (int j = threadIdx.y; j < kT; j += blockDim.y) {
    const int y = sy + j, x = x0 + threadIdx.x;
    if (y < H && x < W) p[(size_t)y * W + x] = tile[j][threadIdx.x];
  }
}

// WF-TiS: the tiles (ty, tx) with ty + tx == diag, all bins, in one launch.
// The tile's 2-D inclusive scan in shared memory, plus the final values of
// the column to its left and the row above (Eq. 6's wavefront order makes
// both final), minus their shared corner.
__global__ void wf_diag_kernel(uint32_t *__restrict__ a, int H, int W, int ntx, int nty, int diag) {
  __shared__ uint32_t tile[kT][kT + 1];
  __shared__ uint32_t s_left[kT], s_top[kT];
  const int b = blockIdx.z;
  const int tx_lo = max(0, diag - (nty - 1));
  const int tx = tx_lo + blockIdx.x, ty = diag - tx;
  if (tx >= ntx || ty < 0) return;
  const int x0 = tx * kT, y0 = ty * kT;
  uint32_t *p = a + (size_t)b * H * W;
  for (int j = threadIdx.y; j < kT; j += blockDim.y) {
    const int y = y0 + j, x = x0 + threadIdx.x;
    tile[j][threadIdx.x] = (y < H && x < W) ? p[(size_t)y * W + x] : 0u;
  }
  if (threadIdx.y == 0) {
    const int y = y0 + threadIdx.x, x = x0 + threadIdx.x;
    s_left[threadIdx.x] = (x0 > 0 && y < H) ? p[(size_t)y * W + x0 - 1] : 0u;
    s_top[threadIdx.x] = (y0 > 0 && x < W) ? p[(size_t)(y0 - 1) * W + x] : 0u;
  }
  __syncthreads();
  const uint32_t corner = (x0 > 0 && y0 > 0) ? p[(size_t)(y0 - 1) * W + x0 - 1] : 0u;
  if (threadIdx.y == 0) {  // row scans
    uint32_t run = 0u;
    for (int i = 0; i < kT; ++i) {
      run += tile[threadIdx.x][i];
      tile[threadIdx.x][i] = run;
    }
  }
  __syncthreads();
  if (threadIdx.y == 0) {  // column scans
    uint32_t run = 0u;
    for (int i = 0; i < kT; ++i) {
      run += tile[i][threadIdx.x];
      tile[i][threadIdx.x] = run;
    }
  }
  __syncthreads();
  for (int j = threadIdx.y; j < kT; j += blockDim.y) {
    const int y = y0 + j, x = x0 + threadIdx.x;
    if (y < H && x < W) p[(size_t)y * W + x] = tile[j][threadIdx.x] + s_left[j] + s_top[threadIdx.x] - corner;
  }
}

int launch_ok() { return cudaGetLastError() == cudaSuccess ? IHIST_OK : IHIST_ERR_CUDA; }

}  // namespace

extern "C" size_t ihist_mapping_workspace_bytes(int mapping, int h, int w, int nbins) {
  if (h < 1 || w < 1 || nbins < 1) return 0;
  // CW-STS keeps a transposed copy of the tensor; the tiled mappings work in place
  return mapping == IHIST_MAPPING_CW_STS ? (size_t)h * w * nbins * sizeof(uint32_t) : 0;
}

extern "C" int ihist_mapping_compute(int mapping, int h, int w, int nbins, const uint8_t *d_in, size_t in_pitch,
                                     uint32_t *d_out, void *d_work, void *stream) {
  if (h < 1 || w < 1 || h > 65535 || w > 65535 || nbins < 1 || nbins > 256 || !d_in || !d_out ||
      in_pitch < (size_t)w)
    return IHIST_ERR_INVALID_ARG;
  if ((unsigned long long)h * w >= (1ull << 32)) return IHIST_ERR_INVALID_ARG;
  if (mapping != IHIST_MAPPING_CW_STS && mapping != IHIST_MAPPING_CW_TIS && mapping != IHIST_MAPPING_WF_TIS)
    return IHIST_ERR_INVALID_ARG;
  if (mapping == IHIST_MAPPING_CW_STS && !d_work) return IHIST_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const long long total = (long long)h * w * nbins;
  const unsigned int g1 = (unsigned int)std::min<long long>((total + 255) / 256, 152ll * 32);
  onehot_kernel<<<g1, 256, 0, s>>>(d_in, (long long)in_pitch, h, w, nbins, d_out);
  int rc = launch_ok();
  if (rc != IHIST_OK) return rc;
  const int ntx = (w + kT - 1) / kT, nty = (h + kT - 1) / kT;
  const dim3 blk(kT, 8);
  if (mapping == IHIST_MAPPING_CW_STS) {
    uint32_t *t = static_cast<uint32_t *>(d_work);
    const long long rows_h = (long long)nbins * h, rows_w = (long long)nbins * w;
    row_scan_kernel<<<(unsigned int)std::min<long long>(rows_h, 65535ll * 8), 256, 0, s>>>(d_out, rows_h, w);
    transpose_kernel<<<dim3(ntx, nty, nbins), blk, 0, s>>>(d_out, t, h, w);
    row_scan_kernel<<<(unsigned int)std::min<long long>(rows_w, 65535ll * 8), 256, 0, s>>>(t, rows_w, h);
    transpose_kernel<<<dim3(nty, ntx, nbins), blk, 0, s>>>(t, d_out, w, h);
    return launch_ok();
  }
  if (mapping == IHIST_MAPPING_CW_TIS) {
    for (int sx = 0; sx < w; sx += kT) tis_hstrip_kernel<<<dim3(1, nty, nbins), blk, 0, s>>>(d_out, h, w, sx);
    for (int sy = 0; sy < h; sy += kT) tis_vstrip_kernel<<<dim3(ntx, 1, nbins), blk, 0, s>>>(d_out, h, w, sy);
    return launch_ok();
  }
  for (int d = 0; d < ntx + nty - 1; ++d) {
    const int tx_lo = std::max(0, d - (nty - 1)), tx_hi = std::min(ntx - 1, d);
    wf_diag_kernel<<<dim3(tx_hi - tx_lo + 1, 1, nbins), blk, 0, s>>>(d_out, h, w, ntx, nty, d);
  }
  return launch_ok();
}

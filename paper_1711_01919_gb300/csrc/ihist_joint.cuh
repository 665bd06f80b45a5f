// ihist_joint.cuh -- joint bins of multi-channel frames: the
// higher-dimensional (e.g. colour) histograms that arXiv 1711.01919 names as
// uses of the integral histogram (Sec. 1, Sec. 2.1).
//
// A pixel p = (v_0 .. v_{C-1}) of a frame with C interleaved channels has
// the joint bin k = sum_c q_c * s_c, where q_c = floor(v_c * B_c / 256) is
// its bin among channel c's B_c uniform bins and s_{C-1} = 1,
// s_c = s_{c+1} * B_{c+1} (channel 0 is the most significant digit), for
// B = prod B_c <= 256 joint bins.  This pass writes k as one byte per pixel;
// the scan kernel then reads that plane with the identity binning (q = v)
// and builds the B planes of Eq. 1 exactly as for a one-channel frame.
#pragma once

#include <cstdint>

namespace ihist {

struct JointBins {
  int C;
  int mul[4];     // B_c
  int stride[4];  // s_c
};

// One thread per 4 consecutive pixels of a row (grid-stride).  idx rows are
// idx_pitch bytes, a multiple of 16 at least W rounded up to 4, so the
// 4-byte store of the last quad of a row stays inside the row.
__global__ void __launch_bounds__(256) joint_index_kernel(const uint8_t *__restrict__ in, long long pitch,
                                                          int H, int W, JointBins jb,
                                                          uint8_t *__restrict__ idx,
                                                          long long idx_pitch) {
  const unsigned int quads = ((unsigned)W + 3u) >> 2;
  const unsigned long long total = (unsigned long long)H * quads;
  for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const int y = (int)(t / quads);
    const int x0 = (int)(t - (unsigned long long)y * quads) * 4;
    const uint8_t *row = in + (long long)y * pitch;
    uint32_t packed = 0u;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int x = x0 + i;
      if (x < W) {
        uint32_t k = 0u;
        for (int c = 0; c < jb.C; ++c)
          k += (((uint32_t)__ldg(row + (long long)x * jb.C + c) * (uint32_t)jb.mul[c]) >> 8) *
               (uint32_t)jb.stride[c];
        packed |= k << (8 * i);
      }
    }
    *reinterpret_cast<uint32_t *>(idx + (long long)y * idx_pitch + x0) = packed;
  }
}

}  // namespace ihist

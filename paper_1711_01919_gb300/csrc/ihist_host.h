// ihist_host.h -- host-side helpers shared by the plan (ihist_api.cu) and
// batch (ihist_batch_api.cu) halves of libihist.so; not part of the C ABI.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "ihist.h"
#include "ihist_device.cuh"

namespace ihist {
namespace host {

constexpr unsigned int kDefaultTimeoutUs = 2000000u;

inline int mmax_for(int m) { return m <= 1 ? 1 : m <= 2 ? 2 : m <= 4 ? 4 : 8; }

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link-time dependency on libcuda); nullptr if unavailable.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// Shape limits shared by plans and batch frames (ihist_plan's doc).
int validate_shape(int h, int w, int nbins, int layout);

// Eq. 2 launch shared by plans and batches.
int launch_query(int H, int W, int B, int layout, int sms, Ctrl *ctrl, const uint32_t *d_hist,
                 const int32_t *d_rects, int n, uint32_t *d_hist_out, void *stream);

// Joint bins of C interleaved channels (ihist_plan_joint's rules):
// IHIST_OK and the joint bin count in *nbins, or the error code.
int joint_bin_count(int channels, const int *bins_per_channel, int *nbins);

// The joint-bin plane of one multi-channel frame (one byte per pixel,
// rows idx_pitch bytes, a multiple of 16) on `stream`.
int launch_joint_index(const uint8_t *in, long long pitch, int H, int W, int channels,
                       const int *bins_per_channel, uint8_t *idx, long long idx_pitch, int sms,
                       void *stream);

// Synchronise `stream`, read and clear the device status word.
int read_status(Ctrl *ctrl, void *stream, int *device_status);

}  // namespace host
}  // namespace ihist

// ihist_noalloc.cu -- integral histogram of one frame without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Who needs it: code that runs where allocating device memory is not
// allowed or not safe -- inside a host callback or another library's
// allocator hook, under a memory pool that must not grow, or in a process
// whose allocations are owned by a framework the caller cannot reach.  The
// regular path (ihist_plan + ihist_compute) allocates the carry workspace at
// plan time; this entry point instead uses a fixed scratch array that lives
// in the library image itself.
//
// The scratch below is a file-scope device array of kScratchBytes (8 MiB).
// Every GPU that loads libihist.so holds it until the process exits.  All
// calls share it and it keeps the previous call's contents, so the parts
// that must start at zero (the control block and the carry flags) are
// cleared on the caller's stream at the start of every call.  Two calls
// whose work may overlap on the GPU (different streams, or different host
// threads on one device) race on the scratch and give wrong results; issue
// them on one stream, one after the other.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "ihist.h"
#include "ihist_host.h"
#include "ihist_kernels.h"

using namespace ihist;
using namespace ihist::host;

namespace {

constexpr size_t kScratchBytes = 8u << 20;  // 8 MiB per device
constexpr int kMaxDevices = 64;
constexpr int kG = 4;                        // bins per CTA on this path
constexpr unsigned int kTimeoutUs = 2000000u;

// The scratch: control block, carry flags, column-count aggregates, left
// counts and inclusive rows of one frame (see ihist_scan.cuh).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceSetup {
  bool ready;
  unsigned char *scratch;  // device address of g_scratch on that device
  int sms;
  size_t dyn_smem_max;     // dynamic shared memory the kernels may use
};

DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Once per device, with that device current: the device address of the
// scratch array (the host-side name of a __device__ array is not a device
// address) and the shared-memory limits of the kernels this path launches.
int setup_device(int dev, DeviceSetup **out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup &s = g_setup[dev];
  if (!s.ready) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return IHIST_ERR_CUDA;
    }
    int sms = 0, optin = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return IHIST_ERR_CUDA;
    size_t dyn = (size_t)optin;
    for (int m = 1; m <= 8; m <<= 1)
      for (int tma = 0; tma < 2; ++tma)
        for (int vec = 0; vec < 2; ++vec) {
          ScanFn fn = scan_fn(kG, m, tma != 0, vec != 0);
          cudaFuncAttributes a;
          if (!fn || cudaFuncGetAttributes(&a, fn) != cudaSuccess) {
            cudaGetLastError();
            return IHIST_ERR_CUDA;
          }
          const size_t d = (size_t)optin > a.sharedSizeBytes ? (size_t)optin - a.sharedSizeBytes : 0;
          if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d) != cudaSuccess) {
            cudaGetLastError();
            return IHIST_ERR_CUDA;
          }
          dyn = std::min(dyn, d);
        }
    s.scratch = static_cast<unsigned char *>(ptr);
    s.sms = sms;
    s.dyn_smem_max = dyn;
    s.ready = true;
  }
  *out = &s;
  return IHIST_OK;
}

// Scratch bytes for nci (band, bin group, chunk) carry slots.
size_t scratch_bytes(size_t nci, size_t *o_flags, size_t *o_cnt, size_t *o_left, size_t *o_incl) {
  size_t off = align_up(sizeof(Ctrl), 256);
  *o_flags = off;
  off = align_up(off + nci * 4, 256);
  *o_cnt = off;
  off = align_up(off + nci * kChunk * (kG / 4) * 4, 256);
  *o_left = off;
  off = align_up(off + nci * kG * 4, 256);
  *o_incl = off;
  off = align_up(off + nci * kG * kChunk * 4, 256);
  return off;
}

}  // namespace

extern "C" int ihist_compute_noalloc(int h, int w, int nbins, int layout, const uint8_t *d_in,
                                     size_t in_pitch, uint32_t *d_out, void *stream,
                                     int *device_status) {
  if (h < 1 || w < 1 || h > 65535 || w > 65535 || nbins < 1 || nbins > 256) return IHIST_ERR_INVALID_ARG;
  if ((unsigned long long)h * (unsigned long long)w >= (1ull << 32)) return IHIST_ERR_INVALID_ARG;
  if (layout != IHIST_BIN_MAJOR && layout != IHIST_PIXEL_MAJOR && layout != IHIST_QUAD_MAJOR)
    return IHIST_ERR_INVALID_ARG;
  if (layout == IHIST_QUAD_MAJOR && nbins % 4 != 0) return IHIST_ERR_INVALID_ARG;
  if (!d_in || !d_out || in_pitch < (size_t)w || in_pitch > (size_t)LLONG_MAX) return IHIST_ERR_INVALID_ARG;
  if (((uintptr_t)d_out & 3u) != 0) return IHIST_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IHIST_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return IHIST_ERR_UNSUPPORTED;
  DeviceSetup *ds = nullptr;
  int rc = setup_device(dev, &ds);
  if (rc != IHIST_OK) return rc;

  // tiling: 4 bins per CTA, one CTA per band spanning the width; rows per
  // band start near two work items per SM and grow until the carries fit
  // the scratch.  A frame whose carries cannot fit is rejected.
  const int nchunks = (w + kChunk - 1) / kChunk;
  const int m = nchunks <= 16 ? 1 : nchunks <= 32 ? 2 : nchunks <= 64 ? 4 : 8;
  const int NW = (nchunks + m - 1) / m;
  if (NW > 16) return IHIST_ERR_UNSUPPORTED;
  const int ngroups = (nbins + kG - 1) / kG;
  int R = (int)std::max(8LL, std::min(64LL, (long long)h * ngroups / (2LL * ds->sms)));
  R = std::min(R, h);
  size_t o_flags = 0, o_cnt = 0, o_left = 0, o_incl = 0, need = 0, nci = 0;
  for (;; ++R) {
    const int nbands = (h + R - 1) / R;
    nci = (size_t)nbands * ngroups * nchunks;
    need = scratch_bytes(nci, &o_flags, &o_cnt, &o_left, &o_incl);
    if (need <= kScratchBytes) break;
    if (R >= std::min(h, 255)) return IHIST_ERR_UNSUPPORTED;  // frame too large for the fixed scratch
  }
  const size_t smem = smem_layout(NW, R, kG, nchunks).bytes;
  if (smem > ds->dyn_smem_max) return IHIST_ERR_UNSUPPORTED;

  FrameDesc f;
  std::memset(&f, 0, sizeof(f));
  f.in = d_in;
  f.pitch = (long long)in_pitch;
  f.out = d_out;
  f.H = h;
  f.W = w;
  f.B = nbins;
  f.qmul = nbins;
  f.layout = layout;
  f.R = R;
  f.nbands = (h + R - 1) / R;
  f.ngroups = ngroups;
  f.nchunks = nchunks;
  f.m = m;
  f.wpg = NW;
  f.gpc = 1;
  f.ngsets = ngroups;
  f.fault_skip_band = -1;
  f.nitems = (unsigned int)f.nbands * (unsigned int)ngroups;
  unsigned char *base = ds->scratch;
  Ctrl *ctrl = reinterpret_cast<Ctrl *>(base);
  f.flags = reinterpret_cast<uint32_t *>(base + o_flags);
  f.agg_cnt = reinterpret_cast<uint32_t *>(base + o_cnt);
  f.agg_left = reinterpret_cast<uint32_t *>(base + o_left);
  f.incl = reinterpret_cast<uint32_t *>(base + o_incl);

  const bool vec = (w % 4 == 0) && ((uintptr_t)d_out % 16 == 0);
  bool tma = !((uintptr_t)d_in & 15u) && !(in_pitch & 15u) && w >= kChunk && in_pitch < (1ull << 40);
  CUtensorMap tmap;
  std::memset(&tmap, 0, sizeof(tmap));
  if (tma) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    cuuint64_t gdim[2] = {(cuuint64_t)w, (cuuint64_t)h};
    cuuint64_t gstride[1] = {(cuuint64_t)in_pitch};
    cuuint32_t box[2] = {(cuuint32_t)kChunk, (cuuint32_t)R};
    cuuint32_t estride[2] = {1u, 1u};
    tma = enc && enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(d_in), gdim, gstride,
                     box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  ScanFn fn = scan_fn(kG, mmax_for(m), tma, vec);
  int occ = 0;
  if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, NW * 32, smem) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    return IHIST_ERR_UNSUPPORTED;
  }

  cudaStream_t s = (cudaStream_t)stream;
  // the scratch keeps the last call's contents: clear the control block
  // (ticket, done count, epoch, status) and this frame's carry flags
  if (cudaMemsetAsync(base, 0, o_cnt, s) != cudaSuccess) return IHIST_ERR_CUDA;
  const unsigned int grid = std::min<unsigned int>(f.nitems, (unsigned int)(occ * ds->sms));
  fn<<<grid, NW * 32, smem, s>>>(f, tmap, ctrl, (unsigned long long)kTimeoutUs * 1000ull);
  if (cudaGetLastError() != cudaSuccess) return IHIST_ERR_CUDA;
  if (device_status) {
    int v = 0;
    if (cudaStreamSynchronize(s) != cudaSuccess ||
        cudaMemcpy(&v, &ctrl->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return IHIST_ERR_CUDA;
    *device_status = v;
  }
  return IHIST_OK;
}

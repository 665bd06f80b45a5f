// ihist_api.cu -- host side of libihist.so: argument validation, plan and
// workspace management, kernel selection and launches.  Declared in
// include/ihist.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <new>

#include "../../include/ihist.h"
#include "ihist_query.cuh"
#include "ihist_scan.cuh"

using namespace ihist;

namespace {

using ScanFn = void (*)(FrameDesc, Ctrl *, unsigned long long);

template <int G, int MMAX>
ScanFn pick_vec(bool vec) {
  return vec ? scan_kernel<G, MMAX, true> : scan_kernel<G, MMAX, false>;
}

template <int G>
ScanFn pick_m(int mmax, bool vec) {
  switch (mmax) {
    case 1: return pick_vec<G, 1>(vec);
    case 2: return pick_vec<G, 2>(vec);
    case 4: return pick_vec<G, 4>(vec);
    default: return pick_vec<G, 8>(vec);
  }
}

// G = 16 keeps 64 accumulators per lane; it is built for up to 2 chunks per warp only.
ScanFn pick_scan(int G, int mmax, bool vec) {
  switch (G) {
    case 4: return pick_m<4>(mmax, vec);
    case 8: return pick_m<8>(mmax, vec);
    default:
      if (mmax == 1) return pick_vec<16, 1>(vec);
      if (mmax == 2) return pick_vec<16, 2>(vec);
      return nullptr;
  }
}

int mmax_for(int m) { return m <= 1 ? 1 : m <= 2 ? 2 : m <= 4 ? 4 : 8; }

constexpr unsigned int kDefaultTimeoutUs = 2000000u;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct ihist_plan_s {
  int device;
  int sms;
  int H, W, B, layout;
  int R, G, m, NW, nbands, ngroups, nchunks;
  unsigned int nitems;
  int ctas_per_sm;
  unsigned int timeout_us;
  int fault_skip_band;
  size_t smem_bytes;
  void *ws;
  size_t ws_bytes;
  Ctrl *ctrl;
  uint32_t *flags, *agg_cnt, *agg_left, *incl;
  cudaEvent_t ev_uploaded[2];  // sequence pipeline: slot filled
  cudaEvent_t ev_consumed[2];  // sequence pipeline: slot read by its compute
};

extern "C" size_t ihist_output_bytes(int h, int w, int nbins) {
  if (h <= 0 || w <= 0 || nbins <= 0) return 0;
  return (size_t)h * (size_t)w * (size_t)nbins * sizeof(uint32_t);
}

extern "C" const char *ihist_error_string(int code) {
  switch (code) {
    case IHIST_OK: return "ok";
    case IHIST_ERR_INVALID_ARG: return "invalid argument";
    case IHIST_ERR_UNSUPPORTED: return "unsupported request";
    case IHIST_ERR_OOM: return "device workspace allocation failed";
    case IHIST_ERR_CUDA: return "CUDA runtime error";
    case IHIST_ERR_LOOKBACK_TIMEOUT: return "carry look-back wait timed out; result invalid";
    case IHIST_ERR_BAD_RECT: return "query rectangle out of range; its histogram is zero";
    default: return "unknown status";
  }
}

static int validate_shape(int h, int w, int nbins, int layout) {
  if (h < 1 || w < 1 || h > 65535 || w > 65535) return IHIST_ERR_INVALID_ARG;
  if ((unsigned long long)h * (unsigned long long)w >= (1ull << 32)) return IHIST_ERR_INVALID_ARG;
  if (nbins < 1 || nbins > 256) return IHIST_ERR_INVALID_ARG;
  if (layout != IHIST_BIN_MAJOR && layout != IHIST_PIXEL_MAJOR) return IHIST_ERR_INVALID_ARG;
  if (w > 16384) return IHIST_ERR_UNSUPPORTED;
  return IHIST_OK;
}

// Default tiling: G = 8 bins per CTA (4 for B < 8); m so that the CTA has at
// most 16 warps for w <= 8192; R so that bands x groups gives about two work
// items per SM.
static void default_tune(int h, int w, int nbins, int sms, ihist_tune_t *t) {
  const int nchunks = (w + kChunk - 1) / kChunk;
  if (t->bins_per_cta == 0) t->bins_per_cta = nbins >= 8 ? 8 : 4;
  if (t->chunks_per_warp == 0)
    t->chunks_per_warp = nchunks <= 16 ? 1 : nchunks <= 32 ? 2 : nchunks <= 64 ? 4 : 8;
  if (t->rows_per_band == 0) {
    const int ngroups = (nbins + t->bins_per_cta - 1) / t->bins_per_cta;
    long long r = (long long)h * ngroups / (2LL * sms);
    r = std::max(8LL, std::min(128LL, r));
    t->rows_per_band = (int)std::min<long long>(r, h);
  }
  if (t->timeout_us == 0) t->timeout_us = kDefaultTimeoutUs;
}

extern "C" int ihist_plan_tuned(int h, int w, int nbins, int layout, const ihist_tune_t *tune,
                                ihist_plan_t *out) {
  if (!out) return IHIST_ERR_INVALID_ARG;
  int rc = validate_shape(h, w, nbins, layout);
  if (rc != IHIST_OK) return rc;
  ihist_tune_t t;
  std::memset(&t, 0, sizeof(t));
  t.fault_skip_band = -1;
  if (tune) t = *tune;
  if (t.rows_per_band < 0 || t.rows_per_band > 255) return IHIST_ERR_INVALID_ARG;
  if (t.bins_per_cta != 0 && t.bins_per_cta != 4 && t.bins_per_cta != 8 && t.bins_per_cta != 16)
    return IHIST_ERR_INVALID_ARG;
  if (t.chunks_per_warp != 0 && t.chunks_per_warp != 1 && t.chunks_per_warp != 2 &&
      t.chunks_per_warp != 4 && t.chunks_per_warp != 8)
    return IHIST_ERR_INVALID_ARG;
  if (t.ctas_per_sm < 0 || t.ctas_per_sm > 32) return IHIST_ERR_INVALID_ARG;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IHIST_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return IHIST_ERR_CUDA;
  default_tune(h, w, nbins, sms, &t);

  ihist_plan_s *p = new (std::nothrow) ihist_plan_s;
  if (!p) return IHIST_ERR_OOM;
  std::memset(p, 0, sizeof(*p));
  p->device = dev;
  p->sms = sms;
  p->H = h;
  p->W = w;
  p->B = nbins;
  p->layout = layout;
  p->G = t.bins_per_cta;
  p->m = t.chunks_per_warp;
  p->R = std::min(t.rows_per_band, h);
  p->nchunks = (w + kChunk - 1) / kChunk;
  p->NW = (p->nchunks + p->m - 1) / p->m;
  if (p->NW > 16 || !pick_scan(p->G, mmax_for(p->m), true)) {
    delete p;
    return IHIST_ERR_UNSUPPORTED;
  }
  p->nbands = (h + p->R - 1) / p->R;
  p->ngroups = (nbins + p->G - 1) / p->G;
  p->nitems = (unsigned int)p->nbands * (unsigned int)p->ngroups;
  p->timeout_us = t.timeout_us;
  p->fault_skip_band = t.fault_skip_band;
  p->smem_bytes = ((size_t)p->NW * p->R * p->G + (size_t)p->nchunks * p->G) * sizeof(uint32_t);

  ScanFn fn = pick_scan(p->G, mmax_for(p->m), true);
  ScanFn fn2 = pick_scan(p->G, mmax_for(p->m), false);
  if (p->smem_bytes > 48 * 1024) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem_bytes) !=
            cudaSuccess ||
        cudaFuncSetAttribute(fn2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)p->smem_bytes) != cudaSuccess) {
      cudaGetLastError();
      delete p;
      return IHIST_ERR_UNSUPPORTED;
    }
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, p->NW * 32, p->smem_bytes) !=
          cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    delete p;
    return IHIST_ERR_UNSUPPORTED;
  }
  p->ctas_per_sm = t.ctas_per_sm > 0 ? std::min(t.ctas_per_sm, occ) : occ;

  // workspace: control block, flags, column-count aggregates, left counts, inclusive rows
  const size_t nci = (size_t)p->nitems * p->nchunks;
  size_t off = 0;
  const size_t o_ctrl = off;
  off = align_up(off + sizeof(Ctrl), 256);
  const size_t o_flags = off;
  off = align_up(off + nci * sizeof(uint32_t), 256);
  const size_t o_cnt = off;
  off = align_up(off + nci * kChunk * (p->G / 4) * sizeof(uint32_t), 256);
  const size_t o_left = off;
  off = align_up(off + nci * p->G * sizeof(uint32_t), 256);
  const size_t o_incl = off;
  off = align_up(off + nci * p->G * kChunk * sizeof(uint32_t), 256);
  p->ws_bytes = off;
  if (cudaMalloc(&p->ws, p->ws_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return IHIST_ERR_OOM;
  }
  char *base = static_cast<char *>(p->ws);
  p->ctrl = reinterpret_cast<Ctrl *>(base + o_ctrl);
  p->flags = reinterpret_cast<uint32_t *>(base + o_flags);
  p->agg_cnt = reinterpret_cast<uint32_t *>(base + o_cnt);
  p->agg_left = reinterpret_cast<uint32_t *>(base + o_left);
  p->incl = reinterpret_cast<uint32_t *>(base + o_incl);
  if (cudaMemset(p->ws, 0, o_cnt) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p->ws);
    delete p;
    return IHIST_ERR_CUDA;
  }
  for (int i = 0; i < 2; ++i) {
    if (cudaEventCreateWithFlags(&p->ev_uploaded[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_consumed[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      for (int j = 0; j <= i; ++j) {
        if (p->ev_uploaded[j]) cudaEventDestroy(p->ev_uploaded[j]);
        if (p->ev_consumed[j]) cudaEventDestroy(p->ev_consumed[j]);
      }
      cudaFree(p->ws);
      delete p;
      return IHIST_ERR_CUDA;
    }
  }
  *out = p;
  return IHIST_OK;
}

extern "C" int ihist_plan(int h, int w, int nbins, int layout, ihist_plan_t *out) {
  return ihist_plan_tuned(h, w, nbins, layout, nullptr, out);
}

extern "C" int ihist_plan_get_tune(ihist_plan_t p, ihist_tune_t *out) {
  if (!p || !out) return IHIST_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->rows_per_band = p->R;
  out->bins_per_cta = p->G;
  out->chunks_per_warp = p->m;
  out->ctas_per_sm = p->ctas_per_sm;
  out->timeout_us = p->timeout_us;
  out->fault_skip_band = p->fault_skip_band;
  return IHIST_OK;
}

extern "C" size_t ihist_workspace_bytes(ihist_plan_t p) { return p ? p->ws_bytes : 0; }

static int check_device(const ihist_plan_s *p) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return IHIST_ERR_CUDA;
  return dev == p->device ? IHIST_OK : IHIST_ERR_INVALID_ARG;
}

extern "C" int ihist_compute(ihist_plan_t p, const uint8_t *d_in, size_t in_pitch, uint32_t *d_out,
                             void *stream) {
  if (!p || !d_in || !d_out) return IHIST_ERR_INVALID_ARG;
  if (in_pitch < (size_t)p->W || in_pitch > (size_t)LLONG_MAX) return IHIST_ERR_INVALID_ARG;
  if (((uintptr_t)d_out & 3u) != 0) return IHIST_ERR_INVALID_ARG;
  int rc = check_device(p);
  if (rc != IHIST_OK) return rc;
  const bool vec = ((uintptr_t)d_in % 4 == 0) && (in_pitch % 4 == 0) && (p->W % 4 == 0) &&
                   ((uintptr_t)d_out % 16 == 0);
  FrameDesc f;
  std::memset(&f, 0, sizeof(f));
  f.in = d_in;
  f.pitch = (long long)in_pitch;
  f.out = d_out;
  f.H = p->H;
  f.W = p->W;
  f.B = p->B;
  f.layout = p->layout;
  f.R = p->R;
  f.nbands = p->nbands;
  f.ngroups = p->ngroups;
  f.nchunks = p->nchunks;
  f.m = p->m;
  f.fault_skip_band = p->fault_skip_band;
  f.nitems = p->nitems;
  f.agg_cnt = p->agg_cnt;
  f.agg_left = p->agg_left;
  f.incl = p->incl;
  f.flags = p->flags;
  const unsigned int grid =
      std::min<unsigned int>(p->nitems, (unsigned int)(p->ctas_per_sm * p->sms));
  ScanFn fn = pick_scan(p->G, mmax_for(p->m), vec);
  const unsigned long long timeout_ns = (unsigned long long)p->timeout_us * 1000ull;
  fn<<<grid, p->NW * 32, p->smem_bytes, (cudaStream_t)stream>>>(f, p->ctrl, timeout_ns);
  if (cudaGetLastError() != cudaSuccess) return IHIST_ERR_CUDA;
  return IHIST_OK;
}

extern "C" int ihist_query(ihist_plan_t p, const uint32_t *d_hist, const int32_t *d_rects, int n,
                           uint32_t *d_hist_out, void *stream) {
  if (!p || n < 0) return IHIST_ERR_INVALID_ARG;
  if (n == 0) return IHIST_OK;
  if (!d_hist || !d_rects || !d_hist_out) return IHIST_ERR_INVALID_ARG;
  if (((uintptr_t)d_hist & 3u) || ((uintptr_t)d_rects & 3u) || ((uintptr_t)d_hist_out & 3u))
    return IHIST_ERR_INVALID_ARG;
  if ((unsigned long long)n * (unsigned long long)p->B > 0x7fffffffull) return IHIST_ERR_UNSUPPORTED;
  int rc = check_device(p);
  if (rc != IHIST_OK) return rc;
  const unsigned int total = (unsigned int)n * (unsigned int)p->B;
  const unsigned int threads = 256;
  const unsigned int grid =
      std::min<unsigned int>((total + threads - 1) / threads, (unsigned int)p->sms * 16u);
  if (p->layout == IHIST_BIN_MAJOR)
    query_kernel<0><<<grid, threads, 0, (cudaStream_t)stream>>>(d_hist, p->H, p->W, p->B, d_rects,
                                                                total, d_hist_out, p->ctrl);
  else
    query_kernel<1><<<grid, threads, 0, (cudaStream_t)stream>>>(d_hist, p->H, p->W, p->B, d_rects,
                                                                total, d_hist_out, p->ctrl);
  if (cudaGetLastError() != cudaSuccess) return IHIST_ERR_CUDA;
  return IHIST_OK;
}

extern "C" int ihist_sequence_host(ihist_plan_t p, const uint8_t *h_frames, size_t frame_stride,
                                   int nframes, uint8_t *d_slots, uint32_t *d_outs, int nouts,
                                   const int32_t *d_rects, int nrects, uint32_t *d_query,
                                   uint32_t *h_query_out, void *stream, void *copy_stream) {
  if (!p || nframes < 0 || nouts < 1 || nrects < 0) return IHIST_ERR_INVALID_ARG;
  if (nframes == 0) return IHIST_OK;
  const size_t fbytes = (size_t)p->H * (size_t)p->W;
  if (!h_frames || !d_slots || !d_outs || frame_stride < fbytes) return IHIST_ERR_INVALID_ARG;
  if (nrects > 0 && (!d_rects || !d_query || !h_query_out)) return IHIST_ERR_INVALID_ARG;
  int rc = check_device(p);
  if (rc != IHIST_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream, cs = (cudaStream_t)copy_stream;
  const size_t obytes = ihist_output_bytes(p->H, p->W, p->B);
  const size_t qwords = (size_t)nrects * (size_t)p->B;
  for (int i = 0; i < nframes; ++i) {
    const int slot = i & 1;
    uint8_t *d_in = d_slots + (size_t)slot * fbytes;
    // the slot may be refilled only once the compute that read it (frame i-2) is done
    if (i >= 2 && cudaStreamWaitEvent(cs, p->ev_consumed[slot], 0) != cudaSuccess) return IHIST_ERR_CUDA;
    if (cudaMemcpyAsync(d_in, h_frames + (size_t)i * frame_stride, fbytes, cudaMemcpyHostToDevice,
                        cs) != cudaSuccess)
      return IHIST_ERR_CUDA;
    if (cudaEventRecord(p->ev_uploaded[slot], cs) != cudaSuccess) return IHIST_ERR_CUDA;
    if (cudaStreamWaitEvent(s, p->ev_uploaded[slot], 0) != cudaSuccess) return IHIST_ERR_CUDA;
    uint32_t *d_out = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(d_outs) +
                                                   (size_t)(i % nouts) * obytes);
    rc = ihist_compute(p, d_in, (size_t)p->W, d_out, stream);
    if (rc != IHIST_OK) return rc;
    if (cudaEventRecord(p->ev_consumed[slot], s) != cudaSuccess) return IHIST_ERR_CUDA;
    if (nrects > 0) {
      rc = ihist_query(p, d_out, d_rects, nrects, d_query, stream);
      if (rc != IHIST_OK) return rc;
      if (cudaMemcpyAsync(h_query_out + (size_t)i * qwords, d_query, qwords * sizeof(uint32_t),
                          cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return IHIST_ERR_CUDA;
    }
  }
  // later work on the copy stream must not overtake this sequence's computes
  if (cudaStreamWaitEvent(cs, p->ev_consumed[(nframes - 1) & 1], 0) != cudaSuccess) return IHIST_ERR_CUDA;
  return IHIST_OK;
}

extern "C" int ihist_status(ihist_plan_t p, void *stream, int *device_status) {
  if (!p || !device_status) return IHIST_ERR_INVALID_ARG;
  int rc = check_device(p);
  if (rc != IHIST_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  int v = 0;
  if (cudaStreamSynchronize(s) != cudaSuccess) return IHIST_ERR_CUDA;
  if (cudaMemcpy(&v, &p->ctrl->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return IHIST_ERR_CUDA;
  if (cudaMemset(&p->ctrl->status, 0, sizeof(int)) != cudaSuccess) return IHIST_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return IHIST_ERR_CUDA;
  *device_status = v;
  return IHIST_OK;
}

extern "C" void ihist_destroy(ihist_plan_t p) {
  if (!p) return;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != p->device) cudaSetDevice(p->device);
  for (int i = 0; i < 2; ++i) {
    if (p->ev_uploaded[i]) cudaEventDestroy(p->ev_uploaded[i]);
    if (p->ev_consumed[i]) cudaEventDestroy(p->ev_consumed[i]);
  }
  cudaFree(p->ws);
  if (prev != p->device && prev >= 0) cudaSetDevice(prev);
  delete p;
}

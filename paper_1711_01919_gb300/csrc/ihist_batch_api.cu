// ihist_batch_api.cu -- host side of libihist.so for batches: one persistent
// launch over many frames of uneven size (slot planning, rebinding, uploads,
// launches and queries).  Declared in include/ihist.h.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "ihist.h"
#include "ihist_host.h"
#include "ihist_kernels.h"
#include "ihist_query.cuh"

using namespace ihist;
using namespace ihist::host;

// ---------------------------------------------------------------- batches
//
// A batch plan owns `cap` frame slots.  Slot i's carry workspace is sized
// for the frame it was planned with; ihist_batch_set_io may later bind any
// n <= cap frames whose tilings fit their slots (same or smaller carries,
// rows per band and width), so one plan serves a stream of changing
// batches without allocating.  Every kernel variant (TMA / plain input,
// 16-byte / scalar output) is prepared at plan time and the launch picks
// the one the current frames allow.

namespace {

constexpr int kBatchWarps = 16;  // default warps per CTA of the batched kernel

// Tiling of one frame in a batched launch of `warps`-warp CTAs: m chunks
// per warp (at most max_m) and gpc bin groups per CTA, chunks per CTA group
// x gpc at most max_ncg (the per-CTA carry width the launch's shared memory
// was sized for), maximising the share of the CTA's warps x m chunk slots
// that hold columns, smaller m on ties.  A frame wider than warps x max_m
// chunks is split into width segments of equal chunk counts (one work item
// each, see the scan kernel); segments are used only when no tiling without
// them exists, or for the whole-record pixel-major tilings below.  Returns
// false if no tiling fits max_ncg.
bool batch_frame_tiling(int h, int w, int nbins, int layout, int G, int R_req, int max_m, int max_ncg,
                        int warps, FrameDesc *f) {
  const int nchunks = (w + kChunk - 1) / kChunk;
  const int ngroups = (nbins + G - 1) / G;
  double best = -1.0;
  int bm = 1, bwpg = nchunks, bgpc = 1, bsegs = 1;
  // Pixel-major frames of two to four bin groups whose records the scan
  // kernel can store whole (its record path): take a tiling with every
  // group in the CTA when one fits, width segments allowed (64 pixel-major
  // 1080p x 64 frames: 7.95 -> 7.85 ms).
  if (pm_staged(layout, G) && ngroups >= 2 && ngroups <= 4 && ngroups <= warps && pm_record_bins(nbins)) {
    const int per = warps / ngroups;  // warps of one group
    for (int m = 1; m <= max_m; m <<= 1) {
      const int wpg_all = (nchunks + m - 1) / m;
      const int nsegs = (wpg_all + per - 1) / per;
      const int wpg = (wpg_all + nsegs - 1) / nsegs;
      const int ncl = std::min(nchunks, wpg * m);
      if (ncl * ngroups > max_ncg) continue;
      const double util = (double)nchunks * ngroups / ((double)nsegs * warps * m);
      if (util > best + 1e-9) {
        best = util;
        bm = m;
        bwpg = wpg;
        bgpc = ngroups;
        bsegs = nsegs;
      }
    }
  }
  for (int pass = 0; pass < 2 && best < 0.0; ++pass) {
    for (int m = 1; m <= max_m; m <<= 1) {
      const int wpg_all = (nchunks + m - 1) / m;
      const int nsegs = pass == 0 ? 1 : (wpg_all + warps - 1) / warps;
      const int wpg = (wpg_all + nsegs - 1) / nsegs;
      if (wpg > warps) continue;
      const int ncl = std::min(nchunks, wpg * m);
      const int gpc = std::min(std::min(ngroups, warps / wpg), max_ncg / ncl);
      if (gpc < 1) continue;
      const double util = (double)nchunks * gpc / ((double)nsegs * warps * m);
      if (util > best + 1e-9) {
        best = util;
        bm = m;
        bwpg = wpg;
        bgpc = gpc;
        bsegs = nsegs;
      }
    }
  }
  std::memset(f, 0, sizeof(*f));
  f->H = h;
  f->W = w;
  f->B = nbins;
  f->qmul = nbins;
  f->layout = layout;
  f->R = std::min(R_req, h);
  f->nbands = (h + f->R - 1) / f->R;
  f->ngroups = ngroups;
  f->nchunks = nchunks;
  f->m = bm;
  f->wpg = bwpg;
  f->gpc = bgpc;
  f->nsegs = bsegs;
  f->cps = bsegs > 1 ? bwpg * bm : nchunks;
  f->ngsets = (ngroups + bgpc - 1) / bgpc;
  f->nitems = (unsigned int)f->nbands * (unsigned int)f->ngsets * (unsigned int)bsegs;
  f->fault_skip_band = -1;
  return best >= 0.0;
}

// Chunks of one CTA's bin group (the shared-memory carry width per group).
int frame_ncl(const FrameDesc &f) { return std::min(f.nchunks, f.cps); }

// Segment records of a segmented frame (0 otherwise) and their words.
size_t frame_nhs(const FrameDesc &f) { return f.nsegs > 1 ? (size_t)f.nbands * f.ngroups * f.nsegs : 0; }
size_t frame_hagg_words(const FrameDesc &f, int G) { return frame_nhs(f) * ((size_t)f.R * G + G); }

size_t frame_nci(const FrameDesc &f) { return (size_t)f.nbands * f.ngroups * f.nchunks; }

// Joint-bin frames (2..4 interleaved channels): the scan reads the frame's
// joint-bin plane, which the batch computes into its workspace (rows
// idx_pitch bytes) just before the scan.
bool frame_joint(const ihist_frame_t &fr) { return fr.channels >= 2; }
int frame_channels(const ihist_frame_t &fr) { return frame_joint(fr) ? fr.channels : 1; }
size_t idx_pitch_of(int w) { return align_up((size_t)w, 16); }
size_t idx_bytes_of(const ihist_frame_t &fr) {
  return frame_joint(fr) ? (size_t)fr.h * idx_pitch_of(fr.w) : 0;
}

// A joint frame's channels and bins follow ihist_plan_joint's rules, its
// bins multiply to nbins and it has no value -> bin table.
int joint_ok(const ihist_frame_t &fr) {
  if (fr.channels < 0 || fr.channels > 4) return IHIST_ERR_INVALID_ARG;
  if (!frame_joint(fr)) return IHIST_OK;
  int nb = 0;
  const int rc = joint_bin_count(fr.channels, fr.bins_per_channel, &nb);
  if (rc != IHIST_OK) return rc;
  if (nb != fr.nbins || fr.bin_of_value) return IHIST_ERR_INVALID_ARG;
  if ((long long)fr.w * fr.channels > 65535) return IHIST_ERR_UNSUPPORTED;
  return IHIST_OK;
}

bool frame_tma_ok(const ihist_frame_t &fr) {
  if (frame_joint(fr)) return fr.w >= kChunk;  // the plane is 16-byte aligned, pitch a multiple of 16
  return !((uintptr_t)fr.d_in & 15u) && !(fr.in_pitch & 15u) && fr.w >= kChunk &&
         fr.in_pitch < (1ull << 40);
}

bool frame_vec_ok(const ihist_frame_t &fr) {
  return fr.w % 4 == 0 && !((uintptr_t)fr.d_out & 15u);
}

// A frame's value -> bin table, if it has one, maps every value to a bin
// in [0, nbins) or to -1 (no bin).
bool table_ok(const ihist_frame_t &fr) {
  if (!fr.bin_of_value) return true;
  for (int v = 0; v < 256; ++v)
    if (fr.bin_of_value[v] < -1 || fr.bin_of_value[v] >= fr.nbins) return false;
  return true;
}

// The kernel's form of a frame's binning: 8 * bin of each value, or kNoBin;
// uniform frames of a table batch get the table of q = floor(v * B / 256),
// joint frames the identity on their joint-bin plane.
void fill_table(const ihist_frame_t &fr, uint32_t *dst) {
  for (int v = 0; v < 256; ++v) {
    if (fr.bin_of_value)
      dst[v] = fr.bin_of_value[v] >= 0 ? 8u * (uint32_t)fr.bin_of_value[v] : kNoBin;
    else if (frame_joint(fr))
      dst[v] = v < fr.nbins ? 8u * (uint32_t)v : kNoBin;
    else
      dst[v] = 8u * (((uint32_t)v * (uint32_t)fr.nbins) >> 8);
  }
}

}  // namespace

struct ihist_batch_s {
  int device, sms, cap, n, G, warps, mmax, R_req, R_max, ncg_max, ctas_cap, stage;
  int fault_skip_band;  // test hook, -1 off
  int ctas_per_sm[2][2];  // occupancy of each (tma, vec) variant
  bool tma, vec;          // variant the current frames allow
  bool lut;               // frames bin through per-slot value -> bin tables
  unsigned int timeout_us, total;
  size_t smem_bytes, ws_bytes;
  unsigned long long bins_total;
  void *ws;
  Ctrl *ctrl;
  FrameDesc *d_fd;   // descriptors in work-list order (the scan)
  FrameDesc *d_fdq;  // descriptors in the caller's frame order (the queries)
  CUtensorMap *d_tm;
  unsigned int *d_end, *d_bins_end;
  uint32_t *d_lut;                                    // table batches: [slot][256]
  std::vector<size_t> slot_nci;                       // carry capacity of each slot
  std::vector<size_t> slot_nhs, slot_hwords;          // width-segment records and their words per slot
  std::vector<uint32_t *> slot_flags, slot_cnt, slot_left, slot_incl, slot_hflags, slot_hagg;
  std::vector<size_t> slot_idx_cap;                   // joint-bin plane bytes of each slot
  std::vector<uint8_t *> slot_idx;
  std::vector<FrameDesc> fd;                          // current frames
  std::vector<ihist_frame_t> io;
  // Pinned staging of the descriptors, two sets used by alternate bindings:
  // a binding waits only for the copy made from its set two bindings ago,
  // so a caller can bind and launch ahead of the GPU.  h_* point at the set
  // of the binding being built; staged[i] marks set i's last copy done.
  struct Staging {
    FrameDesc *fd, *fdq;
    CUtensorMap *tm;
    unsigned int *end, *bins_end;
    uint32_t *lut;
  } stage_sets[2];
  cudaEvent_t staged[2];
  int stage_cur;
  FrameDesc *h_fd, *h_fdq;
  CUtensorMap *h_tm;
  unsigned int *h_end, *h_bins_end;
  uint32_t *h_lut;
  cudaEvent_t uploaded, computed;
  bool launched;
};

// TMA descriptor of the plane the scan reads (the frame, or its joint-bin plane).
static bool encode_frame_map(const uint8_t *in, size_t pitch, int h, int w, int R, CUtensorMap *map) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t gdim[2] = {(cuuint64_t)w, (cuuint64_t)h};
  cuuint64_t gstride[1] = {(cuuint64_t)pitch};
  cuuint32_t box[2] = {(cuuint32_t)kChunk, (cuuint32_t)R};
  cuuint32_t estride[2] = {1u, 1u};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(in), gdim, gstride,
             box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Point h_* at staging set i.
static void use_staging(ihist_batch_s *b, int i) {
  b->stage_cur = i;
  b->h_fd = b->stage_sets[i].fd;
  b->h_fdq = b->stage_sets[i].fdq;
  b->h_tm = b->stage_sets[i].tm;
  b->h_end = b->stage_sets[i].end;
  b->h_bins_end = b->stage_sets[i].bins_end;
  b->h_lut = b->stage_sets[i].lut;
}

// Tile the given frames into the plan's slots and fill the pinned staging
// copies (descriptors, tensor maps, item and bin prefix sums).  Nothing is
// committed to b->fd / b->io unless every frame fits.
static int batch_bind(ihist_batch_s *b, const ihist_frame_t *frames, int n) {
  if (n < 1 || n > b->cap) return IHIST_ERR_INVALID_ARG;
  std::vector<FrameDesc> fd(n);
  bool tma = true, vec = true;
  unsigned long long total = 0, bsum = 0;
  for (int i = 0; i < n; ++i) {
    const ihist_frame_t &fr = frames[i];
    int rc = validate_shape(fr.h, fr.w, fr.nbins, fr.layout);
    if (rc != IHIST_OK) return rc;
    rc = joint_ok(fr);
    if (rc != IHIST_OK) return rc;
    if (!fr.d_in || !fr.d_out || fr.in_pitch < (size_t)fr.w * frame_channels(fr) || ((uintptr_t)fr.d_out & 3u) ||
        fr.in_pitch > (size_t)LLONG_MAX || !table_ok(fr))
      return IHIST_ERR_INVALID_ARG;
    if (fr.bin_of_value && !b->lut) return IHIST_ERR_UNSUPPORTED;  // planned without tables
    if (idx_bytes_of(fr) > b->slot_idx_cap[i]) return IHIST_ERR_UNSUPPORTED;  // no joint-bin plane that large
    FrameDesc &f = fd[i];
    if (!batch_frame_tiling(fr.h, fr.w, fr.nbins, fr.layout, b->G, b->R_req, b->mmax, b->ncg_max, b->warps,
                            &f) ||
        frame_nci(f) > b->slot_nci[i] || f.R > b->R_max || frame_ncl(f) * f.gpc > b->ncg_max ||
        mmax_for(f.m) > b->mmax || frame_nhs(f) > b->slot_nhs[i] || frame_hagg_words(f, b->G) > b->slot_hwords[i])
      return IHIST_ERR_UNSUPPORTED;  // does not fit the slot planned for it
    f.in = frame_joint(fr) ? b->slot_idx[i] : fr.d_in;
    f.pitch = frame_joint(fr) ? (long long)idx_pitch_of(fr.w) : (long long)fr.in_pitch;
    if (frame_joint(fr)) f.qmul = 256;  // the plane holds bin indices
    f.out = fr.d_out;
    f.flags = b->slot_flags[i];
    f.agg_cnt = b->slot_cnt[i];
    f.agg_left = b->slot_left[i];
    f.incl = b->slot_incl[i];
    f.hflags = frame_nhs(f) ? b->slot_hflags[i] : nullptr;
    f.hagg = frame_nhs(f) ? b->slot_hagg[i] : nullptr;
    f.fault_skip_band = b->fault_skip_band;
    tma = tma && frame_tma_ok(fr);
    vec = vec && frame_vec_ok(fr);
    total += f.nitems;
    bsum += (unsigned long long)fr.nbins;
  }
  if (total >= 0xffffffffull) return IHIST_ERR_UNSUPPORTED;
  // Work-list order: largest outputs first, so the launch ends on small
  // frames (the 256-frame batch of 320x240 .. 1920x1080 frames with 16-64
  // bins: 5.235 -> 5.142 ms against the caller's order).  Each frame's descriptor carries its own slot's
  // carries, table and plane, so only the order of the items changes.
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    return ihist_output_bytes(frames[a].h, frames[a].w, frames[a].nbins) >
           ihist_output_bytes(frames[c].h, frames[c].w, frames[c].nbins);
  });
  unsigned long long brun = 0;
  for (int i = 0; i < n; ++i) {
    brun += (unsigned long long)frames[i].nbins;
    b->h_bins_end[i] = (unsigned int)brun;
    if (b->lut) {
      fill_table(frames[i], b->h_lut + (size_t)i * 256);
      fd[i].lut = b->d_lut + (size_t)i * 256;
    }
    b->h_fdq[i] = fd[i];
  }
  unsigned long long run = 0;
  for (int k = 0; k < n; ++k) {
    const int i = order[k];
    if (tma) {
      if (!encode_frame_map(fd[i].in, (size_t)fd[i].pitch, frames[i].h, frames[i].w, fd[i].R, &b->h_tm[k]))
        return IHIST_ERR_CUDA;
    } else {
      std::memset(&b->h_tm[k], 0, sizeof(CUtensorMap));
    }
    run += fd[i].nitems;
    b->h_end[k] = (unsigned int)run;
    b->h_fd[k] = fd[i];
  }
  b->fd.assign(fd.begin(), fd.end());
  b->io.assign(frames, frames + n);
  b->n = n;
  b->tma = tma;
  b->vec = vec;
  b->total = (unsigned int)total;
  b->bins_total = bsum;
  return IHIST_OK;
}

static int batch_upload(ihist_batch_s *b, cudaStream_t s) {
  const int n = b->n;
  if (cudaMemcpyAsync(b->d_fd, b->h_fd, (size_t)n * sizeof(FrameDesc), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(b->d_fdq, b->h_fdq, (size_t)n * sizeof(FrameDesc), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(b->d_tm, b->h_tm, (size_t)n * sizeof(CUtensorMap), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(b->d_end, b->h_end, (size_t)n * sizeof(unsigned int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(b->d_bins_end, b->h_bins_end, (size_t)n * sizeof(unsigned int), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      (b->lut && cudaMemcpyAsync(b->d_lut, b->h_lut, (size_t)n * 256 * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                 s) != cudaSuccess) ||
      cudaEventRecord(b->staged[b->stage_cur], s) != cudaSuccess)
    return IHIST_ERR_CUDA;
  return IHIST_OK;
}

extern "C" void ihist_batch_destroy(ihist_batch_t b) {
  if (!b) return;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  for (int i = 0; i < 2; ++i) {
    if (b->staged[i]) cudaEventSynchronize(b->staged[i]);
    if (b->staged[i]) cudaEventDestroy(b->staged[i]);
  }
  if (b->uploaded) cudaEventDestroy(b->uploaded);
  if (b->computed) cudaEventDestroy(b->computed);
  for (int i = 0; i < 2; ++i) {
    ihist_batch_s::Staging &st = b->stage_sets[i];
    if (st.fd) cudaFreeHost(st.fd);
    if (st.fdq) cudaFreeHost(st.fdq);
    if (st.tm) cudaFreeHost(st.tm);
    if (st.end) cudaFreeHost(st.end);
    if (st.bins_end) cudaFreeHost(st.bins_end);
    if (st.lut) cudaFreeHost(st.lut);
  }
  if (b->ws) cudaFree(b->ws);
  if (prev != b->device && prev >= 0) cudaSetDevice(prev);
  delete b;
}

extern "C" int ihist_batch_plan(const ihist_frame_t *frames, int n, const ihist_tune_t *tune,
                                ihist_batch_t *out) {
  if (!frames || n < 1 || !out) return IHIST_ERR_INVALID_ARG;
  ihist_tune_t t;
  std::memset(&t, 0, sizeof(t));
  if (tune) t = *tune;
  // frames with value -> bin tables make a table batch (every frame bins
  // through a table; 4 or 8 bins per CTA)
  bool lut = false;
  for (int i = 0; i < n; ++i) lut = lut || frames[i].bin_of_value != nullptr;
  if (t.bins_per_cta == 0) {
    // larger bin groups when any frame is pixel-major (longer contiguous
    // pieces per pixel record): 16 when every frame has at least 16 bins and
    // fits 16 warps x 2 chunks, else 8
    bool pm = false, wide16 = !lut;
    for (int i = 0; i < n; ++i) {
      pm = pm || frames[i].layout == IHIST_PIXEL_MAJOR;
      wide16 = wide16 && frames[i].nbins >= 16 && frames[i].w <= kBatchWarps * 2 * kChunk;
    }
    t.bins_per_cta = pm ? (wide16 ? 16 : 8) : 4;
  }
  if (t.bins_per_cta != 4 && t.bins_per_cta != 8 && t.bins_per_cta != 16) return IHIST_ERR_INVALID_ARG;
  if (lut && t.bins_per_cta == 16) return IHIST_ERR_UNSUPPORTED;
  if (t.rows_per_band < 0 || t.rows_per_band > 255) return IHIST_ERR_INVALID_ARG;
  if (t.ctas_per_sm < 0 || t.ctas_per_sm > 32) return IHIST_ERR_INVALID_ARG;
  if (t.warps_per_cta != 0 && t.warps_per_cta != 4 && t.warps_per_cta != 8 && t.warps_per_cta != 16)
    return IHIST_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    int rc = validate_shape(frames[i].h, frames[i].w, frames[i].nbins, frames[i].layout);
    if (rc != IHIST_OK) return rc;
    rc = joint_ok(frames[i]);
    if (rc != IHIST_OK) return rc;
    if (!table_ok(frames[i])) return IHIST_ERR_INVALID_ARG;
  }
  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IHIST_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return IHIST_ERR_CUDA;

  ihist_batch_s *b = new (std::nothrow) ihist_batch_s();
  if (!b) return IHIST_ERR_OOM;
  b->device = dev;
  b->sms = sms;
  b->cap = n;
  b->G = t.bins_per_cta;
  b->lut = lut;
  b->fault_skip_band = t.fault_skip_band >= 1 ? t.fault_skip_band - 1 : -1;
  // pixel-major frames stage their rows in shared memory
  b->stage = 0;
  for (int i = 0; i < n; ++i)
    if (pm_staged(frames[i].layout, b->G)) b->stage = 1;
  const int max_m = b->G == 16 ? 2 : 4;  // chunks per warp the instantiations cover
  b->warps = t.warps_per_cta;
  if (b->warps == 0) {
    // 8-warp CTAs (4 per SM overlap their count, look-back and emit phases
    // better than 2 of 16 warps: 5% faster on 1080p frames), except 16 for
    // staged pixel-major rows in 8-bin groups (64 pixel-major 1080p frames:
    // 8 bins 10.5 ms with 16 warps against 11.7 with 8; 16 bins 8.2 ms with
    // 8 warps against 8.5 with 16) and for frames wider than 8 warps x
    // max_m chunks
    b->warps = (b->stage && b->G != 16) ? kBatchWarps : 8;
    for (int i = 0; i < n; ++i)
      if (frames[i].w > 8 * max_m * kChunk) b->warps = kBatchWarps;
  }
  b->timeout_us = t.timeout_us ? t.timeout_us : kDefaultTimeoutUs;
  // every kernel variant the batch may launch may use the opt-in shared memory
  for (int mm = 1; mm <= max_m; mm <<= 1)
    for (int tma = 0; tma < 2; ++tma)
      for (int vec = 0; vec < 2; ++vec) {
        BatchFn fn = batch_fn(b->G, mm, tma != 0, vec != 0, b->lut);
        cudaFuncAttributes a;
        if (!fn || cudaFuncGetAttributes(&a, fn) != cudaSuccess) {
          cudaGetLastError();
          delete b;
          return fn ? IHIST_ERR_CUDA : IHIST_ERR_UNSUPPORTED;
        }
        const size_t dyn_max = (size_t)optin > a.sharedSizeBytes ? (size_t)optin - a.sharedSizeBytes : 0;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max) != cudaSuccess) {
          cudaGetLastError();
          delete b;
          return IHIST_ERR_CUDA;
        }
      }
  // default rows per band: the largest R (at most 64) at which the kernel
  // still keeps 32 warps per SM (each warp stages R rows of input and row
  // carries in shared memory), as the occupancy calculator reports it
  // every frame must have a tiling in CTAs of this many warps
  for (int i = 0; i < n; ++i) {
    FrameDesc f;
    if (!batch_frame_tiling(frames[i].h, frames[i].w, frames[i].nbins, frames[i].layout, b->G, 8, max_m,
                            INT_MAX, b->warps, &f)) {
      delete b;
      return IHIST_ERR_UNSUPPORTED;
    }
  }
  b->R_req = t.rows_per_band;
  if (b->R_req == 0) {
    // the largest R (at most 64) that keeps the CTAs per SM that the
    // smallest bands allow (registers permitting: 4 of 8 warps or 2 of 16
    // warps with 4 or 8 bins per CTA, 1 with 16)
    auto occ_at = [&](int r) {
      int rmax = 1, ncg = 1, mm = 1;
      for (int i = 0; i < n; ++i) {
        FrameDesc f;
        batch_frame_tiling(frames[i].h, frames[i].w, frames[i].nbins, frames[i].layout, b->G, r, max_m, INT_MAX,
                           b->warps, &f);
        rmax = std::max(rmax, f.R);
        ncg = std::max(ncg, frame_ncl(f) * f.gpc);
        mm = std::max(mm, f.m);
      }
      int occ = 0;
      const size_t smem = smem_layout(b->warps, rmax, b->G, ncg, b->stage != 0).bytes;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_fn(b->G, mmax_for(mm), true, true, b->lut),
                                                        b->warps * 32, smem) != cudaSuccess) {
        cudaGetLastError();
        occ = 0;
      }
      return occ;
    };
    const int target = std::max(1, occ_at(8));
    b->R_req = 8;
    for (int r = 64; r >= 8; --r) {
      if (occ_at(r) >= target) {
        b->R_req = r;
        break;
      }
    }
  }
  // slot capacities from the planned frames
  std::vector<FrameDesc> plan_fd(n);
  int mm = 1;
  size_t nci_total = 0;
  for (int i = 0; i < n; ++i) {
    batch_frame_tiling(frames[i].h, frames[i].w, frames[i].nbins, frames[i].layout, b->G, b->R_req, max_m,
                       INT_MAX, b->warps, &plan_fd[i]);
    mm = std::max(mm, plan_fd[i].m);
    b->R_max = std::max(b->R_max, plan_fd[i].R);
    b->ncg_max = std::max(b->ncg_max, frame_ncl(plan_fd[i]) * plan_fd[i].gpc);
    b->slot_nci.push_back(frame_nci(plan_fd[i]));
    b->slot_nhs.push_back(frame_nhs(plan_fd[i]));
    b->slot_hwords.push_back(frame_hagg_words(plan_fd[i], b->G));
    nci_total += frame_nci(plan_fd[i]) + frame_nhs(plan_fd[i]);
  }
  b->mmax = mmax_for(mm);
  b->smem_bytes = smem_layout(b->warps, b->R_max, b->G, b->ncg_max, b->stage != 0).bytes;
  for (int tma = 0; tma < 2; ++tma)
    for (int vec = 0; vec < 2; ++vec) {
      BatchFn fn = batch_fn(b->G, b->mmax, tma != 0, vec != 0, b->lut);
      cudaFuncAttributes a;
      if (!fn || cudaFuncGetAttributes(&a, fn) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fn ? IHIST_ERR_CUDA : IHIST_ERR_UNSUPPORTED;
      }
      const size_t dyn_max = (size_t)optin > a.sharedSizeBytes ? (size_t)optin - a.sharedSizeBytes : 0;
      int occ = 0;
      if (b->smem_bytes > dyn_max ||
          cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, b->warps * 32, b->smem_bytes) != cudaSuccess ||
          occ < 1) {
        cudaGetLastError();
        delete b;
        return IHIST_ERR_UNSUPPORTED;
      }
      b->ctas_per_sm[tma][vec] = t.ctas_per_sm > 0 ? std::min(t.ctas_per_sm, occ) : occ;
    }

  // workspace: control block and flags (cleared), descriptor arrays
  // (written only by copies), then each slot's carries
  size_t off = 0;
  const size_t o_ctrl = off;
  off = align_up(off + sizeof(Ctrl), 256);
  const size_t o_flags = off;
  off = align_up(off + nci_total * sizeof(uint32_t), 256);
  const size_t zero_end = off;
  const size_t o_fd = off;
  off = align_up(off + (size_t)n * sizeof(FrameDesc), 256);
  const size_t o_fdq = off;
  off = align_up(off + (size_t)n * sizeof(FrameDesc), 256);
  const size_t o_tm = off;
  off = align_up(off + (size_t)n * sizeof(CUtensorMap), 256);
  const size_t o_end = off;
  off = align_up(off + (size_t)n * sizeof(unsigned int), 256);
  const size_t o_bend = off;
  off = align_up(off + (size_t)n * sizeof(unsigned int), 256);
  const size_t o_lut = off;
  if (lut) off = align_up(off + (size_t)n * 256 * sizeof(uint32_t), 256);
  const size_t o_carry = off;
  for (int i = 0; i < n; ++i) {
    const size_t nci = b->slot_nci[i];
    off = align_up(off + nci * kChunk * (b->G / 4) * 4, 256);
    off = align_up(off + nci * b->G * 4, 256);
    off = align_up(off + nci * b->G * kChunk * 4, 256);
    off = align_up(off + b->slot_hwords[i] * 4, 256);
  }
  const size_t o_idx = off;  // joint-bin planes of the slots planned with joint frames
  for (int i = 0; i < n; ++i) {
    b->slot_idx_cap.push_back(idx_bytes_of(frames[i]));
    off = align_up(off + b->slot_idx_cap[i], 256);
  }
  b->ws_bytes = off;
  if (cudaMalloc(&b->ws, b->ws_bytes) != cudaSuccess ||
      [&]() {
        for (int i = 0; i < 2; ++i) {
          ihist_batch_s::Staging &st = b->stage_sets[i];
          if (cudaMallocHost((void **)&st.fd, (size_t)n * sizeof(FrameDesc)) != cudaSuccess ||
              cudaMallocHost((void **)&st.fdq, (size_t)n * sizeof(FrameDesc)) != cudaSuccess ||
              cudaMallocHost((void **)&st.tm, (size_t)n * sizeof(CUtensorMap)) != cudaSuccess ||
              cudaMallocHost((void **)&st.end, (size_t)n * sizeof(unsigned int)) != cudaSuccess ||
              cudaMallocHost((void **)&st.bins_end, (size_t)n * sizeof(unsigned int)) != cudaSuccess ||
              (lut && cudaMallocHost((void **)&st.lut, (size_t)n * 256 * sizeof(uint32_t)) != cudaSuccess) ||
              cudaEventCreateWithFlags(&b->staged[i], cudaEventDisableTiming) != cudaSuccess)
            return false;
        }
        return true;
      }() == false ||
      cudaEventCreateWithFlags(&b->uploaded, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->computed, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    ihist_batch_destroy(b);
    return IHIST_ERR_OOM;
  }
  char *base = static_cast<char *>(b->ws);
  b->ctrl = reinterpret_cast<Ctrl *>(base + o_ctrl);
  b->d_fd = reinterpret_cast<FrameDesc *>(base + o_fd);
  b->d_fdq = reinterpret_cast<FrameDesc *>(base + o_fdq);
  b->d_tm = reinterpret_cast<CUtensorMap *>(base + o_tm);
  b->d_end = reinterpret_cast<unsigned int *>(base + o_end);
  b->d_bins_end = reinterpret_cast<unsigned int *>(base + o_bend);
  if (lut) b->d_lut = reinterpret_cast<uint32_t *>(base + o_lut);
  size_t fo = o_flags, co = o_carry;
  for (int i = 0; i < n; ++i) {
    const size_t nci = b->slot_nci[i];
    b->slot_flags.push_back(reinterpret_cast<uint32_t *>(base + fo));
    fo += nci * sizeof(uint32_t);
    b->slot_hflags.push_back(reinterpret_cast<uint32_t *>(base + fo));  // segment flags, cleared with the rest
    fo += b->slot_nhs[i] * sizeof(uint32_t);
    b->slot_cnt.push_back(reinterpret_cast<uint32_t *>(base + co));
    co = align_up(co + nci * kChunk * (b->G / 4) * 4, 256);
    b->slot_left.push_back(reinterpret_cast<uint32_t *>(base + co));
    co = align_up(co + nci * b->G * 4, 256);
    b->slot_incl.push_back(reinterpret_cast<uint32_t *>(base + co));
    co = align_up(co + nci * b->G * kChunk * 4, 256);
    b->slot_hagg.push_back(reinterpret_cast<uint32_t *>(base + co));
    co = align_up(co + b->slot_hwords[i] * 4, 256);
  }
  size_t xo = o_idx;
  for (int i = 0; i < n; ++i) {
    b->slot_idx.push_back(b->slot_idx_cap[i] ? reinterpret_cast<uint8_t *>(base + xo) : nullptr);
    xo = align_up(xo + b->slot_idx_cap[i], 256);
  }
  use_staging(b, 0);
  int rc = batch_bind(b, frames, n);
  if (rc != IHIST_OK) {
    ihist_batch_destroy(b);
    return rc;
  }
  // clear the control block and the flags only; the descriptor arrays are
  // written once per binding by the copies
  if (cudaMemset(b->ws, 0, zero_end) != cudaSuccess || batch_upload(b, 0) != IHIST_OK ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    ihist_batch_destroy(b);
    return IHIST_ERR_CUDA;
  }
  (void)o_ctrl;
  *out = b;
  return IHIST_OK;
}

static int check_batch_device(const ihist_batch_s *b) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return IHIST_ERR_CUDA;
  return dev == b->device ? IHIST_OK : IHIST_ERR_INVALID_ARG;
}

extern "C" int ihist_batch_get_tune(ihist_batch_t b, ihist_tune_t *out) {
  if (!b || !out) return IHIST_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->rows_per_band = b->R_req;
  out->bins_per_cta = b->G;
  out->chunks_per_warp = b->mmax;
  out->ctas_per_sm = b->ctas_per_sm[1][1];
  out->timeout_us = b->timeout_us;
  out->fault_skip_band = b->fault_skip_band + 1;  // 0 = off
  out->groups_per_cta = 0;  // chosen per frame
  out->warps_per_cta = b->warps;
  return IHIST_OK;
}

extern "C" int ihist_batch_set_io(ihist_batch_t b, const ihist_frame_t *frames, int n, void *stream) {
  if (!b || !frames) return IHIST_ERR_INVALID_ARG;
  int rc = check_batch_device(b);
  if (rc != IHIST_OK) return rc;
  // build the binding in the other staging set, once that set's previous
  // copy (two bindings back) has been made; on failure the current binding
  // (already copied from its own set) stays in force
  const int prev = b->stage_cur, next = prev ^ 1;
  if (cudaEventSynchronize(b->staged[next]) != cudaSuccess) return IHIST_ERR_CUDA;
  use_staging(b, next);
  rc = batch_bind(b, frames, n);
  if (rc != IHIST_OK) {
    use_staging(b, prev);
    return rc;
  }
  return batch_upload(b, (cudaStream_t)stream);
}

extern "C" int ihist_batch_compute(ihist_batch_t b, void *stream) {
  if (!b) return IHIST_ERR_INVALID_ARG;
  int rc = check_batch_device(b);
  if (rc != IHIST_OK) return rc;
  // joint frames: their joint-bin planes first (the scan waits for them)
  for (int i = 0; i < b->n; ++i) {
    const ihist_frame_t &fr = b->io[i];
    if (!frame_joint(fr)) continue;
    rc = launch_joint_index(fr.d_in, (long long)fr.in_pitch, fr.h, fr.w, fr.channels, fr.bins_per_channel,
                            b->slot_idx[i], (long long)idx_pitch_of(fr.w), b->sms, stream);
    if (rc != IHIST_OK) return rc;
  }
  BatchFn fn = batch_fn(b->G, b->mmax, b->tma, b->vec, b->lut);
  const int cps = b->ctas_per_sm[b->tma ? 1 : 0][b->vec ? 1 : 0];
  const unsigned int grid = std::min<unsigned int>(b->total, (unsigned int)(cps * b->sms));
  const unsigned long long timeout_ns = (unsigned long long)b->timeout_us * 1000ull;
  fn<<<grid, b->warps * 32, b->smem_bytes, (cudaStream_t)stream>>>(
      b->d_fd, b->d_tm, b->d_end, b->n, b->R_max, b->ncg_max, b->stage, b->ctrl, timeout_ns);
  if (cudaGetLastError() != cudaSuccess) return IHIST_ERR_CUDA;
  if (cudaEventRecord(b->computed, (cudaStream_t)stream) != cudaSuccess) return IHIST_ERR_CUDA;
  b->launched = true;
  return IHIST_OK;
}

extern "C" int ihist_batch_upload_compute(ihist_batch_t b, const uint8_t *const *h_frames, void *stream,
                                          void *copy_stream) {
  if (!b || !h_frames) return IHIST_ERR_INVALID_ARG;
  for (int i = 0; i < b->n; ++i)
    if (!h_frames[i]) return IHIST_ERR_INVALID_ARG;
  int rc = check_batch_device(b);
  if (rc != IHIST_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream, cs = (cudaStream_t)copy_stream;
  // inputs are overwritten only after the previous compute of this batch read them
  if (b->launched && cudaStreamWaitEvent(cs, b->computed, 0) != cudaSuccess) return IHIST_ERR_CUDA;
  for (int i = 0; i < b->n; ++i) {
    const ihist_frame_t &fr = b->io[i];
    const size_t row = (size_t)fr.w * frame_channels(fr);
    if (cudaMemcpy2DAsync(const_cast<uint8_t *>(fr.d_in), fr.in_pitch, h_frames[i], row, row, (size_t)fr.h,
                          cudaMemcpyHostToDevice, cs) != cudaSuccess)
      return IHIST_ERR_CUDA;
  }
  if (cudaEventRecord(b->uploaded, cs) != cudaSuccess ||
      cudaStreamWaitEvent(s, b->uploaded, 0) != cudaSuccess)
    return IHIST_ERR_CUDA;
  return ihist_batch_compute(b, stream);
}

extern "C" int ihist_batch_query_all(ihist_batch_t b, const int32_t *d_rects, int n, uint32_t *d_out,
                                     void *stream) {
  if (!b || n < 0) return IHIST_ERR_INVALID_ARG;
  if (n == 0) return IHIST_OK;
  if (!d_rects || !d_out || ((uintptr_t)d_rects & 3u) || ((uintptr_t)d_out & 3u))
    return IHIST_ERR_INVALID_ARG;
  int rc = check_batch_device(b);
  if (rc != IHIST_OK) return rc;
  if (b->bins_total * (unsigned long long)n >= (1ull << 40)) return IHIST_ERR_UNSUPPORTED;
  const unsigned long long total = b->bins_total * (unsigned long long)n;
  const unsigned int threads = 256;
  const unsigned long long want = (total + threads - 1) / threads;
  const unsigned int grid = (unsigned int)std::min<unsigned long long>(want, (unsigned long long)b->sms * 16ull);
  query_batch_kernel<FrameDesc><<<grid, threads, 0, (cudaStream_t)stream>>>(
      b->d_fdq, b->d_bins_end, b->n, d_rects, (unsigned int)n, total, d_out, b->ctrl);
  if (cudaGetLastError() != cudaSuccess) return IHIST_ERR_CUDA;
  return IHIST_OK;
}

extern "C" int ihist_batch_query(ihist_batch_t b, int frame, const uint32_t *d_hist,
                                 const int32_t *d_rects, int n, uint32_t *d_hist_out, void *stream) {
  if (!b || frame < 0 || frame >= b->n || n < 0) return IHIST_ERR_INVALID_ARG;
  if (n == 0) return IHIST_OK;
  int rc = check_batch_device(b);
  if (rc != IHIST_OK) return rc;
  const FrameDesc &f = b->fd[frame];
  return launch_query(f.H, f.W, f.B, f.layout, b->sms, b->ctrl, d_hist, d_rects, n, d_hist_out, stream);
}

extern "C" int ihist_batch_status(ihist_batch_t b, void *stream, int *device_status) {
  if (!b || !device_status) return IHIST_ERR_INVALID_ARG;
  int rc = check_batch_device(b);
  if (rc != IHIST_OK) return rc;
  return read_status(b->ctrl, stream, device_status);
}

extern "C" size_t ihist_batch_workspace_bytes(ihist_batch_t b) { return b ? b->ws_bytes : 0; }

extern "C" unsigned int ihist_batch_items(ihist_batch_t b) { return b ? b->total : 0u; }

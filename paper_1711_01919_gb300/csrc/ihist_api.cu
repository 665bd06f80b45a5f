// ihist_api.cu -- host side of libihist.so for single-frame plans: argument
// validation, plan and workspace management, kernel selection and launches
// (batches are in ihist_batch_api.cu).  Declared in include/ihist.h.
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
#include "ihist_joint.cuh"
#include "ihist_kernels.h"
#include "ihist_query.cuh"
#include "ihist_query_sorted.cuh"
#include "ihist_window.cuh"

using namespace ihist;

using namespace ihist::host;

PFN_cuTensorMapEncodeTiled_v12000 ihist::host::tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

enum Binning { kUniform = 0, kTable = 1, kJoint = 2 };

struct ihist_plan_s {
  int device;
  int sms;
  int H, W, B, layout;
  int binning;          // Binning
  JointBins joint;      // kJoint: channels and their bins
  uint32_t *lut;        // kTable: device table, 8 * bin of each intensity or kNoBin
  uint8_t *idx;         // kJoint: joint-bin plane [H][idx_pitch]
  size_t idx_pitch;
  int R, G, m, NW, nbands, ngroups, nchunks, wpg, gpc, ngsets;
  int nsegs, cps;       // width segments per band and chunks per segment
  unsigned int nitems;
  int ctas_per_sm;
  unsigned int timeout_us;
  int fault_skip_band;
  int overlap;          // launch with programmatic dependent launch
  size_t smem_bytes;
  void *ws;
  size_t ws_bytes;
  Ctrl *ctrl;
  Ctrl *ctrl_alt;  // control block of every other launch (epochs of the other parity)
  unsigned long long launches;
  uint32_t *flags, *agg_cnt, *agg_left, *incl;
  uint32_t *hflags, *hagg;     // width segments (nsegs > 1): flags and per-row totals
  cudaEvent_t ev_uploaded[2];  // sequence pipeline: slot filled
  cudaEvent_t ev_consumed[2];  // sequence pipeline: slot read by its compute
  cudaEvent_t ev_queried;      // sequence pipeline: a frame's query rows are in d_query
  cudaEvent_t ev_copied;       // sequence pipeline: those rows have reached the host
  struct {
    const void *ptr;
    size_t pitch;
    bool ok;
    CUtensorMap map;
  } tmaps[4];                  // TMA descriptors of recent inputs (round robin)
  int tmap_next;
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
    case IHIST_ERR_CHECK_FAILED: return "checked build caught an out-of-range access; result invalid";
    default: return "unknown status";
  }
}

int ihist::host::validate_shape(int h, int w, int nbins, int layout) {
  if (h < 1 || w < 1 || h > 65535 || w > 65535) return IHIST_ERR_INVALID_ARG;
  if ((unsigned long long)h * (unsigned long long)w >= (1ull << 32)) return IHIST_ERR_INVALID_ARG;
  if (nbins < 1 || nbins > 256) return IHIST_ERR_INVALID_ARG;
  if (layout != IHIST_BIN_MAJOR && layout != IHIST_PIXEL_MAJOR && layout != IHIST_QUAD_MAJOR)
    return IHIST_ERR_INVALID_ARG;
  if (layout == IHIST_QUAD_MAJOR && nbins % 4 != 0) return IHIST_ERR_INVALID_ARG;
  return IHIST_OK;
}

// Largest dynamic shared memory a CTA may opt into, set once on every
// instantiation a plan may launch so that occupancy queries and launches
// can use any tile size up to it.
static int prepare_kernels(int G, int mmax, int dev, size_t *optin, bool lut = false) {
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return IHIST_ERR_CUDA;
  size_t dyn = (size_t)v;
  for (int tma = 0; tma < 2; ++tma)
    for (int vec = 0; vec < 2; ++vec) {
      ScanFn fn = scan_fn(G, mmax, tma != 0, vec != 0, lut);
      if (!fn) return IHIST_ERR_UNSUPPORTED;
      cudaFuncAttributes a;
      if (cudaFuncGetAttributes(&a, fn) != cudaSuccess) {
        cudaGetLastError();
        return IHIST_ERR_CUDA;
      }
      // dynamic + static shared memory must fit the opt-in limit
      const size_t d = (size_t)v > a.sharedSizeBytes ? (size_t)v - a.sharedSizeBytes : 0;
      if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d) != cudaSuccess) {
        cudaGetLastError();
        return IHIST_ERR_CUDA;
      }
      dyn = std::min(dyn, d);
    }
  *optin = dyn;
  return IHIST_OK;
}

static int occupancy(ScanFn fn, int threads, size_t smem) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}

// Default tiling: the (rows per band R, bin groups per CTA) that maximise
// (fraction of persistent-CTA slot time the work items fill, counting the
// last partial wave) x (1 - carry overhead, about 1.25/R of the output
// bytes) x (warps per SM, up to 24) x (fraction of CTA bin groups in use).
// Fields the caller fixed (non-zero) are kept.
static void default_tiling(int h, int ngroups, int wpg, int G, int ncl, int nsegs, int sms, ScanFn fn,
                           size_t optin, int layout, int max_warps, int *R, int *gpc) {
  double best = -1.0;
  int best_r = *R ? *R : std::min(h, 8), best_g = *gpc ? *gpc : 1;
  const int g_lo = *gpc ? *gpc : 1;
  const int g_hi = *gpc ? *gpc : std::max(1, std::min(ngroups, max_warps / wpg));
  for (int gp = g_lo; gp <= g_hi; ++gp) {
    const int NW = gp * wpg;
    const int ngsets = (ngroups + gp - 1) / gp;
    const double used = (double)ngroups / (double)(ngsets * gp);
    const int r_lo = *R ? *R : std::min(h, 8), r_hi = *R ? *R : std::min(h, 255);
    for (int r = r_lo; r <= r_hi; ++r) {
      const size_t smem = smem_layout(NW, r, G, ncl * gp, pm_staged(layout, G)).bytes;
      if (smem > optin) break;
      const int occ = occupancy(fn, NW * 32, smem);
      if (occ < 1) break;
      const long long slots = (long long)occ * sms;
      const long long items = (long long)((h + r - 1) / r) * ngsets * nsegs;
      const long long waves = (items + slots - 1) / slots;
      const double fill = (double)items / (double)(waves * slots);
      const double carry = 1.0 - 1.25 / r;
      const double warps = std::min(1.0, occ * NW / 24.0);
      const double score = fill * carry * warps * used;
      if (score > best) {
        best = score;
        best_r = r;
        best_g = gp;
      }
    }
  }
  // A frame that fills less than one wave even in the smallest bands (the
  // score above then settles on the smallest R) runs each CTA's one item at
  // a time: its time grows with the band's rows and with the look-back
  // chain (the band count).  Measured on 640x480 x 32, T ~ 0.18 R + 0.085
  // (h / R) us (R = 8: 25.3 us, 16: 24.2, 24: 24.8), so R near sqrt(h / 2)
  // instead (640x480 x 32: 29.1 -> 24.8 us per frame; 1280x720 x 16: 34.5 ->
  // 30.9 us).  Frames for which the score picked a larger R keep it: there
  // the larger sqrt(h / 2) measured slower (1280x720 x 32, 1920x1080 x 16).
  if (!*R && best_r == std::min(h, 8)) {
    const int NW = best_g * wpg;
    const int ngsets = (ngroups + best_g - 1) / best_g;
    const size_t smem0 = smem_layout(NW, best_r, G, ncl * best_g, pm_staged(layout, G)).bytes;
    const long long slots0 = (long long)occupancy(fn, NW * 32, smem0) * sms;
    if ((long long)((h + best_r - 1) / best_r) * ngsets * nsegs <= slots0) {
      double best_t = 1e30;
      int pick = best_r;
      for (int r = std::min(h, 8); r <= std::min(h, 255); ++r) {
        const size_t smem = smem_layout(NW, r, G, ncl * best_g, pm_staged(layout, G)).bytes;
        if (smem > optin || occupancy(fn, NW * 32, smem) < 1) break;
        const double t = r + 0.5 * ((h + r - 1) / r);
        if (t < best_t) {
          best_t = t;
          pick = r;
        }
      }
      best_r = pick;
    }
  }
  *R = best_r;
  *gpc = best_g;
}

// Plan for uniform bins (bin_map and joint null), a value -> bin table
// (bin_map: 256 ints in [-1, nbins)) or joint bins of a multi-channel frame.
static int plan_create(int h, int w, int nbins, int layout, const ihist_tune_t *tune, const int *bin_map,
                       const JointBins *joint, ihist_plan_t *out) {
  if (!out) return IHIST_ERR_INVALID_ARG;
  int rc = validate_shape(h, w, nbins, layout);
  if (rc != IHIST_OK) return rc;
  const bool table = bin_map != nullptr;
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
  if (t.groups_per_cta < 0 || t.groups_per_cta > 16) return IHIST_ERR_INVALID_ARG;
  if (t.overlap != 0 && t.overlap != 1) return IHIST_ERR_INVALID_ARG;
  if (t.warps_per_cta < 0 || t.warps_per_cta > 16) return IHIST_ERR_INVALID_ARG;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IHIST_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return IHIST_ERR_CUDA;
  const int nchunks = (w + kChunk - 1) / kChunk;
  // Pixel-major output: a pixel's counts of one bin group are G contiguous
  // words and the groups of a pixel belong to different CTAs, so larger
  // groups give longer contiguous pieces per pixel record; rows are staged
  // in shared memory so that a warp store writes whole pieces (measured on
  // 1080p x 64 per frame: G = 4 unstaged 762 us; G = 16 unstaged 325 us,
  // staged 159 us).
  const bool pm_wide = layout == IHIST_PIXEL_MAJOR && nbins >= 16 && nchunks <= 32 && !table;
  if (t.bins_per_cta == 0) t.bins_per_cta = layout == IHIST_PIXEL_MAJOR ? (pm_wide ? 16 : 8) : 4;
  // Frames wider than 16 chunks (bin- and quad-major): one chunk per warp
  // in CTAs of at most 8 warps, each band split into width segments, 48
  // rows per band -- more, smaller CTAs per SM and the one-chunk kernel,
  // against one 16-warp CTA spanning the width with several chunks per
  // warp (measured per frame: 3840x2160 x 64 405 -> 357 us, 7680x4320 x 32
  // 830 -> 690 us, 16384x2048 x 16 503 -> 374 us, 8192x8192 x 128 5.38 ->
  // 5.01 ms; frames of up to 16 chunks are faster in one CTA).
  if (nchunks > 16 && layout != IHIST_PIXEL_MAJOR && t.chunks_per_warp == 0 && t.warps_per_cta == 0) {
    t.chunks_per_warp = 1;
    t.warps_per_cta = 8;
    if (t.rows_per_band == 0) t.rows_per_band = std::min(h, 48);
  }
  if (t.chunks_per_warp == 0) {
    t.chunks_per_warp = nchunks <= 16 ? 1 : nchunks <= 32 ? 2 : nchunks <= 64 ? 4 : 8;
    if (t.bins_per_cta == 16) t.chunks_per_warp = std::min(t.chunks_per_warp, 2);  // the 16-bin kernels' limit
  }
  const int cta_warps = t.warps_per_cta ? t.warps_per_cta : 16;  // upper bound on a CTA's warps
  if (t.timeout_us == 0) t.timeout_us = kDefaultTimeoutUs;
  // Frames wider than W warps x m chunks (W = warps_per_cta, default 16;
  // W / groups_per_cta warps when that is given) split each band into width
  // segments of equal chunk counts, one work item each (see the scan kernel).
  struct Split {
    int nsegs, wpg, cps, ncl;  // ncl: chunks of one CTA's group
  };
  auto split_for = [&](int gpc) {
    Split sp;
    const int wpg_all = (nchunks + t.chunks_per_warp - 1) / t.chunks_per_warp;
    const int seg_warps = std::max(1, cta_warps / std::max(1, gpc));  // warps of one group
    sp.nsegs = (wpg_all + seg_warps - 1) / seg_warps;
    sp.wpg = (wpg_all + sp.nsegs - 1) / sp.nsegs;
    sp.cps = sp.wpg * t.chunks_per_warp;
    sp.ncl = std::min(nchunks, sp.cps);
    return sp;
  };
  Split sp = split_for(t.groups_per_cta);
  const int mmax = mmax_for(t.chunks_per_warp);
  if (sp.wpg * std::max(1, t.groups_per_cta) > cta_warps || !scan_fn(t.bins_per_cta, mmax, true, true, table))
    return IHIST_ERR_UNSUPPORTED;
  size_t optin = 0;
  rc = prepare_kernels(t.bins_per_cta, mmax, dev, &optin, table);
  if (rc != IHIST_OK) return rc;
  ScanFn fn = scan_fn(t.bins_per_cta, mmax, true, true, table);
  const int ngroups = (nbins + t.bins_per_cta - 1) / t.bins_per_cta;
  if (t.groups_per_cta > ngroups) t.groups_per_cta = ngroups;
  if (t.rows_per_band == 0 || t.groups_per_cta == 0) {
    const bool gpc_free = t.groups_per_cta == 0;
    const int r_req = t.rows_per_band;
    default_tiling(h, ngroups, sp.wpg, t.bins_per_cta, sp.ncl, sp.nsegs, sms, fn, optin, layout, cta_warps,
                   &t.rows_per_band, &t.groups_per_cta);
    // Staged pixel-major frames whose one-group items fit in one wave of
    // CTAs: one group per CTA, the most CTAs side by side (640x480 x 64,
    // 16 bins per group: 70.5 us per frame with 2 groups per CTA, 61.7 us
    // with 1; 640x480 x 32: 62.4 -> 61.3 us).
    if (gpc_free && t.groups_per_cta > 1 && pm_staged(layout, t.bins_per_cta)) {
      int R = r_req, g = 1;
      default_tiling(h, ngroups, sp.wpg, t.bins_per_cta, sp.ncl, sp.nsegs, sms, fn, optin, layout, cta_warps, &R, &g);
      const size_t smem = smem_layout(sp.wpg, R, t.bins_per_cta, sp.ncl, true).bytes;
      const int occ = smem <= optin ? occupancy(fn, sp.wpg * 32, smem) : 0;
      const long long items = (long long)((h + R - 1) / R) * ngroups * sp.nsegs;
      if (occ >= 1 && items <= (long long)occ * sms) {
        t.groups_per_cta = 1;
        t.rows_per_band = R;
      }
    }
    // Pixel-major frames of two to four bin groups whose records the scan
    // kernel can store whole (see pm_record): all groups in one CTA, so the
    // warps of a column range write complete records, when those coarser
    // items still fill a wave of CTAs (1080p x 64, 16 bins per group: 156
    // -> 151 us per frame, 151 -> 144 us overlapped; smaller frames, whose
    // items would leave SMs idle, measured 11-19% slower that way).
    if (gpc_free && t.groups_per_cta != ngroups && ngroups >= 2 && ngroups <= 4 &&
        pm_staged(layout, t.bins_per_cta) && pm_record_bins(nbins) && !table) {
      const Split sr = split_for(ngroups);
      int R = r_req, g = ngroups;
      default_tiling(h, ngroups, sr.wpg, t.bins_per_cta, sr.ncl, sr.nsegs, sms, fn, optin, layout, cta_warps, &R, &g);
      const int nw = sr.wpg * ngroups;
      const size_t smem = smem_layout(nw, R, t.bins_per_cta, sr.ncl * ngroups, true).bytes;
      const int occ = (nw <= cta_warps && smem <= optin) ? occupancy(fn, nw * 32, smem) : 0;
      const long long items = (long long)((h + R - 1) / R) * sr.nsegs;
      if (occ >= 1 && items >= (long long)occ * sms) {
        t.groups_per_cta = ngroups;
        t.rows_per_band = R;
        sp = sr;
      }
    }
  }
  const int nsegs = sp.nsegs, wpg = sp.wpg, cps = sp.cps, ncl = sp.ncl;

  ihist_plan_s *p = new (std::nothrow) ihist_plan_s;
  if (!p) return IHIST_ERR_OOM;
  std::memset(p, 0, sizeof(*p));
  p->device = dev;
  p->sms = sms;
  p->H = h;
  p->W = w;
  p->B = nbins;
  p->layout = layout;
  p->binning = table ? kTable : joint ? kJoint : kUniform;
  if (joint) p->joint = *joint;
  p->G = t.bins_per_cta;
  p->m = t.chunks_per_warp;
  p->R = std::min(t.rows_per_band, h);
  p->nchunks = nchunks;
  p->wpg = wpg;
  p->gpc = t.groups_per_cta;
  p->NW = wpg * p->gpc;
  p->nbands = (h + p->R - 1) / p->R;
  p->ngroups = ngroups;
  p->ngsets = (ngroups + p->gpc - 1) / p->gpc;
  p->nsegs = nsegs;
  p->cps = nsegs > 1 ? cps : nchunks;
  if ((unsigned long long)p->nbands * p->ngsets * nsegs >= 0xffffffffull) {
    delete p;
    return IHIST_ERR_UNSUPPORTED;
  }
  p->nitems = (unsigned int)p->nbands * (unsigned int)p->ngsets * (unsigned int)nsegs;
  p->timeout_us = t.timeout_us;
  p->fault_skip_band = t.fault_skip_band >= 1 ? t.fault_skip_band - 1 : -1;  // 1-based in the tune struct
  p->overlap = t.overlap;
  p->smem_bytes = smem_layout(p->NW, p->R, p->G, ncl * p->gpc, pm_staged(layout, p->G)).bytes;
  const int occ = p->smem_bytes <= optin ? occupancy(fn, p->NW * 32, p->smem_bytes) : 0;
  if (occ < 1) {
    delete p;
    return IHIST_ERR_UNSUPPORTED;
  }
  p->ctas_per_sm = t.ctas_per_sm > 0 ? std::min(t.ctas_per_sm, occ) : occ;

  // workspace: control block, flags, column-count aggregates, left counts, inclusive rows
  const size_t nci = (size_t)p->nbands * p->ngroups * p->nchunks;
  size_t off = 0;
  const size_t o_ctrl = off;
  off = align_up(off + sizeof(Ctrl), 256);
  const size_t o_ctrl_alt = off;
  off = align_up(off + sizeof(Ctrl), 256);
  const size_t o_flags = off;
  off = align_up(off + nci * sizeof(uint32_t), 256);
  const size_t nhs = nsegs > 1 ? (size_t)p->nbands * p->ngroups * nsegs : 0;  // segment records
  const size_t o_hflags = off;
  off = align_up(off + nhs * sizeof(uint32_t), 256);
  const size_t o_cnt = off;
  off = align_up(off + nci * kChunk * (p->G / 4) * sizeof(uint32_t), 256);
  const size_t o_left = off;
  off = align_up(off + nci * p->G * sizeof(uint32_t), 256);
  const size_t o_incl = off;
  off = align_up(off + nci * p->G * kChunk * sizeof(uint32_t), 256);
  const size_t o_hagg = off;
  off = align_up(off + nhs * ((size_t)p->R * p->G + p->G) * sizeof(uint32_t), 256);
  const size_t o_lut = off;
  if (table) off = align_up(off + 256 * sizeof(uint32_t), 256);
  const size_t o_idx = off;
  p->idx_pitch = align_up((size_t)w, 16);
  if (joint) off = align_up(off + (size_t)h * p->idx_pitch, 256);
  p->ws_bytes = off;
  if (cudaMalloc(&p->ws, p->ws_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return IHIST_ERR_OOM;
  }
  char *base = static_cast<char *>(p->ws);
  p->ctrl = reinterpret_cast<Ctrl *>(base + o_ctrl);
  p->ctrl_alt = reinterpret_cast<Ctrl *>(base + o_ctrl_alt);
  p->flags = reinterpret_cast<uint32_t *>(base + o_flags);
  p->agg_cnt = reinterpret_cast<uint32_t *>(base + o_cnt);
  p->agg_left = reinterpret_cast<uint32_t *>(base + o_left);
  p->incl = reinterpret_cast<uint32_t *>(base + o_incl);
  if (nhs) {
    p->hflags = reinterpret_cast<uint32_t *>(base + o_hflags);
    p->hagg = reinterpret_cast<uint32_t *>(base + o_hagg);
  }
  if (table) p->lut = reinterpret_cast<uint32_t *>(base + o_lut);
  if (joint) p->idx = reinterpret_cast<uint8_t *>(base + o_idx);
  uint32_t host_lut[256];
  for (int v = 0; v < 256; ++v)
    host_lut[v] = table && bin_map[v] >= 0 ? 8u * (uint32_t)bin_map[v] : kNoBin;
  // Launches alternate between the two control blocks and each advances its
  // block's epoch by 2, so the epochs of neighbouring launches (which may
  // run at the same time with overlap on) never match each other's flags.
  const unsigned int epoch_alt = 1u;
  if (cudaMemset(p->ws, 0, o_cnt) != cudaSuccess ||
      cudaMemcpy(&p->ctrl_alt->epoch, &epoch_alt, sizeof(epoch_alt), cudaMemcpyHostToDevice) != cudaSuccess ||
      (table && cudaMemcpy(p->lut, host_lut, sizeof(host_lut), cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p->ws);
    delete p;
    return IHIST_ERR_CUDA;
  }
  for (int i = 0; i < 2; ++i) {
    if (cudaEventCreateWithFlags(&p->ev_uploaded[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_consumed[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(i == 0 ? &p->ev_queried : &p->ev_copied, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      for (int j = 0; j <= i; ++j) {
        if (p->ev_uploaded[j]) cudaEventDestroy(p->ev_uploaded[j]);
        if (p->ev_consumed[j]) cudaEventDestroy(p->ev_consumed[j]);
      }
      if (p->ev_queried) cudaEventDestroy(p->ev_queried);
      if (p->ev_copied) cudaEventDestroy(p->ev_copied);
      cudaFree(p->ws);
      delete p;
      return IHIST_ERR_CUDA;
    }
  }
  *out = p;
  return IHIST_OK;
}

extern "C" int ihist_plan_tuned(int h, int w, int nbins, int layout, const ihist_tune_t *tune,
                                ihist_plan_t *out) {
  return plan_create(h, w, nbins, layout, tune, nullptr, nullptr, out);
}

extern "C" int ihist_plan(int h, int w, int nbins, int layout, ihist_plan_t *out) {
  return plan_create(h, w, nbins, layout, nullptr, nullptr, nullptr, out);
}

extern "C" int ihist_plan_lut(int h, int w, int nbins, int layout, const int *bin_of_value,
                              const ihist_tune_t *tune, ihist_plan_t *out) {
  if (!bin_of_value || nbins < 1 || nbins > 256) return IHIST_ERR_INVALID_ARG;
  for (int v = 0; v < 256; ++v)
    if (bin_of_value[v] < -1 || bin_of_value[v] >= nbins) return IHIST_ERR_INVALID_ARG;
  if (tune && tune->bins_per_cta == 16) return IHIST_ERR_UNSUPPORTED;
  return plan_create(h, w, nbins, layout, tune, bin_of_value, nullptr, out);
}

extern "C" int ihist_edges_table(int nbins, const int *edges, int *bin_of_value) {
  if (!edges || !bin_of_value || nbins < 1 || nbins > 256) return IHIST_ERR_INVALID_ARG;
  if (edges[0] < 0 || edges[nbins] > 256) return IHIST_ERR_INVALID_ARG;
  for (int k = 0; k < nbins; ++k)
    if (edges[k] >= edges[k + 1]) return IHIST_ERR_INVALID_ARG;
  // bin k holds edges[k] <= v < edges[k + 1]; v walks up once, k with it
  int k = 0;
  for (int v = 0; v < 256; ++v) {
    while (k < nbins && v >= edges[k + 1]) ++k;
    bin_of_value[v] = (k < nbins && v >= edges[k]) ? k : -1;
  }
  return IHIST_OK;
}

extern "C" int ihist_plan_edges(int h, int w, int nbins, int layout, const int *edges,
                                const ihist_tune_t *tune, ihist_plan_t *out) {
  int table[256];
  const int rc = ihist_edges_table(nbins, edges, table);
  if (rc != IHIST_OK) return rc;
  return ihist_plan_lut(h, w, nbins, layout, table, tune, out);
}

int ihist::host::joint_bin_count(int channels, const int *bins_per_channel, int *nbins) {
  if (channels < 1 || channels > 4 || !bins_per_channel) return IHIST_ERR_INVALID_ARG;
  long long n = 1;
  for (int c = 0; c < channels; ++c) {
    if (bins_per_channel[c] < 1 || bins_per_channel[c] > 256) return IHIST_ERR_INVALID_ARG;
    n *= bins_per_channel[c];
    if (n > 256) return IHIST_ERR_UNSUPPORTED;
  }
  *nbins = (int)n;
  return IHIST_OK;
}

// Digit weights of the joint bin: channel 0 most significant.
static JointBins joint_bins(int channels, const int *bins_per_channel) {
  JointBins jb;
  std::memset(&jb, 0, sizeof(jb));
  jb.C = channels;
  for (int c = 0; c < channels; ++c) jb.mul[c] = bins_per_channel[c];
  int stride = 1;
  for (int c = channels - 1; c >= 0; --c) {
    jb.stride[c] = stride;
    stride *= jb.mul[c];
  }
  return jb;
}

int ihist::host::launch_joint_index(const uint8_t *in, long long pitch, int H, int W, int channels,
                                    const int *bins_per_channel, uint8_t *idx, long long idx_pitch, int sms,
                                    void *stream) {
  const JointBins jb = joint_bins(channels, bins_per_channel);
  const unsigned long long quads = (unsigned long long)H * (((unsigned)W + 3u) / 4u);
  const unsigned int grid =
      (unsigned int)std::min<unsigned long long>((quads + 255) / 256, (unsigned long long)sms * 8ull);
  joint_index_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(in, pitch, H, W, jb, idx, idx_pitch);
  return cudaGetLastError() == cudaSuccess ? IHIST_OK : IHIST_ERR_CUDA;
}

extern "C" int ihist_plan_joint(int h, int w, int channels, const int *bins_per_channel, int layout,
                                const ihist_tune_t *tune, ihist_plan_t *out) {
  int nbins = 0;
  const int rc = joint_bin_count(channels, bins_per_channel, &nbins);
  if (rc != IHIST_OK) return rc;
  if ((long long)w * channels > 65535) return IHIST_ERR_UNSUPPORTED;
  const JointBins jb = joint_bins(channels, bins_per_channel);
  return plan_create(h, w, nbins, layout, tune, nullptr, &jb, out);
}

extern "C" int ihist_plan_channels(ihist_plan_t p) {
  if (!p) return 0;
  return p->binning == kJoint ? p->joint.C : 1;
}

extern "C" int ihist_plan_get_tune(ihist_plan_t p, ihist_tune_t *out) {
  if (!p || !out) return IHIST_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->rows_per_band = p->R;
  out->bins_per_cta = p->G;
  out->chunks_per_warp = p->m;
  out->ctas_per_sm = p->ctas_per_sm;
  out->timeout_us = p->timeout_us;
  out->fault_skip_band = p->fault_skip_band + 1;  // 0 = off
  out->groups_per_cta = p->gpc;
  out->warps_per_cta = p->NW;
  out->overlap = p->overlap;
  return IHIST_OK;
}

extern "C" size_t ihist_workspace_bytes(ihist_plan_t p) { return p ? p->ws_bytes : 0; }

static int check_device(const ihist_plan_s *p) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return IHIST_ERR_CUDA;
  return dev == p->device ? IHIST_OK : IHIST_ERR_INVALID_ARG;
}

// TMA descriptor of the input frame: 2-D uint8 tensor {w, h} with row stride
// `pitch`, box {128 columns, R rows}, zero fill outside the frame.  Needs a
// 16-byte aligned base and pitch (the tensor-map rules) and w >= 128.
static const CUtensorMap *input_map(ihist_plan_s *p, const uint8_t *d_in, size_t pitch) {
  if (((uintptr_t)d_in & 15u) || (pitch & 15u) || p->W < kChunk || pitch >= (1ull << 40))
    return nullptr;
  for (auto &e : p->tmaps)
    if (e.ptr == d_in && e.pitch == pitch) return e.ok ? &e.map : nullptr;
  auto &e = p->tmaps[p->tmap_next];
  p->tmap_next = (p->tmap_next + 1) % 4;
  e.ptr = d_in;
  e.pitch = pitch;
  e.ok = false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return nullptr;
  cuuint64_t gdim[2] = {(cuuint64_t)p->W, (cuuint64_t)p->H};
  cuuint64_t gstride[1] = {(cuuint64_t)pitch};
  cuuint32_t box[2] = {(cuuint32_t)kChunk, (cuuint32_t)p->R};
  cuuint32_t estride[2] = {1u, 1u};
  e.ok = enc(&e.map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(d_in), gdim, gstride, box,
             estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  return e.ok ? &e.map : nullptr;
}

// One frame (ihist_compute).  Every scan is launched with programmatic
// stream serialization, so its CTAs may start while the previous kernel on
// the stream finishes; they take their first work item and then wait for
// that kernel (griddepcontrol.wait) before reading the frame, or, with
// overlap, only before their first store, after staging and counting their
// first band.
static int compute_frame(ihist_plan_s *p, const uint8_t *d_in, size_t in_pitch, uint32_t *d_out,
                         void *stream, bool overlap) {
  if (!p || !d_in || !d_out) return IHIST_ERR_INVALID_ARG;
  const size_t row_bytes = (size_t)p->W * (size_t)ihist_plan_channels(p);
  if (in_pitch < row_bytes || in_pitch > (size_t)LLONG_MAX) return IHIST_ERR_INVALID_ARG;
  if (((uintptr_t)d_out & 3u) != 0) return IHIST_ERR_INVALID_ARG;
  int rc = check_device(p);
  if (rc != IHIST_OK) return rc;
  if (p->binning == kJoint) {
    // joint bins first, one byte per pixel; the scan then reads that plane
    int rc2 = launch_joint_index(d_in, (long long)in_pitch, p->H, p->W, p->joint.C, p->joint.mul, p->idx,
                                 (long long)p->idx_pitch, p->sms, stream);
    if (rc2 != IHIST_OK) return rc2;
    d_in = p->idx;
    in_pitch = p->idx_pitch;
    overlap = false;  // the scan reads the plane the kernel just launched writes
  }
  const bool vec = (p->W % 4 == 0) && ((uintptr_t)d_out % 16 == 0);
  const CUtensorMap *tm = input_map(p, d_in, in_pitch);
  CUtensorMap tmap;
  if (tm)
    tmap = *tm;
  else
    std::memset(&tmap, 0, sizeof(tmap));
  FrameDesc f;
  std::memset(&f, 0, sizeof(f));
  f.in = d_in;
  f.pitch = (long long)in_pitch;
  f.out = d_out;
  f.H = p->H;
  f.W = p->W;
  f.B = p->B;
  f.layout = p->layout;
  f.qmul = p->binning == kJoint ? 256 : p->B;
  f.lut = p->lut;
  f.R = p->R;
  f.nbands = p->nbands;
  f.ngroups = p->ngroups;
  f.nchunks = p->nchunks;
  f.m = p->m;
  f.wpg = p->wpg;
  f.gpc = p->gpc;
  f.ngsets = p->ngsets;
  f.fault_skip_band = p->fault_skip_band;
  f.nitems = p->nitems;
  f.late_wait = overlap ? 1 : 0;
  f.agg_cnt = p->agg_cnt;
  f.agg_left = p->agg_left;
  f.incl = p->incl;
  f.flags = p->flags;
  f.nsegs = p->nsegs;
  f.cps = p->cps;
  f.hagg = p->hagg;
  f.hflags = p->hflags;
  const unsigned int grid =
      std::min<unsigned int>(p->nitems, (unsigned int)(p->ctas_per_sm * p->sms));
  ScanFn fn = scan_fn(p->G, mmax_for(p->m), tm != nullptr, vec, p->binning == kTable);
  const unsigned long long timeout_ns = (unsigned long long)p->timeout_us * 1000ull;
  Ctrl *ctrl = (p->launches++ & 1ull) ? p->ctrl_alt : p->ctrl;
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(p->NW * 32);
  cfg.dynamicSmemBytes = p->smem_bytes;
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, fn, f, tmap, ctrl, timeout_ns) != cudaSuccess) {
    cudaGetLastError();
    return IHIST_ERR_CUDA;
  }
  return IHIST_OK;
}

extern "C" int ihist_compute(ihist_plan_t p, const uint8_t *d_in, size_t in_pitch, uint32_t *d_out,
                             void *stream) {
  return compute_frame(p, d_in, in_pitch, d_out, stream, p && p->overlap != 0);
}

int ihist::host::launch_query(int H, int W, int B, int layout, int sms, Ctrl *ctrl, const uint32_t *d_hist,
                        const int32_t *d_rects, int n, uint32_t *d_hist_out, void *stream) {
  if (n < 0) return IHIST_ERR_INVALID_ARG;
  if (n == 0) return IHIST_OK;
  if (!d_hist || !d_rects || !d_hist_out) return IHIST_ERR_INVALID_ARG;
  if (((uintptr_t)d_hist & 3u) || ((uintptr_t)d_rects & 3u) || ((uintptr_t)d_hist_out & 3u))
    return IHIST_ERR_INVALID_ARG;
  if ((unsigned long long)n * (unsigned long long)B > 0x7fffffffull) return IHIST_ERR_UNSUPPORTED;
  const unsigned int total = (unsigned int)n * (unsigned int)B;
  const unsigned int threads = 256;
  const unsigned int grid =
      std::min<unsigned int>((total + threads - 1) / threads, (unsigned int)sms * 16u);
  // may start while the kernel before it finishes; waits for it first thing
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e =
      layout == IHIST_BIN_MAJOR
          ? cudaLaunchKernelEx(&cfg, query_kernel<0>, d_hist, H, W, B, d_rects, total, d_hist_out, ctrl)
      : layout == IHIST_PIXEL_MAJOR
          ? cudaLaunchKernelEx(&cfg, query_kernel<1>, d_hist, H, W, B, d_rects, total, d_hist_out, ctrl)
          : cudaLaunchKernelEx(&cfg, query_kernel<2>, d_hist, H, W, B, d_rects, total, d_hist_out, ctrl);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return IHIST_ERR_CUDA;
  }
  return IHIST_OK;
}

extern "C" int ihist_query(ihist_plan_t p, const uint32_t *d_hist, const int32_t *d_rects, int n,
                           uint32_t *d_hist_out, void *stream) {
  if (!p || n < 0) return IHIST_ERR_INVALID_ARG;
  if (n == 0) return IHIST_OK;
  int rc = check_device(p);
  if (rc != IHIST_OK) return rc;
  return launch_query(p->H, p->W, p->B, p->layout, p->sms, p->ctrl, d_hist, d_rects, n, d_hist_out,
                      stream);
}

// Scratch of ihist_query_sorted: row counts (zero between calls), row
// offsets, the corners' (y, x) in row order, each rectangle's four corner
// positions and the gathered corner values of one bin group.
struct SortedQueryWork {
  size_t o_cnt, o_off, o_pts, o_slot, o_val, bytes;
};

static SortedQueryWork sorted_query_work(int H, size_t n, int nb) {
  SortedQueryWork w;
  size_t off = 0;
  w.o_cnt = off;
  off = align_up(off + (size_t)H * 4, 256);
  w.o_off = off;
  off = align_up(off + ((size_t)H + 1) * 4, 256);
  w.o_pts = off;
  off = align_up(off + 4 * n * 4, 256);
  w.o_slot = off;
  off = align_up(off + n * 16, 256);
  w.o_val = off;
  off = align_up(off + 4 * n * (size_t)nb * 4, 256);
  w.bytes = off;
  return w;
}

static int sorted_group(int bins_per_pass) { return bins_per_pass == 0 ? 8 : bins_per_pass; }

extern "C" size_t ihist_query_work_bytes(ihist_plan_t p, int n, int bins_per_pass) {
  if (!p || n < 0 || (bins_per_pass != 0 && bins_per_pass != 4 && bins_per_pass != 8 && bins_per_pass != 16))
    return 0;
  return sorted_query_work(p->H, (size_t)n, sorted_group(bins_per_pass)).bytes;
}

extern "C" int ihist_query_sorted(ihist_plan_t p, const uint32_t *d_hist, const int32_t *d_rects, int n,
                                  uint32_t *d_hist_out, int bins_per_pass, void *d_work, size_t work_bytes,
                                  void *stream) {
  if (!p || n < 0) return IHIST_ERR_INVALID_ARG;
  if (bins_per_pass != 0 && bins_per_pass != 4 && bins_per_pass != 8 && bins_per_pass != 16)
    return IHIST_ERR_INVALID_ARG;
  if (n == 0) return IHIST_OK;
  if (!d_hist || !d_rects || !d_hist_out || !d_work) return IHIST_ERR_INVALID_ARG;
  if (((uintptr_t)d_hist & 3u) || ((uintptr_t)d_rects & 3u) || ((uintptr_t)d_hist_out & 3u) ||
      ((uintptr_t)d_work & 255u))
    return IHIST_ERR_INVALID_ARG;
  if (p->layout != IHIST_BIN_MAJOR) return IHIST_ERR_UNSUPPORTED;
  if ((unsigned long long)n * (unsigned long long)p->B > 0x7fffffffull || (unsigned long long)n >= (1ull << 29))
    return IHIST_ERR_UNSUPPORTED;
  const int nb = sorted_group(bins_per_pass);
  const SortedQueryWork w = sorted_query_work(p->H, (size_t)n, nb);
  if (work_bytes < w.bytes) return IHIST_ERR_INVALID_ARG;
  int rc = check_device(p);
  if (rc != IHIST_OK) return rc;
  char *base = static_cast<char *>(d_work);
  unsigned int *cnt = reinterpret_cast<unsigned int *>(base + w.o_cnt);
  unsigned int *off = reinterpret_cast<unsigned int *>(base + w.o_off);
  uint32_t *pts = reinterpret_cast<uint32_t *>(base + w.o_pts);
  uint4 *slot = reinterpret_cast<uint4 *>(base + w.o_slot);
  uint32_t *val = reinterpret_cast<uint32_t *>(base + w.o_val);
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned int un = (unsigned int)n;
  const unsigned int cap = (unsigned int)p->sms * 16u;
  const unsigned int g_rect = std::min<unsigned int>((un + 255u) / 256u, cap);
  const unsigned int g_pts = std::min<unsigned int>((unsigned int)(((unsigned long long)un * 4ull + 255ull) / 256ull), cap);
  if (cudaMemsetAsync(cnt, 0, (size_t)p->H * 4, s) != cudaSuccess) return IHIST_ERR_CUDA;
  corner_count_kernel<<<g_rect, 256, 0, s>>>(d_rects, un, p->H, p->W, cnt, p->ctrl);
  row_offsets_kernel<<<1, 1024, 0, s>>>(cnt, p->H, off);
  corner_scatter_kernel<<<g_rect, 256, 0, s>>>(d_rects, un, p->H, p->W, cnt, off, pts, slot);
  for (int b0 = 0; b0 < p->B; b0 += nb) {
    const int cur = std::min(nb, p->B - b0);
    const unsigned int g_comb = std::min<unsigned int>(
        (unsigned int)(((unsigned long long)un * nb + 255ull) / 256ull), cap);
    switch (nb) {
      case 4:
        corner_gather_kernel<4><<<g_pts, 256, 0, s>>>(d_hist, p->H, p->W, b0, cur, pts, off, val);
        corner_combine_kernel<4><<<g_comb, 256, 0, s>>>(slot, un, p->B, b0, cur, val, d_hist_out);
        break;
      case 8:
        corner_gather_kernel<8><<<g_pts, 256, 0, s>>>(d_hist, p->H, p->W, b0, cur, pts, off, val);
        corner_combine_kernel<8><<<g_comb, 256, 0, s>>>(slot, un, p->B, b0, cur, val, d_hist_out);
        break;
      default:
        corner_gather_kernel<16><<<g_pts, 256, 0, s>>>(d_hist, p->H, p->W, b0, cur, pts, off, val);
        corner_combine_kernel<16><<<g_comb, 256, 0, s>>>(slot, un, p->B, b0, cur, val, d_hist_out);
        break;
    }
  }
  return cudaGetLastError() == cudaSuccess ? IHIST_OK : IHIST_ERR_CUDA;
}

extern "C" int ihist_window_search(ihist_plan_t p, const uint32_t *d_hist, const uint32_t *d_target, int win_h,
                                   int win_w, int stride, uint32_t *d_scores, unsigned long long *d_best,
                                   void *stream) {
  if (!p || !d_hist || !d_target || (!d_scores && !d_best)) return IHIST_ERR_INVALID_ARG;
  if (win_h < 1 || win_w < 1 || win_h > p->H || win_w > p->W || stride < 1) return IHIST_ERR_INVALID_ARG;
  if (((uintptr_t)d_hist & 3u) || ((uintptr_t)d_target & 3u) || ((uintptr_t)d_scores & 3u) ||
      ((uintptr_t)d_best & 7u))
    return IHIST_ERR_INVALID_ARG;
  if (p->layout == IHIST_QUAD_MAJOR) return IHIST_ERR_UNSUPPORTED;
  int rc = check_device(p);
  if (rc != IHIST_OK) return rc;
  if (d_best && cudaMemsetAsync(d_best, 0, sizeof(unsigned long long), (cudaStream_t)stream) != cudaSuccess)
    return IHIST_ERR_CUDA;
  const int ny = (p->H - win_h) / stride + 1, nx = (p->W - win_w) / stride + 1;
  const long long total = (long long)ny * nx;
  const unsigned int threads = 256;
  const size_t smem = (size_t)p->B * sizeof(uint32_t);
  cudaStream_t s = (cudaStream_t)stream;
  if (p->layout == IHIST_BIN_MAJOR) {
    const unsigned int grid =
        (unsigned int)std::min<long long>((total + threads - 1) / threads, (long long)p->sms * 8);
    // the map-only search keeps the plain kernel (no best-window tracking in its loop)
    if (d_best)
      window_kernel_bin_major<true><<<grid, threads, smem, s>>>(d_hist, p->H, p->W, p->B, d_target, win_h, win_w,
                                                                stride, ny, nx, d_scores, d_best);
    else
      window_kernel_bin_major<false><<<grid, threads, smem, s>>>(d_hist, p->H, p->W, p->B, d_target, win_h, win_w,
                                                                 stride, ny, nx, d_scores, nullptr);
  } else {
    const unsigned int grid =
        (unsigned int)std::min<long long>((total + threads / 32 - 1) / (threads / 32), (long long)p->sms * 8);
    if (d_best)
      window_kernel_pixel_major<true><<<grid, threads, smem, s>>>(d_hist, p->H, p->W, p->B, d_target, win_h, win_w,
                                                                  stride, ny, nx, d_scores, d_best);
    else
      window_kernel_pixel_major<false><<<grid, threads, smem, s>>>(d_hist, p->H, p->W, p->B, d_target, win_h,
                                                                   win_w, stride, ny, nx, d_scores, nullptr);
  }
  if (cudaGetLastError() != cudaSuccess) return IHIST_ERR_CUDA;
  return IHIST_OK;
}

extern "C" int ihist_sequence_host(ihist_plan_t p, const uint8_t *h_frames, size_t frame_stride,
                                   int nframes, uint8_t *d_slots, uint32_t *d_outs, int nouts,
                                   const int32_t *d_rects, int nrects, uint32_t *d_query,
                                   uint32_t *h_query_out, void *stream, void *copy_stream) {
  if (!p || nframes < 0 || nouts < 1 || nrects < 0) return IHIST_ERR_INVALID_ARG;
  if (nframes == 0) return IHIST_OK;
  const size_t row_bytes = (size_t)p->W * (size_t)ihist_plan_channels(p);
  const size_t fbytes = (size_t)p->H * row_bytes;
  if (!h_frames || !d_slots || !d_outs || frame_stride < fbytes) return IHIST_ERR_INVALID_ARG;
  if (nrects > 0 && (!d_rects || !d_query || !h_query_out)) return IHIST_ERR_INVALID_ARG;
  int rc = check_device(p);
  if (rc != IHIST_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream, cs = (cudaStream_t)copy_stream;
  const size_t obytes = ihist_output_bytes(p->H, p->W, p->B);
  const size_t qwords = (size_t)nrects * (size_t)p->B;
  // frame i's upload into slot i % 2, once the compute that read the slot
  // (frame i-2) is done
  auto upload = [&](int i) -> int {
    const int slot = i & 1;
    if (i >= 2 && cudaStreamWaitEvent(cs, p->ev_consumed[slot], 0) != cudaSuccess) return IHIST_ERR_CUDA;
    if (cudaMemcpyAsync(d_slots + (size_t)slot * fbytes, h_frames + (size_t)i * frame_stride, fbytes,
                        cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaEventRecord(p->ev_uploaded[slot], cs) != cudaSuccess)
      return IHIST_ERR_CUDA;
    return IHIST_OK;
  };
  rc = upload(0);
  if (rc != IHIST_OK) return rc;
  for (int i = 0; i < nframes; ++i) {
    const int slot = i & 1;
    // frame i+1's upload goes on the copy stream before frame i's copy back,
    // so it overlaps frame i's compute
    if (i + 1 < nframes) {
      rc = upload(i + 1);
      if (rc != IHIST_OK) return rc;
    }
    if (cudaStreamWaitEvent(s, p->ev_uploaded[slot], 0) != cudaSuccess) return IHIST_ERR_CUDA;
    uint32_t *d_out = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(d_outs) +
                                                   (size_t)(i % nouts) * obytes);
    // frames arrive by copy, so no kernel before a compute writes its frame
    rc = compute_frame(p, d_slots + (size_t)slot * fbytes, row_bytes, d_out, stream, true);
    if (rc != IHIST_OK) return rc;
    if (cudaEventRecord(p->ev_consumed[slot], s) != cudaSuccess) return IHIST_ERR_CUDA;
    if (nrects > 0) {
      // the rows go back on the copy stream, off the compute stream, so the
      // next frame's scan follows this query directly; d_query is reused
      // once the previous frame's rows have left it
      if (i > 0 && cudaStreamWaitEvent(s, p->ev_copied, 0) != cudaSuccess) return IHIST_ERR_CUDA;
      rc = ihist_query(p, d_out, d_rects, nrects, d_query, stream);
      if (rc != IHIST_OK) return rc;
      if (cudaEventRecord(p->ev_queried, s) != cudaSuccess || cudaStreamWaitEvent(cs, p->ev_queried, 0) != cudaSuccess ||
          cudaMemcpyAsync(h_query_out + (size_t)i * qwords, d_query, qwords * sizeof(uint32_t),
                          cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
          cudaEventRecord(p->ev_copied, cs) != cudaSuccess)
        return IHIST_ERR_CUDA;
    }
  }
  // a caller that synchronises `stream` finds every row on the host
  if (nrects > 0 && cudaStreamWaitEvent(s, p->ev_copied, 0) != cudaSuccess) return IHIST_ERR_CUDA;
  // later work on the copy stream must not overtake this sequence's computes
  if (cudaStreamWaitEvent(cs, p->ev_consumed[(nframes - 1) & 1], 0) != cudaSuccess) return IHIST_ERR_CUDA;
  return IHIST_OK;
}

int ihist::host::read_status(Ctrl *ctrl, void *stream, int *device_status) {
  cudaStream_t s = (cudaStream_t)stream;
  int v = 0;
  if (cudaStreamSynchronize(s) != cudaSuccess) return IHIST_ERR_CUDA;
  if (cudaMemcpy(&v, &ctrl->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return IHIST_ERR_CUDA;
  if (cudaMemset(&ctrl->status, 0, sizeof(int)) != cudaSuccess) return IHIST_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return IHIST_ERR_CUDA;
  *device_status = v;
  return IHIST_OK;
}

extern "C" int ihist_status(ihist_plan_t p, void *stream, int *device_status) {
  if (!p || !device_status) return IHIST_ERR_INVALID_ARG;
  int rc = check_device(p);
  if (rc != IHIST_OK) return rc;
  int st_alt = 0;
  rc = read_status(p->ctrl_alt, stream, &st_alt);
  if (rc != IHIST_OK) return rc;
  rc = read_status(p->ctrl, stream, device_status);  // also the queries' status
  if (rc == IHIST_OK && *device_status == IHIST_OK) *device_status = st_alt;
  return rc;
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
  if (p->ev_queried) cudaEventDestroy(p->ev_queried);
  if (p->ev_copied) cudaEventDestroy(p->ev_copied);
  cudaFree(p->ws);
  if (prev != p->device && prev >= 0) cudaSetDevice(prev);
  delete p;
}

/*
 * ihist.h -- C ABI of libihist.so, a GB300 (sm_103a) integral-histogram
 * engine for the method of Poostchi et al., "Fast Integral Histogram
 * Computations on GPU for Real-Time Video Analytics" (arXiv 1711.01919).
 *
 * What is computed
 *   For a uint8 frame I of h rows and w columns and B uniform bins
 *   Q(v) = floor(v * B / 256), the integral histogram (Eq. 1, Sec. 2.1) is
 *       H[b][y][x] = #{ (x', y') : x' <= x, y' <= y, Q(I[y'][x']) == b }
 *   -- the per-bin inclusive 2-D prefix count that Algorithm 1 builds with
 *   H(k,x,y) = H(k,x-1,y) + H(k,x,y-1) - H(k,x-1,y-1) + Q(k, I(x,y)).
 *   Row index y runs top to bottom, column index x left to right, origin at
 *   the top-left corner (Fig. 1).  Counts are exact uint32 ("4 byte integer",
 *   Sec. 4.6).  The region histogram of an inclusive rectangle is Eq. 2:
 *       h(R, b) = H[y1][x1] - H[y0-1][x1] - H[y1][x0-1] + H[y0-1][x0-1]
 *   with every term whose index is -1 taken as zero.
 *
 * Conventions for every entry point
 *   - Pointers named d_* are DEVICE pointers on the plan's device, owned by
 *     the caller; the library never frees them.  h_* pointers are host
 *     pointers.  Streams are passed as `void *` holding a cudaStream_t (NULL =
 *     the legacy default stream).
 *   - Work is enqueued asynchronously on the stream; the return code reports
 *     host-side validation and launch errors only.  Errors detected on the
 *     device (a look-back wait that ran out of time, a bad rectangle) are
 *     latched in the plan's device status word and read with ihist_status().
 *   - A plan owns its workspace (allocated once by ihist_plan*); compute and
 *     query calls allocate nothing.  One plan must not be used by two
 *     launches that may run concurrently (two streams); create one plan per
 *     stream.  Calls on one plan from several host threads need external
 *     locking.
 *   - Return codes are the IHIST_* values below; nothing aborts or traps.
 */
#ifndef IHIST_H
#define IHIST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return / status codes. */
enum {
  IHIST_OK = 0,
  IHIST_ERR_INVALID_ARG = 1,      /* bad size, pointer, alignment or layout */
  IHIST_ERR_UNSUPPORTED = 2,      /* valid request outside what this build handles */
  IHIST_ERR_OOM = 3,              /* workspace allocation failed */
  IHIST_ERR_CUDA = 4,             /* a CUDA runtime call failed */
  IHIST_ERR_LOOKBACK_TIMEOUT = 5, /* device: a carry wait ran out of time (result invalid) */
  IHIST_ERR_BAD_RECT = 6,         /* device: a query rectangle was out of range (its row is zero) */
  IHIST_ERR_CHECK_FAILED = 7      /* device, checked builds only: an out-of-range access was caught and
                                     skipped (result invalid; a library bug) */
};

/* Output layouts of H.  Bin-major is the paper's b x h x w tensor mapped
 * row-major to 1-D (Sec. 3.1, Fig. 2): H[b][y][x] at ((b*h + y)*w + x).
 * Pixel-major keeps each pixel's B counts together: H[y][x][b] at
 * ((y*w + x)*B + b), so a region query reads four contiguous vectors.
 * Quad-major keeps each pixel's counts of four consecutive bins together:
 * H[b/4][y][x][b%4] at (((b/4)*h + y)*w + x)*4 + b%4 (B a multiple of 4,
 * else IHIST_ERR_INVALID_ARG) -- one 16-byte word per pixel and quad, so a
 * region query reads a quarter of the bin-major layout's DRAM sectors
 * (64 x 1080p x 64: queries 0.25 instead of 0.41 ms, the scan 5.5 instead of
 * 5.2 ms).  Not a layout of the paper; ihist_window_search does not take
 * it (IHIST_ERR_UNSUPPORTED). */
enum { IHIST_BIN_MAJOR = 0, IHIST_PIXEL_MAJOR = 1, IHIST_QUAD_MAJOR = 2 };

typedef struct ihist_plan_s *ihist_plan_t;

/* Tile shape of the fused scan kernel.  Zero fields take the library's
 * default for the frame shape.
 *   rows_per_band   R, rows one CTA owns (1..255)
 *   bins_per_cta    G, bins one CTA owns (4, 8 or 16; default 4, or for
 *                   pixel-major output 16 (8 with fewer than 16 bins or
 *                   more than 4096 columns): longer contiguous pieces of
 *                   each pixel's record)
 *   chunks_per_warp m, 128-column chunks one warp owns (1, 2, 4 or 8;
 *                   at most 2 with bins_per_cta 16)
 *   groups_per_cta  bin groups one CTA serves side by side (warps = groups
 *                   x ceil(ceil(w/128)/m), at most 16 in all; frames split
 *                   into width segments count the warps of one segment);
 *                   narrow frames fill a CTA this way.  Pixel-major output
 *                   with every group in the CTA (8 or 16 bins per CTA,
 *                   nbins / 4 a power of two) stores whole pixel records:
 *                   the default for 2 to 4 groups when those items still
 *                   fill a wave of CTAs, and in batches
 *   ctas_per_sm     persistent grid = ctas_per_sm x SMs (0 = occupancy limit)
 *   timeout_us      limit of each carry wait before it gives up and latches
 *                   IHIST_ERR_LOOKBACK_TIMEOUT (default 2,000,000 us)
 *   fault_skip_band test hook, 0 (or negative) = off: a value k >= 1
 *                   makes the CTAs of band k-1 publish no carries, so the
 *                   band below must time out (in every frame of a batch).
 *                   Used only to test failure detection; never set it
 *                   otherwise.  A zero-initialised struct leaves it off.
 *   warps_per_cta   batched launches: warps per CTA (4, 8 or 16; default
 *                   8, or 16 for pixel-major batches with 8 bins per CTA
 *                   and for frames wider than 8 warps can cover).  A frame
 *                   wider than 4 x warps_per_cta chunks of 128 columns (2 x
 *                   with 16 bins per CTA) is split into width segments.
 *                   Plans: an upper bound on the warps of one CTA (1..16,
 *                   0 = 16; frames wider than it x chunks_per_warp chunks
 *                   split into width segments); ihist_plan_get_tune reports
 *                   the warps the plan uses, which recreates the same
 *                   tiling when passed back.
 *   overlap         plans: every ihist_compute (and ihist_query) is launched
 *                   with programmatic dependent launch, so its CTAs may
 *                   start while the kernel launched just before it on the
 *                   stream is still finishing.  By default (0) a scan's CTAs
 *                   take their first work item and then wait for that kernel
 *                   to complete before reading anything of the frame, which
 *                   is always safe.  1 = overlap further: they stage and
 *                   count their first band of the frame before waiting (every
 *                   store still waits), so the frame (d_in) must not be
 *                   written by the kernel launched just before ihist_compute
 *                   on the same stream (a copy, an event wait or another
 *                   kernel in between makes it safe again).  1080p x 64 per
 *                   frame, back to back: 115 us plain launches, 104 us with
 *                   the default, 99 us with 1.  Joint plans treat 1 as 0
 *                   (their scan reads the joint-bin plane the kernel before
 *                   it writes); ihist_sequence_host always uses 1 (its
 *                   frames arrive by copy).  Batches ignore it.            */
typedef struct {
  int rows_per_band;
  int bins_per_cta;
  int chunks_per_warp;
  int ctas_per_sm;
  unsigned int timeout_us;
  int fault_skip_band;
  int groups_per_cta;
  int warps_per_cta;
  int overlap;
  int reserved;
} ihist_tune_t;

/* Create a plan for frames of h rows x w columns and nbins bins in the given
 * layout, with default tiling.  Limits: 1 <= h, w <= 65535, h*w < 2^32,
 * 1 <= nbins <= 256.  A frame wider than one CTA's warps cover (16 warps x
 * chunks_per_warp x 128 columns) has each band split into width segments of
 * equal chunk counts, one work item each; a segment adds the per-row bin
 * totals that the segments to its left publish right after counting (Eq. 1's
 * row sums split at the segment edges).  Allocates the plan's device
 * workspace on the current device.  *out is set only on IHIST_OK. */
int ihist_plan(int h, int w, int nbins, int layout, ihist_plan_t *out);

/* As ihist_plan with explicit tiling (NULL = defaults). */
int ihist_plan_tuned(int h, int w, int nbins, int layout, const ihist_tune_t *tune,
                     ihist_plan_t *out);

/* Other bin structures (Sec. 1 / Sec. 2.1: the paper leaves the binning Q
 * of Eq. 1 open).  Same limits, tiling, workspace and error rules as
 * ihist_plan_tuned (tune may be NULL); bins_per_cta must be 4 or 8.
 *   ihist_plan_lut    any value -> bin map: bin_of_value is a HOST array of
 *                     256 ints, bin_of_value[v] in [0, nbins) is the bin of
 *                     intensity v and -1 puts v in no bin (such pixels count
 *                     nowhere).  The table is copied into the plan.
 *   ihist_plan_edges  bins by edges: edges is a HOST array of nbins + 1
 *                     strictly increasing ints in [0, 256]; bin k holds the
 *                     intensities edges[k] <= v < edges[k+1] and values
 *                     outside [edges[0], edges[nbins]) are in no bin.
 * The map is applied inside the scan kernel from a 256-entry table in
 * shared memory; ihist_compute, ihist_query and ihist_sequence_host work on
 * these plans unchanged.  IHIST_ERR_INVALID_ARG for an entry out of range or
 * edges that do not increase. */
int ihist_plan_lut(int h, int w, int nbins, int layout, const int *bin_of_value,
                   const ihist_tune_t *tune, ihist_plan_t *out);
int ihist_plan_edges(int h, int w, int nbins, int layout, const int *edges,
                     const ihist_tune_t *tune, ihist_plan_t *out);

/* The value -> bin table of bins by edges (Sec. 2.1 leaves the binning Q of
 * Eq. 1 open; this is the table ihist_plan_edges bins with).  edges: HOST
 * array of nbins + 1 strictly increasing ints in [0, 256] (1 <= nbins <=
 * 256); bin_of_value: HOST array of 256 ints, filled with the bin k of each
 * intensity v, edges[k] <= v < edges[k+1], or -1 for values outside
 * [edges[0], edges[nbins]).  Pass the table as ihist_frame_t.bin_of_value to
 * bin a batch frame by edges.  Host-only (no device, no allocation);
 * IHIST_ERR_INVALID_ARG for a NULL pointer, nbins out of range or edges that
 * do not increase within [0, 256]. */
int ihist_edges_table(int nbins, const int *edges, int *bin_of_value);

/* Joint histogram of a multi-channel frame (the higher-dimensional, e.g.
 * colour, histograms of Sec. 1 / Sec. 2.1).  Frames hold `channels` (1..4)
 * interleaved bytes per pixel: pixel (y, x) channel c at
 * d_in[y * in_pitch + x * channels + c], in_pitch >= w * channels.  Channel
 * c is cut into bins_per_channel[c] uniform bins, q_c = floor(v_c * B_c /
 * 256), and the pixel's bin is the mixed-radix number
 * k = (...(q_0 * B_1 + q_1) * B_2 + ...) + q_{C-1}   (channel 0 most
 * significant), so the plan has nbins = prod B_c planes, at most 256
 * (IHIST_ERR_UNSUPPORTED above that or when w * channels > 65535).
 * bins_per_channel is a HOST array of `channels` ints in 1..256.  Each
 * ihist_compute first writes the pixels' joint bins into a plane the plan
 * owns (h x w bytes, one extra read of the frame), then runs the scan on it;
 * the output is H[k][y][x] (or pixel-major) exactly as for nbins uniform
 * bins.  ihist_query and ihist_sequence_host (frames of h * w * channels
 * bytes) work unchanged. */
int ihist_plan_joint(int h, int w, int channels, const int *bins_per_channel, int layout,
                     const ihist_tune_t *tune, ihist_plan_t *out);

/* Bytes per pixel of the plan's input frames: the channel count of a joint
 * plan, 1 otherwise (0 for a NULL plan). */
int ihist_plan_channels(ihist_plan_t plan);

/* The tiling a plan resolved to (all fields filled). */
int ihist_plan_get_tune(ihist_plan_t plan, ihist_tune_t *out);

/* Device workspace bytes the plan holds (carry vectors, flags, control). */
size_t ihist_workspace_bytes(ihist_plan_t plan);

/* Bytes of one integral histogram: h * w * nbins * 4. */
size_t ihist_output_bytes(int h, int w, int nbins);

/* Integral histogram of one frame (Eq. 1; fused quantise, row scan, column
 * scan and carry passing).  d_in: h rows of w bytes (w * channels for a
 * joint plan), row stride in_pitch (>= that) bytes.  d_out:
 * ihist_output_bytes(h, w, nbins) bytes in the plan's layout; every word is
 * written exactly once.  The fast path wants d_in and in_pitch 4-byte
 * aligned and d_out 16-byte aligned with w % 4 == 0; anything else takes a
 * slower element-wise path with the same result.
 * Stand-alone use (results wanted in host memory, Alg. 6's copy back,
 * Sec. 4.3-4.4): d_out may be page-locked host memory the device can address
 * (cudaHostAlloc, or cudaHostRegister'ed with mapping).  The kernel's stores
 * then cross the CPU-GPU link themselves, so no device copy of H and no
 * separate transfer is needed; the frame rate is that of the link (on a
 * GB300 about the same as a device-to-host copy of the same bytes).  Use
 * the bin-major layout there: pixel-major stores are too scattered for the
 * link.  The caller synchronises `stream` before reading d_out on the host. */
int ihist_compute(ihist_plan_t plan, const uint8_t *d_in, size_t in_pitch, uint32_t *d_out,
                  void *stream);

/* Region histograms by Eq. 2.  d_hist: an integral histogram made by this
 * plan's layout and shape.  d_rects: n x {x0, y0, x1, y1} int32, inclusive,
 * x = column.  d_hist_out: n x nbins uint32, row i = histogram of rect i.
 * A rectangle with x0 > x1, y0 > y1 or a corner outside the frame yields a
 * zero row and latches IHIST_ERR_BAD_RECT.  n == 0 is a no-op.  The
 * launch may start while the kernel before it on the stream finishes when
 * that kernel is one of this library's (a scan): it then reads d_rects at
 * once (no library kernel writes rectangles) and d_hist only after that
 * kernel completed.  After any other kernel it starts when that one ends. */
int ihist_query(ihist_plan_t plan, const uint32_t *d_hist, const int32_t *d_rects, int n,
                uint32_t *d_hist_out, void *stream);

/* Region histograms by Eq. 2 for large batches of rectangles on a bin-major
 * H, with the corner lookups put in row order first (same results as
 * ihist_query, word for word).  ihist_query reads each corner word where it
 * lies, so random rectangles on a large bin-major H cost one DRAM line per
 * 4-byte corner; here the corners of all n rectangles are bucketed by row
 * (a counting sort, once per call), then each group of bins_per_pass bins
 * reads them bucket by bucket, so the corners of a row share the lines they
 * fall on, and a second pass combines each rectangle's four corners.
 *   bins_per_pass  bins gathered per pass: 4, 8 or 16 (0 = 8)
 *   d_work         device scratch of ihist_query_work_bytes(plan, n,
 *                  bins_per_pass) bytes, 256-byte aligned, owned by the
 *                  caller; about 32 + 16 * bins_per_pass bytes per rectangle
 *                  plus 8 per frame row.  Its contents need not be kept
 *                  between calls; two calls sharing it must not overlap.
 * Other arguments and the bad-rectangle rule as for ihist_query.  Bin-major
 * plans only (IHIST_ERR_UNSUPPORTED otherwise); n < 2^29;
 * IHIST_ERR_INVALID_ARG if work_bytes is too small.  Five kinds of launch on
 * `stream` (count, offsets, scatter, then a gather and a combine per group
 * of bins); allocates nothing. */
size_t ihist_query_work_bytes(ihist_plan_t plan, int n, int bins_per_pass);
int ihist_query_sorted(ihist_plan_t plan, const uint32_t *d_hist, const int32_t *d_rects, int n,
                       uint32_t *d_hist_out, int bins_per_pass, void *d_work, size_t work_bytes,
                       void *stream);

/* Sliding-window histogram search over a resident integral histogram (the
 * detection / tracking use of Sec. 1).  Window (i, j) covers rows
 * i*stride .. i*stride + win_h - 1 and columns j*stride .. j*stride + win_w - 1
 * for i < ny = (h - win_h) / stride + 1 and j < nx = (w - win_w) / stride + 1
 * (only windows inside the frame).  Its histogram comes from Eq. 2 and its
 * score is the histogram intersection sum_b min(h_b, target_b), an exact
 * integer <= win_h * win_w.
 *   d_hist    an integral histogram made with this plan's shape and layout
 *             (pixel-major reads each corner as one contiguous vector and is
 *             the faster layout here)
 *   d_target  nbins uint32 counts, device
 *   d_scores  ny * nx uint32, row-major [i][j], device; may be NULL
 *   d_best    one uint64, device, 8-byte aligned; may be NULL: receives the
 *             best window as (score << 32) | (0xffffffff - (i * nx + j)),
 *             the highest score and among equal scores the first window in
 *             row-major order (0 if there is none); the call clears it first
 * At least one of d_scores and d_best must be given.  IHIST_ERR_INVALID_ARG
 * if the window does not fit the frame or stride < 1.  Asynchronous on
 * stream; allocates nothing. */
int ihist_window_search(ihist_plan_t plan, const uint32_t *d_hist, const uint32_t *d_target, int win_h,
                        int win_w, int stride, uint32_t *d_scores, unsigned long long *d_best, void *stream);

/* The paper's own GPU mappings, rebuilt on this GPU as comparison kernels
 * for measuring the fused look-back design against them (not a fast path):
 *   IHIST_MAPPING_CW_STS  Sec. 3.3 / Alg. 3: one-hot tensor, one row-scan
 *                         launch, 3-D transpose, row scan, transpose back
 *   IHIST_MAPPING_CW_TIS  Sec. 3.4 / Alg. 4: one-hot tensor, a launch per
 *                         vertical strip of 32-column tiles (row scans),
 *                         then a launch per horizontal strip (column scans)
 *   IHIST_MAPPING_WF_TIS  Sec. 3.5 / Alg. 5 / Eq. 6: one-hot tensor, then a
 *                         launch per anti-diagonal of 32 x 32 tiles, each
 *                         tile scanned in shared memory and offset by the
 *                         final column to its left and row above
 * All three write exactly the H of Eq. 1, bin-major, into d_out (which also
 * holds the one-hot tensor while they run).  d_work: a device buffer of
 * ihist_mapping_workspace_bytes() bytes (0, and d_work may be NULL, for
 * the tiled mappings).  Shape limits as ihist_plan; asynchronous on stream.
 * IHIST_ERR_INVALID_ARG for an unknown mapping or a bad shape or pointer. */
enum { IHIST_MAPPING_CW_STS = 1, IHIST_MAPPING_CW_TIS = 2, IHIST_MAPPING_WF_TIS = 3 };
size_t ihist_mapping_workspace_bytes(int mapping, int h, int w, int nbins);
int ihist_mapping_compute(int mapping, int h, int w, int nbins, const uint8_t *d_in, size_t in_pitch,
                          uint32_t *d_out, void *d_work, void *stream);

/* A sequence of frames from HOST memory (the dual-buffered pipeline of
 * Algorithm 6, Sec. 4.4): frame i+1 is uploaded on copy_stream into one of
 * two device input slots while frame i is computed on stream.
 *   h_frames      nframes frames of h x w bytes, frame i at h_frames +
 *                 i * frame_stride, rows packed (pitch w).  Page-locked
 *                 memory is needed for the copies to overlap compute.
 *   d_slots       2 * h * w bytes of device memory (the upload ring).
 *   d_outs        nouts integral histograms (ihist_output_bytes each, back
 *                 to back); frame i is written to slot i % nouts.
 *   d_rects, nrects  optional (nrects may be 0): rectangles queried on every
 *                 frame's histogram (Eq. 2) into d_query (nrects * nbins
 *                 uint32) and copied to h_query_out + i * nrects * nbins.
 * Frame i+1's upload is issued before frame i's rows go back, and the rows
 * go back on copy_stream, so the compute stream runs scan, query, scan, ...
 * (the scans overlapped, see tune.overlap).  All work is enqueued; the call
 * returns before it finishes.  The caller synchronises `stream` (which is
 * made to wait for the last copy and compute) before reading h_query_out or
 * reusing h_frames.  Uses events the plan owns, so it must not overlap
 * another sequence call on the same plan. */
int ihist_sequence_host(ihist_plan_t plan, const uint8_t *h_frames, size_t frame_stride,
                        int nframes, uint8_t *d_slots, uint32_t *d_outs, int nouts,
                        const int32_t *d_rects, int nrects, uint32_t *d_query,
                        uint32_t *h_query_out, void *stream, void *copy_stream);

/* ---- Batches: many frames of uneven size in one persistent launch -------
 *
 * A batch is a work-list over several frames (any mix of shapes, bin counts
 * and layouts): one launch computes every frame's integral histogram, so the
 * ramp and tail of a launch are paid once per batch instead of once per
 * frame.  The same fused kernel runs on each frame (Eq. 1; Sec. 4.4's image
 * sequences as one launch), and results equal ihist_compute's word for word.
 * The launch needs no host-side reset between calls, so it can be captured
 * in a CUDA graph and replayed. */
typedef struct ihist_batch_s *ihist_batch_t;

/* One frame of a batch.  d_in: h rows of w bytes, row stride in_pitch;
 * d_out: ihist_output_bytes(h, w, nbins) bytes in `layout`.  Both are device
 * pointers the caller owns and keeps valid while the batch may run.
 * bin_of_value: NULL for uniform bins, or a HOST array of 256 ints as for
 * ihist_plan_lut (bin of each intensity in [0, nbins), -1 = no bin; bins by
 * edges are such a table), read during ihist_batch_plan / ihist_batch_set_io
 * and copied into the batch.
 * channels: 0 or 1 for one byte per pixel; 2..4 for a joint-bin frame as
 * for ihist_plan_joint: d_in holds `channels` interleaved bytes per pixel
 * (in_pitch >= w * channels), channel c is cut into bins_per_channel[c]
 * uniform bins (channel 0 the most significant digit) and nbins must equal
 * their product; bin_of_value must then be NULL.  The batch computes each
 * joint frame's joint-bin plane (one byte per pixel, in its workspace) just
 * before the scan.  A zero-initialised struct is a uniform one-channel
 * frame. */
typedef struct {
  int h, w, nbins, layout;
  const uint8_t *d_in;
  size_t in_pitch;
  uint32_t *d_out;
  const int *bin_of_value;
  int channels;
  int bins_per_channel[4];
} ihist_frame_t;

/* Plan a batch of n >= 1 frames (limits per frame as for ihist_plan); the
 * frames also fix the capacity of the batch's n slots (see
 * ihist_batch_set_io).  tune may be NULL; its bins_per_cta (4, 8 or 16;
 * default 4, or 16 / 8 when a frame is pixel-major), rows_per_band and
 * warps_per_cta apply to every frame; chunks per warp and groups per CTA
 * are chosen per frame to fill the CTA's warps.  Frames wider than
 * 4 x warps_per_cta chunks of 128 columns (2 x with 16 bins per CTA) are
 * split into width segments as in ihist_plan.  Frames bound
 * later by ihist_batch_set_io keep within the launch shape the planned
 * frames fixed (chunks per warp, carry width per CTA), which may leave some
 * of a narrower frame's CTA idle.  If any planned frame has a bin table
 * (bin_of_value), the batch is a table batch: every frame bins through a
 * per-slot table in shared memory (uniform frames get the table of
 * floor(v * nbins / 256)), bins_per_cta is 4 or 8 (default 8 when a frame is
 * pixel-major; 16 gives IHIST_ERR_UNSUPPORTED) and later bindings may mix
 * table and uniform frames; a batch planned without tables refuses tables
 * later (IHIST_ERR_UNSUPPORTED).  A table entry outside [-1, nbins) gives
 * IHIST_ERR_INVALID_ARG.  A launch works through the bound frames largest
 * output first (results do not depend on the order).  Allocates the batch's
 * device workspace and pinned staging buffers. */
int ihist_batch_plan(const ihist_frame_t *frames, int n, const ihist_tune_t *tune,
                     ihist_batch_t *out);

/* The launch shape a batch resolved to: rows_per_band (the requested band
 * height; short frames use fewer rows), bins_per_cta, chunks_per_warp (the
 * largest any frame may use), ctas_per_sm, timeout_us, warps_per_cta;
 * groups_per_cta is 0 (chosen per frame). */
int ihist_batch_get_tune(ihist_batch_t batch, ihist_tune_t *out);

/* Bind the batch to n frames (1 <= n <= the planned count), for example a
 * new set of requests.  Frame i takes slot i, whose carry workspace was
 * sized for the i-th planned frame: any frame fits whose carries are no
 * larger (same or smaller height, width and bin count always do);
 * otherwise IHIST_ERR_UNSUPPORTED and the previous binding stays.  The new
 * descriptors are copied on `stream`, so later launches on it see them; the
 * descriptors are staged in one of two pinned buffers used by alternate
 * bindings, so the call waits (on the host) only for the copy made two
 * bindings earlier, and a caller may bind and launch ahead of the GPU.
 * Nothing is allocated. */
int ihist_batch_set_io(ihist_batch_t batch, const ihist_frame_t *frames, int n, void *stream);

/* Compute every bound frame of the batch in one launch on `stream`. */
int ihist_batch_compute(ihist_batch_t batch, void *stream);

/* Region histograms (Eq. 2) on frame `frame` of the batch; arguments as for
 * ihist_query. */
int ihist_batch_query(ihist_batch_t batch, int frame, const uint32_t *d_hist,
                      const int32_t *d_rects, int n, uint32_t *d_hist_out, void *stream);

/* Region histograms (Eq. 2) on every frame of the batch in one launch.
 * d_rects: nframes x n rectangles ({x0, y0, x1, y1} int32, inclusive),
 * frame f's at d_rects + 4*n*f.  d_out: frame f's n x nbins_f rows start
 * after those of frames 0..f-1 (offset n * sum of their bin counts words).
 * Out-of-range rectangles give zero rows and latch IHIST_ERR_BAD_RECT. */
int ihist_batch_query_all(ihist_batch_t batch, const int32_t *d_rects, int n, uint32_t *d_out,
                          void *stream);

/* Upload every frame of the batch from page-locked HOST memory on
 * copy_stream (h_frames[i]: h x w bytes, rows packed; w * channels bytes
 * per row for a joint frame) into the batch's
 * device inputs, then compute the batch on `stream` once the copies land
 * (Algorithm 6's dual buffering, one batch at a time).  Two batches driven
 * alternately overlap one batch's upload with the other's compute.  The
 * copies of a call wait for this batch's previous compute, so inputs are
 * never overwritten while still being read. */
int ihist_batch_upload_compute(ihist_batch_t batch, const uint8_t *const *h_frames, void *stream,
                               void *copy_stream);

/* As ihist_status, for the batch's status word. */
int ihist_batch_status(ihist_batch_t batch, void *stream, int *device_status);

/* Device workspace bytes the batch holds; number of work items per launch. */
size_t ihist_batch_workspace_bytes(ihist_batch_t batch);
unsigned int ihist_batch_items(ihist_batch_t batch);

/* Release the batch (NULL is a no-op); no launch of it may still be running. */
void ihist_batch_destroy(ihist_batch_t batch);

/* ---- Integral histogram without any device allocation -----------------
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc (code running inside a host callback or an
 * allocator hook, under a memory pool that must not grow, or in a process
 * whose device allocations belong to a framework the caller cannot reach).
 * It computes exactly what ihist_plan + ihist_compute compute (same kernel,
 * same words) for one frame, but takes its carry scratch from a fixed
 * 8 MiB array inside the library image instead of a plan.
 *   - Allocates nothing: no cudaMalloc, no cudaFree, no plan.
 *   - The scratch exists once per device, for as long as the process keeps
 *     the library loaded (8 MiB of every device that loads it).
 *   - The first call on a device sets that device up (looks up the device
 *     address of the scratch and the kernels' shared-memory limits) with
 *     the device current; make that first call before any stream capture.
 *   - All calls share the scratch, which keeps the previous call's
 *     contents; each call clears the parts that must start at zero on its
 *     stream.  Calls whose work may overlap on the GPU (other streams, other
 *     host threads) race on the scratch: keep them on one stream.
 *   - A frame whose carries do not fit the scratch returns
 *     IHIST_ERR_UNSUPPORTED (roughly: up to 1920 x 1080 with 64 bins fits;
 *     8192 x 8192 with 128 bins does not -- use a plan there).
 * Arguments as for ihist_plan / ihist_compute.  device_status: NULL for a
 * fully asynchronous call; otherwise the call waits for the stream and
 * stores the device status (IHIST_OK or IHIST_ERR_LOOKBACK_TIMEOUT). */
int ihist_compute_noalloc(int h, int w, int nbins, int layout, const uint8_t *d_in,
                          size_t in_pitch, uint32_t *d_out, void *stream, int *device_status);

/* Synchronise the stream, then read and clear the plan's device status word
 * into *device_status (IHIST_OK if no device error was latched since the
 * last read).  Returns IHIST_OK or a host/CUDA error code. */
int ihist_status(ihist_plan_t plan, void *stream, int *device_status);

/* Release the plan and its workspace (NULL is a no-op).  The caller must
 * make sure no work using the plan is still running. */
void ihist_destroy(ihist_plan_t plan);

/* Static description of a status code. */
const char *ihist_error_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* IHIST_H */

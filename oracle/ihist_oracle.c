/*
 * ihist_oracle.c -- CPU oracle for the integral histogram.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / --impl reference legs use it.  It shares no code, header,
 * table or constant with the CUDA library in paper_1711_01919_gb300/csrc.
 *
 * What it computes (Poostchi et al., "Fast Integral Histogram Computations on
 * GPU for Real-Time Video Analytics", arXiv 1711.01919):
 *
 *   H(x, y, b) = sum_{r<=x} sum_{c<=y} Q(I(r, c), b)                  (Eq. 1)
 *
 * computed with the sequential recurrence of Algorithm 1 (Sec. 2.1):
 *
 *   H(k, x, y) = H(k, x-1, y) + H(k, x, y-1) - H(k, x-1, y-1) + Q(k, I(x, y))
 *
 * looping over bins k, then rows x, then columns y.  The paper's x is the
 * row index and y the column index (Alg. 1 runs x over h and y over w).
 *
 * Readings taken where the paper is silent or ambiguous:
 *   - 0-based indices; any term with index -1 is zero (Alg. 1 is 1-based
 *     with an implicit zero border).
 *   - inclusive sums: a pixel counts in its own H (Eq. 1 sums r<=x, c<=y).
 *   - Q(v, b) = 1 iff floor(v * B / 256) == b for uint8 v and B uniform bins
 *     (the paper leaves the bin edges open, Sec. 2.1).
 *   - output layout [b][row][col] row-major, uint32 counts ("4 byte integer",
 *     Sec. 4.6; 3-D array mapped row-major to 1-D, Sec. 3.1 / Fig. 2).
 *   - region query (Eq. 2) for an inclusive rectangle (x0, y0, x1, y1) with
 *     x = column, y = row:
 *       h = H[y1][x1] - H[y0-1][x1] - H[y1][x0-1] + H[y0-1][x0-1]
 *     with index -1 terms zero, evaluated in uint32 modular arithmetic
 *     (the true result lies in [0, area], so intermediate wrap is harmless).
 *
 * Every function is plain, single-threaded and unblocked, except
 * oracle_ih_threads(), the bins-parallel variant used only to time the CPU
 * with all host cores (the paper's multi-threaded CPU comparison, Sec. 4.7);
 * it runs the same per-plane function on disjoint bins.
 */
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

/* Binning function Q of Eq. 1 (Sec. 2.1): the bin of intensity v among
 * nbins uniform bins over [0, 256). */
int oracle_bin_of(int v, int nbins) { return (v * nbins) / 256; }

/* One bin plane k of Algorithm 1.  img: h rows of w bytes, row stride pitch.
 * plane: [h][w] uint32, fully overwritten. */
void oracle_ih_plane(const uint8_t *img, size_t pitch, int h, int w, int nbins,
                     int k, uint32_t *plane) {
  for (int x = 0; x < h; ++x) {
    for (int y = 0; y < w; ++y) {
      uint32_t above = (x > 0) ? plane[(size_t)(x - 1) * w + y] : 0u;
      uint32_t left = (y > 0) ? plane[(size_t)x * w + (y - 1)] : 0u;
      uint32_t diag = (x > 0 && y > 0) ? plane[(size_t)(x - 1) * w + (y - 1)] : 0u;
      uint32_t q = (oracle_bin_of(img[(size_t)x * pitch + y], nbins) == k) ? 1u : 0u;
      plane[(size_t)x * w + y] = above + left - diag + q;
    }
  }
}

/* Algorithm 1 over all bins: out is [nbins][h][w] uint32. */
void oracle_ih(const uint8_t *img, size_t pitch, int h, int w, int nbins,
               uint32_t *out) {
  for (int k = 0; k < nbins; ++k)
    oracle_ih_plane(img, pitch, h, w, nbins, k, out + (size_t)k * h * w);
}

/* Region histogram by Eq. 2 from a bin-major integral histogram hist
 * ([nbins][h][w]).  rects: n x {x0, y0, x1, y1}, inclusive, x = column.
 * out: [n][nbins].  Returns the number of rectangles that were out of range
 * (those get an all-zero histogram). */
int oracle_query(const uint32_t *hist, int h, int w, int nbins,
                 const int32_t *rects, int n, uint32_t *out) {
  int bad = 0;
  for (int i = 0; i < n; ++i) {
    int x0 = rects[4 * i + 0], y0 = rects[4 * i + 1];
    int x1 = rects[4 * i + 2], y1 = rects[4 * i + 3];
    int ok = (0 <= x0 && x0 <= x1 && x1 < w && 0 <= y0 && y0 <= y1 && y1 < h);
    for (int b = 0; b < nbins; ++b) {
      uint32_t r = 0u;
      if (ok) {
        const uint32_t *P = hist + (size_t)b * h * w;
        uint32_t br = P[(size_t)y1 * w + x1];
        uint32_t tr = (y0 > 0) ? P[(size_t)(y0 - 1) * w + x1] : 0u;
        uint32_t bl = (x0 > 0) ? P[(size_t)y1 * w + (x0 - 1)] : 0u;
        uint32_t tl = (y0 > 0 && x0 > 0) ? P[(size_t)(y0 - 1) * w + (x0 - 1)] : 0u;
        r = br - tr - bl + tl;
      }
      out[(size_t)i * nbins + b] = r;
    }
    if (!ok) ++bad;
  }
  return bad;
}

/* Brute-force region histogram: counts the pixels of the rectangle directly
 * (the definition of a histogram over R, Sec. 2.1); independent of Eq. 2.
 * out: [nbins].  Returns 0, or -1 for an out-of-range rectangle. */
int oracle_region_brute(const uint8_t *img, size_t pitch, int h, int w,
                        int nbins, int x0, int y0, int x1, int y1,
                        uint32_t *out) {
  for (int b = 0; b < nbins; ++b) out[b] = 0u;
  if (!(0 <= x0 && x0 <= x1 && x1 < w && 0 <= y0 && y0 <= y1 && y1 < h)) return -1;
  for (int r = y0; r <= y1; ++r)
    for (int c = x0; c <= x1; ++c) out[oracle_bin_of(img[(size_t)r * pitch + c], nbins)] += 1u;
  return 0;
}

/* ---- other bin structures and joint (multi-channel) histograms ---------
 *
 * Eq. 1 holds for any binning function Q: the paper leaves the bin layout
 * open (Sec. 2.1) and names other bin structures and higher-dimensional
 * histograms, such as joint colour histograms, as uses of the same integral
 * (Sec. 1, Sec. 2.1).  Readings taken here:
 *   - bins by edges: nbins + 1 strictly increasing integers
 *     e[0] < e[1] < ... < e[nbins] in [0, 256]; bin k holds the intensities
 *     v with e[k] <= v < e[k+1]; intensities outside [e[0], e[nbins]) are in
 *     no bin (they count nowhere).
 *   - any value -> bin map: map[v] in [-1, nbins), -1 meaning no bin.
 *   - joint bins of a pixel with C interleaved channels (p_0 .. p_{C-1}),
 *     channel c cut into bins[c] uniform bins as above: the joint bin is the
 *     mixed-radix number of the channel bins, channel 0 most significant,
 *       k = (...((q_0 * bins[1] + q_1) * bins[2] + q_2) ...)
 *     with q_c = Q(p_c) among bins[c] bins; nbins = prod bins[c].
 * Every plane is still built by Algorithm 1's recurrence. */

/* The bin of intensity v for bins given by edges, or -1. */
int oracle_bin_of_edges(int v, const int *edges, int nbins) {
  for (int k = 0; k < nbins; ++k)
    if (edges[k] <= v && v < edges[k + 1]) return k;
  return -1;
}

/* Algorithm 1 with Q(k, v) = [map[v] == k]; out is [nbins][h][w] uint32. */
void oracle_ih_mapped(const uint8_t *img, size_t pitch, int h, int w,
                      const int *map, int nbins, uint32_t *out) {
  for (int k = 0; k < nbins; ++k) {
    uint32_t *plane = out + (size_t)k * h * w;
    for (int x = 0; x < h; ++x) {
      for (int y = 0; y < w; ++y) {
        uint32_t above = (x > 0) ? plane[(size_t)(x - 1) * w + y] : 0u;
        uint32_t left = (y > 0) ? plane[(size_t)x * w + (y - 1)] : 0u;
        uint32_t diag = (x > 0 && y > 0) ? plane[(size_t)(x - 1) * w + (y - 1)] : 0u;
        uint32_t q = (map[img[(size_t)x * pitch + y]] == k) ? 1u : 0u;
        plane[(size_t)x * w + y] = above + left - diag + q;
      }
    }
  }
}

/* Joint bin of one pixel px[0 .. channels-1]. */
int oracle_joint_bin(const uint8_t *px, int channels, const int *bins) {
  int k = 0;
  for (int c = 0; c < channels; ++c) k = k * bins[c] + oracle_bin_of(px[c], bins[c]);
  return k;
}

/* Algorithm 1 over the joint bins of a pixel-interleaved C-channel frame:
 * img holds h rows of w * channels bytes at row stride pitch; out is
 * [prod bins][h][w] uint32. */
void oracle_ih_joint(const uint8_t *img, size_t pitch, int h, int w,
                     int channels, const int *bins, uint32_t *out) {
  int nbins = 1;
  for (int c = 0; c < channels; ++c) nbins *= bins[c];
  for (int k = 0; k < nbins; ++k) {
    uint32_t *plane = out + (size_t)k * h * w;
    for (int x = 0; x < h; ++x) {
      for (int y = 0; y < w; ++y) {
        uint32_t above = (x > 0) ? plane[(size_t)(x - 1) * w + y] : 0u;
        uint32_t left = (y > 0) ? plane[(size_t)x * w + (y - 1)] : 0u;
        uint32_t diag = (x > 0 && y > 0) ? plane[(size_t)(x - 1) * w + (y - 1)] : 0u;
        const uint8_t *px = img + (size_t)x * pitch + (size_t)y * channels;
        uint32_t q = (oracle_joint_bin(px, channels, bins) == k) ? 1u : 0u;
        plane[(size_t)x * w + y] = above + left - diag + q;
      }
    }
  }
}

/* ---- a consumer of the integral histogram: sliding-window search -------
 *
 * Detection and tracking compare the histogram of every candidate window
 * with a target histogram (Sec. 1), which is what the O(1) region query is
 * for.  Readings taken here: windows of win_h x win_w pixels whose top-left
 * corners lie on the grid (i * stride, j * stride), i = 0 .. ny-1,
 * j = 0 .. nx-1, ny = (h - win_h) / stride + 1, nx = (w - win_w) / stride + 1
 * (integer division: only windows inside the frame); the score of a window
 * is the histogram intersection sum_b min(count_b, target_b) of Swain and
 * Ballard (1991), an exact integer.  This oracle counts each window's pixels
 * directly, without Eq. 2. */
void oracle_window_intersection(const uint8_t *img, size_t pitch, int h, int w, int nbins,
                                const uint32_t *target, int win_h, int win_w, int stride,
                                uint32_t *out) {
  const int ny = (h - win_h) / stride + 1, nx = (w - win_w) / stride + 1;
  uint32_t *count = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)nbins);
  if (!count) return;
  for (int i = 0; i < ny; ++i) {
    for (int j = 0; j < nx; ++j) {
      for (int b = 0; b < nbins; ++b) count[b] = 0u;
      for (int r = i * stride; r < i * stride + win_h; ++r)
        for (int c = j * stride; c < j * stride + win_w; ++c)
          count[oracle_bin_of(img[(size_t)r * pitch + c], nbins)] += 1u;
      uint32_t score = 0u;
      for (int b = 0; b < nbins; ++b) score += count[b] < target[b] ? count[b] : target[b];
      out[(size_t)i * nx + j] = score;
    }
  }
  free(count);
}

/* ---- bins-parallel variant, for timing the CPU on all host cores ------ */

typedef struct {
  const uint8_t *img;
  size_t pitch;
  int h, w, nbins, first, stride;
  uint32_t *out;
} oracle_job_t;

static void *oracle_worker(void *arg) {
  oracle_job_t *j = (oracle_job_t *)arg;
  for (int k = j->first; k < j->nbins; k += j->stride)
    oracle_ih_plane(j->img, j->pitch, j->h, j->w, j->nbins, k,
                    j->out + (size_t)k * j->h * j->w);
  return NULL;
}

/* Same result as oracle_ih(); bins are split round-robin over nthreads
 * POSIX threads.  Returns the number of threads actually used. */
int oracle_ih_threads(const uint8_t *img, size_t pitch, int h, int w,
                      int nbins, uint32_t *out, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > nbins) nthreads = nbins;
  pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
  oracle_job_t *jobs = (oracle_job_t *)malloc(sizeof(oracle_job_t) * (size_t)nthreads);
  char *running = (char *)calloc((size_t)nthreads, 1);
  if (!tid || !jobs || !running) {
    free(tid);
    free(jobs);
    free(running);
    oracle_ih(img, pitch, h, w, nbins, out);
    return 1;
  }
  int started = 0;
  for (int t = 0; t < nthreads; ++t) {
    oracle_job_t jb = {img, pitch, h, w, nbins, t, nthreads, out};
    jobs[t] = jb;
    if (pthread_create(&tid[t], NULL, oracle_worker, &jobs[t]) == 0) {
      running[t] = 1;
      ++started;
    } else {
      oracle_worker(&jobs[t]); /* run this share inline */
    }
  }
  for (int t = 0; t < nthreads; ++t)
    if (running[t]) pthread_join(tid[t], NULL);
  free(tid);
  free(jobs);
  free(running);
  return started > 0 ? started : 1;
}

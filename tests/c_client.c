/* A plain C (C11) client of libihist.so: no Python, no torch.  It reads a
 * uint8 frame and rectangles from files, computes the integral histogram
 * (Eq. 1) with a plan and as frame 0 of a two-frame batch, queries the
 * rectangles (Eq. 2), and writes H and the query rows to files.  Used by
 * tests/test_c_client.py, which compares the files with the oracle.
 *
 *   c_client <h> <w> <nbins> <frame.u8> <rects.i32> <nrects> <hist.u32> <rows.u32>
 *
 * Exit status 0 on success; any library or CUDA error prints a message and
 * exits 1. */
#include <cuda_runtime_api.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "ihist.h"

/* the struct sizes the Python binding mirrors (ctypes) */
_Static_assert(sizeof(ihist_frame_t) == 72, "ihist_frame_t layout");
_Static_assert(sizeof(ihist_tune_t) == 40, "ihist_tune_t layout");

static int fail(const char *what, int code) {
  fprintf(stderr, "%s failed: %d (%s)\n", what, code, ihist_error_string(code));
  return 1;
}

static void *read_file(const char *path, size_t bytes) {
  FILE *f = fopen(path, "rb");
  void *buf = malloc(bytes ? bytes : 1);
  if (!f || !buf || fread(buf, 1, bytes, f) != bytes) {
    fprintf(stderr, "cannot read %zu bytes from %s\n", bytes, path);
    exit(1);
  }
  fclose(f);
  return buf;
}

static int write_file(const char *path, const void *buf, size_t bytes) {
  FILE *f = fopen(path, "wb");
  if (!f || fwrite(buf, 1, bytes, f) != bytes) return 1;
  return fclose(f) != 0;
}

int main(int argc, char **argv) {
  if (argc != 9) {
    fprintf(stderr, "usage: %s h w nbins frame.u8 rects.i32 nrects hist.u32 rows.u32\n", argv[0]);
    return 2;
  }
  const int h = atoi(argv[1]), w = atoi(argv[2]), nbins = atoi(argv[3]), nrects = atoi(argv[6]);
  const size_t frame_bytes = (size_t)h * (size_t)w;
  const size_t out_bytes = ihist_output_bytes(h, w, nbins);
  const size_t rows_bytes = (size_t)nrects * (size_t)nbins * sizeof(uint32_t);
  uint8_t *frame = (uint8_t *)read_file(argv[4], frame_bytes);
  int32_t *rects = (int32_t *)read_file(argv[5], (size_t)nrects * 4 * sizeof(int32_t));

  uint8_t *d_in = NULL;
  uint32_t *d_out = NULL, *d_out2 = NULL, *d_rows = NULL;
  int32_t *d_rects = NULL;
  if (cudaMalloc((void **)&d_in, frame_bytes) != cudaSuccess ||
      cudaMalloc((void **)&d_out, out_bytes) != cudaSuccess ||
      cudaMalloc((void **)&d_out2, out_bytes) != cudaSuccess ||
      cudaMalloc((void **)&d_rows, rows_bytes ? rows_bytes : 4) != cudaSuccess ||
      cudaMalloc((void **)&d_rects, (size_t)nrects * 16 + 16) != cudaSuccess) {
    fprintf(stderr, "cudaMalloc failed\n");
    return 1;
  }
  cudaMemcpy(d_in, frame, frame_bytes, cudaMemcpyHostToDevice);
  cudaMemcpy(d_rects, rects, (size_t)nrects * 16, cudaMemcpyHostToDevice);

  /* one frame through a plan, then its region histograms */
  ihist_plan_t plan = NULL;
  int rc = ihist_plan(h, w, nbins, IHIST_BIN_MAJOR, &plan);
  if (rc != IHIST_OK) return fail("ihist_plan", rc);
  rc = ihist_compute(plan, d_in, (size_t)w, d_out, NULL);
  if (rc != IHIST_OK) return fail("ihist_compute", rc);
  rc = ihist_query(plan, d_out, d_rects, nrects, d_rows, NULL);
  if (rc != IHIST_OK) return fail("ihist_query", rc);
  int device_status = -1;
  rc = ihist_status(plan, NULL, &device_status);
  if (rc != IHIST_OK) return fail("ihist_status", rc);
  if (device_status != IHIST_OK) return fail("device status", device_status);

  /* the same frame as frame 0 of a batch (frame 1: its top half) */
  ihist_frame_t frames[2];
  memset(frames, 0, sizeof(frames));
  frames[0].h = h;
  frames[0].w = w;
  frames[0].nbins = nbins;
  frames[0].layout = IHIST_BIN_MAJOR;
  frames[0].d_in = d_in;
  frames[0].in_pitch = (size_t)w;
  frames[0].d_out = d_out2;
  frames[1] = frames[0];
  frames[1].h = h / 2 > 0 ? h / 2 : 1;
  uint32_t *d_out3 = NULL;
  if (cudaMalloc((void **)&d_out3, ihist_output_bytes(frames[1].h, w, nbins)) != cudaSuccess) return 1;
  frames[1].d_out = d_out3;
  ihist_batch_t batch = NULL;
  rc = ihist_batch_plan(frames, 2, NULL, &batch);
  if (rc != IHIST_OK) return fail("ihist_batch_plan", rc);
  rc = ihist_batch_compute(batch, NULL);
  if (rc != IHIST_OK) return fail("ihist_batch_compute", rc);
  rc = ihist_batch_status(batch, NULL, &device_status);
  if (rc != IHIST_OK) return fail("ihist_batch_status", rc);
  if (device_status != IHIST_OK) return fail("batch device status", device_status);

  uint32_t *hist = (uint32_t *)malloc(out_bytes), *hist2 = (uint32_t *)malloc(out_bytes);
  uint32_t *rows = (uint32_t *)malloc(rows_bytes ? rows_bytes : 4);
  if (!hist || !hist2 || !rows) return 1;
  if (cudaMemcpy(hist, d_out, out_bytes, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(hist2, d_out2, out_bytes, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(rows, d_rows, rows_bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
    fprintf(stderr, "cudaMemcpy back failed\n");
    return 1;
  }
  if (memcmp(hist, hist2, out_bytes) != 0) {
    fprintf(stderr, "batched and planned results differ\n");
    return 1;
  }
  if (write_file(argv[7], hist, out_bytes) || write_file(argv[8], rows, rows_bytes)) {
    fprintf(stderr, "cannot write the results\n");
    return 1;
  }
  ihist_batch_destroy(batch);
  ihist_destroy(plan);
  cudaFree(d_in);
  cudaFree(d_out);
  cudaFree(d_out2);
  cudaFree(d_out3);
  cudaFree(d_rows);
  cudaFree(d_rects);
  free(frame);
  free(rects);
  free(hist);
  free(hist2);
  free(rows);
  printf("c client ok\n");
  return 0;
}

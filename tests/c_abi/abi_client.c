/* A plain C client of the FNR library's C ABI (include/ir_filter.h): no
 * Python, no torch. It builds a synthetic 14-bit frame with impulses, filters
 * it with ir_filter_run2 (flagged count on the device), ir_filter_run (in
 * place) and a two-frame batch, and compares every pixel and the count with
 * the CPU oracle (oracle/fnr_oracle.c, linked as test infrastructure).
 * Exit status 0 = all bit-exact. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <cuda_runtime.h>
#include "ir_filter.h"

long long oracle_fnr(const void *in, long long in_pitch, void *out, long long out_pitch,
                     int H, int W, int esize, int k);

static unsigned long long lcg(unsigned long long *s) {
  *s = *s * 6364136223846793005ull + 1442695040888963407ull;
  return *s >> 33;
}

#define CHECK(x) do { ir_status st_ = (x); if (st_ != IR_OK) { \
  fprintf(stderr, "%s -> %s: %s\n", #x, ir_status_string(st_), ir_filter_last_error(h)); return 1; } } while (0)
#define CUDA(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { \
  fprintf(stderr, "%s -> %s\n", #x, cudaGetErrorString(e_)); return 1; } } while (0)

int main(void) {
  const int H = 301, W = 517, k = 5;
  const size_t pitch = W * 2;
  unsigned short *frame = malloc(pitch * H), *want = malloc(pitch * H), *got = malloc(pitch * H);
  unsigned long long seed = 12013972ull;
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      unsigned v = 4000 + 10 * (unsigned)(x + y) + (unsigned)(lcg(&seed) % 17);
      unsigned u = (unsigned)(lcg(&seed) % 100);
      frame[y * W + x] = (unsigned short)(u < 8 ? 0 : (u < 16 ? 16383 : v));
    }
  long long want_flagged = oracle_fnr(frame, (long long)pitch, want, (long long)pitch, H, W, 2, k);
  ir_filter *h = NULL;
  CHECK(ir_filter_create(&h, 0));
  void *d_in, *d_out;
  unsigned long long *d_cnt, cnt = 0;
  CUDA(cudaMalloc(&d_in, pitch * H));
  CUDA(cudaMalloc(&d_out, pitch * H));
  CUDA(cudaMalloc((void **)&d_cnt, 2 * sizeof(unsigned long long)));
  CUDA(cudaMemcpy(d_in, frame, pitch * H, cudaMemcpyHostToDevice));
  /* out of place, with the flagged count */
  CHECK(ir_filter_run2(h, d_in, pitch, d_out, pitch, H, W, IR_U14, k, NULL, d_cnt));
  CUDA(cudaMemcpy(got, d_out, pitch * H, cudaMemcpyDeviceToHost));
  CUDA(cudaMemcpy(&cnt, d_cnt, sizeof cnt, cudaMemcpyDeviceToHost));
  if (memcmp(got, want, pitch * H) != 0 || (long long)cnt != want_flagged) {
    fprintf(stderr, "run2 differs from the oracle (flagged %llu vs %lld)\n", cnt, want_flagged);
    return 1;
  }
  /* in place */
  CUDA(cudaMemcpy(d_out, frame, pitch * H, cudaMemcpyHostToDevice));
  CHECK(ir_filter_run(h, d_out, H, W, pitch, IR_U14, k, NULL));
  CUDA(cudaMemcpy(got, d_out, pitch * H, cudaMemcpyDeviceToHost));
  if (memcmp(got, want, pitch * H) != 0) { fprintf(stderr, "run (in place) differs\n"); return 1; }
  /* a batch of two: the same frame as two halves of one allocation */
  void *d_out2;
  CUDA(cudaMalloc(&d_out2, pitch * H));
  ir_frame_desc d[2];
  memset(d, 0, sizeof d);
  d[0].in = d_in; d[0].out = d_out; d[0].H = H; d[0].W = W; d[0].in_pitch = pitch; d[0].out_pitch = pitch;
  d[0].dtype = IR_U14; d[0].k = k; d[0].flagged_count = d_cnt;
  d[1] = d[0]; d[1].out = d_out2; d[1].flagged_count = d_cnt + 1;
  CUDA(cudaMemset(d_out, 0, pitch * H));
  CHECK(ir_filter_run_batch(h, d, 2, NULL));
  CHECK(ir_filter_sync_status(h));
  unsigned long long c2[2];
  CUDA(cudaMemcpy(c2, d_cnt, sizeof c2, cudaMemcpyDeviceToHost));
  for (int i = 0; i < 2; ++i) {
    CUDA(cudaMemcpy(got, i ? d_out2 : d_out, pitch * H, cudaMemcpyDeviceToHost));
    if (memcmp(got, want, pitch * H) != 0 || (long long)c2[i] != want_flagged) {
      fprintf(stderr, "batch frame %d differs\n", i);
      return 1;
    }
  }
  /* argument errors come back as statuses */
  if (ir_filter_run2(h, d_in, pitch, d_out, pitch, H, W, IR_U14, 4, NULL, NULL) != IR_EINVAL) return 1;
  printf("C ABI client: run2, run and batch bit-exact, flagged %lld, %llu launches\n", want_flagged,
         ir_filter_launch_count(h));
  cudaFree(d_in); cudaFree(d_out); cudaFree(d_out2); cudaFree(d_cnt);
  ir_filter_destroy(h);
  free(frame); free(want); free(got);
  return 0;
}

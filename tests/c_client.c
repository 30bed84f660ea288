/*
 * c_client.c -- a plain C caller of the fiberx C ABI (no Python, no torch):
 * reads a case from a binary file, uploads the fibers (cubic or quadratic)
 * from host memory, copies rays and the candidate CSR to the device with the
 * CUDA runtime, runs intersect_closest (and intersect_pairs with per-pair
 * status bytes), then intersect_backward for L = the sum of the hit t,
 * copies the results back and writes them to a binary file.
 *
 *   c_client IN OUT DEPTH FLAGS VARIANT
 *
 * IN:  int64 n_seg, n_ray, n_pair, n_cp (4: cubic, 3: quadratic);
 *      float cps[n_seg * n_cp * 4]; float rays[n_ray * 8];
 *      int32 row_ptr[n_ray + 1]; int32 seg_idx[n_pair]
 * OUT: float tu[n_ray * 2]; int32 seg[n_ray]; int32 leaf[n_ray];
 *      float tu_pairs[n_pair * 2]; uint8 pair_flags[n_pair]; uint32 status;
 *      float grad_cps[n_seg * n_cp * 4]
 * Exit status 0 on success; any failing call prints fx_last_error().
 */
#include <cuda_runtime_api.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "fiberx.h"

#define CHECK_FX(call)                                                        \
  do {                                                                        \
    fx_status st_ = (call);                                                   \
    if (st_ != FX_OK) {                                                       \
      fprintf(stderr, "%s failed (%d): %s\n", #call, (int)st_, fx_last_error()); \
      return 1;                                                               \
    }                                                                         \
  } while (0)

#define CHECK_CUDA(call)                                                      \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      fprintf(stderr, "%s failed: %s\n", #call, cudaGetErrorString(e_));      \
      return 1;                                                               \
    }                                                                         \
  } while (0)

static void *read_n(FILE *f, size_t bytes) {
  void *p = malloc(bytes ? bytes : 1);
  if (p && bytes && fread(p, 1, bytes, f) != bytes) {
    free(p);
    return NULL;
  }
  return p;
}

static void *to_device(const void *h, size_t bytes) {
  void *d = NULL;
  if (cudaMalloc(&d, bytes ? bytes : 1) != cudaSuccess) return NULL;
  if (bytes && cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return NULL;
  return d;
}

int main(int argc, char **argv) {
  if (argc != 6) {
    fprintf(stderr, "usage: %s IN OUT DEPTH FLAGS VARIANT\n", argv[0]);
    return 2;
  }
  const int32_t depth = atoi(argv[3]);
  const uint32_t flags = (uint32_t)strtoul(argv[4], NULL, 0);
  const int32_t variant = atoi(argv[5]);
  FILE *in = fopen(argv[1], "rb");
  if (!in) return 2;
  int64_t n[4];
  if (fread(n, sizeof(int64_t), 4, in) != 4) return 2;
  const int64_t n_seg = n[0], n_ray = n[1], n_pair = n[2], n_cp = n[3];
  if (n_cp != 3 && n_cp != 4) return 2;
  const size_t cp_floats = (size_t)n_seg * (size_t)n_cp * 4;
  float *cps = (float *)read_n(in, cp_floats * sizeof(float));
  float *rays = (float *)read_n(in, (size_t)n_ray * 8 * sizeof(float));
  int32_t *row_ptr = (int32_t *)read_n(in, (size_t)(n_ray + 1) * sizeof(int32_t));
  int32_t *seg_idx = (int32_t *)read_n(in, (size_t)n_pair * sizeof(int32_t));
  fclose(in);
  if (!cps || !rays || !row_ptr || !seg_idx) return 2;

  fx_fibers *fib = NULL;
  fx_upload_opts opts = {8, 1};
  if (n_cp == 4)
    CHECK_FX(fiber_upload(cps, n_seg, 0, &opts, NULL, &fib));
  else
    CHECK_FX(fiber_upload_quadratic(cps, n_seg, 0, &opts, NULL, &fib));
  fx_launch launch;
  CHECK_FX(fx_get_launch(fib, &launch));
  launch.variant = variant;
  CHECK_FX(fx_set_launch(fib, &launch));

  float *d_rays = (float *)to_device(rays, (size_t)n_ray * 8 * sizeof(float));
  int32_t *d_rp = (int32_t *)to_device(row_ptr, (size_t)(n_ray + 1) * sizeof(int32_t));
  int32_t *d_si = (int32_t *)to_device(seg_idx, (size_t)n_pair * sizeof(int32_t));
  float *d_tu = NULL, *d_tup = NULL;
  int32_t *d_seg = NULL, *d_leaf = NULL;
  uint8_t *d_pf = NULL;
  if (!d_rays || !d_rp || !d_si) return 1;
  CHECK_CUDA(cudaMalloc((void **)&d_tu, (size_t)n_ray * 2 * sizeof(float) + 1));
  CHECK_CUDA(cudaMalloc((void **)&d_seg, (size_t)n_ray * sizeof(int32_t) + 1));
  CHECK_CUDA(cudaMalloc((void **)&d_leaf, (size_t)n_ray * sizeof(int32_t) + 1));
  CHECK_CUDA(cudaMalloc((void **)&d_tup, (size_t)n_pair * 2 * sizeof(float) + 1));
  CHECK_CUDA(cudaMalloc((void **)&d_pf, (size_t)n_pair + 1));

  CHECK_FX(intersect_closest(fib, d_rays, n_ray, d_rp, d_si, n_pair, depth, NULL, flags, d_tu, d_seg, d_leaf,
                             NULL));
  CHECK_FX(intersect_pairs(fib, d_rays, n_ray, d_rp, d_si, n_pair, depth, NULL, flags & ~FX_POLISH_FP64, d_tup,
                           NULL, d_pf, NULL));
  /* adjoint of L = sum of the hit t: dL/dt = 1 for every ray (misses add nothing) */
  float *ones = (float *)malloc((size_t)n_ray * sizeof(float) + 1);
  float *d_gt = NULL, *d_grad = NULL;
  if (!ones) return 1;
  for (int64_t i = 0; i < n_ray; ++i) ones[i] = 1.0f;
  d_gt = (float *)to_device(ones, (size_t)n_ray * sizeof(float));
  if (!d_gt) return 1;
  CHECK_CUDA(cudaMalloc((void **)&d_grad, cp_floats * sizeof(float) + 1));
  CHECK_CUDA(cudaMemset(d_grad, 0, cp_floats * sizeof(float) + 1));
  CHECK_FX(intersect_backward(fib, d_rays, n_ray, d_tu, d_seg, d_gt, d_grad, NULL, NULL));
  uint32_t status = 0;
  CHECK_FX(fx_stream_status(fib, NULL, &status));

  float *tu = (float *)malloc((size_t)n_ray * 2 * sizeof(float) + 1);
  int32_t *seg = (int32_t *)malloc((size_t)n_ray * sizeof(int32_t) + 1);
  int32_t *leaf = (int32_t *)malloc((size_t)n_ray * sizeof(int32_t) + 1);
  float *tup = (float *)malloc((size_t)n_pair * 2 * sizeof(float) + 1);
  uint8_t *pf = (uint8_t *)malloc((size_t)n_pair + 1);
  float *grad = (float *)malloc(cp_floats * sizeof(float) + 1);
  if (!tu || !seg || !leaf || !tup || !pf || !grad) return 1;
  CHECK_CUDA(cudaMemcpy(tu, d_tu, (size_t)n_ray * 2 * sizeof(float), cudaMemcpyDeviceToHost));
  CHECK_CUDA(cudaMemcpy(seg, d_seg, (size_t)n_ray * sizeof(int32_t), cudaMemcpyDeviceToHost));
  CHECK_CUDA(cudaMemcpy(leaf, d_leaf, (size_t)n_ray * sizeof(int32_t), cudaMemcpyDeviceToHost));
  CHECK_CUDA(cudaMemcpy(tup, d_tup, (size_t)n_pair * 2 * sizeof(float), cudaMemcpyDeviceToHost));
  CHECK_CUDA(cudaMemcpy(pf, d_pf, (size_t)n_pair, cudaMemcpyDeviceToHost));
  CHECK_CUDA(cudaMemcpy(grad, d_grad, cp_floats * sizeof(float), cudaMemcpyDeviceToHost));

  FILE *out = fopen(argv[2], "wb");
  if (!out) return 2;
  fwrite(tu, sizeof(float), (size_t)n_ray * 2, out);
  fwrite(seg, sizeof(int32_t), (size_t)n_ray, out);
  fwrite(leaf, sizeof(int32_t), (size_t)n_ray, out);
  fwrite(tup, sizeof(float), (size_t)n_pair * 2, out);
  fwrite(pf, 1, (size_t)n_pair, out);
  fwrite(&status, sizeof(status), 1, out);
  fwrite(grad, sizeof(float), cp_floats, out);
  fclose(out);
  cudaFree(d_gt);
  cudaFree(d_grad);
  free(ones);
  free(grad);

  cudaFree(d_rays);
  cudaFree(d_rp);
  cudaFree(d_si);
  cudaFree(d_tu);
  cudaFree(d_seg);
  cudaFree(d_leaf);
  cudaFree(d_tup);
  cudaFree(d_pf);
  fiber_free(fib);
  free(cps);
  free(rays);
  free(row_ptr);
  free(seg_idx);
  free(tu);
  free(seg);
  free(leaf);
  free(tup);
  free(pf);
  printf("c_client ok: fiberx %d, %lld rays, %lld pairs\n", fx_version(), (long long)n_ray, (long long)n_pair);
  return 0;
}

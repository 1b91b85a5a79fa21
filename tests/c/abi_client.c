/* A plain C client of the C ABI: no Python, no torch.  Reads a segment and a
 * batch from a binary file, evaluates it on the GPU through include/td.h and
 * writes log L and chi2.
 *
 * Input file:  int64 n, int64 K, int64 has_mask, double acf[n],
 *              uint8 mask[n] (if has_mask), float R[K][N'] (column k = residual k)
 * Output file: double logL[K], double chi2[K], double logdet, double same
 *   (same = 1 when a segment saved to "<output>.ckpt" with td_segment_save and
 *   read back with td_segment_load gives the same log L bits, else 0)
 * Exit status 0 on success; a td_status or CUDA failure prints td_last_error(). */
#include <cuda_runtime_api.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "td.h"

#define CHECK_TD(call)                                                           \
  do {                                                                           \
    td_status st_ = (call);                                                      \
    if (st_ != TD_OK) {                                                          \
      fprintf(stderr, "%s failed: %d (%s)\n", #call, (int)st_, td_last_error()); \
      return 2;                                                                  \
    }                                                                            \
  } while (0)
#define CHECK_CUDA(call)                                                     \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      fprintf(stderr, "%s failed: %s\n", #call, cudaGetErrorString(e_));     \
      return 3;                                                              \
    }                                                                        \
  } while (0)

int main(int argc, char** argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: %s input output\n", argv[0]);
    return 1;
  }
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 1;
  int64_t hdr[3];
  if (fread(hdr, sizeof(int64_t), 3, f) != 3) return 1;
  const int64_t n = hdr[0], K = hdr[1];
  double* acf = (double*)malloc((size_t)n * sizeof(double));
  uint8_t* mask = hdr[2] ? (uint8_t*)malloc((size_t)n) : NULL;
  if (fread(acf, sizeof(double), (size_t)n, f) != (size_t)n) return 1;
  int64_t nk = n;
  if (mask) {
    if (fread(mask, 1, (size_t)n, f) != (size_t)n) return 1;
    nk = 0;
    for (int64_t i = 0; i < n; ++i) nk += mask[i] != 0;
  }
  float* R = (float*)malloc((size_t)(nk * K) * sizeof(float));
  if (fread(R, sizeof(float), (size_t)(nk * K), f) != (size_t)(nk * K)) return 1;
  fclose(f);

  td_segment* s = NULL;
  CHECK_TD(td_segment_create(acf, n, mask, NULL, &s));
  CHECK_TD(td_factor(s, NULL));
  if (td_kept(s) != nk) return 4;
  double logdet = 0.0;
  CHECK_TD(td_logdet(s, &logdet));

  float* dR = NULL;
  double *dL = NULL, *dC = NULL;
  CHECK_CUDA(cudaMalloc((void**)&dR, (size_t)(nk * K) * sizeof(float)));
  CHECK_CUDA(cudaMalloc((void**)&dL, (size_t)K * sizeof(double)));
  CHECK_CUDA(cudaMalloc((void**)&dC, (size_t)K * sizeof(double)));
  CHECK_CUDA(cudaMemcpy(dR, R, (size_t)(nk * K) * sizeof(float), cudaMemcpyHostToDevice));
  td_options opt;
  td_options_default(&opt);
  CHECK_TD(td_loglike_batch(s, dR, nk, K, dL, &opt, dC, NULL));
  CHECK_TD(td_check(s, NULL));

  double* out = (double*)malloc((size_t)(2 * K + 2) * sizeof(double));
  CHECK_CUDA(cudaMemcpy(out, dL, (size_t)K * sizeof(double), cudaMemcpyDeviceToHost));
  CHECK_CUDA(cudaMemcpy(out + K, dC, (size_t)K * sizeof(double), cudaMemcpyDeviceToHost));
  out[2 * K] = logdet;

  /* factor checkpoint and resume through the same ABI */
  char* ckpt = (char*)malloc(strlen(argv[2]) + 6);
  sprintf(ckpt, "%s.ckpt", argv[2]);
  CHECK_TD(td_segment_save(s, ckpt, NULL));
  td_segment* s2 = NULL;
  CHECK_TD(td_segment_load(ckpt, NULL, &s2));
  CHECK_TD(td_loglike_batch(s2, dR, nk, K, dL, &opt, NULL, NULL));
  CHECK_TD(td_check(s2, NULL));
  double* again = (double*)malloc((size_t)K * sizeof(double));
  CHECK_CUDA(cudaMemcpy(again, dL, (size_t)K * sizeof(double), cudaMemcpyDeviceToHost));
  out[2 * K + 1] = memcmp(again, out, (size_t)K * sizeof(double)) == 0 ? 1.0 : 0.0;
  td_segment_destroy(s2);
  remove(ckpt);
  free(ckpt);
  free(again);

  f = fopen(argv[2], "wb");
  if (!f) return 1;
  fwrite(out, sizeof(double), (size_t)(2 * K + 2), f);
  fclose(f);

  cudaFree(dR);
  cudaFree(dL);
  cudaFree(dC);
  td_segment_destroy(s);
  free(acf);
  free(mask);
  free(R);
  free(out);
  return 0;
}

/* A plain C caller of libdmpt.so (test driver).
 *
 * Reads one problem from a raw file -- n x n H, then k blocks of n x n H1,
 * all float64 row-major -- solves it through dmpt_sp2_response_host (host
 * buffers in and out; the only device memory it manages is the workspace),
 * and writes P then the k blocks of P1 to the output file.  Prints
 * "status layers d0_layer converged" on stdout.
 *
 * usage: dmpt_host_solve n n_occ k input.bin output.bin
 */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "dmpt.h"

static int read_all(const char* path, double* buf, size_t count) {
  FILE* f = fopen(path, "rb");
  if (!f) return 0;
  size_t got = fread(buf, sizeof(double), count, f);
  fclose(f);
  return got == count;
}

static int write_all(const char* path, const double* a, size_t na, const double* b, size_t nb) {
  FILE* f = fopen(path, "wb");
  if (!f) return 0;
  int ok = fwrite(a, sizeof(double), na, f) == na && fwrite(b, sizeof(double), nb, f) == nb;
  fclose(f);
  return ok;
}

int main(int argc, char** argv) {
  if (argc != 6) {
    fprintf(stderr, "usage: %s n n_occ k input.bin output.bin\n", argv[0]);
    return 2;
  }
  const long long n = atoll(argv[1]), n_occ = atoll(argv[2]);
  const int k = atoi(argv[3]);
  const size_t nn = (size_t)n * (size_t)n;
  double* in = (double*)malloc(sizeof(double) * nn * (1 + k));
  double* P = (double*)malloc(sizeof(double) * nn);
  double* P1 = (double*)malloc(sizeof(double) * nn * (k > 0 ? k : 1));
  if (!in || !P || !P1 || !read_all(argv[4], in, nn * (1 + k))) {
    fprintf(stderr, "cannot read %s\n", argv[4]);
    return 2;
  }
  dmpt_handle h = NULL;
  dmpt_status st = dmpt_create(&h, 0);
  if (st != DMPT_OK) {
    fprintf(stderr, "dmpt_create: %s\n", dmpt_status_string(st));
    return 1;
  }
  dmpt_options o;
  dmpt_default_options(&o);
  const size_t ws_bytes = dmpt_workspace_size_host(n, k, &o);
  void* ws = NULL;
  if (ws_bytes == 0 || cudaMalloc(&ws, ws_bytes) != cudaSuccess) {
    fprintf(stderr, "workspace of %zu bytes\n", ws_bytes);
    return 1;
  }
  const double* Hs[1] = {in};
  const double* H1s[1] = {in + nn};
  double* Ps[1] = {P};
  double* P1s[1] = {P1};
  dmpt_info info;
  st = dmpt_sp2_response_host(h, 1, Hs, H1s, k, n, n_occ, &o, Ps, k > 0 ? P1s : NULL, &info, ws,
                              ws_bytes, NULL);
  printf("%d %d %d %d\n", (int)st, info.layers, info.d0_layer, info.converged);
  if (st != DMPT_OK) fprintf(stderr, "dmpt_sp2_response_host: %s\n", dmpt_last_error(h));
  const int ok = write_all(argv[5], P, nn, P1, nn * (size_t)k);
  cudaFree(ws);
  dmpt_destroy(h);
  free(in);
  free(P);
  free(P1);
  return (st == DMPT_OK && ok) ? 0 : 1;
}

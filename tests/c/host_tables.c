/* Uses the C ABI from plain C (host-only entry points, no GPU): builds the tables of a
 * 2 x 1 x 1 box with one refined base cell, prints the counts, adapts it with all
 * refinable elements marked for refinement and prints the new leaf count, then reads the
 * Jacobi-diagonal tables. */
#include <stdio.h>
#include <stdlib.h>

#include "tm.h"

int main(void) {
  /* base cell (0,0,0) split into its 8 children (level 1), base cell (1,0,0) whole (level 0); L = 1 */
  int32_t leaves[4 * 9];
  int n = 0;
  for (int k = 0; k < 8; ++k) {
    leaves[4 * n + 0] = k & 1;
    leaves[4 * n + 1] = (k >> 1) & 1;
    leaves[4 * n + 2] = (k >> 2) & 1;
    leaves[4 * n + 3] = 1;
    ++n;
  }
  leaves[4 * n + 0] = 2; leaves[4 * n + 1] = 0; leaves[4 * n + 2] = 0; leaves[4 * n + 3] = 0;
  ++n;
  tm_mesh_desc d = {2, 1, 1, 1, 1.0, n, leaves, 1u, 1.0, 1e-9, 0.3, 3.0};
  tm_tables *t = NULL;
  tm_mesh_info info;
  char err[256];
  int rc = tm_tables_build(&d, &t, &info, err, (int)sizeof err);
  if (rc != TM_OK) {
    fprintf(stderr, "tm_tables_build: %d %s\n", rc, err);
    return 1;
  }
  printf("Ne %lld Nn %lld hanging %lld free %lld blocks %d\n", (long long)info.Ne, (long long)info.Nn,
         (long long)info.n_hanging, (long long)info.n_free, info.n_blocks);
  int8_t *mark = (int8_t *)calloc((size_t)info.Ne, 1);
  double *rho = (double *)malloc(sizeof(double) * (size_t)info.Ne);
  for (int64_t e = 0; e < info.Ne; ++e) rho[e] = 0.5;
  /* the level-0 element is the last in Morton order here: refine it */
  mark[info.Ne - 1] = 1;
  int32_t out_leaves[4 * 64];
  double out_rho[64];
  int64_t n_out = 0;
  rc = tm_tables_adapt(t, mark, rho, 64, out_leaves, out_rho, &n_out);
  printf("adapt rc %d leaves %lld\n", rc, (long long)n_out);
  /* a malformed request is refused with TM_EINVAL, not a crash */
  mark[info.Ne - 1] = 0;
  mark[0] = 1;               /* level 1 == L: cannot refine */
  rc = tm_tables_adapt(t, mark, rho, 64, out_leaves, out_rho, &n_out);
  printf("bad mark rc %d\n", rc);
  /* the Jacobi-diagonal tables: sizes first, then the arrays; the diagonal's component-0 sum at
   * rho = 1 (c_e = h_e: level-1 elements 0..7 have h = 1/2, the level-0 element h = 1) */
  int64_t n_entries = 0, n_triples = 0;
  rc = tm_tables_diag(t, NULL, NULL, NULL, NULL, &n_entries, &n_triples);
  int32_t *ptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(info.Nn + 1));
  int32_t *elem = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_entries);
  uint16_t *q = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n_entries);
  double *tab = (double *)malloc(sizeof(double) * 3 * (size_t)n_triples);
  if (rc == TM_OK) rc = tm_tables_diag(t, ptr, elem, q, tab, &n_entries, &n_triples);
  double dsum = 0.0;
  for (int64_t nd = 0; nd < info.Nn; ++nd)
    for (int32_t j = ptr[nd]; j < ptr[nd + 1]; ++j) dsum += (elem[j] == info.Ne - 1 ? 1.0 : 0.5) * tab[3 * q[j]];
  printf("diag rc %d entries %lld triples %lld sum0 %.17g\n", rc, (long long)n_entries, (long long)n_triples, dsum);
  tm_tables_free(t);
  free(ptr);
  free(elem);
  free(q);
  free(tab);
  free(mark);
  free(rho);
  return 0;
}

/* A plain C99 consumer of include/apsp.h: compiles with -pedantic -Werror,
 * links against libapsp.so and calls the entry points that need no GPU,
 * through the header's own types (so the header, not a binding, is checked
 * against the library).  Prints "ok" on success. */
#include <stdio.h>
#include <string.h>

#include "apsp.h"

static int fails = 0;
#define CHECK(c)                                                   \
  do {                                                             \
    if (!(c)) {                                                    \
      printf("FAIL line %d: %s\n", __LINE__, #c);                  \
      ++fails;                                                     \
    }                                                              \
  } while (0)

int main(void) {
  apsp_config cfg;
  int32_t d[9];
  int16_t via[9];
  int64_t path[8], len = -1;
  int i;

  CHECK(apsp_version() > 0);
  CHECK(strcmp(apsp_status_str(APSP_OK), "APSP_OK") == 0);
  CHECK(strcmp(apsp_status_str(APSP_EINVAL), "APSP_EINVAL") == 0);
  CHECK(apsp_status_str(12345) != NULL);

  /* configuration queries fill the header's struct */
  memset(&cfg, 0x55, sizeof cfg);
  CHECK(apsp_query_config(16384, APSP_F32, 0, &cfg) == APSP_OK);
  CHECK(cfg.kblock == 128 && cfg.rounds == 128 && cfg.phase3_tma == 1 && cfg.phase3_threads == 256);
  CHECK(cfg.phase3_relax_per_round == (int64_t)(16384 - 128) * (16384 - 128) * 128);
  CHECK(cfg.lookahead == 1 && cfg.strips == 0);
  CHECK(apsp_query_config(1024, APSP_I32, 0, &cfg) == APSP_OK);
  CHECK(cfg.kblock == 64 && cfg.rounds == 16 && cfg.lookahead == 1 && cfg.strips == 1);
  CHECK(apsp_query_config(100, APSP_I16, 128, &cfg) == APSP_OK && cfg.kblock == 128 && cfg.rounds == 1);
  CHECK(apsp_query_config(100, APSP_I32, 96, &cfg) == APSP_EINVAL);
  CHECK(apsp_query_config(100, 7, 0, &cfg) == APSP_EINVAL);
  CHECK(apsp_workspace_bytes(16384, APSP_F32, 0) == (int64_t)2 * 128 * 16384 * 4);
  CHECK(apsp_workspace_bytes(-1, APSP_F32, 0) == 0);

  /* argument checks come before any device work */
  CHECK(apsp_fw(NULL, 10, 10, APSP_I32, NULL) == APSP_EINVAL);
  CHECK(apsp_fw(d, 3, 2, APSP_I32, NULL) == APSP_EINVAL);     /* ld < n */
  CHECK(apsp_fw(d, -1, 3, APSP_I32, NULL) == APSP_EINVAL);
  CHECK(apsp_fw(d, 3, 3, 9, NULL) == APSP_EINVAL);            /* dtype */
  CHECK(apsp_fw(d, 0, 0, APSP_F32, NULL) == APSP_OK);         /* empty graph */

  /* apsp_path on a solved 3-vertex graph (host arrays): edges 0->1 (10),
   * 0->2 (1), 2->1 (2), 1->0 (1); the solve lowers d_01 to 3 through vertex 2
   * in stage 0 (one k-block of 64), d_12 to 2 and d_21 stays the edge. */
  {
    const int32_t solved[9] = {0, 3, 1, 1, 0, 2, 3, 2, 0};
    const int16_t rec[9] = {-1, 0, -1, -1, -1, 0, 0, -1, -1};
    memcpy(d, solved, sizeof d);
    memcpy(via, rec, sizeof via);
  }
  CHECK(apsp_path(d, via, 3, 3, 3, APSP_I32, 64, 0, 1, path, 8, &len) == APSP_OK);
  CHECK(len == 3 && path[0] == 0 && path[1] == 2 && path[2] == 1);
  CHECK(apsp_path(d, via, 3, 3, 3, APSP_I32, 64, 2, 0, path, 8, &len) == APSP_OK);
  CHECK(len == 3 && path[0] == 2 && path[1] == 1 && path[2] == 0);
  CHECK(apsp_path(d, via, 3, 3, 3, APSP_I32, 64, 1, 1, path, 8, &len) == APSP_OK && len == 1 && path[0] == 1);
  CHECK(apsp_path(d, via, 3, 3, 3, APSP_I32, 64, 0, 1, path, 2, &len) == APSP_ENOMEM && len == 3);
  CHECK(apsp_path(d, via, 3, 3, 3, APSP_I32, 64, 0, 5, path, 8, &len) == APSP_EINVAL);
  for (i = 0; i < 9; ++i) CHECK(d[i] >= 0 && d[i] < APSP_INF_I32); /* apsp_path does not write the matrix */

  if (fails) return 1;
  printf("ok\n");
  return 0;
}

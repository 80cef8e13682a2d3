/* A plain C client of the C ABI: compiled against include/aiwc.h, linked to
 * libaiwc.so, and run without a GPU. It exercises only calls that need no
 * device: the defaults, argument checks, host-side aggregation over
 * invocations (Sec. VI) and the serving configuration checks. */
#include <stdio.h>
#include <string.h>

#include "aiwc.h"

#define CHECK(c)                                                    \
  do {                                                              \
    if (!(c)) {                                                     \
      fprintf(stderr, "c client: line %d: %s\n", __LINE__, #c);     \
      return 1;                                                     \
    }                                                               \
  } while (0)

int main(void) {
  aiwc_config cfg;
  aiwc_config_default(&cfg);
  CHECK(cfg.history_len == 16 && cfg.cover_num == 9 && cfg.cover_den == 10);
  CHECK(cfg.space_mask == 0xF && cfg.n_opcodes == 65535 && cfg.precision == 0);

  /* invalid configurations are refused before any device is touched */
  aiwc_handle* h = (aiwc_handle*)&cfg;
  cfg.history_len = 0;
  CHECK(aiwc_create(&cfg, &h) == AIWC_EINVAL && h == NULL);
  CHECK(strstr(aiwc_last_error(NULL), "history_len") != NULL);
  aiwc_config_default(&cfg);
  cfg.partitions = 3;
  CHECK(aiwc_create(&cfg, &h) == AIWC_EINVAL);
  CHECK(aiwc_create(NULL, &h) == AIWC_EINVAL);
  CHECK(aiwc_push_mem(NULL, NULL, 0, 0) == AIWC_EINVAL);
  CHECK(aiwc_compute(NULL, NULL) == AIWC_EINVAL);
  CHECK(aiwc_destroy(NULL) == AIWC_OK);

  /* whole-application view: sums and medians over three invocations */
  aiwc_metrics runs[3], out;
  memset(runs, 0, sizeof runs);
  runs[0].footprint = 10;
  runs[1].footprint = 30;
  runs[2].footprint = 20;
  runs[0].albe = 0.5;
  runs[1].albe = 0.25;
  runs[2].albe = 1.0;
  runs[0].entropy[3] = 2.0;
  runs[1].entropy[3] = 4.0;
  memset(&out, 0, sizeof out);
  CHECK(aiwc_aggregate(runs, 3, AIWC_AGG_SUM, &out) == AIWC_OK);
  CHECK(out.footprint == 60 && out.albe == 1.75 && out.entropy[3] == 6.0);
  CHECK(aiwc_aggregate(runs, 3, AIWC_AGG_MEDIAN, &out) == AIWC_OK);
  CHECK(out.footprint == 20 && out.albe == 0.5 && out.entropy[3] == 2.0);
  CHECK(aiwc_aggregate(runs, 2, AIWC_AGG_MEDIAN, &out) == AIWC_OK);
  CHECK(out.footprint == 10 && out.albe == 0.375); /* integers: lower middle; reals: mean of the middles */
  CHECK(aiwc_aggregate(runs, 3, 7, &out) == AIWC_EINVAL);
  CHECK(aiwc_aggregate(NULL, 3, AIWC_AGG_SUM, &out) == AIWC_EINVAL);

  /* serving configuration */
  aiwc_server_config sc;
  aiwc_server_config_default(&sc);
  CHECK(sc.max_jobs == 32 && sc.workers == 4 && sc.hbm_budget == (120ull << 30));
  sc.max_jobs = 0;
  aiwc_server* s = NULL;
  CHECK(aiwc_server_create(&sc, &s) == AIWC_EINVAL && s == NULL);

  printf("c client ok\n");
  return 0;
}

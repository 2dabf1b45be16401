/* A C11 client of include/tectonic.h: compiles the header as plain C under
 * -pedantic, links libtectonic.so and runs the calls that need no device
 * (argument checks and the error buffer).  Prints "ok" and exits 0 on
 * success; prints the failed check and exits 1 otherwise. */
#include <stdio.h>
#include <string.h>

#include "tectonic.h"

#define CHECK(cond)                                          \
    do {                                                     \
        if (!(cond)) {                                       \
            printf("failed: %s (line %d)\n", #cond, __LINE__); \
            return 1;                                        \
        }                                                    \
    } while (0)

int main(void) {
    char buf[256];
    int64_t n = -1, m = -1;
    int64_t p[2] = {1, 2}, q[2] = {128, 128};
    tec_graph *g = NULL;
    tec_measure meas = TEC_TECTONIC;
    tec_rule rule = TEC_RULE_LARGEST_JUMP;

    CHECK(tec_version() == 100);
    CHECK(tec_graph_free(NULL) == TEC_OK);
    CHECK(tec_graph_info(NULL, &n, &m) == TEC_EINVAL);
    CHECK(tec_last_error(buf, sizeof buf) > 0 && strlen(buf) > 0);
    CHECK(tec_last_error(NULL, 0) == strlen(buf));
    CHECK(tec_graph_create(-1, 0, NULL, &g) == TEC_EINVAL && g == NULL);
    CHECK(tec_prune(NULL, meas, 1, 10, NULL, NULL) == TEC_EINVAL);
    CHECK(tec_sweep(NULL, meas, p, q, 2, NULL, 0, NULL, NULL) == TEC_EINVAL);
    CHECK(tec_rule_of_thumb(NULL, p, q, 0, 1, rule, NULL, NULL) == TEC_EINVAL);
    CHECK(tec_picker_thresholds(NULL, -1, NULL, NULL, NULL) == TEC_EINVAL);
    CHECK(TEC_PICKER_PARAMS == TEC_PICKER_HIDDEN * TEC_PICKER_INPUTS + TEC_PICKER_HIDDEN +
                                   TEC_PICKER_HIDDEN * TEC_PICKER_HIDDEN + TEC_PICKER_HIDDEN +
                                   TEC_PICKER_HIDDEN + 1);
    CHECK(sizeof(tec_sweep_stat) == 5 * 8);
    printf("ok\n");
    return 0;
}

/* Test client: include/tm.h compiled as strict C99 and linked against
 * libtm.so by a C compiler, calling host-only entry points and argument
 * checks (no GPU needed).  Built and run by tests/test_abi.py; prints one
 * line per check and exits non-zero on the first failure. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "tm.h"

#define CHECK(cond)                                                       \
    do {                                                                  \
        if (!(cond)) {                                                    \
            printf("FAILED: %s (line %d)\n", #cond, __LINE__);            \
            return 1;                                                     \
        }                                                                 \
        printf("ok: %s\n", #cond);                                        \
    } while (0)

int main(void)
{
    tm_config cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.p = 1024;
    CHECK(tm_version() > 0);
    CHECK(strlen(tm_status_str(TM_ERR_INVALID)) > 0);
    CHECK(strcmp(tm_last_cuda_error(), "cudaSuccess") == 0);
    CHECK(tm_merge_blocks((int64_t)1 << 20, (int64_t)1 << 19, &cfg) == 1024);
    CHECK(tm_merge_blocks(0, 0, NULL) == 1);
    CHECK(tm_merge_workspace_size((int64_t)1 << 20, (int64_t)1 << 19, &cfg) >= 256 + 2 * 1025 * 8);
    CHECK(tm_tile_record_bytes() == 48);
    CHECK(tm_merge_tile_cap(10, 7, 3) == 4 + 3);
    CHECK(tm_plan_tile_count(10, 3, 5) == 5 + 3);
    CHECK(tm_merge(TM_KEY_I32, NULL, NULL, -1, NULL, NULL, 0, NULL, NULL, NULL, 0, NULL, NULL) == TM_ERR_INVALID);
    CHECK(tm_merge((tm_key_type)9, NULL, NULL, 0, NULL, NULL, 0, NULL, NULL, NULL, 0, NULL, NULL)
          == TM_ERR_UNSUPPORTED);
    CHECK(tm_merge_sort(TM_KEY_U64, NULL, NULL, -1, NULL, NULL, NULL, 0, NULL, NULL) == TM_ERR_INVALID);
    CHECK(tm_merge_batched_workspace_size(-1, 0, 0, NULL) == 0);
    CHECK(tm_cdf_model_bytes(4096, 64) % 256 == 0 && tm_cdf_model_bytes(1, 64) == 0);
    CHECK(tm_graph_capture_begin(NULL) == TM_ERR_INVALID);
    tm_graph_destroy(NULL);
    CHECK(tm_autotune_clear() == 0);
    printf("all ok\n");
    return 0;
}

/* Test client: prints the byte layout of the public structs of include/tm.h
 * as the C compiler lays them out ("name offset size" per field, then the
 * struct size), for tests/test_abi.py to compare with the binding's ctypes
 * declarations. */
#include <stddef.h>
#include <stdio.h>

#include "tm.h"

#define FIELD(s, f) printf(#f " %zu %zu\n", offsetof(s, f), sizeof(((s*)0)->f))

int main(void)
{
    FIELD(tm_config, p);
    FIELD(tm_config, tile);
    FIELD(tm_config, threads);
    FIELD(tm_config, grid);
    FIELD(tm_config, stages);
    FIELD(tm_config, split);
    FIELD(tm_config, wait_ms);
    FIELD(tm_config, test_drop_tile);
    FIELD(tm_config, unfused);
    FIELD(tm_config, partition);
    FIELD(tm_config, payload_bytes);
    FIELD(tm_config, trace);
    FIELD(tm_config, merge_ways);
    printf("sizeof %zu\n", sizeof(tm_config));
    return 0;
}

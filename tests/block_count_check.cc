// Edge values of the block-count helpers of the library (csrc/block_count.h), on the host:
// tests/test_library_cpu.py compiles and runs this file.  Exit status 0 when every check holds.
#include <cstdint>
#include <cstdio>

#include "block_count.h"

using cbessfm::blocks_for;
using cbessfm::too_many_blocks;

static int failures = 0;

static void check(bool ok, const char* what) {
    if (!ok) {
        std::printf("failed: %s\n", what);
        ++failures;
    }
}

int main() {
    const long long M = (1ll << 31) - 1;
    check(blocks_for(1, 3840) == 1, "one sample is one block");
    check(blocks_for(3840, 3840) == 1, "V samples are one block");
    check(blocks_for(3841, 3840) == 2, "V + 1 samples are two blocks");
    check(blocks_for(INT64_MAX, 1) == INT64_MAX, "no overflow at the largest length, V = 1");
    check(blocks_for(INT64_MAX, 3840) == INT64_MAX / 3840 + 1, "no overflow at the largest length");
    check(!too_many_blocks(M, 1), "2^31 - 1 blocks are allowed");
    check(too_many_blocks(M + 1, 1), "2^31 blocks are refused");
    check(!too_many_blocks(M / 7, 7) && too_many_blocks(M / 7 + 1, 7), "the limit with batch 7");
    check(too_many_blocks(INT64_MAX / 3840 + 1, 2147483647), "the largest call is refused");
    check(!too_many_blocks(1, 2147483647), "one block per sequence at the largest batch");
    return failures == 0 ? 0 : 1;
}

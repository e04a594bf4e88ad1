// block_count.h -- overlap-and-save block counts of a call, computed without overflow.
//
// A launch indexes its (realization, block) items with 32-bit integers, so every entry point
// refuses calls of more than 2^31 - 1 blocks.  That check runs before any size derived from
// n_samples * batch (byte counts for the alias checks, workspace sizes), which it bounds.
#pragma once

#include <cstdint>

namespace cbessfm {

// Blocks of V valid samples covering n_samples >= 1 samples: ceil(n_samples / V).
inline long long blocks_for(int64_t n_samples, int V) {
    return n_samples / V + (n_samples % V != 0 ? 1 : 0);
}

// Whether batch >= 1 sequences of n_blocks blocks each exceed 2^31 - 1 blocks in total.
inline bool too_many_blocks(long long n_blocks, int batch) {
    return n_blocks > ((1ll << 31) - 1) / batch;
}

}  // namespace cbessfm

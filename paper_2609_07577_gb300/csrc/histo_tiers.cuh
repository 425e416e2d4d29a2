// Work thresholds of the histogram tiers (histo.cuh), settable per handle.
#pragma once
#include <stdint.h>

namespace snn {

constexpr int64_t HT_WWORK = 8192;      // most elements one warp takes alone
constexpr int64_t HT_BWORK = 1 << 16;   // most elements one 256-thread block takes
constexpr int64_t HT_GWORK = 1 << 22;   // most elements one large block takes

struct HtTiers {
    int64_t wwork = HT_WWORK;
    int64_t bwork = HT_BWORK;
    int64_t gwork = HT_GWORK;
};

}  // namespace snn

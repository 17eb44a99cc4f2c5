// eis_internal.h -- what other translation units of the library may see of a
// context (internal; the public boundary is include/eis.h).
#pragma once

#include <cstdint>

#include <nvtx3/nvToolsExt.h>

#include "eis.h"

struct eis_ctx_view {
    int device;
    const uint32_t *d_primes;  // odd primes < 2^22 on the device
    const uint64_t *d_sqtab;   // their division-free square-divisibility table
    uint32_t nprimes;
    uint32_t walk_grid;        // persistent walk grid (SMs x resident CTAs)
    uint32_t giant_grid;       // one-warp blocks of k_giant that fit at once (SMs x 4)
    int giant_compose;         // EIS_COMPOSE_*
    uint32_t step_limit;
};

// Baby-step count and log2 table size of the giant-step search for d up to
// `d` (forced > 0 picks the baby-step count).
void eis_giant_params(uint64_t d, int64_t forced, int &nbaby, int &log2n);

eis_ctx_view eis_ctx_get_view(eis_ctx *ctx);
// Account `bytes` of device memory against the context budget; false if over.
bool eis_ctx_reserve(eis_ctx *ctx, uint64_t bytes);
void eis_ctx_release(eis_ctx *ctx, uint64_t bytes);

// Host-side NVTX range for the phases a profiler timeline should show
// (plan build and launch, single queries, autotuning, server batches).  The
// header-only NVTX API costs nothing when no tool is attached.
struct EisNvtxRange {
    explicit EisNvtxRange(const char *name) { nvtxRangePushA(name); }
    ~EisNvtxRange() { nvtxRangePop(); }
    EisNvtxRange(const EisNvtxRange &) = delete;
    EisNvtxRange &operator=(const EisNvtxRange &) = delete;
};

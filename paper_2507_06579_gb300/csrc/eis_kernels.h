// eis_kernels.h -- kernel declarations shared by the .cu files of the library
// (internal; the public boundary is include/eis.h).
#pragma once

#include <cstdint>

#include "eis_bsgs.cuh"
#include "eis_common.cuh"

namespace eis {

__global__ void k_sieve(const Tile *tiles, const Seg *segs, const uint32_t *primes,
                        uint32_t nprimes, uint32_t *sqfree, uint32_t *tile_pop, int primes_only);
__global__ void k_scan_tiles(const uint32_t *tile_pop, uint32_t *tile_off, uint32_t ntiles,
                             uint32_t *total);
__global__ void k_compact(const Tile *tiles, const uint32_t *sqfree, const uint32_t *tile_off,
                          uint32_t *surv);
__global__ void k_count(const Tile *tiles, const uint32_t *flags, const uint32_t *sqfree,
                        unsigned long long *counts, const uint8_t *glog, unsigned long long *cls);
__global__ void k_expand_codes(const uint32_t *flags, const uint32_t *sqfree, uint64_t ncand,
                               uint8_t *codes);
__global__ void k_fill(uint32_t *buf, uint64_t nwords, uint32_t v);

__global__ void k_walk_plain(uint64_t d_first, uint64_t cand_first, uint32_t ncand,
                             const uint32_t *sqfree, uint32_t *flags, uint8_t *glog,
                             unsigned long long *steps_acc, int *status, uint32_t step_limit);
__global__ void k_walk_persistent(const Seg *segs, uint32_t nseg, const uint32_t *surv,
                                  const uint32_t *n_surv_ptr, uint32_t *next_ptr, uint32_t *flags,
                                  uint8_t *glog, unsigned long long *steps_acc, int *status,
                                  uint32_t step_limit, uint32_t defer_after, uint32_t *defer_list,
                                  uint32_t *defer_count, uint32_t defer_cap, int fast);
__global__ void k_giant(const uint64_t *ds, const Seg *segs, uint32_t nseg, const uint32_t *cands,
                        const uint32_t *n_ptr, uint32_t n_fixed, uint32_t *next_ptr,
                        const uint32_t *primes, const uint64_t *sqtab, uint32_t nprimes,
                        int8_t *out_g, uint32_t *flags,
                        uint8_t *glog, unsigned long long *acc, int *status, int nbaby, int log2n,
                        uint32_t max_rounds, int compose, const uint32_t *sq_flag);
__global__ void k_walk_single(uint64_t d, const uint32_t *primes, const uint64_t *sqtab,
                              uint32_t nprimes, int *out, int *status, uint32_t step_limit,
                              const uint32_t *sq_flag);
__global__ void k_sqfree_one(uint64_t d, const uint64_t *sqtab, uint32_t nprimes, uint32_t *flag);

__global__ void k_walk_record(const Seg *segs, uint32_t nseg, const uint32_t *surv,
                              const uint32_t *n_surv_ptr, uint32_t q_lo, uint32_t q_hi,
                              uint32_t *next_ptr, uint32_t *flags, uint8_t *glog,
                              unsigned long long *steps_acc, int *status, uint32_t step_limit,
                              const __grid_constant__ TuneTab tt, DRecord *recs, uint32_t *nrec,
                              uint32_t rec_cap, unsigned char *pool,
                              unsigned long long *handed_acc, int fast);
// The lane search kernel for (fast quotient, composition), and its launch
// (128 threads a block).
const void *k_bsgs_kernel(int fast, int compose);
cudaError_t launch_k_bsgs(uint32_t grid, cudaStream_t st, int fast, int compose, const Seg *segs,
                          uint32_t nseg, const DRecord *recs, const uint32_t *nrec, uint32_t rec_cap,
                          uint32_t *next_ptr, const unsigned char *pool, uint32_t *flags,
                          uint8_t *glog, unsigned long long *acc, int *status, uint32_t *fb_list,
                          uint32_t *fb_count, uint32_t fb_cap, const TuneTab &tt,
                          uint32_t max_cycles, uint32_t walk_cap, uint32_t walk_window);

}  // namespace eis

// k_sieve.cu -- candidate sieve, survivor compaction and counting kernels.
//
// Candidates are d == 5 (mod 8) (Section 1: D = { d == 5 mod 8, square-free }).
// Such d are odd, so d is square-free iff no odd prime square p^2 divides it.
// For odd p, p^2 == 1 (mod 8), hence the candidates divisible by p^2 are
// exactly d = p^2 m with m == 5 (mod 8): consecutive hits are 8 p^2 apart in
// d, p^2 apart in candidate index.  Each CTA sieves one tile of 2^16
// candidates in shared memory (8 KB bitmap) and writes it to HBM once.
#include "eis_common.cuh"
#include "eis_kernels.h"

namespace eis {

namespace {

// Primes whose hits per tile exceed this many are sieved by the whole CTA,
// larger ones by one thread each.
constexpr uint32_t kCoopP2 = 4096;

__device__ __forceinline__ void clear_bit(uint32_t *bits, uint32_t idx) {
    atomicAnd(&bits[idx >> 5], ~(1u << (idx & 31)));
}

}  // namespace

// K1: one CTA per tile.  sqfree bit k = [candidate k is square-free];
// tile_pop[t] = number of square-free candidates of tile t.
// primes_only: bit k = [candidate k is prime] instead (prime subsequence,
// Section 3.2).  For an odd prime p, p m == 5 (mod 8) iff m == 5p (mod 8)
// (p^2 == 1 mod 8), so the multiples p m (m >= 2) among the candidates are
// p apart in candidate index.
__global__ void __launch_bounds__(256) k_sieve(const Tile *__restrict__ tiles,
                                               const Seg *__restrict__ segs,
                                               const uint32_t *__restrict__ primes,
                                               uint32_t nprimes, uint32_t *__restrict__ sqfree,
                                               uint32_t *__restrict__ tile_pop, int primes_only) {
    __shared__ uint32_t bits[kTileWords];
    __shared__ uint32_t red[32];
    const Tile t = tiles[blockIdx.x];
    const Seg s = segs[t.seg];
    const uint64_t dfirst = s.d0 + 8 * (t.cand0 - s.cand0);
    const uint64_t dlast = dfirst + 8 * (uint64_t)(t.ncand - 1);
    const uint32_t nw = (t.ncand + 31) >> 5;
    for (uint32_t w = threadIdx.x; w < kTileWords; w += blockDim.x) {
        uint32_t v = 0;
        if (w < nw) {
            const uint32_t rem = t.ncand - w * 32;
            v = rem >= 32 ? kFull : ((1u << rem) - 1);
        }
        bits[w] = v;
    }
    __syncthreads();
    if (primes_only) {
        uint32_t i = 0;
        // small primes: the whole CTA strides over the hits of one prime
        for (; i < nprimes; ++i) {
            const uint64_t p = primes[i];
            if (p >= 1024 || p * p > dlast) break;
            uint64_t m = (dfirst + p - 1) / p;
            if (m < 2) m = 2;
            m += (5 * p + 8 - m % 8) % 8;  // m == 5p (mod 8)
            const uint64_t dh = m * p;
            if (dh > dlast) continue;
            const uint32_t first = (uint32_t)((dh - dfirst) >> 3);
            const uint32_t nh = (uint32_t)((dlast - dh) / (8 * p)) + 1;
            for (uint32_t h = threadIdx.x; h < nh; h += blockDim.x)
                clear_bit(bits, first + h * (uint32_t)p);
        }
        for (uint32_t j = i + threadIdx.x; j < nprimes; j += blockDim.x) {
            const uint64_t p = primes[j];
            if (p * p > dlast) break;
            uint64_t m = (dfirst + p - 1) / p;
            if (m < 2) m = 2;
            m += (5 * p + 8 - m % 8) % 8;
            for (uint64_t dh = m * p; dh <= dlast; dh += 8 * p)
                clear_bit(bits, (uint32_t)((dh - dfirst) >> 3));
        }
    } else {
    // Small primes: the whole CTA strides over the hits of one prime.
    uint32_t i = 0;
    for (; i < nprimes; ++i) {
        const uint64_t p = primes[i];
        const uint64_t p2 = p * p;
        if (p2 >= kCoopP2 || p2 > dlast) break;
        uint64_t m = (dfirst + p2 - 1) / p2;
        m += (13 - m % 8) % 8;  // m == 5 (mod 8)
        const uint64_t dh = m * p2;
        if (dh > dlast) continue;
        const uint32_t first = (uint32_t)((dh - dfirst) >> 3);
        const uint32_t nh = (uint32_t)((dlast - dh) / (8 * p2)) + 1;
        for (uint32_t h = threadIdx.x; h < nh; h += blockDim.x)
            clear_bit(bits, first + h * (uint32_t)p2);
    }
    // Larger primes: one thread per prime.
    for (uint32_t j = i + threadIdx.x; j < nprimes; j += blockDim.x) {
        const uint64_t p = primes[j];
        const uint64_t p2 = p * p;
        if (p2 > dlast) break;
        uint64_t m = (dfirst + p2 - 1) / p2;
        m += (13 - m % 8) % 8;
        for (uint64_t dh = m * p2; dh <= dlast; dh += 8 * p2)
            clear_bit(bits, (uint32_t)((dh - dfirst) >> 3));
    }
    }
    __syncthreads();
    uint32_t pop = 0;
    const uint64_t wbase = t.cand0 >> 5;
    for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) {
        const uint32_t v = bits[w];
        sqfree[wbase + w] = v;
        pop += __popc(v);
    }
    pop = block_sum(pop, red);
    if (threadIdx.x == 0) tile_pop[blockIdx.x] = pop;
}

// Exclusive scan of tile_pop into tile_off (single CTA) and the total.
__global__ void __launch_bounds__(1024) k_scan_tiles(const uint32_t *__restrict__ tile_pop,
                                                     uint32_t *__restrict__ tile_off,
                                                     uint32_t ntiles, uint32_t *__restrict__ total) {
    __shared__ uint32_t red[32];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < ntiles; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < ntiles ? tile_pop[i] : 0;
        uint32_t tot;
        const uint32_t ex = block_excl_scan(v, red, &tot);
        if (i < ntiles) tile_off[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// K1b: the square-free candidates of each tile, in increasing order, as
// a compact queue from tile_off[tile].  The tile is taken in chunks of 256
// bitmap words, one per thread and read coalesced.  A block scan of the
// words' popcounts places each word's survivors in a shared-memory stage,
// and the block copies the stage to the queue with consecutive threads
// writing consecutive entries, so the queue is written in whole lines.
__global__ void __launch_bounds__(256) k_compact(const Tile *__restrict__ tiles,
                                                 const uint32_t *__restrict__ sqfree,
                                                 const uint32_t *__restrict__ tile_off,
                                                 uint32_t *__restrict__ surv) {
    __shared__ uint32_t red[32];
    __shared__ uint32_t stage[256 * 32];  // one chunk: at most 8192 survivors
    const Tile t = tiles[blockIdx.x];
    const uint32_t nw = (t.ncand + 31) >> 5;
    const uint64_t wbase = t.cand0 >> 5;
    uint32_t out = tile_off[blockIdx.x];
    for (uint32_t c0 = 0; c0 < nw; c0 += 256) {
        const uint32_t w = c0 + threadIdx.x;
        uint32_t x = (w < nw) ? sqfree[wbase + w] : 0u;
        uint32_t tot;
        uint32_t o = block_excl_scan((uint32_t)__popc(x), red, &tot);
        const uint32_t cbase = (uint32_t)(t.cand0 + 32u * w);
        while (x) {
            stage[o++] = cbase + (uint32_t)(__ffs(x) - 1);
            x &= x - 1;
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < tot; i += 256) surv[out + i] = stage[i];
        out += tot;
        __syncthreads();
    }
}

// K4: per-interval counts.  counts[2*seg] += #E, counts[2*seg+1] += #D over
// the tile's words (ballot/popcount data already packed in the bitmaps).
// With glog, cls[3*seg + g] += #{d : log eps_d = g} for g = 0, 1, 2 (the
// class of eps_d in F_4* = {1, omega, omega^2}).
__global__ void __launch_bounds__(256) k_count(const Tile *__restrict__ tiles,
                                               const uint32_t *__restrict__ flags,
                                               const uint32_t *__restrict__ sqfree,
                                               unsigned long long *__restrict__ counts,
                                               const uint8_t *__restrict__ glog,
                                               unsigned long long *__restrict__ cls) {
    __shared__ uint32_t red[32];
    const Tile t = tiles[blockIdx.x];
    const uint32_t nw = (t.ncand + 31) >> 5;
    const uint64_t wbase = t.cand0 >> 5;
    uint32_t e = 0, dd = 0;
    for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) {
        e += __popc(flags[wbase + w]);
        dd += __popc(sqfree[wbase + w]);
    }
    e = block_sum(e, red);
    __syncthreads();
    dd = block_sum(dd, red);
    if (threadIdx.x == 0) {
        atomicAdd(&counts[2 * t.seg], (unsigned long long)e);
        atomicAdd(&counts[2 * t.seg + 1], (unsigned long long)dd);
    }
    if (glog && cls) {
        uint32_t c[3] = {0, 0, 0};
        for (uint32_t k = threadIdx.x; k < t.ncand; k += blockDim.x) {
            const uint32_t v = glog[t.cand0 + k];
            c[0] += (v == 1);
            c[1] += (v == 2);
            c[2] += (v == 3);
        }
        for (int g = 0; g < 3; ++g) {
            __syncthreads();
            const uint32_t sum = block_sum(c[g], red);
            if (threadIdx.x == 0) atomicAdd(&cls[3 * t.seg + g], (unsigned long long)sum);
        }
    }
}

// Byte codes per candidate: 0 = not in D, 1 = in D \ E, 2 = in E.
__global__ void __launch_bounds__(256) k_expand_codes(const uint32_t *__restrict__ flags,
                                                      const uint32_t *__restrict__ sqfree,
                                                      uint64_t ncand, uint8_t *__restrict__ codes) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < ncand;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t b = 1u << (k & 31);
        const uint32_t sq = sqfree[k >> 5] & b, fl = flags[k >> 5] & b;
        codes[k] = fl ? 2 : (sq ? 1 : 0);
    }
}

// L2 flush helper for benchmarks: overwrite a buffer larger than L2.
__global__ void k_fill(uint32_t *__restrict__ buf, uint64_t nwords, uint32_t v) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < nwords;
         k += (uint64_t)gridDim.x * blockDim.x)
        buf[k] = v;
}

}  // namespace eis

// k_noalloc.cu -- eis_classify_range_noalloc: classification without any
// device allocation.
//
// Who needs this: code that must not allocate device memory -- a custom
// allocator hook (calling cudaMalloc from inside it would recurse into the
// allocator it implements), a process whose GPU memory is owned by another
// framework's pool (a cudaMalloc behind the pool's back can fail or break its
// accounting), or a real-time loop that forbids allocation after start-up.
// eis_create itself allocates (prime table, stream), so such callers cannot
// hold a context.  This call does make CUDA runtime calls (memsets, launches,
// one copy and a stream synchronisation), so it is not for host functions
// enqueued with cudaLaunchHostFunc, where CUDA calls are not allowed.
//
// The scratch the pipeline needs (survivor queue, tile counts, counters and,
// when the caller does not want it, the square-free bitmap) lives in one
// file-scope __device__ array of fixed size.  Every GPU that loads the
// library holds it until the process exits.  The caller passes only the
// outputs.  The square-free sieve here tests every odd k with k^2 <= d instead
// of a prime table, so no table has to be allocated or uploaded.
#include <cstring>
#include <mutex>

#include "eis.h"
#include "eis_kernels.h"

namespace eis {
namespace {

constexpr uint64_t kNaMaxCands = (uint64_t)1 << 20;       // candidates per call
// Byte layout of the scratch array.
constexpr size_t kOffCounters = 0;      // u32 n_surv, u32 next, int status, u32 pad,
                                        // u64 steps, u64 count_E, u64 count_D
constexpr size_t kOffSeg = 256;         // one Seg
constexpr size_t kOffTilePop = 512;     // one u32 per tile (at most 16 tiles)
constexpr size_t kOffSqfree = 1024;     // kNaMaxCands / 32 words
constexpr size_t kOffQueue = kOffSqfree + kNaMaxCands / 8;  // kNaMaxCands u32
constexpr size_t kScratchBytes = kOffQueue + kNaMaxCands * 4;

static __device__ __align__(256) unsigned char g_na_scratch[kScratchBytes];

// Square-free sieve of the single interval (variant of k_sieve): odd k >= 3
// with k^2 <= d_last, composites included (their squares add nothing), so it
// needs no prime table.  Block 0 also writes the Seg the walk kernel reads.
__global__ void __launch_bounds__(256) k_na_sieve(uint64_t d0, uint32_t ncand,
                                                  uint32_t *__restrict__ sqfree) {
    __shared__ uint32_t bits[kTileWords];
    __shared__ uint32_t red[32];
    const uint32_t t = blockIdx.x;
    const uint32_t c0 = t * kTileCands;
    const uint32_t nc = min((uint32_t)kTileCands, ncand - c0);
    const uint64_t dfirst = d0 + 8ull * c0;
    const uint64_t dlast = dfirst + 8ull * (nc - 1);
    if (t == 0 && threadIdx.x == 0) {
        Seg *s = reinterpret_cast<Seg *>(g_na_scratch + kOffSeg);
        s->d0 = d0;
        s->ncand = ncand;
        s->cand0 = 0;
    }
    const uint32_t nw = (nc + 31) >> 5;
    for (uint32_t w = threadIdx.x; w < kTileWords; w += blockDim.x) {
        uint32_t v = 0;
        if (w < nw) {
            const uint32_t rem = nc - w * 32;
            v = rem >= 32 ? kFull : ((1u << rem) - 1);
        }
        bits[w] = v;
    }
    __syncthreads();
    for (uint64_t k = 3 + 2ull * threadIdx.x; k * k <= dlast; k += 2ull * blockDim.x) {
        const uint64_t k2 = k * k;
        uint64_t m = (dfirst + k2 - 1) / k2;
        m += (13 - m % 8) % 8;  // k^2 == 1 (mod 8), so k^2 m == 5 (mod 8) iff m == 5
        for (uint64_t dh = m * k2; dh <= dlast; dh += 8 * k2) {
            const uint32_t idx = (uint32_t)((dh - dfirst) >> 3);
            atomicAnd(&bits[idx >> 5], ~(1u << (idx & 31)));
        }
    }
    __syncthreads();
    uint32_t pop = 0;
    for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) {
        sqfree[(c0 >> 5) + w] = bits[w];
        pop += __popc(bits[w]);
    }
    for (int o = 16; o > 0; o >>= 1) pop += __shfl_xor_sync(kFull, pop, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = pop;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (uint32_t i = 0; i < (blockDim.x >> 5); ++i) s += red[i];
        reinterpret_cast<uint32_t *>(g_na_scratch + kOffTilePop)[t] = s;
    }
}

// Prefix of at most 16 tile counts, then the survivor queue (variant of
// k_scan_tiles + k_compact for one interval).  As in k_compact, the tile is
// taken in chunks of 256 bitmap words, one per thread; a block scan of the
// words' popcounts places each word's survivors in a shared-memory stage,
// which the block copies to the queue with consecutive threads writing
// consecutive entries.
__global__ void __launch_bounds__(256) k_na_compact(uint32_t ncand, uint32_t ntiles,
                                                    const uint32_t *__restrict__ sqfree) {
    __shared__ uint32_t red[32];
    __shared__ uint32_t stage[256 * 32];  // one chunk: at most 8192 survivors
    __shared__ uint32_t base_s;
    const uint32_t t = blockIdx.x;
    const uint32_t *pop = reinterpret_cast<const uint32_t *>(g_na_scratch + kOffTilePop);
    if (threadIdx.x == 0) {
        uint32_t b = 0;
        for (uint32_t i = 0; i < t; ++i) b += pop[i];
        base_s = b;
        if (t == ntiles - 1) {
            uint32_t *ctr = reinterpret_cast<uint32_t *>(g_na_scratch + kOffCounters);
            ctr[0] = b + pop[t];
        }
    }
    __syncthreads();
    uint32_t out = base_s;
    const uint32_t c0 = t * kTileCands;
    const uint32_t nc = min((uint32_t)kTileCands, ncand - c0);
    const uint32_t nw = (nc + 31) >> 5;
    uint32_t *queue = reinterpret_cast<uint32_t *>(g_na_scratch + kOffQueue);
    for (uint32_t w0 = 0; w0 < nw; w0 += 256) {
        const uint32_t w = w0 + threadIdx.x;
        uint32_t x = (w < nw) ? sqfree[(c0 >> 5) + w] : 0u;
        uint32_t tot;
        uint32_t o = block_excl_scan((uint32_t)__popc(x), red, &tot);
        const uint32_t cb = c0 + 32u * w;
        while (x) {
            stage[o++] = cb + (uint32_t)(__ffs(x) - 1);
            x &= x - 1;
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < tot; i += 256) queue[out + i] = stage[i];
        out += tot;
        __syncthreads();
    }
}

// #E and #D of the interval into the counters.
__global__ void __launch_bounds__(256) k_na_count(uint32_t nwords, const uint32_t *__restrict__ flags,
                                                  const uint32_t *__restrict__ sqfree) {
    unsigned long long e = 0, dd = 0;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += gridDim.x * blockDim.x) {
        e += __popc(flags[w]);
        dd += __popc(sqfree[w]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(kFull, e, o);
        dd += __shfl_xor_sync(kFull, dd, o);
    }
    if ((threadIdx.x & 31) == 0) {
        unsigned long long *c64 =
            reinterpret_cast<unsigned long long *>(g_na_scratch + kOffCounters + 16);
        atomicAdd(&c64[1], e);
        atomicAdd(&c64[2], dd);
    }
}

// Per-device set-up: the address of g_na_scratch (host code may not use the
// symbol itself) and the persistent grid size.
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
bool g_na_ready[kNaMaxDevices];
unsigned char *g_na_ptr[kNaMaxDevices];
int g_na_grid[kNaMaxDevices];

int na_setup(int device) {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (g_na_ready[device]) return EIS_OK;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || p == nullptr) return EIS_EDEVICE;
    int sms = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_walk_persistent, 256, 0) != cudaSuccess)
        return EIS_EDEVICE;
    g_na_ptr[device] = static_cast<unsigned char *>(p);
    g_na_grid[device] = sms * (occ > 0 ? occ : 1);
    g_na_ready[device] = true;
    return EIS_OK;
}

// Makes `device` current for the call and gives the caller's device back on
// every return path.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int device) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = (prev == device) || cudaSetDevice(device) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Launch with the launch's own status as the return value, so the call never
// reads (and clears) an error left pending by the caller's earlier work.
template <class... Params, class... Args>
cudaError_t launch(void (*kernel)(Params...), uint32_t grid, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace
}  // namespace eis

using namespace eis;

extern "C" int eis_classify_range_noalloc(int device, uint64_t lo, uint64_t hi, uint32_t *flags_out,
                                          uint32_t *sqfree_out, uint64_t *count_out, void *stream) {
    if (!flags_out || lo > hi || device < 0 || device >= kNaMaxDevices) return EIS_EINVAL;
    if (hi > EIS_D_LIMIT) return EIS_ERANGE;
    const uint64_t d0 = lo + ((13 - lo % 8) % 8);
    const uint64_t n = hi > d0 ? (hi - d0 + 7) / 8 : 0;
    if (n > kNaMaxCands) return EIS_ETOOLARGE;
    DeviceGuard guard(device);
    if (!guard.ok) return EIS_EDEVICE;
    int rc = na_setup(device);
    if (rc != EIS_OK) return rc;
    if (n == 0) {
        if (count_out) *count_out = 0;
        return EIS_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *base = g_na_ptr[device];
    const uint32_t ncand = (uint32_t)n, nwords = (ncand + 31) / 32;
    const uint32_t ntiles = (ncand + kTileCands - 1) / kTileCands;
    uint32_t *sq = sqfree_out ? sqfree_out : reinterpret_cast<uint32_t *>(base + kOffSqfree);
    uint32_t *ctr = reinterpret_cast<uint32_t *>(base + kOffCounters);
    unsigned long long *c64 = reinterpret_cast<unsigned long long *>(base + kOffCounters + 16);
    // The array keeps the previous call's contents: clear the counters and
    // the caller's flag words, which the walk only ORs into.
    if (cudaMemsetAsync(base + kOffCounters, 0, 64, s) != cudaSuccess ||
        cudaMemsetAsync(flags_out, 0, (size_t)nwords * 4, s) != cudaSuccess)
        return EIS_EDEVICE;
    const uint32_t count_grid = (nwords + 255) / 256 < 304 ? (nwords + 255) / 256 : 304;
    if (launch(k_na_sieve, ntiles, s, d0, ncand, sq) != cudaSuccess ||
        launch(k_na_compact, ntiles, s, ncand, ntiles, (const uint32_t *)sq) != cudaSuccess ||
        launch(k_walk_persistent, (uint32_t)g_na_grid[device], s,
               reinterpret_cast<const Seg *>(base + kOffSeg), 1u,
               reinterpret_cast<const uint32_t *>(base + kOffQueue), (const uint32_t *)ctr,
               ctr + 1, flags_out, (uint8_t *)nullptr, c64, reinterpret_cast<int *>(ctr + 2),
               1u << 26, 0u, (uint32_t *)nullptr, (uint32_t *)nullptr, 0u,
               d0 + 8 * (n - 1) < kFastDLimit ? 1 : 0) != cudaSuccess ||
        launch(k_na_count, count_grid, s, nwords, (const uint32_t *)flags_out,
               (const uint32_t *)sq) != cudaSuccess)
        return EIS_EDEVICE;
    unsigned long long host[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(host, base + kOffCounters, sizeof(host), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return EIS_EDEVICE;
    // host[0]: survivors | queue head, host[1]: status, host[2]: steps, host[3]: #E
    int status = 0;
    std::memcpy(&status, &host[1], sizeof(int));
    if (status & kErrSteps) return EIS_ESTEPS;
    if (count_out) *count_out = host[3];
    return EIS_OK;
}

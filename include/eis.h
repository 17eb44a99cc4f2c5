/*
 * eis.h -- C-ABI of the GB300 (sm_103a) Eisenstein-discriminant library.
 *
 * What it computes (Breuer & Punch, "Quadratic units and cubic fields"):
 *   D  = { d > 0 : d == 5 (mod 8), d square-free }              (Section 1)
 *   E  = { d in D : eps_d == 1 (mod 2O_K) }, eps_d the fundamental unit of
 *        K = Q(sqrt d), O_K = Z[(1+sqrt d)/2]                     (Section 1)
 *   pi_E(x) = #{ d in E : d <= x }                                (Section 1)
 * eps_d mod 2O_K is found by the infrastructure baby steps of Appendix A
 * with every generator reduced into (O_K/2O_K)* = F_4* = Z/3 (Appendix A,
 * last paragraphs before the implementation notes).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Ranges are half-open [lo, hi); pi_E(x) = count over [0, x+1).  Supported
 * values: hi <= EIS_D_LIMIT (2^44); larger give EIS_ERANGE.
 *
 * Candidates: the d == 5 (mod 8) in [lo, hi), d = d0 + 8k, k = 0..n-1, with
 * d0 the least such d >= lo.  Bit-packed outputs use 32-bit words, bit
 * (k & 31) of word (k >> 5), little-endian bit order; unused high bits of
 * the last word are 0.  Flag bit = [d in E]; square-free bit = [d in D];
 * a candidate that is not square-free has flag 0.
 *
 * Ownership: the caller owns every output buffer; the context owns its
 * device memory (prime table, bitmaps, work queues), streams and graphs.
 * A context is not thread-safe: one host thread uses it at a time.
 *
 * Errors: every function returns EIS_OK (0) or a negative EIS_E* code and
 * then writes no output.  eis_strerror() names a code.  Device memory is
 * allocated only in eis_create / eis_plan_create / the convenience calls
 * (which size their work to the context's memory budget), never inside
 * eis_plan_launch.
 */
#ifndef EIS_GB300_H
#define EIS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EIS_OK 0
#define EIS_EINVAL -1    /* null pointer where one is required, lo > hi, bad option */
#define EIS_ENOTD -2     /* is_eisenstein: d is not in D (no result written) */
#define EIS_ERANGE -3    /* hi (or d) above EIS_D_LIMIT */
#define EIS_ENOMEM -4    /* device or host allocation failed / over budget */
#define EIS_ETIMEOUT -5  /* a wait for a result ran past its limit */
#define EIS_EDEVICE -6   /* a CUDA call failed; the context should be destroyed */
#define EIS_ESTEPS -7    /* a walk ran past its step limit (never expected) */
#define EIS_EBUSY -8     /* serving: request not admitted (queue or memory full) */
#define EIS_ENOTFOUND -9 /* serving: unknown request id */
#define EIS_ETOOLARGE -10 /* eis_classify_range_noalloc: more candidates than its */
                          /* fixed scratch holds (EIS_NOALLOC_MAX_CANDIDATES)      */
#define EIS_ECANCELED -11 /* serving: the request was cancelled                    */

/* Exclusive upper bound on hi (and on d): 2^44.  Below it every baby-step
 * quantity (P, Q, P + floor(sqrt d)) is an integer below 2^23, which the
 * kernels carry exactly in fp32 registers. */
#define EIS_D_LIMIT (((uint64_t)1) << 44)

/* Execution modes (eis_set_option(EIS_OPT_MODE)). */
#define EIS_MODE_PLAIN 0      /* one launch per 2^24-wide block of d, one    */
                              /* thread per candidate                         */
#define EIS_MODE_PERSISTENT 1 /* sieve + compaction + one persistent launch   */
                              /* whose lanes steal d's from a global queue   */
                              /* (CUDA-graph captured per plan)               */

/* Options (eis_set_option / eis_get_option). */
#define EIS_OPT_MODE 1           /* EIS_MODE_*; default EIS_MODE_PERSISTENT   */
#define EIS_OPT_CTAS_PER_SM 2    /* persistent grid: CTAs per SM (default 0 = */
                                 /* occupancy maximum)                        */
#define EIS_OPT_THREADS 3        /* threads per CTA of the walk kernels (256) */
#define EIS_OPT_STEP_LIMIT 4     /* per-d baby-step limit before EIS_ESTEPS   */
#define EIS_OPT_USE_GRAPH 5      /* 1: capture plans into CUDA graphs (1)     */
#define EIS_OPT_GIANT_THRESHOLD 6 /* baby steps after which a d is handed to  */
                                  /* the giant-step kernel (0 = never)        */
#define EIS_OPT_GIANT_STRIDE 7   /* giant-step stride in baby steps (0: auto) */
#define EIS_OPT_GIANT_COMPOSE 8  /* giant-step composition: EIS_COMPOSE_*      */
#define EIS_OPT_MEM_BUDGET 9     /* read-only: the context's device-memory    */
                                 /* budget in bytes                           */
#define EIS_OPT_MEM_IN_USE 10    /* read-only: bytes charged to the budget    */
                                 /* (context tables, live plans and servers,  */
                                 /* and the lane-search table pool a freed    */
                                 /* plan leaves for the next; a plan that     */
                                 /* needs the room reclaims it)               */
#define EIS_OPT_GIANT_KERNEL 11  /* which search takes walks past the          */
                                 /* threshold: EIS_GIANT_* (EIS_GIANT_LANE)    */
#define EIS_OPT_MARK_EVERY 12    /* lane search: about 1 state in this many is */
                                 /* marked and kept in the baby table (16)     */
#define EIS_OPT_BSGS_CHUNK 13    /* lane search: survivors per round of record */
                                 /* walk + search (2^23); sizes the table pool */
#define EIS_OPT_BSGS_WALK_CAP 14 /* lane search: steps a giant cycle may walk  */
                                 /* without meeting a marked state before its  */
                                 /* d is finished by the plain walk (2^14)     */
#define EIS_OPT_BSGS_WINDOW 15   /* lane search: steps a lane walks per search */
                                 /* iteration before the warp's composition    */
                                 /* (64; 0: until every lane's walk has ended) */

/* Giant-step searches of plans (EIS_OPT_GIANT_KERNEL).  Both run after
 * EIS_OPT_GIANT_THRESHOLD baby steps without a centre. */
#define EIS_GIANT_LANE 0 /* one d per lane: the baby walk keeps the marked states  */
                         /* (Q < 1.39/mark_every * floor(sqrt d)) in a table, and   */
                         /* each giant cycle walks to a marked state and looks it  */
                         /* up (plans of >= 2^18 candidates; smaller plans walk)   */
#define EIS_GIANT_WARP 1 /* one d per warp: the full baby table in shared memory  */
                         /* (the single-query kernel)                              */

/* Giant-step compositions (EIS_OPT_GIANT_COMPOSE). */
#define EIS_COMPOSE_TEXTBOOK 0 /* product of forms, then rho until reduced      */
                               /* (default: measured slightly faster below 2^44)*/
#define EIS_COMPOSE_NUCOMP 1   /* NUCOMP / NUDUPL / NUCOMPchoose (Algorithms    */
                               /* 2-4): near-reduced output, ~1 rho step after  */

typedef struct eis_ctx eis_ctx;
typedef struct eis_plan eis_plan;

/* Per-call statistics of the last plan launch / convenience call. */
typedef struct {
    uint64_t candidates;  /* d == 5 (mod 8) examined */
    uint64_t in_D;        /* square-free candidates (#D) */
    uint64_t in_E;        /* #E */
    uint64_t baby_steps;  /* rho steps walked by the walk kernels */
    uint64_t giant_steps; /* giant steps (compositions) */
    uint64_t deferred;    /* d handed from the baby to the giant kernel */
    double ms_total;      /* device time of the whole plan (CUDA events) */
    double ms_walk;       /* device time of the walk kernel(s) */
    double ms_sieve;      /* device time of sieve + compaction */
    double ms_giant;      /* device time of the giant-step kernel(s) (lane search: */
                          /* search and fallback walk of every round)           */
    int launches;         /* kernels launched by the plan */
    int sm_count;
    uint64_t search_steps; /* of baby_steps, those walked by the lane search's   */
                           /* giant cycles (to their marked states)              */
} eis_stats;

/* ---------------------------------------------------------------------
 * Context
 * ------------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  mem_budget_bytes bounds the
 * device memory the context and its plans may hold (0: 3/4 of free memory).
 * Builds the odd-prime table up to 2^22 (for the square-free sieve of d <
 * 2^44) on the device.  *out receives the context. */
int eis_create(eis_ctx **out, int device, uint64_t mem_budget_bytes);

/* Release every resource of the context (plans made from it must be
 * destroyed first).  NULL is accepted. */
int eis_destroy(eis_ctx *ctx);

/* Static text for an EIS_* code. */
const char *eis_strerror(int code);

/* Text of the CUDA error behind the calling thread's last EIS_EDEVICE. */
const char *eis_last_cuda_error_string(void);

int eis_set_option(eis_ctx *ctx, int key, int64_t value);
int eis_get_option(eis_ctx *ctx, int key, int64_t *value);

/* Statistics of the most recent call on this context. */
int eis_get_stats(eis_ctx *ctx, eis_stats *out);

/* ---------------------------------------------------------------------
 * Convenience calls (synchronous; allocate and free per call, chunked to
 * the memory budget)
 * ------------------------------------------------------------------- */

/* *count_out = #E cap [lo, hi)   (pi_E(x) = count over [0, x+1), Section 1). */
int eis_count_range(eis_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t *count_out);

/* Classify every candidate of [lo, hi).
 *   flags_out  : ceil(n/32) words, bit = [d in E]            (nullable)
 *   sqfree_out : ceil(n/32) words, bit = [d in D]            (nullable)
 *   out_on_device : 1 if flags_out/sqfree_out are device pointers (written
 *                   in stream order on `stream`), 0 for host memory
 *   count_out  : #E cap [lo, hi)                             (nullable)
 *   stream     : cudaStream_t to run on (NULL: the context's stream)
 * Returns after the results are complete. */
int eis_classify_range(eis_ctx *ctx, uint64_t lo, uint64_t hi, uint32_t *flags_out,
                       uint32_t *sqfree_out, int out_on_device, uint64_t *count_out,
                       void *stream);

/* One byte per candidate: 0 = d not in D, 1 = d in D \ E, 2 = d in E. */
int eis_classify_range_u8(eis_ctx *ctx, uint64_t lo, uint64_t hi, uint8_t *codes_out,
                          int out_on_device, uint64_t *count_out, void *stream);

/* One byte per candidate: 0 = d not in D, else 1 + log_omega(eps_d mod 2O_K)
 * in F_4* = {1, omega, omega^2} (so 1 = d in E, 2 = eps_d == omega,
 * 3 = eps_d == omega^2 = 1 + omega), eps_d the unit reached by walking the
 * cycle forward from O_K (Appendix A: theta_{l+1}).  For the distribution
 * of eps_d mod 2O_K over the three classes (Section 1's a-priori 1/3). */
int eis_classify_range_log(eis_ctx *ctx, uint64_t lo, uint64_t hi, uint8_t *log_out,
                           int out_on_device, void *stream);

/* *result_out = 1 if d is in E, 0 if d is in D \ E (Section 1, Lemma 1.1(i)).
 * d not in D (d != 5 mod 8, or p^2 | d for an odd prime p): EIS_ENOTD and
 * nothing written; d >= EIS_D_LIMIT: EIS_ERANGE; a walk or giant-step
 * search past its limit: EIS_ESTEPS.  The square-free test spreads the prime
 * table over the whole GPU; then, in EIS_MODE_PERSISTENT (default), one warp
 * runs the baby-step giant-step search of Algorithm 1 (composition per
 * EIS_OPT_GIANT_COMPOSE), and in EIS_MODE_PLAIN one lane walks the half
 * period.  Synchronous on the context's stream; eis_get_stats reports the
 * baby and giant steps taken. */
int eis_is_eisenstein(eis_ctx *ctx, uint64_t d, int *result_out);

/* counts_out[i] = #E cap [lo[i], hi[i]) for i < n, all intervals classified
 * in one plan (one persistent launch). */
int eis_count_batch(eis_ctx *ctx, const uint64_t *lo, const uint64_t *hi, size_t n,
                    uint64_t *counts_out);

/* ---------------------------------------------------------------------
 * Autotuning
 * ------------------------------------------------------------------- */

typedef struct {
    int32_t ctas_per_sm;     /* persistent walk CTAs per SM chosen */
    int64_t giant_threshold; /* baby steps before a walk goes to a giant-step  */
                             /* search (0: never)                               */
    int64_t giant_stride;    /* warp-per-d search: baby count N (0: automatic)  */
    double ms_best;          /* device time of one pass with the chosen setting */
    double ms_default;       /* ... and with the context's previous setting     */
    int32_t trials;          /* settings timed                                  */
    int32_t giant_kernel;    /* EIS_GIANT_LANE (1 thread per d) or             */
                             /* EIS_GIANT_WARP (32 threads per d)               */
    int32_t mark_every;      /* lane search: marking density (unchanged here)   */
    int64_t bsgs_chunk;      /* lane search: survivors per round (chunk size)   */
} eis_tune_result;

/* Per-decade settings of the lane search (EIS_GIANT_LANE): a row covers the
 * d below its d_hi (rows sorted by d_hi; the last row also covers every larger
 * d).  nbaby = 0 walks those d to the centre of their period. */
typedef struct {
    uint64_t d_hi;
    int32_t nbaby;       /* baby steps before a d is handed to the search */
    int32_t mark_every;  /* about 1 state in this many is marked          */
} eis_tune_row;

#define EIS_TUNE_MAX_ROWS 8

/* Install a table of n <= EIS_TUNE_MAX_ROWS rows (n = 0 removes it).  While a
 * table is installed, plans take each d's settings from its row instead of
 * EIS_OPT_GIANT_THRESHOLD / EIS_OPT_MARK_EVERY; the search kernel is the lane
 * search.  Rows must have increasing d_hi, nbaby >= 0, 2 <= mark_every <= 4096. */
int eis_set_tune_table(eis_ctx *ctx, const eis_tune_row *rows, size_t n);

/* Copy the installed table into rows (capacity cap); *n_out = its length. */
int eis_get_tune_table(eis_ctx *ctx, eis_tune_row *rows, size_t cap, size_t *n_out);

/* For every decade [10^k, 10^(k+1)) that meets [d_lo, d_hi): time the walk
 * alone and the lane search at a grid of (nbaby, mark_every) on the top
 * 2^22 candidates of the decade inside [d_lo, d_hi), and keep the fastest
 * (the walk unless a setting is 2% faster; every setting must give the same
 * count).  The rows found replace those of the installed table for the same
 * decades (the table keeps at most EIS_TUNE_MAX_ROWS rows, merging equal
 * neighbours) and are copied to rows_out (capacity cap, *n_out rows). */
int eis_autotune_decades(eis_ctx *ctx, uint64_t d_lo, uint64_t d_hi, eis_tune_row *rows_out,
                         size_t cap, size_t *n_out);

/* Time candidate settings on the sample [lo, hi) -- a window of the d-range
 * the context will serve -- with any tuning table set aside: CTAs per SM of
 * the persistent walk; threads per d (the walk alone, the lane search at one
 * thread per d, or the warp-per-d kernel at 32 with its threshold); and the
 * lane search's round size (chunk of survivors).  The fastest stays in the
 * context, provided it beats the previous setting by more than 2% (else the
 * previous stays); the table is restored.  Every candidate runs a full plan
 * (sieve, walks, count); results are identical for every setting, only time
 * differs.  Takes a few passes of the sample. */
int eis_autotune(eis_ctx *ctx, uint64_t lo, uint64_t hi, eis_tune_result *out);

/* ---------------------------------------------------------------------
 * Classification without device allocation
 * ------------------------------------------------------------------- */

/* Largest number of candidates (d == 5 mod 8) one call of
 * eis_classify_range_noalloc accepts: 2^20, i.e. hi - lo <= 8 * 2^20. */
#define EIS_NOALLOC_MAX_CANDIDATES (((uint64_t)1) << 20)

/* The paper has no counterpart to this entry point: it exists for callers
 * that must not allocate device memory -- an allocator hook (a cudaMalloc
 * inside it would recurse into the allocator it implements), a process whose
 * GPU memory is owned by another framework's pool (an allocation behind the
 * pool's back can fail or break its accounting), or a real-time loop that
 * forbids allocation after start-up.  Such callers cannot call eis_create (it
 * allocates), so this call takes no context and calls no cudaMalloc, cudaFree
 * or any allocating library routine.  It does make other CUDA runtime calls
 * (memsets, kernel launches, one copy, a stream synchronisation), so it may
 * not be called from a host function enqueued with cudaLaunchHostFunc, where
 * CUDA calls are not allowed.
 *
 * It classifies the candidates of [lo, hi) on `device` like
 * eis_classify_range (same bit layout):
 *   flags_out  : device pointer, ceil(n/32) words, bit = [d in E]   (required)
 *   sqfree_out : device pointer, ceil(n/32) words, bit = [d in D]   (nullable)
 *   count_out  : host pointer, #E cap [lo, hi)                      (nullable)
 *   stream     : cudaStream_t, NULL for the legacy default stream
 * It returns after the results are complete.  More than
 * EIS_NOALLOC_MAX_CANDIDATES candidates give EIS_ETOOLARGE (nothing written);
 * hi above EIS_D_LIMIT gives EIS_ERANGE.  The caller's current device is the
 * same on return as on entry.  The call checks each CUDA call's own return
 * code and never reads or clears an error the caller left pending; when one
 * of its own calls fails it returns EIS_EDEVICE and that error stays pending
 * in the thread's CUDA error state, as for any failed runtime call.
 *
 * Its scratch (survivor queue, counters, a bitmap when sqfree_out is NULL,
 * about 4.2 MB) is one fixed array in the library's device memory, which every
 * GPU that loads the library holds until the process exits.  The first call
 * on a device looks up that array's device address (with the device made
 * current); make that first call before any stream capture.  All calls share
 * the array: the call clears what must start at zero, but two calls whose
 * work overlaps on the GPU (other host threads, other streams) race on it,
 * so issue them one after another. */
int eis_classify_range_noalloc(int device, uint64_t lo, uint64_t hi, uint32_t *flags_out,
                               uint32_t *sqfree_out, uint64_t *count_out, void *stream);

/* ---------------------------------------------------------------------
 * Plans: device-resident, re-launchable pipelines over a fixed set of
 * intervals (what the benchmark times).
 * ------------------------------------------------------------------- */

/* Build a plan for the n intervals [lo[i], hi[i]) in `mode`.  Allocates all
 * device memory the pipeline needs (bitmaps, survivor queue, counters) and,
 * if EIS_OPT_USE_GRAPH, captures the pipeline into a CUDA graph. */
int eis_plan_create(eis_ctx *ctx, const uint64_t *lo, const uint64_t *hi, size_t n,
                    int mode, eis_plan **out);

/* Plan flags (eis_plan_create_ex). */
#define EIS_PLAN_CLASSES 1u /* keep log eps_d per candidate and count the class  */
                            /* of eps_d in F_4* per interval                     */
#define EIS_PLAN_PRIMES 2u  /* classify the prime d == 5 (mod 8) only: the      */
                            /* "square-free" bitmap and #D then hold the primes, */
                            /* #E counts E cap P (Section 3.2)                   */

/* eis_plan_create with flags (EIS_PLAN_*). */
int eis_plan_create_ex(eis_ctx *ctx, const uint64_t *lo, const uint64_t *hi, size_t n, int mode,
                       uint32_t flags, eis_plan **out);

/* For a plan made with EIS_PLAN_CLASSES: out[3 i + g] = number of d in
 * interval i with eps_d == omega^g (mod 2O_K), g = 0 (d in E), 1, 2. */
int eis_plan_class_counts(eis_plan *plan, uint64_t *out);

/* Class counts over [lo, hi): out[g] = #{d in D : eps_d == omega^g mod 2O_K}
 * (primes_only: over the prime d only).  The a-priori expectation is 1/3 each
 * (Section 1). */
int eis_class_counts(eis_ctx *ctx, uint64_t lo, uint64_t hi, int primes_only, uint64_t out[3]);

/* Enqueue one full pass (sieve, walk, count) on `stream` (NULL: the
 * context's stream).  Asynchronous; allocates nothing. */
int eis_plan_launch(eis_plan *plan, void *stream);

/* Wait for the last launch and copy the per-interval #E to counts_out[n]. */
int eis_plan_counts(eis_plan *plan, uint64_t *counts_out);

/* Wait for the last launch and copy the per-interval #D (square-free
 * candidates, Section 1) to counts_D_out[n]. */
int eis_plan_counts_D(eis_plan *plan, uint64_t *counts_D_out);

/* Device pointers to the plan's bitmaps (valid until eis_plan_destroy):
 * flags/sqfree words for the concatenated candidates; interval i starts at
 * word word_offset[i] (host array of n entries, written if non-NULL). */
int eis_plan_bitmaps(eis_plan *plan, const uint32_t **flags, const uint32_t **sqfree,
                     uint64_t *word_offset, uint64_t *total_words);

/* Wait for the last launch and copy the plan's bitmaps (total_words words
 * each, layout as eis_plan_bitmaps) to caller memory: host pointers if
 * out_on_device is 0, device pointers otherwise.  Either may be NULL. */
int eis_plan_copy_bitmaps(eis_plan *plan, uint32_t *flags_out, uint32_t *sqfree_out,
                          int out_on_device);

/* Wait for the last launch and fill `out` (device times from CUDA events). */
int eis_plan_stats(eis_plan *plan, eis_stats *out);

int eis_plan_destroy(eis_plan *plan);

/* ---------------------------------------------------------------------
 * Serving: continuous batching of range counts and membership queries
 * ------------------------------------------------------------------- */

#define EIS_REQ_COUNT 0  /* #E cap [lo, hi) */
#define EIS_REQ_MEMBER 1 /* is d = lo in E (result 1/0; EIS_ENOTD if d is not in D) */

typedef struct eis_server eis_server;

typedef struct {
    uint32_t slots;           /* batches in flight at once, one stream each (4)  */
    uint64_t slot_candidates; /* candidates one batch holds (2^22); larger       */
                              /* requests are split into parts                   */
    uint32_t slot_requests;   /* request parts one batch holds (4096)            */
    uint32_t max_pending;     /* queued parts before submit refuses (2^20)       */
    uint32_t giant_after;     /* baby steps after which a walk is handed to the  */
                              /* warp-per-d giant-step kernel (131072); this  */
                              /* cuts the latency of batches holding a very   */
                              /* long period; 0xffffffff: never               */
    uint32_t giant_max;       /* at most this many walks per batch go to the     */
                              /* giant-step kernel (0: slot_candidates / 8)      */
    uint32_t fail_launches;   /* test hook (0): the first n batch launches fail  */
                              /* on the host before anything is enqueued, as a   */
                              /* rejected launch would; their requests complete  */
                              /* with EIS_EDEVICE and the server stops taking    */
                              /* new batches                                     */
} eis_server_config;

typedef struct {
    uint64_t requests_submitted;
    uint64_t requests_done;
    uint64_t rejected;        /* submits refused with EIS_EBUSY */
    uint64_t batches;
    uint64_t parts;
    uint64_t max_batch_parts;
    uint64_t pending_parts;
    uint64_t reserved_bytes;  /* device memory of the slots */
    uint64_t deferred;        /* walks of range parts handed to the giant-step */
                              /* kernel after giant_after baby steps           */
} eis_server_counters;

/* Start a server on ctx's device.  Device memory for `slots` batches is
 * allocated here and charged to the context budget (EIS_ENOMEM if it does not
 * fit); a dispatcher thread then packs queued requests into whichever slot is
 * free, so batches overlap on the device while new requests queue.  cfg may
 * be NULL (defaults in the struct comments).  The context must outlive the
 * server and must not be destroyed while it runs. */
int eis_server_create(eis_ctx *ctx, const eis_server_config *cfg, eis_server **out);

/* Queue a request (kind EIS_REQ_COUNT: [lo, hi); EIS_REQ_MEMBER: d = lo, hi
 * ignored).  Returns at once with *id_out; EIS_EBUSY when the queue is full
 * (nothing queued).  Thread-safe. */
int eis_server_submit(eis_server *srv, int kind, uint64_t lo, uint64_t hi, uint64_t *id_out);

/* *done_out = 1 once the request has finished. */
int eis_server_poll(eis_server *srv, uint64_t id, int *done_out);

/* Wait up to timeout_ms for a request.  On completion returns the request's
 * status (EIS_OK, EIS_ENOTD for a member query on d not in D, EIS_ESTEPS,
 * EIS_ECANCELED, EIS_EDEVICE), writes the result (#E, or 1/0 for a member
 * query) and the latency from submit to completion in microseconds, and
 * forgets the request.  EIS_ETIMEOUT leaves it queued. */
int eis_server_wait(eis_server *srv, uint64_t id, double timeout_ms, uint64_t *result_out,
                    double *latency_us_out);

/* Cancel a request: parts not yet on the device are dropped; the request
 * completes with EIS_ECANCELED. */
int eis_server_cancel(eis_server *srv, uint64_t id);

int eis_server_stats(eis_server *srv, eis_server_counters *out);

/* Finish the work in flight and queued, stop the dispatcher, free the slots. */
int eis_server_destroy(eis_server *srv);

/* Load replay: a native client thread submits request i at t_arrival_s[i]
 * seconds after the call starts (kind[i], lo[i], hi[i]); results_out[i],
 * status_out[i] and latency_us_out[i] (completion minus scheduled arrival)
 * are written for every request; *wall_s_out = total time.  Output arrays
 * are nullable.  Returns EIS_OK or the first error other than EIS_ENOTD. */
int eis_server_replay(eis_server *srv, size_t n, const double *t_arrival_s, const int *kind,
                      const uint64_t *lo, const uint64_t *hi, uint64_t *results_out,
                      int *status_out, double *latency_us_out, double *wall_s_out);

#ifdef __cplusplus
}
#endif
#endif

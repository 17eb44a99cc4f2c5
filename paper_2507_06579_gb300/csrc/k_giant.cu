// k_giant.cu -- infrastructure baby-step giant-step kernel (Algorithm 1),
// one warp per discriminant, generator classes in Z/3 (Appendix A).
//
// Baby steps: all 32 lanes run the same walk from O_K (fp32 walk of
// eis_common.cuh; it is deterministic, so every lane holds the same state),
// stopping early at the centre of a short period.  Lane t keeps state j with
// j = t mod 32 in registers, and after every 32 steps the lanes insert their
// states at once, so the hash inserts stay off the walk's dependency chain.
// Each state goes into the warp's shared-memory table twice:
//   direct  (Q_j, P_j)      -> S_j, the position delta_j of state j;
//   mirror  (Q_j, P_{j+1})  -> S_j, which is state l - j (the period is
//                               palindromic), position R - delta_j,
// and O_K itself as (2, P_1) -> 0.  The table therefore covers the window
// [R - delta_N, R + delta_N] around the regulator R.
// Giant steps: G = state N+1; lane t starts at G^(t+2) and strides by G^32,
// so round r looks up positions about (32 r + t + 2) delta_{N+1}.  Every
// giant step is reduce(G^32 * mu) (eis_infra.cuh), by the textbook
// composition or by NUCOMP/NUDUPL/NUCOMPchoose (Algorithms 2-4).  The stride
// is shorter than the window, so the first hit in (round, lane) order is the
// first giant step inside it:
//   mirror hit on j (position R - delta_j, no wrap): log eps = g(mu) + S_j,
//     because S_l - S_{l-j} = S_j;
//   direct hit on j (position R + delta_j, one wrap): log eps = g(mu) - S_j.
// G^2 already lies beyond delta_N, so no giant step can hit before the window.
#include "eis_common.cuh"
#include "eis_infra.cuh"
#include "eis_kernels.h"

namespace eis {

namespace {

struct GiantOut {
    int g;         // log eps in Z/3, or -1 (error), or -2 (not in D)
    uint32_t baby;
    uint32_t giant;
};

// The baby phase, run by all 32 lanes: states 1..N into the table (direct and
// mirror keys); done = 1 with gres = log eps_d if the centre comes first (or
// gres = -1 if the table overflowed); otherwise G = state N+1.  All outputs
// are the same on every lane.
template <bool kFast>
__device__ __forceinline__ void baby_phase(uint64_t d, uint64_t *tab, int log2n, int nbaby,
                                           int lane, int &done, int &gres, int &nb, int64_t &Ga,
                                           int64_t &Gb, int &Gg) {
    WalkState w;
    int g;
    nb = 1;
    if (walk_init<kFast>(d, w, g)) {
        done = 1;
        gres = g;
        return;
    }
    bool ok = true;
    if (lane == 0) {
        const int64_t P1 = __float_as_int(w.Pm) & 0x7fffff;
        ok = infra_insert_cas(tab, log2n, infra_key(2, P1), 0, 0);
    }
    // The state this lane holds, as the walk's raw registers (the integer
    // keys are formed at insert time).
    float kQ = 0.0f, kPm = 0.0f, kPn = 0.0f;
    int kAcc = 0;
    int j = 1;  // the next state to step from
    // Whole batches of 32 steps, unrolled with no branch inside: lane t holds
    // state j + t.  A centre anywhere in the batch sends the warp back to the
    // batch's first state to find it step by step (once per d at most).
    for (; j + 31 <= nbaby; j += 32) {
        const WalkState w0 = w;
        bool cen = false;
#pragma unroll
        for (int t = 0; t < 32; ++t) {
            const bool mine = lane == t;
            kQ = mine ? w.Q : kQ;
            kPm = mine ? w.Pm : kPm;
            kAcc = mine ? w.acc2 : kAcc;
            cen |= walk_step<kFast>(w);
            kPn = mine ? w.Pm : kPn;
        }
        if (cen) {
            w = w0;
            for (int t = 0; t < 32; ++t) {
                ++nb;
                if (walk_step<kFast>(w)) break;
            }
            done = 1;
            gres = walk_finish(w);
            return;
        }
        nb += 32;
        const int64_t Qj = (int64_t)kQ;
        const int64_t Pj = __float_as_int(kPm) & 0x7fffff;
        const int64_t Pn = __float_as_int(kPn) & 0x7fffff;
        const int Sj = (kAcc >> 1) % 3;
        ok &= infra_insert_cas(tab, log2n, infra_key(Qj, Pj), 0, Sj);
        ok &= infra_insert_cas(tab, log2n, infra_key(Qj, Pn), kMirror, Sj);
        __syncwarp();
    }
    // The rest (N not a multiple of 32), one step at a time: lane t holds
    // state j0 + t of this last batch.
    const int j0 = j;
    for (; j <= nbaby; ++j) {
        const bool mine = (j - j0) == lane;
        kQ = mine ? w.Q : kQ;
        kPm = mine ? w.Pm : kPm;
        kAcc = mine ? w.acc2 : kAcc;
        const bool centre = walk_step<kFast>(w);
        ++nb;
        if (centre) {
            done = 1;
            gres = walk_finish(w);
            return;
        }
        kPn = mine ? w.Pm : kPn;
    }
    if (lane < j - j0) {
        const int64_t Qj = (int64_t)kQ;
        const int64_t Pj = __float_as_int(kPm) & 0x7fffff;
        const int64_t Pn = __float_as_int(kPn) & 0x7fffff;
        const int Sj = (kAcc >> 1) % 3;
        ok &= infra_insert_cas(tab, log2n, infra_key(Qj, Pj), 0, Sj);
        ok &= infra_insert_cas(tab, log2n, infra_key(Qj, Pn), kMirror, Sj);
    }
    __syncwarp();
    if (!__all_sync(kFull, ok)) {
        done = 1;
        gres = -1;
        return;
    }
    Ga = (int64_t)w.Q / 2;
    Gb = __float_as_int(w.Pm) & 0x7fffff;
    Gg = (w.acc2 >> 1) % 3;
}

// reduce(X * Y): the textbook composition (compose = 0) or NUCOMP (1).
__device__ __forceinline__ bool giant_mul(int compose, const Ideal &X, const Ideal &Y, int64_t d,
                                          int64_t s, int64_t L, Ideal &out) {
    return compose ? ideal_mul_nucomp(X, Y, d, s, L, out) : ideal_mul(X, Y, d, s, out);
}

// The BSGS of one d by one warp (all 32 lanes call it with the same d).
__device__ GiantOut giant_one(uint64_t d, uint64_t *tab, int log2n, int nbaby, uint32_t max_rounds,
                              int compose) {
    const int lane = threadIdx.x & 31;
    GiantOut res{-1, 0, 0};
    for (uint32_t i = lane; i < (1u << log2n); i += 32) tab[i] = 0;
    __syncwarp();
    // ---- baby steps (all lanes)
    int done = 0, gres = 0, nb = 0;
    int64_t Ga = 0, Gb = 0;
    int Gg = 0;
    if (d < kFastDLimit)
        baby_phase<true>(d, tab, log2n, nbaby, lane, done, gres, nb, Ga, Gb, Gg);
    else
        baby_phase<false>(d, tab, log2n, nbaby, lane, done, gres, nb, Ga, Gb, Gg);
    __syncwarp();
    res.baby = (uint32_t)nb;
    if (done) {
        res.g = gres;
        return res;
    }
    Ideal G;
    G.a = Ga;
    G.b = Gb;
    G.g = Gg;
    const int64_t s = (int64_t)isqrt44(d);
    const int64_t dd = (int64_t)d;
    const int64_t L = (int64_t)isqrt44((uint64_t)s);  // floor(d^(1/4))
    // ---- lane t: mu = G^(t+1) by a product scan over the lanes (five rounds
    // of shuffles, each a composition on the lanes that receive), the stride
    // G^32 from lane 31, then mu = G^(t+2): six compositions deep.
    Ideal mu = G;
    bool ok = true;
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        Ideal o;
        o.a = __shfl_up_sync(kFull, mu.a, k);
        o.b = __shfl_up_sync(kFull, mu.b, k);
        o.g = __shfl_up_sync(kFull, mu.g, k);
        if (lane >= k) {
            Ideal t;
            ok &= giant_mul(compose, mu, o, dd, s, L, t);
            mu = t;
        }
    }
    Ideal stride;  // G^32
    stride.a = __shfl_sync(kFull, mu.a, 31);
    stride.b = __shfl_sync(kFull, mu.b, 31);
    stride.g = __shfl_sync(kFull, mu.g, 31);
    {
        Ideal t;
        ok &= giant_mul(compose, mu, G, dd, s, L, t);
        mu = t;
    }
    uint32_t giants = 6;  // compositions on a lane's way to its first giant step
    if (!__all_sync(kFull, ok)) return res;
    // the stride is fixed from here on: the textbook composition takes the
    // search's lean product (fp32 Euclid, c of the stride computed once)
    const int64_t cS = compose ? 0 : lean_cG(stride, dd);
    for (uint32_t r = 0; r < max_rounds; ++r) {
        const uint64_t e = infra_find(tab, log2n, infra_key(2 * mu.a, mu.b));
        const unsigned hit = __ballot_sync(kFull, e != 0);
        if (hit) {
            const int win = __ffs(hit) - 1;
            int g = 0;
            if (lane == win) {
                const int Sj = (int)(e & 3);
                g = (e & 4) ? (mu.g + Sj) % 3 : (mu.g + 3 - Sj) % 3;
            }
            res.g = __shfl_sync(kFull, g, win);
            res.giant = giants + 32 * r + (uint32_t)win;
            return res;
        }
        Ideal t;
        int64_t Qm;
        ok = compose ? giant_mul(compose, mu, stride, dd, s, L, t) : lean_mul(mu, stride, cS, dd, s, t, Qm);
        mu = t;
        if (!__all_sync(kFull, ok)) return res;
        giants += 32;
    }
    return res;  // no hit within max_rounds: error
}

}  // namespace

// One warp per item; items are taken from a global counter.
//   ds != nullptr : item i is d = ds[i]; out_g[i] = 0 (not in D),
//                   1 + log eps_d, or -1 (error); the square-free test runs
//                   against the prime table (division-free, eis_common.cuh),
//                   unless sq_flag (one d) holds the answer of k_sqfree_one.
//   ds == nullptr : item i is candidate cands[i] of the Seg layout (already
//                   square-free); its flag bit / log byte are written.
// Dynamic shared memory: (blockDim.x / 32) tables of 2^log2n uint64.
__global__ void __launch_bounds__(32) k_giant(const uint64_t *__restrict__ ds,
                                               const Seg *__restrict__ segs, uint32_t nseg,
                                               const uint32_t *__restrict__ cands,
                                               const uint32_t *__restrict__ n_ptr, uint32_t n_fixed,
                                               uint32_t *__restrict__ next_ptr,
                                               const uint32_t *__restrict__ primes,
                                               const uint64_t *__restrict__ sqtab, uint32_t nprimes,
                                               int8_t *__restrict__ out_g,
                                               uint32_t *__restrict__ flags,
                                               uint8_t *__restrict__ glog,
                                               unsigned long long *__restrict__ acc,
                                               int *__restrict__ status, int nbaby, int log2n,
                                               uint32_t max_rounds, int compose,
                                               const uint32_t *__restrict__ sq_flag) {
    extern __shared__ uint64_t smem_tab[];
    uint64_t *tab = smem_tab + (size_t)(threadIdx.x >> 5) * (1u << log2n);
    const int lane = threadIdx.x & 31;
    const uint32_t n = n_ptr ? min(*n_ptr, n_fixed) : n_fixed;
    unsigned long long baby = 0, giant = 0;
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(next_ptr, 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= n) break;
        if (ds) {
            const uint64_t d = ds[item];
            const bool sq = sq_flag ? (*sq_flag == 0)
                                    : warp_squarefree_fast(d, primes, sqtab, nprimes);
            if (d % 8 != 5 || !sq) {
                if (lane == 0) out_g[item] = 0;
                continue;
            }
            const GiantOut r = giant_one(d, tab, log2n, nbaby, max_rounds, compose);
            if (lane == 0) {
                out_g[item] = (int8_t)(r.g >= 0 ? 1 + r.g : -1);
                if (r.g < 0) atomicOr(status, kErrGiant);
            }
            baby += r.baby;
            giant += r.giant;
        } else {
            const uint32_t cand = cands[item];
            const uint64_t d = cand_to_d(segs, nseg, cand);
            const GiantOut r = giant_one(d, tab, log2n, nbaby, max_rounds, compose);
            if (lane == 0) {
                if (r.g < 0) {
                    atomicOr(status, kErrGiant);
                } else {
                    if (r.g == 0) atomicOr(&flags[cand >> 5], 1u << (cand & 31));
                    if (glog) glog[cand] = (uint8_t)(1 + r.g);
                }
            }
            baby += r.baby;
            giant += r.giant;
        }
        __syncwarp();
    }
    if (lane == 0 && acc) {
        atomicAdd(&acc[0], baby);
        atomicAdd(&acc[1], giant);
    }
}

}  // namespace eis

// Host model of the lane-per-d infrastructure search (eis_bsgs.cuh), used by
// test_bsgs_host.py.  The baby steps here are plain 64-bit integer steps of
// the continued fraction; the table, its index, the marking threshold, the
// giant steps (eis_infra.cuh) and the search order are the library's own
// code.  Reads lines
//     d N tau compose extra verify wide
// (compose: 0 the lean textbook product, 1 the lean NUCOMP, 2 the general
// textbook code, 3 the general NUCOMP) and
// prints one line per d:
//     status g babysteps cycles walksteps k jl hit
// status 0 = centre reached in the baby walk (g = log eps_d), 1 = found by
// the giant-step search, 2 = fallback (too few marked states: the search
// declines the d), negative = failure.  `extra` > 0 makes every cycle walk
// up to that many further steps after its marked state (pseudo-random per
// cycle), as lanes of a warp do while they wait for each other; extra = -1
// is the kernel's order: each cycle looks up its first marked state x only
// (under both keys) and the next composition starts from state x + 1.  With
// verify = 1 the whole period is walked first and every hit is checked to
// lie at position l - j or l + j of the first period (hit = 1 if checked).
// wide = 1 strides by G' = reduce(a_jl * a_j'), a_j' the last table state at
// least kBsgsWideGap steps before jl (the kernels' stride), wide = 0 by a_jl.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <map>
#include <utility>
#include <vector>

#include "eis_bsgs.cuh"

using namespace eis;

static int64_t isqrt_host(int64_t d) {
    int64_t s = (int64_t)std::sqrt((double)d);
    while (s * s > d) --s;
    while ((s + 1) * (s + 1) <= d) ++s;
    return s;
}

static int cls(int64_t P) { return 1 + (int)((P >> 1) & 1); }  // log of a step's factor mod 2

struct St {
    int64_t P, Q, Qp;
};

// One baby step; true when the new state is a centre of the period.
static bool step(St &w, int64_t s) {
    const int64_t q = (w.P + s) / w.Q;
    const int64_t Pn = q * w.Q - w.P;
    const int64_t Qn = w.Qp + q * (w.P - Pn);
    const bool centre = (Qn == w.Q) || (Pn == w.P);
    w.Qp = w.Q;
    w.Q = Qn;
    w.P = Pn;
    return centre;
}

int main() {
    long long d_, N, compose, extra, verify, wide;
    double tau_d;
    while (std::scanf("%lld %lld %lf %lld %lld %lld %lld", &d_, &N, &tau_d, &compose, &extra,
                      &verify, &wide) == 7) {
        const int64_t d = d_;
        const int64_t s = isqrt_host(d), L = isqrt_host(s);
        const bool fast = (uint64_t)d < kFastDLimit;
        const float T = bsgs_threshold((float)tau_d, (uint64_t)s);
        uint64_t rng = (uint64_t)d * 0x9E3779B97F4A7C15ull + 1;
        // whole period (verify): position of every state (Q, P) of a_1..a_l
        std::map<std::pair<int64_t, int64_t>, int64_t> pos;
        int64_t ell = 0;
        // baby walk from a_1
        const int64_t a0 = (1 + s) / 2;
        const int64_t P1 = 2 * a0 - 1, Q1 = (d - P1 * P1) / 2;
        if (verify) {
            St w{P1, Q1, 2};
            int64_t j = 1;
            pos[{w.Q, w.P}] = 1;
            while (w.Q != 2) {
                step(w, s);
                ++j;
                pos[{w.Q, w.P}] = j;
            }
            ell = j;  // a_l has Q = 2
        }
        if (Q1 == 2) {
            std::printf("0 %d 1 0 0 0 0 0\n", cls(P1) % 3);
            continue;
        }
        std::vector<DEntry> tab;
        tab.push_back(DEntry{float_bits(2.0f), float_bits(bsgs_num(P1, s, fast)), 0u, 0u});
        // pad holds the entry's baby position j here (the library leaves it 0)
        St w{P1, Q1, 2};
        int S = cls(P1) % 3;
        int64_t j = 1, jl = 0;
        int g = -1;
        for (;;) {
            if ((float)w.Q < T && (int)tab.size() < kBsgsKmax) {
                tab.push_back(DEntry{float_bits((float)w.Q), float_bits(bsgs_num(w.P, s, fast)),
                                     (uint32_t)S, (uint32_t)j});
                jl = j;
            }
            if (j >= N || (int)tab.size() == kBsgsKmax) break;
            const bool c = step(w, s);
            ++j;
            S = (S + cls(w.P)) % 3;
            if (c) {
                // centre at state j: odd type (l = 2j - 1 ... as the kernels' rule)
                // Q_j == Q_{j-1}: l = 2(j-1)+1, log eps = 2 S_{j-1} + log P_j;
                // P_j == P_{j-1}: l = 2(j-1),   log eps = 2 S_{j-1}.
                const int Sprev = (S - cls(w.P) % 3 + 3) % 3;
                g = (w.Q == w.Qp) ? (2 * Sprev + cls(w.P)) % 3 : (2 * Sprev) % 3;
                break;
            }
        }
        if (g >= 0) {
            std::printf("0 %d %lld 0 0 %d %lld 0\n", g, (long long)j, (int)tab.size(), (long long)jl);
            continue;
        }
        const int64_t baby = j;
        if (jl < kBsgsMinJl) {
            std::printf("2 -1 %lld 0 0 %d %lld 0\n", (long long)baby, (int)tab.size(), (long long)jl);
            continue;
        }
        std::vector<uint8_t> slots(kBsgsSlots);
        bsgs_index(tab.data(), (int)tab.size(), slots.data());
        const DEntry &ge = tab.back();
        const Ideal G{(int64_t)bits_float(ge.q) / 2,
                      (int64_t)bits_float(ge.num) - s, (int)(ge.s % 3)};
        // the stride Y: a_jl, or reduce(a_jl * a_j') (taken by the first cycle)
        int ej = -1;
        if (wide)
            for (int e = 1; e + 1 < (int)tab.size(); ++e)
                if ((int64_t)tab[e].pad + kBsgsWideGap <= jl) ej = e;
        Ideal Y = G;
        int64_t cY = lean_cG(G, d);
        Ideal Aj = G;
        int64_t cAj = cY;
        if (ej > 0) {
            Aj = Ideal{(int64_t)bits_float(tab[ej].q) / 2, (int64_t)bits_float(tab[ej].num) - s,
                       (int)(tab[ej].s % 3)};
            cAj = lean_cG(Aj, d);
        }
        Ideal mu = G;
        int64_t wmu = cY;  // mu = G
        int64_t cycles = 0, walked = 0;
        int status = -1, hitok = 0;
        // verify: absolute position (steps from a_0, not reduced mod l) of the
        // state the search stands on
        int64_t abs_pos = jl, cur_pos = jl;  // cur_pos = position mod l in [1, l]
        auto where = [&](int64_t Q, int64_t P) -> int64_t { return pos.at({Q, P}); };
        for (; cycles < (1 << 20) && status < 0; ++cycles) {
            Ideal nx;
            int64_t Qm = 0;
            const bool first = cycles == 0 && ej > 0;
            if (!bsgs_giant((int)compose, mu, wmu, first ? Aj : Y, first ? cAj : cY, d, s, L, nx, Qm)) {
                status = -2;
                break;
            }
            if (first) {  // G' = reduce(a_jl * a_j') is the stride from now on
                Y = nx;
                cY = -Qm / 2;  // (b^2 - d)/(4a) = -Q_{-1}/2
            }
            St v{nx.b, 2 * nx.a, Qm};
            if (verify) {
                const int64_t np = where(v.Q, v.P);
                abs_pos += ((np - cur_pos) % ell + ell) % ell;
                cur_pos = np;
            }
            int gc = nx.g;
            bool passed = false, pending = false;
            int64_t Qx = 0;
            int gx = 0;
            int64_t more = 0;  // extra steps after the cycle's marked state
            int64_t nstep = 0;
            for (;;) {
                step(v, s);
                ++nstep;
                ++walked;
                if (verify) {
                    ++abs_pos;
                    cur_pos = cur_pos % ell + 1;
                }
                gc = (gc + cls(v.P)) % 3;
                const uint32_t num = float_bits(bsgs_num(v.P, s, fast));
                if (pending) {  // mirror key (Q_x, P_{x+1}) of the marked state x before
                    const int e = bsgs_find(tab.data(), slots.data(), float_bits((float)Qx), num);
                    pending = false;
                    if (e >= 0) {
                        g = (gx + (int)(tab[e].s % 3)) % 3;
                        if (verify) hitok = (abs_pos - 1 == ell - (int64_t)tab[e].pad) ? 1 : -1;
                        status = 1;
                        break;
                    }
                    if (extra < 0) break;  // kernel order: compose from x + 1
                }
                if ((float)v.Q < T) {
                    const int e = bsgs_find(tab.data(), slots.data(), float_bits((float)v.Q), num);
                    passed = true;
                    if (e >= 0) {  // direct key (Q_x, P_x)
                        g = (gc - (int)(tab[e].s % 3) + 3) % 3;
                        if (verify) hitok = (abs_pos == ell + (int64_t)tab[e].pad) ? 1 : -1;
                        status = 1;
                        break;
                    }
                    pending = true;
                    Qx = v.Q;
                    gx = gc;
                    if (extra > 0) {
                        rng = rng * 6364136223846793005ull + 1442695040888963407ull;
                        more = (int64_t)((rng >> 33) % (uint64_t)(extra + 1));
                    }
                }
                if (passed && !pending) {
                    if (more <= 0) break;
                    --more;
                }
                if (nstep > (1 << 22)) {
                    status = -3;
                    break;
                }
            }
            mu = Ideal{v.Q / 2, v.P, gc};
            wmu = -v.Qp / 2;
        }
        std::printf("%d %d %lld %lld %lld %d %lld %d\n", status, g, (long long)baby, (long long)cycles,
                    (long long)walked, (int)tab.size(), (long long)jl, hitok);
        std::fflush(stdout);
    }
    return 0;
}

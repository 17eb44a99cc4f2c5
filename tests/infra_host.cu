// Host driver for the giant-step ideal arithmetic (eis_infra.cuh), used by
// test_infra_host.py.  Reads lines "d a1 b1 g1 a2 b2 g2" (two ideals
// [a, (b + sqrt d)/2] with generator classes g in Z/3) and prints, for the
// textbook composition, for NUCOMP/NUDUPL/NUCOMPchoose, for the search's
// lean textbook product (fp32 Euclid, the second ideal's c precomputed) and
// for its lean NUCOMP (fp32 Euclid runs, both c's passed in), whether the
// reduced product was formed and its (a, b, g):
//   okT aT bT gT okN aN bN gN okL aL bL gL okM aM bM gM
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "eis_bsgs.cuh"
#include "eis_infra.cuh"

static int64_t isqrt_host(int64_t d) {
    int64_t s = (int64_t)std::sqrt((double)d);
    while (s * s > d) --s;
    while ((s + 1) * (s + 1) <= d) ++s;
    return s;
}

int main() {
    long long d, a1, b1, g1, a2, b2, g2;
    while (std::scanf("%lld %lld %lld %lld %lld %lld %lld", &d, &a1, &b1, &g1, &a2, &b2, &g2) == 7) {
        const int64_t s = isqrt_host(d), L = isqrt_host(s);
        const eis::Ideal X{a1, b1, (int)g1}, Y{a2, b2, (int)g2};
        eis::Ideal T{0, 0, 0}, N{0, 0, 0}, Le{0, 0, 0};
        const bool okT = eis::ideal_mul(X, Y, d, s, T);
        const bool okN = eis::ideal_mul_nucomp(X, Y, d, s, L, N);
        int64_t Qm = 0;
        bool okL = eis::lean_mul(X, Y, eis::lean_cG(Y, d), d, s, Le, Qm);
        // Q_{-1} of the result must be (d - P^2) / Q
        okL = okL && Qm * 2 * Le.a == d - Le.b * Le.b;
        eis::Ideal M{0, 0, 0};
        int64_t Qm2 = 0;
        bool okM = eis::lean_nucomp(X, eis::lean_cG(X, d), Y, eis::lean_cG(Y, d), d, s, L, M, Qm2);
        okM = okM && Qm2 * 2 * M.a == d - M.b * M.b;
        std::printf("%d %lld %lld %d %d %lld %lld %d %d %lld %lld %d %d %lld %lld %d\n", okT ? 1 : 0,
                    (long long)T.a, (long long)T.b, T.g, okN ? 1 : 0, (long long)N.a, (long long)N.b, N.g,
                    okL ? 1 : 0, (long long)Le.a, (long long)Le.b, Le.g, okM ? 1 : 0, (long long)M.a,
                    (long long)M.b, M.g);
        std::fflush(stdout);  // one answer per line, for interactive use
    }
    return 0;
}

// Host driver for the integer helpers of eis_common.cuh used by
// test_common_host.py: reads one d per line and prints isqrt44(d).
#include <cstdint>
#include <cstdio>

#include "eis_common.cuh"

int main() {
    unsigned long long d;
    while (std::scanf("%llu", &d) == 1) std::printf("%llu\n", (unsigned long long)eis::isqrt44(d));
    return 0;
}

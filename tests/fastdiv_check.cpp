// Check of the multiply-shift division of rism3d_internal.h (make_fastdiv, the round-up
// method of Granlund and Montgomery) against the hardware quotient n / d. The kernels
// evaluate q = (umulhi(n, mul) + n) >> l in 32-bit unsigned arithmetic; here the high
// product is taken from a 64-bit multiply. Covered: every divisor up to 1024 with every
// n below 2^18, and every divisor of the form 2^a 3^b 5^c below 2^27 (the plane, row and
// grid sizes the solver divides by) with n at and around 2000 multiples of d spread up to
// 2^31 - 1. Prints "OK" and exits 0 when every quotient matches.
#include "rism3d_internal.h"

#include <cstdint>
#include <cstdio>
#include <vector>

static unsigned quotient(unsigned n, const rism::FastDiv &f) {
    const unsigned hi = (unsigned)(((uint64_t)n * f.mul) >> 32);
    return (hi + n) >> f.l;
}

int main() {
    long long checked = 0, bad = 0;
    auto check = [&](unsigned n, unsigned d, const rism::FastDiv &f) {
        ++checked;
        if (quotient(n, f) != n / d) {
            if (bad < 5) std::printf("mismatch: n %u d %u got %u want %u\n", n, d, quotient(n, f), n / d);
            ++bad;
        }
    };
    for (unsigned d = 1; d <= 1024; ++d) {
        const rism::FastDiv f = rism::make_fastdiv(d);
        for (unsigned n = 0; n < (1u << 18); ++n) check(n, d, f);
    }
    std::vector<unsigned> smooth;
    for (uint64_t a = 1; a < (1ull << 27); a *= 2)
        for (uint64_t b = a; b < (1ull << 27); b *= 3)
            for (uint64_t c = b; c < (1ull << 27); c *= 5) smooth.push_back((unsigned)c);
    const uint64_t top = (1ull << 31) - 1;
    for (unsigned d : smooth) {
        const rism::FastDiv f = rism::make_fastdiv(d);
        const uint64_t qmax = top / d;
        for (int i = 0; i <= 2000; ++i) {
            const uint64_t q = qmax * (uint64_t)i / 2000;
            for (int64_t off = -1; off <= 1; ++off) {
                const int64_t n = (int64_t)(q * d) + off;
                if (n >= 0 && (uint64_t)n <= top) check((unsigned)n, d, f);
            }
            const uint64_t last = q * d + d - 1;      // largest n with quotient q
            if (last <= top) check((unsigned)last, d, f);
        }
        check((unsigned)top, d, f);
    }
    std::printf("%lld quotients, %lld mismatches, %zu smooth divisors\n", checked, bad, smooth.size());
    std::printf("%s\n", bad ? "FAILED" : "OK");
    return bad != 0;
}

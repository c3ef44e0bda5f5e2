// Host check of the exact binary64 running sum used by the FP64 sweeps
// (paper_0912_4506_gb300/csrc/emusum.cuh): every form of it, fed 6-tuples of
// positive normal doubles, must give the host's sequential IEEE-754 sum
// ((((x0 + x1) + x2) + x3) + x4) + x5 bit for bit whenever it does not flag the
// tuple for the FP64 unit, and all forms must flag the same tuples.
// Usage: emusum_check SEED COUNT; prints counts, exits 1 on any mismatch.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>

#include "../paper_0912_4506_gb300/csrc/emusum.cuh"

using namespace jac::emusum;

static uint64_t bits(double x) {
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
}

template <int F>
static double word_sum(const double* x, uint32_t* bad) {
    const Mul k = make_mul(1u);
    Words w = first_w<F>(unpack_w(x[0], k), unpack_w(x[1], k), k);
    for (int i = 2; i < 6; ++i) add_w<F>(w, unpack_w(x[i], k), k);
    *bad = w.bad;
    return pack_w(w, k);
}

int main(int argc, char** argv) {
    std::mt19937_64 rng(argc > 1 ? atoi(argv[1]) : 1);
    const long long n = argc > 2 ? atoll(argv[2]) : 1000000;
    std::uniform_real_distribution<double> U(0.0, 1.0);
    long long fast = 0, errors = 0;
    for (long long it = 0; it < n; ++it) {
        double x[6];
        const int mode = (int)(it % 5);
        for (int i = 0; i < 6; ++i) {
            if (mode == 0) {
                x[i] = U(rng);  // U[0,1)
            } else if (mode == 1) {
                x[i] = 0.5 + 0.01 * U(rng);  // a smooth field
            } else if (mode == 2) {
                x[i] = std::ldexp(1.0 + U(rng), -(int)(rng() % 12));  // gaps 0..11
            } else if (mode == 3) {  // random significands over 48 binades
                const uint64_t b = (uint64_t)(1000 + rng() % 48) << 52 | (rng() >> 12);
                memcpy(&x[i], &b, 8);
            } else {  // short significands, close exponents: many exact ties
                const uint64_t b = (uint64_t)(1023 - (int)(rng() % 6)) << 52 |
                                   ((rng() >> 12) & ~((1ull << (rng() % 52)) - 1));
                memcpy(&x[i], &b, 8);
            }
            if (x[i] < 1e-300) x[i] = 0.25;  // positive normal operands only
        }
        double want = x[0] + x[1];
        for (int i = 2; i < 6; ++i) want = want + x[i];
        Acc a = first(unpack(x[0]), unpack(x[1]));
        for (int i = 2; i < 6; ++i) add(a, unpack(x[i]));
        uint32_t b0, b1, b2, b3;
        const double w0 = word_sum<0>(x, &b0), w1 = word_sum<1>(x, &b1);
        const double w2 = word_sum<2>(x, &b2), w3 = word_sum<3>(x, &b3);
        const bool flagged = a.bad != 0;
        if ((b0 != 0) != flagged || (b1 != 0) != flagged || (b2 != 0) != flagged ||
            (b3 != 0) != flagged) {
            ++errors;
            continue;
        }
        if (flagged) continue;
        ++fast;
        const uint64_t w = bits(want);
        if (bits(pack(a)) != w || bits(w0) != w || bits(w1) != w || bits(w2) != w ||
            bits(w3) != w) {
            if (errors < 5) printf("mismatch (mode %d): want %a got %a\n", mode, want, pack(a));
            ++errors;
        }
    }
    printf("tuples %lld fast %lld errors %lld\n", n, fast, errors);
    return errors != 0;
}

// Host check of the sampled-capacity bound of the row-tile update: for count
// vectors of a 1-in-samp sample of m packets (sum <= m/samp + tile), the sum
// of sample_capacity() over the tiles must not exceed
// sample_capacity_bound(), which places the overflow list in the workspace.
// Prints one line per case: "m nb kind sum bound".  Built and run by
// tests/test_capacity_bound.py.
#include <cstdio>
#include <cstdint>
#include <random>
#include <vector>

#include "update_binned.h"

int main() {
    const uint32_t samp = 16, tile = 1024;
    std::mt19937_64 rng(7);
    const uint64_t ms[] = {1ull << 16, 1ull << 20, 3ull << 22, 1ull << 26, 1ull << 28};
    const uint32_t nbs[] = {1, 7, 1024, 8192};
    for (uint64_t m : ms) {
        for (uint32_t nb : nbs) {
            const uint64_t total = m / samp + tile;          // sampled packets, the largest possible
            for (int kind = 0; kind < 4; ++kind) {
                std::vector<uint64_t> c(nb, 0);
                if (kind == 0) {                             // even
                    for (uint32_t b = 0; b < nb; ++b) c[b] = total / nb + (b < total % nb);
                } else if (kind == 1) {                      // one tile takes everything
                    c[0] = total;
                } else if (kind == 2) {                      // geometric halves
                    uint64_t left = total;
                    for (uint32_t b = 0; b < nb && left; ++b) {
                        const uint64_t t = b + 1 < nb ? (left + 1) / 2 : left;
                        c[b] = t;
                        left -= t;
                    }
                } else {                                     // random split
                    std::vector<double> w(nb);
                    double sw = 0;
                    for (auto &x : w) { x = std::exponential_distribution<double>(1.0)(rng); sw += x; }
                    uint64_t used = 0;
                    for (uint32_t b = 0; b < nb; ++b) { c[b] = (uint64_t)(total * (w[b] / sw)); used += c[b]; }
                    c[0] += total - used;
                }
                uint64_t sum = 0;
                for (uint32_t b = 0; b < nb; ++b) sum += cbaa::sample_capacity((uint32_t)c[b], samp);
                const uint64_t bound = cbaa::sample_capacity_bound(m, nb, samp, tile);
                std::printf("%llu %u %d %llu %llu\n", (unsigned long long)m, nb, kind, (unsigned long long)sum,
                            (unsigned long long)bound);
            }
        }
    }
    // the exact ceiling of sqrt(c + 1) inside sample_capacity
    for (uint64_t c = 0; c < 200000; c += 1 + c / 7) {
        const uint32_t cap = cbaa::sample_capacity((uint32_t)c, 1);
        uint64_t r = 1;
        while (r * r < c + 1) ++r;
        const uint64_t want = c + c / 8 + 4 * r + 256;
        if (cap != want) { std::printf("bad %llu %u %llu\n", (unsigned long long)c, cap, (unsigned long long)want); return 1; }
    }
    return 0;
}

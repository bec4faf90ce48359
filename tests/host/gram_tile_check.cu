// Host check of the Gram kernels' tile numbering (gram_tile in blockops.h):
// for every tile count T = 1..16 the threads 0 .. 767 cover each tile of the
// three outputs exactly once (outputs 0 and 1: the upper tiles ti <= tj only), the
// numbered tiles come first and every thread past them gets none.
// Prints "ok" and exits 0, or prints the first mismatch and exits 1.
#include <cstdio>
#include <set>
#include <tuple>

#include "blockops.h"

int main() {
    for (int T = 1; T <= 16; ++T) {
        std::set<std::tuple<int, int, int>> seen;
        int last = -1;
        for (int t = 0; t < 768; ++t) {
            int g = -1, ti = -1, tj = -1;
            if (!plhr::gram_tile(t, T, g, ti, tj)) continue;
            if (t != last + 1) { std::printf("T=%d: tile at t=%d after a gap\n", T, t); return 1; }
            last = t;
            const bool valid = g >= 0 && g <= 2 && ti >= 0 && ti < T && tj >= 0 && tj < T && (g == 2 || ti <= tj);
            if (!valid || !seen.insert({g, ti, tj}).second) {
                std::printf("T=%d: t=%d gives (%d, %d, %d)\n", T, t, g, ti, tj);
                return 1;
            }
        }
        const size_t want = (size_t)T * (T + 1) + (size_t)T * T;
        if (seen.size() != want || (size_t)(last + 1) != want) {
            std::printf("T=%d: %zu tiles, want %zu\n", T, seen.size(), want);
            return 1;
        }
    }
    std::printf("ok\n");
    return 0;
}

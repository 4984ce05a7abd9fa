// Host build of csrc/packed.cuh for tests/test_packed_index.py.
//   check_packed            -> the layout and the inverse for every n up to
//                              300 (all positions) and for large n up to
//                              65535 (every row start, its neighbours and
//                              random positions); prints "ok <positions>"
//   check_packed dump <n>   -> tri_index(n, a, b) for a <= b, row by row
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>

#include "../../paper_2608_06536_b300/csrc/packed.cuh"

using jk::packed::tri_count;
using jk::packed::tri_index;
using jk::packed::tri_advance;
using jk::packed::tri_row_col;

static long long checked = 0;

static bool inverse_ok(int n, long long t) {
    int a = -1, b = -1;
    tri_row_col(n, t, &a, &b);
    ++checked;
    if (a < 0 || a > b || b >= n || tri_index(n, a, b) != t) {
        printf("n=%d t=%lld -> (%d, %d)\n", n, t, a, b);
        return false;
    }
    return true;
}

int main(int argc, char **argv) {
    if (argc == 3 && !strcmp(argv[1], "dump")) {
        const int n = atoi(argv[2]);
        for (int a = 0; a < n; a++)
            for (int b = a; b < n; b++) printf("%lld\n", tri_index(n, a, b));
        return 0;
    }
    // small n: the positions are 0, 1, ..., n(n+1)/2 - 1 in row-major order,
    // and every position inverts
    for (int n = 1; n <= 300; n++) {
        long long want = 0;
        for (int a = 0; a < n; a++)
            for (int b = a; b < n; b++) {
                if (tri_index(n, a, b) != want) {
                    printf("layout n=%d (%d, %d)\n", n, a, b);
                    return 1;
                }
                if (!inverse_ok(n, want)) return 1;
                ++want;
            }
        if (want != tri_count(n)) return 1;
    }
    // large n: row starts (where the square root's rounding matters), their
    // neighbours, the last position and random positions
    std::mt19937_64 rng(7);
    const int big[] = {1000, 4095, 4096, 23170, 46340, 46341, 65521, 65534, 65535};
    for (int n : big) {
        const long long tc = tri_count(n);
        for (int a = 0; a < n; a++) {
            const long long s = tri_index(n, a, a);
            if (a > 0 && s != tri_index(n, a - 1, n - 1) + 1) {
                printf("row start n=%d a=%d\n", n, a);
                return 1;
            }
            for (long long t : {s - 1, s, s + 1})
                if (t >= 0 && t < tc && !inverse_ok(n, t)) return 1;
        }
        if (tri_index(n, n - 1, n - 1) != tc - 1 || !inverse_ok(n, tc - 1)) return 1;
        for (int i = 0; i < 200000; i++)
            if (!inverse_ok(n, static_cast<long long>(rng() % static_cast<unsigned long long>(tc)))) return 1;
    }
    // stepping: from each position, tri_advance by `step` lands on the
    // position's (row, column) that tri_row_col gives
    for (int n : {1, 2, 3, 7, 31, 64, 255, 256, 257, 400, 1000}) {
        const long long tc = tri_count(n);
        for (int step : {1, 3, 64, 256, 1000}) {
            for (long long t0 = 0; t0 < step && t0 < tc; t0++) {
                int a, b;
                tri_row_col(n, t0, &a, &b);
                for (long long t = t0 + step; t < tc; t += step) {
                    tri_advance(n, step, &a, &b);
                    int ra, rb;
                    tri_row_col(n, t, &ra, &rb);
                    ++checked;
                    if (a != ra || b != rb) {
                        printf("advance n=%d step=%d t=%lld -> (%d, %d), want (%d, %d)\n", n, step, t, a, b, ra, rb);
                        return 1;
                    }
                }
            }
        }
    }
    printf("ok %lld\n", checked);
    return 0;
}

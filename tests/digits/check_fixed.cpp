// Host build of csrc/fixed.cuh for tests/test_fixed.py: reads one case per
// line from stdin and prints the function's result as hex bits.
//   i64  <v as 16 hex digits, two's complement> <e2>      -> i64_to_f64_scaled
//   i128 <high 64 bits hex> <low 64 bits hex> <e2>         -> i128_to_f64_scaled
//   fx   <bits of x, hex> <e>                              -> to_fixed48 (as 64-bit two's complement)
//   fxn  <nbits> <bits of x, hex> <e>                      -> to_fixed(x, e, nbits)
//   em   <bits of max|x|, hex>                             -> exponent_of_max (decimal)
#include <cinttypes>
#include <cstdio>
#include <cstring>

#include "../../paper_2608_06536_b300/csrc/fixed.cuh"

int main() {
    char op[8];
    unsigned long long a, b;
    int e, nb;
    while (scanf("%7s", op) == 1) {
        if (!strcmp(op, "i64") && scanf("%llx %d", &a, &e) == 2) {
            const double r = jk::fixed::i64_to_f64_scaled(static_cast<long long>(a), e);
            printf("%016" PRIx64 "\n", jk::fixed::f64_bits(r));
        } else if (!strcmp(op, "i128") && scanf("%llx %llx %d", &a, &b, &e) == 3) {
            const __int128 v = static_cast<__int128>((static_cast<unsigned __int128>(a) << 64) | b);
            const double r = jk::fixed::i128_to_f64_scaled(v, e);
            printf("%016" PRIx64 "\n", jk::fixed::f64_bits(r));
        } else if (!strcmp(op, "fx") && scanf("%llx %d", &a, &e) == 2) {
            const long long F = jk::fixed::to_fixed48(jk::fixed::bits_f64(a), e);
            printf("%016" PRIx64 "\n", static_cast<uint64_t>(F));
        } else if (!strcmp(op, "fxn") && scanf("%d %llx %d", &nb, &a, &e) == 3) {
            const long long F = jk::fixed::to_fixed(jk::fixed::bits_f64(a), e, nb);
            printf("%016" PRIx64 "\n", static_cast<uint64_t>(F));
        } else if (!strcmp(op, "em") && scanf("%llx", &a) == 1) {
            printf("%d\n", jk::fixed::exponent_of_max(a));
        } else {
            fprintf(stderr, "bad line\n");
            return 2;
        }
    }
    return 0;
}

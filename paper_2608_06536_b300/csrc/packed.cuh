// Row-major upper triangles of symmetric n x n matrices (diagonal included):
// entry (a, b), a <= b, sits at position
//   t(a, b) = a*n - a(a-1)/2 + (b - a),   0 <= t < n(n+1)/2,
// the layout of a packed factor L^P (the host link's half-size upload) and
// the thread numbering of the symmetric J back-contraction.  Host-compilable,
// so that a CPU test checks the index and its inverse for every n the
// library accepts (nbf <= 65535).
#pragma once

#if !defined(JK_HD)
#if defined(__CUDACC__)
#define JK_HD __host__ __device__ __forceinline__
#else
#define JK_HD static inline
#endif
#endif

#include <math.h>

namespace jk {
namespace packed {

// Entries of one packed triangle.
JK_HD long long tri_count(int n) { return static_cast<long long>(n) * (n + 1) / 2; }

// Position of (a, b), a <= b < n.
JK_HD long long tri_index(int n, long long a, long long b) { return a * n - a * (a - 1) / 2 + (b - a); }

// Inverse: the (a, b) at position t < tri_count(n).  Row a is the largest
// with tri_index(n, a, a) <= t; the closed form (a root of the quadratic in
// a) is corrected by at most a step or two where the FP64 square root rounds.
JK_HD void tri_row_col(int n, long long t, int *a, int *b) {
    const double nn = 2.0 * n + 1.0;
    int mu = static_cast<int>((nn - sqrt(nn * nn - 8.0 * static_cast<double>(t))) * 0.5);
    if (mu < 0) mu = 0;
    if (mu > n - 1) mu = n - 1;
    while (mu > 0 && tri_index(n, mu, mu) > t) mu--;
    while (mu < n - 1 && tri_index(n, mu + 1, mu + 1) <= t) mu++;
    *a = mu;
    *b = mu + static_cast<int>(t - tri_index(n, mu, mu));
}

// (a, b) of position t + step, given (a, b) of position t (both positions
// below tri_count(n)): whole rows are skipped without a square root.
JK_HD void tri_advance(int n, int step, int *a, int *b) {
    int r = *a, c = *b + step;
    while (c >= n && r < n - 1) {
        c -= n - r - 1;      // row r + 1 starts at column r + 1
        r++;
    }
    *a = r;
    *b = c;
}

}  // namespace packed
}  // namespace jk

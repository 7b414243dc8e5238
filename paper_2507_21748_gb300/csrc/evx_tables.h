// Host-side plans and tables shared by the grid runtime and the
// allocation-free entry point, so that both run the same radix order and the
// same FP32-rounded twiddle and wave-number tables.
#pragma once
#include <cmath>
#include <vector>

#include "evx_internal.h"

namespace evxrt {

// true when n has no prime factor other than 2, 3 and 5
inline bool smooth235(int n) {
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

// radix order of the generic mixed-radix kernels: 5s, 3s, 16s, then one 8, 4 or 2
inline evx::Plan make_plan(int L) {
    evx::Plan pl{};
    int n = L;
    while (n % 5 == 0) { pl.r[pl.n++] = 5; n /= 5; }
    while (n % 3 == 0) { pl.r[pl.n++] = 3; n /= 3; }
    while (n % 16 == 0) { pl.r[pl.n++] = 16; n /= 16; }
    if (n == 8 || n == 4 || n == 2) { pl.r[pl.n++] = n; n = 1; }
    return pl;
}

// t[m] = exp(-2 pi i m / L), m < count (count = L by default), FP64 then rounded
inline std::vector<float2> twiddles(int L, int count = -1) {
    std::vector<float2> t(count < 0 ? L : count);
    for (size_t m = 0; m < t.size(); ++m) {
        const double ang = -2.0 * M_PI * (double)m / (double)L;
        t[m] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    return t;
}

// |k|^2 of the spectral wave number k = 2 pi m~ / (n h), m~ the signed index, m < count
inline std::vector<float> k2table(int n, double h, int count) {
    std::vector<float> t(count);
    for (int m = 0; m < count; ++m) {
        const int ms = m <= n / 2 ? m : m - n;
        const double k = 2.0 * M_PI * (double)ms / ((double)n * h);
        t[m] = (float)(k * k);
    }
    return t;
}

}  // namespace evxrt

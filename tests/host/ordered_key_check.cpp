// Host check of ordered_key (sph_internal.cuh): for non-NaN doubles a, b the
// keys order as the values (a < b exactly when key(a) < key(b), -0 == +0),
// and a NaN passes no two-sided bound test [lo, hi) with finite bounds, as it
// passes no double comparison.  Prints the number of mismatches.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>
#include <vector>

#include "sph_internal.cuh"

static double from_bits(uint64_t u) {
    double d;
    memcpy(&d, &u, sizeof d);
    return d;
}

int main() {
    std::vector<double> v = {0.0, -0.0, 1.0, -1.0, 0.5, -0.5, 1e-300, -1e-300,
                             std::numeric_limits<double>::denorm_min(),
                             -std::numeric_limits<double>::denorm_min(),
                             std::numeric_limits<double>::max(), -std::numeric_limits<double>::max(),
                             std::numeric_limits<double>::infinity(),
                             -std::numeric_limits<double>::infinity(), 100.0, -100.0, 0.0125,
                             -0.0125, 3.0, 2.9999999999999996};
    uint64_t s = 0x9E3779B97F4A7C15ull;
    for (int k = 0; k < 20000; ++k) {   // xorshift: random bit patterns, NaNs dropped
        s ^= s << 13;
        s ^= s >> 7;
        s ^= s << 17;
        double d = from_bits(s);
        if (!std::isnan(d)) v.push_back(d);
        if (k % 4 == 0 && !std::isnan(d)) v.push_back(std::nextafter(d, 0.0));
    }
    long bad = 0;
    for (size_t i = 0; i < v.size(); ++i)
        for (size_t j = i; j < v.size() && j < i + 64; ++j) {
            double a = v[i], b = v[(j * 7919) % v.size()];
            long long ka = sph::ordered_key(a), kb = sph::ordered_key(b);
            if ((a < b) != (ka < kb) || (a == b) != (ka == kb)) ++bad;
        }
    const double nans[] = {std::numeric_limits<double>::quiet_NaN(),
                           -std::numeric_limits<double>::quiet_NaN(),
                           from_bits(0x7FF0000000000001ull), from_bits(0xFFF0000000000001ull)};
    const double bounds[][2] = {{-5.0, 5.0}, {0.0, 1.0}, {-1e300, 1e300}, {-0.0, 0.0}};
    for (double x : nans)
        for (auto &bd : bounds) {
            long long k = sph::ordered_key(x);
            if (k >= sph::ordered_key(bd[0]) && k < sph::ordered_key(bd[1])) ++bad;
        }
    printf("%zu values, mismatches %ld\n", v.size(), bad);
    return bad != 0;
}

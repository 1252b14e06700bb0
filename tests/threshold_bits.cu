// Host check of the list thresholds' integer arithmetic (apr_internal.cuh): the
// ceiling of (2 h / delta)^2 read off the bits of the double against ceil() and the
// float64 conversion, and the integer root R (smallest with R^2 >= threshold) reached
// from the start the threshold kernel takes, over random magnitudes, whole numbers,
// square roots of whole numbers and their successors, subnormals and special values.
// Exit status 0 when every case agrees.
#include <cmath>
#include <cstdio>
#include <random>

#include "apr_internal.cuh"

typedef unsigned long long u64;

static u64 reference_threshold(double t)
{
    const double t2 = t * t;
    if (!(t2 < 4.6e18)) return 4611686018427387904ULL;
    return (u64)std::ceil(t2);
}

static int check(double t, long* bad)
{
    const u64 a = apr::lattice_threshold_t(t), b = reference_threshold(t);
    int steps = 0;
    u64 r = a >= 4611686018427387904ULL ? 2147483648ULL : apr::ceil_bits(t);
    while (r > 0 && (r - 1) * (r - 1) >= a && steps < 100) {
        --r;
        ++steps;
    }
    while (r * r < a && steps < 100) {
        ++r;
        ++steps;
    }
    const bool root_ok = r * r >= a && (r == 0 || (r - 1) * (r - 1) < a);
    if (a != b || !root_ok || steps > 2) {
        if (*bad < 5) printf("t=%.17g threshold %llu expected %llu, root %llu after %d steps\n", t, a, b, r, steps);
        ++*bad;
    }
    return steps;
}

int main()
{
    std::mt19937_64 g(20260918);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    long bad = 0, n = 0;
    for (long k = 0; k < 4000000; ++k) {
        double t;
        switch (k % 5) {
        case 0: t = std::ldexp(U(g), (int)(g() % 70) - 40); break;
        case 1: t = (double)(g() % 3000000000ULL); break;
        case 2: t = std::sqrt((double)(g() % (1ULL << 62))); break;
        case 3: t = std::nextafter(std::sqrt((double)(g() % (1ULL << 40))), 1e300); break;
        default: t = std::ldexp(U(g), -1074 + (int)(g() % 60)); break;
        }
        check(t, &bad);
        ++n;
    }
    const double special[] = {0.0, -0.0, 4.9e-324, 1e-300, 0.5, 1.0, 2144761059.9, 2144761060.0,
                              2144761061.0, 2147483647.9, 1e300, INFINITY, NAN};
    for (double t : special) {
        check(t, &bad);
        ++n;
    }
    printf("%ld cases, %ld disagreements\n", n, bad);
    return bad == 0 ? 0 : 1;
}

// Host check of the time-step limit's running minimum (apr_dtmin.cuh): the
// log-domain integer pre-test of add_keyed() may skip a particle's float64 cross
// products only where they would not prefer it, so a sequence of particles fed to
// add_keyed() and to add() (the plain cross products) leaves the same winners, bit
// for bit.  Random magnitudes over many decades, near ties (keys within a few units
// in the last place and within 1e-6), equal keys, zeros, subnormals, negative and
// non-finite values.  Exit status 0 when every sequence agrees.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "apr_dtmin.cuh"

static bool same(double a, double b) { return memcmp(&a, &b, sizeof a) == 0; }

int main()
{
    std::mt19937_64 g(20260918);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    auto logu = [&](double lo, double hi) { return std::exp(lo + (hi - lo) * U(g)); };
    long bad = 0, seqs = 0, parts = 0;
    for (int s = 0; s < 200000; ++s) {
        apr::DtMin a, b;
        const int len = (s % 7 == 0) ? 1000 : 26;
        double hb = logu(-8, 3), vb = logu(-6, 4), ab = logu(-10, 10);
        for (int k = 0; k < len; ++k) {
            double h, vsig, ax, ay, az;
            const int mode = (int)(g() % 10);
            if (mode < 4) {  // independent draws over many decades
                h = logu(-10, 5);
                vsig = logu(-8, 6);
                ax = (U(g) - 0.5) * logu(-12, 12);
                ay = (U(g) - 0.5) * logu(-12, 12);
                az = (U(g) - 0.5) * logu(-12, 12);
            } else if (mode < 8) {  // near ties with the sequence's reference values
                const double e = (mode == 4) ? std::ldexp(1.0, -52) * (double)(g() % 9)
                                             : 1e-6 * (U(g) - 0.5);
                h = hb * (1.0 + e);
                vsig = vb * (1.0 + ((mode == 5) ? -e : 0.0));
                ax = ab * (1.0 + e);
                ay = (mode == 6) ? ab : 0.0;
                az = (mode == 7) ? -ab * (1.0 - e) : 0.0;
            } else {  // special values
                const double sp[] = {0.0, -0.0, 4.9e-324, 1e-310, -1.0, INFINITY, NAN, 1e300};
                h = (g() % 4 == 0) ? sp[g() % 8] : hb;
                vsig = (g() % 2 == 0) ? sp[g() % 8] : vb;
                ax = sp[g() % 8];
                ay = (g() % 2) ? ab : sp[g() % 8];
                az = sp[g() % 8];
            }
            a.add(h, vsig, ax * ax + ay * ay + az * az);
            b.add_keyed(h, vsig, ax, ay, az);
            ++parts;
        }
        ++seqs;
        if (!(same(a.cn, b.cn) && same(a.cd, b.cd) && same(a.fn, b.fn) && same(a.fd, b.fd) &&
              same(a.fh, b.fh))) {
            if (bad < 5)
                printf("sequence %d: courant (%.17g, %.17g) vs (%.17g, %.17g), force (%.17g, %.17g) vs (%.17g, %.17g)\n",
                       s, a.cn, a.cd, b.cn, b.cd, a.fn, a.fd, b.fn, b.fd);
            ++bad;
        }
    }
    // the bound itself: for positive normal x the high word H(x) read as an integer
    // lies within [L - HL_ERR, L], L = 2^20 (log2 x + 1023); the largest gap comes
    // at the mantissa 1 / ln 2 (about 90,252), so a smaller HL_ERR fails here
    long double worst = 0.0L;
    for (long k = 0; k < 4000000; ++k) {
        double x = std::ldexp(1.0 + U(g), (int)(g() % 2040) - 1020);
        if (k % 4 == 0) x = std::ldexp(1.0 / std::log(2.0) * (1.0 + 1e-7 * (U(g) - 0.5)), (int)(g() % 200) - 100);
        const long double L = 1048576.0L * (std::log2((long double)x) + 1023.0L);
        const long double gap = L - (long double)apr::hiword(x);
        if (gap < -1e-6L || gap > (long double)apr::HL_ERR) {
            if (bad < 10) printf("x=%.17g gap %.3Lf\n", x, gap);
            ++bad;
        }
        if (gap > worst) worst = gap;
    }
    if (!((long double)apr::HL_LOG3 >= 1048576.0L * std::log2(3.0L))) ++bad;
    printf("%ld sequences, %ld particles, largest high-word gap %.1Lf, %ld disagreements\n", seqs,
           parts, worst, bad);
    return bad == 0 ? 0 : 1;
}

// Host check of the accretion pre-test (apr_sinkpre.cuh): SinkPre::maybe_inside()
// may answer "certainly outside" only for particles the float64 test
// |x - s|^2 < r_acc^2 rejects.  Positions and radii over many decades, particles on
// the accretion sphere to within a few units in the last place, coordinates far from
// the origin with small radii, radii whose square leaves the float range, zero,
// NaN.  The float64 test is taken both with separately rounded products and with
// fused multiply-adds (the device may contract it).  Exit status 0 when no particle
// inside is answered "outside", and the pre-test rejects nine in ten of the
// particles at least two radii out, where the radius is above 1e-4 of the point
// mass's distance from the origin (smaller radii float coordinates cannot resolve).
#include <cmath>
#include <cstdio>
#include <random>

#include "apr_sinkpre.cuh"

int main()
{
    std::mt19937_64 g(20260918);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    std::uniform_real_distribution<double> U01(0.0, 1.0);
    long bad = 0, inside = 0, far = 0, far_rejected = 0, n = 0;
    for (long t = 0; t < 4000000; ++t) {
        double s[3], x[3], racc;
        const int mode = (int)(t % 6);
        const double scale = std::ldexp(1.0, (int)(g() % 120) - 60);
        for (int k = 0; k < 3; ++k) s[k] = U(g) * scale * ((mode == 3) ? 1e6 : 1.0);
        racc = std::ldexp(U01(g) + 0.5, (int)(g() % 80) - 60);
        if (mode == 4) racc = (g() % 2) ? std::ldexp(1.0, -70 + (int)(g() % 20)) : std::ldexp(1.0, 50 + (int)(g() % 20));
        if (mode == 5) {
            const double sp[] = {0.0, NAN, INFINITY, 1e-300, 1e300};
            racc = sp[g() % 5];
        }
        // a direction and a distance: around the sphere (modes 0, 3), inside, outside
        double d[3], nrm = 0.0;
        for (int k = 0; k < 3; ++k) {
            d[k] = U(g);
            nrm += d[k] * d[k];
        }
        nrm = std::sqrt(nrm);
        double dist;
        if (mode == 0 || mode == 3) dist = racc * (1.0 + std::ldexp(U(g), -50 + (int)(g() % 30)));
        else if (mode == 1) dist = racc * U01(g);
        else dist = racc * std::ldexp(1.0 + U01(g), (int)(g() % 40) - 10);
        for (int k = 0; k < 3; ++k) x[k] = s[k] + dist * d[k] / nrm;
        apr::SinkPre pre;
        pre.set(s, racc);
        const bool maybe = pre.maybe_inside((float)x[0], (float)x[1], (float)x[2]);
        const double dx = x[0] - s[0], dy = x[1] - s[1], dz = x[2] - s[2];
        const double r2a = dx * dx + dy * dy + dz * dz;
        const double r2b = std::fma(dz, dz, std::fma(dy, dy, dx * dx));
        const double R2 = racc * racc;
        const bool in = (r2a < R2) || (r2b < R2);
        ++n;
        if (in) {
            ++inside;
            if (!maybe) {
                if (bad < 5) printf("inside but rejected: s=(%.17g %.17g %.17g) x=(%.17g %.17g %.17g) racc=%.17g\n",
                                    s[0], s[1], s[2], x[0], x[1], x[2], racc);
                ++bad;
            }
        } else if (r2a > 4.0 * R2 && mode == 2 && pre.on &&
                   racc > 1e-4 * std::fmax(std::fabs(s[0]), std::fmax(std::fabs(s[1]), std::fabs(s[2])))) {
            // well outside, and a radius that float coordinates resolve
            ++far;
            if (!maybe) ++far_rejected;
        }
    }
    printf("%ld particles, %ld inside, %ld wrongly rejected; %ld of %ld well outside rejected\n", n,
           inside, bad, far_rejected, far);
    if (far == 0 || far_rejected < far * 9 / 10) ++bad;
    return bad == 0 ? 0 : 1;
}

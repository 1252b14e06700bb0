// Pair arithmetic shared by the SPH sums and the split adjoint: the M4 cubic
// spline, a compensated accumulator and the relative position of two sorted
// particles (float on relative lattice coordinates, or double).
#pragma once

#include "apr_internal.cuh"

namespace apr {

template <typename R>
struct Num;
template <>
struct Num<float> {
    __device__ static float sqrt_(float x) { return sqrtf(x); }
    __device__ static float rsqrt_(float x) { return rsqrtf(x); }
    __device__ static float mass(int level) { return level_mass_f(level); }
};
template <>
struct Num<double> {
    __device__ static double sqrt_(double x) { return sqrt(x); }
    __device__ static double rsqrt_(double x) { return 1.0 / sqrt(x); }
    __device__ static double mass(int level) { return level_mass_d(level); }
};

// M4 cubic spline: f(q) and f'(q), zero for q >= 2
template <typename R>
__device__ __forceinline__ void m4(R q, R& f, R& df)
{
    if (q < R(1)) {
        f = R(1) - R(1.5) * q * q + R(0.75) * q * q * q;
        df = R(-3) * q + R(2.25) * q * q;
    } else if (q < R(2)) {
        R t = R(2) - q;
        f = R(0.25) * t * t * t;
        df = R(-0.75) * t * t;
    } else {
        f = R(0);
        df = R(0);
    }
}

// Wendland C2 (support 2h): f(q) = (1 - q/2)^4 (2q + 1), f'(q) = -5 q (1 - q/2)^3
template <typename R>
__device__ __forceinline__ void wendland_c2(R q, R& f, R& df)
{
    if (q < R(2)) {
        const R t = R(1) - R(0.5) * q;
        const R t3 = t * t * t;
        f = t3 * t * (R(2) * q + R(1));
        df = R(-5) * q * t3;
    } else {
        f = R(0);
        df = R(0);
    }
}

// the configured kernel (the branch is uniform across the grid)
template <typename R>
__device__ __forceinline__ void kern(int kernel, R q, R& f, R& df)
{
    if (kernel == APR_KERNEL_WENDLAND_C2)
        wendland_c2<R>(q, f, df);
    else
        m4<R>(q, f, df);
}

// compensated (Kahan) accumulator
template <typename R>
struct Acc {
    R s, c;
    __device__ __forceinline__ Acc() : s(0), c(0) {}
    __device__ __forceinline__ void add(R x)
    {
        R y = x - c;
        R t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// relative position a - b of two sorted particles
template <typename R>
struct Rel;
template <>
struct Rel<float> {
    __device__ static void get(const DevCfg& dc, const int4& pa, const int4& pb, const double*,
                               const double*, const double*, int, int, float d[3])
    {
        int dx = min_image32(pa.x - pb.x, dc.periodic[0], (int)dc.Lint[0]);
        int dy = min_image32(pa.y - pb.y, dc.periodic[1], (int)dc.Lint[1]);
        int dz = min_image32(pa.z - pb.z, dc.periodic[2], (int)dc.Lint[2]);
        d[0] = (float)dx * dc.deltaf;
        d[1] = (float)dy * dc.deltaf;
        d[2] = (float)dz * dc.deltaf;
    }
};
template <>
struct Rel<double> {
    __device__ static void get(const DevCfg& dc, const int4&, const int4&, const double* sx,
                               const double* sy, const double* sz, int a, int b, double d[3])
    {
        d[0] = sx[a] - sx[b];
        d[1] = sy[a] - sy[b];
        d[2] = sz[a] - sz[b];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (dc.periodic[k]) {
                if (d[k] > 0.5 * dc.L[k]) d[k] -= dc.L[k];
                else if (d[k] < -0.5 * dc.L[k]) d[k] += dc.L[k];
            }
    }
};

}  // namespace apr

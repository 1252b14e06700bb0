// Pair arithmetic shared by the SPH sums and the split adjoint: the M4 cubic
// spline, a compensated accumulator and the relative position of two sorted
// particles (float on relative lattice coordinates, or double).
#pragma once

#include <cfloat>

#include "apr_internal.cuh"

namespace apr {

template <typename R>
struct Num;
template <>
struct Num<float> {
    __device__ static float sqrt_(float x) { return sqrtf(x); }
    __device__ static float rsqrt_(float x) { return rsqrtf(x); }
    // sqrt of a pair's r^2 for a kernel argument: r^2 / sqrt(r^2) (0 stays 0)
    __device__ static float root_(float x) { return x * rsqrtf(fmaxf(x, FLT_MIN)); }
    __device__ static float max_(float a, float b) { return fmaxf(a, b); }
    __device__ static float mass(int level) { return level_mass_f(level); }
};
template <>
struct Num<double> {
    __device__ static double sqrt_(double x) { return sqrt(x); }
    __device__ static double rsqrt_(double x) { return 1.0 / sqrt(x); }
    __device__ static double root_(double x) { return sqrt(x); }
    __device__ static double max_(double a, double b) { return fmax(a, b); }
    __device__ static double mass(int level) { return level_mass_d(level); }
};

// Float arithmetic that rounds the same whether or not its unit is compiled with
// multiply-add contraction: every product that feeds a sum is either an explicit
// fused multiply-add or a separately rounded product (these intrinsics are never
// contracted).  The kernel functions and the density terms are written with it,
// so that the list kernel (a unit compiled without contraction) and the density
// kernel give the same bits for the same terms.
template <typename R>
struct Rn;
template <>
struct Rn<float> {
    __device__ static float mul(float a, float b) { return __fmul_rn(a, b); }
    __device__ static float add(float a, float b) { return __fadd_rn(a, b); }
    __device__ static float sub(float a, float b) { return __fsub_rn(a, b); }
    __device__ static float fma(float a, float b, float c) { return fmaf(a, b, c); }
};
// double: the plain operators, contracted as the compiler sees fit (only the density
// kernel's unit evaluates these in double, and its FP64 pipe is the limit there)
template <>
struct Rn<double> {
    __device__ static double mul(double a, double b) { return a * b; }
    __device__ static double add(double a, double b) { return a + b; }
    __device__ static double sub(double a, double b) { return a - b; }
    __device__ static double fma(double a, double b, double c) { return ::fma(a, b, c); }
};

// M4 cubic spline: f(q) and f'(q), zero for q >= 2.  Without branches: with
// t = max(2 - q, 0) and s = max(1 - q, 0), f = t^3 / 4 - s^3 and
// f' = 3 s^2 - 3 t^2 / 4 (for q < 1 this expands to 1 - 3q^2/2 + 3q^3/4 and
// -3q + 9q^2/4; for 1 <= q < 2 s vanishes)
template <typename R>
__device__ __forceinline__ void m4(R q, R& f, R& df)
{
    using O = Rn<R>;
    const R t = Num<R>::max_(O::sub(R(2), q), R(0)), s = Num<R>::max_(O::sub(R(1), q), R(0));
    const R t2 = O::mul(t, t), s2 = O::mul(s, s);
    f = O::fma(O::mul(R(0.25), t2), t, -O::mul(s2, s));
    df = O::fma(R(3), s2, -O::mul(R(0.75), t2));
}

// Wendland C2 (support 2h): f(q) = (1 - q/2)^4 (2q + 1), f'(q) = -5 q (1 - q/2)^3,
// with t = max(1 - q/2, 0) so that both vanish for q >= 2
template <typename R>
__device__ __forceinline__ void wendland_c2(R q, R& f, R& df)
{
    using O = Rn<R>;
    const R t = Num<R>::max_(O::fma(R(-0.5), q, R(1)), R(0));
    const R t3 = O::mul(O::mul(t, t), t);
    f = O::mul(O::mul(t3, t), O::fma(R(2), q, R(1)));
    df = O::mul(O::mul(R(-5), q), t3);
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

// f'' as well: M4 f'' = 3 t / 2 - 6 s; Wendland C2 f'' = -5 t^3 + 15 q t^2 / 2 (t = 1 - q/2)
template <int KT, typename R>
__device__ __forceinline__ void kern2_t(R q, R& f, R& df, R& ddf)
{
    using O = Rn<R>;
    if constexpr (KT == APR_KERNEL_WENDLAND_C2) {
        const R t = Num<R>::max_(O::fma(R(-0.5), q, R(1)), R(0));
        const R t2 = O::mul(t, t), t3 = O::mul(t2, t);
        f = O::mul(O::mul(t3, t), O::fma(R(2), q, R(1)));
        df = O::mul(O::mul(R(-5), q), t3);
        ddf = O::fma(O::mul(R(7.5), q), t2, O::mul(R(-5), t3));
    } else {
        const R t = Num<R>::max_(O::sub(R(2), q), R(0)), s = Num<R>::max_(O::sub(R(1), q), R(0));
        const R t2 = O::mul(t, t), s2 = O::mul(s, s);
        f = O::fma(O::mul(R(0.25), t2), t, -O::mul(s2, s));
        df = O::fma(R(3), s2, -O::mul(R(0.75), t2));
        ddf = O::fma(R(1.5), t, -O::mul(R(6), s));
    }
}

// the kernel fixed at compile time (KT: APR_KERNEL_M4 or APR_KERNEL_WENDLAND_C2)
template <int KT, typename R>
__device__ __forceinline__ void kern_t(R q, R& f, R& df)
{
    if constexpr (KT == APR_KERNEL_WENDLAND_C2)
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

// compensated by groups: the terms of a group summed plainly (products fused into
// the sum), each group's sum added to the total with Kahan's compensation at
// flush(); the pair kernels flush every four terms, so the rounding error is that of
// a compensated sum of the group sums plus a few units in the last place of each
// group (one compensation step per four terms instead of one per term)
template <typename R>
struct AccB {
    R s, c, g;
    __device__ __forceinline__ AccB() : s(0), c(0), g(0) {}
    __device__ __forceinline__ void add(R x) { g += x; }  // (a product may fuse into it)
    __device__ __forceinline__ void add_prod(R a, R b) { g = Rn<R>::fma(a, b, g); }
    __device__ __forceinline__ void flush()
    {
        R y = g - c;
        R t = s + y;
        c = (t - s) - y;
        s = t;
        g = R(0);
    }
};

// relative position a - b of two sorted particles; PER false: no axis is periodic
// (the minimum-image tests are compiled out)
template <typename R>
struct Rel;
template <>
struct Rel<float> {
    template <bool PER = true>
    __device__ static void get(const DevCfg& dc, const int4& pa, const int4& pb, const double*,
                               const double*, const double*, int, int, float d[3])
    {
        int dx = pa.x - pb.x, dy = pa.y - pb.y, dz = pa.z - pb.z;
        if constexpr (PER) {
            dx = min_image32(dx, dc.periodic[0], (int)dc.Lint[0]);
            dy = min_image32(dy, dc.periodic[1], (int)dc.Lint[1]);
            dz = min_image32(dz, dc.periodic[2], (int)dc.Lint[2]);
        }
        d[0] = (float)dx * dc.deltaf;
        d[1] = (float)dy * dc.deltaf;
        d[2] = (float)dz * dc.deltaf;
    }
};
template <>
struct Rel<double> {
    template <bool PER = true>
    __device__ static void get(const DevCfg& dc, const int4&, const int4&, const double* sx,
                               const double* sy, const double* sz, int a, int b, double d[3])
    {
        d[0] = sx[a] - sx[b];
        d[1] = sy[a] - sy[b];
        d[2] = sz[a] - sz[b];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (PER && dc.periodic[k]) {
                if (d[k] > 0.5 * dc.L[k]) d[k] -= dc.L[k];
                else if (d[k] < -0.5 * dc.L[k]) d[k] += dc.L[k];
            }
    }
};

}  // namespace apr

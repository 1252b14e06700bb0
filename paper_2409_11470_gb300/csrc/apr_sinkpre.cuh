// The accretion test |x - s|^2 < r_acc^2 (Sec. 3: gas inside a point mass's
// accretion radius joins it), evaluated in float64, preceded by a float test that
// answers only "possibly inside" or "certainly outside": the float64 test then runs
// for the few particles near an accretion radius.  Host and device: a test compiles
// it for the host.
#pragma once

#include "apr_internal.cuh"

namespace apr {

struct SinkPre {
    float s[3];  // the point mass's position in float
    float r2;    // r_acc^2 in float, widened by 2^-20
    bool on;     // r_acc^2 a float in [1e-30, 1e30]; otherwise every particle is "possibly inside"
    __host__ __device__ __forceinline__ void set(const double x[3], double racc)
    {
        for (int k = 0; k < 3; ++k) s[k] = (float)x[k];
        const float q = (float)(racc * racc);
        on = q >= 1e-30f && q <= 1e30f;
        r2 = q * (1.0f + 1.0f / 1048576.0f);
    }
    // With v_f the float of a double v, |v_f - v| <= 2^-24 |v| <= 2^-24 (1 + 2^-24) |v_f|,
    // and the float difference adds at most 2^-24 |x_f - s_f|, so per axis
    // |x_f - s_f| - (|x_f| + |s_f|) 2^-22 never exceeds the float64 separation; the
    // sum of the squared bounds (rounded, hence the factor 1 - 2^-20) at or above the
    // widened radius means the float64 test fails.  Overflow gives a NaN or an
    // infinite bound (read as zero, or far outside), underflow a smaller one: both keep
    // the answer on the safe side.
    __host__ __device__ __forceinline__ bool maybe_inside(float xf, float yf, float zf) const
    {
        if (!on) return true;
        const float k = 1.0f / 4194304.0f;
        const float gx = fmaxf(0.0f, fabsf(xf - s[0]) - (fabsf(xf) + fabsf(s[0])) * k);
        const float gy = fmaxf(0.0f, fabsf(yf - s[1]) - (fabsf(yf) + fabsf(s[1])) * k);
        const float gz = fmaxf(0.0f, fabsf(zf - s[2]) - (fabsf(zf) + fabsf(s[2])) * k);
        return fmaf(gz, gz, fmaf(gy, gy, gx * gx)) * (1.0f - 1.0f / 1048576.0f) < r2;
    }
};

}  // namespace apr

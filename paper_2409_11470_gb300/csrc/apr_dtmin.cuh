// The time-step limit's running minimum (Sec. 2.5): per particle the Courant
// criterion h / v_sig and the force criterion sqrt(h / |a|), reduced over the
// particles by cross products of (numerator, denominator) pairs.  Host and device:
// a test compiles it for the host.
#pragma once

#include "apr_internal.cuh"

namespace apr {

// the high word of a double as an integer
__host__ __device__ __forceinline__ int hiword(double x) { return (int)(dbits(x) >> 32); }

// smallest time-step limit min(ccour h / v_sig, cforce sqrt(h / |a|)) without a
// division or square root per particle (FP64 is a slow pipe on this part): each
// criterion keeps its best (numerator, denominator) pair, compared by cross
// products (h / |a| compares as h^2 / a^2); the winner's quotient is formed once
// per block with the same expressions as per particle
// The high word of a positive normal double, read as an integer, is 2^20 (log2 x +
// 1023) less at most 2^20 max_f (log2(1 + f) - f) + 1 < 90,254 (the mantissa's
// linear reading of log2 and its truncation to 20 bits): a key compared in this
// log domain with that error on both sides settles most candidates with integer
// arithmetic only.
constexpr long long HL_ERR = 90300;
constexpr long long HL_LOG3 = 1662000;  // 2^20 log2 3, rounded up
__host__ __device__ __forceinline__ bool hl_normal(int hi) { return hi >= 0x00100000 && hi < 0x7ff00000; }
constexpr long long HL_NONE = 1LL << 60;  // no log-domain key: no candidate is skipped

struct DtMin {
    double cn = 0.0, cd = 0.0;  // courant: h, v_sig (cd == 0: none yet)
    double fn = 0.0, fd = 0.0;  // force: h^2, a^2 (fd == 0: none yet)
    double fh = 0.0;            // the force winner's h
    // log-domain keys of the winners (HL_NONE: none, or not normal)
    long long ck = HL_NONE, fk = HL_NONE;
    // add() for a particle whose courant key h / v_sig or force key h^2 / |a|^2 is
    // certainly larger than the winner's skips that criterion's float64 test: with
    // a_max the largest |a| component, |a|^2 lies in [a_max^2, 3 a_max^2], so the
    // log-domain key 2 (H(h) - H(a_max)) is within 2 HL_ERR + 2^20 log2 3 of the
    // key's log; a skip needs the two keys' logs apart by at least 2^-19, far
    // beyond the rounding of the float64 cross products, which then never prefer it
    __host__ __device__ __forceinline__ void add_keyed(double h, double vsig, double ax, double ay,
                                                       double az)
    {
        const int Ah = hiword(h), Av = hiword(vsig);
        const bool nh = hl_normal(Ah);
        const long long kc = (nh && hl_normal(Av)) ? (long long)Ah - Av : HL_NONE;
        if (!(kc != HL_NONE && kc > ck + 2 * HL_ERR + 2)) {
            if (vsig > 0.0 && (cd == 0.0 || h * cd < cn * vsig)) {
                cn = h;
                cd = vsig;
                ck = kc;
            }
        }
        const int mx = hiword(ax) & 0x7fffffff, my = hiword(ay) & 0x7fffffff,
                  mz = hiword(az) & 0x7fffffff;
        const int Am = mx > my ? (mx > mz ? mx : mz) : (my > mz ? my : mz);
        const long long kf = (nh && hl_normal(Am)) ? 2 * ((long long)Ah - Am) : HL_NONE;
        if (!(kf != HL_NONE && kf > fk + 4 * HL_ERR + HL_LOG3 + 2)) {
            const double a2 = ax * ax + ay * ay + az * az;
            const double h2 = h * h;
            if (a2 > 0.0 && (fd == 0.0 || h2 * fd < fn * a2)) {
                fn = h2;
                fd = a2;
                fh = h;
                fk = kf;
            }
        }
    }
    __host__ __device__ void add(double h, double vsig, double a2)
    {
        if (vsig > 0.0 && (cd == 0.0 || h * cd < cn * vsig)) {
            cn = h;
            cd = vsig;
        }
        const double h2 = h * h;
        if (a2 > 0.0 && (fd == 0.0 || h2 * fd < fn * a2)) {
            fn = h2;
            fd = a2;
            fh = h;
        }
    }
    __host__ __device__ void merge(const DtMin& o)
    {
        if (o.cd > 0.0 && (cd == 0.0 || o.cn * cd < cn * o.cd)) {
            cn = o.cn;
            cd = o.cd;
        }
        if (o.fd > 0.0 && (fd == 0.0 || o.fn * fd < fn * o.fd)) {
            fn = o.fn;
            fd = o.fd;
            fh = o.fh;
        }
    }
    __device__ void shfl_down(int o)
    {
        DtMin t;
        t.cn = __shfl_down_sync(0xffffffffu, cn, o);
        t.cd = __shfl_down_sync(0xffffffffu, cd, o);
        t.fn = __shfl_down_sync(0xffffffffu, fn, o);
        t.fd = __shfl_down_sync(0xffffffffu, fd, o);
        t.fh = __shfl_down_sync(0xffffffffu, fh, o);
        merge(t);
    }
    __host__ __device__ double value(const DevCfg& dc) const
    {
        double dt = INFINITY;
        if (cd > 0.0) dt = fmin(dt, dc.ccour * cn / cd);
        if (fd > 0.0) dt = fmin(dt, dc.cforce * sqrt(fh / sqrt(fd)));
        return dt;
    }
};

}  // namespace apr

// The h-rho Newton-Raphson of one particle, in pieces that two kernels share:
// the density kernel (every pass over a particle's list) and the list kernel
// (the first pass, fused into the list build while the candidates sit in
// shared memory).  Both evaluate the same terms in the same (list) order, so a
// first pass gives the same bits in either.
//
// The grad-h form (Sec. 2.2 cites Phantom's iteration): h is the root of
// g(h) = sum_b mu_b f(r_ab/h) + mu_a - pi mu_a h_fact^3 (mu = 2^-level, Eq. 1),
// monotone in h, so a bracket safeguards every Newton step.
#pragma once

#include "apr_internal.cuh"
#include "apr_pair.cuh"

namespace apr {

// the exact square of a lattice separation
__device__ __forceinline__ unsigned long long lattice_sq(const int d[3])
{
    return (unsigned long long)((long long)d[0] * d[0]) + (unsigned long long)((long long)d[1] * d[1]) +
           (unsigned long long)((long long)d[2] * d[2]);
}

// float r^2 of a lattice separation: the unit times each integer component, squared
// and summed with explicit fused multiply-adds (the same rounding wherever it is used)
__device__ __forceinline__ float lattice_r2f(float unit, const int d[3])
{
    const float x = (float)d[0] * unit, y = (float)d[1] * unit, z = (float)d[2] * unit;
    return fmaf(z, z, fmaf(y, y, x * x));
}

// one density term mu_b f(q), mu_b q f'(q) (and with U2, mu_b q^2 f''(q)) for a
// pair inside 2h
template <int KT, bool U2, typename R>
__device__ __forceinline__ void density_term(R r2, R hinv, R r2max, int levb, AccB<R>& S,
                                             AccB<R>& T, AccB<R>& U, unsigned int& npair)
{
    using O = Rn<R>;
    if (r2 >= r2max) return;
    const R q = O::mul(Num<R>::root_(r2), hinv);
    const R mub = Num<R>::mass(levb);
    const R mq = O::mul(mub, q);
    R f, df;
    if constexpr (U2) {
        R ddf;
        kern2_t<KT, R>(q, f, df, ddf);
        U.add_prod(O::mul(mq, q), ddf);
    } else {
        kern_t<KT, R>(q, f, df);
    }
    S.add_prod(mub, f);
    T.add_prod(mq, df);
    ++npair;
}

template <typename R>
__device__ __forceinline__ R round_down(double x);
template <>
__device__ __forceinline__ float round_down<float>(double x) { return __double2float_rd(x); }
template <>
__device__ __forceinline__ double round_down<double>(double x) { return x; }

// The nearest lattice neighbour (the exact integer minimum of the squared lattice
// distance over the list).  FP64: every entry's exact square.  FP32: the exact
// square only of entries whose float r^2 lies within a relative 2^-20 of the
// smallest float r^2 seen so far.  This is the exact minimum: the float r^2 of any
// entry is its exact lattice r^2 times the (power-of-two) unit squared, to a
// relative 5 u (u = 2^-24: three conversions, three products, two sums), so the
// exact nearest's float r^2 is within a relative 10.1 u of the smallest float
// r^2 of the list, hence within 2^-20 = 16 u of the running minimum when it is
// met; the entries skipped are farther than it.
template <typename R>
__device__ __forceinline__ void near_update(R r2f, const int d[3], R& bestf, unsigned long long& best)
{
    if constexpr (sizeof(R) == 4) {
        if (r2f <= bestf * (1.0f + 1.0f / (1 << 20))) {
            const unsigned long long q = lattice_sq(d);
            best = q < best ? q : best;
            bestf = fminf(bestf, r2f);
        }
    } else {
        const unsigned long long q = lattice_sq(d);
        best = q < best ? q : best;
    }
}

// a profiling count added once per warp (the threads present at the call; one
// atomic per thread on a single word would serialise on it)
__device__ __forceinline__ void count_warp(unsigned long long* counter, unsigned int v)
{
    const unsigned mask = __activemask();
    const unsigned tot = __reduce_add_sync(mask, v);
    if ((threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(counter, (unsigned long long)tot);
}

// the largest growth of h in one density attempt beyond its list's reach, allowed to
// a particle whose list fills at most an eighth of its capacity (the list around the
// grown h holds about (1.4 x 1.06)^3 = 3.3 times as many entries)
constexpr double RETRY_GROWTH = 1.4;

// where an uncovered step may stop: RETRY_GROWTH times the reach for a short list
// (m entries of capacity K), else the reach itself
template <typename R>
__device__ __forceinline__ R retry_cap(R hreach, int m, int K)
{
    return 8LL * m <= (long long)K ? R(RETRY_GROWTH) * hreach : hreach;
}

// one particle's iteration state between passes over its list
template <typename R>
struct NRState {
    R h;            // current smoothing length
    R lo, hi;       // bracket of the root (hi == 0: none yet)
    R D;            // sum mu_b (3 f + q f') at the last evaluated h
    bool conv, uncovered;
};

// One Newton-Raphson update from the sums S, T (and U) of a pass at st.h; returns
// true when the iteration stops (converged, or the root lies beyond the list's
// reach hreach).  ACCEPT (FP32): a step whose predicted successor is below the
// tolerance is taken without a confirming pass.
template <typename R, bool ACCEPT>
__device__ __forceinline__ bool nr_update(NRState<R>& st, R S, R T, R U, R mua, R target, R tol,
                                          R hreach, R hcap)
{
    using O = Rn<R>;
    const R h = st.h;
    const R hinv = R(1) / h;
    const R Sm = O::add(S, mua);
    const R g = O::sub(Sm, target);  // pi h^3 (rho_sum - rho_h) / m0
    const R dg = -O::mul(T, hinv);   // dg/dh >= 0
    st.D = O::fma(R(3), Sm, T);
    if (g < R(0)) st.lo = h;
    else st.hi = h;
    R hn;
    bool newton = dg > R(0);
    if (newton) hn = O::sub(h, g / dg);
    else hn = O::mul(h, R(1.25992105));
    // a Newton step that leaves the bracket is replaced by bisection (or growth)
    if (hn < st.lo || (st.hi > R(0) && hn > st.hi) || !(hn == hn)) {
        hn = st.hi > R(0) ? O::mul(R(0.5), O::add(st.lo, st.hi)) : O::mul(h, R(1.25992105));
        newton = false;
    }
    if (hn > O::mul(R(2), h)) {
        hn = O::mul(R(2), h);
        newton = false;
    }
    if (hn < O::mul(R(0.5), h)) {
        hn = O::mul(R(0.5), h);
        newton = false;
    }
    bool done = fabs(O::sub(hn, h)) <= O::mul(tol, h);
    if (ACCEPT && newton && !done) {
        // the next Newton correction predicted from g'' = (2T + U) / h^2
        // (g(hn) ~ g'' d^2 / 2 after the step d, exact to a relative O(d / h)); a
        // step whose successor is below the tolerance is taken without a
        // confirming pass, and D is carried to hn to first order
        // (dD/dh = -(4T + U) / h)
        const R d = O::sub(hn, h);
        const R g2 = O::mul(O::mul(O::fma(R(2), T, U), hinv), hinv);
        if (fabs(O::mul(O::mul(O::mul(R(0.5), g2), d), d)) <= O::mul(O::mul(tol, hn), dg)) {
            st.D = O::fma(-O::mul(O::fma(R(4), T, U), hinv), d, st.D);
            done = true;
        }
    }
    if (hn > hreach) {
        // the step leaves this list's reach: stop at its target, but at most at hcap
        // (retry_cap); the host builds the particle's list at the reach around it
        // and the iteration continues there
        st.h = hn < hcap ? hn : hcap;
        st.uncovered = true;
        return true;
    }
    st.h = hn;
    if (done) {
        st.conv = true;
        return true;
    }
    return false;
}

// one slot's force records: A = (1/h, P/(Omega rho^2), c_s, rho), V = (v, u),
// B = (P, 1/(Omega rho), h, mass factor).  FP32-mixed: float4, every quotient
// formed in float from the float values the density solve settled (the gather
// forms the same from the stored values, which are exact widenings of them);
// FP64: four doubles each.
__device__ __forceinline__ void store_force_data_f(void* A, void* V, void* B, long long s, float h,
                                                   float r, float om, float P, float cs, double vx,
                                                   double vy, double vz, double u, int level)
{
    const float omr = __fmul_rn(om, r);
    if (B) {
        ((float4*)A)[s] = make_float4(1.0f / h, P / __fmul_rn(omr, r), cs, r);
        ((float4*)B)[s] = make_float4(P, 1.0f / omr, h, level_mass_f(level));
    } else {
        // without conductivity the force needs of B only 1/(Omega rho) (here in A's
        // last slot) and the mass (from the level): two records per slot
        ((float4*)A)[s] = make_float4(1.0f / h, P / __fmul_rn(omr, r), cs, 1.0f / omr);
    }
    ((float4*)V)[s] = make_float4((float)vx, (float)vy, (float)vz, (float)u);
}

// the FP32-mixed force records use the two-record layout (A, V) unless the run
// has artificial conductivity, which needs pressure and density of the neighbour
__host__ __device__ inline bool force_two_records(const DevCfg& dc)
{
    return !(dc.eos == APR_EOS_ADIABATIC && dc.alpha_u > 0.0);
}

__device__ __forceinline__ void store_force_data_d(void* A, void* V, void* B, long long s, double h,
                                                   double r, double om, double P, double cs,
                                                   double vx, double vy, double vz, double u,
                                                   int level)
{
    double* a = (double*)A + 4 * s;
    double* v = (double*)V + 4 * s;
    double* b = (double*)B + 4 * s;
    a[0] = 1.0 / h;
    a[1] = P / (om * r * r);
    a[2] = cs;
    a[3] = r;
    v[0] = vx;
    v[1] = vy;
    v[2] = vz;
    v[3] = u;
    b[0] = P;
    b[1] = 1.0 / (om * r);
    b[2] = h;
    b[3] = level_mass_d(level);
}

// where a settled particle's results go: caller-order arrays through the sort's
// permutation, and (fA non-null) the sorted force records
struct DensityIO {
    const unsigned int* perm;
    const double *x, *y, *u, *vx, *vy, *vz;
    double *h_out, *rho_out, *omega_out, *dnn_out, *pres_out, *cs_out;
    void *fA, *fV, *fB;
};

// The first Newton-Raphson pass of the density solve, fused into the list build
// (FP32-mixed, symmetric lists at the density reach): every entry a lane writes is
// also added, in list order, to that lane's sums at the list's h, from the
// candidate's exact lattice coordinates in shared memory.  The terms, their order
// and the update after the pass are those of the density kernel's first pass, so a
// particle settled here has the bits the density kernel would give it; the others
// are queued for the density kernel, which starts them afresh.
struct FuseArgs {
    const double* sh;  // sorted h: the lists' h and the pass's starting point
    double reach;      // the lists' reach factor (h may not pass reach * h_list)
    DensityIO io;      // where settled particles' results go
    int* dq;           // particles left for the density kernel
    int* dq_n;
};

// the results of a density pass of context c (force_data: with the force records)
DensityIO density_io(apr_ctx* c, bool force_data);

// A settled particle's outputs: h, the nearest lattice neighbour within 2h, density
// (rho = m (h_fact / h)^3), Omega = 1 - D / (3 target), the equation of state
// (adiabatic, or locally isothermal c_s = c_s0 R^-q) and the force records.
// FP32-mixed: density, Omega, pressure and sound speed in float at the pair sums'
// precision (this part's FP64 unit runs at a small fraction of the FP32 rate),
// widened on store.
template <typename R>
__device__ __forceinline__ void density_store(const DevCfg& dc, const DensityIO& io, int a,
                                              const int4& pa, R h, R D, R target,
                                              unsigned long long best)
{
    const unsigned i = io.perm[a];
    const double hd = (double)h;
    io.h_out[i] = hd;
    // nearest lattice neighbour within 2h: the list holds every particle within
    // the reach, so the overall nearest counts iff it lies inside 2h
    const unsigned long long thr = lattice_threshold(dc, hd);
    io.dnn_out[i] = best < thr ? sqrt((double)best) * dc.delta : (double)INFINITY;
    if constexpr (sizeof(R) == 4) {
        // (the products and sums rounded as written: the list kernel's unit is
        // compiled without multiply-add contraction, the density kernel's with it)
        using O = Rn<float>;
        const float hr = dc.hfactf / h;
        const float rho = O::mul(O::mul(O::mul(O::mul(dc.m0f, level_mass_f(pa.w)), hr), hr), hr);
        const float om = O::sub(1.0f, D / O::mul(3.0f, target));
        float P, cs;
        if (dc.eos == APR_EOS_ADIABATIC) {
            const float uf = (float)io.u[i];
            const float gm1 = O::sub(dc.gammaf, 1.0f);
            P = O::mul(O::mul(gm1, rho), uf);
            cs = sqrtf(O::mul(O::mul(dc.gammaf, gm1), uf));
        } else {
            const float xf = (float)io.x[i], yf = (float)io.y[i];
            cs = O::mul(dc.cs0f, powf(sqrtf(O::fma(yf, yf, O::mul(xf, xf))), -dc.qcsf));
            P = O::mul(O::mul(cs, cs), rho);
        }
        io.rho_out[i] = (double)rho;
        io.omega_out[i] = (double)om;
        io.pres_out[i] = (double)P;
        io.cs_out[i] = (double)cs;
        if (io.fA)
            store_force_data_f(io.fA, io.fV, force_two_records(dc) ? nullptr : io.fB, a, h, rho, om,
                               P, cs, io.vx[i], io.vy[i], io.vz[i], io.u[i], pa.w);
    } else {
        const double hr = dc.hfact / hd;
        const double rho = dc.m0 * (double)level_mass_d(pa.w) * hr * hr * hr;
        const double om = 1.0 - (double)D / (3.0 * (double)target);
        double P, cs;
        if (dc.eos == APR_EOS_ADIABATIC) {
            P = (dc.gamma - 1.0) * rho * io.u[i];
            cs = sqrt(dc.gamma * P / rho);
        } else {
            double Rc = sqrt(io.x[i] * io.x[i] + io.y[i] * io.y[i]);
            cs = dc.cs0 * pow(Rc, -dc.qcs);
            P = cs * cs * rho;
        }
        io.rho_out[i] = rho;
        io.omega_out[i] = om;
        io.pres_out[i] = P;
        io.cs_out[i] = cs;
        if (io.fA)
            store_force_data_d(io.fA, io.fV, io.fB, a, hd, rho, om, P, cs, io.vx[i], io.vy[i],
                               io.vz[i], io.u[i], pa.w);
    }
}

}  // namespace apr

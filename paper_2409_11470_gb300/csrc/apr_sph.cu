// SPH density (h-rho Newton-Raphson) and force / energy sums over particles of
// mixed mass (Eq. 1: m = m0 / 2^level) and smoothing length, on sm_103a.
//
// The paper solves for h and rho iteratively as Phantom does (cited in
// Sec. 2.2); the kernels below take the standard grad-h form: h is the root of
// rho_sum(h) = m_a (h_fact / h)^3 with rho_sum(h) = sum_b m_b W(r_ab, h)
// (self included), M4 kernel W = f(q) / (pi h^3), support 2h.  Newton-Raphson
// is applied to g(h) = pi h^3 (rho_sum - rho_h) / m0 = sum_b mu_b f(r_ab/h)
// + mu_a - pi mu_a h_fact^3 (mu = 2^-level), which has the same root and is
// monotone, so a bracket can safeguard every step.
//
// FP32-mixed: pair sums in float on relative lattice coordinates
// (dx = float(dx_lattice) * D), Kahan-compensated; results widened to double.
// FP64: the same kernels in double on the float64 coordinates.
#include <cfloat>

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

// ----------------------------------------------------------------- density

template <typename R>
__global__ void __launch_bounds__(128)
    k_density(DevCfg dc, long long n, long long cap, double reach, const int4* __restrict__ pk,
              const double* __restrict__ sh, const unsigned int* __restrict__ nbr,
              const int* __restrict__ ncnt, const double* __restrict__ sx,
              const double* __restrict__ sy, const double* __restrict__ sz,
              const unsigned int* __restrict__ perm, const double* __restrict__ x,
              const double* __restrict__ y, const double* __restrict__ u,
              double* __restrict__ h_out, double* __restrict__ rho_out,
              double* __restrict__ omega_out, double* __restrict__ dnn_out,
              double* __restrict__ pres_out, double* __restrict__ cs_out, int* status,
              unsigned long long* counters)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int a = (int)s;
    const int4 pa = pk[a];
    const double hlist = sh[a];
    const R mua = Num<R>::mass(pa.w);
    const R target = R(3.14159265358979323846) * mua * R(dc.hfact * dc.hfact * dc.hfact);
    const int m = ncnt[a];
    if (m < 0) {
        // the list at this h overflowed (e.g. an initial h far too large at a
        // density jump): shrink h and let the host rebuild the lists
        h_out[perm[a]] = 0.8 * hlist;
        atomicAdd(&status[ST_UNCOVERED], 1);
        atomicAdd(&status[ST_SHRINK], 1);
        return;
    }
    R h = (R)hlist;
    R lo = R(0), hi = R(0);  // bracket of the root; hi == 0: none yet
    R D = R(0);              // sum mu_b (3 f + q f') at the last evaluated h
    bool conv = false, uncovered = false;
    unsigned long long npair = 0;
    for (int it = 0; it < dc.nr_maxit; ++it) {
        const R hinv = R(1) / h;
        const R r2max = R(4) * h * h;
        Acc<R> S, T;
        for (int k = 0; k < m; ++k) {
            const int b = (int)nbr[(long long)k * cap + a];
            const int4 pb = pk[b];
            R d[3];
            Rel<R>::get(dc, pa, pb, sx, sy, sz, a, b, d);
            const R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 >= r2max) continue;
            const R q = Num<R>::sqrt_(r2) * hinv;
            R f, df;
            m4<R>(q, f, df);
            const R mub = Num<R>::mass(pb.w);
            S.add(mub * f);
            T.add(mub * q * df);
            ++npair;
        }
        const R g = (S.s + mua) - target;           // pi h^3 (rho_sum - rho_h) / m0
        const R dg = -(T.s) * hinv;                   // dg/dh >= 0
        D = R(3) * (S.s + mua) + T.s;
        if (g < R(0)) lo = h;
        else hi = h;
        R hn;
        if (dg > R(0)) hn = h - g / dg;
        else hn = h * R(1.25992105);
        // a Newton step that leaves the bracket is replaced by bisection (or growth)
        if (hn < lo || (hi > R(0) && hn > hi) || !(hn == hn))
            hn = hi > R(0) ? R(0.5) * (lo + hi) : h * R(1.25992105);
        if (hn > R(2) * h) hn = R(2) * h;
        if (hn < R(0.5) * h) hn = R(0.5) * h;
        const bool done = fabs((double)(hn - h)) <= dc.nr_tol * (double)h;
        if ((double)hn > reach * hlist) {
            // the root lies beyond this list's reach: stop at the reach; the host
            // rebuilds the lists there and the iteration continues (growth is
            // bounded per attempt, so lists stay short)
            h = (R)(reach * hlist);
            uncovered = true;
            break;
        }
        h = hn;
        if (done) {
            conv = true;
            break;
        }
    }
    if (dc.prof) atomicAdd(&counters[APR_PROF_DENSITY], npair);
    const unsigned i = perm[a];
    const double hd = (double)h;
    h_out[i] = hd;
    if (uncovered) {
        atomicAdd(&status[ST_UNCOVERED], 1);
        return;
    }
    if (!conv) atomicAdd(&status[ST_NOCONV], 1);
    // nearest neighbour on the lattice among the neighbours at the final h
    const unsigned long long thr = neighbour_threshold(hd, dc.delta);
    unsigned long long best = ~0ULL;
    for (int k = 0; k < m; ++k) {
        const int b = (int)nbr[(long long)k * cap + a];
        const int4 pb = pk[b];
        long long dx = min_image((long long)pa.x - pb.x, dc.periodic[0], dc.Lint[0]);
        long long dy = min_image((long long)pa.y - pb.y, dc.periodic[1], dc.Lint[1]);
        long long dz = min_image((long long)pa.z - pb.z, dc.periodic[2], dc.Lint[2]);
        unsigned long long r2 = (unsigned long long)(dx * dx) + (unsigned long long)(dy * dy) +
                                (unsigned long long)(dz * dz);
        if (r2 < thr && r2 < best) best = r2;
    }
    dnn_out[i] = best == ~0ULL ? (double)INFINITY : sqrt((double)best) * dc.delta;
    const double hr = dc.hfact / hd;
    const double rho = dc.m0 * (double)level_mass_d(pa.w) * hr * hr * hr;
    rho_out[i] = rho;
    omega_out[i] = 1.0 - (double)D / (3.0 * (double)target);
    double P, cs;
    if (dc.eos == APR_EOS_ADIABATIC) {
        P = (dc.gamma - 1.0) * rho * u[i];
        cs = sqrt(dc.gamma * P / rho);
    } else {
        double Rc = sqrt(x[i] * x[i] + y[i] * y[i]);
        cs = dc.cs0 * pow(Rc, -dc.qcs);
        P = cs * cs * rho;
    }
    pres_out[i] = P;
    cs_out[i] = cs;
}

apr_status density_pass(apr_ctx* c, long long* uncovered, long long* noconv)
{
    Workspace& W = c->W;
    const long long n = c->n;
    cudaStream_t st = c->stream;
    cudaMemsetAsync(&W.status[ST_UNCOVERED], 0, 2 * sizeof(int), st);
    cudaMemsetAsync(&W.status[ST_SHRINK], 0, sizeof(int), st);
    int ps = prof_begin(c, APR_PROF_DENSITY);
    if (n > 0) {
        const double reach = DENSITY_REACH;
        if (c->cfg.precision == APR_PREC_FP64)
            APR_LAUNCH(c, k_density<double>, nblocks(n, 128), 128, 
                c->dc, n, c->cap, reach, W.pk, W.sh, W.nbr, W.ncnt, W.sx, W.sy, W.sz, W.perm,
                c->p.x, c->p.y, c->p.u, c->p.h, c->p.rho, c->p.omega, c->p.dnn, c->p.pres, c->p.cs,
                W.status, W.counters);
        else
            APR_LAUNCH(c, k_density<float>, nblocks(n, 128), 128, 
                c->dc, n, c->cap, reach, W.pk, W.sh, W.nbr, W.ncnt, W.sx, W.sy, W.sz, W.perm,
                c->p.x, c->p.y, c->p.u, c->p.h, c->p.rho, c->p.omega, c->p.dnn, c->p.pres, c->p.cs,
                W.status, W.counters);
    }
    prof_end(c, ps);
    cudaMemcpyAsync(c->hbuf, &W.status[ST_UNCOVERED], (ST_SHRINK - ST_UNCOVERED + 1) * sizeof(int),
                    cudaMemcpyDeviceToHost, st);
    apr_status s = cuda_check(c, cudaStreamSynchronize(st), "density");
    if (s != APR_OK) return s;
    *uncovered = ((int*)c->hbuf)[0];
    *noconv = ((int*)c->hbuf)[1];
    c->last_shrink = ((int*)c->hbuf)[ST_SHRINK - ST_UNCOVERED];
    return APR_OK;
}

// ------------------------------------------------------------------- force

__global__ void k_gather_force_f32(long long n, const unsigned int* __restrict__ perm,
                                   const int4* __restrict__ pk, const double* __restrict__ h,
                                   const double* __restrict__ rho, const double* __restrict__ omega,
                                   const double* __restrict__ pres, const double* __restrict__ cs,
                                   const double* __restrict__ vx, const double* __restrict__ vy,
                                   const double* __restrict__ vz, const double* __restrict__ u,
                                   float4* __restrict__ A, float4* __restrict__ V,
                                   float4* __restrict__ B)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    unsigned i = perm[s];
    double r = rho[i], om = omega[i], P = pres[i];
    A[s] = make_float4((float)(1.0 / h[i]), (float)(P / (om * r * r)), (float)cs[i], (float)r);
    V[s] = make_float4((float)vx[i], (float)vy[i], (float)vz[i], (float)u[i]);
    B[s] = make_float4((float)P, (float)(1.0 / (om * r)), (float)h[i], level_mass_f(pk[s].w));
}

__global__ void k_gather_force_f64(long long n, const unsigned int* __restrict__ perm,
                                   const int4* __restrict__ pk, const double* __restrict__ h,
                                   const double* __restrict__ rho, const double* __restrict__ omega,
                                   const double* __restrict__ pres, const double* __restrict__ cs,
                                   const double* __restrict__ vx, const double* __restrict__ vy,
                                   const double* __restrict__ vz, const double* __restrict__ u,
                                   double* __restrict__ A, double* __restrict__ V,
                                   double* __restrict__ B)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    unsigned i = perm[s];
    double r = rho[i], om = omega[i], P = pres[i];
    A[4 * s + 0] = 1.0 / h[i];
    A[4 * s + 1] = P / (om * r * r);
    A[4 * s + 2] = cs[i];
    A[4 * s + 3] = r;
    V[4 * s + 0] = vx[i];
    V[4 * s + 1] = vy[i];
    V[4 * s + 2] = vz[i];
    V[4 * s + 3] = u[i];
    B[4 * s + 0] = P;
    B[4 * s + 1] = 1.0 / (om * r);
    B[4 * s + 2] = h[i];
    B[4 * s + 3] = level_mass_d(pk[s].w);
}

apr_status gather_force_data(apr_ctx* c)
{
    Workspace& W = c->W;
    const long long n = c->n;
    if (n <= 0) return APR_OK;
    if (c->cfg.precision == APR_PREC_FP64)
        APR_LAUNCH(c, k_gather_force_f64, nblocks(n, 256), 256, 
            n, W.perm, W.pk, c->p.h, c->p.rho, c->p.omega, c->p.pres, c->p.cs, c->p.vx, c->p.vy,
            c->p.vz, c->p.u, W.dA, W.dV, W.dB);
    else
        APR_LAUNCH(c, k_gather_force_f32, nblocks(n, 256), 256, 
            n, W.perm, W.pk, c->p.h, c->p.rho, c->p.omega, c->p.pres, c->p.cs, c->p.vx, c->p.vy,
            c->p.vz, c->p.u, W.fA, W.fV, W.fB);
    return cuda_check(c, cudaGetLastError(), "gather force data");
}

template <typename R>
struct F4 {
    R x, y, z, w;
};

template <typename R>
__device__ __forceinline__ F4<R> ld4(const void* base, long long s);
template <>
__device__ __forceinline__ F4<float> ld4<float>(const void* base, long long s)
{
    float4 v = ((const float4*)base)[s];
    return {v.x, v.y, v.z, v.w};
}
template <>
__device__ __forceinline__ F4<double> ld4<double>(const void* base, long long s)
{
    const double2* p = (const double2*)base;
    double2 a = p[2 * s], b = p[2 * s + 1];
    return {a.x, a.y, b.x, b.y};
}

template <typename R>
__global__ void __launch_bounds__(128)
    k_force(DevCfg dc, long long n, long long cap, const int4* __restrict__ pk,
            const void* __restrict__ Ab, const void* __restrict__ Vb, const void* __restrict__ Bb,
            const unsigned int* __restrict__ nbr, const int* __restrict__ ncnt,
            const double* __restrict__ sx, const double* __restrict__ sy,
            const double* __restrict__ sz, const unsigned int* __restrict__ perm,
            double* __restrict__ ax_out, double* __restrict__ ay_out, double* __restrict__ az_out,
            double* __restrict__ dudt_out, double* __restrict__ vsig_out,
            unsigned long long* counters)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int a = (int)s;
    const int4 pa = pk[a];
    const F4<R> A = ld4<R>(Ab, a), V = ld4<R>(Vb, a), B = ld4<R>(Bb, a);
    const R hinv_a = A.x, pro_a = A.y, cs_a = A.z, rho_a = A.w;
    const R P_a = B.x, ior_a = B.y;
    const R h4a = hinv_a * hinv_a * hinv_a * hinv_a;
    const R alpha = (R)dc.alpha_av, beta = (R)dc.beta_av, alpha_u = (R)dc.alpha_u;
    const bool adiabatic = dc.eos == APR_EOS_ADIABATIC;
    const bool cond = adiabatic && dc.alpha_u > 0.0;
    Acc<R> fx, fy, fz, du;
    R vsig = cs_a;
    unsigned long long npair = 0;
    const int m = ncnt[a];
    for (int k = 0; k < m; ++k) {
        const int b = (int)nbr[(long long)k * cap + a];
        const int4 pb = pk[b];
        R d[3];
        Rel<R>::get(dc, pa, pb, sx, sy, sz, a, b, d);
        const F4<R> Ab4 = ld4<R>(Ab, b), Vb4 = ld4<R>(Vb, b), Bb4 = ld4<R>(Bb, b);
        const R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const R rinv = Num<R>::rsqrt_(r2);
        const R r = r2 * rinv;
        const R hinv_b = Ab4.x;
        const R qa = r * hinv_a, qb = r * hinv_b;
        if (!(qa < R(2) || qb < R(2))) continue;
        ++npair;
        R fa, dfa, fb, dfb;
        m4<R>(qa, fa, dfa);
        m4<R>(qb, fb, dfb);
        const R Fa = dfa * h4a;
        const R Fb = dfb * (hinv_b * hinv_b * hinv_b * hinv_b);
        const R vr = ((V.x - Vb4.x) * d[0] + (V.y - Vb4.y) * d[1] + (V.z - Vb4.z) * d[2]) * rinv;
        R ta = pro_a, tb = Ab4.y;
        if (vr < R(0)) {
            const R vsa = alpha * cs_a - beta * vr;
            const R vsb = alpha * Ab4.z - beta * vr;
            ta -= R(0.5) * vsa * vr * ior_a;
            tb -= R(0.5) * vsb * vr * Bb4.y;
        }
        const R mub = Bb4.w;
        const R fac = mub * (ta * Fa + tb * Fb) * rinv;
        fx.add(-fac * d[0]);
        fy.add(-fac * d[1]);
        fz.add(-fac * d[2]);
        if (adiabatic) {
            R e = mub * ta * vr * Fa;
            if (cond) {
                const R dP = P_a - Bb4.x;
                const R vsu = Num<R>::sqrt_(fabs(dP) / (R(0.5) * (rho_a + Ab4.w)));
                e += mub * alpha_u * vsu * (V.w - Vb4.w) * R(0.5) * (Fa * ior_a + Fb * Bb4.y);
            }
            du.add(e);
        }
        const R vs = cs_a + beta * (vr < R(0) ? -vr : R(0));
        vsig = vs > vsig ? vs : vsig;
    }
    if (dc.prof) atomicAdd(&counters[APR_PROF_FORCE], npair);
    const double scale = dc.m0 / 3.14159265358979323846;
    const unsigned i = perm[a];
    ax_out[i] = scale * ((double)fx.s - (double)fx.c);
    ay_out[i] = scale * ((double)fy.s - (double)fy.c);
    az_out[i] = scale * ((double)fz.s - (double)fz.c);
    dudt_out[i] = adiabatic ? scale * ((double)du.s - (double)du.c) : 0.0;
    vsig_out[i] = (double)vsig;
}

apr_status force_pass(apr_ctx* c)
{
    Workspace& W = c->W;
    const long long n = c->n;
    if (n <= 0) return APR_OK;
    const int ps = prof_begin(c, APR_PROF_FORCE);
    if (c->cfg.precision == APR_PREC_FP64)
        APR_LAUNCH(c, k_force<double>, nblocks(n, 128), 128, 
            c->dc, n, c->cap, W.pk, W.dA, W.dV, W.dB, W.nbr, W.ncnt, W.sx, W.sy, W.sz, W.perm,
            c->p.ax, c->p.ay, c->p.az, c->p.dudt, c->p.vsig, W.counters);
    else
        APR_LAUNCH(c, k_force<float>, nblocks(n, 128), 128, 
            c->dc, n, c->cap, W.pk, W.fA, W.fV, W.fB, W.nbr, W.ncnt, W.sx, W.sy, W.sz, W.perm,
            c->p.ax, c->p.ay, c->p.az, c->p.dudt, c->p.vsig, W.counters);
    prof_end(c, ps);
    return cuda_check(c, cudaGetLastError(), "force");
}

}  // namespace apr

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
// (dx = float(dx_lattice) * D), compensated (Kahan) by groups of four terms; results
// widened to double.
// FP64: the same kernels in double on the float64 coordinates.
#include <cfloat>

#include "apr_density.cuh"
#include "apr_internal.cuh"
#include "apr_pair.cuh"

namespace apr {

// ----------------------------------------------------------------- density

// exact lattice separation (minimum image; PER false: no axis is periodic)
template <bool PER>
__device__ __forceinline__ void lattice_d(const DevCfg& dc, const int4& pa, const int4& pb, int d[3])
{
    d[0] = pa.x - pb.x;
    d[1] = pa.y - pb.y;
    d[2] = pa.z - pb.z;
    if constexpr (PER) {
        d[0] = min_image32(d[0], dc.periodic[0], (int)dc.Lint[0]);
        d[1] = min_image32(d[1], dc.periodic[1], (int)dc.Lint[1]);
        d[2] = min_image32(d[2], dc.periodic[2], (int)dc.Lint[2]);
    }
}

template <typename R>
__device__ __forceinline__ R rel_r2(const DevCfg& dc, const int d[3], const double* sx,
                                    const double* sy, const double* sz, int a, int b);
template <>
__device__ __forceinline__ float rel_r2<float>(const DevCfg& dc, const int d[3], const double*,
                                               const double*, const double*, int, int)
{
    return lattice_r2f(dc.deltaf, d);
}
template <>
__device__ __forceinline__ double rel_r2<double>(const DevCfg& dc, const int*, const double* sx,
                                                 const double* sy, const double* sz, int a, int b)
{
    double d[3];
    Rel<double>::get<true>(dc, int4(), int4(), sx, sy, sz, a, b, d);
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

// Newton-Raphson on g(h) with a bracket over this particle's (symmetric,
// reach-scaled) list; the first pass also finds the nearest lattice neighbour.
// Four list entries are loaded ahead so that several gathers are in flight.
// threads per block of the pair kernels (one particle each): a block's particles
// are consecutive in Morton order and share most of their neighbours in L1 (float
// force: 256 measured 2-3% faster than 128 and 512 on the shock tube; density: 128)
constexpr int DENSITY_THREADS = 128;
template <typename R>
__host__ __device__ constexpr int force_threads() { return sizeof(R) == 4 ? 256 : 128; }

// resident blocks per SM asked of the compiler: the float kernels are bound by
// gather latency, so more warps in flight pay; the double kernels keep their registers
template <typename R>
constexpr int density_min_blocks() { return sizeof(R) == 4 ? 1024 / DENSITY_THREADS : 1; }
template <typename R>
constexpr int force_min_blocks() { return sizeof(R) == 4 ? 1024 / force_threads<R>() : 1; }

// PER false: no periodic axis (minimum-image tests compiled out)
template <typename R, int KT, bool PER>
__global__ void __launch_bounds__(DENSITY_THREADS, density_min_blocks<R>())
    k_density(DevCfg dc, long long n, long long cap, double reach, const int4* __restrict__ pk,
              const double* __restrict__ sh, const unsigned int* __restrict__ nbr,
              const int* __restrict__ ncnt, const double* __restrict__ sx,
              const double* __restrict__ sy, const double* __restrict__ sz, DensityIO io,
              int* status, unsigned long long* counters, const int* __restrict__ active,
              long long nactive, int* __restrict__ retry_q, int* __restrict__ retry_n)
{
    // FP32: Newton steps are accepted on their predicted successor (nr_update)
    constexpr bool ACCEPT = sizeof(R) == 4;
    // all particles, or (active != nullptr) only the queued ones of a retry
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= (active ? nactive : n)) return;
    const int a = active ? active[s] : (int)s;
    if (a < 0 || a >= n) return;
    const int4 pa = pk[a];
    const double hlist = sh[a];
    const int m = ncnt[a];
    if (m < 0) {
        // the list at this h overflowed (e.g. an initial h far too large at a
        // density jump): shrink h and let the host rebuild the lists
        io.h_out[io.perm[a]] = 0.8 * hlist;
        atomicAdd(&status[ST_UNCOVERED], 1);
        atomicAdd(&status[ST_SHRINK], 1);
        retry_q[atomicAdd(retry_n, 1)] = a;
        return;
    }
    const R mua = Num<R>::mass(pa.w);
    const R target = R(dc.knorm_inv) * mua * R(dc.hfact * dc.hfact * dc.hfact);
    // this particle's list: a row of max_neigh entries (a multiple of 4), the first m
    // kept; mpad = m rounded up to 4 (<= max_neigh) bounds the 16-byte loads
    const unsigned int* row = nbr + (long long)a * dc.max_neigh;
    const int mpad = (m + 3) & ~3;
    // the list's reach (float: rounded down, so that h stays inside it) and the
    // convergence tolerance at the iteration's precision
    const R hreach = round_down<R>(reach * hlist);
    const R hcap = retry_cap<R>(hreach, m, dc.max_neigh);
    const R tol = (R)dc.nr_tol;
    NRState<R> st{(R)hlist, R(0), R(0), R(0), false, false};
    unsigned int npair = 0;
    unsigned long long best = ~0ULL;
    // FP32: the nearest lattice neighbour through the float r^2 (see near_update)
    R bestf = R(INFINITY);
    for (int it = 0; it < dc.nr_maxit; ++it) {
        const R hinv = R(1) / st.h;
        const R r2max = R(4) * st.h * st.h;
        // compensated by groups of four list entries (AccB)
        AccB<R> S, T, U;
        const bool first_pass = it == 0;
        int k = 0;
        // the next four list entries are loaded one step ahead (one 16-byte load), so
        // that only the gathers of a step wait on memory
        uint4 nx = make_uint4(0u, 0u, 0u, 0u);
        if (m >= 4) nx = *reinterpret_cast<const uint4*>(row);
        for (; k + 4 <= m; k += 4) {
            const int b0 = (int)nx.x, b1 = (int)nx.y, b2 = (int)nx.z, b3 = (int)nx.w;
            if (k + 8 <= mpad) nx = *reinterpret_cast<const uint4*>(row + k + 4);
            const int4 p0 = pk[b0], p1 = pk[b1], p2 = pk[b2], p3 = pk[b3];
            int d0[3], d1[3], d2[3], d3[3];
            lattice_d<PER>(dc, pa, p0, d0);
            lattice_d<PER>(dc, pa, p1, d1);
            lattice_d<PER>(dc, pa, p2, d2);
            lattice_d<PER>(dc, pa, p3, d3);
            const R r0 = rel_r2<R>(dc, d0, sx, sy, sz, a, b0), r1 = rel_r2<R>(dc, d1, sx, sy, sz, a, b1);
            const R r2 = rel_r2<R>(dc, d2, sx, sy, sz, a, b2), r3 = rel_r2<R>(dc, d3, sx, sy, sz, a, b3);
            if (first_pass) {
                // the nearest lattice neighbour, on the first pass only
                near_update<R>(r0, d0, bestf, best);
                near_update<R>(r1, d1, bestf, best);
                near_update<R>(r2, d2, bestf, best);
                near_update<R>(r3, d3, bestf, best);
            }
            density_term<KT, ACCEPT, R>(r0, hinv, r2max, p0.w, S, T, U, npair);
            density_term<KT, ACCEPT, R>(r1, hinv, r2max, p1.w, S, T, U, npair);
            density_term<KT, ACCEPT, R>(r2, hinv, r2max, p2.w, S, T, U, npair);
            density_term<KT, ACCEPT, R>(r3, hinv, r2max, p3.w, S, T, U, npair);
            S.flush();
            T.flush();
            U.flush();
        }
        for (; k < m; ++k) {
            const int b = (int)row[k];
            const int4 pb = pk[b];
            int d[3];
            lattice_d<PER>(dc, pa, pb, d);
            const R rb = rel_r2<R>(dc, d, sx, sy, sz, a, b);
            if (first_pass) near_update<R>(rb, d, bestf, best);
            density_term<KT, ACCEPT, R>(rb, hinv, r2max, pb.w, S, T, U, npair);
        }
        S.flush();
        T.flush();
        U.flush();
        if (nr_update<R, ACCEPT>(st, S.s, T.s, U.s, mua, target, tol, hreach, hcap)) break;
    }
    if (dc.prof) count_warp(&counters[APR_PROF_DENSITY], npair);
    if (st.uncovered) {
        io.h_out[io.perm[a]] = (double)st.h;
        atomicAdd(&status[ST_UNCOVERED], 1);
        retry_q[atomicAdd(retry_n, 1)] = a;
        return;
    }
    if (!st.conv) atomicAdd(&status[ST_NOCONV], 1);
    density_store<R>(dc, io, a, pa, st.h, st.D, target, best);
}

DensityIO density_io(apr_ctx* c, bool force_data)
{
    Workspace& W = c->W;
    const bool f64 = c->cfg.precision == APR_PREC_FP64;
    void* fa = f64 ? (void*)W.dA : (void*)W.fA;
    void* fv = f64 ? (void*)W.dV : (void*)W.fV;
    void* fb = f64 ? (void*)W.dB : (void*)W.fB;
    return DensityIO{W.perm,     c->p.x,     c->p.y,   c->p.u,    c->p.vx,  c->p.vy,
                     c->p.vz,    c->p.h,     c->p.rho, c->p.omega, c->p.dnn, c->p.pres,
                     c->p.cs,    force_data ? fa : nullptr, fv, fb};
}

// one Newton-Raphson pass over all particles (active == nullptr) or over the
// nactive queued ones; particles that need another attempt go to retry_q[out_q]
apr_status density_pass(apr_ctx* c, long long* uncovered, long long* noconv, const int* active,
                        long long nactive, int out_q, bool force_data)
{
    Workspace& W = c->W;
    const long long n = c->n;
    cudaStream_t st = c->stream;
    cudaMemsetAsync(&W.status[ST_UNCOVERED], 0, 2 * sizeof(int), st);
    cudaMemsetAsync(&W.status[ST_SHRINK], 0, sizeof(int), st);
    cudaMemsetAsync(&W.status[ST_RETRY_N + out_q], 0, sizeof(int), st);
    int ps = prof_begin(c, APR_PROF_DENSITY);
    const long long work = active ? nactive : n;
    if (work > 0) {
        const double reach = DENSITY_REACH;
        const bool c2 = c->cfg.kernel == APR_KERNEL_WENDLAND_C2;
        const DensityIO io = density_io(c, force_data);
#define APR_DENSITY_P(R, KT, P)                                                                      \
    APR_LAUNCH(c, (k_density<R, KT, P>), nblocks(work, DENSITY_THREADS), DENSITY_THREADS, c->dc, n, c->cap, reach, W.pk, W.sh,  \
               W.nbr, W.ncnt, W.sx, W.sy, W.sz, io, W.status, W.counters, active, nactive,         \
               W.retry_q[out_q], &W.status[ST_RETRY_N + out_q])
#define APR_DENSITY(R, KT)                                                                           \
    do {                                                                                             \
        if (any_periodic(c->dc)) APR_DENSITY_P(R, KT, true);                                         \
        else APR_DENSITY_P(R, KT, false);                                                            \
    } while (0)
        if (c->cfg.precision == APR_PREC_FP64) {
            if (c2) APR_DENSITY(double, APR_KERNEL_WENDLAND_C2);
            else APR_DENSITY(double, APR_KERNEL_M4);
        } else {
            if (c2) APR_DENSITY(float, APR_KERNEL_WENDLAND_C2);
            else APR_DENSITY(float, APR_KERNEL_M4);
        }
#undef APR_DENSITY
#undef APR_DENSITY_P
    }
    prof_end(c, ps);
    // one read-back for the index status words and the density counters
    cudaMemcpyAsync(c->hbuf, W.status, (ST_SHRINK + 1) * sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync((int*)c->hbuf + 16, &W.status[ST_SORT_ERR], sizeof(int), cudaMemcpyDeviceToHost,
                    st);
    apr_status s = cuda_check(c, cudaStreamSynchronize(st), "density");
    if (s != APR_OK) return s;
    const int* hs = (const int*)c->hbuf;
    if (hs[16]) return fail(c, APR_ERR_STATE, "Morton sort: a tile gave up waiting for its predecessors");
    if (hs[ST_TREE_BAD]) return fail(c, APR_ERR_STATE, "internal error: malformed radix tree");
    if (hs[ST_NEIGH_OVERFLOW] || hs[ST_CAND_OVERFLOW])
        return fail(c, APR_ERR_NEIGH_OVERFLOW, "a neighbour list overflowed");
    *uncovered = hs[ST_UNCOVERED];
    *noconv = hs[ST_NOCONV];
    c->last_shrink = hs[ST_SHRINK];
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
    // the FP32-mixed density solve stores float values widened to double: the
    // narrowing is exact, and the records equal the ones it writes itself
    store_force_data_f(A, V, B, s, (float)h[i], (float)rho[i], (float)omega[i], (float)pres[i],
                       (float)cs[i], vx[i], vy[i], vz[i], u[i], pk[s].w);  // B null: two records
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
    store_force_data_d(A, V, B, s, h[i], rho[i], omega[i], pres[i], cs[i], vx[i], vy[i], vz[i], u[i],
                       pk[s].w);
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
            c->p.vz, c->p.u, W.fA, W.fV, force_two_records(c->dc) ? nullptr : W.fB);
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

// per-particle state the force sums need
template <typename R>
struct ForceSelf {
    R hinv, h4, pro, cs, rho, P, ior, vx, vy, vz, u;
};

// one pair of the force / energy sums (pairs outside both supports add nothing);
// B2: the two-record layout (1/(Omega rho) in A's last slot, mass from the level,
// no conductivity)
template <int KT, typename R, bool B2>
__device__ __forceinline__ void force_pair(const DevCfg& dc, const ForceSelf<R>& A, const R d[3],
                                           const F4<R>& Ab, const F4<R>& Vb, const F4<R>& Bb,
                                           int levb, bool adiabatic, bool cond, AccB<R>& fx,
                                           AccB<R>& fy, AccB<R>& fz, AccB<R>& du, R& vsig,
                                           unsigned int& npair)
{
    const R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const R rinv = Num<R>::rsqrt_(r2);
    const R r = r2 * rinv;
    const R hinv_b = Ab.x;
    const R qa = r * A.hinv, qb = r * hinv_b;
    if (!(qa < R(2) || qb < R(2))) return;
    ++npair;
    R fa, dfa, fb, dfb;
    kern_t<KT, R>(qa, fa, dfa);
    kern_t<KT, R>(qb, fb, dfb);
    // float copies of the coefficients: no double-to-float conversion per pair
    R alpha, beta, alpha_u;
    if constexpr (sizeof(R) == 4) {
        alpha = dc.alpha_avf;
        beta = dc.beta_avf;
        alpha_u = dc.alpha_uf;
    } else {
        alpha = dc.alpha_av;
        beta = dc.beta_av;
        alpha_u = dc.alpha_u;
    }
    const R Fa = dfa * A.h4;
    const R Fb = dfb * (hinv_b * hinv_b * hinv_b * hinv_b);
    const R vr = ((A.vx - Vb.x) * d[0] + (A.vy - Vb.y) * d[1] + (A.vz - Vb.z) * d[2]) * rinv;
    R ta = A.pro, tb = Ab.y;
    if (vr < R(0)) {
        const R vsa = alpha * A.cs - beta * vr;
        const R vsb = alpha * Ab.z - beta * vr;
        ta -= R(0.5) * vsa * vr * A.ior;
        tb -= R(0.5) * vsb * vr * (B2 ? Ab.w : Bb.y);
    }
    const R mub = B2 ? Num<R>::mass(levb) : Bb.w;
    const R fac = mub * (ta * Fa + tb * Fb) * rinv;
    fx.add(-fac * d[0]);
    fy.add(-fac * d[1]);
    fz.add(-fac * d[2]);
    if (adiabatic) {
        R e = mub * ta * vr * Fa;
        if (!B2 && cond) {
            const R dP = A.P - Bb.x;
            const R vsu = Num<R>::sqrt_(fabs(dP) / (R(0.5) * (A.rho + Ab.w)));
            e += mub * alpha_u * vsu * (A.u - Vb.w) * R(0.5) * (Fa * A.ior + Fb * Bb.y);
        }
        du.add(e);
    }
    const R vs = A.cs + beta * (vr < R(0) ? -vr : R(0));
    vsig = vs > vsig ? vs : vsig;
}

// B2: the two-record layout (A, V) of runs without conductivity (FP32-mixed)
template <typename R, int KT, bool B2>
__global__ void __launch_bounds__(force_threads<R>(), force_min_blocks<R>())
    k_force(DevCfg dc, long long n, long long cap, const int4* __restrict__ pk,
            const void* __restrict__ Abuf, const void* __restrict__ Vbuf,
            const void* __restrict__ Bbuf, const unsigned int* __restrict__ nbr,
            const int* __restrict__ ncnt, const double* __restrict__ sx,
            const double* __restrict__ sy, const double* __restrict__ sz,
            const unsigned int* __restrict__ perm, double* __restrict__ ax_out,
            double* __restrict__ ay_out, double* __restrict__ az_out,
            double* __restrict__ dudt_out, double* __restrict__ vsig_out,
            unsigned long long* counters, const int* __restrict__ active, long long nactive)
{
    // all particles, or (active != nullptr) the nactive listed sorted slots
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= (active ? nactive : n)) return;
    const int a = active ? active[s] : (int)s;
    if (a < 0 || a >= n) return;
    const int4 pa = pk[a];
    const F4<R> Aa = ld4<R>(Abuf, a), Va = ld4<R>(Vbuf, a);
    const F4<R> Ba = B2 ? F4<R>{R(0), R(0), R(0), R(0)} : ld4<R>(Bbuf, a);
    ForceSelf<R> A;
    A.hinv = Aa.x;
    A.h4 = Aa.x * Aa.x * Aa.x * Aa.x;
    A.pro = Aa.y;
    A.cs = Aa.z;
    A.rho = Aa.w;
    A.P = Ba.x;
    A.ior = B2 ? Aa.w : Ba.y;
    A.vx = Va.x;
    A.vy = Va.y;
    A.vz = Va.z;
    A.u = Va.w;
    const bool adiabatic = dc.eos == APR_EOS_ADIABATIC;
    const bool cond = adiabatic && dc.alpha_u > 0.0;
    AccB<R> fx, fy, fz, du;  // compensated by groups of four pairs
    R vsig = A.cs;
    unsigned int npair = 0;
    const int m = ncnt[a];
    // this particle's list row; mpad = m rounded up to 4 (<= max_neigh) bounds the
    // 16-byte loads
    const unsigned int* row = nbr + (long long)a * dc.max_neigh;
    const int mpad = (m + 3) & ~3;
    int k = 0;
    // the list entries come four at a time (one 16-byte load), the next four while the
    // second pair of the current ones is evaluated, so that only the gathers of a step
    // wait on memory (two at a time measured slower on the shock tube, whose
    // conductivity adds a third record per neighbour to what L1 holds)
    uint4 w4 = make_uint4(0u, 0u, 0u, 0u);
    if (m >= 2) w4 = *reinterpret_cast<const uint4*>(row);
    const F4<R> zero{R(0), R(0), R(0), R(0)};
    for (; k + 2 <= m; k += 2) {
        const bool upper = (k & 2) != 0;
        const int b0 = (int)(upper ? w4.z : w4.x), b1 = (int)(upper ? w4.w : w4.y);
        if (upper && k + 6 <= mpad) w4 = *reinterpret_cast<const uint4*>(row + k + 2);
        const int4 p0 = pk[b0], p1 = pk[b1];
        const F4<R> A0 = ld4<R>(Abuf, b0), V0 = ld4<R>(Vbuf, b0), B0 = B2 ? zero : ld4<R>(Bbuf, b0);
        const F4<R> A1 = ld4<R>(Abuf, b1), V1 = ld4<R>(Vbuf, b1), B1 = B2 ? zero : ld4<R>(Bbuf, b1);
        R d0[3], d1[3];
        Rel<R>::get(dc, pa, p0, sx, sy, sz, a, b0, d0);
        Rel<R>::get(dc, pa, p1, sx, sy, sz, a, b1, d1);
        force_pair<KT, R, B2>(dc, A, d0, A0, V0, B0, p0.w, adiabatic, cond, fx, fy, fz, du, vsig, npair);
        force_pair<KT, R, B2>(dc, A, d1, A1, V1, B1, p1.w, adiabatic, cond, fx, fy, fz, du, vsig, npair);
        if (upper) {
            fx.flush();
            fy.flush();
            fz.flush();
            du.flush();
        }
    }
    for (; k < m; ++k) {
        const int b = (int)row[k];
        const int4 pb = pk[b];
        const F4<R> Ab = ld4<R>(Abuf, b), Vb = ld4<R>(Vbuf, b), Bb = B2 ? zero : ld4<R>(Bbuf, b);
        R d[3];
        Rel<R>::get(dc, pa, pb, sx, sy, sz, a, b, d);
        force_pair<KT, R, B2>(dc, A, d, Ab, Vb, Bb, pb.w, adiabatic, cond, fx, fy, fz, du, vsig, npair);
    }
    fx.flush();
    fy.flush();
    fz.flush();
    du.flush();
    if (dc.prof) count_warp(&counters[APR_PROF_FORCE], npair);
    const double scale = dc.m0_knorm;
    const unsigned i = perm[a];
    ax_out[i] = scale * ((double)fx.s - (double)fx.c);
    ay_out[i] = scale * ((double)fy.s - (double)fy.c);
    az_out[i] = scale * ((double)fz.s - (double)fz.c);
    dudt_out[i] = adiabatic ? scale * ((double)du.s - (double)du.c) : 0.0;
    vsig_out[i] = (double)vsig;
}

apr_status force_pass(apr_ctx* c, const int* active, long long nactive)
{
    Workspace& W = c->W;
    const long long n = c->n;
    const long long work = active ? nactive : n;
    if (n <= 0 || work <= 0) return APR_OK;
    const int ps = prof_begin(c, APR_PROF_FORCE);
    const bool c2 = c->cfg.kernel == APR_KERNEL_WENDLAND_C2;
// (the force kernel keeps the run-time minimum-image tests: compiled out they made it
// slower on the flyby and the disc, 3.14 -> 3.22 and 0.70 -> 0.74 ms)
#define APR_FORCE(R, KT, B2, A, V, B)                                                                \
    APR_LAUNCH(c, (k_force<R, KT, B2>), nblocks(work, force_threads<R>()), force_threads<R>(), c->dc, n, c->cap, W.pk, A, V, B, W.nbr, \
               W.ncnt, W.sx, W.sy, W.sz, W.perm, c->p.ax, c->p.ay, c->p.az, c->p.dudt, c->p.vsig,   \
               W.counters, active, nactive)
    if (c->cfg.precision == APR_PREC_FP64) {
        if (c2) APR_FORCE(double, APR_KERNEL_WENDLAND_C2, false, W.dA, W.dV, W.dB);
        else APR_FORCE(double, APR_KERNEL_M4, false, W.dA, W.dV, W.dB);
    } else if (force_two_records(c->dc)) {
        if (c2) APR_FORCE(float, APR_KERNEL_WENDLAND_C2, true, W.fA, W.fV, W.fB);
        else APR_FORCE(float, APR_KERNEL_M4, true, W.fA, W.fV, W.fB);
    } else {
        if (c2) APR_FORCE(float, APR_KERNEL_WENDLAND_C2, false, W.fA, W.fV, W.fB);
        else APR_FORCE(float, APR_KERNEL_M4, false, W.fA, W.fV, W.fB);
    }
#undef APR_FORCE
    prof_end(c, ps);
    return cuda_check(c, cudaGetLastError(), "force");
}

}  // namespace apr

// Relaxing (Sec. 2.4) on sm_103a: the particles a split/merge pass introduced
// (flag NEW) are shuffled towards a reference set (the particles before the
// split/merge) by dx = 0.5 dt^2 (a_new - a_ref), dt = 0.3 h / c_s, |dx| capped
// at h, where a_new is the current acceleration and a_ref the reference set's
// accelerations interpolated to the particle, sum over the reference set of
// (m_b / rho_b) a_b W(|x - x_b|, h_b).
//
// The reference set is staged once in the spare bound slots [n, n + nref).
// For the interpolation the index (Morton sort, radix tree, symmetric lists at
// 2 max(h_a, h_b)) is built over the current and staged particles together;
// the lists then hold every reference particle whose support reaches a NEW
// particle.  Sums in FP32 on relative lattice coordinates with compensated
// accumulation (FP64 in the FP64 path); the shuffle energy in FP64.
#include "apr_internal.cuh"
#include "apr_pair.cuh"

namespace apr {

constexpr unsigned RELAX_TARGET = 1u;  // a NEW particle of the current set
constexpr unsigned RELAX_REF = 2u;     // a staged reference particle

__global__ void k_relax_stage(long long n, long long nref, apr_particles ref, apr_particles p)
{
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nref) return;
    const long long j = n + k;
    p.x[j] = ref.x[k];
    p.y[j] = ref.y[k];
    p.z[j] = ref.z[k];
    p.h[j] = ref.h[k];
    p.rho[j] = ref.rho[k];
    p.ax[j] = ref.ax[k];
    p.ay[j] = ref.ay[k];
    p.az[j] = ref.az[k];
    p.level[j] = ref.level[k];
    p.flags[j] = ref.flags[k] & APR_FLAG_DEAD;
}

// caller order: NEW live particles of [0, n) are targets, live staged ones references
__global__ void k_relax_roles(long long n, long long nt, const unsigned char* __restrict__ flags,
                              unsigned int* __restrict__ role)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const unsigned char f = flags[i];
    unsigned r = 0;
    if (!(f & APR_FLAG_DEAD)) {
        if (i >= n) r = RELAX_REF;
        else if (f & APR_FLAG_NEW) r = RELAX_TARGET;
    }
    role[i] = r;
}

// a_ref of every target, written to its caller slot (3 doubles per slot)
template <typename R>
__global__ void __launch_bounds__(128)
    k_relax_interp(DevCfg dc, long long nt, long long cap, const int4* __restrict__ pk,
                   const double* __restrict__ sh, const unsigned int* __restrict__ perm,
                   const unsigned int* __restrict__ role, const unsigned int* __restrict__ nbr,
                   const int* __restrict__ ncnt, const double* __restrict__ sx,
                   const double* __restrict__ sy, const double* __restrict__ sz,
                   const double* __restrict__ rho, const double* __restrict__ ax,
                   const double* __restrict__ ay, const double* __restrict__ az,
                   double* __restrict__ aref)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nt) return;
    const unsigned i = perm[s];
    if (role[i] != RELAX_TARGET) return;
    const int a = (int)s;
    const int4 pa = pk[a];
    Acc<R> gx, gy, gz;
    const int m = ncnt[a];
    for (int k = 0; k < m; ++k) {
        const int b = (int)nbr[(long long)a * dc.max_neigh + k];
        const unsigned j = perm[b];
        if (role[j] != RELAX_REF) continue;
        R d[3];
        Rel<R>::get(dc, pa, pk[b], sx, sy, sz, a, b, d);
        const R r = Num<R>::sqrt_(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const R hinv = (R)(1.0 / sh[b]);
        R f, df;
        kern<R>(dc.kernel, r * hinv, f, df);
        if (f == R(0)) continue;
        // (mu_b / rho_b) f / h_b^3; m0 / knorm_inv applied once below
        const R wgt = Num<R>::mass(pk[b].w) / (R)rho[j] * f * (hinv * hinv * hinv);
        gx.add(wgt * (R)ax[j]);
        gy.add(wgt * (R)ay[j]);
        gz.add(wgt * (R)az[j]);
    }
    const double scale = dc.m0_knorm;
    aref[3 * (long long)i] = scale * ((double)gx.s - (double)gx.c);
    aref[3 * (long long)i + 1] = scale * ((double)gy.s - (double)gy.c);
    aref[3 * (long long)i + 2] = scale * ((double)gz.s - (double)gz.c);
}

__device__ __forceinline__ double wrap_coord(const DevCfg& dc, int k, double v)
{
    if (dc.periodic[k]) {
        if (v < dc.lo[k]) v += dc.L[k];
        else if (v >= dc.hi[k]) v -= dc.L[k];
    }
    return v;
}

// the shift of every NEW particle; block partials of the shuffle energy
__global__ void __launch_bounds__(256)
    k_relax_shift(DevCfg dc, long long n, apr_particles p, const unsigned int* __restrict__ role,
                  const double* __restrict__ aref, double* __restrict__ partials)
{
    double ke = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (role[i] != RELAX_TARGET) continue;
        const double h = p.h[i];
        const double dt = 0.3 * h / p.cs[i];
        const double c = 0.5 * dt * dt;
        double d[3] = {c * (p.ax[i] - aref[3 * i]), c * (p.ay[i] - aref[3 * i + 1]),
                       c * (p.az[i] - aref[3 * i + 2])};
        double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (len > h) {
            const double sc = h / len;
            d[0] = d[0] * sc;
            d[1] = d[1] * sc;
            d[2] = d[2] * sc;
            len = h;
        }
        p.x[i] = wrap_coord(dc, 0, p.x[i] + d[0]);
        p.y[i] = wrap_coord(dc, 1, p.y[i] + d[1]);
        p.z[i] = wrap_coord(dc, 2, p.z[i] + d[2]);
        ke += len / (dt * dt);
    }
    __shared__ double sm[8];
    for (int o = 16; o > 0; o >>= 1) ke += __shfl_down_sync(0xffffffffu, ke, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = ke;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sm[w];
        partials[blockIdx.x * 32] = t;
    }
}

__global__ void k_relax_final(int nblk, const double* __restrict__ partials, double* __restrict__ out)
{
    __shared__ double sm[256];
    double x = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 256) x += partials[b * 32];
    sm[threadIdx.x] = x;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sm[0];
}

__global__ void k_clear_new(long long n, unsigned char* flags)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = flags[i] & (unsigned char)~APR_FLAG_NEW;
}

apr_status relax_stage(apr_ctx* c, const apr_particles* ref, long long nref)
{
    if (nref > 0)
        APR_LAUNCH(c, k_relax_stage, nblocks(nref, 256), 256, c->n, nref, *ref, c->p);
    return cuda_check(c, cudaGetLastError(), "relax stage");
}

// a_ref of the NEW particles, into W.acc_sum (3 doubles per caller slot); the
// bound count is n + nref while the index is built and n again on return
apr_status relax_interp(apr_ctx* c, long long nref, apr_status (*index)(apr_ctx*))
{
    Workspace& W = c->W;
    const long long n = c->n, nt = n + nref;
    if (nt <= 0) return APR_OK;
    APR_LAUNCH(c, k_relax_roles, nblocks(nt, 256), 256, n, nt, c->p.flags, W.uflag);
    c->n = nt;
    apr_status s = index(c);
    if (s == APR_OK) {
        if (c->cfg.precision == APR_PREC_FP64)
            APR_LAUNCH(c, k_relax_interp<double>, nblocks(nt, 128), 128, c->dc, nt, c->cap, W.pk, W.sh,
                       W.perm, W.uflag, W.nbr, W.ncnt, W.sx, W.sy, W.sz, c->p.rho, c->p.ax, c->p.ay,
                       c->p.az, (double*)W.acc_sum);
        else
            APR_LAUNCH(c, k_relax_interp<float>, nblocks(nt, 128), 128, c->dc, nt, c->cap, W.pk, W.sh,
                       W.perm, W.uflag, W.nbr, W.ncnt, W.sx, W.sy, W.sz, c->p.rho, c->p.ax, c->p.ay,
                       c->p.az, (double*)W.acc_sum);
        s = cuda_check(c, cudaGetLastError(), "relax interpolation");
    }
    c->n = n;
    return s;
}

apr_status relax_shift(apr_ctx* c, double* ke)
{
    Workspace& W = c->W;
    const long long n = c->n;
    int grid = (int)nblocks(n, 256);
    if (grid > RED_BLOCKS) grid = RED_BLOCKS;
    if (grid < 1) grid = 1;
    APR_LAUNCH(c, k_relax_shift, grid, 256, c->dc, n, c->p, W.uflag, (const double*)W.acc_sum, W.red);
    APR_LAUNCH(c, k_relax_final, 1, 256, grid, W.red, W.redout);
    cudaMemcpyAsync(c->hbuf, W.redout, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    apr_status s = cuda_check(c, cudaStreamSynchronize(c->stream), "relax shift");
    if (s != APR_OK) return s;
    memcpy(ke, c->hbuf, sizeof(double));
    return APR_OK;
}

apr_status clear_new(apr_ctx* c)
{
    if (c->n > 0) APR_LAUNCH(c, k_clear_new, nblocks(c->n, 256), 256, c->n, c->p.flags);
    return cuda_check(c, cudaGetLastError(), "clear new");
}

}  // namespace apr

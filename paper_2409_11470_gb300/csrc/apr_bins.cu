// Individual time steps in bins (Sec. 2.5) on sm_103a: particle i in bin b_i
// steps dt_max / 2^b_i on the grid of the 2^B substeps of a step of dt_max.
// These kernels do the per-particle parts: binning by the time-step limit
// min(ccour h / v_sig, cforce sqrt(h / |a|)), the half kicks at the start and
// the end of each particle's step, the flag that keeps split/merge to the
// particles whose step ends, the queue of those particles (sorted slots), and
// their new bins.
#include "apr_internal.cuh"

namespace apr {

__device__ __forceinline__ double particle_dt(const DevCfg& dc, const apr_particles& p, long long i)
{
    double dt = INFINITY;
    const double h = p.h[i];
    if (p.vsig[i] > 0.0) dt = fmin(dt, dc.ccour * h / p.vsig[i]);
    const double a = sqrt(p.ax[i] * p.ax[i] + p.ay[i] * p.ay[i] + p.az[i] * p.az[i]);
    if (a > 0.0) dt = fmin(dt, dc.cforce * sqrt(h / a));
    return dt;
}

// the smallest bin b <= B with dt_max / 2^b <= dt (B if none); the halving is exact
__device__ __forceinline__ int wanted_bin(double dt, double dt_max, int B)
{
    int b = 0;
    double d = dt_max;
    while (b < B && d > dt) {
        d *= 0.5;
        ++b;
    }
    return b;
}

__global__ void k_bins_init(DevCfg dc, long long n, apr_particles p, double dt_max, int B)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p.bin[i] = (unsigned char)wanted_bin(particle_dt(dc, p, i), dt_max, B);
}

// half kick of the particles whose step starts at substep k (end_of_step 0) or
// ends at the end of substep k (end_of_step 1)
__global__ void k_bins_kick(DevCfg dc, long long n, apr_particles p, double dt_max, int B,
                            long long k, int end_of_step)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (p.flags[i] & (APR_FLAG_FIXED | APR_FLAG_DEAD)) return;
    const int b = p.bin[i];
    const long long period = (1LL << B) >> b;
    const long long t = end_of_step ? k + 1 : k;
    if (t % period != 0) return;
    const double hdt = 0.5 * dt_max / (double)(1LL << b);
    p.vx[i] += hdt * p.ax[i];
    p.vy[i] += hdt * p.ay[i];
    p.vz[i] += hdt * p.az[i];
    if (dc.eos == APR_EOS_ADIABATIC) p.u[i] += hdt * p.dudt[i];
}

// flag (or unflag) the particles whose step does not end at the end of substep k
__global__ void k_bins_mark(long long n, apr_particles p, int B, long long k, int on)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (on) {
        const long long period = (1LL << B) >> p.bin[i];
        if ((k + 1) % period != 0) p.flags[i] = p.flags[i] | APR_FLAG_INACTIVE;
    } else {
        p.flags[i] = p.flags[i] & (unsigned char)~APR_FLAG_INACTIVE;
    }
}

// the sorted slots of the live particles whose step ends at the end of substep k
__global__ void k_bins_queue(long long n, const unsigned int* __restrict__ perm,
                             const unsigned char* __restrict__ bin,
                             const unsigned char* __restrict__ flags, int B, long long k,
                             int* __restrict__ queue, int* __restrict__ count)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const unsigned i = perm[s];
    if (flags[i] & APR_FLAG_DEAD) return;
    const long long period = (1LL << B) >> bin[i];
    if ((k + 1) % period == 0) queue[atomicAdd(count, 1)] = (int)s;
}

// new bins of the active particles at the grid point k + 1
__global__ void k_bins_rebin(DevCfg dc, long long nq, const int* __restrict__ queue,
                             const unsigned int* __restrict__ perm, apr_particles p, double dt_max,
                             int B, int aligned, double dt_min, int* saturated)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nq) return;
    const unsigned i = perm[queue[t]];
    const double dti = particle_dt(dc, p, i);
    int b;
    if (p.flags[i] & APR_FLAG_CHANGED) {
        b = B;  // split or merged this substep: the shortest step (Sec. 2.5)
    } else {
        b = wanted_bin(dti, dt_max, B);
        if (b < aligned) b = aligned;
    }
    if (dti < dt_min) atomicAdd(saturated, 1);
    p.bin[i] = (unsigned char)b;
}

apr_status bins_init(apr_ctx* c, double dt_max, int B)
{
    if (c->n > 0) APR_LAUNCH(c, k_bins_init, nblocks(c->n, 256), 256, c->dc, c->n, c->p, dt_max, B);
    return cuda_check(c, cudaGetLastError(), "bins init");
}

apr_status bins_kick(apr_ctx* c, double dt_max, int B, long long k, int end_of_step)
{
    if (c->n > 0)
        APR_LAUNCH(c, k_bins_kick, nblocks(c->n, 256), 256, c->dc, c->n, c->p, dt_max, B, k,
                   end_of_step);
    return cuda_check(c, cudaGetLastError(), "bins kick");
}

apr_status bins_mark_inactive(apr_ctx* c, long long k, int B, bool on)
{
    if (c->n > 0) APR_LAUNCH(c, k_bins_mark, nblocks(c->n, 256), 256, c->n, c->p, B, k, on ? 1 : 0);
    return cuda_check(c, cudaGetLastError(), "bins mark");
}

// queue of the active sorted slots (after index_sort); *nact on the host
apr_status bins_active_queue(apr_ctx* c, long long k, int B, long long* nact)
{
    Workspace& W = c->W;
    cudaMemsetAsync(&W.status[ST_ACTIVE_N], 0, sizeof(int), c->stream);
    if (c->n > 0)
        APR_LAUNCH(c, k_bins_queue, nblocks(c->n, 256), 256, c->n, W.perm, c->p.bin, c->p.flags, B, k,
                   W.active_q, &W.status[ST_ACTIVE_N]);
    cudaMemcpyAsync(c->hbuf, &W.status[ST_ACTIVE_N], sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    apr_status s = cuda_check(c, cudaStreamSynchronize(c->stream), "bins queue");
    if (s != APR_OK) return s;
    *nact = ((int*)c->hbuf)[0];
    return APR_OK;
}

apr_status bins_rebin(apr_ctx* c, double dt_max, int B, long long k, long long nq)
{
    Workspace& W = c->W;
    const long long nsub = 1LL << B;
    int aligned = B;  // the longest step whose grid contains k + 1
    while (aligned > 0 && (k + 1) % (nsub >> (aligned - 1)) == 0) --aligned;
    if (nq > 0)
        APR_LAUNCH(c, k_bins_rebin, nblocks(nq, 256), 256, c->dc, nq, W.active_q, W.perm, c->p, dt_max,
                   B, aligned, dt_max / (double)nsub, &W.status[ST_SATURATED]);
    return cuda_check(c, cudaGetLastError(), "bins rebin");
}

}  // namespace apr

// Density error of one split pass and its adjoint, on sm_103a.
//
// Not an operation of the paper's method: the paper chooses the child
// separation (Sec. 2.2, Eq. 2) and relaxes new children (Sec. 2.5) so that the
// split set reproduces the density of the original set.  This file measures
// that error and its gradient with respect to the children's offsets and
// smoothing lengths, so that child placement can be optimised.
//
// Reference set: the bound particles [0, n) at their own h.  Split k puts two
// children at x_p + d_k and x_p - d_k (one level finer, Eq. 1 mass) with their
// own smoothing lengths; the new set is the reference set without the parents
// plus the children.  With e_a = rho_new(a) - rho_ref(x_a),
//   rho_new(a) = sum_{b in new set} m_b W(r_ab, h_a)   (self included, h fixed)
//   rho_ref(x) = sum_{b in reference set} m_b W(|x - x_b|, h_b)
//   J = sum_{children a} e_a^2
// and, with W' = f'(q)/(pi h^4) and u_ab the unit vector from b to a,
//   dJ/dx_a = 2 e_a [sum_{b new} m_b W'(r_ab, h_a) u_ab - sum_{b ref} m_b W'(r_ab, h_b) u_ab]
//             + sum_{children c} 2 e_c m_a W'(r_ac, h_c) u_ac
//   dJ/dh_a = 2 e_a sum_{b new} m_b dW/dh(r_ab, h_a),  dW/dh = -(3 f + q f')/(pi h^4)
//   dJ/dd_k = dJ/dx_(child 2k) - dJ/dx_(child 2k+1).
//
// The children are written into the spare bound slots [n, n + 2k) and the index
// (Morton sort, radix tree, symmetric lists at 2 max(h_a, h_b)) is built over
// the combined set: one symmetric list holds every pair that any of the three
// sums needs.  Pair sums in FP32 on relative lattice coordinates with Kahan
// compensation (FP64 in the FP64 path); J is reduced in FP64 in a fixed order.
#include "apr_internal.cuh"
#include "apr_pair.cuh"

namespace apr {

constexpr unsigned ROLE_NEW = 1u;    // member of the new (split) set
constexpr unsigned ROLE_REF = 2u;    // member of the reference set
constexpr unsigned ROLE_CHILD = 4u;  // a child: a loss term and a variable
constexpr int ADJ_THREADS = 128;

// caller order: live reference particles are in both sets; the rest in neither
__global__ void k_adj_roles(long long n, long long nt, const unsigned char* __restrict__ flags,
                            unsigned int* __restrict__ role)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    role[i] = (i < n && !(flags[i] & APR_FLAG_DEAD)) ? (ROLE_NEW | ROLE_REF) : 0u;
}

// the children of split k at slots n + 2k (x_p + d_k) and n + 2k + 1 (x_p - d_k);
// a bad split (parent out of range, dead or repeated, h not positive, a value not
// finite) writes nothing and raises the status word
__global__ void k_adj_children(DevCfg dc, long long n, long long npar,
                               const long long* __restrict__ parent, const double* __restrict__ d,
                               const double* __restrict__ hc, apr_particles p,
                               unsigned int* __restrict__ role, int* status)
{
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npar) return;
    const long long q = parent[k];
    const double h0 = hc[2 * k], h1 = hc[2 * k + 1];
    const double dk[3] = {d[3 * k], d[3 * k + 1], d[3 * k + 2]};
    bool ok = q >= 0 && q < n && h0 > 0.0 && h1 > 0.0 && isfinite(h0) && isfinite(h1) &&
              isfinite(dk[0]) && isfinite(dk[1]) && isfinite(dk[2]);
    if (ok) ok = p.level[q] < 255;
    // the parent leaves the new set; a second claim finds it already gone
    if (ok) ok = atomicCAS(&role[q], ROLE_NEW | ROLE_REF, ROLE_REF) == (ROLE_NEW | ROLE_REF);
    if (!ok) {
        atomicOr(&status[ST_ADJ_BAD], 1);
        return;
    }
    const double xp[3] = {p.x[q], p.y[q], p.z[q]};
    for (int side = 0; side < 2; ++side) {
        const long long j = n + 2 * k + side;
        const double sg = side == 0 ? 1.0 : -1.0;
        double x[3];
        for (int m = 0; m < 3; ++m) {
            double v = xp[m] + sg * dk[m];
            if (dc.periodic[m]) {
                if (v < dc.lo[m]) v += dc.L[m];
                else if (v >= dc.hi[m]) v -= dc.L[m];
            }
            x[m] = v;
        }
        p.x[j] = x[0];
        p.y[j] = x[1];
        p.z[j] = x[2];
        p.h[j] = side == 0 ? h0 : h1;
        p.level[j] = (unsigned char)(p.level[q] + 1);
        p.flags[j] = 0;
        role[j] = ROLE_NEW | ROLE_CHILD;
    }
}

// per sorted slot: (1/h, 2^-level, role) for the pair loops
template <typename R>
struct AdjSlot {
    R hinv, mu;
    unsigned role, pad;
};

template <typename R>
__global__ void k_adj_prep(long long nt, const unsigned int* __restrict__ perm,
                           const unsigned int* __restrict__ role, const int4* __restrict__ pk,
                           const double* __restrict__ sh, AdjSlot<R>* __restrict__ X)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nt) return;
    AdjSlot<R> v;
    v.hinv = (R)(1.0 / sh[s]);
    v.mu = Num<R>::mass(pk[s].w);
    v.role = role[perm[s]];
    v.pad = 0;
    X[s] = v;
}

// fixed-shape block sum of one double into partials[block * 32]
__device__ __forceinline__ void adj_block_sum(double v, double* partials)
{
    __shared__ double sm[ADJ_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < ADJ_THREADS / 32; ++w) t += sm[w];
        partials[blockIdx.x * 32] = t;
    }
}

// forward: e_a of every child, and the block partials of J
template <typename R>
__global__ void __launch_bounds__(ADJ_THREADS)
    k_adj_forward(DevCfg dc, long long nt, long long cap, const int4* __restrict__ pk,
                  const AdjSlot<R>* __restrict__ X, const unsigned int* __restrict__ nbr,
                  const int* __restrict__ ncnt, const double* __restrict__ sx,
                  const double* __restrict__ sy, const double* __restrict__ sz,
                  const unsigned int* __restrict__ perm, R* __restrict__ E,
                  double* __restrict__ rho_out, double* __restrict__ partials)
{
    double jsum = 0.0;
    const double scale = dc.m0_knorm;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < nt;
         s += (long long)gridDim.x * blockDim.x) {
        const AdjSlot<R> xa = X[s];
        if (!(xa.role & ROLE_CHILD)) continue;
        const int a = (int)s;
        const int4 pa = pk[a];
        Acc<R> Sn, Sr;  // sum mu_b f(q_a) (new set), sum mu_b f(q_b) / h_b^3 (reference set)
        Sn.add(xa.mu);  // self, f(0) = 1
        const int m = ncnt[a];
        for (int k = 0; k < m; ++k) {
            const int b = (int)nbr[(long long)a * dc.max_neigh + k];
            const AdjSlot<R> xb = X[b];
            if (!(xb.role & (ROLE_NEW | ROLE_REF))) continue;
            R d[3];
            Rel<R>::get(dc, pa, pk[b], sx, sy, sz, a, b, d);
            const R r = Num<R>::sqrt_(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            R f, df;
            if (xb.role & ROLE_NEW) {
                kern<R>(dc.kernel, r * xa.hinv, f, df);
                Sn.add(xb.mu * f);
            }
            if (xb.role & ROLE_REF) {
                kern<R>(dc.kernel, r * xb.hinv, f, df);
                Sr.add(xb.mu * f * (xb.hinv * xb.hinv * xb.hinv));
            }
        }
        const double ha3 = (double)xa.hinv * (double)xa.hinv * (double)xa.hinv;
        const double e = scale * (((double)Sn.s - (double)Sn.c) * ha3 - ((double)Sr.s - (double)Sr.c));
        E[a] = (R)e;
        rho_out[perm[a]] = e;
        jsum += e * e;
    }
    adj_block_sum(jsum, partials);
}

// three compensated sums of t * d[0..2]
template <typename R>
struct Acc3 {
    Acc<R> x, y, z;
    __device__ __forceinline__ void add(R t, const R d[3])
    {
        x.add(t * d[0]);
        y.add(t * d[1]);
        z.add(t * d[2]);
    }
    __device__ __forceinline__ double get(int c) const
    {
        const Acc<R>& a = c == 0 ? x : (c == 1 ? y : z);
        return (double)a.s - (double)a.c;
    }
};

// reverse: dJ/dx and dJ/dh of every child, written to its caller slot
template <typename R>
__global__ void __launch_bounds__(ADJ_THREADS)
    k_adj_reverse(DevCfg dc, long long nt, long long cap, const int4* __restrict__ pk,
                  const AdjSlot<R>* __restrict__ X, const R* __restrict__ E,
                  const unsigned int* __restrict__ nbr, const int* __restrict__ ncnt,
                  const double* __restrict__ sx, const double* __restrict__ sy,
                  const double* __restrict__ sz, const unsigned int* __restrict__ perm,
                  double* __restrict__ gx_out, double* __restrict__ gy_out,
                  double* __restrict__ gz_out, double* __restrict__ gh_out)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nt) return;
    const AdjSlot<R> xa = X[s];
    if (!(xa.role & ROLE_CHILD)) return;
    const int a = (int)s;
    const int4 pa = pk[a];
    const R ea = E[a];
    // own-set gradient at h_a, reference interpolant, other children's sums, h derivative
    Acc3<R> on, rf, rv;
    Acc<R> dh;
    dh.add(R(-3) * xa.mu);  // self: -(3 f(0) + 0)
    const int m = ncnt[a];
    for (int k = 0; k < m; ++k) {
        const int b = (int)nbr[(long long)a * dc.max_neigh + k];
        const AdjSlot<R> xb = X[b];
        if (!xb.role) continue;
        R d[3];
        Rel<R>::get(dc, pa, pk[b], sx, sy, sz, a, b, d);
        const R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const R r = Num<R>::sqrt_(r2);
        const R rinv = r > R(0) ? R(1) / r : R(0);  // coincident pair: f'(0) = 0
        R f, df;
        if (xb.role & ROLE_NEW) {
            const R q = r * xa.hinv;
            kern<R>(dc.kernel, q, f, df);
            dh.add(-xb.mu * (R(3) * f + q * df));
            on.add(xb.mu * df * rinv, d);
        }
        if (xb.role & ROLE_REF) {
            kern<R>(dc.kernel, r * xb.hinv, f, df);
            const R h4 = (xb.hinv * xb.hinv) * (xb.hinv * xb.hinv);
            rf.add(xb.mu * df * h4 * rinv, d);
        }
        if (xb.role & ROLE_CHILD) {
            kern<R>(dc.kernel, r * xb.hinv, f, df);
            const R h4 = (xb.hinv * xb.hinv) * (xb.hinv * xb.hinv);
            rv.add(E[b] * df * h4 * rinv, d);
        }
    }
    const double scale = dc.m0_knorm;
    const double ha = (double)xa.hinv, ha4 = (ha * ha) * (ha * ha);
    const double e2 = 2.0 * (double)ea, mua = (double)xa.mu;
    double g[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double own = on.get(c) * ha4 - rf.get(c);
        g[c] = e2 * scale * own + 2.0 * scale * mua * rv.get(c);
    }
    const unsigned i = perm[a];
    gx_out[i] = g[0];
    gy_out[i] = g[1];
    gz_out[i] = g[2];
    gh_out[i] = e2 * scale * ha4 * ((double)dh.s - (double)dh.c);
}

// the split's chain rule: dJ/dd_k = g(child +) - g(child -); dJ/dhc = g_h
__global__ void k_adj_chain(long long n, long long npar, const double* __restrict__ gx,
                            const double* __restrict__ gy, const double* __restrict__ gz,
                            const double* __restrict__ gh, double* __restrict__ grad_d,
                            double* __restrict__ grad_hc)
{
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npar) return;
    const long long j0 = n + 2 * k, j1 = j0 + 1;
    grad_d[3 * k] = gx[j0] - gx[j1];
    grad_d[3 * k + 1] = gy[j0] - gy[j1];
    grad_d[3 * k + 2] = gz[j0] - gz[j1];
    grad_hc[2 * k] = gh[j0];
    grad_hc[2 * k + 1] = gh[j1];
}

__global__ void k_adj_final(int nblk, const double* __restrict__ partials, double* __restrict__ out)
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

template <typename R>
static apr_status adjoint_sums_t(apr_ctx* c, long long n, long long npar, double* loss,
                                 double* grad_d, double* grad_hc, AdjSlot<R>* X, R* E)
{
    Workspace& W = c->W;
    const long long nt = c->n;
    APR_LAUNCH(c, k_adj_prep<R>, nblocks(nt, 256), 256, nt, W.perm, W.uflag, W.pk, W.sh, X);
    const int grid = (int)min((long long)RED_BLOCKS, (nt + ADJ_THREADS - 1) / ADJ_THREADS);
    APR_LAUNCH(c, k_adj_forward<R>, grid, ADJ_THREADS, c->dc, nt, c->cap, W.pk, X, W.nbr, W.ncnt,
               W.sx, W.sy, W.sz, W.perm, E, c->p.rho, W.red);
    APR_LAUNCH(c, k_adj_reverse<R>, nblocks(nt, ADJ_THREADS), ADJ_THREADS, c->dc, nt, c->cap, W.pk,
               X, E, W.nbr, W.ncnt, W.sx, W.sy, W.sz, W.perm, c->p.ax, c->p.ay, c->p.az,
               c->p.dudt);
    APR_LAUNCH(c, k_adj_chain, nblocks(npar, 256), 256, n, npar, c->p.ax, c->p.ay, c->p.az, c->p.dudt,
               grad_d, grad_hc);
    APR_LAUNCH(c, k_adj_final, 1, 256, grid, W.red, W.redout);
    cudaMemcpyAsync(c->hbuf, W.redout, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    apr_status s = cuda_check(c, cudaStreamSynchronize(c->stream), "density loss");
    if (s != APR_OK) return s;
    memcpy(loss, c->hbuf, sizeof(double));
    return APR_OK;
}

apr_status adjoint_children(apr_ctx* c, long long npar, const long long* parent, const double* d,
                            const double* hc, bool* bad)
{
    Workspace& W = c->W;
    const long long n = c->n, nt = n + 2 * npar;
    cudaStream_t st = c->stream;
    APR_LAUNCH(c, k_adj_roles, nblocks(nt, 256), 256, n, nt, c->p.flags, W.uflag);
    cudaMemsetAsync(&W.status[ST_ADJ_BAD], 0, sizeof(int), st);
    APR_LAUNCH(c, k_adj_children, nblocks(npar, 256), 256, c->dc, n, npar, parent, d, hc, c->p,
               W.uflag, W.status);
    cudaMemcpyAsync(c->hbuf, &W.status[ST_ADJ_BAD], sizeof(int), cudaMemcpyDeviceToHost, st);
    apr_status s = cuda_check(c, cudaStreamSynchronize(st), "density loss: children");
    if (s != APR_OK) return s;
    *bad = ((int*)c->hbuf)[0] != 0;
    return APR_OK;
}

apr_status adjoint_sums(apr_ctx* c, long long n, long long npar, double* loss, double* grad_d,
                        double* grad_hc)
{
    Workspace& W = c->W;
    if (c->cfg.precision == APR_PREC_FP64)
        return adjoint_sums_t<double>(c, n, npar, loss, grad_d, grad_hc,
                                      reinterpret_cast<AdjSlot<double>*>(W.dA), W.dV);
    return adjoint_sums_t<float>(c, n, npar, loss, grad_d, grad_hc,
                                 reinterpret_cast<AdjSlot<float>*>(W.fA),
                                 reinterpret_cast<float*>(W.fB));
}

}  // namespace apr

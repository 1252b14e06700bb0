// Refinement (split / merge), point masses and time integration on sm_103a.
//
// Split (Sec. 2.2, Eq. 2): a particle below its zone's level becomes two
// children at +-r_sep along a unit vector tangential to the zone boundary,
// rotated by a random angle; r_sep = min(0.2 h, 0.35 d_nn); h' = (1/2)^(1/3) h.
// The parent keeps its slot, the new child is appended at n + rank where rank
// is the exclusive prefix count of split parents in index order.
// Merge (Sec. 2.3, Eq. 3): the candidates of one level are paired by a tree
// cut through the centre of mass with an even count on each side; a pair whose
// centre of mass lies at a lower level merges into the lower index.  The tree
// is built level-synchronously: every round cuts all open segments at once
// with segmented reductions, then a stable partition.
// This file is compiled without fused multiply-add contraction so that every
// float64 operation rounds exactly as written (the geometry is bit-exact).
#include <cfloat>
#include <climits>

#include "apr_internal.cuh"

namespace apr {

constexpr double SPLIT_HFAC = 0.7937005259840998;  // (1/2)^(1/3), Eq. 2
constexpr double MERGE_HFAC = 1.2599210498948732;  // 2^(1/3), Eq. 3

// ------------------------------------------------------------ zone levels

__device__ int region_level(const DevRegion& r, double px, double py, double pz)
{
    int lev = 0;
    for (int k = 0; k < r.nlev; ++k) {
        bool inside;
        if (r.shape == APR_SHAPE_SPHERE) {
            double dx = px - r.centre[0], dy = py - r.centre[1], dz = pz - r.centre[2];
            double d2 = dx * dx + dy * dy + dz * dz;
            inside = d2 < r.R[k] * r.R[k];
        } else {
            double p = r.axis == 0 ? px : (r.axis == 1 ? py : pz);
            inside = fabs(p - r.centre[r.axis]) < r.R[k];
        }
        if (inside) lev = k + 1;
    }
    return lev;
}

__device__ int target_level(const DevCfg& dc, const DevRegions& rg, double px, double py,
                            double pz, int* which)
{
    int best = 0, w = -1;
    for (int j = 0; j < rg.n; ++j) {
        int l = region_level(rg.r[j], px, py, pz);
        if (l > best) {
            best = l;
            w = j;
        }
    }
    if (best > dc.lmax) best = dc.lmax;
    if (which) *which = w;
    return best;
}

// ------------------------------------------------------------------ split

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double split_uniform(unsigned long long seed, unsigned long long id,
                                                unsigned long long step)
{
    unsigned long long z = splitmix64(splitmix64(splitmix64(seed) ^ id) ^ step);
    return (double)(z >> 11) * 2.220446049250313e-16 - 1.0;
}

// unit vector tangential to the zone boundary at p, rotated about the normal
__device__ void split_direction(const DevRegion& r, double px, double py, double pz, double t,
                                double w[3])
{
    double v[3];
    if (r.shape == APR_SHAPE_SPHERE) {
        v[0] = px - r.centre[0];
        v[1] = py - r.centre[1];
        v[2] = pz - r.centre[2];
        double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (vn > 0.0) {
            v[0] = v[0] / vn;
            v[1] = v[1] / vn;
            v[2] = v[2] / vn;
        } else {
            v[0] = 1.0;
            v[1] = 0.0;
            v[2] = 0.0;
        }
    } else {
        v[0] = v[1] = v[2] = 0.0;
        double p = r.axis == 0 ? px : (r.axis == 1 ? py : pz);
        v[r.axis] = p - r.centre[r.axis] >= 0.0 ? 1.0 : -1.0;
    }
    int k = 0;
    for (int j = 1; j < 3; ++j)
        if (fabs(v[j]) < fabs(v[k])) k = j;
    double e[3] = {0.0, 0.0, 0.0};
    e[k] = 1.0;
    double w1[3] = {v[1] * e[2] - v[2] * e[1], v[2] * e[0] - v[0] * e[2], v[0] * e[1] - v[1] * e[0]};
    double n1 = sqrt(w1[0] * w1[0] + w1[1] * w1[1] + w1[2] * w1[2]);
    w1[0] = w1[0] / n1;
    w1[1] = w1[1] / n1;
    w1[2] = w1[2] / n1;
    double w2[3] = {v[1] * w1[2] - v[2] * w1[1], v[2] * w1[0] - v[0] * w1[2],
                    v[0] * w1[1] - v[1] * w1[0]};
    double den = 1.0 + t * t;
    double cs = (1.0 - t * t) / den;
    double sn = (2.0 * t) / den;
    for (int j = 0; j < 3; ++j) w[j] = cs * w1[j] + sn * w2[j];
}

__device__ __forceinline__ double wrap1(const DevCfg& dc, int k, double x)
{
    if (dc.periodic[k]) {
        if (x >= dc.hi[k]) x -= dc.L[k];
        else if (x < dc.lo[k]) x += dc.L[k];
    }
    return x;
}

__global__ void k_split_flag(DevCfg dc, DevRegions rg, long long n, int level,
                             const double* __restrict__ x, const double* __restrict__ y,
                             const double* __restrict__ z, const unsigned char* __restrict__ lev,
                             const unsigned char* __restrict__ flags, unsigned int* __restrict__ out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned f = 0;
    if (lev[i] == level && !(flags[i] & (APR_FLAG_CHANGED | APR_FLAG_FIXED | APR_FLAG_DEAD)))
        f = target_level(dc, rg, x[i], y[i], z[i], nullptr) > level ? 1u : 0u;
    out[i] = f;
}

__global__ void k_split_apply(DevCfg dc, DevRegions rg, long long n, int level,
                              unsigned long long step, long long next_id,
                              const unsigned int* __restrict__ flag,
                              const unsigned int* __restrict__ rank, apr_particles p)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    const long long j = n + rank[i];
    const double px = p.x[i], py = p.y[i], pz = p.z[i];
    int which;
    target_level(dc, rg, px, py, pz, &which);
    const double t = split_uniform(dc.seed, p.id[i], step);
    double w[3];
    split_direction(rg.r[which], px, py, pz, t, w);
    double rsep = dc.rsep_fac * p.h[i];
    double cap = dc.dnn_cap * p.dnn[i];
    if (cap < rsep) rsep = cap;
    // the new child: a copy of the parent
    p.vx[j] = p.vx[i];
    p.vy[j] = p.vy[i];
    p.vz[j] = p.vz[i];
    p.u[j] = p.u[i];
    p.rho[j] = p.rho[i];
    p.omega[j] = p.omega[i];
    p.ax[j] = p.ax[i];
    p.ay[j] = p.ay[i];
    p.az[j] = p.az[i];
    p.dudt[j] = p.dudt[i];
    p.vsig[j] = p.vsig[i];
    p.dnn[j] = p.dnn[i];
    p.pres[j] = p.pres[i];
    p.cs[j] = p.cs[i];
    p.x[i] = wrap1(dc, 0, px + rsep * w[0]);
    p.y[i] = wrap1(dc, 1, py + rsep * w[1]);
    p.z[i] = wrap1(dc, 2, pz + rsep * w[2]);
    p.x[j] = wrap1(dc, 0, px - rsep * w[0]);
    p.y[j] = wrap1(dc, 1, py - rsep * w[1]);
    p.z[j] = wrap1(dc, 2, pz - rsep * w[2]);
    const double hn = p.h[i] * SPLIT_HFAC;
    p.h[i] = hn;
    p.h[j] = hn;
    p.level[i] = (unsigned char)(level + 1);
    p.level[j] = (unsigned char)(level + 1);
    p.flags[i] = p.flags[i] | APR_FLAG_CHANGED;
    p.flags[j] = p.flags[i];
    p.id[j] = (unsigned long long)(next_id + (long long)rank[i]);
}

// ------------------------------------------------------------ merge tree

__global__ void k_merge_flag(long long n, int level, const unsigned char* __restrict__ lev,
                             const unsigned char* __restrict__ flags, unsigned int* __restrict__ out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = (lev[i] == level &&
              !(flags[i] & (APR_FLAG_CHANGED | APR_FLAG_FIXED | APR_FLAG_DEAD))) ? 1u : 0u;
}

__global__ void k_merge_collect(long long n, const unsigned int* __restrict__ flag,
                                const unsigned int* __restrict__ pos, unsigned int* __restrict__ set)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) set[pos[i]] = (unsigned)i;
}

__global__ void k_seg_init(int m, int* __restrict__ lo, int* __restrict__ hi, int4* acc_lo,
                           int4* acc_hi, unsigned long long* acc_sum, unsigned int* acc_k,
                           unsigned int* acc_k2, unsigned long long* acc_key,
                           unsigned long long* acc_key2)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    lo[p] = 0;
    hi[p] = m;
    if (p == 0) {
        acc_lo[0] = make_int4(INT_MAX, INT_MAX, INT_MAX, 0);
        acc_hi[0] = make_int4(INT_MIN, INT_MIN, INT_MIN, 0);
        acc_sum[0] = 0;
        acc_k[0] = 0;
        acc_k2[0] = 0;
        acc_key[0] = 0;
        acc_key2[0] = ~0ULL;
    }
}

// lanes of one warp that work on the same segment reduce before one atomic
__device__ __forceinline__ unsigned seg_peers(bool active, int seg)
{
    int key = active ? seg : -1 - (int)(threadIdx.x & 31);
    return __match_any_sync(0xffffffffu, key);
}

__device__ __forceinline__ bool seg_leader(unsigned peers)
{
    return (int)(threadIdx.x & 31) == __ffs(peers) - 1;
}

__global__ void k_tree_bbox(int m, const unsigned int* __restrict__ set, const int* __restrict__ lo,
                            const int* __restrict__ hi, const int4* __restrict__ xi, int4* acc_lo,
                            int4* acc_hi)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    bool act = false;
    int seg = 0;
    int4 q = make_int4(0, 0, 0, 0);
    if (p < m) {
        seg = lo[p];
        act = hi[p] - seg > 2;
        if (act) q = xi[set[p]];
    }
    unsigned peers = seg_peers(act, seg);
    if (!act) return;
    int mnx = __reduce_min_sync(peers, q.x), mny = __reduce_min_sync(peers, q.y),
        mnz = __reduce_min_sync(peers, q.z);
    int mxx = __reduce_max_sync(peers, q.x), mxy = __reduce_max_sync(peers, q.y),
        mxz = __reduce_max_sync(peers, q.z);
    if (seg_leader(peers)) {
        atomicMin(&acc_lo[seg].x, mnx);
        atomicMin(&acc_lo[seg].y, mny);
        atomicMin(&acc_lo[seg].z, mnz);
        atomicMax(&acc_hi[seg].x, mxx);
        atomicMax(&acc_hi[seg].y, mxy);
        atomicMax(&acc_hi[seg].z, mxz);
    }
}

__device__ __forceinline__ int seg_axis(const int4& a, const int4& b)
{
    int ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z;
    int ax = 0, e = ex;
    if (ey > e) {
        ax = 1;
        e = ey;
    }
    if (ez > e) ax = 2;
    return ax;
}

__device__ __forceinline__ int comp(const int4& q, int ax) { return ax == 0 ? q.x : (ax == 1 ? q.y : q.z); }

__global__ void k_tree_sum(int m, const unsigned int* __restrict__ set, const int* __restrict__ lo,
                           const int* __restrict__ hi, const int4* __restrict__ xi,
                           const int4* __restrict__ acc_lo, const int4* __restrict__ acc_hi,
                           unsigned long long* acc_sum)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    bool act = false;
    int seg = 0;
    unsigned v = 0;
    if (p < m) {
        seg = lo[p];
        act = hi[p] - seg > 2;
        if (act) v = (unsigned)comp(xi[set[p]], seg_axis(acc_lo[seg], acc_hi[seg]));
    }
    unsigned peers = seg_peers(act, seg);
    if (!act) return;
    unsigned s_hi = __reduce_add_sync(peers, v >> 15);
    unsigned s_lo = __reduce_add_sync(peers, v & 0x7fffu);
    if (seg_leader(peers))
        atomicAdd(&acc_sum[seg], ((unsigned long long)s_hi << 15) + (unsigned long long)s_lo);
}

__global__ void k_tree_count(int m, const unsigned int* __restrict__ set, const int* __restrict__ lo,
                             const int* __restrict__ hi, const int4* __restrict__ xi,
                             const int4* __restrict__ acc_lo, const int4* __restrict__ acc_hi,
                             const unsigned long long* __restrict__ acc_sum, unsigned int* acc_k,
                             unsigned int* acc_k2)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    bool act = false;
    int seg = 0;
    unsigned lt = 0, le = 0;
    if (p < m) {
        seg = lo[p];
        int size = hi[p] - seg;
        act = size > 2;
        if (act) {
            long long com = (long long)(acc_sum[seg] / (unsigned long long)size);
            long long v = comp(xi[set[p]], seg_axis(acc_lo[seg], acc_hi[seg]));
            lt = v < com;
            le = v <= com;
        }
    }
    unsigned peers = seg_peers(act, seg);
    if (!act) return;
    unsigned clt = __reduce_add_sync(peers, lt), cle = __reduce_add_sync(peers, le);
    if (seg_leader(peers)) {
        atomicAdd(&acc_k[seg], clt);
        atomicAdd(&acc_k2[seg], cle);
    }
}

// the cut of one segment: predicate (< or <=), count, and the final left count
struct Cut {
    bool use_le, coincident;
    int k, kfinal;
    long long com;
    int ax;
};

__device__ __forceinline__ Cut seg_cut(int seg, int size, const int4* acc_lo, const int4* acc_hi,
                                       const unsigned long long* acc_sum, const unsigned int* acc_k,
                                       const unsigned int* acc_k2)
{
    Cut c;
    c.ax = seg_axis(acc_lo[seg], acc_hi[seg]);
    c.com = (long long)(acc_sum[seg] / (unsigned long long)size);
    c.k = (int)acc_k[seg];
    c.use_le = false;
    if (c.k == 0) {
        c.k = (int)acc_k2[seg];
        c.use_le = true;
    }
    c.coincident = c.k == size;
    if (c.coincident) {
        c.kfinal = 2 * (size / 4);
    } else if (c.k % 2) {
        int a = c.k - 1, b = c.k + 1;
        int da = abs(2 * a - size), db = abs(2 * b - size);
        c.kfinal = (da <= db) ? a : b;
    } else {
        c.kfinal = c.k;
    }
    return c;
}

// for an odd cut: the largest (coordinate, index) on the low side moves up, or
// the smallest on the high side moves down
__global__ void k_tree_key(int m, const unsigned int* __restrict__ set, const int* __restrict__ lo,
                           const int* __restrict__ hi, const int4* __restrict__ xi,
                           const int4* __restrict__ acc_lo, const int4* __restrict__ acc_hi,
                           const unsigned long long* __restrict__ acc_sum,
                           const unsigned int* __restrict__ acc_k,
                           const unsigned int* __restrict__ acc_k2, unsigned long long* acc_key,
                           unsigned long long* acc_key2)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    int seg = lo[p], size = hi[p] - seg;
    if (size <= 2) return;
    Cut c = seg_cut(seg, size, acc_lo, acc_hi, acc_sum, acc_k, acc_k2);
    if (c.coincident || c.kfinal == c.k) return;
    unsigned idx = set[p];
    long long v = comp(xi[idx], c.ax);
    bool low = c.use_le ? v <= c.com : v < c.com;
    unsigned long long key = ((unsigned long long)v << 32) | idx;
    if (c.kfinal < c.k && low) atomicMax(&acc_key[seg], key);
    if (c.kfinal > c.k && !low) atomicMin(&acc_key2[seg], key);
}

__global__ void k_tree_flag(int m, const unsigned int* __restrict__ set, const int* __restrict__ lo,
                            const int* __restrict__ hi, const int4* __restrict__ xi,
                            const int4* __restrict__ acc_lo, const int4* __restrict__ acc_hi,
                            const unsigned long long* __restrict__ acc_sum,
                            const unsigned int* __restrict__ acc_k,
                            const unsigned int* __restrict__ acc_k2,
                            const unsigned long long* __restrict__ acc_key,
                            const unsigned long long* __restrict__ acc_key2,
                            unsigned int* __restrict__ lflag)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    int seg = lo[p], size = hi[p] - seg;
    if (size <= 2) {
        lflag[p] = 0;
        return;
    }
    Cut c = seg_cut(seg, size, acc_lo, acc_hi, acc_sum, acc_k, acc_k2);
    unsigned idx = set[p];
    bool left;
    if (c.coincident) {
        left = (p - seg) < c.kfinal;  // segments stay in ascending index order
    } else {
        long long v = comp(xi[idx], c.ax);
        left = c.use_le ? v <= c.com : v < c.com;
        unsigned long long key = ((unsigned long long)v << 32) | idx;
        if (c.kfinal < c.k && key == acc_key[seg]) left = false;
        if (c.kfinal > c.k && key == acc_key2[seg]) left = true;
    }
    lflag[p] = left ? 1u : 0u;
}

__global__ void k_tree_scatter(int m, const unsigned int* __restrict__ set,
                               const int* __restrict__ lo, const int* __restrict__ hi,
                               const int4* __restrict__ acc_lo, const int4* __restrict__ acc_hi,
                               const unsigned long long* __restrict__ acc_sum,
                               const unsigned int* __restrict__ acc_k,
                               const unsigned int* __restrict__ acc_k2,
                               const unsigned int* __restrict__ lflag,
                               const unsigned int* __restrict__ lscan, unsigned int* __restrict__ set2,
                               int* __restrict__ lo2, int* __restrict__ hi2, int4* acc_lo_n,
                               int4* acc_hi_n, unsigned long long* acc_sum_n,
                               unsigned int* acc_k_n, unsigned int* acc_k2_n,
                               unsigned long long* acc_key_n, unsigned long long* acc_key2_n,
                               int* maxseg)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    int seg = lo[p], end = hi[p], size = end - seg;
    int np = p, nlo = seg, nhi = end;
    if (size > 2) {
        Cut c = seg_cut(seg, size, acc_lo, acc_hi, acc_sum, acc_k, acc_k2);
        int before = (int)(lscan[p] - lscan[seg]);  // left items before p in this segment
        if (lflag[p]) {
            np = seg + before;
            nhi = seg + c.kfinal;
        } else {
            np = seg + c.kfinal + ((p - seg) - before);
            nlo = seg + c.kfinal;
        }
        atomicMax(maxseg, nhi - nlo);
    }
    set2[np] = set[p];
    lo2[np] = nlo;
    hi2[np] = nhi;
    if (np == nlo && nhi - nlo > 2) {
        acc_lo_n[np] = make_int4(INT_MAX, INT_MAX, INT_MAX, 0);
        acc_hi_n[np] = make_int4(INT_MIN, INT_MIN, INT_MIN, 0);
        acc_sum_n[np] = 0;
        acc_k_n[np] = 0;
        acc_k2_n[np] = 0;
        acc_key_n[np] = 0;
        acc_key2_n[np] = ~0ULL;
    }
}

// pairs the merge candidates of one level; returns the count m (even) and the
// spare index; on return W.mset[*cur] holds the pairs at (2j, 2j+1)
static apr_status pair_tree(apr_ctx* c, int level, int* m_out, long long* spare, int* cur_out)
{
    Workspace& W = c->W;
    cudaStream_t st = c->stream;
    const long long n = c->n;
    APR_LAUNCH(c, k_merge_flag, nblocks(n, 256), 256, n, level, c->p.level, c->p.flags, W.uflag);
    scan_u32(c, W.uflag, W.uscan, n, (unsigned*)&W.status[ST_COUNT_A]);
    APR_LAUNCH(c, k_merge_collect, nblocks(n, 256), 256, n, W.uflag, W.uscan, W.mset[0]);
    cudaMemcpyAsync(c->hbuf, &W.status[ST_COUNT_A], sizeof(int), cudaMemcpyDeviceToHost, st);
    apr_status s = cuda_check(c, cudaStreamSynchronize(st), "merge candidates");
    if (s != APR_OK) return s;
    int m = ((int*)c->hbuf)[0];
    *spare = -1;
    if (m % 2) {
        cudaMemcpyAsync(c->hbuf, W.mset[0] + (m - 1), sizeof(unsigned), cudaMemcpyDeviceToHost,
                        st);
        s = cuda_check(c, cudaStreamSynchronize(st), "spare");
        if (s != APR_OK) return s;
        *spare = ((unsigned*)c->hbuf)[0];
        --m;
    }
    *m_out = m;
    *cur_out = 0;
    if (m <= 2) return APR_OK;
    // accumulators live in two banks indexed by segment start
    unsigned long long* key2[2] = {W.acc_key + c->cap, W.acc_key + 2 * c->cap};
    int4* alo[2] = {W.acc_lo, W.acc_lo + c->cap};
    int4* ahi[2] = {W.acc_hi, W.acc_hi + c->cap};
    unsigned long long* asum[2] = {W.acc_sum, W.acc_sum + c->cap};
    unsigned int* ak[2] = {W.acc_k, W.acc_k + c->cap};
    unsigned int* ak2[2] = {W.acc_k2, W.acc_k2 + c->cap};
    unsigned long long* akey[2] = {W.acc_key, W.acc_key + 3 * c->cap};
    APR_LAUNCH(c, k_seg_init, nblocks(m, 256), 256, m, W.seg_lo[0], W.seg_hi[0], alo[0], ahi[0], asum[0],
                                               ak[0], ak2[0], akey[0], key2[0]);
    int cur = 0;
    const int nb = nblocks(m, 256);
    for (int round = 0; round < 4 * m + 64; ++round) {
        APR_LAUNCH(c, k_tree_bbox, nb, 256, m, W.mset[cur], W.seg_lo[cur], W.seg_hi[cur], W.xi,
                                        alo[cur], ahi[cur]);
        APR_LAUNCH(c, k_tree_sum, nb, 256, m, W.mset[cur], W.seg_lo[cur], W.seg_hi[cur], W.xi, alo[cur],
                                       ahi[cur], asum[cur]);
        APR_LAUNCH(c, k_tree_count, nb, 256, m, W.mset[cur], W.seg_lo[cur], W.seg_hi[cur], W.xi,
                                         alo[cur], ahi[cur], asum[cur], ak[cur], ak2[cur]);
        APR_LAUNCH(c, k_tree_key, nb, 256, m, W.mset[cur], W.seg_lo[cur], W.seg_hi[cur], W.xi, alo[cur],
                                       ahi[cur], asum[cur], ak[cur], ak2[cur], akey[cur], key2[cur]);
        APR_LAUNCH(c, k_tree_flag, nb, 256, m, W.mset[cur], W.seg_lo[cur], W.seg_hi[cur], W.xi,
                                        alo[cur], ahi[cur], asum[cur], ak[cur], ak2[cur], akey[cur],
                                        key2[cur], W.lflag);
        scan_u32(c, W.lflag, W.uscan, m, nullptr);
        cudaMemsetAsync(&W.status[ST_MAXSEG], 0, sizeof(int), st);
        const int nx = cur ^ 1;
        APR_LAUNCH(c, k_tree_scatter, nb, 256, m, W.mset[cur], W.seg_lo[cur], W.seg_hi[cur], alo[cur],
                                           ahi[cur], asum[cur], ak[cur], ak2[cur], W.lflag, W.uscan,
                                           W.mset[nx], W.seg_lo[nx], W.seg_hi[nx], alo[nx], ahi[nx],
                                           asum[nx], ak[nx], ak2[nx], akey[nx], key2[nx],
                                           &W.status[ST_MAXSEG]);
        cur = nx;
        cudaMemcpyAsync(c->hbuf, &W.status[ST_MAXSEG], sizeof(int), cudaMemcpyDeviceToHost, st);
        s = cuda_check(c, cudaStreamSynchronize(st), "pairing tree");
        if (s != APR_OK) return s;
        if (((int*)c->hbuf)[0] <= 2) break;
    }
    *cur_out = cur;
    return APR_OK;
}

__global__ void k_merge_apply(DevCfg dc, DevRegions rg, int npairs, int level,
                              const unsigned int* __restrict__ set, apr_particles p,
                              int* __restrict__ count)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= npairs) return;
    unsigned a = set[2 * j], b = set[2 * j + 1];
    if (b < a) {
        unsigned t = a;
        a = b;
        b = t;
    }
    double pa[3] = {p.x[a], p.y[a], p.z[a]}, pb[3] = {p.x[b], p.y[b], p.z[b]};
    double com[3];
    for (int k = 0; k < 3; ++k) {
        double d = pb[k] - pa[k];
        if (dc.periodic[k]) {
            if (d > 0.5 * dc.L[k]) d -= dc.L[k];
            else if (d < -0.5 * dc.L[k]) d += dc.L[k];
        }
        com[k] = wrap1(dc, k, pa[k] + 0.5 * d);
    }
    if (target_level(dc, rg, com[0], com[1], com[2], nullptr) >= level) return;
    p.x[a] = com[0];
    p.y[a] = com[1];
    p.z[a] = com[2];
    p.vx[a] = 0.5 * (p.vx[a] + p.vx[b]);
    p.vy[a] = 0.5 * (p.vy[a] + p.vy[b]);
    p.vz[a] = 0.5 * (p.vz[a] + p.vz[b]);
    p.u[a] = 0.5 * (p.u[a] + p.u[b]);
    p.h[a] = p.h[a] * MERGE_HFAC;
    p.level[a] = (unsigned char)(level - 1);
    p.flags[a] = p.flags[a] | APR_FLAG_CHANGED;
    p.flags[b] = p.flags[b] | APR_FLAG_DEAD;
    atomicAdd(count, 1);
}

__global__ void k_pairs_out(int npairs, const unsigned int* __restrict__ set,
                            long long* __restrict__ out)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < 2 * npairs) out[j] = set[j];
}

apr_status merge_pairs_debug(apr_ctx* c, int level, long long* pairs, long long cap,
                             long long* npairs, long long* spare)
{
    apr_status s = quantise(c);
    if (s != APR_OK) return s;
    int m, cur;
    s = pair_tree(c, level, &m, spare, &cur);
    if (s != APR_OK) return s;
    *npairs = m / 2;
    if (m / 2 > cap) return fail(c, APR_ERR_ARG, "merge_pairs: cap too small");
    if (m == 0) return APR_OK;
    long long* dev = (long long*)c->W.tmp8;
    APR_LAUNCH(c, k_pairs_out, nblocks(m, 256), 256, m / 2, c->W.mset[cur], dev);
    s = cuda_check(c, cudaMemcpyAsync(pairs, dev, sizeof(long long) * m, cudaMemcpyDeviceToHost,
                                      c->stream), "pairs out");
    if (s != APR_OK) return s;
    return cuda_check(c, cudaStreamSynchronize(c->stream), "pairs out");
}

// ------------------------------------------------------------ compaction

template <typename T>
__global__ void k_compact_field(long long n, const unsigned char* __restrict__ flags,
                                const unsigned int* __restrict__ pos, const T* __restrict__ in,
                                T* __restrict__ out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(flags[i] & APR_FLAG_DEAD)) out[pos[i]] = in[i];
}

__global__ void k_live_flag(long long n, const unsigned char* __restrict__ flags,
                            unsigned int* __restrict__ out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (flags[i] & APR_FLAG_DEAD) ? 0u : 1u;
}

template <typename T>
static void compact_one(apr_ctx* c, T* field, long long n, long long nlive)
{
    T* tmp = (T*)c->W.tmp8;
    APR_LAUNCH(c, k_compact_field<T>, nblocks(n, 256), 256, n, c->p.flags, c->W.uscan, field, tmp);
    cudaMemcpyAsync(field, tmp, sizeof(T) * (size_t)nlive, cudaMemcpyDeviceToDevice, c->stream);
}

apr_status compact(apr_ctx* c, long long* removed)
{
    const long long n = c->n;
    Workspace& W = c->W;
    APR_LAUNCH(c, k_live_flag, nblocks(n, 256), 256, n, c->p.flags, W.uflag);
    scan_u32(c, W.uflag, W.uscan, n, (unsigned*)&W.status[ST_COUNT_B]);
    cudaMemcpyAsync(c->hbuf, &W.status[ST_COUNT_B], sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    apr_status s = cuda_check(c, cudaStreamSynchronize(c->stream), "compaction count");
    if (s != APR_OK) return s;
    long long nlive = (unsigned)((int*)c->hbuf)[0];
    *removed = n - nlive;
    if (nlive == n) return APR_OK;
    apr_particles& p = c->p;
    double* d[] = {p.x, p.y, p.z, p.vx, p.vy, p.vz, p.u, p.h, p.rho, p.omega,
                   p.ax, p.ay, p.az, p.dudt, p.vsig, p.dnn, p.pres, p.cs};
    for (double* f : d) compact_one<double>(c, f, n, nlive);
    compact_one<unsigned long long>(c, p.id, n, nlive);
    compact_one<unsigned char>(c, p.level, n, nlive);
    compact_one<unsigned char>(c, p.flags, n, nlive);  // last: the others read the flags
    c->n = nlive;
    return cuda_check(c, cudaGetLastError(), "compaction");
}

// ------------------------------------------------------- split/merge pass

__global__ void k_clear_changed(long long n, unsigned char* flags)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = flags[i] & (unsigned char)~APR_FLAG_CHANGED;
}

apr_status clear_changed(apr_ctx* c)
{
    if (c->n > 0) APR_LAUNCH(c, k_clear_changed, nblocks(c->n, 256), 256, c->n, c->p.flags);
    return cuda_check(c, cudaGetLastError(), "clear changed");
}

static apr_status split_merge_body(apr_ctx* c, apr_counts* cnt);

apr_status split_merge_pass(apr_ctx* c, apr_counts* cnt)
{
    const int ps = prof_begin(c, APR_PROF_REFINE);
    apr_status s = split_merge_body(c, cnt);
    prof_end(c, ps);
    return s;
}

static apr_status split_merge_body(apr_ctx* c, apr_counts* cnt)
{
    Workspace& W = c->W;
    cudaStream_t st = c->stream;
    const DevRegions rg = dev_regions(c);
    memset(cnt, 0, sizeof(*cnt));
    apr_status s;
    if (c->n > 0) APR_LAUNCH(c, k_clear_changed, nblocks(c->n, 256), 256, c->n, c->p.flags);
    for (int l = 0; l < c->cfg.lmax; ++l) {
        const long long n = c->n;
        if (n == 0) break;
        APR_LAUNCH(c, k_split_flag, nblocks(n, 256), 256, c->dc, rg, n, l, c->p.x, c->p.y, c->p.z,
                                                      c->p.level, c->p.flags, W.uflag);
        scan_u32(c, W.uflag, W.uscan, n, (unsigned*)&W.status[ST_COUNT_A]);
        cudaMemcpyAsync(c->hbuf, &W.status[ST_COUNT_A], sizeof(int), cudaMemcpyDeviceToHost, st);
        s = cuda_check(c, cudaStreamSynchronize(st), "split count");
        if (s != APR_OK) return s;
        long long ns = (unsigned)((int*)c->hbuf)[0];
        if (n + ns > c->cap)
            return fail(c, APR_ERR_CAPACITY, "split would exceed the bound capacity");
        if (ns > 0) {
            APR_LAUNCH(c, k_split_apply, nblocks(n, 256), 256, c->dc, rg, n, l, c->step, c->next_id,
                                                           W.uflag, W.uscan, c->p);
            c->n = n + ns;
            c->next_id += ns;
        }
        cnt->n_split[l] = ns;
    }
    bool any_merge = false;
    if (c->cfg.lmax >= 1 && c->n > 0) {
        s = quantise(c);
        if (s != APR_OK) return s;
    }
    for (int l = c->cfg.lmax; l >= 1; --l) {
        if (c->n == 0) break;
        int m, cur;
        long long spare;
        s = pair_tree(c, l, &m, &spare, &cur);
        if (s != APR_OK) return s;
        cnt->n_spare[l] = spare >= 0 ? 1 : 0;
        if (m < 2) continue;
        cudaMemsetAsync(&W.status[ST_COUNT_B], 0, sizeof(int), st);
        APR_LAUNCH(c, k_merge_apply, nblocks(m / 2, 256), 256, c->dc, rg, m / 2, l, W.mset[cur], c->p,
                                                         &W.status[ST_COUNT_B]);
        cudaMemcpyAsync(c->hbuf, &W.status[ST_COUNT_B], sizeof(int), cudaMemcpyDeviceToHost, st);
        s = cuda_check(c, cudaStreamSynchronize(st), "merge");
        if (s != APR_OK) return s;
        cnt->n_merge[l] = ((int*)c->hbuf)[0];
        if (cnt->n_merge[l]) any_merge = true;
    }
    (void)any_merge;
    long long removed = 0;
    if (c->n > 0) {
        s = compact(c, &removed);
        if (s != APR_OK) return s;
    }
    cnt->n_dead = removed;
    c->step += 1;
    return APR_OK;
}

// ------------------------------------------------------------- reductions

// fixed-shape block reduction of NV doubles; partials[block * 32 + v]
template <int NV>
__device__ void block_reduce_store(double (&v)[NV], double* partials)
{
    __shared__ double sm[NV][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sm[k][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double x = 0.0;
        for (int w = 0; w < 8; ++w) x += sm[threadIdx.x][w];
        partials[blockIdx.x * 32 + threadIdx.x] = x;
    }
}

__global__ void k_reduce_final(int nblk, int nv, const double* __restrict__ partials,
                               double* __restrict__ out, int op_min)
{
    int k = threadIdx.x;
    if (k >= nv) return;
    double x = op_min ? INFINITY : 0.0;
    for (int b = 0; b < nblk; ++b) {
        double y = partials[b * 32 + k];
        x = op_min ? fmin(x, y) : x + y;
    }
    out[k] = x;
}

static apr_status reduce_readback(apr_ctx* c, int nv, int op_min, double* host)
{
    APR_LAUNCH(c, k_reduce_final, 1, 32, RED_BLOCKS, nv, c->W.red, c->W.redout, op_min);
    cudaMemcpyAsync(c->hbuf, c->W.redout, sizeof(double) * nv, cudaMemcpyDeviceToHost, c->stream);
    apr_status s = cuda_check(c, cudaStreamSynchronize(c->stream), "reduce");
    if (s != APR_OK) return s;
    memcpy(host, c->hbuf, sizeof(double) * nv);
    return APR_OK;
}

__global__ void __launch_bounds__(256) k_stats(DevCfg dc, long long n, apr_particles p,
                                               double* partials)
{
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (p.flags[i] & APR_FLAG_DEAD) continue;
        double m = dc.m0 * level_mass_d(p.level[i]);
        double vx = p.vx[i], vy = p.vy[i], vz = p.vz[i];
        v[0] += m;
        v[1] += m * vx;
        v[2] += m * vy;
        v[3] += m * vz;
        v[4] += m * (p.y[i] * vz - p.z[i] * vy);
        v[5] += m * (p.z[i] * vx - p.x[i] * vz);
        v[6] += m * (p.x[i] * vy - p.y[i] * vx);
        v[7] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        if (dc.eos == APR_EOS_ADIABATIC) v[8] += m * p.u[i];
    }
    block_reduce_store<9>(v, partials);
}

apr_status compute_stats(apr_ctx* c, apr_stats* st)
{
    APR_LAUNCH(c, k_stats, RED_BLOCKS, 256, c->dc, c->n, c->p, c->W.red);
    double r[9];
    apr_status s = reduce_readback(c, 9, 0, r);
    if (s != APR_OK) return s;
    st->mass = r[0];
    for (int k = 0; k < 3; ++k) {
        st->mom[k] = r[1 + k];
        st->ang[k] = r[4 + k];
    }
    st->ekin = r[7];
    st->etherm = r[8];
    for (int j = 0; j < c->nsink; ++j) {
        const apr_sink& k = c->sinks[j];
        double m = k.m;
        st->mass += m;
        for (int d = 0; d < 3; ++d) st->mom[d] += m * k.v[d];
        st->ang[0] += m * (k.x[1] * k.v[2] - k.x[2] * k.v[1]);
        st->ang[1] += m * (k.x[2] * k.v[0] - k.x[0] * k.v[2]);
        st->ang[2] += m * (k.x[0] * k.v[1] - k.x[1] * k.v[0]);
        st->ekin += 0.5 * m * (k.v[0] * k.v[0] + k.v[1] * k.v[1] + k.v[2] * k.v[2]);
    }
    return APR_OK;
}

__global__ void __launch_bounds__(256) k_timestep(DevCfg dc, long long n, apr_particles p,
                                                  double* partials)
{
    double dt = INFINITY;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (p.flags[i] & (APR_FLAG_DEAD | APR_FLAG_FIXED)) continue;
        double h = p.h[i];
        if (p.vsig[i] > 0.0) dt = fmin(dt, dc.ccour * h / p.vsig[i]);
        double a = sqrt(p.ax[i] * p.ax[i] + p.ay[i] * p.ay[i] + p.az[i] * p.az[i]);
        if (a > 0.0) dt = fmin(dt, dc.cforce * sqrt(h / a));
    }
    __shared__ double sm[8];
    for (int o = 16; o > 0; o >>= 1) dt = fmin(dt, __shfl_down_sync(0xffffffffu, dt, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = dt;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = sm[0];
        for (int w = 1; w < 8; ++w) x = fmin(x, sm[w]);
        partials[blockIdx.x * 32] = x;
    }
}

apr_status compute_timestep(apr_ctx* c, double* dt)
{
    APR_LAUNCH(c, k_timestep, RED_BLOCKS, 256, c->dc, c->n, c->p, c->W.red);
    return reduce_readback(c, 1, 1, dt);
}

// ------------------------------------------------------- point masses

__global__ void __launch_bounds__(256) k_sink_gravity(DevCfg dc, DevSinks sk, long long n,
                                                      apr_particles p, double* partials)
{
    double v[3 * APR_MAXSINK];
    for (int k = 0; k < 3 * APR_MAXSINK; ++k) v[k] = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (p.flags[i] & APR_FLAG_DEAD) continue;
        const double mi = dc.m0 * level_mass_d(p.level[i]);
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int j = 0; j < sk.n; ++j) {
            double dx = p.x[i] - sk.x[j][0], dy = p.y[i] - sk.x[j][1], dz = p.z[i] - sk.x[j][2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double r = sqrt(r2);
            double f = dc.G / (r2 * r);
            ax -= f * sk.m[j] * dx;
            ay -= f * sk.m[j] * dy;
            az -= f * sk.m[j] * dz;
            v[3 * j + 0] += f * mi * dx;
            v[3 * j + 1] += f * mi * dy;
            v[3 * j + 2] += f * mi * dz;
        }
        p.ax[i] += ax;
        p.ay[i] += ay;
        p.az[i] += az;
    }
    block_reduce_store<3 * APR_MAXSINK>(v, partials);
}

apr_status sink_gravity(apr_ctx* c)
{
    if (c->nsink == 0) return APR_OK;
    APR_LAUNCH(c, k_sink_gravity, RED_BLOCKS, 256, c->dc, dev_sinks(c), c->n, c->p, c->W.red);
    double r[3 * APR_MAXSINK];
    apr_status s = reduce_readback(c, 3 * c->nsink, 0, r);
    if (s != APR_OK) return s;
    for (int j = 0; j < c->nsink; ++j) {
        apr_sink& k = c->sinks[j];
        for (int d = 0; d < 3; ++d) k.a[d] = r[3 * j + d];
    }
    for (int j = 0; j < c->nsink; ++j)
        for (int l = 0; l < c->nsink; ++l) {
            if (l == j) continue;
            apr_sink& a = c->sinks[j];
            const apr_sink& b = c->sinks[l];
            double dx = a.x[0] - b.x[0], dy = a.x[1] - b.x[1], dz = a.x[2] - b.x[2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double rr = sqrt(r2);
            double f = c->cfg.G * b.m / (r2 * rr);
            a.a[0] -= f * dx;
            a.a[1] -= f * dy;
            a.a[2] -= f * dz;
        }
    return APR_OK;
}

__global__ void __launch_bounds__(256) k_accrete(DevCfg dc, DevSinks sk, long long n,
                                                 apr_particles p, double* partials, int* count)
{
    double v[7 * APR_MAXSINK];
    for (int k = 0; k < 7 * APR_MAXSINK; ++k) v[k] = 0.0;
    int cnt = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (p.flags[i] & (APR_FLAG_DEAD | APR_FLAG_FIXED)) continue;
        for (int j = 0; j < sk.n; ++j) {
            double dx = p.x[i] - sk.x[j][0], dy = p.y[i] - sk.x[j][1], dz = p.z[i] - sk.x[j][2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < sk.racc[j] * sk.racc[j])) continue;
            double mi = dc.m0 * level_mass_d(p.level[i]);
            v[7 * j + 0] += mi;
            v[7 * j + 1] += mi * p.vx[i];
            v[7 * j + 2] += mi * p.vy[i];
            v[7 * j + 3] += mi * p.vz[i];
            v[7 * j + 4] += mi * p.x[i];
            v[7 * j + 5] += mi * p.y[i];
            v[7 * j + 6] += mi * p.z[i];
            p.flags[i] = p.flags[i] | APR_FLAG_DEAD;
            ++cnt;
            break;
        }
    }
    if (cnt) atomicAdd(count, cnt);
    // 7 per sink, at most 4 sinks per reduction slot set of 32
    block_reduce_store<28>(*reinterpret_cast<double(*)[28]>(v), partials);
}

apr_status accrete(apr_ctx* c, long long* naccreted)
{
    *naccreted = 0;
    if (c->nsink == 0 || c->n == 0) return APR_OK;
    if (c->nsink > 4) return fail(c, APR_ERR_ARG, "accretion supports at most 4 sinks");
    cudaMemsetAsync(&c->W.status[ST_COUNT_B], 0, sizeof(int), c->stream);
    APR_LAUNCH(c, k_accrete, RED_BLOCKS, 256, c->dc, dev_sinks(c), c->n, c->p, c->W.red,
                                                 &c->W.status[ST_COUNT_B]);
    double r[28];
    apr_status s = reduce_readback(c, 7 * c->nsink, 0, r);
    if (s != APR_OK) return s;
    cudaMemcpyAsync(c->hbuf, &c->W.status[ST_COUNT_B], sizeof(int), cudaMemcpyDeviceToHost,
                    c->stream);
    s = cuda_check(c, cudaStreamSynchronize(c->stream), "accrete");
    if (s != APR_OK) return s;
    *naccreted = ((int*)c->hbuf)[0];
    for (int j = 0; j < c->nsink; ++j) {
        double M = r[7 * j];
        if (!(M > 0.0)) continue;
        apr_sink& k = c->sinks[j];
        double mt = k.m + M;
        for (int d = 0; d < 3; ++d) {
            k.v[d] = (k.m * k.v[d] + r[7 * j + 1 + d]) / mt;
            k.x[d] = (k.m * k.x[d] + r[7 * j + 4 + d]) / mt;
        }
        k.m = mt;
    }
    return APR_OK;
}

// ------------------------------------------------------------ integration

__global__ void k_kick(DevCfg dc, long long n, double hdt, apr_particles p)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (p.flags[i] & (APR_FLAG_FIXED | APR_FLAG_DEAD))) return;
    p.vx[i] += hdt * p.ax[i];
    p.vy[i] += hdt * p.ay[i];
    p.vz[i] += hdt * p.az[i];
    if (dc.eos == APR_EOS_ADIABATIC) p.u[i] += hdt * p.dudt[i];
}

__global__ void k_drift(DevCfg dc, long long n, double dt, apr_particles p)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (p.flags[i] & (APR_FLAG_FIXED | APR_FLAG_DEAD))) return;
    p.x[i] = wrap1(dc, 0, p.x[i] + dt * p.vx[i]);
    p.y[i] = wrap1(dc, 1, p.y[i] + dt * p.vy[i]);
    p.z[i] = wrap1(dc, 2, p.z[i] + dt * p.vz[i]);
}

apr_status kick(apr_ctx* c, double hdt)
{
    if (c->n > 0) APR_LAUNCH(c, k_kick, nblocks(c->n, 256), 256, c->dc, c->n, hdt, c->p);
    for (int j = 0; j < c->nsink; ++j)
        for (int d = 0; d < 3; ++d) c->sinks[j].v[d] += hdt * c->sinks[j].a[d];
    return cuda_check(c, cudaGetLastError(), "kick");
}

apr_status drift(apr_ctx* c, double dt)
{
    if (c->n > 0) APR_LAUNCH(c, k_drift, nblocks(c->n, 256), 256, c->dc, c->n, dt, c->p);
    for (int j = 0; j < c->nsink; ++j)
        for (int d = 0; d < 3; ++d) c->sinks[j].x[d] += dt * c->sinks[j].v[d];
    return cuda_check(c, cudaGetLastError(), "drift");
}

}  // namespace apr

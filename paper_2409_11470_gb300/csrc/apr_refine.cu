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
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cstring>
#include <vector>

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

// split parents of every level: key = level for a parent, 255 otherwise.  A stable
// sort by this key ranks the parents by (level, index), which is the order in
// which level-by-level passes (lowest level first) append the new children.
__global__ void k_split_keys(DevCfg dc, DevRegions rg, long long n, const double* __restrict__ x,
                             const double* __restrict__ y, const double* __restrict__ z,
                             const unsigned char* __restrict__ lev,
                             const unsigned char* __restrict__ flags,
                             unsigned long long* __restrict__ key, unsigned int* __restrict__ val)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = lev[i];
    bool split = false;
    if (l < dc.lmax && !(flags[i] & (APR_FLAG_CHANGED | APR_FLAG_FIXED | APR_FLAG_DEAD)))
        split = target_level(dc, rg, x[i], y[i], z[i], nullptr) > l;
    key[i] = split ? (unsigned long long)l : 255ULL;
    val[i] = (unsigned)i;
}

__global__ void k_split_rank(int total, const unsigned int* __restrict__ sorted,
                             unsigned int* __restrict__ rank)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < total) rank[sorted[r]] = (unsigned)r;
}

__global__ void k_split_apply(DevCfg dc, DevRegions rg, int total, long long n,
                              unsigned long long step, long long next_id,
                              const unsigned int* __restrict__ sorted, apr_particles p)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= total) return;
    const unsigned i = sorted[r];
    const long long j = n + r;
    const int level = p.level[i];
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
    p.id[j] = (unsigned long long)(next_id + (long long)r);
}

// ------------------------------------------------------------ merge tree
//
// The candidates of every level are paired at once (their trees are
// independent): one stable radix pass groups them by level in ascending
// index order; global level-synchronous rounds cut every segment larger than
// TREE_LOCAL; then one CTA per chunk finishes its segments in shared memory.

constexpr int TREE_LOCAL = 512;      // largest segment left to the shared-memory phase
constexpr int TREE_LOC_CAP = 1024;   // positions one CTA can hold (< 2 * TREE_LOCAL)
constexpr int TREE_LOC_THREADS = 256;

struct LevelOffsets {
    int off[APR_MAXLEV + 2];  // candidates of level l occupy [off[l], off[l+1])
    int lmax;
};

__global__ void k_merge_keys(long long n, const unsigned char* __restrict__ lev,
                             const unsigned char* __restrict__ flags,
                             unsigned long long* __restrict__ key, unsigned int* __restrict__ val)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = lev[i];
    const bool cand = l >= 1 && !(flags[i] & (APR_FLAG_CHANGED | APR_FLAG_FIXED | APR_FLAG_DEAD));
    key[i] = cand ? (unsigned long long)l : 255ULL;
    val[i] = (unsigned)i;
}


// one segment per level (even count); an odd level's last candidate is the spare
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

__device__ __forceinline__ int axis_of(int ex, int ey, int ez)
{
    int ax = 0, e = ex;
    if (ey > e) {
        ax = 1;
        e = ey;
    }
    if (ez > e) ax = 2;
    return ax;
}

__device__ __forceinline__ int seg_axis(const int4& a, const int4& b)
{
    return axis_of(b.x - a.x, b.y - a.y, b.z - a.z);
}

__device__ __forceinline__ int comp(const int4& q, int ax) { return ax == 0 ? q.x : (ax == 1 ? q.y : q.z); }

// the cut of one segment from its count below the centre of mass (Sec. 2.3 reading):
// k = #{x < com}; if 0, #{x <= com}; all coincident: 2 floor(n/4) by index; odd: k+-1
struct Cut {
    bool use_le, coincident;
    int k, kfinal;
};

__device__ __forceinline__ Cut make_cut(int size, int k_lt, int k_le)
{
    Cut c;
    c.k = k_lt;
    c.use_le = false;
    if (c.k == 0) {
        c.k = k_le;
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

// ---- global rounds: segments larger than `thresh`
//
// Per segment (indexed by its first slot): bounding box, coordinate sums on all
// three axes, counts below the centre of mass for < and <=, and the four keys an
// odd cut could move (largest (x, index) below / smallest above, for both tests).

struct SegAcc {
    int4* lo;                    // bbox min (x, y, z)
    int4* hi;                    // bbox max
    unsigned long long* sum;     // 3 per segment: sum[3 * s + axis]
    unsigned int* k;             // count x < com
    unsigned int* k2;            // count x <= com
    unsigned long long* key;     // 4 per segment: max low(<), min high(>=), max low(<=), min high(>)
};

__device__ __forceinline__ void acc_reset_all(const SegAcc& A, int s)
{
    A.lo[s] = make_int4(INT_MAX, INT_MAX, INT_MAX, 0);
    A.hi[s] = make_int4(INT_MIN, INT_MIN, INT_MIN, 0);
    A.sum[3 * s] = A.sum[3 * s + 1] = A.sum[3 * s + 2] = 0;
    A.k[s] = 0;
    A.k2[s] = 0;
    A.key[4 * s + 0] = 0;
    A.key[4 * s + 1] = ~0ULL;
    A.key[4 * s + 2] = 0;
    A.key[4 * s + 3] = ~0ULL;
}

__device__ __forceinline__ void warp_sum_u64(unsigned peers, unsigned v, bool leader,
                                             unsigned long long* dst)
{
    unsigned sh = __reduce_add_sync(peers, v >> 15), sl = __reduce_add_sync(peers, v & 0x7fffu);
    if (leader) atomicAdd(dst, ((unsigned long long)sh << 15) + (unsigned long long)sl);
}

__global__ void k_seg_setup(int M, LevelOffsets lo_off, int* __restrict__ lo, int* __restrict__ hi,
                            SegAcc A)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    int l = 1;
    while (l < lo_off.lmax && p >= lo_off.off[l + 1]) ++l;
    const int a = lo_off.off[l], m = lo_off.off[l + 1] - a, be = a + (m & ~1);
    if (p < be) {
        lo[p] = a;
        hi[p] = be;
    } else {
        lo[p] = p;
        hi[p] = p + 1;
    }
    if (p == a && be - a > TREE_LOCAL) acc_reset_all(A, a);
}

__global__ void k_tree_bbox_sum(int m, int thresh, const unsigned int* __restrict__ set,
                                const int* __restrict__ lo, const int* __restrict__ hi,
                                const int4* __restrict__ xi, SegAcc A)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    bool act = false;
    int seg = 0;
    int4 q = make_int4(0, 0, 0, 0);
    if (p < m) {
        seg = lo[p];
        act = hi[p] - seg > thresh;
        if (act) q = xi[set[p]];
    }
    unsigned peers = seg_peers(act, seg);
    if (!act) return;
    const bool lead = seg_leader(peers);
    int mnx = __reduce_min_sync(peers, q.x), mny = __reduce_min_sync(peers, q.y),
        mnz = __reduce_min_sync(peers, q.z);
    int mxx = __reduce_max_sync(peers, q.x), mxy = __reduce_max_sync(peers, q.y),
        mxz = __reduce_max_sync(peers, q.z);
    if (lead) {
        atomicMin(&A.lo[seg].x, mnx);
        atomicMin(&A.lo[seg].y, mny);
        atomicMin(&A.lo[seg].z, mnz);
        atomicMax(&A.hi[seg].x, mxx);
        atomicMax(&A.hi[seg].y, mxy);
        atomicMax(&A.hi[seg].z, mxz);
    }
    warp_sum_u64(peers, (unsigned)q.x, lead, &A.sum[3 * seg + 0]);
    warp_sum_u64(peers, (unsigned)q.y, lead, &A.sum[3 * seg + 1]);
    warp_sum_u64(peers, (unsigned)q.z, lead, &A.sum[3 * seg + 2]);
}

// largest (v, idx) over the lanes in `peers` that have pred; 0 if none
__device__ __forceinline__ unsigned long long warp_max_key(unsigned peers, bool pred, int v,
                                                           unsigned idx)
{
    int vm = __reduce_max_sync(peers, pred ? v : -1);
    unsigned im = __reduce_max_sync(peers, (pred && v == vm) ? idx : 0u);
    return vm < 0 ? 0ULL : (((unsigned long long)vm << 32) | im);
}

// smallest (v, idx) over the lanes in `peers` that have pred; ~0 if none
__device__ __forceinline__ unsigned long long warp_min_key(unsigned peers, bool pred, int v,
                                                           unsigned idx)
{
    int vm = __reduce_min_sync(peers, pred ? v : INT_MAX);
    unsigned im = __reduce_min_sync(peers, (pred && v == vm) ? idx : 0xffffffffu);
    return vm == INT_MAX ? ~0ULL : (((unsigned long long)vm << 32) | im);
}

__device__ __forceinline__ long long seg_com(const SegAcc& A, int seg, int size, int ax)
{
    return (long long)(A.sum[3 * seg + ax] / (unsigned long long)size);
}

__global__ void k_tree_count_key(int m, int thresh, const unsigned int* __restrict__ set,
                                 const int* __restrict__ lo, const int* __restrict__ hi,
                                 const int4* __restrict__ xi, SegAcc A)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    bool act = false;
    int seg = 0, v = 0;
    unsigned idx = 0;
    bool lt = false, le = false;
    if (p < m) {
        seg = lo[p];
        int size = hi[p] - seg;
        act = size > thresh;
        if (act) {
            const int ax = seg_axis(A.lo[seg], A.hi[seg]);
            const long long com = seg_com(A, seg, size, ax);
            idx = set[p];
            v = comp(xi[idx], ax);
            lt = v < com;
            le = v <= com;
        }
    }
    unsigned peers = seg_peers(act, seg);
    if (!act) return;
    const bool lead = seg_leader(peers);
    unsigned clt = __reduce_add_sync(peers, lt ? 1u : 0u), cle = __reduce_add_sync(peers, le ? 1u : 0u);
    unsigned long long k0 = warp_max_key(peers, lt, v, idx);
    unsigned long long k1 = warp_min_key(peers, !lt, v, idx);
    unsigned long long k2 = warp_max_key(peers, le, v, idx);
    unsigned long long k3 = warp_min_key(peers, !le, v, idx);
    if (lead) {
        atomicAdd(&A.k[seg], clt);
        atomicAdd(&A.k2[seg], cle);
        if (k0) atomicMax(&A.key[4 * seg + 0], k0);
        if (k1 != ~0ULL) atomicMin(&A.key[4 * seg + 1], k1);
        if (k2) atomicMax(&A.key[4 * seg + 2], k2);
        if (k3 != ~0ULL) atomicMin(&A.key[4 * seg + 3], k3);
    }
}

__global__ void k_tree_flag(int m, int thresh, const unsigned int* __restrict__ set,
                            const int* __restrict__ lo, const int* __restrict__ hi,
                            const int4* __restrict__ xi, SegAcc A, unsigned int* __restrict__ lflag)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    int seg = lo[p], size = hi[p] - seg;
    if (size <= thresh) {
        lflag[p] = 0;
        return;
    }
    Cut c = make_cut(size, (int)A.k[seg], (int)A.k2[seg]);
    unsigned idx = set[p];
    bool left;
    if (c.coincident) {
        left = (p - seg) < c.kfinal;  // segments stay in ascending index order
    } else {
        const int ax = seg_axis(A.lo[seg], A.hi[seg]);
        const long long com = seg_com(A, seg, size, ax);
        long long v = comp(xi[idx], ax);
        left = c.use_le ? v <= com : v < com;
        unsigned long long key = ((unsigned long long)v << 32) | idx;
        const int kk = c.use_le ? 2 : 0;
        if (c.kfinal < c.k && key == A.key[4 * seg + kk]) left = false;
        if (c.kfinal > c.k && key == A.key[4 * seg + kk + 1]) left = true;
    }
    lflag[p] = left ? 1u : 0u;
}

__global__ void k_tree_scatter(int m, int thresh, const unsigned int* __restrict__ set,
                               const int* __restrict__ lo, const int* __restrict__ hi, SegAcc A,
                               const unsigned int* __restrict__ lflag,
                               const unsigned int* __restrict__ lscan, unsigned int* __restrict__ set2,
                               int* __restrict__ lo2, int* __restrict__ hi2, SegAcc An, int* maxseg)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    int seg = lo[p], end = hi[p], size = end - seg;
    int np = p, nlo = seg, nhi = end;
    if (size > thresh) {
        Cut c = make_cut(size, (int)A.k[seg], (int)A.k2[seg]);
        int before = (int)(lscan[p] - lscan[seg]);  // low items before p in this segment
        if (lflag[p]) {
            np = seg + before;
            nhi = seg + c.kfinal;
        } else {
            np = seg + c.kfinal + ((p - seg) - before);
            nlo = seg + c.kfinal;
        }
        if (nhi - nlo > thresh) atomicMax(maxseg, nhi - nlo);
    }
    set2[np] = set[p];
    lo2[np] = nlo;
    hi2[np] = nhi;
    if (np == nlo && nhi - nlo > thresh) acc_reset_all(An, np);
}

// ---- shared-memory phase: every segment of size <= TREE_LOCAL, one CTA per chunk

struct LocalSmem {
    int X[TREE_LOC_CAP], Y[TREE_LOC_CAP], Z[TREE_LOC_CAP];
    unsigned I[TREE_LOC_CAP];
    short P[2][TREE_LOC_CAP];              // permutation of local slots
    short Lo[2][TREE_LOC_CAP], Hi[2][TREE_LOC_CAP];
    unsigned Fl[TREE_LOC_CAP];             // low flags
    unsigned F[TREE_LOC_CAP];              // their exclusive prefix over the block's slots
    int amin[3][TREE_LOC_CAP], amax[3][TREE_LOC_CAP];
    unsigned long long asum[TREE_LOC_CAP];
    unsigned ak[TREE_LOC_CAP], ak2[TREE_LOC_CAP];
    unsigned long long akey[TREE_LOC_CAP], akey2[TREE_LOC_CAP];
    unsigned wsum[TREE_LOC_THREADS / 32];
    int range_lo, range_hi, any;
};

__device__ __forceinline__ int lcomp(const LocalSmem& S, int q, int ax)
{
    return ax == 0 ? S.X[q] : (ax == 1 ? S.Y[q] : S.Z[q]);
}

__device__ __forceinline__ int laxis(const LocalSmem& S, int seg)
{
    return axis_of(S.amax[0][seg] - S.amin[0][seg], S.amax[1][seg] - S.amin[1][seg],
                   S.amax[2][seg] - S.amin[2][seg]);
}

__global__ void __launch_bounds__(TREE_LOC_THREADS)
    k_tree_local(int M, const int4* __restrict__ xi, unsigned int* __restrict__ set,
                 int* __restrict__ glo, int* __restrict__ ghi)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LocalSmem& S = *reinterpret_cast<LocalSmem*>(smem_raw);
    const int tid = threadIdx.x;
    const int c0 = blockIdx.x * TREE_LOCAL, c1 = min(M, c0 + TREE_LOCAL);
    if (tid == 0) {
        S.range_lo = INT_MAX;
        S.range_hi = INT_MIN;
    }
    __syncthreads();
    // segments starting in [c0, c1) belong to this block
    for (int p = c0 + tid; p < c1; p += TREE_LOC_THREADS)
        if (glo[p] == p) {
            atomicMin(&S.range_lo, p);
            atomicMax(&S.range_hi, ghi[p]);
        }
    __syncthreads();
    const int base = S.range_lo, s = S.range_hi - S.range_lo;
    if (base == INT_MAX || s <= 0 || s > TREE_LOC_CAP) return;  // s <= 2*TREE_LOCAL - 1 by construction
    for (int q = tid; q < s; q += TREE_LOC_THREADS) {
        unsigned e = set[base + q];
        int4 v = xi[e];
        S.X[q] = v.x;
        S.Y[q] = v.y;
        S.Z[q] = v.z;
        S.I[q] = e;
        S.P[0][q] = (short)q;
        S.Lo[0][q] = (short)(glo[base + q] - base);
        S.Hi[0][q] = (short)(ghi[base + q] - base);
    }
    __syncthreads();
    const int lane = tid & 31, wid = tid >> 5;
    int cur = 0;
    for (int level = 0; level < 4 * TREE_LOC_CAP; ++level) {
        // open segments (size > 2) reset their accumulators
        for (int p = tid; p < s; p += TREE_LOC_THREADS) {
            int l = S.Lo[cur][p], h = S.Hi[cur][p];
            if (l == p && h - l > 2) {
                for (int k = 0; k < 3; ++k) {
                    S.amin[k][p] = INT_MAX;
                    S.amax[k][p] = INT_MIN;
                }
                S.asum[p] = 0;
                S.ak[p] = 0;
                S.ak2[p] = 0;
                S.akey[p] = 0;
                S.akey2[p] = ~0ULL;
            }
        }
        if (tid == 0) S.any = 0;
        __syncthreads();
        // bounding boxes
        for (int p0 = 0; p0 < s; p0 += TREE_LOC_THREADS) {
            int p = p0 + tid;
            bool act = false;
            int seg = 0, q = 0;
            if (p < s) {
                seg = S.Lo[cur][p];
                act = S.Hi[cur][p] - seg > 2;
                q = S.P[cur][p];
            }
            unsigned peers = seg_peers(act, seg);
            if (act) {
                int mn[3] = {__reduce_min_sync(peers, S.X[q]), __reduce_min_sync(peers, S.Y[q]),
                             __reduce_min_sync(peers, S.Z[q])};
                int mx[3] = {__reduce_max_sync(peers, S.X[q]), __reduce_max_sync(peers, S.Y[q]),
                             __reduce_max_sync(peers, S.Z[q])};
                if (seg_leader(peers))
                    for (int k = 0; k < 3; ++k) {
                        atomicMin(&S.amin[k][seg], mn[k]);
                        atomicMax(&S.amax[k][seg], mx[k]);
                    }
            }
        }
        __syncthreads();
        // coordinate sums along each segment's widest axis
        for (int p0 = 0; p0 < s; p0 += TREE_LOC_THREADS) {
            int p = p0 + tid;
            bool act = false;
            int seg = 0;
            unsigned v = 0;
            if (p < s) {
                seg = S.Lo[cur][p];
                act = S.Hi[cur][p] - seg > 2;
                if (act) v = (unsigned)lcomp(S, S.P[cur][p], laxis(S, seg));
            }
            unsigned peers = seg_peers(act, seg);
            if (act) {
                unsigned sh = __reduce_add_sync(peers, v >> 15), sl = __reduce_add_sync(peers, v & 0x7fffu);
                if (seg_leader(peers))
                    atomicAdd(&S.asum[seg], ((unsigned long long)sh << 15) + (unsigned long long)sl);
            }
        }
        __syncthreads();
        // counts below the centre of mass
        for (int p0 = 0; p0 < s; p0 += TREE_LOC_THREADS) {
            int p = p0 + tid;
            bool act = false;
            int seg = 0;
            unsigned lt = 0, le = 0;
            if (p < s) {
                seg = S.Lo[cur][p];
                int size = S.Hi[cur][p] - seg;
                act = size > 2;
                if (act) {
                    long long com = (long long)(S.asum[seg] / (unsigned long long)size);
                    long long v = lcomp(S, S.P[cur][p], laxis(S, seg));
                    lt = v < com;
                    le = v <= com;
                }
            }
            unsigned peers = seg_peers(act, seg);
            if (act) {
                unsigned clt = __reduce_add_sync(peers, lt), cle = __reduce_add_sync(peers, le);
                if (seg_leader(peers)) {
                    atomicAdd(&S.ak[seg], clt);
                    atomicAdd(&S.ak2[seg], cle);
                }
            }
        }
        __syncthreads();
        // odd cuts: the particle that crosses (reduced per warp, one atomic per segment run)
        for (int p0 = 0; p0 < s; p0 += TREE_LOC_THREADS) {
            int p = p0 + tid;
            bool act = false, down = false;
            int seg = 0, v = 0;
            unsigned idx = 0;
            if (p < s) {
                seg = S.Lo[cur][p];
                int size = S.Hi[cur][p] - seg;
                if (size > 2) {
                    Cut c = make_cut(size, (int)S.ak[seg], (int)S.ak2[seg]);
                    if (!c.coincident && c.kfinal != c.k) {
                        int q = S.P[cur][p];
                        long long com = (long long)(S.asum[seg] / (unsigned long long)size);
                        v = lcomp(S, q, laxis(S, seg));
                        bool low = c.use_le ? v <= com : v < com;
                        down = c.kfinal < c.k;
                        act = down ? low : !low;
                        idx = S.I[q];
                    }
                }
            }
            // the cut direction is a property of the segment, so peers share it
            unsigned peers = seg_peers(act, seg);
            if (act) {
                if (down) {
                    unsigned long long k0 = warp_max_key(peers, true, v, idx);
                    if (seg_leader(peers)) atomicMax(&S.akey[seg], k0);
                } else {
                    unsigned long long k1 = warp_min_key(peers, true, v, idx);
                    if (seg_leader(peers)) atomicMin(&S.akey2[seg], k1);
                }
            }
        }
        __syncthreads();
        // low flags
        for (int p = tid; p < s; p += TREE_LOC_THREADS) {
            int seg = S.Lo[cur][p], size = S.Hi[cur][p] - seg;
            unsigned f = 0;
            if (size > 2) {
                Cut c = make_cut(size, (int)S.ak[seg], (int)S.ak2[seg]);
                if (c.coincident) {
                    f = (p - seg) < c.kfinal;  // segments stay in ascending index order
                } else {
                    int q = S.P[cur][p];
                    long long com = (long long)(S.asum[seg] / (unsigned long long)size);
                    long long v = lcomp(S, q, laxis(S, seg));
                    bool left = c.use_le ? v <= com : v < com;
                    unsigned long long key = ((unsigned long long)v << 32) | S.I[q];
                    if (c.kfinal < c.k && key == S.akey[seg]) left = false;
                    if (c.kfinal > c.k && key == S.akey2[seg]) left = true;
                    f = left;
                }
            }
            S.Fl[p] = f;
        }
        __syncthreads();
        // exclusive prefix of the flags over the block's slots (a contiguous run per thread)
        {
            const int per = (s + TREE_LOC_THREADS - 1) / TREE_LOC_THREADS;
            const int b0 = min(s, tid * per), b1 = min(s, b0 + per);
            unsigned run = 0;
            for (int p = b0; p < b1; ++p) run += S.Fl[p];
            unsigned incl = run;
            for (int o = 1; o < 32; o <<= 1) {
                unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane == 31) S.wsum[wid] = incl;
            __syncthreads();
            unsigned ex = incl - run;
            for (int w = 0; w < wid; ++w) ex += S.wsum[w];
            for (int p = b0; p < b1; ++p) {
                S.F[p] = ex;
                ex += S.Fl[p];
            }
        }
        __syncthreads();
        // stable partition of every open segment into the other buffer
        const int nx = cur ^ 1;
        for (int p = tid; p < s; p += TREE_LOC_THREADS) {
            int seg = S.Lo[cur][p], end = S.Hi[cur][p], size = end - seg;
            int np = p, nlo = seg, nhi = end;
            if (size > 2) {
                Cut c = make_cut(size, (int)S.ak[seg], (int)S.ak2[seg]);
                int before = (int)(S.F[p] - S.F[seg]);  // low slots in [seg, p)
                if (S.Fl[p]) {
                    np = seg + before;
                    nhi = seg + c.kfinal;
                } else {
                    np = seg + c.kfinal + ((p - seg) - before);
                    nlo = seg + c.kfinal;
                }
                if (nhi - nlo > 2) S.any = 1;
            }
            S.P[nx][np] = S.P[cur][p];
            S.Lo[nx][np] = (short)nlo;
            S.Hi[nx][np] = (short)nhi;
        }
        __syncthreads();
        cur = nx;
        if (!S.any) break;
        __syncthreads();
    }
    for (int p = tid; p < s; p += TREE_LOC_THREADS) {
        set[base + p] = S.I[S.P[cur][p]];
        glo[base + p] = base + S.Lo[cur][p];
        ghi[base + p] = base + S.Hi[cur][p];
    }
}

// the merge decision of every leaf pair of every level (Sec. 2.3, Eq. 3)
__global__ void k_merge_apply(DevCfg dc, DevRegions rg, int M, const unsigned int* __restrict__ set,
                              const int* __restrict__ glo, const int* __restrict__ ghi,
                              apr_particles p, int* __restrict__ count_per_level)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= M || glo[q] != q || ghi[q] - q != 2) return;
    unsigned a = set[q], b = set[q + 1];
    if (b < a) {
        unsigned t = a;
        a = b;
        b = t;
    }
    const int level = p.level[a];
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
    atomicAdd(&count_per_level[level], 1);
}

// the pairing trees of all levels.  On return (*set)[0..M) holds the candidates
// grouped by level (ascending), each level's leaves at consecutive slots, and
// (*lo, *hi) the leaf bounds of every slot; off[l] is the first slot of level l
// (off[lmax+1] = M).
static apr_status pair_trees(apr_ctx* c, int* off, unsigned int** set_out, int** lo_out,
                             int** hi_out)
{
    Workspace& W = c->W;
    cudaStream_t st = c->stream;
    const long long n = c->n;
    const int lmax = c->cfg.lmax;
    APR_LAUNCH(c, k_merge_keys, nblocks(n, 256), 256, n, c->p.level, c->p.flags, W.key[0], W.val[0]);
    apr_status s = radix_pass8(c, W.key[0], W.val[0], W.key[1], W.mset[0], n, 0, &W.status[ST_BINS],
                               lmax + 2);
    if (s != APR_OK) return s;
    cudaMemcpyAsync(c->hbuf, &W.status[ST_BINS], sizeof(int) * (lmax + 2), cudaMemcpyDeviceToHost, st);
    s = cuda_check(c, cudaStreamSynchronize(st), "merge candidates");
    if (s != APR_OK) return s;
    const int* bins = (const int*)c->hbuf;
    // bins[l] = first sorted slot of level l; candidates are levels 1..lmax
    LevelOffsets lo_off;
    memset(&lo_off, 0, sizeof(lo_off));
    lo_off.lmax = lmax;
    const int first = lmax >= 1 ? bins[1] : 0;
    for (int l = 1; l <= lmax + 1; ++l) {
        off[l] = (l <= lmax + 1 ? bins[l] : bins[lmax + 1]) - first;
        lo_off.off[l] = off[l];
    }
    off[0] = 0;
    const int M = off[lmax + 1];
    *set_out = W.mset[1];
    *lo_out = W.seg_lo[0];
    *hi_out = W.seg_hi[0];
    if (M <= 0) return APR_OK;
    if (first > 0)  // level-0 particles sorted first: move the candidates to slot 0
        cudaMemcpyAsync(W.mset[1], W.mset[0] + first, sizeof(unsigned) * M, cudaMemcpyDeviceToDevice,
                        st);
    else
        cudaMemcpyAsync(W.mset[1], W.mset[0], sizeof(unsigned) * M, cudaMemcpyDeviceToDevice, st);
    const long long C = c->cap;
    SegAcc acc[2];
    for (int k = 0; k < 2; ++k) {
        acc[k].lo = W.acc_lo + k * C;
        acc[k].hi = W.acc_hi + k * C;
        acc[k].sum = W.acc_sum + 3 * k * C;
        acc[k].k = W.acc_k + k * C;
        acc[k].k2 = W.acc_k2 + k * C;
        acc[k].key = W.acc_key + 4 * k * C;
    }
    // buffers: set[] alternates between mset[1] and mset[0]
    unsigned int* sets[2] = {W.mset[1], W.mset[0]};
    APR_LAUNCH(c, k_seg_setup, nblocks(M, 256), 256, M, lo_off, W.seg_lo[0], W.seg_hi[0], acc[0]);
    int maxm = 0;
    for (int l = 1; l <= lmax; ++l) maxm = max(maxm, off[l + 1] - off[l]);
    int cur = 0;
    const int nb = nblocks(M, 256);
    int rounds_left = 0;
    if (maxm > TREE_LOCAL) {
        int est = 1;
        while ((TREE_LOCAL << est) < maxm) ++est;
        rounds_left = est + 1;
    }
    for (int total = 0; rounds_left > 0 && total < 64 + 4 * 32; ) {
        for (int r = 0; r < rounds_left; ++r, ++total) {
            APR_LAUNCH(c, k_tree_bbox_sum, nb, 256, M, TREE_LOCAL, sets[cur], W.seg_lo[cur],
                       W.seg_hi[cur], W.xi, acc[cur]);
            APR_LAUNCH(c, k_tree_count_key, nb, 256, M, TREE_LOCAL, sets[cur], W.seg_lo[cur],
                       W.seg_hi[cur], W.xi, acc[cur]);
            APR_LAUNCH(c, k_tree_flag, nb, 256, M, TREE_LOCAL, sets[cur], W.seg_lo[cur],
                       W.seg_hi[cur], W.xi, acc[cur], W.lflag);
            scan_u32(c, W.lflag, W.uscan, M, nullptr);
            cudaMemsetAsync(&W.status[ST_MAXSEG], 0, sizeof(int), st);
            const int nx = cur ^ 1;
            APR_LAUNCH(c, k_tree_scatter, nb, 256, M, TREE_LOCAL, sets[cur], W.seg_lo[cur],
                       W.seg_hi[cur], acc[cur], W.lflag, W.uscan, sets[nx], W.seg_lo[nx],
                       W.seg_hi[nx], acc[nx], &W.status[ST_MAXSEG]);
            cur = nx;
        }
        cudaMemcpyAsync(c->hbuf, &W.status[ST_MAXSEG], sizeof(int), cudaMemcpyDeviceToHost, st);
        s = cuda_check(c, cudaStreamSynchronize(st), "pairing tree");
        if (s != APR_OK) return s;
        rounds_left = ((int*)c->hbuf)[0] > TREE_LOCAL ? 2 : 0;
    }
    if (rounds_left > 0) return fail(c, APR_ERR_STATE, "pairing tree did not reach its leaves");
    if (!c->tree_smem_set) {
        s = cuda_check(c, cudaFuncSetAttribute(k_tree_local,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)sizeof(LocalSmem)), "tree smem");
        if (s != APR_OK) return s;
        c->tree_smem_set = true;
    }
    APR_LAUNCH_SMEM(c, k_tree_local, nblocks(M, TREE_LOCAL), TREE_LOC_THREADS, sizeof(LocalSmem), M,
                    W.xi, sets[cur], W.seg_lo[cur], W.seg_hi[cur]);
    *set_out = sets[cur];
    *lo_out = W.seg_lo[cur];
    *hi_out = W.seg_hi[cur];
    return cuda_check(c, cudaGetLastError(), "pairing tree");
}

__global__ void k_pairs_out(int m, const unsigned int* __restrict__ set, long long* __restrict__ out)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) out[j] = set[j];
}

apr_status merge_pairs_debug(apr_ctx* c, int level, long long* pairs, long long cap,
                             long long* npairs, long long* spare)
{
    *npairs = 0;
    *spare = -1;
    if (level > c->cfg.lmax || c->n == 0) return APR_OK;
    apr_status s = quantise(c);
    if (s != APR_OK) return s;
    int off[APR_MAXLEV + 2];
    unsigned int* set;
    int *lo, *hi;
    s = pair_trees(c, off, &set, &lo, &hi);
    if (s != APR_OK) return s;
    const int a = off[level], m = off[level + 1] - a, me = m & ~1;
    *npairs = me / 2;
    if (me / 2 > cap) return fail(c, APR_ERR_ARG, "merge_pairs: cap too small");
    if (m == 0) return APR_OK;
    long long* dev = (long long*)c->W.tmp8;
    APR_LAUNCH(c, k_pairs_out, nblocks(m, 256), 256, m, set + a, dev);
    std::vector<long long> buf(m);
    s = cuda_check(c, cudaMemcpyAsync(buf.data(), dev, sizeof(long long) * m, cudaMemcpyDeviceToHost,
                                      c->stream), "pairs out");
    if (s != APR_OK) return s;
    s = cuda_check(c, cudaStreamSynchronize(c->stream), "pairs out");
    if (s != APR_OK) return s;
    for (int j = 0; j < me; ++j) pairs[j] = buf[j];
    if (m % 2) *spare = buf[m - 1];
    return APR_OK;
}

// ------------------------------------------------------------ compaction

struct FieldPtrs {
    double* d[18];
    unsigned long long* id;
    unsigned char* level;
    unsigned char* flags;
};

static FieldPtrs field_ptrs(const apr_particles& p)
{
    FieldPtrs f;
    double* d[18] = {p.x,  p.y,  p.z,  p.vx,   p.vy,   p.vz,  p.u,    p.h,    p.rho,
                     p.omega, p.ax, p.ay, p.az, p.dudt, p.vsig, p.dnn, p.pres, p.cs};
    for (int k = 0; k < 18; ++k) f.d[k] = d[k];
    f.id = p.id;
    f.level = p.level;
    f.flags = p.flags;
    return f;
}

__global__ void k_live_flag(long long n, const unsigned char* __restrict__ flags,
                            unsigned int* __restrict__ out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (flags[i] & APR_FLAG_DEAD) ? 0u : 1u;
}

// live particles to their compacted slots in scratch laid out field by field
__global__ void k_compact_out(long long n, long long cap, FieldPtrs f,
                              const unsigned int* __restrict__ pos, double* __restrict__ tmp)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned char fl = f.flags[i];
    if (fl & APR_FLAG_DEAD) return;
    const long long j = pos[i];
    for (int k = 0; k < 18; ++k) tmp[k * cap + j] = f.d[k][i];
    ((unsigned long long*)(tmp + 18 * cap))[j] = f.id[i];
    unsigned char* b = (unsigned char*)(tmp + 19 * cap);
    b[j] = f.level[i];
    b[cap + j] = fl;
}

__global__ void k_compact_back(long long nlive, long long cap, FieldPtrs f,
                               const double* __restrict__ tmp)
{
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nlive) return;
    for (int k = 0; k < 18; ++k) f.d[k][j] = tmp[k * cap + j];
    f.id[j] = ((const unsigned long long*)(tmp + 18 * cap))[j];
    const unsigned char* b = (const unsigned char*)(tmp + 19 * cap);
    f.level[j] = b[j];
    f.flags[j] = b[cap + j];
}

// stable removal of dead particles.  The neighbour-list memory serves as scratch
// (the lists are rebuilt after any change of the particle set).
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
    const FieldPtrs f = field_ptrs(c->p);
    double* tmp = (double*)W.nbr;  // 20 x cap x 8 bytes <= max_neigh x cap x 4 bytes
    APR_LAUNCH(c, k_compact_out, nblocks(n, 256), 256, n, c->cap, f, W.uscan, tmp);
    APR_LAUNCH(c, k_compact_back, nblocks(nlive, 256), 256, nlive, c->cap, f, tmp);
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
    if (c->cfg.lmax >= 1 && c->n > 0) {
        const long long n = c->n;
        APR_LAUNCH(c, k_split_keys, nblocks(n, 256), 256, c->dc, rg, n, c->p.x, c->p.y, c->p.z,
                   c->p.level, c->p.flags, W.key[0], W.val[0]);
        s = radix_pass8(c, W.key[0], W.val[0], W.key[1], W.val[1], n, 0, &W.status[ST_BINS],
                        c->cfg.lmax + 1);
        if (s != APR_OK) return s;
        cudaMemcpyAsync(c->hbuf, &W.status[ST_BINS], sizeof(int) * (c->cfg.lmax + 1),
                        cudaMemcpyDeviceToHost, st);
        s = cuda_check(c, cudaStreamSynchronize(st), "split count");
        if (s != APR_OK) return s;
        const int* bins = (const int*)c->hbuf;  // parents of level l: [bins[l], bins[l+1])
        const int total = bins[c->cfg.lmax];
        for (int l = 0; l < c->cfg.lmax; ++l) cnt->n_split[l] = bins[l + 1] - bins[l];
        if (n + total > c->cap)
            return fail(c, APR_ERR_CAPACITY, "split would exceed the bound capacity");
        if (total > 0) {
            APR_LAUNCH(c, k_split_apply, nblocks(total, 256), 256, c->dc, rg, total, n, c->step,
                       c->next_id, W.val[1], c->p);
            c->n = n + total;
            c->next_id += total;
        }
    }
    if (c->cfg.lmax >= 1 && c->n > 0) {
        s = quantise(c);
        if (s != APR_OK) return s;
        int off[APR_MAXLEV + 2];
        unsigned int* set;
        int *lo, *hi;
        s = pair_trees(c, off, &set, &lo, &hi);
        if (s != APR_OK) return s;
        const int M = off[c->cfg.lmax + 1];
        for (int l = 1; l <= c->cfg.lmax; ++l) cnt->n_spare[l] = (off[l + 1] - off[l]) & 1;
        if (M >= 2) {
            cudaMemsetAsync(&W.status[ST_MERGES], 0, sizeof(int) * APR_MAXLEV, st);
            APR_LAUNCH(c, k_merge_apply, nblocks(M, 256), 256, c->dc, rg, M, set, lo, hi, c->p,
                       &W.status[ST_MERGES]);
            cudaMemcpyAsync(c->hbuf, &W.status[ST_MERGES], sizeof(int) * APR_MAXLEV,
                            cudaMemcpyDeviceToHost, st);
            s = cuda_check(c, cudaStreamSynchronize(st), "merge");
            if (s != APR_OK) return s;
            for (int l = 1; l <= c->cfg.lmax; ++l) cnt->n_merge[l] = ((int*)c->hbuf)[l];
        }
    }
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

// fixed-shape reduction of the block partials (one block): deterministic
__global__ void __launch_bounds__(256) k_reduce_final(int nblk, int nv,
                                                      const double* __restrict__ partials,
                                                      double* __restrict__ out,
                                                      unsigned int min_mask)
{
    __shared__ double sm[256];
    for (int k = 0; k < nv; ++k) {
        const bool op_min = (min_mask >> k) & 1u;
        double x = op_min ? INFINITY : 0.0;
        for (int b = threadIdx.x; b < nblk; b += 256) {
            double y = partials[b * 32 + k];
            x = op_min ? fmin(x, y) : x + y;
        }
        sm[threadIdx.x] = x;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s)
                sm[threadIdx.x] = op_min ? fmin(sm[threadIdx.x], sm[threadIdx.x + s])
                                         : sm[threadIdx.x] + sm[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sm[0];
        __syncthreads();
    }
}

static apr_status reduce_readback_n(apr_ctx* c, int nblk, int nv, unsigned int min_mask,
                                   double* host)
{
    APR_LAUNCH(c, k_reduce_final, 1, 256, nblk, nv, c->W.red, c->W.redout, min_mask);
    cudaMemcpyAsync(c->hbuf, c->W.redout, sizeof(double) * nv, cudaMemcpyDeviceToHost, c->stream);
    apr_status s = cuda_check(c, cudaStreamSynchronize(c->stream), "reduce");
    if (s != APR_OK) return s;
    memcpy(host, c->hbuf, sizeof(double) * nv);
    return APR_OK;
}

static apr_status reduce_readback(apr_ctx* c, int nv, unsigned int min_mask, double* host)
{
    APR_LAUNCH(c, k_reduce_final, 1, 256, RED_BLOCKS, nv, c->W.red, c->W.redout, min_mask);
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

// conservation sums (9) and the time-step limit (slot 9, a minimum) in one pass
__global__ void __launch_bounds__(256) k_stats_dt(DevCfg dc, long long n, apr_particles p,
                                                  double* partials)
{
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    double dt = INFINITY;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned char fl = p.flags[i];
        if (fl & APR_FLAG_DEAD) continue;
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
        if (fl & APR_FLAG_FIXED) continue;
        double h = p.h[i];
        if (p.vsig[i] > 0.0) dt = fmin(dt, dc.ccour * h / p.vsig[i]);
        double a = sqrt(p.ax[i] * p.ax[i] + p.ay[i] * p.ay[i] + p.az[i] * p.az[i]);
        if (a > 0.0) dt = fmin(dt, dc.cforce * sqrt(h / a));
    }
    __shared__ double sm[10][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 9; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sm[k][wid] = x;
    }
    for (int o = 16; o > 0; o >>= 1) dt = fmin(dt, __shfl_down_sync(0xffffffffu, dt, o));
    if (lane == 0) sm[9][wid] = dt;
    __syncthreads();
    if (threadIdx.x < 10) {
        double x = sm[threadIdx.x][0];
        for (int w = 1; w < 8; ++w)
            x = threadIdx.x == 9 ? fmin(x, sm[threadIdx.x][w]) : x + sm[threadIdx.x][w];
        partials[blockIdx.x * 32 + threadIdx.x] = x;
    }
}

static void stats_from(const apr_ctx* c, const double* r, apr_stats* st)
{
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
}

apr_status compute_stats_dt(apr_ctx* c, apr_stats* st, double* dt)
{
    const int nblk = (int)std::min<long long>(RED_BLOCKS, std::max<long long>(1, (c->n + 2047) / 2048));
    APR_LAUNCH(c, k_stats_dt, nblk, 256, c->dc, c->n, c->p, c->W.red);
    double r[10];
    apr_status s = reduce_readback_n(c, nblk, 10, 1u << 9, r);
    if (s != APR_OK) return s;
    stats_from(c, r, st);
    *dt = r[9];
    return APR_OK;
}

apr_status compute_stats(apr_ctx* c, apr_stats* st)
{
    APR_LAUNCH(c, k_stats, RED_BLOCKS, 256, c->dc, c->n, c->p, c->W.red);
    double r[9];
    apr_status s = reduce_readback(c, 9, 0u, r);
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
    return reduce_readback(c, 1, 1u, dt);
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
    apr_status s = reduce_readback(c, 3 * c->nsink, 0u, r);
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
    apr_status s = reduce_readback(c, 7 * c->nsink, 0u, r);
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

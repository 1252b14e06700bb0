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
#include "apr_dtmin.cuh"
#include "apr_sinkpre.cuh"
#include "apr_pair.cuh"

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
        } else if (r.shape == APR_SHAPE_CYLINDER) {
            // distance from the axis line: the two other components, in axis order
            double d[3] = {px - r.centre[0], py - r.centre[1], pz - r.centre[2]};
            const int a1 = r.axis == 0 ? 1 : 0, a2 = r.axis == 2 ? 1 : 2;
            double d2 = d[a1] * d[a1] + d[a2] * d[a2];
            inside = d2 < r.R[k] * r.R[k];
        } else {
            double p = r.axis == 0 ? px : (r.axis == 1 ? py : pz);
            inside = fabs(p - r.centre[r.axis]) < r.R[k];
        }
        if (inside) lev = k + 1;
    }
    return lev;
}

// target level (Sec. 2.1): refinement (level_default 0) takes the deepest zone,
// capped at lmax; derefinement (level_default L) lowers L by the deepest zone's
// depth, floored at 0.  *which: the deciding zone (the deepest; in derefinement
// a point outside every zone is decided by zone 0), -1 if there is none.
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
    int t;
    if (dc.level_default > 0) {
        t = dc.level_default - best;
        if (t < 0) t = 0;
        if (w < 0 && rg.n > 0) w = 0;
    } else {
        t = best > dc.lmax ? dc.lmax : best;
    }
    if (which) *which = w;
    return t;
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
    } else if (r.shape == APR_SHAPE_CYLINDER) {
        // the radial direction from the axis line (the axis component removed)
        v[0] = px - r.centre[0];
        v[1] = py - r.centre[1];
        v[2] = pz - r.centre[2];
        v[r.axis] = 0.0;
        double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (vn > 0.0) {
            v[0] = v[0] / vn;
            v[1] = v[1] / vn;
            v[2] = v[2] / vn;
        } else {
            v[0] = v[1] = v[2] = 0.0;
            v[r.axis == 0 ? 1 : 0] = 1.0;
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
// the level a single zone asks for at p with every boundary shrunk by a relative
// 1e-8: a point that reaches level l here lies inside the level-l boundary by more
// than the rounding of any midpoint formed from it
__device__ int region_level_inset(const DevRegion& r, double px, double py, double pz)
{
    constexpr double INSET = 1.0 - 1e-8;
    int lev = 0;
    for (int k = 0; k < r.nlev; ++k) {
        const double R = r.R[k] * INSET;
        bool inside;
        if (r.shape == APR_SHAPE_SPHERE) {
            double dx = px - r.centre[0], dy = py - r.centre[1], dz = pz - r.centre[2];
            inside = dx * dx + dy * dy + dz * dz < R * R;
        } else if (r.shape == APR_SHAPE_CYLINDER) {
            double d[3] = {px - r.centre[0], py - r.centre[1], pz - r.centre[2]};
            const int a1 = r.axis == 0 ? 1 : 0, a2 = r.axis == 2 ? 1 : 2;
            inside = d[a1] * d[a1] + d[a2] * d[a2] < R * R;
        } else {
            double p = r.axis == 0 ? px : (r.axis == 1 ? py : pz);
            inside = fabs(p - r.centre[r.axis]) < R;
        }
        if (inside) lev = k + 1;
    }
    return lev;
}

// split keys (level of a split candidate, 255 otherwise) and the pass's summary in
// sm[]: split candidates, dead particles, and (check_merge: one convex zone, see
// merge_shortcut_ok) merge candidates per level and whether one of them is not
// safely inside its level's zone
__global__ void k_split_keys(DevCfg dc, DevRegions rg, long long n, const double* __restrict__ x,
                             const double* __restrict__ y, const double* __restrict__ z,
                             const unsigned char* __restrict__ lev,
                             const unsigned char* __restrict__ flags,
                             unsigned long long* __restrict__ key, unsigned int* __restrict__ val,
                             int check_merge, int* __restrict__ sm)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < n;
    int l = 0;
    bool split = false, dead = false, cand = false, loose = false;
    if (live) {
        l = lev[i];
        const unsigned char f = flags[i];
        dead = (f & APR_FLAG_DEAD) != 0;
        const bool free_ = !(f & (APR_FLAG_CHANGED | APR_FLAG_FIXED | APR_FLAG_DEAD | APR_FLAG_INACTIVE));
        if (l < dc.lmax && free_) split = target_level(dc, rg, x[i], y[i], z[i], nullptr) > l;
        if (check_merge && l >= 1 && free_) {
            cand = true;
            int t = region_level_inset(rg.r[0], x[i], y[i], z[i]);
            if (t > dc.lmax) t = dc.lmax;
            loose = t < l;
        }
        key[i] = split ? (unsigned long long)l : 255ULL;
        val[i] = (unsigned)i;
    }
    const unsigned FULL = 0xffffffffu;
    const bool lead = (threadIdx.x & 31) == 0;
    const unsigned ns = __popc(__ballot_sync(FULL, split));
    const bool any_dead = __any_sync(FULL, dead), any_loose = __any_sync(FULL, loose);
    if (lead) {
        if (ns) atomicAdd(&sm[ST_SM_NSPLIT - ST_SM_NSPLIT], (int)ns);
        if (any_dead || any_loose) atomicOr(&sm[ST_SM_FLAGS - ST_SM_NSPLIT], (any_dead ? 1 : 0) | (any_loose ? 2 : 0));
    }
    if (check_merge && __any_sync(FULL, cand)) {
        for (int k = 1; k <= dc.lmax; ++k) {
            const unsigned c = __popc(__ballot_sync(FULL, cand && l == k));
            if (lead && c) atomicAdd(&sm[ST_SM_NCAND - ST_SM_NSPLIT + k], (int)c);
        }
    }
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
    if (which >= 0) {
        split_direction(rg.r[which], px, py, pz, t, w);
    } else {
        // no zone decides (derefinement without zones): a sphere centred on the
        // parent, whose direction falls back to the x axis
        DevRegion self;
        self.shape = APR_SHAPE_SPHERE;
        self.axis = 0;
        self.nlev = 0;
        self.centre[0] = px;
        self.centre[1] = py;
        self.centre[2] = pz;
        split_direction(self, px, py, pz, t, w);
    }
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
    if (p.bin) p.bin[j] = p.bin[i];
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
    p.flags[i] = p.flags[i] | APR_FLAG_CHANGED | APR_FLAG_NEW;
    p.flags[j] = p.flags[i];
    p.id[j] = (unsigned long long)(next_id + (long long)r);
}

// ------------------------------------------------------------ merge tree
//
// The candidates of every level are paired at once (their trees are
// independent): one stable radix pass groups them by level in ascending
// index order; a cooperative kernel cuts every segment larger than TREE_WARP
// round by round; then one warp per segment finishes it in registers.

constexpr int TREE_WARP = 32;          // segments of at most this size finish in one warp
constexpr int COOP_THREADS = 1024;
constexpr unsigned BARRIER_SPIN_LIMIT = 1u << 22;  // polls of ~32 ns + latency: well above 0.1 s

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
    const bool cand = l >= 1 && !(flags[i] & (APR_FLAG_CHANGED | APR_FLAG_FIXED | APR_FLAG_DEAD | APR_FLAG_INACTIVE));
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
    if (p == a && be - a > TREE_WARP) acc_reset_all(A, a);
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


// ---- global rounds: one cooperative persistent kernel
//
// Every round cuts all segments larger than TREE_WARP at once, in three phases
// separated by grid barriers: (B) counts below the centre of mass and the keys
// an odd cut could move; (C) low flags and their prefix within each block's
// chunk, and the reset of the children's accumulators; (D) the chunk offsets
// (scanned again in every block), the stable partition into the other
// buffers, and the children's bounding boxes and coordinate sums for the next
// round.  The loop ends on the device when no segment is larger than
// TREE_WARP.  The grid is no larger than the number of co-resident blocks
// (cooperative launch), so every barrier is reached by all blocks; each wait
// is still bounded and records a timeout.

struct Coop {
    unsigned* btot;     // per block: low flags in its chunk
    unsigned* bar;      // [0] arrivals, [1] generation
    int* maxseg;        // [3], rotating: largest open segment after a round
    int* rounds;        // rounds taken
    int* err;           // 1: a barrier wait timed out; 2: the leaves were not reached
};

__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned* p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void red_add_release_gpu(unsigned* p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// all blocks of the (co-resident) grid: the block's writes before, everyone's after
__device__ __forceinline__ void grid_barrier(const Coop& co)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned* gen = co.bar + 1;
        const unsigned g = ld_relaxed_gpu(gen);
        if (atom_add_acq_rel_gpu(co.bar, 1u) == gridDim.x - 1) {
            atomicExch(co.bar, 0u);
            red_add_release_gpu(gen, 1u);
        } else {
            // poll without acquire semantics, then acquire once
            unsigned it = 0;
            while (ld_relaxed_gpu(gen) == g) {
                if (++it > BARRIER_SPIN_LIMIT) {
                    atomicOr(co.err, 1);
                    break;
                }
            }
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
    }
    __syncthreads();
}

// one particle's bounding box and coordinate sums into its segment (warp-aggregated)
__device__ __forceinline__ void accumulate_box_sum(bool act, int seg, const int4& q, const SegAcc& A)
{
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

__device__ __forceinline__ void round_count_key(int p, int m, int thresh,
                                                const unsigned int* __restrict__ set,
                                                const int* __restrict__ lo,
                                                const int* __restrict__ hi,
                                                const int4* __restrict__ xi, const SegAcc& A)
{
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

__device__ __forceinline__ unsigned round_flag(int p, int thresh, const unsigned int* __restrict__ set,
                                               const int* __restrict__ lo, const int* __restrict__ hi,
                                               const int4* __restrict__ xi, const SegAcc& A)
{
    int seg = lo[p], size = hi[p] - seg;
    if (size <= thresh) return 0u;
    Cut c = make_cut(size, (int)A.k[seg], (int)A.k2[seg]);
    if (c.coincident) return (p - seg) < c.kfinal ? 1u : 0u;  // segments keep ascending index order
    unsigned idx = set[p];
    const int ax = seg_axis(A.lo[seg], A.hi[seg]);
    const long long com = seg_com(A, seg, size, ax);
    long long v = comp(xi[idx], ax);
    bool left = c.use_le ? v <= com : v < com;
    unsigned long long key = ((unsigned long long)v << 32) | idx;
    const int kk = c.use_le ? 2 : 0;
    if (c.kfinal < c.k && key == A.key[4 * seg + kk]) left = false;
    if (c.kfinal > c.k && key == A.key[4 * seg + kk + 1]) left = true;
    return left ? 1u : 0u;
}

// exclusive block scan of one value per thread; returns the block total in *total
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned* total)
{
    __shared__ unsigned wsum[COOP_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    unsigned before = 0, all = 0;
    for (int w = 0; w < COOP_THREADS / 32; ++w) {
        if (w < wid) before += wsum[w];
        all += wsum[w];
    }
    __syncthreads();
    *total = all;
    return before + incl - v;
}

__global__ void __launch_bounds__(COOP_THREADS)
    k_tree_rounds(int M, int thresh, int max_rounds, const int4* __restrict__ xi,
                  unsigned int* set0, unsigned int* set1, int* lo0, int* lo1, int* hi0, int* hi1,
                  SegAcc A0, SegAcc A1, unsigned int* lflag, unsigned int* lscan, Coop co)
{
    __shared__ unsigned s_off[COOP_MAX_BLOCKS];
    __shared__ int s_stop;
    const int G = gridDim.x;
    const int gtid = blockIdx.x * COOP_THREADS + threadIdx.x, gstride = G * COOP_THREADS;
    const int chunk = (M + G - 1) / G;
    // the first cut's boxes and sums (accumulators reset by the setup kernel)
    for (int p0 = 0; p0 < M; p0 += gstride) {
        const int p = p0 + gtid;
        bool act = false;
        int seg = 0;
        int4 q = make_int4(0, 0, 0, 0);
        if (p < M) {
            seg = lo0[p];
            act = hi0[p] - seg > thresh;
            if (act) q = xi[set0[p]];
        }
        accumulate_box_sum(act, seg, q, A0);
    }
    grid_barrier(co);
    int cur = 0, r = 0;
    while (r < max_rounds) {
        // this round's buffers (selected, not indexed, so that they stay in registers)
        unsigned int* const sc = cur ? set1 : set0;
        unsigned int* const sn = cur ? set0 : set1;
        const int* const lc = cur ? lo1 : lo0;
        int* const ln = cur ? lo0 : lo1;
        const int* const hc = cur ? hi1 : hi0;
        int* const hn = cur ? hi0 : hi1;
        const SegAcc Ac = cur ? A1 : A0;
        const SegAcc An = cur ? A0 : A1;
        if (gtid == 0) co.maxseg[(r + 1) % 3] = 0;
        // (B) counts below the centre of mass and the odd-cut keys
        for (int p0 = 0; p0 < M; p0 += gstride) round_count_key(p0 + gtid, M, thresh, sc, lc, hc, xi, Ac);
        grid_barrier(co);
        // (C) low flags and their prefix within this block's chunk; the children's
        // accumulators are reset by the thread at the start of the parent segment
        {
            const int c0 = blockIdx.x * chunk, c1 = min(M, c0 + chunk);
            unsigned run = 0;
            for (int base = c0; base < c1; base += COOP_THREADS) {
                const int p = base + threadIdx.x;
                unsigned f = 0u;
                if (p < c1) {
                    f = round_flag(p, thresh, sc, lc, hc, xi, Ac);
                    const int seg = lc[p], size = hc[p] - seg;
                    if (p == seg && size > thresh) {
                        const Cut c = make_cut(size, (int)Ac.k[seg], (int)Ac.k2[seg]);
                        if (c.kfinal > thresh) acc_reset_all(An, seg);
                        if (size - c.kfinal > thresh) acc_reset_all(An, seg + c.kfinal);
                    }
                }
                unsigned tot;
                const unsigned ex = block_exclusive_scan(f, &tot);
                if (p < c1) {
                    lflag[p] = f;
                    lscan[p] = run + ex;
                }
                run += tot;
            }
            if (threadIdx.x == 0) co.btot[blockIdx.x] = run;
        }
        grid_barrier(co);
        // (D) chunk offsets (every block scans them), stable partition, and the
        // children's boxes and sums for the next round
        {
            unsigned run = 0;
            for (int base = 0; base < G; base += COOP_THREADS) {
                const int j = base + threadIdx.x;
                const unsigned v = j < G ? __ldcg(&co.btot[j]) : 0u;
                unsigned tot;
                const unsigned ex = block_exclusive_scan(v, &tot);
                if (j < G) s_off[j] = run + ex;
                run += tot;
            }
            __syncthreads();
        }
        for (int p0 = 0; p0 < M; p0 += gstride) {
            const int p = p0 + gtid;
            bool act = false;
            int np = 0, nlo = 0, nhi = 0;
            int4 q = make_int4(0, 0, 0, 0);
            if (p < M) {
                const int seg = lc[p], end = hc[p], size = end - seg;
                np = p;
                nlo = seg;
                nhi = end;
                const unsigned e = sc[p];
                if (size > thresh) {
                    const Cut c = make_cut(size, (int)Ac.k[seg], (int)Ac.k2[seg]);
                    const unsigned gp = s_off[p / chunk] + lscan[p];
                    const unsigned gs = s_off[seg / chunk] + lscan[seg];
                    const int before = (int)(gp - gs);  // low items before p in this segment
                    if (lflag[p]) {
                        np = seg + before;
                        nhi = seg + c.kfinal;
                    } else {
                        np = seg + c.kfinal + ((p - seg) - before);
                        nlo = seg + c.kfinal;
                    }
                    act = nhi - nlo > thresh;
                    if (act) {
                        atomicMax(&co.maxseg[r % 3], nhi - nlo);
                        q = xi[e];
                    }
                }
                sn[np] = e;
                ln[np] = nlo;
                hn[np] = nhi;
            }
            accumulate_box_sum(act, nlo, q, An);
        }
        grid_barrier(co);
        cur ^= 1;
        // one decision per block (thread 0 reads, everyone follows), so that no
        // thread leaves the loop while the rest of its block waits at a barrier
        if (threadIdx.x == 0)
            s_stop = (*((volatile int*)&co.maxseg[r % 3]) <= thresh || *((volatile int*)co.err)) ? 1 : 0;
        __syncthreads();
        const int stop = s_stop;
        ++r;
        if (stop) break;
    }
    if (cur == 1)  // leave the result in buffer 0 (the end of the kernel orders this)
        for (int p = gtid; p < M; p += gstride) {
            set0[p] = set1[p];
            lo0[p] = lo1[p];
            hi0[p] = hi1[p];
        }
    if (gtid == 0) {
        *co.rounds = r;
        if (*((volatile int*)&co.maxseg[(r + 2) % 3]) > thresh) atomicOr(co.err, 2);
    }
}

// ---- segments of at most TREE_BLOCK: one block per window of TREE_BLOCK slots
//
// The block takes every segment that starts in its window (at most
// 2 TREE_BLOCK - 1 slots) into shared memory and cuts, level by level with
// block barriers, every segment larger than TREE_WARP.  Open segments are
// larger than TREE_WARP, so their starts are more than TREE_WARP slots apart
// and start / TREE_WARP indexes their accumulators without collisions.

constexpr int TREE_BLOCK = 1024;
constexpr int BLK_CAP = 2 * TREE_BLOCK;         // slots one block can hold
constexpr int BLK_ACC = BLK_CAP / TREE_WARP;    // accumulator entries

struct BlockSmem {
    int4 Q[2][BLK_CAP];         // (x, y, z, particle index), two buffers
    short Lo[2][BLK_CAP], Hi[2][BLK_CAP];
    unsigned F[BLK_CAP];        // low flags
    unsigned S[BLK_CAP];        // their exclusive prefix over the block's slots
    // per open segment, 32-bit only (shared-memory atomics stay native)
    int mn[BLK_ACC][3], mx[BLK_ACC][3];
    unsigned sh[BLK_ACC][3], sl[BLK_ACC][3];  // coordinate sums: high 15-bit parts and low parts
    unsigned k[BLK_ACC], k2[BLK_ACC];
    int vk[BLK_ACC][4];         // largest x below (<), smallest above, largest below (<=), smallest above
    unsigned ik[BLK_ACC][4];    // the index that breaks the tie among those x
    unsigned wsum[TREE_BLOCK / 32];
    int range_lo, range_hi, any;
};

__device__ __forceinline__ int blk_axis(const BlockSmem& S, int e)
{
    return axis_of(S.mx[e][0] - S.mn[e][0], S.mx[e][1] - S.mn[e][1], S.mx[e][2] - S.mn[e][2]);
}

__device__ __forceinline__ long long blk_com(const BlockSmem& S, int e, int ax, int size)
{
    const unsigned long long sum = ((unsigned long long)S.sh[e][ax] << 15) + S.sl[e][ax];
    return (long long)(sum / (unsigned long long)size);
}

__global__ void __launch_bounds__(TREE_BLOCK)
    k_tree_block(int M, unsigned int* __restrict__ set, int* __restrict__ glo, int* __restrict__ ghi,
                 const int4* __restrict__ xi, int* err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BlockSmem& S = *reinterpret_cast<BlockSmem*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int w0 = blockIdx.x * TREE_BLOCK, w1 = min(M, w0 + TREE_BLOCK);
    if (tid == 0) {
        S.range_lo = INT_MAX;
        S.range_hi = INT_MIN;
    }
    __syncthreads();
    {
        const int p = w0 + tid;
        if (p < w1 && glo[p] == p) {
            atomicMin(&S.range_lo, p);
            atomicMax(&S.range_hi, ghi[p]);
        }
    }
    __syncthreads();
    const int base = S.range_lo, n = S.range_hi - S.range_lo;
    if (base == INT_MAX || n <= 0) return;
    if (n > BLK_CAP) {  // a segment larger than TREE_BLOCK reached this kernel
        if (tid == 0) atomicOr(err, 2);
        return;
    }
    for (int q = tid; q < n; q += TREE_BLOCK) {
        const unsigned e = set[base + q];
        const int4 v = xi[e];
        S.Q[0][q] = make_int4(v.x, v.y, v.z, (int)e);
        S.Lo[0][q] = (short)(glo[base + q] - base);
        S.Hi[0][q] = (short)(ghi[base + q] - base);
    }
    int cur = 0;
    for (int level = 0; level < 4 * BLK_CAP; ++level) {
        // accumulators of this level
        for (int e = tid; e < BLK_ACC; e += TREE_BLOCK) {
            for (int a = 0; a < 3; ++a) {
                S.mn[e][a] = INT_MAX;
                S.mx[e][a] = INT_MIN;
                S.sh[e][a] = S.sl[e][a] = 0u;
            }
            S.k[e] = S.k2[e] = 0u;
            S.vk[e][0] = S.vk[e][2] = -1;
            S.vk[e][1] = S.vk[e][3] = INT_MAX;
            S.ik[e][0] = S.ik[e][2] = 0u;
            S.ik[e][1] = S.ik[e][3] = 0xffffffffu;
        }
        if (tid == 0) S.any = 0;
        __syncthreads();
        // bounding boxes and coordinate sums
        for (int q0 = 0; q0 < BLK_CAP; q0 += TREE_BLOCK) {
            const int q = q0 + tid;
            bool act = false;
            int seg = 0;
            int4 v = make_int4(0, 0, 0, 0);
            if (q < n) {
                seg = S.Lo[cur][q];
                act = S.Hi[cur][q] - seg > TREE_WARP;
                v = S.Q[cur][q];
            }
            const unsigned peers = seg_peers(act, seg);
            if (act) {
                const int e = seg / TREE_WARP;
                const int mnx = __reduce_min_sync(peers, v.x), mny = __reduce_min_sync(peers, v.y),
                          mnz = __reduce_min_sync(peers, v.z);
                const int mxx = __reduce_max_sync(peers, v.x), mxy = __reduce_max_sync(peers, v.y),
                          mxz = __reduce_max_sync(peers, v.z);
                const unsigned hx = __reduce_add_sync(peers, (unsigned)v.x >> 15),
                               lx = __reduce_add_sync(peers, (unsigned)v.x & 0x7fffu);
                const unsigned hy = __reduce_add_sync(peers, (unsigned)v.y >> 15),
                               ly = __reduce_add_sync(peers, (unsigned)v.y & 0x7fffu);
                const unsigned hz = __reduce_add_sync(peers, (unsigned)v.z >> 15),
                               lz = __reduce_add_sync(peers, (unsigned)v.z & 0x7fffu);
                if (seg_leader(peers)) {
                    atomicMin(&S.mn[e][0], mnx);
                    atomicMin(&S.mn[e][1], mny);
                    atomicMin(&S.mn[e][2], mnz);
                    atomicMax(&S.mx[e][0], mxx);
                    atomicMax(&S.mx[e][1], mxy);
                    atomicMax(&S.mx[e][2], mxz);
                    atomicAdd(&S.sh[e][0], hx);
                    atomicAdd(&S.sl[e][0], lx);
                    atomicAdd(&S.sh[e][1], hy);
                    atomicAdd(&S.sl[e][1], ly);
                    atomicAdd(&S.sh[e][2], hz);
                    atomicAdd(&S.sl[e][2], lz);
                }
            }
        }
        __syncthreads();
        // counts below the centre of mass and the extreme coordinates on either side
        for (int q0 = 0; q0 < BLK_CAP; q0 += TREE_BLOCK) {
            const int q = q0 + tid;
            bool act = false, blt = false, ble = false;
            int seg = 0, v = 0;
            if (q < n) {
                seg = S.Lo[cur][q];
                const int size = S.Hi[cur][q] - seg;
                act = size > TREE_WARP;
                if (act) {
                    const int e = seg / TREE_WARP;
                    const int ax = blk_axis(S, e);
                    const long long com = blk_com(S, e, ax, size);
                    v = comp(S.Q[cur][q], ax);
                    blt = v < com;
                    ble = v <= com;
                }
            }
            const unsigned peers = seg_peers(act, seg);
            if (act) {
                const int e = seg / TREE_WARP;
                const unsigned clt = __reduce_add_sync(peers, blt ? 1u : 0u);
                const unsigned cle = __reduce_add_sync(peers, ble ? 1u : 0u);
                const int v0 = __reduce_max_sync(peers, blt ? v : -1);
                const int v1 = __reduce_min_sync(peers, !blt ? v : INT_MAX);
                const int v2 = __reduce_max_sync(peers, ble ? v : -1);
                const int v3 = __reduce_min_sync(peers, !ble ? v : INT_MAX);
                if (seg_leader(peers)) {
                    atomicAdd(&S.k[e], clt);
                    atomicAdd(&S.k2[e], cle);
                    atomicMax(&S.vk[e][0], v0);
                    atomicMin(&S.vk[e][1], v1);
                    atomicMax(&S.vk[e][2], v2);
                    atomicMin(&S.vk[e][3], v3);
                }
            }
        }
        __syncthreads();
        // where the cut moves by one particle: the index among the extreme coordinates
        for (int q0 = 0; q0 < BLK_CAP; q0 += TREE_BLOCK) {
            const int q = q0 + tid;
            bool act = false, pick = false;
            int seg = 0, slot = 0;
            unsigned idx = 0;
            if (q < n) {
                seg = S.Lo[cur][q];
                const int size = S.Hi[cur][q] - seg;
                if (size > TREE_WARP) {
                    const int e = seg / TREE_WARP;
                    const Cut c = make_cut(size, (int)S.k[e], (int)S.k2[e]);
                    if (!c.coincident && c.kfinal != c.k) {
                        act = true;
                        const int ax = blk_axis(S, e);
                        const long long com = blk_com(S, e, ax, size);
                        const int4 t = S.Q[cur][q];
                        const int v = comp(t, ax);
                        const bool pl = c.use_le ? v <= com : v < com;
                        slot = (c.use_le ? 2 : 0) + (c.kfinal < c.k ? 0 : 1);
                        pick = (c.kfinal < c.k ? pl : !pl) && v == S.vk[e][slot];
                        idx = (unsigned)t.w;
                    }
                }
            }
            // the slot is a property of the segment, so peers share it
            const unsigned peers = seg_peers(act, seg);
            if (act) {
                const int e = seg / TREE_WARP;
                // lanes without a pick give the identity, so an empty group changes nothing
                if ((slot & 1) == 0) {
                    const unsigned im = __reduce_max_sync(peers, pick ? idx : 0u);
                    if (seg_leader(peers)) atomicMax(&S.ik[e][slot], im);
                } else {
                    const unsigned im = __reduce_min_sync(peers, pick ? idx : 0xffffffffu);
                    if (seg_leader(peers)) atomicMin(&S.ik[e][slot], im);
                }
            }
        }
        __syncthreads();
        // low flags
        for (int q = tid; q < BLK_CAP; q += TREE_BLOCK) {
            unsigned f = 0;
            if (q < n) {
                const int seg = S.Lo[cur][q], size = S.Hi[cur][q] - seg;
                if (size > TREE_WARP) {
                    const int e = seg / TREE_WARP;
                    const Cut c = make_cut(size, (int)S.k[e], (int)S.k2[e]);
                    if (c.coincident) {
                        f = (q - seg) < c.kfinal;  // segments keep ascending index order
                    } else {
                        const int ax = blk_axis(S, e);
                        const long long com = blk_com(S, e, ax, size);
                        const int4 t = S.Q[cur][q];
                        const int v = comp(t, ax);
                        bool left = c.use_le ? v <= com : v < com;
                        const int kk = c.use_le ? 2 : 0;
                        if (c.kfinal < c.k && v == S.vk[e][kk] && (unsigned)t.w == S.ik[e][kk])
                            left = false;
                        if (c.kfinal > c.k && v == S.vk[e][kk + 1] && (unsigned)t.w == S.ik[e][kk + 1])
                            left = true;
                        f = left;
                    }
                }
            }
            S.F[q] = f;
        }
        __syncthreads();
        // exclusive prefix of the flags: two consecutive slots per thread
        {
            const unsigned a0 = S.F[2 * tid], a1 = S.F[2 * tid + 1];
            const unsigned run = a0 + a1;
            unsigned incl = run;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane == 31) S.wsum[wid] = incl;
            __syncthreads();
            unsigned ex = incl - run;
            for (int w = 0; w < wid; ++w) ex += S.wsum[w];
            S.S[2 * tid] = ex;
            S.S[2 * tid + 1] = ex + a0;
        }
        __syncthreads();
        // stable partition of every open segment into the other buffer
        const int nx = cur ^ 1;
        for (int q = tid; q < n; q += TREE_BLOCK) {
            const int seg = S.Lo[cur][q], end = S.Hi[cur][q], size = end - seg;
            int np = q, nlo = seg, nhi = end;
            if (size > TREE_WARP) {
                const int e = seg / TREE_WARP;
                const Cut c = make_cut(size, (int)S.k[e], (int)S.k2[e]);
                const int before = (int)(S.S[q] - S.S[seg]);  // low slots in [seg, q)
                if (S.F[q]) {
                    np = seg + before;
                    nhi = seg + c.kfinal;
                } else {
                    np = seg + c.kfinal + ((q - seg) - before);
                    nlo = seg + c.kfinal;
                }
                if (nhi - nlo > TREE_WARP) S.any = 1;
            }
            if (np >= 0 && np < n) {  // always true for a consistent cut
                S.Q[nx][np] = S.Q[cur][q];
                S.Lo[nx][np] = (short)nlo;
                S.Hi[nx][np] = (short)nhi;
            }
        }
        __syncthreads();
        cur = nx;
        if (!S.any) break;
        __syncthreads();
    }
    for (int q = tid; q < n; q += TREE_BLOCK) {
        set[base + q] = (unsigned)S.Q[cur][q].w;
        glo[base + q] = base + S.Lo[cur][q];
        ghi[base + q] = base + S.Hi[cur][q];
    }
}

// ---- segments of at most TREE_WARP: one warp each, one particle per lane
//
// The same cut as the rounds above, with the segment in registers: warp
// reductions over the lanes of each open sub-segment, the stable partition by
// ballot ranks, and an exchange through shared memory.

__global__ void __launch_bounds__(128)
    k_tree_warp(int M, const int4* __restrict__ xi, unsigned int* __restrict__ set,
                int* __restrict__ glo, int* __restrict__ ghi)
{
    __shared__ int4 xbuf[4][32];
    __shared__ int2 bbuf[4][32];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int nwin = (M + 31) / 32;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int win = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; win < nwin; win += nwarps) {
        const int p = win * 32 + lane;
        const bool start = p < M && glo[p] == p && ghi[p] - p > 2;
        unsigned sm = __ballot_sync(FULL, start);
        while (sm) {
            const int src = __ffs(sm) - 1;
            sm &= sm - 1;
            const int base = win * 32 + src;
            const int s = min(ghi[base] - base, TREE_WARP);
            const bool own = lane < s;
            unsigned idx = own ? set[base + lane] : 0u;
            int4 q = own ? xi[idx] : make_int4(0, 0, 0, 0);
            int slo = 0, shi = s;
            for (int round = 0; round < TREE_WARP; ++round) {
                const int size = shi - slo;
                const bool act = own && size > 2;
                if (!__any_sync(FULL, act)) break;
                const unsigned peers = seg_peers(act, slo);
                int np = lane, nlo = slo, nhi = shi;
                if (act) {
                    const int mn0 = __reduce_min_sync(peers, q.x), mx0 = __reduce_max_sync(peers, q.x);
                    const int mn1 = __reduce_min_sync(peers, q.y), mx1 = __reduce_max_sync(peers, q.y);
                    const int mn2 = __reduce_min_sync(peers, q.z), mx2 = __reduce_max_sync(peers, q.z);
                    const int ax = axis_of(mx0 - mn0, mx1 - mn1, mx2 - mn2);
                    const int v = comp(q, ax);
                    const unsigned sh = __reduce_add_sync(peers, (unsigned)v >> 15);
                    const unsigned sl = __reduce_add_sync(peers, (unsigned)v & 0x7fffu);
                    const unsigned long long sum = ((unsigned long long)sh << 15) + sl;
                    const long long com = (long long)(sum / (unsigned long long)size);
                    const bool blt = v < com, ble = v <= com;
                    const int klt = (int)__reduce_add_sync(peers, blt ? 1u : 0u);
                    const int kle = (int)__reduce_add_sync(peers, ble ? 1u : 0u);
                    const Cut c = make_cut(size, klt, kle);
                    bool low;
                    if (c.coincident) {
                        low = (lane - slo) < c.kfinal;  // lanes hold ascending index order
                    } else {
                        const bool pl = c.use_le ? ble : blt;
                        low = pl;
                        const unsigned long long key = ((unsigned long long)v << 32) | idx;
                        if (c.kfinal < c.k && key == warp_max_key(peers, pl, v, idx)) low = false;
                        if (c.kfinal > c.k && key == warp_min_key(peers, !pl, v, idx)) low = true;
                    }
                    const unsigned lm = __ballot_sync(peers, low) & peers;
                    if (low) {
                        np = slo + __popc(lm & lt);
                        nhi = slo + c.kfinal;
                    } else {
                        np = slo + c.kfinal + __popc(~lm & peers & lt);
                        nlo = slo + c.kfinal;
                    }
                }
                __syncwarp();
                if (own && np >= 0 && np < TREE_WARP) {  // always true for a consistent cut
                    xbuf[w][np] = make_int4(q.x, q.y, q.z, (int)idx);
                    bbuf[w][np] = make_int2(nlo, nhi);
                }
                __syncwarp();
                if (own) {
                    const int4 t = xbuf[w][lane];
                    q = make_int4(t.x, t.y, t.z, 0);
                    idx = (unsigned)t.w;
                    const int2 b = bbuf[w][lane];
                    slo = b.x;
                    shi = b.y;
                }
                __syncwarp();
            }
            if (own) {
                set[base + lane] = idx;
                glo[base + lane] = base + slo;
                ghi[base + lane] = base + shi;
            }
            __syncwarp();
        }
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
    p.flags[a] = p.flags[a] | APR_FLAG_CHANGED | APR_FLAG_NEW;
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
    if (maxm > TREE_BLOCK) {
        if (c->coop_blocks <= 0) {
            int per_sm = 0, nsm = 0;
            s = cuda_check(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tree_rounds,
                                                                            COOP_THREADS, 0),
                           "pairing tree occupancy");
            if (s != APR_OK) return s;
            s = cuda_check(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device),
                           "SM count");
            if (s != APR_OK) return s;
            c->coop_blocks = min(per_sm * nsm, COOP_MAX_BLOCKS);
            if (c->coop_blocks <= 0) return fail(c, APR_ERR_CUDA, "pairing tree: no resident block");
        }
        const int grid = max(1, min(c->coop_blocks, (M + COOP_THREADS - 1) / COOP_THREADS));
        Coop co;
        co.btot = W.coop;
        co.bar = W.coop + 2 * COOP_MAX_BLOCKS;
        co.maxseg = (int*)(co.bar + 2);
        co.rounds = co.maxseg + 3;
        co.err = &W.status[ST_TREE_ERR];
        cudaMemsetAsync(co.bar, 0, sizeof(unsigned) * 8, st);
        cudaMemsetAsync(co.err, 0, sizeof(int), st);
        int M_ = M, thresh = TREE_BLOCK, max_rounds = 64 + 4 * 32;
        void* args[] = {&M_, &thresh, &max_rounds, (void*)&W.xi, (void*)&sets[0], (void*)&sets[1],
                        (void*)&W.seg_lo[0], (void*)&W.seg_lo[1], (void*)&W.seg_hi[0],
                        (void*)&W.seg_hi[1], (void*)&acc[0], (void*)&acc[1], (void*)&W.lflag,
                        (void*)&W.uscan, (void*)&co};
        ++c->launches;
        s = cuda_check(c, cudaLaunchCooperativeKernel((const void*)k_tree_rounds, dim3(grid),
                                                      dim3(COOP_THREADS), args, 0, st),
                       "pairing tree rounds");
        if (s != APR_OK) return s;
    }
    // the rounds leave their result in buffer 0
    if (maxm > TREE_WARP) {
        if (!c->tree_smem_set) {
            s = cuda_check(c, cudaFuncSetAttribute(k_tree_block,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)sizeof(BlockSmem)), "tree smem");
            if (s != APR_OK) return s;
            c->tree_smem_set = true;
        }
        APR_LAUNCH_SMEM(c, k_tree_block, (M + TREE_BLOCK - 1) / TREE_BLOCK, TREE_BLOCK,
                        sizeof(BlockSmem), M, sets[0], W.seg_lo[0], W.seg_hi[0], W.xi,
                        &W.status[ST_TREE_ERR]);
    }
    APR_LAUNCH(c, k_tree_warp, min(nblocks((long long)((M + 31) / 32) * 32, 128), 152 * 16), 128, M,
               W.xi, sets[0], W.seg_lo[0], W.seg_hi[0]);
    *set_out = sets[0];
    *lo_out = W.seg_lo[0];
    *hi_out = W.seg_hi[0];
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
    int terr = 0;
    s = cuda_check(c, cudaMemcpyAsync(buf.data(), dev, sizeof(long long) * m, cudaMemcpyDeviceToHost,
                                      c->stream), "pairs out");
    if (s != APR_OK) return s;
    cudaMemcpyAsync(&terr, &c->W.status[ST_TREE_ERR], sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    s = cuda_check(c, cudaStreamSynchronize(c->stream), "pairs out");
    if (s != APR_OK) return s;
    if (terr) return fail(c, APR_ERR_STATE, "pairing tree: a grid barrier timed out");
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
    unsigned char* bin;  // may be null
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
    f.bin = p.bin;
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
    if (f.bin) b[2 * cap + j] = f.bin[i];
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
    if (f.bin) f.bin[j] = b[2 * cap + j];
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
    c->order_valid = false;
    return cuda_check(c, cudaGetLastError(), "compaction");
}

// every field of the particle in canonical slot perm[j] to position j of the scratch:
// scattered reads, coalesced writes; k_compact_back then writes the fields back in order
__global__ void k_reorder_out(long long n, long long cap, FieldPtrs f,
                              const unsigned int* __restrict__ perm, double* __restrict__ tmp)
{
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const long long i = perm[j];
    for (int k = 0; k < 18; ++k) tmp[k * cap + j] = f.d[k][i];
    ((unsigned long long*)(tmp + 18 * cap))[j] = f.id[i];
    unsigned char* b = (unsigned char*)(tmp + 19 * cap);
    b[j] = f.level[i];
    b[cap + j] = f.flags[i];
    if (f.bin) b[2 * cap + j] = f.bin[i];
}

__global__ void k_iota(long long n, unsigned int* __restrict__ out)
{
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = (unsigned int)j;
}

// The bound arrays permuted into the index's Morton order.  The sorted order, the
// radix tree over it and the force records keep their meaning (slot j now holds
// canonical particle j), so the kept order stays valid with the identity as its
// permutation and every later gather through it reads consecutive addresses.
apr_status reorder(apr_ctx* c)
{
    const long long n = c->n;
    if (n < 2) return APR_OK;
    if (!(c->order_valid && c->order_n == n)) {
        apr_status s = index_sort(c);
        if (s != APR_OK) return s;
    }
    Workspace& W = c->W;
    const FieldPtrs f = field_ptrs(c->p);
    double* tmp = (double*)W.nbr;  // 20 x cap x 8 bytes <= the list memory
    APR_LAUNCH(c, k_reorder_out, nblocks(n, 256), 256, n, c->cap, f, W.perm_keep, tmp);
    APR_LAUNCH(c, k_compact_back, nblocks(n, 256), 256, n, c->cap, f, tmp);
    APR_LAUNCH(c, k_iota, nblocks(n, 256), 256, n, W.perm_keep);
    W.perm = W.perm_keep;
    c->lists_fresh = false;  // the scratch overwrote them
    c->force_data_fresh = false;
    return cuda_check(c, cudaGetLastError(), "reorder");
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

// The split/merge pass may skip its sorts, pairing trees and compaction when it
// provably changes nothing (see split_merge_body).  That needs one zone of the
// refinement kind (the set a level asks for is then the convex inside of one
// boundary) and midpoints that are formed without a periodic wrap across the zone:
// on every periodic axis the zone constrains, the zone lies inside the box and
// two points inside it are closer than half the box; coordinates at most 1e6
// times the innermost radius keep a midpoint's rounding far below the 1e-8 inset.
static bool merge_shortcut_ok(const apr_ctx* c)
{
    if (c->nreg != 1 || c->cfg.level_default != 0 || c->cfg.lmax < 1) return false;
    const apr_region& r = c->regions[0];
    if (r.nlev < 1 || r.nlev > APR_MAXLEV) return false;
    double Rout = 0.0, Rin = INFINITY;
    for (int k = 0; k < r.nlev; ++k) {
        Rout = std::max(Rout, r.R[k]);
        Rin = std::min(Rin, r.R[k]);
    }
    if (!(Rin > 0.0)) return false;
    bool axes[3] = {true, true, true};
    if (r.shape == APR_SHAPE_SLAB) {
        for (int k = 0; k < 3; ++k) axes[k] = k == r.axis;
    } else if (r.shape == APR_SHAPE_CYLINDER) {
        axes[r.axis] = false;
    } else if (r.shape != APR_SHAPE_SPHERE) {
        return false;
    }
    for (int k = 0; k < 3; ++k) {
        const double lo = c->cfg.box_lo[k], hi = c->cfg.box_hi[k];
        if (std::max(std::fabs(lo), std::fabs(hi)) > 1e6 * Rin) return false;
        if (axes[k] && c->cfg.periodic[k] &&
            (r.centre[k] - Rout < lo || r.centre[k] + Rout > hi || 4.0 * Rout >= hi - lo))
            return false;
    }
    return true;
}

// host words for the merge counts and the pairing-tree status, apart from the
// words the compaction count uses
static int* merge_hbuf(apr_ctx* c) { return (int*)c->hbuf + 512; }

static apr_status split_merge_body(apr_ctx* c, apr_counts* cnt)
{
    Workspace& W = c->W;
    cudaStream_t st = c->stream;
    const DevRegions rg = dev_regions(c);
    memset(cnt, 0, sizeof(*cnt));
    apr_status s;
    bool merged = false;
    if (c->n > 0) APR_LAUNCH(c, k_clear_changed, nblocks(c->n, 256), 256, c->n, c->p.flags);
    if (c->cfg.lmax >= 1 && c->n > 0) {
        const long long n = c->n;
        // the summary costs a host synchronisation: read it while passes keep being
        // quiet, else only every eighth pass (a busy zone rarely turns quiet)
        const bool shortcut = merge_shortcut_ok(c) && (c->quiet_pass || c->step % 8 == 0);
        int* sm = &W.status[ST_SM_NSPLIT];
        cudaMemsetAsync(sm, 0, sizeof(int) * (2 + APR_MAXLEV), st);
        APR_LAUNCH(c, k_split_keys, nblocks(n, 256), 256, c->dc, rg, n, c->p.x, c->p.y, c->p.z,
                   c->p.level, c->p.flags, W.key[0], W.val[0], shortcut ? 1 : 0, sm);
        int nsplit = -1;  // unknown until read
        if (shortcut) {
            // the pass's summary first: a pass with nothing to split, no dead particle
            // and every merge candidate safely inside its (convex) zone changes nothing
            // (a pair's centre of mass lies inside a convex zone with both particles),
            // so the sort by level, the pairing trees and the compaction are skipped
            cudaMemcpyAsync((int*)c->hbuf + 600, sm, sizeof(int) * (2 + APR_MAXLEV),
                            cudaMemcpyDeviceToHost, st);
            s = cuda_check(c, cudaStreamSynchronize(st), "split/merge summary");
            if (s != APR_OK) return s;
            const int* h = (const int*)c->hbuf + 600;
            nsplit = h[0];
            if (nsplit == 0 && h[1] == 0) {
                for (int l = 1; l <= c->cfg.lmax; ++l) cnt->n_spare[l] = h[2 + l] & 1;
                c->step += 1;
                c->quiet_pass = true;
                return APR_OK;
            }
        }
        c->quiet_pass = false;
        int total = 0;
        if (nsplit != 0) {
            s = radix_pass8(c, W.key[0], W.val[0], W.key[1], W.val[1], n, 0, &W.status[ST_BINS],
                            c->cfg.lmax + 1);
            if (s != APR_OK) return s;
            cudaMemcpyAsync(c->hbuf, &W.status[ST_BINS], sizeof(int) * (c->cfg.lmax + 1),
                            cudaMemcpyDeviceToHost, st);
            s = cuda_check(c, cudaStreamSynchronize(st), "split count");
            if (s != APR_OK) return s;
            const int* bins = (const int*)c->hbuf;  // parents of level l: [bins[l], bins[l+1])
            total = bins[c->cfg.lmax];
            for (int l = 0; l < c->cfg.lmax; ++l) cnt->n_split[l] = bins[l + 1] - bins[l];
        }
        if (n + total > c->cap)
            return fail(c, APR_ERR_CAPACITY, "split would exceed the bound capacity");
        if (total > 0) {
            APR_LAUNCH(c, k_split_apply, nblocks(total, 256), 256, c->dc, rg, total, n, c->step,
                       c->next_id, W.val[1], c->p);
            c->n = n + total;
            c->next_id += total;
            c->order_valid = false;
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
            // read back with the compaction count below (one host synchronisation)
            cudaMemcpyAsync(merge_hbuf(c), &W.status[ST_MERGES], sizeof(int) * APR_MAXLEV,
                            cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(merge_hbuf(c) + APR_MAXLEV, &W.status[ST_TREE_ERR], sizeof(int),
                            cudaMemcpyDeviceToHost, st);
            merged = true;
        }
    }
    long long removed = 0;
    if (c->n > 0) {
        s = compact(c, &removed);
        if (s != APR_OK) return s;
    }
    if (merged) {
        if (merge_hbuf(c)[APR_MAXLEV])
            return fail(c, APR_ERR_STATE, "pairing tree: a grid barrier timed out or the "
                                          "leaves were not reached");
        for (int l = 1; l <= c->cfg.lmax; ++l) cnt->n_merge[l] = merge_hbuf(c)[l];
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

// blocks of a fixed-shape reduction over n particles: one to eight per SM (the
// same number on every SM, so that none takes twice the FP64 work of another), with
// at least about four particles per thread so that the per-block shuffled sums stay
// a small share of the work
static int red_grid(long long n)
{
    const long long per_sm = std::max<long long>(1, std::min<long long>(8, n / (152LL * 256 * 4)));
    return (int)std::min<long long>(RED_BLOCKS, 152 * per_sm);
}

// one particle's terms of the conservation sums in units of m0 (the host scales
// them): w = 2^-level makes every product with it exact
__device__ __forceinline__ void stats_terms(const DevCfg& dc, const apr_particles& p, long long i,
                                            double w, double vx, double vy, double vz, double* v)
{
    const double mx = w * vx, my = w * vy, mz = w * vz;
    const double x = p.x[i], y = p.y[i], z = p.z[i];
    v[0] += w;
    v[1] += mx;
    v[2] += my;
    v[3] += mz;
    v[4] = fma(-z, my, fma(y, mz, v[4]));
    v[5] = fma(-x, mz, fma(z, mx, v[5]));
    v[6] = fma(-y, mx, fma(x, my, v[6]));
    v[7] = fma(mz, vz, fma(my, vy, fma(mx, vx, v[7])));
    if (dc.eos == APR_EOS_ADIABATIC) v[8] = fma(w, p.u[i], v[8]);
}

// the sums' units: m0 for all, m0 / 2 for the kinetic energy (slot 7)
static void stats_scale(const apr_ctx* c, double* r)
{
    for (int k = 0; k < 9; ++k) r[k] *= k == 7 ? 0.5 * c->dc.m0 : c->dc.m0;
}

__global__ void __launch_bounds__(256) k_stats(DevCfg dc, long long n, apr_particles p,
                                               double* partials)
{
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (p.flags[i] & APR_FLAG_DEAD) continue;
        stats_terms(dc, p, i, level_mass_d(p.level[i]), p.vx[i], p.vy[i], p.vz[i], v);
    }
    block_reduce_store<9>(v, partials);
}

// conservation sums (9) and the time-step limit (slot 9, a minimum) in one pass
// hdt != 0: first the closing half kick of the step (as k_kick), then the sums
__global__ void __launch_bounds__(256) k_stats_dt(DevCfg dc, long long n, apr_particles p,
                                                  double hdt, double* partials)
{
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    DtMin best;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned char fl = p.flags[i];
        if (fl & APR_FLAG_DEAD) continue;
        const double w = level_mass_d(p.level[i]);
        double vx = p.vx[i], vy = p.vy[i], vz = p.vz[i];
        if (hdt != 0.0 && !(fl & APR_FLAG_FIXED)) {
            vx += hdt * p.ax[i];
            vy += hdt * p.ay[i];
            vz += hdt * p.az[i];
            p.vx[i] = vx;
            p.vy[i] = vy;
            p.vz[i] = vz;
            if (dc.eos == APR_EOS_ADIABATIC) p.u[i] += hdt * p.dudt[i];
        }
        stats_terms(dc, p, i, w, vx, vy, vz, v);
        if (fl & APR_FLAG_FIXED) continue;
        best.add_keyed(p.h[i], p.vsig[i], p.ax[i], p.ay[i], p.az[i]);
    }
    __shared__ double sm[10][8];
    __shared__ DtMin sd[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 9; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sm[k][wid] = x;
    }
    for (int o = 16; o > 0; o >>= 1) best.shfl_down(o);
    if (lane == 0) sd[wid] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        DtMin b = sd[0];
        for (int w = 1; w < 8; ++w) b.merge(sd[w]);
        sm[9][0] = b.value(dc);
        for (int w = 1; w < 8; ++w) sm[9][w] = INFINITY;
    }
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

apr_status compute_stats_dt(apr_ctx* c, apr_stats* st, double* dt, double kick_hdt)
{
    // about four particles per thread: enough to hide the loads, few enough blocks
    // that the per-block FP64 reduction (ten shuffled sums) stays small
    const int nblk = red_grid(c->n);
    APR_LAUNCH(c, k_stats_dt, nblk, 256, c->dc, c->n, c->p, kick_hdt, c->W.red);
    double r[10];
    apr_status s = reduce_readback_n(c, nblk, 10, 1u << 9, r);
    if (s != APR_OK) return s;
    stats_scale(c, r);
    stats_from(c, r, st);
    *dt = r[9];
    return APR_OK;
}

apr_status compute_stats(apr_ctx* c, apr_stats* st)
{
    const int nblk = red_grid(c->n);
    APR_LAUNCH(c, k_stats, nblk, 256, c->dc, c->n, c->p, c->W.red);
    double r[9];
    apr_status s = reduce_readback_n(c, nblk, 9, 0u, r);
    if (s != APR_OK) return s;
    stats_scale(c, r);
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
    DtMin best;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (p.flags[i] & (APR_FLAG_DEAD | APR_FLAG_FIXED)) continue;
        best.add(p.h[i], p.vsig[i], p.ax[i] * p.ax[i] + p.ay[i] * p.ay[i] + p.az[i] * p.az[i]);
    }
    __shared__ DtMin sd[8];
    for (int o = 16; o > 0; o >>= 1) best.shfl_down(o);
    if ((threadIdx.x & 31) == 0) sd[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        DtMin b = sd[0];
        for (int w = 1; w < 8; ++w) b.merge(sd[w]);
        partials[blockIdx.x * 32] = b.value(dc);
    }
}

apr_status compute_timestep(apr_ctx* c, double* dt)
{
    const int nblk = red_grid(c->n);
    APR_LAUNCH(c, k_timestep, nblk, 256, c->dc, c->n, c->p, c->W.red);
    return reduce_readback_n(c, nblk, 1, 1u, dt);
}

// ------------------------------------------------------- point masses

// 1 / sqrt(x) in FP64 without a division or a square root (FP64 runs on a narrow
// pipe on this part): the FP32 estimate refined by two Newton steps for
// f(y) = 1/y^2 - x, y <- y (3 - x y^2) / 2, each of which squares the relative
// error (2^-22 -> 2^-44 -> below FP64 rounding); outside the FP32 normal range the
// plain quotient
__device__ __forceinline__ double rsqrt_newton(double x)
{
    if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
    double y = (double)rsqrtf((float)x);
    y = y * (1.5 - 0.5 * x * y * y);
    y = y * (1.5 - 0.5 * x * y * y);
    return y;
}

// every live particle pulls the point masses; with B >= 0 (time-step bins) only
// the particles whose step ends at substep boundary `sub` take their pull.
// NS bounds the number of point masses (the per-block sums are 3 NS wide).  F32
// (the FP32-mixed path): the separation is formed in FP64 and the pull evaluated
// in FP32, like the pair sums; the point masses' sums are compensated in FP32 per
// thread and added in FP64 across threads.
template <int NS, bool F32>
__global__ void __launch_bounds__(256) k_sink_gravity(DevCfg dc, DevSinks sk, long long n,
                                                      apr_particles p, int B, long long sub,
                                                      double* partials)
{
    if constexpr (F32) {
        // the point masses' pull by this thread's particles, compensated in float
        // like the pair sums (the FP64 pipe is narrow on this part); the threads'
        // sums are added in float64
        Acc<float> w[3 * NS];
        const int ns = sk.n < NS ? sk.n : NS;
        const float G = (float)dc.G;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            if (p.flags[i] & APR_FLAG_DEAD) continue;
            // float(m0 2^-level) = float(m0) 2^-level: a power of two scales exactly
            const float mi = dc.m0f * level_mass_f(p.level[i]);
            const bool pulled = B < 0 || sub % ((1LL << B) >> p.bin[i]) == 0;
            float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
            for (int j = 0; j < NS; ++j) {
                if (j >= ns) break;
                const float dx = (float)(p.x[i] - sk.x[j][0]), dy = (float)(p.y[i] - sk.x[j][1]),
                            dz = (float)(p.z[i] - sk.x[j][2]);
                const float r2 = dx * dx + dy * dy + dz * dz;
                const float y = rsqrtf(r2);
                const float f = G * (y * y * y);
                const float fm = f * (float)sk.m[j];
                ax -= fm * dx;
                ay -= fm * dy;
                az -= fm * dz;
                const float fi = f * mi;
                w[3 * j + 0].add(fi * dx);
                w[3 * j + 1].add(fi * dy);
                w[3 * j + 2].add(fi * dz);
            }
            if (pulled) {
                p.ax[i] += (double)ax;
                p.ay[i] += (double)ay;
                p.az[i] += (double)az;
            }
        }
        double v[3 * NS];
        for (int k = 0; k < 3 * NS; ++k) v[k] = (double)w[k].s - (double)w[k].c;
        block_reduce_store<3 * NS>(v, partials);
        return;
    }
    double v[3 * NS];
    for (int k = 0; k < 3 * NS; ++k) v[k] = 0.0;
    const int ns = sk.n < NS ? sk.n : NS;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (p.flags[i] & APR_FLAG_DEAD) continue;
        const double mi = dc.m0 * level_mass_d(p.level[i]);
        const bool pulled = B < 0 || sub % ((1LL << B) >> p.bin[i]) == 0;
        double ax = 0.0, ay = 0.0, az = 0.0;
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            if (j >= ns) break;
            double dx = p.x[i] - sk.x[j][0], dy = p.y[i] - sk.x[j][1], dz = p.z[i] - sk.x[j][2];
            double r2 = dx * dx + dy * dy + dz * dz;
            const double y = rsqrt_newton(r2);
            double f = dc.G * (y * y * y);
            ax -= f * sk.m[j] * dx;
            ay -= f * sk.m[j] * dy;
            az -= f * sk.m[j] * dz;
            v[3 * j + 0] += f * mi * dx;
            v[3 * j + 1] += f * mi * dy;
            v[3 * j + 2] += f * mi * dz;
        }
        if (pulled) {
            p.ax[i] += ax;
            p.ay[i] += ay;
            p.az[i] += az;
        }
    }
    block_reduce_store<3 * NS>(v, partials);
}

apr_status sink_gravity(apr_ctx* c, int B, long long sub)
{
    if (c->nsink == 0) return APR_OK;
    const int nblk = red_grid(c->n);
    const bool f32 = c->cfg.precision == APR_PREC_FP32_MIXED;
#define APR_SINKS(NS, F)                                                                             \
    APR_LAUNCH(c, (k_sink_gravity<NS, F>), nblk, 256, c->dc, dev_sinks(c), c->n, c->p, B, sub, c->W.red)
    if (c->nsink <= 2) {
        if (f32) APR_SINKS(2, true);
        else APR_SINKS(2, false);
    } else {
        if (f32) APR_SINKS(APR_MAXSINK, true);
        else APR_SINKS(APR_MAXSINK, false);
    }
#undef APR_SINKS
    double r[3 * APR_MAXSINK];
    apr_status s = reduce_readback_n(c, nblk, 3 * c->nsink, 0u, r);
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
    // a particle certainly outside every accretion radius by the float pre-test
    // (SinkPre) needs no float64 test
    SinkPre pre[APR_MAXSINK];
    const int ns = sk.n < APR_MAXSINK ? sk.n : APR_MAXSINK;
    for (int j = 0; j < ns; ++j) pre[j].set(sk.x[j], sk.racc[j]);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (p.flags[i] & (APR_FLAG_DEAD | APR_FLAG_FIXED)) continue;
        const float xf = (float)p.x[i], yf = (float)p.y[i], zf = (float)p.z[i];
        bool near = false;
        for (int j = 0; j < ns; ++j) near = near || pre[j].maybe_inside(xf, yf, zf);
        if (!near) continue;
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
    // 7 per sink, at most 4 sinks per reduction slot set of 32; a block that absorbed
    // nothing stores zeros without the shuffled sums (the usual case)
    if (!__syncthreads_or(cnt)) {
        if (threadIdx.x < 28) partials[blockIdx.x * 32 + threadIdx.x] = 0.0;
        return;
    }
    block_reduce_store<28>(*reinterpret_cast<double(*)[28]>(v), partials);
}

apr_status accrete(apr_ctx* c, long long* naccreted)
{
    *naccreted = 0;
    if (c->nsink == 0 || c->n == 0) return APR_OK;
    if (c->nsink > 4) return fail(c, APR_ERR_ARG, "accretion supports at most 4 sinks");
    cudaMemsetAsync(&c->W.status[ST_COUNT_B], 0, sizeof(int), c->stream);
    const int nblk = red_grid(c->n);
    APR_LAUNCH(c, k_accrete, nblk, 256, c->dc, dev_sinks(c), c->n, c->p, c->W.red,
               &c->W.status[ST_COUNT_B]);
    // the sums and the count in one read-back
    APR_LAUNCH(c, k_reduce_final, 1, 256, nblk, 7 * c->nsink, c->W.red, c->W.redout, 0u);
    cudaMemcpyAsync(c->hbuf, c->W.redout, sizeof(double) * 7 * c->nsink, cudaMemcpyDeviceToHost,
                    c->stream);
    cudaMemcpyAsync((double*)c->hbuf + 28, &c->W.status[ST_COUNT_B], sizeof(int),
                    cudaMemcpyDeviceToHost, c->stream);
    apr_status s = cuda_check(c, cudaStreamSynchronize(c->stream), "accrete");
    if (s != APR_OK) return s;
    double r[28];
    memcpy(r, c->hbuf, sizeof(double) * 7 * c->nsink);
    *naccreted = *(const int*)((const double*)c->hbuf + 28);
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

// the opening half kick and the drift of one global step in one pass (as k_kick
// then k_drift)
__global__ void k_kick_drift(DevCfg dc, long long n, double hdt, double dt, apr_particles p)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (p.flags[i] & (APR_FLAG_FIXED | APR_FLAG_DEAD))) return;
    const double vx = p.vx[i] + hdt * p.ax[i], vy = p.vy[i] + hdt * p.ay[i],
                 vz = p.vz[i] + hdt * p.az[i];
    p.vx[i] = vx;
    p.vy[i] = vy;
    p.vz[i] = vz;
    if (dc.eos == APR_EOS_ADIABATIC) p.u[i] += hdt * p.dudt[i];
    p.x[i] = wrap1(dc, 0, p.x[i] + dt * vx);
    p.y[i] = wrap1(dc, 1, p.y[i] + dt * vy);
    p.z[i] = wrap1(dc, 2, p.z[i] + dt * vz);
}

apr_status kick_drift(apr_ctx* c, double hdt, double dt)
{
    if (c->n > 0) APR_LAUNCH(c, k_kick_drift, nblocks(c->n, 256), 256, c->dc, c->n, hdt, dt, c->p);
    for (int j = 0; j < c->nsink; ++j)
        for (int d = 0; d < 3; ++d) {
            c->sinks[j].v[d] += hdt * c->sinks[j].a[d];
            c->sinks[j].x[d] += dt * c->sinks[j].v[d];
        }
    return cuda_check(c, cudaGetLastError(), "kick and drift");
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

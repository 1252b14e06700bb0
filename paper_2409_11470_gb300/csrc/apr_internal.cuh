// Internal declarations of the GB300 APR SPH library: device configuration,
// the opaque context, the workspace layout and small device helpers shared by
// the translation units.  Nothing here is part of the C ABI (include/apr.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <string>

#include "apr.h"

namespace apr {

constexpr int COORD_BITS = 30;               // lattice coordinates are in [0, 2^30)
constexpr long long COORD_MAX = (1LL << COORD_BITS) - 1;
constexpr int CELL_MAX = 32;                 // particles per cell (one warp)
constexpr int KEY_BITS = 16;                 // Morton key bits per axis (48-bit keys, 6 passes)
// candidate cells per cell: 128, or 256 for runs with neighbour lists longer than
// the default (discs, whose sparse vertical tails have large h: more of their cells
// keep their candidates instead of falling back to per-particle tree walks; on the
// uniform shock tube 256 cost 11% of the list time, on the flyby it saved 6%)
constexpr int MAX_CAND_SMALL = 128, MAX_CAND_LARGE = 256;
constexpr int RADIX_TILE = 2048;             // items per radix-sort block (256 x 8)
constexpr int SORT_SWEEP_MAX_TILES = 256;     // Morton sort: single-sweep passes up to this many tiles
constexpr int SCAN_BLOCK = 1024;             // items per scan block (256 x 4)
constexpr int RED_BLOCKS = 1216;             // 8 x 152 SMs: fixed-shape f64 reductions
constexpr int DEFAULT_MAX_NEIGH = 512;
inline int max_cand_of(int max_neigh)
{
    return max_neigh > DEFAULT_MAX_NEIGH ? MAX_CAND_LARGE : MAX_CAND_SMALL;
}
// density lists cover r < 2 * 1.06 * h: room for the h-rho iteration to grow h by 6%
// without a new list (a particle whose root lies farther is retried with a list at
// its new h); 1.06 measured faster than 1.125 (fewer list entries for the density and
// force passes to skip) and than 1.03 (more retries) on the tube and both discs
constexpr float DENSITY_REACH = 1.06f;

// status words written by kernels (device, read back by the host)
enum {
    ST_NEIGH_OVERFLOW = 0,   // a particle's list exceeded max_neigh
    ST_CAND_OVERFLOW = 1,    // a cell's candidate list exceeded max_cand
    ST_UNCOVERED = 2,        // density: h grew beyond the list's reach
    ST_NOCONV = 3,           // density: Newton-Raphson not converged
    ST_COUNT_A = 4,          // generic counters for split/merge passes
    ST_COUNT_B = 5,
    ST_MAXSEG = 6,           // merge tree: largest open segment
    ST_TREE_BAD = 7,         // radix tree walk left its bounds (must never happen)
    ST_SHRINK = 8,           // density: lists overflowed, h shrunk for a retry
    ST_NCELL = 9,            // number of cells of the current index
    ST_ADJ_BAD = 10,         // density loss: a bad split in the input
    ST_POINT_N = 11,         // lists: particles queued for the per-particle search
    ST_TREE_ERR = 12,        // pairing tree: 1 barrier timeout, 2 leaves not reached
    ST_RETRY_N = 13,         // density: lengths of the two retry queues (2 words)
    ST_ACTIVE_N = 15,        // time-step bins: length of the active queue
    ST_SATURATED = 40,       // time-step bins: updates whose limit was below dt_min
    ST_RELIST_N = 41,        // density retries: particles whose lists are rebuilt after
    ST_RETRIED_N = 42,       //   them, and how many of those were retried themselves
    ST_SORT_ERR = 43,        // Morton sort: a tile's look-back gave up waiting (bounded)
    ST_SORT_TICKET = 44,     // Morton sort: tile tickets of the passes (6 words, 44..49)
    ST_ACELL_N = 50,         // lists of the cells that hold a queued particle: cell count
    ST_SM_NSPLIT = 51,       // split/merge pass: split candidates,
    ST_SM_FLAGS = 52,        //   1: a dead particle, 2: a merge candidate not safely inside its zone,
    ST_SM_NCAND = 53,        //   merge candidates per level (APR_MAXLEV words, 53..60)
    ST_BINS = 16,            // merge: first slot of each level's candidates (10 words)
    ST_MERGES = 32,          // merge: merges per level (8 words)
    ST_NSTATUS = 16
};

constexpr int COOP_MAX_BLOCKS = 2048;  // blocks of the cooperative pairing-tree kernel
constexpr int PROF_POOL = 256;              // event pairs recorded before a drain

// launch a kernel on the context's stream and count it
#define APR_LAUNCH(c, kern, grid, block, ...)                                  \
    do {                                                                       \
        ++(c)->launches;                                                       \
        kern<<<(grid), (block), 0, (c)->stream>>>(__VA_ARGS__);                \
    } while (0)

// the same with dynamic shared memory
#define APR_LAUNCH_SMEM(c, kern, grid, block, smem, ...)                       \
    do {                                                                       \
        ++(c)->launches;                                                       \
        kern<<<(grid), (block), (smem), (c)->stream>>>(__VA_ARGS__);           \
    } while (0)

// configuration as the kernels see it (passed by value)
struct DevCfg {
    double lo[3], hi[3], L[3];
    int periodic[3];
    long long Lint[3];
    double delta;
    float deltaf;
    double inv_delta;          // 1 / delta when delta is a power of two (exact), else 0
    double inv_delta2;         // 2 inv_delta (exact; 0 with inv_delta)
    double hfact, gamma;
    int eos;
    double cs0, qcs;
    double alpha_av, beta_av, alpha_u;
    float alpha_avf, beta_avf, alpha_uf;  // the same in float for the FP32 pair loops
    float hfactf, gammaf, cs0f, qcsf, m0f;  // float copies for the FP32-mixed density epilogue
    double rsep_fac, dnn_cap;
    double m0;
    int lmax;
    unsigned long long seed;
    double ccour, cforce, G;
    double nr_tol;
    int nr_maxit;
    int max_neigh;
    int max_cand;              // candidate cells per cell (MAX_CAND_SMALL or _LARGE)
    int prof;                  // count pair evaluations into Workspace::counters
    int kernel;                // APR_KERNEL_M4 or APR_KERNEL_WENDLAND_C2
    double knorm_inv;          // W = f(q) / (knorm_inv h^3): pi (M4), 16 pi / 21 (Wendland C2)
    double m0_knorm;           // m0 / knorm_inv, the factor of the pair sums
    int level_default;         // 0: zones refine; L >= 1: zones derefine from level L
};

struct DevRegion {
    int shape, axis, nlev, pad;
    double centre[3];
    double R[APR_MAXLEV];
};

struct DevRegions {
    int n;
    DevRegion r[APR_MAXREG];
};

struct DevSinks {
    int n;
    double x[APR_MAXSINK][3];
    double m[APR_MAXSINK];
    double racc[APR_MAXSINK];
};

// pointers into the caller's workspace
struct Workspace {
    // index build
    int4* xi;                 // canonical-order lattice coordinates + level
    unsigned long long* key[2];
    unsigned int* val[2];
    unsigned int* hist;
    unsigned int* sort_hist;  // Morton sort: digit counts of every pass (6 x 256), then offsets
    unsigned int* sort_tile;  // Morton sort: per pass and tile, 256 published digit counts
    unsigned int* scan_tmp;
    unsigned int* perm;       // sorted slot -> canonical index
    unsigned int* perm_keep;  // the last sort's order (perm points here after an index build)
    unsigned long long* skey; // sorted keys (aliases key[0] or key[1])
    int4* pk;                 // sorted lattice coordinates + level
    unsigned long long* sthr; // sorted neighbour thresholds of the current list
    unsigned int* sreach;     // smallest integer R with R^2 >= sthr
    double* sh;               // sorted h (float64)
    float4* fA;               // FP32 force data: hinv, P/(Omega rho^2), cs, rho
    float4* fV;               // FP32 velocities + u
    float4* fB;               // FP32 P, 1/(Omega rho), h, level-mass factor
    double* sx;               // FP64 sorted positions
    double* sy;
    double* sz;
    double* dA;               // FP64 force data (4 per particle)
    double* dV;
    double* dB;
    // radix tree over sorted keys
    int* left;
    int* right;
    int* parent_int;
    int* parent_leaf;
    int* visit;
    unsigned char* nlocal;    // radix tree: 1 if a node's leaf range lies in one bottom-up block
    int4* nlo;                // node bbox min (x,y,z) + count
    int4* nhi;                // node bbox max (x,y,z) + first sorted slot
    double* nhmax;            // node max h
    unsigned long long* nthr; // node neighbour threshold at the current reach
    // cells
    unsigned int* cflag;
    unsigned int* cscan;
    int* cell_first;
    int* cell_cnt;
    int* cell_node;
    int* cmark;               // node of the cell starting at a sorted slot
    int* acell_first;         // the cells that hold a queued particle (any order)
    int* acell_cnt;
    int* acell_node;
    unsigned char* amark;     // per sorted slot: queued
    int2* cand;               // max_cand (first slot, count) per cell
    int* ncand;
    int* point_q;             // particles of cells whose candidate list overflowed
    int* retry_q[2];          // density: particles that need another attempt
    int* active_q;            // time-step bins: sorted slots of the active particles
    int* relist_q;            // density retries: retried slots, then their list partners
    unsigned int* qmark;      // per slot: 2 retried, 1 in a retried particle's list
    unsigned long long* sthr0; // density retries: the first list build's thresholds
    // neighbour lists, a row per sorted slot: nbr[slot * max_neigh + k] (a lane writes
    // and reads its own list four entries, 16 bytes, at a time)
    unsigned int* nbr;
    int* ncnt;
    // status words and profile counters
    int* status;
    unsigned long long* counters;
    // split / merge / compaction scratch
    unsigned char* tgt;
    unsigned int* uflag;
    unsigned int* uscan;
    double* tmp8;             // one field's worth of compaction scratch
    unsigned int* mset[2];    // merge tree: particle order within segments
    int* seg_lo[2];
    int* seg_hi[2];
    int4* acc_lo;             // per segment (indexed by its first position)
    int4* acc_hi;
    unsigned long long* acc_sum;
    unsigned int* acc_k;
    unsigned int* acc_k2;
    unsigned long long* acc_key;
    unsigned int* lflag;
    unsigned int* coop;       // pairing-tree rounds: block totals, offsets, barrier, counters
    // reductions
    double* red;              // RED_BLOCKS x 32 partial sums
    double* redout;           // 32 final sums
    size_t bytes;
};

size_t workspace_layout(const apr_config& cfg, long long cap, char* base, Workspace* W);

}  // namespace apr

struct apr_ctx {
    apr_config cfg;
    apr::DevCfg dc;
    cudaStream_t stream;
    int device;
    apr_particles p;
    long long n, cap, next_id;
    unsigned long long step;
    char* ws;
    size_t ws_bytes;
    apr::Workspace W;
    apr_region regions[APR_MAXREG];
    int nreg;
    apr_sink sinks[APR_MAXSINK];
    int nsink;
    long long* hbuf;          // pinned host read-back buffer
    std::string err;
    bool bound;
    bool have_force;
    int coop_blocks;          // co-resident blocks of the pairing-tree kernel (0: unknown)
    long long prof_attempts, prof_unc, prof_shrink;  // density-solve counters
    bool lists_fresh;         // the current lists hold every pair at the current h
    bool force_data_fresh;    // the last density solve wrote every slot's force records
    bool lists_unchecked;     // lists were built after the last read of the status words
    bool quiet_pass;          // the last split/merge pass changed nothing
    bool order_valid;         // the kept Morton order is a permutation of the current set
    long long order_n;        //   of this many particles,
    int order_age;            //   refitted this many times since its sort
    int ncell;
    int last_shrink;
    bool tree_smem_set;       // dynamic shared memory opt-in of the pairing-tree kernel
    bool dt_valid;            // dt_next belongs to the current forces
    double dt_next;
    // profiling
    long long launches;
    bool prof;
    cudaEvent_t ev[2 * apr::PROF_POOL];
    int ev_group[apr::PROF_POOL];
    int ev_used;
    double prof_ms[APR_NPROF];
    long long prof_calls[APR_NPROF];
};

namespace apr {

// ---------------------------------------------------------------- helpers

__host__ __device__ inline unsigned long long neighbour_threshold(double h, double delta)
{
    // b is within the kernel radius 2h of a iff r2_lattice(a, b) < thr(h)
    double t = (2.0 * h) / delta;
    double t2 = t * t;
    if (!(t2 < 4.6e18)) return 4611686018427387904ULL;
    return (unsigned long long)ceil(t2);
}

// the same threshold with dc's lattice unit: a multiplication where the unit is a
// power of two (then x * (1/delta) equals x / delta exactly), else the division
// the bits of a double (host and device: the threshold arithmetic below is also
// compiled for the host by a test)
__host__ __device__ __forceinline__ unsigned long long dbits(double d)
{
    unsigned long long b;
    memcpy(&b, &d, sizeof b);
    return b;
}

// ceil(|d|) of a double with |d| < 2^62 as an integer, read off its bits with
// integer operations (the FP64 pipe, which rounds and converts, is narrow on this part)
__host__ __device__ __forceinline__ unsigned long long ceil_bits(double d)
{
    const unsigned long long b = dbits(d) & 0x7fffffffffffffffULL;
    const int e = (int)(b >> 52) - 1023;
    if (e < 0) return b != 0ULL ? 1ULL : 0ULL;
    const unsigned long long m = (b & ((1ULL << 52) - 1ULL)) | (1ULL << 52);
    if (e >= 52) return m << (e - 52);
    const unsigned long long ip = m >> (52 - e);
    return ip + ((m & ((1ULL << (52 - e)) - 1ULL)) != 0ULL ? 1ULL : 0ULL);
}

// the lattice radius 2 h / delta (as the oracle forms it: with a power-of-two unit
// (2 h) inv_delta = h (2 inv_delta), both one rounding of the same product)
__host__ __device__ __forceinline__ double lattice_radius(const DevCfg& dc, double h)
{
    return dc.inv_delta > 0.0 ? h * dc.inv_delta2 : (2.0 * h) / dc.delta;
}

// ceil(t^2) of t = lattice_radius, capped at 2^62; t^2 in [0, 4.6e18) (compared as
// bits: for non-negative doubles the bit patterns order as the values, and a NaN's
// lie above) takes ceil_bits
__host__ __device__ __forceinline__ unsigned long long lattice_threshold_t(double t)
{
    const double t2 = t * t;
    if (!(dbits(t2) < dbits(4.6e18)))
        return 4611686018427387904ULL;
    return ceil_bits(t2);
}

__device__ __forceinline__ unsigned long long lattice_threshold(const DevCfg& dc, double h)
{
    return lattice_threshold_t(lattice_radius(dc, h));
}

__device__ __forceinline__ long long min_image(long long d, int periodic, long long L)
{
    if (periodic) {
        if (2 * d > L) d -= L;
        else if (2 * d < -L) d += L;
    }
    return d;
}

inline bool any_periodic(const DevCfg& dc)
{
    return dc.periodic[0] || dc.periodic[1] || dc.periodic[2];
}

__device__ __forceinline__ int min_image32(int d, int periodic, int L)
{
    if (periodic) {
        if (2 * d > L) d -= L;
        else if (2 * d < -L) d += L;
    }
    return d;
}

// relative mass 2^-level as an exact float
__device__ __forceinline__ float level_mass_f(int level) { return __int_as_float((127 - level) << 23); }
__device__ __forceinline__ double level_mass_d(int level)
{
    return __longlong_as_double((long long)(1023 - level) << 52);
}

// ------------------------------------------------------ launch plumbing

// host-side helpers (apr_api.cu)
apr_status fail(apr_ctx* c, apr_status s, const std::string& msg);
apr_status cuda_check(apr_ctx* c, cudaError_t e, const char* what);
DevRegions dev_regions(const apr_ctx* c);
int prof_begin(apr_ctx* c, int group);        // -1 when profiling is off
void prof_end(apr_ctx* c, int slot);
DevSinks dev_sinks(const apr_ctx* c);

// index build (apr_index.cu)
apr_status scan_u32(apr_ctx* c, const unsigned int* in, unsigned int* out, long long n,
                    unsigned int* total_dev);
apr_status quantise(apr_ctx* c);
// one stable 8-bit radix pass; bin_starts[d] (d < nbins) = first output slot of digit d
apr_status radix_pass8(apr_ctx* c, const unsigned long long* kin, const unsigned int* vin,
                       unsigned long long* kout, unsigned int* vout, long long n, int shift,
                       int* bin_starts, int nbins);
apr_status index_sort(apr_ctx* c);           // quantise, Morton sort, gather, tree, node data
apr_status index_refresh_h(apr_ctx* c);      // re-gather h and node hmax after a density pass
// lists after density retries: relist_mark records a retry queue before its
// attempt (the first call clears the marks); relist_finish rebuilds, at the final
// h, the lists of every retried particle and of every particle in a retried
// particle's last list, so that all lists hold every force pair
apr_status relist_mark(apr_ctx* c, const int* queue, const int* qlen_dev, bool first);
apr_status relist_finish(apr_ctx* c);
// mode 0: gather lists (r < 2 reach h_a); mode 1: symmetric lists (r < 2 reach max(h_a, h_b)).
// graceful: an overflowing list is marked (count -1) instead of flagged as an error.
struct FuseArgs;
apr_status index_lists(apr_ctx* c, int mode, double reach, bool graceful = false,
                       const FuseArgs* fz = nullptr);
// lists of the queued particles only, by a per-particle tree walk: symmetric
// (sym) or gather lists; node_reach > 0: the nodes' largest h are in units of
// h / node_reach (see relist_finish)
apr_status index_lists_queue(apr_ctx* c, const int* queue, const int* qlen_dev, double reach,
                             bool graceful = true, bool sym = true, double node_reach = -1.0);
// symmetric lists of every particle in a cell that holds a queued particle
apr_status index_lists_cells_of(apr_ctx* c, const int* queue, const int* qlen_dev, double reach,
                                bool graceful);
apr_status index_refresh_sh(apr_ctx* c);     // re-gather h only (no node h maxima)
// re-gather the h of the queued slots only
apr_status index_refresh_sh_queue(apr_ctx* c, const int* queue, const int* qlen_dev);

// SPH passes (apr_sph.cu)
// force_data: also write the force pass's per-slot records of the iterated particles
apr_status density_pass(apr_ctx* c, long long* uncovered, long long* noconv,
                        const int* active = nullptr, long long nactive = 0, int out_q = 0,
                        bool force_data = false);
apr_status force_pass(apr_ctx* c, const int* active = nullptr, long long nactive = 0);
apr_status gather_force_data(apr_ctx* c);

// refinement, sinks, integration (apr_refine.cu)
apr_status split_merge_pass(apr_ctx* c, apr_counts* cnt);
apr_status clear_changed(apr_ctx* c);
apr_status merge_pairs_debug(apr_ctx* c, int level, long long* pairs, long long cap,
                             long long* npairs, long long* spare);
// point-mass gravity; B >= 0: only the particles whose time-step bin ends at
// substep boundary `sub` take the pull (the point masses feel every particle)
apr_status sink_gravity(apr_ctx* c, int B = -1, long long sub = 0);
apr_status accrete(apr_ctx* c, long long* naccreted);
apr_status kick(apr_ctx* c, double hdt);
apr_status drift(apr_ctx* c, double dt);
apr_status kick_drift(apr_ctx* c, double hdt, double dt);  // opening half kick + drift
apr_status compute_stats(apr_ctx* c, apr_stats* st);
apr_status compute_timestep(apr_ctx* c, double* dt);
// conservation sums and the step limit; kick_hdt != 0 applies the step's closing
// half kick to the gas first (the same pass)
apr_status compute_stats_dt(apr_ctx* c, apr_stats* st, double* dt, double kick_hdt = 0.0);
// individual time steps (apr_bins.cu)
apr_status bins_init(apr_ctx* c, double dt_max, int B);
apr_status bins_kick(apr_ctx* c, double dt_max, int B, long long k, int end_of_step);
apr_status bins_mark_inactive(apr_ctx* c, long long k, int B, bool on);
apr_status bins_active_queue(apr_ctx* c, long long k, int B, long long* nact);
apr_status bins_rebin(apr_ctx* c, double dt_max, int B, long long k, long long nq);

// relaxing (apr_relax.cu)
apr_status relax_stage(apr_ctx* c, const apr_particles* ref, long long nref);
apr_status relax_interp(apr_ctx* c, long long nref, apr_status (*index)(apr_ctx*));
apr_status relax_shift(apr_ctx* c, double* ke);
apr_status clear_new(apr_ctx* c);

// density error of a split and its adjoint (apr_adjoint.cu)
apr_status adjoint_children(apr_ctx* c, long long npar, const long long* parent, const double* d,
                            const double* hc, bool* bad);
apr_status adjoint_sums(apr_ctx* c, long long n, long long npar, double* loss, double* grad_d,
                        double* grad_hc);
apr_status compact(apr_ctx* c, long long* removed);
apr_status reorder(apr_ctx* c);  // bound arrays into the index's Morton order

inline int nblocks(long long n, int bs) { return (int)((n + bs - 1) / bs); }

}  // namespace apr

/*
 * apr.h -- C ABI of the GB300 adaptive particle refinement (APR) SPH library.
 *
 * Method: Nealon & Price, "Adaptive particle refinement for compressible
 * smoothed particle hydrodynamics" (arXiv 2409.11470).  The library runs the
 * data-parallel hot path of one time step on one GPU: refinement zones
 * (Sec. 2.1), split (Sec. 2.2, Eq. 2), pairing tree and merge (Sec. 2.3,
 * Eq. 3, Eq. 4) in the per-step order of Sec. 2.6, the neighbour search, the
 * h-rho density solve and the force / energy sums over particles of mixed
 * mass (Eq. 1) and smoothing length, point-mass gravity with accretion, and a
 * kick-drift-kick update.
 *
 * Conventions (all entry points):
 *  - Plain C types only.  Particle arrays and the workspace are DEVICE
 *    pointers owned by the caller; the library owns only the opaque context
 *    and a few bytes of pinned host memory for status read-back.
 *  - All GPU work is ordered on the stream given to apr_create; calls return
 *    after the host has read whatever counts it reports (a short
 *    device-to-host copy), so the particle count is always current on return.
 *  - Nothing is allocated on the device after apr_bind.
 *  - Errors are status codes; no exception crosses the ABI.  apr_last_error
 *    returns a text for the last failing call on that context.
 *  - Particle order is the caller's: indices are stable except that split
 *    children are appended at the end (slot n + rank), merged-away or
 *    accreted particles are removed by a stable compaction, and apr_reorder
 *    permutes every array into spatial order when the caller asks for it.
 */
#ifndef APR_H
#define APR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define APR_MAXLEV 8
#define APR_MAXREG 8
#define APR_MAXSINK 8

typedef enum {
    APR_OK = 0,
    APR_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, bad config) */
    APR_ERR_CAPACITY = 2,       /* a split would exceed the bound capacity; state unchanged */
    APR_ERR_NR_NOCONV = 3,      /* some h-rho iterations did not converge (best effort kept) */
    APR_ERR_NEIGH_OVERFLOW = 4, /* a neighbour or candidate list exceeded its capacity */
    APR_ERR_CUDA = 5,           /* a CUDA runtime call failed */
    APR_ERR_STATE = 6,          /* call out of order (e.g. before apr_bind) */
    APR_ERR_WORKSPACE = 7       /* workspace too small for the bound capacity */
} apr_status;

/* particle flag bits: CHANGED by the current split/merge pass; FIXED never moves,
   splits or merges; DEAD removed at the next compaction; NEW introduced by a split
   or merge and not yet relaxed (apr_relax clears it) */
enum { APR_FLAG_CHANGED = 1, APR_FLAG_FIXED = 2, APR_FLAG_DEAD = 4, APR_FLAG_NEW = 8,
       APR_FLAG_INACTIVE = 16 /* set only inside apr_step_bins: not at the end of its step */ };
enum { APR_SHAPE_SPHERE = 0, APR_SHAPE_SLAB = 1, APR_SHAPE_CYLINDER = 2 };
enum { APR_EOS_ADIABATIC = 0, APR_EOS_LOCALLY_ISOTHERMAL = 1 };
enum { APR_PREC_FP32_MIXED = 0, APR_PREC_FP64 = 1 };
enum { APR_KERNEL_M4 = 0, APR_KERNEL_WENDLAND_C2 = 1 };

/*
 * Run configuration.  box_lo/box_hi: domain; periodic axes wrap.  delta: the
 * quantisation unit D of the integer lattice x_int = floor((x - lo)/D) on
 * which all decisions (neighbour membership, nearest-neighbour distance,
 * pairing-tree cuts) are taken; (hi - lo)/D must be <= 2^30 and an exact
 * integer on periodic axes.  hfact: h = hfact (m/rho)^(1/3) (Table 2).
 * m0: mass at level 0 (Eq. 1).  lmax: deepest level.  rsep_fac, dnn_cap: the
 * split separation min(rsep_fac h, dnn_cap d_nn) (Sec. 2.2; 0.2 and 0.35).
 * alpha_av, beta_av: artificial viscosity; alpha_u: artificial conductivity.
 * precision: APR_PREC_FP32_MIXED (pair sums in float on relative lattice
 * coordinates, compensated; state, integration and global sums in double) or
 * APR_PREC_FP64.  nr_tol, nr_maxit: h-rho Newton-Raphson stopping rule.
 * max_neigh: capacity of one particle's neighbour list (0 = default 512; else a
 * positive multiple of 4, the lists being written and read 16 bytes at a time).
 * kernel: APR_KERNEL_M4 (cubic spline, h_fact 1.2) or APR_KERNEL_WENDLAND_C2
 * (the applications' kernel of Sec. 3, h_fact 1.3); both have support 2h.
 * level_default: 0 refines (a point inside k nested boundaries of a zone asks
 * for level k, the maximum over zones); L >= 1 derefines (every point asks for
 * level L, a point inside k boundaries for L - k, the minimum over zones), the
 * mode Sec. 2.1 and Sec. 4 describe for zones of lower resolution.
 * fused_density: 1 lets the FP32-mixed path take the first Newton-Raphson
 * pass of a step's density solve inside the neighbour-list build, from the
 * candidates staged in shared memory (the same terms in the same order, hence
 * the same results); 0 (default, faster on GB300) runs every pass in the
 * density kernel.  The FP64 path always does the latter.
 */
typedef struct {
    double box_lo[3], box_hi[3];
    int periodic[3];
    double delta;
    double hfact, gamma;
    int eos;
    double cs0, qcs;
    double alpha_av, beta_av, alpha_u;
    double rsep_fac, dnn_cap;
    double m0;
    int lmax;
    unsigned long long seed;
    double ccour, cforce, G;
    int precision;
    double nr_tol;
    int nr_maxit;
    int max_neigh;
    int kernel;
    int level_default;
    int fused_density;
} apr_config;

/*
 * A refinement zone (Sec. 2.1, Table 1): nested boundaries R[0] > R[1] > ...,
 * a point strictly inside R[k] asks for level k + 1.  shape sphere:
 * |x - centre| < R; slab: |x[axis] - centre[axis]| < R; cylinder along axis:
 * the distance from the line through centre along axis < R (the circular zone
 * of a thin box, appendix sound-wave test).  track_sink >= 0 makes
 * the centre follow that sink every step (co-moving zone, Sec. 2.1).
 */
typedef struct {
    int shape, axis, track_sink, nlev;
    double centre[3];
    double R[APR_MAXLEV];
} apr_region;

/* a point mass: position, velocity, acceleration, mass, accretion radius */
typedef struct {
    double x[3], v[3], a[3];
    double m, racc;
} apr_sink;

/*
 * Particle state: caller-owned DEVICE arrays of length >= capacity, in the
 * caller's order.  Inputs: x..h, level, flags, id.  Outputs written by the
 * library: rho, omega (grad-h term), ax..az, dudt, vsig (signal speed), dnn
 * (nearest-neighbour distance on the lattice, +inf if none within 2h), pres,
 * cs.  Mass is m0 / 2^level (Eq. 1) and is not stored.
 */
typedef struct {
    double *x, *y, *z, *vx, *vy, *vz, *u, *h;
    double *rho, *omega, *ax, *ay, *az, *dudt, *vsig, *dnn, *pres, *cs;
    unsigned char *level, *flags;
    unsigned long long *id;
    unsigned char* bin; /* time-step bin (apr_step_bins); may be NULL otherwise */
} apr_particles;

typedef struct {
    long long n_split[APR_MAXLEV], n_merge[APR_MAXLEV], n_spare[APR_MAXLEV];
    long long n_accreted, n_dead;
} apr_counts;

/* float64 conservation sums over live gas particles and sinks */
typedef struct {
    double mass, mom[3], ang[3], ekin, etherm;
} apr_stats;

/* kernel groups timed by the profiler (apr_profile_enable) */
enum {
    APR_PROF_SORT = 0,      /* lattice quantisation, Morton keys, radix sort, gathers */
    APR_PROF_TREE = 1,      /* radix tree construction and bottom-up node boxes */
    APR_PROF_LISTS = 2,     /* cells, candidate cells, neighbour lists */
    APR_PROF_DENSITY = 3,   /* the h-rho Newton-Raphson kernel */
    APR_PROF_FORCE = 4,     /* the force / energy kernel */
    APR_PROF_REFINE = 5,    /* split / merge pass */
    APR_PROF_OTHER = 6,     /* force-data gathers, gravity, accretion, integration, sums */
    APR_NPROF = 8
};

/*
 * Profile counters.  ms/calls: device time (CUDA events recorded on the
 * library's stream around each group) and number of timed calls per group,
 * accumulated while profiling is enabled.  pairs: pair evaluations done by
 * the density kernel (pairs inside 2h, summed over Newton-Raphson iterations)
 * and by the force kernel (pairs inside max(2h_a, 2h_b)).  launches: every
 * kernel the library launched since the context was created (always counted).
 * density_attempts: list builds + Newton-Raphson passes of the density solve;
 * uncovered: particles, summed over attempts, that needed another attempt
 * (h beyond the lists' reach, or a list that overflowed); shrunk: those of
 * them whose list overflowed (h reduced).
 */
typedef struct {
    double ms[APR_NPROF];
    long long calls[APR_NPROF];
    double pairs[APR_NPROF];
    long long launches;
    long long density_attempts;
    long long uncovered;
    long long shrunk;
} apr_profile;

typedef struct apr_ctx apr_ctx;

/* Create a context on the current CUDA device; stream may be NULL (legacy default). */
apr_status apr_create(apr_ctx** ctx, const apr_config* cfg, void* stream);
void apr_destroy(apr_ctx* ctx);
const char* apr_last_error(const apr_ctx* ctx);

/* Bytes of device workspace needed for `capacity` particles. */
apr_status apr_workspace_size(const apr_config* cfg, long long capacity, size_t* bytes);

/*
 * Attach particle arrays (n live particles, room for `capacity`), the next id
 * to hand to a split child, and a caller-owned device workspace of at least
 * apr_workspace_size bytes (256-byte aligned).
 */
apr_status apr_bind(apr_ctx* ctx, const apr_particles* p, long long n, long long capacity,
                    long long next_id, void* workspace, size_t bytes);

/*
 * Host exchange of the bound particle state, for callers that keep it in host
 * memory between steps (the paper has no counterpart: these move data only).  host:
 * an apr_particles of HOST pointers (page-locked memory lets
 * the copies run asynchronously); a NULL field is skipped.
 *
 * apr_upload copies n particles (0 <= n <= capacity) into the bound arrays on
 * the context's stream and makes n the bound count.  The cached time-step
 * limit and lists are dropped (call apr_timestep before uploading if the next
 * step should use the limit of the last pass); the forces a step needs are
 * whatever the uploaded ax..dudt hold.  APR_ERR_ARG for a bad n,
 * APR_ERR_STATE if a given field has no bound array (bin).
 *
 * apr_download copies the current particles to host arrays of room for cap
 * particles, waits for the copies, and stores the count in *n_out (may be
 * NULL); APR_ERR_CAPACITY (nothing copied) if cap is too small.
 */
apr_status apr_upload(apr_ctx* ctx, const apr_particles* host, long long n);
apr_status apr_download(apr_ctx* ctx, const apr_particles* host, long long cap,
                        long long* n_out);

/* Refinement zones and point masses (host arrays, copied). */
apr_status apr_set_regions(apr_ctx* ctx, const apr_region* r, int nregions);
apr_status apr_set_sinks(apr_ctx* ctx, const apr_sink* s, int nsinks);
apr_status apr_get_sinks(apr_ctx* ctx, apr_sink* s, int nsinks);

/* Current particle count, next id and split/merge step counter. */
apr_status apr_get_count(apr_ctx* ctx, long long* n, long long* next_id,
                         unsigned long long* step);

/*
 * Initial refinement with the given refinement zones and levels (Sec. 2.1
 * rules 1-3, Table 1; Sec. 2.6 applied until no particle changes level):
 * the zones are installed as by apr_set_regions, moved onto the sinks they
 * track, and {density; split/merge pass} is repeated until nothing changes,
 * so that particles reach the full depth of nested zones; then density and
 * forces.  regions: HOST array of nregions zones (copied; nregions 0 with a
 * non-NULL array removes every zone); NULL keeps the zones already set (then
 * nregions must be 0).  *passes (may be NULL) receives the number of
 * split/merge passes.  APR_ERR_ARG for a bad zone (nothing changed),
 * APR_ERR_CAPACITY if the splits would exceed the bound capacity; errors of
 * the density solve and the lists as for apr_sph_density.
 */
apr_status apr_init(apr_ctx* ctx, const apr_region* regions, int nregions, int* passes);

/*
 * One split/merge pass (Sec. 2.6): clear the changed marks; split levels
 * 0..lmax-1 ascending (Sec. 2.2, Eq. 2); merge levels lmax..1 descending
 * through the pairing tree (Sec. 2.3, Eq. 3; an odd candidate is left over);
 * compact.  Each particle changes level at most once.  APR_ERR_CAPACITY is
 * detected before any particle is written.
 */
apr_status apr_split_merge(apr_ctx* ctx, long long* n_out, apr_counts* counts);

/*
 * Density solve: h, rho, omega, dnn, pres, cs of every live particle from
 * the h-rho relation rho = m (hfact/h)^3 = sum_b m_b W(r_ab, h) (cited in
 * Sec. 2.2) by Newton-Raphson from the current h.  *n_unconverged (may be
 * NULL) receives the count still unconverged after nr_maxit iterations.
 */
apr_status apr_sph_density(apr_ctx* ctx, long long* n_unconverged);

/*
 * Force and energy sums (the standard grad-h SPH equations the paper takes
 * from Phantom, cited in Sec. 2.2 and Sec. 3; mixed masses by Eq. 1):
 *   a_a = -sum_b m_b [(P_a + q_a)/(Omega_a rho_a^2) F_a + (P_b + q_b)/(Omega_b rho_b^2) F_b] r_hat
 *   du_a/dt = (P_a + q_a)/(Omega_a rho_a^2) sum_b m_b (v_ab . r_hat) F_a + conductivity
 * over pairs with |r_ab| < 2 max(h_a, h_b), F = dW/dr at each particle's own
 * h, q the artificial viscosity of approaching pairs (alpha, beta) and the
 * conductivity alpha_u (Sec. 4's shock tube); vsig_a = max over neighbours of
 * c_s + beta max(0, -v_ab . r_hat).  Point masses (Sec. 3) add
 * -G M (x - x_s)/|x - x_s|^3.  Reads x, v, u, h, rho, omega, pres, cs, level,
 * flags of every live particle (rho .. cs as the last density pass left
 * them); writes ax, ay, az, dudt, vsig.  APR_ERR_STATE before apr_bind;
 * errors of the lists as for apr_sph_density.
 */
apr_status apr_sph_force(apr_ctx* ctx);

/*
 * One kick-drift-kick step of length dt (dt <= 0: the limit of apr_timestep
 * from the last force pass), with the paper's per-step order (Sec. 2.6,
 * Fig. 1) placed between the drift and the closing kick: half kick (gas and
 * sinks), drift, accretion (Sec. 3), zones updated onto their sinks (Sec. 2.1),
 * split passes ascending and merge passes descending (Sec. 2.2, 2.3),
 * compaction, density, forces, half kick, float64 conservation sums.
 * dt_used receives the step taken; stats the sums at the end; counts the
 * split/merge/accretion counts; each may be NULL.  Errors as for
 * apr_split_merge, apr_sph_density and apr_sph_force; APR_ERR_STATE before a
 * force pass.
 */
apr_status apr_step(apr_ctx* ctx, double dt, double* dt_used, apr_stats* stats,
                    apr_counts* counts);

/*
 * Global time-step limit from the last force pass (the step whose halving
 * defines the bins of Sec. 2.5; the paper cites Phantom's criteria):
 * min over live, unfixed particles of ccour h / vsig (vsig > 0) and
 * cforce sqrt(h / |a|) (|a| > 0); ccour 0.3, cforce 0.25.  +inf if no
 * particle constrains it.  *dt: HOST.  APR_ERR_STATE before a force pass.
 */
apr_status apr_timestep(apr_ctx* ctx, double* dt);

/*
 * Float64 conservation sums of the current state, over live gas particles
 * (mass m0 / 2^level, Eq. 1) and sinks: total mass (exactly conserved by
 * split and merge, Sec. 2.2-2.3), momentum, angular momentum about the
 * origin, kinetic and thermal energy.  Fixed-order reduction (the same result
 * for the same state on every call).  *stats: HOST.
 */
apr_status apr_stats_compute(apr_ctx* ctx, apr_stats* stats);

/*
 * Memory layout, no counterpart in the paper: permutes every bound particle
 * array (all fields of apr_particles, bin too when bound) in place into the
 * order of the index's last Morton sort (sorting first if the particle set
 * changed since), so that particles close in space sit close in memory and the
 * passes' gathers through the sort read consecutive addresses.  Ids travel with
 * their particles; indices the caller kept from before (apr_merge_pairs, the
 * parents of apr_density_loss_grad) name other particles afterwards.  Later
 * results are those without the call, except for the order of equal Morton
 * keys in the next sort and hence the summation order of sums.  The
 * neighbour-list memory is its scratch, so the next pass rebuilds the lists.
 * Errors: APR_ERR_STATE before apr_bind; APR_ERR_CUDA on a launch error.
 */
apr_status apr_reorder(apr_ctx* ctx);

/*
 * Debug / parity: neighbour lists on the quantised lattice at the current h,
 * into HOST buffers in CSR form (offsets[n+1], idx[total]; particle indices
 * in the caller's order; order within a list unspecified).  mode 0: b != a
 * with |r_ab| < 2 h_a; mode 1: |r_ab| < 2 max(h_a, h_b).  Returns
 * APR_ERR_NEIGH_OVERFLOW with *total set if cap is too small.
 */
apr_status apr_neighbour_lists(apr_ctx* ctx, int mode, long long* offsets, int* idx,
                               long long cap, long long* total);

/*
 * Debug / parity: the pairing tree (Sec. 2.3) of the merge candidates of
 * `level` in the current state, without merging.  pairs: HOST buffer of
 * 2*cap particle indices; *npairs receives the pair count, *spare the index
 * left out for an odd count (-1 if none).
 */
apr_status apr_merge_pairs(apr_ctx* ctx, int level, long long* pairs, long long cap,
                           long long* npairs, long long* spare);

/*
 * One step of length dt_max with individual time steps (Sec. 2.5).  Particle i
 * sits in bin b_i (0..max_bin) and steps dt_max / 2^b_i on the grid of the
 * 2^max_bin substeps of dt_min = dt_max / 2^max_bin.  Per substep: half kick of
 * the particles whose step starts (old accelerations), drift of every
 * particle, then for the particles whose step ends (the active ones), in the
 * order of apr_step: split/merge restricted to them (APR over active particles
 * only), their density and forces (the others keep their last values), their
 * second half kick, and their new bin: split or merged particles go to
 * max_bin; the others to the longest step dt_max / 2^b not above their limit
 * min(ccour h / v_sig, cforce sqrt(h / |a|)), moving to a longer step only
 * where its grid meets the current time.  Point masses take every substep:
 * half kick, drift, accretion and zones moved onto them after the drift; after
 * the active particles' forces, their pull on the active particles only and
 * their own accelerations from every live particle; then the closing half
 * kick.  init_bins != 0 first bins every particle by its limit.  With
 * max_bin = 0 this is apr_step(dt_max).
 *
 * Needs the bound bin array and forces from a previous pass (apr_init or a
 * step).  counts: summed over the substeps (n_accreted included); updates:
 * particle force updates done; saturated: updates whose limit was below dt_min
 * (kept in max_bin); stats: conservation sums at the end.  Any of them may be
 * NULL.
 */
apr_status apr_step_bins(apr_ctx* ctx, double dt_max, int max_bin, int init_bins,
                         apr_counts* counts, long long* updates, long long* saturated,
                         apr_stats* stats);

/*
 * Relaxing (Sec. 2.4): shuffle the particles flagged APR_FLAG_NEW (introduced
 * by the split/merge passes since the last relax) towards a reference set, the
 * particles as they were before those passes.  Each shuffle computes density
 * and forces of the current particles (a_new), interpolates the reference
 * accelerations to every NEW particle, a_ref = sum over the reference set of
 * (m_b / rho_b) a_b W(|x - x_b|, h_b) (each reference particle at its own h),
 * and moves it by dx = 0.5 dt^2 (a_new - a_ref) with dt = 0.3 h / c_s, |dx|
 * capped at h.  The shuffle's energy is the sum of |dx| / dt^2; shuffles stop
 * when it is at most tol times the first one's, or after max_iter (the paper:
 * 0.005 and 50).  Then density and forces are recomputed and the NEW flags
 * cleared.
 *
 * ref: DEVICE arrays x, y, z, h, rho, ax, ay, az, level, flags of nref
 * particles (dead ones take no part; other fields are not read), caller-owned.
 * iters (may be NULL): shuffles done; ke_ratio (may be NULL): last energy /
 * first.  Needs n + nref <= capacity (APR_ERR_CAPACITY otherwise): the
 * reference set is staged in the spare bound slots [n, n + nref), which are
 * scratch.  Errors of the density solve or the lists are returned as by
 * apr_sph_density.  Synchronises the stream.
 */
apr_status apr_relax(apr_ctx* ctx, const apr_particles* ref, long long nref, int max_iter,
                     double tol, int* iters, double* ke_ratio);

/*
 * Density error of one split pass and its gradient (adjoint).  The paper's
 * method has no such call: it chooses the child separation (Sec. 2.2, Eq. 2)
 * and relaxes new children (Sec. 2.5) so that the split set reproduces the
 * density of the original set; this call measures that error and its gradient
 * with respect to the children's offsets and smoothing lengths, so that child
 * placement can be optimised.
 *
 * Reference set: the n bound particles as they are, each at its own h (dead
 * ones take no part).  Split k replaces parent[k] by two children at
 * x_p + d[k] and x_p - d[k], one level finer (mass by Eq. 1), with smoothing
 * lengths hc[2k] and hc[2k+1].  The new set is the reference set without the
 * parents, plus the children.
 *   J = sum over children a of (rho_new(a) - rho_ref(x_a))^2
 *   rho_new(a) = sum over the new set of m_b W(|x_a - x_b|, h_a)   (h fixed, self included)
 *   rho_ref(x) = sum over the reference set of m_b W(|x - x_b|, h_b)
 * M4 kernel, minimum image on periodic axes.
 *
 * parent: DEVICE, npar int64 indices into [0, n), each live and used once.
 * d: DEVICE, npar x 3 float64, row-major.  hc: DEVICE, 2*npar float64, > 0.
 * loss: HOST, receives J.  grad_d: DEVICE npar x 3 float64 (dJ/dd), grad_hc:
 * DEVICE 2*npar float64 (dJ/dhc).  All buffers are the caller's.  Pair sums
 * run in float on relative lattice coordinates with compensated accumulation
 * (double with APR_PREC_FP64); J is reduced in float64 in a fixed order.
 *
 * Needs n + 2*npar <= capacity, else APR_ERR_CAPACITY and nothing is written.
 * The spare bound slots [n, n + 2*npar) are scratch: on return they hold the
 * children (x, y, z, h, level), each child's density error in rho and its
 * position and h gradients in ax, ay, az and dudt.  Particles [0, n) and the
 * count n are unchanged; the next density or force call rebuilds the index.
 * APR_ERR_ARG for a bad split (parent out of range, dead or repeated, an
 * offset not finite, hc not finite and positive); APR_ERR_NEIGH_OVERFLOW if a
 * list exceeds max_neigh.  Synchronises the stream.
 */
apr_status apr_density_loss_grad(apr_ctx* ctx, long long npar, const long long* parent,
                                 const double* d, const double* hc, double* loss, double* grad_d,
                                 double* grad_hc);

/*
 * Profiling (not part of the method): on != 0 starts timing kernel groups with
 * CUDA events on the bound stream and counting pair evaluations, and clears
 * the counters; on == 0 stops.  The event pool is created here, not in the
 * hot calls.
 */
apr_status apr_profile_enable(apr_ctx* ctx, int on);

/* Read (and with reset != 0 clear) the profile counters; synchronises the stream. */
apr_status apr_profile_read(apr_ctx* ctx, apr_profile* out, int reset);

/*
 * Measurement probe (not a step of the method; the paper has no
 * counterpart): the arithmetic peak of this GPU's fused multiply-add pipes,
 * against which the pair kernels' FLOP rates are stated.  precision
 * APR_PREC_FP32_MIXED probes the FP32 pipes, APR_PREC_FP64 the FP64 pipe.
 * One warm-up launch, then one launch timed with CUDA events on `stream`
 * (NULL = legacy default): every SM holds as many 256-thread blocks as fit,
 * each thread runs 8 independent FMA chains for iters x 16 steps (2 flops per
 * FMA).  *tflops and *ms (HOST) receive the rate and the timed launch's
 * duration.  Synchronises the stream; allocates no device memory.
 * APR_ERR_ARG for iters < 1 or another precision, APR_ERR_CUDA if a CUDA call
 * fails.
 */
apr_status apr_probe_fma_peak(int precision, int iters, void* stream, double* tflops,
                              double* ms);

/*
 * Conservation sums like apr_stats_compute, for callers that cannot allocate
 * device memory.  The paper has no counterpart: this is a convenience of the
 * library, not a step of the method.
 *
 * Who needs it: code running under another framework's memory manager (a raw
 * cudaMalloc there bypasses the framework's pool and accounting) and
 * latency-critical callbacks where an allocation could implicitly synchronise
 * the device or fail under a memory cap.  This call takes no context and no
 * workspace and allocates nothing (no cudaMalloc, cudaFree or allocating
 * library routine): its scratch is a fixed 512 KB device array built into the
 * library, present on every GPU that loads the library until the process
 * exits.
 *
 * cfg: only m0 and eos are read.  p: DEVICE arrays x, y, z, vx, vy, vz, u,
 * level, flags of n particles (dead-flagged ones are skipped); at most
 * 16,777,216 particles, larger n returns APR_ERR_ARG with a message.  sinks:
 * HOST array of nsinks point masses added to the sums (may be NULL if 0).
 * stream: the CUDA stream to run on (NULL = legacy default); the call
 * synchronises it before returning.  out: HOST result.  err/errlen: optional
 * buffer for a message (empty on success).
 *
 * The first call on each device looks up the device address of the built-in
 * array (with that device current).  No call may run on a stream under
 * capture: every call reads its result back to host memory and synchronises
 * the stream, so a call on a capturing stream returns APR_ERR_ARG without
 * launching anything.  Every call overwrites the whole scratch it uses, so nothing
 * carries over between calls, but two calls that overlap on the GPU (from
 * different streams or threads) share the array and race.
 */
apr_status apr_stats_noalloc(const apr_config* cfg, const apr_particles* p, long long n,
                             const apr_sink* sinks, int nsinks, void* stream, apr_stats* out,
                             char* err, size_t errlen);

#ifdef __cplusplus
}
#endif

#endif /* APR_H */

// C ABI of the GB300 APR SPH library (declared in include/apr.h): argument
// checks, the caller-owned workspace layout, and the host-side order of the
// passes of one step (Sec. 2.6: zones -> split ascending -> merge descending
// -> density -> forces, inside a kick-drift-kick update).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "apr_density.cuh"
#include "apr_internal.cuh"

namespace apr {

apr_status fail(apr_ctx* c, apr_status s, const std::string& msg)
{
    if (c) c->err = msg;
    return s;
}

apr_status cuda_check(apr_ctx* c, cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return APR_OK;
    return fail(c, APR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

DevRegions dev_regions(const apr_ctx* c)
{
    DevRegions r;
    memset(&r, 0, sizeof(r));
    r.n = c->nreg;
    for (int j = 0; j < c->nreg; ++j) {
        const apr_region& s = c->regions[j];
        r.r[j].shape = s.shape;
        r.r[j].axis = s.axis;
        r.r[j].nlev = s.nlev;
        for (int k = 0; k < 3; ++k) r.r[j].centre[k] = s.centre[k];
        for (int k = 0; k < APR_MAXLEV; ++k) r.r[j].R[k] = s.R[k];
    }
    return r;
}

DevSinks dev_sinks(const apr_ctx* c)
{
    DevSinks s;
    memset(&s, 0, sizeof(s));
    s.n = c->nsink;
    for (int j = 0; j < c->nsink; ++j) {
        for (int k = 0; k < 3; ++k) s.x[j][k] = c->sinks[j].x[k];
        s.m[j] = c->sinks[j].m;
        s.racc[j] = c->sinks[j].racc;
    }
    return s;
}

// ---------------------------------------------------------------- profiling

static void prof_drain(apr_ctx* c)
{
    if (c->ev_used == 0) return;
    cudaStreamSynchronize(c->stream);
    for (int s = 0; s < c->ev_used; ++s) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[2 * s], c->ev[2 * s + 1]) == cudaSuccess) {
            c->prof_ms[c->ev_group[s]] += ms;
            c->prof_calls[c->ev_group[s]] += 1;
        }
    }
    c->ev_used = 0;
}

int prof_begin(apr_ctx* c, int group)
{
    if (!c->prof) return -1;
    if (c->ev_used == PROF_POOL) prof_drain(c);
    int s = c->ev_used++;
    c->ev_group[s] = group;
    cudaEventRecord(c->ev[2 * s], c->stream);
    return s;
}

void prof_end(apr_ctx* c, int slot)
{
    if (slot >= 0) cudaEventRecord(c->ev[2 * slot + 1], c->stream);
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t workspace_layout(const apr_config& cfg, long long cap, char* base, Workspace* W)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        off = align256(off);
        void* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    const size_t C = (size_t)(cap > 0 ? cap : 1);
    const size_t K = (size_t)(cfg.max_neigh > 0 ? cfg.max_neigh : DEFAULT_MAX_NEIGH);
    const size_t ntiles = (C + RADIX_TILE - 1) / RADIX_TILE;
    const size_t scan_n = C > 256 * ntiles ? C : 256 * ntiles;
    const bool f64 = cfg.precision == APR_PREC_FP64;
    Workspace w;
    memset(&w, 0, sizeof(w));
    w.xi = (int4*)take(16 * C);
    w.key[0] = (unsigned long long*)take(8 * C);
    w.key[1] = (unsigned long long*)take(8 * C);
    w.val[0] = (unsigned int*)take(4 * C);
    w.val[1] = (unsigned int*)take(4 * C);
    w.perm_keep = (unsigned int*)take(4 * C);
    w.hist = (unsigned int*)take(4 * 256 * ntiles * 2);
    w.sort_hist = (unsigned int*)take(4 * 256 * 6);
    w.sort_tile = (unsigned int*)take(4 * 256 * std::min<size_t>(ntiles, SORT_SWEEP_MAX_TILES) * 6);
    w.scan_tmp = (unsigned int*)take(4 * (scan_n / 256 + 8192));
    w.pk = (int4*)take(16 * C);
    w.sthr = (unsigned long long*)take(8 * C);
    w.sreach = (unsigned int*)take(4 * C);
    w.sh = (double*)take(8 * C);
    if (f64) {
        w.sx = (double*)take(8 * C);
        w.sy = (double*)take(8 * C);
        w.sz = (double*)take(8 * C);
        w.dA = (double*)take(32 * C);
        w.dV = (double*)take(32 * C);
        w.dB = (double*)take(32 * C);
    } else {
        w.fA = (float4*)take(16 * C);
        w.fV = (float4*)take(16 * C);
        w.fB = (float4*)take(16 * C);
    }
    w.left = (int*)take(4 * C);
    w.right = (int*)take(4 * C);
    w.parent_int = (int*)take(4 * C);
    w.parent_leaf = (int*)take(4 * C);
    w.visit = (int*)take(4 * C);
    w.nlocal = (unsigned char*)take(C);
    w.nlo = (int4*)take(16 * C);
    w.nhi = (int4*)take(16 * C);
    w.nhmax = (double*)take(8 * C);
    w.nthr = (unsigned long long*)take(8 * C);
    w.cflag = (unsigned int*)take(4 * C);
    w.cscan = (unsigned int*)take(4 * C);
    w.cell_first = (int*)take(4 * C);
    w.cell_cnt = (int*)take(4 * C);
    w.cell_node = (int*)take(4 * C);
    w.cmark = (int*)take(4 * C);
    w.acell_first = (int*)take(4 * C);
    w.acell_cnt = (int*)take(4 * C);
    w.acell_node = (int*)take(4 * C);
    w.amark = (unsigned char*)take(C);
    w.cand = (int2*)take(8 * (size_t)max_cand_of((int)K) * C);
    w.ncand = (int*)take(4 * C);
    w.point_q = (int*)take(4 * C);
    w.retry_q[0] = (int*)take(4 * C);
    w.retry_q[1] = (int*)take(4 * C);
    w.active_q = (int*)take(4 * C);
    w.relist_q = (int*)take(4 * C);
    w.qmark = (unsigned int*)take(4 * C);
    w.sthr0 = (unsigned long long*)take(8 * C);
    // the list memory doubles as compaction scratch (20 x 8 bytes per particle)
    w.nbr = (unsigned int*)take((4 * K > 160 ? 4 * K : 160) * C);
    w.ncnt = (int*)take(4 * C);
    w.status = (int*)take(4 * 64);
    w.counters = (unsigned long long*)take(8 * 16);
    w.tgt = (unsigned char*)take(C);
    w.uflag = (unsigned int*)take(4 * C);
    w.uscan = (unsigned int*)take(4 * C);
    w.tmp8 = (double*)take(8 * C);
    w.mset[0] = (unsigned int*)take(4 * C);
    w.mset[1] = (unsigned int*)take(4 * C);
    w.seg_lo[0] = (int*)take(4 * C);
    w.seg_lo[1] = (int*)take(4 * C);
    w.seg_hi[0] = (int*)take(4 * C);
    w.seg_hi[1] = (int*)take(4 * C);
    w.acc_lo = (int4*)take(16 * C * 2);
    w.acc_hi = (int4*)take(16 * C * 2);
    w.acc_sum = (unsigned long long*)take(8 * C * 6);
    w.acc_k = (unsigned int*)take(4 * C * 2);
    w.acc_k2 = (unsigned int*)take(4 * C * 2);
    w.acc_key = (unsigned long long*)take(8 * C * 8);
    w.lflag = (unsigned int*)take(4 * C);
    w.coop = (unsigned int*)take(4 * (2 * COOP_MAX_BLOCKS + 16));
    w.red = (double*)take(8 * 32 * (size_t)RED_BLOCKS);
    w.redout = (double*)take(8 * 32);
    w.bytes = align256(off);
    if (W) *W = w;
    return w.bytes;
}

static apr_status check_cfg(const apr_config* cfg, DevCfg* dc, std::string* why)
{
    if (!cfg) {
        *why = "null config";
        return APR_ERR_ARG;
    }
    if (!(cfg->delta > 0.0) || !(cfg->hfact > 0.0) || !(cfg->m0 > 0.0)) {
        *why = "delta, hfact and m0 must be positive";
        return APR_ERR_ARG;
    }
    if (cfg->lmax < 0 || cfg->lmax >= APR_MAXLEV) {
        *why = "lmax out of range";
        return APR_ERR_ARG;
    }
    if (cfg->precision != APR_PREC_FP32_MIXED && cfg->precision != APR_PREC_FP64) {
        *why = "unknown precision";
        return APR_ERR_ARG;
    }
    if (cfg->kernel != APR_KERNEL_M4 && cfg->kernel != APR_KERNEL_WENDLAND_C2) {
        *why = "unknown kernel";
        return APR_ERR_ARG;
    }
    if (cfg->level_default < 0 || cfg->level_default > cfg->lmax) {
        *why = "level_default must lie in [0, lmax]";
        return APR_ERR_ARG;
    }
    memset(dc, 0, sizeof(*dc));
    dc->kernel = cfg->kernel;
    // W = f(q) / (knorm_inv h^3): M4 1/pi; Wendland C2 21/(16 pi) (unit integral over its support)
    dc->knorm_inv = cfg->kernel == APR_KERNEL_WENDLAND_C2 ? 16.0 * M_PI / 21.0 : M_PI;
    dc->level_default = cfg->level_default;
    for (int k = 0; k < 3; ++k) {
        double L = cfg->box_hi[k] - cfg->box_lo[k];
        if (!(L > 0.0)) {
            *why = "empty box";
            return APR_ERR_ARG;
        }
        double units = L / cfg->delta;
        if (units > (double)(1LL << COORD_BITS)) {
            *why = "box / delta exceeds 2^30 lattice units";
            return APR_ERR_ARG;
        }
        long long Li = llround(units);
        if (cfg->periodic[k] && (double)Li != units) {
            *why = "periodic length is not a whole number of lattice units";
            return APR_ERR_ARG;
        }
        dc->lo[k] = cfg->box_lo[k];
        dc->hi[k] = cfg->box_hi[k];
        dc->L[k] = L;
        dc->periodic[k] = cfg->periodic[k] ? 1 : 0;
        dc->Lint[k] = Li;
    }
    dc->delta = cfg->delta;
    dc->deltaf = (float)cfg->delta;
    {
        int ex = 0;
        const double mant = std::frexp(cfg->delta, &ex);
        dc->inv_delta = mant == 0.5 ? std::ldexp(1.0, 1 - ex) : 0.0;
        dc->inv_delta2 = 2.0 * dc->inv_delta;
    }
    dc->alpha_avf = (float)cfg->alpha_av;
    dc->hfactf = (float)cfg->hfact;
    dc->gammaf = (float)cfg->gamma;
    dc->cs0f = (float)cfg->cs0;
    dc->qcsf = (float)cfg->qcs;
    dc->m0f = (float)cfg->m0;
    dc->beta_avf = (float)cfg->beta_av;
    dc->alpha_uf = (float)cfg->alpha_u;
    dc->hfact = cfg->hfact;
    dc->gamma = cfg->gamma;
    dc->eos = cfg->eos;
    dc->cs0 = cfg->cs0;
    dc->qcs = cfg->qcs;
    dc->alpha_av = cfg->alpha_av;
    dc->beta_av = cfg->beta_av;
    dc->alpha_u = cfg->alpha_u;
    dc->rsep_fac = cfg->rsep_fac;
    dc->dnn_cap = cfg->dnn_cap;
    dc->m0 = cfg->m0;
    dc->m0_knorm = cfg->m0 / dc->knorm_inv;
    dc->lmax = cfg->lmax;
    dc->seed = cfg->seed;
    dc->ccour = cfg->ccour;
    dc->cforce = cfg->cforce;
    dc->G = cfg->G;
    dc->nr_tol = cfg->nr_tol > 0.0 ? cfg->nr_tol
                                   : (cfg->precision == APR_PREC_FP64 ? 1e-12 : 1e-6);
    dc->nr_maxit = cfg->nr_maxit > 0 ? cfg->nr_maxit : 50;
    if (cfg->max_neigh < 0 || cfg->max_neigh % 4 != 0) {
        *why = "max_neigh must be 0 (the default) or a positive multiple of 4";
        return APR_ERR_ARG;
    }
    dc->max_neigh = cfg->max_neigh > 0 ? cfg->max_neigh : DEFAULT_MAX_NEIGH;
    dc->max_cand = max_cand_of(dc->max_neigh);
    return APR_OK;
}

// ------------------------------------------------------------ pass drivers

static apr_status read_status(apr_ctx* c, int first, int count, int* out)
{
    cudaMemcpyAsync(c->hbuf, &c->W.status[first], sizeof(int) * count, cudaMemcpyDeviceToHost,
                    c->stream);
    apr_status s = cuda_check(c, cudaStreamSynchronize(c->stream), "status");
    if (s == APR_OK) memcpy(out, c->hbuf, sizeof(int) * count);
    return s;
}

static apr_status check_overflow(apr_ctx* c)
{
    int st[8];
    // the Morton sort's status word rides along in the same read-back
    cudaMemcpyAsync((int*)c->hbuf + 16, &c->W.status[ST_SORT_ERR], sizeof(int),
                    cudaMemcpyDeviceToHost, c->stream);
    apr_status s = read_status(c, 0, 8, st);
    if (s != APR_OK) return s;
    if (((int*)c->hbuf)[16])
        return fail(c, APR_ERR_STATE, "Morton sort: a tile gave up waiting for its predecessors");
    if (st[ST_TREE_BAD]) return fail(c, APR_ERR_STATE, "internal error: malformed radix tree");
    if (st[0]) return fail(c, APR_ERR_NEIGH_OVERFLOW, "a neighbour list exceeded max_neigh");
    if (st[1]) return fail(c, APR_ERR_NEIGH_OVERFLOW, "a candidate-cell list overflowed");
    return APR_OK;
}

static apr_status run_density(apr_ctx* c, long long* noconv_out)
{
    c->force_data_fresh = false;
    apr_status s = index_sort(c);
    if (s != APR_OK) return s;
    long long unc = 0, noconv = 0, shrinks = 0;
    int attempts = 0, q = 0;
    for (int attempt = 0; attempt < 64; ++attempt) {
        cudaMemsetAsync(c->W.status, 0, 2 * sizeof(int), c->stream);
        if (attempt == 0) {
            // symmetric lists at the reach: if every h converges within it, they
            // also hold every force pair, r < 2 max(h_a, h_b)
            if (c->cfg.precision == APR_PREC_FP32_MIXED && c->cfg.fused_density) {
                // the first pass inside the list build; the particles it does not
                // settle (queued in retry_q[1]) take the density kernel from the start
                int* dq_n = &c->W.status[ST_RETRY_N + 1];
                cudaMemsetAsync(dq_n, 0, sizeof(int), c->stream);
                const FuseArgs fz{c->W.sh, (double)DENSITY_REACH, density_io(c, true), c->W.retry_q[1],
                                  dq_n};
                s = index_lists(c, 1, DENSITY_REACH, true, &fz);
                int nq = 0;
                if (s == APR_OK) s = read_status(c, ST_RETRY_N + 1, 1, &nq);
                if (s != APR_OK) return s;
                s = density_pass(c, &unc, &noconv, c->W.retry_q[1], (long long)nq, q, true);
            } else {
                s = index_lists(c, 1, DENSITY_REACH, true);
                if (s != APR_OK) return s;
                s = density_pass(c, &unc, &noconv, nullptr, 0, q, true);
            }
        } else {
            // only the particles queued by the last pass: their gather lists by a
            // per-particle tree walk at their new h, then their Newton-Raphson
            // (the symmetric lists the force needs are rebuilt after the last attempt)
            s = relist_mark(c, c->W.retry_q[q], &c->W.status[ST_RETRY_N + q], attempt == 1);
            if (s == APR_OK)
                s = index_refresh_sh_queue(c, c->W.retry_q[q], &c->W.status[ST_RETRY_N + q]);
            if (s != APR_OK) return s;
            s = index_lists_queue(c, c->W.retry_q[q], &c->W.status[ST_RETRY_N + q], DENSITY_REACH,
                                  true, false);
            if (s != APR_OK) return s;
            const long long nq = unc;
            s = density_pass(c, &unc, &noconv, c->W.retry_q[q], nq, q ^ 1, true);
            q ^= 1;
        }
        if (s != APR_OK) return s;
        ++attempts;
        shrinks += c->last_shrink;
        c->prof_attempts += 1;
        c->prof_unc += unc;
        c->prof_shrink += c->last_shrink;
        if (unc == 0) break;
    }
    // after retries, the lists around the retried particles are rebuilt at the
    // final h; with them every list holds its force pairs
    c->lists_fresh = attempts == 1;
    if (attempts > 1 && unc == 0) {
        s = relist_finish(c);
        if (s != APR_OK) return s;
        c->lists_fresh = true;
        c->lists_unchecked = true;
    }
    if (noconv_out) *noconv_out = noconv + unc;
    if (unc && shrinks)
        return fail(c, APR_ERR_NEIGH_OVERFLOW,
                    "neighbour lists cannot hold the particles within reach: raise max_neigh");
    if (unc) return fail(c, APR_ERR_NR_NOCONV, "smoothing lengths kept outgrowing their lists");
    // every slot's force records were written by the pass that settled its h
    c->force_data_fresh = true;
    if (noconv) return fail(c, APR_ERR_NR_NOCONV, "h-rho iteration did not converge everywhere");
    return APR_OK;
}

// reuse_density_lists: the lists of a density pass that has just converged on the
// same positions (every h within the lists' reach) contain every force pair
static apr_status run_force(apr_ctx* c, bool reuse_density_lists)
{
    apr_status s;
    if (!reuse_density_lists || !c->lists_fresh) {
        c->lists_unchecked = true;
        if (reuse_density_lists) {
            // same positions as the density pass: the sort stands, only h moved
            s = index_refresh_h(c);
        } else {
            s = index_sort(c);
        }
        if (s != APR_OK) return s;
        cudaMemsetAsync(c->W.status, 0, 2 * sizeof(int), c->stream);
        s = index_lists(c, 1, 1.0);
        if (s != APR_OK) return s;
        c->lists_fresh = true;
    }
    if (!(reuse_density_lists && c->force_data_fresh)) {
        int ps = prof_begin(c, APR_PROF_OTHER);
        s = gather_force_data(c);
        prof_end(c, ps);
        if (s != APR_OK) return s;
    }
    c->force_data_fresh = false;
    s = force_pass(c);
    if (s != APR_OK) return s;
    // lists the density pass built and checked need no second read of the status
    if (c->lists_unchecked) {
        s = check_overflow(c);
        if (s != APR_OK) return s;
        c->lists_unchecked = false;
    }
    int ps = prof_begin(c, APR_PROF_OTHER);
    s = sink_gravity(c);
    prof_end(c, ps);
    if (s != APR_OK) return s;
    c->have_force = true;
    return APR_OK;
}

static void kick_sinks(apr_ctx* c, double hdt)
{
    for (int j = 0; j < c->nsink; ++j)
        for (int d = 0; d < 3; ++d) c->sinks[j].v[d] += hdt * c->sinks[j].a[d];
}

static void track_regions(apr_ctx* c)
{
    for (int j = 0; j < c->nreg; ++j) {
        int t = c->regions[j].track_sink;
        if (t >= 0 && t < c->nsink)
            for (int k = 0; k < 3; ++k) c->regions[j].centre[k] = c->sinks[t].x[k];
    }
}

}  // namespace apr

using namespace apr;

// ---------------------------------------------------------------- the ABI

extern "C" {

apr_status apr_create(apr_ctx** out, const apr_config* cfg, void* stream)
{
    if (!out) return APR_ERR_ARG;
    *out = nullptr;
    DevCfg dc;
    std::string why;
    apr_status s = check_cfg(cfg, &dc, &why);
    if (s != APR_OK) return s;
    apr_ctx* c = new (std::nothrow) apr_ctx();
    if (!c) return APR_ERR_ARG;
    c->cfg = *cfg;
    c->dc = dc;
    c->stream = (cudaStream_t)stream;
    c->bound = false;
    c->have_force = false;
    c->coop_blocks = 0;
    c->lists_fresh = false;
    c->force_data_fresh = false;
    c->prof_attempts = c->prof_unc = c->prof_shrink = 0;
    c->n = c->cap = c->next_id = 0;
    c->step = 0;
    c->nreg = c->nsink = 0;
    c->ncell = 0;
    c->last_shrink = 0;
    c->dt_valid = false;
    c->dt_next = 0.0;
    c->tree_smem_set = false;
    c->launches = 0;
    c->prof = false;
    c->ev_used = 0;
    for (int g = 0; g < APR_NPROF; ++g) {
        c->prof_ms[g] = 0.0;
        c->prof_calls[g] = 0;
    }
    for (int k = 0; k < 2 * PROF_POOL; ++k) c->ev[k] = nullptr;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaMallocHost((void**)&c->hbuf, 4096) != cudaSuccess) {
        delete c;
        return APR_ERR_CUDA;
    }
    *out = c;
    return APR_OK;
}

void apr_destroy(apr_ctx* c)
{
    if (!c) return;
    for (int k = 0; k < 2 * PROF_POOL; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->hbuf) cudaFreeHost(c->hbuf);
    delete c;
}

const char* apr_last_error(const apr_ctx* c) { return c ? c->err.c_str() : "null context"; }

apr_status apr_workspace_size(const apr_config* cfg, long long capacity, size_t* bytes)
{
    if (!cfg || !bytes || capacity < 0) return APR_ERR_ARG;
    *bytes = workspace_layout(*cfg, capacity, nullptr, nullptr);
    return APR_OK;
}

apr_status apr_bind(apr_ctx* c, const apr_particles* p, long long n, long long capacity,
                    long long next_id, void* workspace, size_t bytes)
{
    if (!c || !p) return APR_ERR_ARG;
    if (n < 0 || capacity < n || capacity >= (1LL << 31))
        return fail(c, APR_ERR_ARG, "need 0 <= n <= capacity < 2^31");
    const void* ptrs[] = {p->x,  p->y,    p->z,  p->vx,   p->vy,   p->vz,   p->u,
                          p->h,  p->rho,  p->omega, p->ax, p->ay,   p->az,   p->dudt,
                          p->vsig, p->dnn, p->pres, p->cs, p->level, p->flags, p->id};
    for (const void* q : ptrs)
        if (!q) return fail(c, APR_ERR_ARG, "null particle array");
    size_t need = workspace_layout(c->cfg, capacity, nullptr, nullptr);
    if (!workspace || bytes < need) return fail(c, APR_ERR_WORKSPACE, "workspace too small");
    if (((uintptr_t)workspace) & 255) return fail(c, APR_ERR_ARG, "workspace not 256-byte aligned");
    c->p = *p;
    c->n = n;
    c->cap = capacity;
    c->next_id = next_id;
    c->ws = (char*)workspace;
    c->ws_bytes = bytes;
    workspace_layout(c->cfg, capacity, c->ws, &c->W);
    apr_status s =
        cuda_check(c, cudaMemsetAsync(c->W.status, 0, 4 * 64 + 8 * 16 + 256, c->stream), "bind");
    if (s != APR_OK) return s;
    c->bound = true;
    c->order_valid = false;
    c->have_force = false;
    c->dt_valid = false;
    return APR_OK;
}

// the fields of an apr_particles with their element sizes (bin last, optional)
static int particle_fields(const apr_particles* p, void** ptr, size_t* size)
{
    double* const* d[] = {&p->x,   &p->y,     &p->z,  &p->vx, &p->vy, &p->vz,
                          &p->u,   &p->h,     &p->rho, &p->omega, &p->ax, &p->ay,
                          &p->az,  &p->dudt,  &p->vsig, &p->dnn, &p->pres, &p->cs};
    int k = 0;
    for (double* const* q : d) {
        ptr[k] = *q;
        size[k++] = sizeof(double);
    }
    ptr[k] = p->level;
    size[k++] = 1;
    ptr[k] = p->flags;
    size[k++] = 1;
    ptr[k] = p->id;
    size[k++] = sizeof(unsigned long long);
    ptr[k] = p->bin;
    size[k++] = 1;
    return k;
}

// Host exchange.  Fields whose host arrays are page-locked (hence visible to the
// device) move in one kernel that reads or writes host memory directly: a copy
// call per field costs more than its bytes at these sizes.  Other host arrays go
// through one cudaMemcpyAsync each.
constexpr int COPY_FIELDS = 24;
struct FieldCopy {
    const unsigned char* src[COPY_FIELDS];
    unsigned char* dst[COPY_FIELDS];
    unsigned long long bytes[COPY_FIELDS];
    int n;
};

__global__ void __launch_bounds__(256) k_copy_fields(FieldCopy f)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int j = 0; j < f.n; ++j) {
        const unsigned char* src = f.src[j];
        unsigned char* dst = f.dst[j];
        const long long nb = (long long)f.bytes[j];
        const bool vec = ((reinterpret_cast<size_t>(src) | reinterpret_cast<size_t>(dst)) & 15) == 0;
        const long long nv = vec ? nb / 16 : 0;  // 16-byte words, then single bytes
        for (long long i = t; i < nv; i += stride)
            reinterpret_cast<int4*>(dst)[i] = reinterpret_cast<const int4*>(src)[i];
        for (long long i = 16 * nv + t; i < nb; i += stride) dst[i] = src[i];
    }
}

// the device's address of host memory, or nullptr if it is not page-locked
static void* host_device_ptr(const void* h)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// k fields of n particles between host (hp) and device (dp) arrays
static apr_status copy_fields(apr_ctx* c, void* const* hp, void* const* dp, const size_t* sz, int k,
                              long long n, bool to_device, const char* what)
{
    FieldCopy f;
    f.n = 0;
    long long total = 0;
    for (int j = 0; j < k; ++j) {
        if (!hp[j] || !dp[j] || n == 0) continue;
        const size_t bytes = sz[j] * (size_t)n;
        void* hd = host_device_ptr(hp[j]);
        if (hd && f.n < COPY_FIELDS) {
            f.src[f.n] = (const unsigned char*)(to_device ? hd : dp[j]);
            f.dst[f.n] = (unsigned char*)(to_device ? dp[j] : hd);
            f.bytes[f.n++] = bytes;
            total += (long long)bytes;
            continue;
        }
        apr_status s = cuda_check(
            c,
            cudaMemcpyAsync(to_device ? dp[j] : hp[j], to_device ? hp[j] : dp[j], bytes,
                            to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, c->stream),
            what);
        if (s != APR_OK) return s;
    }
    if (f.n == 0) return APR_OK;
    const long long words = total / 16 + 1;
    const int grid = (int)std::min<long long>(152 * 8, (words + 255) / 256);
    APR_LAUNCH(c, k_copy_fields, grid, 256, f);
    return cuda_check(c, cudaGetLastError(), what);
}

apr_status apr_upload(apr_ctx* c, const apr_particles* host, long long n)
{
    if (!c || !host) return APR_ERR_ARG;
    if (!c->bound) return fail(c, APR_ERR_STATE, "apr_bind first");
    if (n < 0 || n > c->cap) return fail(c, APR_ERR_ARG, "upload needs 0 <= n <= capacity");
    void *hp[24], *dp[24];
    size_t sz[24];
    const int k = particle_fields(host, hp, sz);
    particle_fields(&c->p, dp, sz);
    for (int j = 0; j < k; ++j)
        if (hp[j] && n > 0 && !dp[j])
            return fail(c, APR_ERR_STATE, "upload: no bound array for a given field");
    apr_status s = copy_fields(c, hp, dp, sz, k, n, true, "upload");
    if (s != APR_OK) return s;
    if (n != c->n) c->order_valid = false;  // the kept order is a permutation of n particles
    c->n = n;
    c->dt_valid = false;
    c->lists_fresh = false;
    c->force_data_fresh = false;
    return APR_OK;
}

apr_status apr_download(apr_ctx* c, const apr_particles* host, long long cap, long long* n_out)
{
    if (!c || !host) return APR_ERR_ARG;
    if (!c->bound) return fail(c, APR_ERR_STATE, "apr_bind first");
    const long long n = c->n;
    if (n_out) *n_out = n;
    if (n > cap) return fail(c, APR_ERR_CAPACITY, "download: the host arrays hold fewer than n");
    void *hp[24], *dp[24];
    size_t sz[24];
    const int k = particle_fields(host, hp, sz);
    particle_fields(&c->p, dp, sz);
    apr_status s = copy_fields(c, hp, dp, sz, k, n, false, "download");
    if (s != APR_OK) return s;
    return cuda_check(c, cudaStreamSynchronize(c->stream), "download");
}

apr_status apr_set_regions(apr_ctx* c, const apr_region* r, int nregions)
{
    if (!c || nregions < 0 || nregions > APR_MAXREG || (nregions > 0 && !r)) return APR_ERR_ARG;
    for (int j = 0; j < nregions; ++j) {
        if (r[j].nlev < 0 || r[j].nlev > APR_MAXLEV || r[j].axis < 0 || r[j].axis > 2 ||
            (r[j].shape != APR_SHAPE_SPHERE && r[j].shape != APR_SHAPE_SLAB &&
             r[j].shape != APR_SHAPE_CYLINDER))
            return fail(c, APR_ERR_ARG, "bad region");
        c->regions[j] = r[j];
    }
    c->nreg = nregions;
    return APR_OK;
}

apr_status apr_set_sinks(apr_ctx* c, const apr_sink* s, int nsinks)
{
    if (!c || nsinks < 0 || nsinks > APR_MAXSINK || (nsinks > 0 && !s)) return APR_ERR_ARG;
    for (int j = 0; j < nsinks; ++j) c->sinks[j] = s[j];
    c->nsink = nsinks;
    return APR_OK;
}

apr_status apr_get_sinks(apr_ctx* c, apr_sink* s, int nsinks)
{
    if (!c || nsinks < 0 || nsinks > c->nsink || (nsinks > 0 && !s)) return APR_ERR_ARG;
    for (int j = 0; j < nsinks; ++j) s[j] = c->sinks[j];
    return APR_OK;
}

apr_status apr_get_count(apr_ctx* c, long long* n, long long* next_id, unsigned long long* step)
{
    if (!c) return APR_ERR_ARG;
    if (n) *n = c->n;
    if (next_id) *next_id = c->next_id;
    if (step) *step = c->step;
    return APR_OK;
}

apr_status apr_reorder(apr_ctx* c)
{
    if (!c) return APR_ERR_ARG;
    if (!c->bound) return fail(c, APR_ERR_STATE, "apr_bind first");
    return reorder(c);
}

apr_status apr_sph_density(apr_ctx* c, long long* n_unconverged)
{
    if (!c) return APR_ERR_ARG;
    if (!c->bound) return fail(c, APR_ERR_STATE, "apr_bind first");
    c->dt_valid = false;
    return run_density(c, n_unconverged);
}

apr_status apr_sph_force(apr_ctx* c)
{
    if (!c) return APR_ERR_ARG;
    if (!c->bound) return fail(c, APR_ERR_STATE, "apr_bind first");
    c->dt_valid = false;
    return run_force(c, false);
}

apr_status apr_split_merge(apr_ctx* c, long long* n_out, apr_counts* counts)
{
    if (!c) return APR_ERR_ARG;
    if (!c->bound) return fail(c, APR_ERR_STATE, "apr_bind first");
    apr_counts cnt;
    track_regions(c);
    c->dt_valid = false;
    apr_status s = split_merge_pass(c, &cnt);
    if (n_out) *n_out = c->n;
    if (counts) *counts = cnt;
    return s;
}

apr_status apr_init(apr_ctx* c, const apr_region* regions, int nregions, int* passes)
{
    if (!c) return APR_ERR_ARG;
    if (!c->bound) return fail(c, APR_ERR_STATE, "apr_bind first");
    if (regions) {
        const apr_status sr = apr_set_regions(c, regions, nregions);
        if (sr != APR_OK) return sr;
    } else if (nregions != 0) {
        return fail(c, APR_ERR_ARG, "apr_init: nregions without a region array");
    }
    track_regions(c);
    int np = 0;
    apr_status s;
    for (;;) {
        s = run_density(c, nullptr);
        if (s != APR_OK && s != APR_ERR_NR_NOCONV) return s;
        apr_counts cnt;
        s = split_merge_pass(c, &cnt);
        if (s != APR_OK) return s;
        ++np;
        long long changed = 0;
        for (int l = 0; l < APR_MAXLEV; ++l) changed += cnt.n_split[l] + cnt.n_merge[l];
        if (changed == 0 || np > 4 * APR_MAXLEV) break;
    }
    s = clear_changed(c);
    if (s != APR_OK) return s;
    s = run_density(c, nullptr);
    if (s != APR_OK) return s;
    s = run_force(c, true);
    if (passes) *passes = np;
    if (s != APR_OK) return s;
    apr_stats st_local;
    s = compute_stats_dt(c, &st_local, &c->dt_next);
    c->dt_valid = s == APR_OK;
    return s;
}

apr_status apr_timestep(apr_ctx* c, double* dt)
{
    if (!c || !dt) return APR_ERR_ARG;
    if (!c->bound || !c->have_force) return fail(c, APR_ERR_STATE, "no force pass yet");
    if (c->dt_valid) {
        *dt = c->dt_next;
        return APR_OK;
    }
    return compute_timestep(c, dt);
}

apr_status apr_stats_compute(apr_ctx* c, apr_stats* st)
{
    if (!c || !st) return APR_ERR_ARG;
    if (!c->bound) return fail(c, APR_ERR_STATE, "apr_bind first");
    return compute_stats(c, st);
}

apr_status apr_step(apr_ctx* c, double dt, double* dt_used, apr_stats* stats,
                    apr_counts* counts)
{
    if (!c) return APR_ERR_ARG;
    if (!c->bound || !c->have_force) return fail(c, APR_ERR_STATE, "apr_init or a force pass first");
    apr_status s;
    if (!(dt > 0.0)) {
        if (c->dt_valid) {
            dt = c->dt_next;
        } else {
            s = compute_timestep(c, &dt);
            if (s != APR_OK) return s;
        }
    }
    const double hdt = 0.5 * dt;
    int ps = prof_begin(c, APR_PROF_OTHER);
    s = kick_drift(c, hdt, dt);
    if (s != APR_OK) return s;
    long long na = 0;
    s = accrete(c, &na);
    prof_end(c, ps);
    if (s != APR_OK) return s;
    track_regions(c);
    apr_counts cnt;
    s = split_merge_pass(c, &cnt);
    if (s != APR_OK) return s;
    cnt.n_accreted = na;
    s = run_density(c, nullptr);
    if (s != APR_OK) return s;
    s = run_force(c, true);
    if (s != APR_OK) return s;
    if (dt_used) *dt_used = dt;
    if (counts) *counts = cnt;
    // the closing half kick (point masses here, the gas in the same pass as the
    // conservation sums and the next step's limit)
    kick_sinks(c, hdt);
    apr_stats st_local;
    ps = prof_begin(c, APR_PROF_OTHER);
    s = compute_stats_dt(c, stats ? stats : &st_local, &c->dt_next, hdt);
    prof_end(c, ps);
    if (s != APR_OK) return s;
    c->dt_valid = true;
    return APR_OK;
}

apr_status apr_neighbour_lists(apr_ctx* c, int mode, long long* offsets, int* idx, long long cap,
                               long long* total)
{
    if (!c || !offsets || (mode != 0 && mode != 1)) return APR_ERR_ARG;
    if (!c->bound) return fail(c, APR_ERR_STATE, "apr_bind first");
    const long long n = c->n;
    apr_status s = index_sort(c);
    if (s != APR_OK) return s;
    cudaMemsetAsync(c->W.status, 0, 2 * sizeof(int), c->stream);
    s = index_lists(c, mode, 1.0);
    if (s != APR_OK) return s;
    s = check_overflow(c);
    if (s != APR_OK) return s;
    const int K = c->dc.max_neigh;
    std::vector<unsigned> perm(n), nb((size_t)K * n);
    std::vector<int> cnt(n);
    if (n > 0) {
        cudaMemcpyAsync(perm.data(), c->W.perm, 4 * n, cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(cnt.data(), c->W.ncnt, 4 * n, cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(nb.data(), c->W.nbr, 4 * (size_t)K * n, cudaMemcpyDeviceToHost, c->stream);
    }
    s = cuda_check(c, cudaStreamSynchronize(c->stream), "neighbour lists");
    if (s != APR_OK) return s;
    std::vector<long long> cnt_can(n, 0);
    for (long long sl = 0; sl < n; ++sl) cnt_can[perm[sl]] = cnt[sl];
    offsets[0] = 0;
    for (long long a = 0; a < n; ++a) offsets[a + 1] = offsets[a] + cnt_can[a];
    const long long tot = n > 0 ? offsets[n] : 0;
    if (total) *total = tot;
    if (tot > cap || (tot > 0 && !idx)) return fail(c, APR_ERR_NEIGH_OVERFLOW, "idx too small");
    for (long long sl = 0; sl < n; ++sl) {
        long long a = perm[sl], o = offsets[a];
        for (int k = 0; k < cnt[sl]; ++k) idx[o + k] = (int)perm[nb[(size_t)sl * K + k]];
    }
    return APR_OK;
}

// density of the nq particles of the active queue (sorted slots), with retries
// over the ones that outgrow their lists; their lists come from the cell pass
// when they are many, from per-particle tree walks when they are few
static apr_status run_density_active(apr_ctx* c, long long nq, bool all)
{
    Workspace& W = c->W;
    c->force_data_fresh = false;
    long long unc = 0, noconv = 0, shrinks = 0;
    int attempts = 0, q = 0;
    apr_status s = APR_OK;
    for (int attempt = 0; attempt < 64; ++attempt) {
        cudaMemsetAsync(W.status, 0, 2 * sizeof(int), c->stream);
        if (attempt == 0) {
            s = all ? index_lists(c, 1, DENSITY_REACH, true)
                    : index_lists_cells_of(c, W.active_q, &W.status[ST_ACTIVE_N], DENSITY_REACH,
                                           true);
            if (s == APR_OK) s = density_pass(c, &unc, &noconv, W.active_q, nq, q);
        } else {
            s = relist_mark(c, W.retry_q[q], &W.status[ST_RETRY_N + q], attempt == 1);
            if (s == APR_OK) s = index_refresh_sh_queue(c, W.retry_q[q], &W.status[ST_RETRY_N + q]);
            if (s == APR_OK)
                s = index_lists_queue(c, W.retry_q[q], &W.status[ST_RETRY_N + q], DENSITY_REACH,
                                      true, false);
            const long long nr = unc;
            if (s == APR_OK) s = density_pass(c, &unc, &noconv, W.retry_q[q], nr, q ^ 1);
            q ^= 1;
        }
        if (s != APR_OK) return s;
        ++attempts;
        shrinks += c->last_shrink;
        c->prof_attempts += 1;
        c->prof_unc += unc;
        c->prof_shrink += c->last_shrink;
        if (unc == 0) break;
    }
    c->lists_fresh = attempts == 1;
    if (attempts > 1 && unc == 0) {
        // as in run_density; lists rebuilt for inactive partners go unused
        s = relist_finish(c);
        if (s != APR_OK) return s;
        c->lists_fresh = true;
        c->lists_unchecked = true;
    }
    if (unc && shrinks)
        return fail(c, APR_ERR_NEIGH_OVERFLOW,
                    "neighbour lists cannot hold the particles within reach: raise max_neigh");
    if (unc) return fail(c, APR_ERR_NR_NOCONV, "smoothing lengths kept outgrowing their lists");
    if (noconv) return fail(c, APR_ERR_NR_NOCONV, "h-rho iteration did not converge everywhere");
    return APR_OK;
}

// forces of the particles of the active queue
static apr_status run_force_active(apr_ctx* c, long long nq, bool all)
{
    Workspace& W = c->W;
    apr_status s;
    if (!c->lists_fresh) {
        s = index_refresh_h(c);
        if (s != APR_OK) return s;
        cudaMemsetAsync(W.status, 0, 2 * sizeof(int), c->stream);
        s = all ? index_lists(c, 1, 1.0)
                : index_lists_cells_of(c, W.active_q, &W.status[ST_ACTIVE_N], 1.0, false);
        if (s != APR_OK) return s;
        c->lists_fresh = true;
        c->lists_unchecked = true;
    }
    int ps = prof_begin(c, APR_PROF_OTHER);
    s = gather_force_data(c);
    prof_end(c, ps);
    if (s != APR_OK) return s;
    s = force_pass(c, W.active_q, nq);
    if (s != APR_OK || !c->lists_unchecked) return s;
    c->lists_unchecked = false;
    return check_overflow(c);
}

apr_status apr_step_bins(apr_ctx* c, double dt_max, int B, int init_bins, apr_counts* counts,
                         long long* updates, long long* saturated, apr_stats* stats)
{
    if (!c) return APR_ERR_ARG;
    if (!c->bound) return fail(c, APR_ERR_STATE, "apr_bind first");
    if (!c->p.bin) return fail(c, APR_ERR_STATE, "step_bins: no bin array bound");
    if (!(dt_max > 0.0) || B < 0 || B > 20) return fail(c, APR_ERR_ARG, "step_bins: bad dt_max or max_bin");
    if (!c->have_force) return fail(c, APR_ERR_STATE, "apr_init or a force pass first");
    Workspace& W = c->W;
    apr_counts total;
    memset(&total, 0, sizeof(total));
    long long upd = 0;
    cudaMemsetAsync(&W.status[ST_SATURATED], 0, sizeof(int), c->stream);
    apr_status s = APR_OK;
    if (init_bins) s = bins_init(c, dt_max, B);
    const long long nsub = 1LL << B;
    const double dtmin = dt_max / (double)nsub;
    long long nacc = 0;
    for (long long k = 0; k < nsub && s == APR_OK; ++k) {
        // point masses take every substep (bin B)
        int ps = prof_begin(c, APR_PROF_OTHER);
        s = bins_kick(c, dt_max, B, k, 0);
        kick_sinks(c, 0.5 * dtmin);
        if (s == APR_OK) s = drift(c, dtmin);
        long long na = 0;
        if (s == APR_OK) s = accrete(c, &na);
        prof_end(c, ps);
        if (s != APR_OK) break;
        nacc += na;
        track_regions(c);
        // split/merge over the particles whose step ends now (Sec. 2.5)
        apr_counts cs;
        s = bins_mark_inactive(c, k, B, true);
        if (s == APR_OK) s = split_merge_pass(c, &cs);
        apr_status s2 = bins_mark_inactive(c, k, B, false);
        if (s == APR_OK) s = s2;
        if (s != APR_OK) break;
        for (int l = 0; l < APR_MAXLEV; ++l) {
            total.n_split[l] += cs.n_split[l];
            total.n_merge[l] += cs.n_merge[l];
            total.n_spare[l] = cs.n_spare[l];
        }
        total.n_dead += cs.n_dead;
        long long nq = 0;
        s = index_sort(c);
        ps = prof_begin(c, APR_PROF_OTHER);
        if (s == APR_OK) s = bins_active_queue(c, k, B, &nq);
        prof_end(c, ps);
        const bool all = nq > c->n / 4;
        if (s == APR_OK && nq > 0) s = run_density_active(c, nq, all);
        if (s == APR_OK && nq > 0) s = run_force_active(c, nq, all);
        ps = prof_begin(c, APR_PROF_OTHER);
        if (s == APR_OK) s = sink_gravity(c, B, k + 1);
        if (s == APR_OK) s = bins_kick(c, dt_max, B, k, 1);
        kick_sinks(c, 0.5 * dtmin);
        if (s == APR_OK) s = bins_rebin(c, dt_max, B, k, nq);
        prof_end(c, ps);
        upd += nq;
    }
    c->dt_valid = false;
    c->lists_fresh = false;
    c->force_data_fresh = false;
    if (s != APR_OK) return s;
    int sat = 0;
    cudaMemcpyAsync(c->hbuf, &W.status[ST_SATURATED], sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    s = cuda_check(c, cudaStreamSynchronize(c->stream), "step_bins");
    if (s != APR_OK) return s;
    sat = ((int*)c->hbuf)[0];
    if (stats) {
        s = compute_stats(c, stats);
        if (s != APR_OK) return s;
    }
    total.n_accreted = nacc;
    if (counts) *counts = total;
    if (updates) *updates = upd;
    if (saturated) *saturated = sat;
    c->have_force = true;
    return APR_OK;
}

// the index over the bound particles with symmetric lists at 2 max(h_a, h_b)
static apr_status relax_index(apr_ctx* c)
{
    apr_status s = index_sort(c);
    if (s != APR_OK) return s;
    cudaMemsetAsync(c->W.status, 0, 2 * sizeof(int), c->stream);
    s = index_lists(c, 1, 1.0);
    if (s != APR_OK) return s;
    return check_overflow(c);
}

apr_status apr_relax(apr_ctx* c, const apr_particles* ref, long long nref, int max_iter, double tol,
                     int* iters, double* ke_ratio)
{
    if (!c || !ref || nref < 0 || max_iter < 0 || !(tol >= 0.0)) return APR_ERR_ARG;
    if (!c->bound) return fail(c, APR_ERR_STATE, "apr_bind first");
    if (iters) *iters = 0;
    if (ke_ratio) *ke_ratio = 0.0;
    if (nref > 0 && (!ref->x || !ref->y || !ref->z || !ref->h || !ref->rho || !ref->ax || !ref->ay ||
                     !ref->az || !ref->level || !ref->flags))
        return fail(c, APR_ERR_ARG, "relax: null reference array");
    if (nref > c->cap - c->n) return fail(c, APR_ERR_CAPACITY, "relax needs n + nref <= capacity");
    apr_status s = relax_stage(c, ref, nref);
    if (s != APR_OK) return s;
    double ke0 = 0.0, ke = 0.0;
    int it = 0;
    for (it = 0; it < max_iter; ++it) {
        // a_new at the current positions, then a_ref there, then the shift
        s = run_density(c, nullptr);
        if (s == APR_OK) s = run_force(c, true);
        if (s == APR_OK) s = relax_interp(c, nref, relax_index);
        if (s == APR_OK) s = relax_shift(c, &ke);
        if (s != APR_OK) return s;
        if (it == 0) ke0 = ke;
        if (ke0 <= 0.0 || ke <= tol * ke0) {
            ++it;
            break;
        }
    }
    s = run_density(c, nullptr);
    if (s == APR_OK) s = run_force(c, true);
    if (s == APR_OK) s = clear_new(c);
    c->dt_valid = false;
    if (s != APR_OK) return s;
    if (iters) *iters = it;
    if (ke_ratio) *ke_ratio = ke0 > 0.0 ? ke / ke0 : 0.0;
    return APR_OK;
}

apr_status apr_density_loss_grad(apr_ctx* c, long long npar, const long long* parent,
                                 const double* d, const double* hc, double* loss, double* grad_d,
                                 double* grad_hc)
{
    if (!c || !loss || npar < 0) return APR_ERR_ARG;
    if (!c->bound) return fail(c, APR_ERR_STATE, "apr_bind first");
    *loss = 0.0;
    if (npar > 0 && (!parent || !d || !hc || !grad_d || !grad_hc))
        return fail(c, APR_ERR_ARG, "density loss: null pointer");
    const long long n = c->n;
    if (npar > (c->cap - n) / 2)
        return fail(c, APR_ERR_CAPACITY, "density loss needs n + 2 npar <= capacity");
    if (npar == 0) return APR_OK;
    bool bad = false;
    apr_status s = adjoint_children(c, npar, parent, d, hc, &bad);
    if (s != APR_OK) return s;
    if (bad)
        return fail(c, APR_ERR_ARG,
                    "density loss: a parent is out of range, dead or repeated, or an offset or "
                    "smoothing length is not finite and positive");
    // the index over the combined set; the bound count is restored on every path
    c->n = n + 2 * npar;
    s = index_sort(c);
    if (s == APR_OK) {
        cudaMemsetAsync(c->W.status, 0, 2 * sizeof(int), c->stream);
        s = index_lists(c, 1, 1.0);
    }
    if (s == APR_OK) s = check_overflow(c);
    if (s == APR_OK) s = adjoint_sums(c, n, npar, loss, grad_d, grad_hc);
    c->n = n;
    c->have_force = false;
    c->dt_valid = false;
    c->lists_fresh = false;
    c->force_data_fresh = false;
    return s;
}

apr_status apr_profile_enable(apr_ctx* c, int on)
{
    if (!c) return APR_ERR_ARG;
    if (on) {
        for (int k = 0; k < 2 * PROF_POOL; ++k)
            if (!c->ev[k] && cudaEventCreate(&c->ev[k]) != cudaSuccess)
                return fail(c, APR_ERR_CUDA, "event pool");
        prof_drain(c);
        for (int g = 0; g < APR_NPROF; ++g) {
            c->prof_ms[g] = 0.0;
            c->prof_calls[g] = 0;
        }
        if (c->bound) cudaMemsetAsync(c->W.counters, 0, 8 * 16, c->stream);
    } else {
        prof_drain(c);
    }
    c->prof = on != 0;
    c->dc.prof = on ? 1 : 0;
    return cuda_check(c, cudaGetLastError(), "profile enable");
}

apr_status apr_profile_read(apr_ctx* c, apr_profile* out, int reset)
{
    if (!c || !out) return APR_ERR_ARG;
    prof_drain(c);
    memset(out, 0, sizeof(*out));
    for (int g = 0; g < APR_NPROF; ++g) {
        out->ms[g] = c->prof_ms[g];
        out->calls[g] = c->prof_calls[g];
    }
    out->launches = c->launches;
    out->density_attempts = c->prof_attempts;
    out->uncovered = c->prof_unc;
    out->shrunk = c->prof_shrink;
    if (c->bound) {
        unsigned long long cnt[APR_NPROF];
        apr_status s = cuda_check(c, cudaMemcpyAsync(cnt, c->W.counters, sizeof(cnt),
                                                     cudaMemcpyDeviceToHost, c->stream), "profile");
        if (s == APR_OK) s = cuda_check(c, cudaStreamSynchronize(c->stream), "profile");
        if (s != APR_OK) return s;
        for (int g = 0; g < APR_NPROF; ++g) out->pairs[g] = (double)cnt[g];
        if (reset) cudaMemsetAsync(c->W.counters, 0, 8 * 16, c->stream);
    }
    if (reset) {
        for (int g = 0; g < APR_NPROF; ++g) {
            c->prof_ms[g] = 0.0;
            c->prof_calls[g] = 0;
        }
        c->prof_attempts = c->prof_unc = c->prof_shrink = 0;
    }
    return APR_OK;
}

apr_status apr_merge_pairs(apr_ctx* c, int level, long long* pairs, long long cap,
                           long long* npairs, long long* spare)
{
    if (!c || !pairs || !npairs || !spare || level < 1) return APR_ERR_ARG;
    if (!c->bound) return fail(c, APR_ERR_STATE, "apr_bind first");
    return merge_pairs_debug(c, level, pairs, cap, npairs, spare);
}

}  // extern "C"

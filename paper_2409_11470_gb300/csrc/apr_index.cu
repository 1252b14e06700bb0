// Neighbour index of the APR SPH hot path on sm_103a.
//
// The paper finds neighbours with Phantom's k-d tree (cited in Sec. 2.2 and
// Sec. 2.3); on the GPU the index is rebuilt every density pass instead:
//   1. positions -> integer lattice coordinates -> 63-bit Morton keys;
//   2. stable LSD radix sort of (key, index), 8 passes of 8 bits;
//   3. a binary radix tree over the sorted keys (Karras 2012 construction);
//   4. bottom-up node boxes, particle counts and max h;
//   5. cells = the largest subtrees with <= 32 particles (one warp each);
//   6. per cell, the candidate cells whose box is within kernel reach;
//   7. per particle, the exact neighbour list on the integer lattice,
//      one warp per cell with candidates broadcast lane to lane.
// Every membership decision is an exact integer comparison, so the lists are
// bit-identical to a brute-force search on the same lattice.
#include <cstdio>
#include <type_traits>

#include "apr_density.cuh"
#include "apr_internal.cuh"

namespace apr {

// ------------------------------------------------------------------- scan

// block-local exclusive scan of SCAN_BLOCK items; bsum[block] = the block's total;
// with a single block, *total receives the total
__global__ void k_scan_block(const unsigned int* __restrict__ in, unsigned int* __restrict__ out,
                             unsigned int* __restrict__ bsum, long long n,
                             unsigned int* __restrict__ total)
{
    __shared__ unsigned int wsum[8];
    const long long base = (long long)blockIdx.x * SCAN_BLOCK + 4 * threadIdx.x;
    unsigned int v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0u;
        s += v[k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        unsigned int w = lane < 8 ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            unsigned int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < 8) wsum[lane] = w;
    }
    __syncthreads();
    unsigned int run = incl - s + (wid > 0 ? wsum[wid - 1] : 0u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 255) {
        if (bsum) bsum[blockIdx.x] = wsum[7];
        if (total && gridDim.x == 1) *total = wsum[7];
    }
}

// adds the sum of the preceding block totals (computed here, no second pass);
// the last block writes the grand total
__global__ void k_scan_fix(unsigned int* __restrict__ out, const unsigned int* __restrict__ bsum,
                           long long n, unsigned int* __restrict__ total)
{
    __shared__ unsigned int red[256];
    unsigned int s = 0;
    for (int j = threadIdx.x; j < (int)blockIdx.x; j += 256) s += bsum[j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const unsigned int off = red[0];
    const long long base = (long long)blockIdx.x * SCAN_BLOCK + 4 * threadIdx.x;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (base + k < n) out[base + k] += off;
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = off + bsum[blockIdx.x];
}

__global__ void k_scan_add(unsigned int* __restrict__ out, const unsigned int* __restrict__ boff,
                           long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += boff[i / SCAN_BLOCK];
}

__global__ void k_scan_total(const unsigned int* in, const unsigned int* out, long long n,
                             unsigned int* total)
{
    *total = n > 0 ? out[n - 1] + in[n - 1] : 0u;
}

constexpr long long SCAN_FIX_MAX_BLOCKS = 4096;

static void scan_rec(apr_ctx* c, const unsigned int* in, unsigned int* out, long long n,
                     unsigned int* tmp, unsigned int* total)
{
    const long long nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    if (nb <= 1) {
        APR_LAUNCH(c, k_scan_block, 1, 256, in, out, nullptr, n, total);
        return;
    }
    unsigned int* sums = tmp;
    APR_LAUNCH(c, k_scan_block, (unsigned)nb, 256, in, out, sums, n, nullptr);
    if (nb <= SCAN_FIX_MAX_BLOCKS) {
        APR_LAUNCH(c, k_scan_fix, (unsigned)nb, 256, out, sums, n, total);
        return;
    }
    unsigned int* offs = tmp + nb;
    scan_rec(c, sums, offs, nb, tmp + 2 * nb, nullptr);
    APR_LAUNCH(c, k_scan_add, nblocks(n, 256), 256, out, offs, n);
    if (total) APR_LAUNCH(c, k_scan_total, 1, 1, in, out, n, total);
}

apr_status scan_u32(apr_ctx* c, const unsigned int* in, unsigned int* out, long long n,
                    unsigned int* total_dev)
{
    if (n > 0) scan_rec(c, in, out, n, c->W.scan_tmp, total_dev);
    else if (total_dev) cudaMemsetAsync(total_dev, 0, sizeof(unsigned int), c->stream);
    return cuda_check(c, cudaGetLastError(), "scan");
}

// --------------------------------------------------- lattice and Morton keys

__device__ __forceinline__ long long quant1(const DevCfg& dc, int k, double x)
{
    // a power-of-two unit multiplies (exactly the quotient); the remainder only for
    // the rare coordinate outside the periodic box
    const double t = dc.inv_delta > 0.0 ? (x - dc.lo[k]) * dc.inv_delta : (x - dc.lo[k]) / dc.delta;
    long long q = (long long)floor(t);
    if (dc.periodic[k]) {
        long long L = dc.Lint[k];
        if (q < 0 || q >= L) {
            q %= L;
            if (q < 0) q += L;
        }
    } else {
        if (q < 0) q = 0;
        if (q > COORD_MAX) q = COORD_MAX;
    }
    return q;
}

// spread the low 21 bits of v so that bit k lands on bit 3k
__device__ __forceinline__ unsigned long long spread21(unsigned int v)
{
    unsigned long long x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffULL;
    x = (x | (x << 16)) & 0x001f0000ff0000ffULL;
    x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
    x = (x | (x << 2)) & 0x1249249249249249ULL;
    return x;
}

__global__ void k_quantise(DevCfg dc, const double* __restrict__ x, const double* __restrict__ y,
                           const double* __restrict__ z, const unsigned char* __restrict__ level,
                           long long n, int4* __restrict__ xi, unsigned long long* __restrict__ key,
                           unsigned int* __restrict__ val)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    long long qx = quant1(dc, 0, x[i]), qy = quant1(dc, 1, y[i]), qz = quant1(dc, 2, z[i]);
    xi[i] = make_int4((int)qx, (int)qy, (int)qz, (int)level[i]);
    if (key) {
        const int sh = COORD_BITS - KEY_BITS;
        key[i] = (spread21((unsigned)(qx >> sh)) << 2) | (spread21((unsigned)(qy >> sh)) << 1) |
                 spread21((unsigned)(qz >> sh));
        val[i] = (unsigned)i;
    }
}

apr_status quantise(apr_ctx* c)
{
    APR_LAUNCH(c, k_quantise, nblocks(c->n, 256), 256, c->dc, c->p.x, c->p.y, c->p.z,
                                                          c->p.level, c->n, c->W.xi, nullptr,
                                                          nullptr);
    return cuda_check(c, cudaGetLastError(), "quantise");
}

// ------------------------------------------------------------- radix sort

__global__ void k_radix_hist(const unsigned long long* __restrict__ keys, long long n, int shift,
                             unsigned int* __restrict__ hist, int ntiles)
{
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * RADIX_TILE;
#pragma unroll
    for (int r = 0; r < RADIX_TILE / 256; ++r) {
        long long i = base + r * 256 + threadIdx.x;
        if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// stable scatter: rank of an item = items of the same digit before it in the tile
__global__ void k_radix_scatter(const unsigned long long* __restrict__ kin,
                                const unsigned int* __restrict__ vin,
                                unsigned long long* __restrict__ kout, unsigned int* __restrict__ vout,
                                long long n, int shift, const unsigned int* __restrict__ hoff,
                                int ntiles)
{
    __shared__ unsigned int run[256];
    __shared__ unsigned int wcnt[8][256];
    __shared__ unsigned int goff[256];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    run[t] = 0;
    goff[t] = hoff[(long long)t * ntiles + blockIdx.x];
    for (int w = 0; w < 8; ++w) wcnt[w][t] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const long long base = (long long)blockIdx.x * RADIX_TILE;
    for (int r = 0; r < RADIX_TILE / 256; ++r) {
        long long i = base + r * 256 + t;
        bool valid = i < n;
        unsigned long long k = valid ? kin[i] : 0ULL;
        unsigned int v = valid ? vin[i] : 0u;
        unsigned d = valid ? (unsigned)(k >> shift) & 255u : 256u + lane;  // invalid: unique
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank = __popc(peers & lt);
        if (valid && (peers & lt) == 0) wcnt[wid][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            unsigned pos = goff[d] + run[d] + rank;
            for (int w = 0; w < wid; ++w) pos += wcnt[w][d];
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        unsigned tot = 0;
        for (int w = 0; w < 8; ++w) {
            tot += wcnt[w][t];
            wcnt[w][t] = 0;
        }
        run[t] += tot;
        __syncthreads();
    }
}

__global__ void k_bin_starts(const unsigned int* __restrict__ hoff, int ntiles, int nbins,
                             int* __restrict__ out)
{
    int d = threadIdx.x;
    if (d < nbins) out[d] = (int)hoff[(long long)d * ntiles];
}

apr_status radix_pass8(apr_ctx* c, const unsigned long long* kin, const unsigned int* vin,
                       unsigned long long* kout, unsigned int* vout, long long n, int shift,
                       int* bin_starts, int nbins)
{
    Workspace& W = c->W;
    const int ntiles = nblocks(n, RADIX_TILE);
    APR_LAUNCH(c, k_radix_hist, ntiles, 256, kin, n, shift, W.hist, ntiles);
    scan_u32(c, W.hist, W.hist + (size_t)256 * ntiles, (long long)256 * ntiles, nullptr);
    APR_LAUNCH(c, k_radix_scatter, ntiles, 256, kin, vin, kout, vout, n, shift,
               W.hist + (size_t)256 * ntiles, ntiles);
    if (bin_starts)
        APR_LAUNCH(c, k_bin_starts, 1, 32, W.hist + (size_t)256 * ntiles, ntiles, nbins, bin_starts);
    return cuda_check(c, cudaGetLastError(), "radix pass");
}

// ---- Morton sort in one sweep per digit
//
// The six 8-bit digit histograms are counted in one read of the keys and scanned
// once; each pass then needs a single launch: a tile takes a ticket (so that
// every lower ticket belongs to a block that has already started), counts its
// digits, publishes them, and adds up the counts of the tiles before it by
// looking back over their published words (count with a flag: aggregate only, or
// inclusive prefix), stopping at the first inclusive one.  Its items then go to
// digit offset + tiles before + rank in the tile, the same stable order as a
// histogram-scan-scatter pass.  Waits are bounded; a wait that gives up sets
// ST_SORT_ERR, and no write leaves [0, n).

static_assert(3 * KEY_BITS == 48, "the single-sweep sort takes six 8-bit digits");
constexpr unsigned SORT_FLAG_A = 1u << 30;   // the tile's own counts
constexpr unsigned SORT_FLAG_P = 2u << 30;   // counts of this tile and all before it
constexpr unsigned SORT_COUNT = (1u << 30) - 1u;
constexpr unsigned SORT_SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(256)
    k_sort_hist6(const unsigned long long* __restrict__ keys, long long n,
                 unsigned int* __restrict__ hist6)
{
    __shared__ unsigned int h[6][256];
    for (int k = 0; k < 6; ++k) h[k][threadIdx.x] = 0;
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[i];
#pragma unroll
        for (int k = 0; k < 6; ++k) atomicAdd(&h[k][(unsigned)(key >> (8 * k)) & 255u], 1u);
    }
    __syncthreads();
    for (int k = 0; k < 6; ++k) {
        const unsigned v = h[k][threadIdx.x];
        if (v) atomicAdd(&hist6[k * 256 + threadIdx.x], v);
    }
}

// counts -> exclusive offsets, one pass per warp-group of the block
__global__ void __launch_bounds__(256) k_sort_scan6(unsigned int* __restrict__ hist6)
{
    __shared__ unsigned wsum[8];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int k = 0; k < 6; ++k) {
        const unsigned v = hist6[k * 256 + t];
        unsigned incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        unsigned ex = incl - v;
        for (int w = 0; w < wid; ++w) ex += wsum[w];
        hist6[k * 256 + t] = ex;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
    k_sort_pass(const unsigned long long* __restrict__ kin, const unsigned int* __restrict__ vin,
                unsigned long long* __restrict__ kout, unsigned int* __restrict__ vout, long long n,
                int shift, const unsigned int* __restrict__ goff, unsigned int* tiles,
                unsigned int* ticket, int* err)
{
    __shared__ unsigned s_tile;
    __shared__ unsigned h[256], excl[256], run[256];
    __shared__ unsigned wcnt[8][256];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    if (t == 0) s_tile = atomicAdd(ticket, 1u);
    h[t] = 0;
    run[t] = 0;
    for (int w = 0; w < 8; ++w) wcnt[w][t] = 0;
    __syncthreads();
    const unsigned tile = s_tile;
    const long long base = (long long)tile * RADIX_TILE;
    constexpr int R = RADIX_TILE / 256;
    unsigned long long k[R];
    unsigned int v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const long long i = base + r * 256 + t;
        k[r] = i < n ? kin[i] : 0ULL;
        v[r] = i < n ? vin[i] : 0u;
        if (i < n) atomicAdd(&h[(unsigned)(k[r] >> shift) & 255u], 1u);
    }
    __syncthreads();
    // publish, then the counts of every tile before this one
    unsigned* mine = tiles + (size_t)tile * 256;
    const unsigned own = h[t];
    if (tile == 0) {
        st_release_u32(&mine[t], SORT_FLAG_P | own);
        excl[t] = 0;
    } else {
        st_release_u32(&mine[t], SORT_FLAG_A | own);
        unsigned acc = 0;
        for (long long j = (long long)tile - 1; j >= 0; --j) {
            const unsigned* w = tiles + (size_t)j * 256 + t;
            unsigned word = ld_acquire_u32(w);
            unsigned spins = 0;
            while ((word & ~SORT_COUNT) == 0u && ++spins < SORT_SPIN_LIMIT) word = ld_acquire_u32(w);
            if ((word & ~SORT_COUNT) == 0u) {
                atomicOr(err, 1);
                break;
            }
            acc += word & SORT_COUNT;
            if ((word & ~SORT_COUNT) == SORT_FLAG_P) break;
        }
        excl[t] = acc;
        st_release_u32(&mine[t], SORT_FLAG_P | ((acc + own) & SORT_COUNT));
    }
    __syncthreads();
    // stable ranks within the tile, round by round as the items were loaded
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const long long i = base + r * 256 + t;
        const bool valid = i < n;
        const unsigned d = valid ? (unsigned)(k[r] >> shift) & 255u : 256u + lane;  // invalid: unique
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned rank = __popc(peers & lt);
        if (valid && (peers & lt) == 0) wcnt[wid][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            unsigned long long pos = (unsigned long long)goff[d] + excl[d] + run[d] + rank;
            for (int w = 0; w < wid; ++w) pos += wcnt[w][d];
            if (pos < (unsigned long long)n) {
                kout[pos] = k[r];
                vout[pos] = v[r];
            } else {
                atomicOr(err, 2);
            }
        }
        __syncthreads();
        unsigned tot = 0;
        for (int w = 0; w < 8; ++w) {
            tot += wcnt[w][t];
            wcnt[w][t] = 0;
        }
        run[t] += tot;
        __syncthreads();
    }
}

static apr_status radix_sort(apr_ctx* c, long long n)
{
    Workspace& W = c->W;
    const int ntiles = nblocks(n, RADIX_TILE);
    int cur = 0;
    // the look-back walks past every predecessor that has not yet published its
    // prefix; with all tiles in flight at once that grows with the square of the
    // tile count, so large sorts keep the histogram-scan-scatter passes (measured:
    // 103 tiles 19% faster, 550 tiles 8% slower)
    if (ntiles <= SORT_SWEEP_MAX_TILES) {
        cudaMemsetAsync(W.sort_hist, 0, sizeof(unsigned) * 256 * 6, c->stream);
        cudaMemsetAsync(W.sort_tile, 0, sizeof(unsigned) * 256 * (size_t)ntiles * 6, c->stream);
        cudaMemsetAsync(&W.status[ST_SORT_TICKET], 0, sizeof(int) * 6, c->stream);
        APR_LAUNCH(c, k_sort_hist6, min(ntiles, 152 * 4), 256, W.key[0], n, W.sort_hist);
        APR_LAUNCH(c, k_sort_scan6, 1, 256, W.sort_hist);
        for (int pass = 0; pass < 6; ++pass) {
            APR_LAUNCH(c, k_sort_pass, ntiles, 256, W.key[cur], W.val[cur], W.key[cur ^ 1],
                       W.val[cur ^ 1], n, 8 * pass, W.sort_hist + 256 * pass,
                       W.sort_tile + (size_t)256 * ntiles * pass,
                       (unsigned*)&W.status[ST_SORT_TICKET + pass], &W.status[ST_SORT_ERR]);
            cur ^= 1;
        }
    } else {
        for (int shift = 0; shift < 3 * KEY_BITS; shift += 8) {
            APR_LAUNCH(c, k_radix_hist, ntiles, 256, W.key[cur], n, shift, W.hist, ntiles);
            scan_u32(c, W.hist, W.hist + (size_t)256 * ntiles, (long long)256 * ntiles, nullptr);
            APR_LAUNCH(c, k_radix_scatter, ntiles, 256, W.key[cur], W.val[cur], W.key[cur ^ 1],
                       W.val[cur ^ 1], n, shift, W.hist + (size_t)256 * ntiles, ntiles);
            cur ^= 1;
        }
    }
    W.skey = W.key[cur];
    W.perm = W.val[cur];
    return cuda_check(c, cudaGetLastError(), "radix sort");
}

// ------------------------------------------------------- gather sorted data

__global__ void k_gather_index(long long n, const unsigned int* __restrict__ perm,
                               const int4* __restrict__ xi, const double* __restrict__ h,
                               const double* __restrict__ x, const double* __restrict__ y,
                               const double* __restrict__ z, int4* __restrict__ pk,
                               double* __restrict__ sh, double* __restrict__ sx,
                               double* __restrict__ sy, double* __restrict__ sz)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    unsigned i = perm[s];
    pk[s] = xi[i];
    sh[s] = h[i];
    if (sx) {
        sx[s] = x[i];
        sy[s] = y[i];
        sz[s] = z[i];
    }
}

__global__ void k_gather_h(long long n, const unsigned int* __restrict__ perm,
                           const double* __restrict__ h, double* __restrict__ sh)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) sh[s] = h[perm[s]];
}

// the same for the queued slots only (the h of no other slot has changed since it
// was last needed: between the attempts of a density solve only the queued
// particles are listed and iterated, and the rebuild after them refreshes all)
__global__ void k_gather_h_queue(const int* __restrict__ queue, const int* __restrict__ qlen,
                                 long long n, const unsigned int* __restrict__ perm,
                                 const double* __restrict__ h, double* __restrict__ sh)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= min((long long)*qlen, n)) return;
    const int a = queue[i];
    if (a >= 0 && a < n) sh[a] = h[perm[a]];
}

// ------------------------------------------------------------ radix tree

__device__ __forceinline__ int prefix_len(const unsigned long long* __restrict__ k, int n, int i,
                                          int j)
{
    if (j < 0 || j >= n) return -1;
    unsigned long long a = k[i], b = k[j];
    if (a == b) return 64 + __clz((unsigned)i ^ (unsigned)j);
    return __clzll(a ^ b);
}

// leaves per block of the bottom-up pass (k_tree_up): a node whose leaf range lies
// inside one such block is merged with a shared-memory arrival counter
constexpr int TREE_UP_T = 1024;

__global__ void k_tree_internal(const unsigned long long* __restrict__ k, int n,
                                int* __restrict__ left, int* __restrict__ right,
                                int* __restrict__ parent_int, int* __restrict__ parent_leaf,
                                unsigned char* __restrict__ nlocal)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (prefix_len(k, n, i, i + 1) - prefix_len(k, n, i, i - 1)) > 0 ? 1 : -1;
    int dmin = prefix_len(k, n, i, i - d);
    int lmax = 2;
    while (prefix_len(k, n, i, i + lmax * d) > dmin) lmax *= 2;
    int l = 0;
    for (int t = lmax / 2; t >= 1; t /= 2)
        if (prefix_len(k, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = prefix_len(k, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (prefix_len(k, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int g = i + s * d + (d < 0 ? -1 : 0);
    int lo = min(i, j), hi = max(i, j);
    nlocal[i] = lo / TREE_UP_T == hi / TREE_UP_T;
    int L = (lo == g) ? ~g : g;
    int R = (hi == g + 1) ? ~(g + 1) : g + 1;
    left[i] = L;
    right[i] = R;
    if (L >= 0) parent_int[L] = i;
    else parent_leaf[~L] = i;
    if (R >= 0) parent_int[R] = i;
    else parent_leaf[~R] = i;
}

struct NodeData {
    int lo[3], hi[3], count, first;
    double hmax;
};

__device__ __forceinline__ NodeData node_data(int c, const int4* pk, const double* sh,
                                              const int4* nlo, const int4* nhi, const double* nhmax)
{
    NodeData r;
    if (c < 0) {
        int s = ~c;
        int4 p = pk[s];
        r.lo[0] = r.hi[0] = p.x;
        r.lo[1] = r.hi[1] = p.y;
        r.lo[2] = r.hi[2] = p.z;
        r.count = 1;
        r.first = s;
        r.hmax = sh[s];
    } else {
        int4 a = __ldcg(&nlo[c]), b = __ldcg(&nhi[c]);
        r.lo[0] = a.x;
        r.lo[1] = a.y;
        r.lo[2] = a.z;
        r.count = a.w;
        r.hi[0] = b.x;
        r.hi[1] = b.y;
        r.hi[2] = b.z;
        r.first = b.w;
        r.hmax = __ldcg(&nhmax[c]);
    }
    return r;
}

__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned* p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned atom_add_acq_rel_cta_shared(unsigned* p, unsigned v)
{
    unsigned old;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;"
                 : "=r"(old)
                 : "r"(a), "r"(v)
                 : "memory");
    return old;
}

// bottom-up: the second child to arrive at a node merges both children.  A block
// takes TREE_UP_T consecutive leaves; a node whose leaf range lies inside them
// (nlocal, from the build) is reached only by this block's threads and counts
// arrivals in shared memory, the others in global memory.  Its index is an end of
// its range, so it falls inside the block's index window.
__global__ void __launch_bounds__(TREE_UP_T)
    k_tree_up(int n, const int4* __restrict__ pk, const double* __restrict__ sh,
              const int* __restrict__ left, const int* __restrict__ right,
              const int* __restrict__ parent_int, const int* __restrict__ parent_leaf,
              const unsigned char* __restrict__ nlocal, int* __restrict__ visit, int4* nlo,
              int4* nhi, double* nhmax, int* status)
{
    __shared__ unsigned vis[TREE_UP_T];
    __shared__ unsigned char loc[TREE_UP_T];
    const int b0 = blockIdx.x * TREE_UP_T;
    vis[threadIdx.x] = 0u;
    loc[threadIdx.x] = b0 + (int)threadIdx.x < n - 1 ? nlocal[b0 + threadIdx.x] : 0;
    __syncthreads();
    const int s = b0 + threadIdx.x;
    if (s >= n || n < 2) return;
    int node = parent_leaf[s];
    for (int depth = 0;; ++depth) {
        if (depth > 4 * 64 || node < 0 || node >= n - 1) {  // a valid tree is < 96 deep
            atomicOr(&status[ST_TREE_BAD], 1);
            return;
        }
        // the topology (written by the build, read-only here) loads with the arrival
        // count instead of after it
        const int lcn = __ldg(&left[node]), rcn = __ldg(&right[node]);
        const int par = __ldg(&parent_int[node]);
        // release: this thread's child data (stored just before) is visible to the
        // sibling's thread; acquire: the sibling's child data is visible here (the
        // same block's threads for a local node, any thread for the others)
        const bool local = node >= b0 && node < b0 + TREE_UP_T && loc[node - b0];
        const unsigned old = local ? atom_add_acq_rel_cta_shared(&vis[node - b0], 1u)
                                   : atom_add_acq_rel_u32((unsigned*)&visit[node], 1u);
        if (old == 0u) return;
        NodeData a = node_data(lcn, pk, sh, nlo, nhi, nhmax);
        NodeData b = node_data(rcn, pk, sh, nlo, nhi, nhmax);
        int4 lo = make_int4(min(a.lo[0], b.lo[0]), min(a.lo[1], b.lo[1]), min(a.lo[2], b.lo[2]),
                            a.count + b.count);
        int4 hi = make_int4(max(a.hi[0], b.hi[0]), max(a.hi[1], b.hi[1]), max(a.hi[2], b.hi[2]),
                            min(a.first, b.first));
        __stcg(&nlo[node], lo);
        __stcg(&nhi[node], hi);
        __stcg(&nhmax[node], fmax(a.hmax, b.hmax));
        if (node == 0) return;
        node = par;
    }
}

static apr_status tree_up(apr_ctx* c)
{
    Workspace& W = c->W;
    int n = (int)c->n;
    if (n < 2) return APR_OK;
    cudaMemsetAsync(W.visit, 0, sizeof(int) * (size_t)(n - 1), c->stream);
    APR_LAUNCH(c, k_tree_up, nblocks(n, TREE_UP_T), TREE_UP_T, n, W.pk, W.sh, W.left, W.right,
               W.parent_int, W.parent_leaf, W.nlocal, W.visit, W.nlo, W.nhi, W.nhmax, W.status);
    return cuda_check(c, cudaGetLastError(), "tree up");
}

// The index: a Morton sort and the radix tree over it, or, while the particle set
// and its canonical order are those of a recent sort, a refit: the same order and
// tree topology with every node's box recomputed from the current positions.  The
// lists are exact either way (the candidate search prunes by true bounding boxes
// of each subtree's current members); the order only decides how tight the boxes
// are, so a full sort comes at least every REFIT_MAX + 1 builds.
constexpr int REFIT_MAX = 3;

apr_status index_sort(apr_ctx* c)
{
    Workspace& W = c->W;
    long long n = c->n;
    if (n <= 0) return APR_OK;
    const bool refit = c->order_valid && c->order_n == n && c->order_age < REFIT_MAX;
    int ps = prof_begin(c, APR_PROF_SORT);
    APR_LAUNCH(c, k_quantise, nblocks(n, 256), 256, c->dc, c->p.x, c->p.y, c->p.z, c->p.level,
                                                       n, W.xi, refit ? nullptr : W.key[0],
                                                       refit ? nullptr : W.val[0]);
    apr_status s;
    if (!refit) {
        s = radix_sort(c, n);
        if (s != APR_OK) return s;
        // the order outlives the key buffers, which other passes reuse as scratch
        cudaMemcpyAsync(W.perm_keep, W.perm, sizeof(unsigned) * (size_t)n, cudaMemcpyDeviceToDevice,
                        c->stream);
    }
    W.perm = W.perm_keep;
    const bool f64 = c->cfg.precision == APR_PREC_FP64;
    APR_LAUNCH(c, k_gather_index, nblocks(n, 256), 256, n, W.perm, W.xi, c->p.h, c->p.x, c->p.y,
                                                           c->p.z, W.pk, W.sh, f64 ? W.sx : nullptr,
                                                           W.sy, W.sz);
    prof_end(c, ps);
    ps = prof_begin(c, APR_PROF_TREE);
    if (n >= 2 && !refit)
        APR_LAUNCH(c, k_tree_internal, nblocks(n - 1, 256), 256, W.skey, (int)n, W.left, W.right,
                   W.parent_int, W.parent_leaf, W.nlocal);
    s = cuda_check(c, cudaGetLastError(), "index sort");
    if (s != APR_OK) return s;
    s = tree_up(c);
    prof_end(c, ps);
    if (refit) {
        ++c->order_age;
    } else {
        c->order_valid = true;
        c->order_n = n;
        c->order_age = 0;
    }
    return s;
}

apr_status index_refresh_sh(apr_ctx* c)
{
    if (c->n <= 0) return APR_OK;
    int ps = prof_begin(c, APR_PROF_TREE);
    APR_LAUNCH(c, k_gather_h, nblocks(c->n, 256), 256, c->n, c->W.perm, c->p.h, c->W.sh);
    prof_end(c, ps);
    return cuda_check(c, cudaGetLastError(), "refresh sh");
}

apr_status index_refresh_sh_queue(apr_ctx* c, const int* queue, const int* qlen_dev)
{
    if (c->n <= 0) return APR_OK;
    int ps = prof_begin(c, APR_PROF_TREE);
    APR_LAUNCH(c, k_gather_h_queue, nblocks(c->n, 256), 256, queue, qlen_dev, c->n, c->W.perm,
               c->p.h, c->W.sh);
    prof_end(c, ps);
    return cuda_check(c, cudaGetLastError(), "refresh sh (queue)");
}

apr_status index_refresh_h(apr_ctx* c)
{
    if (c->n <= 0) return APR_OK;
    int ps = prof_begin(c, APR_PROF_TREE);
    APR_LAUNCH(c, k_gather_h, nblocks(c->n, 256), 256, c->n, c->W.perm, c->p.h, c->W.sh);
    apr_status s = cuda_check(c, cudaGetLastError(), "refresh h");
    if (s != APR_OK) return s;
    s = tree_up(c);
    prof_end(c, ps);
    return s;
}

// ------------------------------------------------------------------ cells

__device__ __forceinline__ int node_count(int c, const int4* nlo) { return c < 0 ? 1 : nlo[c].w; }
__device__ __forceinline__ int node_first(int c, const int4* nhi) { return c < 0 ? ~c : nhi[c].w; }

__global__ void k_cells_mark(int n, const int* __restrict__ left, const int* __restrict__ right,
                             const int4* __restrict__ nlo, const int4* __restrict__ nhi,
                             unsigned int* __restrict__ cflag, int* __restrict__ cmark)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    if (nlo[i].w <= CELL_MAX) return;
    int ch[2] = {left[i], right[i]};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        int cc = ch[k];
        if (node_count(cc, nlo) <= CELL_MAX) {
            int f = node_first(cc, nhi);
            if (f >= 0 && f < n) {
                cflag[f] = 1u;
                cmark[f] = cc;
            }
        }
    }
}

__global__ void k_cells_root(int n, unsigned int* cflag, int* cmark)
{
    cflag[0] = 1u;
    cmark[0] = n >= 2 ? 0 : ~0;
}

__global__ void k_cells_compact(int n, const unsigned int* __restrict__ cflag,
                                const unsigned int* __restrict__ cscan,
                                const int* __restrict__ cmark, const int4* __restrict__ nlo,
                                int* __restrict__ cell_first, int* __restrict__ cell_cnt,
                                int* __restrict__ cell_node)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n || !cflag[s]) return;
    int id = (int)cscan[s];
    int node = cmark[s];
    cell_first[id] = s;
    cell_cnt[id] = node_count(node, nlo);
    cell_node[id] = node;
}

// squared lattice distance between two boxes (minimum image on periodic axes)
__device__ __forceinline__ unsigned long long box_dist2(const DevCfg& dc, const int* alo,
                                                        const int* ahi, const int* blo,
                                                        const int* bhi)
{
    unsigned long long d2 = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        long long g = max(0LL, max((long long)blo[k] - ahi[k], (long long)alo[k] - bhi[k]));
        if (dc.periodic[k]) {
            long long L = dc.Lint[k];
            long long g1 = max(0LL, max((long long)blo[k] + L - ahi[k], (long long)alo[k] - bhi[k] - L));
            long long g2 = max(0LL, max((long long)blo[k] - L - ahi[k], (long long)alo[k] - bhi[k] + L));
            g = min(g, min(g1, g2));
        }
        d2 += (unsigned long long)(g * g);
    }
    return d2;
}

// node thresholds thr(reach * max h of the subtree); thr is monotone in h, so the
// symmetric test max(thr_a, thr_b) needs no float64 work during the traversal
__global__ void k_node_thr(DevCfg dc, int n, double reach, const double* __restrict__ nhmax,
                           unsigned long long* __restrict__ nthr)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n - 1) nthr[i] = lattice_threshold(dc, reach * nhmax[i]);
}

struct NodeBox {
    int lo[3], hi[3], count, first;
    unsigned long long thr;
};

// read-only view of a node for the traversal (the tree is complete by now)
__device__ __forceinline__ NodeBox node_box(int c, const int4* __restrict__ pk,
                                            const unsigned long long* __restrict__ sthr,
                                            const int4* __restrict__ nlo,
                                            const int4* __restrict__ nhi,
                                            const unsigned long long* __restrict__ nthr)
{
    NodeBox r;
    if (c < 0) {
        int s = ~c;
        int4 p = __ldg(&pk[s]);
        r.lo[0] = r.hi[0] = p.x;
        r.lo[1] = r.hi[1] = p.y;
        r.lo[2] = r.hi[2] = p.z;
        r.count = 1;
        r.first = s;
        r.thr = __ldg(&sthr[s]);
    } else {
        int4 a = __ldg(&nlo[c]), b = __ldg(&nhi[c]);
        r.lo[0] = a.x;
        r.lo[1] = a.y;
        r.lo[2] = a.z;
        r.count = a.w;
        r.hi[0] = b.x;
        r.hi[1] = b.y;
        r.hi[2] = b.z;
        r.first = b.w;
        r.thr = __ldg(&nthr[c]);
    }
    return r;
}

// candidate cells: one warp per cell walks the tree from the root, popping up to
// 32 nodes at a time from a shared-memory stack and testing them in parallel;
// cells within reach are emitted in a fixed (lane) order, internal nodes within
// reach push their children.  mode 0: the cell's own reach (gather); otherwise
// the larger of the two reaches (symmetric).
constexpr int CAND_STACK = 1024;

__global__ void __launch_bounds__(128)
    k_candidates(DevCfg dc, int mode, const int* __restrict__ ncell_dev, int n,
                 const int* __restrict__ cell_node, const int* __restrict__ left,
                 const int* __restrict__ right, const int4* __restrict__ pk,
                 const unsigned long long* __restrict__ sthr, const int4* __restrict__ nlo,
                 const int4* __restrict__ nhi, const unsigned long long* __restrict__ nthr,
                 int2* __restrict__ cand, int* __restrict__ ncand, int* status, int graceful)
{
    __shared__ int stk[4][CAND_STACK];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int ncell = *ncell_dev;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int cid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; cid < ncell; cid += nwarps) {
        const NodeBox me = node_box(cell_node[cid], pk, sthr, nlo, nhi, nthr);
        const unsigned long long thr_self = me.thr;
        const bool nonper = !(dc.periodic[0] || dc.periodic[1] || dc.periodic[2]);
        __syncwarp();
        if (lane == 0) stk[w][0] = n >= 2 ? 0 : ~0;
        __syncwarp();
        int sp = 1, k = 0;
        bool overflow = false;
        while (sp > 0) {
            const int take = sp < 32 ? sp : 32;
            const bool have = lane < take;
            const int node = have ? stk[w][sp - 1 - lane] : 0;
            sp -= take;
            bool pass = false, cell = false;
            int first = 0, count = 0, lc = 0, rc = 0;
            if (have) {
                const NodeBox o = node_box(node, pk, sthr, nlo, nhi, nthr);
                // the children's indices in the same round trip as the node's box (needed
                // only if it passes, but a second dependent load per round costs more)
                if (node >= 0) {
                    lc = __ldg(&left[node]);
                    rc = __ldg(&right[node]);
                }
                const unsigned long long thr = (mode == 0 || o.thr < thr_self) ? thr_self : o.thr;
                if (nonper) {
                    // in float, widened by 2^-16 relative: a superset of the exact test
                    // (the list kernel culls every staged candidate exactly)
                    const float gx = (float)max(0, max(o.lo[0] - me.hi[0], me.lo[0] - o.hi[0]));
                    const float gy = (float)max(0, max(o.lo[1] - me.hi[1], me.lo[1] - o.hi[1]));
                    const float gz = (float)max(0, max(o.lo[2] - me.hi[2], me.lo[2] - o.hi[2]));
                    pass = fmaf(gz, gz, fmaf(gy, gy, gx * gx)) < (float)thr * (1.0f + 1.0f / 65536.0f);
                } else {
                    pass = box_dist2(dc, me.lo, me.hi, o.lo, o.hi) < thr;
                }
                cell = o.count <= CELL_MAX;
                first = o.first;
                count = o.count;
            }
            const unsigned cm = __ballot_sync(0xffffffffu, pass && cell);
            if (pass && cell) {
                const int pos = k + __popc(cm & lt);
                if (pos < dc.max_cand) cand[(long long)cid * dc.max_cand + pos] = make_int2(first, count);
            }
            k += __popc(cm);
            const unsigned im = __ballot_sync(0xffffffffu, pass && !cell);
            const int nint = __popc(im);
            __syncwarp();  // every lane has read its node before the stack is overwritten
            if (sp + 2 * nint > CAND_STACK) {
                overflow = true;
                break;
            }
            if (pass && !cell) {
                const int pos = sp + 2 * __popc(im & lt);
                stk[w][pos] = rc;
                stk[w][pos + 1] = lc;
            }
            sp += 2 * nint;
            __syncwarp();
        }
        overflow = overflow || k > dc.max_cand;
        // an overflowed cell is not an error: its particles take the per-particle search
        if (lane == 0) ncand[cid] = overflow ? -1 : k;
    }
}

// per particle: the squared-distance threshold and the smallest integer R with
// R^2 >= thr (every neighbour has |dx|, |dy|, |dz| < R on the lattice)
__global__ void k_thresholds(DevCfg dc, long long n, double reach, const double* __restrict__ sh,
                             unsigned long long* __restrict__ thr, unsigned int* __restrict__ rint,
                             int* status)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0) status[ST_POINT_N] = 0;  // the per-particle queue of this list build
    if (s >= n) return;
    const double rad = lattice_radius(dc, reach * sh[s]);
    const unsigned long long t = lattice_threshold_t(rad);
    thr[s] = t;
    // ceil(|radius|) as the start (its square is at least radius^2, so it lies at
    // most a step or two from the root), made exact by the integer steps below
    unsigned long long r = t >= 4611686018427387904ULL ? 2147483648ULL : ceil_bits(rad);
    while (r > 0 && (r - 1) * (r - 1) >= t) --r;
    while (r * r < t) ++r;
    rint[s] = r > 0xffffffffULL ? 0xffffffffu : (unsigned)r;
}

// thresholds of the queued slots only (gather lists of a queue read no other slot's)
__global__ void k_thresholds_queue(DevCfg dc, const int* __restrict__ queue,
                                   const int* __restrict__ qlen, long long n, double reach,
                                   const double* __restrict__ sh, unsigned long long* __restrict__ thr,
                                   unsigned int* __restrict__ rint)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= min((long long)*qlen, n)) return;
    const int s = queue[i];
    if (s < 0 || s >= n) return;
    const double rad = lattice_radius(dc, reach * sh[s]);
    const unsigned long long t = lattice_threshold_t(rad);
    thr[s] = t;
    // ceil(|radius|) as the start (its square is at least radius^2, so it lies at
    // most a step or two from the root), made exact by the integer steps below
    unsigned long long r = t >= 4611686018427387904ULL ? 2147483648ULL : ceil_bits(rad);
    while (r > 0 && (r - 1) * (r - 1) >= t) --r;
    while (r * r < t) ++r;
    rint[s] = r > 0xffffffffULL ? 0xffffffffu : (unsigned)r;
}

// exact lists: warp per cell.  The particles of each candidate cell are culled
// against the cell's bounding box first (exact: a particle whose squared gap to
// the box is >= the larger threshold reaches no particle inside it), moved to
// their periodic image nearest the box centre, and packed into a per-warp batch
// in shared memory; a full batch is read back as broadcasts.  A pair is
// rejected early by the exact per-axis test |d| >= R (R^2 >= thr); the rest
// take the exact 64-bit r^2 < thr.  The image shift is exact while
// w + 2R + 1 <= L on every periodic axis (w: box width): a pair whose true
// minimum image differs from the shifted one is then at least
// L/2 - ceil(w/2) >= R apart on that axis, so both readings reject it.
// Batches holding a particle that breaks this take the per-pair minimum image.
// A batch is tested once it holds LIST_FLUSH candidates (a candidate cell adds at
// most 32): three or four chunks of 32 per batch, so that a batch's ragged last
// chunk and fixed costs are shared by more candidates than with batches of 32.
constexpr int LIST_FLUSH = 96;
constexpr int LIST_BUF = LIST_FLUSH + 32;

__device__ __forceinline__ int wrap_near(int d, int L)
{
    return 2 * d > L ? d - L : (2 * d < -L ? d + L : d);
}

// The first Newton-Raphson pass of the density solve fused into the list build
// (FuseArgs): the per-lane sums of that pass, or nothing.

template <int KT>
struct FusedLane {
    static constexpr bool on = true;
    const unsigned char* lev;  // the staged candidates' levels (their .w holds the slot)
    float unit, hinv, r2max, bestf;
    AccB<float> S, T, U;  // flushed every four entries, as the density kernel does
    unsigned long long best;
    unsigned int npair, nent;
    __device__ __forceinline__ void init(float h, float delta_f)
    {
        unit = delta_f;
        hinv = 1.0f / h;
        r2max = 4.0f * h * h;
        bestf = INFINITY;
        best = ~0ULL;
        npair = 0;
        nent = 0;
    }
    __device__ __forceinline__ void flush()
    {
        S.flush();
        T.flush();
        U.flush();
    }
    // a list entry of lane particle pa: the staged candidate l, q its coordinates as
    // staged (periodic axes: the image nearest the cell; the minimum image is taken
    // again per axis)
    template <int PX, int PY, int PZ>
    __device__ __forceinline__ void hit(const int4& pa, const int4& q, int l, int Lx, int Ly, int Lz)
    {
        int d[3] = {pa.x - q.x, pa.y - q.y, pa.z - q.z};
        if (PX) d[0] = wrap_near(d[0], Lx);
        if (PY) d[1] = wrap_near(d[1], Ly);
        if (PZ) d[2] = wrap_near(d[2], Lz);
        const float r2 = lattice_r2f(unit, d);
        near_update<float>(r2, d, bestf, best);
        density_term<KT, true, float>(r2, hinv, r2max, (int)lev[l], S, T, U, npair);
        if ((++nent & 3u) == 0u) flush();
    }
};

struct NoFuse {
    static constexpr bool on = false;
    template <int PX, int PY, int PZ>
    __device__ __forceinline__ void hit(const int4&, const int4&, int, int, int, int)
    {
    }
};

// gap from coordinate v to [lo, hi], minimum over the periodic images when P
template <int P>
__device__ __forceinline__ long long axis_gap(int v, int lo, int hi, int L)
{
    long long g = max(0LL, max((long long)lo - v, (long long)v - hi));
    if (P) {
        long long g1 = max(0LL, max((long long)lo - (v + (long long)L), (long long)v + L - hi));
        long long g2 = max(0LL, max((long long)lo - (v - (long long)L), (long long)v - L - hi));
        g = min(g, min(g1, g2));
    }
    return g;
}

// the exact test of one staged candidate l against this lane's particle a
// gap from v to [lo, hi]; P: v is the periodic image nearest the box centre, and
// the gap less one (never more than the smallest gap over the images)
template <int P>
__device__ __forceinline__ long long box_gap(int v, int lo, int hi)
{
    const int g = max(0, max(lo - v, v - hi));
    return P ? (long long)max(0, g - 1) : (long long)g;
}

template <int PX, int PY, int PZ, int SYM, bool WRAP>
__device__ __forceinline__ bool exact_pair(const int4& q, unsigned long long tq, unsigned int rq,
                                           const int4& pa, int a, bool own, unsigned long long ta,
                                           unsigned int Ra, int Lx, int Ly, int Lz)
{
    int dx = pa.x - q.x, dy = pa.y - q.y, dz = pa.z - q.z;
    if (WRAP) {
        if (PX) dx = wrap_near(dx, Lx);
        if (PY) dy = wrap_near(dy, Ly);
        if (PZ) dz = wrap_near(dz, Lz);
    }
    unsigned int R = Ra;
    if (SYM) R = (own && rq > R) ? rq : R;
    if ((unsigned)abs(dx) >= R || (unsigned)abs(dy) >= R || (unsigned)abs(dz) >= R) return false;
    if (q.w == a) return false;
    const unsigned long long r2 = (unsigned long long)((long long)dx * dx) +
                                  (unsigned long long)((long long)dy * dy) +
                                  (unsigned long long)((long long)dz * dz);
    unsigned long long th = ta;
    if (SYM) th = tq > th ? tq : th;
    return r2 < th;
}

// A lane's list: slot a's entries go to its row nbr[a * K ...] four at a time (one
// 16-byte store per four entries; K is a multiple of four); entries past K are
// counted but not kept (the list then reads as overflowed)
struct RowWriter {
    unsigned e0 = 0, e1 = 0, e2 = 0, e3 = 0;
    __device__ __forceinline__ void push(unsigned* __restrict__ row, int& m, int K, unsigned v)
    {
        if (m < K) {
            // the last four entries, newest in e3
            e0 = e1;
            e1 = e2;
            e2 = e3;
            e3 = v;
            if ((m & 3) == 3) *reinterpret_cast<uint4*>(row + (m - 3)) = make_uint4(e0, e1, e2, e3);
        }
        ++m;
    }
    // the same with m < K known
    __device__ __forceinline__ void push_room(unsigned* __restrict__ row, int& m, unsigned v)
    {
        e0 = e1;
        e1 = e2;
        e2 = e3;
        e3 = v;
        if ((m & 3) == 3) *reinterpret_cast<uint4*>(row + (m - 3)) = make_uint4(e0, e1, e2, e3);
        ++m;
    }
    // the last one to three entries kept
    __device__ __forceinline__ void finish(unsigned* __restrict__ row, int m, int K) const
    {
        const int mw = m < K ? m : K;
        const int c = mw & 3, base = mw - c;
        if (c == 1) row[base] = e3;
        if (c == 2) {
            row[base] = e2;
            row[base + 1] = e3;
        }
        if (c == 3) {
            row[base] = e1;
            row[base + 1] = e2;
            row[base + 2] = e3;
        }
    }
};

template <int PX, int PY, int PZ, int SYM, bool WRAP, class FZ>
__device__ __forceinline__ void list_batch(int nb, const int4* __restrict__ cq,
                                           const unsigned long long* __restrict__ ct,
                                           const unsigned int* __restrict__ cr, const int4& pa,
                                           int a, bool own, unsigned long long ta, unsigned int Ra,
                                           int Lx, int Ly, int Lz, int K,
                                           unsigned int* __restrict__ row, RowWriter& wr, int& m,
                                           FZ& fz)
{
    for (int l = 0; l < nb; ++l) {
        const int4 q = cq[l];
        if (exact_pair<PX, PY, PZ, SYM, WRAP>(q, SYM ? ct[l] : 0ULL, SYM ? cr[l] : 0u, pa, a, own, ta,
                                             Ra, Lx, Ly, Lz)) {
            wr.push(row, m, K, (unsigned)q.w);
            fz.template hit<PX, PY, PZ>(pa, q, l, Lx, Ly, Lz);
        }
    }
}

// The same decisions through a float filter: the candidate and the lane's
// particle as float coordinates relative to the cell centre (tf: the float
// threshold), r^2 in float; the exact test runs only inside the band
// |r2f - th| <= FILTER_EPS th.  With V the largest relative coordinate of the
// batch and the cell, u = 2^-24, |r2f - r^2| <= 6.93 u V r + 5 u r^2, which at
// r^2 ~ th is at most 1.1e-4 th while V <= FILTER_SPAN sqrt(th); the caller
// checks that bound (th >= the smallest own threshold) before it takes this path.
constexpr float FILTER_EPS = 1.0f / 1024.0f;
constexpr long long FILTER_SPAN = 256;

template <int PX, int PY, int PZ, int SYM, class FZ>
__device__ __forceinline__ void list_batch_fast(int nb, const int4* __restrict__ cq,
                                                const float4* __restrict__ cf,
                                                const unsigned long long* __restrict__ ct,
                                                const unsigned int* __restrict__ cr,
                                                const int4& pa, float pfx, float pfy, float pfz,
                                                float tfa, int a, bool own, unsigned long long ta,
                                                unsigned int Ra, int Lx, int Ly, int Lz, int K,
                                                unsigned int* __restrict__ row, RowWriter& wr,
                                                int& m, FZ& fz)
{
    // Per chunk of 32 staged candidates: first the float tests of every
    // candidate into two bit masks (inside the band's lower edge: a hit; inside
    // the band: undecided), with no branch or store; then the exact tests of
    // the undecided ones (rare: only when some lane of the warp has one); then
    // the hits written in candidate order.  The entries and their order are
    // those of a test-and-write loop over the candidates.  Idle lanes carry NaN
    // coordinates, so none of their tests passes.
    // the band's lower edge th (1 - eps) comes scaled with the thresholds (the
    // staged candidates' too: fl(max(a, b) k) = max(fl(a k), fl(b k))), its upper
    // edge is that times (1 + eps)/(1 - eps); below the upper edge and not a hit
    // is the band
    const float lo_k = 1.0f - FILTER_EPS, hl_k = (1.0f + FILTER_EPS) / (1.0f - FILTER_EPS);
    const float tfl = tfa * lo_k;
    for (int base = 0; base < nb; base += 32) {
        const int cnt = min(32, nb - base);
        unsigned hit = 0u, band = 0u;
        if (cnt == 32) {
            // fully unrolled: every bit position is a constant
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float4 f = cf[base + j];
                const float dx = pfx - f.x, dy = pfy - f.y, dz = pfz - f.z;
                const float r2f = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const float lo = SYM ? fmaxf(tfl, f.w) : tfl;
                hit |= (r2f < lo ? 1u : 0u) << j;
                band |= (r2f <= lo * hl_k ? 1u : 0u) << j;
            }
        } else {
            for (int j = 0; j < cnt; ++j) {
                const float4 f = cf[base + j];
                const float dx = pfx - f.x, dy = pfy - f.y, dz = pfz - f.z;
                const float r2f = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const float lo = SYM ? fmaxf(tfl, f.w) : tfl;
                hit |= (r2f < lo ? 1u : 0u) << j;
                band |= (r2f <= lo * hl_k ? 1u : 0u) << j;
            }
        }
        band &= ~hit;
        if (__any_sync(0xffffffffu, band != 0u)) {
            unsigned bm = band;
            while (bm) {
                const int j = __ffs(bm) - 1;
                bm &= bm - 1u;
                const int l = base + j;
                if (exact_pair<PX, PY, PZ, SYM, false>(cq[l], SYM ? ct[l] : 0ULL, SYM ? cr[l] : 0u,
                                                       pa, a, own, ta, Ra, Lx, Ly, Lz))
                    hit |= 1u << j;
            }
        }
        if (!FZ::on && m + __popc(hit) <= K) {
            // room for every hit of the chunk: no per-entry bound test
            while (hit) {
                const int j = __ffs(hit) - 1;
                hit &= hit - 1u;
                const int b = cq[base + j].w;
                if (b != a) wr.push_room(row, m, (unsigned)b);
            }
        }
        while (hit) {
            const int j = __ffs(hit) - 1;
            hit &= hit - 1u;
            if constexpr (FZ::on) {
                const int4 q = cq[base + j];
                if (q.w != a) {
                    wr.push(row, m, K, (unsigned)q.w);
                    fz.template hit<PX, PY, PZ>(pa, q, base + j, Lx, Ly, Lz);
                }
            } else {
                const int b = cq[base + j].w;
                if (b != a) wr.push(row, m, K, (unsigned)b);
            }
        }
    }
}

// one staged batch: the float filter when the batch's relative coordinates stay
// within FILTER_SPAN times the smallest own R (R - 1 <= sqrt(threshold)), else,
// and for batches that need the per-pair minimum image, the exact tests
template <int PX, int PY, int PZ, int SYM, class FZ>
__device__ __forceinline__ void flush_batch(int nb, bool wrapb, long long vlane, long long vown,
                                            unsigned int rmin, const int4* cq, const float4* cf,
                                            const unsigned long long* ct, const unsigned int* cr,
                                            const int4& pa, float pfx, float pfy, float pfz,
                                            float tfa, int a, bool own, unsigned long long ta,
                                            unsigned int Ra, int Lx, int Ly, int Lz, int K,
                                            unsigned int* row, RowWriter& wr, int& m, FZ& fz)
{
    const long long v = max(vown, (long long)__reduce_max_sync(0xffffffffu, (unsigned)vlane));
    const bool fast = !wrapb && rmin >= 2u && rmin != 0xffffffffu &&
                      v <= FILTER_SPAN * (long long)(rmin - 1u);
    if (wrapb)
        list_batch<PX, PY, PZ, SYM, true>(nb, cq, ct, cr, pa, a, own, ta, Ra, Lx, Ly, Lz, K, row, wr,
                                          m, fz);
    else if (fast)
        list_batch_fast<PX, PY, PZ, SYM>(nb, cq, cf, ct, cr, pa, pfx, pfy, pfz, tfa, a, own, ta, Ra, Lx,
                                         Ly, Lz, K, row, wr, m, fz);
    else
        list_batch<PX, PY, PZ, SYM, false>(nb, cq, ct, cr, pa, a, own, ta, Ra, Lx, Ly, Lz, K, row, wr,
                                           m, fz);
}

// threads per block of the cell list kernel (a warp per cell; a block's cells are
// consecutive in Morton order and share candidate particles in L1)
constexpr int LIST_THREADS = 128;

// FUSE: 0, or 1 + the kernel type of a fused first density pass (FuseArgs)
template <int PX, int PY, int PZ, int SYM, int FUSE>
__global__ void __launch_bounds__(LIST_THREADS)
    k_lists(DevCfg dc, const int* __restrict__ ncell_dev, int n, long long cap,
            const int* __restrict__ cell_first,
            const int* __restrict__ cell_cnt, const int2* __restrict__ cand,
            const int* __restrict__ ncand, const int4* __restrict__ pk,
            const unsigned long long* __restrict__ thr, const unsigned int* __restrict__ rint,
            unsigned int* __restrict__ nbr, int* __restrict__ ncnt, int* __restrict__ point_q,
            int* status, int graceful, unsigned long long* counters, FuseArgs fa)
{
    using FZ = typename std::conditional<FUSE != 0, FusedLane<FUSE - 1>, NoFuse>::type;
    __shared__ int4 cq[LIST_THREADS / 32][LIST_BUF];
    __shared__ float4 cf[LIST_THREADS / 32][LIST_BUF];
    __shared__ unsigned long long ct[LIST_THREADS / 32][LIST_BUF];
    __shared__ unsigned int cr[LIST_THREADS / 32][LIST_BUF];
    __shared__ unsigned char clev[LIST_THREADS / 32][FUSE != 0 ? LIST_BUF : 1];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int ncell = *ncell_dev;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int Lx = (int)dc.Lint[0], Ly = (int)dc.Lint[1], Lz = (int)dc.Lint[2];
    const int K = dc.max_neigh;
    for (int cid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; cid < ncell; cid += nwarps) {
    const int first = cell_first[cid], cnt = cell_cnt[cid];
    if (first < 0 || cnt < 1 || cnt > CELL_MAX || first + cnt > n) continue;
    const bool own = lane < cnt;
    const int a = first + (own ? lane : 0);
    const int4 pa = pk[a];
    const unsigned long long ta = own ? thr[a] : 0ULL;
    const unsigned int Ra = own ? rint[a] : 0u;  // 0: every test fails for idle lanes
    int m = 0;
    const int nc = ncand[cid];
    if (nc < 0) {  // candidate list overflowed: this cell's particles search one by one
        if (own) {
            const int q = atomicAdd(&status[ST_POINT_N], 1);
            if (q < n) point_q[q] = a;
            if constexpr (FUSE != 0) fa.dq[atomicAdd(fa.dq_n, 1)] = a;
        }
        continue;
    }
    // this lane's list row (idle lanes find no entry and write nothing)
    unsigned int* const row = nbr + (long long)a * K;
    RowWriter wr;
    FZ fz;
    double hlist = 1.0;
    if constexpr (FUSE != 0) {
        if (own) hlist = fa.sh[a];
        fz.init((float)hlist, dc.deltaf);
        fz.lev = clev[w];
    }
    // the cell's box, largest threshold and largest R
    const int lox = __reduce_min_sync(FULL, own ? pa.x : INT_MAX);
    const int loy = __reduce_min_sync(FULL, own ? pa.y : INT_MAX);
    const int loz = __reduce_min_sync(FULL, own ? pa.z : INT_MAX);
    const int hix = __reduce_max_sync(FULL, own ? pa.x : INT_MIN);
    const int hiy = __reduce_max_sync(FULL, own ? pa.y : INT_MIN);
    const int hiz = __reduce_max_sync(FULL, own ? pa.z : INT_MIN);
    const unsigned th_hi = __reduce_max_sync(FULL, (unsigned)(ta >> 32));
    const unsigned th_lo = __reduce_max_sync(FULL, (unsigned)(ta >> 32) == th_hi ? (unsigned)ta : 0u);
    const unsigned long long tcell = ((unsigned long long)th_hi << 32) | th_lo;
    const unsigned int rcell = __reduce_max_sync(FULL, Ra);
    const int cx = lox + ((hix - lox) >> 1), cy = loy + ((hiy - loy) >> 1), cz = loz + ((hiz - loz) >> 1);
    // the float filter: this lane's coordinates relative to the centre, the float
    // threshold (-1: idle lane), the smallest own R and the largest relative
    // coordinate so far (own particles: at most half the box, rounded up)
    // idle lanes: NaN coordinates (no float test passes) and no threshold
    const float nan = __int_as_float(0x7fc00000);
    const float pfx = own ? (float)(pa.x - cx) : nan, pfy = own ? (float)(pa.y - cy) : nan,
                pfz = own ? (float)(pa.z - cz) : nan;
    const float tfa = own ? (float)ta : -1.0f;
    const unsigned int rmin = __reduce_min_sync(FULL, own ? Ra : 0xffffffffu);
    const long long vown = max(max(hix - lox, hiy - loy), hiz - loz) / 2 + 1;
    long long vlane = 0;  // largest |coordinate - centre| this lane staged into the batch
    int nb = 0;
    bool wrapb = false;
    // The candidate cells are software-pipelined: the particles of cell j + 1 are
    // loaded (and the entry of cell j + 2 read) before cell j is culled and
    // staged, so that two cells' loads are in flight instead of a chain of two
    // dependent loads per cell.
    const int2* __restrict__ cc = cand + (long long)cid * dc.max_cand;
    auto valid = [&](const int2& c) { return c.x >= 0 && c.y >= 0 && c.y <= CELL_MAX && c.x + c.y <= n; };
    int2 cb_n = nc > 0 ? cc[0] : make_int2(-1, 0);
    int4 q_n = make_int4(0, 0, 0, 0);
    unsigned long long tq_n = 0;
    unsigned int rq_n = 0;
    if (valid(cb_n) && lane < cb_n.y) {
        const int b = cb_n.x + lane;
        q_n = pk[b];
        tq_n = thr[b];
        rq_n = rint[b];
    }
    int2 cb_nn = nc > 1 ? cc[1] : make_int2(-1, 0);
    for (int j = 0; j < nc; ++j) {
        const int2 cb = cb_n;
        int4 q = q_n;
        const unsigned long long tq = tq_n;
        const unsigned int rq = rq_n;
        cb_n = cb_nn;
        if (valid(cb_n) && lane < cb_n.y) {
            const int b = cb_n.x + lane;
            q_n = pk[b];
            tq_n = thr[b];
            rq_n = rint[b];
        }
        cb_nn = j + 2 < nc ? cc[j + 2] : make_int2(-1, 0);
        if (!valid(cb)) continue;
        bool keep = false, nw = false;
        const int lev = q.w;  // pk's fourth word: the level (the staged copy holds the slot)
        if (lane < cb.y) {
            q.w = cb.x + lane;
            const unsigned long long T = (SYM && tq > tcell) ? tq : tcell;
            // periodic axes: the image nearest the box centre is at most one unit
            // farther from the box than the nearest image (the centre rounds
            // down), so its gap less one keeps the culling conservative
            if (PX) q.x = cx + wrap_near(q.x - cx, Lx);
            if (PY) q.y = cy + wrap_near(q.y - cy, Ly);
            if (PZ) q.z = cz + wrap_near(q.z - cz, Lz);
            const long long gx = box_gap<PX>(q.x, lox, hix);
            const long long gy = box_gap<PY>(q.y, loy, hiy);
            const long long gz = box_gap<PZ>(q.z, loz, hiz);
            keep = (unsigned long long)(gx * gx) + (unsigned long long)(gy * gy) +
                       (unsigned long long)(gz * gz) < T;
            if (keep) {
                const long long R2 = 2LL * (long long)((SYM && rq > rcell) ? rq : rcell);
                if (PX) nw = nw || (long long)(hix - lox) + R2 + 1 > Lx;
                if (PY) nw = nw || (long long)(hiy - loy) + R2 + 1 > Ly;
                if (PZ) nw = nw || (long long)(hiz - loz) + R2 + 1 > Lz;
            }
        }
        const unsigned km = __ballot_sync(FULL, keep);
        wrapb = wrapb || __any_sync(FULL, nw);
        if (keep) {
            const int pos = nb + __popc(km & lt);
            const int rx = q.x - cx, ry = q.y - cy, rz = q.z - cz;
            cq[w][pos] = q;
            if constexpr (FUSE != 0) clev[w][pos] = (unsigned char)lev;
            cf[w][pos] = make_float4((float)rx, (float)ry, (float)rz,
                                     (float)tq * (1.0f - FILTER_EPS));
            vlane = max(vlane, (long long)max(max(abs(rx), abs(ry)), abs(rz)));
            if (SYM) {
                ct[w][pos] = tq;
                cr[w][pos] = rq;
            }
        }
        nb += __popc(km);
        __syncwarp();
        if (nb >= LIST_FLUSH) {
            flush_batch<PX, PY, PZ, SYM>(nb, wrapb, vlane, vown, rmin, cq[w], cf[w], ct[w], cr[w], pa,
                                         pfx, pfy, pfz, tfa, a, own, ta, Ra, Lx, Ly, Lz, K, row, wr,
                                         m, fz);
            nb = 0;
            wrapb = false;
            vlane = 0;
            __syncwarp();
        }
    }
    if (nb > 0)
        flush_batch<PX, PY, PZ, SYM>(nb, wrapb, vlane, vown, rmin, cq[w], cf[w], ct[w], cr[w], pa, pfx,
                                     pfy, pfz, tfa, a, own, ta, Ra, Lx, Ly, Lz, K, row, wr, m, fz);
    if (own) {
        wr.finish(row, m, K);
        ncnt[a] = m > K ? -1 : m;
        if (m > K && !graceful) atomicOr(&status[ST_NEIGH_OVERFLOW], 1);
    }
    if constexpr (FUSE != 0) {
        // the pass's Newton-Raphson update, as the density kernel's first iteration
        if (own) {
            bool settled = false;
            if (m <= K) {
                const float mua = level_mass_f(pa.w);
                const float target = float(dc.knorm_inv) * mua * float(dc.hfact * dc.hfact * dc.hfact);
                NRState<float> st{(float)hlist, 0.0f, 0.0f, 0.0f, false, false};
                fz.flush();
                const float hreach = round_down<float>(fa.reach * hlist);
                if (nr_update<float, true>(st, fz.S.s, fz.T.s, fz.U.s, mua, target, (float)dc.nr_tol,
                                           hreach, retry_cap<float>(hreach, m, K)) &&
                    st.conv) {
                    density_store<float>(dc, fa.io, a, pa, st.h, st.D, target, fz.best);
                    settled = true;
                }
            }
            if (!settled) fa.dq[atomicAdd(fa.dq_n, 1)] = a;
        }
    }
    if (dc.prof) {  // list entries written (profiling only)
        const unsigned tot = __reduce_add_sync(FULL, own ? (unsigned)min(m, K) : 0u);
        if (lane == 0) atomicAdd(&counters[APR_PROF_LISTS], (unsigned long long)tot);
    }
    __syncwarp();
    }
}

// the particles of cells whose candidate-cell list overflowed (a large cell in a
// sparse region with a large smoothing length): one warp per particle walks the
// radix tree with the particle's own point-to-box test and tests the particles
// of every cell within reach exactly, a cell at a time in lane order
template <int PX, int PY, int PZ, int SYM>
__global__ void __launch_bounds__(128)
    k_lists_point(DevCfg dc, const int* __restrict__ qlen, const int* __restrict__ point_q, int n,
                  long long cap, const int* __restrict__ left, const int* __restrict__ right,
                  const int4* __restrict__ pk, const unsigned long long* __restrict__ sthr,
                  const int4* __restrict__ nlo, const int4* __restrict__ nhi,
                  const unsigned long long* __restrict__ nthr, unsigned int* __restrict__ nbr,
                  int* __restrict__ ncnt, int* status, int graceful, unsigned long long* counters)
{
    __shared__ int stk[4][CAND_STACK];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int nq = min(*qlen, n);
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int Lx = (int)dc.Lint[0], Ly = (int)dc.Lint[1], Lz = (int)dc.Lint[2];
    const int K = dc.max_neigh;
    for (int qi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; qi < nq; qi += nwarps) {
        const int a = point_q[qi];
        if (a < 0 || a >= n) continue;
        const int4 pa = pk[a];
        const unsigned long long ta = sthr[a];
        __syncwarp();
        if (lane == 0) stk[w][0] = n >= 2 ? 0 : ~0;
        __syncwarp();
        int sp = 1, m = 0;
        bool overflow = false;
        while (sp > 0) {
            const int take = sp < 32 ? sp : 32;
            const bool have = lane < take;
            const int node = have ? stk[w][sp - 1 - lane] : 0;
            sp -= take;
            bool pass = false, cell = false;
            int first = 0, count = 0, lc = 0, rc = 0;
            if (have) {
                const NodeBox o = node_box(node, pk, sthr, nlo, nhi, nthr);
                if (node >= 0) {  // children with the box (see k_candidates)
                    lc = __ldg(&left[node]);
                    rc = __ldg(&right[node]);
                }
                const unsigned long long T = (SYM && o.thr > ta) ? o.thr : ta;
                const long long gx = axis_gap<PX>(pa.x, o.lo[0], o.hi[0], Lx);
                const long long gy = axis_gap<PY>(pa.y, o.lo[1], o.hi[1], Ly);
                const long long gz = axis_gap<PZ>(pa.z, o.lo[2], o.hi[2], Lz);
                pass = (unsigned long long)(gx * gx) + (unsigned long long)(gy * gy) +
                           (unsigned long long)(gz * gz) < T;
                cell = o.count <= CELL_MAX;
                first = o.first;
                count = o.count;
            }
            unsigned cm = __ballot_sync(FULL, pass && cell);
            while (cm) {
                const int src = __ffs(cm) - 1;
                cm &= cm - 1;
                const int f = __shfl_sync(FULL, first, src), cnt = __shfl_sync(FULL, count, src);
                const int b = f + lane;
                bool hit = false;
                if (lane < cnt && b >= 0 && b < n && b != a) {
                    const int4 q = pk[b];
                    int dx = pa.x - q.x, dy = pa.y - q.y, dz = pa.z - q.z;
                    if (PX) dx = wrap_near(dx, Lx);
                    if (PY) dy = wrap_near(dy, Ly);
                    if (PZ) dz = wrap_near(dz, Lz);
                    const unsigned long long r2 = (unsigned long long)((long long)dx * dx) +
                                                  (unsigned long long)((long long)dy * dy) +
                                                  (unsigned long long)((long long)dz * dz);
                    unsigned long long th = ta;
                    if (SYM) {
                        const unsigned long long tb = sthr[b];
                        th = tb > th ? tb : th;
                    }
                    hit = r2 < th;
                }
                const unsigned hm = __ballot_sync(FULL, hit);
                if (hit) {
                    const int pos = m + __popc(hm & lt);
                    if (pos < K) nbr[(long long)a * K + pos] = (unsigned)b;
                }
                m += __popc(hm);
            }
            const unsigned im = __ballot_sync(FULL, pass && !cell);
            const int nint = __popc(im);
            __syncwarp();  // every lane has read its node before the stack is overwritten
            if (sp + 2 * nint > CAND_STACK) {
                overflow = true;
                break;
            }
            if (pass && !cell) {
                const int pos = sp + 2 * __popc(im & lt);
                stk[w][pos] = rc;
                stk[w][pos + 1] = lc;
            }
            sp += 2 * nint;
            __syncwarp();
        }
        if (lane == 0) {
            const bool over = overflow || m > K;
            ncnt[a] = over ? -1 : m;
            if (over && !graceful) atomicOr(&status[ST_NEIGH_OVERFLOW], 1);
            if (dc.prof) atomicAdd(&counters[APR_PROF_LISTS], (unsigned long long)min(m, K));
        }
    }
}

template <int SYM, int FUSE>
static void launch_lists_t(apr_ctx* c, const int* ncell_dev, int n, bool graceful,
                           const int* cell_first, const int* cell_cnt, const FuseArgs& fa)
{
    Workspace& W = c->W;
    const int mask = (c->dc.periodic[0] ? 1 : 0) | (c->dc.periodic[1] ? 2 : 0) |
                     (c->dc.periodic[2] ? 4 : 0);
    const int grid = min(nblocks((long long)n * 32, LIST_THREADS), 152 * 16 * 128 / LIST_THREADS);
#define APR_LISTS_CASE(M, X, Y, Z)                                                                   \
    case M:                                                                                          \
        APR_LAUNCH(c, (k_lists<X, Y, Z, SYM, FUSE>), grid, LIST_THREADS, c->dc, ncell_dev, n, c->cap, \
                   cell_first,                                                                       \
                   cell_cnt, W.cand, W.ncand, W.pk, W.sthr, W.sreach, W.nbr, W.ncnt, W.point_q,      \
                   W.status, graceful ? 1 : 0, W.counters, fa);                                      \
        APR_LAUNCH(c, (k_lists_point<X, Y, Z, SYM>), 152 * 4, 128, c->dc, &W.status[ST_POINT_N],     \
                   W.point_q, n, c->cap, W.left, W.right, W.pk, W.sthr, W.nlo, W.nhi, W.nthr, W.nbr, \
                   W.ncnt, W.status, graceful ? 1 : 0, W.counters);                                  \
        break;
    switch (mask) {
        APR_LISTS_CASE(0, 0, 0, 0)
        APR_LISTS_CASE(1, 1, 0, 0)
        APR_LISTS_CASE(2, 0, 1, 0)
        APR_LISTS_CASE(3, 1, 1, 0)
        APR_LISTS_CASE(4, 0, 0, 1)
        APR_LISTS_CASE(5, 1, 0, 1)
        APR_LISTS_CASE(6, 0, 1, 1)
        APR_LISTS_CASE(7, 1, 1, 1)
    }
#undef APR_LISTS_CASE
}

// fz: the fused first density pass (symmetric lists only), or null
template <int SYM>
static void launch_lists(apr_ctx* c, const int* ncell_dev, int n, bool graceful,
                         const int* cell_first, const int* cell_cnt, const FuseArgs* fz = nullptr)
{
    if constexpr (SYM == 1) {
        if (fz) {
            if (c->cfg.kernel == APR_KERNEL_WENDLAND_C2)
                launch_lists_t<1, 1 + APR_KERNEL_WENDLAND_C2>(c, ncell_dev, n, graceful, cell_first,
                                                              cell_cnt, *fz);
            else
                launch_lists_t<1, 1 + APR_KERNEL_M4>(c, ncell_dev, n, graceful, cell_first, cell_cnt,
                                                     *fz);
            return;
        }
    }
    launch_lists_t<SYM, 0>(c, ncell_dev, n, graceful, cell_first, cell_cnt, FuseArgs{});
}

// lists (graceful: an overflow marks the list, the density pass shrinks h) of the
// queued particles only; the cells and candidate lists are not touched.  sym:
// symmetric lists (r < 2 reach max(h_a, h_b), node h maxima must be current);
// else gather lists (r < 2 reach h_a), which read no neighbour's h
template <int SYM>
static void launch_queue_lists(apr_ctx* c, const int* queue, const int* qlen_dev, int n,
                               bool graceful)
{
    Workspace& W = c->W;
    const int mask = (c->dc.periodic[0] ? 1 : 0) | (c->dc.periodic[1] ? 2 : 0) |
                     (c->dc.periodic[2] ? 4 : 0);
#define APR_QUEUE_CASE(M, X, Y, Z)                                                                   \
    case M:                                                                                          \
        APR_LAUNCH(c, (k_lists_point<X, Y, Z, SYM>), 152 * 4, 128, c->dc, qlen_dev, queue, n, c->cap, \
                   W.left, W.right, W.pk, W.sthr, W.nlo, W.nhi, W.nthr, W.nbr, W.ncnt, W.status,      \
                   graceful ? 1 : 0, W.counters);                                                    \
        break;
    switch (mask) {
        APR_QUEUE_CASE(0, 0, 0, 0)
        APR_QUEUE_CASE(1, 1, 0, 0)
        APR_QUEUE_CASE(2, 0, 1, 0)
        APR_QUEUE_CASE(3, 1, 1, 0)
        APR_QUEUE_CASE(4, 0, 0, 1)
        APR_QUEUE_CASE(5, 1, 0, 1)
        APR_QUEUE_CASE(6, 0, 1, 1)
        APR_QUEUE_CASE(7, 1, 1, 1)
    }
#undef APR_QUEUE_CASE
}

apr_status index_lists_queue(apr_ctx* c, const int* queue, const int* qlen_dev, double reach,
                             bool graceful, bool sym, double node_reach)
{
    Workspace& W = c->W;
    const int n = (int)c->n;
    if (n <= 0) return APR_OK;
    int ps = prof_begin(c, APR_PROF_LISTS);
    if (sym) {
        // symmetric lists read every slot's threshold and the nodes' largest h
        APR_LAUNCH(c, k_thresholds, nblocks(n, 256), 256, c->dc, n, reach, W.sh, W.sthr, W.sreach,
                   W.status);
        if (n >= 2)
            APR_LAUNCH(c, k_node_thr, nblocks(n - 1, 256), 256, c->dc, n,
                       node_reach > 0.0 ? node_reach : reach, W.nhmax, W.nthr);
        launch_queue_lists<1>(c, queue, qlen_dev, n, graceful);
    } else {
        // gather lists read only the queued slots' own thresholds
        APR_LAUNCH(c, k_thresholds_queue, nblocks(n, 256), 256, c->dc, queue, qlen_dev, n, reach,
                   W.sh, W.sthr, W.sreach);
        launch_queue_lists<0>(c, queue, qlen_dev, n, graceful);
    }
    prof_end(c, ps);
    return cuda_check(c, cudaGetLastError(), "queue lists");
}

// ------------------------------------------------- lists after density retries
//
// A density pass keeps the symmetric lists of its first attempt for the force
// when every h converged within their reach.  A particle b that needed retries
// may end with h_b beyond that reach, so a partner y that converged at once can
// lack b in its first list although r_yb < 2 h_b.  Such a y lies in b's last
// list (built at b's last reach): rebuilding, at the final h, the lists of every
// retried particle and of every partner in their last lists that lacks a pair the
// force needs restores every force pair; all other lists already hold theirs.

// mark the slots of a retry queue as retried (2) and queue each once
__global__ void k_relist_mark_queue(const int* __restrict__ queue, const int* __restrict__ qlen,
                                    int n, unsigned int* __restrict__ mark,
                                    int* __restrict__ relist_q, int* __restrict__ relist_n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= min(*qlen, n)) return;
    const int a = queue[i];
    if (a < 0 || a >= n) return;
    if (atomicExch(&mark[a], 2u) != 2u) relist_q[atomicAdd(relist_n, 1)] = a;
}

// warp per retried slot b: a slot y in b's last list is marked (1) and queued when
// the force needs the pair because of b's final h (lattice r^2 below the threshold
// at h_b) and y's first list lacks b (r^2 at or above the larger of the two
// first-build thresholds, which decided that list's membership)
__global__ void k_relist_mark_reach(DevCfg dc, int n, long long cap, int K,
                                    const int* __restrict__ nretried,
                                    const unsigned int* __restrict__ nbr,
                                    const int* __restrict__ ncnt, const int4* __restrict__ pk,
                                    const unsigned int* __restrict__ perm,
                                    const double* __restrict__ h,
                                    const unsigned long long* __restrict__ sthr0,
                                    unsigned int* __restrict__ mark, int* __restrict__ relist_q,
                                    int* __restrict__ relist_n)
{
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int nr = min(*nretried, n);
    const int Lx = (int)dc.Lint[0], Ly = (int)dc.Lint[1], Lz = (int)dc.Lint[2];
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nr; w += nw) {
        const int b = relist_q[w];
        const int m = min(ncnt[b], K);
        const int4 pb = pk[b];
        const unsigned long long tf = lattice_threshold(dc, h[perm[b]]);
        const unsigned long long tb0 = sthr0[b];
        for (int k = lane; k < m; k += 32) {
            const int y = (int)nbr[(long long)b * K + k];
            if (y < 0 || y >= n) continue;
            const int4 py = pk[y];
            const long long dx = min_image32(pb.x - py.x, dc.periodic[0], Lx);
            const long long dy = min_image32(pb.y - py.y, dc.periodic[1], Ly);
            const long long dz = min_image32(pb.z - py.z, dc.periodic[2], Lz);
            const unsigned long long r2 = (unsigned long long)(dx * dx) +
                                          (unsigned long long)(dy * dy) +
                                          (unsigned long long)(dz * dz);
            const unsigned long long t0 = sthr0[y] > tb0 ? sthr0[y] : tb0;
            if (r2 < tf && r2 >= t0 && atomicCAS(&mark[y], 0u, 1u) == 0u)
                relist_q[atomicAdd(relist_n, 1)] = y;
        }
    }
}

apr_status relist_mark(apr_ctx* c, const int* queue, const int* qlen_dev, bool first)
{
    Workspace& W = c->W;
    const int n = (int)c->n;
    if (first) {
        cudaMemsetAsync(W.qmark, 0, sizeof(unsigned) * (size_t)n, c->stream);
        cudaMemsetAsync(&W.status[ST_RELIST_N], 0, sizeof(int), c->stream);
        // the first build's thresholds, before the retries recompute them
        cudaMemcpyAsync(W.sthr0, W.sthr, sizeof(unsigned long long) * (size_t)n,
                        cudaMemcpyDeviceToDevice, c->stream);
    }
    if (n > 0)
        APR_LAUNCH(c, k_relist_mark_queue, nblocks(n, 256), 256, queue, qlen_dev, n, W.qmark,
                   W.relist_q, &W.status[ST_RELIST_N]);
    return cuda_check(c, cudaGetLastError(), "relist mark");
}

// After a density solve with retries, the radix tree's largest h per node is
// brought up to date without a bottom-up pass over the whole tree: a particle that
// converged on its first list ended within that list's reach, reach x its h at the
// build, so reach x the build's node maximum bounds it; a retried particle raises
// its ancestors' maxima itself.  The values are stored in build units (h / reach,
// rounded up) and compared as their float64 bit patterns, which order like the
// values for positive numbers; an ancestor already at or above the value stops
// the walk (every ancestor of a node holds at least its maximum).
__global__ void k_hmax_raise(const int* __restrict__ queue, const int* __restrict__ qlen, int n,
                             const double* __restrict__ sh, const int* __restrict__ parent_leaf,
                             const int* __restrict__ parent_int, double* nhmax, double inv_reach)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= min(*qlen, n) || n < 2) return;
    const int s = queue[i];
    if (s < 0 || s >= n) return;
    const double v = sh[s] * inv_reach * (1.0 + 0x1p-50);
    const unsigned long long vb = (unsigned long long)__double_as_longlong(v);
    int node = parent_leaf[s];
    for (int depth = 0; depth < 4 * 64 && node >= 0 && node < n - 1; ++depth) {
        const unsigned long long old = atomicMax((unsigned long long*)&nhmax[node], vb);
        if (old >= vb || node == 0) break;
        node = parent_int[node];
    }
}

apr_status relist_finish(apr_ctx* c)
{
    Workspace& W = c->W;
    const int n = (int)c->n;
    if (n <= 0) return APR_OK;
    int ps = prof_begin(c, APR_PROF_LISTS);
    cudaMemcpyAsync(&W.status[ST_RETRIED_N], &W.status[ST_RELIST_N], sizeof(int),
                    cudaMemcpyDeviceToDevice, c->stream);
    APR_LAUNCH(c, k_relist_mark_reach, 152 * 8, 256, c->dc, n, c->cap, c->dc.max_neigh,
               &W.status[ST_RETRIED_N], W.nbr, W.ncnt, W.pk, W.perm, c->p.h, W.sthr0, W.qmark,
               W.relist_q, &W.status[ST_RELIST_N]);
    prof_end(c, ps);
    apr_status s = index_refresh_sh(c);
    if (s != APR_OK) return s;
    ps = prof_begin(c, APR_PROF_TREE);
    // the retried particles are the first ST_RETRIED_N entries of the relist queue
    APR_LAUNCH(c, k_hmax_raise, nblocks(n, 256), 256, W.relist_q, &W.status[ST_RETRIED_N], n, W.sh,
               W.parent_leaf, W.parent_int, W.nhmax, 1.0 / (double)DENSITY_REACH);
    prof_end(c, ps);
    s = cuda_check(c, cudaGetLastError(), "node h raise");
    if (s != APR_OK) return s;
    return index_lists_queue(c, W.relist_q, &W.status[ST_RELIST_N], 1.0, false, true,
                             (double)DENSITY_REACH);
}

apr_status index_lists(apr_ctx* c, int mode, double reach, bool graceful, const FuseArgs* fz)
{
    Workspace& W = c->W;
    int n = (int)c->n;
    if (n <= 0) {
        c->ncell = 0;
        return APR_OK;
    }
    cudaStream_t st = c->stream;
    int ps = prof_begin(c, APR_PROF_LISTS);
    cudaMemsetAsync(W.cflag, 0, sizeof(unsigned) * (size_t)n, st);
    if (n <= CELL_MAX)
        APR_LAUNCH(c, k_cells_root, 1, 1, n, W.cflag, W.cmark);
    else
        APR_LAUNCH(c, k_cells_mark, nblocks(n - 1, 256), 256, n, W.left, W.right, W.nlo, W.nhi, W.cflag,
                                                           W.cmark);
    int* ncell_dev = &W.status[ST_NCELL];
    scan_u32(c, W.cflag, W.cscan, n, (unsigned*)ncell_dev);
    APR_LAUNCH(c, k_cells_compact, nblocks(n, 256), 256, n, W.cflag, W.cscan, W.cmark, W.nlo,
               W.cell_first, W.cell_cnt, W.cell_node);
    APR_LAUNCH(c, k_thresholds, nblocks(n, 256), 256, c->dc, n, reach, W.sh, W.sthr, W.sreach,
               W.status);
    if (n >= 2) APR_LAUNCH(c, k_node_thr, nblocks(n - 1, 256), 256, c->dc, n, reach, W.nhmax, W.nthr);
    APR_LAUNCH(c, k_candidates, min(nblocks((long long)n * 32, 128), 152 * 16), 128, c->dc, mode,
               ncell_dev, n,
               W.cell_node, W.left, W.right, W.pk, W.sthr, W.nlo, W.nhi, W.nthr, W.cand, W.ncand,
               W.status, graceful ? 1 : 0);
    if (mode == 0)
        launch_lists<0>(c, ncell_dev, n, graceful, W.cell_first, W.cell_cnt);
    else
        launch_lists<1>(c, ncell_dev, n, graceful, W.cell_first, W.cell_cnt, fz);
    prof_end(c, ps);
    return cuda_check(c, cudaGetLastError(), "lists");
}

// ---- symmetric lists of the cells that hold a queued particle
//
// For a queue that is a small part of the particles (the active particles of a
// time-step bin), clustered in space as bins follow the flow: the cells that
// hold one of them take the warp-per-cell path, which costs a few particles'
// worth of a per-particle tree walk.  Every particle of such a cell gets its
// list; the queued ones are among them.

__global__ void k_mark_queue_slots(const int* __restrict__ queue, const int* __restrict__ qlen,
                                   int n, unsigned char* __restrict__ amark)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= min(*qlen, n)) return;
    const int a = queue[i];
    if (a >= 0 && a < n) amark[a] = 1;
}

// the cells with a marked slot, appended in any order (each cell's lists are
// built on their own)
__global__ void k_active_cells(const int* __restrict__ ncell_dev, int n,
                               const int* __restrict__ cell_first, const int* __restrict__ cell_cnt,
                               const int* __restrict__ cell_node,
                               const unsigned char* __restrict__ amark, int* __restrict__ acell_first,
                               int* __restrict__ acell_cnt, int* __restrict__ acell_node,
                               int* __restrict__ nactive)
{
    const int cid = blockIdx.x * blockDim.x + threadIdx.x;
    if (cid >= min(*ncell_dev, n)) return;
    const int f = cell_first[cid], cnt = cell_cnt[cid];
    if (f < 0 || cnt < 1 || f + cnt > n) return;
    bool any = false;
    for (int k = 0; k < cnt && !any; ++k) any = amark[f + k] != 0;
    if (!any) return;
    const int slot = atomicAdd(nactive, 1);
    acell_first[slot] = f;
    acell_cnt[slot] = cnt;
    acell_node[slot] = cell_node[cid];
}

apr_status index_lists_cells_of(apr_ctx* c, const int* queue, const int* qlen_dev, double reach,
                                bool graceful)
{
    Workspace& W = c->W;
    int n = (int)c->n;
    if (n <= 0) return APR_OK;
    cudaStream_t st = c->stream;
    int ps = prof_begin(c, APR_PROF_LISTS);
    cudaMemsetAsync(W.cflag, 0, sizeof(unsigned) * (size_t)n, st);
    if (n <= CELL_MAX)
        APR_LAUNCH(c, k_cells_root, 1, 1, n, W.cflag, W.cmark);
    else
        APR_LAUNCH(c, k_cells_mark, nblocks(n - 1, 256), 256, n, W.left, W.right, W.nlo, W.nhi, W.cflag,
                   W.cmark);
    int* ncell_dev = &W.status[ST_NCELL];
    scan_u32(c, W.cflag, W.cscan, n, (unsigned*)ncell_dev);
    APR_LAUNCH(c, k_cells_compact, nblocks(n, 256), 256, n, W.cflag, W.cscan, W.cmark, W.nlo,
               W.cell_first, W.cell_cnt, W.cell_node);
    cudaMemsetAsync(W.amark, 0, (size_t)n, st);
    cudaMemsetAsync(&W.status[ST_ACELL_N], 0, sizeof(int), st);
    APR_LAUNCH(c, k_mark_queue_slots, nblocks(n, 256), 256, queue, qlen_dev, n, W.amark);
    APR_LAUNCH(c, k_active_cells, nblocks(n, 256), 256, ncell_dev, n, W.cell_first, W.cell_cnt,
               W.cell_node, W.amark, W.acell_first, W.acell_cnt, W.acell_node, &W.status[ST_ACELL_N]);
    APR_LAUNCH(c, k_thresholds, nblocks(n, 256), 256, c->dc, n, reach, W.sh, W.sthr, W.sreach,
               W.status);
    if (n >= 2) APR_LAUNCH(c, k_node_thr, nblocks(n - 1, 256), 256, c->dc, n, reach, W.nhmax, W.nthr);
    int* nac = &W.status[ST_ACELL_N];
    APR_LAUNCH(c, k_candidates, min(nblocks((long long)n * 32, 128), 152 * 16), 128, c->dc, 1, nac, n,
               W.acell_node, W.left, W.right, W.pk, W.sthr, W.nlo, W.nhi, W.nthr, W.cand, W.ncand,
               W.status, graceful ? 1 : 0);
    launch_lists<1>(c, nac, n, graceful, W.acell_first, W.acell_cnt);
    prof_end(c, ps);
    return cuda_check(c, cudaGetLastError(), "active-cell lists");
}

}  // namespace apr

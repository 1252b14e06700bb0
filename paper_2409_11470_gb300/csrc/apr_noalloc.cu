// Conservation sums that allocate nothing.
//
// apr_stats_compute reduces into the caller's workspace.  Some callers have
// no workspace to give and may not call cudaMalloc at all: code that runs
// inside another framework's memory manager (a raw allocation would bypass
// its accounting and pool), or a latency-critical callback where an
// allocation could implicitly synchronise the device or fail under a memory
// cap.  This entry point serves them: its scratch (one row of partial sums
// per thread block plus the final sums) is a file-scope device array that
// exists from library load until process exit on every GPU that loads the
// library.
#include <cstring>
#include <mutex>

#include "apr_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_ITEMS = 16;                     // particles per thread
constexpr int NA_MAX_BLOCKS = 4096;
constexpr int NA_NV = 9;                         // sums per block
constexpr long long NA_MAX_N = (long long)NA_MAX_BLOCKS * NA_THREADS * NA_ITEMS;  // 16,777,216
constexpr int NA_ROW = 16;                       // doubles per partial row
constexpr int NA_MAX_DEVICES = 64;

// the scratch: NA_MAX_BLOCKS partial rows, then one row of final sums (512 KB + 128 B)
static __device__ __align__(256) double g_na_scratch[(NA_MAX_BLOCKS + 1) * NA_ROW];

__global__ void __launch_bounds__(NA_THREADS)
    k_na_partial(long long n, double m0, int adiabatic, apr_particles p, double* scratch)
{
    double v[NA_NV];
    for (int k = 0; k < NA_NV; ++k) v[k] = 0.0;
    const long long base = (long long)blockIdx.x * NA_THREADS * NA_ITEMS + threadIdx.x;
    for (int r = 0; r < NA_ITEMS; ++r) {
        const long long i = base + (long long)r * NA_THREADS;
        if (i >= n || (p.flags[i] & APR_FLAG_DEAD)) continue;
        const double m = m0 * apr::level_mass_d(p.level[i]);
        const double vx = p.vx[i], vy = p.vy[i], vz = p.vz[i];
        v[0] += m;
        v[1] += m * vx;
        v[2] += m * vy;
        v[3] += m * vz;
        v[4] += m * (p.y[i] * vz - p.z[i] * vy);
        v[5] += m * (p.z[i] * vx - p.x[i] * vz);
        v[6] += m * (p.x[i] * vy - p.y[i] * vx);
        v[7] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        if (adiabatic) v[8] += m * p.u[i];
    }
    __shared__ double sm[NA_NV][NA_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < NA_NV; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sm[k][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < NA_NV) {
        double x = 0.0;
        for (int w = 0; w < NA_THREADS / 32; ++w) x += sm[threadIdx.x][w];
        scratch[(long long)blockIdx.x * NA_ROW + threadIdx.x] = x;  // every row is overwritten
    }
}

// one block: fixed-shape tree over the used rows -> final row
__global__ void __launch_bounds__(NA_THREADS) k_na_final(int nblk, double* scratch)
{
    __shared__ double sm[NA_THREADS];
    double* out = scratch + (long long)NA_MAX_BLOCKS * NA_ROW;
    for (int k = 0; k < NA_NV; ++k) {
        double x = 0.0;
        for (int b = threadIdx.x; b < nblk; b += NA_THREADS) x += scratch[(long long)b * NA_ROW + k];
        sm[threadIdx.x] = x;
        __syncthreads();
        for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sm[0];
        __syncthreads();
    }
}

std::mutex g_na_mutex;
double* g_na_ptr[NA_MAX_DEVICES];

void put_err(char* err, size_t len, const char* msg)
{
    if (err && len > 0) {
        strncpy(err, msg, len - 1);
        err[len - 1] = '\0';
    }
}

}  // namespace

extern "C" apr_status apr_stats_noalloc(const apr_config* cfg, const apr_particles* p,
                                        long long n, const apr_sink* sinks, int nsinks,
                                        void* stream, apr_stats* out, char* err, size_t errlen)
{
    if (!cfg || !p || !out || n < 0 || nsinks < 0 || nsinks > APR_MAXSINK || (nsinks && !sinks)) {
        put_err(err, errlen, "apr_stats_noalloc: null pointer or negative size");
        return APR_ERR_ARG;
    }
    if (n > NA_MAX_N) {
        put_err(err, errlen,
                "apr_stats_noalloc: n exceeds the fixed scratch (at most 16,777,216 particles); "
                "use apr_stats_compute with a workspace");
        return APR_ERR_ARG;
    }
    if (n > 0 && (!p->x || !p->y || !p->z || !p->vx || !p->vy || !p->vz || !p->u || !p->level ||
                  !p->flags)) {
        put_err(err, errlen, "apr_stats_noalloc: null particle array");
        return APR_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        put_err(err, errlen, "apr_stats_noalloc: no current CUDA device");
        return APR_ERR_CUDA;
    }
    {
        // every call reads its result back and synchronises the stream, neither of
        // which a stream under capture allows
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess ||
            cs != cudaStreamCaptureStatusNone) {
            (void)cudaGetLastError();
            put_err(err, errlen, "apr_stats_noalloc: the stream is under capture (or invalid)");
            return APR_ERR_ARG;
        }
    }
    double* scratch;
    {
        // once per device, with that device current: the device address of the array
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_na_scratch);
            if (e != cudaSuccess || !ptr) {
                put_err(err, errlen, "apr_stats_noalloc: cudaGetSymbolAddress failed");
                return APR_ERR_CUDA;
            }
            g_na_ptr[dev] = (double*)ptr;
        }
        scratch = g_na_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nblk = (int)((n + (long long)NA_THREADS * NA_ITEMS - 1) / ((long long)NA_THREADS * NA_ITEMS));
    if (nblk > 0)
        k_na_partial<<<nblk, NA_THREADS, 0, st>>>(n, cfg->m0, cfg->eos == APR_EOS_ADIABATIC ? 1 : 0,
                                                  *p, scratch);
    k_na_final<<<1, NA_THREADS, 0, st>>>(nblk, scratch);
    // a launch that failed leaves the final row as the previous call wrote it:
    // report the launch error instead of reading that row back
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        put_err(err, errlen, cudaGetErrorString(e));
        return APR_ERR_CUDA;
    }
    double r[NA_NV];
    e = cudaMemcpyAsync(r, scratch + (long long)NA_MAX_BLOCKS * NA_ROW, sizeof(r),
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        put_err(err, errlen, cudaGetErrorString(e));
        return APR_ERR_CUDA;
    }
    memset(out, 0, sizeof(*out));
    out->mass = r[0];
    for (int k = 0; k < 3; ++k) {
        out->mom[k] = r[1 + k];
        out->ang[k] = r[4 + k];
    }
    out->ekin = r[7];
    out->etherm = r[8];
    for (int j = 0; j < nsinks; ++j) {
        const apr_sink& s = sinks[j];
        out->mass += s.m;
        for (int d = 0; d < 3; ++d) out->mom[d] += s.m * s.v[d];
        out->ang[0] += s.m * (s.x[1] * s.v[2] - s.x[2] * s.v[1]);
        out->ang[1] += s.m * (s.x[2] * s.v[0] - s.x[0] * s.v[2]);
        out->ang[2] += s.m * (s.x[0] * s.v[1] - s.x[1] * s.v[0]);
        out->ekin += 0.5 * s.m * (s.v[0] * s.v[0] + s.v[1] * s.v[1] + s.v[2] * s.v[2]);
    }
    put_err(err, errlen, "");
    return APR_OK;
}

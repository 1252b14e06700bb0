// Arithmetic peak probe of the fused multiply-add pipes (a measurement aid for
// the pair kernels' rooflines, not a step of the method).
//
// Every thread runs PROBE_CHAINS independent FMA chains x <- x * a + b, so the
// pipes never wait on a result; the grid fills every SM with the largest number
// of resident blocks.  FLOPs per launch = 2 * PROBE_CHAINS * PROBE_UNROLL *
// iters * threads.  The chains converge to b / (1 - a) and stay finite; their
// sum is compared with a value it never takes, so that the compiler keeps them
// (nothing is stored in practice).
#include "apr_internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_UNROLL = 16;

static __device__ double g_probe_sink;

__device__ __forceinline__ float fma_(float x, float a, float b) { return fmaf(x, a, b); }
__device__ __forceinline__ double fma_(double x, double a, double b) { return fma(x, a, b); }

template <typename R>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_chain(int iters, R a, R b, R never)
{
    R x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = R(threadIdx.x + k) * R(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u) {
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fma_(x[k], a, b);
        }
    }
    R s = R(0);
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
    if (s == never) g_probe_sink = (double)s;
}

template <typename R>
apr_status run_probe(int iters, cudaStream_t st, double* tflops, double* ms_out)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chain<R>, PROBE_THREADS, 0) !=
            cudaSuccess ||
        sms <= 0 || per_sm <= 0)
        return APR_ERR_CUDA;
    const int grid = sms * per_sm;
    const R a = R(0.9999999), b = R(1e-7), never = R(-1);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return APR_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return APR_ERR_CUDA;
    }
    k_fma_chain<R><<<grid, PROBE_THREADS, 0, st>>>(iters, a, b, never);  // warm-up
    cudaEventRecord(e0, st);
    k_fma_chain<R><<<grid, PROBE_THREADS, 0, st>>>(iters, a, b, never);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || ms <= 0.0f) return APR_ERR_CUDA;
    const double flops =
        2.0 * PROBE_CHAINS * PROBE_UNROLL * (double)iters * (double)grid * PROBE_THREADS;
    *tflops = flops / (ms * 1e-3) / 1e12;
    *ms_out = ms;
    return APR_OK;
}

}  // namespace

extern "C" apr_status apr_probe_fma_peak(int precision, int iters, void* stream, double* tflops,
                                         double* ms)
{
    if (!tflops || !ms || iters < 1 ||
        (precision != APR_PREC_FP32_MIXED && precision != APR_PREC_FP64))
        return APR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    return precision == APR_PREC_FP64 ? run_probe<double>(iters, st, tflops, ms)
                                      : run_probe<float>(iters, st, tflops, ms);
}

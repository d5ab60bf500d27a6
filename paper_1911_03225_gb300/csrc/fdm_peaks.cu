// fdm_peaks.cu -- measured arithmetic rates of the GPU, the denominators of the roofline
// fractions of the step kernels that are bound by arithmetic rather than by memory.
//
// Each thread runs kChains independent multiply-add chains (enough independent work for
// the pipe's latency), on every SM, for a number of iterations calibrated so that a timed
// launch lasts about 50 ms; the rate is the multiply-adds done over the launch's CUDA-event
// duration, two flops each.  The double-word rate counts one double-word multiply followed
// by one double-word add (the library's FP32-pair arithmetic) as two FP64-equivalent flops.
#include <cmath>

#include "fdm_device.cuh"
#include "fdm_host.h"

namespace fdm {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T> __device__ __forceinline__ T fma_step(T a, T b, T c);
template <> __device__ __forceinline__ double fma_step(double a, double b, double c) { return __fma_rn(a, b, c); }
template <> __device__ __forceinline__ float fma_step(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ df fma_step(df a, df b, df c) { return a * b + c; }

template <typename T> __device__ __forceinline__ double as_double(T v) { return (double)v; }

// a <- a b + c converges to c / (1 - b) for |b| < 1, so the chains stay finite for any
// iteration count; the store depends on every chain, so no chain can be dropped
template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(long long iters, double* sink) {
    T a[kChains];
    const T b = T(0.999999f), c = T(1e-7f);
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = T(float(threadIdx.x + k) * 1e-3f);
    for (long long i = 0; i < iters; i += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma_step(a[k], b, c);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += as_double(a[k]);
    if (s == -1.0) sink[blockIdx.x] = s;   // never true; keeps the chains live
}

template <typename T>
fdm_status measure(cudaStream_t st, double* gflops) {
    int dev = 0, sms = 0;
    FDM_CK(cudaGetDevice(&dev));
    FDM_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = 0;
    FDM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chain_kernel<T>, kThreads, 0));
    if (per_sm < 1) return FDM_ERR_DEVICE;
    const int blocks = sms * per_sm;
    double* sink = nullptr;
    if (cudaMalloc(&sink, (size_t)blocks * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return FDM_ERR_OOM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    fdm_status rc = FDM_OK;
    auto timed = [&](long long iters, float* ms) -> cudaError_t {
        cudaError_t e;
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess) return e;
        fma_chain_kernel<T><<<blocks, kThreads, 0, st>>>(iters, sink);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaEventRecord(e1, st)) != cudaSuccess) return e;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
        return cudaEventElapsedTime(ms, e0, e1);
    };
    do {
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) { rc = FDM_ERR_DEVICE; break; }
        // calibrate: grow the iteration count until a launch takes a few ms, then scale to ~50 ms
        long long iters = 256;
        float ms = 0.f;
        for (;;) {
            if (timed(iters, &ms) != cudaSuccess) { rc = FDM_ERR_DEVICE; break; }
            if (ms > 5.f || iters > (1ll << 40)) break;
            iters *= 4;
        }
        if (rc != FDM_OK) break;
        iters = (long long)((double)iters * 50.0 / (double)ms) / 4 * 4;
        if (iters < 4) iters = 4;
        float best = 0.f;
        for (int r = 0; r < 3; ++r) {
            if (timed(iters, &ms) != cudaSuccess) { rc = FDM_ERR_DEVICE; break; }
            if (r == 0 || ms < best) best = ms;
        }
        if (rc != FDM_OK) break;
        const double fmas = (double)blocks * kThreads * kChains * (double)iters;
        *gflops = 2.0 * fmas / ((double)best * 1e-3) / 1e9;
    } while (0);
    if (rc != FDM_OK) cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
}

// y[i] = the FP64 stencil's reciprocal square root (op 0) or reciprocal (op 1) of x[i]
__global__ void fp64_math_kernel(int op, const double* __restrict__ x, double* __restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = op == 0 ? trsqrt(x[i]) : trcp(x[i]);
}

}  // namespace
}  // namespace fdm

using namespace fdm;

extern "C" fdm_status fdm_debug_fp64_math(int32_t op, const double* x, double* y, int64_t n) {
    if ((op != 0 && op != 1) || n < 0 || (n > 0 && (!x || !y))) return FDM_ERR_INVALID_ARG;
    if (n == 0) return FDM_OK;
    double* d = nullptr;
    if (cudaMalloc(&d, (size_t)n * 2 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return FDM_ERR_OOM;
    }
    fdm_status rc = FDM_OK;
    if (cudaMemcpy(d, x, (size_t)n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) rc = FDM_ERR_DEVICE;
    if (rc == FDM_OK) {
        const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
        fp64_math_kernel<<<blocks, 256>>>(op, d, d + n, (long long)n);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(y, d + n, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = FDM_ERR_DEVICE;
    }
    if (rc != FDM_OK) cudaGetLastError();
    cudaFree(d);
    return rc;
}

extern "C" fdm_status fdm_measure_arith_rate(int32_t precision, void* stream, double* gflops) {
    if (!gflops) return FDM_ERR_INVALID_ARG;
    *gflops = 0.0;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == FDM_FP64) return measure<double>(s, gflops);
    if (precision == FDM_MIXED) return measure<float>(s, gflops);
    if (precision == FDM_DF64) return measure<df>(s, gflops);
    return FDM_ERR_INVALID_ARG;
}

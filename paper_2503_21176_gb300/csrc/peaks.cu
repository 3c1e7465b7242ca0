// Throughput microbenchmarks of the pipes the real-space pair sum runs on: FP32
// fused multiply-add, FP64 fused multiply-add and the special-function unit
// (MUFU, one reciprocal square root per operation).  The real-space kernels are
// bound by these pipes rather than by memory, so their roofline fractions are
// quoted against the rates measured here on the running GPU and clock.
//
// Each kernel runs independent dependency chains per thread (enough of them to
// hide the pipe latency), over a grid of resident blocks on every SM, and keeps
// its result alive through a store that never happens.  Rates are operations
// per second from CUDA events, best of three timed launches after a warm-up.

#include "internal.cuh"

namespace qeq {
namespace {

constexpr int kPeakThreads = 512;
constexpr int kPeakBlocksPerSm = 2;

template <int ILP>
__global__ void __launch_bounds__(kPeakThreads) k_peak_fma32(int iters, float b, float c,
                                                            float *sink) {
    float a[ILP];
#pragma unroll
    for (int i = 0; i < ILP; ++i) a[i] = 1e-3f * (float)(threadIdx.x + i);
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int i = 0; i < ILP; ++i) a[i] = fmaf(a[i], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < ILP; ++i) s += a[i];
    if (s == -1.25e30f) sink[blockIdx.x] = s;
}

template <int ILP>
__global__ void __launch_bounds__(kPeakThreads) k_peak_fma64(int iters, double b, double c,
                                                            double *sink) {
    double a[ILP];
#pragma unroll
    for (int i = 0; i < ILP; ++i) a[i] = 1e-3 * (double)(threadIdx.x + i);
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int i = 0; i < ILP; ++i) a[i] = fma(a[i], b, c);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < ILP; ++i) s += a[i];
    if (s == -1.25e300) sink[blockIdx.x] = s;
}

__device__ __forceinline__ float mufu_rsqrt(float x) {
    float y;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x <- 1 / sqrt(x) converges to 1 and stays finite; one MUFU instruction per step.
template <int ILP>
__global__ void __launch_bounds__(kPeakThreads) k_peak_mufu(int iters, float *sink) {
    float a[ILP];
#pragma unroll
    for (int i = 0; i < ILP; ++i) a[i] = 1.5f + 1e-3f * (float)(threadIdx.x + i);
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int i = 0; i < ILP; ++i) a[i] = mufu_rsqrt(a[i]);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < ILP; ++i) s += a[i];
    if (s == -1.25e30f) sink[blockIdx.x] = s;
}

constexpr int kIlp32 = 8, kIlp64 = 4, kIlpMufu = 8;

// Best rate (operations per second) of three timed launches; ops_per_launch
// counts one FMA as two floating-point operations.
template <typename Launch>
int time_best(Launch launch, double ops_per_launch, cudaStream_t s, double *rate) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return QEQ_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return QEQ_ERR_CUDA;
    }
    launch();  // warm-up (clocks ramp, module load)
    double best = 0.0;
    cudaError_t err = cudaGetLastError();
    for (int r = 0; r < 3 && err == cudaSuccess; ++r) {
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
        err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && ms > 0.f) {
            const double r_ops = ops_per_launch / (1e-3 * (double)ms);
            if (r_ops > best) best = r_ops;
        }
    }
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *rate = best;
    return err == cudaSuccess ? QEQ_OK : QEQ_ERR_CUDA;
}

}  // namespace
}  // namespace qeq

using namespace qeq;

QEQ_API int qeq_measure_peaks(double *out4, void *stream) {
    if (!out4) return set_error(nullptr, QEQ_ERR_INVALID, "measure_peaks: out4 is NULL");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms <= 0)
        return set_error(nullptr, QEQ_ERR_CUDA, "measure_peaks: device query failed");
    cudaStream_t s = (cudaStream_t)stream;
    float *sink32 = nullptr;
    double *sink64 = nullptr;
    const int blocks = sms * kPeakBlocksPerSm;
    e = cudaMalloc(&sink32, sizeof(float) * blocks);
    if (e == cudaSuccess) e = cudaMalloc(&sink64, sizeof(double) * blocks);
    if (e != cudaSuccess) {
        cudaFree(sink32);
        return set_error(nullptr, QEQ_ERR_NOMEM, "measure_peaks: sink allocation failed");
    }
    const double threads = (double)blocks * kPeakThreads;
    // iteration counts sized for a few milliseconds per launch at the nominal rates
    const int it32 = 16384, it64 = 512, itm = 2048;
    int rc = time_best(
        [&] { k_peak_fma32<kIlp32><<<blocks, kPeakThreads, 0, s>>>(it32, 0.999f, 1e-3f, sink32); },
        2.0 * threads * kIlp32 * 8.0 * it32, s, &out4[0]);
    if (!rc)
        rc = time_best(
            [&] { k_peak_fma64<kIlp64><<<blocks, kPeakThreads, 0, s>>>(it64, 0.999, 1e-3, sink64); },
            2.0 * threads * kIlp64 * 8.0 * it64, s, &out4[1]);
    if (!rc)
        rc = time_best([&] { k_peak_mufu<kIlpMufu><<<blocks, kPeakThreads, 0, s>>>(itm, sink32); },
                       threads * kIlpMufu * 8.0 * itm, s, &out4[2]);
    out4[3] = (double)sms;
    cudaFree(sink32);
    cudaFree(sink64);
    if (rc) return set_error(nullptr, rc, "measure_peaks: a timed launch failed");
    return QEQ_OK;
}

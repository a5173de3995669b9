// Throughput probes of the SM's arithmetic pipes: the measured denominators of the rooflines of
// the ALU-bound kernels (FP32 multiply-add for the FP32 path, FP64 multiply-add for the MIXED
// update, the special-function unit for the sin/cos/log/rsqrt of propagation and scattering).
// Each thread runs kChains independent dependency chains, so the pipe, not the latency of one
// chain, bounds the rate; the chains' ends are stored so that no work is optimised away.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

template <class T> __global__ void __launch_bounds__(kProbeThreads) k_probe_fma(T *out, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_sfu(float *out, int iters)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __sinf(x[c]);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

// Best of `reps` timed launches (after one untimed), in ms.
template <class F> int time_best(F launch, cudaStream_t s, int reps, float *best_ms)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return TKF_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return TKF_ERR_CUDA;
    }
    int rc = TKF_OK;
    launch();
    *best_ms = 1e30f;
    for (int r = 0; r < reps && rc == TKF_OK; ++r) {
        float ms = 0.f;
        if (cudaEventRecord(e0, s) != cudaSuccess) rc = TKF_ERR_CUDA;
        launch();
        if (rc == TKF_OK && (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
                             cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = TKF_ERR_CUDA;
        if (rc == TKF_OK) *best_ms = std::min(*best_ms, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace

extern "C" int tkf_probe_alu(tkf_stream stream, double *fp32_tflops, double *fp64_tflops, double *sfu_tops)
{
    if (!fp32_tflops || !fp64_tflops || !sfu_tops) return TKF_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return TKF_ERR_CUDA;
    const int blocks = sms * 8;  // 2048 threads per SM
    const size_t n = (size_t)blocks * kProbeThreads;
    double *buf = nullptr;
    if (cudaMalloc((void **)&buf, n * sizeof(double)) != cudaSuccess) return TKF_ERR_NOMEM;
    const int it32 = 4096, it64 = 64, itsfu = 1024;
    float ms32 = 0.f, ms64 = 0.f, mssfu = 0.f;
    int rc = time_best(
        [&] { k_probe_fma<float><<<blocks, kProbeThreads, 0, s>>>((float *)buf, it32, 0.9999999f, 1e-7f); }, s, 3,
        &ms32);
    if (rc == TKF_OK)
        rc = time_best([&] { k_probe_fma<double><<<blocks, kProbeThreads, 0, s>>>(buf, it64, 0.9999999, 1e-7); }, s,
                       3, &ms64);
    if (rc == TKF_OK)
        rc = time_best([&] { k_probe_sfu<<<blocks, kProbeThreads, 0, s>>>((float *)buf, itsfu); }, s, 3, &mssfu);
    cudaFree(buf);
    if (rc != TKF_OK) return rc;
    const double ops = (double)n * kChains * 4;  // per loop iteration, every thread
    *fp32_tflops = 2.0 * ops * it32 / (ms32 * 1e-3) / 1e12;
    *fp64_tflops = 2.0 * ops * it64 / (ms64 * 1e-3) / 1e12;
    *sfu_tops = ops * itsfu / (mssfu * 1e-3) / 1e12;
    return TKF_OK;
}

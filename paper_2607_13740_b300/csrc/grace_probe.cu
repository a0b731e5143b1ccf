// Throughput probes for the roofline denominators of this part: FP64 FMA,
// FP32 FMA and FP64 -> FP32 conversion rates of the CUDA cores.
#include "grace_internal.h"

namespace grace {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

__global__ void fma64_kernel(double seed, double *out)
{
    double a[kChains];
    for (int i = 0; i < kChains; ++i) a[i] = seed + threadIdx.x * 1e-9 + i;
    const double m = 0.999999999, c = 1e-9;
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], m, c);
    double s = 0.0;
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == 12345.678) out[0] = s;   // keeps the chains alive
}

__global__ void fma32_kernel(float seed, float *out)
{
    float a[kChains];
    for (int i = 0; i < kChains; ++i) a[i] = seed + threadIdx.x * 1e-6f + i;
    const float m = 0.9999999f, c = 1e-7f;
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], m, c);
    float s = 0.f;
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == 12345.678f) out[0] = s;
}

__global__ void cvt_kernel(double seed, float *out)
{
    double a[kChains];
    float f[kChains];
    for (int i = 0; i < kChains; ++i) {
        a[i] = seed + threadIdx.x * 1e-9 + i;
        f[i] = 0.f;
    }
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            f[i] += (float)a[i];                       // one FP64 -> FP32 conversion + FP32 add
            a[i] = __longlong_as_double(__double_as_longlong(a[i]) + 1);   // integer bump
        }
    float s = 0.f;
    for (int i = 0; i < kChains; ++i) s += f[i];
    if (s == 12345.678f) out[0] = s;
}

}  // namespace
}  // namespace grace

using namespace grace;

extern "C" grace_status grace_probe_rates(int device, double *rates)
{
    if (!rates || device < 0) {
        set_error("grace_probe_rates: null output or negative device");
        return GRACE_ERR_ARG;
    }
    Guard guard(device);
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    double *d64 = nullptr;
    float *d32 = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d64, 64);
    if (e == cudaSuccess) e = cudaMalloc(&d32, 64);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    const int blocks = sms * 8, threads = 256;
    const double ops = (double)blocks * threads * kIters * kChains;
    for (int kind = 0; kind < 3 && e == cudaSuccess; ++kind) {
        float best = 1e30f;
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
            cudaEventRecord(a, 0);
            if (kind == 0) fma64_kernel<<<blocks, threads>>>(1.0 + rep, d64);
            if (kind == 1) fma32_kernel<<<blocks, threads>>>(1.0f + rep, d32);
            if (kind == 2) cvt_kernel<<<blocks, threads>>>(1.0 + rep, d32);
            cudaEventRecord(b, 0);
            e = cudaEventSynchronize(b);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            if (rep > 0 && ms < best) best = ms;
        }
        rates[kind] = ops / (best * 1e-3);   // operations (FMA or conversion) per second
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(d64);
    cudaFree(d32);
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_probe_rates");
}

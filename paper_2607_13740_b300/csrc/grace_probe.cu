// Throughput probes for the roofline denominators of this part: FP64 FMA,
// FP32 FMA and FP64 -> FP32 conversion rates of the CUDA cores, and the dense
// tcgen05.mma rate (kind::tf32, kind::f16 with bf16) of the tensor cores.
#include <cstdint>

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

// Dense tensor-core rate: one CTA per SM allocates a 256-column TMEM accumulator and one thread
// issues `iters` back-to-back tcgen05.mma with M = 128, N = n and K = 32 bytes (8 TF32 or 16 BF16
// values) from shared-memory operands in the contraction kernel's layouts (A: 128-byte swizzled
// K-major rows; B: 32-byte swizzled K-major rows), then waits (bounded) for their completion.
constexpr int kProbeKsteps = 4;          // k-steps cycled through (one A atom)
constexpr long long kProbeWait = 4000000000LL;

__device__ __forceinline__ uint32_t probe_smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

template <int PREC>
__global__ void __launch_bounds__(128, 1) mma_probe_kernel(int n, int iters, int *err)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    const uint32_t raw = probe_smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gen = smem_raw + (base - raw);
    const uint32_t a_bytes = 128u * 128u, b_bytes = (uint32_t)n * 32u * kProbeKsteps;
    // small non-zero operands (values do not matter for the rate)
    for (uint32_t i = threadIdx.x; i < (a_bytes + b_bytes) / 4; i += blockDim.x)
        reinterpret_cast<uint32_t *>(gen)[i] = 0x3C003C00u ^ (i & 0x00FF00FFu);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(probe_smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
                         probe_smem_u32(&tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t d = tmem_base;
    if (threadIdx.x == 0) {
        const uint32_t fmt = PREC == GRACE_TF32 ? 2u : 1u;
        const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
        for (int i = 0; i < iters; ++i) {
            const int ks = i & (kProbeKsteps - 1);
            const uint32_t aa = base + (uint32_t)ks * 32u, bb = base + a_bytes + (uint32_t)ks * (uint32_t)n * 32u;
            const uint64_t ad = (uint64_t)((aa >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
                                ((uint64_t)1u << 46) | ((uint64_t)2u << 61);
            const uint64_t bd = (uint64_t)((bb >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(256u >> 4) << 32) |
                                ((uint64_t)1u << 46) | ((uint64_t)6u << 61);
            const uint32_t acc = i > 0 ? 1u : 0u;
            if (PREC == GRACE_TF32)
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                             "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                             : "memory");
            else
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                             "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                             : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         probe_smem_u32(&bar))
                     : "memory");
        const long long t0 = clock64();
        uint32_t ok = 0;
        while (!ok) {
            asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(ok)
                         : "r"(probe_smem_u32(&bar))
                         : "memory");
            if (!ok && clock64() - t0 > kProbeWait) {
                atomicOr(err, 1);
                break;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(d) : "memory");
}

}  // namespace
}  // namespace grace

using namespace grace;

extern "C" grace_status grace_probe_mma(int device, int precision, int n, double *flops_per_s)
{
    if (!flops_per_s || device < 0 || (precision != GRACE_TF32 && precision != GRACE_BF16X3) || n < 16 ||
        n > 256 || n % 16 != 0) {
        set_error("grace_probe_mma: precision must be GRACE_TF32 or GRACE_BF16X3, n a multiple of 16 in [16, 256]");
        return GRACE_ERR_ARG;
    }
    Guard guard(device);
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int *d_err = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    const int smem = 1024 + 128 * 128 + n * 32 * kProbeKsteps;
    if (e == cudaSuccess)
        e = precision == GRACE_TF32
                ? cudaFuncSetAttribute(mma_probe_kernel<GRACE_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                : cudaFuncSetAttribute(mma_probe_kernel<GRACE_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem);
    const int iters = 16384;
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(a, 0);
        if (precision == GRACE_TF32) mma_probe_kernel<GRACE_TF32><<<sms, 128, smem>>>(n, iters, d_err);
        else mma_probe_kernel<GRACE_BF16X3><<<sms, 128, smem>>>(n, iters, d_err);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(b, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;
    }
    int h_err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(d_err);
    if (e != cudaSuccess) return cuda_fail(e, "grace_probe_mma");
    if (h_err) {
        set_error("grace_probe_mma: the completion wait gave up");
        return GRACE_ERR_TIMEOUT;
    }
    const double k_elems = precision == GRACE_TF32 ? 8.0 : 16.0;
    *flops_per_s = 2.0 * 128.0 * n * k_elems * (double)iters * sms / (best * 1e-3);
    return GRACE_OK;
}

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

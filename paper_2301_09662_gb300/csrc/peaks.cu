// Peak-rate probes of the arithmetic pipes the imaging kernels use, so that
// their roofline fractions rest on measured rates: FP32 FMA (scalar and packed
// pairs), FP64 FMA, and dense FP16 tcgen05 MMA.  Each probe is a long run of
// independent multiply-adds (eight chains per thread, enough to cover the
// pipe latency) or of back-to-back MMAs from shared memory into TMEM, one CTA
// per SM, timed with CUDA events; nothing here is on the imaging path.
#include <algorithm>

#include "dft_small.cuh"
#include "epic_internal.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace epic {
namespace {

constexpr int kChains = 8;

template <class T>
__global__ void __launch_bounds__(512) fma_probe(int iters, T seed, T *sink)
{
    T a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; i++) a[i] = seed + static_cast<T>(threadIdx.x + i);
    const T b = seed * static_cast<T>(0.999), c = static_cast<T>(1e-7);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int r = 0; r < 16; r++)
#pragma unroll
            for (int i = 0; i < kChains; i++) a[i] = fma(a[i], b, c);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; i++) s += a[i];
    if (s == static_cast<T>(-1.2345)) sink[blockIdx.x] = s;   // never true: keeps the chains live
}

// packed FP32 pairs: one fma.rn.f32x2 does two FMAs
__global__ void __launch_bounds__(512) fma2_probe(int iters, float seed, float *sink)
{
    float2 a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; i++) a[i] = make_float2(seed + threadIdx.x + i, seed - i);
    const float2 b = make_float2(seed * 0.999f, seed * 0.998f), c = make_float2(1e-7f, 2e-7f);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int r = 0; r < 16; r++)
#pragma unroll
            for (int i = 0; i < kChains; i++) a[i] = pfma(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; i++) s += a[i].x + a[i].y;
    if (s == -1.2345f) sink[blockIdx.x] = s;
}

// dense FP16 tcgen05: 128 x 256 x 16 MMAs from a zeroed shared-memory A and B
// into one TMEM accumulator, issued back to back by one thread per CTA; a
// bounded wait on the final commit (budget ~2 s at the maximum clock)
__global__ void __launch_bounds__(128, 1) tc_probe(int n_mma, int *status)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t slot;
    const int tid = threadIdx.x;
    for (int i = tid; i < (128 + 256) * 16 * 2 / 16; i += blockDim.x) reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
    if (tid < 32) tc::tmem_alloc(&slot, 256);
    if (tid == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = slot;
    if (tid == 0) {
        const uint32_t a = tc::smem_u32(sm), b = a + 128 * 16 * 2;
        const uint64_t ad = tc::smem_desc(a, tcc::kLBO, 256), bd = tc::smem_desc(b, tcc::kLBO, 256);
        constexpr uint32_t id = tcc::idesc_kk(128, 256, false);
        for (int i = 0; i < n_mma; i++) tc::mma_f16(taddr, ad, bd, id, i > 0 ? 1u : 0u);
        tc::mma_commit(&bar);
        if (!tc::mbar_wait(&bar, 0, 4000000000LL)) atomicOr(status, kStatusTimeout);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid < 32) tc::tmem_dealloc(taddr, 256);
}

}  // namespace
}  // namespace epic

extern "C" int epic_measure_peak(int what, int ms, double *tflops, void *cuda_stream)
{
    using namespace epic;
    if (!tflops || ms < 1 || ms > 10000 || what < EPIC_PEAK_FP32 || what > EPIC_PEAK_FP16_TC) return EPIC_ERR_ARG;
    *tflops = 0.0;
    auto s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return EPIC_ERR_CUDA;
    void *buf = nullptr;
    if (cudaMalloc(&buf, 4096) != cudaSuccess) return EPIC_ERR_NOMEM;
    if (cudaMemsetAsync(buf, 0, 4096, s) != cudaSuccess) {
        cudaFree(buf);
        return EPIC_ERR_CUDA;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) ? EPIC_OK : EPIC_ERR_CUDA;
    const int blocks = 4 * sms, threads = 512;
    const int tc_smem = (128 + 256) * 16 * 2;
    if (rc == EPIC_OK && what == EPIC_PEAK_FP16_TC &&
        cudaFuncSetAttribute(tc_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem) != cudaSuccess)
        rc = EPIC_ERR_CUDA;
    // flops of one launch with `work` iterations (fma probes) or MMAs per CTA (tensor probe)
    auto launch = [&](int work) -> double {
        switch (what) {
        case EPIC_PEAK_FP32:
            fma_probe<float><<<blocks, threads, 0, s>>>(work, 1.0001f, static_cast<float *>(buf));
            return 2.0 * kChains * 16 * static_cast<double>(work) * blocks * threads;
        case EPIC_PEAK_FP32X2:
            fma2_probe<<<blocks, threads, 0, s>>>(work, 1.0001f, static_cast<float *>(buf));
            return 4.0 * kChains * 16 * static_cast<double>(work) * blocks * threads;
        case EPIC_PEAK_FP64:
            fma_probe<double><<<blocks, threads, 0, s>>>(work, 1.0001, static_cast<double *>(buf));
            return 2.0 * kChains * 16 * static_cast<double>(work) * blocks * threads;
        default:
            tc_probe<<<sms, 128, tc_smem, s>>>(work, static_cast<int *>(buf));
            return 2.0 * 128 * 256 * 16 * static_cast<double>(work) * sms;
        }
    };
    auto timed = [&](int work, float &msec) -> double {
        double f = 0;
        if (cudaEventRecord(e0, s) != cudaSuccess) return -1;
        f = launch(work);
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&msec, e0, e1) != cudaSuccess)
            return -1;
        return f;
    };
    if (rc == EPIC_OK) {
        // size one launch to about `ms` milliseconds from a short calibration run, then take the
        // best of three such launches
        int work = what == EPIC_PEAK_FP16_TC ? 256 : what == EPIC_PEAK_FP64 ? 4 : 64;
        float t = 0.f;
        if (timed(work, t) < 0) rc = EPIC_ERR_CUDA;
        for (int k = 0; rc == EPIC_OK && k < 3 && t < 0.2f * ms; k++) {
            const double scale = std::min(1000.0, std::max(2.0, static_cast<double>(ms) / std::max(static_cast<double>(t), 1e-3)));
            work = static_cast<int>(std::min(2.0e9, static_cast<double>(work) * scale));
            if (timed(work, t) < 0) rc = EPIC_ERR_CUDA;
        }
        double best = 0;
        for (int k = 0; rc == EPIC_OK && k < 3; k++) {
            const double f = timed(work, t);
            if (f < 0) rc = EPIC_ERR_CUDA;
            else best = std::max(best, f / (t * 1e-3) / 1e12);
        }
        *tflops = best;
    }
    int st = 0;
    if (rc == EPIC_OK && what == EPIC_PEAK_FP16_TC &&
        (cudaMemcpy(&st, buf, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || st != 0))
        rc = st ? EPIC_ERR_TIMEOUT : EPIC_ERR_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (rc == EPIC_OK && cudaGetLastError() != cudaSuccess) rc = EPIC_ERR_CUDA;
    return rc;
}

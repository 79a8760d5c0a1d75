// E-field-domain gain solver for one calibrator (the feedback calibration Sec. 1
// cites for EPIC, and the real-time calibration Sec. 5 names as future work).
// Per (channel, polarisation), from unit gains, n_iter times:
//
//   E(t) = (1/A) sum_a g_a e_a(t) conj(phi_a)              the calibrator field
//   g_a  = phi_a sum_t E(t) conj(e_a(t)) / sum_t |e_a(t)|^2  per-antenna least squares
//   then antenna 0's phase -> 0 and the RMS |g| -> 1
//
// phi_a = exp(-2 pi i (kx_a lx + ky_a ly) / N) for a source at the image offset
// (lx, ly) = (l N du, m N du) pixels (a source there has e_a ~ phi_a and appears
// at +(lx, ly) in the image).  One CTA per (channel, polarisation); phi, the gains,
// the integer |e|^2 sums and E(t) stay in shared memory.
#include <algorithm>
#include <cmath>

#include "dft_small.cuh"
#include "epic_internal.cuh"

namespace epic {
namespace {

constexpr int kCalThreads = 256;

__device__ __forceinline__ float block_sum(float x, float *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    float s = 0.f;
    for (int w = 0; w < kCalThreads / 32; w++) s += red[w];
    return s;
}

__global__ void __launch_bounds__(kCalThreads)
gain_solve_kernel(const uint8_t *__restrict__ v, const short2 *__restrict__ cells, const int *__restrict__ chans,
                  int A, int C, int P, int T, int N, double lx, double ly, int n_iter, float2 *__restrict__ gains)
{
    extern __shared__ float2 sm[];
    float2 *phi = sm;                        // [A]
    float2 *g = phi + A;                     // [A]
    float2 *E = g + A;                       // [T]
    int *den = reinterpret_cast<int *>(E + T);   // [A] exact sum_t |e_a(t)|^2
    __shared__ float red[kCalThreads / 32];
    __shared__ float2 ref;
    const int c = chans[blockIdx.x / P], p = blockIdx.x % P;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto byte = [&](int t, int a) {
        return static_cast<uint32_t>(__ldg(v + ((static_cast<size_t>(t) * C + c) * A + a) * P + p));
    };

    for (int a = tid; a < A; a += kCalThreads) {
        const short2 k = cells[static_cast<size_t>(c) * A + a];
        double turns = (static_cast<double>(k.x) * lx + static_cast<double>(k.y) * ly) / N;
        turns -= rint(turns);
        double s, co;
        sincospi(-2.0 * turns, &s, &co);
        phi[a] = make_float2(static_cast<float>(co), static_cast<float>(s));
        g[a] = make_float2(1.f, 0.f);
        int acc = 0;
#pragma unroll 8
        for (int t = 0; t < T; t++) {
            const float2 e = ci4_decode(byte(t, a));
            acc += static_cast<int>(e.x * e.x + e.y * e.y);
        }
        den[a] = acc;
    }
    __syncthreads();

    const float invA = 1.f / static_cast<float>(A);
    for (int it = 0; it < n_iter; it++) {
        // E(t) = (1/A) sum_a g_a conj(phi_a) e_a(t): one warp per sample
        for (int t = warp; t < T; t += kCalThreads / 32) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8
            for (int a = lane; a < A; a += 32) {
                const float2 w = cmul(g[a], make_float2(phi[a].x, -phi[a].y));
                const float2 e = ci4_decode(byte(t, a));
                acc.x = fmaf(w.x, e.x, fmaf(-w.y, e.y, acc.x));
                acc.y = fmaf(w.x, e.y, fmaf(w.y, e.x, acc.y));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
            if (lane == 0) E[t] = make_float2(acc.x * invA, acc.y * invA);
        }
        __syncthreads();
        // g_a = phi_a sum_t E(t) conj(e_a(t)) / sum_t |e_a(t)|^2
        for (int a = tid; a < A; a += kCalThreads) {
            float2 num = make_float2(0.f, 0.f);
#pragma unroll 8
            for (int t = 0; t < T; t++) {
                const float2 e = ci4_decode(byte(t, a));
                const float2 x = E[t];
                num.x = fmaf(x.x, e.x, fmaf(x.y, e.y, num.x));    // x conj(e)
                num.y = fmaf(x.y, e.x, fmaf(-x.x, e.y, num.y));
            }
            g[a] = den[a] > 0 ? cscale(cmul(phi[a], num), 1.f / static_cast<float>(den[a])) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        // antenna 0's phase to zero, then RMS amplitude to one
        if (tid == 0) {
            const float2 g0 = g[0];
            const float r = sqrtf(g0.x * g0.x + g0.y * g0.y);
            ref = r > 0.f ? make_float2(g0.x / r, -g0.y / r) : make_float2(1.f, 0.f);
        }
        float ss = 0.f;
        for (int a = tid; a < A; a += kCalThreads) ss += g[a].x * g[a].x + g[a].y * g[a].y;
        ss = block_sum(ss, red);
        const float rms = sqrtf(ss * invA);
        const float sc = rms > 0.f ? 1.f / rms : 1.f;
        for (int a = tid; a < A; a += kCalThreads) g[a] = cscale(cmul(g[a], ref), sc);
        __syncthreads();
    }
    for (int a = tid; a < A; a += kCalThreads) gains[(static_cast<size_t>(c) * A + a) * P + p] = g[a];
}

size_t cal_smem(int A, int T) { return sizeof(float2) * (2 * static_cast<size_t>(A) + T) + sizeof(int) * A; }

}  // namespace
}  // namespace epic

extern "C" int epic_solve_gains(epic_plan_t plan, const uint8_t *ci4, int n_spectra, double l, double m, int n_iter,
                                float *gains_out, void *stream)
{
    if (!plan || !ci4 || !gains_out || n_spectra < 1 || n_spectra > plan->max_spectra || n_iter < 1 || n_iter > 64 ||
        !std::isfinite(l) || !std::isfinite(m))
        return EPIC_ERR_ARG;
    const size_t smem = epic::cal_smem(plan->A, n_spectra);
    if (smem > 200 * 1024) return EPIC_ERR_TOO_LARGE;
    if (cudaFuncSetAttribute(epic::gain_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
        return EPIC_ERR_CUDA;
    auto s = static_cast<cudaStream_t>(stream);
    for (const auto &g : plan->groups) {
        const double lx = l * g.N * plan->du, ly = m * g.N * plan->du;
        epic::gain_solve_kernel<<<static_cast<unsigned>(g.n_chan * plan->P), epic::kCalThreads, smem, s>>>(
            ci4, plan->d_cells, g.d_chans, plan->A, plan->C, plan->P, n_spectra, g.N, lx, ly, n_iter,
            reinterpret_cast<float2 *>(gains_out));
        if (cudaGetLastError() != cudaSuccess) return EPIC_ERR_CUDA;
    }
    return EPIC_OK;
}

// Transient search on the image cube: incoherent de-dispersion of every
// pixel's dynamic spectrum and a boxcar single-pulse search of the
// de-dispersed light curves (Sec. 4: light curves extracted per channel, the
// dispersive delay corrected across the band, single pulses searched; Sec. 5
// names de-dispersion and transient detection as the next modules).
//
//  * shifts: s[d][c] = floor(k_DM DM_d (f_c^-2 - f_max^-2) / dt + 1/2) samples,
//    f in MHz, computed once on the host in FP64 (the plan);
//  * dedisperse_staged_kernel: D[d][t][p] = sum_c I[t + s[d][c]][c][p].  A
//    block is 16 trial DMs (warps) x 32 pixels (lanes, coalesced) x 32 output
//    samples; per channel the union of the sixteen sweeps is staged in shared
//    memory once (cp.async, four channels in flight) and every warp sums its
//    window from there.  dedisperse_kernel (each warp loading its own sweep)
//    serves DM grids too coarse for the staging buffer.  The cube is read
//    through (time, channel, pixel) strides, so the Stokes-I slot of an image
//    series (complex64 layout) is searched in place;
//  * curve_stats_kernel + single_pulse_kernel: one thread per (DM, pixel) light
//    curve: mean and standard deviation in one blocked FP32 pass (a low-register
//    kernel of its own), then running window sums of x - mu for every boxcar
//    width 2^k <= 32 (the previous 32 samples in registers); the best S/N, its
//    start and width are kept;
//  * candidates_kernel: one block compacts the (DM, pixel) pairs whose best S/N
//    reaches the threshold, in index order (deterministic).
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "epic_internal.cuh"

struct epic_search_s {
    int C = 0, n_dm = 0, npix = 0, T = 0, T_out = 0, smax = 0;
    unsigned widths = 0;          // bit k: boxcar width 2^k (k < 6)
    int *d_shift = nullptr;       // [n_dm][C]
    float2 *d_stats = nullptr;    // [n_dm][npix] mean, standard deviation of each light curve
    bool staged = true;           // every block's sweep spread fits the staging buffer
};

namespace epic {
namespace {

constexpr double kDM = 4.148808e3;   // s MHz^2 pc^-1 cm^3
constexpr int kPixB = 32, kDmB = 8, kTT = 32;
constexpr int kRows = 96;                        // staged rows per channel: kTT + spread <= kRows
constexpr int kDmS = 16;                         // trial DMs (warps) per block of the staged form
constexpr int kStages = 4;                       // channels in flight (cp.async ring)

// Direct form: each warp (one DM) loads its own sweep; L1 shares what the
// eight DMs of a block have in common.
__global__ void __launch_bounds__(kPixB * kDmB)
dedisperse_kernel(const float *__restrict__ cube, long long ts, long long cs, long long ps, int C, int npix,
                  int T_out, const int *__restrict__ shift, int n_dm, float *__restrict__ dd)
{
    extern __shared__ int sh[];                       // [kDmB][C]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int d0 = blockIdx.y * kDmB;
    for (int i = threadIdx.x; i < kDmB * C; i += blockDim.x) {
        const int d = d0 + i / C;
        sh[i] = d < n_dm ? shift[static_cast<size_t>(d) * C + i % C] : 0;
    }
    __syncthreads();
    const int pix = blockIdx.x * kPixB + lane, d = d0 + w, t0 = blockIdx.z * kTT;
    if (pix >= npix || d >= n_dm) return;
    const int nt = min(kTT, T_out - t0);
    float acc[kTT];
#pragma unroll
    for (int j = 0; j < kTT; j++) acc[j] = 0.f;
    const float *base = cube + static_cast<long long>(pix) * ps;
    for (int c = 0; c < C; c++) {
        const float *src = base + static_cast<long long>(t0 + sh[w * C + c]) * ts + c * cs;
#pragma unroll
        for (int j = 0; j < kTT; j++)
            if (j < nt) acc[j] += __ldg(src + j * ts);
    }
    float *out = dd + (static_cast<size_t>(d) * T_out + t0) * npix + pix;
#pragma unroll
    for (int j = 0; j < kTT; j++)
        if (j < nt) out[static_cast<size_t>(j) * npix] = acc[j];
}

__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Staged form.  Block (DM block x, pixel block y, time tile z): for each channel
// the rows t0 + min_d s[d][c] .. t0 + max_d s[d][c] + kTT of its 32 pixels are
// copied to shared memory once (coalesced cp.async, kStages channels in
// flight), and each warp (one DM) sums its window from there.
__global__ void __launch_bounds__(kPixB * kDmS)
dedisperse_staged_kernel(const float *__restrict__ cube, long long ts, long long cs, long long ps, int C, int npix,
                         int T_out, const int *__restrict__ shift, int n_dm, float *__restrict__ dd)
{
    extern __shared__ float dyn[];                   // [kStages][kRows][kPixB], then the tables
    float *ring = dyn;
    int *sh = reinterpret_cast<int *>(dyn + kStages * kRows * kPixB);   // [kDmS][C]
    int *smin = sh + kDmS * C, *srows = smin + C;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int d0 = blockIdx.x * kDmS, pix = blockIdx.y * kPixB + lane, t0 = blockIdx.z * kTT;
    const int nt = min(kTT, T_out - t0);
    const int nd = min(kDmS, n_dm - d0);
    for (int i = threadIdx.x; i < kDmS * C; i += blockDim.x) {
        const int d = i / C;
        sh[i] = shift[static_cast<size_t>(d0 + min(d, nd - 1)) * C + i % C];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        int lo = sh[c], hi = sh[c];
        for (int d = 1; d < nd; d++) {
            lo = min(lo, sh[d * C + c]);
            hi = max(hi, sh[d * C + c]);
        }
        smin[c] = lo;
        srows[c] = nt + hi - lo;                      // <= kRows, checked when the plan was made
    }
    __syncthreads();
    const bool pin = pix < npix;
    const float *base = cube + static_cast<long long>(min(pix, npix - 1)) * ps;
    auto issue = [&](int c) {                        // channel c into ring slot c mod kStages
        if (c < C) {
            const float *src = base + static_cast<long long>(t0 + smin[c]) * ts + c * cs;
            float *dst = ring + (c % kStages) * kRows * kPixB + lane;
            const int rows = srows[c];
            for (int r = w; r < rows; r += kDmS)
                cp_async4(dst + r * kPixB, src + static_cast<long long>(r) * ts, pin);
        }
        cp_async_commit();                           // one group per channel, empty past the end
    };
    float acc[kTT];
#pragma unroll
    for (int j = 0; j < kTT; j++) acc[j] = 0.f;
#pragma unroll
    for (int c = 0; c < kStages - 1; c++) issue(c);
    for (int c = 0; c < C; c++) {
        cp_async_wait<kStages - 2>();                // channel c has landed (this thread's part)
        __syncthreads();                             // ... everyone's; slot (c - 1) mod kStages is free
        issue(c + kStages - 1);
        const int off = sh[w * C + c] - smin[c];
        const float *row = ring + (c % kStages) * kRows * kPixB + off * kPixB + lane;
#pragma unroll
        for (int j = 0; j < kTT; j++) acc[j] += row[j * kPixB];   // rows past nt + spread are never stored
    }
    cp_async_wait<0>();
    if (!pin || w >= nd) return;
    float *out = dd + (static_cast<size_t>(d0 + w) * T_out + t0) * npix + pix;
#pragma unroll
    for (int j = 0; j < kTT; j++)
        if (j < nt) out[static_cast<size_t>(j) * npix] = acc[j];
}

size_t staged_smem(int C)
{
    return sizeof(float) * kStages * kRows * kPixB + sizeof(int) * (kDmS + 2) * static_cast<size_t>(C);
}

// better S/N, then the smaller width, then the earlier start
__device__ __forceinline__ void keep_best(float s, int t, int w, float &bs, int &bt, int &bw)
{
    if (s > bs || (s == bs && (w < bw || (w == bw && t < bt)))) {
        bs = s;
        bt = t;
        bw = w;
    }
}

// Mean and population standard deviation of every (DM, pixel) light curve, one
// shifted pass (x - x_0, x_0 the first sample, keeps the two sums small),
// summed in blocks of 16.  Few registers, so many warps hide the loads.
__global__ void __launch_bounds__(256)
curve_stats_kernel(const float *__restrict__ dd, int T_out, int npix, int n_dm, float2 *__restrict__ stats)
{
    const int pix = blockIdx.x * blockDim.x + threadIdx.x, d = blockIdx.y;
    if (pix >= npix || d >= n_dm) return;
    const float *x = dd + static_cast<size_t>(d) * T_out * npix + pix;
    const float x0 = __ldg(x);
    float s1 = 0.f, s2 = 0.f;
    for (int t0 = 0; t0 < T_out; t0 += 16) {
        float b1 = 0.f, b2 = 0.f;
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const float y = t0 + k < T_out ? __ldg(x + static_cast<size_t>(t0 + k) * npix) - x0 : 0.f;
            b1 += y;
            b2 = fmaf(y, y, b2);
        }
        s1 += b1;
        s2 += b2;
    }
    const float m1 = s1 / static_cast<float>(T_out);
    stats[static_cast<size_t>(d) * npix + pix] =
        make_float2(x0 + m1, sqrtf(fmaxf(s2 / static_cast<float>(T_out) - m1 * m1, 0.f)));
}

// Boxcar search of every light curve: y = x - mu streamed 32 samples at a time;
// for each width w = 2^k the running window sum S_w gains y_e and drops y_{e-w}
// (the previous 32 samples stay in registers), and S_w / (sigma sqrt(w)) is the
// S/N of the window starting at e - w + 1.
__global__ void __launch_bounds__(128)
single_pulse_kernel(const float *__restrict__ dd, const float2 *__restrict__ stats, int T_out, int npix, int n_dm,
                    unsigned widths, float *__restrict__ best_snr, int *__restrict__ best_t, int *__restrict__ best_w)
{
    const int pix = blockIdx.x * blockDim.x + threadIdx.x, d = blockIdx.y;
    if (pix >= npix || d >= n_dm) return;
    const float *x = dd + static_cast<size_t>(d) * T_out * npix + pix;
    const float2 ms = stats[static_cast<size_t>(d) * npix + pix];
    const float mu = ms.x, sigma = ms.y;
    int wmin = 0;
    while (wmin < 6 && !((widths >> wmin) & 1u)) wmin++;
    float bs = -INFINITY;
    int bt = 0, bw = 1 << wmin;
    if (!(sigma > 0.f)) {
        bs = 0.f;
    } else {
        float inv[6], S[6];
#pragma unroll
        for (int k = 0; k < 6; k++) {
            inv[k] = 1.f / (sigma * sqrtf(static_cast<float>(1 << k)));
            S[k] = 0.f;
        }
        float prev[32], cur[32];
#pragma unroll
        for (int j = 0; j < 32; j++) prev[j] = 0.f;
        for (int base = 0; base < T_out; base += 32) {
#pragma unroll
            for (int j = 0; j < 32; j++)
                cur[j] = base + j < T_out ? __ldg(x + static_cast<size_t>(base + j) * npix) - mu : 0.f;
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const int e = base + j;
#pragma unroll
                for (int k = 0; k < 6; k++) {
                    const int w = 1 << k;
                    const float old = j - w >= 0 ? cur[j - w] : prev[32 + j - w];
                    S[k] += cur[j] - old;
                    if (((widths >> k) & 1u) && e >= w - 1 && e < T_out)
                        keep_best(S[k] * inv[k], e - w + 1, w, bs, bt, bw);
                }
            }
#pragma unroll
            for (int j = 0; j < 32; j++) prev[j] = cur[j];
        }
    }
    const size_t o = static_cast<size_t>(d) * npix + pix;
    best_snr[o] = bs;
    best_t[o] = bt;
    best_w[o] = bw;
}

// One block: (d, p) pairs with best S/N >= threshold, in index order.
__global__ void __launch_bounds__(1024)
candidates_kernel(const float *__restrict__ best_snr, int n, float threshold, int2 *__restrict__ cand, int cap,
                  int npix, int *__restrict__ n_cand)
{
    __shared__ int part[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (n + nt - 1) / nt;
    const int i0 = min(n, tid * per), i1 = min(n, i0 + per);
    int cnt = 0;
    for (int i = i0; i < i1; i++) cnt += best_snr[i] >= threshold;
    part[tid] = cnt;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {          // inclusive scan
        const int v = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int pos = part[tid] - cnt;
    for (int i = i0; i < i1; i++)
        if (best_snr[i] >= threshold) {
            if (pos < cap) cand[pos] = make_int2(i / npix, i % npix);
            pos++;
        }
    if (tid == nt - 1) *n_cand = part[tid];
}

}  // namespace
}  // namespace epic

extern "C" {

int epic_search_plan(epic_search_t *out, const double *freq_hz, int n_chan, double dt_s, const double *dm,
                     int n_dm, int n_pix, int n_time, unsigned width_mask)
{
    if (!out) return EPIC_ERR_ARG;
    *out = nullptr;
    if (!freq_hz || !dm || n_chan < 1 || n_dm < 1 || n_pix < 1 || n_time < 1 || !(dt_s > 0)) return EPIC_ERR_ARG;
    if ((width_mask & 63u) == 0 || (width_mask & ~63u)) return EPIC_ERR_ARG;
    double fmax = 0;
    for (int c = 0; c < n_chan; c++) {
        if (!(freq_hz[c] > 0)) return EPIC_ERR_ARG;
        fmax = std::max(fmax, freq_hz[c] / 1e6);
    }
    std::vector<int> shift(static_cast<size_t>(n_dm) * n_chan);
    int smax = 0;
    for (int d = 0; d < n_dm; d++) {
        if (!(dm[d] >= 0)) return EPIC_ERR_ARG;
        for (int c = 0; c < n_chan; c++) {
            const double f = freq_hz[c] / 1e6;
            const double x = epic::kDM * dm[d] * (1.0 / (f * f) - 1.0 / (fmax * fmax)) / dt_s;
            const double r = std::floor(x + 0.5);
            if (r > static_cast<double>(n_time)) return EPIC_ERR_TOO_LARGE;
            shift[static_cast<size_t>(d) * n_chan + c] = static_cast<int>(r);
            smax = std::max(smax, static_cast<int>(r));
        }
    }
    if (smax >= n_time) return EPIC_ERR_TOO_LARGE;
    int wmin = 0;
    while (!((width_mask >> wmin) & 1u)) wmin++;
    if ((1 << wmin) > n_time - smax) return EPIC_ERR_TOO_LARGE;   // no boxcar fits the output
    auto *s = new (std::nothrow) epic_search_s;
    if (!s) return EPIC_ERR_NOMEM;
    s->C = n_chan;
    s->n_dm = n_dm;
    s->npix = n_pix;
    s->T = n_time;
    s->smax = smax;
    s->T_out = n_time - smax;
    s->widths = width_mask;
    // the staged kernel holds kTT + (spread of the shifts over one block's DMs) rows per channel
    for (int d0 = 0; d0 < n_dm && s->staged; d0 += epic::kDmS)
        for (int c = 0; c < n_chan; c++) {
            int lo = shift[static_cast<size_t>(d0) * n_chan + c], hi = lo;
            for (int d = d0; d < std::min(n_dm, d0 + epic::kDmS); d++) {
                lo = std::min(lo, shift[static_cast<size_t>(d) * n_chan + c]);
                hi = std::max(hi, shift[static_cast<size_t>(d) * n_chan + c]);
            }
            if (epic::kTT + hi - lo > epic::kRows) {
                s->staged = false;
                break;
            }
        }
    if (cudaMalloc(&s->d_shift, shift.size() * sizeof(int)) != cudaSuccess) {
        delete s;
        return EPIC_ERR_NOMEM;
    }
    if (cudaMemcpy(s->d_shift, shift.data(), shift.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(s->d_shift);
        delete s;
        return EPIC_ERR_CUDA;
    }
    if (cudaMalloc(&s->d_stats, sizeof(float2) * static_cast<size_t>(n_dm) * n_pix) != cudaSuccess) {
        cudaFree(s->d_shift);
        delete s;
        return EPIC_ERR_NOMEM;
    }
    *out = s;
    return EPIC_OK;
}

int epic_search_info(epic_search_t s, int *t_out, int *max_shift)
{
    if (!s) return EPIC_ERR_ARG;
    if (t_out) *t_out = s->T_out;
    if (max_shift) *max_shift = s->smax;
    return EPIC_OK;
}

int epic_dedisperse(epic_search_t s, const float *cube, long long t_stride, long long c_stride, long long pix_stride,
                    float *dd, void *stream)
{
    if (!s || !cube || !dd || t_stride < 1 || c_stride < 1 || pix_stride < 1) return EPIC_ERR_ARG;
    const unsigned pb = static_cast<unsigned>((s->npix + epic::kPixB - 1) / epic::kPixB);
    const unsigned tb = static_cast<unsigned>((s->T_out + epic::kTT - 1) / epic::kTT);
    auto st = static_cast<cudaStream_t>(stream);
    const size_t smem_staged = epic::staged_smem(s->C);
    if (s->staged && smem_staged <= 200 * 1024 &&
        cudaFuncSetAttribute(epic::dedisperse_staged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem_staged)) == cudaSuccess) {
        // DM blocks fastest: the blocks that read the same rows run together and share L2
        const unsigned db = static_cast<unsigned>((s->n_dm + epic::kDmS - 1) / epic::kDmS);
        epic::dedisperse_staged_kernel<<<dim3(db, pb, tb), epic::kPixB * epic::kDmS, smem_staged, st>>>(
            cube, t_stride, c_stride, pix_stride, s->C, s->npix, s->T_out, s->d_shift, s->n_dm, dd);
    } else {
        const unsigned db = static_cast<unsigned>((s->n_dm + epic::kDmB - 1) / epic::kDmB);
        const size_t smem = sizeof(int) * epic::kDmB * s->C;
        if (smem > 48 * 1024) return EPIC_ERR_UNSUPPORTED;
        epic::dedisperse_kernel<<<dim3(pb, db, tb), epic::kPixB * epic::kDmB, smem, st>>>(
            cube, t_stride, c_stride, pix_stride, s->C, s->npix, s->T_out, s->d_shift, s->n_dm, dd);
    }
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

int epic_single_pulse(epic_search_t s, const float *dd, float threshold, float *best_snr, int *best_t, int *best_w,
                      int *cand, int cand_cap, int *n_cand, void *stream)
{
    if (!s || !dd || !best_snr || !best_t || !best_w || cand_cap < 0 || (cand_cap > 0 && !cand) || !n_cand)
        return EPIC_ERR_ARG;
    auto st = static_cast<cudaStream_t>(stream);
    epic::curve_stats_kernel<<<dim3(static_cast<unsigned>((s->npix + 255) / 256), static_cast<unsigned>(s->n_dm)),
                                256, 0, st>>>(dd, s->T_out, s->npix, s->n_dm, s->d_stats);
    if (cudaGetLastError() != cudaSuccess) return EPIC_ERR_CUDA;
    const dim3 grid(static_cast<unsigned>((s->npix + 127) / 128), static_cast<unsigned>(s->n_dm));
    epic::single_pulse_kernel<<<grid, 128, 0, st>>>(dd, s->d_stats, s->T_out, s->npix, s->n_dm, s->widths, best_snr,
                                                     best_t, best_w);
    if (cudaGetLastError() != cudaSuccess) return EPIC_ERR_CUDA;
    epic::candidates_kernel<<<1, 1024, 0, st>>>(best_snr, s->n_dm * s->npix, threshold,
                                                reinterpret_cast<int2 *>(cand), cand_cap, s->npix, n_cand);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

void epic_search_destroy(epic_search_t s)
{
    if (!s) return;
    cudaFree(s->d_shift);
    cudaFree(s->d_stats);
    delete s;
}

}  // extern "C"

// Transient search on the image cube: incoherent de-dispersion of every
// pixel's dynamic spectrum and a boxcar single-pulse search of the
// de-dispersed light curves (Sec. 4: light curves extracted per channel, the
// dispersive delay corrected across the band, single pulses searched; Sec. 5
// names de-dispersion and transient detection as the next modules).
//
//  * shifts: s[d][c] = floor(k_DM DM_d (f_c^-2 - f_max^-2) / dt + 1/2) samples,
//    f in MHz, computed once on the host in FP64 (the plan);
//  * dedisperse_staged_kernel: D[d][t][p] = sum_c I[t + s[d][c]][c][p].  A
//    block is 32 (or 16) trial DMs, two per warp, x 32 pixels (lanes,
//    coalesced) x 28 output samples; per channel the union of the block's
//    sweeps is staged in shared memory once (cp.async, eight channels in
//    flight) and every warp sums its two windows from there.  dedisperse_kernel
//    (each warp loading its own sweep) serves DM grids too coarse for the
//    staging buffer.  The cube is read
//    through (time, channel, pixel) strides, so the Stokes-I slot of an image
//    series (complex64 layout) is searched in place;
//  * single_pulse_kernel: one thread per (DM, pixel) light curve, one pass:
//    population moments and, per boxcar width 2^k <= 32, the largest running
//    window sum (the previous 32 samples in registers), normalised by mu and
//    sigma at the end; a warp ballot marks the pairs whose best S/N reaches the
//    threshold;
//  * candidates_kernel: one block compacts the marked (DM, pixel) pairs in index
//    order (deterministic).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <new>
#include <vector>

#include "epic_internal.cuh"

struct epic_search_s {
    int C = 0, n_dm = 0, npix = 0, T = 0, T_out = 0, smax = 0;
    unsigned widths = 0;          // bit k: boxcar width 2^k (k < 6)
    int *d_shift = nullptr;       // [n_dm][C]
    unsigned *d_mask = nullptr;   // [n_dm][wpr] candidate bits, wpr = ceil(npix / 32)
    int wpr = 0;
    int dm_block = 0;             // trial DMs per block of the staged form (32 or 16); 0: direct form
    int rows = 0;                 // staged rows per channel slot: kTS + the largest spread of a block
};

namespace epic {
namespace {

constexpr double kDM = 4.148808e3;   // s MHz^2 pc^-1 cm^3
constexpr int kPixB = 32, kDmB = 8, kTT = 32;
constexpr int kTS = 28;                          // output samples per block of the staged form (2 x 28 accumulators)
constexpr int kRows = 96;                        // largest staged rows per channel: kTS + spread <= kRows
constexpr int kStages = 8;                       // channels in flight (cp.async ring)

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

// Staged form.  Block (DM block x, pixel block y, time tile z), WARPS warps and
// two trial DMs (d, d + 1) per warp: for each channel the rows t0 + min_d s[d][c]
// .. t0 + max_d s[d][c] + kTS of its 32 pixels are copied to shared memory once
// (coalesced cp.async, kStages channels in flight).  A warp reads the window of
// its first DM into registers and adds it; the second DM's window starts
// delta = s[d+1][c] - s[d][c] rows later, so for delta 0 or 1 (adjacent trials
// finer than one sample of sweep, the usual DM grid) it is the same registers,
// shifted, plus one row; other deltas read their own window.  Shared-memory
// reads per add are about halved.
template <int WARPS>
__global__ void __launch_bounds__(kPixB * WARPS, 512 / (kPixB * WARPS))
dedisperse_staged_kernel(const float *__restrict__ cube, long long ts, long long cs, long long ps, int C, int npix,
                         int T_out, const int *__restrict__ shift, int n_dm, int rows_max, float *__restrict__ dd)
{
    constexpr int DMB = 2 * WARPS;                   // trial DMs per block
    extern __shared__ float dyn[];                   // [kStages][rows_max][kPixB], then the tables
    float *ring = dyn;
    int *sh = reinterpret_cast<int *>(dyn + kStages * rows_max * kPixB);   // [DMB][C]
    int *smin = sh + DMB * C, *srows = smin + C;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int d0 = blockIdx.x * DMB, pix = blockIdx.y * kPixB + lane, t0 = blockIdx.z * kTS;
    const int nt = min(kTS, T_out - t0);
    const int nd = min(DMB, n_dm - d0);
    for (int i = threadIdx.x; i < DMB * C; i += blockDim.x) {
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
        srows[c] = nt + hi - lo;                      // kTS + hi - lo <= rows_max, found when the plan was made
    }
    __syncthreads();
    const bool pin = pix < npix;
    const float *base = cube + static_cast<long long>(min(pix, npix - 1)) * ps;
    auto issue = [&](int c) {                        // channel c into ring slot c mod kStages
        if (c < C) {
            const float *src = base + static_cast<long long>(t0 + smin[c]) * ts + c * cs;
            float *dst = ring + (c % kStages) * rows_max * kPixB + lane;
            const int rows = srows[c];
            for (int r = w; r < rows; r += WARPS)
                cp_async4(dst + r * kPixB, src + static_cast<long long>(r) * ts, pin);
        }
        cp_async_commit();                           // one group per channel, empty past the end
    };
    float acc0[kTS], acc1[kTS];
#pragma unroll
    for (int j = 0; j < kTS; j++) acc0[j] = acc1[j] = 0.f;
#pragma unroll
    for (int c = 0; c < kStages - 1; c++) issue(c);
    for (int c = 0; c < C; c++) {
        cp_async_wait<kStages - 2>();                // channel c has landed (this thread's part)
        __syncthreads();                             // ... everyone's; slot (c - 1) mod kStages is free
        issue(c + kStages - 1);
        const int o0 = sh[2 * w * C + c] - smin[c], o1 = sh[(2 * w + 1) * C + c] - smin[c];
        const float *slot = ring + (c % kStages) * rows_max * kPixB + lane;
        const float *row = slot + o0 * kPixB;
        // rows at or past nt + spread are never stored: they only feed outputs j >= nt, never written
        const int delta = o1 - o0;                   // warp-uniform
        if (delta == 0) {
#pragma unroll
            for (int j = 0; j < kTS; j++) {
                const float v = row[j * kPixB];
                acc0[j] += v;
                acc1[j] += v;
            }
        } else if (delta == 1) {
#pragma unroll
            for (int j = 0; j < kTS; j++) {
                const float v = row[j * kPixB];
                acc0[j] += v;
                if (j) acc1[j - 1] += v;
            }
            acc1[kTS - 1] += row[kTS * kPixB];       // row o1 + kTS - 1 < rows_max
        } else {
            const float *row1 = slot + o1 * kPixB;
#pragma unroll
            for (int j = 0; j < kTS; j++) {
                acc0[j] += row[j * kPixB];
                acc1[j] += row1[j * kPixB];
            }
        }
    }
    cp_async_wait<0>();
    if (!pin) return;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        if (2 * w + h >= nd) break;
        float *out = dd + (static_cast<size_t>(d0 + 2 * w + h) * T_out + t0) * npix + pix;
#pragma unroll
        for (int j = 0; j < kTS; j++)
            if (j < nt) out[static_cast<size_t>(j) * npix] = h ? acc1[j] : acc0[j];
    }
}

size_t staged_smem(int C, int dm_block, int rows)
{
    return sizeof(float) * kStages * rows * kPixB + sizeof(int) * (dm_block + 2) * static_cast<size_t>(C);
}

// Largest kTS + (spread of the shifts over one block of dm_block trials), over blocks and channels.
int staged_rows(const std::vector<int> &shift, int n_dm, int C, int dm_block)
{
    int need = 0;
    for (int d0 = 0; d0 < n_dm; d0 += dm_block)
        for (int c = 0; c < C; c++) {
            int lo = shift[static_cast<size_t>(d0) * C + c], hi = lo;
            for (int d = d0; d < std::min(n_dm, d0 + dm_block); d++) {
                lo = std::min(lo, shift[static_cast<size_t>(d) * C + c]);
                hi = std::max(hi, shift[static_cast<size_t>(d) * C + c]);
            }
            need = std::max(need, kTS + hi - lo);
        }
    return need;
}

// Running boxcar sums of one 32-sample chunk of a light curve (y = x - x0).
// For width w = 2^k the window sum S_w gains y_e and drops y_{e-w} (the previous
// chunk stays in registers); the largest S_w and the end e of its first
// occurrence are kept per width.  FIRST: windows ending before w - 1 are not
// complete; TAIL: samples at or past T_out are not part of the curve.
template <bool FIRST, bool TAIL>
__device__ __forceinline__ void boxcar_chunk(const float (&cur)[32], const float (&prev)[32], int base, int T_out,
                                             float (&S)[6], float (&bS)[6], int (&bE)[6])
{
#pragma unroll
    for (int j = 0; j < 32; j++) {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const int w = 1 << k;
            const float old = j - w >= 0 ? cur[j - w] : (FIRST ? 0.f : prev[32 + j - w]);
            S[k] += cur[j] - old;
            const bool full = !FIRST || j >= w - 1;
            const bool in = !TAIL || base + j < T_out;
            if (full && in && S[k] > bS[k]) {
                bS[k] = S[k];
                bE[k] = base + j;
            }
        }
    }
}

// Boxcar search of every light curve in one pass: one thread per (DM, pixel),
// samples shifted by the first one (y = x - x0: constant curves give exact
// zeros, and the sums stay small).  The pass accumulates sum y and sum y^2
// (population moments) and, per width, the largest window sum; since mu and
// sigma are the same for every window of a curve, the S/N of width w is
// maximised by the largest window sum, normalised at the end:
// (max S_w - w (mu - x0)) / (sigma sqrt(w)).  Ties: smaller width, then earlier
// start.  A warp ballot of "best S/N >= threshold" gives the candidate mask
// (bit p mod 32 of word d * wpr + p / 32).
__global__ void __launch_bounds__(128)
single_pulse_kernel(const float *__restrict__ dd, int T_out, int npix, unsigned widths, float threshold,
                    float *__restrict__ best_snr, int *__restrict__ best_t, int *__restrict__ best_w,
                    unsigned *__restrict__ mask, int wpr)
{
    const int pix = blockIdx.x * blockDim.x + threadIdx.x, d = blockIdx.y;
    const bool valid = pix < npix;
    const float *x = dd + static_cast<size_t>(d) * T_out * npix + min(pix, npix - 1);
    int wmin = 0;
    while (wmin < 6 && !((widths >> wmin) & 1u)) wmin++;
    float S[6], bS[6];
    int bE[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        S[k] = 0.f;
        bS[k] = -INFINITY;
        bE[k] = 0;
    }
    float s1 = 0.f, s2 = 0.f;
    const float x0 = __ldg(x);
    float prev[32], cur[32];
    auto load = [&](int base) {
#pragma unroll
        for (int j = 0; j < 32; j++)
            cur[j] = base + j < T_out ? __ldg(x + static_cast<size_t>(base + j) * npix) - x0 : 0.f;
        float b1 = 0.f, b2 = 0.f;
#pragma unroll
        for (int j = 0; j < 32; j++) {
            b1 += cur[j];
            b2 = fmaf(cur[j], cur[j], b2);
        }
        s1 += b1;
        s2 += b2;
    };
#pragma unroll
    for (int j = 0; j < 32; j++) prev[j] = 0.f;
    load(0);
    if (T_out <= 32) {
        boxcar_chunk<true, true>(cur, prev, 0, T_out, S, bS, bE);
    } else {
        boxcar_chunk<true, false>(cur, prev, 0, T_out, S, bS, bE);
        int base = 32;
        for (; base + 32 <= T_out; base += 32) {
#pragma unroll
            for (int j = 0; j < 32; j++) prev[j] = cur[j];
            load(base);
            boxcar_chunk<false, false>(cur, prev, base, T_out, S, bS, bE);
        }
        if (base < T_out) {
#pragma unroll
            for (int j = 0; j < 32; j++) prev[j] = cur[j];
            load(base);
            boxcar_chunk<false, true>(cur, prev, base, T_out, S, bS, bE);
        }
    }
    const float m1 = s1 / static_cast<float>(T_out);
    const float sigma = sqrtf(fmaxf(s2 / static_cast<float>(T_out) - m1 * m1, 0.f));
    float bs = 0.f;
    int bt = 0, bw = 1 << wmin;
    if (sigma > 0.f) {
        bs = -INFINITY;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const float w = static_cast<float>(1 << k);
            if (((widths >> k) & 1u) && bS[k] > -INFINITY) {
                const float snr = (bS[k] - w * m1) / (sigma * sqrtf(w));
                if (snr > bs) {
                    bs = snr;
                    bt = bE[k] - (1 << k) + 1;
                    bw = 1 << k;
                }
            }
        }
    }
    const unsigned hits = __ballot_sync(0xffffffffu, valid && bs >= threshold);
    if (!valid) return;
    const size_t o = static_cast<size_t>(d) * npix + pix;
    best_snr[o] = bs;
    best_t[o] = bt;
    best_w[o] = bw;
    if ((threadIdx.x & 31) == 0) mask[static_cast<size_t>(d) * wpr + (pix >> 5)] = hits;
}

// One block: the (d, p) pairs set in the candidate mask, in index order
// (deterministic).  Each thread owns a contiguous run of mask words.
__global__ void __launch_bounds__(1024)
candidates_kernel(const unsigned *__restrict__ mask, int n_words, int wpr, int2 *__restrict__ cand, int cap,
                  int *__restrict__ n_cand)
{
    __shared__ int part[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (n_words + nt - 1) / nt;
    const int i0 = min(n_words, tid * per), i1 = min(n_words, i0 + per);
    int cnt = 0;
    for (int i = i0; i < i1; i++) cnt += __popc(mask[i]);
    part[tid] = cnt;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {          // inclusive scan
        const int v = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int pos = part[tid] - cnt;
    for (int i = i0; i < i1 && pos < cap; i++) {
        unsigned m = mask[i];
        while (m && pos < cap) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            cand[pos++] = make_int2(i / wpr, (i % wpr) * 32 + b);
        }
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
    // the staged kernel holds kTS + (spread of the shifts over one block's DMs) rows per channel;
    // EPIC_SEARCH_DM_BLOCK caps the block: 16 asks for the smaller block even where 32 trials
    // fit, 0 for the direct form
    const char *env = std::getenv("EPIC_SEARCH_DM_BLOCK");
    const int cap = env && *env ? std::atoi(env) : 32;
    const int rows32 = epic::staged_rows(shift, n_dm, n_chan, 32);
    const int rows16 = epic::staged_rows(shift, n_dm, n_chan, 16);
    if (cap >= 32 && rows32 <= epic::kRows) {
        s->dm_block = 32;
        s->rows = rows32;
    } else if (cap >= 16 && rows16 <= epic::kRows) {
        s->dm_block = 16;
        s->rows = rows16;
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
    s->wpr = (n_pix + 31) / 32;
    if (cudaMalloc(&s->d_mask, sizeof(unsigned) * static_cast<size_t>(n_dm) * s->wpr) != cudaSuccess) {
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
    const int dmb = s->dm_block;
    const size_t smem_staged = dmb ? epic::staged_smem(s->C, dmb, s->rows) : 0;
    auto staged = dmb == 32 ? epic::dedisperse_staged_kernel<16> : epic::dedisperse_staged_kernel<8>;
    if (dmb && smem_staged <= 200 * 1024 &&
        cudaFuncSetAttribute(staged, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem_staged)) == cudaSuccess) {
        // DM blocks fastest: the blocks that read the same rows run together and share L2
        const unsigned db = static_cast<unsigned>((s->n_dm + dmb - 1) / dmb);
        const unsigned tbs = static_cast<unsigned>((s->T_out + epic::kTS - 1) / epic::kTS);
        staged<<<dim3(db, pb, tbs), epic::kPixB * (dmb / 2), smem_staged, st>>>(
            cube, t_stride, c_stride, pix_stride, s->C, s->npix, s->T_out, s->d_shift, s->n_dm, s->rows, dd);
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
    const dim3 grid(static_cast<unsigned>((s->npix + 127) / 128), static_cast<unsigned>(s->n_dm));
    epic::single_pulse_kernel<<<grid, 128, 0, st>>>(dd, s->T_out, s->npix, s->widths, threshold, best_snr, best_t,
                                                     best_w, s->d_mask, s->wpr);
    if (cudaGetLastError() != cudaSuccess) return EPIC_ERR_CUDA;
    epic::candidates_kernel<<<1, 1024, 0, st>>>(s->d_mask, s->n_dm * s->wpr, s->wpr,
                                                reinterpret_cast<int2 *>(cand), cand_cap, n_cand);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

void epic_search_destroy(epic_search_t s)
{
    if (!s) return;
    cudaFree(s->d_shift);
    cudaFree(s->d_mask);
    delete s;
}

}  // extern "C"

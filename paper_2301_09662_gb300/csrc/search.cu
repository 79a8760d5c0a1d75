// Transient search on the image cube: incoherent de-dispersion of every
// pixel's dynamic spectrum and a boxcar single-pulse search of the
// de-dispersed light curves (Sec. 4: light curves extracted per channel, the
// dispersive delay corrected across the band, single pulses searched; Sec. 5
// names de-dispersion and transient detection as the next modules).
//
//  * shifts: s[d][c] = floor(k_DM DM_d (f_c^-2 - f_max^-2) / dt + 1/2) samples,
//    f in MHz, computed once on the host in FP64 (the plan);
//  * dedisperse_staged_kernel: D[d][t][p] = sum_c I[t + s[d][c]][c][p].  A
//    block is 16 (or 32) trial DMs, two per warp, x 32 pixels (lanes,
//    coalesced) x 28 output samples; per channel the union of the block's
//    sweeps is staged in shared memory once (cp.async, eight channels in
//    flight) and every warp sums its two windows from there.  dedisperse_kernel
//    (each warp loading its own sweep) serves DM grids too coarse for the
//    staging buffer.  The cube is read
//    through (time, channel, pixel) strides, so the Stokes-I slot of an image
//    series (complex64 layout) is searched in place;
//  * single_pulse_kernel: one thread per (DM, pixel) light curve, one pass:
//    population moments and, per boxcar width 2^k <= 32, the largest window
//    sum (sums by doubling, S_2w(e) = S_w(e) + S_w(e - w), histories in
//    registers), normalised by mu and sigma at the end; a warp ballot marks the
//    pairs whose best S/N reaches the threshold;
//  * candidates_kernel: one block compacts the marked (DM, pixel) pairs in index
//    order (deterministic).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <new>
#include <vector>

#include <cudaTypedefs.h>

#include "epic_internal.cuh"
#include "tc_ptx.cuh"

struct epic_search_s {
    int C = 0, n_dm = 0, npix = 0, T = 0, T_out = 0, smax = 0;
    unsigned widths = 0;          // bit k: boxcar width 2^k (k < 6)
    int *d_shift = nullptr;       // [n_dm][C]
    unsigned *d_mask = nullptr;   // [n_dm][wpr] candidate bits, wpr = ceil(npix / 32)
    int wpr = 0;
    int dm_block = 0;             // trial DMs per block of the staged forms (32 or 16); 0: direct form
    int spread = 0;               // largest spread of the shifts over one block's trials (rows)
    bool pix2 = true;             // the two-pixel forms may serve cubes with unit pixel stride
    bool tma = true;              // the TMA form may serve cubes with 16-byte row pitches
    int *d_status = nullptr;      // sticky device status word (EPIC_ERR_TIMEOUT)
    long long wait_budget = 0;    // clock cycles before a device-side wait gives up
    int withhold = 0;             // failure-detection hook: the TMA form never loads channel 0
};

namespace epic {
namespace {

constexpr double kDM = 4.148808e3;   // s MHz^2 pc^-1 cm^3
constexpr int kPixB = 32, kDmB = 8, kTT = 32;
constexpr int kTS = 28;                          // output samples per block of the staged form (2 x 28 accumulators)
constexpr int kPix2 = 64, kT2 = 16;              // pixels and output samples per block of the two-pixel forms
constexpr int kStagesT = 8;                      // ring slots of the TMA form (a power of two)
constexpr long long kWaitBudget = 2000000000LL;  // clock cycles (about a second) before a wait gives up
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

__device__ __forceinline__ void cp_async8(float *dst, const float *src, int src_bytes)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}

// Two IEEE round-to-nearest FP32 adds in one instruction (the same results as two adds).
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    unsigned long long x, y, r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.x), "f"(b.y));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    float2 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
    return o;
}

// Staged form for a cube with unit pixel stride: as dedisperse_staged_kernel,
// but a lane owns two adjacent pixels (a warp 64), so one 8-byte shared load
// feeds two packed adds per trial DM; kT2 output samples per block.  Sums run
// in channel order, bit-identical to the other forms.
template <int WARPS>
__global__ void __launch_bounds__(32 * WARPS, 512 / (32 * WARPS))
dedisperse_staged2_kernel(const float *__restrict__ cube, long long ts, long long cs, int C, int npix, int T_out,
                          const int *__restrict__ shift, int n_dm, int rows_max, float *__restrict__ dd)
{
    constexpr int DMB = 2 * WARPS;
    extern __shared__ float dyn[];                   // [kStages][rows_max][kPix2], then the tables
    float *ring = dyn;
    int *sh = reinterpret_cast<int *>(dyn + kStages * rows_max * kPix2);   // [DMB][C]
    int *smin = sh + DMB * C, *srows = smin + C;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int d0 = blockIdx.x * DMB, p0 = blockIdx.y * kPix2, pix = p0 + 2 * lane, t0 = blockIdx.z * kT2;
    const int nt = min(kT2, T_out - t0);
    const int nd = min(DMB, n_dm - d0);
    const int valid = min(max(npix - pix, 0), 2);   // pixels of this lane inside the image
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
        srows[c] = nt + hi - lo;                      // kT2 + hi - lo <= rows_max, found when the plan was made
    }
    __syncthreads();
    const float *base = cube + (valid ? pix : p0);   // an aligned address inside the cube even when empty
    auto issue = [&](int c) {
        if (c < C) {
            const float *src = base + static_cast<long long>(t0 + smin[c]) * ts + c * cs;
            float *dst = ring + (c % kStages) * rows_max * kPix2 + 2 * lane;
            const int rows = srows[c];
            for (int r = w; r < rows; r += WARPS)
                cp_async8(dst + r * kPix2, src + static_cast<long long>(r) * ts, 4 * valid);
        }
        cp_async_commit();
    };
    float2 acc0[kT2], acc1[kT2];
#pragma unroll
    for (int j = 0; j < kT2; j++) acc0[j] = acc1[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < kStages - 1; c++) issue(c);
    for (int c = 0; c < C; c++) {
        cp_async_wait<kStages - 2>();
        __syncthreads();
        issue(c + kStages - 1);
        const int o0 = sh[2 * w * C + c] - smin[c], o1 = sh[(2 * w + 1) * C + c] - smin[c];
        const float2 *slot = reinterpret_cast<const float2 *>(ring + (c % kStages) * rows_max * kPix2) + lane;
        const float2 *row = slot + o0 * (kPix2 / 2);
        const int delta = o1 - o0;                   // warp-uniform
        if (delta == 0) {
#pragma unroll
            for (int j = 0; j < kT2; j++) {
                const float2 v = row[j * (kPix2 / 2)];
                acc0[j] = add2(acc0[j], v);
                acc1[j] = add2(acc1[j], v);
            }
        } else if (delta == 1) {
#pragma unroll
            for (int j = 0; j < kT2; j++) {
                const float2 v = row[j * (kPix2 / 2)];
                acc0[j] = add2(acc0[j], v);
                if (j) acc1[j - 1] = add2(acc1[j - 1], v);
            }
            acc1[kT2 - 1] = add2(acc1[kT2 - 1], row[kT2 * (kPix2 / 2)]);   // row o1 + kT2 - 1 < rows_max
        } else {
            const float2 *row1 = slot + o1 * (kPix2 / 2);
#pragma unroll
            for (int j = 0; j < kT2; j++) {
                acc0[j] = add2(acc0[j], row[j * (kPix2 / 2)]);
                acc1[j] = add2(acc1[j], row1[j * (kPix2 / 2)]);
            }
        }
    }
    cp_async_wait<0>();
    if (!valid) return;
    const bool pair = valid == 2 && !(npix & 1);     // 8-byte aligned pair stores
#pragma unroll
    for (int h = 0; h < 2; h++) {
        if (2 * w + h >= nd) break;
        float *out = dd + (static_cast<size_t>(d0 + 2 * w + h) * T_out + t0) * npix + pix;
#pragma unroll
        for (int j = 0; j < kT2; j++) {
            if (j >= nt) break;
            const float2 v = h ? acc1[j] : acc0[j];
            float *o = out + static_cast<size_t>(j) * npix;
            if (pair) {
                *reinterpret_cast<float2 *>(o) = v;
            } else {
                o[0] = v.x;
                if (valid == 2) o[1] = v.y;
            }
        }
    }
}

// TMA form (cube with unit pixel stride and 16-byte row pitches): WARPS
// consumer warps (two trial DMs and two pixels per lane each, as the two-pixel
// form) and one producer warp.  The producer loads each channel's rows
// t0 + min_d s[d][c] .. + rows of the block's 64 pixels with one 3-D tensor
// copy into an 8-slot ring (pixels and rows past the cube arrive as zeros);
// "full" barriers count the bytes, "empty" barriers the consumer warps that
// are done with a slot, so no block-wide barrier runs per channel.  Every wait
// is bounded: on a timeout the block sets the status word, waits (bounded) for
// the copies it has in flight and writes nothing.
template <int WARPS>
__global__ void __launch_bounds__(32 * (WARPS + 1), WARPS <= 8 ? 2 : 1)
dedisperse_tma_kernel(const __grid_constant__ CUtensorMap map, int C, int npix, int T_out,
                      const int *__restrict__ shift, int n_dm, int rows, float *__restrict__ dd,
                      int *__restrict__ status, long long budget, int withhold)
{
    constexpr int DMB = 2 * WARPS;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t pad = (1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u;
    float *ring = reinterpret_cast<float *>(smem_raw + pad);          // [kStagesT][rows][kPix2]
    uint64_t *full = reinterpret_cast<uint64_t *>(ring + kStagesT * rows * kPix2);
    uint64_t *empty = full + kStagesT;
    int *last = reinterpret_cast<int *>(empty + kStagesT);            // channel last loaded into each slot
    volatile int *flag = last + kStagesT;                             // a wait ran out
    int *sh = last + kStagesT + 1;                                    // [DMB][C]
    int *smin = sh + DMB * C;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int d0 = blockIdx.x * DMB, p0 = blockIdx.y * kPix2, pix = p0 + 2 * lane, t0 = blockIdx.z * kT2;
    const int nt = min(kT2, T_out - t0);
    const int nd = min(DMB, n_dm - d0);
    for (int i = threadIdx.x; i < DMB * C; i += blockDim.x) {
        const int d = i / C;
        sh[i] = shift[static_cast<size_t>(d0 + min(d, nd - 1)) * C + i % C];
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStagesT; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], WARPS);
            last[s] = -1;
        }
        *flag = 0;
        tc::fence_mbar_init();
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        int lo = sh[c];
        for (int d = 1; d < nd; d++) lo = min(lo, sh[d * C + c]);
        smin[c] = lo;
    }
    __syncthreads();
    if (w == WARPS) {                                 // producer
        if (lane == 0) {
            const uint32_t bytes = static_cast<uint32_t>(rows) * kPix2 * sizeof(float);
            for (int c = 0; c < C; c++) {
                const int s = c & (kStagesT - 1);
                if (c >= kStagesT && !tc::mbar_wait(&empty[s], ((c / kStagesT) - 1) & 1, budget)) {
                    *flag = 1;
                    break;
                }
                if (*flag) break;
                if (withhold && c == 0) continue;     // failure-detection hook: channel 0 never arrives
                tc::mbar_expect_tx(&full[s], bytes);
                tc::tma_load_3d(ring + s * rows * kPix2, &map, p0, c, t0 + smin[c], &full[s]);
                last[s] = c;
            }
        }
        __syncwarp();
    } else {                                          // consumers
        float2 acc0[kT2], acc1[kT2];
#pragma unroll
        for (int j = 0; j < kT2; j++) acc0[j] = acc1[j] = make_float2(0.f, 0.f);
        const int *sh0 = sh + 2 * w * C, *sh1 = sh0 + C;
        for (int c = 0; c < C; c++) {
            const int s = c & (kStagesT - 1);
            const bool ok = tc::mbar_wait(&full[s], (c / kStagesT) & 1, budget);
            if (!__all_sync(0xffffffffu, ok)) {
                *flag = 1;
                break;
            }
            const int o0 = sh0[c] - smin[c], o1 = sh1[c] - smin[c];
            const float2 *slot = reinterpret_cast<const float2 *>(ring + s * rows * kPix2) + lane;
            const float2 *row = slot + o0 * (kPix2 / 2);
            const int delta = o1 - o0;               // warp-uniform
            if (delta == 0) {
#pragma unroll
                for (int j = 0; j < kT2; j++) {
                    const float2 v = row[j * (kPix2 / 2)];
                    acc0[j] = add2(acc0[j], v);
                    acc1[j] = add2(acc1[j], v);
                }
            } else if (delta == 1) {
#pragma unroll
                for (int j = 0; j < kT2; j++) {
                    const float2 v = row[j * (kPix2 / 2)];
                    acc0[j] = add2(acc0[j], v);
                    if (j) acc1[j - 1] = add2(acc1[j - 1], v);
                }
                acc1[kT2 - 1] = add2(acc1[kT2 - 1], row[kT2 * (kPix2 / 2)]);   // row o1 + kT2 - 1 < rows
            } else {
                const float2 *row1 = slot + o1 * (kPix2 / 2);
#pragma unroll
                for (int j = 0; j < kT2; j++) {
                    acc0[j] = add2(acc0[j], row[j * (kPix2 / 2)]);
                    acc1[j] = add2(acc1[j], row1[j * (kPix2 / 2)]);
                }
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&empty[s]);
        }
        tc::named_bar_sync(1, 32 * (WARPS + 1));
        if (*flag) return;
        const int valid = min(max(npix - pix, 0), 2);
        if (!valid) return;
        const bool pair = valid == 2 && !(npix & 1);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            if (2 * w + h >= nd) break;
            float *out = dd + (static_cast<size_t>(d0 + 2 * w + h) * T_out + t0) * npix + pix;
#pragma unroll
            for (int j = 0; j < kT2; j++) {
                if (j >= nt) break;
                const float2 v = h ? acc1[j] : acc0[j];
                float *o = out + static_cast<size_t>(j) * npix;
                if (pair) {
                    *reinterpret_cast<float2 *>(o) = v;
                } else {
                    o[0] = v.x;
                    if (valid == 2) o[1] = v.y;
                }
            }
        }
        return;
    }
    tc::named_bar_sync(1, 32 * (WARPS + 1));          // the producer warp meets the consumers here
    if (*flag && threadIdx.x == 32 * WARPS) {
        atomicCAS(status, 0, static_cast<int>(EPIC_ERR_TIMEOUT));
        for (int s = 0; s < kStagesT; s++)            // copies still in flight land before the block exits
            if (last[s] >= 0) tc::mbar_wait(&full[s], (last[s] / kStagesT) & 1, budget);
    }
}

// cuTensorMapEncodeTiled from the driver, looked up once (null if absent).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

size_t tma_smem(int C, int dm_block, int rows)
{
    return 1024 + sizeof(float) * kStagesT * rows * kPix2 + sizeof(uint64_t) * 2 * kStagesT +
           sizeof(int) * (kStagesT + 1) + sizeof(int) * (dm_block + 1) * static_cast<size_t>(C);
}

size_t staged_smem(int C, int dm_block, int rows, int pix_block)
{
    return sizeof(float) * kStages * rows * pix_block + sizeof(int) * (dm_block + 2) * static_cast<size_t>(C);
}

// Largest spread of the shifts over one block of dm_block trials, over blocks and channels.
int staged_spread(const std::vector<int> &shift, int n_dm, int C, int dm_block)
{
    int need = 0;
    for (int d0 = 0; d0 < n_dm; d0 += dm_block)
        for (int c = 0; c < C; c++) {
            int lo = shift[static_cast<size_t>(d0) * C + c], hi = lo;
            for (int d = d0; d < std::min(n_dm, d0 + dm_block); d++) {
                lo = std::min(lo, shift[static_cast<size_t>(d) * C + c]);
                hi = std::max(hi, shift[static_cast<size_t>(d) * C + c]);
            }
            need = std::max(need, hi - lo);
        }
    return need;
}

// Boxcar sums of one 16-sample chunk of a light curve (y = x - x0) by
// doubling: S_1(e) = y_e and S_2w(e) = S_w(e) + S_w(e - w), so each width costs
// one add per sample and every window sum carries at most five roundings.
// h_w holds S_w of the previous w samples (slot e mod w; chunks start at
// multiples of 16, so the slots are compile-time).  Per width the largest S_w
// and the end e of its first occurrence are kept.  CHECK (the chunks that
// start before sample 32 or reach past T_out): windows ending before w - 1
// are not complete, samples at or past T_out are not part of the curve.
struct Boxcar {
    float h1[1], h2[2], h4[4], h8[8], h16[16];
    float bS[6];
    int bE[6];
};

template <bool CHECK>
__device__ __forceinline__ void boxcar_chunk(const float (&y)[16], int base, int T_out, Boxcar &b)
{
#pragma unroll
    for (int j = 0; j < 16; j++) {
        float S[6];
        S[0] = y[j];
        S[1] = S[0] + b.h1[0];
        b.h1[0] = S[0];
        S[2] = S[1] + b.h2[j & 1];
        b.h2[j & 1] = S[1];
        S[3] = S[2] + b.h4[j & 3];
        b.h4[j & 3] = S[2];
        S[4] = S[3] + b.h8[j & 7];
        b.h8[j & 7] = S[3];
        S[5] = S[4] + b.h16[j];
        b.h16[j] = S[4];
        const int e = base + j;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const bool ok = !CHECK || (e >= (1 << k) - 1 && e < T_out);
            if (ok && S[k] > b.bS[k]) {
                b.bS[k] = S[k];
                b.bE[k] = e;
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
// start.  Chunks are double-buffered: the loads of the next 16 samples are in
// flight while the current ones are scored.  A warp ballot of "best S/N >=
// threshold" gives the candidate mask (bit p mod 32 of word d * wpr + p / 32).
__global__ void __launch_bounds__(128, 5)
single_pulse_kernel(const float *__restrict__ dd, int T_out, int npix, unsigned widths, float threshold,
                    float *__restrict__ best_snr, int *__restrict__ best_t, int *__restrict__ best_w,
                    unsigned *__restrict__ mask, int wpr)
{
    const int pix = blockIdx.x * blockDim.x + threadIdx.x, d = blockIdx.y;
    const bool valid = pix < npix;
    const float *x = dd + static_cast<size_t>(d) * T_out * npix + min(pix, npix - 1);
    int wmin = 0;
    while (wmin < 6 && !((widths >> wmin) & 1u)) wmin++;
    Boxcar b;
    b.h1[0] = 0.f;
#pragma unroll
    for (int i = 0; i < 2; i++) b.h2[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 4; i++) b.h4[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 8; i++) b.h8[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 16; i++) b.h16[i] = 0.f;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        b.bS[k] = -INFINITY;
        b.bE[k] = 0;
    }
    float s1 = 0.f, s2 = 0.f;
    const float x0 = __ldg(x);
    auto load = [&](float (&y)[16], int base) {       // raw samples; 0 past the end
#pragma unroll
        for (int j = 0; j < 16; j++)
            y[j] = base + j < T_out ? __ldg(x + static_cast<size_t>(base + j) * npix) : x0;
    };
    auto score = [&](float (&y)[16], int base) {
        float b1 = 0.f, b2 = 0.f;
#pragma unroll
        for (int j = 0; j < 16; j++) {
            y[j] -= x0;
            b1 += y[j];
            b2 = fmaf(y[j], y[j], b2);
        }
        s1 += b1;
        s2 += b2;
        if (base < 32 || base + 16 > T_out)
            boxcar_chunk<true>(y, base, T_out, b);
        else
            boxcar_chunk<false>(y, base, T_out, b);
    };
    float ya[16], yb[16];
    load(ya, 0);
    for (int base = 0;; base += 32) {
        if (base + 16 < T_out) load(yb, base + 16);
        score(ya, base);
        if (base + 16 >= T_out) break;
        if (base + 32 < T_out) load(ya, base + 32);
        score(yb, base + 16);
        if (base + 32 >= T_out) break;
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
            if (((widths >> k) & 1u) && b.bS[k] > -INFINITY) {
                const float snr = (b.bS[k] - w * m1) / (sigma * sqrtf(w));
                if (snr > bs) {
                    bs = snr;
                    bt = b.bE[k] - (1 << k) + 1;
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
    constexpr unsigned kDiag = EPIC_SEARCH_DIAG_DM32 | EPIC_SEARCH_DIAG_DIRECT | EPIC_SEARCH_DIAG_NO_PIX2 |
                               EPIC_SEARCH_DIAG_NO_TMA | EPIC_SEARCH_DIAG_WITHHOLD_TMA;
    const unsigned diag = width_mask & kDiag;
    width_mask &= ~kDiag;
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
    // the staged kernels hold a tile + (spread of the shifts over one block's DMs) rows per
    // channel.  Blocks of 16 trials (two blocks per SM) measured faster than 32 in every staged
    // form; the diagnostic options ask for 32-trial blocks where they fit, or for the direct form.
    const int want = (diag & EPIC_SEARCH_DIAG_DIRECT) ? 0 : (diag & EPIC_SEARCH_DIAG_DM32) ? 32 : 16;
    const int spread32 = epic::staged_spread(shift, n_dm, n_chan, 32);
    const int spread16 = epic::staged_spread(shift, n_dm, n_chan, 16);
    if (want == 32 && epic::kTS + spread32 <= epic::kRows) {
        s->dm_block = 32;
        s->spread = spread32;
    } else if (want != 0 && epic::kTS + spread16 <= epic::kRows) {
        s->dm_block = 16;
        s->spread = spread16;
    }
    // diagnostics: keep unit-stride cubes on the one-pixel staged form, or on the cp.async forms
    s->pix2 = !(diag & EPIC_SEARCH_DIAG_NO_PIX2);
    s->tma = !(diag & EPIC_SEARCH_DIAG_NO_TMA);
    s->wait_budget = epic::kWaitBudget;
    // Fault injection for the failure-detection test: the TMA form's producer
    // skips channel 0, the consumers' wait runs out after a short budget and
    // the status word reports EPIC_ERR_TIMEOUT.
    if (diag & EPIC_SEARCH_DIAG_WITHHOLD_TMA) {
        s->withhold = 1;
        s->wait_budget = 2000000;   // ~1 ms
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
    if (cudaMalloc(&s->d_status, sizeof(int)) != cudaSuccess || cudaMemset(s->d_status, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(s->d_status);
        cudaFree(s->d_shift);
        delete s;
        return EPIC_ERR_NOMEM;
    }
    if (cudaMalloc(&s->d_mask, sizeof(unsigned) * static_cast<size_t>(n_dm) * s->wpr) != cudaSuccess) {
        cudaFree(s->d_status);
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
    // DM blocks fastest in every staged grid: the blocks that read the same rows run together and share L2
    const unsigned db = dmb ? static_cast<unsigned>((s->n_dm + dmb - 1) / dmb) : 0;
    if (dmb && s->pix2 && s->tma && pix_stride == 1 && t_stride % 4 == 0 && c_stride % 4 == 0 &&
        reinterpret_cast<uintptr_t>(cube) % 16 == 0) {
        const int rows = epic::kT2 + s->spread;
        const size_t smem = epic::tma_smem(s->C, dmb, rows);
        auto k = dmb == 32 ? epic::dedisperse_tma_kernel<16> : epic::dedisperse_tma_kernel<8>;
        const auto encode = epic::tensor_map_encoder();
        CUtensorMap map;
        const cuuint64_t dims[3] = {static_cast<cuuint64_t>(s->npix), static_cast<cuuint64_t>(s->C),
                                    static_cast<cuuint64_t>(s->T)};
        const cuuint64_t strides[2] = {static_cast<cuuint64_t>(c_stride) * sizeof(float),
                                       static_cast<cuuint64_t>(t_stride) * sizeof(float)};
        const cuuint32_t box[3] = {static_cast<cuuint32_t>(epic::kPix2), 1u, static_cast<cuuint32_t>(rows)};
        const cuuint32_t unit[3] = {1u, 1u, 1u};
        if (encode && rows <= 256 && smem <= 200 * 1024 &&
            encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(cube), dims, strides, box, unit,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS &&
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) ==
                cudaSuccess) {
            const dim3 grid(db, static_cast<unsigned>((s->npix + epic::kPix2 - 1) / epic::kPix2),
                            static_cast<unsigned>((s->T_out + epic::kT2 - 1) / epic::kT2));
            k<<<grid, 32 * (dmb / 2 + 1), smem, st>>>(map, s->C, s->npix, s->T_out, s->d_shift, s->n_dm, rows, dd,
                                                      s->d_status, s->wait_budget, s->withhold);
            return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
        }
    }
    if (dmb && s->pix2 && pix_stride == 1 && t_stride % 2 == 0 && c_stride % 2 == 0 &&
        reinterpret_cast<uintptr_t>(cube) % 8 == 0) {
        const int rows = epic::kT2 + s->spread;
        const size_t smem = epic::staged_smem(s->C, dmb, rows, epic::kPix2);
        auto k = dmb == 32 ? epic::dedisperse_staged2_kernel<16> : epic::dedisperse_staged2_kernel<8>;
        if (smem <= 200 * 1024 &&
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) == cudaSuccess) {
            const dim3 grid(db, static_cast<unsigned>((s->npix + epic::kPix2 - 1) / epic::kPix2),
                            static_cast<unsigned>((s->T_out + epic::kT2 - 1) / epic::kT2));
            k<<<grid, 32 * (dmb / 2), smem, st>>>(cube, t_stride, c_stride, s->C, s->npix, s->T_out, s->d_shift,
                                                  s->n_dm, rows, dd);
            return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
        }
    }
    const int rows = epic::kTS + s->spread;
    const size_t smem_staged = dmb ? epic::staged_smem(s->C, dmb, rows, epic::kPixB) : 0;
    auto staged = dmb == 32 ? epic::dedisperse_staged_kernel<16> : epic::dedisperse_staged_kernel<8>;
    if (dmb && smem_staged <= 200 * 1024 &&
        cudaFuncSetAttribute(staged, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem_staged)) == cudaSuccess) {
        const unsigned tbs = static_cast<unsigned>((s->T_out + epic::kTS - 1) / epic::kTS);
        staged<<<dim3(db, pb, tbs), epic::kPixB * (dmb / 2), smem_staged, st>>>(
            cube, t_stride, c_stride, pix_stride, s->C, s->npix, s->T_out, s->d_shift, s->n_dm, rows, dd);
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

int epic_search_status(epic_search_t s)
{
    if (!s) return EPIC_ERR_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return EPIC_ERR_CUDA;
    int st = 0;
    if (cudaMemcpy(&st, s->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return EPIC_ERR_CUDA;
    if (cudaMemset(s->d_status, 0, sizeof(int)) != cudaSuccess) return EPIC_ERR_CUDA;
    return st;
}

void epic_search_destroy(epic_search_t s)
{
    if (!s) return;
    cudaFree(s->d_shift);
    cudaFree(s->d_mask);
    cudaFree(s->d_status);
    delete s;
}

}  // extern "C"

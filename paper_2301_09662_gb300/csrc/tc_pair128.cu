// Tensor-core form for grid side 128 (dual polarisation): one CTA images two
// pixel classes of one channel from a single gridding of each sample.  The same
// kernel with CLS = 1 images grid side 64 (one class, no folding): the row
// stage, class 0's column stage and its products, nothing of class 1.
//
// With l = 2 m + h (h in {0, 1}^2) the image of class h is the 64-point 2-D DFT
// of the folded aperture Gf_h(j) = sum_{k = j mod 64} G(k) w_128^{k.h}.  The
// class phase is separable, w_128^{kx hx} w_128^{ky hy}.  A CTA owns the two
// classes (hx, 0) and (hx, 1): the x factor goes into the gridding (into the
// gains per antenna and the taps per column), so both classes share one
// gridded sample, one row transform and one conversion of its result; the y
// factor turns each folded input row of the column transform, and so goes
// into that transform's operand.  That needs one unfolded row ky per folded
// row jy among the cells any footprint touches (the aperture spans at most 64
// rows, as with 2x padding); the plan checks it per channel and lists the rows
// with ky >= 64, and then w_128^{ky} = w_128^{jy} (-1)^{ky >= 64}.
//
//   row stage     D1[(pol, jy)][r] = sum_k G16[(pol, jy)][k] X[r][k]
//                 G16 = the gridded sample in FP16 hi + lo (shared memory,
//                 K-major, A operand), X = the 64-point DFT in real 2 x 2 block
//                 form (shared memory, K-major, B operand)
//   column stage  D2_hy[r][n] = sum_k X_hy[r][k] H16[n][k],  n = (mx, pol)
//                 H16 = D1 as FP16 hi + lo (shared memory, MN-major, B
//                 operand); X_0 = X (shared memory), X_1 = X with input row jy
//                 turned by w_128^{ky} (TMEM, A operand, built once per CTA).
//                 The two classes' column stages run back to back, class 1's
//                 into D1's columns (D1 has been converted by then), class 0's
//                 into a second buffer; the next sample's row stage takes that
//                 one once class 0's products have read it, so the two buffers
//                 swap roles every sample and no stage waits for the products
//                 of the stage before it.
//
// Both stages take three MMAs per 16-deep k-block (hi hi + hi lo + lo hi).
//
// Gridding is a gather (the FP32 register kernel's lists, 16-bit entries): a
// lane sums the (antenna, tap pair) list of one pair of horizontally adjacent
// folded cells in FP32 registers and writes both cells' hi and lo straight into
// G16, so there is no FP32 grid and no conversion pass.  The lists write the
// same cells every sample and the transforms run in TMEM, so cells no list
// names stay zero from the start.
//
// TMEM columns: buffers P [0,128) and Q [256,384) (sample t: D1 and then D2_1
// in R(t), D2_0 in A(t); R = P for even t, Q for odd), X_1 [128,256) (hi, lo),
// the time sums of class hy = 1 [384,512); class hy = 0 keeps its time sums in
// registers.  Shared memory: X, G16 and
// H16 (64 KB each, hi and lo), the channel's gather lists, calibrated
// voltages (two samples), gains, tap pairs.
//
// Warps 0-7 (TMEM warps), iteration t: wait for the row stage of t, D1 -> H16
// and arrive on bar_h; grid the first part of their lists of sample t+1; wait
// for class 0's column stage, add its products and arrive on bar_fa; grid the
// second part and arrive on bar_g; wait for class 1's column stage, add its
// products and arrive on bar_fb.  Warps 8-10 only grid: after the row stage of t
// they take a larger share of sample t+1's lists (the plan deals the lists so
// that each warp's work, conversions and products included, is about equal)
// and arrive on bar_g; then, while the TMEM warps form products, they unpack
// and calibrate sample t+2 (its bytes copied asynchronously since the
// iteration began) into the other of two voltage buffers, so no unpacking lies
// between a row stage and the next gridding.  Warp 11 issues, in order, the
// row stage of t after bar_g (and, from the second sample on, bar_fa of
// t - 1), then after bar_h (and bar_fb of t - 1) the column stages of classes
// 0 and 1, each committed to its own mbarrier.  Each of its waits costs a
// shared-memory round trip of a few hundred cycles under the gridding's load,
// so it waits first for the barrier that is usually complete (bar_fa, bar_fb)
// and last for the one on the path (bar_g, bar_h), and reads the abort flag
// once a sample while the row stage runs.  Every wait is bounded; a timeout is
// recorded in the plan's status word and stops the CTA.  Twelve warps cost no registers over nine: a
// scheduler holding three warps already limits a thread to 168.
#include <algorithm>
#include <array>
#include <cstdlib>

#include "dft_small.cuh"
#include "epic_internal.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace epic {
namespace {

using namespace tcc;

constexpr int kTmemWarps = 8;                    // warps 0-7: grid, convert the row stage, form products
constexpr int kGathW = kTmemWarps + kPairHelpers; // + warps that only grid
constexpr int kSimtP = kTmemWarps * 32;          // threads that touch TMEM (bar_h arrivals)
constexpr int kGath = kGathW * 32;               // threads that grid (bar_g arrivals, the named barrier)
constexpr int kMmaWarp = kGathW;                 // the MMA-issuing warp
constexpr int kPairThreads = (kGathW + 1) * 32;
constexpr int kBarP = 6;                         // named barrier of the gridding warps
constexpr int kBarH = 7;                         // named barrier of the gridding-only warps
constexpr uint32_t kColP = 0, kColXt = 128, kColQ = 256, kColAcc1 = 384;
// sample t's row stage and class 1's column stage use buffer R(t), class 0's column stage A(t);
// the two swap every sample
__device__ __forceinline__ uint32_t col_r(int t) { return (t & 1) ? kColQ : kColP; }
__device__ __forceinline__ uint32_t col_a(int t) { return (t & 1) ? kColP : kColQ; }
constexpr uint16_t kNone = 0xFFFFu;

// XX, YY, XY of one sample added to the time sums of one class: TMEM lanes
// 32 (w mod 4) + l = (my, part), the column block 64 hh .. (hh = w / 4,
// pixels mx = 32 hh ..) of the column stage's result at column d2.  Lane l keeps pixels mx = 32 hh + 16 part + j,
// j < 16; Re and Im of a pixel are exchanged between lanes l and l ^ 16 by one
// shuffle.  Two halves of 8 pixels (x8 loads of the own and the partner's
// columns) bound the live registers.  Class hy = 0 sums into registers (acc),
// class hy = 1 into TMEM columns kColAcc1 + 64 hh .. (4 per pixel).
template <bool REG>
__device__ __forceinline__ void products(uint32_t lane_addr, uint32_t d2, int hh, int part, float4 (&acc)[16])
{
#pragma unroll
    for (int half = 0; half < 2; half++) {
        // columns 8 half .. (part 0's pixels) and 16 + 8 half .. (part 1's) of each polarisation
        // in the column block 64 hh .. of D2 (polarisation 0 at + 0-31, 1 at + 32-63); a TMEM load's
        // address is warp-uniform, so each lane then picks its own part and the one its partner needs
        uint32_t x0[8], y0[8], x1[8], y1[8];
        const uint32_t base = lane_addr + d2 + 64 * hh + 8 * half;
        tc::tmem_ld8_issue(base, x0);
        tc::tmem_ld8_issue(base + 16, x1);
        tc::tmem_ld8_issue(base + 32, y0);
        tc::tmem_ld8_issue(base + 48, y1);
        uint32_t s[32];
        const uint32_t at = lane_addr + kColAcc1 + 64 * hh + 32 * half;
        if constexpr (!REG) tc::tmem_ld32_issue(at, s);
        tc::tmem_wait_ld();
        tc::reg_fence8(x0);
        tc::reg_fence8(x1);
        tc::reg_fence8(y0);
        tc::reg_fence8(y1);
        if constexpr (!REG) tc::reg_fence32(s);
#pragma unroll
        for (int jj = 0; jj < 8; jj++) {
            const uint32_t ox = part ? x1[jj] : x0[jj], oy = part ? y1[jj] : y0[jj];
            const uint32_t sx = part ? x0[jj] : x1[jj], sy = part ? y0[jj] : y1[jj];
            // (a, b) = (own, partner's) parts of F_X, (c, d) of F_Y: (Re, Im) on part-0 lanes,
            // (Im, Re) on part-1 lanes.  XX, YY and Re XY are symmetric in that swap; Im XY =
            // b c - a d on part-0 lanes and its negative on part-1 lanes, fixed at the end.
            const float b = __shfl_xor_sync(0xffffffffu, __uint_as_float(sx), 16);
            const float d = __shfl_xor_sync(0xffffffffu, __uint_as_float(sy), 16);
            const float a = __uint_as_float(ox), c = __uint_as_float(oy);
            if constexpr (REG) {
                float4 &q = acc[8 * half + jj];
                q.x = fmaf(a, a, fmaf(b, b, q.x));
                q.y = fmaf(c, c, fmaf(d, d, q.y));
                q.z = fmaf(a, c, fmaf(b, d, q.z));
                q.w = fmaf(b, c, fmaf(-a, d, q.w));
            } else {
                uint32_t *a4 = s + 4 * jj;
                a4[0] = __float_as_uint(fmaf(a, a, fmaf(b, b, __uint_as_float(a4[0]))));
                a4[1] = __float_as_uint(fmaf(c, c, fmaf(d, d, __uint_as_float(a4[1]))));
                a4[2] = __float_as_uint(fmaf(a, c, fmaf(b, d, __uint_as_float(a4[2]))));
                a4[3] = __float_as_uint(fmaf(b, c, fmaf(-a, d, __uint_as_float(a4[3]))));
            }
        }
        if constexpr (!REG) {
            tc::tmem_st32_issue(at, s);
            tc::tmem_wait_st();
        }
    }
}

// Shared memory (dynamic, 1024-aligned): X, G16, H16 (each hi then lo), then
// es [2][A*P], gp [A*P], tw2 [K (K + 1) + 1][8] (float4: eight interleaved copies,
// lane l reads copy l mod 8, so the eight lanes of one 16-byte request never
// share a bank group; the last slot is zero, for the lists' empty steps),
// stage [(A*P + 3) / 4] (u32), the channel's lists [words] (u16).
template <int VAR, int CLS, int MF>
__global__ void __launch_bounds__(kPairThreads, 1)
tc_pair128_kernel(const uint8_t *__restrict__ v, const float2 *__restrict__ gains,
                  const short2 *__restrict__ cells, const float2 *__restrict__ kern, int K,
                  const int *__restrict__ chans, const float2 *__restrict__ twN,
                  const uint16_t *__restrict__ ptab, const int2 *__restrict__ pchan, const int4 *__restrict__ pidx,
                  const unsigned long long *__restrict__ upper,
                  const uint8_t *__restrict__ dft_ops, int A, int C, int T, int n_items_out, int n_tau,
                  float *__restrict__ partial, int *__restrict__ status, long long wait_budget, int withhold_mma,
                  const float *__restrict__ dfreq, const float4 *__restrict__ dtab)
{
    constexpr int P = 2;
    // grid side: two classes of folded side MF (128 or 96), or side 64 unfolded; a 48-point DFT
    // sits in the 64-point operands' first 48 rows and columns (the rest zero)
    constexpr int N = CLS == 2 ? 2 * MF : MF;
    static_assert(MF == 64 || (MF == 48 && CLS == 2), "folded sides 64 and 48");
    auto wrap = [](int x) { return ((x % N) + N) % N; };
    constexpr bool kBF16 = VAR == 2;
    constexpr bool kSplit = VAR != 1;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *opX = smem;                                      // [2 parts][32 KB] K-major
    uint8_t *opG = smem + 2 * kPart;                          // [2 parts][32 KB] K-major
    uint8_t *opH = smem + 4 * kPart;                          // [2 parts][32 KB] MN-major
    const int AP = A * P, KK = K * K, hk = (K - 1) / 2;
    const int APW = (AP + 3) >> 2;
    float2 *es = reinterpret_cast<float2 *>(smem + 6 * kPart);   // sample t in es + (t & 1) AP
    float2 *gp = es + 2 * AP;
    float4 *tw2 = reinterpret_cast<float4 *>(gp + AP);
    const int TPN = K * (K + 1);                             // the zero tap slot
    uint32_t *stage = reinterpret_cast<uint32_t *>(tw2 + 8 * (TPN + 1));
    uint16_t *stab = reinterpret_cast<uint16_t *>(stage + APW);
    __shared__ __align__(8) uint64_t bar_x, bar_g, bar_h, bar_fa, bar_fb, bar_m1, bar_m2[2];
    __shared__ uint32_t tmem_slot;
    __shared__ float red[kGathW];
    __shared__ int abort_flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool simt = warp < kGathW;             // a gridding warp (TMEM warps included)
    const bool tmw = warp < kTmemWarps;
    const int n_pairs = gridDim.x / n_tau;                    // CTAs per time chunk: channels x CLS
    const int item = blockIdx.x % n_pairs;
    const int tau = blockIdx.x / n_pairs;
    const int ci = CLS == 2 ? item >> 1 : item, hx = CLS == 2 ? item & 1 : 0;
    const int c = chans[ci];
    const int t0 = static_cast<int>(static_cast<long long>(T) * tau / n_tau);
    const int t1 = static_cast<int>(static_cast<long long>(T) * (tau + 1) / n_tau);
    const int2 my_chan = pchan[ci];

    if (warp == 0) tc::tmem_alloc(&tmem_slot, 512);
    if (tid == 0) {
        abort_flag = 0;
        tc::mbar_init(&bar_x, 1);
        tc::mbar_init(&bar_g, kGath);
        tc::mbar_init(&bar_h, kSimtP);
        tc::mbar_init(&bar_m1, 1);
        tc::mbar_init(&bar_fa, kSimtP);
        tc::mbar_init(&bar_fb, kSimtP);
        tc::mbar_init(&bar_m2[0], 1);
        tc::mbar_init(&bar_m2[1], 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {   // the DFT operand, hi and lo, one bulk copy each
        tc::mbar_expect_tx(&bar_x, 2 * kPart);
        tc::bulk_g2s(opX, dft_ops, kPart, &bar_x);
        tc::bulk_g2s(opX + kPart, dft_ops + kPart, kPart, &bar_x);
    }

    // ---- set-up: gains and taps with the class-x phase, the largest gain for the FP16 scale,
    // a zero G16, the channel's lists, the bytes of the first sample
    float gmax = 0.f;
    for (int a = simt ? tid : A; a < A; a += kGath) {
        const short2 k = cells[static_cast<size_t>(c) * A + a];
        if (k.x < hk || k.x >= N - hk || k.y < hk || k.y >= N - hk) atomicOr(status, kStatusDevice);
        const float2 ph = twN[wrap(k.x * hx)];
        for (int p = 0; p < P; p++) {
            const float2 g = gains ? gains[(static_cast<size_t>(c) * A + a) * P + p] : make_float2(1.f, 0.f);
            const float2 gg = cmul(g, ph);
            gp[a * P + p] = gg;
            gmax = fmaxf(gmax, sqrtf(gg.x * gg.x + gg.y * gg.y));
        }
    }
    // tap pairs (w(dy, dxl), w(dy, dxl + 1)), zero outside the footprint row, with w_128^{dx hx}
    for (int i = simt ? tid : 8 * (TPN + 1); i < 8 * (TPN + 1); i += kGath) {
        const int tp = i >> 3, dyi = tp / (K + 1), j = tp % (K + 1);
        float2 w[2];
        for (int u = 0; u < 2; u++) {
            const int dx = j - 1 + u;
            w[u] = (tp < TPN && dx >= 0 && dx < K) ? cmul(kern[dyi * K + dx], twN[wrap((dx - hk) * hx)])
                                                   : make_float2(0.f, 0.f);
        }
        tw2[i] = make_float4(w[0].x, w[0].y, w[1].x, w[1].y);
    }
    for (int i = simt ? tid : 2 * static_cast<int>(kPart) / 16; i < 2 * static_cast<int>(kPart) / 16; i += kGath)
        reinterpret_cast<uint4 *>(opG)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = simt ? tid : my_chan.y; i < my_chan.y; i += kGath) stab[i] = __ldg(ptab + my_chan.x + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    if (simt && lane == 0) red[warp] = gmax;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tmem_slot;
    const uint32_t lane_addr = taddr + (static_cast<uint32_t>(32 * (warp & 3)) << 16);
    float scale = 1.f;
    if constexpr (!kBF16) {
        // |H| <= sum_a |e~_a| sum_taps |w| bounds both stages' operands: keep it below 2^13
        float gm = 0.f;
        for (int w = 0; w < kGathW; w++) gm = fmaxf(gm, red[w]);
        float wsum = 0.f;
        for (int i = 0; i < KK; i++) wsum += sqrtf(kern[i].x * kern[i].x + kern[i].y * kern[i].y);
        const float bound = 2.f * static_cast<float>(A) * 11.3137085f * gm * wsum;
        int e2 = 0;
        if (bound > 0.f) e2 = static_cast<int>(floorf(log2f(16384.f / bound)));
        scale = ldexpf(1.f, max(-40, min(40, e2)));
    }
    for (int i = simt ? tid : AP; i < AP; i += kGath) gp[i] = cscale(gp[i], scale);
    if (CLS == 2 && tmw) {
        // zero the TMEM time sums of class hy = 1: lanes 32 (w mod 4) .., columns kColAcc1 + 64 (w / 4) ..
        uint32_t z[32];
#pragma unroll
        for (int j = 0; j < 32; j++) z[j] = 0u;
        const uint32_t acc = lane_addr + kColAcc1 + 64 * (warp >> 2);
        tc::tmem_st32_issue(acc, z);
        tc::tmem_st32_issue(acc + 32, z);
        // the column-stage operand of class hy = 1 (A operand in TMEM): X with input row jy
        // turned by w_N^{ky}, ky = jy + MF [row listed as upper], i.e. the rotation by
        // w_N^{2 jy my + ky} in real 2 x 2 form (N = 2 MF).  Lane = output (my, part), columns k / 2 of
        // k = 64 im_in + jy (hi, then lo 64 columns on); warp half w / 4 = im_in.
        const int myo = 16 * (warp & 3) + (lane & 15), prt = lane >> 4, imin = warp >> 2;
        const unsigned long long up = upper[ci];
        uint32_t xh[32], xl[32];
#pragma unroll
        for (int w = 0; w < 32; w++) {
            float a2[2];
#pragma unroll
            for (int u = 0; u < 2; u++) {
                const int j = 2 * w + u;
                const int kyj = j + (((up >> j) & 1ull) ? MF : 0);
                const float2 e = twN[wrap(2 * j * myo + kyj)];
                a2[u] = prt == 0 ? (imin ? -e.y : e.x) : (imin ? e.x : e.y);
                if (MF < 64 && (j >= MF || myo >= MF)) a2[u] = 0.f;   // outside the 48-point DFT
            }
            split_pair<kBF16, kSplit>(a2[0], a2[1], xh[w], xl[w]);
        }
        tc::tmem_st32_issue(lane_addr + kColXt + 32 * imin, xh);
        if constexpr (kSplit) tc::tmem_st32_issue(lane_addr + kColXt + 64 + 32 * imin, xl);
        tc::tmem_wait_st();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    constexpr uint32_t idesc_row = idesc_kk(128, 128, kBF16);
    constexpr uint32_t idesc_col = idesc_kmn(128, 128, kBF16);
    const uint32_t x_base = tc::smem_u32(opX), g_base = tc::smem_u32(opG), h_base = tc::smem_u32(opH);

    if (!simt) {
        // ---- the MMA warp (kMmaWarp): row stage of t after bar_g, column stages of (t, 0) and (t, 1)
        // after the next two completions of bar_h
        if (lane == 0) {
            bool ok = tc::mbar_wait(&bar_x, 0, wait_budget);
            uint32_t pg = 0, ph = 0, pf = 0;
            for (int t = t0; t < t1 && ok; t++) {
                if (t > t0)   // R(t) = A(t - 1): the products of (t - 1, 0) have read it
                    ok = tc::mbar_wait(&bar_fa, pf, wait_budget);
                ok = ok && tc::mbar_wait(&bar_g, pg, wait_budget);
                pg ^= 1u;
                if (!ok) break;
                tc::fence_after_sync();
                if (!withhold_mma) {
#pragma unroll
                    for (int kb = 0; kb < 8; kb++) {
                        if (MF < 64 && (kb & 3) * 16 >= MF) continue;   // k beyond the folded side: zeros
                        const uint64_t g_hi = tc::smem_desc(g_base + kb * 256, kLBO, kSBO);
                        const uint64_t x_hi = tc::smem_desc(x_base + kb * 256, kLBO, kSBO);
                        tc::mma_f16(taddr + col_r(t), g_hi, x_hi, idesc_row, kb > 0 ? 1u : 0u);
                        if constexpr (kSplit) {
                            const uint64_t g_lo = tc::smem_desc(g_base + kPart + kb * 256, kLBO, kSBO);
                            const uint64_t x_lo = tc::smem_desc(x_base + kPart + kb * 256, kLBO, kSBO);
                            tc::mma_f16(taddr + col_r(t), g_hi, x_lo, idesc_row, 1u);
                            tc::mma_f16(taddr + col_r(t), g_lo, x_hi, idesc_row, 1u);
                        }
                    }
                    tc::mma_commit(&bar_m1);
                }
                if (abort_flag) {
                    ok = false;
                    break;
                }
                if (CLS == 2 && t > t0)   // A(t) = R(t - 1): the products of (t - 1, 1) have read it
                    ok = tc::mbar_wait(&bar_fb, pf, wait_budget);
                ok = ok && tc::mbar_wait(&bar_h, ph, wait_budget);
                ph ^= 1u;
                if (t > t0) pf ^= 1u;
                if (!ok) break;
                tc::fence_after_sync();
                if (!withhold_mma) {
                    // class hy = 0: A = X (shared memory) into A(t); class hy = 1: A = the turned X in
                    // TMEM into R(t) (converted to H16 by now)
                    for (int hy = 0; hy < CLS; hy++) {
                        const uint32_t d2 = taddr + (hy ? col_r(t) : col_a(t));
#pragma unroll
                        for (int kb = 0; kb < 8; kb++) {
                            if (MF < 64 && (kb & 3) * 16 >= MF) continue;
                            const uint64_t h_hi = tc::smem_desc(h_base + kb * 256, kLBO, kSBO);
                            const uint64_t h_lo = tc::smem_desc(h_base + kPart + kb * 256, kLBO, kSBO);
                            if (hy == 0) {
                                const uint64_t x_hi = tc::smem_desc(x_base + kb * 256, kLBO, kSBO);
                                tc::mma_f16(d2, x_hi, h_hi, idesc_col, kb > 0 ? 1u : 0u);
                                if constexpr (kSplit) {
                                    const uint64_t x_lo = tc::smem_desc(x_base + kPart + kb * 256, kLBO, kSBO);
                                    tc::mma_f16(d2, x_hi, h_lo, idesc_col, 1u);
                                    tc::mma_f16(d2, x_lo, h_hi, idesc_col, 1u);
                                }
                            } else {
                                const uint32_t a_hi = taddr + kColXt + kb * 8;
                                mma_ts(d2, a_hi, h_hi, idesc_col, kb > 0 ? 1u : 0u);
                                if constexpr (kSplit) {
                                    mma_ts(d2, a_hi, h_lo, idesc_col, 1u);
                                    mma_ts(d2, a_hi + 64, h_hi, idesc_col, 1u);
                                }
                            }
                        }
                        tc::mma_commit(&bar_m2[hy]);
                    }
                }
            }
            if (!ok) {
                atomicOr(status, kStatusTimeout);
                abort_flag = 1;
            }
        }
        __syncwarp();
    } else {
        const int m = 32 * (warp & 3) + lane;          // TMEM warps: lane m = (pol, jy) in D1, (my, part) in D2
        const int hp = (warp >> 2) & 1;                 // which half of the columns
        const bool prod_rows = 16 * (warp & 3) < MF;    // the warp's pixel rows my = 16 (w mod 4) .. exist
        const int part = lane >> 4;
        const int pol = m >> 6, jy = m & 63;
        const int4 my_idx = pidx[ci * kGathW + warp];   // (first batch, batches in half 1, second half's start, batches in half 2)

        // a1, a2: unpack and calibrate sample t into es + (t & 1) AP, from the bytes at `src`
        // (global or staged), by threads first, first + stride, ...
        auto unpack = [&](int t, const uint8_t *src, int first, int stride) {
            float2 *dst = es + (t & 1) * AP;
            for (int i = first; i < AP; i += stride) {
                float2 e = cmul(gp[i], ci4_decode(src[i]));
                if (dtab) e = cmul(e, delay_phase(dtab[static_cast<size_t>(t) * A + i / P], dfreq[c]));
                dst[i] = e;
            }
        };
        auto bytes_of = [&](int t) { return v + (static_cast<size_t>(t) * C + c) * AP; };
        const bool helper = !tmw;
        const int htid = tid - kSimtP;                  // helpers: 0 .. 32 kPairHelpers - 1
        // a3: gather gridding of n batches from offset `at` (u16 units) straight into G16.  A
        // batch is [d][32 G16 byte offsets of the lanes' cell pairs (pol 0, Re, hi part), or
        // 0xFFFF][d x 32 entries tp << 10 | a]; empty steps name the zero tap slot.
        auto gather = [&](int at, int n, int t) {
            const uint16_t *bt = stab + at;
            const float4 *es4 = reinterpret_cast<const float4 *>(es + (t & 1) * AP);
            const float4 *tw8 = tw2 + (lane & 7);
            const uint32_t empty = static_cast<uint32_t>(TPN) << 10;
            // the next batch's header and first entry are loaded a batch ahead (every batch has d >= 1)
            int d = 0;
            uint32_t off = kNone, e0 = empty;
            if (n > 0) {
                d = bt[0];
                off = bt[1 + lane];
                e0 = bt[33 + lane];
            }
            for (int b = 0; b < n; b++) {
                const uint16_t *ent = bt + 33 + lane;
                const uint16_t *nbt = bt + 33 + 32 * d;
                int dn = 0;
                uint32_t offn = kNone, e0n = empty;
                if (b + 1 < n) {
                    dn = nbt[0];
                    offn = nbt[1 + lane];
                    e0n = nbt[33 + lane];
                }
                float2 acc[P][2];
#pragma unroll
                for (int p = 0; p < P; p++) acc[p][0] = acc[p][1] = make_float2(0.f, 0.f);
                // software-pipelined: the entry two steps ahead and the taps and voltages one step
                // ahead are in flight while the current step's multiply-adds run (unrolled by four)
                uint32_t en1 = d > 1 ? ent[32] : empty;
                float4 ww = tw8[(e0 >> 10) << 3];
                float4 ee = es4[e0 & 1023u];
#pragma unroll 4
                for (int j = 0; j < d; j++) {
                    const uint32_t en2 = j + 2 < d ? ent[(j + 2) * 32] : empty;
                    const float4 wwn = tw8[(en1 >> 10) << 3];
                    const float4 een = es4[en1 & 1023u];
                    // cell u += w_u e_p (complex), as scalar FMAs with the sign folded in
                    const float wr[2] = {ww.x, ww.z}, wi[2] = {ww.y, ww.w};
                    const float er[2] = {ee.x, ee.z}, ei[2] = {ee.y, ee.w};
#pragma unroll
                    for (int p = 0; p < P; p++)
#pragma unroll
                        for (int u = 0; u < 2; u++) {
                            acc[p][u].x = fmaf(-wi[u], ei[p], fmaf(wr[u], er[p], acc[p][u].x));
                            acc[p][u].y = fmaf(wi[u], er[p], fmaf(wr[u], ei[p], acc[p][u].y));
                        }
                    ww = wwn;
                    ee = een;
                    en1 = en2;
                }
                if (off != kNone) {
                    // Re at off, Im at + 1024 (K + 64), polarisation 1 at + 16384 (rows + 64)
#pragma unroll
                    for (int p = 0; p < P; p++) {
                        uint32_t rh, rl, ih, il;
                        split_pair<kBF16, kSplit>(acc[p][0].x, acc[p][1].x, rh, rl);
                        split_pair<kBF16, kSplit>(acc[p][0].y, acc[p][1].y, ih, il);
                        uint8_t *at0 = opG + off + 16384 * p;
                        *reinterpret_cast<uint32_t *>(at0) = rh;
                        *reinterpret_cast<uint32_t *>(at0 + 1024) = ih;
                        if constexpr (kSplit) {
                            *reinterpret_cast<uint32_t *>(at0 + kPart) = rl;
                            *reinterpret_cast<uint32_t *>(at0 + kPart + 1024) = il;
                        }
                    }
                }
                bt = nbt;
                d = dn;
                off = offn;
                e0 = e0n;
            }
        };
        // D1 (row transform of the sample) -> H16, shared by both classes (class hy = 1's turn is in
        // its column-stage operand).  Thread: lane m = (pol, jy), columns 64 hp .. 64 hp + 63 = Re
        // and Im of mx = 32 hp .. 32 hp + 31; H16 row n = 64 hp + 32 pol + (mx - 32 hp), so each
        // half buffer of the column stage reads one contiguous N = 64 block.
        auto to_h16 = [&](uint32_t d1) {
#pragma unroll
            for (int q = 0; q < 2; q++) {
                uint32_t d[32];
                tc::tmem_ld32_issue(lane_addr + d1 + 64 * hp + 32 * q, d);
                tc::tmem_wait_ld();
                tc::reg_fence32(d);
#pragma unroll
                for (int g8 = 0; g8 < 2; g8++) {
                    uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
                    for (int w = 0; w < 4; w++) {
                        const int i = 8 * g8 + 2 * w;
                        split_pair<kBF16, kSplit>(__uint_as_float(d[i]), __uint_as_float(d[i + 1]), rh[w], rl[w]);
                        split_pair<kBF16, kSplit>(__uint_as_float(d[16 + i]), __uint_as_float(d[17 + i]), ih[w], il[w]);
                    }
                    const int n0 = 64 * hp + 32 * pol + 16 * q + 8 * g8;
                    *reinterpret_cast<uint4 *>(opH + mn_off(n0, jy)) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
                    *reinterpret_cast<uint4 *>(opH + mn_off(n0, 64 + jy)) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
                    if constexpr (kSplit) {
                        *reinterpret_cast<uint4 *>(opH + kPart + mn_off(n0, jy)) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
                        *reinterpret_cast<uint4 *>(opH + kPart + mn_off(n0, 64 + jy)) =
                            make_uint4(il[0], il[1], il[2], il[3]);
                    }
                }
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            tc::mbar_arrive(&bar_h);
        };
        // helpers: the bytes of sample t copied asynchronously into the stage
        auto stage_async = [&](int t) {
            if (t >= t1) return;
            const uint32_t *row = reinterpret_cast<const uint32_t *>(bytes_of(t));
            for (int w = htid; w < APW; w += 32 * kPairHelpers) tc::cp_async4(stage + w, row + w);
        };
        auto fail = [&]() {
            atomicOr(status, kStatusTimeout);
            abort_flag = 1;
        };

        float4 acc0[16];
#pragma unroll
        for (int j = 0; j < 16; j++) acc0[j] = make_float4(0.f, 0.f, 0.f, 0.f);

        // prologue: samples t0 and t0 + 1 unpacked, t0 gridded into G16
        if (t0 < t1) {
            unpack(t0, bytes_of(t0), tid, kGath);
            if (t0 + 1 < t1) unpack(t0 + 1, bytes_of(t0 + 1), tid, kGath);
            tc::named_bar_sync(kBarP, kGath);
            gather(my_idx.x, my_idx.y, t0);
            gather(my_idx.z, my_idx.w, t0);
            tc::fence_proxy_async();
            tc::fence_before_sync();
            tc::mbar_arrive(&bar_g);
            tc::named_bar_sync(kBarP, kGath);
        }
        uint32_t p1 = 0, p2 = 0;
        for (int t = t0; t < t1; t++) {
            const bool nxt = t + 1 < t1;
            if (helper) stage_async(t + 2);
            // row stage of t done: G16 is free for sample t + 1; the TMEM warps convert D1 -> H16
            if (!abort_flag) {
                if (!tc::mbar_wait(&bar_m1, p1, wait_budget)) fail();
                else if (tmw) {
                    tc::fence_after_sync();
                    to_h16(col_r(t));
                }
            }
            p1 ^= 1u;
            if (tmw) {
                if (nxt && !abort_flag) gather(my_idx.x, my_idx.y, t + 1);
                // a5, a6: products of (t, 0)
                if (!abort_flag) {
                    if (!tc::mbar_wait(&bar_m2[0], p2, wait_budget)) fail();
                    else {
                        tc::fence_after_sync();
                        if (prod_rows) products<true>(lane_addr, col_a(t), hp, part, acc0);
                        tc::fence_before_sync();
                        tc::mbar_arrive(&bar_fa);
                    }
                }
            }
            if (nxt && !abort_flag) {
                if (tmw) gather(my_idx.z, my_idx.w, t + 1);
                else gather(my_idx.x, my_idx.y, t + 1);
                tc::fence_proxy_async();
                tc::fence_before_sync();
                tc::mbar_arrive(&bar_g);
            }
            if (helper && t + 2 < t1) {
                // sample t + 2 into the buffer sample t used (all gridding of t ended at the last
                // iteration's closing barrier); the closing barrier below publishes it
                tc::cp_async_wait_all();
                tc::named_bar_sync(kBarH, 32 * kPairHelpers);   // every helper's copies landed
                unpack(t + 2, reinterpret_cast<const uint8_t *>(stage), htid, 32 * kPairHelpers);
            }
            if (CLS == 2 && tmw && !abort_flag) {
                // products of (t, 1), from R(t), which is then free for class 0's column stage of t + 1
                if (!tc::mbar_wait(&bar_m2[1], p2, wait_budget)) fail();
                else {
                    tc::fence_after_sync();
                    if (prod_rows) products<false>(lane_addr, col_r(t), hp, part, acc0);
                    tc::fence_before_sync();
                    tc::mbar_arrive(&bar_fb);
                }
            }
            p2 ^= 1u;
            tc::fence_before_sync();
            if (tc::named_bar_or(kBarP, kGath, abort_flag != 0)) break;   // the same answer in every warp
        }

        if (helper) tc::cp_async_wait_all();             // no copy outlives the loop
        // ---- partial images of both classes (undo the FP16 scale exactly)
        tc::fence_after_sync();
        if (tmw) {
            const float inv = 1.f / (scale * scale);
            const float inv_im = part ? -inv : inv;        // Im XY was summed with the lane's part sign
            const int my = 16 * (warp & 3) + (lane & 15);
            // items: channel ci's classes h = 2 hy + hx (side 128), or channel ci (side 64)
            float4 *dst0 = reinterpret_cast<float4 *>(partial) +
                           (static_cast<size_t>(tau) * n_items_out + (CLS == 2 ? ci * 4 + hx : ci)) * (MF * MF);
            float4 *dst1 = reinterpret_cast<float4 *>(partial) +
                           (static_cast<size_t>(tau) * n_items_out + ci * 4 + 2 + hx) * (MF * MF);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int mx = 32 * hp + 16 * part + j;
                if (my < MF && mx < MF)
                    dst0[my * MF + mx] = make_float4(acc0[j].x * inv, acc0[j].y * inv, acc0[j].z * inv, acc0[j].w * inv_im);
            }
#pragma unroll
            for (int half = 0; half < (CLS == 2 ? 2 : 0); half++) {
                uint32_t s[32];
                tc::tmem_ld32_issue(lane_addr + kColAcc1 + 64 * hp + 32 * half, s);
                tc::tmem_wait_ld();
                tc::reg_fence32(s);
#pragma unroll
                for (int jj = 0; jj < 8; jj++) {
                    const int mx = 32 * hp + 16 * part + 8 * half + jj;
                    if (my < MF && mx < MF)
                        dst1[my * MF + mx] = make_float4(__uint_as_float(s[4 * jj]) * inv, __uint_as_float(s[4 * jj + 1]) * inv,
                                                         __uint_as_float(s[4 * jj + 2]) * inv,
                                                         __uint_as_float(s[4 * jj + 3]) * inv_im);
                }
            }
        }
    }
    // an aborted CTA may still have MMAs in flight: give them a bounded chance to land
    if (tid == kMmaWarp * 32 && abort_flag) {
        tc::mbar_wait(&bar_m1, 0, wait_budget);
        tc::mbar_wait(&bar_m1, 1, wait_budget);
        for (int i = 0; i < 2; i++) {
            tc::mbar_wait(&bar_m2[i], 0, wait_budget);
            tc::mbar_wait(&bar_m2[i], 1, wait_budget);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, 512);
}

size_t pair_smem(int A, int K, int words)
{
    const int AP = A * 2;
    size_t b = 6 * static_cast<size_t>(kPart);
    b += sizeof(float2) * 3 * static_cast<size_t>(AP) + sizeof(float4) * 8 * (static_cast<size_t>(K) * (K + 1) + 1);
    b += sizeof(uint32_t) * ((AP + 3) / 4) + sizeof(uint16_t) * static_cast<size_t>(words);
    return (b + 15) & ~static_cast<size_t>(15);
}

template <class F>
int pair_dispatch(int precision, F &&f)
{
    switch (precision) {
    case EPIC_TC_SPLIT_FP16: return f(std::integral_constant<int, 0>{});
    case EPIC_TC_FP16: return f(std::integral_constant<int, 1>{});
    default: return f(std::integral_constant<int, 2>{});
    }
}

// the instantiation for a group: two classes of folded side 64 (grid side 128) or 48 (96), or one
// class of side 64
template <int VAR>
const void *pair_kernel(int cls, int mf)
{
    if (cls == 1) return reinterpret_cast<const void *>(tc_pair128_kernel<VAR, 1, 64>);
    return mf == 48 ? reinterpret_cast<const void *>(tc_pair128_kernel<VAR, 2, 48>)
                    : reinterpret_cast<const void *>(tc_pair128_kernel<VAR, 2, 64>);
}

}  // namespace

// The gather lists of the pair kernel, rebuilt from the FP32 kernel's table of
// the same channels (build_gather_table, fold side 64, dual polarisation: per
// pair of adjacent folded cells, the (antenna, tap pair) entries of the
// footprints that cover it).  Batches of 32 cell pairs are formed again for
// this kernel: pairs sorted by list length, and each batch takes, from a
// window of the next pairs, ones whose 32-bit stores into G16 fall in distinct
// banks -- a pair (y, 2 xp) is stored at bank 4 (y mod 8) + xp mod 4 of every
// part, so 32 pairs with distinct (y mod 8, xp mod 4) store without conflicts.
// Within each group of 8 lanes (one 16-byte request of the voltage loads) the
// step order is then chosen so that one step reads distinct banks, antenna
// a mod 8, as far as the lists allow.  Storage: [list length d][32 G16 byte
// offsets k_off(y, 2 xp) of the pairs (0xFFFF: an empty lane)][d x 32 entries
// tp << 10 | a] in 16-bit words, an empty step naming tap slot K (K + 1)
// (zeros) and an antenna its step loads anyway; no zero lists (G16 keeps the
// cells no list names at zero).  Before that a batch's lists are grouped into
// the four 8-lane groups so that each group's antennas spread over the bank
// slots, and the greedy step order is then improved by a local search (swaps
// within a lane's list) on the voltage loads' wavefronts.  The
// batches are dealt to the kernel's gridding warps longest first, each to the
// warp with the least work so far (a batch costs 4 d + 6, about 37 cycles a
// unit): the 8 TMEM warps start with sched.tmem_load units for their
// conversions and products, the gridding-only warps with none.  A TMEM warp's
// batches are split in two parts for the two gridding phases of an iteration,
// about sched.first_pct percent of the work in the first (it overlaps class 0's
// column stage, the second only part of class 1's, after class 0's products); a
// gridding-only warp has one list.  The defaults (90 units, 80 %) are the
// measured best on the LWA-like layout; epic_autotune measures a few others.  idx[ci * kPairGatherWarps + w]
// = (first half's offset, its batches, second half's offset, its batches),
// offsets in words from the channel block's start; chan[ci] = (block start,
// block words).  The upper mask of a channel lists the folded rows whose cells
// lie in unfolded rows 64..127; EPIC_ERR_UNSUPPORTED when a folded row holds
// cells of both halves, when A > 1024, or when K (K + 1) > 63.
int build_pair_tables(const std::vector<short2> &cells, int A, int K, const std::vector<int> &chans,
                      const std::vector<uint32_t> &tab32, const std::vector<int4> &idx32,
                      const std::vector<int2> &chan32, std::vector<uint16_t> &tab, std::vector<int4> &idx,
                      std::vector<int2> &chan, std::vector<unsigned long long> &upper, const PairSchedule &sched,
                      int M)
{
    constexpr int W32 = 8, W = kPairGatherWarps, kWindow = 96;
    const int S = M + 1;
    const long long kTmemLoad = sched.tmem_load;
    if (A > 1024 || K * (K + 1) > 63 || sched.tmem_load < 0 || sched.first_pct < 0 || sched.first_pct > 100 ||
        (M != 64 && M != 48))
        return EPIC_ERR_UNSUPPORTED;
    const int nc = static_cast<int>(chans.size()), h = (K - 1) / 2;
    tab.clear();
    idx.assign(static_cast<size_t>(nc) * W, make_int4(0, 0, 0, 0));
    chan.assign(nc, make_int2(0, 0));
    upper.assign(nc, 0ull);
    for (int ci = 0; ci < nc; ci++) {
        unsigned long long lo_rows = 0, hi_rows = 0;
        for (int a = 0; a < A; a++) {
            const short2 k = cells[static_cast<size_t>(chans[ci]) * A + a];
            for (int dy = -h; dy <= h; dy++) {
                const int ky = k.y + dy;
                if (ky < 0 || ky >= 2 * M) return EPIC_ERR_UNSUPPORTED;
                if (ky >= M) hi_rows |= 1ull << (ky - M);
                else lo_rows |= 1ull << ky;
            }
        }
        if (lo_rows & hi_rows) return EPIC_ERR_UNSUPPORTED;
        upper[ci] = hi_rows;
        // every cell pair of the channel with its entries (tp << 10 | a)
        const uint32_t *blk = tab32.data() + chan32[ci].x;
        std::vector<std::pair<int, std::vector<uint16_t>>> pairs;   // (y * 32 + xp, entries)
        for (int w = 0; w < W32; w++) {
            const int4 i32 = idx32[static_cast<size_t>(ci) * W32 + w];
            int at = i32.z;
            for (int b = 0; b < i32.w; b++) {
                const int d = static_cast<int>(blk[at]);
                for (int l = 0; l < 32; l++) {
                    const uint32_t cw = blk[at + 1 + l];
                    if (cw == ~0u) continue;
                    std::vector<uint16_t> ent;
                    for (int j = 0; j < d; j++) {
                        const uint32_t en = blk[at + 33 + 32 * j + l];
                        if (en != ~0u) ent.push_back(static_cast<uint16_t>(((en & 0xFFu) << 10) | (en >> 8)));
                    }
                    pairs.push_back({static_cast<int>(cw / S) * 32 + static_cast<int>(cw % S) / 2, std::move(ent)});
                }
                at += 33 + 32 * d;
            }
        }
        std::stable_sort(pairs.begin(), pairs.end(),
                         [](const auto &u, const auto &v) { return u.second.size() > v.second.size(); });
        // batches of 32 pairs with distinct store banks where the window allows
        std::vector<std::vector<int>> batches;
        std::vector<char> taken(pairs.size(), 0);
        size_t first = 0;
        while (first < pairs.size()) {
            std::vector<int> bt;
            bool bank[32] = {};
            for (size_t q = first; q < pairs.size() && q < first + kWindow && bt.size() < 32; q++) {
                if (taken[q]) continue;
                const int pos = pairs[q].first, r = 4 * ((pos >> 5) & 7) + (pos & 3);
                if (bank[r]) continue;
                bank[r] = true;
                taken[q] = 1;
                bt.push_back(static_cast<int>(q));
            }
            for (size_t q = first; q < pairs.size() && bt.size() < 32; q++)   // fill: conflicts allowed
                if (!taken[q]) {
                    taken[q] = 1;
                    bt.push_back(static_cast<int>(q));
                }
            while (first < pairs.size() && taken[first]) first++;
            batches.push_back(std::move(bt));
        }
        // repair store-bank conflicts: a pair whose bank its batch already uses is exchanged with a
        // pair of another batch whose bank is free there, when its own bank is free in the other
        // batch and neither batch's longest list grows (so no batch gains steps)
        {
            auto bank_of = [&](int q) { const int pos = pairs[q].first; return 4 * ((pos >> 5) & 7) + (pos & 3); };
            const int nb = static_cast<int>(batches.size());
            std::vector<std::array<int, 32>> cnt(nb);
            std::vector<size_t> dmax(nb, 0);
            for (int b = 0; b < nb; b++) {
                cnt[b].fill(0);
                for (int q : batches[b]) {
                    cnt[b][bank_of(q)]++;
                    dmax[b] = std::max(dmax[b], pairs[q].second.size());
                }
            }
            for (int pass = 0; pass < 3; pass++) {
                bool moved = false;
                for (int b1 = 0; b1 < nb; b1++)
                    for (size_t i1 = 0; i1 < batches[b1].size(); i1++) {
                        const int q1 = batches[b1][i1], r1 = bank_of(q1);
                        if (cnt[b1][r1] < 2) continue;
                        const size_t len = pairs[q1].second.size();
                        bool done = false;
                        for (int b2 = 0; b2 < nb && !done; b2++) {
                            if (b2 == b1 || cnt[b2][r1] > 0 || len > dmax[b2]) continue;   // r1 free in b2
                            for (size_t i2 = 0; i2 < batches[b2].size() && !done; i2++) {
                                const int q2 = batches[b2][i2], r2 = bank_of(q2);
                                if (pairs[q2].second.size() > dmax[b1] || cnt[b1][r2] > 0) continue;   // r2 free in b1
                                batches[b1][i1] = q2;
                                batches[b2][i2] = q1;
                                cnt[b1][r1]--;
                                cnt[b1][r2]++;
                                cnt[b2][r2]--;
                                cnt[b2][r1]++;
                                done = moved = true;
                            }
                        }
                    }
                if (!moved) break;
            }
        }
        // each batch as words: length, positions, then the steps with distinct voltage banks per
        // group of 8 lanes where possible
        std::vector<std::vector<uint16_t>> words(batches.size());
        std::vector<int> blen(batches.size());
        for (size_t b = 0; b < batches.size(); b++) {
            auto &bt = batches[b];
            // the batch's lanes into 4 groups of 8 (one 16-byte voltage request each) so that a
            // group's antennas spread over the 8 bank slots a mod 8: a group needs at least
            // max(its longest list, the most distinct antennas on one slot) wavefronts per
            // sample; lists go longest first to the group that bound grows least for, then
            // swaps of two lists between groups while the sum falls (the store banks do not
            // depend on the lane)
            if (bt.size() > 8) {
                const int nq = static_cast<int>(bt.size());
                std::vector<int> ord(nq);
                for (int i = 0; i < nq; i++) ord[i] = i;
                std::stable_sort(ord.begin(), ord.end(), [&](int u, int v) {
                    return pairs[bt[u]].second.size() > pairs[bt[v]].second.size();
                });
                auto bound = [&](const int *lanes, int n) {
                    uint64_t seen[16] = {};          // antennas < 1024
                    int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0}, mx = 0, dl = 0;
                    for (int k = 0; k < n; k++) {
                        const auto &lst = pairs[bt[lanes[k]]].second;
                        dl = std::max(dl, static_cast<int>(lst.size()));
                        for (uint16_t e : lst) {
                            const int a = e & 1023;
                            const uint64_t bit = 1ull << (a & 63);
                            if (seen[a >> 6] & bit) continue;
                            seen[a >> 6] |= bit;
                            mx = std::max(mx, ++cnt[a & 7]);
                        }
                    }
                    return std::max(dl, mx);
                };
                int grp[4][8], gn[4] = {0, 0, 0, 0};
                for (int i : ord) {
                    int best_g = -1, best_inc = 0;
                    for (int g = 0; g < 4; g++) {
                        if (gn[g] >= 8) continue;
                        const int before = bound(grp[g], gn[g]);
                        grp[g][gn[g]] = i;
                        const int inc = bound(grp[g], gn[g] + 1) - before;
                        if (best_g < 0 || inc < best_inc) {
                            best_g = g;
                            best_inc = inc;
                        }
                    }
                    grp[best_g][gn[best_g]++] = i;
                }
                int cost[4];
                for (int g = 0; g < 4; g++) cost[g] = bound(grp[g], gn[g]);
                bool better = true;
                for (int pass = 0; pass < 4 && better; pass++) {
                    better = false;
                    for (int g1 = 0; g1 < 4; g1++)
                        for (int g2 = g1 + 1; g2 < 4; g2++)
                            for (int i1 = 0; i1 < gn[g1]; i1++)
                                for (int i2 = 0; i2 < gn[g2]; i2++) {
                                    std::swap(grp[g1][i1], grp[g2][i2]);
                                    const int c1 = bound(grp[g1], gn[g1]), c2 = bound(grp[g2], gn[g2]);
                                    if (c1 + c2 < cost[g1] + cost[g2]) {
                                        cost[g1] = c1;
                                        cost[g2] = c2;
                                        better = true;
                                    } else {
                                        std::swap(grp[g1][i1], grp[g2][i2]);
                                    }
                                }
                }
                // every group at its own 8-lane slot (a group of fewer than 8 leaves empty lanes, -1)
                std::vector<int> placed(32, -1);
                for (int g = 0; g < 4; g++)
                    for (int k = 0; k < gn[g]; k++) placed[8 * g + k] = bt[grp[g][k]];
                bt = placed;
            }
            int d = 0;
            for (int q : bt)
                if (q >= 0) d = std::max(d, static_cast<int>(pairs[q].second.size()));
            blen[b] = d;
            auto &wd = words[b];
            const int empty_tp = K * (K + 1);                                    // the zero tap slot
            const uint16_t empty = static_cast<uint16_t>(empty_tp << 10);
            wd.assign(1 + 32 + static_cast<size_t>(d) * 32, empty);
            wd[0] = static_cast<uint16_t>(d);
            for (int l = 0; l < 32; l++) {
                if (l >= static_cast<int>(bt.size()) || bt[l] < 0) {
                    wd[1 + l] = 0xFFFFu;
                    continue;
                }
                const int pos = pairs[bt[l]].first;
                wd[1 + l] = static_cast<uint16_t>(k_off(pos >> 5, 2 * (pos & 31)));   // pol 0, Re, hi part
            }
            for (int g0 = 0; g0 < 32; g0 += 8) {
                std::vector<std::vector<uint16_t>> rem(8);
                for (int l = 0; l < 8; l++)
                    if (g0 + l < static_cast<int>(bt.size()) && bt[g0 + l] >= 0) rem[l] = pairs[bt[g0 + l]].second;
                for (int j = 0; j < d; j++) {
                    std::vector<int> order(8);
                    for (int l = 0; l < 8; l++) order[l] = l;
                    std::stable_sort(order.begin(), order.end(),
                                     [&](int u, int v) { return rem[u].size() > rem[v].size(); });
                    int slot[8];
                    for (int &x : slot) x = -1;
                    for (int l : order) {
                        auto &r = rem[l];
                        if (r.empty()) continue;
                        const bool must = static_cast<int>(r.size()) >= d - j;
                        int pick = -1;
                        for (size_t q = 0; q < r.size() && pick < 0; q++) {
                            const int a = r[q] & 1023, sl = a & 7;
                            if (slot[sl] < 0 || slot[sl] == a) pick = static_cast<int>(q);
                        }
                        if (pick < 0 && must) pick = 0;
                        if (pick < 0) continue;
                        const uint16_t e = r[pick];
                        r.erase(r.begin() + pick);
                        slot[(e & 1023) & 7] = e & 1023;
                        wd[1 + 32 + static_cast<size_t>(j) * 32 + g0 + l] = e;
                    }
                }
                // then a local search over each lane's order (two of its steps swapped, empty ones
                // included) while the group's voltage loads need fewer wavefronts: a step costs the
                // most distinct antennas any 16-byte bank group (a mod 8) receives
                auto at = [&](int j, int l) -> uint16_t & { return wd[1 + 32 + static_cast<size_t>(j) * 32 + g0 + l]; };
                auto step_cost = [&](int j) {
                    int seen[8], ns = 0, cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0}, mx = 1;
                    for (int l = 0; l < 8; l++) {
                        const uint16_t e = at(j, l);
                        if ((e >> 10) == empty_tp) continue;
                        const int a = e & 1023;
                        bool dup = false;
                        for (int q = 0; q < ns; q++) dup = dup || seen[q] == a;
                        if (dup) continue;
                        seen[ns++] = a;
                        mx = std::max(mx, ++cnt[a & 7]);
                    }
                    return mx;
                };
                bool improved = d <= 24;   // (bounded: plan time grows as d^2 per pass)
                for (int pass = 0; pass < 4 && improved; pass++) {
                    improved = false;
                    for (int l = 0; l < 8; l++)
                        for (int j1 = 0; j1 < d; j1++)
                            for (int j2 = j1 + 1; j2 < d; j2++) {
                                uint16_t &x = at(j1, l), &y = at(j2, l);
                                if (x == y) continue;
                                const int before = step_cost(j1) + step_cost(j2);
                                std::swap(x, y);
                                if (step_cost(j1) + step_cost(j2) < before) improved = true;
                                else std::swap(x, y);
                            }
                }
                // an empty step loads an antenna its step loads anyway (its tap pair is zero)
                for (int j = 0; j < d; j++) {
                    int a0 = 0;
                    for (int l = 0; l < 8; l++)
                        if ((at(j, l) >> 10) != empty_tp) {
                            a0 = at(j, l) & 1023;
                            break;
                        }
                    for (int l = 0; l < 8; l++)
                        if ((at(j, l) >> 10) == empty_tp) at(j, l) = static_cast<uint16_t>((empty_tp << 10) | a0);
                }
            }
        }
        // deal to the gridding warps
        std::vector<int> ord(batches.size());
        for (size_t b = 0; b < ord.size(); b++) ord[b] = static_cast<int>(b);
        std::stable_sort(ord.begin(), ord.end(), [&](int u, int v) { return blen[u] > blen[v]; });
        std::vector<std::vector<int>> per(W);
        std::vector<long long> load(W, 0);
        for (int w = 0; w < 8; w++) load[w] = kTmemLoad;
        for (int b : ord) {
            const int w = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
            per[w].push_back(b);
            load[w] += 4LL * blen[b] + 6;
        }
        const size_t start = tab.size();
        for (int w = 0; w < W; w++) {
            long long total = 0;
            for (int b : per[w]) total += 4LL * blen[b] + 6;
            size_t split = per[w].size();   // gridding-only warps: one list
            if (w < 8) {
                // the prefix closest to first_pct percent of the warp's gridding
                long long run = 0, best = -1;
                for (size_t i = 0; i <= per[w].size(); i++) {
                    const long long dev = std::llabs(100 * run - sched.first_pct * total);
                    if (best < 0 || dev < best) {
                        best = dev;
                        split = i;
                    }
                    if (i < per[w].size()) run += 4LL * blen[per[w][i]] + 6;
                }
            }
            int4 &o = idx[static_cast<size_t>(ci) * W + w];
            for (int half = 0; half < 2; half++) {
                const size_t b0 = half ? split : 0, b1 = half ? per[w].size() : split;
                const int off = static_cast<int>(tab.size() - start);
                if (half) {
                    o.z = off;
                    o.w = static_cast<int>(b1 - b0);
                } else {
                    o.x = off;
                    o.y = static_cast<int>(b1 - b0);
                }
                for (size_t q = b0; q < b1; q++) tab.insert(tab.end(), words[per[w][q]].begin(), words[per[w][q]].end());
            }
        }
        const size_t nwords = tab.size() - start;
        if (nwords > 0xFFFFFFull || start > 0x7FFFFFFFull) return EPIC_ERR_UNSUPPORTED;
        chan[ci] = make_int2(static_cast<int>(start), static_cast<int>(nwords));
    }
    if (tab.empty()) tab.push_back(0);
    return EPIC_OK;
}

size_t tc_pair_smem_bytes(int A, int K, int words) { return pair_smem(A, K, words); }

int prepare_tc_pair(const epic_plan_s *plan, size_t smem)
{
    return pair_dispatch(plan->precision, [&](auto vv) {
        constexpr int V = decltype(vv)::value;
        int rc = raise_dyn_smem_cap(pair_kernel<V>(2, 64), smem);
        if (rc == EPIC_OK) rc = raise_dyn_smem_cap(pair_kernel<V>(1, 64), smem);
        return rc != EPIC_OK ? rc : raise_dyn_smem_cap(pair_kernel<V>(2, 48), smem);
    });
}

int launch_tc_pair(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau_out,
                   cudaStream_t stream)
{
    int n_tau = choose_tau(plan, g, T);
    if (n_tau > g.tau_cap) n_tau = g.tau_cap;
    *n_tau_out = n_tau;
    const int cls = g.Q1 == 2 ? 2 : 1;
    const dim3 grid(static_cast<unsigned>(g.n_chan * cls * n_tau));
    const size_t smem = pair_smem(plan->A, plan->K, g.pwords);
    const uint8_t *dft = g.M == 48 ? plan->d_dft48 : plan->d_dft;
    return pair_dispatch(plan->precision, [&](auto vv) {
        constexpr int V = decltype(vv)::value;
        auto kfn = cls == 1 ? tc_pair128_kernel<V, 1, 64> : g.M == 48 ? tc_pair128_kernel<V, 2, 48> : tc_pair128_kernel<V, 2, 64>;
        kfn<<<grid, kPairThreads, smem, stream>>>(
            v, gains, plan->d_cells, plan->d_kernel, plan->K, g.d_chans, g.d_twN, g.d_ptab, g.d_pchan, g.d_pidx,
            g.d_upper, dft, plan->A, plan->C, T, g.n_items, n_tau, g.d_partial, plan->d_status,
            plan->wait_budget, plan->test_withhold_mma, plan->d_dfreq, plan->delays ? plan->d_dtab : nullptr);
        return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
    });
}

}  // namespace epic

// Two-stage tensor-core form (folded side M = 64, dual polarisation): both
// 64-point DFTs of every sample run as real GEMMs on tcgen05, the CUDA cores
// only unpack, grid, convert operands and form the products.
//
//   row stage     D1[(pol, jy)][r] = sum_k G16[(pol, jy)][k] X[r][k]
//                 k = 64 part' + jx, G16 = the gridded sample (hi, lo) in TMEM
//                 (A operand), X = the 64-point DFT in real 2 x 2 block form in
//                 shared memory (B operand, K-major), so D1 holds the row
//                 transform H: column r = (part, kx) in the drain order below
//   column stage  D2[r][(mx, pol)] = sum_k X[r][k] H16[(mx, pol)][k]
//                 k = 64 part + jy, X again (now the A operand, from shared
//                 memory), H16 = D1 re-packed as FP16 (hi, lo) in shared memory
//                 (B operand, MN-major, columns n = mx + 64 pol)
//
// Both stages take three MMAs per 16-deep k-block (hi hi + hi lo + lo hi), so
// each product keeps ~22 significant bits.  Row r of X is (my, part) with
// r = 32 q + l, my = 16 q + (l mod 16), part = l / 16: the Re and Im rows of a
// pixel sit in lanes l and l ^ 16 of one TMEM lane quarter.
//
// TMEM columns: G16 [0,128) (hi [0,64), lo [64,128); two 16-bit K values per
// 32-bit column, lower K in the low half), D1 [128,256), D2 [256,384), time
// sums [384,512) (lane r keeps XX, YY, Re XY, Im XY of 16 pixels per column
// half).  Shared memory: X (hi, lo: 64 KB, one bulk copy per CTA), H16 (64 KB),
// the FP32 grid (66.5 KB).
//
// Warps 0-7 (SIMT), iteration t: convert G(t) -> G16 in TMEM and arrive on
// bar_g (G is never cleared: each cell's first write in the static gridding
// schedule stores instead of adding); unpack, calibrate and grid sample t+1 while the row stage
// of t runs; sum the products of D2(t-1); wait for the row stage of t, convert
// D1 -> H16 and arrive on bar_h.  Warp 8 issues the row stage of t after bar_g
// and the column stage after bar_h, each committed to its own mbarrier; the
// column stage of t runs while G(t+1) is converted.  Every wait is bounded; a
// timeout is recorded in the plan's status word and stops the CTA.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dft_small.cuh"
#include "epic_internal.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

#include <cmath>
#include <type_traits>
#include <vector>

namespace epic {
namespace {

constexpr int M64 = 64;
constexpr int S64 = 65;
using namespace tcc;
constexpr uint32_t kColG = 0, kColD1 = 128, kColD2 = 256, kColAcc = 384;
constexpr int kSimt = kThreads;                 // warps 0-7
constexpr int kDualThreads = kSimt + 32;        // + the MMA warp
constexpr int kBarSimt = 5;

// XX, YY, XY of one sample added to this warp's time sums: TMEM lanes 32 (w mod 4) + l
// = (my, part), columns 32 hh .. 32 hh + 31 of each polarisation (hh = w / 4).  Lane l
// keeps the pixels j = 16 part .. 16 part + 15 of the half at sum columns
// kColAcc + 64 hh + 4 (j mod 16); Re and Im of a pixel are exchanged between lanes l
// and l ^ 16 by one shuffle.
__device__ __forceinline__ void products(uint32_t lane_addr, int hh, int part)
{
    uint32_t rx[32], ry[32], s0[32], s1[32];
    const uint32_t acc = lane_addr + kColAcc + 64 * hh;
    tc::tmem_ld32_issue(lane_addr + kColD2 + 32 * hh, rx);
    tc::tmem_ld32_issue(lane_addr + kColD2 + 64 + 32 * hh, ry);
    tc::tmem_ld32_issue(acc, s0);
    tc::tmem_ld32_issue(acc + 32, s1);
    tc::tmem_wait_ld();
    tc::reg_fence32(rx);
    tc::reg_fence32(ry);
    tc::reg_fence32(s0);
    tc::reg_fence32(s1);
#pragma unroll
    for (int j = 0; j < 16; j++) {
        const float ox = __uint_as_float(part ? rx[16 + j] : rx[j]);
        const float oy = __uint_as_float(part ? ry[16 + j] : ry[j]);
        const float sx = __uint_as_float(part ? rx[j] : rx[16 + j]);
        const float sy = __uint_as_float(part ? ry[j] : ry[16 + j]);
        const float gx = __shfl_xor_sync(0xffffffffu, sx, 16);
        const float gy = __shfl_xor_sync(0xffffffffu, sy, 16);
        const float xr = part ? gx : ox, xi = part ? ox : gx;
        const float yr = part ? gy : oy, yi = part ? oy : gy;
        uint32_t *a4 = j < 8 ? s0 + 4 * j : s1 + 4 * (j - 8);
        a4[0] = __float_as_uint(fmaf(xr, xr, fmaf(xi, xi, __uint_as_float(a4[0]))));
        a4[1] = __float_as_uint(fmaf(yr, yr, fmaf(yi, yi, __uint_as_float(a4[1]))));
        a4[2] = __float_as_uint(fmaf(xr, yr, fmaf(xi, yi, __uint_as_float(a4[2]))));
        a4[3] = __float_as_uint(fmaf(xi, yr, fmaf(-xr, yi, __uint_as_float(a4[3]))));
    }
    tc::tmem_st32_issue(acc, s0);
    tc::tmem_st32_issue(acc + 32, s1);
    tc::tmem_wait_st();
}

template <int VAR, int KC>
__global__ void __launch_bounds__(kDualThreads, 1)
tc_dual64_kernel(const uint8_t *__restrict__ v, const float2 *__restrict__ gains,
                 const short2 *__restrict__ cells, const float2 *__restrict__ kern, int K_rt,
                 const int *__restrict__ chans, const float2 *__restrict__ twN,
                 const uint32_t *__restrict__ sched, const int *__restrict__ nrounds, int rmax,
                 const uint8_t *__restrict__ dft_ops, int A, int C, int T, int N, int Q1, int n_items, int n_tau,
                 float *__restrict__ partial, int *__restrict__ status, long long wait_budget, int withhold_mma,
                 const float *__restrict__ dfreq, const float4 *__restrict__ dtab,
                 const uint16_t *__restrict__ first, const float2 *__restrict__ gf, int accumulate, int npol)
{
    // npol = 1: single polarisation; the Y rows of the operands stay zero and only XX is written
    const int P = npol;
    constexpr bool kBF16 = VAR == 2;
    constexpr bool kSplit = VAR != 1;
    constexpr int BUF = M64 * S64;
    const int K = KC > 0 ? KC : K_rt;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *opX = smem;                                              // [2 parts][32 KB] K-major
    uint8_t *opH = smem + 2 * kPart;                                  // [2 parts][32 KB] MN-major
    float2 *G = reinterpret_cast<float2 *>(smem + 4 * kPart);         // [2][64][65] (X, Y)
    const int AP = A * P, KK = K * K, hk = (K - 1) / 2;
    const int APW = (AP + 3) >> 2;
    float2 *es = G + 2 * BUF;
    float2 *gp = es + AP;
    float2 *tapw = gp + AP;
    uint32_t *stage = reinterpret_cast<uint32_t *>(tapw + KK);
    __shared__ __align__(8) uint64_t bar_x, bar_g, bar_h, bar_m1, bar_m2;
    __shared__ uint32_t tmem_slot;
    __shared__ float red[kSimt / 32];
    __shared__ int abort_flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool simt = warp < 8;
    const int item = blockIdx.x % n_items;
    const int tau = blockIdx.x / n_items;
    const int Q = Q1 * Q1;
    const int ci = item / Q, h = item % Q, hx = h % Q1, hy = h / Q1;
    const int c = chans[ci];
    const int t0 = static_cast<int>(static_cast<long long>(T) * tau / n_tau);
    const int t1 = static_cast<int>(static_cast<long long>(T) * (tau + 1) / n_tau);
    const uint32_t *my_sched = sched + (static_cast<size_t>(ci) * 8 + min(warp, 7)) * rmax * 32;
    // first: per descriptor, the taps whose cell no earlier round writes.  Those store instead of
    // adding, so G (gridded values only: the transforms run in TMEM) needs no clearing between
    // samples -- cells no footprint touches stay zero from the start
    const uint16_t *my_first = first + (static_cast<size_t>(ci) * 8 + min(warp, 7)) * rmax * 32;
    const int my_rounds = simt ? nrounds[ci * 8 + warp] : 0;

    if (warp == 0) tc::tmem_alloc(&tmem_slot, 512);
    if (tid == 0) {
        abort_flag = 0;
        tc::mbar_init(&bar_x, 1);
        tc::mbar_init(&bar_g, kSimt);
        tc::mbar_init(&bar_h, kSimt);
        tc::mbar_init(&bar_m1, 1);
        tc::mbar_init(&bar_m2, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {   // the DFT operand, hi and lo, one bulk copy each
        tc::mbar_expect_tx(&bar_x, 2 * kPart);
        tc::bulk_g2s(opX, dft_ops, kPart, &bar_x);
        tc::bulk_g2s(opX + kPart, dft_ops + kPart, kPart, &bar_x);
    }

    // ---- set-up: phase-folded gains and taps, the largest gain for the FP16 scale.  With gf
    // (large grid sides) the class grids arrive folded from alias_fold_kernel: no per-antenna
    // tables (the launch does not even allocate them), only the largest gain for the scale.
    const bool lg = gf != nullptr;
    float gmax = 0.f;
    for (int a = simt ? tid : A; a < A; a += kSimt) {
        const short2 k = cells[static_cast<size_t>(c) * A + a];
        if (k.x < hk || k.x >= N - hk || k.y < hk || k.y >= N - hk) atomicOr(status, kStatusDevice);
        const float2 ph = twN[((k.x * hx + k.y * hy) % N + N) % N];
        for (int p = 0; p < P; p++) {
            const float2 g = gains ? gains[(static_cast<size_t>(c) * A + a) * P + p] : make_float2(1.f, 0.f);
            const float2 gg = cmul(g, ph);
            if (!lg) gp[a * P + p] = gg;
            gmax = fmaxf(gmax, sqrtf(gg.x * gg.x + gg.y * gg.y));
        }
    }
    for (int i = simt && !lg ? tid : KK; i < KK; i += kSimt) {
        const int dy = i / K - hk, dx = i % K - hk;
        tapw[i] = cmul(kern[i], twN[((dx * hx + dy * hy) % N + N) % N]);
    }
    for (int i = simt ? tid : 2 * BUF; i < 2 * BUF; i += kSimt) G[i] = make_float2(0.f, 0.f);
    if (simt && t0 < t1 && !lg) {
        const uint32_t *row = reinterpret_cast<const uint32_t *>(v + (static_cast<size_t>(t0) * C + c) * AP);
        for (int w = tid; w < APW; w += kSimt) stage[w] = row[w];
    }
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
        for (int w = 0; w < kSimt / 32; w++) gm = fmaxf(gm, red[w]);
        float wsum = 0.f;
        for (int i = 0; i < KK; i++) {
            const float2 w = lg ? kern[i] : tapw[i];       // the class phases have unit modulus
            wsum += sqrtf(w.x * w.x + w.y * w.y);
        }
        const float bound = 2.f * static_cast<float>(A) * 11.3137085f * gm * wsum;
        int e2 = 0;
        if (bound > 0.f) e2 = static_cast<int>(floorf(log2f(16384.f / bound)));
        scale = ldexpf(1.f, max(-40, min(40, e2)));
    }
    for (int i = simt && !lg ? tid : AP; i < AP; i += kSimt) gp[i] = cscale(gp[i], scale);
    if (simt) {
        // zero this warp's time sums: lanes 32 (w mod 4) .., columns kColAcc + 64 (w / 4) ..
        uint32_t z[32];
#pragma unroll
        for (int j = 0; j < 32; j++) z[j] = 0u;
        const uint32_t acc = lane_addr + kColAcc + 64 * (warp >> 2);
        tc::tmem_st32_issue(acc, z);
        tc::tmem_st32_issue(acc + 32, z);
        tc::tmem_wait_st();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    constexpr uint32_t idesc_row = idesc_kk(128, 128, kBF16);
    constexpr uint32_t idesc_col = idesc_kmn(128, 128, kBF16);
    const uint32_t x_base = tc::smem_u32(opX), h_base = tc::smem_u32(opH);

    if (!simt) {
        // ---- the MMA warp: row stage after bar_g, column stage after bar_h
        if (lane == 0) {
            bool ok = tc::mbar_wait(&bar_x, 0, wait_budget);
            uint32_t ph = 0;
            for (int t = t0; t < t1 && ok; t++, ph ^= 1u) {
                ok = tc::mbar_wait(&bar_g, ph, wait_budget) && !abort_flag;
                if (!ok) break;
                tc::fence_after_sync();
                if (!withhold_mma) {
#pragma unroll
                    for (int kb = 0; kb < 8; kb++) {
                        const uint32_t a_hi = taddr + kColG + kb * 8;
                        const uint64_t x_hi = tc::smem_desc(x_base + kb * 256, kLBO, kSBO);
                        mma_ts(taddr + kColD1, a_hi, x_hi, idesc_row, kb > 0 ? 1u : 0u);
                        if constexpr (kSplit) {
                            const uint64_t x_lo = tc::smem_desc(x_base + kPart + kb * 256, kLBO, kSBO);
                            mma_ts(taddr + kColD1, a_hi, x_lo, idesc_row, 1u);
                            mma_ts(taddr + kColD1, a_hi + 64, x_hi, idesc_row, 1u);
                        }
                    }
                    tc::mma_commit(&bar_m1);
                }
                ok = tc::mbar_wait(&bar_h, ph, wait_budget) && !abort_flag;
                if (!ok) break;
                tc::fence_after_sync();
                if (!withhold_mma) {
#pragma unroll
                    for (int kb = 0; kb < 8; kb++) {
                        const uint64_t x_hi = tc::smem_desc(x_base + kb * 256, kLBO, kSBO);
                        const uint64_t h_hi = tc::smem_desc(h_base + kb * 256, kLBO, kSBO);
                        tc::mma_f16(taddr + kColD2, x_hi, h_hi, idesc_col, kb > 0 ? 1u : 0u);
                        if constexpr (kSplit) {
                            const uint64_t x_lo = tc::smem_desc(x_base + kPart + kb * 256, kLBO, kSBO);
                            const uint64_t h_lo = tc::smem_desc(h_base + kPart + kb * 256, kLBO, kSBO);
                            tc::mma_f16(taddr + kColD2, x_hi, h_lo, idesc_col, 1u);
                            tc::mma_f16(taddr + kColD2, x_lo, h_hi, idesc_col, 1u);
                        }
                    }
                    tc::mma_commit(&bar_m2);
                }
            }
            if (!ok) {
                atomicOr(status, kStatusTimeout);
                abort_flag = 1;
            }
        }
        __syncwarp();
    } else {
        constexpr int kPreW = kMaxAP / 4 / kSimt;
        const int m = 32 * (warp & 3) + lane;          // this thread's TMEM lane / grid row (pol, jy)
        const int hp = warp >> 2;                       // which half of the row's work
        const int part = lane >> 4;
        // a1, a2: unpack and calibrate sample t from the staged bytes
        auto unpack = [&](int t) {
            for (int i = tid; i < AP; i += kSimt) {
                const uint32_t b = reinterpret_cast<const uint8_t *>(stage)[i];
                float2 e = cmul(gp[i], ci4_decode(b));
                if (dtab) e = cmul(e, delay_phase(dtab[static_cast<size_t>(t) * A + i / P], dfreq[c]));
                es[i] = e;
            }
        };
        // a3: scheduled gridding of the unpacked sample into G
        auto grid = [&]() {
            for (int r = 0; r < my_rounds; r++) {
                const uint32_t d = __ldg(my_sched + r * 32 + lane);
                if (d >> 31) {
                    const uint32_t fm = __ldg(my_first + r * 32 + lane);
                    const int a = static_cast<int>(d & 0xFFFu);
                    const int dyi = static_cast<int>((d >> 12) & 0xFu);
                    const int y = static_cast<int>((d >> 16) & 0x3Fu);
                    const int x0 = static_cast<int>((d >> 22) & 0x3Fu);
                    const float2 e0 = es[a * P], e1 = P == 2 ? es[a * P + 1] : make_float2(0.f, 0.f);
                    const float2 e0s = pswap(e0), e1s = pswap(e1);
                    const float2 *wrow = tapw + dyi * K;
                    float2 *gy = G + y * S64;
#pragma unroll
                    for (int dx = 0; dx < (KC > 0 ? KC : K); dx++) {
                        // cell = (first write ? 0 : cell) + w e as two packed FMAs:
                        // w.x (e.x, e.y) + (-w.y, w.y) (e.y, e.x)
                        const float2 w = wrow[dx];
                        const float2 wr = make_float2(w.x, w.x), wi = make_float2(-w.y, w.y);
                        const int x = (x0 + dx) & (M64 - 1);
                        const bool fresh = (fm >> dx) & 1u;
                        const float2 z = make_float2(0.f, 0.f);
                        gy[x] = pfma(wi, e0s, pfma(wr, e0, fresh ? z : gy[x]));
                        if (P == 2) gy[BUF + x] = pfma(wi, e1s, pfma(wr, e1, fresh ? z : gy[BUF + x]));
                    }
                }
                __syncwarp();
            }
        };
        auto load_stage = [&](int t, uint32_t (&pre)[kPreW]) {
            const uint32_t *row = reinterpret_cast<const uint32_t *>(v + (static_cast<size_t>(t) * C + c) * AP);
#pragma unroll
            for (int r = 0; r < kPreW; r++) {
                const int w = tid + r * kSimt;
                pre[r] = (t < t1 && w < APW) ? __ldg(row + w) : 0u;
            }
        };
        auto put_stage = [&](const uint32_t (&pre)[kPreW]) {
#pragma unroll
            for (int r = 0; r < kPreW; r++) {
                const int w = tid + r * kSimt;
                if (w < APW) stage[w] = pre[r];
            }
        };

        // large grid sides: sample t's folded class grid (gf [T][n_items][P][64][64]) into G,
        // scaled like the gridded voltages
        auto load_grid = [&](int t) {
            const float4 *src = reinterpret_cast<const float4 *>(gf + (static_cast<size_t>(t) * n_items + item) * P * 4096);
            for (int i = tid; i < P * 4096 / 2; i += kSimt) {
                const float4 f = __ldg(src + i);
                const int e = 2 * i, pl = e >> 12, y = (e >> 6) & 63, x = e & 63;
                G[pl * BUF + y * S64 + x] = make_float2(f.x * scale, f.y * scale);
                G[pl * BUF + y * S64 + x + 1] = make_float2(f.z * scale, f.w * scale);
            }
        };

        // prologue: sample t0 gridded, the bytes of t0 + 1 staged
        if (t0 < t1) {
            if (lg) {
                load_grid(t0);
            } else {
                unpack(t0);
                tc::named_bar_sync(kBarSimt, kSimt);
                grid();
                uint32_t pre[kPreW];
                load_stage(t0 + 1, pre);
                put_stage(pre);
            }
            tc::named_bar_sync(kBarSimt, kSimt);
        }
        // Iteration t: G(t) -> G16 (row stage of t starts); unpack and grid t+1 while it
        // runs; products of t-1; D1(t) -> H16 (column stage of t starts).
        uint32_t ph = 0;                                // parity of sample t - t0
        for (int t = t0; t <= t1; t++) {
            const bool work = t < t1, nxt = t + 1 < t1;
            // ---- G (FP32) -> G16 in TMEM (row stage A operand).
            // Thread: lane m = (pol, jy); half hp takes jx = 32 hp .. 32 hp + 31.
            if (work) {
                float2 *line = G + (m >> 6) * BUF + (m & 63) * S64 + 32 * hp;
                uint32_t rh[16], ih[16], rl[16], il[16];
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const float2 a = line[2 * j], b = line[2 * j + 1];   // no clearing: see my_first
                    split_pair<kBF16, kSplit>(a.x, b.x, rh[j], rl[j]);
                    split_pair<kBF16, kSplit>(a.y, b.y, ih[j], il[j]);
                }
                // k = 64 part' + jx -> column k / 2: Re words 16 hp .., Im words 32 + 16 hp ..
                tc::tmem_st16_issue(lane_addr + kColG + 16 * hp, rh);
                tc::tmem_st16_issue(lane_addr + kColG + 32 + 16 * hp, ih);
                if constexpr (kSplit) {
                    tc::tmem_st16_issue(lane_addr + kColG + 64 + 16 * hp, rl);
                    tc::tmem_st16_issue(lane_addr + kColG + 96 + 16 * hp, il);
                }
                tc::tmem_wait_st();
                tc::fence_before_sync();
                tc::mbar_arrive(&bar_g);
            }
            tc::named_bar_sync(kBarSimt, kSimt);        // G has been read, es is free

            // ---- sample t+1: unpack and grid (or load its folded grid) while the row stage of t runs
            uint32_t pre[kPreW];
            if (!lg) load_stage(t + 2, pre);
            if (nxt) {
                if (lg) {
                    load_grid(t + 1);
                } else {
                    unpack(t + 1);
                    tc::named_bar_sync(kBarSimt, kSimt);
                    grid();
                }
            }

            // ---- a5, a6: products of sample t-1 (column stage in D2) into the time sums
            if (t > t0 && !abort_flag) {
                if (!tc::mbar_wait(&bar_m2, ph ^ 1u, wait_budget)) {
                    atomicOr(status, kStatusTimeout);
                    abort_flag = 1;
                } else {
                    tc::fence_after_sync();
                    products(lane_addr, hp, part);
                }
            }

            // ---- D1 (row transform H of sample t) -> H16 in shared memory (column stage B operand).
            // Thread: lane m = (pol, jy); half hp takes part hp (Re or Im) of every kx.
            if (work && !abort_flag) {
                if (!tc::mbar_wait(&bar_m1, ph, wait_budget)) {
                    atomicOr(status, kStatusTimeout);
                    abort_flag = 1;
                } else {
                    tc::fence_after_sync();
                    const int pol = m >> 6, jy = m & 63;
                    const int k2 = 64 * hp + jy;
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        // columns r = 32 q + 16 hp + i hold part hp of H at kx = 16 q + i
                        uint32_t d[16];
                        tc::tmem_ld16_issue(lane_addr + kColD1 + 32 * q + 16 * hp, d);
                        tc::tmem_wait_ld();
                        tc::reg_fence16(d);
#pragma unroll
                        for (int half = 0; half < 2; half++) {
                            uint32_t hw[4], lw[4];
#pragma unroll
                            for (int w = 0; w < 4; w++)
                                split_pair<kBF16, kSplit>(__uint_as_float(d[8 * half + 2 * w]),
                                                          __uint_as_float(d[8 * half + 2 * w + 1]), hw[w], lw[w]);
                            const int n0 = 16 * q + 8 * half + 64 * pol;
                            *reinterpret_cast<uint4 *>(opH + mn_off(n0, k2)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                            if constexpr (kSplit)
                                *reinterpret_cast<uint4 *>(opH + kPart + mn_off(n0, k2)) =
                                    make_uint4(lw[0], lw[1], lw[2], lw[3]);
                        }
                    }
                    tc::fence_proxy_async();
                    tc::fence_before_sync();
                    tc::mbar_arrive(&bar_h);
                }
            }
            if (!lg && t + 2 < t1) put_stage(pre);      // bytes of t+2 for the next iteration
            tc::named_bar_sync(kBarSimt, kSimt);
            if (abort_flag) break;
            ph ^= 1u;
        }

        // ---- partial image from the time sums (undo the FP16 scale exactly)
        tc::fence_after_sync();
        const float inv = 1.f / (scale * scale);
        const int my = 16 * (warp & 3) + (lane & 15);
        float4 *dst = reinterpret_cast<float4 *>(partial) + (static_cast<size_t>(tau) * n_items + item) * (M64 * M64);
        uint32_t s0[32], s1[32];
        const uint32_t acc = lane_addr + kColAcc + 64 * hp;
        tc::tmem_ld32_issue(acc, s0);
        tc::tmem_ld32_issue(acc + 32, s1);
        tc::tmem_wait_ld();
        tc::reg_fence32(s0);
        tc::reg_fence32(s1);
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const int mx = 32 * hp + 16 * part + j;
            const uint32_t *a4 = j < 8 ? s0 + 4 * j : s1 + 4 * (j - 8);
            float4 o = make_float4(__uint_as_float(a4[0]) * inv, __uint_as_float(a4[1]) * inv,
                                   __uint_as_float(a4[2]) * inv, __uint_as_float(a4[3]) * inv);
            if (P == 1) {                                  // XX only: one float per pixel
                float *d1 = partial + (static_cast<size_t>(tau) * n_items + item) * (M64 * M64);
                d1[my * M64 + mx] = accumulate ? d1[my * M64 + mx] + o.x : o.x;
                continue;
            }
            if (accumulate) {                              // a later time batch of a large-side group
                const float4 q = dst[my * M64 + mx];
                o = make_float4(q.x + o.x, q.y + o.y, q.z + o.z, q.w + o.w);
            }
            dst[my * M64 + mx] = o;
        }
    }
    // an aborted CTA may still have MMAs in flight: give them a bounded chance to land
    if (tid == kSimt && abort_flag) {
        tc::mbar_wait(&bar_m1, 0, wait_budget);
        tc::mbar_wait(&bar_m1, 1, wait_budget);
        tc::mbar_wait(&bar_m2, 0, wait_budget);
        tc::mbar_wait(&bar_m2, 1, wait_budget);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, 512);
}

size_t dual_smem(int A, int K)
{
    const int AP = A * 2;
    size_t b = 4 * static_cast<size_t>(kPart);
    b += sizeof(float2) * (static_cast<size_t>(2) * M64 * S64 + 2 * AP + K * K);
    b += sizeof(uint32_t) * ((AP + 3) / 4);
    return (b + 15) & ~static_cast<size_t>(15);
}

template <int VAR, int KC>
int launch_dual_t(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau_out,
                  cudaStream_t stream)
{
    int n_tau = choose_tau(plan, g, T);
    if (n_tau > g.tau_cap) n_tau = g.tau_cap;
    *n_tau_out = n_tau;
    const dim3 grid(static_cast<unsigned>(g.n_items * n_tau));
    tc_dual64_kernel<VAR, KC><<<grid, kDualThreads, dual_smem(plan->A, plan->K), stream>>>(
        v, gains, plan->d_cells, plan->d_kernel, plan->K, g.d_chans, g.d_twN, g.d_sched, g.d_nrounds, g.rmax,
        plan->d_dft, plan->A, plan->C, T, g.N, g.Q1, g.n_items, n_tau, g.d_partial, plan->d_status,
        plan->wait_budget, plan->test_withhold_mma, plan->d_dfreq, plan->delays ? plan->d_dtab : nullptr,
        g.d_first, nullptr, 0, plan->P);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

// Large grid sides: one time batch of folded class grids (gf), time sums into
// partial slot 0 (added to it when accumulate is set).  Shared memory: the
// operands and G only.
size_t dual_fold_smem() { return 4 * static_cast<size_t>(kPart) + sizeof(float2) * 2 * M64 * S64; }

template <int VAR, int KC>
int launch_dual_fold_t(epic_plan_s *plan, const GroupCfg &g, const float2 *gains, const float2 *gf, int nb,
                       bool accumulate, cudaStream_t stream)
{
    const dim3 grid(static_cast<unsigned>(g.n_items));
    tc_dual64_kernel<VAR, KC><<<grid, kDualThreads, dual_fold_smem(), stream>>>(
        nullptr, gains, plan->d_cells, plan->d_kernel, plan->K, g.d_chans, g.d_twN, g.d_sched, g.d_nrounds, g.rmax,
        plan->d_dft, plan->A, plan->C, nb, g.N, g.Q1, g.n_items, 1, g.d_partial, plan->d_status,
        plan->wait_budget, plan->test_withhold_mma, plan->d_dfreq, nullptr, g.d_first, gf, accumulate ? 1 : 0, 2);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

template <class F>
int dual_dispatch(int precision, int K, F &&f)
{
    const int var = precision == EPIC_TC_SPLIT_FP16 ? 0 : precision == EPIC_TC_FP16 ? 1 : 2;
    auto with_k = [&](auto vv) {
        switch (K) {
        case 1: return f(vv, std::integral_constant<int, 1>{});
        case 5: return f(vv, std::integral_constant<int, 5>{});
        default: return f(vv, std::integral_constant<int, 0>{});
        }
    };
    switch (var) {
    case 0: return with_k(std::integral_constant<int, 0>{});
    case 1: return with_k(std::integral_constant<int, 1>{});
    default: return with_k(std::integral_constant<int, 2>{});
    }
}

}  // namespace

size_t tc_dual_smem_bytes(int A, int K) { return dual_smem(A, K); }

// The cap is per kernel and process (raise_dyn_smem_cap): a later plan that
// needs less cannot lower it under this one.
int prepare_tc_dual(const epic_plan_s *plan, size_t smem)
{
    return dual_dispatch(plan->precision, plan->K, [&](auto vv, auto kc) {
        return raise_dyn_smem_cap(
            reinterpret_cast<const void *>(tc_dual64_kernel<decltype(vv)::value, decltype(kc)::value>), smem);
    });
}

size_t tc_dual_fold_smem_bytes() { return dual_fold_smem(); }

int launch_tc_dual_fold(epic_plan_s *plan, const GroupCfg &g, const float2 *gains, const float2 *gf, int nb,
                        bool accumulate, cudaStream_t stream)
{
    return dual_dispatch(plan->precision, plan->K, [&](auto vv, auto kc) {
        return launch_dual_fold_t<decltype(vv)::value, decltype(kc)::value>(plan, g, gains, gf, nb, accumulate,
                                                                            stream);
    });
}

int launch_tc_dual(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau,
                   cudaStream_t stream)
{
    return dual_dispatch(plan->precision, plan->K, [&](auto vv, auto kc) {
        return launch_dual_t<decltype(vv)::value, decltype(kc)::value>(plan, g, v, gains, T, n_tau, stream);
    });
}

// The M-point DFT X[r][k] (M = 64, or 48 in the first 48 of the 64 frequencies and inputs, the
// rest zero) in real 2 x 2 block form, hi and lo parts, K-major: row r = 32 q + l -> (my = 16 q
// + l mod 16, part = l / 16), column k = 64 part' + j, X = exp(+2 pi i j my / M) as
// [[cos, -sin], [sin, cos]] over (part, part').  The lo part is what the hi part leaves of the
// FP64 value, rounded once more.
void build_dft_operand(bool bf16, std::vector<uint16_t> &words, int M)
{
    words.assign(2 * kPart / 2, 0);
    auto to16 = [bf16](double x, double &back) -> uint16_t {
        if (bf16) {
            const __nv_bfloat16 h = __float2bfloat16_rn(static_cast<float>(x));
            back = static_cast<double>(__bfloat162float(h));
            return __bfloat16_as_ushort(h);
        }
        const __half h = __float2half_rn(static_cast<float>(x));
        back = static_cast<double>(__half2float(h));
        return __half_as_ushort(h);
    };
    for (int r = 0; r < 128; r++) {
        const int q = r / 32, l = r % 32;
        const int my = 16 * q + (l % 16), part = l / 16;
        for (int k = 0; k < 128; k++) {
            const int j = k % 64;
            const bool im_in = k >= 64;
            // an M-point DFT (M = 64, or 48 in the first 48 rows and columns, the rest zero)
            const long e = (static_cast<long>(j) * my) % M;
            const double th = 2.0 * M_PI * static_cast<double>(e) / M;
            double a;
            if (part == 0) a = im_in ? -std::sin(th) : std::cos(th);
            else a = im_in ? std::cos(th) : std::sin(th);
            if (j >= M || my >= M) a = 0.0;
            double hi_back = 0, lo_back = 0;
            const uint16_t hi = to16(a, hi_back);
            const uint16_t lo = to16(a - hi_back, lo_back);
            words[k_off(r, k) / 2] = hi;
            words[(kPart + k_off(r, k)) / 2] = lo;
        }
    }
}

}  // namespace epic

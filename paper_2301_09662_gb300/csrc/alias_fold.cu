// Large grid sides (N = 8 x 64, 64 pixel classes): gridding once per
// (channel, sample) instead of once per class.
//
// The M = 64 kernels transform, per pixel class h = (hx, hy), the folded grid
//   G_h(m) = sum_j G(m + 64 j) w_N^{(m + 64 j).h}  =  w_N^{m.h} sum_j G(m + 64 j) w_8^{j.h},
// j the alias block of the full N x N grid G (Eq. 4's gridded aperture).  At
// N = 512 re-gridding every footprint for each of the 64 classes dominates the
// run.  alias_fold_kernel grids the calibrated voltages once into the occupied
// alias blocks (the aperture spans at most half of each axis, so at most 4 x 4
// of the 8 x 8 blocks), then forms all 64 folded grids with one 8 x 8 DFT over
// the alias index per folded cell (factored: 4 rows of 8-point DFTs over jx,
// then 8 columns over jy) and the class phase w_N^{m.h}.  fp32_fold64_kernel
// (or, for a tensor plan, tc_dual64_kernel in its folded-grid mode) then loads
// each class's grid and transforms it.
//
// Block = (8-row band of the folded grid, channel, sample x polarisation); warp
// w owns folded row 8 band + w, so the alias buffers are written without
// atomics and in a fixed order (deterministic): its footprint rows (plan list,
// a << 8 | dyi) are taken 32 at a time, each lane calibrating one, then applied
// one after another with lane dx adding tap dx.
#include <algorithm>
#include <utility>
#include <vector>

#include "dft_small.cuh"
#include "epic_internal.cuh"

namespace epic {
namespace {

constexpr int kAliasThreads = 256;   // 8 warps = 8 folded rows of a band
constexpr int kNJ = 4;               // occupied alias blocks per axis
constexpr int kCS = kNJ * kNJ + 1;   // float2 per folded cell in shared memory (odd: no bank conflicts)

// exp(+2 pi i k / 8); indexed with warp-uniform k (alias block x class), a broadcast read
__constant__ float2 c_w8[8] = {{1.f, 0.f},   {kSqrtHalf, kSqrtHalf},   {0.f, 1.f},  {-kSqrtHalf, kSqrtHalf},
                               {-1.f, 0.f},  {-kSqrtHalf, -kSqrtHalf}, {0.f, -1.f}, {kSqrtHalf, -kSqrtHalf}};

// s += a w8^K with K known at compile time: +-1 and +-i are adds, the odd
// powers (+-1 +-i) sqrt(1/2) two FMAs per component
template <int K>
__device__ __forceinline__ void cmac8(float2 &s, float2 a)
{
    constexpr int k = K & 7;
    if constexpr (k == 0) {
        s.x += a.x;
        s.y += a.y;
    } else if constexpr (k == 2) {
        s.x -= a.y;
        s.y += a.x;
    } else if constexpr (k == 4) {
        s.x -= a.x;
        s.y -= a.y;
    } else if constexpr (k == 6) {
        s.x += a.y;
        s.y -= a.x;
    } else {
        constexpr float c = (k == 1 || k == 7) ? kSqrtHalf : -kSqrtHalf;
        constexpr float d = (k == 1 || k == 3) ? kSqrtHalf : -kSqrtHalf;
        s.x = fmaf(a.x, c, fmaf(-a.y, d, s.x));
        s.y = fmaf(a.x, d, fmaf(a.y, c, s.y));
    }
}

template <class F, int... I>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F &&f)
{
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

__global__ void __launch_bounds__(kAliasThreads)
alias_fold_kernel(const uint8_t *__restrict__ v, const float2 *__restrict__ gains, const short2 *__restrict__ cells,
                  const float2 *__restrict__ kern, int K, const int *__restrict__ chans,
                  const short2 *__restrict__ j0tab, const uint32_t *__restrict__ bseg, const int *__restrict__ boff,
                  const float2 *__restrict__ twN, int A, int C, int P, int N, int n_items, int tb0,
                  const float *__restrict__ dfreq, const float4 *__restrict__ dtab, float2 *__restrict__ gf)
{
    extern __shared__ float2 al[];                 // [8 rows][64 x][kCS: kNJ * kNJ aliases + pad], then taps [K][K]
    float2 *tap = al + 8 * 64 * kCS;
    const int band = blockIdx.x, ci = blockIdx.y, bt = blockIdx.z / P, p = blockIdx.z % P;
    const int t = tb0 + bt, c = chans[ci];
    const int tid = threadIdx.x, lane = tid & 31, row = tid >> 5;
    const int h = (K - 1) / 2;
    const short2 j0 = j0tab[ci];
    for (int i = tid; i < 8 * 64 * kCS; i += kAliasThreads) al[i] = make_float2(0.f, 0.f);
    for (int i = tid; i < K * K; i += kAliasThreads) tap[i] = kern[i];
    __syncthreads();

    // ---- grid this warp's folded row my = 8 band + row into its alias blocks
    const int my = 8 * band + row;
    const int s0 = boff[ci * 64 + my], s1 = boff[ci * 64 + my + 1];
    float2 *arow = al + row * 64 * kCS;
    for (int sb = s0; sb < s1; sb += 32) {
        const int n = min(32, s1 - sb);
        int a = 0, dyi = 0, cx = 0, iy = 0;
        float2 e = make_float2(0.f, 0.f);
        if (lane < n) {                            // lane l calibrates footprint row sb + l
            const uint32_t seg = bseg[sb + lane];
            a = static_cast<int>(seg >> 8);
            dyi = static_cast<int>(seg & 255u);
            const short2 k = cells[static_cast<size_t>(c) * A + a];
            cx = k.x;
            iy = ((k.y + dyi - h) >> 6) - j0.y;
            e = ci4_decode(v[((static_cast<size_t>(t) * C + c) * A + a) * P + p]);
            if (gains) e = cmul(gains[(static_cast<size_t>(c) * A + a) * P + p], e);
            if (dtab) e = cmul(e, delay_phase(dtab[static_cast<size_t>(t) * A + a], dfreq[c]));
        }
        for (int i = 0; i < n; i++) {
            const float ex = __shfl_sync(0xffffffffu, e.x, i), ey = __shfl_sync(0xffffffffu, e.y, i);
            const int di = __shfl_sync(0xffffffffu, dyi, i), kx0 = __shfl_sync(0xffffffffu, cx, i) - h;
            const int ay = __shfl_sync(0xffffffffu, iy, i);
            if (lane < K) {                        // distinct cells within one footprint row
                const int kx = kx0 + lane;
                const float2 w = cmul(tap[di * K + lane], make_float2(ex, ey));
                float2 *cell = arow + (kx & 63) * kCS + ay * kNJ + ((kx >> 6) - j0.x);
                const float2 o = *cell;
                *cell = make_float2(o.x + w.x, o.y + w.y);
            }
            __syncwarp();
        }
    }
    __syncthreads();

    // ---- fold: per folded cell (my, mx), the kNJ x kNJ aliases -> 8 x 8 class values.
    // w_N^{m.h} w8^{(j0 + i).h} = fx(hx) fy(hy) w8^{i.h}: the alias offset j0 and the class
    // phase go into per-cell factors fx, fy, the remaining 4-input 8-point DFTs have
    // compile-time roots
    for (int cl = tid; cl < 8 * 64; cl += kAliasThreads) {
        const int r = cl >> 6, mx = cl & 63, mfy = 8 * band + r;
        const float2 *src = al + cl * kCS;
        float2 fx[8], fy[8];
#pragma unroll
        for (int hh = 0; hh < 8; hh++) {
            fx[hh] = cmul(c_w8[(j0.x * hh) & 7], twN[(mx * hh) % N]);
            fy[hh] = cmul(c_w8[(j0.y * hh) & 7], twN[(mfy * hh) % N]);
        }
        float2 B[kNJ][8];                          // B[iy][hx] = fx(hx) sum_ix A[iy][ix] w8^{ix hx}
        static_for<kNJ>([&](auto iy) {
            float2 av[kNJ];
#pragma unroll
            for (int ix = 0; ix < kNJ; ix++) av[ix] = src[iy.value * kNJ + ix];
            static_for<8>([&](auto hx) {
                float2 acc2 = make_float2(0.f, 0.f);
                static_for<kNJ>([&](auto ix) { cmac8<ix.value * hx.value>(acc2, av[ix.value]); });
                B[iy.value][hx.value] = cmul(acc2, fx[hx.value]);
            });
        });
        float2 *out = gf + (static_cast<size_t>(bt) * n_items + ci * 64) * P * 4096 + p * 4096 + mfy * 64 + mx;
        static_for<8>([&](auto hy) {
            static_for<8>([&](auto hx) {
                float2 acc2 = make_float2(0.f, 0.f);
                static_for<kNJ>([&](auto iy) { cmac8<iy.value * hy.value>(acc2, B[iy.value][hx.value]); });
                out[static_cast<size_t>(hy.value * 8 + hx.value) * P * 4096] = cmul(acc2, fy[hy.value]);
            });
        });
    }
}

size_t alias_smem(int K) { return sizeof(float2) * (8 * 64 * kCS + static_cast<size_t>(K) * K); }

}  // namespace

// Host tables: per channel the first occupied alias block of each axis (the
// footprints must span at most kNJ blocks, else EPIC_ERR_UNSUPPORTED and the
// plan keeps the per-class gridding) and, per (channel, folded row), the
// footprint rows landing on it.
int build_alias_tables(const std::vector<short2> &cells, int A, int K, int N, const std::vector<int> &chans,
                       std::vector<short2> &j0, std::vector<uint32_t> &bseg, std::vector<int> &boff)
{
    const int h = (K - 1) / 2;
    if (N != 8 * 64 || A >= (1 << 24) || K > 255) return EPIC_ERR_UNSUPPORTED;
    const int nc = static_cast<int>(chans.size());
    j0.assign(nc, make_short2(0, 0));
    std::vector<std::vector<uint32_t>> rows(static_cast<size_t>(nc) * 64);
    for (int ci = 0; ci < nc; ci++) {
        const int c = chans[ci];
        int jx0 = 1 << 20, jx1 = -1, jy0 = 1 << 20, jy1 = -1;
        for (int a = 0; a < A; a++) {
            const short2 k = cells[static_cast<size_t>(c) * A + a];
            jx0 = std::min(jx0, (k.x - h) >> 6);
            jx1 = std::max(jx1, (k.x + h) >> 6);
            jy0 = std::min(jy0, (k.y - h) >> 6);
            jy1 = std::max(jy1, (k.y + h) >> 6);
            for (int dyi = 0; dyi < K; dyi++)
                rows[static_cast<size_t>(ci) * 64 + ((k.y + dyi - h) & 63)].push_back(
                    (static_cast<uint32_t>(a) << 8) | static_cast<uint32_t>(dyi));
        }
        if (jx1 - jx0 >= kNJ || jy1 - jy0 >= kNJ) return EPIC_ERR_UNSUPPORTED;
        j0[ci] = make_short2(static_cast<short>(jx0), static_cast<short>(jy0));
    }
    bseg.clear();
    boff.assign(static_cast<size_t>(nc) * 64 + 1, 0);
    for (size_t i = 0; i < rows.size(); i++) {
        boff[i] = static_cast<int>(bseg.size());
        bseg.insert(bseg.end(), rows[i].begin(), rows[i].end());
    }
    boff[rows.size()] = static_cast<int>(bseg.size());
    return EPIC_OK;
}

// The cap is per kernel and process, and this plan's size depends on K
// (raise_dyn_smem_cap: a later plan with a smaller K cannot lower it).
int prepare_alias(const epic_plan_s *plan)
{
    const int rc = raise_dyn_smem_cap(reinterpret_cast<const void *>(alias_fold_kernel), alias_smem(plan->K));
    return rc != EPIC_OK ? rc : prepare_fold64(plan->P);
}

// One integration: per batch of alias_tb samples, fold every class of every
// channel, then transform and sum the batch into partial slot 0.
int launch_alias(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau,
                 cudaStream_t stream)
{
    *n_tau = 1;
    const size_t smem = alias_smem(plan->K);
    for (int tb0 = 0; tb0 < T; tb0 += g.alias_tb) {
        const int nb = std::min(g.alias_tb, T - tb0);
        const dim3 grid(8, static_cast<unsigned>(g.n_chan), static_cast<unsigned>(nb * plan->P));
        alias_fold_kernel<<<grid, kAliasThreads, smem, stream>>>(
            v, gains, plan->d_cells, plan->d_kernel, plan->K, g.d_chans, g.d_j0, g.d_bseg, g.d_boff, g.d_twN,
            plan->A, plan->C, plan->P, g.N, g.n_items, tb0, plan->d_dfreq, plan->delays ? plan->d_dtab : nullptr,
            g.d_gf);
        if (cudaGetLastError() != cudaSuccess) return EPIC_ERR_CUDA;
        const int rc = g.tensor ? launch_tc_dual_fold(plan, g, gains, g.d_gf, nb, tb0 > 0, stream)
                                : launch_fold64(g, plan->P, g.d_gf, nb, tb0 > 0, stream);
        if (rc != EPIC_OK) return rc;
    }
    return EPIC_OK;
}

}  // namespace epic

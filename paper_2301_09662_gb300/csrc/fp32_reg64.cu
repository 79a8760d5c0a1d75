// FP32 form, folded side M = 64 or 48: the imaging kernel used for grid sides
// 64, 128, 256, 512 (M = 64) and 96 (M = 48), one pixel class of one channel
// per CTA, as in fp32_image.cu (see the derivation there).
//
// What differs from the general kernel, and why (measured: the general kernel
// is bound by the shared-memory pipe, ~17 000 wavefronts per CTA and sample):
//  * gridding without atomics: the plan splits every antenna footprint into K
//    row segments and packs them into rounds of 32 lanes in which no two
//    segments touch the same cell and no two lanes of a half-warp hit the same
//    bank; warp w owns the grid rows y = w (mod 8), so a round is a plain
//    read-add-write of K cells per lane with no inter-warp race;
//  * the M-point transforms run in registers (one row or column per thread),
//    so each axis costs one shared-memory read and one write;
//  * two time samples per iteration share the schedule, the twiddles and the
//    synchronisation;
//  * the transforms and the gridding multiply-adds run on packed FP32 pairs
//    (add/sub/mul/fma .f32x2: one instruction for both lanes of a float2).
#include <type_traits>

#include "epic_internal.cuh"
#include "fft48.cuh"
#include "fft64.cuh"

namespace epic {
namespace {

constexpr int M64 = 64;
constexpr int S64 = 65;                       // padded row stride (float2)

template <int P>
struct Acc64;
template <> struct Acc64<1> { using T = float; };
template <> struct Acc64<2> { using T = float4; };

constexpr int NPOS64 = M64 * M64 / kThreads;   // pixels whose time sums a thread keeps

// Register transforms of the folded side M: 64 points (8 x 8) or 48 (8 x 6, grid side 96).
template <int M, class Sink>
__device__ __forceinline__ void fft_reg(float2 (&x)[M], Sink &&sink)
{
    static_assert(M == 64 || M == 48, "folded sides 64 and 48");
    if constexpr (M == 64) {
        fft64p_stage1(x);
        fft64p_stage2(x, sink);
    } else {
        fft48p_stage1(x);
        fft48p_stage2(x, sink);
    }
}

// a4-a6 on the TS x P planes of G ([ts][p][y][x], x < M at stride M + 1): rows
// then columns, one M-point transform per thread, then the products of every
// pixel added to the thread's time sums; CLEAR zeroes the planes for the next
// gridding.  Rows outside rows_used are empty and stay zero.
template <int M, int P, int TS, bool CLEAR>
__device__ __forceinline__ void transform_products(float2 *G, unsigned long long rows_used,
                                                   typename Acc64<P>::T (&acc)[M * M / kThreads], int tid)
{
    constexpr int S = M + 1, BUF = M * S, NPOS = M * M / kThreads;
    for (int q = tid; q < TS * P * M; q += kThreads) {
        if (!((rows_used >> (q % M)) & 1ull)) continue;   // empty row: stays zero
        float2 *line = G + (q / M) * BUF + (q % M) * S;
        float2 x[M];
#pragma unroll
        for (int i = 0; i < M; i++) x[i] = line[i];
        fft_reg<M>(x, [&](int k, float2 val) { line[k] = val; });
    }
    __syncthreads();
    for (int q = tid; q < TS * P * M; q += kThreads) {
        float2 *col = G + (q / M) * BUF + (q % M);
        float2 x[M];
#pragma unroll
        for (int i = 0; i < M; i++) x[i] = col[i * S];
        fft_reg<M>(x, [&](int k, float2 val) { col[k * S] = val; });
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < NPOS; r++) {
        const int pos = tid + r * kThreads;
        int idx;
        if constexpr (M == 64) idx = (pos >> 6) * S64 + (pos & 63);
        else idx = (pos / M) * S + (pos % M);
#pragma unroll
        for (int ts = 0; ts < TS; ts++) {
            const float2 f0 = G[(ts * P) * BUF + idx];
            if constexpr (CLEAR) G[(ts * P) * BUF + idx] = make_float2(0.f, 0.f);
            if constexpr (P == 2) {
                const float2 f1 = G[(ts * P + 1) * BUF + idx];
                if constexpr (CLEAR) G[(ts * P + 1) * BUF + idx] = make_float2(0.f, 0.f);
                acc[r].x = fmaf(f0.x, f0.x, fmaf(f0.y, f0.y, acc[r].x));
                acc[r].y = fmaf(f1.x, f1.x, fmaf(f1.y, f1.y, acc[r].y));
                acc[r].z = fmaf(f0.x, f1.x, fmaf(f0.y, f1.y, acc[r].z));
                acc[r].w = fmaf(f0.y, f1.x, fmaf(-f0.x, f1.y, acc[r].w));
            } else {
                acc[r] = fmaf(f0.x, f0.x, fmaf(f0.y, f0.y, acc[r]));
            }
        }
    }
}

// Folded side M (64, or 48 for grid side 96).  Grid buffers: G[ts][p][y][x] with
// x < M at stride M + 1.  KC > 0 fixes the
// kernel side at compile time (the gridding loop then unrolls fully); KC = 0
// takes it from K.  DL: voltages take the geometric-delay phase of the
// per-integration table dtab (Sec. 2.2 delay correction), once per antenna.  rowmask[ci] marks the folded rows any footprint touches:
// the others stay zero and their row transforms are skipped.
template <int M, int P, int TS, int KC, bool DL>
__global__ void __launch_bounds__(kThreads, 1)
fp32_reg64_kernel(const uint8_t *__restrict__ v, const float2 *__restrict__ gains,
                  const short2 *__restrict__ cells, const float2 *__restrict__ kern, int K_rt,
                  const int *__restrict__ chans, const float2 *__restrict__ twN,
                  const uint32_t *__restrict__ sched, const int *__restrict__ nrounds, int rmax,
                  const unsigned long long *__restrict__ rowmask,
                  int A, int C, int T, int N, int Q1, int n_items, int n_tau,
                  float *__restrict__ partial, int *__restrict__ status, int nker,
                  const float *__restrict__ dfreq, const float4 *__restrict__ dtab)
{
    const int K = KC > 0 ? KC : K_rt;
    constexpr int NPOS = M * M / kThreads;       // pixels per thread (16 at M = 64, 9 at 48)
    constexpr int S = M + 1;                     // padded row stride (float2)
    constexpr int BUF = M * S;                   // one [y][x] plane
    extern __shared__ float4 smem_raw[];
    const int AP = A * P, KK = K * K, hk = (K - 1) / 2;
    const int APW = (AP + 3) >> 2;
    float2 *G = reinterpret_cast<float2 *>(smem_raw);          // [TS][P][M][M + 1]
    float2 *es = G + TS * P * BUF;                             // [TS][A*P]
    float2 *gp = es + TS * AP;                                 // [A*P]
    float2 *tapw = gp + AP;                                    // [nker][K*K]
    uint32_t *stage = reinterpret_cast<uint32_t *>(tapw + nker * KK); // [TS][APW]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int item = blockIdx.x % n_items;
    const int tau = blockIdx.x / n_items;
    const int Q = Q1 * Q1;
    const int ci = item / Q, h = item % Q, hx = h % Q1, hy = h / Q1;
    const int c = chans[ci];
    const int t0 = static_cast<int>(static_cast<long long>(T) * tau / n_tau);
    const int t1 = static_cast<int>(static_cast<long long>(T) * (tau + 1) / n_tau);
    const uint32_t *my_sched = sched + (static_cast<size_t>(ci) * 8 + warp) * rmax * 32;
    const int my_rounds = nrounds[ci * 8 + warp];
    const unsigned long long rows_used = rowmask[ci];

    // ---- set-up: phase-folded gains and taps (class phase w_N^{k.h})
    for (int a = tid; a < A; a += kThreads) {
        const short2 k = cells[static_cast<size_t>(c) * A + a];
        if (k.x < hk || k.x >= N - hk || k.y < hk || k.y >= N - hk) atomicOr(status, kStatusDevice);
        const float2 ph = twN[((k.x * hx + k.y * hy) % N + N) % N];
        for (int p = 0; p < P; p++) {
            const float2 g = gains ? gains[(static_cast<size_t>(c) * A + a) * P + p] : make_float2(1.f, 0.f);
            gp[a * P + p] = cmul(g, ph);
        }
    }
    for (int i = tid; i < nker * KK; i += kThreads) {
        const int tap = i % KK;
        const int dy = tap / K - hk, dx = tap % K - hk;
        tapw[i] = cmul(kern[i], twN[((dx * hx + dy * hy) % N + N) % N]);
    }
    for (int i = tid; i < TS * P * BUF; i += kThreads) G[i] = make_float2(0.f, 0.f);
    for (int ts = 0; ts < TS; ts++) {
        if (t0 + ts < t1) {
            const uint32_t *row = reinterpret_cast<const uint32_t *>(v + (static_cast<size_t>(t0 + ts) * C + c) * AP);
            for (int w = tid; w < APW; w += kThreads) stage[ts * APW + w] = row[w];
        }
    }

    typename Acc64<P>::T acc[NPOS];
#pragma unroll
    for (int r = 0; r < NPOS; r++) {
        if constexpr (P == 2) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        else acc[r] = 0.f;
    }
    __syncthreads();

    constexpr int kPreW = kMaxAP / 4 / kThreads;
    for (int t = t0; t < t1; t += TS) {
        // ---- a1, a2: unpack and calibrate TS samples (an absent sample grids zeros)
#pragma unroll
        for (int ts = 0; ts < TS; ts++) {
            const bool ok = t + ts < t1;
            if constexpr (DL) {
                // delay phase once per antenna, shared by its polarisations
                for (int a = tid; a < A; a += kThreads) {
                    const float2 ph = ok ? delay_phase(dtab[static_cast<size_t>(t + ts) * A + a], dfreq[c])
                                         : make_float2(0.f, 0.f);
#pragma unroll
                    for (int p = 0; p < P; p++) {
                        const int i = a * P + p;
                        const uint32_t b = reinterpret_cast<const uint8_t *>(stage + ts * APW)[i];
                        es[ts * AP + i] = cmul(cmul(gp[i], ci4_decode(b)), ph);
                    }
                }
            } else {
                for (int i = tid; i < AP; i += kThreads) {
                    const uint32_t b = reinterpret_cast<const uint8_t *>(stage + ts * APW)[i];
                    es[ts * AP + i] = ok ? cmul(gp[i], ci4_decode(b)) : make_float2(0.f, 0.f);
                }
            }
        }
        // prefetch the next TS samples while this group is gridded and transformed
        uint32_t pre[TS][kPreW];
#pragma unroll
        for (int ts = 0; ts < TS; ts++) {
            const int tn = t + TS + ts;
            const uint32_t *row = reinterpret_cast<const uint32_t *>(v + (static_cast<size_t>(tn) * C + c) * AP);
#pragma unroll
            for (int r = 0; r < kPreW; r++) {
                const int w = tid + r * kThreads;
                pre[ts][r] = (tn < t1 && w < APW) ? __ldg(row + w) : 0u;
            }
        }
        __syncthreads();

        // ---- a3: scheduled gridding, warp w owns rows y = w (mod 8)
        for (int r = 0; r < my_rounds; r++) {
            const uint32_t d = __ldg(my_sched + r * 32 + lane);
            if (d >> 31) {
                const int a = static_cast<int>(d & 0xFFFu);
                const int dyi = static_cast<int>((d >> 12) & 0xFu);
                const int y = static_cast<int>((d >> 16) & 0x3Fu);
                const int x0 = static_cast<int>((d >> 22) & 0x3Fu);
                float2 e[TS][P], eswap[TS][P];
#pragma unroll
                for (int ts = 0; ts < TS; ts++)
#pragma unroll
                    for (int p = 0; p < P; p++) {
                        e[ts][p] = es[ts * AP + a * P + p];
                        eswap[ts][p] = pswap(e[ts][p]);
                    }
                const float2 *wrow = tapw + (nker > 1 ? a * KK : 0) + dyi * K;
#pragma unroll
                for (int dx = 0; dx < (KC > 0 ? KC : K); dx++) {
                    // cell += w e as two packed FMAs: w.x (e.x, e.y) + (-w.y, w.y) (e.y, e.x)
                    const float2 w = wrow[dx];
                    const float2 wr = make_float2(w.x, w.x), wi = make_float2(-w.y, w.y);
                    int x;
                    if constexpr (M == 64) x = (x0 + dx) & (M64 - 1);
                    else x = x0 + dx >= M ? x0 + dx - M : x0 + dx;   // x0 < M, dx < K <= 15
#pragma unroll
                    for (int ts = 0; ts < TS; ts++)
#pragma unroll
                        for (int p = 0; p < P; p++) {
                            float2 *cell = G + (ts * P + p) * BUF + y * S + x;
                            *cell = pfma(wi, eswap[ts][p], pfma(wr, e[ts][p], *cell));
                        }
                }
            }
            __syncwarp();
        }
        __syncthreads();

        // ---- a4, a5, a6: transforms, products summed over time; planes cleared for the next group
        transform_products<M, P, TS, true>(G, rows_used, acc, tid);
#pragma unroll
        for (int ts = 0; ts < TS; ts++)
#pragma unroll
            for (int r = 0; r < kPreW; r++) {
                const int w = tid + r * kThreads;
                if (w < APW) stage[ts * APW + w] = pre[ts][r];
            }
        __syncthreads();
    }

    float *dst = partial + (static_cast<size_t>(tau) * n_items + item) * (M * M) * (P == 2 ? 4 : 1);
#pragma unroll
    for (int r = 0; r < NPOS; r++) {
        const int pos = tid + r * kThreads;
        if constexpr (P == 2) reinterpret_cast<float4 *>(dst)[pos] = acc[r];
        else dst[pos] = acc[r];
    }
}

// Large grid sides: the folded grids of every pixel class were formed once per
// (channel, sample) by alias_fold_kernel; this kernel loads its class's grid
// for each sample of a time batch instead of gridding, then transforms and
// sums products like fp32_reg64_kernel.  Two grid buffers: the next sample's
// grid streams in (cp.async) while the current one is transformed.  gf is
// [nb][n_items][P][64][64]; the time sums go to partial slot 0, added to what
// is there when accumulate is set (batches of one integration follow each other
// on the stream).
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

template <int P>
__global__ void __launch_bounds__(kThreads, 1)
fp32_fold64_kernel(const float2 *__restrict__ gf, int nb, int accumulate, float *__restrict__ partial)
{
    constexpr int BUF = M64 * S64;
    extern __shared__ float4 smem_raw[];
    float2 *Gb = reinterpret_cast<float2 *>(smem_raw);         // two x [P][64][65]
    const int item = blockIdx.x, n_items = gridDim.x, tid = threadIdx.x;
    float *dst = partial + static_cast<size_t>(item) * (M64 * M64) * (P == 2 ? 4 : 1);
    typename Acc64<P>::T acc[NPOS64];
#pragma unroll
    for (int r = 0; r < NPOS64; r++) {
        const int pos = tid + r * kThreads;
        if constexpr (P == 2) acc[r] = accumulate ? reinterpret_cast<const float4 *>(dst)[pos] : make_float4(0.f, 0.f, 0.f, 0.f);
        else acc[r] = accumulate ? dst[pos] : 0.f;
    }
    auto issue = [&](int bt) {                       // sample bt of the batch into buffer bt mod 2
        if (bt < nb) {
            const float2 *src = gf + (static_cast<size_t>(bt) * n_items + item) * P * (M64 * M64);
            float2 *G = Gb + (bt & 1) * P * BUF;
            for (int i = tid; i < P * M64 * M64; i += kThreads)
                cp_async8(G + (i >> 12) * BUF + ((i >> 6) & 63) * S64 + (i & 63), src + i);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    issue(0);
    for (int bt = 0; bt < nb; bt++) {
        issue(bt + 1);
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // sample bt has landed (this thread's part)
        __syncthreads();
        transform_products<64, P, 1, false>(Gb + (bt & 1) * P * BUF, ~0ull, acc, tid);
        __syncthreads();                             // buffer bt mod 2 is refilled two samples on
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
#pragma unroll
    for (int r = 0; r < NPOS64; r++) {
        const int pos = tid + r * kThreads;
        if constexpr (P == 2) reinterpret_cast<float4 *>(dst)[pos] = acc[r];
        else dst[pos] = acc[r];
    }
}

template <int M, int P, int TS>
size_t reg64_smem(int A, int K, int nker)
{
    const int AP = A * P;
    size_t b = sizeof(float2) * (static_cast<size_t>(TS) * P * M * (M + 1) + static_cast<size_t>(TS) * AP + AP +
                                 static_cast<size_t>(nker) * K * K);
    b += sizeof(uint32_t) * TS * ((AP + 3) / 4);
    return (b + 15) & ~static_cast<size_t>(15);
}

template <int M, int P, int TS, int KC, bool DL>
int launch_reg64_t(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau_out,
                   cudaStream_t stream)
{
    auto kfn = fp32_reg64_kernel<M, P, TS, KC, DL>;
    const size_t smem = reg64_smem<M, P, TS>(plan->A, plan->K, plan->nker);
    int n_tau = choose_tau(plan, g, T);
    if (n_tau > g.tau_cap) n_tau = g.tau_cap;
    *n_tau_out = n_tau;
    const dim3 grid(static_cast<unsigned>(g.n_items * n_tau));
    kfn<<<grid, kThreads, smem, stream>>>(v, gains, plan->d_cells, plan->d_kernel, plan->K, g.d_chans, g.d_twN,
                                          g.d_sched, g.d_nrounds, g.rmax, g.d_rowmask, plan->A, plan->C, T, g.N, g.Q1,
                                          g.n_items, n_tau, g.d_partial, plan->d_status, plan->nker, plan->d_dfreq,
                                          DL ? plan->d_dtab : nullptr);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

template <int M, int P, int TS, int KC>
int prepare_reg64_t(const epic_plan_s *plan)
{
    const int smem = static_cast<int>(reg64_smem<M, P, TS>(plan->A, plan->K, plan->nker));
    const bool ok = cudaFuncSetAttribute(fp32_reg64_kernel<M, P, TS, KC, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess &&
                    cudaFuncSetAttribute(fp32_reg64_kernel<M, P, TS, KC, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess;
    return ok ? EPIC_OK : EPIC_ERR_UNSUPPORTED;
}

// Which instantiation serves a plan: at M = 64 dual polarisation gets kernels
// specialised for the kernel sides in use here (1: image-domain taper, 5:
// LWA-like, 7: dense), at M = 48 (grid side 96) for side 5; anything else runs
// the generic loop.
struct Reg64Key {
    int M, P, TS, KC;
};

Reg64Key reg64_key(const epic_plan_s *plan, const GroupCfg &g)
{
    int kc = 0;
    if (plan->P == 2 && (plan->K == 5 || (g.M == 64 && (plan->K == 1 || plan->K == 7)))) kc = plan->K;
    return {g.M, plan->P, g.ts, kc};
}

template <int V>
using IC = std::integral_constant<int, V>;

template <int M, class F>
int reg64_dispatch_m(const Reg64Key &k, F &&f)
{
    if (k.P == 2) {
        auto with_ts = [&](auto ts) {
            switch (k.KC) {
            case 5: return f(IC<M>{}, IC<2>{}, ts, IC<5>{});
            case 1:
                if constexpr (M == 64) return f(IC<M>{}, IC<2>{}, ts, IC<1>{});
                else return f(IC<M>{}, IC<2>{}, ts, IC<0>{});
            case 7:
                if constexpr (M == 64) return f(IC<M>{}, IC<2>{}, ts, IC<7>{});
                else return f(IC<M>{}, IC<2>{}, ts, IC<0>{});
            default: return f(IC<M>{}, IC<2>{}, ts, IC<0>{});
            }
        };
        return k.TS == 2 ? with_ts(IC<2>{}) : with_ts(IC<1>{});
    }
    return k.TS == 2 ? f(IC<M>{}, IC<1>{}, IC<2>{}, IC<0>{}) : f(IC<M>{}, IC<1>{}, IC<1>{}, IC<0>{});
}

template <class F>
int reg64_dispatch(const Reg64Key &k, F &&f)
{
    return k.M == 48 ? reg64_dispatch_m<48>(k, f) : reg64_dispatch_m<64>(k, f);
}

}  // namespace

int prepare_reg64(const epic_plan_s *plan, const GroupCfg &g)
{
    return reg64_dispatch(reg64_key(plan, g), [&](auto m_, auto p_, auto ts_, auto kc_) {
        return prepare_reg64_t<decltype(m_)::value, decltype(p_)::value, decltype(ts_)::value,
                               decltype(kc_)::value>(plan);
    });
}

size_t reg64_smem_bytes(int M, int P, int TS, int A, int K, int nker)
{
    if (M == 48) {
        if (P == 2) return TS == 2 ? reg64_smem<48, 2, 2>(A, K, nker) : reg64_smem<48, 2, 1>(A, K, nker);
        return TS == 2 ? reg64_smem<48, 1, 2>(A, K, nker) : reg64_smem<48, 1, 1>(A, K, nker);
    }
    if (P == 2) return TS == 2 ? reg64_smem<64, 2, 2>(A, K, nker) : reg64_smem<64, 2, 1>(A, K, nker);
    return TS == 2 ? reg64_smem<64, 1, 2>(A, K, nker) : reg64_smem<64, 1, 1>(A, K, nker);
}

size_t fold64_smem_bytes(int P) { return 2 * sizeof(float2) * static_cast<size_t>(P) * M64 * S64; }

int prepare_fold64(int P)
{
    const int smem = static_cast<int>(fold64_smem_bytes(P));
    const cudaError_t e = P == 2 ? cudaFuncSetAttribute(fp32_fold64_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                                 : cudaFuncSetAttribute(fp32_fold64_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e == cudaSuccess ? EPIC_OK : EPIC_ERR_UNSUPPORTED;
}

int launch_fold64(const GroupCfg &g, int P, const float2 *gf, int nb, bool accumulate, cudaStream_t stream)
{
    const size_t smem = fold64_smem_bytes(P);
    const dim3 grid(static_cast<unsigned>(g.n_items));
    if (P == 2) fp32_fold64_kernel<2><<<grid, kThreads, smem, stream>>>(gf, nb, accumulate ? 1 : 0, g.d_partial);
    else fp32_fold64_kernel<1><<<grid, kThreads, smem, stream>>>(gf, nb, accumulate ? 1 : 0, g.d_partial);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

int launch_reg64(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau,
                 cudaStream_t stream)
{
    return reg64_dispatch(reg64_key(plan, g), [&](auto m_, auto p_, auto ts_, auto kc_) {
        constexpr int M = decltype(m_)::value, P = decltype(p_)::value, TS = decltype(ts_)::value,
                      KC = decltype(kc_)::value;
        // the delay-corrected form is a separate instantiation, so the plain one carries no trace of it
        return plan->delays ? launch_reg64_t<M, P, TS, KC, true>(plan, g, v, gains, T, n_tau, stream)
                            : launch_reg64_t<M, P, TS, KC, false>(plan, g, v, gains, T, n_tau, stream);
    });
}

}  // namespace epic

// FP32 form, folded side M = 64 or 48: the imaging kernel used for grid sides
// 64, 128, 256, 512 (M = 64) and 96 (M = 48), one pixel class of one channel
// per CTA, as in fp32_image.cu (see the derivation there).
//
// What differs from the general kernel, and why (measured: the general kernel
// is bound by the shared-memory pipe, ~17 000 wavefronts per CTA and sample):
//  * gridding as a gather, without atomics and without reading the grid: the
//    plan lists, per pair of adjacent folded cells, the antennas whose
//    footprints cover them with the matching pair of taps; a lane sums one
//    pair's list in registers and stores both cells once (cells no footprint
//    covers get zeros), so the grid is never cleared, each cell costs one store
//    per plane instead of a read-add-write per tap, and one voltage load serves
//    two cells;
//  * the M-point transforms run in registers (one row or column per thread),
//    so each axis costs one shared-memory read and one write;
//  * two time samples per iteration share the gather lists (one entry and tap
//    load serve both samples), the twiddles and the synchronisation;
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
// gridding.  Rows outside rows_used are empty: the row pass skips them and the
// column pass reads them as zeros (their cells hold whatever the last
// transform left there).
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
        for (int i = 0; i < M; i++) x[i] = ((rows_used >> i) & 1ull) ? col[i * S] : make_float2(0.f, 0.f);
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

// E-field images (epic_image_efield): the same two transform passes, then each
// of the TS x P transformed planes is written out as F_p(l, t) on the shifted
// layout instead of being squared and summed.  Class (hx, hy) pixel (my, mx) is
// l = (Q1 mx + hx, Q1 my + hy), stored at out[t][off_c + p N^2 + i N + j] with
// (i, j) = (l_y + N/2, l_x + N/2) mod N.
template <int M, int P, int TS>
__device__ __forceinline__ void transform_store(float2 *G, unsigned long long rows_used, float2 *__restrict__ out,
                                                long long stride, long long off_c, int t, int t1, int N, int Q1,
                                                int hx, int hy, int tid)
{
    constexpr int S = M + 1, BUF = M * S;
    for (int q = tid; q < TS * P * M; q += kThreads) {
        if (!((rows_used >> (q % M)) & 1ull)) continue;
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
        for (int i = 0; i < M; i++) x[i] = ((rows_used >> i) & 1ull) ? col[i * S] : make_float2(0.f, 0.f);
        fft_reg<M>(x, [&](int k, float2 val) { col[k * S] = val; });
    }
    __syncthreads();
    const long long NN = static_cast<long long>(N) * N;
    for (int e = tid; e < TS * P * M * M; e += kThreads) {
        const int pos = e % (M * M), plane = e / (M * M), ts = plane / P, p = plane % P;
        if (t + ts >= t1) continue;
        const int my = pos / M, mx = pos % M;
        // shifted row and column: Q1 m + h + N/2 lies in [0, 2N), so one conditional subtraction
        int i = Q1 * my + hy + N / 2, j = Q1 * mx + hx + N / 2;
        i -= i >= N ? N : 0;
        j -= j >= N ? N : 0;
        out[static_cast<long long>(t + ts) * stride + off_c + p * NN + static_cast<long long>(i) * N + j] =
            G[plane * BUF + my * S + mx];
    }
}

// Folded side M (64, or 48 for grid side 96).  Grid buffers: G[ts][p][y][x] with
// x < M at stride M + 1.  DL: voltages take the geometric-delay phase of the
// per-integration table dtab (Sec. 2.2 delay correction), once per antenna.
// gtab/gidx/gchan: the gather table (per channel a block of per-warp zero lists
// and batches of 32 cells with their (antenna, tap) lists; layout in the plan's
// builder); GS: the channel's block is copied to shared memory first (when it
// fits beside the grids), else it is read through the L1 cache.  rowmask[ci]
// marks the folded rows any footprint touches: the others are never written
// and their transforms are skipped.
// EF: write the E-field images (transform_store) instead of summing products;
// ef_out / ef_off / ef_stride are its output, per-channel offsets and per-sample
// stride (complex elements), unused otherwise.
template <int M, int P, int TS, bool DL, bool GS, bool EF>
__global__ void __launch_bounds__(kThreads, 1)
fp32_reg64_kernel(const uint8_t *__restrict__ v, const float2 *__restrict__ gains,
                  const short2 *__restrict__ cells, const float2 *__restrict__ kern, int K,
                  const int *__restrict__ chans, const float2 *__restrict__ twN,
                  const uint32_t *__restrict__ gtab, const int4 *__restrict__ gidx, const int2 *__restrict__ gchan,
                  const unsigned long long *__restrict__ rowmask,
                  int A, int C, int T, int N, int Q1, int n_items, int n_tau,
                  float *__restrict__ partial, int *__restrict__ status, int nker,
                  const float *__restrict__ dfreq, const float4 *__restrict__ dtab,
                  float2 *__restrict__ ef_out, const long long *__restrict__ ef_off, long long ef_stride)
{
    constexpr int NPOS = M * M / kThreads;       // pixels per thread (16 at M = 64, 9 at 48)
    constexpr int S = M + 1;                     // padded row stride (float2)
    constexpr int BUF = M * S;                   // one [y][x] plane
    extern __shared__ float4 smem_raw[];
    const int AP = A * P, KK = K * K, hk = (K - 1) / 2;
    const int APW = (AP + 3) >> 2;
    float2 *G = reinterpret_cast<float2 *>(smem_raw);          // [TS][P][M][M + 1]
    float4 *tw2 = reinterpret_cast<float4 *>(G + TS * P * BUF);  // [K][K + 1] tap pairs (one kernel)
    float2 *es = reinterpret_cast<float2 *>(tw2 + K * (K + 1)); // [TS][A*P]
    float2 *gp = es + TS * AP;                                 // [A*P]
    float2 *tapw = gp + AP;                                    // [nker][K*K]
    uint32_t *stage = reinterpret_cast<uint32_t *>(tapw + nker * KK); // [TS][APW]
    uint32_t *stab = stage + TS * APW;                         // [block words] (GS)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int item = blockIdx.x % n_items;
    const int tau = blockIdx.x / n_items;
    const int Q = Q1 * Q1;
    const int ci = item / Q, h = item % Q, hx = h % Q1, hy = h / Q1;
    const int c = chans[ci];
    const int t0 = static_cast<int>(static_cast<long long>(T) * tau / n_tau);
    const int t1 = static_cast<int>(static_cast<long long>(T) * (tau + 1) / n_tau);
    const int4 my_idx = gidx[ci * 8 + warp];
    const int2 my_chan = gchan[ci];
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
    // tap pairs of the gather: (w(dy, dxl), w(dy, dxl + 1)) with zero outside the footprint row
    for (int i = tid; i < K * (K + 1); i += kThreads) {
        const int dyi = i / (K + 1), j = i % (K + 1);
        float2 w[2];
        for (int u = 0; u < 2; u++) {
            const int dx = j - 1 + u;
            w[u] = (dx >= 0 && dx < K)
                       ? cmul(kern[dyi * K + dx], twN[(((dx - hk) * hx + (dyi - hk) * hy) % N + N) % N])
                       : make_float2(0.f, 0.f);
        }
        tw2[i] = make_float4(w[0].x, w[0].y, w[1].x, w[1].y);
    }
    for (int i = tid; i < TS * P * BUF; i += kThreads) G[i] = make_float2(0.f, 0.f);
    if constexpr (GS)
        for (int i = tid; i < my_chan.y; i += kThreads) stab[i] = __ldg(gtab + my_chan.x + i);
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

        // ---- a3: gridding as a gather: zeros for the uncovered cells of touched rows, then
        // each lane sums its cell pair's (antenna, tap pair) list in registers and stores the
        // two cells once
        {
            const uint32_t *tb;
            if constexpr (GS) tb = stab;
            else tb = gtab + my_chan.x;
            auto ld = [&](const uint32_t *q) -> uint32_t {
                if constexpr (GS) return *q;
                else return __ldg(q);
            };
            const uint32_t *zl = tb + my_idx.x + lane;
#pragma unroll 4
            for (int r = 0; r < my_idx.y; r++) {
                const uint32_t cell = ld(zl + r * 32);
                if (cell != ~0u) {
#pragma unroll
                    for (int q = 0; q < TS * P; q++) G[q * BUF + cell] = make_float2(0.f, 0.f);
                }
            }
            const uint32_t *bt = tb + my_idx.z;
            uint32_t hdr = my_idx.w > 0 ? ld(bt) : 0u;
            for (int b = 0; b < my_idx.w; b++) {
                const int d = static_cast<int>(hdr);
                const uint32_t cell = ld(bt + 1 + lane);              // left cell of the lane's pair
                const uint32_t *ent = bt + 33 + lane;
                const uint32_t *next = bt + 33 + d * 32;
                if (b + 1 < my_idx.w) hdr = ld(next);                 // next batch's length in flight
                float2 acc_g[TS][P][2];
#pragma unroll
                for (int ts = 0; ts < TS; ts++)
#pragma unroll
                    for (int p = 0; p < P; p++) acc_g[ts][p][0] = acc_g[ts][p][1] = make_float2(0.f, 0.f);
                uint32_t en = d > 0 ? ld(ent) : ~0u;
                for (int j = 0; j < d; j++) {
                    const uint32_t cur = en;
                    if (j + 1 < d) en = ld(ent + (j + 1) * 32);        // next step's entry in flight
                    if (cur != ~0u) {
                        const int a = static_cast<int>(cur >> 8), tp = static_cast<int>(cur & 0xFFu);
                        float2 w[2];
                        if (nker > 1) {   // per-antenna kernels: the pair from the antenna's taps
                            const int dyi = tp / (K + 1), dxl = tp - dyi * (K + 1) - 1;
                            const float2 *wrow = tapw + a * KK + dyi * K;
                            w[0] = dxl >= 0 ? wrow[dxl] : make_float2(0.f, 0.f);
                            w[1] = dxl + 1 < K ? wrow[dxl + 1] : make_float2(0.f, 0.f);
                        } else {
                            const float4 ww = tw2[tp];
                            w[0] = make_float2(ww.x, ww.y);
                            w[1] = make_float2(ww.z, ww.w);
                        }
                        // cell += w e as two packed FMAs: w.x (e.x, e.y) + (-w.y, w.y) (e.y, e.x)
                        float2 wr[2], wi[2];
#pragma unroll
                        for (int u = 0; u < 2; u++) {
                            wr[u] = make_float2(w[u].x, w[u].x);
                            wi[u] = make_float2(-w[u].y, w[u].y);
                        }
#pragma unroll
                        for (int ts = 0; ts < TS; ts++) {
                            float2 e[P];
                            if constexpr (P == 2) {
                                const float4 e2 = reinterpret_cast<const float4 *>(es + ts * AP)[a];
                                e[0] = make_float2(e2.x, e2.y);
                                e[1] = make_float2(e2.z, e2.w);
                            } else {
                                e[0] = es[ts * AP + a];
                            }
#pragma unroll
                            for (int p = 0; p < P; p++) {
                                const float2 esw = pswap(e[p]);
#pragma unroll
                                for (int u = 0; u < 2; u++)
                                    acc_g[ts][p][u] = pfma(wi[u], esw, pfma(wr[u], e[p], acc_g[ts][p][u]));
                            }
                        }
                    }
                }
                if (cell != ~0u) {
#pragma unroll
                    for (int ts = 0; ts < TS; ts++)
#pragma unroll
                        for (int p = 0; p < P; p++) {
                            G[(ts * P + p) * BUF + cell] = acc_g[ts][p][0];
                            G[(ts * P + p) * BUF + cell + 1] = acc_g[ts][p][1];
                        }
                }
                bt = next;
            }
        }
        __syncthreads();

        // ---- a4, a5, a6: transforms, products summed over time (the next gather overwrites
        // every cell of the touched rows, so nothing is cleared); or the E-field images
        if constexpr (EF)
            transform_store<M, P, TS>(G, rows_used, ef_out, ef_stride, ef_off[ci], t, t1, N, Q1, hx, hy, tid);
        else
            transform_products<M, P, TS, false>(G, rows_used, acc, tid);
#pragma unroll
        for (int ts = 0; ts < TS; ts++)
#pragma unroll
            for (int r = 0; r < kPreW; r++) {
                const int w = tid + r * kThreads;
                if (w < APW) stage[ts * APW + w] = pre[ts][r];
            }
        __syncthreads();
    }

    if constexpr (!EF) {
        float *dst = partial + (static_cast<size_t>(tau) * n_items + item) * (M * M) * (P == 2 ? 4 : 1);
#pragma unroll
        for (int r = 0; r < NPOS; r++) {
            const int pos = tid + r * kThreads;
            if constexpr (P == 2) reinterpret_cast<float4 *>(dst)[pos] = acc[r];
            else dst[pos] = acc[r];
        }
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
    b += sizeof(float4) * static_cast<size_t>(K) * (K + 1);
    b += sizeof(uint32_t) * TS * ((AP + 3) / 4);
    return (b + 15) & ~static_cast<size_t>(15);
}

template <int M, int P, int TS, bool DL, bool GS, bool EF = false>
int launch_reg64_t(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau_out,
                   cudaStream_t stream, float2 *ef_out = nullptr, long long ef_stride = 0)
{
    auto kfn = fp32_reg64_kernel<M, P, TS, DL, GS, EF>;
    const size_t smem = reg64_smem<M, P, TS>(plan->A, plan->K, plan->nker) +
                        (GS ? sizeof(uint32_t) * static_cast<size_t>(g.gwords) : 0);
    int n_tau = choose_tau(plan, g, T);
    if (n_tau > g.tau_cap) n_tau = g.tau_cap;
    *n_tau_out = n_tau;
    const dim3 grid(static_cast<unsigned>(g.n_items * n_tau));
    kfn<<<grid, kThreads, smem, stream>>>(v, gains, plan->d_cells, plan->d_kernel, plan->K, g.d_chans, g.d_twN,
                                          g.d_gtab, g.d_gidx, g.d_gchan, g.d_rowmask, plan->A, plan->C, T, g.N,
                                          g.Q1, g.n_items, n_tau, g.d_partial, plan->d_status, plan->nker,
                                          plan->d_dfreq, DL ? plan->d_dtab : nullptr, ef_out, g.d_ef_off, ef_stride);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

// The dynamic shared-memory cap is set to the device's opt-in limit, not to this
// group's size: the cap is per kernel and process, and another group or plan with
// a smaller table must not lower it under this one.
template <int M, int P, int TS, bool GS>
int prepare_reg64_t(const epic_plan_s *plan, const GroupCfg &g)
{
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return EPIC_ERR_CUDA;
    const size_t need = reg64_smem<M, P, TS>(plan->A, plan->K, plan->nker) +
                        (GS ? sizeof(uint32_t) * static_cast<size_t>(g.gwords) : 0);
    if (need > static_cast<size_t>(optin)) return EPIC_ERR_UNSUPPORTED;
    const int smem = optin;
    const bool ok = cudaFuncSetAttribute(fp32_reg64_kernel<M, P, TS, false, GS, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess &&
                    cudaFuncSetAttribute(fp32_reg64_kernel<M, P, TS, true, GS, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess &&
                    cudaFuncSetAttribute(fp32_reg64_kernel<M, P, TS, false, GS, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess;
    return ok ? EPIC_OK : EPIC_ERR_UNSUPPORTED;
}

template <int V>
using IC = std::integral_constant<int, V>;

// The instantiation that serves a group: fold side, polarisations, samples per
// iteration, and whether the gather table is staged in shared memory.
template <class F>
int reg64_dispatch(const epic_plan_s *plan, const GroupCfg &g, F &&f)
{
    auto with_m = [&](auto m_) {
        auto with_p = [&](auto p_) {
            auto with_ts = [&](auto ts_) {
                return g.gstage ? f(m_, p_, ts_, IC<1>{}) : f(m_, p_, ts_, IC<0>{});
            };
            return g.ts == 2 ? with_ts(IC<2>{}) : with_ts(IC<1>{});
        };
        return plan->P == 2 ? with_p(IC<2>{}) : with_p(IC<1>{});
    };
    return g.M == 48 ? with_m(IC<48>{}) : with_m(IC<64>{});
}

}  // namespace

int prepare_reg64(const epic_plan_s *plan, const GroupCfg &g)
{
    return reg64_dispatch(plan, g, [&](auto m_, auto p_, auto ts_, auto gs_) {
        return prepare_reg64_t<decltype(m_)::value, decltype(p_)::value, decltype(ts_)::value,
                               decltype(gs_)::value != 0>(plan, g);
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

int launch_reg64_efield(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T,
                        float2 *out, long long stride, cudaStream_t stream)
{
    return reg64_dispatch(plan, g, [&](auto m_, auto p_, auto ts_, auto gs_) {
        constexpr int M = decltype(m_)::value, P = decltype(p_)::value, TS = decltype(ts_)::value;
        constexpr bool GS = decltype(gs_)::value != 0;
        int n_tau = 1;
        return launch_reg64_t<M, P, TS, false, GS, true>(plan, g, v, gains, T, &n_tau, stream, out, stride);
    });
}

int launch_reg64(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau,
                 cudaStream_t stream)
{
    return reg64_dispatch(plan, g, [&](auto m_, auto p_, auto ts_, auto gs_) {
        constexpr int M = decltype(m_)::value, P = decltype(p_)::value, TS = decltype(ts_)::value;
        constexpr bool GS = decltype(gs_)::value != 0;
        // the delay-corrected form is a separate instantiation, so the plain one carries no trace of it
        return plan->delays ? launch_reg64_t<M, P, TS, true, GS>(plan, g, v, gains, T, n_tau, stream)
                            : launch_reg64_t<M, P, TS, false, GS>(plan, g, v, gains, T, n_tau, stream);
    });
}

}  // namespace epic

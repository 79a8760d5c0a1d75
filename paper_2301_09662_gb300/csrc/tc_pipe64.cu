// Pipelined tensor-core form (folded side M = 64, dual polarisation).
//
// Same arithmetic as tc_col64.cu -- the column transform of each sample is the
// real GEMM D[128 x 128] = A[128 x 128] B^T with FP16 (or BF16) hi + lo
// operands, 3 MMAs per 16-deep k-block -- but laid out so that the tensor
// cores work while the CUDA cores do the rest:
//
//  * A (the 64-point DFT in real 2 x 2 block form, hi and lo) lives in tensor
//    memory for the whole CTA (loaded once with tcgen05.st), which frees the
//    shared memory for two B buffers;
//  * B is MN-major with columns n = 8 (mx mod 8) + mx / 8 (+ 64 for pol Y):
//    a stage-2 radix-8 block of the row transform of grid row jy yields 8
//    consecutive columns, stored as one 16-byte word per part straight from
//    registers, so H never goes back through the grid;
//  * two B buffers: the MMA of sample t runs while sample t+1 is unpacked,
//    gridded and row-transformed; its products are summed after that row
//    transform, before the MMA of t+1 is issued, so one accumulator suffices;
//  * all eight SIMT warps share every phase: a row (pol, jy) is transformed by
//    warps w and w + 4 (half of each radix-8 stage, the stage-1 values
//    exchanged in place through the grid row under a 64-thread named barrier),
//    and warp w sums the products of TMEM lanes 32 (w mod 4) .. and column
//    half w / 4; a ninth warp only issues the MMAs.
//
// TMEM columns: D [0,128), A_hi [128,192), A_lo [192,256) (A packs two 16-bit
// K values per 32-bit column, lower K in the low half), and the time sums
// [256,512).  Lane r = (my, part) holds the Re (part 0) or Im (part 1) row of
// D, and accumulates, for each of its 64 pixels, the partial sums that need no
// other lane: own_X^2, own_Y^2, own_X own_Y, and other_X own_Y with other_X the
// partner lane's (l ^ 16) value -- one shuffle per pixel.  The two lanes'
// partials combine into XX, YY, Re XY, Im XY once, when the partial image is
// written.
// Every wait is bounded; a timeout is recorded in the plan's status word.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "epic_internal.cuh"
#include "fft64.cuh"
#include "tc_ptx.cuh"

#include <type_traits>
#include <vector>

namespace epic {
namespace {

constexpr int M64 = 64;
constexpr int S64 = 65;
constexpr uint32_t kPart = 128u * 128u * 2u;     // one 128 x 128 16-bit B part (32 KB)
constexpr uint32_t kLBO = 128;                  // K-adjacent core matrices
constexpr uint32_t kSBO = 2048;                 // N-adjacent core matrices (16 along K x 128 B)
constexpr uint32_t kColA = 128;                 // first TMEM column of A (D is [0, 128))
constexpr uint32_t kColAcc = 256;               // first TMEM column of the time sums
constexpr int kSimt = kThreads;                 // warps 0-7: unpack, gridding, row transforms, products
constexpr int kPipeThreads = kSimt + 32;        // warp 8: issues the MMAs
constexpr int kBarSimt = 5;                     // named barrier of the eight SIMT warps

// byte offset of B element (n, k) in the MN-major canonical layout
__host__ __device__ constexpr uint32_t b_off(int n, int k)
{
    return static_cast<uint32_t>((n >> 3) * kSBO + (k >> 3) * kLBO + (k & 7) * 16 + (n & 7) * 2);
}

// Two FP32 values as one packed 16-bit pair (a in the low half) and, for the
// split forms, the pair of their rounding residuals (exact in FP32).
template <bool BF16, bool SPLIT>
__device__ __forceinline__ void split_pair(float a, float b, uint32_t &hi, uint32_t &lo)
{
    if constexpr (BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        if constexpr (SPLIT) {
            const float2 back = __bfloat1622float2(h);
            const __nv_bfloat162 l = __floats2bfloat162_rn(a - back.x, b - back.y);
            lo = *reinterpret_cast<const uint32_t *>(&l);
        }
    } else {
        const __half2 h = __floats2half2_rn(a, b);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        if constexpr (SPLIT) {
            const float2 back = __half22float2(h);
            const __half2 l = __floats2half2_rn(a - back.x, b - back.y);
            lo = *reinterpret_cast<const uint32_t *>(&l);
        }
    }
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n"
        "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]),
        "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]),
        "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

// D(tmem) (+)= A(tmem) x B(smem)^T
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// instruction descriptor: FP32 accumulate, A K-major, B MN-major, M x N
__host__ __device__ constexpr uint32_t idesc_mn(int M, int N, bool bf16)
{
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | (1u << 16) |
           (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

// Half H of stage 1 of the 8 x 8 row transform (fft64.cuh): for n2 = 4 H .. 4 H + 3,
// DFT8 over line[n2 + 8 n1], twiddled by w64^(n2 k1), back in place.  H is
// warp-uniform, so both halves run one copy of the code.
__device__ __forceinline__ void row_stage1(float2 *line, int H)
{
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int n2 = 4 * H + i;
        float2 t[8];
#pragma unroll
        for (int n1 = 0; n1 < 8; n1++) t[n1] = line[n2 + 8 * n1];
        dft8(t);
        line[n2] = t[0];
#pragma unroll
        for (int k1 = 1; k1 < 8; k1++) line[n2 + 8 * k1] = cmul(t[k1], c_tw64.w[n2 * k1]);
    }
}

// Half H of stage 2: for k1 = 4 H .. 4 H + 3, DFT8 over line[n2 + 8 k1] (zeroed
// for the next sample's gridding), which yields X[k1 + 8 k2] for the 8
// consecutive B columns n = 8 k1 + k2 (+ 64 p): one 16-byte store per part.
template <bool BF16, bool SPLIT>
__device__ __forceinline__ void row_stage2(float2 *line, uint8_t *bb, int p, int jy, int H)
{
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int k1 = 4 * H + j;
        float2 t[8];
#pragma unroll
        for (int n2 = 0; n2 < 8; n2++) {
            t[n2] = line[n2 + 8 * k1];
            line[n2 + 8 * k1] = make_float2(0.f, 0.f);
        }
        dft8(t);
        uint32_t rh[4], ih[4], rl[4], il[4];
#pragma unroll
        for (int w = 0; w < 4; w++) {
            split_pair<BF16, SPLIT>(t[2 * w].x, t[2 * w + 1].x, rh[w], rl[w]);
            split_pair<BF16, SPLIT>(t[2 * w].y, t[2 * w + 1].y, ih[w], il[w]);
        }
        const int n0 = 8 * k1 + 64 * p;
        *reinterpret_cast<uint4 *>(bb + b_off(n0, jy)) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
        *reinterpret_cast<uint4 *>(bb + b_off(n0, 64 + jy)) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
        if constexpr (SPLIT) {
            *reinterpret_cast<uint4 *>(bb + kPart + b_off(n0, jy)) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
            *reinterpret_cast<uint4 *>(bb + kPart + b_off(n0, 64 + jy)) = make_uint4(il[0], il[1], il[2], il[3]);
        }
    }
}

// Partial products of one sample added to this warp's time sums.  The warp
// reads TMEM lanes 32 (w mod 4) + l = (my, part) and B columns 32 hh .. 32 hh + 31
// of each polarisation (pixels j = 0 .. 31 of the half); pixel j's four partial
// sums sit at columns kColAcc + 128 hh + 4 j.  Two passes of 16 pixels keep the
// registers at 96.
__device__ __forceinline__ void drain_sample(uint32_t lane_addr, int hh)
{
#pragma unroll 1
    for (int q = 0; q < 2; q++) {
        uint32_t rx[16], ry[16], s0[32], s1[32];
        const uint32_t acc = lane_addr + kColAcc + 128 * hh + 64 * q;
        tc::tmem_ld16_issue(lane_addr + 32 * hh + 16 * q, rx);
        tc::tmem_ld16_issue(lane_addr + 64 + 32 * hh + 16 * q, ry);
        tc::tmem_ld32_issue(acc, s0);
        tc::tmem_ld32_issue(acc + 32, s1);
        tc::tmem_wait_ld();
        tc::reg_fence16(rx);
        tc::reg_fence16(ry);
        tc::reg_fence32(s0);
        tc::reg_fence32(s1);
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const float x = __uint_as_float(rx[j]), y = __uint_as_float(ry[j]);
            const float xo = __shfl_xor_sync(0xffffffffu, x, 16);
            uint32_t *a4 = j < 8 ? s0 + 4 * j : s1 + 4 * (j - 8);
            a4[0] = __float_as_uint(fmaf(x, x, __uint_as_float(a4[0])));
            a4[1] = __float_as_uint(fmaf(y, y, __uint_as_float(a4[1])));
            a4[2] = __float_as_uint(fmaf(x, y, __uint_as_float(a4[2])));
            a4[3] = __float_as_uint(fmaf(xo, y, __uint_as_float(a4[3])));
        }
        tc::tmem_st32_issue(acc, s0);
        tc::tmem_st32_issue(acc + 32, s1);
        tc::tmem_wait_st();
    }
}

template <int VAR, int KC>
__global__ void __launch_bounds__(kPipeThreads, 1)
tc_pipe64_kernel(const uint8_t *__restrict__ v, const float2 *__restrict__ gains,
                 const short2 *__restrict__ cells, const float2 *__restrict__ kern, int K_rt,
                 const int *__restrict__ chans, const float2 *__restrict__ twN,
                 const uint32_t *__restrict__ sched, const int *__restrict__ nrounds, int rmax,
                 const unsigned long long *__restrict__ rowmask, const uint16_t *__restrict__ dft_rows,
                 int A, int C, int T, int N, int Q1, int n_items, int n_tau,
                 float *__restrict__ partial, int *__restrict__ status, long long wait_budget, int withhold_mma,
                 const float *__restrict__ dfreq, const float4 *__restrict__ dtab)
{
    constexpr int P = 2;
    constexpr bool kBF16 = VAR == 2;
    constexpr bool kSplit = VAR != 1;
    constexpr int BUF = M64 * S64;
    const int K = KC > 0 ? KC : K_rt;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *opB = smem;                                              // [2 buffers][2 parts][32 KB]
    float2 *G = reinterpret_cast<float2 *>(smem + 4 * kPart);         // [P][64][65]
    const int AP = A * P, KK = K * K, hk = (K - 1) / 2;
    const int APW = (AP + 3) >> 2;
    float2 *es = G + P * BUF;
    float2 *gp = es + AP;
    float2 *tapw = gp + AP;
    uint32_t *stage = reinterpret_cast<uint32_t *>(tapw + KK);
    __shared__ __align__(8) uint64_t bar_mma[2];
    __shared__ uint32_t tmem_slot;
    __shared__ float red[kThreads / 32];
    __shared__ int abort_flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int item = blockIdx.x % n_items;
    const int tau = blockIdx.x / n_items;
    const int Q = Q1 * Q1;
    const int ci = item / Q, h = item % Q, hx = h % Q1, hy = h / Q1;
    const int c = chans[ci];
    const int t0 = static_cast<int>(static_cast<long long>(T) * tau / n_tau);
    const int t1 = static_cast<int>(static_cast<long long>(T) * (tau + 1) / n_tau);
    const uint32_t *my_sched = sched + (static_cast<size_t>(ci) * 8 + warp) * rmax * 32;
    const int my_rounds = warp < 8 ? nrounds[ci * 8 + warp] : 0;
    const unsigned long long rows_used = rowmask[ci];

    if (warp == 0) tc::tmem_alloc(&tmem_slot, 512);
    if (tid == 0) {
        abort_flag = 0;
        tc::mbar_init(&bar_mma[0], 1);
        tc::mbar_init(&bar_mma[1], 1);
        tc::fence_mbar_init();
    }

    // ---- set-up: phase-folded gains and taps, the largest gain for the FP16 scale
    float gmax = 0.f;
    const bool simt = warp < 8;
    for (int a = simt ? tid : A; a < A; a += kThreads) {
        const short2 k = cells[static_cast<size_t>(c) * A + a];
        if (k.x < hk || k.x >= N - hk || k.y < hk || k.y >= N - hk) atomicOr(status, kStatusDevice);
        const float2 ph = twN[((k.x * hx + k.y * hy) % N + N) % N];
        for (int p = 0; p < P; p++) {
            const float2 g = gains ? gains[(static_cast<size_t>(c) * A + a) * P + p] : make_float2(1.f, 0.f);
            const float2 gg = cmul(g, ph);
            gp[a * P + p] = gg;
            gmax = fmaxf(gmax, sqrtf(gg.x * gg.x + gg.y * gg.y));
        }
    }
    for (int i = simt ? tid : KK; i < KK; i += kThreads) {
        const int dy = i / K - hk, dx = i % K - hk;
        tapw[i] = cmul(kern[i], twN[((dx * hx + dy * hy) % N + N) % N]);
    }
    for (int i = simt ? tid : P * BUF; i < P * BUF; i += kThreads) G[i] = make_float2(0.f, 0.f);
    for (int i = simt ? tid : static_cast<int>(4 * kPart / 16); i < static_cast<int>(4 * kPart / 16); i += kThreads)
        reinterpret_cast<uint4 *>(opB)[i] = make_uint4(0u, 0u, 0u, 0u);   // rows never written stay zero
    if (simt && t0 < t1) {
        const uint32_t *row = reinterpret_cast<const uint32_t *>(v + (static_cast<size_t>(t0) * C + c) * AP);
        for (int w = tid; w < APW; w += kThreads) stage[w] = row[w];
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
        float gm = 0.f;
        for (int w = 0; w < kThreads / 32; w++) gm = fmaxf(gm, red[w]);
        float wsum = 0.f;
        for (int i = 0; i < KK; i++) wsum += sqrtf(tapw[i].x * tapw[i].x + tapw[i].y * tapw[i].y);
        const float bound = 2.f * static_cast<float>(A) * 11.3137085f * gm * wsum;
        int e2 = 0;
        if (bound > 0.f) e2 = static_cast<int>(floorf(log2f(16384.f / bound)));
        scale = ldexpf(1.f, max(-40, min(40, e2)));
    }
    for (int i = simt ? tid : AP; i < AP; i += kThreads) gp[i] = cscale(gp[i], scale);
    // A (hi, lo) into TMEM: warp w < 4 writes rows 32w .. 32w+31
    if (warp < 4) {
        const int r = 32 * warp + lane;
        for (int part = 0; part < 2; part++)
            for (int half = 0; half < 2; half++) {
                uint32_t w[32];
                const uint16_t *src = dft_rows + (static_cast<size_t>(part) * 128 + r) * 128 + half * 64;
#pragma unroll
                for (int j = 0; j < 32; j++) w[j] = static_cast<uint32_t>(src[2 * j]) | (static_cast<uint32_t>(src[2 * j + 1]) << 16);
                tmem_st32(taddr + (static_cast<uint32_t>(32 * warp) << 16) + kColA + part * 64 + half * 32, w);
            }
    }
    if (simt) {
        // zero this warp's time sums: TMEM lanes 32 (w mod 4) .., columns kColAcc + 128 (w / 4) ..
        uint32_t z[32];
#pragma unroll
        for (int j = 0; j < 32; j++) z[j] = 0u;
        const uint32_t acc = lane_addr + kColAcc + 128 * (warp >> 2);
        for (int cc = 0; cc < 128; cc += 32) tc::tmem_st32_issue(acc + cc, z);
        tc::tmem_wait_st();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    constexpr uint32_t idesc = idesc_mn(128, 128, kBF16);
    const uint32_t b_base = tc::smem_u32(opB);
    uint32_t phase = 0u;                          // bit b: parity of bar_mma[b]
    constexpr int kPreW = kMaxAP / 4 / kThreads;
    if (!simt) {
        // ---- a4 (columns): D = A B[buf]^T for each sample, issued by one thread
        // once the eight SIMT warps have written B[buf] and drained D (block barrier)
        for (int t = t0; t <= t1; t++) {
            tc::fence_before_sync();
            __syncthreads();
            if (abort_flag) break;
            if (t < t1 && lane == 0 && !withhold_mma) {
                tc::fence_after_sync();
                const int buf = (t - t0) & 1;
                const uint32_t d_tmem = taddr;
                const uint32_t bb = b_base + buf * 2 * kPart;
#pragma unroll
                for (int kb = 0; kb < 8; kb++) {
                    const uint64_t b_hi = tc::smem_desc(bb + kb * 256, kLBO, kSBO);
                    const uint32_t a_hi = taddr + kColA + kb * 8;
                    mma_ts(d_tmem, a_hi, b_hi, idesc, kb > 0 ? 1u : 0u);
                    if constexpr (kSplit) {
                        const uint64_t b_lo = tc::smem_desc(bb + kPart + kb * 256, kLBO, kSBO);
                        mma_ts(d_tmem, a_hi, b_lo, idesc, 1u);
                        mma_ts(d_tmem, a_hi + 64, b_hi, idesc, 1u);
                    }
                }
                tc::mma_commit(&bar_mma[buf]);
            }
            __syncwarp();
        }
    } else for (int t = t0; t <= t1; t++) {
        const bool work = t < t1;
        const int buf = (t - t0) & 1;
        // ---- a1, a2 (sample t) and prefetch of t+1
        if (work) {
            for (int i = tid; i < AP; i += kThreads) {
                const uint32_t b = reinterpret_cast<const uint8_t *>(stage)[i];
                float2 e = cmul(gp[i], ci4_decode(b));
                if (dtab) e = cmul(e, delay_phase(dtab[static_cast<size_t>(t) * A + i / P], dfreq[c]));
                es[i] = e;
            }
        }
        const bool has_next = t + 1 < t1;
        uint32_t pre[kPreW];
        {
            const uint32_t *row = reinterpret_cast<const uint32_t *>(v + (static_cast<size_t>(t + 1) * C + c) * AP);
#pragma unroll
            for (int r = 0; r < kPreW; r++) {
                const int w = tid + r * kThreads;
                pre[r] = (has_next && w < APW) ? __ldg(row + w) : 0u;
            }
        }
        tc::named_bar_sync(kBarSimt, kSimt);

        // ---- a3: scheduled gridding of sample t (the MMA of t-1 is running)
        if (work) {
            for (int r = 0; r < my_rounds; r++) {
                const uint32_t d = __ldg(my_sched + r * 32 + lane);
                if (d >> 31) {
                    const int a = static_cast<int>(d & 0xFFFu);
                    const int dyi = static_cast<int>((d >> 12) & 0xFu);
                    const int y = static_cast<int>((d >> 16) & 0x3Fu);
                    const int x0 = static_cast<int>((d >> 22) & 0x3Fu);
                    const float2 e0 = es[a * P], e1 = es[a * P + 1];
                    const float2 *wrow = tapw + dyi * K;
                    float2 *gy = G + y * S64;
                    if constexpr (KC > 0) {
                        // the KC cells of one lane are distinct, so every load of the
                        // round can be issued before its first store
                        float2 o0[KC], o1[KC];
#pragma unroll
                        for (int dx = 0; dx < KC; dx++) {
                            const int x = (x0 + dx) & (M64 - 1);
                            o0[dx] = gy[x];
                            o1[dx] = gy[BUF + x];
                        }
#pragma unroll
                        for (int dx = 0; dx < KC; dx++) {
                            const float2 w = wrow[dx];
                            const float2 v0 = cmul(w, e0), v1 = cmul(w, e1);
                            const int x = (x0 + dx) & (M64 - 1);
                            gy[x] = make_float2(o0[dx].x + v0.x, o0[dx].y + v0.y);
                            gy[BUF + x] = make_float2(o1[dx].x + v1.x, o1[dx].y + v1.y);
                        }
                    } else {
                        for (int dx = 0; dx < K; dx++) {
                            const float2 w = wrow[dx];
                            const int x = (x0 + dx) & (M64 - 1);
                            const float2 v0 = cmul(w, e0), v1 = cmul(w, e1);
                            const float2 o0 = gy[x], o1 = gy[BUF + x];
                            gy[x] = make_float2(o0.x + v0.x, o0.y + v0.y);
                            gy[BUF + x] = make_float2(o1.x + v1.x, o1.y + v1.y);
                        }
                    }
                }
                __syncwarp();
            }
        }
        tc::named_bar_sync(kBarSimt, kSimt);

        // ---- a4 (rows) of sample t into B[buf]: row (pol, jy) = tid mod 128 is
        // shared by warps w and w + 4, each taking half of both radix-8 stages;
        // the twiddled stage-1 values go back through the grid row between them
        {
            const int q = tid & 127, jy = q & 63, p = q >> 6;
            const bool row_on = work && ((rows_used >> jy) & 1ull);
            float2 *line = G + p * BUF + jy * S64;
            if (row_on) row_stage1(line, warp >> 2);
            tc::named_bar_sync(1 + (warp & 3), 64);
            if (row_on) {
                uint8_t *bb = opB + buf * 2 * kPart;
                row_stage2<kBF16, kSplit>(line, bb, p, jy, warp >> 2);
            }
        }
        // ---- a5, a6: products of sample t-1 (D, written from B[buf ^ 1]) into the time sums
        if (t > t0 && !abort_flag) {
            const int pb = buf ^ 1;
            if (!tc::mbar_wait(&bar_mma[pb], (phase >> pb) & 1u, wait_budget)) {
                atomicOr(status, kStatusTimeout);
                abort_flag = 1;
            } else {
                tc::fence_after_sync();
                drain_sample(lane_addr, warp >> 2);
            }
            phase ^= 1u << pb;
        }
        tc::fence_proxy_async();
        if (has_next) {
#pragma unroll
            for (int r = 0; r < kPreW; r++) {
                const int w = tid + r * kThreads;
                if (w < APW) stage[w] = pre[r];
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        if (abort_flag) break;
    }

    // ---- partial image from each warp's TMEM lanes and column half: the Re and
    // Im lanes' partials combine into XX, YY, Re XY, Im XY (FP16 scale undone exactly)
    if (simt) {
        tc::fence_after_sync();
        const float inv = 1.f / (scale * scale);
        const int hh = warp >> 2, part = lane >> 4;
        const int my = 16 * (warp & 3) + (lane & 15);
        float4 *dst = reinterpret_cast<float4 *>(partial) + (static_cast<size_t>(tau) * n_items + item) * (M64 * M64);
#pragma unroll 1
        for (int q = 0; q < 2; q++) {
            uint32_t s0[32], s1[32];
            const uint32_t acc = lane_addr + kColAcc + 128 * hh + 64 * q;
            tc::tmem_ld32_issue(acc, s0);
            tc::tmem_ld32_issue(acc + 32, s1);
            tc::tmem_wait_ld();
            tc::reg_fence32(s0);
            tc::reg_fence32(s1);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const uint32_t *a4 = j < 8 ? s0 + 4 * j : s1 + 4 * (j - 8);
                float v[4], o[4];
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    v[i] = __uint_as_float(a4[i]);
                    o[i] = __shfl_xor_sync(0xffffffffu, v[i], 16);
                }
                // lane part 0 holds sum xi yr in v[3], part 1 holds sum xr yi
                const float im = part ? o[3] - v[3] : v[3] - o[3];
                if ((j >> 3) == part) {
                    const int n = 32 * hh + 16 * q + j;         // B column -> mx = n / 8 + 8 (n mod 8)
                    const int mx = (n >> 3) + 8 * (n & 7);
                    dst[my * M64 + mx] = make_float4((v[0] + o[0]) * inv, (v[1] + o[1]) * inv,
                                                     (v[2] + o[2]) * inv, im * inv);
                }
            }
        }
    }
    // an aborted CTA may still have an MMA in flight: give it a bounded chance to land
    if (tid == 0 && abort_flag) {
        tc::mbar_wait(&bar_mma[0], phase & 1u, wait_budget);
        tc::mbar_wait(&bar_mma[1], (phase >> 1) & 1u, wait_budget);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, 512);
}

size_t pipe_smem(int A, int K)
{
    const int AP = A * 2;
    size_t b = 4 * static_cast<size_t>(kPart);
    b += sizeof(float2) * (static_cast<size_t>(2) * M64 * S64 + 2 * AP + K * K);
    b += sizeof(uint32_t) * ((AP + 3) / 4);
    return (b + 15) & ~static_cast<size_t>(15);
}

template <int VAR, int KC>
int prepare_pipe_t(const epic_plan_s *plan)
{
    return cudaFuncSetAttribute(tc_pipe64_kernel<VAR, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(pipe_smem(plan->A, plan->K))) == cudaSuccess
               ? EPIC_OK
               : EPIC_ERR_UNSUPPORTED;
}

template <int VAR, int KC>
int launch_pipe_t(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau_out,
                  cudaStream_t stream)
{
    int n_tau = choose_tau(plan, g, T);
    if (n_tau > g.tau_cap) n_tau = g.tau_cap;
    *n_tau_out = n_tau;
    const dim3 grid(static_cast<unsigned>(g.n_items * n_tau));
    tc_pipe64_kernel<VAR, KC><<<grid, kPipeThreads, pipe_smem(plan->A, plan->K), stream>>>(
        v, gains, plan->d_cells, plan->d_kernel, plan->K, g.d_chans, g.d_twN, g.d_sched, g.d_nrounds, g.rmax,
        g.d_rowmask, plan->d_dft_rows, plan->A, plan->C, T, g.N, g.Q1, g.n_items, n_tau, g.d_partial,
        plan->d_status, plan->wait_budget, plan->test_withhold_mma, plan->d_dfreq,
        plan->delays ? plan->d_dtab : nullptr);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

template <class F>
int pipe_dispatch(int precision, int K, F &&f)
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

size_t tc_pipe_smem_bytes(int A, int K) { return pipe_smem(A, K); }

int prepare_tc_pipe(const epic_plan_s *plan)
{
    return pipe_dispatch(plan->precision, plan->K, [&](auto vv, auto kc) {
        return prepare_pipe_t<decltype(vv)::value, decltype(kc)::value>(plan);
    });
}

int launch_tc_pipe(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau,
                   cudaStream_t stream)
{
    return pipe_dispatch(plan->precision, plan->K, [&](auto vv, auto kc) {
        return launch_pipe_t<decltype(vv)::value, decltype(kc)::value>(plan, g, v, gains, T, n_tau, stream);
    });
}

// The column-DFT operand as plain rows for tcgen05.st: [part][128 rows][128 K]
// 16-bit words, hi part then lo part, FP16 or BF16 bit patterns.
void build_dft_rows(bool bf16, std::vector<uint16_t> &words)
{
    words.assign(2 * 128 * 128, 0);
    auto to16h = [bf16](double x, double &back) -> uint16_t {
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
            const int jy = k % 64;
            const bool im_in = k >= 64;
            const long e = (static_cast<long>(jy) * my) % 64;
            const double th = 2.0 * M_PI * static_cast<double>(e) / 64.0;
            double a;
            if (part == 0) a = im_in ? -std::sin(th) : std::cos(th);
            else a = im_in ? std::cos(th) : std::sin(th);
            double hb = 0, lb = 0;
            words[static_cast<size_t>(r) * 128 + k] = to16h(a, hb);
            words[static_cast<size_t>(128 * 128) + static_cast<size_t>(r) * 128 + k] = to16h(a - hb, lb);
        }
    }
}

}  // namespace epic

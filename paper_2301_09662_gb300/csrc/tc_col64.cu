// Tensor-core form (folded side M = 64, dual polarisation): gridding and the
// row transform run in FP32 exactly as in fp32_reg64.cu; the column transform
// is a DFT-as-GEMM on the 5th-generation tensor cores.
//
// Per time sample and CTA (one pixel class of one channel), with H the
// row-transformed folded grid, the column DFT in real form is one GEMM
//     D[r][n] = sum_k A[r][k] B[n][k],   M = N = K = 128,
//   rows r = (my, Re/Im): r = 32 q + l, my = 16 q + (l mod 16), part = l / 16,
//   K    k = (Re/Im, jy): k < 64 -> Re H(jy = k), k >= 64 -> Im H(jy = k - 64),
//   cols n = (mx, pol):  n = mx + 64 p,
//   A = [[cos, -sin], [sin, cos]] of theta = 2 pi jy my / 64 (sign +, Eq. 4).
// FP16 operands carry about 11 bits, so both A and H are split x = hi + lo
// and the GEMM is A_hi B_hi + A_hi B_lo + A_lo B_hi (the lo x lo term is
// below FP32 rounding); the single-FP16 variant keeps only A_hi B_hi, and the
// BF16 variant uses the same two-part split with 8-bit mantissas.  H is scaled
// by a power of two so |H| stays inside the FP16 range; the scale is undone
// exactly on the finished partial sums.  The accumulator D (128 lanes x 128
// FP32 columns) lives in tensor memory; the products XX, YY, XY are formed
// straight from it and summed over time in registers.
//
// The DFT operand (2 x 32 KB, built once per plan) is staged into shared
// memory by one bulk TMA copy per CTA.  The MMA is issued by one thread and
// completes on an mbarrier; every wait is bounded and a timeout is recorded in
// the plan's status word.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "epic_internal.cuh"
#include "fft64.cuh"
#include "tc_ptx.cuh"

namespace epic {
namespace {

constexpr int M64 = 64;
constexpr int S64 = 65;
constexpr int KT = 128;                          // K of one operand part
constexpr uint32_t kPartBytes = 128u * KT * 2u;   // one 128 x 128 16-bit operand part
constexpr uint32_t kLBO = 128;                   // K-adjacent core matrices
constexpr uint32_t kSBO = KT * 16;               // M/N-adjacent core matrices (2048 B)

__host__ __device__ constexpr uint32_t op_off(int row, int k)
{
    return static_cast<uint32_t>((row >> 3) * kSBO + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

template <bool BF16>
struct Half16;
template <>
struct Half16<false> {
    static __device__ __forceinline__ uint16_t bits(float x, float &back)
    {
        const __half h = __float2half_rn(x);
        back = __half2float(h);
        return __half_as_ushort(h);
    }
};
template <>
struct Half16<true> {
    static __device__ __forceinline__ uint16_t bits(float x, float &back)
    {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        back = __bfloat162float(h);
        return __bfloat16_as_ushort(h);
    }
};

// VAR: 0 = FP16 two-part split (3 MMAs per k-block), 1 = single FP16, 2 = BF16 two-part split
template <int VAR>
__global__ void __launch_bounds__(kThreads, 1)
tc_col64_kernel(const uint8_t *__restrict__ v, const float2 *__restrict__ gains,
                const short2 *__restrict__ cells, const float2 *__restrict__ kern, int K,
                const int *__restrict__ chans, const float2 *__restrict__ twN,
                const uint32_t *__restrict__ sched, const int *__restrict__ nrounds, int rmax,
                const uint8_t *__restrict__ dft_ops, int A, int C, int T, int N, int Q1, int n_items, int n_tau,
                float *__restrict__ partial, int *__restrict__ status, long long wait_budget, int withhold_mma,
                const float *__restrict__ dfreq, const float4 *__restrict__ dtab)
{
    constexpr int P = 2;
    constexpr bool kBF16 = VAR == 2;
    constexpr bool kSplit = VAR != 1;
    constexpr int BUF = M64 * S64;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *opA = smem;                                          // [2 parts][128 x 128] 16-bit
    uint8_t *opB = smem + 2 * kPartBytes;                         // [2 parts][128 x 128] 16-bit
    float2 *G = reinterpret_cast<float2 *>(smem + 4 * kPartBytes); // [P][64][65]
    const int AP = A * P, KK = K * K, hk = (K - 1) / 2;
    const int APW = (AP + 3) >> 2;
    float2 *es = G + P * BUF;                                     // [A*P]
    float2 *gp = es + AP;                                         // [A*P]
    float2 *tapw = gp + AP;                                       // [K*K]
    uint32_t *stage = reinterpret_cast<uint32_t *>(tapw + KK);    // [APW]
    __shared__ __align__(8) uint64_t bar_ops, bar_mma;
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
    const int my_rounds = nrounds[ci * 8 + warp];

    if (warp == 0) tc::tmem_alloc(&tmem_slot, 128);
    if (tid == 0) {
        abort_flag = 0;
        tc::mbar_init(&bar_ops, 1);
        tc::mbar_init(&bar_mma, 1);
        tc::fence_mbar_init();
    }

    // ---- set-up: phase-folded gains and taps, the largest gain for the FP16 scale
    float gmax = 0.f;
    for (int a = tid; a < A; a += kThreads) {
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
    for (int i = tid; i < KK; i += kThreads) {
        const int dy = i / K - hk, dx = i % K - hk;
        tapw[i] = cmul(kern[i], twN[((dx * hx + dy * hy) % N + N) % N]);
    }
    for (int i = tid; i < P * BUF; i += kThreads) G[i] = make_float2(0.f, 0.f);
    if (t0 < t1) {
        const uint32_t *row = reinterpret_cast<const uint32_t *>(v + (static_cast<size_t>(t0) * C + c) * AP);
        for (int w = tid; w < APW; w += kThreads) stage[w] = row[w];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    if (lane == 0) red[warp] = gmax;
    __syncthreads();
    // |H| <= sum_a |g~_a| * 8 sqrt 2 * sum |W|; scale it below 2^14 (FP16 max 65504)
    float scale = 1.f;
    if constexpr (!kBF16) {
        float gm = 0.f;
        for (int w = 0; w < kThreads / 32; w++) gm = fmaxf(gm, red[w]);
        float wsum = 0.f;
        for (int i = 0; i < KK; i++) wsum += sqrtf(tapw[i].x * tapw[i].x + tapw[i].y * tapw[i].y);
        const float bound = 2.f * static_cast<float>(A) * 11.3137085f * gm * wsum;
        int e2 = 0;
        if (bound > 0.f) e2 = static_cast<int>(floorf(log2f(16384.f / bound)));
        scale = ldexpf(1.f, max(-40, min(40, e2)));   // an exact power of two
    }
    for (int i = tid; i < AP; i += kThreads) gp[i] = cscale(gp[i], scale);
    if (tid == 0) {
        tc::mbar_expect_tx(&bar_ops, 2 * kPartBytes);
        tc::bulk_g2s(opA, dft_ops, kPartBytes, &bar_ops);
        tc::bulk_g2s(opA + kPartBytes, dft_ops + kPartBytes, kPartBytes, &bar_ops);
    }
    float4 acc[16];
#pragma unroll
    for (int j = 0; j < 16; j++) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tmem_slot;

    constexpr uint32_t idesc = tc::idesc_f16(128, 128, kBF16);
    const uint32_t a_base = tc::smem_u32(opA), b_base = tc::smem_u32(opB);
    uint32_t phase = 0;
    bool ops_ready = false;
    constexpr int kPreW = kMaxAP / 4 / kThreads;
    for (int t = t0; t < t1; t++) {
        // ---- a1, a2
        for (int i = tid; i < AP; i += kThreads) {
            const uint32_t b = reinterpret_cast<const uint8_t *>(stage)[i];
            float2 e = cmul(gp[i], ci4_decode(b));
            if (dtab) e = cmul(e, delay_phase(dtab[static_cast<size_t>(t) * A + i / P], dfreq[c]));
            es[i] = e;
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
        __syncthreads();

        // ---- a3: scheduled gridding (warp-owned rows, no atomics)
        for (int r = 0; r < my_rounds; r++) {
            const uint32_t d = __ldg(my_sched + r * 32 + lane);
            if (d >> 31) {
                const int a = static_cast<int>(d & 0xFFFu);
                const int dyi = static_cast<int>((d >> 12) & 0xFu);
                const int y = static_cast<int>((d >> 16) & 0x3Fu);
                const int x0 = static_cast<int>((d >> 22) & 0x3Fu);
                const float2 e0 = es[a * P], e1 = es[a * P + 1];
                const float2 *wrow = tapw + dyi * K;
                for (int dx = 0; dx < K; dx++) {
                    const float2 w = wrow[dx];
                    const int x = (x0 + dx) & (M64 - 1);
                    float2 *c0 = G + y * S64 + x;
                    float2 *c1 = c0 + BUF;
                    const float2 v0 = cmul(w, e0), v1 = cmul(w, e1);
                    float2 o0 = *c0, o1 = *c1;
                    o0.x += v0.x;
                    o0.y += v0.y;
                    o1.x += v1.x;
                    o1.y += v1.y;
                    *c0 = o0;
                    *c1 = o1;
                }
            }
            __syncwarp();
        }
        __syncthreads();

        // ---- a4 (rows): 64-point transforms in registers, back into G
        for (int q = tid; q < P * M64; q += kThreads) {
            float2 *line = G + (q / M64) * BUF + (q % M64) * S64;
            float2 x[64];
#pragma unroll
            for (int i = 0; i < 64; i++) x[i] = line[i];
            fft64_stage1(x);
            fft64_stage2(x, [&](int k, float2 val) { line[k] = val; });
        }
        __syncthreads();

        // ---- pack H into the B operand (hi, lo parts), clearing G
        {
            const int n = tid & 127, kh = tid >> 7;
            const int mx = n & 63, p = n >> 6;
            float2 *col = G + p * BUF + mx;
#pragma unroll
            for (int jb = 0; jb < 4; jb++) {
                const int jy0 = 32 * kh + 8 * jb;
                uint16_t rh[8], ih[8], rl[8], il[8];
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const float2 hv = col[(jy0 + j) * S64];
                    col[(jy0 + j) * S64] = make_float2(0.f, 0.f);
                    float br, bi;
                    rh[j] = Half16<kBF16>::bits(hv.x, br);
                    ih[j] = Half16<kBF16>::bits(hv.y, bi);
                    if constexpr (kSplit) {
                        float dummy;
                        rl[j] = Half16<kBF16>::bits(hv.x - br, dummy);
                        il[j] = Half16<kBF16>::bits(hv.y - bi, dummy);
                    }
                }
                auto pack = [](const uint16_t *s) {
                    return make_uint4(s[0] | (static_cast<uint32_t>(s[1]) << 16), s[2] | (static_cast<uint32_t>(s[3]) << 16),
                                      s[4] | (static_cast<uint32_t>(s[5]) << 16), s[6] | (static_cast<uint32_t>(s[7]) << 16));
                };
                *reinterpret_cast<uint4 *>(opB + op_off(n, jy0)) = pack(rh);
                *reinterpret_cast<uint4 *>(opB + op_off(n, 64 + jy0)) = pack(ih);
                if constexpr (kSplit) {
                    *reinterpret_cast<uint4 *>(opB + kPartBytes + op_off(n, jy0)) = pack(rl);
                    *reinterpret_cast<uint4 *>(opB + kPartBytes + op_off(n, 64 + jy0)) = pack(il);
                }
            }
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();

        // ---- a4 (columns): D = A x B^T on the tensor cores, one thread issues
        if (tid == 0) {
            tc::fence_after_sync();
            bool ok = true;
            if (!ops_ready) {
                ok = tc::mbar_wait(&bar_ops, 0, wait_budget);
                ops_ready = ok;
            }
            // withhold_mma (fault-injection test hook): issue nothing and arrive
            // nowhere, so every thread's bounded wait below runs out
            if (ok && !withhold_mma) {
#pragma unroll
                for (int kb = 0; kb < 8; kb++) {
                    const uint32_t koff = static_cast<uint32_t>(kb) * 2u * 128u;
                    const uint64_t a_hi = tc::smem_desc(a_base + koff, kLBO, kSBO);
                    const uint64_t b_hi = tc::smem_desc(b_base + koff, kLBO, kSBO);
                    tc::mma_f16(taddr, a_hi, b_hi, idesc, kb > 0 ? 1u : 0u);
                    if constexpr (kSplit) {
                        const uint64_t a_lo = tc::smem_desc(a_base + kPartBytes + koff, kLBO, kSBO);
                        const uint64_t b_lo = tc::smem_desc(b_base + kPartBytes + koff, kLBO, kSBO);
                        tc::mma_f16(taddr, a_hi, b_lo, idesc, 1u);
                        tc::mma_f16(taddr, a_lo, b_hi, idesc, 1u);
                    }
                }
                tc::mma_commit(&bar_mma);
            } else if (!ok) {
                atomicOr(status, kStatusTimeout);
                abort_flag = 1;
            }
        }
        __syncthreads();
        if (abort_flag) break;
        if (!tc::mbar_wait(&bar_mma, phase, wait_budget)) {
            atomicOr(status, kStatusTimeout);
            abort_flag = 1;
        }
        phase ^= 1u;
        tc::fence_after_sync();

        // ---- a5, a6: products from tensor memory, summed in registers
        if (!abort_flag) {
            const int qd = warp & 3, half = warp >> 2, part = lane >> 4;
            const uint32_t row_addr = taddr + (static_cast<uint32_t>(32 * qd) << 16);
            float vx[32], vy[32];
            tc::tmem_ld32(row_addr + 32 * half, vx);
            tc::tmem_ld32(row_addr + 64 + 32 * half, vy);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                // keep mx sub-range [16 part, 16 part + 16) of this half, trade the other
                const float ox = part ? vx[16 + j] : vx[j], oy = part ? vy[16 + j] : vy[j];
                const float sx = part ? vx[j] : vx[16 + j], sy = part ? vy[j] : vy[16 + j];
                const float gx = __shfl_xor_sync(0xffffffffu, sx, 16);
                const float gy = __shfl_xor_sync(0xffffffffu, sy, 16);
                const float xr = part ? gx : ox, xi = part ? ox : gx;
                const float yr = part ? gy : oy, yi = part ? oy : gy;
                acc[j].x = fmaf(xr, xr, fmaf(xi, xi, acc[j].x));
                acc[j].y = fmaf(yr, yr, fmaf(yi, yi, acc[j].y));
                acc[j].z = fmaf(xr, yr, fmaf(xi, yi, acc[j].z));
                acc[j].w = fmaf(xi, yr, fmaf(-xr, yi, acc[j].w));
            }
        }
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

    // ---- partial sums (undo the FP16 scale exactly: products carry scale^2)
    {
        const float inv = 1.f / (scale * scale);
        const int qd = warp & 3, half = warp >> 2, part = lane >> 4;
        const int my = 16 * qd + (lane & 15);
        float4 *dst = reinterpret_cast<float4 *>(partial) + (static_cast<size_t>(tau) * n_items + item) * (M64 * M64);
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const int mx = 32 * half + 16 * part + j;
            const float4 a4 = acc[j];
            dst[my * M64 + mx] = make_float4(a4.x * inv, a4.y * inv, a4.z * inv, a4.w * inv);
        }
    }
    // an aborted CTA may still have a copy or an MMA in flight: give them a bounded chance to land
    if (tid == 0 && abort_flag) {
        if (!ops_ready) tc::mbar_wait(&bar_ops, 0, wait_budget);
        tc::mbar_wait(&bar_mma, phase ^ 1u, wait_budget);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, 128);
}

size_t tc_smem(int A, int K)
{
    const int AP = A * 2;
    size_t b = 4 * static_cast<size_t>(kPartBytes);
    b += sizeof(float2) * (static_cast<size_t>(2) * M64 * S64 + 2 * AP + K * K);
    b += sizeof(uint32_t) * ((AP + 3) / 4);
    return (b + 15) & ~static_cast<size_t>(15);
}

template <int VAR>
int prepare_tc_t(const epic_plan_s *plan)
{
    return cudaFuncSetAttribute(tc_col64_kernel<VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(tc_smem(plan->A, plan->K))) == cudaSuccess
               ? EPIC_OK
               : EPIC_ERR_UNSUPPORTED;
}

template <int VAR>
int launch_tc_t(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau_out,
                cudaStream_t stream)
{
    int n_tau = choose_tau(plan, g, T);
    if (n_tau > g.tau_cap) n_tau = g.tau_cap;
    *n_tau_out = n_tau;
    const dim3 grid(static_cast<unsigned>(g.n_items * n_tau));
    tc_col64_kernel<VAR><<<grid, kThreads, tc_smem(plan->A, plan->K), stream>>>(
        v, gains, plan->d_cells, plan->d_kernel, plan->K, g.d_chans, g.d_twN, g.d_sched, g.d_nrounds, g.rmax,
        plan->d_dft, plan->A, plan->C, T, g.N, g.Q1, g.n_items, n_tau, g.d_partial, plan->d_status,
        plan->wait_budget, plan->test_withhold_mma, plan->d_dfreq, plan->delays ? plan->d_dtab : nullptr);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

int tc_variant(int precision)
{
    switch (precision) {
    case EPIC_TC_SPLIT_FP16: return 0;
    case EPIC_TC_FP16: return 1;
    case EPIC_TC_SPLIT_BF16: return 2;
    default: return -1;
    }
}

}  // namespace

size_t tc_smem_bytes(int A, int K) { return tc_smem(A, K); }

int prepare_tc(const epic_plan_s *plan)
{
    switch (tc_variant(plan->precision)) {
    case 0: return prepare_tc_t<0>(plan);
    case 1: return prepare_tc_t<1>(plan);
    case 2: return prepare_tc_t<2>(plan);
    default: return EPIC_ERR_UNSUPPORTED;
    }
}

int launch_tc(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau,
              cudaStream_t stream)
{
    switch (tc_variant(plan->precision)) {
    case 0: return launch_tc_t<0>(plan, g, v, gains, T, n_tau, stream);
    case 1: return launch_tc_t<1>(plan, g, v, gains, T, n_tau, stream);
    case 2: return launch_tc_t<2>(plan, g, v, gains, T, n_tau, stream);
    default: return EPIC_ERR_UNSUPPORTED;
    }
}

// The column-DFT operand A (hi part, then lo part) in the canonical K-major
// layout, as 16-bit words: FP16 or BF16 bit patterns.
void build_dft_operand(bool bf16, std::vector<uint16_t> &words)
{
    words.assign(2 * kPartBytes / 2, 0);
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
            const int jy = k % 64;
            const bool im_in = k >= 64;
            const long e = (static_cast<long>(jy) * my) % 64;
            const double th = 2.0 * M_PI * static_cast<double>(e) / 64.0;
            double a;
            if (part == 0) a = im_in ? -std::sin(th) : std::cos(th);
            else a = im_in ? std::cos(th) : std::sin(th);
            double hi_back = 0, lo_back = 0;
            const uint16_t hi = to16(a, hi_back);
            const uint16_t lo = to16(a - hi_back, lo_back);
            words[op_off(r, k) / 2] = hi;
            words[(kPartBytes + op_off(r, k)) / 2] = lo;
        }
    }
}

}  // namespace epic

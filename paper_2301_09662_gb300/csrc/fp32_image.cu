// FP32 form of the EPIC imaging path: one fused kernel per grid side that
// unpacks and calibrates the ci4 voltages, grids them in shared memory, runs
// the 2-D transform in shared memory, forms the polarisation products and sums
// them over time in registers (Eq. 4; blocks of Sec. 2.2 fused).
//
// Work split.  With the sky index written l = Q1 m + h (h in [0, Q1)^2), the
// transform restricted to one pixel class h is
//     F(Q1 m + h) = sum_{j in [0,M)^2} w_M^{j.m} Gf_h(j),
//     Gf_h(j)     = sum_{k = j mod M} G(k) w_N^{k.h},       M = N / Q1,
// so a CTA that owns class h grids every antenna straight into an M x M folded
// aperture, with the phase w_N^{k.h} split into a per-antenna factor (folded
// into the gain) and a per-tap factor (folded into the kernel), and then runs
// an M x M FFT.  The CTA's M^2 pixels keep their XX, YY, XY sums in registers
// for the whole time range, so nothing but the finished partial sums goes back
// to memory.  Channels x classes x time chunks fill the GPU.
//
// Each 1-D transform of length M = R1 R2 is two in-place shared-memory passes
// (radix R1 with twiddles, then radix R2).  Position p = R2 k1 + k2 then holds
// frequency k1 + R1 k2; the epilogue undoes that digit order.
#include <cstdio>

#include "dft_small.cuh"
#include <algorithm>

#include "epic_internal.cuh"

namespace epic {
namespace {

template <int M>
struct Radix;
template <> struct Radix<32> { static constexpr int R1 = 8, R2 = 4; };
template <> struct Radix<48> { static constexpr int R1 = 8, R2 = 6; };
template <> struct Radix<64> { static constexpr int R1 = 8, R2 = 8; };

// pass 1 of a length-M transform along rows (ROWS) or columns, both pols:
// element n2 + R2 n1 -> DFT over n1, twiddle w_M^{n2 k1}, back to n2 + R2 k1
template <int M, int P, bool ROWS>
__device__ __forceinline__ void fft_pass1(float2 *Gf, const float2 *twM)
{
    constexpr int R1 = Radix<M>::R1, R2 = Radix<M>::R2, S = M + 1;
    constexpr int TASKS = P * M * R2;
    for (int q = threadIdx.x; q < TASKS; q += kThreads) {
        const int line = q % M;
        const int rest = q / M;
        const int n2 = rest % R2;
        const int p = rest / R2;
        float2 *base = Gf + p * M * S + (ROWS ? line * S : line);
        const int step = ROWS ? 1 : S;
        float2 x[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; n1++) x[n1] = base[(n2 + R2 * n1) * step];
        dft<R1>(x);
#pragma unroll
        for (int k1 = 1; k1 < R1; k1++) x[k1] = cmul(x[k1], twM[n2 * k1]);
#pragma unroll
        for (int k1 = 0; k1 < R1; k1++) base[(n2 + R2 * k1) * step] = x[k1];
    }
}

// pass 2: element R2 k1 + n2 -> DFT over n2, back in place (digit-reversed order)
template <int M, int P, bool ROWS>
__device__ __forceinline__ void fft_pass2(float2 *Gf)
{
    constexpr int R1 = Radix<M>::R1, R2 = Radix<M>::R2, S = M + 1;
    constexpr int TASKS = P * M * R1;
    for (int q = threadIdx.x; q < TASKS; q += kThreads) {
        const int line = q % M;
        const int rest = q / M;
        const int k1 = rest % R1;
        const int p = rest / R1;
        float2 *base = Gf + p * M * S + (ROWS ? line * S : line);
        const int step = ROWS ? 1 : S;
        float2 x[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; n2++) x[n2] = base[(R2 * k1 + n2) * step];
        dft<R2>(x);
#pragma unroll
        for (int k2 = 0; k2 < R2; k2++) base[(R2 * k1 + k2) * step] = x[k2];
    }
}

template <int P>
struct Acc;
template <> struct Acc<1> { using T = float; };
template <> struct Acc<2> { using T = float4; };

template <int M, int P>
__global__ void __launch_bounds__(kThreads, 2)
fp32_image_kernel(const uint8_t *__restrict__ v, const float2 *__restrict__ gains,
                  const short2 *__restrict__ cells, const float2 *__restrict__ kern, int K,
                  const int *__restrict__ chans, const float2 *__restrict__ twN,
                  int A, int C, int T, int N, int Q1, int n_items, int n_tau,
                  float *__restrict__ partial, int *__restrict__ status, int nker,
                  const float *__restrict__ dfreq, const float4 *__restrict__ dtab)
{
    constexpr int S = M + 1;
    constexpr int NPOS = (M * M + kThreads - 1) / kThreads;
    extern __shared__ float4 smem_raw[];
    const int AP = A * P, KK = K * K, hk = (K - 1) / 2;
    float2 *Gf = reinterpret_cast<float2 *>(smem_raw);   // [P][M][S]
    float2 *es = Gf + P * M * S;                          // [A*P] calibrated voltages
    float2 *gp = es + AP;                                 // [A*P] gains x class phase
    float2 *tapw = gp + AP;                               // [nker][K*K] kernel(s) x class phase
    float2 *twM = tapw + nker * KK;                       // [M]
    uint32_t *antj = reinterpret_cast<uint32_t *>(twM + M);  // [A] folded cell
    uint32_t *tapd = antj + A;                            // [K*K] packed offsets
    uint32_t *stage = tapd + KK;                          // [ceil(AP/4)] ci4 words

    const int tid = threadIdx.x;
    const int item = blockIdx.x % n_items;
    const int tau = blockIdx.x / n_items;
    const int Q = Q1 * Q1;
    const int ci = item / Q, h = item % Q, hx = h % Q1, hy = h / Q1;
    const int c = chans[ci];
    const int t0 = static_cast<int>(static_cast<long long>(T) * tau / n_tau);
    const int t1 = static_cast<int>(static_cast<long long>(T) * (tau + 1) / n_tau);
    const bool words = (AP & 3) == 0;
    const int APW = (AP + 3) >> 2;

    // ---- per-CTA set-up: folded cells, phase-folded gains and taps, twiddles
    for (int a = tid; a < A; a += kThreads) {
        const short2 k = cells[static_cast<size_t>(c) * A + a];
        int kx = k.x, ky = k.y;
        if (kx < hk || kx >= N - hk || ky < hk || ky >= N - hk) {
            atomicOr(status, kStatusDevice);   // plan guarantees this never happens
            kx = ky = N / 2;
        }
        antj[a] = static_cast<uint32_t>(kx % M) | (static_cast<uint32_t>(ky % M) << 16);
        const float2 ph = twN[(kx * hx + ky * hy) % N];
        for (int p = 0; p < P; p++) {
            const float2 g = gains ? gains[(static_cast<size_t>(c) * A + a) * P + p] : make_float2(1.f, 0.f);
            gp[a * P + p] = cmul(g, ph);
        }
    }
    for (int i = tid; i < nker * KK; i += kThreads) {
        const int tap = i % KK;
        const int dy = tap / K - hk, dx = tap % K - hk;
        const int e = ((dx * hx + dy * hy) % N + N) % N;
        tapw[i] = cmul(kern[i], twN[e]);
        if (i < KK) tapd[i] = static_cast<uint32_t>(dx + 16) | (static_cast<uint32_t>(dy + 16) << 8);
    }
    for (int k = tid; k < M; k += kThreads) twM[k] = twN[k * Q1];
    for (int i = tid; i < P * M * S; i += kThreads) Gf[i] = make_float2(0.f, 0.f);

    const uint8_t *vrow0 = v + (static_cast<size_t>(t0) * C + c) * AP;
    if (t0 < t1) {
        if (words) {
            for (int w = tid; w < APW; w += kThreads) stage[w] = reinterpret_cast<const uint32_t *>(vrow0)[w];
        } else {
            for (int i = tid; i < AP; i += kThreads) reinterpret_cast<uint8_t *>(stage)[i] = vrow0[i];
        }
    }

    typename Acc<P>::T acc[NPOS];
#pragma unroll
    for (int r = 0; r < NPOS; r++) {
        if constexpr (P == 2) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        else acc[r] = 0.f;
    }
    __syncthreads();

    constexpr int kPreW = kMaxAP / 4 / kThreads;   // ci4 words prefetched per thread
    for (int t = t0; t < t1; t++) {
        // ---- a1, a2: unpack and calibrate this time sample
        for (int i = tid; i < AP; i += kThreads) {
            const uint32_t b = reinterpret_cast<const uint8_t *>(stage)[i];
            float2 e = cmul(gp[i], ci4_decode(b));
            if (dtab) e = cmul(e, delay_phase(dtab[static_cast<size_t>(t) * A + i / P], dfreq[c]));
            es[i] = e;
        }
        // prefetch the next sample's bytes while this one is gridded and transformed
        const bool has_next = t + 1 < t1;
        const uint8_t *vnext = v + (static_cast<size_t>(t + 1) * C + c) * AP;
        uint32_t pre[kPreW];
#pragma unroll
        for (int r = 0; r < kPreW; r++) {
            const int w = tid + r * kThreads;
            pre[r] = (has_next && words && w < APW) ? __ldg(reinterpret_cast<const uint32_t *>(vnext) + w) : 0u;
        }
        __syncthreads();

        // ---- a3: gridding into the folded aperture (shared-memory atomics)
        for (int a = tid; a < A; a += kThreads) {
            const uint32_t j = antj[a];
            const int jx = static_cast<int>(j & 0xFFFFu), jy = static_cast<int>(j >> 16);
            const float2 e0 = es[a * P];
            const float2 e1 = P == 2 ? es[a * P + 1] : make_float2(0.f, 0.f);
            for (int i = 0; i < KK; i++) {
                const uint32_t d = tapd[i];
                int x = jx + static_cast<int>(d & 0xFFu) - 16;
                int y = jy + static_cast<int>((d >> 8) & 0xFFu) - 16;
                x += x < 0 ? M : 0;
                x -= x >= M ? M : 0;
                y += y < 0 ? M : 0;
                y -= y >= M ? M : 0;
                const float2 w = tapw[(nker > 1 ? a * KK : 0) + i];
                float2 *cell = Gf + y * S + x;
                const float2 c0 = cmul(w, e0);
                atomicAdd(&cell->x, c0.x);
                atomicAdd(&cell->y, c0.y);
                if constexpr (P == 2) {
                    const float2 c1 = cmul(w, e1);
                    atomicAdd(&cell[M * S].x, c1.x);
                    atomicAdd(&cell[M * S].y, c1.y);
                }
            }
        }
        __syncthreads();

        // ---- a4: M x M transform, rows then columns
        fft_pass1<M, P, true>(Gf, twM);
        __syncthreads();
        fft_pass2<M, P, true>(Gf);
        __syncthreads();
        fft_pass1<M, P, false>(Gf, twM);
        __syncthreads();
        fft_pass2<M, P, false>(Gf);
        __syncthreads();

        // ---- a5, a6: products summed over time; clear the grid for the next sample
#pragma unroll
        for (int r = 0; r < NPOS; r++) {
            const int pos = tid + r * kThreads;
            if (pos < M * M) {
                const int idx = (pos / M) * S + (pos % M);
                const float2 f0 = Gf[idx];
                Gf[idx] = make_float2(0.f, 0.f);
                if constexpr (P == 2) {
                    const float2 f1 = Gf[M * S + idx];
                    Gf[M * S + idx] = make_float2(0.f, 0.f);
                    acc[r].x = fmaf(f0.x, f0.x, fmaf(f0.y, f0.y, acc[r].x));
                    acc[r].y = fmaf(f1.x, f1.x, fmaf(f1.y, f1.y, acc[r].y));
                    acc[r].z = fmaf(f0.x, f1.x, fmaf(f0.y, f1.y, acc[r].z));
                    acc[r].w = fmaf(f0.y, f1.x, fmaf(-f0.x, f1.y, acc[r].w));
                } else {
                    acc[r] = fmaf(f0.x, f0.x, fmaf(f0.y, f0.y, acc[r]));
                }
            }
        }
        if (has_next) {
            if (words) {
#pragma unroll
                for (int r = 0; r < kPreW; r++) {
                    const int w = tid + r * kThreads;
                    if (w < APW) stage[w] = pre[r];
                }
            } else {
                for (int i = tid; i < AP; i += kThreads) reinterpret_cast<uint8_t *>(stage)[i] = vnext[i];
            }
        }
        __syncthreads();
    }

    // ---- partial sums of this (channel, class, time chunk)
    float *dst = partial + (static_cast<size_t>(tau) * n_items + item) * (M * M) * (P == 2 ? 4 : 1);
#pragma unroll
    for (int r = 0; r < NPOS; r++) {
        const int pos = tid + r * kThreads;
        if (pos < M * M) {
            if constexpr (P == 2) reinterpret_cast<float4 *>(dst)[pos] = acc[r];
            else dst[pos] = acc[r];
        }
    }
}

template <int M, int P>
size_t smem_bytes(int A, int K, int nker = 1)
{
    const int AP = A * P, KK = K * K;
    size_t b = sizeof(float2) * (static_cast<size_t>(P) * M * (M + 1) + 2 * AP + static_cast<size_t>(nker) * KK + M);
    b += sizeof(uint32_t) * (A + KK + (AP + 3) / 4);
    return (b + 15) & ~static_cast<size_t>(15);
}

int pick_tau(int n_items, int T, int sms)
{
    if (T <= 1) return 1;
    // Pick the time split that balances work across SMs: an SM's throughput is
    // about the same with one or two resident CTAs, so the integration takes
    // about (CTAs on the busiest SM) x (samples per CTA + ~2 samples of set-up
    // and partial write).
    int best = 1;
    double best_cost = 1e300;
    for (int n = 1; n <= kMaxTau && n <= T; n++) {
        const long long blocks = static_cast<long long>(n_items) * n;
        const long long waves = (blocks + sms - 1) / sms;
        const double per = static_cast<double>((T + n - 1) / n) + 2.0;
        const double cost = waves * per;
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = n;
        }
    }
    return best;
}

template <int M, int P>
int launch_group(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T,
                 int *n_tau_out, cudaStream_t stream)
{
    auto kfn = fp32_image_kernel<M, P>;
    const size_t smem = smem_bytes<M, P>(plan->A, plan->K, plan->nker);
    int n_tau = choose_tau(plan, g, T);
    if (n_tau > g.tau_cap) n_tau = g.tau_cap;
    *n_tau_out = n_tau;
    const dim3 grid(static_cast<unsigned>(g.n_items * n_tau));
    kfn<<<grid, kThreads, smem, stream>>>(v, gains, plan->d_cells, plan->d_kernel, plan->K, g.d_chans, g.d_twN,
                                          plan->A, plan->C, T, g.N, g.Q1, g.n_items, n_tau, g.d_partial,
                                          plan->d_status, plan->nker, plan->d_dfreq,
                                          plan->delays ? plan->d_dtab : nullptr);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

template <int M, int P>
int prepare_group(const epic_plan_s *plan)
{
    auto kfn = fp32_image_kernel<M, P>;
    const size_t smem = smem_bytes<M, P>(plan->A, plan->K, plan->nker);
    if (const int rc = raise_dyn_smem_cap(reinterpret_cast<const void *>(kfn), smem); rc != EPIC_OK) return rc;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kThreads, smem) != cudaSuccess || per_sm < 1)
        return EPIC_ERR_UNSUPPORTED;
    return EPIC_OK;
}

template <int M, int P>
int launch_raw(const RawImage &r, const uint8_t *v, const float2 *gains, cudaStream_t stream)
{
    auto kfn = fp32_image_kernel<M, P>;
    const size_t smem = smem_bytes<M, P>(r.A, r.K);
    if (const int rc = raise_dyn_smem_cap(reinterpret_cast<const void *>(kfn), smem); rc != EPIC_OK) return rc;
    const dim3 grid(static_cast<unsigned>(r.n_items * r.n_tau));
    kfn<<<grid, kThreads, smem, stream>>>(v, gains, r.cells, r.kernel, r.K, r.chans, r.twN, r.A, r.C, r.T, r.N, r.Q1,
                                          r.n_items, r.n_tau, r.partial, r.status, 1, nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

}  // namespace

int fp32_pick_tau(int n_items, int T, int sms) { return pick_tau(n_items, T, sms); }

int choose_tau(const epic_plan_s *plan, const GroupCfg &g, int T)
{
    int n = plan->force_tau > 0                       ? plan->force_tau
            : (g.tuned_tau > 0 && g.tuned_T == T) ? g.tuned_tau
                                                  : pick_tau(g.launch_items, T, plan->sm_count);
    return std::max(1, std::min(n, g.tau_cap));
}

size_t fp32_smem_bytes(int M, int P, int A, int K)
{
    switch (M * 4 + P) {
    case 32 * 4 + 1: return smem_bytes<32, 1>(A, K);
    case 32 * 4 + 2: return smem_bytes<32, 2>(A, K);
    case 48 * 4 + 1: return smem_bytes<48, 1>(A, K);
    case 48 * 4 + 2: return smem_bytes<48, 2>(A, K);
    case 64 * 4 + 1: return smem_bytes<64, 1>(A, K);
    case 64 * 4 + 2: return smem_bytes<64, 2>(A, K);
    default: return 0;
    }
}

int launch_fp32_raw(const RawImage &r, const uint8_t *v, const float2 *gains, cudaStream_t stream)
{
    switch (r.M * 4 + r.P) {
    case 32 * 4 + 1: return launch_raw<32, 1>(r, v, gains, stream);
    case 32 * 4 + 2: return launch_raw<32, 2>(r, v, gains, stream);
    case 48 * 4 + 1: return launch_raw<48, 1>(r, v, gains, stream);
    case 48 * 4 + 2: return launch_raw<48, 2>(r, v, gains, stream);
    case 64 * 4 + 1: return launch_raw<64, 1>(r, v, gains, stream);
    case 64 * 4 + 2: return launch_raw<64, 2>(r, v, gains, stream);
    default: return EPIC_ERR_UNSUPPORTED;
    }
}

int prepare_fp32(const epic_plan_s *plan, const GroupCfg &g)
{
    if (g.reg64) return prepare_reg64(plan, g);
    switch (g.M * 4 + plan->P) {
    case 32 * 4 + 1: return prepare_group<32, 1>(plan);
    case 32 * 4 + 2: return prepare_group<32, 2>(plan);
    case 48 * 4 + 1: return prepare_group<48, 1>(plan);
    case 48 * 4 + 2: return prepare_group<48, 2>(plan);
    case 64 * 4 + 1: return prepare_group<64, 1>(plan);
    case 64 * 4 + 2: return prepare_group<64, 2>(plan);
    default: return EPIC_ERR_UNSUPPORTED;
    }
}

int launch_imaging(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau,
                   cudaStream_t s)
{
    if (g.alias && plan->force_tau == 0) return launch_alias(plan, g, v, gains, T, n_tau, s);
    if (g.tensor && !g.tc_regular) return EPIC_ERR_UNSUPPORTED;   // e.g. an image series: no fold path there
    if (g.tensor) return g.pair ? launch_tc_pair(plan, g, v, gains, T, n_tau, s) : launch_tc_dual(plan, g, v, gains, T, n_tau, s);
    if (g.reg64) return launch_reg64(plan, g, v, gains, T, n_tau, s);
    switch (g.M * 4 + plan->P) {
    case 32 * 4 + 2: return launch_group<32, 2>(plan, g, v, gains, T, n_tau, s);
    case 48 * 4 + 2: return launch_group<48, 2>(plan, g, v, gains, T, n_tau, s);
    case 64 * 4 + 2: return launch_group<64, 2>(plan, g, v, gains, T, n_tau, s);
    case 32 * 4 + 1: return launch_group<32, 1>(plan, g, v, gains, T, n_tau, s);
    case 48 * 4 + 1: return launch_group<48, 1>(plan, g, v, gains, T, n_tau, s);
    case 64 * 4 + 1: return launch_group<64, 1>(plan, g, v, gains, T, n_tau, s);
    default: return EPIC_ERR_UNSUPPORTED;
    }
}

// Launch every kernel of one integration.  With fork, the auto-power kernel
// runs on `stream` while each grid side's imaging kernel runs on its own side
// stream; each epilogue waits for its imaging kernel and for the auto-power,
// and `stream` joins all branches at the end (the shape captured into the
// plan's CUDA graph).
int image_fp32(epic_plan_s *plan, const uint8_t *v, const float2 *gains, int T, float2 *out, cudaStream_t stream,
               bool fork)
{
    if (T == 0) {
        return cudaMemsetAsync(out, 0, plan->out_floats * sizeof(float), stream) == cudaSuccess ? EPIC_OK
                                                                                                : EPIC_ERR_CUDA;
    }
    const bool autosub = !(plan->flags & EPIC_NO_AUTOSUB);
    fork = fork && !plan->side.empty();
    int rc = EPIC_OK;
    int stage = 0;
    prof_begin(plan);
    if (plan->delays && (rc = launch_delay_prep(plan, T, stream)) != EPIC_OK) return rc;
    if (fork && cudaEventRecord(plan->ev_fork, stream) != cudaSuccess) return EPIC_ERR_CUDA;
    if (autosub) {
        prof_mark(plan, stream, stage, true);
        rc = launch_autopower(plan, v, T, stream);
        prof_mark(plan, stream, stage++, false);
        if (rc != EPIC_OK) return rc;
        if (fork && cudaEventRecord(plan->ev_auto, stream) != cudaSuccess) return EPIC_ERR_CUDA;
    }
    for (size_t gi = 0; gi < plan->groups.size(); gi++) {
        const GroupCfg &g = plan->groups[gi];
        cudaStream_t s = fork ? plan->side[gi] : stream;
        if (fork && cudaStreamWaitEvent(s, plan->ev_fork, 0) != cudaSuccess) return EPIC_ERR_CUDA;
        int n_tau = 1;
        prof_mark(plan, s, stage, true);
        rc = launch_imaging(plan, g, v, gains, T, &n_tau, s);
        prof_mark(plan, s, stage++, false);
        if (rc != EPIC_OK) return rc;
        if (fork && autosub && cudaStreamWaitEvent(s, plan->ev_auto, 0) != cudaSuccess) return EPIC_ERR_CUDA;
        prof_mark(plan, s, stage, true);
        if (autosub && plan->nker > 1) rc = launch_auto_rho(plan, g, gains, s);
        if (rc == EPIC_OK) rc = launch_epilogue(plan, g, gains, T, n_tau, out, s);
        prof_mark(plan, s, stage++, false);
        if (rc != EPIC_OK) return rc;
        if (fork) {
            if (cudaEventRecord(plan->ev_join[gi], s) != cudaSuccess) return EPIC_ERR_CUDA;
            if (cudaStreamWaitEvent(stream, plan->ev_join[gi], 0) != cudaSuccess) return EPIC_ERR_CUDA;
        }
    }
    return rc;
}

}  // namespace epic

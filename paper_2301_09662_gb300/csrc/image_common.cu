// Stages shared by every arithmetic form: the exact integer auto-power (a7)
// and the epilogue that sums the partial images, subtracts the
// autocorrelation term and writes the shifted output (a8).
//
// Autocorrelation removal (Sec. 2.2): the a = b terms of F_p F_q^* are
// e~_ap e~_aq^* |W^(l)|^2 for every antenna, so their sum over the integration
// is A_pq |W^(l)|^2 with A_pq = sum_a g_ap g_aq^* sum_t e_ap e_aq^*.  The inner
// time sum is exact in int32 (|e e^*| components <= 128, T <= 10^5); the
// antenna sum and the subtraction run in FP64 because the auto term can be
// much larger than what is left after it is removed.
#include <algorithm>

#include "epic_internal.cuh"

namespace epic {
namespace {

__device__ __forceinline__ void ci4_parts(uint32_t b, int &re, int &im)
{
    re = static_cast<int>(static_cast<int8_t>(b & 0xF0u)) >> 4;
    im = static_cast<int>(static_cast<int8_t>((b << 4) & 0xF0u)) >> 4;
}

// grid (C, n_chunks): per antenna, integer sums over one time chunk
//   [0] sum |e_X|^2   [1] sum |e_Y|^2   [2] Re sum e_X e_Y^*   [3] Im sum e_X e_Y^*
__global__ void __launch_bounds__(kThreads)
autopower_kernel(const uint8_t *__restrict__ v, int T, int C, int A, int P, int n_chunks,
                 size_t chunk_stride, int *__restrict__ autoint)
{
    const int c = blockIdx.x;
    const int chunk = blockIdx.y;
    const int t0 = static_cast<int>(static_cast<long long>(T) * chunk / n_chunks);
    const int t1 = static_cast<int>(static_cast<long long>(T) * (chunk + 1) / n_chunks);
    for (int a = threadIdx.x; a < A; a += blockDim.x) {
        int sxx = 0, syy = 0, sxyr = 0, sxyi = 0;
        for (int t = t0; t < t1; t++) {
            const uint8_t *row = v + (static_cast<size_t>(t) * C + c) * A * P + static_cast<size_t>(a) * P;
            int xr, xi;
            ci4_parts(row[0], xr, xi);
            sxx += xr * xr + xi * xi;
            if (P == 2) {
                int yr, yi;
                ci4_parts(row[1], yr, yi);
                syy += yr * yr + yi * yi;
                sxyr += xr * yr + xi * yi;
                sxyi += xi * yr - xr * yi;
            }
        }
        // chunk_stride 0: every chunk adds into one sum; else one sum per chunk (image series)
        int *dst = autoint + chunk * chunk_stride + (static_cast<size_t>(c) * A + a) * 4;
        atomicAdd(dst + 0, sxx);
        if (P == 2) {
            atomicAdd(dst + 1, syy);
            atomicAdd(dst + 2, sxyr);
            atomicAdd(dst + 3, sxyi);
        }
    }
}

// grid (pixel tiles, group channels).  Partial layout written by the imaging
// kernels: [tau][item][pos][NPF] with item = ci * Q + (hy * Q1 + hx) and
// pos = py * M + px, where folded frequency m sits at digit position
// up (R2 (m mod R1) + m / R1) (R1 = 1, R2 = M for natural order; up = 2 when a
// side-32 grid was transformed zero-padded to 64 points, whose even
// frequencies are the 32-point transform).
template <int M, int P>
__global__ void __launch_bounds__(kThreads)
epilogue_kernel(const float *__restrict__ partial, int n_tau, int n_items, int N, int Q1, int R1, int R2,
                const int *__restrict__ chans, const long long *__restrict__ out_off,
                const double *__restrict__ wpow, const int *__restrict__ autoint,
                const float2 *__restrict__ gains, int A, int T, unsigned flags, float2 *__restrict__ out,
                size_t auto_stride, long long out_stride,
                const double2 *__restrict__ Yauto, const double2 *__restrict__ tw64, int K, int up)
{
    // blockIdx.z = image: it sums time chunks [z n_tau, (z + 1) n_tau) and uses
    // the auto sums and output block of index z (one image unless a series)
    const int img = blockIdx.z;
    partial += static_cast<size_t>(img) * n_tau * n_items * (M * M) * (P == 2 ? 4 : 1);
    autoint += img * auto_stride;
    out += img * out_stride;
    constexpr int NPF = P == 2 ? 4 : 1;
    constexpr int NP = P == 2 ? 4 : 1;
    const int ci = blockIdx.y;
    const int c = chans[ci];
    const bool autosub = !(flags & EPIC_NO_AUTOSUB);

    // A_pq(c) in FP64, reduced in a fixed order (deterministic)
    __shared__ double red[kThreads / 32][6];
    __shared__ double apq[6];   // XX, YY, Re XY, Im XY (YX = conj XY)
    const bool ant_kernels = Yauto != nullptr;   // auto image from the per-antenna auto-correlation grid
    if (autosub && !ant_kernels) {
        double s[6] = {0, 0, 0, 0, 0, 0};
        for (int a = threadIdx.x; a < A; a += kThreads) {
            const int *ia = autoint + (static_cast<size_t>(c) * A + a) * 4;
            double gxr = 1, gxi = 0, gyr = 1, gyi = 0;
            if (gains) {
                const float2 gx = gains[(static_cast<size_t>(c) * A + a) * P];
                gxr = gx.x;
                gxi = gx.y;
                if (P == 2) {
                    const float2 gy = gains[(static_cast<size_t>(c) * A + a) * P + 1];
                    gyr = gy.x;
                    gyi = gy.y;
                }
            }
            s[0] += (gxr * gxr + gxi * gxi) * static_cast<double>(ia[0]);
            if (P == 2) {
                s[1] += (gyr * gyr + gyi * gyi) * static_cast<double>(ia[1]);
                // g_x g_y^* (I_re + i I_im)
                const double pr = gxr * gyr + gxi * gyi, pi = gxi * gyr - gxr * gyi;
                s[2] += pr * ia[2] - pi * ia[3];
                s[3] += pr * ia[3] + pi * ia[2];
            }
        }
        // fixed-order tree: within each warp by shuffles, then the warps' sums by thread 0..3
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_down_sync(0xffffffffu, s[k], o);
        if ((threadIdx.x & 31) == 0)
            for (int k = 0; k < 4; k++) red[threadIdx.x >> 5][k] = s[k];
        __syncthreads();
        if (threadIdx.x < 4) {
            double tot = 0;
            for (int i = 0; i < kThreads / 32; i++) tot += red[i][threadIdx.x];
            apq[threadIdx.x] = tot;
        }
        __syncthreads();
    }

    const double scale = ((flags & EPIC_MEAN) && T > 0) ? 1.0 / T : 1.0;
    const int NN = N * N;
    const int Q = Q1 * Q1;
    float2 *oc = out + out_off[ci];
    for (int pix = blockIdx.x * kThreads + threadIdx.x; pix < NN; pix += gridDim.x * kThreads) {
        const int i = pix / N, j = pix % N;
        const int ly = (i + N / 2) % N, lx = (j + N / 2) % N;   // (i - N/2) mod N
        const int hx = lx % Q1, mx = lx / Q1, hy = ly % Q1, my = ly / Q1;
        const int item = ci * Q + hy * Q1 + hx;
        const int px = up * (R2 * (mx % R1) + mx / R1), py = up * (R2 * (my % R1) + my / R1);
        const size_t pos = static_cast<size_t>(py) * M + px;
        // time chunks added in time order as compensated FP32 (hi, lo) pairs: TwoSum keeps
        // hi + lo equal to the exact running sum up to the roundings of lo, far below FP32;
        // FP64 only for the pair and the auto-term subtraction (FP64 is ~2 ops/clock/SM here)
        float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
        auto two_sum = [](float &h, float &l, float x) {
            const float t = h + x;
            const float bp = t - h;
            l += (h - (t - bp)) + (x - bp);
            h = t;
        };
        const float *src0 = partial + (static_cast<size_t>(item) * (M * M) + pos) * NPF;
        const size_t tau_stride = static_cast<size_t>(n_items) * (M * M) * NPF;
        for (int tau = 0; tau < n_tau; tau++) {
            const float *src = src0 + tau * tau_stride;
            if constexpr (P == 2) {
                const float4 f = __ldg(reinterpret_cast<const float4 *>(src));
                two_sum(hi[0], lo[0], f.x);
                two_sum(hi[1], lo[1], f.y);
                two_sum(hi[2], lo[2], f.z);
                two_sum(hi[3], lo[3], f.w);
            } else {
                two_sum(hi[0], lo[0], __ldg(src));
            }
        }
        double s[4];
#pragma unroll
        for (int k = 0; k < 4; k++) s[k] = static_cast<double>(hi[k]) + static_cast<double>(lo[k]);
        const double w = wpow[pix];
        if (ant_kernels) {
            if (autosub) {
                // auto_pq(l) = sum_{rho_y} Y_pq(rho_y, l_x) exp(+2 pi i rho_y l_y / N)
                const int R = 2 * K - 1;
                const int lyv = i - N / 2;
                double ax = 0, ay = 0, axr = 0, axi = 0;
                for (int ry = 0; ry < R; ry++) {
                    const int m = (((ry - (K - 1)) * lyv) % N + N) % N;
                    const double2 tw = tw64[m];
                    const double2 y0 = Yauto[(static_cast<size_t>(ci) * 3 * R + ry) * N + j];
                    ax += y0.x * tw.x - y0.y * tw.y;
                    if (P == 2) {
                        const double2 y1 = Yauto[(static_cast<size_t>(ci) * 3 * R + R + ry) * N + j];
                        const double2 y2 = Yauto[(static_cast<size_t>(ci) * 3 * R + 2 * R + ry) * N + j];
                        ay += y1.x * tw.x - y1.y * tw.y;
                        axr += y2.x * tw.x - y2.y * tw.y;
                        axi += y2.x * tw.y + y2.y * tw.x;
                    }
                }
                s[0] -= ax;
                if (P == 2) {
                    s[1] -= ay;
                    s[2] -= axr;
                    s[3] -= axi;
                }
            }
        } else if (flags & EPIC_KERNEL_TAPER) {
            // point-gridded sums: subtract the bare autos, then apply |W^(l)|^2
            for (int k = 0; k < (P == 2 ? 4 : 1); k++) s[k] = (s[k] - (autosub ? apq[k] : 0.0)) * w;
        } else if (autosub) {
            s[0] -= apq[0] * w;
            if (P == 2) {
                s[1] -= apq[1] * w;
                s[2] -= apq[2] * w;
                s[3] -= apq[3] * w;
            }
        }
        if (P == 2 && (flags & EPIC_STOKES)) {
            // I = XX + YY, Q = XX - YY, U = 2 Re XY, V = 2 Im XY
            const double st[4] = {s[0] + s[1], s[0] - s[1], 2.0 * s[2], 2.0 * s[3]};
            for (int k = 0; k < 4; k++) oc[k * NN + pix] = make_float2(static_cast<float>(st[k] * scale), 0.f);
            continue;
        }
        oc[pix] = make_float2(static_cast<float>(s[0] * scale), 0.f);
        if constexpr (NP == 4) {
            oc[NN + pix] = make_float2(static_cast<float>(s[1] * scale), 0.f);
            oc[2 * NN + pix] = make_float2(static_cast<float>(s[2] * scale), static_cast<float>(s[3] * scale));
            oc[3 * NN + pix] = make_float2(static_cast<float>(s[2] * scale), static_cast<float>(-s[3] * scale));
        }
    }
}

// Per-antenna kernels (Eq. 3's W_a): the a = b terms of F_p F_q^* sum to
// sum_a A_a,pq |W^_a(l)|^2 = sum_rho X_pq(rho) exp(+2 pi i rho.l / N) with the
// auto-correlation grid X_pq(rho) = sum_a A_a,pq B_aa(rho),
// B_aa = W_a (x) W_a^* on the (2K-1)^2 offsets rho (Sec. 2.2's "auto-correlation
// grids from individual antenna voltages").  One block per (channel, product):
// X in FP64, then the l_x half of the separable transform,
// Y(rho_y, l_x) = sum_rho_x X(rho_x, rho_y) exp(+2 pi i rho_x l_x / N), for the
// epilogue to finish along l_y.
__global__ void __launch_bounds__(kThreads)
auto_rho_kernel(const int *__restrict__ autoint, const float2 *__restrict__ gains,
                const double2 *__restrict__ bauto, const int *__restrict__ chans, const double2 *__restrict__ tw64,
                int A, int P, int K, int N, double2 *__restrict__ Y)
{
    extern __shared__ double2 X[];     // [R][R]
    const int R = 2 * K - 1, RR = R * R;
    const int ci = blockIdx.x, pq = blockIdx.y;
    const int c = chans[ci];
    for (int rho = threadIdx.x; rho < RR; rho += blockDim.x) {
        double xr = 0, xi = 0;
        for (int a = 0; a < A; a++) {
            const int *ia = autoint + (static_cast<size_t>(c) * A + a) * 4;
            double ar, ai;
            double gxr = 1, gxi = 0, gyr = 1, gyi = 0;
            if (gains) {
                const float2 gx = gains[(static_cast<size_t>(c) * A + a) * P];
                gxr = gx.x;
                gxi = gx.y;
                if (P == 2) {
                    const float2 gy = gains[(static_cast<size_t>(c) * A + a) * P + 1];
                    gyr = gy.x;
                    gyi = gy.y;
                }
            }
            if (pq == 0) {
                ar = (gxr * gxr + gxi * gxi) * ia[0];
                ai = 0;
            } else if (pq == 1) {
                ar = (gyr * gyr + gyi * gyi) * ia[1];
                ai = 0;
            } else {
                const double pr = gxr * gyr + gxi * gyi, pi = gxi * gyr - gxr * gyi;
                ar = pr * ia[2] - pi * ia[3];
                ai = pr * ia[3] + pi * ia[2];
            }
            const double2 b = bauto[static_cast<size_t>(a) * RR + rho];
            xr += ar * b.x - ai * b.y;
            xi += ar * b.y + ai * b.x;
        }
        X[rho] = make_double2(xr, xi);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < R * N; e += blockDim.x) {
        const int ry = e / N, j = e % N;
        const int lx = j - N / 2;
        double yr = 0, yi = 0;
        for (int rx = 0; rx < R; rx++) {
            const int m = (((rx - (K - 1)) * lx) % N + N) % N;
            const double2 tw = tw64[m], x = X[ry * R + rx];
            yr += x.x * tw.x - x.y * tw.y;
            yi += x.x * tw.y + x.y * tw.x;
        }
        Y[(static_cast<size_t>(ci) * 3 * R + static_cast<size_t>(pq) * R + ry) * N + j] = make_double2(yr, yi);
    }
}

template <int M, int P>
int launch_epi(epic_plan_s *plan, const GroupCfg &g, const float2 *gains, int T, int n_tau, float2 *out,
               cudaStream_t stream)
{
    const int NN = g.N * g.N;
    // 8 pixels a thread: fewer blocks, each reducing the channel's auto-power sums once
    const int tiles = (NN + kThreads * 8 - 1) / (kThreads * 8);
    const dim3 grid(static_cast<unsigned>(tiles), static_cast<unsigned>(g.n_chan));
    epilogue_kernel<M, P><<<grid, kThreads, 0, stream>>>(g.d_partial, n_tau, g.n_items, g.N, g.Q1, g.R1, g.R2,
                                                         g.d_chans,
                                                         g.d_out_off, g.d_wpow, plan->d_autoint, gains, plan->A, T,
                                                         plan->flags, out, 0, 0,
                                                         plan->nker > 1 ? g.d_Y : nullptr, g.d_tw64, plan->K, g.up);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

template <int M, int P>
int launch_epi_raw(const RawImage &r, const float2 *gains, float2 *out, cudaStream_t stream)
{
    const int NN = r.N * r.N;
    const int tiles = (NN + kThreads * 4 - 1) / (kThreads * 4);
    const dim3 grid(static_cast<unsigned>(tiles), static_cast<unsigned>(r.C));
    epilogue_kernel<M, P><<<grid, kThreads, 0, stream>>>(r.partial, r.n_tau, r.n_items, r.N, r.Q1, 8, M / 8,
                                                         r.chans,
                                                         r.out_off, r.wpow, r.autoint, gains, r.A, r.T, r.flags,
                                                         out, 0, 0, nullptr, nullptr, 0, 1);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

// Per (t, antenna): the FP64 part of the delay phase, once per integration,
// so the imaging kernels need only FP32 (Sec. 2.2 delay correction).
__global__ void delay_prep_kernel(const double *__restrict__ delays, int n, double f_ref, float4 *__restrict__ tab)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double tau = delays[i];
        double b = f_ref * tau;
        b -= rint(b);
        const float hi = static_cast<float>(tau);
        const float lo = static_cast<float>(tau - static_cast<double>(hi));
        tab[i] = make_float4(static_cast<float>(b), hi, lo, 0.f);
    }
}

}  // namespace

int launch_autopower_raw(const RawImage &r, const uint8_t *v, int sm_count, cudaStream_t stream)
{
    if (r.T == 0) return EPIC_OK;
    int chunks = (4 * sm_count + r.C - 1) / r.C;
    if (chunks > r.T) chunks = r.T;
    if (chunks < 1) chunks = 1;
    const dim3 grid(static_cast<unsigned>(r.C), static_cast<unsigned>(chunks));
    autopower_kernel<<<grid, kThreads, 0, stream>>>(v, r.T, r.C, r.A, r.P, chunks, 0, r.autoint);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

int launch_epilogue_raw(const RawImage &r, const float2 *gains, float2 *out, cudaStream_t stream)
{
    switch (r.M * 4 + r.P) {
    case 32 * 4 + 1: return launch_epi_raw<32, 1>(r, gains, out, stream);
    case 32 * 4 + 2: return launch_epi_raw<32, 2>(r, gains, out, stream);
    case 48 * 4 + 1: return launch_epi_raw<48, 1>(r, gains, out, stream);
    case 48 * 4 + 2: return launch_epi_raw<48, 2>(r, gains, out, stream);
    case 64 * 4 + 1: return launch_epi_raw<64, 1>(r, gains, out, stream);
    case 64 * 4 + 2: return launch_epi_raw<64, 2>(r, gains, out, stream);
    default: return EPIC_ERR_UNSUPPORTED;
    }
}

template <int M, int P>
int launch_epi_series(epic_plan_s *plan, const GroupCfg &g, const float2 *gains, int spi, int n_img, float2 *out,
                      cudaStream_t stream)
{
    const int NN = g.N * g.N;
    const int tiles = (NN + kThreads * 4 - 1) / (kThreads * 4);
    const dim3 grid(static_cast<unsigned>(tiles), static_cast<unsigned>(g.n_chan), static_cast<unsigned>(n_img));
    epilogue_kernel<M, P><<<grid, kThreads, 0, stream>>>(g.d_partial, 1, g.n_items, g.N, g.Q1, g.R1, g.R2, g.d_chans,
                                                         g.d_out_off, g.d_wpow, plan->d_autoint, gains, plan->A, spi,
                                                         plan->flags, out,
                                                         static_cast<size_t>(plan->C) * plan->A * 4,
                                                         static_cast<long long>(plan->out_floats / 2), nullptr,
                                                         nullptr, 0, g.up);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

int launch_autopower_series(epic_plan_s *plan, const uint8_t *v, int spi, int n_img, cudaStream_t stream)
{
    const size_t stride = static_cast<size_t>(plan->C) * plan->A * 4;
    if (cudaMemsetAsync(plan->d_autoint, 0, stride * n_img * sizeof(int), stream) != cudaSuccess) return EPIC_ERR_CUDA;
    const dim3 grid(static_cast<unsigned>(plan->C), static_cast<unsigned>(n_img));
    autopower_kernel<<<grid, kThreads, 0, stream>>>(v, spi * n_img, plan->C, plan->A, plan->P, n_img, stride,
                                                    plan->d_autoint);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

int launch_epilogue_series(epic_plan_s *plan, const GroupCfg &g, const float2 *gains, int spi, int n_img,
                           float2 *out, cudaStream_t stream)
{
    switch (g.M * 4 + plan->P) {
    case 32 * 4 + 1: return launch_epi_series<32, 1>(plan, g, gains, spi, n_img, out, stream);
    case 32 * 4 + 2: return launch_epi_series<32, 2>(plan, g, gains, spi, n_img, out, stream);
    case 48 * 4 + 1: return launch_epi_series<48, 1>(plan, g, gains, spi, n_img, out, stream);
    case 48 * 4 + 2: return launch_epi_series<48, 2>(plan, g, gains, spi, n_img, out, stream);
    case 64 * 4 + 1: return launch_epi_series<64, 1>(plan, g, gains, spi, n_img, out, stream);
    case 64 * 4 + 2: return launch_epi_series<64, 2>(plan, g, gains, spi, n_img, out, stream);
    default: return EPIC_ERR_UNSUPPORTED;
    }
}

int launch_delay_prep(epic_plan_s *plan, int T, cudaStream_t stream)
{
    const int n = T * plan->A;
    if (n <= 0) return EPIC_OK;
    const int blocks = std::min((n + kThreads - 1) / kThreads, 4 * plan->sm_count);
    delay_prep_kernel<<<blocks, kThreads, 0, stream>>>(plan->delays, n, plan->f_ref, plan->d_dtab);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

int launch_auto_rho(epic_plan_s *plan, const GroupCfg &g, const float2 *gains, cudaStream_t stream)
{
    const int R = 2 * plan->K - 1;
    const dim3 grid(static_cast<unsigned>(g.n_chan), static_cast<unsigned>(plan->P == 2 ? 3 : 1));
    auto_rho_kernel<<<grid, kThreads, sizeof(double2) * R * R, stream>>>(
        plan->d_autoint, gains, plan->d_bauto, g.d_chans, g.d_tw64, plan->A, plan->P, plan->K, g.N, g.d_Y);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

int launch_autopower(epic_plan_s *plan, const uint8_t *v, int T, cudaStream_t stream)
{
    const size_t n = static_cast<size_t>(plan->C) * plan->A * 4;
    if (cudaMemsetAsync(plan->d_autoint, 0, n * sizeof(int), stream) != cudaSuccess) return EPIC_ERR_CUDA;
    if (T == 0) return EPIC_OK;
    int chunks = (4 * plan->sm_count + plan->C - 1) / plan->C;
    if (chunks > T) chunks = T;
    if (chunks < 1) chunks = 1;
    const dim3 grid(static_cast<unsigned>(plan->C), static_cast<unsigned>(chunks));
    autopower_kernel<<<grid, kThreads, 0, stream>>>(v, T, plan->C, plan->A, plan->P, chunks, 0, plan->d_autoint);
    return cudaGetLastError() == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

int launch_epilogue(epic_plan_s *plan, const GroupCfg &g, const float2 *gains, int T, int n_tau, float2 *out,
                    cudaStream_t stream)
{
    if (plan->P == 2) {
        switch (g.M) {
        case 32: return launch_epi<32, 2>(plan, g, gains, T, n_tau, out, stream);
        case 48: return launch_epi<48, 2>(plan, g, gains, T, n_tau, out, stream);
        case 64: return launch_epi<64, 2>(plan, g, gains, T, n_tau, out, stream);
        }
    } else {
        switch (g.M) {
        case 32: return launch_epi<32, 1>(plan, g, gains, T, n_tau, out, stream);
        case 48: return launch_epi<48, 1>(plan, g, gains, T, n_tau, out, stream);
        case 64: return launch_epi<64, 1>(plan, g, gains, T, n_tau, out, stream);
        }
    }
    return EPIC_ERR_UNSUPPORTED;
}

}  // namespace epic

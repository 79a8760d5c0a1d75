// epic_image_static: one FP32 integration with no device allocation at all.
//
// Who needs this.  epic_plan allocates its tables and workspace with
// cudaMalloc.  Some programs that want an image cannot make that call: a
// telescope pipeline whose GPU memory is all reserved up front by its own pool
// allocator (a stray cudaMalloc would fail or fragment it), a real-time capture
// loop in which cudaMalloc / cudaFree would quietly synchronise the whole
// device and stall the stream that must keep pace with the antennas, or a
// plug-in that may not leave allocations behind in its host process.  Such a
// caller still owns its input voltages, gains and output image; this entry
// point takes exactly those and keeps everything else it needs -- the
// antenna-to-cell map, the kernel and its image, twiddles, the exact integer
// auto-power sums and the partial image sums -- in one fixed-size array in
// device global memory that the library declares at file scope.
//
// The array costs every GPU that loads libepic kStaticScratchBytes of device
// memory until the process exits.  All calls share it: a call overwrites what
// the previous one left (the parts that must start at zero are cleared on the
// call's stream), so calls whose work overlaps on the GPU -- on different
// streams, or from different host threads -- race and must be ordered by the
// caller.
#include <cstring>
#include <mutex>
#include <vector>

#include "epic_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = static_cast<size_t>(32) << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

// File-scope scratch: tables first, then auto-power sums, then partial images.
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void *g_scratch_dev[kMaxDevices] = {};   // device address of g_static_scratch per device

// Device address of the scratch array on the current device.  In host code the
// name g_static_scratch is only a host-side stand-in, so the real address is
// asked for once per device, with that device current.
int scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return EPIC_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return EPIC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return EPIC_ERR_CUDA;
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return EPIC_OK;
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

int fold_for(int n)
{
    switch (n) {
    case 32: return 1;
    case 64: return 1;
    case 96: return 2;
    case 128: return 2;
    default: return 0;
    }
}

}  // namespace

extern "C" int epic_image_static(const double *ant_xy_m, int n_ant, int n_pol, const float *kernel_c64, int K,
                                 int grid_n, const double *freq_hz, int n_chan, double du, const uint8_t *ci4,
                                 const float *gains_c64, int n_spectra, unsigned flags, float *out_c64,
                                 void *cuda_stream)
{
    using namespace epic;
    if (!ant_xy_m || !kernel_c64 || !freq_hz || !out_c64) return EPIC_ERR_ARG;
    if (n_ant < 1 || (n_pol != 1 && n_pol != 2) || K < 1 || (K % 2) == 0 || K > kMaxK || n_chan < 1 ||
        !(du > 0.0) || du > 0.5 || n_spectra < 0 || (n_spectra > 0 && !ci4))
        return EPIC_ERR_ARG;
    if (flags & ~(EPIC_MEAN | EPIC_NO_AUTOSUB)) return EPIC_ERR_ARG;
    const int Q1 = fold_for(grid_n);
    if (Q1 == 0) return EPIC_ERR_UNSUPPORTED;
    if (static_cast<long long>(n_ant) * n_pol > kMaxAP) return EPIC_ERR_UNSUPPORTED;
    for (int c = 0; c < n_chan; c++)
        if (!(freq_hz[c] > 0.0)) return EPIC_ERR_ARG;
    auto stream = static_cast<cudaStream_t>(cuda_stream);

    // ---- host tables
    std::vector<int> gn(n_chan, grid_n);
    std::vector<short2> cells;
    int rc = host_cell_map(ant_xy_m, n_ant, freq_hz, n_chan, gn.data(), du, K, cells);
    if (rc != EPIC_OK) return rc;
    const int N = grid_n, M = N / Q1, NP = n_pol == 2 ? 4 : 1, NPF = n_pol == 2 ? 4 : 1;
    std::vector<double> wpow;
    host_kernel_power(kernel_c64, K, N, wpow);

    // ---- scratch layout (all offsets 256-byte aligned)
    size_t off = 0;
    const size_t o_status = off;   off = align256(off + sizeof(int));
    const size_t o_cells = off;    off = align256(off + cells.size() * sizeof(short2));
    const size_t o_kernel = off;   off = align256(off + static_cast<size_t>(K) * K * sizeof(float2));
    const size_t o_chans = off;    off = align256(off + static_cast<size_t>(n_chan) * sizeof(int));
    const size_t o_outoff = off;   off = align256(off + static_cast<size_t>(n_chan) * sizeof(long long));
    const size_t o_wpow = off;     off = align256(off + wpow.size() * sizeof(double));
    const size_t o_twN = off;      off = align256(off + static_cast<size_t>(N) * sizeof(float2));
    const size_t table_bytes = off;
    const size_t o_auto = off;     off = align256(off + static_cast<size_t>(n_chan) * n_ant * 4 * sizeof(int));
    const size_t o_partial = off;
    const int n_items = n_chan * Q1 * Q1;
    const size_t per_tau = static_cast<size_t>(n_items) * M * M * NPF * sizeof(float);
    if (o_partial + per_tau > kStaticScratchBytes) return EPIC_ERR_TOO_LARGE;

    void *base = nullptr;
    rc = scratch_address(&base);
    if (rc != EPIC_OK) return rc;
    auto *scratch = static_cast<unsigned char *>(base);

    if (n_spectra == 0)
        return cudaMemsetAsync(out_c64, 0, static_cast<size_t>(n_chan) * NP * N * N * 2 * sizeof(float), stream) ==
                       cudaSuccess
                   ? EPIC_OK
                   : EPIC_ERR_CUDA;

    std::vector<unsigned char> img(table_bytes, 0);
    std::memcpy(img.data() + o_cells, cells.data(), cells.size() * sizeof(short2));
    std::memcpy(img.data() + o_kernel, kernel_c64, static_cast<size_t>(K) * K * sizeof(float2));
    auto *chans = reinterpret_cast<int *>(img.data() + o_chans);
    auto *outoff = reinterpret_cast<long long *>(img.data() + o_outoff);
    for (int c = 0; c < n_chan; c++) {
        chans[c] = c;
        outoff[c] = static_cast<long long>(c) * NP * N * N;
    }
    std::memcpy(img.data() + o_wpow, wpow.data(), wpow.size() * sizeof(double));
    auto *tw = reinterpret_cast<float2 *>(img.data() + o_twN);
    for (int k = 0; k < N; k++) {
        const double ang = 2.0 * M_PI * k / N;
        tw[k] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
    }
    // pageable source: the call returns once the bytes are staged, so img may go
    if (cudaMemcpyAsync(scratch, img.data(), table_bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return EPIC_ERR_CUDA;
    if (cudaMemsetAsync(scratch + o_auto, 0, o_partial - o_auto, stream) != cudaSuccess) return EPIC_ERR_CUDA;

    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return EPIC_ERR_CUDA;

    RawImage r;
    r.A = n_ant;
    r.P = n_pol;
    r.C = n_chan;
    r.K = K;
    r.N = N;
    r.M = M;
    r.Q1 = Q1;
    r.n_items = n_items;
    r.T = n_spectra;
    r.flags = flags;
    const size_t fit = (kStaticScratchBytes - o_partial) / per_tau;
    int n_tau = fp32_pick_tau(n_items, n_spectra, sms);
    if (static_cast<size_t>(n_tau) > fit) n_tau = static_cast<int>(fit);
    r.n_tau = n_tau < 1 ? 1 : n_tau;
    r.cells = reinterpret_cast<const short2 *>(scratch + o_cells);
    r.kernel = reinterpret_cast<const float2 *>(scratch + o_kernel);
    r.chans = reinterpret_cast<const int *>(scratch + o_chans);
    r.out_off = reinterpret_cast<const long long *>(scratch + o_outoff);
    r.wpow = reinterpret_cast<const double *>(scratch + o_wpow);
    r.twN = reinterpret_cast<const float2 *>(scratch + o_twN);
    r.autoint = reinterpret_cast<int *>(scratch + o_auto);
    r.partial = reinterpret_cast<float *>(scratch + o_partial);
    r.status = reinterpret_cast<int *>(scratch + o_status);

    const auto *gains = reinterpret_cast<const float2 *>(gains_c64);
    if (!(flags & EPIC_NO_AUTOSUB)) {
        rc = launch_autopower_raw(r, ci4, sms, stream);
        if (rc != EPIC_OK) return rc;
    }
    rc = launch_fp32_raw(r, ci4, gains, stream);
    if (rc != EPIC_OK) return rc;
    return launch_epilogue_raw(r, gains, reinterpret_cast<float2 *>(out_c64), stream);
}

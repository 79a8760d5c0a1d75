// Internal declarations shared by the libepic translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "epic.h"

namespace epic {

constexpr double kC0 = 299792458.0;
constexpr int kThreads = 256;          // threads per CTA of the imaging kernels
constexpr int kMaxTau = 64;            // most time chunks one channel item is split into
constexpr int kMaxK = 15;
constexpr int kMaxAP = 4096;           // n_ant * n_pol handled by one CTA's staging
constexpr int kPairHelpers = 3;        // pair kernel (tc_pair128.cu): gridding-only warps beside its 8 TMEM warps
constexpr int kPairGatherWarps = 8 + kPairHelpers;

// How one grid side N is imaged by the FP32 kernel: the sky is split into
// Q1 x Q1 pixel classes l = (Q1 m + h) and each CTA owns one class, so it grids
// into an M x M folded aperture (M = N / Q1) and runs an M x M transform.
// One 4+4-bit complex voltage byte: Re = the high nibble, Im = the low nibble,
// both two's complement (-8..7; Sec. 3's "4+4 complex integers", reading 1).
__device__ __forceinline__ float2 ci4_decode(uint32_t b)
{
    const int re = static_cast<int>(static_cast<int8_t>(b & 0xF0u)) >> 4;
    const int im = static_cast<int>(static_cast<int8_t>((b << 4) & 0xF0u)) >> 4;
    return make_float2(static_cast<float>(re), static_cast<float>(im));
}

// How the pair kernel's lists are dealt (build_pair_tables): the 8 TMEM warps start with
// tmem_load work units (~37 cycles each) for their conversion and products, and a TMEM warp's
// share is split so that about first_pct percent is gridded under class 0's column stage.
struct PairSchedule {
    int tmem_load = 90;
    int first_pct = 80;
};

struct GroupCfg {
    int N = 0, M = 0, Q1 = 1, Q = 1;
    int n_chan = 0;
    std::vector<int> chans;            // plan channel indices in this group
    int *d_chans = nullptr;            // device copy of chans
    long long *d_out_off = nullptr;    // device: output offset (complex elements) per group channel
    double *d_wpow = nullptr;          // device: |W^(l)|^2 on the shifted [N][N] layout
    double2 *d_tw64 = nullptr;         // per-antenna kernels: exp(+2 pi i k / N) in FP64
    double2 *d_Y = nullptr;            // per-antenna kernels: [n_chan][3][2K-1][N] partial auto images
    float2 *d_twN = nullptr;           // device: exp(+2 pi i k / N), k < N
    int n_items = 0;                   // n_chan * Q
    int tau_cap = 1;                   // time chunks the partial buffer holds
    float *d_partial = nullptr;        // device: [tau_cap][n_items][M*M][NPF] partial sums
    // partial-sum pixel order: folded frequency m sits at up (R2 (m mod R1) + m / R1)
    int R1 = 1, R2 = 1;
    int up = 1;                        // 2: a side-32 group transformed zero-padded to 64 points (tensor form)
    // register-transform kernels (fold side 64 or 48): gridding tables and samples per iteration
    bool reg64 = false;
    bool tensor = false;               // a tensor plan's group that folds to 64 runs the tensor kernel
    bool tc_regular = true;            // the tensor kernel's per-antenna buffers fit (else only the fold path)
    int tuned_tau = 0, tuned_T = -1;   // time chunks epic_autotune measured fastest for T = tuned_T
    int ts = 1;
    int rmax = 0;
    uint32_t *d_sched = nullptr;       // device: [n_chan][8 warps][rmax][32] segment descriptors
    uint16_t *d_first = nullptr;       // device (tensor plans): per descriptor, taps that write their cell first
    int *d_nrounds = nullptr;          // device: [n_chan][8] rounds per warp
    unsigned long long *d_rowmask = nullptr;  // device: [n_chan] folded rows touched by any footprint
    uint32_t *d_gtab = nullptr;        // device (FP32 register kernel): gather table, build_gather_table
    int4 *d_gidx = nullptr;            // device: [n_chan][8 warps] (zero offset, zero steps, batch offset, batches)
    int2 *d_gchan = nullptr;           // device: [n_chan] (block start, block words)
    int gwords = 0;                    // largest channel block (words)
    bool gstage = false;               // blocks staged in shared memory
    // large grid sides (8 x 8 pixel classes): grid once per (channel, sample) into the occupied
    // alias blocks, fold all classes with one 8 x 8 DFT per folded cell (alias_fold_kernel), then
    // transform each class's loaded grid (fp32_fold64_kernel), in time batches of alias_tb samples
    bool alias = false;
    int alias_tb = 0;
    float2 *d_gf = nullptr;            // device: [alias_tb][n_items][P][64][64] folded grids
    short2 *d_j0 = nullptr;            // device: [n_chan] first occupied alias block (x, y)
    uint32_t *d_bseg = nullptr;        // device: footprint rows (a << 8 | dyi) per (channel, 8-row band)
    int *d_boff = nullptr;             // device: [n_chan * 8 + 1] offsets into d_bseg
    // grid sides 128 and 64 in a tensor plan: the pair kernel (tc_pair128.cu)
    bool pair = false;
    PairSchedule psched;               // how its lists are dealt to the warps (epic_autotune measures a few)
    std::vector<uint32_t> h_tab32;     // host: the FP32 gather table of the group (kept to re-deal the lists)
    std::vector<int4> h_idx32;
    std::vector<int2> h_chan32;
    size_t ptab_n = 0, pidx_n = 0;     // sizes of the device lists and warp offsets
    int launch_items = 0;              // CTAs per time chunk (n_items, or n_chan * 2 for the pair kernel)
    int pwords = 0;                    // largest channel block of the pair lists (16-bit words)
    uint16_t *d_ptab = nullptr;        // device: pair-kernel gather lists (build_pair_tables)
    int2 *d_pchan = nullptr;           // device: [n_chan] (block start, block words)
    int4 *d_pidx = nullptr;            // device: [n_chan][8 warps] (half 1 offset, batches, half 2 offset, batches)
    unsigned long long *d_upper = nullptr;  // device: [n_chan] folded rows whose cells lie in unfolded rows 64..127
    long long *d_ef_off = nullptr;     // device (E-field images): per group channel, complex offset within a sample
};

struct KernelTables {
    const short2 *cells;               // [C][A] (kx, ky)
    const float2 *kernel;              // [K*K]
    int A, P, C, K;
};

}  // namespace epic

struct epic_plan_s {
    int device = 0;
    int A = 0, P = 0, NP = 0, C = 0, K = 0, max_spectra = 0, precision = 0;
    int nker = 1;                      // kernels: 1 shared, or A (one per antenna)
    double2 *d_bauto = nullptr;        // per-antenna kernels: [A][(2K-1)^2] B_aa(rho) = W_a (x) W_a^*
    unsigned flags = 0;
    int sm_count = 0;
    std::vector<int> grid_n;
    std::vector<long long> out_off;    // complex-element offset of each channel's image
    size_t out_floats = 0;
    long long ef_stride = 0;           // E-field images: complex elements per sample (sum_c P N_c^2)
    uint8_t *d_dft = nullptr;          // tensor form: the 64-point DFT operand (hi, lo parts)
    uint8_t *d_dft48 = nullptr;        // the 48-point DFT in the same 128 x 128 operands (grid side 96)
    short2 *d_cells = nullptr;         // [C][A]
    float2 *d_kernel = nullptr;        // [K*K]
    int *d_autoint = nullptr;          // [C][A][4] exact integer auto sums
    int *d_status = nullptr;           // sticky device status word
    double f_ref = 0;                  // delay phases: reference frequency (mid-band, Hz)
    double du = 0.5;                   // grid cell size in wavelengths
    float *d_dfreq = nullptr;          // [C] f_c - f_ref (Hz)
    float4 *d_dtab = nullptr;          // [max_spectra][A] (frac(f_ref tau), tau_hi, tau_lo, 0) of the current call
    const double *delays = nullptr;    // device [T][A] geometric delays (s) of the current call, or null
    std::vector<epic::GroupCfg> groups;
    int force_tau = 0;                 // > 0: time chunks of the next launches (image series)
    long long wait_budget = 4000000000LL;  // clock cycles a device-side wait may take (~2 s)
    int test_withhold_mma = 0;         // fault-injection hook: tensor kernel withholds its MMA
    int series_cap = 1;                // images one series batch can hold (partials, auto sums)
    // stage timing (epic_set_profiling)
    bool profiling = false;
    std::vector<cudaEvent_t> events;   // 2 per recorded stage
    int n_recorded = 0;
    // CUDA graph of one integration, re-captured when T, pointers or profiling change
    bool use_graph = true;
    cudaStream_t cap = nullptr;        // capture stream
    std::vector<cudaStream_t> side;    // one branch per grid side
    cudaEvent_t ev_fork = nullptr, ev_auto = nullptr;
    std::vector<cudaEvent_t> ev_join;
    cudaGraphExec_t gexec = nullptr;
    const void *g_v = nullptr, *g_gains = nullptr, *g_delays = nullptr;
    void *g_out = nullptr;
    int g_T = -1;
    bool g_prof = false;
    std::vector<short2> h_cells;       // host copy of the cell map, kept when a group uses the pair kernel
    // host-buffer entry point staging (allocated on first use)
    uint8_t *d_stage_v = nullptr;
    float *d_stage_g = nullptr;
    float *d_stage_out = nullptr;
    // pipelined host-buffer entry point (epic_image_host_async; allocated on first use): two
    // slots of upload and download buffers, an upload and a download stream, and the events
    // that order them against the imaging on the caller's stream
    uint8_t *d_ring_v[2] = {nullptr, nullptr};
    float *d_ring_g[2] = {nullptr, nullptr};
    float *d_ring_out[2] = {nullptr, nullptr};
    cudaStream_t s_up = nullptr, s_down = nullptr;
    cudaEvent_t ev_up[2] = {nullptr, nullptr}, ev_in_free[2] = {nullptr, nullptr};
    cudaEvent_t ev_img[2] = {nullptr, nullptr}, ev_out_free[2] = {nullptr, nullptr};
    long long n_async = 0;
};

namespace epic {

// Stage timing helpers: no-ops unless profiling is on.
void prof_begin(epic_plan_s *plan);
void prof_mark(epic_plan_s *plan, cudaStream_t stream, int stage, bool start);

// FP32 form: launch every kernel of one integration on `stream` (with fork,
// the grid sides run on the plan's side streams and join back).
int image_fp32(epic_plan_s *plan, const uint8_t *v, const float2 *gains, int T,
               float2 *out, cudaStream_t stream, bool fork);
// one integration through the plan's CUDA graph (or direct launches)
int run_image(epic_plan_s *plan, const uint8_t *v, const float2 *gains, int T, float2 *out, cudaStream_t stream);
// per-group kernel attributes (dynamic shared memory), set once at plan time
int prepare_fp32(const epic_plan_s *plan, const GroupCfg &g);
int prepare_reg64(const epic_plan_s *plan, const GroupCfg &g);

// shared pieces (image_common.cu)
int launch_autopower(epic_plan_s *plan, const uint8_t *v, int T, cudaStream_t stream);
int launch_epilogue(epic_plan_s *plan, const GroupCfg &g, const float2 *gains, int T, int n_tau,
                    float2 *out, cudaStream_t stream);
// per-antenna kernels: auto-correlation grid X(rho) -> Y(rho_y, l_x) per channel and product
int launch_auto_rho(epic_plan_s *plan, const GroupCfg &g, const float2 *gains, cudaStream_t stream);
// delay table of the current call (plan->delays, [T][A] seconds) into plan->d_dtab
int launch_delay_prep(epic_plan_s *plan, int T, cudaStream_t stream);
// image series: per-image auto sums and one epilogue image per time chunk
int launch_autopower_series(epic_plan_s *plan, const uint8_t *v, int spi, int n_img, cudaStream_t stream);
int launch_epilogue_series(epic_plan_s *plan, const GroupCfg &g, const float2 *gains, int spi, int n_img,
                           float2 *out, cudaStream_t stream);
// imaging kernel of one group (FP32 or tensor form as the plan says)
int launch_imaging(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau,
                   cudaStream_t stream);

// tensor-core form, both 64-point DFT stages on tcgen05 (tc_dual64.cu)
void build_dft_operand(bool bf16, std::vector<uint16_t> &words, int M = 64);
size_t tc_dual_smem_bytes(int A, int K);
int prepare_tc_dual(const epic_plan_s *plan, size_t smem);
size_t tc_dual_fold_smem_bytes();
int launch_tc_dual_fold(epic_plan_s *plan, const GroupCfg &g, const float2 *gains, const float2 *gf, int nb,
                        bool accumulate, cudaStream_t stream);
int launch_tc_dual(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau,
                   cudaStream_t stream);
// grid sides 128 and 64: the gather-gridding pair kernel (tc_pair128.cu)
int build_pair_tables(const std::vector<short2> &cells, int A, int K, const std::vector<int> &chans,
                      const std::vector<uint32_t> &tab32, const std::vector<int4> &idx32,
                      const std::vector<int2> &chan32, std::vector<uint16_t> &tab, std::vector<int4> &idx,
                      std::vector<int2> &chan, std::vector<unsigned long long> &upper,
                      const PairSchedule &sched = PairSchedule(), int M = 64);
size_t tc_pair_smem_bytes(int A, int K, int words);
int prepare_tc_pair(const epic_plan_s *plan, size_t smem);
int launch_tc_pair(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau,
                   cudaStream_t stream);

// Gather table of the FP32 register-transform kernel for the channels of one group (plan.cu),
// built on up to `threads` host threads (0: automatic); the result does not depend on it.
int build_gather_table(const std::vector<short2> &cells, int A, int K, int M, int P, const std::vector<int> &chans,
                       std::vector<uint32_t> &tab, std::vector<int4> &idx, std::vector<int2> &chan,
                       std::vector<unsigned long long> &rowmask, int threads = 0);
// Register-transform kernels, fold side M = 64 or 48 (fp32_reg64.cu)
size_t reg64_smem_bytes(int M, int P, int TS, int A, int K, int nker);
int launch_reg64(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau,
                 cudaStream_t stream);
// E-field images through the register kernel: out complex [T][stride], channel offsets in g.d_ef_off
int launch_reg64_efield(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T,
                        float2 *out, long long stride, cudaStream_t stream);
// Gridding schedule of the register-transform kernels for the channels of one group (plan.cu).
int build_reg64_schedule(const std::vector<short2> &cells, int A, int K, int M, const std::vector<int> &chans,
                         std::vector<uint32_t> &desc, std::vector<int> &nrounds, int &rmax,
                         std::vector<unsigned long long> &rowmask, std::vector<uint16_t> &first);

// One single-grid-side FP32 imaging job on caller-provided device tables and
// workspace (used by the static-scratch entry point).
struct RawImage {
    int A = 0, P = 0, C = 0, K = 0, N = 0, M = 0, Q1 = 1, n_items = 0, n_tau = 1, T = 0;
    unsigned flags = 0;
    const short2 *cells = nullptr;     // [C][A]
    const float2 *kernel = nullptr;    // [K*K]
    const int *chans = nullptr;        // [C] identity channel list
    const long long *out_off = nullptr;  // [C]
    const double *wpow = nullptr;      // [N][N]
    const float2 *twN = nullptr;       // [N]
    float *partial = nullptr;          // [n_tau][n_items][M*M][NPF]
    int *autoint = nullptr;            // [C][A][4]
    int *status = nullptr;
};
int fp32_pick_tau(int n_items, int T, int sms);
// time chunks of one launch: forced (image series), else autotuned for this T, else the cost model
int choose_tau(const epic_plan_s *plan, const GroupCfg &g, int T);
// large grid sides (GroupCfg::alias)
size_t fold64_smem_bytes(int P);
int prepare_fold64(int P);
int launch_fold64(const GroupCfg &g, int P, const float2 *gf, int nb, bool accumulate, cudaStream_t stream);
int build_alias_tables(const std::vector<short2> &cells, int A, int K, int N, const std::vector<int> &chans,
                       std::vector<short2> &j0, std::vector<uint32_t> &bseg, std::vector<int> &boff);
int prepare_alias(const epic_plan_s *plan);
int launch_alias(epic_plan_s *plan, const GroupCfg &g, const uint8_t *v, const float2 *gains, int T, int *n_tau,
                 cudaStream_t stream);
size_t fp32_smem_bytes(int M, int P, int A, int K);
int launch_fp32_raw(const RawImage &r, const uint8_t *v, const float2 *gains, cudaStream_t stream);
int launch_autopower_raw(const RawImage &r, const uint8_t *v, int sm_count, cudaStream_t stream);
int launch_epilogue_raw(const RawImage &r, const float2 *gains, float2 *out, cudaStream_t stream);
// host tables shared by the plan and the static-scratch entry point
int host_cell_map(const double *ant_xy_m, int n_ant, const double *freq_hz, int n_chan, const int *grid_n,
                  double du, int K, std::vector<short2> &cells);
void host_kernel_power(const float *kern, int K, int N, std::vector<double> &out);
// raise a kernel's dynamic shared-memory cap to the device limit (less its static shared memory);
// EPIC_ERR_UNSUPPORTED if `need` does not fit
int raise_dyn_smem_cap(const void *kfn, size_t need);

// device status bits
constexpr int kStatusDevice = 1;
constexpr int kStatusTimeout = 2;

}  // namespace epic

/*
 * epic.h -- C ABI of libepic, a GB300 (sm_103a) implementation of the
 * E-field Parallel Imaging Correlator's imaging path (Krishnan et al. 2023,
 * "Optimization and Commissioning of the EPIC Commensal Radio Transient Imager
 * for the Long Wavelength Array").
 *
 * What one call computes (Eq. 4 and the GPU block chain of Sec. 2.2): for every
 * channel c and time sample t of one integration, each antenna's 4+4-bit
 * complex voltage is calibrated (e~ = g e), gridded onto a padded N x N
 * aperture grid through the illumination kernel W, Fourier transformed to the
 * sky, F_p(l) = sum_k G_p(k) exp(+2 pi i k.l / N) (unnormalised), and the
 * polarisation products F_p F_q^* (XX, YY, XY, YX; Sec. 3.2) are summed over
 * the integration.  The autocorrelation term A_pq |W^(l)|^2 -- the a = b part
 * of F_p F_q^*, A_pq = sum_a g_ap g_aq^* sum_t e_ap e_aq^*, W^(l) = sum_d W(d)
 * exp(+2 pi i d.l / N) -- is subtracted (Sec. 2.2), which makes the result
 * equal to the FX-correlator dirty image of Eq. 2-3.
 *
 * Conventions shared by every call:
 *   - ci4 byte: real part in the high nibble, imaginary in the low nibble,
 *     two's complement, values -8..7 (Sec. 2.1, "4+4 complex integers").
 *   - complex64 = two interleaved floats (re, im), i.e. float[2*n].
 *   - antenna -> cell map (Sec. 3.1, nearest neighbour on a regular grid of
 *     spacing du wavelengths): per channel, per axis,
 *       k = llround(((x - x_c) * f_c) / (c0 * du)) + N_c / 2,
 *     x_c the centroid of the layout, c0 = 299792458 m/s.  Antenna a's
 *     footprint covers cells k_a + (dx, dy), |dx|, |dy| <= (K-1)/2.
 *   - kernel W: complex64 [K][K], element [dy + h][dx + h], h = (K-1)/2; one
 *     kernel for every antenna, channel and polarisation.
 *   - output image of channel c: complex64 [NP][N_c][N_c], NP = 4 products
 *     (XX, YY, XY, YX) for dual polarisation, 1 (XX) for single; pixel (i, j)
 *     holds direction l = (j - N_c/2, i - N_c/2) in cells of 1/(N_c du), i.e.
 *     the transform is fft-shifted.  Channels are packed one after another in
 *     channel order.
 *   - XX and YY are real (imaginary part written as 0); YX = conj(XY).
 *   - an integration is a sum over time; EPIC_MEAN divides by n_spectra.
 *
 * Ownership: the caller owns every buffer passed in; the plan owns its device
 * tables and workspace.  A plan is used by one stream at a time.
 *
 * Errors: every entry point returns EPIC_OK (0) or a negative EPIC_ERR_* code.
 * Argument errors are detected on the host before anything is launched and
 * leave the output untouched.  Device-side errors (a bounded wait that ran
 * out, an index check that failed) are recorded in the plan's status word and
 * reported by epic_status.
 */
#ifndef EPIC_H
#define EPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct epic_plan_s *epic_plan_t;

enum {
    EPIC_OK = 0,
    EPIC_ERR_ARG = -1,          /* bad argument (null pointer, size, range) */
    EPIC_ERR_OUT_OF_GRID = -2,  /* an antenna footprint leaves [0, N) */
    EPIC_ERR_UNSUPPORTED = -3,  /* valid request this build does not implement */
    EPIC_ERR_CUDA = -4,         /* a CUDA runtime call failed */
    EPIC_ERR_TIMEOUT = -5,      /* a bounded device-side wait ran out */
    EPIC_ERR_NOMEM = -6,        /* device or host allocation failed */
    EPIC_ERR_DEVICE = -7,       /* a device-side index/consistency check failed */
    EPIC_ERR_TOO_LARGE = -8     /* request does not fit epic_image_static's fixed scratch */
};

/* Arithmetic form of the gridding + transform + products stages. */
enum {
    EPIC_FP32 = 0,              /* FP32 SIMT: gather gridding, register FFTs */
    EPIC_TC_SPLIT_FP16 = 1,     /* tensor cores, split hi+lo FP16 operands, FP32 accumulate */
    EPIC_TC_FP16 = 2,           /* tensor cores, single FP16 operands */
    EPIC_TC_SPLIT_BF16 = 3      /* tensor cores, two-part BF16 split (hi + lo, 3 MMAs per k-block): about
                                   16 significant bits, bounded by 1e-4 of the peak, not 1e-5 */
};
/* The tensor-core forms run both DFT stages of every pixel class as tcgen05
 * GEMMs (the complex DFT in real 2 x 2 block form, FP32 accumulation in tensor
 * memory; 64-point, a 32 side as the 64-point DFT of the zero-padded grid, a 96
 * side's 48-point DFTs in the first 48 rows and columns of the same operands).
 * Grid sides 128, 96 and 64 with dual polarisation and one shared kernel run
 * the gather-gridding kernel (gridding straight into the FP16 operand; two
 * pixel classes per CTA from one gridding at sides 128 and 96) when the
 * channel's lists fit in shared memory and no folded row holds cells of both
 * aperture halves; otherwise, and for sides 32, 256 and 512 or single
 * polarisation, the two-stage kernel (one class per CTA) — except side 96,
 * which then runs the FP32 kernel inside the tensor plan (a tensor plan must
 * run at least one group on the tensor cores, else EPIC_ERR_UNSUPPORTED).
 * Accuracy: split FP16 within 1e-5 of the channel peak, single FP16 within
 * 2e-3. */

/* flags */
#define EPIC_MEAN        1u     /* divide the sum over time by n_spectra */
#define EPIC_NO_AUTOSUB  2u     /* keep the autocorrelation term (diagnostics) */
/* Apply the illumination kernel in the image domain: grid each calibrated
 * voltage into its single cell and multiply the finished image by |W^(l)|^2
 * (FP64).  Because every antenna shares one kernel, gridding through W is a
 * convolution and F(l) = W^(l) sum_a e~_a exp(+2 pi i k_a.l / N); the result
 * equals the default (literal gridding) form up to rounding, with K^2 times
 * fewer gridding operations. */
#define EPIC_KERNEL_TAPER 4u
/* Dual polarisation only: write Stokes I = XX + YY, Q = XX - YY, U = 2 Re XY,
 * V = 2 Im XY (XY = F_X F_Y^*) as the four real images instead of the
 * polarisation products. */
#define EPIC_STOKES      8u
/* kernel_c64 holds one kernel per antenna, complex64 [n_ant][K][K] (Eq. 3
 * writes the gridding kernel W_a per antenna: heterogeneous beams,
 * A-projection, Sec. 3.1).  The autocorrelation term becomes
 * sum_a A_a,pq |W^_a(l)|^2, evaluated from the auto-correlation grid
 * sum_a A_a,pq (W_a (x) W_a^*) in FP64.  FP32 form only; not with
 * EPIC_KERNEL_TAPER (which needs one shared kernel) or epic_image_series. */
#define EPIC_ANTENNA_KERNELS 16u

/*
 * Diagnostic plan options, in the flags word from bit 8 up.  They exist for
 * the library's own tests and measurements: each selects another route to the
 * same result (or, for EPIC_DIAG_WITHHOLD_MMA, injects a fault), and nothing
 * but an explicit flag turns one on.
 */
#define EPIC_DIAG_NO_GRAPH       (1u << 8)   /* launch each kernel directly instead of replaying a CUDA graph */
#define EPIC_DIAG_GATHER_GLOBAL  (1u << 9)   /* FP32 register kernel: read the gather table through L1 instead
                                                of staging it in shared memory (bitwise the same result) */
#define EPIC_DIAG_NO_ALIAS       (1u << 10)  /* 512 grid sides: grid per pixel class instead of folding */
#define EPIC_DIAG_WITHHOLD_MMA   (1u << 11)  /* fault injection: the tensor kernel issues no MMA, its bounded
                                                wait (budget ~1 ms) runs out and epic_status reports
                                                EPIC_ERR_TIMEOUT; the context stays usable */
#define EPIC_DIAG_ALIAS_BATCH(n) ((((unsigned)(n)) & 255u) << 16)   /* fold path: at most n (1..255) samples
                                                                        per time batch */
#define EPIC_DIAG_NO_PAIR        (1u << 12)  /* tensor form without the gather-gridding pair kernel (two
                                                classes from one gridding at sides 128 and 96, its one
                                                class at 64): sides 128 and 64 run the two-stage kernel
                                                of the other sides (one pixel class per CTA, scheduled
                                                gridding), side 96 the FP32 register kernel */

/*
 * epic_plan -- validate the array geometry and build every table the imaging
 * calls need (Sec. 3.1 grid and antenna-to-cell map; Eq. 4 kernel image).
 *
 *   out            receives the plan handle (set to NULL on error)
 *   ant_xy_m       host double [n_ant][2], antenna (x, y) positions in metres
 *   n_ant          number of antennas A >= 1
 *   n_pol          1 (single polarisation, product XX) or 2 (X and Y)
 *   kernel_c64     host complex64 [K][K] illumination kernel W, or [n_ant][K][K]
 *                  with EPIC_ANTENNA_KERNELS
 *   K              odd kernel side, 1 <= K <= 15
 *   grid_n         host int [n_chan], grid side N_c per channel; supported
 *                  sides are 32, 64, 96, 128, 256 and 512
 *   freq_hz        host double [n_chan], channel centre frequencies
 *   n_chan         number of channels C >= 1
 *   du_wavelengths cell size in wavelengths, 0 < du <= 0.5 (lambda/2 grid)
 *   max_spectra    largest n_spectra an epic_image call will pass (>= 0)
 *   precision      EPIC_FP32 or one of the EPIC_TC_* forms
 *   flags          EPIC_MEAN | EPIC_NO_AUTOSUB | EPIC_KERNEL_TAPER | EPIC_STOKES |
 *                  EPIC_ANTENNA_KERNELS, plus the EPIC_DIAG_* options above
 *
 * Uses the current CUDA device.  Allocates device memory (tables and
 * workspace) and returns EPIC_ERR_NOMEM if that fails.  The tables include,
 * per channel, the gridding lists of the FP32 kernel (for every pair of
 * adjacent folded cells, the antennas whose footprints cover it: 4 bytes per
 * entry, about A * K * (K + 1) / 2 entries plus padding; 43 KB per channel at
 * A = 256, K = 5), staged in shared memory by the kernel when they fit.
 * Channels with a 512 grid side and one shared kernel wider than one tap are
 * imaged by gridding each (channel, sample) once and folding the 64 pixel
 * classes from it: their workspace adds the folded class grids of one time
 * batch, up to 4 GiB (C * 64 * n_pol * 32 KB per spectrum, batched).  Returns
 * EPIC_ERR_OUT_OF_GRID when some antenna footprint k_a +- (K-1)/2 leaves
 * [0, N_c) in some channel; EPIC_ERR_UNSUPPORTED for a grid side, precision or
 * size this build does not provide.
 */
int epic_plan(epic_plan_t *out,
              const double *ant_xy_m, int n_ant, int n_pol,
              const float *kernel_c64, int K,
              const int *grid_n, const double *freq_hz, int n_chan,
              double du_wavelengths, int max_spectra, int precision,
              unsigned flags);

/*
 * epic_image -- image one integration (Eq. 4 with autocorrelation removal,
 * Sec. 2.2).
 *
 *   plan        from epic_plan
 *   ci4         device uint8 [n_spectra][n_chan][n_ant][n_pol], packed 4+4-bit
 *               voltages (time slowest, polarisation fastest)
 *   gains_c64   device complex64 [n_chan][n_ant][n_pol] per-antenna gains, or
 *               NULL for unit gains (Sec. 4 notes gains are not applied in the
 *               deployed system; they multiply the voltages here)
 *   n_spectra   number of time samples T, 0 <= T <= max_spectra; T = 0 gives
 *               an all-zero image
 *   out_c64     device complex64, epic_out_floats(plan) floats, overwritten
 *   cuda_stream cudaStream_t to order the work on (NULL = legacy default)
 *
 * Asynchronous and stream-ordered; allocates nothing.  Returns EPIC_ERR_ARG
 * (nothing launched) for null pointers or n_spectra out of range, and
 * EPIC_ERR_CUDA if a launch fails.
 */
int epic_image(epic_plan_t plan, const uint8_t *ci4, const float *gains_c64,
               int n_spectra, float *out_c64, void *cuda_stream);

/*
 * epic_autotune -- pick each channel group's launch shape by measurement.
 *
 * For every channel group the imaging and epilogue launches of an n_spectra
 * integration are timed (CUDA events on the stream, zero voltages, unit
 * gains, scratch buffers the call allocates and frees) at a handful of
 * time-chunk counts -- the cost model's choice, its neighbours, and the counts
 * that fill whole waves of SMs -- and the fastest is kept for later epic_image /
 * epic_image_ex calls with the same n_spectra (other counts fall back to the
 * cost model; epic_image_series keeps one chunk per image).  The next call
 * re-captures its CUDA graph.  Blocks the host until the timing runs finish.
 * Results are unchanged up to the FP32 summation order of the time chunks.
 * EPIC_ERR_ARG for a null plan or n_spectra outside [1, max_spectra];
 * EPIC_ERR_NOMEM / EPIC_ERR_CUDA if the scratch buffers or launches fail.
 */
int epic_autotune(epic_plan_t plan, int n_spectra, void *cuda_stream);

/*
 * epic_image_series_ex -- epic_image_series with the geometric-delay correction
 * of epic_image_ex: delays_s is device double [n_spectra][n_ant] (seconds),
 * indexed like the voltages; NULL = no correction (identical to
 * epic_image_series).  Same errors and behaviour as epic_image_series.
 */
int epic_image_series_ex(epic_plan_t plan, const uint8_t *ci4, const float *gains_c64,
                         const double *delays_s, int n_spectra, int spectra_per_image,
                         float *out_c64, void *cuda_stream);

/*
 * epic_image_ex -- epic_image with the geometric-delay correction of Sec. 2.2
 * (the delay-correction block that compensates each antenna's geometric delay
 * at every time step, for every channel, before gridding).  Each calibrated
 * voltage is multiplied by exp(+2 pi i f_c tau_a(t)):
 *
 *   e~_{a,p}(t, c) = g_{c,a,p} * exp(+2 pi i f_c tau_a(t)) * e_{a,p}(t, c)
 *
 * tau_a(t) is the delay of antenna a's signal relative to the phase centre
 * (positive = the wavefront reaches it later), so the product re-phases the
 * array towards the direction the delays were computed for.
 *
 *   delays_s    device double [n_spectra][n_ant], seconds; NULL = no correction
 *               (identical to epic_image)
 *   (the other arguments as for epic_image)
 *
 * A small kernel forms, once per (t, antenna), the FP64 turns at a mid-band
 * reference frequency (reduced to a fraction) and tau as two floats; the
 * imaging kernels add the per-channel remainder (f_c - f_ref) tau in FP32 with
 * an exact two-product and take a single-precision sincospi.  The plan holds
 * that [max_spectra][n_ant] table, so this call allocates nothing either.  The
 * correction has unit modulus and is common to both
 * polarisations of an antenna, so the autocorrelation term is unchanged.
 * Same errors, ordering and allocation behaviour as epic_image.  The delays
 * pointer is part of the captured graph's key: a new pointer re-captures.
 */
int epic_image_ex(epic_plan_t plan, const uint8_t *ci4, const float *gains_c64,
                  const double *delays_s, int n_spectra, float *out_c64,
                  void *cuda_stream);

/*
 * epic_image_host -- the same integration with HOST buffers: copies ci4 and
 * gains to plan-owned device staging (allocated on the first call, reused
 * after), runs epic_image on the given stream, copies the image back into
 * out_c64 (host) and synchronises that stream before returning.  Pinned host
 * memory makes the copies asynchronous DMA; pageable memory works but is
 * slower.  Argument meanings and layouts are those of epic_image.
 */
int epic_image_host(epic_plan_t plan, const uint8_t *ci4_host, const float *gains_c64_host,
                    int n_spectra, float *out_c64_host, void *cuda_stream);

/*
 * epic_image_host_async / epic_host_wait -- the host-buffer integration as a
 * pipeline for a stream of integrations (the paper's deployment images gulp
 * after gulp, Sec. 2.2): epic_image_host_async queues the upload of this
 * integration's ci4 and gains (on a plan-owned upload stream, into one of two
 * plan-owned device slots), its imaging on cuda_stream, and the download of the
 * image into out_c64_host (on a plan-owned download stream), and returns
 * without waiting, so the upload of the next integration and the download of
 * the previous one overlap this one's imaging.  epic_host_wait blocks until
 * every queued upload and download has finished; until then the caller must
 * neither change the host inputs nor read the host outputs of the queued calls.
 * Host buffers should be pinned (pageable memory makes the copies synchronous).
 * Argument meanings, layouts and checks are those of epic_image_host; device
 * buffers are allocated on the first call (EPIC_ERR_NOMEM), copy errors are
 * reported by this call or by epic_host_wait (EPIC_ERR_CUDA), device-side
 * status by epic_status.  The paper has no counterpart.
 */
int epic_image_host_async(epic_plan_t plan, const uint8_t *ci4_host, const float *gains_c64_host,
                          int n_spectra, float *out_c64_host, void *cuda_stream);
int epic_host_wait(epic_plan_t plan);

/*
 * epic_image_series -- time-resolved imaging for transient searches (the
 * millisecond imaging of Sec. 1 and Sec. 4): n_spectra = n_img *
 * spectra_per_image, and image i is the integration of spectra
 * [i * spectra_per_image, (i + 1) * spectra_per_image) with its own
 * autocorrelation subtraction (flags as for the plan; EPIC_MEAN divides by
 * spectra_per_image).  out_c64 holds n_img consecutive outputs of
 * epic_out_floats(plan) floats each.  Other arguments as for epic_image.
 * Returns EPIC_ERR_ARG if n_spectra is not a multiple of spectra_per_image or
 * exceeds max_spectra, and EPIC_ERR_UNSUPPORTED for a tensor-form plan whose
 * 512-side channels only fit the folded path (series need one time chunk per
 * image, which that path does not provide).  Asynchronous; allocates nothing;
 * runs as direct launches (no graph).
 */
int epic_image_series(epic_plan_t plan, const uint8_t *ci4, const float *gains_c64,
                      int n_spectra, int spectra_per_image, float *out_c64, void *cuda_stream);

/*
 * epic_image_efield -- the electric-field images themselves, one per sample (the
 * abstract and Sec. 1: EPIC forms "electric field or intensity images"; the
 * transient mode of Sec. 4 images every sample):
 *
 *   F_p(l, t) = sum_k G_p(k, t) exp(+2 pi i k.l / N_c),
 *   G_p(k, t) = sum_a sum_d W(d) g_{c,a,p} e_{t,c,a,p} [k = k_a(c) + d]
 *
 * for every sample t, channel c and polarisation p: calibrate, grid, transform
 * (steps a1-a4 of epic_image), with no products, no time sum and no
 * autocorrelation term (plan flags other than the kernel choice do not apply).
 *
 *   out_c64     device complex64 [n_spectra][epic_efield_floats(plan) / 2]: per
 *               sample the channels packed in channel order, each
 *               [n_pol][N_c][N_c] on the fft-shifted layout of epic_image
 *               (pixel (i, j) holds l = (j - N_c/2, i - N_c/2)); overwritten
 *   (the other arguments as for epic_image)
 *
 * The output is n_spectra x 8 sum_c n_pol N_c^2 bytes (16.8 GB for 1000 samples
 * of 64 channels of 128 x 128 dual polarisation), written once.  FP32 plans
 * whose grid sides all run the register-transform kernel (sides 64, 96, 128,
 * 256, 512 with n_ant * n_pol a multiple of 4); EPIC_ERR_UNSUPPORTED for
 * others.  Asynchronous; allocates nothing; direct launches (no graph).
 */
int epic_image_efield(epic_plan_t plan, const uint8_t *ci4, const float *gains_c64, int n_spectra,
                      float *out_c64, void *cuda_stream);

/* Floats of one sample of epic_image_efield's output (2 per complex value), or
 * 0 for a NULL plan. */
size_t epic_efield_floats(epic_plan_t plan);

/* Number of floats of one epic_image output (2 per complex value), or 0 for a
 * NULL plan. */
size_t epic_out_floats(epic_plan_t plan);

/*
 * epic_status -- synchronise the device and return the sticky device-side
 * status of the plan: EPIC_OK, EPIC_ERR_TIMEOUT or EPIC_ERR_DEVICE (an
 * in-kernel consistency check failed; the output of that call is undefined),
 * or EPIC_ERR_CUDA if the synchronisation itself reported an error.  Reading
 * the status clears it.
 */
int epic_status(epic_plan_t plan);

/* Free the plan and everything it owns (waits for the device first). NULL is
 * accepted. */
void epic_destroy(epic_plan_t plan);

/*
 * Stage timing (the per-block processing-time breakdown of Table 2, taken on
 * the device).  epic_set_profiling(plan, 1) makes every later epic_image call
 * record CUDA events on its stream around each of its kernel launches;
 * epic_stage_times waits for the last such call and writes the device time in
 * milliseconds of each launch, in launch order: [0] the auto-power kernel
 * (absent with EPIC_NO_AUTOSUB), then for each grid side in ascending order
 * the imaging kernel and its epilogue.  Returns the number of values written
 * (at most max_stages), or a negative EPIC_ERR_* code (EPIC_ERR_ARG if
 * profiling is off or no call was recorded).
 */
int epic_set_profiling(epic_plan_t plan, int enable);
int epic_stage_times(epic_plan_t plan, float *ms, int max_stages);

/*
 * epic_image_static -- one integration in the FP32 form with no device
 * allocation: no plan, no cudaMalloc/cudaFree, no allocating library call.
 * The paper has no counterpart; this entry point exists for callers that
 * cannot allocate device memory themselves or through the library -- a
 * pipeline whose GPU memory is all reserved by its own pool allocator, a
 * real-time capture loop that must not let cudaMalloc/cudaFree synchronise the
 * device under it, a plug-in that may leave no allocations behind.
 *
 * The caller passes the geometry (as for epic_plan, but one grid side
 * grid_n in {32, 64, 96, 128} for every channel), the device inputs (as for
 * epic_image) and the device output (complex64 [n_chan][NP][grid_n][grid_n]).
 * Tables and workspace live in one 32 MiB array in device global memory that
 * the library declares at file scope; every GPU that loads libepic holds it
 * until the process exits.  Requests whose tables, auto-power sums and one set
 * of partial images do not fit it return EPIC_ERR_TOO_LARGE before any work
 * is queued (e.g. 64 channels of 128 x 128 dual polarisation fit; 128 do not).
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current).  Every call shares the array and
 * overwrites what the previous call left in it (what must start at zero is
 * cleared on the call's stream), so calls whose GPU work overlaps -- different
 * streams, different host threads -- race; order them.  The geometry tables
 * are copied from pageable host memory on the stream, so the call may block
 * the host briefly, and it must not be made while the stream is being captured
 * into a CUDA graph.  Asynchronous otherwise.  The return value covers the
 * checks and launches only: the device-side status word that epic_status
 * reports for a plan (e.g. a bounded wait that ran out) lives in the shared
 * array and is not reported to a static caller.  Other errors are those of
 * epic_plan and epic_image.
 */
int epic_image_static(const double *ant_xy_m, int n_ant, int n_pol,
                      const float *kernel_c64, int K, int grid_n,
                      const double *freq_hz, int n_chan, double du_wavelengths,
                      const uint8_t *ci4, const float *gains_c64, int n_spectra,
                      unsigned flags, float *out_c64, void *cuda_stream);

/*
 * epic_solve_gains -- per-antenna complex gains from one calibrator, in the
 * E-field domain (the feedback calibration Sec. 1 cites for EPIC; Sec. 5 lists
 * real-time calibration as future work; the paper gives no algorithm, this is
 * a single-calibrator solver in that spirit).
 *
 * For each channel c and polarisation p, from unit gains, n_iter times:
 *   E(t) = (1/A) sum_a g_a e_a(t) conj(phi_a)           beamformed calibrator field
 *   g_a  = phi_a sum_t E(t) conj(e_a(t)) / sum_t |e_a(t)|^2   (0 if e_a is all zero)
 *   antenna 0's phase set to 0, the RMS of |g_a| set to 1
 * with phi_a = exp(-2 pi i (kx_a lx + ky_a ly) / N_c), (lx, ly) = (l N_c du,
 * m N_c du): the phase the calibrator at direction cosines (l, m) puts on the
 * antenna's cell (it then appears at +(lx, ly) in epic_image's output).  The
 * result is what epic_image's gains_c64 expects (g multiplies e) up to one
 * complex factor per (channel, polarisation), which a single calibrator of
 * unknown flux cannot fix.  The start needs the unit-gain beam to see the
 * calibrator: if the instrumental gains sum to zero, E vanishes and the gains
 * come out zero.
 *
 *   ci4         device uint8 [n_spectra][n_chan][n_ant][n_pol], 1 <= n_spectra <= max_spectra
 *   l, m        calibrator direction cosines
 *   n_iter      1 .. 64 (one iteration suffices when one source dominates)
 *   gains_out   device complex64 [n_chan][n_ant][n_pol], overwritten
 *
 * FP32 sums, exact integer |e|^2 sums; one CTA per (channel, polarisation).
 * Asynchronous on the stream; allocates nothing.  EPIC_ERR_ARG for null
 * pointers or out-of-range arguments, EPIC_ERR_TOO_LARGE when the per-CTA
 * shared memory (8 n_spectra + 20 n_ant bytes) exceeds 200 KB.
 */
int epic_solve_gains(epic_plan_t plan, const uint8_t *ci4, int n_spectra, double l, double m,
                     int n_iter, float *gains_out, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Transient search on the image cube (Sec. 4: per-channel light curves from
 * the images, the dispersive delay corrected across the band, a single-pulse
 * search of the de-dispersed light curves; Sec. 5: real-time de-dispersion
 * and transient detection).  Works on any float intensity cube
 * I[t][c][p] reached through strides -- a plain [T][C][P] array, or the
 * Stokes-I slot of an epic_image_series output made with EPIC_STOKES.
 * ------------------------------------------------------------------------ */
typedef struct epic_search_s *epic_search_t;

/*
 * epic_search_plan -- delay table of a de-dispersion search.
 *
 *   freq_hz     host double [n_chan] channel centre frequencies
 *   dt_s        sampling interval of the cube (s)
 *   dm          host double [n_dm] trial dispersion measures (pc cm^-3, >= 0)
 *   n_pix       pixels per channel image; n_time samples per channel
 *   width_mask  boxcar widths of the single-pulse search: bit k = width 2^k,
 *               k < 6 (1 .. 32 samples); at least one bit
 *
 * width_mask may also carry diagnostic options, from bit 8 up (tests and
 * measurements only; the result is bitwise the same in every form):
 *   EPIC_SEARCH_DIAG_DM32     blocks of 32 trial DMs where they fit (else 16)
 *   EPIC_SEARCH_DIAG_DIRECT   the direct form (each warp loads its own sweep)
 *   EPIC_SEARCH_DIAG_NO_PIX2  unit-stride cubes on the one-pixel staged form
 *   EPIC_SEARCH_DIAG_NO_TMA   no tensor-memory-access copies (cp.async forms)
 *   EPIC_SEARCH_DIAG_WITHHOLD_TMA  fault injection: the TMA form's producer
 *       skips channel 0, the consumers' bounded wait (~1 ms) runs out and
 *       epic_search_status reports EPIC_ERR_TIMEOUT
 *
 * Channel c at trial d is delayed by s = floor(k_DM DM (f_c^-2 - f_max^-2) / dt
 * + 1/2) samples (f in MHz, k_DM = 4.148808e3 s MHz^2 pc^-1 cm^3, FP64 on the
 * host); t_out = n_time - max s output samples remain.  EPIC_ERR_ARG for bad
 * arguments, EPIC_ERR_TOO_LARGE when the largest delay leaves fewer output
 * samples than the smallest width.  The plan owns the device delay table.
 */
#define EPIC_SEARCH_DIAG_DM32         (1u << 8)
#define EPIC_SEARCH_DIAG_DIRECT       (1u << 9)
#define EPIC_SEARCH_DIAG_NO_PIX2      (1u << 10)
#define EPIC_SEARCH_DIAG_NO_TMA       (1u << 11)
#define EPIC_SEARCH_DIAG_WITHHOLD_TMA (1u << 12)
int epic_search_plan(epic_search_t *out, const double *freq_hz, int n_chan, double dt_s,
                     const double *dm, int n_dm, int n_pix, int n_time, unsigned width_mask);

/* Output samples per trial (t_out) and the largest delay (samples); either pointer may be NULL. */
int epic_search_info(epic_search_t s, int *t_out, int *max_shift);

/*
 * epic_dedisperse -- D[d][t][p] = sum_c I[t + s[d][c]][c][p] for t < t_out.
 *
 *   cube       device float; I[t][c][p] = cube[t * t_stride + c * c_stride + p * pix_stride]
 *              (strides in floats, >= 1)
 *   dd         device float [n_dm][t_out][n_pix], overwritten
 *
 * FP32 sums in channel order.  Asynchronous on the stream; allocates nothing.
 * With unit pixel stride and row pitches that are multiples of 4 floats (a
 * 16-byte aligned cube) the rows are fetched by tensor-memory-access copies
 * whose waits are bounded; see epic_search_status.
 */
int epic_dedisperse(epic_search_t s, const float *cube, long long t_stride, long long c_stride,
                    long long pix_stride, float *dd, void *cuda_stream);

/*
 * epic_single_pulse -- boxcar search of every de-dispersed light curve.
 *
 * Per (d, p): mu and sigma are the mean and population standard deviation of
 * D[d][:][p]; S/N(t, w) = (sum_{k<w} D[d][t+k][p] - w mu) / (sigma sqrt(w))
 * for the plan's widths w and t <= t_out - w.  Written per (d, p), device
 * [n_dm][n_pix]: best_snr, best_t and best_w of the largest S/N (ties: the
 * smaller width, then the earlier start; sigma = 0 gives S/N 0 at t = 0 and
 * the smallest width).  Then cand (device int pairs (d, p), capacity
 * cand_cap, may be NULL when cand_cap = 0) receives, in increasing d * n_pix + p
 * order, every pair whose best S/N >= threshold, and *n_cand (device int) their
 * number (which can exceed cand_cap; only the first cand_cap are stored).
 * Asynchronous on the stream; allocates nothing.
 */
int epic_single_pulse(epic_search_t s, const float *dd, float threshold, float *best_snr, int *best_t,
                      int *best_w, int *cand, int cand_cap, int *n_cand, void *cuda_stream);

/*
 * epic_search_status -- synchronise the device and return the sticky
 * device-side status of the search plan: EPIC_OK, or EPIC_ERR_TIMEOUT when a
 * bounded wait inside epic_dedisperse ran out (that call's output is then
 * undefined); EPIC_ERR_CUDA if the synchronisation itself failed.  Reading the
 * status clears it.
 */
int epic_search_status(epic_search_t s);

void epic_search_destroy(epic_search_t s);

/*
 * epic_measure_peak -- measure the peak rate of one arithmetic pipe on the
 * current device, for the roofline fractions of the benchmark; the paper has
 * no counterpart.  what: EPIC_PEAK_FP32 (FP32 FMA), EPIC_PEAK_FP32X2 (FP32 FMA
 * on packed pairs, fma.rn.f32x2), EPIC_PEAK_FP64 (FP64 FMA), EPIC_PEAK_FP16_TC
 * (dense FP16 tcgen05 MMA, 128 x 256 x 16, FP32 accumulate).  Each launch runs
 * long chains of independent multiply-adds (or back-to-back MMAs, one CTA per
 * SM) for about `ms` milliseconds (1 .. 10000); *tflops receives the best of
 * three launches in TFLOP/s (2 per multiply-add).  Synchronises the stream;
 * allocates 4 KB of device memory for the duration of the call.
 * EPIC_ERR_TIMEOUT if the tensor probe's bounded wait ran out.
 */
enum { EPIC_PEAK_FP32 = 0, EPIC_PEAK_FP32X2 = 1, EPIC_PEAK_FP64 = 2, EPIC_PEAK_FP16_TC = 3 };
int epic_measure_peak(int what, int ms, double *tflops, void *cuda_stream);

/* Static, human-readable text for an EPIC_* code. */
const char *epic_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* EPIC_H */

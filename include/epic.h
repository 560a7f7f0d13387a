/*
 * epic.h -- C ABI of the GB300 MOFF imaging library.
 *
 * The library implements the per-sample imaging step of the E-field Parallel Imaging
 * Correlator (Thyagarajan, Beardsley, Bowman & Morales 2015, "A generic and efficient
 * E-field parallel imaging correlator for next-generation radio telescopes"):
 * for every time sample, channel and polarisation the calibrated antenna voltages are
 * gridded with their aperture-illumination kernels (Sec. 3 "Gridding Convolution"),
 * zero-padded and spatially Fourier transformed (Sec. 3 "Spatial Fourier Transform"),
 * squared and time-averaged (Sec. 3 "Time-averaging"), which is the MOFF imaging
 * equation (Eq. "dirty-image-MOFF").
 *
 * Conventions shared by every call:
 *   - All sizes are plain ints; all device pointers are caller-owned (e.g. allocated
 *     by PyTorch) and never freed by the library.  Host pointers are only read during
 *     the call.
 *   - Complex numbers are interleaved (re, im) pairs.
 *   - Grid cell (gy, gx) of the N_g x N_g grid sits at origin + dx * (gx, gy) metres.
 *     The padded grid is N_p x N_p with the gridded field in its corner [0, N_g)^2.
 *   - Spatial transform: F(k) = sum_g E(g) exp(+2 pi i g.k / N_p), unnormalised (the
 *     imaging sign of App. B; a source at direction s appears at +s).
 *   - Images are N_p x N_p, row-major (iy, ix), with k = 0 at pixel (N_p/2, N_p/2):
 *     pixel (iy, ix) is direction (l, m) = ((ix - N_p/2), (iy - N_p/2)) * lambda / (N_p dx).
 *   - Every call returns an epic_status and never aborts; on failure epic_last_error()
 *     returns a thread-local message.  Arguments are validated on the host before any
 *     launch, including the alignment of every device array to its element: voltages to
 *     their sample size (8, 4 or 1 bytes), complex64 and float64 arrays to 8 bytes, float32
 *     arrays to 4 (a misaligned array, e.g. a view at an odd offset, is EPIC_EINVAL).  Calls
 *     are asynchronous on the caller's stream; a CUDA error raised by a launch is reported as
 *     EPIC_ECUDA.
 */
#ifndef EPIC_H
#define EPIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct epic_plan epic_plan;

typedef enum {
    EPIC_OK = 0,
    EPIC_EINVAL = 1,        /* invalid argument (message says which) */
    EPIC_ENOMEM = 2,        /* the plan's device tables could not be allocated */
    EPIC_ECUDA = 3,         /* a CUDA runtime call or launch failed */
    EPIC_EUNSUPPORTED = 4,  /* valid, but outside what this library implements */
    EPIC_ETIMEOUT = 5       /* a kernel's bounded wait (on the tensor cores, or on a cluster
                               exchange) ran out (reported by epic_sync; the outputs of the
                               calls since the last epic_sync are undefined) */
} epic_status;

typedef enum {
    EPIC_VOLT_C64 = 0,      /* complex64: float re, float im (8 bytes) */
    EPIC_VOLT_F16 = 1,      /* complex half: half re, half im (4 bytes) */
    EPIC_VOLT_CI4 = 2       /* 4+4-bit: one byte, high nibble re, low nibble im,
                               each a 4-bit two's-complement integer */
} epic_volt_dtype;

typedef enum {
    EPIC_XFORM_FFT = 0,         /* FP32 shared-memory FFT (all sizes; the default) */
    EPIC_XFORM_DFTGEMM = 1,     /* dense DFT on the tensor cores, FP16 hi+lo operands, FP32
                                   accumulation (N_p = 128 and 256) */
    EPIC_XFORM_DFTGEMM_FP16 = 2,/* reduced precision: FP16 gridding operands (weights and gained
                                   voltages rounded to FP16, products exact, FP32 sums) and one
                                   FP16 product per real product of the DFT (N_p = 128) */
    EPIC_XFORM_FFT_TWOPASS = 3, /* FP32 FFT as a row pass and a column pass with the row-
                                   transformed grid staged in device memory (N_p = 512) */
    EPIC_XFORM_DFTGEMM_FP16_GRID = 4 /* FP16 gridding operands (weights and calibrated voltages
                                   rounded to FP16, products exact, FP32 sums) and the
                                   EPIC_XFORM_DFTGEMM transform with hi+lo operands (N_p = 256) */
} epic_xform;

/*
 * epic_create -- build the antenna-to-grid mapping and the device tables (once per
 * array; Sec. 3 "Antenna-to-Grid Mapping").
 *
 *   plan        out: new plan, owned by the caller until epic_destroy.
 *   n_ant       number of antennas A (1 .. 4096).
 *   pos_xy      host [A][2] float64, antenna positions in metres (x, y).
 *   kern_ptr    host [A+1] int32, CSR row pointers into the footprint tables: antenna a
 *               owns samples kern_ptr[a] .. kern_ptr[a+1]-1 (kern_ptr[0] == 0).
 *   kern_dxdy   host [nt][2] float64, footprint sample offsets from the antenna (m).
 *   kern_w      host [nt][2] float64, complex sample weights of the illumination W_a.
 *   dx          grid spacing in metres (> 0).
 *   origin_xy   host [2] float64, position (m) of the centre of grid cell (0, 0).
 *   n_grid      N_g, the unpadded grid side (1 .. n_pad/2).
 *   n_pad       N_p, the padded grid and image side: 32, 64, 128, 256 or 512.
 *   n_chan      C, channels per call (>= 1).
 *   n_pol       P, polarisations per call (>= 1).
 *   volt_dtype  one of epic_volt_dtype.
 *   device      CUDA device ordinal the plan lives on.
 *
 * Each footprint sample maps to its nearest grid cell, per axis
 * floor((r_a + delta - origin) / dx + 0.5) evaluated in float64; the weights of samples
 * landing in the same cell are summed (the sparse matrix M(r, a) of Sec. 3).  A sample
 * outside [0, N_g)^2 is EPIC_EINVAL.  The mapping is shared by all channels: it is in
 * metres, and channel c's pixel scale follows from its wavelength.  EPIC_EUNSUPPORTED if the
 * forward kernel's shared memory (per-antenna gains and voltages beside the transform
 * buffers) cannot hold n_ant antennas at this n_pad.
 */
epic_status epic_create(epic_plan **plan, int n_ant, const double *pos_xy,
                        const int *kern_ptr, const double *kern_dxdy, const double *kern_w,
                        double dx, const double *origin_xy, int n_grid, int n_pad,
                        int n_chan, int n_pol, int volt_dtype, int device);

/*
 * epic_set_transform -- choose how epic_image computes the zero-padded 2-D spatial transform
 * (Sec. 3 "Spatial Fourier Transform").  EPIC_XFORM_FFT (default) is a float32 radix FFT in
 * shared memory.  EPIC_XFORM_DFTGEMM writes the transform as two dense matrix products with the
 * DFT matrix W[k][n] = exp(+2 pi i n k / N_p) on the tensor cores: every operand is split into
 * two FP16 numbers (hi + lo) and each real product is accumulated as hi*hi + hi*lo + lo*hi in
 * FP32 (per image the gridded field is scaled by a power of two to keep the operands in range).
 * It is available for n_pad == 128 (up to about 2,400 antennas: the kernel keeps four
 * per-antenna arrays in shared memory beside the operand tables; 1,900 for epic_image_xpol) and
 * for n_pad == 256 (up to about 1,860 antennas; two CTAs per image, each computing half of the
 * image rows, the operand tables streamed from global memory; no cross-polarisation form);
 * otherwise EPIC_EUNSUPPORTED.  EPIC_XFORM_DFTGEMM_FP16 (n_pad == 128, single polarisation
 * products only) is the reduced-precision form: the gridding multiplies FP16-rounded weights by
 * FP16-rounded calibrated voltages and sums in FP32, and each real product of the transform is
 * one FP16 product with FP32 accumulation (no lo parts): about a third of the tensor work, with
 * an error of about 1e-3 relative L2 against the exact image instead of about 1e-6.  The first
 * call with a tensor-core form uploads the plan's DFT operand tables (64 KB for n_pad 128,
 * 256 KB for 256).  EPIC_XFORM_FFT_TWOPASS (n_pad == 512) computes the same FP32 transform as the
 * default form in two passes over every SM instead of one 16-CTA cluster per image (only one
 * such cluster fits a GPC): the row pass writes each sample's row-transformed grid (1 MB) to a
 * scratch buffer the plan allocates on the first call (4 x SMs samples, about 608 MB on 152
 * SMs), the column pass reads it back; no cross-polarisation variant.
 * EPIC_XFORM_DFTGEMM_FP16_GRID (n_pad == 256, single polarisation products only) grids with FP16
 * operands -- each weight and each calibrated voltage rounded to FP16 (normal FP16 range: about
 * 6e-5 to 65504 in magnitude), each product exact in FP32, the cells' sums in FP32 -- and then
 * runs the EPIC_XFORM_DFTGEMM transform (hi+lo operands).  Real weights are read as one packed
 * word per mapping entry (the plan builds these for n_pad 256 when every weight is real).  The
 * error is that of the FP16 roundings of the gridding operands (relative L2 about 1e-4 against
 * the exact image; the stated bound is 3e-3).  epic_image_backward always uses the FFT form.
 */
epic_status epic_set_transform(epic_plan *plan, int xform);

/* Release the plan and its device tables.  NULL is accepted. */
void epic_destroy(epic_plan *plan);

/*
 * epic_sync -- wait for the work enqueued on stream and report what the plan's kernels found on
 * the device.  The kernels that hand operands to the tensor cores (epic_image and
 * epic_image_xpol in the EPIC_XFORM_DFTGEMM form, epic_correlate) wait on the tensor pipe with
 * bounded waits; a wait that runs out sets a bit in the plan's device status word (the kernel
 * then waits, with its full limit, for the products still in flight, releases its tensor memory
 * and returns, marking its first output block with NaN).  The FFT form at N_p = 256 and 512 waits,
 * with a fixed bound of about a second, for the row-pass data its cluster peers send it; a wait
 * that runs out sets another bit.  This call synchronises the stream,
 * reads the word, clears it and returns EPIC_ETIMEOUT if any bit was set (the message names the
 * kernel), EPIC_ECUDA if the stream reported an error, else EPIC_OK.  The imaging calls
 * themselves stay asynchronous.  Not meant for use inside a stream capture.
 */
epic_status epic_sync(const epic_plan *plan, void *stream);

/*
 * epic_set_wait_limit -- tries of each bounded wait of the plan's tensor-core pipelines (each try
 * suspends the waiting thread for up to about 1 ms; default 1000, so a wait gives up after about
 * a second).  0 to 1000000; with 0 every such wait reports a timeout at its first check, which
 * exercises the failure path above without a fault (the waits that drain the products in flight
 * always use the full limit).  Applies to calls enqueued after it.
 */
epic_status epic_set_wait_limit(epic_plan *plan, int tries);

/*
 * epic_image -- the MOFF imaging step (Eq. "dirty-image-MOFF") for one block of samples.
 *
 *   volt      device [T][C][P][A] voltages in the plan's volt_dtype.
 *   n_time    T >= 1.
 *   gains     device [C][P][A] complex64 per-antenna gains applied before gridding
 *             (Sec. 3 "Calibration"), or NULL for unit gains.
 *   accum     device [C][P][N_p][N_p] float64: receives sum_t |F_t(k)|^2.  If t_prev > 0
 *             the sum continues onto the values already there (the integration resumes);
 *             if t_prev == 0 it is overwritten.
 *   power     device [C][P][A] float64 or NULL: receives sum_t |g_a V_a(t)|^2 with the same
 *             continue/overwrite rule.  Required when autocorr != NULL.
 *   t_prev    number of samples already integrated into accum / power (>= 0).
 *   image     device [C][P][N_p][N_p] float32 or NULL: accum / (t_prev + T), the
 *             time-averaged image.
 *   autocorr  device [C][P][N_p][N_p] float32 or NULL: the antenna auto-correlation term
 *             of the averaged image (Sec. 4.2), A(k) = sum_a P_a |K_a(k)|^2 with
 *             P_a = power_a / (t_prev + T) and K_a(k) the transform of antenna a's
 *             gridded footprint.  image - autocorr is the cross-correlation-only image.
 *   stream    cudaStream_t to launch on (NULL = the legacy default stream).
 *
 * Work is split across the whole GPU; accum and power are updated with float64 atomic
 * adds, so their low-order bits may differ between runs.
 */
epic_status epic_image(const epic_plan *plan, const void *volt, int n_time, const float *gains,
                       double *accum, double *power, int64_t t_prev,
                       float *image, float *autocorr, void *stream);

/*
 * epic_image_backward -- adjoint of epic_image with respect to the gains.
 *
 * For a real loss L of the averaged image I = (1/T) sum_t |F_t|^2 of one call (t_prev = 0),
 * given grad_image = dL/dI (device [C][P][N_p][N_p] float32, image pixel order), writes
 * grad_gains = dL/dRe(g) + i dL/dIm(g) (device [C][P][A] complex64), i.e.
 *   grad_a = (2/T) sum_t conj(V_a(t)) sum_g conj(M[g, a]) sum_k G(k) F_t(k) exp(-2 pi i g.k/N_p),
 * the chain rule through Eq. "dirty-image-MOFF" with the gains applied as in Sec. 3
 * "Calibration" (their use in feedback calibration).  The per-sample fields F_t are
 * recomputed, not stored.  volt, n_time and gains are as for epic_image.
 * grad_gains is overwritten (accumulated with float32 atomic adds).  EPIC_EUNSUPPORTED if the
 * adjoint kernel's shared memory cannot hold the plan's antennas at its n_pad (it keeps four
 * per-antenna arrays; e.g. at most about 2,880 antennas at n_pad 128).
 */
epic_status epic_image_backward(const epic_plan *plan, const void *volt, int n_time,
                                const float *gains, const float *grad_image, float *grad_gains,
                                void *stream);

/*
 * epic_image_xpol -- the four instrumental cross-polarisation images of dual-polarisation
 * data (Sec. 3 and the image module of App. A produce all four; Eq. "dirty-image-MOFF" with
 * F_p conj(F_q) in place of |F_p|^2): XX = <|F_X|^2>, YY = <|F_Y|^2>, XY = <F_X conj(F_Y)>,
 * YX = conj(XY), averaged over time, for a plan with n_pol == 2 (pol 0 = X, pol 1 = Y).
 *
 *   volt, n_time, gains  as for epic_image ([T][C][2][A], gains [C][2][A] or NULL).
 *   accum4    device [C][4][N_p][N_p] float64: per channel the time sums of |F_v|^2 for
 *             v = X, Y, X + Y, X + iY (the gridded fields g_X V_X, g_Y V_Y, g_X V_X + g_Y V_Y,
 *             g_X V_X + i g_Y V_Y).  Continued if t_prev > 0, overwritten if t_prev == 0.
 *   t_prev    samples already integrated into accum4 (>= 0).
 *   image     device [C][2][N_p][N_p] float32 (XX, YY), or NULL.
 *   cross     device [C][N_p][N_p] complex64 (XY, interleaved re, im), or NULL.
 *
 * XY follows from the four sums by the polarisation identity, evaluated in float64:
 * Re XY = (S_{X+Y} - S_X - S_Y) / 2T, Im XY = (S_{X+iY} - S_X - S_Y) / 2T.  The forward
 * kernel therefore runs 4 C instead of 2 C (channel, pol) images, in the transform
 * epic_set_transform chose (FP32 FFT or tensor-core DFT-GEMM); no auto-correlation term.
 * EPIC_EINVAL if the plan does not have two pols; EPIC_EUNSUPPORTED if the antennas do not
 * fit the chosen kernel's shared memory.
 */
epic_status epic_image_xpol(const epic_plan *plan, const void *volt, int n_time, const float *gains,
                            double *accum4, int64_t t_prev, float *image, float *cross, void *stream);

/*
 * epic_fengine -- the F-engine (Sec. 3 "Temporal Fourier transform"): the time samples of
 * every antenna, in blocks of n_chan consecutive samples, become electric-field spectra,
 *   volt[t][c][p][a] = sum_{j < C} raw[t C + j][p][a] exp(-2 pi i j c / C),  c = 0 .. C-1,
 * an unnormalised forward DFT without window (bins in FFT order: c > C/2 are negative
 * frequencies), the layout epic_image reads (C channels per call).  No plan is needed.
 *
 *   n_ant, n_pol          A, P.
 *   n_chan                C: 32, 64, 128, 256 or 512 (else EPIC_EUNSUPPORTED).
 *   n_time                T, spectra per antenna (raw holds T C samples per antenna).
 *   in_dtype              raw sample format (one of epic_volt_dtype).
 *   raw                   device [T C][P][A] samples.
 *   out_dtype             EPIC_VOLT_C64 (complex64) or EPIC_VOLT_F16 (FP16 pairs, rounded;
 *                         |values| above 65504 overflow).
 *   volt                  device [T][C][P][A], overwritten.
 *   device                CUDA device of the arrays.
 */
epic_status epic_fengine(int n_ant, int n_pol, int n_chan, int n_time, int in_dtype, const void *raw,
                         int out_dtype, void *volt, int device, void *stream);

/*
 * epic_weff -- the effective weighting of the plan's (possibly heterogeneous) array in the
 * optimally weighted image (Sec. 5, Eq. "effective-weighting-optimal"), on the image pixels:
 *   weff(k) = (1 / (A (A - 1))) sum_{a != b} |K_a(k)|^2 |K_b(k)|^2,
 * K_a(k) the transform of antenna a's gridded footprint (equal to its far-field pattern when
 * the gridding kernels are the instrument's, W^G = W^I).  Channel independent: the pixel
 * grid is in units of the aperture grid.
 *
 *   weff      device [N_p][N_p] float32, image pixel order (k = 0 at (N_p/2, N_p/2)).
 *
 * All padded sizes; EPIC_EUNSUPPORTED for footprints too wide for the lag tables; EPIC_EINVAL
 * for fewer than two antennas.  One CTA per 16 image rows; meant to be called once per plan.
 */
epic_status epic_weff(const epic_plan *plan, float *weff, void *stream);

/*
 * epic_isotropic -- the estimate of the isotropically weighted dirty image (Sec. 5,
 * Eq. "effective-weighting"): iso = I' / weff with I' = (image - autocorr) / (A (A - 1)), the
 * mean weighted fringe over antenna pairs a != b.
 *
 *   image, autocorr  device [C][P][N_p][N_p] float32 from epic_image (the same call).
 *   weff      device [N_p][N_p] float32 from epic_weff.
 *   rel_floor pixels where weff < rel_floor * max(weff) are set to NaN (0 <= rel_floor < 1).
 *   iso       device [C][P][N_p][N_p] float32, overwritten.
 */
epic_status epic_isotropic(const epic_plan *plan, const float *image, const float *autocorr,
                           const float *weff, float rel_floor, float *iso, void *stream);

/*
 * epic_correlate -- the X-engine of the FX route (Sec. 3, the FX flow; Eq. "cc-vis"): the
 * visibilities of every ordered antenna pair of every (channel, pol), autocorrelations
 * included,
 *   vis[c][p][a][b] = g_a conj(g_b) (1/T) sum_t V_a(t) conj(V_b(t)),
 * i.e. the time average of E_a conj(E_b) of the calibrated fields.  vis is Hermitian in (a, b).
 *
 *   volt, n_time, gains  as for epic_image; the plan's voltages must be FP16 or 4+4-bit
 *             (EPIC_EUNSUPPORTED for complex64).  n_time <= 131072.
 *   vis       device [C][P][A][A] complex64, row-major (a, b); overwritten; 8-byte aligned.
 *
 * Computed on the tensor cores as real products of the real and imaginary parts with FP16
 * operands (the voltages are exact in FP16) and FP32 accumulation: for 4+4-bit voltages the
 * sums over the call are exact; the gains and 1/T are applied in FP32 afterwards.  Each call is
 * one integration (no continuation).  The plan's mapping is not used.  4+4-bit voltages with A
 * a multiple of 4 in a 4-byte-aligned array are read 4 antennas per load (faster); any other A
 * or alignment, and FP16 voltages, are read voltage by voltage, with the same results.  Uses
 * about 200 KB of shared memory and all 512 tensor-memory columns of each SM it runs on.
 */
epic_status epic_correlate(const epic_plan *plan, const void *volt, int n_time, const float *gains,
                           float *vis, void *stream);

/*
 * epic_fx_image -- the FX route's imaging of one integration's visibilities (Sec. 3, the FX
 * flow; Eqs. "e-field-conv" and "dirty-image-FX"): the visibilities are gridded with the
 * antenna-pair kernels B_ab(d) = sum_g M[g, a] conj(M[g - d, b]) (the cross-correlation of
 * the two sampled footprints) onto the lag plane and transformed once:
 *   image(k) = Re sum_d U(d) exp(+2 pi i d.k / N_p),  U(d) = sum_{a, b} vis_ab B_ab(d).
 * With vis from epic_correlate (autocorrelations included, same gains) this equals
 * epic_image's time-averaged image (Sec. 2: the two routes are equivalent).
 *
 *   vis       device [C][P][A][A] complex64.
 *   image     device [C][P][N_p][N_p] float32, image pixel order; overwritten.
 *
 * n_pad <= 128 (the lag plane is transformed in shared memory), else EPIC_EUNSUPPORTED;
 * A^2 * C * P below 2^31.  The first call builds, on the host, the plan's table of the
 * antenna-pair kernels grouped by lag cell (B_ab(d) of every ordered pair summed over the two
 * footprints' entries: work grows as the square of the mapping entries, 16 bytes of device
 * memory per (pair, lag) entry, at most 2^27 entries, else EPIC_EUNSUPPORTED), uploads it
 * (synchronously, once) and allocates the plan's imaging scratch (A^2 * C * P * 8 bytes for the
 * visibilities in pair-major order, C * P * n_pad^2 * 8 bytes for the lag planes; EPIC_ENOMEM
 * if that fails).  Every call then transposes vis into the scratch, gathers each lag plane U(d)
 * cell by cell from the table (no atomics) and transforms each once (three launches).  The
 * scratch belongs to the plan: calls on one plan whose kernels may overlap (two streams) race
 * on it, so the caller orders them.
 */
epic_status epic_fx_image(const epic_plan *plan, const float *vis, float *image, void *stream);

/*
 * epic_grid -- the gridding step alone (Sec. 3, gridding convolution): for every sample
 * t and (channel, pol), E_t(g) = sum_a M[g, a] g_a V_a(t) on the plan's N_g x N_g grid
 * (no zero padding, no transform), written to device memory.
 *
 *   volt, n_time, gains  as for epic_image.
 *   grid      device [T][C][P][N_g][N_g] complex64 (interleaved re, im float32), row-major
 *             over (y, x); 8-byte aligned.  Overwritten; caller-owned.
 *
 * This is the form in which the gridded fields leave the chip (e.g. for an external
 * transform); epic_image keeps them on chip.  Returns EPIC_EINVAL for NULL or misaligned
 * arrays and n_time < 1.
 */
epic_status epic_grid(const epic_plan *plan, const void *volt, int n_time, const float *gains,
                      float *grid, void *stream);

/*
 * epic_plan_info -- sizes of the plan (any pointer may be NULL):
 *   nnz       non-zeros of the mapping M(r, a) (cells x antennas);
 *   n_cells   occupied grid cells;
 *   lag_side  side L of the per-antenna footprint auto-correlation tables (L x L lags).
 */
epic_status epic_plan_info(const epic_plan *plan, int64_t *nnz, int64_t *n_cells, int *lag_side);

/*
 * Batches: many plans (e.g. heterogeneous sub-arrays, each with its own antennas, kernels,
 * grid and channels) imaged by one persistent launch per padded-size class, the classes
 * forked onto internal streams and joined back into the caller's stream.  The stacking of
 * data streams for array operations is App. A.3's; the batch object owns its streams, events
 * and (for N_p = 512 classes) the two-pass form's scratch buffers, all allocated by
 * epic_batch_create, so epic_batch_image allocates nothing and can be captured in a CUDA graph.
 * Plans must share the device and the voltage format; at most 64 plans per size class are
 * walked by one launch (more are split into further launches).
 */
typedef struct epic_batch epic_batch;

/* Group n_plans plans (the plans must outlive the batch). */
epic_status epic_batch_create(epic_batch **batch, int n_plans, epic_plan *const *plans);

/*
 * Image every plan of the batch: host arrays of n_plans entries; volt[i], n_time[i],
 * gains[i] (or gains == NULL, or gains[i] == NULL, for unit gains) are as for epic_image;
 * accum[i] is overwritten with sum_t |F_t|^2; image[i] (image == NULL or image[i] == NULL to
 * skip) receives accum[i] / n_time[i].  The FFT form is used for every class.
 */
epic_status epic_batch_image(epic_batch *batch, const void *const *volt, const int *n_time,
                             const float *const *gains, double *const *accum, float *const *image,
                             void *stream);

/*
 * Autotune the batch on representative inputs (same arguments as epic_batch_image; accum is
 * overwritten): for each size class, the kernel form and worker count that run it fastest
 * alone -- the persistent form with all, 3/4 or 1/2 of its resident CTAs (clusters), for
 * N_p = 512 classes also the two-pass form, for N_p = 256 classes also the persistent form with
 * one row-pass buffer -- then whether the classes run faster concurrently
 * or back to back (timed alternately; concurrent unless back to back is more than 2 % faster,
 * the stream fork and join per class that eager timing adds and a captured graph does not).
 * Synchronises the stream; not capturable.  The choice is kept in the batch (epic_batch_class
 * reports it).
 */
epic_status epic_batch_autotune(epic_batch *batch, const void *const *volt, const int *n_time,
                                const float *const *gains, double *const *accum, void *stream);

/* The batch's size classes, whether they run concurrently, and the worker cap of each class
 * (0 = all resident; at most max_workers entries written).  Any pointer may be NULL. */
epic_status epic_batch_info(const epic_batch *batch, int *n_classes, int *concurrent, int *workers,
                            int max_workers);

/* Size class k of the batch (0 .. n_classes - 1): its padded size, its worker cap (0 = all
 * resident) and its kernel form, 0 = persistent (one CTA or cluster per image in flight), 1 =
 * two-pass (N_p = 512 classes: a row pass and a column pass over every SM with the row-
 * transformed grids staged in a scratch buffer the batch allocates at creation, 4 x SMs samples
 * of 1 MB for each such class), 2 = persistent with one row-pass buffer (N_p = 256 classes: a
 * cluster barrier per image instead of two buffers used alternately).  The form is what
 * epic_batch_autotune chose (persistent until then).  Any out-pointer may be NULL. */
epic_status epic_batch_class(const epic_batch *batch, int k, int *n_pad, int *workers, int *form);

/* Release the batch (not its plans).  NULL is accepted. */
void epic_batch_destroy(epic_batch *batch);

/*
 * epic_image_noalloc -- epic_image for an n_pad == 512 plan, in the two-pass form, that allocates
 * no device memory.  The paper has no counterpart: this call exists for callers that cannot call
 * cudaMalloc while they image -- a pipeline whose device memory is all reserved up front by
 * another allocator, or a real-time data path that may not stop on an allocation between
 * samples.  The two-pass form stages each sample's row-transformed grid (1 MB) in scratch
 * memory; instead of a buffer of the plan (EPIC_XFORM_FFT_TWOPASS allocates one), this call uses
 * a device array built into the library: 64 MB, held by every GPU that loads the library until
 * the process exits.
 *
 *   volt, n_time, gains, accum, power, t_prev, image, autocorr, stream
 *               as for epic_image (the plan's transform setting is not used).
 *   chunk_items samples staged per pass, 1 .. 64 (the array's capacity); a larger value is
 *               EPIC_EINVAL before anything is launched.  Any number of samples is imaged, in
 *               chunks of this size; more samples per chunk keep more SMs busy.
 *
 * The first call on a device looks up the array's device address (with that device current) and
 * keeps it; make that first call before any stream capture that might include this call.  Every
 * call on a device shares the array and leaves its last chunk's rows in it; nothing in it needs
 * to start at zero.  Calls whose kernels overlap on the GPU (two streams, or two host threads)
 * race on the array: order them.  The call performs no cudaMalloc, cudaFree or other allocation.
 */
epic_status epic_image_noalloc(const epic_plan *plan, const void *volt, int n_time, const float *gains,
                               double *accum, double *power, int64_t t_prev, float *image, float *autocorr,
                               int chunk_items, void *stream);

/* Thread-local message for the last failing call on this thread ("" if none). */
const char *epic_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* EPIC_H */

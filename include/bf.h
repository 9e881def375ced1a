/*
 * bf.h -- C ABI of the GB300 plane-wave receive beamformer (libbf.so).
 *
 * The library forms B-mode images from plane-wave channel data as the paper
 * describes (Sec. II-B): for every pixel and receive channel it computes the
 * transmit + receive time of flight, linearly interpolates the channel's RF,
 * applies the F-number aperture, and combines the channels by delay-and-sum
 * (Eq. (1)), by signed-square-root delay-multiply-and-sum, or by
 * coherence-factor-weighted DAS; results are compounded over plane-wave
 * angles, then optionally envelope-detected along depth (the DMAS image
 * through a [f0, 3 f0] band-pass) and log-compressed to the -70 dB dynamic
 * range the paper's images are shown with (Fig. 3).
 *
 * Definitions every entry point follows (all positions in metres):
 *   element i:  x_i = x_elem_m[i] if given, else (i - (N - 1) / 2) * pitch_m, z_i = 0
 *   pixel (ix, iz):  x_p = x0 + ix * ((x1 - x0) / (nx - 1))   (x0 when nx == 1),
 *                    z_p = z0 + iz * ((z1 - z0) / (nz - 1))   (z0 when nz == 1)
 *   fractional sample index (time zero when the wavefront crosses the array centre):
 *       n = (x_p sin(theta) + z_p cos(theta) + sqrt((x_p - x_i)^2 + z_p^2)) * (fs / c)
 *   channel active:  |x_p - x_i| <= z_p / (2 F)               (inclusive boxcar)
 *   sample:  k = floor(n); v = (1 - (n - k)) u[k] + (n - k) u[k + 1] if 0 <= k <= Ns - 2, else 0
 *   DAS  = sum_theta sum_active v
 *   DMAS = sum_theta ((sum s)^2 - sum s^2) / 2,  s = sign(v) sqrt|v|
 *   CF   = (DAS^2 / (M * sum_theta sum_active v^2)) * DAS, M = active (angle, channel) pairs;
 *          0 when the denominator is 0
 *   pDAS = sum_theta sign(t) |t|^p,  t = sum_active sign(v) |v|^(1/p)   (Eq. (2)-(3); p per handle)
 * The two discrete decisions (aperture membership and 0 <= k <= Ns - 2) are
 * taken on the host in double precision with exactly the expressions above,
 * evaluated left to right without fused multiply-adds; the per-pixel
 * arithmetic runs on the GPU in FP32.
 *
 * Threading: a handle may be used from one thread at a time.  Different
 * handles may be used concurrently.  All device work of a handle is ordered
 * on its stream (bf_set_stream; default: a stream the library creates).
 *
 * Errors: functions return BF_OK (0), BF_PENDING (1) or a negative BF_E*
 * code; nothing is thrown across the ABI.  bf_last_error() returns a
 * thread-local description of the last failure on the calling thread.
 */
#ifndef BF_H
#define BF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define BF_API __attribute__((visibility("default")))
#else
#define BF_API
#endif

/* Linear receive array.  x_elem_m (optional, n_elements entries, strictly
 * increasing) overrides the uniform centred layout.  f_number > 0. */
typedef struct bf_geometry {
    int32_t n_elements;
    double pitch_m;
    const double *x_elem_m;
    double f_number;
} bf_geometry;

/* Pixel grid: inclusive linspaces, x1 >= x0, z1 >= z0 >= 0, nx, nz in [1, 32767]. */
typedef struct bf_grid {
    int32_t nx, nz;
    double x0_m, x1_m, z0_m, z1_m;
} bf_grid;

typedef struct bf_handle bf_handle;
typedef struct bf_batch bf_batch;

/* mode_and_flags: combiner bits (any non-empty subset) ... */
enum { BF_DAS = 1, BF_DMAS = 2, BF_CF = 4, BF_PDAS = 8, BF_MODE_MASK = 15 };
/* ... RF storage precision on the device (bits 4-5; interpolation and sums are always FP32) ... */
enum { BF_PREC_FP32 = 0, BF_PREC_FP16 = 1 << 4, BF_PREC_BF16 = 2 << 4, BF_PREC_MASK = 3 << 4 };
/* ... and the output stage (bits 8-9). */
enum { BF_OUT_RF = 0, BF_OUT_ENV = 1 << 8, BF_OUT_LOGDB = 2 << 8, BF_OUT_MASK = 3 << 8 };
/* IQ combiners (bits 12-13; not with the RF combiners above in one call, FP32
 * storage, n_samples a power of two <= 8192): each channel record is
 * demodulated to complex baseband (analytic signal times exp(-j 2 pi f0 k / fs)),
 * interpolated linearly at the delay and re-modulated by exp(j 2 pi f0 n / fs):
 *   IQ-DAS  = |sum_theta sum_active s|                        (Sec. II-B-1)
 *   BB-DMAS = |sum_theta ((1/M) sum_active sqrt|s| e^{j arg s})^2|, M = channels
 *             inside the aperture                             (Eq. (4))
 * Their outputs are magnitude images: BF_OUT_RF and BF_OUT_ENV both return
 * them, BF_OUT_LOGDB their -70 dB log compression. */
enum { BF_IQDAS = 1 << 12, BF_BBDMAS = 1 << 13, BF_IQ_MASK = 3 << 12 };
/* bf_fkmig only: Stolt's mapping instead of the exact plane-wave one (bit 16). */
enum { BF_FK_STOLT = 1 << 16 };
/* bf_submit_many_into only: the destinations lie in one allocation (bit 17),
 * so that destinations back to back leave in one transfer. */
enum { BF_DEST_ONE_BUFFER = 1 << 17 };

enum {
    BF_OK = 0,
    BF_PENDING = 1,      /* bf_poll: result not ready yet */
    BF_EINVAL = -1,      /* bad argument (message in bf_last_error) */
    BF_EAGAIN = -2,      /* admission refused: no ring slot / device memory now; retry later */
    BF_ENOMEM = -3,      /* a device or host allocation failed */
    BF_ECUDA = -4,       /* a CUDA call failed */
    BF_ETIMEDOUT = -5,   /* bf_poll deadline passed, or a device-side bounded wait gave up */
    BF_ENOTFOUND = -6,   /* unknown ticket */
    BF_ENOSYS = -7       /* feature not available in this build */
};
/* Error-path testing: the environment variable BF_FAULT, a comma-separated
 * list read on every use, injects failures on the host: alloc (device
 * allocations fail with BF_ENOMEM), submit (admission refuses requests with
 * BF_EAGAIN), copy (a request's RF copy fails with BF_ECUDA).  Unset in
 * normal use.  bf_selftest_wait exercises the device-side bounded wait. */

/* Paper: Sec. II-B (array, pixel grid and the time of flight of Eq. (1)).
 * Create a handle for one geometry and pixel grid.  fs_hz: sampling rate,
 * f0_hz: transmit centre frequency (sets the DMAS band-pass), c_mps: speed
 * of sound.  Uploads the geometry tables to the current CUDA device.
 * *out receives the handle (caller owns it; free with bf_destroy). */
BF_API int bf_create(const bf_geometry *geometry, const bf_grid *grid, double fs_hz,
                     double f0_hz, double c_mps, bf_handle **out);

/* Paper: no counterpart (resource lifetime of this implementation).
 * Free a handle and its device memory.  BF_EINVAL while tickets are pending;
 * the handle stays valid then. */
BF_API int bf_destroy(bf_handle *h);

/* Paper: no counterpart (stream ordering of this implementation).
 * Device stream for all of this handle's work (a cudaStream_t; NULL = the
 * library's own non-blocking stream).  The caller keeps ownership of the
 * stream and must keep it alive while the handle uses it. */
BF_API int bf_set_stream(bf_handle *h, void *cuda_stream);

/* Paper: Sec. II-B-3 (Lu's and Stolt's f-k migrations, which the paper
 * evaluates next to the beamformers).  Plane-wave f-k migration of one
 * device-resident frame: per angle the records' spectrum along time
 * (zero-padded to nt, the power of two >= 2 n_samples), the transmit's lateral
 * delay x_i sin(theta) / c removed, the spectrum along the elements
 * (zero-padded to nk >= 2 n_elements), then every output wavenumber
 * (Kx, Kz > 0) takes the spectrum at a temporal frequency, interpolated
 * linearly and weighted by the mapping's Jacobian; the angles' spectra are
 * summed and transformed back.  The mapping:
 *   default: the exact one of the delay model above, f = c k / (2 pi),
 *     k = (Kx^2 + Kz^2) / (2 (Kx sin + Kz cos)), where the receive wave
 *     propagates;
 *   BF_FK_STOLT: Stolt's, for the exploding reflector fitted to the
 *     plane-wave two-way time at the scatterer's lateral position (velocity
 *     c / b, b = sqrt(1 + cos - sin^2 / 2)): f = c sqrt(Kx^2 + Kz'^2) / (2 pi b),
 *     Kz' = (Kz - Kx sin) / b, the shear and scale that map the exploding
 *     reflector's image back onto the native grid, where Kz' > 0.
 * The mapping is tabulated on the host in double precision (kept while the
 * sample count, angles and mapping stay the same); the device only gathers.
 * Output on the native grid, not the handle's pixel grid: out_dev float
 * [n_elements][n_samples], column i at element i, row m at depth m c / (2 fs),
 * holding |image| (flags BF_OUT_RF or BF_OUT_ENV) or its -70 dB log
 * compression (BF_OUT_LOGDB); no flag bits besides these and BF_FK_STOLT.
 * Needs equally spaced elements (2 to 2048), 2 <= n_samples <= 4096; BF_EINVAL
 * otherwise.  Enqueued on the handle's stream; uses scratch owned by the
 * handle. */
BF_API int bf_fkmig(bf_handle *h, const int16_t *rf_dev, int32_t n_samples,
                    const double *angles_rad, int32_t n_angles, uint32_t mode_and_flags,
                    float *out_dev);

/* Paper: Eq. (2)-(3), Sec. II-B-2.
 * Order p of the pDAS combiner of this handle: each delayed sample is
 * compressed to sign(v) |v|^(1/p) before the channel sum, and the sum is
 * raised back to sign(t) |t|^p per angle.  1 <= p <= 16 (BF_EINVAL
 * otherwise); default 2.  Applies to work enqueued or submitted after the
 * call (a prepared batch keeps the value it was created with). */
BF_API int bf_set_pdas_order(bf_handle *h, double p);

/* Paper: no counterpart (buffer sizing).
 * Bytes of one output for the given mode_and_flags: images * nx * nz * 4. */
BF_API size_t bf_output_bytes(const bf_handle *h, uint32_t mode_and_flags);

/* Paper: Sec. II-B, Eq. (1) (delay, interpolation, apodization, sum), the
 * B-mode display of Fig. 3 (envelope, -70 dB), timed as in Sec. III-B.
 * Stream-ordered beamforming of one frame, device-resident data.
 * rf_dev: device int16 [n_angles][n_elements][n_samples] (read during the call's
 * stream work), angles_rad: host array of n_angles plane-wave angles in
 * (-pi/2, pi/2); out_dev: device float [images][nx][nz] (one image per selected
 * combiner in bit order DAS, DMAS, CF, pDAS, IQ-DAS, BB-DMAS; z fastest)
 * receiving the stage selected by BF_OUT_*.
 * The envelope of the DMAS image goes through the [f0, 3 f0] band-pass; the
 * other images are used as they are.
 * Returns after enqueueing; the caller synchronises the stream.  Calls on one
 * handle share its scratch memory and must be ordered on its stream. */
BF_API int bf_beamform(bf_handle *h, const int16_t *rf_dev, int32_t n_samples,
                       const double *angles_rad, int32_t n_angles, uint32_t mode_and_flags,
                       float *out_dev);

/* Paper: Sec. II-B, Eq. (1); the one-frame-per-call GPU execution of Sec. II-A.
 * The same computation as bf_beamform (FP32 storage only) through the plain
 * baseline kernel: one frame per launch, one thread per pixel, records read
 * from global memory without staging.  Kept to measure the batched and served
 * paths against. */
BF_API int bf_beamform_plain(bf_handle *h, const int16_t *rf_dev, int32_t n_samples,
                             const double *angles_rad, int32_t n_angles, uint32_t mode_and_flags,
                             float *out_dev);

/* Paper: the front end streams frames to the host GPU one after another
 * (Sec. II-A); request queueing and batching have no counterpart there.
 * Asynchronous submission (serving path).  rf: host or device int16
 * [n_angles][n_elements][n_samples]; it is copied (host -> pinned staging ->
 * device ring slot) before the call returns, so the caller may reuse it.
 * *ticket_out identifies the request.  BF_EAGAIN when no slot or device
 * memory is free right now. */
BF_API int bf_submit(bf_handle *h, const int16_t *rf, int32_t n_samples,
                     const double *angles_rad, int32_t n_angles, uint32_t mode_and_flags,
                     uint64_t *ticket_out);

/* Paper: the image of one frame the front end streamed in (Sec. II-A) comes
 * back beamformed as bf_beamform computes it (Sec. II-B, Eq. (1), Fig. 3);
 * request tickets have no counterpart.
 * Wait up to timeout_us (0: do not wait; < 0: wait without limit) for a
 * ticket.  BF_PENDING (timeout_us == 0) or BF_ETIMEDOUT (timeout passed) if
 * not ready, leaving the ticket valid; BF_OK after copying the result into
 * out (host or device, out_bytes >= bf_output_bytes; out == NULL discards
 * it), which releases the ticket; other negative codes release it too.
 * BF_ENOTFOUND for an unknown or already released ticket. */
BF_API int bf_poll(bf_handle *h, uint64_t ticket, float *out, size_t out_bytes,
                   int64_t timeout_us);

/* Paper: as bf_submit.  n frames of one geometry, sample count, angle set and
 * flags in one call: rf[k] (host or device) is frame k, tickets_out[k] its
 * ticket.  Every source has been copied when the call returns (one wait for
 * all the copies instead of one per frame; device and page-locked sources
 * move by DMA on several streams).  The engine forms no batch from
 * pending work while the call admits its frames (unless a full batch is
 * pending), so the call's frames ride together.  *n_submitted (optional)
 * receives how many frames got tickets: on BF_EAGAIN the rest can be
 * submitted later. */
BF_API int bf_submit_many(bf_handle *h, int32_t n, const int16_t *const *rf, int32_t n_samples,
                          const double *angles_rad, int32_t n_angles, uint32_t mode_and_flags,
                          uint64_t *tickets_out, int32_t *n_submitted);

/* Paper: as bf_submit; the front end's frames stream in while earlier images
 * leave (Sec. II-A).  bf_submit_many with a destination per frame: outs[k]
 * (host or device, out_bytes >= bf_output_bytes each) receives frame k's
 * result as soon as its batch finishes, copied by the batch itself, so that
 * the transfer of one batch's images overlaps the next batch's kernels
 * without the caller waiting in between.  Device destinations and host
 * memory from cudaHostAlloc / cudaMallocHost are written directly; other host
 * memory through the engine's page-locked staging, copied on by the poll.
 * Each destination must stay valid and untouched until its ticket is polled:
 * bf_poll / bf_poll_many then only wait (their out / outs arguments are
 * ignored for these tickets) and release.  With BF_DEST_ONE_BUFFER in
 * mode_and_flags the caller states that every outs[k] lies in one allocation
 * (views of one buffer): the results of frames whose destinations follow one
 * another in memory (outs[k + 1] == outs[k] + bf_output_bytes / 4) then leave
 * their batch in one transfer.  Errors as bf_submit_many, plus BF_EINVAL for
 * a null or too small destination. */
BF_API int bf_submit_many_into(bf_handle *h, int32_t n, const int16_t *const *rf,
                               int32_t n_samples, const double *angles_rad, int32_t n_angles,
                               uint32_t mode_and_flags, float *const *outs, size_t out_bytes,
                               uint64_t *tickets_out, int32_t *n_submitted);

/* Paper: as bf_poll.  Waits up to timeout_us for all n tickets, then copies
 * every result into outs[k] (host or device, out_bytes each; outs or outs[k]
 * NULL discards) with one synchronisation at the end and releases every
 * ticket; returns the first failure of any ticket (all are released).  On
 * BF_PENDING / BF_ETIMEDOUT / BF_ENOTFOUND nothing is released.  Device
 * destinations and host destinations from cudaHostAlloc / cudaMallocHost are
 * written by one DMA copy each, spread over several streams so that the copy
 * engines run beside the next batch's kernels; other host memory (pageable,
 * or registered with cudaHostRegister) goes through the engine's page-locked
 * staging buffer. */
BF_API int bf_poll_many(bf_handle *h, int32_t n, const uint64_t *tickets, float *const *outs,
                        size_t out_bytes, int64_t timeout_us);

/* Paper: no counterpart (serving-engine introspection of this implementation).
 * The batch a launched ticket rides in and how
 * many frames that batch holds (BF_PENDING while still queued). */
BF_API int bf_ticket_batch(bf_handle *h, uint64_t ticket, int32_t *batch_id,
                           int32_t *batch_frames);

/* Paper: no counterpart (latency measurement of the serving engine).
 * Device time of a ticket's batch once it has finished: when the batch began
 * and ended executing, in ms since the engine started (BF_PENDING before). */
BF_API int bf_ticket_times(bf_handle *h, uint64_t ticket, double *start_ms, double *end_ms);

/* Paper: no counterpart (serving-engine control).
 * Hold (paused != 0) or resume the serving engine's launches on the current
 * device.  Submissions are still admitted while paused; on resume everything
 * queued is launched as batches. */
BF_API int bf_engine_pause(int32_t paused);

/* Paper: no counterpart (serving-engine control).
 * Serving-engine knobs for the current device (values <= 0 keep the current
 * setting): frames per launched batch (default 64), batches in flight
 * (default 3), device memory budget of admitted requests in bytes (default
 * half the device, or BF_MEM_BUDGET_MB from the environment). */
BF_API int bf_engine_configure(int32_t max_batch, int32_t max_inflight,
                               uint64_t memory_budget_bytes);

/* Paper: no counterpart (error reporting of this implementation).
 * Wait for the handle's stream and report device-side failures of its
 * bf_beamform work (BF_ETIMEDOUT when a bounded wait inside a kernel gave up). */
BF_API int bf_sync(bf_handle *h);

/* One frame of a batch: its handle (grid, geometry), device RF, host angles,
 * mode/flags and device output (layout as bf_beamform). */
typedef struct bf_frame {
    bf_handle *h;
    const int16_t *rf_dev;
    int32_t n_samples;
    const double *angles_rad;
    int32_t n_angles;
    uint32_t mode_and_flags;
    float *out_dev;
} bf_frame;

/* Paper: no counterpart (the paper beamforms one frame per call); each frame
 * is computed as bf_beamform computes it (Sec. II-B, Eq. (1)).
 * Prepare a batch of frames with uneven grids and angle counts: builds the
 * per-frame tables and one flat work list over all (frame, pixel tile) items
 * and captures the batch's kernels in a CUDA graph.  The frame descriptors
 * are copied; the RF and output buffers must stay valid while the batch is
 * launched. */
BF_API int bf_batch_create(const bf_frame *frames, int32_t n_frames, bf_batch **out);
/* Paper: as bf_batch_create.  Launch a prepared batch on a stream
 * (cudaStream_t; NULL = default stream): replays its CUDA graph. */
BF_API int bf_batch_launch(bf_batch *b, void *cuda_stream);
/* Paper: no counterpart (error reporting).  Synchronise the stream and report
 * device-side failures of the batch's launches. */
BF_API int bf_batch_status(bf_batch *b, void *cuda_stream);
/* Paper: no counterpart (per-stage timing; the paper times whole
 * reconstructions, Sec. III-B).
 * Device time of the last completed replay, from events captured in the graph
 * on a side branch (each event node follows the stage it closes; no kernel
 * waits on one): ms3[0] ingest (+ resets), ms3[1] beamforming launches,
 * ms3[2] envelope + log.
 * *kernel_launches (optional) receives the number of kernels one replay runs. */
BF_API int bf_batch_timing(bf_batch *b, float *ms3, int32_t *kernel_launches);
/* Paper: no counterpart.  Free a batch (its graph, tables and scratch); the
 * caller's RF and output buffers are not touched. */
BF_API int bf_batch_destroy(bf_batch *b);

/* Paper: the F-number aperture and the record bound of Sec. II-B.
 * Host-only diagnostic (touches no GPU): the double-precision decision
 * tables the device path consumes.  valid_rows [n_angles][nx][n_elements][2]
 * receives the first and last pixel row iz at which channel i's sample
 * counts for column ix and angle a (inside the aperture and
 * 0 <= floor(n) <= Ns - 2; (-1, -1) when none); aperture_count [nx][nz]
 * the number of channels inside the aperture of each pixel.  Either output
 * may be NULL. */
BF_API int bf_host_tables(const bf_geometry *geometry, const bf_grid *grid, double fs_hz,
                          double f0_hz, double c_mps, int32_t n_samples,
                          const double *angles_rad, int32_t n_angles, int32_t *valid_rows,
                          uint16_t *aperture_count);

/* Paper: no counterpart (tiling of this implementation).
 * Plan introspection (builds the plan if needed): info8 receives
 * {window pairs staged per channel, TMA box width, channels per stage, rows
 * per thread, tiles across, tiles down, pairs per channel record, entries of
 * the window table}; wtab (optional, wtab_entries >= info8[7]) the first
 * staged pair of every (angle, tile, channel) window, INT32_MIN when no pixel
 * of the tile counts that channel.  Pair j of a record holds samples j - 2
 * and j - 1.  Tiles are 32 columns wide and 8 * rows deep, numbered across
 * first. */
BF_API int bf_plan_info(bf_handle *h, int32_t n_samples, const double *angles_rad,
                        int32_t n_angles, uint32_t mode_and_flags, int32_t *info8, int32_t *wtab,
                        size_t wtab_entries);

/* Paper: no counterpart (tile shape of this implementation).
 * Autotuner: times the beamforming launches of `frames` (1-256) frames of
 * this workload (grid of the handle, n_samples, angles, the combiner and
 * precision bits of mode_and_flags; the output stage is ignored) under each
 * tile configuration the library knows (rows per thread x channels per
 * pipeline stage), on synthetic zero records, and keeps the fastest: later
 * bf_beamform, bf_submit and bf_batch_create work on this workload uses it.
 * Synchronous; allocates scratch for the frames while it runs.  Optional
 * outputs: the chosen rows per thread and stage bytes, and the median
 * beamforming time in microseconds of every candidate (n_candidates
 * entries; -1 where a configuration does not fit).  Two-row tiles (16 rows,
 * up to four frames of one workload per job sharing every delay) serve DAS
 * and DMAS of RF records and IQ-DAS / BB-DMAS; other work on a workload
 * tuned to them keeps the default tiles.  The environment variable
 * BF_TILE_ROWS=2, 4 or 8 overrides any tuned choice. */
BF_API int bf_autotune(bf_handle *h, int32_t n_samples, const double *angles_rad,
                       int32_t n_angles, uint32_t mode_and_flags, int32_t frames,
                       int32_t *rows_out, int32_t *stage_bytes_out, float *candidate_us,
                       int32_t n_candidates);

/* Paper: no counterpart (safety of this implementation).
 * Self-test of the device-side bounded waits every beamforming kernel uses:
 * launches one warp that waits on a barrier phase nothing completes, for
 * timeout_us microseconds (1 .. 1000000) of the device's global timer, on a
 * private stream of the current device, and waits for it.  Returns
 * BF_ETIMEDOUT when the wait ran out and the kernel reported it (the expected
 * outcome: the path a CTA whose copies never land takes; the CUDA context
 * stays usable), BF_EINVAL for a timeout out of range, BF_ECUDA on a CUDA
 * error. */
BF_API int bf_selftest_wait(int64_t timeout_us);

/* Allocation-free envelope + log compression, for callers that cannot
 * allocate device memory while running (a real-time acquisition loop that
 * must not enter cudaMalloc, an application whose device memory belongs to
 * its own allocator).  The paper has no counterpart: it is a deployment
 * variant of the BF_OUT_LOGDB stage.
 * y_dev: device float [nx][nz] beamformed image (e.g. one mode of a
 * bf_beamform BF_OUT_RF output); db_dev: device float [nx][nz] receiving
 * 20 log10(env / max env) clipped to [-70, 0] dB, env the analytic-signal
 * magnitude along z, through the [f0, 3 f0] band-pass when bandpass != 0
 * (the DMAS image); z0_m, z1_m: the grid's depth range (sets the band).
 * Limits: nz a power of two <= 4096 and nx * nz <= 2^20; BF_EINVAL beyond.
 * Scratch: a fixed 4 MiB array inside the library (held by every GPU that
 * loads it until exit); no cudaMalloc, cudaFree or other allocating routine is
 * called.  Every call shares that array and leaves its contents behind, so
 * calls that overlap on the GPU (different streams, no ordering) race.  The
 * first call on a device looks up the array's device address; make that first
 * call before any stream capture.  Enqueued on cuda_stream (NULL: default
 * stream); returns after enqueueing. */
BF_API int bf_logdb_static(const float *y_dev, int32_t nx, int32_t nz, double z0_m, double z1_m,
                           double f0_hz, double c_mps, int32_t bandpass, float *db_dev,
                           void *cuda_stream);

/* Paper: no counterpart (error reporting of this implementation).
 * Thread-local message of the last failure on the calling thread ("" if
 * none).  The string belongs to the library and stays valid until the next
 * failing call on the same thread. */
BF_API const char *bf_last_error(void);

/* Paper: no counterpart.  Library version: major * 10000 + minor * 100 + patch. */
BF_API int bf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BF_H */

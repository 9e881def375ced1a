// Internal declarations shared by the host engine (C++) and the kernels (CUDA).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace bfi {

// RF sample pairs are stored per channel with this many zero samples in front,
// so that pair j holds samples k = j - kPadL and k + 1.  Samples before 0 and
// from Ns on read as zero, which makes the interpolation continuous across the
// record ends (the host tables decide which samples count).
constexpr int kPadL = 2;
// Pixel tile of one CTA: 32 columns (one per lane) x kWarps * rows-per-thread
// rows (each consumer warp a contiguous band of rows); one more warp issues
// the tensor-memory-accelerator copies.
constexpr int kTileCols = 32;
constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kMaxGroup = 24;         // channels staged per pipeline stage (upper bound)
constexpr int kMaxStages = 3;         // pipeline stages in shared memory (at most)
constexpr int kMaxBox = 256;          // TMA box extent limit per dimension
constexpr int kMaxSmemPerCta = 227 << 10;  // dynamic shared memory one CTA may use
constexpr int kNoWindow = (int)0x80000000;  // window table: no sample of this channel counts
// Columns of the per-(channel, column) tables are padded to a multiple of 4
// so that every table row starts 16-byte aligned (a tensor-map requirement).
inline int pad_cols(int nx) { return (nx + 3) / 4 * 4; }
inline int tile_rows(int rows_per_thread) { return kWarps * rows_per_thread; }

// Tile configurations the autotuner chooses from: rows per thread (tile
// height 8 * rows) and the target bytes of one pipeline stage's sample
// windows (channels per stage).  Entry 0 is the default.  Two-row tiles serve
// DAS / DMAS of RF records and IQ-DAS / BB-DMAS, with up to four frames per
// job.
struct TileConfig {
    int rows, stage_bytes;
};
constexpr TileConfig kTileConfigs[] = {{4, 24 << 10}, {4, 16 << 10}, {4, 32 << 10}, {8, 24 << 10},
                                       {2, 14 << 10}, {2, 12 << 10}, {2, 17 << 10}};
// Pipeline stages of a beamforming CTA: two deep stages (up to 22 channels of
// four frames, the most that keep two CTAs per SM) for two-row tiles, three
// otherwise (measured fastest for each).
__host__ __device__ constexpr int stages_for_rows(int rows) { return rows == 2 ? 2 : 3; }
constexpr int kNumTileConfigs = 7;
// Frames of one plan that one beamforming job may carry (sharing every delay).
constexpr int kMaxFramesPerJob = 4;

// Storage of the staged records: RF sample pairs in FP32 (mid, diff), FP16 or
// BF16, or complex analytic-signal pairs for IQ beamforming (kPrecIQ, FP32).
enum Prec : int { kPrecF32 = 0, kPrecF16 = 1, kPrecBF16 = 2, kPrecIQ = 3 };

// Device-side error bits (written with atomicOr into a per-launch word).
enum DevErr : int { kErrTimeout = 1, kErrWindow = 2, kErrConfig = 4 };

// Everything one frame needs inside the beamforming kernel.  All pointers are
// device pointers owned by the handle / batch that built the job.
struct BfJob {
    const int *colK;      // [na][nx]  nearest integer of kappa * x_p * sin(theta)
    const float *colF;    // [na][nx]  remainder
    const int *rowK;      // [na][nz]  nearest integer of kappa * z_p * (1 + cos(theta))
    const float *rowF;    // [na][nz]  remainder
    const float *rowZ;    // [nz]      kappa * z_p
    const int *wtab;      // [na][tiles][ne] first staged pair of each tile's channel window
    const int *btab;      // [na][tiles][ne] per row band b: bit b some pixel counts the
                          // channel, bit 8 + b every pixel of the band does
    const uint16_t *apcnt;// [nx][nz]  channels inside the aperture (CF denominator)
    const CUtensorMap *rf_map;     // sample pairs [na * ne][nsp]
    const CUtensorMap *valid_map;  // int2 [na * ne][nxp]: first / last counted row, (-1, -1) if none
    const CUtensorMap *dx2_map;    // float [ne][nxp]: max((kappa * (x_p - x_i))^2, 1e-30)
    float *y;             // [nmodes][nx][nz] beamformed output
    // further frames of the same plan sharing every delay (multi-frame jobs;
    // null otherwise): their outputs.  rf_map then covers all the job's
    // frames, interleaved by frame ([row][pair][frame]), and box counts pairs
    // per frame of one copy.
    float *y_more[kMaxFramesPerJob - 1];
    // IQ jobs: the further frames' image maxima (as maxbits below; null where
    // that frame's images do not feed the log stage)
    unsigned *maxbits_more[kMaxFramesPerJob - 1];
    int nx, nz, na, ne;
    int wmax;             // window length (pairs) staged per channel and tile
    int box;              // TMA box width (pairs); wmax is a multiple of it
    int group;            // channels per stage
    int rows;             // rows per thread (tile height = kWarps * rows)
    int modes;            // BF_DAS | BF_DMAS | BF_CF | BF_PDAS
    int tiles_x, tiles_z;
    float out_scale;      // 1 (FP32 pairs) or 32768 (FP16 / BF16 data scaled by 2^-15)
    float pdas_p;         // order p of the pDAS combiner
    float pdas_inv_p;     // 1 / p
    // IQ beamforming: the carrier phase 2 pi (f0 / fs) (alpha' + 1/2) of the
    // fractional offset alpha' in [-1/2, 1/2] is fma(alpha', iq_c1, iq_c2);
    // maxbits (non-null when the magnitude images feed the log stage) receives
    // each image's maximum (float bits), one word per output slot.
    float iq_c1, iq_c2;
    unsigned *maxbits;
};

// Inputs of the per-plan window planner (one job per plan).
struct PlanJob {
    const int *colK;
    const float *colF;
    const int *rowK;
    const float *rowF;
    const float *rowZ;
    const int2 *valid;    // [na][ne][nxp]
    const float *dx2;     // [ne][nxp]
    int *wtab;            // [na][tiles][ne]
    int *btab;            // [na][tiles][ne]
    int nx, nxp, nz, na, ne, rows, tiles_x, tiles_z, wmax, align;
};

// One frame's int16 records to staged sample pairs.
struct IngestJob {
    const int16_t *rf;    // [rows][ns]
    void *pairs;          // [rows][nsp], or [rows][nsp][nf] for nf > 1 (frames interleaved)
    int rows, ns, nsp;
    unsigned *maxbits;    // the frame's 4 image maxima, zeroed by the job's first CTA (or null)
    // the other frames of a multi-frame beamforming job (nf > 1): their records
    // and maxima; pair j of frame f lands at [row][j][f]
    int nf;
    int chunks;           // CTAs per record row: nf * nsp / 8 threads of 256 per CTA
    const int16_t *rf_more[kMaxFramesPerJob - 1];
    unsigned *maxbits_more[kMaxFramesPerJob - 1];
};

// One frame's int16 records to complex analytic-signal pairs for IQ
// beamforming: per record the analytic signal a[k] (one-sided spectrum of a
// power-of-two-length FFT), then pair j (samples k = j - kPadL and k + 1)
// holds mid = (A + B) / 2 and diff = B - A with A = a[k],
// B = a[k + 1] exp(-j 2 pi f0 / fs) (zero outside the record).
//
// Frames of a multi-frame IQ job (nf = 2 or 4) are demodulated in frame pairs
// (frames fi and fi + 1 of the job, one job entry per pair) into the lead
// frame's array, interleaved for the beamformer's paired arithmetic: per pair
// index j a block of 4 nf floats, and in it per frame pair q = fi / 2 eight
// floats (mid.re, mid.im, diff.re, diff.im, each for frames 2q and 2q + 1).
struct DemodJob {
    const int16_t *rf;    // [rows][ns] (the pair's first frame)
    const int16_t *rf2;   // nf > 1: the pair's second frame
    float4 *pairs;        // nf == 1: [rows][nsp] (mid.re, mid.im, diff.re, diff.im)
    int rows, ns, nsp, lgn;
    int nf, fi;           // frames of the beamforming job, the (first) frame's index in it
    unsigned *maxbits2;   // nf > 1: the second frame's image maxima (or null)
    float2 rot;           // exp(-j 2 pi f0 / fs)
    const float2 *tw;     // [ns] exp(-2 pi i k / ns)
    unsigned *maxbits;    // the frame's image maxima, zeroed by the job's first CTA (or null)
};

// Plane-wave f-k migration of one frame (all its angles): see bf_fkmig.
struct FkJob {
    const int16_t *rf;    // [na][ne][ns]
    float2 *D;            // [na][nt/2 + 1][nk] per-angle spectra (time, then lateral transform)
    float2 *spec;         // [nt/2][nk] migrated spectrum, rows Kz bin q = 1 .. nt/2
    float *img;           // [ne][ns] magnitude image
    unsigned *maxbits;    // image maximum (float bits) for the log stage, or null
    const float *beta;    // [na][ne] pi x_i sin(theta_a) / (nt dz): lateral phase per time bin
    // the mapping, decided on the host in double precision: per (angle, Kz bin
    // q = 1 .. nt/2, Kx bin) the temporal bin i0 below the mapped position (-1:
    // the point takes nothing from this angle) and (interpolation weight of
    // bin i0 + 1, spectral weight)
    const int *map_i0;    // [na][nt/2][nk]
    const float2 *map_aw; // [na][nt/2][nk]
    const float2 *tw_t;   // [nt] exp(-2 pi i k / nt)
    const float2 *tw_k;   // [nk] exp(-2 pi i k / nk)
    int na, ne, ns, nt, lgt, nk, lgk;
};

// One (frame, mode) image through the analytic-signal envelope along z.
struct EnvJob {
    const float *y;       // [nx][nz] beamformed image
    float *env;           // [nx][nz] envelope output
    unsigned *maxbits;    // frame maximum of env (float bits), reset to 0 before
    int nx, nz;
    int fft_m;            // transform size (nz itself when nz is a power of two)
    int bluestein;        // 1 when nz is not a power of two
    int band;             // 1: keep only bins [kb_lo, kb_hi] (DMAS second-harmonic band-pass)
    int kb_lo, kb_hi;
    int cols_per_block;   // image columns transformed together by one CTA
    int vec4;             // 1: y and env are 16-byte aligned and nz a multiple of 4 (vector access)
    const float2 *tw;     // [fft_m] exp(-2 pi i k / fft_m)
    const float2 *chirp;  // [nz] exp(i pi n^2 / nz)              (Bluestein only)
    const float2 *bhat;   // [fft_m] DFT of the chirp convolution kernel (Bluestein only)
};

// One (frame, mode) envelope image to decibels against its frame maximum.
struct LogJob {
    const float *env;
    float *out;
    const unsigned *maxbits;
    int n;                // pixels
    int vec4;             // 1: env and out 16-byte aligned and n a multiple of 4
};

// Launch configuration of kernel `k` on the current device, cached per
// (device, kernel) behind a mutex so that host threads and devices do not race:
// raises its dynamic shared-memory limit to at least `smem` when that is above
// the 48 KB default (with the largest shared-memory carveout when
// `max_carveout`), and returns the device's SM count in *sms and, when occ is
// not null, the resident CTAs per SM at `threads` threads and `smem` bytes.
cudaError_t kernel_setup(const void *k, size_t smem, int threads, bool max_carveout, int *sms,
                         int *occ);

// Kernel launchers (bf_kernels.cu).  All enqueue on `stream` and return the
// launch status.  `variant` holds the BF_DMAS / BF_CF bits the launch computes
// (all its jobs must share them, the precision and the rows per thread);
// BF_PDAS adds the p-th-root combiner.
cudaError_t launch_plan(const PlanJob &job, int *err_dev, cudaStream_t stream);
// total_blocks: the jobs' rows x chunks (blk_prefix_dev: each job's first CTA).
cudaError_t launch_ingest(const IngestJob *jobs_dev, const int *blk_prefix_dev, int njobs,
                          int total_blocks, int prec, cudaStream_t stream);
// pairs: some job demodulates a frame pair (four transform buffers per CTA)
cudaError_t launch_demod(const DemodJob *jobs_dev, const int *row_prefix_dev, int njobs,
                         int total_rows, int max_ns, bool pairs, cudaStream_t stream);
size_t demod_smem_bytes(int ns, bool pairs);
// f-k migration launches (bf_kernels.cu), in order on `stream`.
cudaError_t launch_fkmig(const FkJob &job, cudaStream_t stream);
// nf: frames per job (1, 2 or 4, with 4 on two-row tiles only; the frames of
// one job share the delays; DAS / DMAS variants of the RF precisions, or the
// IQ combiners, only when nf > 1 or rows == 2).
cudaError_t launch_beamform(const BfJob *jobs_dev, const int *tile_prefix_dev, int njobs,
                            int total_tiles, size_t smem_bytes, int prec, int variant, int rows,
                            int nf, int *err_dev, cudaStream_t stream);
cudaError_t launch_envelope(const EnvJob *jobs_dev, const int *blk_prefix_dev, int njobs,
                            int total_blocks, size_t smem_bytes, cudaStream_t stream);
cudaError_t launch_log(const LogJob *jobs_dev, const int *blk_prefix_dev, int njobs,
                       int total_blocks, float dynamic_range_db, cudaStream_t stream);
// Envelope of 512-row images by the warp-per-column-pair kernel (bf_envelope.cu):
// the jobs it takes (power-of-two depth of 512, no Bluestein), and its launch
// over total_pairs column pairs (pair_prefix_dev: each job's first pair).
bool envelope_warp_ok(int nz, int fft_m, int bluestein);
cudaError_t launch_envelope_warp(const EnvJob *jobs_dev, const int *pair_prefix_dev, int njobs,
                                 int total_pairs, cudaStream_t stream);
// One frame through the plain baseline kernel (FP32, global loads, one thread
// per pixel); job.y receives the beamformed modes.
cudaError_t launch_plain(const BfJob &job, const int16_t *rf, const int2 *valid, const float *dx2,
                         int nxp, int ns, cudaStream_t stream);
// Dynamic shared memory of a beamforming CTA: header, the multi-frame
// staging area (nf > 1) and the pipeline stages.
size_t beamform_smem_bytes(int wmax, int group, int prec, int nf = 1, int rows = 4);
int log_blocks(long long pixels);
int envelope_cols_per_block(int fft_m);
size_t envelope_smem_bytes(int fft_m, int bluestein);

// Bytes of one stored sample pair for a precision.
inline int pair_bytes(int prec) { return prec == kPrecIQ ? 16 : prec == kPrecF32 ? 8 : 4; }
// Largest TMA box of staged pairs (a box spans at most 256 elements of 8 bytes
// for FP32 and IQ pairs, 4 bytes for FP16 / BF16).
inline int max_box_pairs(int prec) { return prec == kPrecIQ ? 128 : 256; }
// Tensor-map elements per staged pair.
inline int pair_elems(int prec) { return prec == kPrecIQ ? 2 : 1; }

}  // namespace bfi

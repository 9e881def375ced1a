// GB300 (sm_103a) kernels of the plane-wave beamformer.
//
//   plan_kernel      once per (handle, angle set): for every pixel tile, angle
//                    and channel, the first sample pair of the window of the
//                    channel's record the tile reads (or "none")
//   ingest_kernel    int16 channel records of a batch of frames -> staged
//                    sample pairs (FP32 (mid, diff) pairs, or raw FP16 / BF16
//                    pairs), one launch for the whole batch
//   beamform_kernel  persistent CTAs walking the launch's (job, tile) list; a
//                    tile is 32 columns (one per lane) x 8 row bands (one per
//                    consumer warp, `ROWS` contiguous rows per thread).  Per
//                    angle and channel group a producer warp has the tensor
//                    memory accelerator (cp.async.bulk.tensor) copy, into a
//                    3-stage shared-memory ring tracked by mbarriers, the
//                    group's window of every channel's record plus the tile's
//                    per-(channel, column) tables; delays are formed in
//                    registers, samples interpolated linearly and combined
//                    (DAS, signed-sqrt DMAS, coherence factor, pDAS), compounded
//                    over angles (Eq. (1), Sec. II-B).  A job may carry 2 or 4
//                    frames of one plan (their pairs interleaved by frame):
//                    every delay (and for IQ-DAS / BB-DMAS, Eq. (4), the
//                    carrier phase) serves all of them, and a storer warp
//                    writes the staged tile images with bulk copies
//   envelope_kernel  per image column the analytic signal along depth via a
//                    shared-memory radix-8 Stockham FFT (Bluestein for other
//                    lengths), one-sided mask and optional [f0, 3 f0]
//                    band-pass, magnitude, and the frame maximum
//   log_kernel       20 log10(env / max) clipped to the -70 dB range of Fig. 3
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <limits.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "../../include/bf.h"
#include "bf_fft.cuh"
#include "bf_internal.h"

namespace bfi {
namespace {

constexpr float kRoundMagic = 12582912.0f;  // 1.5 * 2^23: x + magic rounds x to an integer
constexpr int kRoundBits = 0x4B400000;      // bit pattern of kRoundMagic
constexpr unsigned long long kWaitNs = 4000000000ull;  // bounded wait per CTA (4 s)

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for a barrier phase until the CTA's deadline; false (and an error bit)
// if it passed.  Every wait of the CTA shares one deadline, so a stuck copy
// costs at most kWaitNs before the CTA gives up on all remaining steps.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity,
                                          unsigned long long deadline, int *err)
{
    if (mbar_try_wait(bar, parity))
        return true;
    while (global_ns() < deadline)
        if (mbar_try_wait(bar, parity))
            return true;
    atomicOr(err, kErrTimeout);
    return false;
}

// One 2-D tensor-map box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *map, int x, int y,
                                       uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x^e for x >= 0, e > 0 as 2^(e log2 x) on the special-function unit
// (x = 0: log2 gives -inf, 2^-inf = 0).
__device__ __forceinline__ float pow_approx(float x, float e)
{
    float l, y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(l * e));
    return y;
}

// sign(v) |v|^(1/p) of one delayed sample; p = 2 takes the square root.
__device__ __forceinline__ float pdas_root(float v, float inv_p, bool square)
{
    const float av = fabsf(v);
    return copysignf(square ? sqrt_approx(av) : pow_approx(av, inv_p), v);
}

// Receive path length beyond the depth term, in samples:
//   q = sqrt(d2 + z^2) - z = d2 / (sqrt(d2 + z^2) + z),
// d2 = (kappa (x_p - x_i))^2, z = kappa z_p.  The large, pixel-only part of
// the delay (transmit leg + depth) comes from the host as an exact integer +
// remainder, so FP32 only has to carry this small term, formed without
// cancellation; its relative error (a few ulp) keeps the delay within ~1e-6
// samples (float32 emulation: 1e-6 rms, 1e-5 max over |x_p - x_i| <= z_p / 3).
// dx2 >= 1e-30 (host floor), so the square root never sees 0; dx2 + z^2 is
// formed with one rounding.
__device__ __forceinline__ float rx_excess(float dx2, float z)
{
    const float s = fmaf(z, z, dx2);
    const float r = s * rsqrt_approx(s);
    return dx2 * rcp_approx(r + z);
}

__device__ __forceinline__ int find_job(const int *__restrict__ prefix, int njobs, int bid)
{
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= bid)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------ plan --

__global__ void __launch_bounds__(128) plan_kernel(const PlanJob J, int *__restrict__ err)
{
    const int t = blockIdx.x, a = blockIdx.y;
    const int tx = t % J.tiles_x, tz = t / J.tiles_x;
    const int th = kWarps * J.rows;
    const int tz0 = tz * th, tz_last = min(tz0 + th - 1, J.nz - 1);
    for (int i = threadIdx.x; i < J.ne; i += blockDim.x) {
        int kmin = INT_MAX, kmax = INT_MIN;
        unsigned any = 0, full = (1u << kWarps) - 1;
        for (int w = 0; w < kTileCols; ++w) {
            const int ix = tx * kTileCols + w;
            if (ix >= J.nx)
                break;
            const int2 vr = J.valid[((size_t)a * J.ne + i) * J.nxp + ix];
            // row bands of the consumer warps: does some / every pixel of this column count?
            for (int b = 0; b < kWarps; ++b) {
                const int b0 = tz0 + b * J.rows, b1 = min(b0 + J.rows - 1, J.nz - 1);
                if (b0 > b1)
                    continue;  // band below the grid: nothing to store there
                if (vr.x <= b1 && vr.y >= b0)
                    any |= 1u << b;
                if (!(vr.x <= b0 && vr.y >= b1))
                    full &= ~(1u << b);
            }
            const int r0 = max(vr.x, tz0), r1 = min(vr.y, tz_last);
            if (r0 > r1)
                continue;
            const float d2 = J.dx2[(size_t)i * J.nxp + ix];
            const int kb = J.colK[a * J.nx + ix];
            const float fb = J.colF[a * J.nx + ix];
            const int k0 = kb + J.rowK[a * J.nz + r0] +
                           __float2int_rd(fb + J.rowF[a * J.nz + r0] +
                                          rx_excess(d2, J.rowZ[r0]));
            const int k1 = kb + J.rowK[a * J.nz + r1] +
                           __float2int_rd(fb + J.rowF[a * J.nz + r1] +
                                          rx_excess(d2, J.rowZ[r1]));
            kmin = min(kmin, min(k0, k1));
            kmax = max(kmax, max(k0, k1));
        }
        int w0 = kNoWindow;
        if (kmin <= kmax) {
            // pairs kmin + kPadL .. kmax + kPadL, two pairs of margin on either side
            w0 = (kmin + kPadL - 2) & ~(J.align - 1);
            if (kmax + kPadL + 2 - w0 + 1 > J.wmax)
                atomicOr(err, kErrWindow);
        }
        const size_t o = ((size_t)a * J.tiles_x * J.tiles_z + t) * J.ne + i;
        J.wtab[o] = w0;
        J.btab[o] = w0 == kNoWindow ? 0 : (int)(any | ((full & any) << 8));
    }
}

// ---------------------------------------------------------------- ingest --

// Pairs j0 .. j0 + 7 of one record row: mid point and difference of samples
// k = j - kPadL and k + 1 (zero outside the record), FP32 or scaled by 2^-15 to
// FP16 / BF16 (two 16-bit halves: sample k low, k + 1 high).
// vec: the row starts 16-byte aligned (samples j0 .. j0 + 7 in one 16-byte
// load, j0 - 2 and j0 - 1 in one 4-byte load when all lie inside the record).
template <int PREC>
__device__ __forceinline__ void row_pairs(const int16_t *__restrict__ u, int ns, int j0, bool vec,
                                          float2 *f, unsigned *h)
{
    static_assert(kPadL == 2, "the vector path loads two samples before j0");
    int s[9];
    if (vec && j0 >= kPadL && j0 + 8 <= ns) {
        const unsigned lo = __ldg(reinterpret_cast<const unsigned *>(u + j0 - kPadL));
        const int4 hi = __ldg(reinterpret_cast<const int4 *>(u + j0));
        const unsigned w[4] = {(unsigned)hi.x, (unsigned)hi.y, (unsigned)hi.z, (unsigned)hi.w};
        s[0] = (int)(int16_t)(lo & 0xffffu);
        s[1] = (int)(int16_t)(lo >> 16);
#pragma unroll
        for (int q = 0; q < 7; ++q)  // samples j0 .. j0 + 6 (little-endian halves)
            s[2 + q] = (int)(int16_t)((w[q >> 1] >> (16 * (q & 1))) & 0xffffu);
    } else {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int k = j0 - kPadL + q;
            s[q] = (k >= 0 && k < ns) ? (int)__ldg(u + k) : 0;
        }
    }
    if (PREC == kPrecF32) {
        // v = mid + (alpha - 1/2) * diff (exact for int16)
#pragma unroll
        for (int q = 0; q < 8; ++q)
            f[q] = make_float2(0.5f * (float)(s[q] + s[q + 1]), (float)(s[q + 1] - s[q]));
    } else {
        const float sc = 1.0f / 32768.0f;
        unsigned b[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            if (PREC == kPrecF16)
                b[q] = __half_as_ushort(__float2half_rn((float)s[q] * sc));
            else
                b[q] = __bfloat16_as_ushort(__float2bfloat16_rn((float)s[q] * sc));
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
            h[q] = b[q] | (b[q + 1] << 16);
    }
}

// Record rows to sample pairs.  A job's CTAs take its rows in order, `chunks`
// CTAs per row.  nf = 1 writes [row][nsp] (thread g: pairs 8 g .. 8 g + 7).
// A multi-frame job (nf = 2, 4) writes its frames interleaved per pair index:
// FP32 as frame pairs, pair j of frames 2q, 2q + 1 at [row][j][q] as
// (mid_2q, mid_2q+1, diff_2q, diff_2q+1) (thread g: frame pair g % (nf / 2),
// pairs 8 (g / (nf / 2)) .. + 7); FP16 / BF16 as one 4-byte pair per frame at
// [row][j][f] (thread g: frame g % nf, pairs 8 (g / nf) .. + 7).
template <int PREC>
__global__ void __launch_bounds__(256) ingest_kernel(const IngestJob *__restrict__ jobs,
                                                     const int *__restrict__ blk_prefix, int njobs)
{
    const int jb = find_job(blk_prefix, njobs, blockIdx.x);
    const IngestJob J = jobs[jb];
    const int local = blockIdx.x - __ldg(blk_prefix + jb);
    const int row = local / J.chunks, chunk = local - row * J.chunks;
    if (row == 0 && chunk == 0 && threadIdx.x < 4) {  // before any later kernel takes a maximum
        if (J.maxbits)
            J.maxbits[threadIdx.x] = 0u;
        for (int f = 1; f < J.nf; ++f) {
            unsigned *m = jobs[jb].maxbits_more[f - 1];
            if (m)
                m[threadIdx.x] = 0u;
        }
    }
    const int nf = J.nf;  // 1, 2 or 4
    const int g = chunk * blockDim.x + threadIdx.x;
    // the other frames' pointers come from the job in global memory: a runtime
    // index into the local copy J would put it on the stack
    auto record = [&](int f) { return f == 0 ? J.rf : jobs[jb].rf_more[f - 1]; };
    auto vec_ok = [&](const int16_t *rf) {
        return (J.ns & 7) == 0 && (reinterpret_cast<unsigned long long>(rf) & 15) == 0;
    };
    float2 fp[8];
    unsigned hp[8];
    if (PREC == kPrecF32 && nf > 1) {
        const int npair = nf / 2;
        const int q = g % npair, j0 = (g / npair) * 8;
        if (j0 >= J.nsp)
            return;
        float2 fq[8];
        const int16_t *ra = record(2 * q), *rb = record(2 * q + 1);
        row_pairs<PREC>(ra + (size_t)row * J.ns, J.ns, j0, vec_ok(ra), fp, hp);
        row_pairs<PREC>(rb + (size_t)row * J.ns, J.ns, j0, vec_ok(rb), fq, hp);
        float4 *o = reinterpret_cast<float4 *>(J.pairs) + ((size_t)row * J.nsp + j0) * npair + q;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            o[(size_t)k * npair] = make_float4(fp[k].x, fq[k].x, fp[k].y, fq[k].y);
        return;
    }
    const int f = g & (nf - 1), j0 = (g / nf) * 8;
    if (j0 >= J.nsp)
        return;
    const int16_t *__restrict__ rf = record(f);
    const int16_t *__restrict__ u = rf + (size_t)row * J.ns;
    row_pairs<PREC>(u, J.ns, j0, vec_ok(rf), fp, hp);
    const size_t at = ((size_t)row * J.nsp + j0) * nf + f;  // slot of pair j0
    if (PREC == kPrecF32) {
        float2 *o = reinterpret_cast<float2 *>(J.pairs) + at;
#pragma unroll
        for (int k = 0; k < 8; k += 2)  // nf == 1: 16-byte stores of two pairs
            reinterpret_cast<float4 *>(o)[k / 2] =
                make_float4(fp[k].x, fp[k].y, fp[k + 1].x, fp[k + 1].y);
    } else {
        unsigned *o = reinterpret_cast<unsigned *>(J.pairs) + at;
        if (nf == 1) {
            reinterpret_cast<uint4 *>(o)[0] = make_uint4(hp[0], hp[1], hp[2], hp[3]);
            reinterpret_cast<uint4 *>(o)[1] = make_uint4(hp[4], hp[5], hp[6], hp[7]);
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                o[(size_t)k * nf] = hp[k];
        }
    }
}

// ------------------------------------------------------------- beamform --

// Shared memory of one beamforming CTA: the header (mbarrier ring, window
// starts, channel lists, delay tables), the image staging area of multi-frame
// jobs, then stages_for_rows(ROWS) stages, each holding the tile's
// per-(channel, column) tables of one channel group and the channels' record
// windows.

// --------------------------------------------------------- demodulation --

// Analytic signal of one int16 record u of length m = 2^lgm, scaled by m:
// length-m transform of u in X (Y the work buffer), one-sided spectrum
// (H = 1 at 0 and m/2, 2 between, 0 above), inverse transform.  Returns the
// buffer (X or Y) holding it.
__device__ float2 *analytic_scaled(const int16_t *__restrict__ u, int m, int lgm, float2 *X,
                                   float2 *Y, const float2 *tw)
{
    for (int k = threadIdx.x; k < m; k += blockDim.x)
        X[k] = make_float2((float)__ldg(u + k), 0.f);
    __syncthreads();
    float2 *S = fft_r8(X, Y, m, lgm, 1, tw, false);
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const float h = (k == 0 || 2 * k == m) ? 1.f : (2 * k < m ? 2.f : 0.f);
        S[k] = make_float2(S[k].x * h, S[k].y * h);
    }
    __syncthreads();
    return fft_r8(S, S == X ? Y : X, m, lgm, 1, tw, true);
}

// Interpolation pair j of an analytic signal A (scaled by m): mid = (a + b) / 2,
// diff = b - a with a = A[k], b = A[k + 1] exp(-j 2 pi f0 / fs), k = j - kPadL
// (zero outside the record).
__device__ __forceinline__ float4 demod_pair(const float2 *A, int j, int m, float2 rot, float inv)
{
    const int k = j - kPadL;
    const float2 a0 = (k >= 0 && k < m) ? A[k] : make_float2(0.f, 0.f);
    const float2 a1 = (k + 1 >= 0 && k + 1 < m) ? A[k + 1] : make_float2(0.f, 0.f);
    const float2 b = cmul(a1, rot);
    return make_float4(0.5f * (a0.x + b.x) * inv, 0.5f * (a0.y + b.y) * inv, (b.x - a0.x) * inv,
                       (b.y - a0.y) * inv);
}

// One channel record per CTA (of one frame, or of the two frames of a frame
// pair of a multi-frame job): analytic signal, then the complex interpolation
// pairs of the IQ beamformer.
__global__ void __launch_bounds__(256) demod_kernel(const DemodJob *__restrict__ jobs,
                                                    const int *__restrict__ row_prefix, int njobs)
{
    extern __shared__ __align__(16) float2 dbuf[];
    const int jb = find_job(row_prefix, njobs, blockIdx.x);
    const DemodJob J = jobs[jb];
    const int row = blockIdx.x - __ldg(row_prefix + jb);
    if (row == 0 && threadIdx.x < 4) {  // before any later kernel takes a maximum
        if (J.maxbits)
            J.maxbits[threadIdx.x] = 0u;
        if (J.maxbits2)
            J.maxbits2[threadIdx.x] = 0u;
    }
    const int m = J.ns, lgm = J.lgn;
    float2 *X = dbuf, *Y = dbuf + m, *tw = dbuf + 2 * (size_t)m, *Z = dbuf + 3 * (size_t)m;
    for (int k = threadIdx.x; k < m; k += blockDim.x)
        tw[k] = __ldg(J.tw + k);
    const float inv = 1.f / (float)m;
    if (J.nf == 1) {
        const float2 *A = analytic_scaled(J.rf + (size_t)row * m, m, lgm, X, Y, tw);
        float4 *__restrict__ out = J.pairs + (size_t)row * J.nsp;
        for (int j = threadIdx.x; j < J.nsp; j += blockDim.x)
            out[j] = demod_pair(A, j, m, J.rot, inv);
        return;
    }
    // frame pair: both records in one transform, z = u_a + i u_b.  Their
    // spectra follow from Z's Hermitian parts, U_a[k] = (Z[k] + conj Z[-k]) / 2
    // and U_b[k] = (Z[k] - conj Z[-k]) / 2i; each gets the one-sided mask and
    // its own inverse transform (three transforms for two records).
    {
        const int16_t *__restrict__ ua = J.rf + (size_t)row * m;
        const int16_t *__restrict__ ub = J.rf2 + (size_t)row * m;
        for (int k = threadIdx.x; k < m; k += blockDim.x)
            X[k] = make_float2((float)__ldg(ua + k), (float)__ldg(ub + k));
    }
    __syncthreads();
    float2 *S = fft_r8(X, Y, m, lgm, 1, tw, false);
    float2 *P = S == X ? Y : X;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const float h = (k == 0 || 2 * k == m) ? 1.f : (2 * k < m ? 2.f : 0.f);
        const float2 zk = S[k], zm = S[(m - k) & (m - 1)];
        const float hh = 0.5f * h;
        P[k] = make_float2((zk.x + zm.x) * hh, (zk.y - zm.y) * hh);
        Z[k] = make_float2((zk.y + zm.y) * hh, (zm.x - zk.x) * hh);
    }
    __syncthreads();
    const float2 *A = fft_r8(P, S, m, lgm, 1, tw, true);  // m * analytic signal of u_a
    const float2 *B = fft_r8(Z, A == P ? S : P, m, lgm, 1, tw, true);  // and of u_b
    // per pair index the pair's eight floats in two 16-byte stores
    float4 *__restrict__ out = J.pairs + (size_t)row * J.nsp * J.nf + J.fi / 2 * 2;
    for (int j = threadIdx.x; j < J.nsp; j += blockDim.x) {
        const float4 a = demod_pair(A, j, m, J.rot, inv), b = demod_pair(B, j, m, J.rot, inv);
        float4 *o = out + (size_t)j * J.nf;
        o[0] = make_float4(a.x, b.x, a.y, b.y);
        o[1] = make_float4(a.z, b.z, a.w, b.w);
    }
}

struct SmemHeader {
    uint64_t full[kMaxStages];   // producer -> consumers: the stage's copies have landed
    uint64_t empty[kMaxStages];  // consumers -> producer: every consumer warp is done with it
    int2 wf[kMaxStages][kMaxGroup];  // (window start, band flags) per staged channel
    // per row band (consumer warp): the stage's channels that every pixel of the
    // band counts, then those that only some pixels count
    uint8_t list[kMaxStages][kWarps][kMaxGroup];
    uint8_t nfull[kMaxStages][kWarps], ntot[kMaxStages][kWarps];
    // per stage that starts an angle: the tile's delay tables (integer part and
    // remainder of the column terms [32], then of the row terms [up to 64];
    // kappa z of the rows)
    int tK[kMaxStages][kTileCols + 64];
    float tF[kMaxStages][kTileCols + 64];
    float tZ[kMaxStages][64];
    // multi-frame jobs: consumers -> storer (the tile's images are staged),
    // storer -> consumers (the staging area is free again)
    uint64_t epi_full, epi_empty;
};
constexpr int kHeaderBytes = 4608;
static_assert(sizeof(SmemHeader) <= kHeaderBytes, "header");

// Sample pairs read from shared memory through 32-bit shared-window addresses.
template <int PREC>
struct PairIO;

template <>
struct PairIO<kPrecF32> {
    static constexpr int kBytes = 8;
    __device__ static __forceinline__ float interp(uint32_t addr, float al)
    {
        float mid, diff;
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(mid), "=f"(diff) : "r"(addr));
        return fmaf(al, diff, mid);
    }
};

template <>
struct PairIO<kPrecF16> {
    static constexpr int kBytes = 4;
    __device__ static __forceinline__ float interp(uint32_t addr, float al)
    {
        unsigned w;
        asm volatile("ld.shared.b32 %0, [%1];" : "=r"(w) : "r"(addr));
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w));
        return fmaf(al + 0.5f, f.y - f.x, f.x);
    }
};

template <>
struct PairIO<kPrecBF16> {
    static constexpr int kBytes = 4;
    __device__ static __forceinline__ float interp(uint32_t addr, float al)
    {
        unsigned w;
        asm volatile("ld.shared.b32 %0, [%1];" : "=r"(w) : "r"(addr));
        const float lo = __uint_as_float(w << 16), hi = __uint_as_float(w & 0xffff0000u);
        return fmaf(al + 0.5f, hi - lo, lo);
    }
};

// Loads through 32-bit shared-window addresses (the consumer loop's tables).
__device__ __forceinline__ float4 lds_f32x4(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr));
    return v;
}

__device__ __forceinline__ int2 lds_int2(uint32_t addr)
{
    int2 v;
    asm volatile("ld.shared.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
    return v;
}

__device__ __forceinline__ float lds_f32(uint32_t addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void sts_f32x2(uint32_t addr, float a, float b)
{
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(a), "f"(b) : "memory");
}

// This thread's shared-memory writes, visible to the async proxy (bulk copies).
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bulk copy shared -> global (16-byte aligned addresses, size a multiple of 16),
// tracked in this thread's bulk groups.
__device__ __forceinline__ void bulk_store(void *gdst, uint32_t ssrc, unsigned bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
                 "r"(ssrc), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Every committed bulk copy of this thread has read its shared-memory source.
__device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Every committed bulk copy of this thread is complete.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Bytes of one pipeline stage: tables (int2 rows + float dx^2) and windows.
// (nf frames' windows per channel in multi-frame jobs)
__host__ __device__ __forceinline__ int stage_bytes(int group, int wmax, int pb, int nf = 1)
{
    return group * (kTileCols * 12 + nf * wmax * pb);
}

// Multi-frame jobs stage their images in shared memory for the storer warp:
// per image plane (frame, combiner) and tile column the tile's rows, then
// kEpiPad floats (16-byte aligned runs for the bulk copies, at most 4-way bank
// conflicts for the consumers' writes).  It sits between the header and the
// pipeline stages.
constexpr int kEpiPad = 4;
__host__ __device__ constexpr int epi_col_floats(int rows) { return kWarps * rows + kEpiPad; }
__host__ __device__ constexpr int epi_bytes(int nf, int rows)
{
    return nf > 1 ? nf * 2 * kTileCols * epi_col_floats(rows) * (int)sizeof(float) : 0;
}
// Threads of a beamforming CTA: the consumer warps, the producer warp and, in
// multi-frame jobs, the storer warp.
template <int NF>
constexpr int beamform_threads()
{
    return kThreads + 32 + (NF > 1 ? 32 : 0);
}

// ---- packed FP32 pairs (Blackwell f32x2 arithmetic): two rows' delays at once
typedef unsigned long long f32x2_t;

__device__ __forceinline__ f32x2_t pk2(float lo, float hi)
{
    f32x2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void upk2(f32x2_t v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ f32x2_t fma2(f32x2_t a, f32x2_t b, f32x2_t c)
{
    f32x2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2_t add2(f32x2_t a, f32x2_t b)
{
    f32x2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2_t sub2(f32x2_t a, f32x2_t b)
{
    f32x2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2_t mul2(f32x2_t a, f32x2_t b)
{
    f32x2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Rounded delays of rows j and j + 1 for one channel (d2 packed twice): the
// rx_excess arithmetic of both rows in paired instructions, each half with
// exactly the scalar version's operations and roundings, plus the pixels'
// remainders.  m holds the delay plus the rounding constant (integer in its
// low bits), al the offset in [-1/2, 1/2].
__device__ __forceinline__ void delay2(f32x2_t D2, f32x2_t Zp, f32x2_t Fp, float &ma, float &mb,
                                       float &ala, float &alb)
{
    const f32x2_t s = fma2(Zp, Zp, D2);
    float sa, sb;
    upk2(s, sa, sb);
    const f32x2_t r = mul2(s, pk2(rsqrt_approx(sa), rsqrt_approx(sb)));
    float da, db;
    upk2(add2(r, Zp), da, db);
    const f32x2_t x = fma2(D2, pk2(rcp_approx(da), rcp_approx(db)), Fp);
    const f32x2_t MG = pk2(kRoundMagic, kRoundMagic);
    const f32x2_t m = add2(x, MG);
    upk2(m, ma, mb);
    upk2(sub2(x, sub2(m, MG)), ala, alb);
}

// Per-angle constants of a thread's rows, packed in row pairs for delay2: the
// depth term z and the remainder f (minus 1/2).
template <int ROWS>
struct RowPack {
    f32x2_t Z[ROWS / 2], F[ROWS / 2];
    __device__ __forceinline__ void set(const float *z, const float *f)
    {
#pragma unroll
        for (int j = 0; j < ROWS; j += 2) {
            Z[j / 2] = pk2(z[j], z[j + 1]);
            F[j / 2] = pk2(f[j], f[j + 1]);
        }
    }
};

// Accumulate one channel into the ROWS pixels of this thread.  CHECK: test
// every pixel's row against the channel's counted rows (otherwise the whole
// row band of the warp counts it).
template <int PREC, bool DMAS, bool CF, bool PDAS, int ROWS, bool CHECK>
__device__ __forceinline__ void accumulate(uint32_t win, int wmax, int w0, float d2, int2 vr,
                                           int r_first, const RowPack<ROWS> &P, const int *Kc,
                                           float *S1, float *T1, float *T2, float *Su2, float *P1,
                                           float inv_p, bool square)
{
    constexpr int PB = PairIO<PREC>::kBytes;
    static_assert(ROWS % 2 == 0, "rows are processed in pairs");
    const unsigned span = (unsigned)(vr.y - vr.x);
    const f32x2_t D2 = pk2(d2, d2);
#pragma unroll
    for (int j = 0; j < ROWS; j += 2) {
        float m[2], al[2];  // al in [-1/2, 1/2]
        delay2(D2, P.Z[j / 2], P.F[j / 2], m[0], m[1], al[0], al[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int jj = j + h;
            const unsigned idx =
                min((unsigned)(__float_as_int(m[h]) + Kc[jj] - w0), (unsigned)(wmax - 1));
            const float v = PairIO<PREC>::interp(win + idx * PB, al[h]);
            if (!CHECK || (unsigned)(r_first + jj - vr.x) <= span) {
                S1[jj] += v;
                if (DMAS) {
                    const float av = fabsf(v);
                    T1[jj] += copysignf(sqrt_approx(av), v);
                    T2[jj] += av;
                }
                if (CF)
                    Su2[jj] = fmaf(v, v, Su2[jj]);
                if (PDAS)
                    P1[jj] += pdas_root(v, inv_p, square);
            }
        }
    }
}

// The NF frames' samples at one window index of a multi-frame job, as NF / 2
// frame pairs (v[q] = frames 2q, 2q + 1).  FP32 records are staged as
// (mid_2q, mid_2q+1, diff_2q, diff_2q+1) per window index and frame pair, so
// one 16-byte load and one paired FMA interpolate two frames; FP16 / BF16
// records keep one 4-byte pair per frame ([pair][frame]).
template <int PREC, int NF>
__device__ __forceinline__ void interp_frames(uint32_t a, float al, f32x2_t *v)
{
    if constexpr (PREC == kPrecF32) {
        const f32x2_t AL = pk2(al, al);
#pragma unroll
        for (int q = 0; q < NF / 2; ++q) {
            f32x2_t mid, diff;
            asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];"
                         : "=l"(mid), "=l"(diff)
                         : "r"(a + (uint32_t)q * 16u));
            v[q] = fma2(AL, diff, mid);
        }
    } else {
        unsigned w[NF];
        if constexpr (NF == 4) {
            asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
                         : "r"(a));
        } else {
            asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(w[0]), "=r"(w[1]) : "r"(a));
        }
        const float t = al + 0.5f;
        float x[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            float lo, hi;
            if constexpr (PREC == kPrecF16) {
                const float2 h = __half22float2(*reinterpret_cast<const __half2 *>(&w[f]));
                lo = h.x;
                hi = h.y;
            } else {
                lo = __uint_as_float(w[f] << 16);
                hi = __uint_as_float(w[f] & 0xffff0000u);
            }
            x[f] = fmaf(t, hi - lo, lo);
        }
#pragma unroll
        for (int q = 0; q < NF / 2; ++q)
            v[q] = pk2(x[2 * q], x[2 * q + 1]);
    }
}

// One channel into the ROWS pixels of this thread for NF frames of one plan:
// the delay of each pixel is formed once and read from every frame's pairs
// (interleaved by frame in the window); the sums of two frames move in paired
// FP32 instructions.  DMAS sums s = sign(v) sqrt|v| and s^2 (= |v| up to the
// square root's rounding, so that the pairwise products the identity
// ((sum s)^2 - sum s^2) / 2 stands for are those of the computed s).
template <int PREC, bool DMAS, int ROWS, int NF, bool CHECK>
__device__ __forceinline__ void accumulate_fn(uint32_t win, int wmax, int w0, float d2, int2 vr,
                                              int r_first, const RowPack<ROWS> &P, const int *Kc,
                                              f32x2_t (&S1)[NF / 2][ROWS],
                                              f32x2_t (&T1)[NF / 2][ROWS],
                                              f32x2_t (&T2)[NF / 2][ROWS])
{
    constexpr int PB = PairIO<PREC>::kBytes;
    const unsigned span = (unsigned)(vr.y - vr.x);
    const f32x2_t D2 = pk2(d2, d2);
#pragma unroll
    for (int j = 0; j < ROWS; j += 2) {
        float m[2], al[2];
        delay2(D2, P.Z[j / 2], P.F[j / 2], m[0], m[1], al[0], al[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int jj = j + h;
            const unsigned idx =
                min((unsigned)(__float_as_int(m[h]) + Kc[jj] - w0), (unsigned)(wmax - 1));
            f32x2_t v[NF / 2];
            interp_frames<PREC, NF>(win + idx * (NF * PB), al[h], v);
            if (!CHECK || (unsigned)(r_first + jj - vr.x) <= span) {
#pragma unroll
                for (int q = 0; q < NF / 2; ++q) {
                    S1[q][jj] = add2(S1[q][jj], v[q]);
                    if (DMAS) {
                        float a, b;
                        upk2(v[q], a, b);
                        const f32x2_t sr = pk2(copysignf(sqrt_approx(fabsf(a)), a),
                                               copysignf(sqrt_approx(fabsf(b)), b));
                        T1[q][jj] = add2(T1[q][jj], sr);
                        T2[q][jj] = fma2(sr, sr, T2[q][jj]);
                    }
                }
            }
        }
    }
}

// Two channels that every pixel of the band counts, interleaved: twice the
// independent dependency chains per thread (square roots, shared loads) for
// the scheduler to overlap.
template <int PREC, bool DMAS, bool CF, bool PDAS, int ROWS>
__device__ __forceinline__ void accumulate2(uint32_t win0, int w00, float d20, uint32_t win1,
                                            int w01, float d21, int wmax, const RowPack<ROWS> &P,
                                            const int *Kc, float *S1, float *T1, float *T2,
                                            float *Su2, float *P1, float inv_p, bool square)
{
    constexpr int PB = PairIO<PREC>::kBytes;
    const f32x2_t D20 = pk2(d20, d20), D21 = pk2(d21, d21);
#pragma unroll
    for (int j = 0; j < ROWS; j += 2) {
        float m0[2], al0[2], m1[2], al1[2];
        delay2(D20, P.Z[j / 2], P.F[j / 2], m0[0], m0[1], al0[0], al0[1]);
        delay2(D21, P.Z[j / 2], P.F[j / 2], m1[0], m1[1], al1[0], al1[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int jj = j + h;
            const unsigned i0 =
                min((unsigned)(__float_as_int(m0[h]) + Kc[jj] - w00), (unsigned)(wmax - 1));
            const unsigned i1 =
                min((unsigned)(__float_as_int(m1[h]) + Kc[jj] - w01), (unsigned)(wmax - 1));
            const float v0 = PairIO<PREC>::interp(win0 + i0 * PB, al0[h]);
            const float v1 = PairIO<PREC>::interp(win1 + i1 * PB, al1[h]);
            S1[jj] += v0 + v1;
            if (DMAS) {
                const float a0 = fabsf(v0), a1 = fabsf(v1);
                T1[jj] += copysignf(sqrt_approx(a0), v0) + copysignf(sqrt_approx(a1), v1);
                T2[jj] += a0 + a1;
            }
            if (CF)
                Su2[jj] = fmaf(v0, v0, fmaf(v1, v1, Su2[jj]));
            if (PDAS)
                P1[jj] += pdas_root(v0, inv_p, square) + pdas_root(v1, inv_p, square);
        }
    }
}

// One channel of IQ beamforming into the ROWS pixels of this thread.  The
// staged pair holds mid = (A + B) / 2, diff = B - A of the analytic samples
// A = a[k], B = a[k + 1] exp(-j 2 pi r) (r = f0 / fs), so that
//   s = exp(j 2 pi r alpha) (mid + (alpha - 1/2) diff)
// is the baseband sample interpolated at n = k + alpha with its carrier
// exp(j 2 pi r n) restored.  IQ-DAS sums s; BB-DMAS (BB) sums
// s / sqrt|s| = sqrt|s| exp(j arg s) per angle.
template <bool BB, int ROWS, bool CHECK>
__device__ __forceinline__ void accumulate_iq(uint32_t win, int wmax, int w0, float d2, int2 vr,
                                              int r_first, const RowPack<ROWS> &P, const int *Kc,
                                              float c1, float c2, float *Yr, float *Yi, float *Tr,
                                              float *Ti)
{
    const unsigned span = (unsigned)(vr.y - vr.x);
    const f32x2_t D2 = pk2(d2, d2);
#pragma unroll
    for (int j = 0; j < ROWS; j += 2) {
        float mm[2], aa[2];
        delay2(D2, P.Z[j / 2], P.F[j / 2], mm[0], mm[1], aa[0], aa[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int jj = j + h;
            const float al = aa[h];  // alpha - 1/2
            const unsigned idx =
                min((unsigned)(__float_as_int(mm[h]) + Kc[jj] - w0), (unsigned)(wmax - 1));
            const float4 p = lds_f32x4(win + idx * 16u);
            const float br = fmaf(al, p.z, p.x), bi = fmaf(al, p.w, p.y);
            float sn, cs;
            __sincosf(fmaf(al, c1, c2), &sn, &cs);
            const float sr = fmaf(br, cs, -bi * sn), si = fmaf(br, sn, bi * cs);
            if (!CHECK || (unsigned)(r_first + jj - vr.x) <= span) {
                Yr[jj] += sr;
                Yi[jj] += si;
                if (BB) {
                    // |s|^(-1/2); the floor keeps s = 0 at 0 instead of 0 * inf
                    const float w = rsqrt_approx(sqrt_approx(fmaf(sr, sr, fmaf(si, si, 1e-30f))));
                    Tr[jj] = fmaf(sr, w, Tr[jj]);
                    Ti[jj] = fmaf(si, w, Ti[jj]);
                }
            }
        }
    }
}

// One channel of IQ beamforming into the ROWS pixels of this thread for NF
// frames of one plan: the delay and the carrier phase of each pixel are formed
// once and serve every frame.  The frames' pairs are staged by frame pair
// (mid.re, mid.im, diff.re, diff.im of frames 2q and 2q + 1, eight floats),
// so two frames move through each paired FP32 instruction; per frame the
// operations and roundings are those of accumulate_iq.
template <bool BB, int ROWS, int NF, bool CHECK>
__device__ __forceinline__ void accumulate_iq_fn(uint32_t win, int wmax, int w0, float d2, int2 vr,
                                                 int r_first, const RowPack<ROWS> &P,
                                                 const int *Kc, float c1, float c2,
                                                 f32x2_t (&Yr)[NF / 2][ROWS],
                                                 f32x2_t (&Yi)[NF / 2][ROWS],
                                                 f32x2_t (&Tr)[NF / 2][ROWS],
                                                 f32x2_t (&Ti)[NF / 2][ROWS])
{
    const unsigned span = (unsigned)(vr.y - vr.x);
    const f32x2_t D2 = pk2(d2, d2);
#pragma unroll
    for (int j = 0; j < ROWS; j += 2) {
        float mm[2], aa[2];
        delay2(D2, P.Z[j / 2], P.F[j / 2], mm[0], mm[1], aa[0], aa[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int jj = j + h;
            const float al = aa[h];  // alpha - 1/2
            const unsigned idx =
                min((unsigned)(__float_as_int(mm[h]) + Kc[jj] - w0), (unsigned)(wmax - 1));
            float sn, cs;
            __sincosf(fmaf(al, c1, c2), &sn, &cs);
            const f32x2_t AL = pk2(al, al), CS = pk2(cs, cs), SN = pk2(sn, sn),
                          NSN = pk2(-sn, -sn);
            const uint32_t a = win + idx * (uint32_t)(NF * 16);
#pragma unroll
            for (int q = 0; q < NF / 2; ++q) {
                f32x2_t mre, mim, dre, dim;
                asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];"
                             : "=l"(mre), "=l"(mim)
                             : "r"(a + (uint32_t)q * 32u));
                asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];"
                             : "=l"(dre), "=l"(dim)
                             : "r"(a + (uint32_t)q * 32u + 16u));
                const f32x2_t br = fma2(AL, dre, mre), bi = fma2(AL, dim, mim);
                const f32x2_t sr = fma2(br, CS, mul2(bi, NSN)), si = fma2(br, SN, mul2(bi, CS));
                if (!CHECK || (unsigned)(r_first + jj - vr.x) <= span) {
                    Yr[q][jj] = add2(Yr[q][jj], sr);
                    Yi[q][jj] = add2(Yi[q][jj], si);
                    if (BB) {
                        float qa, qb;
                        upk2(fma2(sr, sr, fma2(si, si, pk2(1e-30f, 1e-30f))), qa, qb);
                        const f32x2_t w = pk2(rsqrt_approx(sqrt_approx(qa)),
                                              rsqrt_approx(sqrt_approx(qb)));
                        Tr[q][jj] = fma2(sr, w, Tr[q][jj]);
                        Ti[q][jj] = fma2(si, w, Ti[q][jj]);
                    }
                }
            }
        }
    }
}

// Resident CTAs per SM the register budget is sized for: three 16- or 32-row
// tiles, one 64-row tile (measured: capping 64-row tiles at two CTAs per SM
// costs more in spills and lost overlap than the extra warps win).
// Multi-frame jobs hold NF times the accumulators and NF windows per channel
// and stage: two CTAs per SM when NF * ROWS = 8 (two frames of 4 rows, four
// frames of 2 rows), and for every multi-frame IQ job (six complex or paired
// sums per pixel and frame).
template <int PREC, bool DMAS, bool CF, bool PDAS, int ROWS, int NF>
constexpr int beamform_min_blocks()
{
    if (PREC == kPrecIQ && NF > 1)  // complex sums: two CTAs per SM for every multi-frame job
        return 2;
    return ROWS == 8 ? 1 : (NF * ROWS >= 8 ? 2 : 3);
}

template <int PREC, bool DMAS, bool CF, bool PDAS, int ROWS, int NF>
__global__ void __launch_bounds__(beamform_threads<NF>(),
                                  (beamform_min_blocks<PREC, DMAS, CF, PDAS, ROWS, NF>()))
    beamform_kernel(const BfJob *__restrict__ jobs, const int *__restrict__ tile_prefix, int njobs,
                    int total_tiles, int stage_stride, int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    SmemHeader &sh = *reinterpret_cast<SmemHeader *>(smem);
    constexpr bool IQ = PREC == kPrecIQ;
    constexpr int PB = IQ ? 16 : PairIO<IQ ? kPrecF32 : PREC>::kBytes;
    constexpr int XS = IQ ? 2 : 1;  // tensor-map elements per staged pair
    constexpr int TR = kWarps * ROWS;  // tile rows
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Persistent CTAs: tiles blockIdx.x, blockIdx.x + gridDim.x, ... of the
    // launch's flat (frame, tile) list.  The stage ring runs on across tiles
    // (ring position r), so the copies of a CTA's next tile are in flight while
    // it finishes the current one.  Every stage has the launch's largest
    // stage size; inside a stage the layout is the job's: int2 rows [G][32],
    // float dx^2 [G][32], windows [G][wmax].
    constexpr int EPI = epi_bytes(NF, ROWS);
    constexpr int kStages = stages_for_rows(ROWS);
    constexpr int CFL = epi_col_floats(ROWS);
    auto stage_base = [&](int st) {
        return smem + kHeaderBytes + EPI + (size_t)st * stage_stride;
    };
    // multi-frame jobs whose images take the bulk-copy epilogue: 16-byte aligned
    // images and columns (nz a multiple of 4), uniform over the job
    auto staged_job = [&](const BfJob *J) {
        if (NF == 1)
            return false;
        unsigned long long a = reinterpret_cast<unsigned long long>(J->y);
#pragma unroll
        for (int f = 1; f < NF; ++f)
            a |= reinterpret_cast<unsigned long long>(J->y_more[f - 1]);
        return (J->nz & 3) == 0 && (a & 15) == 0;
    };

    if (threadIdx.x == 0) {
        for (int st = 0; st < kStages; ++st) {
            mbar_init(&sh.full[st], 1);
            mbar_init(&sh.empty[st], kWarps);
        }
        mbar_init(&sh.epi_full, kWarps);
        mbar_init(&sh.epi_empty, 1);
        mbar_fence_init();
    }
    __syncthreads();

    if (NF > 1 && warp == kWarps + 1) {
        // ================= storer warp (multi-frame jobs): the consumers' staged
        // images out to global memory, per column and image one bulk copy of
        // the tile's rows (lane = column)
        const uint32_t eb = smem_u32(smem + kHeaderBytes) + (uint32_t)(lane * CFL) * 4u;
        unsigned u = 0;
        for (int tg = blockIdx.x; tg < total_tiles; tg += gridDim.x) {
            const int jb = find_job(tile_prefix, njobs, tg);
            const BfJob *J = jobs + jb;
            if (!staged_job(J))
                continue;
            const int tile = tg - __ldg(tile_prefix + jb);
            const int nx = J->nx, nz = J->nz, modes = J->modes;
            const int tx = tile % J->tiles_x, tz = tile / J->tiles_x;
            const unsigned long long deadline = global_ns() + kWaitNs;
            if (!__all_sync(0xffffffffu, mbar_wait(&sh.epi_full, u & 1u, deadline, err)))
                break;
            const int ix = tx * kTileCols + lane, r0 = tz * TR;
            const unsigned bytes = (unsigned)min(TR, nz - r0) * 4u;
            const size_t plane = (size_t)nx * nz;
            if (ix < nx) {
                int p = 0;
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    float *yf = f == 0 ? J->y : J->y_more[f - 1];
                    float *col = yf + (size_t)ix * nz + r0;
                    int slot = 0;
                    if (modes & BF_DAS)
                        bulk_store(col + (size_t)(slot++) * plane,
                                   eb + (uint32_t)(p++ * kTileCols * CFL) * 4u, bytes);
                    if (modes & BF_DMAS)
                        bulk_store(col + (size_t)(slot++) * plane,
                                   eb + (uint32_t)(p++ * kTileCols * CFL) * 4u, bytes);
                }
            }
            bulk_commit();
            bulk_wait_read();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&sh.epi_empty);
            ++u;
        }
        bulk_wait_all();
        return;
    }

    if (warp == kWarps) {
        // ================= producer warp: TMA copies of every step's stage
        unsigned r = 0;
        for (int tg = blockIdx.x; tg < total_tiles; tg += gridDim.x) {
            const unsigned long long deadline = global_ns() + kWaitNs;
            const int jb = find_job(tile_prefix, njobs, tg);
            const BfJob *J = jobs + jb;
            const int tile = tg - __ldg(tile_prefix + jb);
            const int nx = J->nx, nz = J->nz, ne = J->ne, G = J->group, wmax = J->wmax;
            const int tiles_x = J->tiles_x, ntiles = tiles_x * J->tiles_z;
            const int tx = tile % tiles_x, tz = tile / tiles_x;
            const int ngroups = (ne + G - 1) / G, steps = J->na * ngroups;
            const int *__restrict__ wtab = J->wtab;
            const int *__restrict__ btab = J->btab;
            const CUtensorMap *rf_map = J->rf_map;
            const CUtensorMap *valid_map = J->valid_map;
            const CUtensorMap *dx2_map = J->dx2_map;
            const int box = J->box;
            const unsigned meta_bytes = (unsigned)G * kTileCols * 12;
            // window start and band flags of this lane's channel at step s
            auto window_of = [&](int s) -> int2 {
                const int a = s / ngroups, g = s - a * ngroups;
                const int c = g * G + lane;
                if (s >= steps || lane >= G || c >= ne)
                    return make_int2(kNoWindow, 0);
                const size_t o = ((size_t)a * ntiles + tile) * ne + c;
                return make_int2(__ldg(wtab + o), __ldg(btab + o));
            };
            // the tile's delay tables of angle a: this lane's column and rows lane, lane + 32
            const int cx = min(tx * kTileCols + lane, nx - 1);
            const int rz0 = min(tz * TR + lane, nz - 1), rz1 = min(tz * TR + lane + 32, nz - 1);
            struct Tabs {
                int ck, rk0, rk1;
                float cf, rf0, rf1, z0, z1;
            };
            auto tabs_of = [&](int a) -> Tabs {
                Tabs t;
                t.ck = __ldg(J->colK + a * nx + cx);
                t.cf = __ldg(J->colF + a * nx + cx);
                t.rk0 = __ldg(J->rowK + a * nz + rz0);
                t.rf0 = __ldg(J->rowF + a * nz + rz0);
                t.z0 = __ldg(J->rowZ + rz0);
                t.rk1 = t.rf1 = 0, t.z1 = 0.f;
                if (TR > 32) {
                    t.rk1 = __ldg(J->rowK + a * nz + rz1);
                    t.rf1 = __ldg(J->rowF + a * nz + rz1);
                    t.z1 = __ldg(J->rowZ + rz1);
                }
                return t;
            };
            int2 wf = window_of(0);
            Tabs tb = tabs_of(0);
            bool ok = true;
            for (int s = 0; s < steps; ++s, ++r) {
                const int st = (int)(r % kStages);
                const unsigned use = r / kStages;
                const int a = s / ngroups, g = s - a * ngroups, i0 = g * G;
                // next step's loads in flight while we wait
                const int2 wf_next = window_of(s + 1);
                const bool next_angle = s + 1 < steps && (s + 1) % ngroups == 0;
                Tabs tb_next = tb;
                if (next_angle)
                    tb_next = tabs_of(a + 1);
                if (use > 0 && !mbar_wait(&sh.empty[st], (use - 1) & 1u, deadline, err)) {
                    ok = false;
                    break;
                }
                if (g == 0) {  // delay tables of the angle, read by the consumers at this step
                    sh.tK[st][lane] = tb.ck;
                    sh.tF[st][lane] = tb.cf;
                    sh.tK[st][kTileCols + lane] = tb.rk0;
                    sh.tF[st][kTileCols + lane] = tb.rf0;
                    sh.tZ[st][lane] = tb.z0;
                    if (TR > 32) {
                        sh.tK[st][kTileCols + 32 + lane] = tb.rk1;
                        sh.tF[st][kTileCols + 32 + lane] = tb.rf1;
                        sh.tZ[st][32 + lane] = tb.z1;
                    }
                }
                const bool mine = lane < G && i0 + lane < ne;
                if (mine)
                    sh.wf[st][lane] = wf;
                {  // channel lists of every row band (lane = channel of the group)
                    const unsigned fl = (mine && wf.x != kNoWindow) ? (unsigned)wf.y : 0u;
                    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
                    for (int b = 0; b < kWarps; ++b) {
                        const bool full = (fl >> (8 + b)) & 1u;
                        const bool part = !full && ((fl >> b) & 1u);
                        const unsigned fm = __ballot_sync(0xffffffffu, full);
                        const unsigned pm = __ballot_sync(0xffffffffu, part);
                        if (full)
                            sh.list[st][b][__popc(fm & lt)] = (uint8_t)lane;
                        else if (part)
                            sh.list[st][b][__popc(fm) + __popc(pm & lt)] = (uint8_t)lane;
                        if (lane == 0) {
                            sh.nfull[st][b] = (uint8_t)__popc(fm);
                            sh.ntot[st][b] = (uint8_t)(__popc(fm) + __popc(pm));
                        }
                    }
                }
                const int w0 = wf.x;
                const unsigned bytes = (mine && w0 != kNoWindow) ? (unsigned)(NF * wmax * PB) : 0u;
                unsigned total = bytes;
#pragma unroll
                for (int off = 16; off; off >>= 1)
                    total += __shfl_xor_sync(0xffffffffu, total, off);
                unsigned char *base = stage_base(st);
                // everything written above is read by the consumers after the full barrier
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive_expect_tx(&sh.full[st], total + meta_bytes);
                    tma_2d(base, valid_map, tx * kTileCols, a * ne + i0, &sh.full[st]);
                    tma_2d(base + (size_t)G * kTileCols * 8, dx2_map, tx * kTileCols, i0,
                           &sh.full[st]);
                }
                __syncwarp();
                if (bytes) {
                    unsigned char *dst =
                        base + (size_t)G * kTileCols * 12 + (size_t)lane * NF * wmax * PB;
                    const int row = a * ne + i0 + lane;
                    // multi-frame jobs: the frames' pairs interleaved ([pair][frame]),
                    // box pairs of every frame per copy
                    for (int off = 0; off < wmax; off += box)
                        tma_2d(dst + (size_t)off * NF * PB, rf_map, (w0 + off) * NF * XS, row,
                               &sh.full[st]);
                }
                wf = wf_next;
                tb = tb_next;
            }
            if (!ok)
                return;  // the consumers' waits run out too
        }
        return;
    }

    // ================= consumer warps: one column per lane, ROWS rows per thread
    unsigned r = 0;
    unsigned epi_use = 0;  // staged tiles so far (multi-frame jobs)
    for (int tg = blockIdx.x; tg < total_tiles; tg += gridDim.x) {
        const unsigned long long deadline = global_ns() + kWaitNs;
        const int jb = find_job(tile_prefix, njobs, tg);
        const BfJob *J = jobs + jb;
        const int tile = tg - __ldg(tile_prefix + jb);
        const int nx = J->nx, nz = J->nz, na = J->na, ne = J->ne, G = J->group, wmax = J->wmax;
        const int tx = tile % J->tiles_x, tz = tile / J->tiles_x;
        const int ngroups = (ne + G - 1) / G, steps = na * ngroups;
        const int ix = tx * kTileCols + lane;
        const bool col_ok = ix < nx;
        const int ixc = min(ix, nx - 1);
        const int r_first = tz * TR + warp * ROWS;

        int Kc[ROWS];
        RowPack<ROWS> P;
        float S1[ROWS], T1[ROWS], T2[ROWS], Yd[ROWS], Su2[ROWS], P1[ROWS], Yp[ROWS];
        // NF > 1: per frame pair (frames 2q, 2q + 1 in the two halves)
        constexpr int NP = NF > 1 ? NF / 2 : 1;
        f32x2_t FS1p[NP][ROWS], FT1[NP][ROWS], FT2[NP][ROWS], FYdp[NP][ROWS];
        // IQ, NF > 1: FS1p / FYi the IQ-DAS sums, FT1 / FTi the per-angle BB-DMAS
        // sums, FYdp / FY2i BB-DMAS
        constexpr int NQ = IQ && NF > 1 ? NP : 1;
        f32x2_t FYi[NQ][ROWS], FTi[NQ][ROWS], FY2i[NQ][ROWS];
        const f32x2_t zero2 = pk2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < ROWS; ++j) {
            S1[j] = T1[j] = T2[j] = Yd[j] = Su2[j] = P1[j] = Yp[j] = 0.f;
#pragma unroll
            for (int q = 0; q < NP; ++q)
                FS1p[q][j] = FT1[q][j] = FT2[q][j] = FYdp[q][j] = zero2;
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                FYi[q][j] = FTi[q][j] = FY2i[q][j] = zero2;
            Kc[j] = 0;
        }
#pragma unroll
        for (int j = 0; j < ROWS / 2; ++j)
            P.Z[j] = P.F[j] = zero2;
        const float pdas_p = J->pdas_p, inv_p = J->pdas_inv_p;
        const bool square = pdas_p == 2.0f;  // uniform over the job
        // IQ: S1 / Y1i the IQ-DAS sum, T1 / Ti the per-angle BB-DMAS sum, Yd / Y2i BB-DMAS
        float Y1i[ROWS], Ti[ROWS], Y2i[ROWS], invM[ROWS];
        const float c1 = J->iq_c1, c2 = J->iq_c2;
#pragma unroll
        for (int j = 0; j < ROWS; ++j) {
            Y1i[j] = Ti[j] = Y2i[j] = 0.f;
            invM[j] = 0.f;
            if (IQ && DMAS) {
                const int izc = min(r_first + j, nz - 1);
                const float m = (float)__ldg(J->apcnt + (size_t)ixc * nz + izc);
                invM[j] = m > 0.f ? 1.f / m : 0.f;
            }
        }

        bool ok = true;
#pragma unroll 1
        for (int s = 0; s < steps; ++s, ++r) {
            const int a = s / ngroups, g = s - a * ngroups;
            (void)a;
            const int st = (int)(r % kStages);
            const unsigned use = r / kStages;
            ok = __all_sync(0xffffffffu, mbar_wait(&sh.full[st], use & 1u, deadline, err));
            if (!ok)
                break;
            if (g == 0) {  // this angle's delay tables, staged by the producer
                const int ck = sh.tK[st][lane];
                const float cf = sh.tF[st][lane];
                float Z[ROWS], fp[ROWS];
#pragma unroll
                for (int j = 0; j < ROWS; ++j) {
                    const int rr = warp * ROWS + j;
                    Kc[j] = ck + sh.tK[st][kTileCols + rr] + kPadL - kRoundBits;
                    fp[j] = cf + sh.tF[st][kTileCols + rr] - 0.5f;
                    Z[j] = sh.tZ[st][rr];
                    T1[j] = T2[j] = P1[j] = Ti[j] = 0.f;
#pragma unroll
                    for (int q = 0; q < NP; ++q)
                        FT1[q][j] = FT2[q][j] = zero2;
#pragma unroll
                    for (int q = 0; q < NQ; ++q)
                        FTi[q][j] = zero2;
                }
                P.set(Z, fp);
            }
            const uint32_t base = smem_u32(stage_base(st));
            const uint32_t vrb = base + (uint32_t)lane * 8;                          // int2 [G][32]
            const uint32_t d2b = base + (uint32_t)G * kTileCols * 8 + (uint32_t)lane * 4;  // float [G][32]
            const uint32_t wins = base + (uint32_t)G * kTileCols * 12;
            const uint32_t wfb = smem_u32(&sh.wf[st][0]);
            const int nf = sh.nfull[st][warp], nt = sh.ntot[st][warp];
            const uint8_t *L = sh.list[st][warp];
            auto win_of = [&](int c) { return wins + (uint32_t)(c * NF * wmax * PB); };
            auto w0_of = [&](int c) { return lds_int2(wfb + (uint32_t)c * 8).x; };
            auto d2_of = [&](int c) { return lds_f32(d2b + (uint32_t)c * (kTileCols * 4)); };
            auto vr_of = [&](int c) { return lds_int2(vrb + (uint32_t)c * (kTileCols * 8)); };
            int k = 0;
            if constexpr (IQ && NF > 1) {
                // every channel once, its delay and carrier phase serving every frame
#pragma unroll 1
                for (; k < nf; ++k) {
                    const int c = L[k];
                    accumulate_iq_fn<DMAS, ROWS, NF, false>(win_of(c), wmax, w0_of(c), d2_of(c),
                                                            make_int2(0, 0), r_first, P, Kc, c1,
                                                            c2, FS1p, FYi, FT1, FTi);
                }
#pragma unroll 1
                for (; k < nt; ++k) {
                    const int c = L[k];
                    accumulate_iq_fn<DMAS, ROWS, NF, true>(win_of(c), wmax, w0_of(c), d2_of(c),
                                                           vr_of(c), r_first, P, Kc, c1, c2, FS1p,
                                                           FYi, FT1, FTi);
                }
            } else if constexpr (IQ) {
#pragma unroll 1
                for (; k < nf; ++k) {
                    const int c = L[k];
                    accumulate_iq<DMAS, ROWS, false>(win_of(c), wmax, w0_of(c), d2_of(c),
                                                     make_int2(0, 0), r_first, P, Kc, c1, c2,
                                                     S1, Y1i, T1, Ti);
                }
#pragma unroll 1
                for (; k < nt; ++k) {
                    const int c = L[k];
                    accumulate_iq<DMAS, ROWS, true>(win_of(c), wmax, w0_of(c), d2_of(c), vr_of(c),
                                                    r_first, P, Kc, c1, c2, S1, Y1i, T1, Ti);
                }
            } else if constexpr (NF > 1) {
                // every channel once, each delay serving every frame
#pragma unroll 1
                for (; k < nf; ++k) {
                    const int c = L[k];
                    accumulate_fn<PREC, DMAS, ROWS, NF, false>(win_of(c), wmax, w0_of(c),
                                                               d2_of(c), make_int2(0, 0), r_first,
                                                               P, Kc, FS1p, FT1, FT2);
                }
#pragma unroll 1
                for (; k < nt; ++k) {
                    const int c = L[k];
                    accumulate_fn<PREC, DMAS, ROWS, NF, true>(win_of(c), wmax, w0_of(c), d2_of(c),
                                                              vr_of(c), r_first, P, Kc, FS1p,
                                                              FT1, FT2);
                }
            } else {
                // channels every pixel of the band counts, two at a time (twice the
                // independent dependency chains per thread), then the rest with a
                // per-pixel row test
#pragma unroll 1
                for (; k + 1 < nf; k += 2) {
                    const int c0 = L[k], c1 = L[k + 1];
                    accumulate2<PREC, DMAS, CF, PDAS, ROWS>(win_of(c0), w0_of(c0), d2_of(c0),
                                                            win_of(c1), w0_of(c1), d2_of(c1), wmax,
                                                            P, Kc, S1, T1, T2, Su2, P1, inv_p,
                                                            square);
                }
                if (k < nf) {
                    const int c = L[k++];
                    accumulate<PREC, DMAS, CF, PDAS, ROWS, false>(win_of(c), wmax, w0_of(c),
                                                                  d2_of(c), make_int2(0, 0),
                                                                  r_first, P, Kc, S1, T1, T2,
                                                                  Su2, P1, inv_p, square);
                }
#pragma unroll 1
                for (; k < nt; ++k) {
                    const int c = L[k];
                    accumulate<PREC, DMAS, CF, PDAS, ROWS, true>(win_of(c), wmax, w0_of(c),
                                                                 d2_of(c), vr_of(c), r_first, P,
                                                                 Kc, S1, T1, T2, Su2, P1, inv_p,
                                                                 square);
                }
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&sh.empty[st]);
            if (DMAS && !IQ && g == ngroups - 1) {
#pragma unroll
                for (int j = 0; j < ROWS; ++j) {
                    Yd[j] = fmaf(0.5f * T1[j], T1[j], fmaf(-0.5f, T2[j], Yd[j]));
#pragma unroll
                    for (int q = 0; q < NP; ++q)
                        FYdp[q][j] = fma2(mul2(pk2(0.5f, 0.5f), FT1[q][j]), FT1[q][j],
                                          fma2(pk2(-0.5f, -0.5f), FT2[q][j], FYdp[q][j]));
                }
            }
            if (DMAS && IQ && NF == 1 && g == ngroups - 1) {  // Eq. (4): ((1/M) sum s^)^2 per angle
#pragma unroll
                for (int j = 0; j < ROWS; ++j) {
                    const float ur = T1[j] * invM[j], ui = Ti[j] * invM[j];
                    Yd[j] += fmaf(ur, ur, -ui * ui);
                    Y2i[j] = fmaf(2.f * ur, ui, Y2i[j]);
                }
            }
            if (DMAS && IQ && NF > 1 && g == ngroups - 1) {  // the same per frame
#pragma unroll
                for (int q = 0; q < NQ; ++q)
#pragma unroll
                    for (int j = 0; j < ROWS; ++j) {
                        float tr[2], ti[2], yd[2], y2[2];
                        upk2(FT1[q][j], tr[0], tr[1]);
                        upk2(FTi[q][j], ti[0], ti[1]);
                        upk2(FYdp[q][j], yd[0], yd[1]);
                        upk2(FY2i[q][j], y2[0], y2[1]);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float ur = tr[h] * invM[j], ui = ti[h] * invM[j];
                            yd[h] += fmaf(ur, ur, -ui * ui);
                            y2[h] = fmaf(2.f * ur, ui, y2[h]);
                        }
                        FYdp[q][j] = pk2(yd[0], yd[1]);
                        FY2i[q][j] = pk2(y2[0], y2[1]);
                    }
            }
            if (PDAS && g == ngroups - 1) {  // Eq. (3) per angle, then the coherent sum
#pragma unroll
                for (int j = 0; j < ROWS; ++j)
                    Yp[j] += copysignf(powf(fabsf(P1[j]), pdas_p), P1[j]);
            }
        }
        if (!ok)
            return;  // warp-uniform: a bounded wait ran out (error bit set)

        if constexpr (IQ && NF == 1) {  // magnitude images (and their maxima for the log stage)
            const size_t plane = (size_t)nx * nz;
            float *__restrict__ y = J->y;
            const int modes = J->modes;
            float m0 = 0.f, m1 = 0.f;
            if (ok && col_ok) {
    #pragma unroll
                for (int j = 0; j < ROWS; ++j) {
                    const int iz = r_first + j;
                    if (iz >= nz)
                        break;
                    const size_t o = (size_t)ix * nz + iz;
                    int slot = 0;
                    if (modes & BF_DAS) {
                        const float v = sqrtf(fmaf(S1[j], S1[j], Y1i[j] * Y1i[j]));
                        y[(size_t)(slot++) * plane + o] = v;
                        m0 = fmaxf(m0, v);
                    }
                    if (modes & BF_DMAS) {
                        const float v = sqrtf(fmaf(Yd[j], Yd[j], Y2i[j] * Y2i[j]));
                        y[(size_t)(slot++) * plane + o] = v;
                        m1 = fmaxf(m1, v);
                    }
                }
            }
            if (J->maxbits) {  // uniform per job; every lane of the warp is here
                const unsigned r0 = __reduce_max_sync(0xffffffffu, __float_as_uint(m0));
                const unsigned r1 = __reduce_max_sync(0xffffffffu, __float_as_uint(m1));
                if (lane == 0) {
                    int slot = 0;
                    if (modes & BF_DAS)
                        atomicMax(J->maxbits + slot++, r0);
                    if (modes & BF_DMAS)
                        atomicMax(J->maxbits + slot, r1);
                }
            }
            continue;
        }
        const int modes = J->modes;
        const float scale = J->out_scale;
        const size_t plane = (size_t)nx * nz;
        float *__restrict__ y = J->y;
        if constexpr (NF > 1) {  // every frame of the job (DAS / DMAS only)
            // frame f's sums: the low (even f) or high (odd f) half of its pair
            float FS1[NF][ROWS], FYd[NF][ROWS];
#pragma unroll
            for (int q = 0; q < NP; ++q)
#pragma unroll
                for (int j = 0; j < ROWS; ++j) {
                    upk2(FS1p[q][j], FS1[2 * q][j], FS1[2 * q + 1][j]);
                    upk2(FYdp[q][j], FYd[2 * q][j], FYd[2 * q + 1][j]);
                }
            if constexpr (IQ) {
                // magnitude images, and each frame's maxima for the log stage
                float FYi_[NF][ROWS], FY2i_[NF][ROWS];
#pragma unroll
                for (int q = 0; q < NQ; ++q)
#pragma unroll
                    for (int j = 0; j < ROWS; ++j) {
                        upk2(FYi[q][j], FYi_[2 * q][j], FYi_[2 * q + 1][j]);
                        upk2(FY2i[q][j], FY2i_[2 * q][j], FY2i_[2 * q + 1][j]);
                    }
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    float m0 = 0.f, m1 = 0.f;
#pragma unroll
                    for (int j = 0; j < ROWS; ++j) {
                        FS1[f][j] = sqrtf(fmaf(FS1[f][j], FS1[f][j], FYi_[f][j] * FYi_[f][j]));
                        FYd[f][j] = sqrtf(fmaf(FYd[f][j], FYd[f][j], FY2i_[f][j] * FY2i_[f][j]));
                        if (col_ok && r_first + j < nz) {
                            m0 = fmaxf(m0, FS1[f][j]);
                            m1 = fmaxf(m1, FYd[f][j]);
                        }
                    }
                    unsigned *mb = f == 0 ? J->maxbits : J->maxbits_more[f - 1];
                    if (mb) {  // uniform per job; every lane of the warp is here
                        const unsigned r0 = __reduce_max_sync(0xffffffffu, __float_as_uint(m0));
                        const unsigned r1 = __reduce_max_sync(0xffffffffu, __float_as_uint(m1));
                        if (lane == 0) {
                            int slot = 0;
                            if (modes & BF_DAS)
                                atomicMax(mb + slot++, r0);
                            if (modes & BF_DMAS)
                                atomicMax(mb + slot, r1);
                        }
                    }
                }
            }
            if (staged_job(J)) {
                // the tile's images into the staging area (plane p = frame, then
                // combiner; column = lane), then the storer warp writes them out
                if (epi_use > 0 &&
                    !__all_sync(0xffffffffu,
                                mbar_wait(&sh.epi_empty, (epi_use - 1) & 1u, deadline, err)))
                    return;  // warp-uniform: a bounded wait ran out (error bit set)
                const uint32_t eb =
                    smem_u32(smem + kHeaderBytes) + (uint32_t)(lane * CFL + warp * ROWS) * 4u;
                int p = 0;
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    if (modes & BF_DAS) {
#pragma unroll
                        for (int j = 0; j < ROWS; j += 2)
                            sts_f32x2(eb + (uint32_t)(p * kTileCols * CFL + j) * 4u,
                                      FS1[f][j] * scale, FS1[f][j + 1] * scale);
                        ++p;
                    }
                    if (modes & BF_DMAS) {
#pragma unroll
                        for (int j = 0; j < ROWS; j += 2)
                            sts_f32x2(eb + (uint32_t)(p * kTileCols * CFL + j) * 4u,
                                      FYd[f][j] * scale, FYd[f][j + 1] * scale);
                        ++p;
                    }
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&sh.epi_full);
                ++epi_use;
                continue;
            }
            if (!col_ok)
                continue;
            float *yf[NF];
            yf[0] = y;
#pragma unroll
            for (int f = 1; f < NF; ++f)
                yf[f] = J->y_more[f - 1];
            unsigned long long align = 0;
#pragma unroll
            for (int f = 0; f < NF; ++f)
                align |= reinterpret_cast<unsigned long long>(yf[f]);
            if ((nz & 1) == 0 && (align & 7) == 0 && r_first + ROWS <= nz) {
                // rows in pairs: one 8-byte store per pair (8-byte aligned images,
                // nz even, r_first even)
#pragma unroll
                for (int j = 0; j < ROWS; j += 2) {
                    const size_t o = (size_t)ix * nz + r_first + j;
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        int slot = 0;
                        if (modes & BF_DAS)
                            *reinterpret_cast<float2 *>(yf[f] + (size_t)(slot++) * plane + o) =
                                make_float2(FS1[f][j] * scale, FS1[f][j + 1] * scale);
                        if (modes & BF_DMAS)
                            *reinterpret_cast<float2 *>(yf[f] + (size_t)(slot++) * plane + o) =
                                make_float2(FYd[f][j] * scale, FYd[f][j + 1] * scale);
                    }
                }
                continue;
            }
#pragma unroll
            for (int j = 0; j < ROWS; ++j) {
                const int iz = r_first + j;
                if (iz >= nz)
                    break;
                const size_t o = (size_t)ix * nz + iz;
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    int slot = 0;
                    if (modes & BF_DAS)
                        yf[f][(size_t)(slot++) * plane + o] = FS1[f][j] * scale;
                    if (modes & BF_DMAS)
                        yf[f][(size_t)(slot++) * plane + o] = FYd[f][j] * scale;
                }
            }
        } else {
            if (!col_ok)
                continue;
#pragma unroll
            for (int j = 0; j < ROWS; ++j) {
                const int iz = r_first + j;
                if (iz >= nz)
                    break;
                const size_t o = (size_t)ix * nz + iz;
                int slot = 0;
                if (modes & BF_DAS)
                    y[(size_t)(slot++) * plane + o] = S1[j] * scale;
                if (modes & BF_DMAS)
                    y[(size_t)(slot++) * plane + o] = Yd[j] * scale;
                if (modes & BF_CF) {
                    const float mtot = (float)na * (float)__ldg(J->apcnt + o);
                    const float den = mtot * Su2[j];
                    y[(size_t)(slot++) * plane + o] =
                        den > 0.f ? (S1[j] * S1[j] / den) * S1[j] * scale : 0.f;
                }
                if (modes & BF_PDAS)
                    y[(size_t)(slot++) * plane + o] = Yp[j] * scale;
            }
        }
    }
}

// ----------------------------------------------------- plain (baseline) --

// One frame per launch, one thread per pixel, FP32, the int16 records read
// straight from global memory (no staging, no tiles): the straightforward
// port of the per-pixel loop, kept as the comparison baseline for the batched
// and served paths.  Same tables and the same split delay as beamform_kernel.
template <bool DMAS, bool CF>
__global__ void __launch_bounds__(256) plain_kernel(const BfJob J, const int16_t *__restrict__ rf,
                                                    const int2 *__restrict__ valid,
                                                    const float *__restrict__ dx2, int nxp, int ns)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (long long)J.nx * J.nz)
        return;
    const int ix = (int)(p / J.nz), iz = (int)(p - (long long)ix * J.nz);
    const float Z = __ldg(J.rowZ + iz);
    float S1 = 0.f, Yd = 0.f, Su2 = 0.f, Yp = 0.f;
    const bool pdas = (J.modes & BF_PDAS) != 0;
    for (int a = 0; a < J.na; ++a) {
        const int K = __ldg(J.colK + a * J.nx + ix) + __ldg(J.rowK + a * J.nz + iz);
        const float f = __ldg(J.colF + a * J.nx + ix) + __ldg(J.rowF + a * J.nz + iz) - 0.5f;
        float T1 = 0.f, T2 = 0.f, P1 = 0.f;
        for (int i = 0; i < J.ne; ++i) {
            const int2 vr = __ldg(valid + ((size_t)a * J.ne + i) * nxp + ix);
            if (iz < vr.x || iz > vr.y)
                continue;
            const float x = rx_excess(__ldg(dx2 + (size_t)i * nxp + ix), Z) + f;
            const float m = x + kRoundMagic;
            const float al = x - (m - kRoundMagic);
            // the host decided 0 <= floor(n) <= ns - 2; FP32 rounding may land one sample
            // off at a record end, so clamp and move the weight with it (continuous)
            const int kk = __float_as_int(m) - kRoundBits + K;
            const int k = min(max(kk, 0), ns - 2);
            const int16_t *u = rf + ((size_t)a * J.ne + i) * ns;
            const float u0 = (float)__ldg(u + k), u1 = (float)__ldg(u + k + 1);
            const float v = fmaf(al + 0.5f + (float)(kk - k), u1 - u0, u0);
            S1 += v;
            if (DMAS) {
                const float av = fabsf(v);
                T1 += copysignf(sqrt_approx(av), v);
                T2 += av;
            }
            if (CF)
                Su2 = fmaf(v, v, Su2);
            if (pdas)
                P1 += copysignf(powf(fabsf(v), J.pdas_inv_p), v);
        }
        if (DMAS)
            Yd = fmaf(0.5f * T1, T1, fmaf(-0.5f, T2, Yd));
        if (pdas)
            Yp += copysignf(powf(fabsf(P1), J.pdas_p), P1);
    }
    const size_t plane = (size_t)J.nx * J.nz, o = (size_t)ix * J.nz + iz;
    int slot = 0;
    if (J.modes & BF_DAS)
        J.y[(size_t)(slot++) * plane + o] = S1;
    if (J.modes & BF_DMAS)
        J.y[(size_t)(slot++) * plane + o] = Yd;
    if (J.modes & BF_CF) {
        const float den = (float)J.na * (float)__ldg(J.apcnt + o) * Su2;
        J.y[(size_t)(slot++) * plane + o] = den > 0.f ? (S1 * S1 / den) * S1 : 0.f;
    }
    if (pdas)
        J.y[(size_t)(slot++) * plane + o] = Yp;
}

// ------------------------------------------------------------- envelope --

__device__ __forceinline__ float spectral_weight(int k, int L, int band, int kb_lo, int kb_hi)
{
    float h = (k == 0) ? 1.f : (2 * k < L) ? 2.f : (2 * k == L) ? 1.f : 0.f;
    if (band && (k < kb_lo || k > kb_hi))
        h = 0.f;
    return h;
}

// Envelope transform buffers: plain, or in the swz layout.  Measured on the
// 512 x 512 workload: the swizzle removes the strided passes' bank conflicts
// (shared wavefronts 7.9 M -> 3.2 M per 8 frames) but its index arithmetic
// adds half again the instructions, and the kernel ends no faster; the
// per-pass twiddle table alone takes the envelope + log stages from 0.285 to
// 0.260 ms per 64 frames.
constexpr bool kEnvSwizzle = false;

// Analytic-signal envelope of an image's columns.  The one-sided spectrum
// X * H (H = 1 at 0 and L/2, 2 between, 0 for negative frequencies), times
// the band-pass B for the DMAS image, has as inverse transform r + i h: r is
// the column filtered by B mirrored onto negative frequencies (the column
// itself without band-pass) and h its Hilbert transform, the multiplier
// -i sgn(k) B(|k|) with sgn(0) = sgn(L/2) = 0.  Both are real and linear in
// the column, so two columns a, b go through one complex transform of
// a + i b: the inverse transforms of M(k) (A + iB) give r_a + i r_b and
// h_a + i h_b.
__global__ void __launch_bounds__(256) envelope_kernel(const EnvJob *__restrict__ jobs,
                                                       const int *__restrict__ blk_prefix,
                                                       int njobs)
{
    extern __shared__ __align__(16) float2 sbuf[];
    __shared__ float red[32];
    // blocks in reverse: the beamformer writes a batch's last images last, so
    // those are still in L2 when this kernel starts (and the log stage, in
    // launch order, then reads the envelopes written last first)
    const int blk = gridDim.x - 1 - blockIdx.x;
    // the log stage's blocks may be scheduled as this grid's CTAs finish (they
    // wait for the whole grid before reading its results)
    asm volatile("griddepcontrol.launch_dependents;");
    const int jb = find_job(blk_prefix, njobs, blk);
    const EnvJob J = jobs[jb];
    const int nz = J.nz, m = J.fft_m;
    const int lgm = 31 - __clz(m);
    float lmax = 0.f;

    if (!J.bluestein) {
        const int C = J.cols_per_block >> 1;  // complex columns (pairs of image columns)
        const int c0 = (blk - __ldg(blk_prefix + jb)) * J.cols_per_block;
        float2 *Zb = sbuf, *Pb = sbuf + (size_t)C * m, *Qb = sbuf + (size_t)2 * C * m;
        float2 *tw = sbuf + (size_t)3 * C * m;
        float2 *ptw = tw + m;  // per-pass twiddles of the radix-8 passes
        for (int k = threadIdx.x; k < m; k += blockDim.x)
            tw[k] = __ldg(J.tw + k);
        __syncthreads();
        fill_pass_twiddles(ptw, tw, lgm);
        // Buffers in the swizzled layout (element t at swz(t)): columns in, four
        // depths per thread with 16-byte global loads (m >= 4: nz = m)
        auto at = [](int t) { return swz<kEnvSwizzle>(t); };
        const int vec = J.vec4 ? 4 : 1;
        for (int t = threadIdx.x * vec; t < C * m; t += blockDim.x * vec) {
            const int c = t >> lgm, n = t & (m - 1);
            const int ca = c0 + 2 * c, cb = ca + 1;
            if (vec == 4) {
                const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 a = ca < J.nx ? __ldg(reinterpret_cast<const float4 *>(J.y + (size_t)ca * nz + n)) : z4;
                const float4 b = cb < J.nx ? __ldg(reinterpret_cast<const float4 *>(J.y + (size_t)cb * nz + n)) : z4;
                Zb[at(t)] = make_float2(a.x, b.x);
                Zb[at(t + 1)] = make_float2(a.y, b.y);
                Zb[at(t + 2)] = make_float2(a.z, b.z);
                Zb[at(t + 3)] = make_float2(a.w, b.w);
            } else {
                const float ya = ca < J.nx ? __ldg(J.y + (size_t)ca * nz + n) : 0.f;
                const float yb = cb < J.nx ? __ldg(J.y + (size_t)cb * nz + n) : 0.f;
                Zb[at(t)] = make_float2(ya, yb);
            }
        }
        __syncthreads();
        float2 *S = fft_r8<kEnvSwizzle>(Zb, Pb, m, lgm, C, tw, false, ptw);  // spectrum of a + i b
        float2 *F1 = S == Zb ? Pb : Zb;                                 // free buffer
        const float inv = 1.f / (float)m;
        if (!J.band) {
            for (int t = threadIdx.x; t < C * m; t += blockDim.x) {
                const int k = t & (m - 1);
                const float sg = (k == 0 || 2 * k == m) ? 0.f : (2 * k < m ? 1.f : -1.f);
                const float2 sv = S[at(t)];
                F1[at(t)] = make_float2(sv.y * sg, -sv.x * sg);  // -i sgn(k) S
            }
            __syncthreads();
            const float2 *Hh = fft_r8<kEnvSwizzle>(F1, S, m, lgm, C, tw, true, ptw);
            for (int t = threadIdx.x * vec; t < C * m; t += blockDim.x * vec) {
                const int c = t >> lgm, n = t & (m - 1);
                const int ca = c0 + 2 * c, cb = ca + 1;
                if (vec == 4) {
                    const float2 h0 = Hh[at(t)], h1 = Hh[at(t + 1)], h2 = Hh[at(t + 2)],
                                 h3 = Hh[at(t + 3)];
                    if (ca < J.nx) {
                        const float4 a = __ldg(reinterpret_cast<const float4 *>(J.y + (size_t)ca * nz + n));
                        const float4 e = make_float4(hypotf(a.x, h0.x * inv), hypotf(a.y, h1.x * inv),
                                                     hypotf(a.z, h2.x * inv), hypotf(a.w, h3.x * inv));
                        *reinterpret_cast<float4 *>(J.env + (size_t)ca * nz + n) = e;
                        lmax = fmaxf(lmax, fmaxf(fmaxf(e.x, e.y), fmaxf(e.z, e.w)));
                    }
                    if (cb < J.nx) {
                        const float4 b = __ldg(reinterpret_cast<const float4 *>(J.y + (size_t)cb * nz + n));
                        const float4 e = make_float4(hypotf(b.x, h0.y * inv), hypotf(b.y, h1.y * inv),
                                                     hypotf(b.z, h2.y * inv), hypotf(b.w, h3.y * inv));
                        *reinterpret_cast<float4 *>(J.env + (size_t)cb * nz + n) = e;
                        lmax = fmaxf(lmax, fmaxf(fmaxf(e.x, e.y), fmaxf(e.z, e.w)));
                    }
                    continue;
                }
                const float2 h = Hh[at(t)];
                if (ca < J.nx) {
                    const float e = hypotf(__ldg(J.y + (size_t)ca * nz + n), h.x * inv);
                    J.env[(size_t)ca * nz + n] = e;
                    lmax = fmaxf(lmax, e);
                }
                if (cb < J.nx) {
                    const float e = hypotf(__ldg(J.y + (size_t)cb * nz + n), h.y * inv);
                    J.env[(size_t)cb * nz + n] = e;
                    lmax = fmaxf(lmax, e);
                }
            }
        } else {
            for (int t = threadIdx.x; t < C * m; t += blockDim.x) {
                const int k = t & (m - 1);
                const int kk = 2 * k <= m ? k : m - k;  // |k|
                const float bp = (kk >= J.kb_lo && kk <= J.kb_hi) ? 1.f : 0.f;
                const float sg = (k == 0 || 2 * k == m) ? 0.f : (2 * k < m ? 1.f : -1.f);
                const float2 sv = S[at(t)];
                const float2 r = make_float2(sv.x * bp, sv.y * bp);
                S[at(t)] = r;
                Qb[at(t)] = make_float2(r.y * sg, -r.x * sg);
            }
            __syncthreads();
            float2 *R = fft_r8<kEnvSwizzle>(S, F1, m, lgm, C, tw, true, ptw);
            float2 *F2 = R == S ? F1 : S;
            const float2 *Hh = fft_r8<kEnvSwizzle>(Qb, F2, m, lgm, C, tw, true, ptw);
            for (int t = threadIdx.x * vec; t < C * m; t += blockDim.x * vec) {
                const int c = t >> lgm, n = t & (m - 1);
                const int ca = c0 + 2 * c, cb = ca + 1;
                if (vec == 4) {
                    float2 rr[4], hh[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        rr[u] = R[at(t + u)];
                        hh[u] = Hh[at(t + u)];
                    }
                    if (ca < J.nx) {
                        const float4 e = make_float4(hypotf(rr[0].x, hh[0].x) * inv, hypotf(rr[1].x, hh[1].x) * inv,
                                                     hypotf(rr[2].x, hh[2].x) * inv, hypotf(rr[3].x, hh[3].x) * inv);
                        *reinterpret_cast<float4 *>(J.env + (size_t)ca * nz + n) = e;
                        lmax = fmaxf(lmax, fmaxf(fmaxf(e.x, e.y), fmaxf(e.z, e.w)));
                    }
                    if (cb < J.nx) {
                        const float4 e = make_float4(hypotf(rr[0].y, hh[0].y) * inv, hypotf(rr[1].y, hh[1].y) * inv,
                                                     hypotf(rr[2].y, hh[2].y) * inv, hypotf(rr[3].y, hh[3].y) * inv);
                        *reinterpret_cast<float4 *>(J.env + (size_t)cb * nz + n) = e;
                        lmax = fmaxf(lmax, fmaxf(fmaxf(e.x, e.y), fmaxf(e.z, e.w)));
                    }
                    continue;
                }
                const float2 rv = R[at(t)], hv = Hh[at(t)];
                if (ca < J.nx) {
                    const float e = hypotf(rv.x, hv.x) * inv;
                    J.env[(size_t)ca * nz + n] = e;
                    lmax = fmaxf(lmax, e);
                }
                if (cb < J.nx) {
                    const float e = hypotf(rv.y, hv.y) * inv;
                    J.env[(size_t)cb * nz + n] = e;
                    lmax = fmaxf(lmax, e);
                }
            }
        }
    } else {
        // one column per block through Bluestein's chirp transforms
        const int c0 = blk - __ldg(blk_prefix + jb);
        float2 *A = sbuf, *B = sbuf + m, *tw = sbuf + (size_t)3 * m;
        for (int k = threadIdx.x; k < m; k += blockDim.x)
            tw[k] = __ldg(J.tw + k);
        const float *__restrict__ y = J.y + (size_t)c0 * nz;
        const float2 *__restrict__ w = J.chirp;
        const float2 *__restrict__ bh = J.bhat;
        const float inv_m = 1.f / (float)m;
        // forward DFT: X_k = conj(w_k) * (a (*) w)_k with a_n = y_n conj(w_n)
        for (int n = threadIdx.x; n < m; n += blockDim.x) {
            float2 v = make_float2(0.f, 0.f);
            if (n < nz) {
                const float2 c = __ldg(w + n);
                const float yn = __ldg(y + n);
                v = make_float2(yn * c.x, -yn * c.y);
            }
            A[n] = v;
        }
        __syncthreads();
        float2 *X = fft_r8(A, B, m, lgm, 1, tw, false);
        for (int k = threadIdx.x; k < m; k += blockDim.x)
            X[k] = cmul(X[k], __ldg(bh + k));
        __syncthreads();
        float2 *O = X == A ? B : A;
        float2 *Cb = fft_r8(X, O, m, lgm, 1, tw, true);
        float2 *D = Cb == A ? B : A;
        // masked spectrum, conjugated and pre-multiplied by conj(w) for the second
        // pass: the inverse DFT of S is conj(DFT(conj S)) / nz
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            float2 v = make_float2(0.f, 0.f);
            if (k < nz) {
                const float2 c = __ldg(w + k);
                const float2 cc = make_float2(c.x, -c.y);
                float2 xk = cmul(make_float2(Cb[k].x * inv_m, Cb[k].y * inv_m), cc);
                const float h = spectral_weight(k, nz, J.band, J.kb_lo, J.kb_hi);
                xk = make_float2(xk.x * h, -xk.y * h);
                v = cmul(xk, cc);
            }
            D[k] = v;
        }
        __syncthreads();
        float2 *E = fft_r8(D, Cb, m, lgm, 1, tw, false);
        for (int k = threadIdx.x; k < m; k += blockDim.x)
            E[k] = cmul(E[k], __ldg(bh + k));
        __syncthreads();
        float2 *F = fft_r8(E, E == A ? B : A, m, lgm, 1, tw, true);
        const float inv = inv_m / (float)nz;
        float *__restrict__ env = J.env + (size_t)c0 * nz;
        for (int n = threadIdx.x; n < nz; n += blockDim.x) {
            const float e = hypotf(F[n].x, F[n].y) * inv;
            env[n] = e;
            lmax = fmaxf(lmax, e);
        }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1)
        lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, off));
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = lmax;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
        for (int off = 16; off; off >>= 1)
            v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
        if (threadIdx.x == 0)
            atomicMax(J.maxbits, __float_as_uint(v));  // env >= 0: bit order = value order
    }
}

// ------------------------------------------------------------ f-k migration --

// Per channel record: transform along time (zero-padded to nt), then the
// transmit's lateral delay removed per bin, written to D[a][b][i].
__global__ void __launch_bounds__(256) fk_time_kernel(const FkJob J)
{
    extern __shared__ __align__(16) float2 fbuf[];
    const int row = blockIdx.x, a = row / J.ne, i = row - a * J.ne;
    const int m = J.nt;
    float2 *X = fbuf, *Y = fbuf + m, *tw = fbuf + 2 * (size_t)m;
    const int16_t *__restrict__ u = J.rf + (size_t)row * J.ns;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        tw[k] = __ldg(J.tw_t + k);
        X[k] = make_float2(k < J.ns ? (float)__ldg(u + k) : 0.f, 0.f);
    }
    __syncthreads();
    const float2 *S = fft_r8(X, Y, m, J.lgt, 1, tw, false);
    const float beta = __ldg(J.beta + row);
    const int nf = m / 2 + 1;
    float2 *__restrict__ D = J.D + (size_t)a * nf * J.nk + i;
    for (int b = threadIdx.x; b < nf; b += blockDim.x) {
        float sn, cs;
        sincosf((float)b * beta, &sn, &cs);
        D[(size_t)b * J.nk] = cmul(S[b], make_float2(cs, sn));
    }
}

// Transforms of `rows` rows of length n held with stride n: entries from
// len_in on are taken as zero; `per` rows per CTA.
__global__ void __launch_bounds__(256) fk_rows_kernel(float2 *data, int rows, int len_in, int n,
                                                      int lg, int per, const float2 *tw_g,
                                                      int inverse)
{
    extern __shared__ __align__(16) float2 fbuf[];
    float2 *X = fbuf, *Y = fbuf + (size_t)per * n, *tw = fbuf + 2 * (size_t)per * n;
    const int r0 = blockIdx.x * per;
    const int nr = min(per, rows - r0);
    for (int k = threadIdx.x; k < n; k += blockDim.x)
        tw[k] = __ldg(tw_g + k);
    for (int t = threadIdx.x; t < per * n; t += blockDim.x) {
        const int rr = t / n, k = t - rr * n;
        X[t] = (rr < nr && k < len_in) ? data[(size_t)(r0 + rr) * n + k] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2 *S = fft_r8(X, Y, n, lg, per, tw, inverse != 0);
    for (int t = threadIdx.x; t < nr * n; t += blockDim.x)
        data[(size_t)r0 * n + t] = S[t];
}

// Migrated spectrum at (q = 1 .. nt/2, m): every angle's spectrum of lateral
// bin m, interpolated between temporal bins i0 and i0 + 1 and weighted, summed.
// The mapping (exact plane-wave or Stolt's) is tabulated on the host in double
// precision: this kernel only gathers and sums in FP32.
__global__ void __launch_bounds__(256) fk_map_kernel(const FkJob J)
{
    const int nk = J.nk, half = J.nt / 2;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)half * nk)
        return;
    const int m = (int)(idx % nk);
    const int nf = half + 1;
    float2 acc = make_float2(0.f, 0.f);
    for (int a = 0; a < J.na; ++a) {
        const size_t t = (size_t)a * half * nk + (size_t)idx;
        const int i0 = __ldg(J.map_i0 + t);
        if (i0 < 0)
            continue;
        const float2 aw = __ldg(J.map_aw + t);  // (alpha, weight)
        const int i1 = min(i0 + 1, half);
        const float2 *D = J.D + (size_t)a * nf * nk + m;
        const float2 v0 = D[(size_t)i0 * nk], v1 = D[(size_t)i1 * nk];
        acc.x = fmaf(aw.y, fmaf(aw.x, v1.x - v0.x, v0.x), acc.x);
        acc.y = fmaf(aw.y, fmaf(aw.x, v1.y - v0.y, v0.y), acc.y);
    }
    J.spec[idx] = acc;
}

// Per image column m < ne: inverse transform along depth of the migrated
// spectrum's column (Kz bins 1 .. nt/2, zero elsewhere), magnitude of the
// first ns samples (the 1 / (nt nk) of both inverse transforms applied here).
__global__ void __launch_bounds__(256) fk_depth_kernel(const FkJob J)
{
    extern __shared__ __align__(16) float2 fbuf[];
    __shared__ float red[32];
    const int mcol = blockIdx.x, n = J.nt, half = n / 2;
    float2 *X = fbuf, *Y = fbuf + n, *tw = fbuf + 2 * (size_t)n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        tw[k] = __ldg(J.tw_t + k);
        X[k] = (k >= 1 && k <= half) ? J.spec[(size_t)(k - 1) * J.nk + mcol] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2 *S = fft_r8(X, Y, n, J.lgt, 1, tw, true);
    const float inv = 1.f / ((float)n * (float)J.nk);
    float lmax = 0.f;
    float *__restrict__ out = J.img + (size_t)mcol * J.ns;
    for (int z = threadIdx.x; z < J.ns; z += blockDim.x) {
        const float e = hypotf(S[z].x, S[z].y) * inv;
        out[z] = e;
        lmax = fmaxf(lmax, e);
    }
    if (J.maxbits) {
#pragma unroll
        for (int off = 16; off; off >>= 1)
            lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, off));
        if ((threadIdx.x & 31) == 0)
            red[threadIdx.x >> 5] = lmax;
        __syncthreads();
        if (threadIdx.x < 32) {
            float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
            for (int off = 16; off; off >>= 1)
                v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
            if (threadIdx.x == 0)
                atomicMax(J.maxbits, __float_as_uint(v));
        }
    }
}

// ------------------------------------------------------------------ log --

constexpr int kLogPerBlock = 4096;

__global__ void __launch_bounds__(256) log_kernel(const LogJob *__restrict__ jobs,
                                                  const int *__restrict__ blk_prefix, int njobs,
                                                  float dr)
{
    // blocks in launch order: the envelope kernels walk a batch's images in
    // reverse, so the envelopes written last (still in L2) are read first
    const int blk = blockIdx.x;
    const int jb = find_job(blk_prefix, njobs, blk);
    const LogJob J = jobs[jb];
    const size_t base = (size_t)(blk - __ldg(blk_prefix + jb)) * kLogPerBlock;
    // Launched as a programmatic dependent of the envelope kernel: this block
    // may start while that grid's last CTAs still run, and waits here until
    // the grid has completed and its envelopes and maxima are visible.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const float peak = __uint_as_float(__ldcg(J.maxbits));
    // 20 log10(e / peak) = (20 log10 2) (log2 e - log2 peak), the logarithm on the
    // special-function unit (absolute error ~1e-6 of a unit of log2: ~1e-5 dB)
    const float lp = peak > 0.f ? __log2f(peak) : 0.f;
    auto db = [&](float e) {
        return (e > 0.f && peak > 0.f) ? fminf(fmaxf(6.0205999132796239f * (__log2f(e) - lp), -dr), 0.f)
                                       : -dr;
    };
    if (J.vec4) {  // sixteen pixels per thread as four 16-byte loads issued together
        float4 e[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const size_t pu = base + (size_t)threadIdx.x * 4 + (size_t)u * blockDim.x * 4;
            ok[u] = pu < (size_t)J.n;
            e[u] = ok[u] ? __ldcs(reinterpret_cast<const float4 *>(J.env + pu))
                         : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const size_t pu = base + (size_t)threadIdx.x * 4 + (size_t)u * blockDim.x * 4;
            if (ok[u])
                __stcs(reinterpret_cast<float4 *>(J.out + pu),
                       make_float4(db(e[u].x), db(e[u].y), db(e[u].z), db(e[u].w)));
        }
        return;
    }
    for (int t = threadIdx.x; t < kLogPerBlock; t += blockDim.x) {
        const size_t p = base + t;
        if (p >= (size_t)J.n)
            break;
        J.out[p] = db(__ldg(J.env + p));
    }
}

template <int PREC, bool DMAS, bool CF, bool PDAS, int ROWS, int NF = 1>
cudaError_t launch_bf_t(const BfJob *jobs, const int *prefix, int njobs, int tiles, size_t smem,
                        int *err, cudaStream_t st)
{
    auto k = beamform_kernel<PREC, DMAS, CF, PDAS, ROWS, NF>;
    // several CTAs per SM need the largest shared-memory carveout
    constexpr int threads = beamform_threads<NF>();
    int sms = 0, occ = 0;
    cudaError_t e = kernel_setup((const void *)k, smem, threads, true, &sms, &occ);
    if (e != cudaSuccess)
        return e;
    // persistent grid: every CTA resident at once, each walking the tiles
    const int grid = std::max(1, std::min(tiles, std::max(occ, 1) * sms));
    const int stride = (int)((smem - kHeaderBytes - epi_bytes(NF, ROWS)) / stages_for_rows(ROWS));
    k<<<grid, threads, smem, st>>>(jobs, prefix, njobs, tiles, stride, err);
    return cudaGetLastError();
}

template <int PREC, bool PDAS, int ROWS>
cudaError_t launch_bf_pdr(const BfJob *jobs, const int *prefix, int njobs, int tiles, size_t smem,
                          int dmas, int cf, int *err, cudaStream_t st)
{
    if (dmas && cf)
        return launch_bf_t<PREC, true, true, PDAS, ROWS>(jobs, prefix, njobs, tiles, smem, err, st);
    if (dmas)
        return launch_bf_t<PREC, true, false, PDAS, ROWS>(jobs, prefix, njobs, tiles, smem, err, st);
    if (cf)
        return launch_bf_t<PREC, false, true, PDAS, ROWS>(jobs, prefix, njobs, tiles, smem, err, st);
    return launch_bf_t<PREC, false, false, PDAS, ROWS>(jobs, prefix, njobs, tiles, smem, err, st);
}

// Jobs of NF frames each (DAS / DMAS of the RF precisions).
template <int ROWS, int NF>
cudaError_t launch_bf_frames(const BfJob *j, const int *pf, int njobs, int tiles, size_t smem,
                             int prec, int dmas, int *err, cudaStream_t st)
{
    if (prec == kPrecF32)
        return dmas ? launch_bf_t<kPrecF32, true, false, false, ROWS, NF>(j, pf, njobs, tiles, smem, err, st)
                    : launch_bf_t<kPrecF32, false, false, false, ROWS, NF>(j, pf, njobs, tiles, smem, err, st);
    if (prec == kPrecF16)
        return dmas ? launch_bf_t<kPrecF16, true, false, false, ROWS, NF>(j, pf, njobs, tiles, smem, err, st)
                    : launch_bf_t<kPrecF16, false, false, false, ROWS, NF>(j, pf, njobs, tiles, smem, err, st);
    return dmas ? launch_bf_t<kPrecBF16, true, false, false, ROWS, NF>(j, pf, njobs, tiles, smem, err, st)
                : launch_bf_t<kPrecBF16, false, false, false, ROWS, NF>(j, pf, njobs, tiles, smem, err, st);
}

// IQ-DAS (always) and BB-DMAS (in the DMAS slot) jobs of NF frames each.
template <int ROWS, int NF>
cudaError_t launch_bf_iq(const BfJob *j, const int *pf, int njobs, int tiles, size_t smem, int dmas,
                         int *err, cudaStream_t st)
{
    return dmas ? launch_bf_t<kPrecIQ, true, false, false, ROWS, NF>(j, pf, njobs, tiles, smem, err, st)
                : launch_bf_t<kPrecIQ, false, false, false, ROWS, NF>(j, pf, njobs, tiles, smem, err, st);
}

template <int PREC>
cudaError_t launch_bf_p(const BfJob *jobs, const int *prefix, int njobs, int tiles, size_t smem,
                        int dmas, int cf, int pdas, int rows, int *err, cudaStream_t st)
{
    if (rows == 4)
        return pdas ? launch_bf_pdr<PREC, true, 4>(jobs, prefix, njobs, tiles, smem, dmas, cf, err, st)
                    : launch_bf_pdr<PREC, false, 4>(jobs, prefix, njobs, tiles, smem, dmas, cf, err, st);
    return pdas ? launch_bf_pdr<PREC, true, 8>(jobs, prefix, njobs, tiles, smem, dmas, cf, err, st)
                : launch_bf_pdr<PREC, false, 8>(jobs, prefix, njobs, tiles, smem, dmas, cf, err, st);
}

}  // namespace

size_t beamform_smem_bytes(int wmax, int group, int prec, int nf, int rows)
{
    return (size_t)kHeaderBytes + (size_t)epi_bytes(nf, rows) +
           (size_t)stages_for_rows(rows) * stage_bytes(group, wmax, pair_bytes(prec), nf);
}

// Image columns per envelope CTA for a power-of-two transform: two per
// complex column, up to 2048 complex points per buffer.
int envelope_cols_per_block(int fft_m) { return 2 * (fft_m >= 2048 ? 1 : 2048 / fft_m); }

// Shared memory of an envelope CTA: three transform buffers and the twiddles.
size_t envelope_smem_bytes(int fft_m, int bluestein)
{
    const int c = bluestein ? 1 : envelope_cols_per_block(fft_m) / 2;
    int lgm = 0;
    while ((1 << lgm) < fft_m)
        ++lgm;
    const size_t passes = bluestein ? 0 : (size_t)pass_twiddle_count(lgm);
    return (3u * (size_t)c * fft_m + (size_t)fft_m + passes) * sizeof(float2);
}

cudaError_t launch_plan(const PlanJob &job, int *err_dev, cudaStream_t stream)
{
    dim3 grid(job.tiles_x * job.tiles_z, job.na);
    plan_kernel<<<grid, 128, 0, stream>>>(job, err_dev);
    return cudaGetLastError();
}

cudaError_t launch_ingest(const IngestJob *jobs_dev, const int *blk_prefix_dev, int njobs,
                          int total_blocks, int prec, cudaStream_t stream)
{
    if (njobs <= 0 || total_blocks <= 0)
        return cudaSuccess;
    if (prec == kPrecF32)
        ingest_kernel<kPrecF32><<<total_blocks, 256, 0, stream>>>(jobs_dev, blk_prefix_dev, njobs);
    else if (prec == kPrecF16)
        ingest_kernel<kPrecF16><<<total_blocks, 256, 0, stream>>>(jobs_dev, blk_prefix_dev, njobs);
    else
        ingest_kernel<kPrecBF16><<<total_blocks, 256, 0, stream>>>(jobs_dev, blk_prefix_dev, njobs);
    return cudaGetLastError();
}

size_t demod_smem_bytes(int ns, bool pairs) { return (size_t)(pairs ? 4 : 3) * ns * sizeof(float2); }

cudaError_t launch_demod(const DemodJob *jobs_dev, const int *row_prefix_dev, int njobs,
                         int total_rows, int max_ns, bool pairs, cudaStream_t stream)
{
    if (njobs <= 0 || total_rows <= 0)
        return cudaSuccess;
    const size_t smem = demod_smem_bytes(max_ns, pairs);
    int sms = 0;
    cudaError_t e = kernel_setup((const void *)demod_kernel, smem, 256, false, &sms, nullptr);
    if (e != cudaSuccess)
        return e;
    demod_kernel<<<total_rows, 256, smem, stream>>>(jobs_dev, row_prefix_dev, njobs);
    return cudaGetLastError();
}

cudaError_t launch_beamform(const BfJob *jobs_dev, const int *tile_prefix_dev, int njobs,
                            int total_tiles, size_t smem_bytes, int prec, int variant, int rows,
                            int nf, int *err_dev, cudaStream_t stream)
{
    if (njobs <= 0 || total_tiles <= 0)
        return cudaSuccess;
    const int dmas = (variant & BF_DMAS) ? 1 : 0, cf = (variant & BF_CF) ? 1 : 0;
    const int pdas = (variant & BF_PDAS) ? 1 : 0;
    if (nf > 1 || rows == 2) {
        // frames sharing the delays, and every two-row tile: DAS / DMAS of RF
        // records, IQ-DAS / BB-DMAS of analytic signals
        if (cf || pdas)
            return cudaErrorInvalidValue;
        const BfJob *j = jobs_dev;
        const int *pf = tile_prefix_dev;
        if (prec == kPrecIQ) {
            if (rows == 4 && nf == 2)
                return launch_bf_iq<4, 2>(j, pf, njobs, total_tiles, smem_bytes, dmas, err_dev, stream);
            if (rows == 2 && nf == 4)
                return launch_bf_iq<2, 4>(j, pf, njobs, total_tiles, smem_bytes, dmas, err_dev, stream);
            if (rows == 2 && nf == 2)
                return launch_bf_iq<2, 2>(j, pf, njobs, total_tiles, smem_bytes, dmas, err_dev, stream);
            if (rows == 2 && nf == 1)
                return launch_bf_iq<2, 1>(j, pf, njobs, total_tiles, smem_bytes, dmas, err_dev, stream);
            return cudaErrorInvalidValue;
        }
        if (rows == 4 && nf == 2)
            return launch_bf_frames<4, 2>(j, pf, njobs, total_tiles, smem_bytes, prec, dmas, err_dev, stream);
        if (rows == 2 && nf == 4)
            return launch_bf_frames<2, 4>(j, pf, njobs, total_tiles, smem_bytes, prec, dmas, err_dev, stream);
        if (rows == 2 && nf == 2)
            return launch_bf_frames<2, 2>(j, pf, njobs, total_tiles, smem_bytes, prec, dmas, err_dev, stream);
        if (rows == 2 && nf == 1)
            return launch_bf_frames<2, 1>(j, pf, njobs, total_tiles, smem_bytes, prec, dmas, err_dev, stream);
        return cudaErrorInvalidValue;
    }
    if (prec == kPrecIQ) {  // IQ-DAS always, BB-DMAS in the DMAS slot
        if (rows == 4)
            return dmas ? launch_bf_t<kPrecIQ, true, false, false, 4>(jobs_dev, tile_prefix_dev, njobs,
                                                                     total_tiles, smem_bytes, err_dev, stream)
                        : launch_bf_t<kPrecIQ, false, false, false, 4>(jobs_dev, tile_prefix_dev, njobs,
                                                                      total_tiles, smem_bytes, err_dev, stream);
        return dmas ? launch_bf_t<kPrecIQ, true, false, false, 8>(jobs_dev, tile_prefix_dev, njobs,
                                                                 total_tiles, smem_bytes, err_dev, stream)
                    : launch_bf_t<kPrecIQ, false, false, false, 8>(jobs_dev, tile_prefix_dev, njobs,
                                                                  total_tiles, smem_bytes, err_dev, stream);
    }
    if (prec == kPrecF32)
        return launch_bf_p<kPrecF32>(jobs_dev, tile_prefix_dev, njobs, total_tiles, smem_bytes,
                                     dmas, cf, pdas, rows, err_dev, stream);
    if (prec == kPrecF16)
        return launch_bf_p<kPrecF16>(jobs_dev, tile_prefix_dev, njobs, total_tiles, smem_bytes,
                                     dmas, cf, pdas, rows, err_dev, stream);
    return launch_bf_p<kPrecBF16>(jobs_dev, tile_prefix_dev, njobs, total_tiles, smem_bytes, dmas,
                                  cf, pdas, rows, err_dev, stream);
}

cudaError_t launch_plain(const BfJob &job, const int16_t *rf, const int2 *valid, const float *dx2,
                         int nxp, int ns, cudaStream_t stream)
{
    const long long px = (long long)job.nx * job.nz;
    const int blocks = (int)((px + 255) / 256);
    const int dmas = (job.modes & BF_DMAS) ? 1 : 0, cf = (job.modes & BF_CF) ? 1 : 0;
    if (dmas && cf)
        plain_kernel<true, true><<<blocks, 256, 0, stream>>>(job, rf, valid, dx2, nxp, ns);
    else if (dmas)
        plain_kernel<true, false><<<blocks, 256, 0, stream>>>(job, rf, valid, dx2, nxp, ns);
    else if (cf)
        plain_kernel<false, true><<<blocks, 256, 0, stream>>>(job, rf, valid, dx2, nxp, ns);
    else
        plain_kernel<false, false><<<blocks, 256, 0, stream>>>(job, rf, valid, dx2, nxp, ns);
    return cudaGetLastError();
}

cudaError_t launch_envelope(const EnvJob *jobs_dev, const int *blk_prefix_dev, int njobs,
                            int total_blocks, size_t smem, cudaStream_t stream)
{
    if (njobs <= 0 || total_blocks <= 0)
        return cudaSuccess;
    int sms = 0;
    cudaError_t e = kernel_setup((const void *)envelope_kernel, smem, 256, false, &sms, nullptr);
    if (e != cudaSuccess)
        return e;
    envelope_kernel<<<total_blocks, 256, smem, stream>>>(jobs_dev, blk_prefix_dev, njobs);
    return cudaGetLastError();
}

cudaError_t launch_log(const LogJob *jobs_dev, const int *blk_prefix_dev, int njobs,
                       int total_blocks, float dynamic_range_db, cudaStream_t stream)
{
    if (njobs <= 0 || total_blocks <= 0)
        return cudaSuccess;
    // programmatic stream serialization: the blocks may be scheduled before the
    // envelope kernel ends (the kernel's griddepcontrol.wait orders the reads),
    // which hides this launch behind that kernel's last CTAs
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)total_blocks);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, log_kernel, jobs_dev, blk_prefix_dev, njobs, dynamic_range_db);
}

int log_blocks(long long pixels) { return (int)((pixels + kLogPerBlock - 1) / kLogPerBlock); }

cudaError_t kernel_setup(const void *k, size_t smem, int threads, bool max_carveout, int *sms,
                         int *occ)
{
    struct State {
        size_t configured = 48u * 1024u;  // dynamic shared memory allowed without an attribute
        bool carveout = false;
        std::map<std::pair<size_t, int>, int> occ;  // (smem, threads) -> resident CTAs per SM
    };
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, State> state;
    static std::map<int, int> sm_count;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    std::lock_guard<std::mutex> lock(mu);
    auto sm = sm_count.find(dev);
    if (sm == sm_count.end()) {
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess)
            return e;
        sm = sm_count.emplace(dev, n).first;
    }
    *sms = sm->second;
    State &s = state[{dev, k}];
    if (max_carveout && !s.carveout) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess)
            return e;
        s.carveout = true;
    }
    if (smem > s.configured) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        s.configured = smem;
    }
    if (occ) {
        auto it = s.occ.find({smem, threads});
        if (it == s.occ.end()) {
            int n = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem);
            if (e != cudaSuccess)
                return e;
            it = s.occ.emplace(std::make_pair(smem, threads), n).first;
        }
        *occ = it->second;
    }
    return cudaSuccess;
}

cudaError_t launch_fkmig(const FkJob &J, cudaStream_t st)
{
    int sms = 0;
    const size_t s_nt = (size_t)3 * J.nt * sizeof(float2);
    cudaError_t e = kernel_setup((const void *)fk_time_kernel, s_nt, 256, false, &sms, nullptr);
    if (e == cudaSuccess)
        e = kernel_setup((const void *)fk_depth_kernel, s_nt, 256, false, &sms, nullptr);
    const int per = J.nk >= 2048 ? 1 : 2048 / J.nk;
    const size_t s_rows = ((size_t)2 * per * J.nk + J.nk) * sizeof(float2);
    if (e == cudaSuccess)
        e = kernel_setup((const void *)fk_rows_kernel, s_rows, 256, false, &sms, nullptr);
    if (e != cudaSuccess)
        return e;
    const int nf = J.nt / 2 + 1, half = J.nt / 2;
    fk_time_kernel<<<J.na * J.ne, 256, s_nt, st>>>(J);
    const int drows = J.na * nf;
    fk_rows_kernel<<<(drows + per - 1) / per, 256, s_rows, st>>>(J.D, drows, J.ne, J.nk, J.lgk, per,
                                                                   J.tw_k, 0);
    const long long pts = (long long)half * J.nk;
    fk_map_kernel<<<(int)((pts + 255) / 256), 256, 0, st>>>(J);
    fk_rows_kernel<<<(half + per - 1) / per, 256, s_rows, st>>>(J.spec, half, J.nk, J.nk, J.lgk, per,
                                                                  J.tw_k, 1);
    fk_depth_kernel<<<J.ne, 256, s_nt, st>>>(J);
    return cudaGetLastError();
}

}  // namespace bfi

// GB300 (sm_103a) kernels of the plane-wave beamformer.
//
//   plan_kernel      once per (handle, angle set): for every pixel tile, angle
//                    and channel, the first sample pair of the window of the
//                    channel's record the tile reads (or "none")
//   ingest_kernel    int16 channel records of a batch of frames -> staged
//                    sample pairs (FP32 (mid, diff) pairs, or raw FP16 / BF16
//                    pairs), one launch for the whole batch
//   beamform_kernel  per CTA a tile of 32 columns (one per lane) x 8 row bands
//                    (one per warp, `ROWS` contiguous rows per thread).  Per
//                    angle and channel group the tensor memory accelerator
//                    (cp.async.bulk.tensor) copies, into a double-buffered
//                    shared-memory stage tracked by an mbarrier, the group's
//                    window of every channel's record plus the tile's
//                    per-(channel, column) tables; delays are formed in
//                    registers, samples interpolated linearly and combined
//                    (DAS, signed-sqrt DMAS, coherence factor), compounded over
//                    angles (Eq. (1), Sec. II-B)
//   envelope_kernel  per image column the analytic signal along depth via a
//                    shared-memory radix-2 Stockham FFT (Bluestein for other
//                    lengths), one-sided mask and optional [f0, 3 f0]
//                    band-pass, magnitude, and the frame maximum
//   log_kernel       20 log10(env / max) clipped to the -70 dB range of Fig. 3
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <limits.h>

#include "../../include/bf.h"
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

// Receive path length beyond the depth term, in samples:
//   sqrt(dx^2 + z^2) - z = dx^2 / (sqrt(dx^2 + z^2) + z).
// The large, pixel-only part of the delay (transmit leg + depth) comes from
// the host as an exact integer + remainder, so FP32 only has to carry this
// small term; its relative error (a few ulp) stays far below a sample.
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
        for (int w = 0; w < kTileCols; ++w) {
            const int ix = tx * kTileCols + w;
            if (ix >= J.nx)
                break;
            const int2 vr = J.valid[((size_t)a * J.ne + i) * J.nxp + ix];
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
        J.wtab[((size_t)a * J.tiles_x * J.tiles_z + t) * J.ne + i] = w0;
    }
}

// ---------------------------------------------------------------- ingest --

template <int PREC>
__global__ void __launch_bounds__(256) ingest_kernel(const IngestJob *__restrict__ jobs,
                                                     const int *__restrict__ row_prefix, int njobs)
{
    const int jb = find_job(row_prefix, njobs, blockIdx.x);
    const IngestJob J = jobs[jb];
    const int row = blockIdx.x - __ldg(row_prefix + jb);
    const int16_t *__restrict__ u = J.rf + (size_t)row * J.ns;
    const int ns = J.ns;
    auto sample = [&](int k) -> int { return (k >= 0 && k < ns) ? (int)__ldg(u + k) : 0; };
    for (int j0 = threadIdx.x * 8; j0 < J.nsp; j0 += blockDim.x * 8) {
        int s[9];
#pragma unroll
        for (int q = 0; q < 9; ++q)
            s[q] = sample(j0 - kPadL + q);
        if (PREC == kPrecF32) {
            // mid point and difference: v = mid + (alpha - 1/2) * diff (exact for int16)
            float4 *o = reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(J.pairs) +
                                                   (size_t)row * J.nsp + j0);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                o[q] = make_float4(0.5f * (float)(s[2 * q] + s[2 * q + 1]),
                                   (float)(s[2 * q + 1] - s[2 * q]),
                                   0.5f * (float)(s[2 * q + 1] + s[2 * q + 2]),
                                   (float)(s[2 * q + 2] - s[2 * q + 1]));
        } else {
            const float sc = 1.0f / 32768.0f;
            unsigned h[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                if (PREC == kPrecF16)
                    h[q] = __half_as_ushort(__float2half_rn((float)s[q] * sc));
                else
                    h[q] = __bfloat16_as_ushort(__float2bfloat16_rn((float)s[q] * sc));
            }
            uint4 *o = reinterpret_cast<uint4 *>(reinterpret_cast<unsigned *>(J.pairs) +
                                                 (size_t)row * J.nsp + j0);
            o[0] = make_uint4(h[0] | (h[1] << 16), h[1] | (h[2] << 16), h[2] | (h[3] << 16),
                              h[3] | (h[4] << 16));
            o[1] = make_uint4(h[4] | (h[5] << 16), h[5] | (h[6] << 16), h[6] | (h[7] << 16),
                              h[7] | (h[8] << 16));
        }
    }
}

// ------------------------------------------------------------- beamform --

// Shared memory of one CTA: barriers + window starts, then per stage the
// tile's per-(channel, column) tables and the channels' record windows.
struct SmemHeader {
    uint64_t full[2];
    int w0[2][kMaxGroup];
};
constexpr int kHeaderBytes = 256;
static_assert(sizeof(SmemHeader) <= kHeaderBytes, "header");
constexpr int kVrBytes = kMaxGroup * kTileCols * 8;  // int2 valid rows, one stage
constexpr int kD2Bytes = kMaxGroup * kTileCols * 4;  // float dx^2, one stage
constexpr int kDataOffset = kHeaderBytes + 2 * kVrBytes + 2 * kD2Bytes;

template <int PREC>
struct PairIO;

template <>
struct PairIO<kPrecF32> {
    static constexpr int kBytes = 8;
    __device__ static __forceinline__ float interp(const unsigned char *win, unsigned idx, float al)
    {
        const float2 p = reinterpret_cast<const float2 *>(win)[idx];
        return fmaf(al, p.y, p.x);
    }
};

template <>
struct PairIO<kPrecF16> {
    static constexpr int kBytes = 4;
    __device__ static __forceinline__ float interp(const unsigned char *win, unsigned idx, float al)
    {
        const __half2 h = reinterpret_cast<const __half2 *>(win)[idx];
        const float2 f = __half22float2(h);
        return fmaf(al + 0.5f, f.y - f.x, f.x);
    }
};

template <>
struct PairIO<kPrecBF16> {
    static constexpr int kBytes = 4;
    __device__ static __forceinline__ float interp(const unsigned char *win, unsigned idx, float al)
    {
        const unsigned w = reinterpret_cast<const unsigned *>(win)[idx];
        const float lo = __uint_as_float(w << 16), hi = __uint_as_float(w & 0xffff0000u);
        return fmaf(al + 0.5f, hi - lo, lo);
    }
};

template <int PREC, bool DMAS, bool CF, int ROWS>
__global__ void __launch_bounds__(kThreads, 2) beamform_kernel(const BfJob *__restrict__ jobs,
                                                               const int *__restrict__ tile_prefix,
                                                               int njobs, int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    SmemHeader &sh = *reinterpret_cast<SmemHeader *>(smem);
    int2 *vr_s = reinterpret_cast<int2 *>(smem + kHeaderBytes);                 // [2][G][32]
    float *d2_s = reinterpret_cast<float *>(smem + kHeaderBytes + 2 * kVrBytes);  // [2][G][32]
    unsigned char *data = smem + kDataOffset;
    constexpr int PB = PairIO<PREC>::kBytes;

    // ---- which frame and tile
    const int jb = find_job(tile_prefix, njobs, blockIdx.x);
    const BfJob *J = jobs + jb;
    const int nx = J->nx, nz = J->nz, na = J->na, ne = J->ne;
    const int wmax = J->wmax, box = J->box, G = J->group;
    const int *__restrict__ colK = J->colK;
    const float *__restrict__ colF = J->colF;
    const int *__restrict__ rowK = J->rowK;
    const float *__restrict__ rowF = J->rowF;
    const int *__restrict__ wtab = J->wtab;
    const CUtensorMap *rf_map = J->rf_map;
    const CUtensorMap *valid_map = J->valid_map;
    const CUtensorMap *dx2_map = J->dx2_map;

    const int tile = blockIdx.x - __ldg(tile_prefix + jb);
    const int ntiles = J->tiles_x * J->tiles_z;
    const int tx = tile % J->tiles_x, tz = tile / J->tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ix = tx * kTileCols + lane;
    const bool col_ok = ix < nx;
    const int ixc = min(ix, nx - 1);
    const int r_first = tz * kWarps * ROWS + warp * ROWS;  // this warp's rows
    const int r_last = r_first + ROWS - 1;

    if (threadIdx.x == 0) {
        mbar_init(&sh.full[0], 1);
        mbar_init(&sh.full[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const unsigned long long deadline = global_ns() + kWaitNs;

    const int ngroups = (ne + G - 1) / G;
    const int steps = na * ngroups;
    const unsigned meta_bytes = (unsigned)G * kTileCols * (8 + 4);

    // Producer (warp 0): window start of this lane's channel for a step.
    auto window_of = [&](int s) -> int {
        const int a = s / ngroups, g = s - a * ngroups;
        const int c = g * G + lane;
        if (s >= steps || lane >= G || c >= ne)
            return kNoWindow;
        return __ldg(wtab + ((size_t)a * ntiles + tile) * ne + c);
    };
    auto issue = [&](int s, int w0) {
        const int a = s / ngroups, g = s - a * ngroups, buf = s & 1;
        const int i0 = g * G;
        const bool mine = lane < G && i0 + lane < ne;
        if (mine)
            sh.w0[buf][lane] = w0;
        const unsigned bytes = (mine && w0 != kNoWindow) ? (unsigned)(wmax * PB) : 0u;
        unsigned total = bytes;
#pragma unroll
        for (int off = 16; off; off >>= 1)
            total += __shfl_xor_sync(0xffffffffu, total, off);
        if (lane == 0) {
            mbar_arrive_expect_tx(&sh.full[buf], total + meta_bytes);
            tma_2d(vr_s + (size_t)buf * G * kTileCols, valid_map, tx * kTileCols, a * ne + i0,
                   &sh.full[buf]);
            tma_2d(d2_s + (size_t)buf * G * kTileCols, dx2_map, tx * kTileCols, i0, &sh.full[buf]);
        }
        __syncwarp();
        if (bytes) {
            unsigned char *dst = data + ((size_t)buf * G + lane) * wmax * PB;
            const int row = a * ne + i0 + lane;
            for (int off = 0; off < wmax; off += box)
                tma_2d(dst + (size_t)off * PB, rf_map, w0 + off, row, &sh.full[buf]);
        }
    };

    // ---- per-pixel state: ROWS contiguous rows per thread, one column per lane
    int Kc[ROWS];
    float Z[ROWS], fp[ROWS];
    float S1[ROWS], T1[ROWS], T2[ROWS], Yd[ROWS], Su2[ROWS];
#pragma unroll
    for (int j = 0; j < ROWS; ++j) {
        const int izc = min(r_first + j, nz - 1);
        Z[j] = __ldg(J->rowZ + izc);
        S1[j] = T1[j] = T2[j] = Yd[j] = Su2[j] = 0.f;
        Kc[j] = 0;
        fp[j] = 0.f;
    }

    bool ok = true;
    int w0_next = 0;
    if (warp == 0) {
        const int w0_first = window_of(0);
        w0_next = window_of(1);
        if (steps > 0)
            issue(0, w0_first);
    }
#pragma unroll 1
    for (int s = 0; s < steps; ++s) {
        const int a = s / ngroups, g = s - a * ngroups, buf = s & 1;
        if (g == 0) {
            const int ck = __ldg(colK + a * nx + ixc);
            const float cf = __ldg(colF + a * nx + ixc);
#pragma unroll
            for (int j = 0; j < ROWS; ++j) {
                const int izc = min(r_first + j, nz - 1);
                Kc[j] = ck + __ldg(rowK + a * nz + izc) + kPadL - kRoundBits;
                fp[j] = cf + __ldg(rowF + a * nz + izc) - 0.5f;
                T1[j] = T2[j] = 0.f;
            }
        }
        __syncthreads();  // every warp is done with step s - 1: its stage is free
        if (warp == 0 && s + 1 < steps && ok) {
            issue(s + 1, w0_next);
            w0_next = window_of(s + 2);
        }
        if (ok)
            ok = mbar_wait(&sh.full[buf], (unsigned)((s >> 1) & 1), deadline, err);
        if (ok) {
            const int i0 = g * G, gs = min(G, ne - i0);
            const int2 *vrb = vr_s + (size_t)buf * G * kTileCols;
            const float *d2b = d2_s + (size_t)buf * G * kTileCols;
#pragma unroll 1
            for (int c = 0; c < gs; ++c) {
                const int w0 = sh.w0[buf][c];
                if (w0 == kNoWindow)
                    continue;  // no pixel of the tile counts this channel
                const int2 vr = vrb[c * kTileCols + lane];  // (-1, -1): no row counts
                const bool mine = vr.x <= r_last && vr.y >= r_first;
                if (!__any_sync(0xffffffffu, mine))
                    continue;
                const float d2 = d2b[c * kTileCols + lane];
                const unsigned char *win = data + ((size_t)buf * G + c) * wmax * PB;
                const unsigned span = (unsigned)(vr.y - vr.x);
#pragma unroll
                for (int j = 0; j < ROWS; ++j) {
                    const float x = rx_excess(d2, Z[j]) + fp[j];
                    const float m = x + kRoundMagic;
                    const float al = x - (m - kRoundMagic);  // in [-1/2, 1/2]
                    const unsigned idx =
                        min((unsigned)(__float_as_int(m) + Kc[j] - w0), (unsigned)(wmax - 1));
                    const float v = PairIO<PREC>::interp(win, idx, al);
                    if ((unsigned)(r_first + j - vr.x) <= span) {
                        S1[j] += v;
                        if (DMAS) {
                            const float av = fabsf(v);
                            T1[j] += copysignf(sqrt_approx(av), v);
                            T2[j] += av;
                        }
                        if (CF)
                            Su2[j] = fmaf(v, v, Su2[j]);
                    }
                }
            }
        }
        if (DMAS && g == ngroups - 1) {
#pragma unroll
            for (int j = 0; j < ROWS; ++j)
                Yd[j] = fmaf(0.5f * T1[j], T1[j], fmaf(-0.5f, T2[j], Yd[j]));
        }
    }

    if (!ok || !col_ok)
        return;
    const int modes = J->modes;
    const float scale = J->out_scale;
    const size_t plane = (size_t)nx * nz;
    float *__restrict__ y = J->y;
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
            y[(size_t)(slot++) * plane + o] = den > 0.f ? (S1[j] * S1[j] / den) * S1[j] * scale : 0.f;
        }
    }
}

// ------------------------------------------------------------- envelope --

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Radix-2 Stockham FFTs of `cols` columns of length m (power of two) stored
// back to back in x; twiddles exp(-2 pi i k / m) in shared memory.  The result
// ends in the returned buffer.  inverse: +i exponent, no scaling.
__device__ float2 *fft_cols(float2 *x, float2 *y, int m, int lgm, int cols, const float2 *tw,
                            bool inverse)
{
    const int half = m >> 1;
    const int total = cols * half;
    for (int ns = 1, lg = 0; ns < m; ns <<= 1, ++lg) {
        const int stride_sh = lgm - 1 - lg;  // log2(m / (2 ns))
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int c = t >> (lgm - 1), j = t & (half - 1);
            const float2 *xc = x + (size_t)c * m;
            float2 *yc = y + (size_t)c * m;
            const float2 v0 = xc[j], v1 = xc[j + half];
            const int r = j & (ns - 1);
            float2 w = tw[r << stride_sh];
            if (inverse)
                w.y = -w.y;
            const float2 t2 = cmul(v1, w);
            const int d = ((j - r) << 1) + r;
            yc[d] = make_float2(v0.x + t2.x, v0.y + t2.y);
            yc[d + ns] = make_float2(v0.x - t2.x, v0.y - t2.y);
        }
        __syncthreads();
        float2 *tmp = x;
        x = y;
        y = tmp;
    }
    return x;
}

__device__ __forceinline__ float spectral_weight(int k, int L, int band, int kb_lo, int kb_hi)
{
    float h = (k == 0) ? 1.f : (2 * k < L) ? 2.f : (2 * k == L) ? 1.f : 0.f;
    if (band && (k < kb_lo || k > kb_hi))
        h = 0.f;
    return h;
}

__global__ void __launch_bounds__(256) envelope_kernel(const EnvJob *__restrict__ jobs,
                                                       const int *__restrict__ blk_prefix,
                                                       int njobs)
{
    extern __shared__ __align__(16) float2 sbuf[];
    __shared__ float red[32];
    const int jb = find_job(blk_prefix, njobs, blockIdx.x);
    const EnvJob J = jobs[jb];
    const int C = J.cols_per_block;
    const int c0 = (blockIdx.x - __ldg(blk_prefix + jb)) * C;
    const int cols = min(C, J.nx - c0);
    const int nz = J.nz, m = J.fft_m;
    const int lgm = 31 - __clz(m);
    float2 *A = sbuf, *B = sbuf + (size_t)C * m, *tw = sbuf + (size_t)2 * C * m;
    for (int k = threadIdx.x; k < (m >> 1); k += blockDim.x)
        tw[k] = __ldg(J.tw + k);
    float lmax = 0.f;

    if (!J.bluestein) {
        for (int t = threadIdx.x; t < cols * m; t += blockDim.x) {
            const int c = t / m, n = t - c * m;
            A[t] = make_float2(__ldg(J.y + (size_t)(c0 + c) * nz + n), 0.f);
        }
        __syncthreads();
        float2 *X = fft_cols(A, B, m, lgm, cols, tw, false);
        float2 *O = X == A ? B : A;
        for (int t = threadIdx.x; t < cols * m; t += blockDim.x) {
            const int k = t & (m - 1);
            const float h = spectral_weight(k, nz, J.band, J.kb_lo, J.kb_hi);
            X[t] = make_float2(X[t].x * h, X[t].y * h);
        }
        __syncthreads();
        float2 *R = fft_cols(X, O, m, lgm, cols, tw, true);
        const float inv = 1.f / (float)m;
        for (int t = threadIdx.x; t < cols * m; t += blockDim.x) {
            const int c = t >> lgm, n = t & (m - 1);
            const float e = hypotf(R[t].x, R[t].y) * inv;
            J.env[(size_t)(c0 + c) * nz + n] = e;
            lmax = fmaxf(lmax, e);
        }
    } else {
        // one column per block (C == 1)
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
        float2 *X = fft_cols(A, B, m, lgm, 1, tw, false);
        for (int k = threadIdx.x; k < m; k += blockDim.x)
            X[k] = cmul(X[k], __ldg(bh + k));
        __syncthreads();
        float2 *O = X == A ? B : A;
        float2 *Cb = fft_cols(X, O, m, lgm, 1, tw, true);
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
        float2 *E = fft_cols(D, Cb, m, lgm, 1, tw, false);
        for (int k = threadIdx.x; k < m; k += blockDim.x)
            E[k] = cmul(E[k], __ldg(bh + k));
        __syncthreads();
        float2 *F = fft_cols(E, E == A ? B : A, m, lgm, 1, tw, true);
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

// ------------------------------------------------------------------ log --

constexpr int kLogPerBlock = 1024;

__global__ void __launch_bounds__(256) log_kernel(const LogJob *__restrict__ jobs,
                                                  const int *__restrict__ blk_prefix, int njobs,
                                                  float dr)
{
    const int jb = find_job(blk_prefix, njobs, blockIdx.x);
    const LogJob J = jobs[jb];
    const size_t base = (size_t)(blockIdx.x - __ldg(blk_prefix + jb)) * kLogPerBlock;
    const float peak = __uint_as_float(__ldg(J.maxbits));
    for (int t = threadIdx.x; t < kLogPerBlock; t += blockDim.x) {
        const size_t p = base + t;
        if (p >= (size_t)J.n)
            break;
        const float e = __ldg(J.env + p);
        float d = -dr;
        if (e > 0.f && peak > 0.f)
            d = fminf(fmaxf(20.f * log10f(e / peak), -dr), 0.f);
        J.out[p] = d;
    }
}

template <int PREC, bool DMAS, bool CF, int ROWS>
cudaError_t launch_bf_t(const BfJob *jobs, const int *prefix, int njobs, int tiles, size_t smem,
                        int *err, cudaStream_t st)
{
    auto k = beamform_kernel<PREC, DMAS, CF, ROWS>;
    static size_t configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        configured = smem;
    }
    k<<<tiles, kThreads, smem, st>>>(jobs, prefix, njobs, err);
    return cudaGetLastError();
}

template <int PREC, int ROWS>
cudaError_t launch_bf_pr(const BfJob *jobs, const int *prefix, int njobs, int tiles, size_t smem,
                         int dmas, int cf, int *err, cudaStream_t st)
{
    if (dmas && cf)
        return launch_bf_t<PREC, true, true, ROWS>(jobs, prefix, njobs, tiles, smem, err, st);
    if (dmas)
        return launch_bf_t<PREC, true, false, ROWS>(jobs, prefix, njobs, tiles, smem, err, st);
    if (cf)
        return launch_bf_t<PREC, false, true, ROWS>(jobs, prefix, njobs, tiles, smem, err, st);
    return launch_bf_t<PREC, false, false, ROWS>(jobs, prefix, njobs, tiles, smem, err, st);
}

template <int PREC>
cudaError_t launch_bf_p(const BfJob *jobs, const int *prefix, int njobs, int tiles, size_t smem,
                        int dmas, int cf, int rows, int *err, cudaStream_t st)
{
    if (rows == 4)
        return launch_bf_pr<PREC, 4>(jobs, prefix, njobs, tiles, smem, dmas, cf, err, st);
    return launch_bf_pr<PREC, 8>(jobs, prefix, njobs, tiles, smem, dmas, cf, err, st);
}

}  // namespace

size_t beamform_smem_bytes(int wmax, int group, int prec)
{
    return (size_t)kDataOffset + 2u * (size_t)group * (size_t)wmax * (size_t)pair_bytes(prec);
}

int envelope_cols_per_block(int fft_m) { return fft_m >= 2048 ? 1 : 2048 / fft_m; }

size_t envelope_smem_bytes(int fft_m)
{
    const int c = envelope_cols_per_block(fft_m);
    return (2u * (size_t)c * fft_m + (size_t)(fft_m / 2 > 0 ? fft_m / 2 : 1)) * sizeof(float2);
}

cudaError_t launch_plan(const PlanJob &job, int *err_dev, cudaStream_t stream)
{
    dim3 grid(job.tiles_x * job.tiles_z, job.na);
    plan_kernel<<<grid, 128, 0, stream>>>(job, err_dev);
    return cudaGetLastError();
}

cudaError_t launch_ingest(const IngestJob *jobs_dev, const int *row_prefix_dev, int njobs,
                          int total_rows, int prec, cudaStream_t stream)
{
    if (njobs <= 0 || total_rows <= 0)
        return cudaSuccess;
    if (prec == kPrecF32)
        ingest_kernel<kPrecF32><<<total_rows, 256, 0, stream>>>(jobs_dev, row_prefix_dev, njobs);
    else if (prec == kPrecF16)
        ingest_kernel<kPrecF16><<<total_rows, 256, 0, stream>>>(jobs_dev, row_prefix_dev, njobs);
    else
        ingest_kernel<kPrecBF16><<<total_rows, 256, 0, stream>>>(jobs_dev, row_prefix_dev, njobs);
    return cudaGetLastError();
}

cudaError_t launch_beamform(const BfJob *jobs_dev, const int *tile_prefix_dev, int njobs,
                            int total_tiles, size_t smem_bytes, int prec, int variant, int rows,
                            int *err_dev, cudaStream_t stream)
{
    if (njobs <= 0 || total_tiles <= 0)
        return cudaSuccess;
    const int dmas = (variant & BF_DMAS) ? 1 : 0, cf = (variant & BF_CF) ? 1 : 0;
    if (prec == kPrecF32)
        return launch_bf_p<kPrecF32>(jobs_dev, tile_prefix_dev, njobs, total_tiles, smem_bytes,
                                     dmas, cf, rows, err_dev, stream);
    if (prec == kPrecF16)
        return launch_bf_p<kPrecF16>(jobs_dev, tile_prefix_dev, njobs, total_tiles, smem_bytes,
                                     dmas, cf, rows, err_dev, stream);
    return launch_bf_p<kPrecBF16>(jobs_dev, tile_prefix_dev, njobs, total_tiles, smem_bytes, dmas,
                                  cf, rows, err_dev, stream);
}

cudaError_t launch_envelope(const EnvJob *jobs_dev, const int *blk_prefix_dev, int njobs,
                            int total_blocks, size_t smem, cudaStream_t stream)
{
    if (njobs <= 0 || total_blocks <= 0)
        return cudaSuccess;
    static size_t configured = 0;
    if (smem > 48u * 1024u && smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(envelope_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        configured = smem;
    }
    envelope_kernel<<<total_blocks, 256, smem, stream>>>(jobs_dev, blk_prefix_dev, njobs);
    return cudaGetLastError();
}

cudaError_t launch_log(const LogJob *jobs_dev, const int *blk_prefix_dev, int njobs,
                       int total_blocks, float dynamic_range_db, cudaStream_t stream)
{
    if (njobs <= 0 || total_blocks <= 0)
        return cudaSuccess;
    log_kernel<<<total_blocks, 256, 0, stream>>>(jobs_dev, blk_prefix_dev, njobs, dynamic_range_db);
    return cudaGetLastError();
}

int log_blocks(long long pixels) { return (int)((pixels + kLogPerBlock - 1) / kLogPerBlock); }

}  // namespace bfi

// GB300 (sm_103a) kernels of the plane-wave beamformer.
//
//   ingest_kernel    int16 channel records -> sample pairs staged for the
//                    beamformer (FP32 (mid, diff) pairs, or raw FP16 / BF16 pairs)
//   beamform_kernel  per CTA an 8-column x 64-row pixel tile; per angle and
//                    channel group the needed window of every channel's record
//                    is copied into shared memory by the tensor memory
//                    accelerator (cp.async.bulk.tensor, double buffered on
//                    mbarriers), delays are formed in registers, samples are
//                    interpolated linearly and combined (DAS, signed-sqrt DMAS,
//                    coherence factor) and compounded over angles (Eq. (1),
//                    Sec. II-B)
//   envelope_kernel  per image column the analytic signal along depth via a
//                    shared-memory radix-2 Stockham FFT (Bluestein for other
//                    lengths), one-sided mask and optional [f0, 3 f0] band-pass,
//                    magnitude, and the frame maximum
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

// One 2-D tensor-map box (box pairs of one channel row) into shared memory.
__device__ __forceinline__ void tma_row(void *dst, const CUtensorMap *map, int x, int row,
                                        uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(row), "r"(smem_u32(bar))
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
__device__ __forceinline__ float rx_excess(float dx2, float z, float z2)
{
    float s = fmaxf(dx2 + z2, 1e-30f);
    float r = s * rsqrt_approx(s);
    return dx2 * rcp_approx(r + z);
}

// ---------------------------------------------------------------- ingest --

template <int PREC>
__global__ void __launch_bounds__(256) ingest_kernel(const int16_t *__restrict__ rf,
                                                     void *__restrict__ pairs, int ns, int nsp)
{
    const int row = blockIdx.x;
    const int16_t *u = rf + (size_t)row * ns;
    for (int j = threadIdx.x; j < nsp; j += blockDim.x) {
        const int k = j - kPadL;
        const int a = (k >= 0 && k < ns) ? (int)__ldg(u + k) : 0;
        const int b = (k + 1 >= 0 && k + 1 < ns) ? (int)__ldg(u + k + 1) : 0;
        const size_t o = (size_t)row * nsp + j;
        if (PREC == kPrecF32) {
            // mid point and difference: v = mid + (alpha - 1/2) * diff (exact for int16)
            reinterpret_cast<float2 *>(pairs)[o] = make_float2(0.5f * (float)(a + b), (float)(b - a));
        } else if (PREC == kPrecF16) {
            const float s = 1.0f / 32768.0f;
            reinterpret_cast<__half2 *>(pairs)[o] =
                __halves2half2(__float2half_rn((float)a * s), __float2half_rn((float)b * s));
        } else {
            const float s = 1.0f / 32768.0f;
            reinterpret_cast<__nv_bfloat162 *>(pairs)[o] =
                __halves2bfloat162(__float2bfloat16_rn((float)a * s), __float2bfloat16_rn((float)b * s));
        }
    }
}

// ------------------------------------------------------------- beamform --

struct SmemHeader {
    uint64_t full[2];
    int w0[2][kMaxGroup];
    int2 vr[2][kMaxGroup][kTileCols];
    float dx2[2][kMaxGroup][kTileCols];
};
constexpr int kHeaderBytes = (int)((sizeof(SmemHeader) + 127) / 128 * 128);

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

template <int PREC, bool DMAS, bool CF>
__global__ void __launch_bounds__(kThreads) beamform_kernel(const BfJob *__restrict__ jobs,
                                                            const int *__restrict__ tile_prefix,
                                                            int njobs, int *__restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    SmemHeader &sh = *reinterpret_cast<SmemHeader *>(smem);
    unsigned char *data = smem + kHeaderBytes;
    constexpr int PB = PairIO<PREC>::kBytes;
    constexpr int kAlign = 16 / PB;

    // ---- which frame and tile
    const int bid = blockIdx.x;
    int jlo = 0, jhi = njobs - 1;
    while (jlo < jhi) {
        const int mid = (jlo + jhi + 1) >> 1;
        if (__ldg(tile_prefix + mid) <= bid)
            jlo = mid;
        else
            jhi = mid - 1;
    }
    const BfJob *J = jobs + jlo;
    const int nx = J->nx, nz = J->nz, na = J->na, ne = J->ne;
    const int wmax = J->wmax, box = J->box, G = J->group;
    const int *__restrict__ colK = J->colK;
    const float *__restrict__ colF = J->colF;
    const int *__restrict__ rowK = J->rowK;
    const float *__restrict__ rowF = J->rowF;
    const float *__restrict__ rowZ = J->rowZ;
    const float *__restrict__ rowZ2 = J->rowZ2;
    const float *__restrict__ colDX2 = J->colDX2;
    const int2 *__restrict__ valid = J->valid;
    const CUtensorMap *map = J->rf_map;

    const int t = bid - __ldg(tile_prefix + jlo);
    const int tx = t % J->tiles_x, tz = t / J->tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ix = tx * kTileCols + warp;
    const bool col_ok = ix < nx;
    const int ixc = min(ix, nx - 1);
    const int tz0 = tz * kTileRows;
    const int tz_last = min(tz0 + kTileRows - 1, nz - 1);

    if (threadIdx.x == 0) {
        mbar_init(&sh.full[0], 1);
        mbar_init(&sh.full[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const unsigned long long deadline = global_ns() + kWaitNs;

    const int ngroups = (ne + G - 1) / G;
    const int steps = na * ngroups;

    // Producer (warp 0): windows and TMA copies of one (angle, channel group) step.
    auto issue = [&](int s) {
        const int a = s / ngroups, g = s - a * ngroups, buf = s & 1;
        const int i0 = g * G, gs = min(G, ne - i0);
        int bytes = 0;
        int w0 = 0;
        if (lane < gs) {
            const int i = i0 + lane;
            int kmin = INT_MAX, kmax = INT_MIN;
#pragma unroll 1
            for (int w = 0; w < kTileCols; ++w) {
                const int ixw = tx * kTileCols + w;
                int2 vr = make_int2(1, 0);
                float d2 = 0.f;
                if (ixw < nx) {
                    vr = __ldg(valid + ((size_t)a * nx + ixw) * ne + i);
                    d2 = __ldg(colDX2 + (size_t)ixw * ne + i);
                    const int r0 = max(vr.x, tz0), r1 = min(vr.y, tz_last);
                    if (r0 <= r1) {
                        const int kb = __ldg(colK + a * nx + ixw);
                        const float fb = __ldg(colF + a * nx + ixw);
                        const int k0 = kb + __ldg(rowK + a * nz + r0) +
                                       __float2int_rd(fb + __ldg(rowF + a * nz + r0) +
                                                      rx_excess(d2, __ldg(rowZ + r0), __ldg(rowZ2 + r0)));
                        const int k1 = kb + __ldg(rowK + a * nz + r1) +
                                       __float2int_rd(fb + __ldg(rowF + a * nz + r1) +
                                                      rx_excess(d2, __ldg(rowZ + r1), __ldg(rowZ2 + r1)));
                        kmin = min(kmin, min(k0, k1));
                        kmax = max(kmax, max(k0, k1));
                    }
                }
                sh.vr[buf][lane][w] = vr;
                sh.dx2[buf][lane][w] = d2;
            }
            if (kmin <= kmax) {
                w0 = (kmin + kPadL - 2) & ~(kAlign - 1);
                if (kmax + kPadL + 2 - w0 + 1 > wmax)
                    atomicOr(err, kErrWindow);
                bytes = wmax * PB;
            }
            sh.w0[buf][lane] = w0;
        }
        int total = bytes;
#pragma unroll
        for (int off = 16; off; off >>= 1)
            total += __shfl_xor_sync(0xffffffffu, total, off);
        if (lane == 0)
            mbar_arrive_expect_tx(&sh.full[buf], (unsigned)total);
        __syncwarp();
        if (bytes) {
            unsigned char *dst = data + ((size_t)buf * G + lane) * wmax * PB;
            const int row = a * ne + i0 + lane;
            for (int off = 0; off < wmax; off += box)
                tma_row(dst + (size_t)off * PB, map, w0 + off, row, &sh.full[buf]);
        }
    };

    // ---- per-pixel state: two rows per lane, one column per warp
    int iz[kRowsPerLane], Kc[kRowsPerLane];
    float Z[kRowsPerLane], Z2[kRowsPerLane], fp[kRowsPerLane];
    float S1[kRowsPerLane], T1[kRowsPerLane], T2[kRowsPerLane], Yd[kRowsPerLane], Su2[kRowsPerLane];
#pragma unroll
    for (int j = 0; j < kRowsPerLane; ++j) {
        iz[j] = tz0 + lane + 32 * j;
        const int izc = min(iz[j], nz - 1);
        Z[j] = __ldg(rowZ + izc);
        Z2[j] = __ldg(rowZ2 + izc);
        S1[j] = T1[j] = T2[j] = Yd[j] = Su2[j] = 0.f;
        Kc[j] = 0;
        fp[j] = 0.f;
    }

    bool ok = true;
    if (warp == 0 && steps > 0)
        issue(0);
#pragma unroll 1
    for (int s = 0; s < steps; ++s) {
        const int a = s / ngroups, g = s - a * ngroups, buf = s & 1;
        if (g == 0) {
            const int ck = __ldg(colK + a * nx + ixc);
            const float cf = __ldg(colF + a * nx + ixc);
#pragma unroll
            for (int j = 0; j < kRowsPerLane; ++j) {
                const int izc = min(iz[j], nz - 1);
                Kc[j] = ck + __ldg(rowK + a * nz + izc) + kPadL - kRoundBits;
                fp[j] = cf + __ldg(rowF + a * nz + izc) - 0.5f;
                T1[j] = T2[j] = 0.f;
            }
        }
        __syncthreads();  // every warp is done with step s - 1: its buffer is free
        if (warp == 0 && s + 1 < steps && ok)
            issue(s + 1);
        if (ok)
            ok = mbar_wait(&sh.full[buf], (unsigned)((s >> 1) & 1), deadline, err);
        if (ok && col_ok) {
            const int i0 = g * G, gs = min(G, ne - i0);
#pragma unroll 1
            for (int c = 0; c < gs; ++c) {
                const int2 vr = sh.vr[buf][c][warp];
                if (vr.y < tz0 || vr.x > tz_last || vr.x > vr.y)
                    continue;  // no row of this warp counts this channel
                const float d2 = sh.dx2[buf][c][warp];
                const int w0 = sh.w0[buf][c];
                const unsigned char *win = data + ((size_t)buf * G + c) * wmax * PB;
#pragma unroll
                for (int j = 0; j < kRowsPerLane; ++j) {
                    const float x = rx_excess(d2, Z[j], Z2[j]) + fp[j];
                    const float m = x + kRoundMagic;
                    const float al = x - (m - kRoundMagic);  // in [-1/2, 1/2]
                    const unsigned idx =
                        min((unsigned)(__float_as_int(m) + Kc[j] - w0), (unsigned)(wmax - 1));
                    const float v = PairIO<PREC>::interp(win, idx, al);
                    if ((unsigned)(iz[j] - vr.x) <= (unsigned)(vr.y - vr.x)) {
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
            for (int j = 0; j < kRowsPerLane; ++j)
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
    for (int j = 0; j < kRowsPerLane; ++j) {
        if (iz[j] >= nz)
            continue;
        const size_t o = (size_t)ix * nz + iz[j];
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

// Radix-2 Stockham FFT of length m (power of two) over shared memory; the
// result ends in the returned buffer.  inverse: +i exponent, no scaling.
__device__ float2 *fft_stockham(float2 *x, float2 *y, int m, const float2 *__restrict__ tw,
                                bool inverse)
{
    const int half = m >> 1;
    for (int ns = 1; ns < m; ns <<= 1) {
        const int stride = half / ns;  // m / (2 ns)
        for (int j = threadIdx.x; j < half; j += blockDim.x) {
            const float2 v0 = x[j], v1 = x[j + half];
            const int r = j & (ns - 1);
            float2 w = __ldg(tw + r * stride);
            if (inverse)
                w.y = -w.y;
            const float2 t = cmul(v1, w);
            const int d = ((j - r) << 1) + r;
            y[d] = make_float2(v0.x + t.x, v0.y + t.y);
            y[d + ns] = make_float2(v0.x - t.x, v0.y - t.y);
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
                                                       const int *__restrict__ col_prefix,
                                                       int njobs)
{
    extern __shared__ __align__(16) float2 sbuf[];
    __shared__ float red[32];
    const int bid = blockIdx.x;
    int jlo = 0, jhi = njobs - 1;
    while (jlo < jhi) {
        const int mid = (jlo + jhi + 1) >> 1;
        if (__ldg(col_prefix + mid) <= bid)
            jlo = mid;
        else
            jhi = mid - 1;
    }
    const EnvJob J = jobs[jlo];
    const int ix = bid - __ldg(col_prefix + jlo);
    const int nz = J.nz, m = J.fft_m;
    const float *__restrict__ y = J.y + (size_t)ix * nz;
    float *__restrict__ env = J.env + (size_t)ix * nz;
    float2 *A = sbuf, *B = sbuf + m;
    const int band = J.band;
    float lmax = 0.f;

    if (!J.bluestein) {
        for (int n = threadIdx.x; n < m; n += blockDim.x)
            A[n] = make_float2(__ldg(y + n), 0.f);
        __syncthreads();
        float2 *X = fft_stockham(A, B, m, J.tw, false);
        float2 *O = X == A ? B : A;
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const float h = spectral_weight(k, nz, band, J.kb_lo, J.kb_hi);
            X[k] = make_float2(X[k].x * h, X[k].y * h);
        }
        __syncthreads();
        float2 *R = fft_stockham(X, O, m, J.tw, true);
        const float inv = 1.f / (float)m;
        for (int n = threadIdx.x; n < nz; n += blockDim.x) {
            const float e = hypotf(R[n].x, R[n].y) * inv;
            env[n] = e;
            lmax = fmaxf(lmax, e);
        }
    } else {
        const float2 *__restrict__ w = J.chirp;
        const float2 *__restrict__ bh = J.bhat;
        const float inv_m = 1.f / (float)m;
        // forward DFT of the column: X_k = conj(w_k) * (a (*) w)_k, a_n = y_n conj(w_n)
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
        float2 *X = fft_stockham(A, B, m, J.tw, false);
        for (int k = threadIdx.x; k < m; k += blockDim.x)
            X[k] = cmul(X[k], __ldg(bh + k));
        __syncthreads();
        float2 *O = X == A ? B : A;
        float2 *C = fft_stockham(X, O, m, J.tw, true);
        float2 *D = C == A ? B : A;
        // masked spectrum, conjugated and pre-multiplied by conj(w) for the second pass:
        // the inverse DFT of S is conj(DFT(conj S)) / nz
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            float2 v = make_float2(0.f, 0.f);
            if (k < nz) {
                const float2 c = __ldg(w + k);
                const float2 cc = make_float2(c.x, -c.y);
                float2 xk = cmul(make_float2(C[k].x * inv_m, C[k].y * inv_m), cc);
                const float h = spectral_weight(k, nz, band, J.kb_lo, J.kb_hi);
                xk = make_float2(xk.x * h, -xk.y * h);  // conj of the masked bin
                v = cmul(xk, cc);
            }
            D[k] = v;
        }
        __syncthreads();
        float2 *E = fft_stockham(D, C, m, J.tw, false);
        for (int k = threadIdx.x; k < m; k += blockDim.x)
            E[k] = cmul(E[k], __ldg(bh + k));
        __syncthreads();
        float2 *F = fft_stockham(E, E == A ? B : A, m, J.tw, true);
        const float inv = inv_m / (float)nz;
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
    const int bid = blockIdx.x;
    int jlo = 0, jhi = njobs - 1;
    while (jlo < jhi) {
        const int mid = (jlo + jhi + 1) >> 1;
        if (__ldg(blk_prefix + mid) <= bid)
            jlo = mid;
        else
            jhi = mid - 1;
    }
    const LogJob J = jobs[jlo];
    const size_t base = (size_t)(bid - __ldg(blk_prefix + jlo)) * kLogPerBlock;
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

template <int PREC, bool DMAS, bool CF>
cudaError_t launch_bf_t(const BfJob *jobs, const int *prefix, int njobs, int tiles, size_t smem,
                        int *err, cudaStream_t st)
{
    auto k = beamform_kernel<PREC, DMAS, CF>;
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

template <int PREC>
cudaError_t launch_bf_p(const BfJob *jobs, const int *prefix, int njobs, int tiles, size_t smem,
                        int dmas, int cf, int *err, cudaStream_t st)
{
    if (dmas && cf)
        return launch_bf_t<PREC, true, true>(jobs, prefix, njobs, tiles, smem, err, st);
    if (dmas)
        return launch_bf_t<PREC, true, false>(jobs, prefix, njobs, tiles, smem, err, st);
    if (cf)
        return launch_bf_t<PREC, false, true>(jobs, prefix, njobs, tiles, smem, err, st);
    return launch_bf_t<PREC, false, false>(jobs, prefix, njobs, tiles, smem, err, st);
}

}  // namespace

size_t beamform_smem_bytes(int wmax, int group, int prec)
{
    return (size_t)kHeaderBytes + 2u * (size_t)group * (size_t)wmax * (size_t)pair_bytes(prec);
}

cudaError_t launch_ingest(const int16_t *rf, void *pairs, int rows, int ns, int nsp, int prec,
                          cudaStream_t stream)
{
    if (rows <= 0)
        return cudaSuccess;
    if (prec == kPrecF32)
        ingest_kernel<kPrecF32><<<rows, 256, 0, stream>>>(rf, pairs, ns, nsp);
    else if (prec == kPrecF16)
        ingest_kernel<kPrecF16><<<rows, 256, 0, stream>>>(rf, pairs, ns, nsp);
    else
        ingest_kernel<kPrecBF16><<<rows, 256, 0, stream>>>(rf, pairs, ns, nsp);
    return cudaGetLastError();
}

cudaError_t launch_beamform(const BfJob *jobs_dev, const int *tile_prefix_dev, int njobs,
                            int total_tiles, size_t smem_bytes, int prec, int variant,
                            int *err_dev, cudaStream_t stream)
{
    if (njobs <= 0 || total_tiles <= 0)
        return cudaSuccess;
    const int dmas = (variant & BF_DMAS) ? 1 : 0, cf = (variant & BF_CF) ? 1 : 0;
    if (prec == kPrecF32)
        return launch_bf_p<kPrecF32>(jobs_dev, tile_prefix_dev, njobs, total_tiles, smem_bytes,
                                     dmas, cf, err_dev, stream);
    if (prec == kPrecF16)
        return launch_bf_p<kPrecF16>(jobs_dev, tile_prefix_dev, njobs, total_tiles, smem_bytes,
                                     dmas, cf, err_dev, stream);
    return launch_bf_p<kPrecBF16>(jobs_dev, tile_prefix_dev, njobs, total_tiles, smem_bytes, dmas,
                                  cf, err_dev, stream);
}

cudaError_t launch_envelope(const EnvJob *jobs_dev, const int *col_prefix_dev, int njobs,
                            int total_cols, int max_fft_m, cudaStream_t stream)
{
    if (njobs <= 0 || total_cols <= 0)
        return cudaSuccess;
    const size_t smem = 2u * (size_t)max_fft_m * sizeof(float2);
    static size_t configured = 0;
    if (smem > 48u * 1024u && smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(envelope_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        configured = smem;
    }
    envelope_kernel<<<total_cols, 256, smem, stream>>>(jobs_dev, col_prefix_dev, njobs);
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

// Allocation-free envelope and log-compression entry point.
//
// Some callers cannot allocate device memory once they are running: a scanner's
// real-time acquisition loop that must not call cudaMalloc after start-up (it
// can block and synchronise the device), a host application whose device
// memory is owned by its own allocator or a fixed pool, or code running where
// the allocator must not be entered at all.  bf_logdb_static serves them: it
// takes a beamformed image the caller already holds on the device and writes
// its -70 dB log-compressed envelope into the caller's output, and its only
// scratch (the envelope image and the frame maximum) is a fixed array compiled
// into this library.  Every GPU that loads the library holds that array
// (kStaticPixels floats, 4 MiB) until the process exits.
//
// The computation is the one of the BF_OUT_LOGDB stage of bf_beamform: the
// analytic-signal magnitude along depth, optionally through the [f0, 3 f0]
// band-pass of the DMAS image, then 20 log10(env / max) clipped to -70 dB.
// Twiddle factors are computed on the device, so depths must be powers of two.
#include <algorithm>
#include <mutex>

#include "../../include/bf.h"
#include "bf_engine.h"
#include "bf_fft.cuh"
#include "bf_internal.h"

namespace bfi {
namespace {

constexpr size_t kStaticPixels = (size_t)1 << 20;  // largest nx * nz accepted
constexpr int kMaxDevices = 64;

// [0, kStaticPixels): envelope image; [kStaticPixels]: frame maximum (float bits).
__device__ __align__(256) float g_static_scratch[kStaticPixels + 64];

__global__ void __launch_bounds__(256) static_envelope_kernel(const float *__restrict__ y, int nx,
                                                              int nz, int band, int kb_lo,
                                                              int kb_hi, float *__restrict__ env,
                                                              unsigned *__restrict__ maxbits)
{
    extern __shared__ __align__(16) float2 sbuf[];
    __shared__ float red[32];
    const int m = nz, lgm = 31 - __clz(m);
    const int C = m >= 2048 ? 1 : 2048 / m;  // complex columns: pairs of image columns
    const int c0 = blockIdx.x * 2 * C;
    float2 *Zb = sbuf, *Pb = sbuf + (size_t)C * m, *Qb = sbuf + (size_t)2 * C * m;
    float2 *tw = sbuf + (size_t)3 * C * m;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        float sn, cs;
        sincospif(-2.0f * (float)k / (float)m, &sn, &cs);  // exp(-2 pi i k / m)
        tw[k] = make_float2(cs, sn);
    }
    for (int t = threadIdx.x; t < C * m; t += blockDim.x) {
        const int c = t >> lgm, n = t & (m - 1);
        const int ca = c0 + 2 * c, cb = ca + 1;
        Zb[t] = make_float2(ca < nx ? __ldg(y + (size_t)ca * nz + n) : 0.f,
                            cb < nx ? __ldg(y + (size_t)cb * nz + n) : 0.f);
    }
    __syncthreads();
    float2 *S = fft_r4(Zb, Pb, m, lgm, C, tw, false);
    float2 *F1 = S == Zb ? Pb : Zb;
    const float inv = 1.f / (float)m;
    float lmax = 0.f;
    // spectral multipliers: symmetric band-pass (DMAS) and the Hilbert -i sgn(k)
    for (int t = threadIdx.x; t < C * m; t += blockDim.x) {
        const int k = t & (m - 1);
        const int kk = 2 * k <= m ? k : m - k;
        const float bp = (!band || (kk >= kb_lo && kk <= kb_hi)) ? 1.f : 0.f;
        const float sg = (k == 0 || 2 * k == m) ? 0.f : (2 * k < m ? 1.f : -1.f);
        const float2 r = make_float2(S[t].x * bp, S[t].y * bp);
        S[t] = r;
        Qb[t] = make_float2(r.y * sg, -r.x * sg);
    }
    __syncthreads();
    float2 *R = fft_r4(S, F1, m, lgm, C, tw, true);
    float2 *F2 = R == S ? F1 : S;
    const float2 *Hh = fft_r4(Qb, F2, m, lgm, C, tw, true);
    for (int t = threadIdx.x; t < C * m; t += blockDim.x) {
        const int c = t >> lgm, n = t & (m - 1);
        const int ca = c0 + 2 * c, cb = ca + 1;
        if (ca < nx) {
            const float e = hypotf(R[t].x, Hh[t].x) * inv;
            env[(size_t)ca * nz + n] = e;
            lmax = fmaxf(lmax, e);
        }
        if (cb < nx) {
            const float e = hypotf(R[t].y, Hh[t].y) * inv;
            env[(size_t)cb * nz + n] = e;
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
            atomicMax(maxbits, __float_as_uint(v));
    }
}

__global__ void __launch_bounds__(256) static_log_kernel(const float *__restrict__ env, size_t n,
                                                         const unsigned *__restrict__ maxbits,
                                                         float *__restrict__ out, float dr)
{
    const float peak = __uint_as_float(*maxbits);
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (size_t)gridDim.x * blockDim.x) {
        const float e = env[p];
        float d = -dr;
        if (e > 0.f && peak > 0.f)
            d = fminf(fmaxf(20.f * log10f(e / peak), -dr), 0.f);
        out[p] = d;
    }
}

std::mutex g_static_mu;
float *g_static_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the array's name is only a host-side stand-in in host code).
int static_scratch(float **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(BF_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaGetSymbolAddress (static scratch)");
        g_static_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_static_ptr[dev];
    return BF_OK;
}

// Self-test of the device-side bounded waits: one warp waits on an mbarrier
// phase that nothing completes (no thread arrives) until timeout_ns pass on the
// global timer, then records the timeout in *err, as a beamforming CTA whose
// copies never land does, and returns.
__global__ void __launch_bounds__(32) wait_selftest_kernel(unsigned long long timeout_ns, int *err)
{
    __shared__ unsigned long long bar;
    const unsigned a = (unsigned)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(1u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    const unsigned long long deadline = t + timeout_ns;
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(0u)
            : "memory");
        if (__all_sync(0xffffffffu, done != 0))
            return;  // the phase completed (it cannot: nothing arrives)
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (__any_sync(0xffffffffu, t >= deadline)) {
            if (threadIdx.x == 0)
                atomicOr(err, 1);
            return;
        }
    }
}

}  // namespace
}  // namespace bfi

using namespace bfi;

extern "C" BF_API int bf_selftest_wait(int64_t timeout_us)
{
    if (timeout_us < 1 || timeout_us > 1000000)
        return fail(BF_EINVAL, "timeout_us must be in [1, 1000000], got %lld", (long long)timeout_us);
    int *err_dev = nullptr;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaMalloc(&err_dev, sizeof(int));
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(err_dev, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        wait_selftest_kernel<<<1, 32, 0, st>>>((unsigned long long)timeout_us * 1000ull, err_dev);
        e = cudaGetLastError();
    }
    int err_host = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&err_host, err_dev, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (st)
        cudaStreamDestroy(st);
    if (err_dev)
        cudaFree(err_dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "bounded-wait self-test");
    if (err_host & 1)
        return fail(BF_ETIMEDOUT, "bounded-wait self-test: the wait ran out after %lld us (expected)",
                    (long long)timeout_us);
    return BF_OK;
}

extern "C" BF_API int bf_logdb_static(const float *y_dev, int32_t nx, int32_t nz, double z0_m,
                                      double z1_m, double f0_hz, double c_mps, int32_t bandpass,
                                      float *db_dev, void *cuda_stream)
{
    if (!y_dev || !db_dev)
        return fail(BF_EINVAL, "null image pointer");
    if (nx < 1 || nz < 1 || nz > 4096 || (nz & (nz - 1)) != 0)
        return fail(BF_EINVAL, "bf_logdb_static needs nx >= 1 and a power-of-two nz <= 4096 (got %d x %d)",
                    nx, nz);
    if ((size_t)nx * (size_t)nz > kStaticPixels)
        return fail(BF_EINVAL, "bf_logdb_static handles at most %zu pixels (got %d x %d)",
                    kStaticPixels, nx, nz);
    if (!(z1_m >= z0_m) || !(c_mps > 0.0) || !(f0_hz > 0.0))
        return fail(BF_EINVAL, "bad depth range or acquisition parameters");
    float *scratch = nullptr;
    int rc = static_scratch(&scratch);
    if (rc)
        return rc;
    int kb_lo = 1, kb_hi = 0;
    bandpass_bins(nz, z0_m, z1_m, c_mps, f0_hz, kb_lo, kb_hi);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    float *env = scratch;
    unsigned *maxbits = reinterpret_cast<unsigned *>(scratch + kStaticPixels);
    cudaError_t e = cudaMemsetAsync(maxbits, 0, sizeof(unsigned), st);  // the maximum starts at 0
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync (static scratch)");
    const int C = nz >= 2048 ? 1 : 2048 / nz;
    const size_t smem = (3u * (size_t)C * nz + (size_t)nz) * sizeof(float2);
    int sms = 0;
    e = kernel_setup((const void *)static_envelope_kernel, smem, 256, false, &sms, nullptr);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaFuncSetAttribute");
    const int blocks = (nx + 2 * C - 1) / (2 * C);
    static_envelope_kernel<<<blocks, 256, smem, st>>>(y_dev, nx, nz, bandpass ? 1 : 0, kb_lo, kb_hi,
                                                      env, maxbits);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(e, "envelope launch");
    const size_t n = (size_t)nx * nz;
    const int lb = (int)std::min<size_t>((n + 255) / 256, 4096);
    static_log_kernel<<<lb, 256, 0, st>>>(env, n, maxbits, db_dev, 70.0f);
    e = cudaGetLastError();
    return e == cudaSuccess ? BF_OK : cuda_fail(e, "log launch");
}

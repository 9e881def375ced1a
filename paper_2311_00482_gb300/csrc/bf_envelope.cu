// Warp-per-column-pair envelope kernel for 512-sample depths: the
// analytic-signal envelope along depth of the B-mode display (Fig. 3), with
// the DMAS image's [f0, 3 f0] band-pass, without block-wide barriers.
//
// Two image columns a, b form one complex sequence z[n] = y_a[n] + i y_b[n]
// of length N = 512.  A warp transforms it with the four-step decomposition
// n = 32 n1 + n2, k = k1 + 16 k2 (n1, k1 < 16; n2, k2 < 32):
//   lane n2 holds z[32 n1 + n2] for all n1 (coalesced column loads),
//   16-point DFTs over n1 in registers (4 x 4 radix-4), twiddles W_N^(n2 k1),
//   a transpose through a warp-private shared-memory buffer,
//   32-point DFTs over n2 split over lane pairs: 16-point DFTs of the even and
//   odd n2 and one radix-2 step, the halves exchanged by warp shuffles.
// The inverse runs the same steps backwards and ends in the load layout, so
// the envelope is formed in registers and stored coalesced.  Spectral masks
// (scipy.signal.hilbert's one-sided mask; the band-pass keeps |k| in
// [kb_lo, kb_hi]):
//   no band-pass: the Hilbert transforms of both columns in one inverse,
//     IDFT(-i sgn(k) Z) = H{y_a} + i H{y_b}; env = |y + i H{y}|;
//   band-pass: IDFT(B Z) and IDFT(-i sgn(k) B Z) give the band-passed columns
//     and their Hilbert transforms; env = |y_B + i H{y_B}|.
// The inverse's 1/N (a power of two, exact) rides on the mask.  Complex
// additions, the lane-pair radix-2 step and the magnitudes' squares run as
// paired FP32 instructions; the magnitudes' square roots on the
// special-function unit.  Each image's maximum goes to its maxbits word
// (float bits, env >= 0).
#include <cuda_runtime.h>
#include <stdint.h>

#include "bf_fft.cuh"
#include "bf_internal.h"

namespace bfi {
namespace {

constexpr int kEnvWarps = 8;                 // warps per CTA, each on its own column pairs
constexpr int kR = 16, kN = 32 * kR;         // registers per lane, transform length
// Row pitch (complex values) of the transpose buffers and the twiddle table:
// the lane pairs' strided accesses (row lane / 2, column 2 j + lane % 2) fall
// on distinct banks.
constexpr int kPitch = 34;

// cos, sin of 2 pi e / 32 for e < 16
__device__ __constant__ float2 kW32[16] = {
    {1.000000000e+00f, 0.000000000e+00f},  {9.807852804e-01f, 1.950903220e-01f},
    {9.238795325e-01f, 3.826834324e-01f},  {8.314696123e-01f, 5.555702330e-01f},
    {7.071067812e-01f, 7.071067812e-01f},  {5.555702330e-01f, 8.314696123e-01f},
    {3.826834324e-01f, 9.238795325e-01f},  {1.950903220e-01f, 9.807852804e-01f},
    {0.000000000e+00f, 1.000000000e+00f},  {-1.950903220e-01f, 9.807852804e-01f},
    {-3.826834324e-01f, 9.238795325e-01f}, {-5.555702330e-01f, 8.314696123e-01f},
    {-7.071067812e-01f, 7.071067812e-01f}, {-8.314696123e-01f, 5.555702330e-01f},
    {-9.238795325e-01f, 3.826834324e-01f}, {-9.807852804e-01f, 1.950903220e-01f}};

// Complex add / subtract as one paired FP32 instruction (Blackwell f32x2):
// the real and imaginary parts of a float2 sit in a register pair.
__device__ __forceinline__ float2 c_add(float2 a, float2 b)
{
    unsigned long long ra, rb, rc;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(rc) : "l"(ra), "l"(rb));
    float2 c;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(c.x), "=f"(c.y) : "l"(rc));
    return c;
}

__device__ __forceinline__ float2 c_sub(float2 a, float2 b)
{
    unsigned long long ra, rb, rc;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rc) : "l"(ra), "l"(rb));
    float2 c;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(c.x), "=f"(c.y) : "l"(rc));
    return c;
}

// (a.x^2 + b.x^2, a.y^2 + b.y^2): per half b^2 rounded, then one FMA.
__device__ __forceinline__ float2 c_sqsum(float2 a, float2 b)
{
    unsigned long long ra, rb, rc;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(rc) : "l"(rb));
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(rc) : "l"(ra), "l"(rc));
    float2 c;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(c.x), "=f"(c.y) : "l"(rc));
    return c;
}

// Square root on the special-function unit (relative error about one unit in
// the last place, far inside the envelope's tolerance).
__device__ __forceinline__ float sqrt_fast(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// s * a + b with s a scalar (both halves), as one paired FMA.
__device__ __forceinline__ float2 c_sfma(float s, float2 a, float2 b)
{
    unsigned long long rs, ra, rb, rc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(rs) : "f"(s));
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rc) : "l"(rs), "l"(ra), "l"(rb));
    float2 c;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(c.x), "=f"(c.y) : "l"(rc));
    return c;
}

// b * W_32^e (INV: conjugate), W_32 = exp(-2 pi i / 32), 0 <= e < 32; e is a
// compile-time constant wherever this is used (quarter turns are swaps).
template <bool INV>
__device__ __forceinline__ float2 w32mul(float2 b, int e)
{
    if (e >= 16) {  // W_32^16 = -1
        b = make_float2(-b.x, -b.y);
        e -= 16;
    }
    if (e == 0)
        return b;
    if (e == 8)
        return INV ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x);
    const float2 w = kW32[e];
    const float s = INV ? w.y : -w.y;
    return make_float2(b.x * w.x - b.y * s, b.x * s + b.y * w.x);
}

// 4-point DFT in place: y_k = sum_n x_n W_4^(n k), W_4 = -i (INV: +i).
template <bool INV>
__device__ __forceinline__ void dft4(float2 &a, float2 &b, float2 &c, float2 &d)
{
    const float2 t0 = c_add(a, c), t1 = c_sub(a, c), t2 = c_add(b, d), u = c_sub(b, d);
    a = c_add(t0, t2);
    c = c_sub(t0, t2);
    // t1 +- u W_4 (W_4 = -i, INV: +i): the swapped halves in scalar operations
    if (INV) {
        b = make_float2(t1.x - u.y, t1.y + u.x);
        d = make_float2(t1.x + u.y, t1.y - u.x);
    } else {
        b = make_float2(t1.x + u.y, t1.y - u.x);
        d = make_float2(t1.x - u.y, t1.y + u.x);
    }
}

// In-register 16-point DFT, natural order in and out: x[k] <- sum_n x[n]
// W_16^(n k) (INV: conjugate exponent, no scaling), as 4 x 4 with n = n1 + 4 n2
// and k = 4 k1 + k2: DFTs over n2, twiddles W_16^(n1 k2), DFTs over n1, and a
// transposed read-out (register renaming only).
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&x)[16])
{
    dft4<INV>(x[0], x[4], x[8], x[12]);  // -> B[n1][k2] at n1 + 4 k2
    dft4<INV>(x[1], x[5], x[9], x[13]);
    dft4<INV>(x[2], x[6], x[10], x[14]);
    dft4<INV>(x[3], x[7], x[11], x[15]);
    x[5] = w32mul<INV>(x[5], 2);  // W_16^(n1 k2) = W_32^(2 n1 k2)
    x[9] = w32mul<INV>(x[9], 4);
    x[13] = w32mul<INV>(x[13], 6);
    x[6] = w32mul<INV>(x[6], 4);
    x[10] = w32mul<INV>(x[10], 8);
    x[14] = w32mul<INV>(x[14], 12);
    x[7] = w32mul<INV>(x[7], 6);
    x[11] = w32mul<INV>(x[11], 12);
    x[15] = w32mul<INV>(x[15], 18);
    dft4<INV>(x[0], x[1], x[2], x[3]);  // -> X[4 k1 + k2] at 4 k2 + k1
    dft4<INV>(x[4], x[5], x[6], x[7]);
    dft4<INV>(x[8], x[9], x[10], x[11]);
    dft4<INV>(x[12], x[13], x[14], x[15]);
    float2 t;
    t = x[1], x[1] = x[4], x[4] = t;
    t = x[2], x[2] = x[8], x[8] = t;
    t = x[3], x[3] = x[12], x[12] = t;
    t = x[6], x[6] = x[9], x[9] = t;
    t = x[7], x[7] = x[13], x[13] = t;
    t = x[11], x[11] = x[14], x[14] = t;
}

// Shared-memory accesses through 32-bit shared-window addresses, and global
// stores and reductions through explicitly global instructions: generic
// accesses through pointers the compiler cannot place would keep the
// transforms' register arrays in local memory.
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float2 lds2(uint32_t a)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}

__device__ __forceinline__ void sts2(uint32_t a, float2 v)
{
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}

__device__ __forceinline__ void red_max_global(unsigned *p, unsigned v)
{
    asm volatile("red.global.max.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ float2 shfl_pair(float2 v)
{
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, 1), __shfl_xor_sync(0xffffffffu, v.y, 1));
}

// Length-512 transforms of a warp's sequence (buf: the warp's transpose
// buffer, twt: the [16][kPitch] table of W_N^(k1 n2)).  Forward: in, register
// r of lane n2 holds z[32 r + n2]; out, register k of the lane holds
// X[k1 + 16 k2] with k1 = lane / 2, k2 = 16 (lane % 2) + k.  Inverse (no
// scaling): the other way round.
template <bool INV>
__device__ __forceinline__ void fft_warp(float2 (&v)[kR], uint32_t buf, uint32_t twt, int lane)
{
    const int k1 = lane >> 1, h = lane & 1;
    const float sgn = h ? -1.f : 1.f;
    auto at = [&](int row, int col) { return 8u * (uint32_t)(row * kPitch + col); };
    if constexpr (!INV) {
        dft16<false>(v);  // over n1, for n2 = lane
#pragma unroll
        for (int k = 1; k < kR; ++k)
            v[k] = cmul(v[k], lds2(twt + at(k, lane)));  // W_N^(lane k1)
#pragma unroll
        for (int k = 0; k < kR; ++k)
            sts2(buf + at(k, lane), v[k]);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 16; ++j)
            v[j] = lds2(buf + at(k1, 2 * j + h));
        __syncwarp();
        dft16<false>(v);  // E_h[k] over the even (h = 0) or odd n2
        // X[k1 + 16 k] = E_0 + W_32^k E_1, X[k1 + 16 (k + 16)] = E_0 - W_32^k E_1:
        // the odd lane premultiplies its E_1, then both take sgn * own + other
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float2 tw = w32mul<false>(v[k], k);
            const float2 own = h ? tw : v[k];
            const float2 oth = shfl_pair(own);
            v[k] = c_sfma(sgn, own, oth);
        }
    } else {
        // radix-2 step over k2 (k2 and k2 + 16 in the two lanes): the even lane
        // keeps P + Q, the odd one (P - Q) W_32^-k; then 16-point inverses give
        // the even (h = 0) or odd n2
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float2 oth = shfl_pair(v[k]);
            const float2 s = c_sfma(sgn, v[k], oth);
            v[k] = h ? w32mul<true>(s, k) : s;
        }
        dft16<true>(v);  // register m: n2 = 2 m + h
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int n2 = 2 * m + h;
            const float2 w = lds2(twt + at(k1, n2));  // W_N^(k1 n2), conjugated
            sts2(buf + at(k1, n2), cmul(v[m], make_float2(w.x, -w.y)));
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < kR; ++k)
            v[k] = lds2(buf + at(k, lane));
        __syncwarp();
        dft16<true>(v);  // over k1: register r holds z[32 r + lane]
    }
}

__device__ __forceinline__ int find_pair_job(const int *__restrict__ prefix, int njobs, int g)
{
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(32 * kEnvWarps, 2)
    envelope_warp_kernel(const EnvJob *__restrict__ jobs, const int *__restrict__ pair_prefix,
                         int njobs, int total_pairs)
{
    extern __shared__ __align__(16) float2 esm[];
    // the log stage's blocks may be scheduled as this grid's CTAs finish (they
    // wait for the whole grid before reading its results)
    asm volatile("griddepcontrol.launch_dependents;");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    {
        // [16][kPitch]: W_N^(k1 n2) from the job's table exp(-2 pi i k / N), k < N
        const float2 *tw = jobs[0].tw;
        for (int t = threadIdx.x; t < kR * 32; t += blockDim.x) {
            const int k1 = t >> 5, n2 = t & 31;
            esm[k1 * kPitch + n2] = __ldg(tw + ((k1 * n2) & (kN - 1)));
        }
    }
    __syncthreads();
    const uint32_t twa = smem_addr(esm);
    const uint32_t buf = smem_addr(esm + (1 + warp) * kR * kPitch);  // this warp's transposes
    // this warp's holding area, [r][lane]: at most one transform's registers and
    // one other array are live at a time
    const uint32_t hold = smem_addr(esm + (1 + kEnvWarps) * kR * kPitch) + 8u * (warp * kR * 32 + lane);
    auto hold_at = [&](int r) { return hold + 8u * 32u * (uint32_t)r; };
    // spectrum register k of this lane is bin f = k1 + 16 k + 256 h: sgn(f) is
    // +1 (h = 0) or -1 (h = 1) except at f = 0 and f = N / 2 (k1 = k = 0);
    // |f| = k1 + 16 k (h = 0), 256 - k1 - 16 k (h = 1)
    const int k1 = lane >> 1, h = lane & 1;
    const float sg_lane = h ? -1.f : 1.f;

    int cur = -1;
    float lmax = 0.f;
    int mask_job = -1;     // the job bp_mask belongs to
    unsigned bp_mask = 0u;  // bit k: spectrum register k of this lane is in the band
    unsigned *cur_max = nullptr;
    const float inv = 1.f / (float)kN;
    // Column pairs in reverse launch order: the beamformer writes the last
    // images of a batch last, so those are still in L2 when this kernel starts.
    for (int g0 = blockIdx.x * kEnvWarps + warp; g0 < total_pairs; g0 += gridDim.x * kEnvWarps) {
        const int g = total_pairs - 1 - g0;
        const int jb = find_pair_job(pair_prefix, njobs, g);
        const EnvJob &J = jobs[jb];
        if (jb != cur) {  // flush the previous image's maximum
            if (cur >= 0) {
                const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(lmax));
                if (lane == 0)
                    red_max_global(cur_max, m);
            }
            cur = jb;
            cur_max = J.maxbits;
            lmax = 0.f;
        }
        const int pair = g - __ldg(pair_prefix + jb);
        const int ca = 2 * pair, cb = ca + 1;
        const bool has_b = cb < J.nx;
        const float *__restrict__ ya = J.y + (size_t)ca * kN;
        const float *__restrict__ yb = J.y + (size_t)(has_b ? cb : ca) * kN;
        float2 v[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int n = 32 * r + lane;
            // read once: streaming loads, evicted first, so the envelopes this
            // kernel writes stay in L2 for the log stage
            v[r] = make_float2(__ldcs(ya + n), has_b ? __ldcs(yb + n) : 0.f);
        }
        const bool band = J.band != 0;
        if (!band) {
#pragma unroll
            for (int r = 0; r < kR; ++r)
                sts2(hold_at(r), v[r]);  // the columns themselves, for |y + i H{y}|
        }
        fft_warp<false>(v, buf, twa, lane);
        if (!band) {
            // the inverse transform's 1 / N (a power of two: exact) with the mask
#pragma unroll
            for (int k = 0; k < kR; ++k) {
                const float sg = (k == 0 && k1 == 0) ? 0.f : sg_lane * inv;
                v[k] = make_float2(v[k].y * sg, -v[k].x * sg);  // -i sgn(f) Z / N
            }
            fft_warp<true>(v, buf, twa, lane);
#pragma unroll
            for (int r = 0; r < kR; ++r) {
                const float2 q = c_sqsum(lds2(hold_at(r)), v[r]);  // y^2 + (H y)^2
                v[r] = make_float2(sqrt_fast(q.x), sqrt_fast(q.y));
            }
        } else {
            if (jb != mask_job) {  // this lane's bins inside the band, once per image
                const int lo = J.kb_lo, hi = J.kb_hi;
                bp_mask = 0u;
#pragma unroll
                for (int k = 0; k < kR; ++k) {
                    const int fa = h ? 256 - k1 - 16 * k : k1 + 16 * k;  // |f|
                    bp_mask |= (fa >= lo && fa <= hi) ? (1u << k) : 0u;
                }
                mask_job = jb;
            }
#pragma unroll
            for (int k = 0; k < kR; ++k) {  // the 1 / N of the inverses with the mask
                const float bp = ((bp_mask >> k) & 1u) ? inv : 0.f;
                const float sg = (k == 0 && k1 == 0) ? 0.f : sg_lane;
                v[k] = make_float2(v[k].x * bp, v[k].y * bp);                 // B Z
                sts2(hold_at(k), make_float2(v[k].y * sg, -v[k].x * sg));  // -i sgn(f) B Z
            }
            fft_warp<true>(v, buf, twa, lane);  // the band-passed columns
#pragma unroll
            for (int r = 0; r < kR; ++r) {  // swap: their Hilbert spectrum next
                const float2 q = lds2(hold_at(r));
                sts2(hold_at(r), v[r]);
                v[r] = q;
            }
            fft_warp<true>(v, buf, twa, lane);  // their Hilbert transforms
#pragma unroll
            for (int r = 0; r < kR; ++r) {
                const float2 q = c_sqsum(lds2(hold_at(r)), v[r]);
                v[r] = make_float2(sqrt_fast(q.x), sqrt_fast(q.y));
            }
        }
        float *__restrict__ oa = J.env + (size_t)ca * kN;
        float *__restrict__ ob = J.env + (size_t)cb * kN;
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int n = 32 * r + lane;
            __stcg(oa + n, v[r].x);
            lmax = fmaxf(lmax, v[r].x);
            if (has_b) {
                __stcg(ob + n, v[r].y);
                lmax = fmaxf(lmax, v[r].y);
            }
        }
    }
    if (cur >= 0) {
        const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(lmax));
        if (lane == 0)
            red_max_global(cur_max, m);
    }
}

}  // namespace

bool envelope_warp_ok(int nz, int fft_m, int bluestein)
{
    return !bluestein && fft_m == nz && nz == kN;
}

static size_t envelope_warp_smem_bytes()
{
    return ((size_t)(1 + kEnvWarps) * kR * kPitch + (size_t)kEnvWarps * kR * 32) * sizeof(float2);
}

cudaError_t launch_envelope_warp(const EnvJob *jobs_dev, const int *pair_prefix_dev, int njobs,
                                 int total_pairs, cudaStream_t stream)
{
    if (njobs <= 0 || total_pairs <= 0)
        return cudaSuccess;
    const size_t smem = envelope_warp_smem_bytes();
    int sms = 0, occ = 0;
    cudaError_t e = kernel_setup((const void *)envelope_warp_kernel, smem, 32 * kEnvWarps, false,
                                 &sms, &occ);
    if (e != cudaSuccess)
        return e;
    const int cap = sms * (occ > 0 ? occ : 1);
    const int want = (total_pairs + kEnvWarps - 1) / kEnvWarps;
    envelope_warp_kernel<<<want < cap ? want : cap, 32 * kEnvWarps, smem, stream>>>(
        jobs_dev, pair_prefix_dev, njobs, total_pairs);
    return cudaGetLastError();
}

}  // namespace bfi

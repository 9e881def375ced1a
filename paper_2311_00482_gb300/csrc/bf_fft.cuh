// Shared-memory FFT building blocks used by the envelope kernels.
#pragma once

#include <cuda_runtime.h>

namespace bfi {

static __device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Radix-4 Stockham FFTs (a final radix-2 pass when log2(m) is odd) of `cols`
// complex columns of length m stored back to back in x; tw[k] = exp(-2 pi i
// k / m) for k < m.  inverse: +i exponent, no scaling.  Returns the buffer
// holding the result.
static __device__ float2 *fft_r4(float2 *x, float2 *y, int m, int lgm, int cols, const float2 *tw,
                                bool inverse)
{
    int ns = 1, lg = 0;
    if (m >= 4) {
        const int q = m >> 2;
        for (; (ns << 2) <= m; ns <<= 2, lg += 2) {
            const int sh = lgm - 2 - lg;  // log2(m / (4 ns))
            const int total = cols * q;
            for (int t = threadIdx.x; t < total; t += blockDim.x) {
                const int c = t >> (lgm - 2), j = t & (q - 1);
                const float2 *xc = x + (size_t)c * m;
                float2 *yc = y + (size_t)c * m;
                float2 v0 = xc[j], v1 = xc[j + q], v2 = xc[j + 2 * q], v3 = xc[j + 3 * q];
                const int r = j & (ns - 1);
                const int k1 = r << sh;
                float2 w1 = tw[k1], w2 = tw[2 * k1], w3 = tw[3 * k1];
                if (inverse) {
                    w1.y = -w1.y;
                    w2.y = -w2.y;
                    w3.y = -w3.y;
                }
                v1 = cmul(v1, w1);
                v2 = cmul(v2, w2);
                v3 = cmul(v3, w3);
                const float2 a0 = make_float2(v0.x + v2.x, v0.y + v2.y);
                const float2 a1 = make_float2(v0.x - v2.x, v0.y - v2.y);
                const float2 a2 = make_float2(v1.x + v3.x, v1.y + v3.y);
                const float2 d = make_float2(v1.x - v3.x, v1.y - v3.y);
                // (v1 - v3) times -i (forward) or +i (inverse)
                const float2 a3 = inverse ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
                const int o = ((j - r) << 2) + r;
                yc[o] = make_float2(a0.x + a2.x, a0.y + a2.y);
                yc[o + ns] = make_float2(a1.x + a3.x, a1.y + a3.y);
                yc[o + 2 * ns] = make_float2(a0.x - a2.x, a0.y - a2.y);
                yc[o + 3 * ns] = make_float2(a1.x - a3.x, a1.y - a3.y);
            }
            __syncthreads();
            float2 *tmp = x;
            x = y;
            y = tmp;
        }
    }
    if (ns < m) {  // one radix-2 pass, ns == m / 2
        const int half = m >> 1;
        for (int t = threadIdx.x; t < cols * half; t += blockDim.x) {
            const int c = t >> (lgm - 1), j = t & (half - 1);
            const float2 *xc = x + (size_t)c * m;
            float2 *yc = y + (size_t)c * m;
            float2 w = tw[j];
            if (inverse)
                w.y = -w.y;
            const float2 v0 = xc[j], t2 = cmul(xc[j + half], w);
            yc[j] = make_float2(v0.x + t2.x, v0.y + t2.y);
            yc[j + half] = make_float2(v0.x - t2.x, v0.y - t2.y);
        }
        __syncthreads();
        float2 *tmp = x;
        x = y;
        y = tmp;
    }
    return x;
}

// 8-point DFT of v (forward: exp(-2 pi i / 8) powers; inverse: conjugate), in
// place, outputs in natural order: two radix-2 stages feeding two 4-point DFTs.
static __device__ __forceinline__ void dft8(float2 *v, bool inverse)
{
    const float r2 = 0.70710678118654752f;
    float2 b[8];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        b[p] = make_float2(v[p].x + v[p + 4].x, v[p].y + v[p + 4].y);
        b[p + 4] = make_float2(v[p].x - v[p + 4].x, v[p].y - v[p + 4].y);
    }
    // b5 *= W8, b6 *= W8^2, b7 *= W8^3 (W8 = exp(-+ 2 pi i / 8))
    if (!inverse) {
        b[5] = make_float2(r2 * (b[5].x + b[5].y), r2 * (b[5].y - b[5].x));
        b[6] = make_float2(b[6].y, -b[6].x);
        b[7] = make_float2(r2 * (b[7].y - b[7].x), -r2 * (b[7].x + b[7].y));
    } else {
        b[5] = make_float2(r2 * (b[5].x - b[5].y), r2 * (b[5].y + b[5].x));
        b[6] = make_float2(-b[6].y, b[6].x);
        b[7] = make_float2(-r2 * (b[7].x + b[7].y), r2 * (b[7].x - b[7].y));
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // 4-point DFTs of b[4h .. 4h + 3] -> outputs h, h + 2, h + 4, h + 6
        const float2 c0 = b[4 * h], c1 = b[4 * h + 1], c2 = b[4 * h + 2], c3 = b[4 * h + 3];
        const float2 d0 = make_float2(c0.x + c2.x, c0.y + c2.y);
        const float2 d1 = make_float2(c0.x - c2.x, c0.y - c2.y);
        const float2 d2 = make_float2(c1.x + c3.x, c1.y + c3.y);
        const float2 e = make_float2(c1.x - c3.x, c1.y - c3.y);
        const float2 d3 = inverse ? make_float2(-e.y, e.x) : make_float2(e.y, -e.x);
        v[h] = make_float2(d0.x + d2.x, d0.y + d2.y);
        v[h + 2] = make_float2(d1.x + d3.x, d1.y + d3.y);
        v[h + 4] = make_float2(d0.x - d2.x, d0.y - d2.y);
        v[h + 6] = make_float2(d1.x - d3.x, d1.y - d3.y);
    }
}

// Shared-memory layout of the transform buffers: element i of a buffer lives
// at swz(i) = i ^ g(i), g moving bits 4..6 of i into bits 0..2 and bit 6 into
// bit 3 (a bijection inside every aligned run of 16 elements).  For the
// length-512 envelope transforms it makes every pass's strided reads and
// writes hit 16 distinct bank pairs per half warp.
template <bool SWZ>
static __device__ __forceinline__ int swz(int i)
{
    return SWZ ? (i ^ (((i >> 4) & 7) | ((i >> 3) & 8))) : i;
}

// Per-pass twiddles of the radix-8 passes with stride ns = 8, 64, ... of a
// length-m transform: w^1, w^2, w^4 of k1 = r * m / (8 ns) for r < ns, each
// power's run contiguous in r (consecutive lanes read consecutive entries).
static __host__ __device__ inline int pass_twiddle_count(int lgm)
{
    int n = 0;
    for (int ns = 8, lg = 3; lgm - lg >= 3; ns <<= 3, lg += 3)
        n += 3 * ns;
    return n;
}

static __device__ void fill_pass_twiddles(float2 *ptw, const float2 *tw, int lgm)
{
    int base = 0;
    for (int ns = 8, lg = 3; lgm - lg >= 3; ns <<= 3, lg += 3) {
        const int sh = lgm - 3 - lg;
        for (int r = threadIdx.x; r < ns; r += blockDim.x) {
            const int k1 = r << sh;
            ptw[base + r] = tw[k1];
            ptw[base + ns + r] = tw[2 * k1];
            ptw[base + 2 * ns + r] = tw[4 * k1];
        }
        base += 3 * ns;
    }
}

// Stockham FFTs with radix-8 passes (then one radix-4 or radix-2 pass for the
// remaining factor) of `cols` complex columns of length m stored back to back
// in x; same contract as fft_r4: tw[k] = exp(-2 pi i k / m), inverse = +i
// exponent without scaling, returns the buffer holding the result.  SWZ:
// buffers in the swz layout; ptw (optional): the per-pass twiddle table.
// Without SWZ the first pass (stride 1) writes each thread's eight outputs as
// four 16-byte stores.
template <bool SWZ = false>
static __device__ float2 *fft_r8(float2 *x, float2 *y, int m, int lgm, int cols, const float2 *tw,
                                bool inverse, const float2 *ptw = nullptr)
{
    int ns = 1, lg = 0, pbase = 0;
    while (lgm - lg >= 3) {
        const int q = m >> 3, sh = lgm - 3 - lg;  // sh = log2(m / (8 ns))
        const int total = cols * q;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int c = t >> (lgm - 3), j = t & (q - 1);
            const int cb = c * m;  // column start
            const int r = j & (ns - 1), k1 = r << sh;
            float2 v[8];
            v[0] = x[swz<SWZ>(cb + j)];
            if (ns == 1) {  // first pass: every twiddle is 1
#pragma unroll
                for (int p = 1; p < 8; ++p)
                    v[p] = x[swz<SWZ>(cb + j + p * q)];
            } else {
                // w^1, w^2, w^4 from a table, the other powers by products
                float2 w1, w2, w4;
                if (ptw) {
                    w1 = ptw[pbase + r];
                    w2 = ptw[pbase + ns + r];
                    w4 = ptw[pbase + 2 * ns + r];
                } else {
                    w1 = tw[k1];
                    w2 = tw[2 * k1];
                    w4 = tw[4 * k1];
                }
                if (inverse) {
                    w1.y = -w1.y;
                    w2.y = -w2.y;
                    w4.y = -w4.y;
                }
                const float2 w3 = cmul(w1, w2);
                const float2 w[8] = {make_float2(1.f, 0.f), w1, w2, w3, w4, cmul(w1, w4),
                                     cmul(w2, w4), cmul(w3, w4)};
#pragma unroll
                for (int p = 1; p < 8; ++p)
                    v[p] = cmul(x[swz<SWZ>(cb + j + p * q)], w[p]);
            }
            dft8(v, inverse);
            const int o = cb + ((j - r) << 3) + r;
            if (!SWZ && ns == 1) {
                float4 *y4 = reinterpret_cast<float4 *>(y + o);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    y4[u] = make_float4(v[2 * u].x, v[2 * u].y, v[2 * u + 1].x, v[2 * u + 1].y);
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    y[swz<SWZ>(o + u * ns)] = v[u];
            }
        }
        __syncthreads();
        float2 *tmp = x;
        x = y;
        y = tmp;
        if (ns > 1)
            pbase += 3 * ns;
        ns <<= 3;
        lg += 3;
    }
    if (lgm - lg == 2) {  // one radix-4 pass
        const int q = m >> 2, sh = lgm - 2 - lg;
        for (int t = threadIdx.x; t < cols * q; t += blockDim.x) {
            const int c = t >> (lgm - 2), j = t & (q - 1);
            const int cb = c * m;
            const int r = j & (ns - 1), k1 = r << sh;
            float2 w1 = tw[k1], w2 = tw[2 * k1], w3 = tw[3 * k1];
            if (inverse) {
                w1.y = -w1.y;
                w2.y = -w2.y;
                w3.y = -w3.y;
            }
            const float2 v0 = x[swz<SWZ>(cb + j)], v1 = cmul(x[swz<SWZ>(cb + j + q)], w1),
                         v2 = cmul(x[swz<SWZ>(cb + j + 2 * q)], w2),
                         v3 = cmul(x[swz<SWZ>(cb + j + 3 * q)], w3);
            const float2 a0 = make_float2(v0.x + v2.x, v0.y + v2.y);
            const float2 a1 = make_float2(v0.x - v2.x, v0.y - v2.y);
            const float2 a2 = make_float2(v1.x + v3.x, v1.y + v3.y);
            const float2 d = make_float2(v1.x - v3.x, v1.y - v3.y);
            const float2 a3 = inverse ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
            const int o = cb + ((j - r) << 2) + r;
            y[swz<SWZ>(o)] = make_float2(a0.x + a2.x, a0.y + a2.y);
            y[swz<SWZ>(o + ns)] = make_float2(a1.x + a3.x, a1.y + a3.y);
            y[swz<SWZ>(o + 2 * ns)] = make_float2(a0.x - a2.x, a0.y - a2.y);
            y[swz<SWZ>(o + 3 * ns)] = make_float2(a1.x - a3.x, a1.y - a3.y);
        }
        __syncthreads();
        float2 *tmp = x;
        x = y;
        y = tmp;
    } else if (lgm - lg == 1) {  // one radix-2 pass, ns == m / 2
        const int half = m >> 1;
        for (int t = threadIdx.x; t < cols * half; t += blockDim.x) {
            const int c = t >> (lgm - 1), j = t & (half - 1);
            const int cb = c * m;
            float2 w = tw[j];
            if (inverse)
                w.y = -w.y;
            const float2 v0 = x[swz<SWZ>(cb + j)], t2 = cmul(x[swz<SWZ>(cb + j + half)], w);
            y[swz<SWZ>(cb + j)] = make_float2(v0.x + t2.x, v0.y + t2.y);
            y[swz<SWZ>(cb + j + half)] = make_float2(v0.x - t2.x, v0.y - t2.y);
        }
        __syncthreads();
        float2 *tmp = x;
        x = y;
        y = tmp;
    }
    return x;
}

}  // namespace bfi

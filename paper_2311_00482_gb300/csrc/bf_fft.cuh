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

}  // namespace bfi

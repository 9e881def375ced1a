// Batched copies between host and device memory for the serving engine: one
// kernel moves every frame of a bf_submit_many (records in) or a bf_poll_many
// (images out).  Pinned host buffers are read or written in place through
// their device-mapped addresses over the host link, which beats one
// cudaMemcpyAsync per frame for frames of a few hundred KB (measured on
// GB300: 64 x 256 KB in 0.09 ms instead of 0.28 ms; 64 x 2 MB in 0.70 ms
// instead of 0.86 ms).
#include "bf_internal.h"

namespace bfi {
namespace {

__global__ void __launch_bounds__(256) copy_segments_kernel(const CopyList list, int blocks_per_seg)
{
    const int s = blockIdx.x / blocks_per_seg, b = blockIdx.x - s * blocks_per_seg;
    if (s >= list.n)
        return;
    const CopySeg g = list.seg[s];
    const uint4 *__restrict__ src = static_cast<const uint4 *>(g.src);
    uint4 *__restrict__ dst = static_cast<uint4 *>(g.dst);
    const unsigned long long n16 = g.bytes / 16;
    for (unsigned long long i = (unsigned long long)b * blockDim.x + threadIdx.x; i < n16;
         i += (unsigned long long)blocks_per_seg * blockDim.x)
        dst[i] = src[i];
}

}  // namespace

bool copy_segment_ok(const void *src, const void *dst, size_t bytes)
{
    return bytes > 0 && bytes % 16 == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0 &&
           (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
}

cudaError_t launch_copy_segments(const CopyList &list, int blocks_per_seg, cudaStream_t stream)
{
    if (list.n <= 0)
        return cudaSuccess;
    copy_segments_kernel<<<list.n * blocks_per_seg, 256, 0, stream>>>(list, blocks_per_seg);
    return cudaGetLastError();
}

}  // namespace bfi

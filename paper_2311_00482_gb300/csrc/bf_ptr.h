// How the serving engine moves a caller's buffer (RF records in, images out),
// decided from what cudaPointerGetAttributes and cudaHostGetFlags reported.
// Header-only and free of CUDA calls, so that the decision can be checked on a
// machine without a GPU.
#pragma once

#include <cuda_runtime.h>

namespace bfi {

// Direct: one cudaMemcpyAsync between the buffer and the engine's slot (a copy
// engine moves it, beside whatever kernels run).  Staged: through the slot's
// page-locked staging buffer and a host memcpy.
enum class CopyRoute { kDirect, kStaged };

// type: the buffer's memory type; host_alloc: page-locked host memory from
// cudaHostAlloc / cudaMallocHost (cudaHostGetFlags succeeded), as opposed to
// memory registered with cudaHostRegister, which may be registered read-only
// for the device; write: the copy writes the buffer.
//   device memory (of any device: cudaMemcpyDefault copies across devices)
//   and page-locked host memory are read directly;
//   they are written directly too, except registered host memory;
//   pageable (unregistered) and managed memory go through the staging buffer.
inline CopyRoute copy_route(cudaMemoryType type, bool host_alloc, bool write)
{
    if (type == cudaMemoryTypeDevice)
        return CopyRoute::kDirect;
    if (type == cudaMemoryTypeHost)
        return (!write || host_alloc) ? CopyRoute::kDirect : CopyRoute::kStaged;
    return CopyRoute::kStaged;
}

}  // namespace bfi

// Which address a copy kernel of the serving engine may use for a buffer the
// caller passed (RF records in, images out), decided from what
// cudaPointerGetAttributes reported.  Header-only and free of CUDA calls, so
// that the decision can be checked on a machine without a GPU.
#pragma once

#include <cuda_runtime.h>

namespace bfi {

// a: the buffer's attributes; p: the caller's pointer; device: the engine's
// device (where the copy kernel runs); current: the device that was current
// when `a` was taken (a.devicePointer is valid there only); write: the kernel
// would write the buffer; host_alloc: a page-locked host buffer came from
// cudaHostAlloc / cudaMallocHost (cudaHostGetFlags succeeded), as opposed to
// memory registered with cudaHostRegister, which may be read-only for the
// device.  Returns the address to use, or null when the buffer must take the
// cudaMemcpyAsync path instead:
//   device memory of another device (no peer access is set up);
//   page-locked host memory without a mapping on the engine's device;
//   registered host memory the kernel would write.
inline void *kernel_address(const cudaPointerAttributes &a, const void *p, int device, int current,
                            bool write, bool host_alloc)
{
    if (a.type == cudaMemoryTypeDevice)
        return a.device == device ? const_cast<void *>(p) : nullptr;
    if (a.type == cudaMemoryTypeHost) {
        if (current != device || a.devicePointer == nullptr)
            return nullptr;
        if (write && !host_alloc)
            return nullptr;
        return a.devicePointer;
    }
    return nullptr;  // managed or unregistered memory
}

}  // namespace bfi

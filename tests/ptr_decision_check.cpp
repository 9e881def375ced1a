// Drives bfi::kernel_address (the serving engine's choice between its copy
// kernel and cudaMemcpyAsync) with hand-made pointer attributes; built and run
// by tests/test_host_logic.py with g++ against the CUDA headers only (no GPU,
// no CUDA library).  Prints one line per case: name and 0 (memcpy path) or 1
// (kernel path, with the expected address).
#include <cstdio>
#include <cstring>

#include "bf_ptr.h"

static int kernel_path(cudaMemoryType type, int attr_device, void *p, void *devptr, int engine,
                       int current, bool write, bool host_alloc, void **got)
{
    cudaPointerAttributes a;
    std::memset(&a, 0, sizeof a);
    a.type = type;
    a.device = attr_device;
    a.devicePointer = devptr;
    a.hostPointer = type == cudaMemoryTypeHost ? p : nullptr;
    *got = bfi::kernel_address(a, p, engine, current, write, host_alloc);
    return *got != nullptr;
}

int main()
{
    char buf[64];
    void *p = buf, *mapped = buf + 16, *got = nullptr;
    struct Case {
        const char *name;
        cudaMemoryType type;
        int attr_device, engine, current;
        bool write, host_alloc;
        void *expect;
    } cases[] = {
        {"device_same", cudaMemoryTypeDevice, 1, 1, 1, false, false, p},
        {"device_same_write", cudaMemoryTypeDevice, 1, 1, 1, true, false, p},
        {"device_foreign", cudaMemoryTypeDevice, 0, 1, 1, false, false, nullptr},
        {"device_foreign_write", cudaMemoryTypeDevice, 2, 1, 1, true, false, nullptr},
        {"host_alloc_read", cudaMemoryTypeHost, 0, 0, 0, false, true, mapped},
        {"host_alloc_write", cudaMemoryTypeHost, 0, 0, 0, true, true, mapped},
        {"host_registered_read", cudaMemoryTypeHost, 0, 0, 0, false, false, mapped},
        {"host_registered_write", cudaMemoryTypeHost, 0, 0, 0, true, false, nullptr},
        {"host_other_current", cudaMemoryTypeHost, 0, 1, 0, false, true, nullptr},
        {"managed", cudaMemoryTypeManaged, 0, 0, 0, false, false, nullptr},
        {"unregistered", cudaMemoryTypeUnregistered, 0, 0, 0, false, false, nullptr},
    };
    for (const Case &c : cases) {
        void *devptr = c.type == cudaMemoryTypeHost ? mapped : (c.type == cudaMemoryTypeDevice ? p : nullptr);
        const int k = kernel_path(c.type, c.attr_device, p, devptr, c.engine, c.current, c.write,
                                  c.host_alloc, &got);
        std::printf("%s %d %d\n", c.name, k, got == c.expect);
    }
    return 0;
}

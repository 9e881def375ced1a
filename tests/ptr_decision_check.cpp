// Drives bfi::copy_route (the serving engine's choice between a direct copy and
// the page-locked staging buffer) with every memory type; built and run by
// tests/test_host_logic.py with g++ against the CUDA headers only (no GPU, no
// CUDA library).  Prints one line per case: name and 1 (direct) or 0 (staged).
#include <cstdio>

#include "bf_ptr.h"

int main()
{
    struct Case {
        const char *name;
        cudaMemoryType type;
        bool host_alloc, write;
    } cases[] = {
        {"device_read", cudaMemoryTypeDevice, false, false},
        {"device_write", cudaMemoryTypeDevice, false, true},
        {"host_alloc_read", cudaMemoryTypeHost, true, false},
        {"host_alloc_write", cudaMemoryTypeHost, true, true},
        {"host_registered_read", cudaMemoryTypeHost, false, false},
        {"host_registered_write", cudaMemoryTypeHost, false, true},
        {"managed_read", cudaMemoryTypeManaged, false, false},
        {"managed_write", cudaMemoryTypeManaged, false, true},
        {"unregistered_read", cudaMemoryTypeUnregistered, false, false},
        {"unregistered_write", cudaMemoryTypeUnregistered, false, true},
    };
    for (const Case &c : cases)
        std::printf("%s %d\n", c.name,
                    bfi::copy_route(c.type, c.host_alloc, c.write) == bfi::CopyRoute::kDirect);
    return 0;
}

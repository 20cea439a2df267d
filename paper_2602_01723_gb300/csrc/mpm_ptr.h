// mpm_ptr.h -- where a caller's array lives, as seen from the current CUDA
// device.  Shared by every entry point that takes caller arrays.
//
//  - Where::device: the current device's own memory, or managed memory;
//    kernels on the current device use it directly.
//  - Where::host: pageable or pinned host memory; entry points that accept
//    host arrays copy them through a staging buffer.
//  - Where::other_device: device memory of another GPU.  No entry point sets
//    up peer access, so a kernel given such a pointer would fault: every
//    entry point rejects it with MPM_ERR_INVALID_ARG before any GPU work.
#pragma once
#include <cuda_runtime.h>

#include <initializer_list>

namespace mpm {

enum class Where { none, host, device, other_device };

inline Where where(const void *p) {
    if (!p) return Where::none;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return Where::host;
    }
    if (a.type == cudaMemoryTypeManaged) return Where::device;
    if (a.type != cudaMemoryTypeDevice) return Where::host;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return Where::other_device;
    }
    return a.device == cur ? Where::device : Where::other_device;
}

// true when p is device memory that the current device's kernels can use
inline bool on_this_device(const void *p) { return where(p) == Where::device; }

// true when any of the (nullable) pointers is device memory of another GPU
inline bool any_on_other_device(std::initializer_list<const void *> ps) {
    for (const void *p : ps)
        if (where(p) == Where::other_device) return true;
    return false;
}

}  // namespace mpm

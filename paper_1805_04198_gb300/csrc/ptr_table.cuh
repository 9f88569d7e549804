// ptr_table.cuh -- host arrays of device pointers copied to the device through
// kernel parameters (no host-to-device copy call, so the enqueue stays
// capturable and needs no pinned staging buffer).
#pragma once

#include <algorithm>
#include <cstring>

#include <cuda_runtime.h>

#include "host_util.h"

namespace eik {

constexpr int PTR_CHUNK = 1024;
struct PtrChunk {
    const void *p[PTR_CHUNK];
};

template <int Unused = 0>
__global__ void k_ptr_upload(const void **dst, const __grid_constant__ PtrChunk c, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = c.p[i];
}

// dst[0 .. n) = src[0 .. n) on stream s; returns the number of launches or a
// negative status.
inline int upload_ptrs(const void **dst, const void *const *src, int n, cudaStream_t s) {
    PtrChunk c;
    int launches = 0;
    for (int off = 0; off < n; off += PTR_CHUNK) {
        const int m = std::min(PTR_CHUNK, n - off);
        memcpy(c.p, src + off, sizeof(void *) * (size_t)m);
        k_ptr_upload<<<(m + 255) / 256, 256, 0, s>>>(dst + off, c, m);
        ++launches;
    }
    const int rc = cuda_check(cudaGetLastError(), "pointer table upload");
    return rc ? rc : launches;
}

}  // namespace eik

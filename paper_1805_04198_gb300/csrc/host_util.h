// host_util.h -- host-side helpers of the libeik C ABI (error text, workspace
// carving, launch checks).
#pragma once

#include <cstdarg>
#include <cstddef>
#include <cstdint>
#include <cstdio>

#include <cuda_runtime.h>

#include "eik.h"

namespace eik {

void set_error(const char *fmt, ...);

// Carves 256-byte aligned sub-buffers out of the caller's workspace.  With a
// null base it only measures.
struct Carver {
    char *base;
    size_t used = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <class X>
    X *take(size_t count) {
        size_t off = (used + 255) & ~(size_t)255;
        used = off + count * sizeof(X);
        return base ? reinterpret_cast<X *>(base + off) : nullptr;
    }
};

// Dynamic shared memory of a kernel, and the preference for the largest
// shared-memory carveout: without it the runtime may pick a carveout that
// holds one CTA of a kernel whose CTAs need just under half an SM's shared
// memory, halving its occupancy.
template <class F>
inline cudaError_t set_dyn_smem(F *func, int bytes) {
    cudaError_t e = cudaFuncSetAttribute((const void *)func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void *)func, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

inline int cuda_check(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        set_error("%s: %s", what, cudaGetErrorString(e));
        return EIK_ECUDA;
    }
    return EIK_OK;
}

// Whether the registers of one CTA of `warps` warps of a kernel fit an SM.  The
// register file is split evenly across the SM's four schedulers and a CTA's
// warps are spread over them, so the busiest scheduler holds ceil(warps / 4)
// warps; registers are allocated per thread in multiples of 8.  (A product
// threads x registers against the whole file accepts CTAs that cannot launch.)
inline bool regs_fit(const cudaFuncAttributes &fa, int warps, int regs_per_sm = 65536) {
    const long long per_warp = (long long)((fa.numRegs + 7) & ~7) * 32;
    return per_warp * ((warps + 3) / 4) <= regs_per_sm / 4;
}

inline bool valid_grid_common(const eik_grid *g, int ndim_required) {
    if (!g) {
        set_error("grid is NULL");
        return false;
    }
    if (g->ndim != ndim_required) {
        set_error("ndim = %d not supported here (need %d)", g->ndim, ndim_required);
        return false;
    }
    if (g->dtype != EIK_F32 && g->dtype != EIK_F64) {
        set_error("dtype %d is neither EIK_F32 nor EIK_F64", g->dtype);
        return false;
    }
    if (!(g->h > 0.0)) {
        set_error("h must be > 0");
        return false;
    }
    for (int a = 0; a < g->ndim; ++a) {
        if (g->n[a] < 2 || g->n[a] > (1 << 20)) {
            set_error("n[%d] = %lld out of range [2, 2^20]", a, (long long)g->n[a]);
            return false;
        }
    }
    if (g->stride[0] != 1) {
        set_error("stride[0] must be 1");
        return false;
    }
    if (g->ndim >= 2 && g->stride[1] < g->n[0]) {
        set_error("stride[1] < n[0]");
        return false;
    }
    if (g->ndim >= 3 && g->stride[2] < g->stride[1] * g->n[1]) {
        set_error("stride[2] < stride[1] * n[1]");
        return false;
    }
    return true;
}

}  // namespace eik

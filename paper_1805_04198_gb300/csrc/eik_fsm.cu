// eik_fsm.cu -- plain fast sweeping method on the whole grid (Sec. 1.1), the
// baseline the domain decomposition is compared against, plus the shared host
// helpers of the C ABI (error text, version).
//
// The grid is one box for the warp-systolic engine: one warp per 32-column
// block, all blocks of the grid in one CTA, sweeps cycling through the four
// orderings until a sweep changes nothing.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "engine.cuh"
#include "host_util.h"

namespace eik {

static thread_local char g_err[512];

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

struct FsmDev {
    unsigned long long sweeps;
    int converged;
    int err;
};

template <class T>
struct FsmArgs {
    const T *r;
    const uint8_t *gamma;
    const T *g;
    T *u;
    long long sy;
    int nx, ny, nb, nstepp;
    T *state;
    T *rsk;
    FsmDev *dev;
    T h;
    long long max_sweeps;
};

template <class T>
struct PlainFsmPolicy {
    T h;
    __device__ __forceinline__ T update(T self, T vmx, T vpx, T vmy, T vpy, const T *sv, uint8_t, int, int,
                                        bool &changed) const {
        const T r = sv[0];
        if (!(r > T(0))) return self;  // Gamma
        const T ut = local_solve2_value(vmx, vpx, vmy, vpy, Num<T>::mul(r, h));
        if (ut < self) {
            changed = true;
            return ut;
        }
        return self;
    }
};

template <class T>
__global__ void k_fsm_pack(FsmArgs<T> A) {
    const size_t total = (size_t)A.nx * A.ny;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        int x = (int)(t % A.nx), y = (int)(t / A.nx);
        const size_t gi = (size_t)y * A.sy + x;
        const bool gam = A.gamma[gi] != 0;
        const T rv = gam ? T(-1) : A.r[gi];
        for (int d = 0; d < 4; ++d) A.rsk[skew_index(d, x, y, A.nb, A.ny, A.nstepp)] = rv;
        // Sec. 1.1 initialisation: Gamma fixed at g, everything else large
        A.state[box_index(x, y, A.ny)] = gam ? A.g[gi] : Num<T>::inf();
    }
}

template <class T>
__global__ void k_fsm_run(FsmArgs<T> A) {
    extern __shared__ __align__(16) char smem[];
    Box<T, 1> bx;
    bx.u = A.state;
    bx.st[0] = A.rsk;
    bx.sb = nullptr;
    bx.nx = A.nx;
    bx.ny = A.ny;
    bx.nb = A.nb;
    bx.nstepp = A.nstepp;
    PlainFsmPolicy<T> pol{A.h};
    long long sweeps;
    bool conv;
    if (threadIdx.x == 0) A.dev->err = 0;
    __syncthreads();
    engine_run<T, 1, false>(bx, pol, A.max_sweeps, smem, sweeps, conv, &A.dev->err);
    if (threadIdx.x == 0) {
        A.dev->sweeps = (unsigned long long)sweeps;
        A.dev->converged = conv ? 1 : 0;
    }
}

template <class T>
__global__ void k_fsm_unpack(FsmArgs<T> A, eik_fsm_stats *out) {
    const size_t total = (size_t)A.nx * A.ny;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        int x = (int)(t % A.nx), y = (int)(t / A.nx);
        A.u[(size_t)y * A.sy + x] = A.state[box_index(x, y, A.ny)];
    }
    if (out && blockIdx.x == 0 && threadIdx.x == 0) {
        out->sweeps = (int64_t)A.dev->sweeps;
        out->converged = A.dev->converged;
        out->error = A.dev->err;
    }
}

struct FsmPlan {
    int nx, ny, nb, nstepp;
    size_t smem, bytes;
};

template <class T>
static size_t fsm_layout(const FsmPlan &P, FsmArgs<T> *A, void *ws) {
    Carver cv(ws);
    T *state = cv.take<T>((size_t)P.nb * P.ny * 32);
    T *rsk = cv.take<T>((size_t)4 * P.nb * P.nstepp * 32);
    FsmDev *dev = cv.take<FsmDev>(1);
    if (A) {
        A->state = state;
        A->rsk = rsk;
        A->dev = dev;
    }
    return cv.used + 256;
}

static bool fsm_plan(const eik_grid *grid, FsmPlan &P) {
    if (!valid_grid_common(grid, 2)) return false;
    P.nx = (int)grid->n[0];
    P.ny = (int)grid->n[1];
    P.nb = ceil32(P.nx);
    P.nstepp = nstep_padded(P.ny);
    P.smem = grid->dtype == EIK_F64 ? engine_smem_bytes<double>(P.nb, P.ny) : engine_smem_bytes<float>(P.nb, P.ny);
    P.bytes = grid->dtype == EIK_F64 ? fsm_layout<double>(P, nullptr, nullptr) : fsm_layout<float>(P, nullptr, nullptr);
    return true;
}

template <class T>
static int fsm_run(const eik_grid *grid, const FsmPlan &P, const void *r, const uint8_t *gamma, const void *g,
                   void *u, int64_t max_sweeps, void *ws, eik_fsm_stats *stats, cudaStream_t s) {
    FsmArgs<T> A;
    memset(&A, 0, sizeof(A));
    A.r = static_cast<const T *>(r);
    A.gamma = gamma;
    A.g = static_cast<const T *>(g);
    A.u = static_cast<T *>(u);
    A.sy = grid->stride[1];
    A.nx = P.nx;
    A.ny = P.ny;
    A.nb = P.nb;
    A.nstepp = P.nstepp;
    A.h = (T)grid->h;
    A.max_sweeps = max_sweeps;
    fsm_layout<T>(P, &A, ws);
    int rc;
    int dev, optin = 0, nsm = 0;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if ((int)P.smem > optin || P.nb > 32) {
        set_error("grid of %d x %d nodes needs %zu bytes of shared memory in one CTA (limit %d)", P.nx, P.ny, P.smem,
                  optin);
        return EIK_EUNSUPPORTED;
    }
    if ((rc = cuda_check(cudaFuncSetAttribute(k_fsm_run<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.smem),
                         "smem attr")))
        return rc;
    const size_t total = (size_t)P.nx * P.ny;
    const int tb = (int)std::min<size_t>((total + 255) / 256, (size_t)nsm * 16);
    k_fsm_pack<T><<<tb, 256, 0, s>>>(A);
    k_fsm_run<T><<<1, 32 * P.nb, P.smem, s>>>(A);
    k_fsm_unpack<T><<<tb, 256, 0, s>>>(A, stats);
    return cuda_check(cudaGetLastError(), "fsm launch");
}

}  // namespace eik

using namespace eik;

extern "C" const char *eik_last_error(void) { return g_err; }

extern "C" int eik_version(void) { return 100; }

extern "C" size_t eik_fsm_workspace_size(const eik_grid *grid) {
    FsmPlan P;
    if (!fsm_plan(grid, P)) return 0;
    return P.bytes;
}

extern "C" int eik_fsm(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g, void *u,
                       int64_t max_sweeps, void *ws, size_t ws_bytes, eik_fsm_stats *stats, void *stream) {
    FsmPlan P;
    if (!fsm_plan(grid, P)) return EIK_EINVAL;
    if (!r || !gamma || !g || !u || !ws) {
        set_error("eik_fsm: NULL array argument");
        return EIK_EINVAL;
    }
    if (max_sweeps < 1) {
        set_error("max_sweeps must be >= 1");
        return EIK_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(ws) & 255) {
        set_error("workspace must be 256-byte aligned");
        return EIK_EINVAL;
    }
    if (ws_bytes < P.bytes) {
        set_error("workspace of %zu bytes is smaller than the %zu required", ws_bytes, P.bytes);
        return EIK_ENOMEM;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (grid->dtype == EIK_F64) return fsm_run<double>(grid, P, r, gamma, g, u, max_sweeps, ws, stats, s);
    return fsm_run<float>(grid, P, r, gamma, g, u, max_sweeps, ws, stats, s);
}

// eik_fsm3.cu -- plain fast sweeping method on a whole 3-D grid (Sec. 1.1),
// the baseline the 3-D domain decomposition is compared against.
//
// Sweep k visits the nodes in ordering k mod 8 of the paper's loop nest (sign
// of x = bit 2, y = bit 1, z = bit 0).  Nodes with equal i + j + k (logical
// indices of the ordering) do not depend on each other, so a sweep is the
// sequence of these hyperplanes, each updated by the whole GPU at once: one
// cooperative kernel, a grid barrier between hyperplanes, the update
// u = min(u, u~) with the 3-D Godunov local solve.  The result is that of the
// serial loop nest.  Sweeps stop after the first one that changes nothing.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "host_util.h"
#include "prof.h"

namespace eik {

EIK_SPIN_LIMIT_SETTER(set_spin_limit_fsm3)

struct Fsm3Dev {
    unsigned long long sweeps;
    int converged;
    int err;
    unsigned bar[4];
    int chg[4];
};

template <class T>
struct Fsm3Args {
    const T *r;
    const uint8_t *gamma;
    const T *g;
    T *u;              // caller's output, strides sy, sz
    long long sy, sz;
    int nx, ny, nz;
    T h;
    T *w;              // work copy [nz][ny][nx]
    Fsm3Dev *dev;
    long long max_sweeps;
    int launches;
};

template <class T>
__global__ void k_fsm3_init(Fsm3Args<T> A) {
    const size_t n = (size_t)A.nx * A.ny * A.nz;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(t % A.nx), y = (int)((t / A.nx) % A.ny), z = (int)(t / ((size_t)A.nx * A.ny));
        const size_t gi = (size_t)z * A.sz + (size_t)y * A.sy + x;
        A.w[t] = A.gamma[gi] ? A.g[gi] : Num<T>::inf();  // Sec. 1.1 initialisation
    }
    if (blockIdx.x == 0 && threadIdx.x < 4) {
        A.dev->bar[threadIdx.x] = 0;
        A.dev->chg[threadIdx.x] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.dev->err = 0;
        A.dev->sweeps = 0;
        A.dev->converged = 0;
    }
}

template <class T>
__global__ void k_fsm3_sweeps(Fsm3Args<T> A) {
    const long long wlim = spin_limit();  // limit of the grid-barrier waits
    const T INF = Num<T>::inf();
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const size_t plane = (size_t)nx * ny;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ndiag = nx + ny + nz - 2;
    __shared__ int blk_ch;
    long long k = 0;
    bool conv = false;
    for (; k < A.max_sweeps; ++k) {
        const int q = (int)(k & 7);
        const int sx = (q & 4) ? 1 : -1, sy = (q & 2) ? 1 : -1, sz = (q & 1) ? 1 : -1;
        if (threadIdx.x == 0) blk_ch = 0;
        bool ch = false;
        for (int dg = 0; dg < ndiag; ++dg) {
            const int ilo = max(0, dg - (ny - 1) - (nz - 1)), ihi = min(nx - 1, dg);
            const long long ncand = (long long)(ihi - ilo + 1) * ny;
            for (long long c = tid; c < ncand; c += nthreads) {
                const int ip = ilo + (int)(c / ny), jp = (int)(c % ny), kp = dg - ip - jp;
                if (kp < 0 || kp >= nz) continue;
                const int x = sx > 0 ? ip : nx - 1 - ip;
                const int y = sy > 0 ? jp : ny - 1 - jp;
                const int z = sz > 0 ? kp : nz - 1 - kp;
                const size_t gi = (size_t)z * A.sz + (size_t)y * A.sy + x;
                if (A.gamma[gi]) continue;
                const size_t t = (size_t)z * plane + (size_t)y * nx + x;
                T vm[3], vp[3];
                vm[0] = x > 0 ? A.w[t - 1] : INF;
                vp[0] = x + 1 < nx ? A.w[t + 1] : INF;
                vm[1] = y > 0 ? A.w[t - nx] : INF;
                vp[1] = y + 1 < ny ? A.w[t + nx] : INF;
                vm[2] = z > 0 ? A.w[t - plane] : INF;
                vp[2] = z + 1 < nz ? A.w[t + plane] : INF;
                uint8_t wd;
                const T ut = local_solve3(vm, vp, Num<T>::mul(A.r[gi], A.h), wd);
                if (ut < A.w[t]) {
                    A.w[t] = ut;
                    ch = true;
                }
            }
            if (!grid_barrier(A.dev->bar, &A.dev->err, wlim)) return;
        }
        // sweep k changed something?  slot k % 3, cleared two sweeps ahead
        if (ch) blk_ch = 1;
        __syncthreads();
        if (threadIdx.x == 0 && blk_ch) atomicOr(&A.dev->chg[k % 3], 1);
        if (!grid_barrier(A.dev->bar, &A.dev->err, wlim)) return;
        const int any = *(volatile int *)&A.dev->chg[k % 3];
        if (blockIdx.x == 0 && threadIdx.x == 0) A.dev->chg[(k + 2) % 3] = 0;
        if (!any) {
            conv = true;
            ++k;
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.dev->sweeps = (unsigned long long)(conv ? k : A.max_sweeps);
        A.dev->converged = conv ? 1 : 0;
    }
}

template <class T>
__global__ void k_fsm3_out(Fsm3Args<T> A, eik_fsm_stats *out) {
    const size_t n = (size_t)A.nx * A.ny * A.nz;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(t % A.nx), y = (int)((t / A.nx) % A.ny), z = (int)(t / ((size_t)A.nx * A.ny));
        A.u[(size_t)z * A.sz + (size_t)y * A.sy + x] = A.w[t];
    }
    if (out && blockIdx.x == 0 && threadIdx.x == 0) {
        out->sweeps = (int64_t)A.dev->sweeps;
        out->converged = A.dev->converged;
        out->error = A.dev->err;
        out->updates = (int64_t)A.dev->sweeps * A.nx * A.ny * A.nz;
        out->launches = A.launches;
    }
}

size_t fsm3_workspace_size(const eik_grid *grid) {
    Carver cv(nullptr);
    cv.take<double>((size_t)grid->n[0] * grid->n[1] * grid->n[2]);
    cv.take<Fsm3Dev>(1);
    return cv.used + 256;
}

template <class T>
static int fsm3_run_t(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g, void *u,
                      int64_t max_sweeps, void *ws, eik_fsm_stats *stats, cudaStream_t s) {
    Fsm3Args<T> A;
    memset(&A, 0, sizeof(A));
    A.r = static_cast<const T *>(r);
    A.gamma = gamma;
    A.g = static_cast<const T *>(g);
    A.u = static_cast<T *>(u);
    A.sy = grid->stride[1];
    A.sz = grid->stride[2];
    A.nx = (int)grid->n[0];
    A.ny = (int)grid->n[1];
    A.nz = (int)grid->n[2];
    A.h = (T)grid->h;
    A.max_sweeps = max_sweeps;
    Carver cv(ws);
    A.w = cv.take<T>((size_t)A.nx * A.ny * A.nz);
    A.dev = cv.take<Fsm3Dev>(1);
    A.launches = 3;
    int rc, dev, nsm = 0;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 512;
    int per_sm = 0;
    if ((rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fsm3_sweeps<T>, threads, 0),
                         "occupancy")))
        return rc;
    // one or two CTAs per SM keep the grid barrier short
    const int blocks = std::max(1, std::min(per_sm, 2) * nsm);
    const size_t n = (size_t)A.nx * A.ny * A.nz;
    const int eb = (int)std::min<size_t>((n + 255) / 256, (size_t)nsm * 16);
    EIK_LAUNCH("fsm3_init", s, k_fsm3_init<T><<<eb, 256, 0, s>>>(A));
    void *args[] = {&A};
    int tok = prof_begin("fsm3_sweeps", s);
    rc = cuda_check(cudaLaunchCooperativeKernel((void *)k_fsm3_sweeps<T>, blocks, threads, args, 0, s),
                    "fsm3 cooperative launch");
    prof_end(tok, s);
    if (rc) return rc;
    EIK_LAUNCH("fsm3_out", s, k_fsm3_out<T><<<eb, 256, 0, s>>>(A, stats));
    return cuda_check(cudaGetLastError(), "fsm3 launch");
}

int fsm3_run(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g, void *u, int64_t max_sweeps,
             void *ws, eik_fsm_stats *stats, cudaStream_t s) {
    if (grid->dtype == EIK_F64) return fsm3_run_t<double>(grid, r, gamma, g, u, max_sweeps, ws, stats, s);
    return fsm3_run_t<float>(grid, r, gamma, g, u, max_sweeps, ws, stats, s);
}

}  // namespace eik

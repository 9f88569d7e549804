// eik_dd.cu -- two-scale domain decomposition (Sec. 3.2, Steps 1-4, Alg. 1-5)
// on one GPU, 2-D.
//
// Per parareal iteration k the device runs, on one stream:
//   k_fine   one CTA per subdomain: Step 2 boundary data from (U, W), Step 3
//            FSM sweeps by the warp-systolic engine, then the Alg. 3 winds of
//            the converged state at the subdomain's coarse-set nodes (written
//            as per-subdomain copies) and the fine values of interior nodes;
//   k_alg4   one thread per coarse-set node: Alg. 4 choice among the copies
//            -> u^k, w^k; the skewed per-direction inputs of Alg. 5 (u^k,
//            agreement mask, C_H(nbrs U^k)), U^k for the delta, W = w^k;
//   k_check  stop test (k == max_iter, or k >= 1 and max|U^k - U^{k-1}| < tol);
//   k_step4  one CTA per shifted coarse grid: reset, Alg. 5 sweeps by the
//            same engine;
//   k_causal cooperative: Alg. 2 along every coarse line to its least fixed
//            point (segmented max-scans, rounds until nothing changes);
//   k_delta  max|U^{k+1} - U^k| over the coarse set.
// Every kernel returns at once when the device flag `done` is set, so the
// host enqueues max_iter + 1 iterations without reading anything back.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "dd2_device.cuh"
#include "dd2_host.cuh"
#include "host_util.h"
#include "prof.h"

namespace eik {

EIK_SPIN_LIMIT_SETTER(set_spin_limit_dd)

// Kernel entry points.  Register caps keep two 9-warp subdomain CTAs per SM in
// FP32 and let a 9-warp CTA fit the register file in FP64 (it is split across
// the SM's four schedulers, 16 K registers each, and 3 of the 9 warps share
// one: at most 168 registers a thread).
#define EIK_KERNEL_PAIR(name, RF, RD)                                                  \
    __global__ void __maxnreg__(RF) name##_f32(DDArgs<float> A) {                     \
        extern __shared__ __align__(16) char smem[];                                  \
        name##_body<float>(A, smem, blockIdx.x);                                      \
    }                                                                                 \
    __global__ void __maxnreg__(RD) name##_f64(DDArgs<double> A) {                    \
        extern __shared__ __align__(16) char smem[];                                  \
        name##_body<double>(A, smem, blockIdx.x);                                     \
    }
EIK_KERNEL_PAIR(k_step1, 96, 168)
EIK_KERNEL_PAIR(k_step4, 160, 168)
EIK_KERNEL_PAIR(k_step4a, 160, 168)

// Planning pass of a subdomain launch over tiles [t0, t0 + ntl): which
// subdomains' Step 2 data changed since their previous solve in this call
// (tile_needs_solve, which also records the new data).  Those are listed
// first in A.order, the rest after them, so that the CTAs with work are the
// lowest-numbered ones and are spread one per SM while they are at most as
// many as the SMs.  The order is the atomics' and does not matter: the
// subdomain solves are independent.
template <class T>
__global__ void k_fine_plan(DDArgs<T> A, int t0, int ntl) {
    if (*A.done) return;
    const int tile = t0 + blockIdx.x;
    const bool need = tile_needs_solve(A, tile);
    if (threadIdx.x == 0) {
        if (need) {
            A.order[atomicAdd(A.order_cnt, 1)] = tile;
        } else {
            A.order[ntl - 1 - atomicAdd(A.order_cnt + 1, 1)] = tile;
            atomicAdd(&A.st->fine_skips, 1ull);
        }
    }
}

// Subdomain kernel: with a plan, CTA b solves subdomain A.order[b] when b is
// below the count of subdomains that need a solve; without one, CTA b
// solves subdomain A.tile0 + b if its data changed.
template <class T>
__device__ __forceinline__ void k_fine_entry(const DDArgs<T> &A, char *smem) {
    if (!A.order) {
        k_fine_body<T>(A, smem, A.tile0 + blockIdx.x);
        return;
    }
    if (*A.done || (int)blockIdx.x >= *(volatile const int *)A.order_cnt) return;
    k_fine_body<T>(A, smem, A.order[blockIdx.x], false);
}
__global__ void __maxnreg__(96) k_fine_f32(DDArgs<float> A) {
    extern __shared__ __align__(16) char smem[];
    k_fine_entry<float>(A, smem);
}
__global__ void __maxnreg__(168) k_fine_f64(DDArgs<double> A) {
    extern __shared__ __align__(16) char smem[];
    k_fine_entry<double>(A, smem);
}

template <class T> struct DDKernels;
template <> struct DDKernels<float> {
    static constexpr void (*step1)(DDArgs<float>) = k_step1_f32;
    static constexpr void (*step4)(DDArgs<float>) = k_step4_f32;
    static constexpr void (*step4a)(DDArgs<float>) = k_step4a_f32;
    static constexpr void (*fine)(DDArgs<float>) = k_fine_f32;
};
template <> struct DDKernels<double> {
    static constexpr void (*step1)(DDArgs<double>) = k_step1_f64;
    static constexpr void (*step4)(DDArgs<double>) = k_step4_f64;
    static constexpr void (*step4a)(DDArgs<double>) = k_step4a_f64;
    static constexpr void (*fine)(DDArgs<double>) = k_fine_f64;
};

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------
// 3-D implementation (eik_dd3.cu)
size_t dd3_workspace_size(const eik_grid *grid, const eik_dd_params *p);
bool dd3_validate(const eik_grid *grid, const eik_dd_params *p);
int dd3_run(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g, const eik_dd_params *p,
            void *u_out, void *ws, eik_dd_stats *stats, cudaStream_t s);
// 1-D implementation (eik_dd1.cu)
bool dd1_validate(const eik_grid *grid, const eik_dd_params *p);
size_t dd1_workspace_size(const eik_grid *grid, const eik_dd_params *p);
int dd1_run(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g, const eik_dd_params *p,
            void *u_out, void *ws, eik_dd_stats *stats, cudaStream_t s);

// Parameters of the per-node weight of Sec. 4.2 (2-D and 3-D).
static bool valid_adaptive(const eik_dd_params *p) {
    if (!p->theta_adaptive) return true;
    const double w = p->omega[0] + p->omega[1] + p->omega[2];
    bool ok = std::isfinite(p->sig_delta) && std::isfinite(p->sig_x0) && std::isfinite(p->theta_cap) &&
              p->sig_gamma > 0.0 && std::isfinite(p->sig_gamma) && w > 0.0 && std::isfinite(w);
    for (int s2 = 0; s2 < 3; ++s2) ok = ok && p->omega[s2] >= 0.0;
    if (!ok)
        set_error("adaptive theta: omega must be >= 0 with a positive finite sum, sig_gamma > 0, "
                  "sig_delta, sig_x0 and theta_cap finite");
    return ok;
}

bool dd_validate(const eik_grid *grid, const eik_dd_params *p) {
    if (!p) {
        set_error("params is NULL");
        return false;
    }
    if (grid && grid->ndim == 1) return dd1_validate(grid, p);
    if (grid && grid->ndim == 3) {
        if (!valid_grid_common(grid, 3)) return false;
        if (p->max_iter < 0 || p->max_iter > 100000 || p->max_fsm_sweeps < 1 || p->max_coarse_sweeps < 1 ||
            p->max_fsm_sweeps > MAX_SWEEPS || p->max_coarse_sweeps > MAX_SWEEPS || !std::isfinite(p->theta)) {
            set_error("max_iter must be in [0, 100000], sweep caps in [1, %lld], theta finite", MAX_SWEEPS);
            return false;
        }
        return valid_adaptive(p) && dd3_validate(grid, p);
    }
    if (!valid_grid_common(grid, 2)) return false;
    for (int a = 0; a < 2; ++a) {
        if (p->tiles[a] < 1 || (grid->n[a] - 1) % p->tiles[a] != 0) {
            set_error("tiles[%d] = %d does not divide n[%d]-1 = %lld", a, p->tiles[a], a, (long long)(grid->n[a] - 1));
            return false;
        }
    }
    const int c = p->coarse_ratio;
    if (c < 1) {
        set_error("coarse_ratio must be >= 1");
        return false;
    }
    for (int a = 0; a < 2; ++a) {
        long long S = (grid->n[a] - 1) / p->tiles[a];
        if (S % c != 0) {
            set_error("coarse_ratio %d does not divide the subdomain width %lld", c, S);
            return false;
        }
        if (S + 1 > 1024) {
            set_error("subdomain of %lld nodes per side exceeds 1024", S + 1);
            return false;
        }
        if ((grid->n[a] - 1) / c + 1 > 1024) {
            set_error("coarse grid of %lld nodes per side exceeds 1024", (long long)((grid->n[a] - 1) / c + 1));
            return false;
        }
    }
    if (p->max_iter < 0 || p->max_iter > 100000 || p->max_fsm_sweeps < 1 || p->max_coarse_sweeps < 1 ||
        p->max_fsm_sweeps > MAX_SWEEPS || p->max_coarse_sweeps > MAX_SWEEPS) {
        set_error("max_iter must be in [0, 100000] and sweep caps in [1, %lld]", MAX_SWEEPS);
        return false;
    }
    if (!(std::isfinite(p->theta))) {
        set_error("theta must be finite");
        return false;
    }
    return valid_adaptive(p);
}

// One 2-D DD solve on one stream, in phases: set-up, start (statistics, packed
// statics, Step 1 and its causal sweep), the subdomain solves of a range of
// subdomains (Steps 2-3), the coarse phase of an iteration (Alg. 4, the stop
// test, Step 4, the causal sweep, the update size) and the statistics.  The
// single solve runs them back to back; a sharded solve runs the subdomain
// phase on its own subdomains only and exchanges their copies in between.
template <class T>
struct DDSolve {
    DDPlan P;
    DDArgs<T> A;
    CausalShape cs;
    cudaStream_t s = nullptr;
    int nsm = 0, ew = 256, eb = 0, tb = 0, ntiles = 0, fine_threads = 0;
    size_t fine_smem = 0;
    void (*step4k)(DDArgs<T>) = nullptr;
    long long nl = 0;  // launches made

    int setup(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g, const eik_dd_params *p,
              void *u_out, void *ws, cudaStream_t stream) {
        s = stream;
        P = dd_plan(grid, p);
        memset(&A, 0, sizeof(A));
        A.G = P.G;
        A.r = static_cast<const T *>(r);
        A.gamma = gamma;
        A.g = static_cast<const T *>(g);
        A.u_out = static_cast<T *>(u_out);
        A.sy = grid->stride[1];
        dd_layout<T>(P, &A, ws, p->max_iter);
        A.theta = (T)p->theta;
        A.step4_identity = (!P.adaptive && p->theta == 0.0) ? 1 : 0;
        A.tol = (T)p->tol;
        A.max_iter = p->max_iter;
        A.max_fsm = p->max_fsm_sweeps;
        A.max_coarse = p->max_coarse_sweeps;
        A.adaptive = P.adaptive ? 1 : 0;
        for (int s2 = 0; s2 < 3; ++s2) A.om[s2] = p->omega[s2];
        A.sg = p->sig_gamma;
        A.sd = p->sig_delta;
        A.sx0 = p->sig_x0;
        A.cap = p->theta_cap;
        const DDGeom &G = P.G;
        ntiles = G.tx * G.ty;

        int rc, dev;
        if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
        if ((rc = cuda_check(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "attr"))) return rc;
        int smem_optin = 0;
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        fine_threads = 32 * G.tnb;
        fine_smem = P.fine_smem;
        if ((int)fine_smem > smem_optin || (int)P.step1_smem > smem_optin || (int)P.step4_smem > smem_optin) {
            set_error("shared memory need (%zu, %zu, %zu) exceeds the device limit %d", fine_smem, P.step1_smem,
                      P.step4_smem, smem_optin);
            return EIK_EUNSUPPORTED;
        }
        if ((rc = cuda_check(set_dyn_smem(DDKernels<T>::fine, (int)fine_smem), "smem attr fine")))
            return rc;
        if ((rc = cuda_check(set_dyn_smem(DDKernels<T>::step1, (int)P.step1_smem), "smem attr step1")))
            return rc;
        step4k = P.adaptive ? DDKernels<T>::step4a : DDKernels<T>::step4;
        if ((rc = cuda_check(set_dyn_smem(step4k, (int)P.step4_smem), "smem attr step4")))
            return rc;
        // causal sweep: cooperative grid sized to what is co-resident
        if ((rc = causal_shape<T>((const void *)k_causal<T>, std::max(G.nx, G.ny), std::max(G.ncx, G.ncy) + 1, nsm,
                                  smem_optin, cs)))
            return rc;
        eb = (int)std::min<size_t>((G.coarse_elems + ew - 1) / ew, (size_t)nsm * 8);
        const size_t tiles_nodes = (size_t)ntiles * G.tnx * G.tny;
        tb = (int)std::min<size_t>((tiles_nodes + ew - 1) / ew, (size_t)nsm * 16);
        return EIK_OK;
    }

    int causal(int only_if_not_done) {
        void *args[] = {&A, &only_if_not_done, &cs.lw};
        int tok = prof_begin("dd_causal_sweep", s);
        int rc = cuda_check(cudaLaunchCooperativeKernel((void *)k_causal<T>, cs.blocks, cs.threads, args, cs.smem, s),
                            "causal launch");
        prof_end(tok, s);
        ++nl;
        return rc;
    }

    int start() {
        const DDGeom &G = P.G;
        EIK_LAUNCH("dd_init", s, k_init_stats<T><<<1, 256, 0, s>>>(A)); ++nl;
        EIK_LAUNCH("dd_pack_tiles", s, k_pack_tiles<T><<<tb, ew, 0, s>>>(A)); ++nl;
        EIK_LAUNCH("dd_pack_coarse", s, k_pack_coarse<T><<<eb, ew, 0, s>>>(A)); ++nl;
        EIK_LAUNCH("dd_step1_coarse_fsm", s, DDKernels<T>::step1<<<G.ngrids, P.grid_threads, P.step1_smem, s>>>(A));
        ++nl;
        return causal(0);
    }

    // Steps 2-3 on subdomains [t0, t1)
    int fine(int t0, int t1) {
        if (t1 <= t0) return EIK_OK;
        EIK_LAUNCH("dd_fine_plan", s, k_fine_plan<T><<<t1 - t0, 256, 0, s>>>(A, t0, t1 - t0)); ++nl;
        EIK_LAUNCH("dd_fine_subdomains", s, DDKernels<T>::fine<<<t1 - t0, fine_threads, fine_smem, s>>>(A)); ++nl;
        return EIK_OK;
    }

    // copies of subdomains [t0, t1) to (pack) or from (unpack) their records
    int records(int t0, int t1, void *xbuf, int pack) {
        if (t1 <= t0) return EIK_OK;
        const size_t nodes = (size_t)(t1 - t0) * P.G.tnx * P.G.tny;
        const int nb = (int)std::min<size_t>((nodes + ew - 1) / ew, (size_t)nsm * 16);
        EIK_LAUNCH(pack ? "dd_shard_pack" : "dd_shard_unpack", s,
                   k_shard_records<T><<<nb, ew, 0, s>>>(A, t0, t1, static_cast<unsigned char *>(xbuf), pack));
        ++nl;
        return EIK_OK;
    }

    // Alg. 4 and the stop test of iteration k, then (k < max_iter) Step 4, the
    // causal sweep and the size of the coarse update
    int coarse(int k) {
        EIK_LAUNCH("dd_alg4_restrict", s, k_alg4<T><<<eb, ew, 0, s>>>(A, k)); ++nl;
        EIK_LAUNCH("dd_check", s, k_check<T><<<1, 1, 0, s>>>(A, k)); ++nl;
        if (k == A.max_iter) return EIK_OK;
        if (!A.step4_identity) {
            EIK_LAUNCH("dd_step4_weighted", s, step4k<<<P.G.ngrids, P.grid_threads, P.step4_smem, s>>>(A));
            ++nl;
        }
        int rc = causal(1);
        if (rc) return rc;
        EIK_LAUNCH("dd_delta", s, k_delta<T><<<eb, ew, 0, s>>>(A, k)); ++nl;
        return EIK_OK;
    }

    int finish(eik_dd_stats *stats) {
        ++nl;
        EIK_LAUNCH("dd_finalize", s, k_finalize<T><<<1, 32, 0, s>>>(A, stats, nl));
        return cuda_check(cudaGetLastError(), "dd launch");
    }
};

template <class T>
static int dd_run(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                  const eik_dd_params *p, void *u_out, void *ws, eik_dd_stats *stats, cudaStream_t s) {
    DDSolve<T> D;
    int rc = D.setup(grid, r, gamma, g, p, u_out, ws, s);
    if (!rc) rc = D.start();
    for (int k = 0; !rc && k <= p->max_iter; ++k) {
        rc = D.fine(0, D.ntiles);
        if (!rc) rc = D.coarse(k);
    }
    if (rc) return rc;
    return D.finish(stats);
}

}  // namespace eik

using namespace eik;

extern "C" size_t eik_dd_workspace_size(const eik_grid *grid, const eik_dd_params *params) {
    if (!dd_validate(grid, params)) return 0;
    if (grid->ndim == 1) return dd1_workspace_size(grid, params);
    if (grid->ndim == 3) return dd3_workspace_size(grid, params);
    return dd_plan(grid, params).bytes;
}

extern "C" int eik_dd_solve(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                            const eik_dd_params *params, void *u_out, void *ws, size_t ws_bytes, eik_dd_stats *stats,
                            void *stream) {
    if (!dd_validate(grid, params)) return EIK_EINVAL;
    if (!r || !gamma || !g || !u_out || !ws) {
        set_error("eik_dd_solve: NULL array argument");
        return EIK_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(ws) & 255) {
        set_error("workspace must be 256-byte aligned");
        return EIK_EINVAL;
    }
    const size_t need = grid->ndim == 1   ? dd1_workspace_size(grid, params)
                        : grid->ndim == 3 ? dd3_workspace_size(grid, params)
                                          : dd_plan(grid, params).bytes;
    if (ws_bytes < need) {
        set_error("workspace of %zu bytes is smaller than the %zu required", ws_bytes, need);
        return EIK_ENOMEM;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (grid->ndim == 1) return dd1_run(grid, r, gamma, g, params, u_out, ws, stats, s);
    if (grid->ndim == 3) return dd3_run(grid, r, gamma, g, params, u_out, ws, stats, s);
    if (grid->dtype == EIK_F64) return dd_run<double>(grid, r, gamma, g, params, u_out, ws, stats, s);
    return dd_run<float>(grid, r, gamma, g, params, u_out, ws, stats, s);
}

// --------------------------------------------------------------------------
// Read-back of the coarse state (U, W) of the last iteration of a 2-D solve,
// scattered from the workspace's coarse layout to fine indexing.
// --------------------------------------------------------------------------
namespace eik {

template <class T>
__global__ void k_coarse_state(DDGeom G, const T *U, const uint8_t *W, T *U_out, uint8_t *W_out, long long sy) {
    const long long n = (long long)G.nx * G.ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(e % G.nx), Y = (int)(e / G.nx);
        if (!in_coarse_set(G, X, Y)) continue;
        const size_t ca = coarse_addr(G, X, Y);
        if (U_out) U_out[(size_t)Y * sy + X] = U[ca];
        if (W_out) W_out[(size_t)Y * sy + X] = (uint8_t)(W[ca] & ~WIND_ECHO);
    }
}

template <class T>
static int coarse_state_t(const eik_grid *grid, const eik_dd_params *p, const void *ws, void *U_out, uint8_t *W_out,
                          cudaStream_t s) {
    const DDPlan P = dd_plan(grid, p);
    DDArgs<T> A;
    memset(&A, 0, sizeof(A));
    dd_layout<T>(P, &A, const_cast<void *>(ws), p->max_iter);
    int dev, nsm = 0;
    int rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    EIK_LAUNCH("dd_coarse_state", s,
               k_coarse_state<T><<<4 * nsm, 256, 0, s>>>(P.G, A.U, A.W, static_cast<T *>(U_out), W_out,
                                                          grid->stride[1]));
    return cuda_check(cudaGetLastError(), "coarse state launch");
}

}  // namespace eik

extern "C" int eik_dd_coarse_state(const eik_grid *grid, const eik_dd_params *params, const void *ws,
                                   size_t ws_bytes, void *U_out, uint8_t *W_out, void *stream) {
    if (!dd_validate(grid, params)) return EIK_EINVAL;
    if (grid->ndim != 2) {
        set_error("eik_dd_coarse_state: 2-D solves only");
        return EIK_EUNSUPPORTED;
    }
    if (!ws || (!U_out && !W_out) || (reinterpret_cast<uintptr_t>(ws) & 255)) {
        set_error("eik_dd_coarse_state: NULL or unaligned argument");
        return EIK_EINVAL;
    }
    if (ws_bytes < dd_plan(grid, params).bytes) {
        set_error("workspace of %zu bytes is smaller than the solve's", ws_bytes);
        return EIK_ENOMEM;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (grid->dtype == EIK_F64) return coarse_state_t<double>(grid, params, ws, U_out, W_out, s);
    return coarse_state_t<float>(grid, params, ws, U_out, W_out, s);
}

// --------------------------------------------------------------------------
// Sharded 2-D solve: phases of eik_dd_solve for callers that split the
// subdomain solves over several processes (slabs of subdomain rows) and keep
// the coarse state replicated.
// --------------------------------------------------------------------------
namespace eik {

static int shard_check(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                       const eik_dd_params *params, void *u_out, void *ws, size_t ws_bytes) {
    if (!dd_validate(grid, params)) return EIK_EINVAL;
    if (grid->ndim != 2) {
        set_error("the sharded solve is built for 2-D grids");
        return EIK_EUNSUPPORTED;
    }
    if (!r || !gamma || !g || !u_out || !ws) {
        set_error("NULL array argument");
        return EIK_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(ws) & 255) {
        set_error("workspace must be 256-byte aligned");
        return EIK_EINVAL;
    }
    const size_t need = dd_plan(grid, params).bytes;
    if (ws_bytes < need) {
        set_error("workspace of %zu bytes is smaller than the %zu required", ws_bytes, need);
        return EIK_ENOMEM;
    }
    return EIK_OK;
}

template <class T>
static int shard_phase(int phase, const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                       const eik_dd_params *p, void *u_out, void *ws, int a, int b, void *xbuf,
                       eik_dd_stats *stats, cudaStream_t s) {
    DDSolve<T> D;
    int rc = D.setup(grid, r, gamma, g, p, u_out, ws, s);
    if (rc) return rc;
    const int tx = D.P.G.tx;
    switch (phase) {
        case 0: rc = D.start(); break;
        case 1:  // Steps 2-3 on subdomain rows [a, b), their copies into their records
            rc = D.fine(a * tx, b * tx);
            if (!rc) rc = D.records(a * tx, b * tx, xbuf, 1);
            break;
        default:  // every record into the copies, then the coarse phase of iteration a
            rc = D.records(0, D.ntiles, xbuf, 0);
            if (!rc) rc = D.coarse(a);
            if (!rc && stats) rc = D.finish(stats);
            break;
    }
    if (rc) return rc;
    return cuda_check(cudaGetLastError(), "dd shard launch");
}

static int shard_dispatch(int phase, const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                          const eik_dd_params *p, void *u_out, void *ws, int a, int b, void *xbuf,
                          eik_dd_stats *stats, void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (grid->dtype == EIK_F64) return shard_phase<double>(phase, grid, r, gamma, g, p, u_out, ws, a, b, xbuf, stats, s);
    return shard_phase<float>(phase, grid, r, gamma, g, p, u_out, ws, a, b, xbuf, stats, s);
}

}  // namespace eik

extern "C" size_t eik_dd_shard_exchange_bytes(const eik_grid *grid, const eik_dd_params *params,
                                              size_t *record_bytes) {
    if (!dd_validate(grid, params)) return 0;
    if (grid->ndim != 2) {
        set_error("the sharded solve is built for 2-D grids");
        return 0;
    }
    const DDGeom G = dd_plan(grid, params).G;
    const size_t rec = grid->dtype == EIK_F64 ? tile_record_bytes<double>(G) : tile_record_bytes<float>(G);
    if (record_bytes) *record_bytes = rec;
    return rec * (size_t)G.tx * G.ty;
}

extern "C" int eik_dd_shard_start(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                                  const eik_dd_params *params, void *u_out, void *ws, size_t ws_bytes, void *stream) {
    int rc = shard_check(grid, r, gamma, g, params, u_out, ws, ws_bytes);
    if (rc) return rc;
    return shard_dispatch(0, grid, r, gamma, g, params, u_out, ws, 0, 0, nullptr, nullptr, stream);
}

extern "C" int eik_dd_shard_fine(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                                 const eik_dd_params *params, void *u_out, void *ws, size_t ws_bytes, int row0,
                                 int row1, void *xbuf, void *stream) {
    int rc = shard_check(grid, r, gamma, g, params, u_out, ws, ws_bytes);
    if (rc) return rc;
    if (row0 < 0 || row1 < row0 || row1 > params->tiles[1]) {
        set_error("subdomain rows [%d, %d) outside [0, %d]", row0, row1, params->tiles[1]);
        return EIK_EINVAL;
    }
    if (!xbuf || (reinterpret_cast<uintptr_t>(xbuf) & 15)) {
        set_error("exchange buffer must be non-NULL and 16-byte aligned");
        return EIK_EINVAL;
    }
    return shard_dispatch(1, grid, r, gamma, g, params, u_out, ws, row0, row1, xbuf, nullptr, stream);
}

extern "C" int eik_dd_shard_coarse(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                                   const eik_dd_params *params, void *u_out, void *ws, size_t ws_bytes, int k,
                                   const void *xbuf, eik_dd_stats *stats, void *stream) {
    int rc = shard_check(grid, r, gamma, g, params, u_out, ws, ws_bytes);
    if (rc) return rc;
    if (k < 0 || k > params->max_iter) {
        set_error("iteration %d outside [0, max_iter = %d]", k, params->max_iter);
        return EIK_EINVAL;
    }
    if (!xbuf || (reinterpret_cast<uintptr_t>(xbuf) & 15)) {
        set_error("exchange buffer must be non-NULL and 16-byte aligned");
        return EIK_EINVAL;
    }
    return shard_dispatch(2, grid, r, gamma, g, params, u_out, ws, k, 0, const_cast<void *>(xbuf), stats, stream);
}

// --------------------------------------------------------------------------
// Entry point that allocates nothing: the DD workspace lives in a file-scope
// device array instead of caller memory.
//
// Some callers cannot call cudaMalloc at all: hosts whose allocator is owned
// by another runtime that must not be bypassed, and real-time loops that
// forbid allocation after start-up.  For them the scratch
// is a static __device__ array of EIK_NOALLOC_SCRATCH_BYTES (32 MiB), which
// every GPU that loads this library keeps until the process exits.
// --------------------------------------------------------------------------
#include <mutex>

namespace eik {

static __device__ __align__(256) unsigned char g_dd_scratch[EIK_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
static void *g_scratch_ptr[MAX_DEVICES];
static std::mutex g_scratch_mu;

// Device address of g_dd_scratch on the current device, looked up once per
// device (the host-side name of the array is only a stand-in for it).
static int scratch_address(void **out) {
    int dev = 0;
    int rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if (dev < 0 || dev >= MAX_DEVICES) {
        set_error("device index %d beyond the %d devices this entry point supports", dev, MAX_DEVICES);
        return EIK_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        rc = cuda_check(cudaGetSymbolAddress(&p, g_dd_scratch), "cudaGetSymbolAddress(scratch)");
        if (rc) return rc;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return EIK_OK;
}

}  // namespace eik

extern "C" int eik_dd_solve_noalloc(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                                    const eik_dd_params *params, void *u_out, eik_dd_stats *stats, void *stream) {
    const size_t need = eik_dd_workspace_size(grid, params);
    if (need == 0) return EIK_EINVAL;
    if (need > (size_t)EIK_NOALLOC_SCRATCH_BYTES) {
        set_error("eik_dd_solve_noalloc: problem needs %zu bytes of scratch, the static scratch holds %zu; "
                  "use eik_dd_solve with a caller workspace",
                  need, (size_t)EIK_NOALLOC_SCRATCH_BYTES);
        return EIK_ENOMEM;
    }
    void *ws = nullptr;
    const int rc = scratch_address(&ws);
    if (rc) return rc;
    // The workspace needs no clearing: every word the solve reads is written
    // earlier in the same solve (the statistics and control words included).
    return eik_dd_solve(grid, r, gamma, g, params, u_out, ws, (size_t)EIK_NOALLOC_SCRATCH_BYTES, stats, stream);
}

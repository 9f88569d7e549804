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
EIK_KERNEL_PAIR(k_fine, 96, 168)

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

template <class T>
static int dd_run(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                  const eik_dd_params *p, void *u_out, void *ws, eik_dd_stats *stats, cudaStream_t s) {
    DDPlan P = dd_plan(grid, p);
    DDArgs<T> A;
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
    const int ntiles = G.tx * G.ty;

    int rc;
    int dev;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    int nsm = 0;
    if ((rc = cuda_check(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "attr"))) return rc;
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    auto finek = DDKernels<T>::fine;
    const int fine_threads = 32 * G.tnb;
    const size_t fine_smem = P.fine_smem;
    if ((int)fine_smem > smem_optin || (int)P.step1_smem > smem_optin || (int)P.step4_smem > smem_optin) {
        set_error("shared memory need (%zu, %zu, %zu) exceeds the device limit %d", fine_smem, P.step1_smem,
                  P.step4_smem, smem_optin);
        return EIK_EUNSUPPORTED;
    }
    if ((rc = cuda_check(cudaFuncSetAttribute(finek, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fine_smem),
                         "smem attr fine")))
        return rc;
    if ((rc = cuda_check(cudaFuncSetAttribute(DDKernels<T>::step1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.step1_smem),
                         "smem attr step1")))
        return rc;
    auto step4k = P.adaptive ? DDKernels<T>::step4a : DDKernels<T>::step4;
    if ((rc = cuda_check(cudaFuncSetAttribute(step4k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.step4_smem),
                         "smem attr step4")))
        return rc;
    // causal sweep: cooperative grid sized to what is co-resident
    CausalShape cs;
    if ((rc = causal_shape<T>((const void *)k_causal<T>, std::max(G.nx, G.ny), std::max(G.ncx, G.ncy) + 1, nsm,
                              smem_optin, cs)))
        return rc;

    const int ew = 256;
    const int eb = (int)std::min<size_t>((G.coarse_elems + ew - 1) / ew, (size_t)nsm * 8);
    const size_t tiles_nodes = (size_t)ntiles * G.tnx * G.tny;
    const int tb = (int)std::min<size_t>((tiles_nodes + ew - 1) / ew, (size_t)nsm * 16);

    long long nl = 0;
    EIK_LAUNCH("dd_init", s, k_init_stats<T><<<1, 256, 0, s>>>(A)); ++nl;
    EIK_LAUNCH("dd_pack_tiles", s, k_pack_tiles<T><<<tb, ew, 0, s>>>(A)); ++nl;
    EIK_LAUNCH("dd_pack_coarse", s, k_pack_coarse<T><<<eb, ew, 0, s>>>(A)); ++nl;
    EIK_LAUNCH("dd_step1_coarse_fsm", s, DDKernels<T>::step1<<<G.ngrids, P.grid_threads, P.step1_smem, s>>>(A)); ++nl;
    auto launch_causal = [&](int only) -> int {
        void *args[] = {&A, &only, &cs.lw};
        int tok = prof_begin("dd_causal_sweep", s);
        int r2 = cuda_check(cudaLaunchCooperativeKernel((void *)k_causal<T>, cs.blocks, cs.threads, args, cs.smem, s),
                            "causal launch");
        prof_end(tok, s);
        ++nl;
        return r2;
    };
    if ((rc = launch_causal(0))) return rc;
    for (int k = 0; k <= p->max_iter; ++k) {
        EIK_LAUNCH("dd_fine_subdomains", s, finek<<<ntiles, fine_threads, fine_smem, s>>>(A)); ++nl;
        EIK_LAUNCH("dd_alg4_restrict", s, k_alg4<T><<<eb, ew, 0, s>>>(A, k)); ++nl;
        EIK_LAUNCH("dd_check", s, k_check<T><<<1, 1, 0, s>>>(A, k)); ++nl;
        if (k == p->max_iter) break;
        if (!A.step4_identity) {
            EIK_LAUNCH("dd_step4_weighted", s, step4k<<<G.ngrids, P.grid_threads, P.step4_smem, s>>>(A));
            ++nl;
        }
        if ((rc = launch_causal(1))) return rc;
        EIK_LAUNCH("dd_delta", s, k_delta<T><<<eb, ew, 0, s>>>(A, k)); ++nl;
    }
    ++nl;
    EIK_LAUNCH("dd_finalize", s, k_finalize<T><<<1, 32, 0, s>>>(A, stats, nl));
    return cuda_check(cudaGetLastError(), "dd launch");
}

}  // namespace eik

using namespace eik;

extern "C" size_t eik_dd_workspace_size(const eik_grid *grid, const eik_dd_params *params) {
    if (!dd_validate(grid, params)) return 0;
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
    const size_t need = grid->ndim == 3 ? dd3_workspace_size(grid, params) : dd_plan(grid, params).bytes;
    if (ws_bytes < need) {
        set_error("workspace of %zu bytes is smaller than the %zu required", ws_bytes, need);
        return EIK_ENOMEM;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (grid->ndim == 3) return dd3_run(grid, r, gamma, g, params, u_out, ws, stats, s);
    if (grid->dtype == EIK_F64) return dd_run<double>(grid, r, gamma, g, params, u_out, ws, stats, s);
    return dd_run<float>(grid, r, gamma, g, params, u_out, ws, stats, s);
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

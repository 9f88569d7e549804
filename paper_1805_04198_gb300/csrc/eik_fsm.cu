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
#include "prof.h"
#include "ptr_table.cuh"

#include <string>
#include <vector>

namespace eik {

EIK_SPIN_LIMIT_SETTER(set_spin_limit_fsm)

static thread_local char g_err[512];

// ---- optional per-launch event timing -------------------------------------
struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
};
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof;
static std::vector<cudaEvent_t> g_prof_pool;

static cudaEvent_t prof_event() {
    if (!g_prof_pool.empty()) {
        cudaEvent_t e = g_prof_pool.back();
        g_prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

int prof_begin(const char *name, cudaStream_t s) {
    if (!g_prof_on) return -1;
    ProfRec r{name, prof_event(), prof_event()};
    cudaEventRecord(r.a, s);
    g_prof.push_back(r);
    return (int)g_prof.size() - 1;
}

void prof_end(int token, cudaStream_t s) {
    if (token < 0) return;
    cudaEventRecord(g_prof[token].b, s);
}

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
    T *ghands;   // multi-CTA hand-off columns [nb][ny]
    int *gctl;   // multi-CTA control words
    FsmDev *dev;
    T h;
    long long max_sweeps;
    int launches;
};

template <class T>
struct PlainFsmPolicy {
    T h;
    __device__ __forceinline__ T update(T self, T vmx, T vpx, T vmy, T vpy, const T *sv, uint8_t,
                                        bool &changed) const {
        const T r = sv[0];  // <= 0 on Gamma
        const T ut = local_solve2_value(vmx, vpx, vmy, vpy, Num<T>::mul(r, h));
        const bool take = (r > T(0)) && (ut < self);
        changed = take;
        return take ? ut : self;
    }
};

// Skewed slowness in output order (the inverse of skew_index, so a warp's
// stores are contiguous; positions outside the box get 0), then the state:
// Sec. 1.1 initialisation, Gamma fixed at g, everything else large.
template <class T>
__device__ void fsm_pack_body(const FsmArgs<T> &A, size_t bid, size_t nbid) {
    const size_t chan = (size_t)4 * A.nb * A.nstepp * 32;
    for (size_t e = bid * blockDim.x + threadIdx.x; e < chan; e += nbid * blockDim.x) {
        const int l = (int)(e & 31);
        const size_t row = e >> 5;
        const int st = (int)(row % A.nstepp);
        const int q = (int)((row / A.nstepp) % A.nb);
        const int d = (int)(row / ((size_t)A.nstepp * A.nb));
        const int sx = dir_sx(d), sy = dir_sy(d);
        const int x = 32 * (sx > 0 ? q : A.nb - 1 - q) + (sx > 0 ? l : 31 - l);
        const int lr = st - l;
        T v = T(0);
        if (x < A.nx && lr >= 0 && lr < A.ny) {
            const size_t gi = (size_t)(sy > 0 ? lr : A.ny - 1 - lr) * A.sy + x;
            v = A.gamma[gi] ? T(-1) : A.r[gi];
        }
        A.rsk[e] = v;
    }
    const size_t total = (size_t)A.nx * A.ny;
    for (size_t t = bid * blockDim.x + threadIdx.x; t < total; t += nbid * blockDim.x) {
        int x = (int)(t % A.nx), y = (int)(t / A.nx);
        const size_t gi = (size_t)y * A.sy + x;
        A.state[box_index(x, y, A.ny)] = A.gamma[gi] ? A.g[gi] : Num<T>::inf();
    }
}

template <class T>
__global__ void k_fsm_pack(FsmArgs<T> A) {
    fsm_pack_body(A, blockIdx.x, gridDim.x);
}

template <class T>
__device__ void fsm_run_body(const FsmArgs<T> &A, char *smem) {
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
__global__ void __maxnreg__((RegCap<T, 96, 128>::v)) k_fsm_run(FsmArgs<T> A) {
    extern __shared__ __align__(16) char smem[];
    fsm_run_body(A, smem);
}

// Multi-CTA form for grids wider than one CTA's blocks: cooperative launch,
// hand-offs and control words in global memory.
template <class T>
__global__ void k_fsm_init_global(FsmArgs<T> A) {
    engine_global_init(A.gctl, A.nb);
    if (threadIdx.x == 0) A.dev->err = 0;
}

template <class T>
__device__ void fsm_run_global_body(const FsmArgs<T> &A, char *smem, int cta) {
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
    engine_run<T, 1, false, true>(bx, pol, A.max_sweeps, smem, sweeps, conv, &A.dev->err, A.ghands, A.gctl, cta);
    if (cta == 0 && threadIdx.x == 0) {
        A.dev->sweeps = (unsigned long long)sweeps;
        A.dev->converged = conv ? 1 : 0;
    }
}

template <class T>
__global__ void __maxnreg__((RegCap<T, 104, 160>::v)) k_fsm_run_global(FsmArgs<T> A) {
    extern __shared__ __align__(16) char smem[];
    fsm_run_global_body(A, smem, (int)blockIdx.x);
}

template <class T>
__device__ void fsm_unpack_body(const FsmArgs<T> &A, eik_fsm_stats *out, size_t bid, size_t nbid) {
    const size_t total = (size_t)A.nx * A.ny;
    for (size_t t = bid * blockDim.x + threadIdx.x; t < total; t += nbid * blockDim.x) {
        int x = (int)(t % A.nx), y = (int)(t / A.nx);
        A.u[(size_t)y * A.sy + x] = A.state[box_index(x, y, A.ny)];
    }
    if (out && bid == 0 && threadIdx.x == 0) {
        out->sweeps = (int64_t)A.dev->sweeps;
        out->converged = A.dev->converged;
        out->error = A.dev->err;
        out->updates = (int64_t)A.dev->sweeps * A.nx * A.ny;
        out->launches = A.launches;
    }
}

template <class T>
__global__ void k_fsm_unpack(FsmArgs<T> A, eik_fsm_stats *out) {
    fsm_unpack_body(A, out, blockIdx.x, gridDim.x);
}

struct FsmPlan {
    int nx, ny, nb, nstepp;
    size_t smem, bytes;
    size_t gsmem;  // multi-CTA shared memory per CTA
    int wpc;       // multi-CTA warps (blocks) per CTA
};

template <class T>
static size_t fsm_layout(const FsmPlan &P, FsmArgs<T> *A, void *ws) {
    Carver cv(ws);
    T *state = cv.take<T>((size_t)P.nb * P.ny * 32);
    T *rsk = cv.take<T>((size_t)4 * P.nb * P.nstepp * 32);
    T *ghands = cv.take<T>((size_t)P.nb * P.ny);
    int *gctl = cv.take<int>(engine_global_ints(P.nb));
    FsmDev *dev = cv.take<FsmDev>(1);
    if (A) {
        A->state = state;
        A->rsk = rsk;
        A->ghands = ghands;
        A->gctl = gctl;
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
    P.smem = grid->dtype == EIK_F64 ? engine_smem_bytes<double, 1, false>(P.nb, P.ny)
                                     : engine_smem_bytes<float, 1, false>(P.nb, P.ny);
    P.wpc = 2;
    P.gsmem = grid->dtype == EIK_F64 ? engine_smem_bytes<double, 1, false, true>(P.wpc, P.ny)
                                      : engine_smem_bytes<float, 1, false, true>(P.wpc, P.ny);
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
    A.launches = 3;
    int rc;
    int dev, optin = 0, nsm = 0;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncAttributes fa;
    if ((rc = cuda_check(cudaFuncGetAttributes(&fa, k_fsm_run<T>), "func attr"))) return rc;
    const bool single = (int)P.smem <= optin && P.nb <= 32 && regs_fit(fa, P.nb);
    A.launches = single ? 3 : 4;
    const size_t total = (size_t)P.nx * P.ny;
    const int tb = (int)std::min<size_t>((total + 255) / 256, (size_t)nsm * 16);
    EIK_LAUNCH("fsm_pack", s, k_fsm_pack<T><<<tb, 256, 0, s>>>(A));
    if (single) {
        if ((rc = cuda_check(set_dyn_smem(k_fsm_run<T>, (int)P.smem), "smem attr")))
            return rc;
        EIK_LAUNCH("fsm_sweeps", s, k_fsm_run<T><<<1, 32 * P.nb, P.smem, s>>>(A));
    } else {
        // one CTA per P.wpc blocks, all co-resident
        const int nblk = (P.nb + P.wpc - 1) / P.wpc;
        if ((rc = cuda_check(set_dyn_smem(k_fsm_run_global<T>, (int)P.gsmem), "smem attr")))
            return rc;
        int per_sm = 0;
        if ((rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fsm_run_global<T>, 32 * P.wpc,
                                                                          P.gsmem), "occupancy")))
            return rc;
        if (per_sm * nsm < nblk) {
            set_error("grid of %d x %d nodes needs %d co-resident CTAs, the device holds %d", P.nx, P.ny, nblk,
                      per_sm * nsm);
            return EIK_EUNSUPPORTED;
        }
        EIK_LAUNCH("fsm_init", s, k_fsm_init_global<T><<<1, 256, 0, s>>>(A));
        void *args[] = {&A};
        int tok = prof_begin("fsm_sweeps", s);
        rc = cuda_check(cudaLaunchCooperativeKernel((void *)k_fsm_run_global<T>, nblk, 32 * P.wpc, args, P.gsmem, s),
                        "fsm cooperative launch");
        prof_end(tok, s);
        if (rc) return rc;
    }
    EIK_LAUNCH("fsm_unpack", s, k_fsm_unpack<T><<<tb, 256, 0, s>>>(A, stats));
    return cuda_check(cudaGetLastError(), "fsm launch");
}


// --------------------------------------------------------------------------
// Many right-hand sides (sources Gamma_p, boundary values g_p) on one grid and
// one slowness: the per-problem kernels of fsm_run, each launch covering every
// problem (the multi-CTA sweep form in co-resident groups of problems).
// --------------------------------------------------------------------------
template <class T>
struct FsmMany {
    FsmArgs<T> A;            // shared fields; the per-problem ones are set by fsm_prob
    const void *const *tab;  // [3][nprob]: gamma, g, u
    char *ws0;               // workspace of problem 0; problem p at ws0 + p * per
    size_t per;
    size_t o_state, o_rsk, o_ghands, o_gctl, o_dev;  // offsets inside a problem's region
    int nprob;
};

template <class T>
__device__ __forceinline__ FsmArgs<T> fsm_prob(const FsmMany<T> &M, int p) {
    FsmArgs<T> A = M.A;
    A.gamma = static_cast<const uint8_t *>(M.tab[p]);
    A.g = static_cast<const T *>(M.tab[M.nprob + p]);
    A.u = static_cast<T *>(const_cast<void *>(M.tab[2 * M.nprob + p]));
    char *b = M.ws0 + (size_t)p * M.per;
    A.state = reinterpret_cast<T *>(b + M.o_state);
    A.rsk = reinterpret_cast<T *>(b + M.o_rsk);
    A.ghands = reinterpret_cast<T *>(b + M.o_ghands);
    A.gctl = reinterpret_cast<int *>(b + M.o_gctl);
    A.dev = reinterpret_cast<FsmDev *>(b + M.o_dev);
    return A;
}

template <class T>
__global__ void k_fsmm_pack(FsmMany<T> M) {
    fsm_pack_body(fsm_prob(M, blockIdx.y), blockIdx.x, gridDim.x);
}

template <class T>
__global__ void __maxnreg__((RegCap<T, 104, 128>::v)) k_fsmm_run(FsmMany<T> M) {
    extern __shared__ __align__(16) char smem[];
    fsm_run_body(fsm_prob(M, blockIdx.x), smem);
}

template <class T>
__global__ void k_fsmm_init_global(FsmMany<T> M) {
    const FsmArgs<T> A = fsm_prob(M, blockIdx.x);
    engine_global_init(A.gctl, A.nb);
    if (threadIdx.x == 0) A.dev->err = 0;
}

// CTA c of the launch serves problem p0 + c / nblk as its CTA c % nblk
template <class T>
__global__ void __maxnreg__((RegCap<T, 96, 160>::v)) k_fsmm_run_global(FsmMany<T> M, int p0, int nblk) {
    extern __shared__ __align__(16) char smem[];
    fsm_run_global_body(fsm_prob(M, p0 + (int)blockIdx.x / nblk), smem, (int)blockIdx.x % nblk);
}

template <class T>
__global__ void k_fsmm_unpack(FsmMany<T> M, eik_fsm_stats *out) {
    fsm_unpack_body(fsm_prob(M, blockIdx.y), out ? out + blockIdx.y : nullptr, blockIdx.x, gridDim.x);
}

struct FsmManyPlan {
    FsmPlan P;
    size_t tab_bytes, per, bytes;
};

static bool fsm_many_plan(const eik_grid *grid, int nprob, FsmManyPlan &M) {
    if (nprob < 1 || nprob > 65535) {
        set_error("nprob = %d out of range [1, 65535]", nprob);
        return false;
    }
    if (!fsm_plan(grid, M.P)) return false;
    M.tab_bytes = ((size_t)3 * nprob * sizeof(void *) + 255) & ~(size_t)255;
    M.per = (M.P.bytes + 255) & ~(size_t)255;
    M.bytes = M.tab_bytes + (size_t)nprob * M.per + 256;
    return true;
}

template <class T>
static int fsm_many_run(const eik_grid *grid, const FsmManyPlan &MP, int nprob, const void *r,
                        const uint8_t *const *gamma, const void *const *g, void *const *u, int64_t max_sweeps,
                        void *ws, eik_fsm_stats *stats, cudaStream_t s) {
    const FsmPlan &P = MP.P;
    FsmMany<T> M;
    memset(&M, 0, sizeof(M));
    FsmArgs<T> &A = M.A;
    A.r = static_cast<const T *>(r);
    A.sy = grid->stride[1];
    A.nx = P.nx;
    A.ny = P.ny;
    A.nb = P.nb;
    A.nstepp = P.nstepp;
    A.h = (T)grid->h;
    A.max_sweeps = max_sweeps;
    // offsets of one problem's region (measured against a dummy base)
    char *const dummy = reinterpret_cast<char *>(256);
    FsmArgs<T> L;
    fsm_layout<T>(P, &L, dummy);
    M.o_state = reinterpret_cast<char *>(L.state) - dummy;
    M.o_rsk = reinterpret_cast<char *>(L.rsk) - dummy;
    M.o_ghands = reinterpret_cast<char *>(L.ghands) - dummy;
    M.o_gctl = reinterpret_cast<char *>(L.gctl) - dummy;
    M.o_dev = reinterpret_cast<char *>(L.dev) - dummy;
    M.tab = static_cast<const void *const *>(ws);
    M.ws0 = static_cast<char *>(ws) + MP.tab_bytes;
    M.per = MP.per;
    M.nprob = nprob;

    int rc, dev, optin = 0, nsm = 0;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncAttributes fa;
    if ((rc = cuda_check(cudaFuncGetAttributes(&fa, k_fsmm_run<T>), "func attr"))) return rc;
    const bool single = (int)P.smem <= optin && P.nb <= 32 && regs_fit(fa, P.nb);
    const int nblk = (P.nb + P.wpc - 1) / P.wpc;
    int group = nprob;  // problems per cooperative launch
    if (!single) {
        if ((rc = cuda_check(set_dyn_smem(k_fsmm_run_global<T>, (int)P.gsmem), "smem attr")))
            return rc;
        int per_sm = 0;
        if ((rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fsmm_run_global<T>, 32 * P.wpc,
                                                                          P.gsmem), "occupancy")))
            return rc;
        group = std::min(nprob, per_sm * nsm / nblk);
        if (group < 1) {
            set_error("grid of %d x %d nodes needs %d co-resident CTAs, the device holds %d", P.nx, P.ny, nblk,
                      per_sm * nsm);
            return EIK_EUNSUPPORTED;
        }
    } else if ((rc = cuda_check(set_dyn_smem(k_fsmm_run<T>, (int)P.smem), "smem attr"))) {
        return rc;
    }
    // pointer table: gamma, g, u
    std::vector<const void *> tab((size_t)3 * nprob);
    for (int p = 0; p < nprob; ++p) {
        tab[p] = gamma[p];
        tab[nprob + p] = g[p];
        tab[2 * nprob + p] = u[p];
    }
    int nl = upload_ptrs(const_cast<const void **>(M.tab), tab.data(), 3 * nprob, s);
    if (nl < 0) return nl;
    const int ngroups = (nprob + group - 1) / group;
    nl += 2 + (single ? 1 : 1 + ngroups);
    A.launches = nl;
    const size_t total = (size_t)P.nx * P.ny;
    const dim3 eg((unsigned)std::max<size_t>(1, std::min<size_t>((total + 255) / 256, (size_t)nsm * 16 / nprob + 1)),
                  (unsigned)nprob);
    EIK_LAUNCH("fsm_pack", s, k_fsmm_pack<T><<<eg, 256, 0, s>>>(M));
    if (single) {
        EIK_LAUNCH("fsm_sweeps", s, k_fsmm_run<T><<<nprob, 32 * P.nb, P.smem, s>>>(M));
    } else {
        EIK_LAUNCH("fsm_init", s, k_fsmm_init_global<T><<<nprob, 256, 0, s>>>(M));
        for (int p0 = 0; p0 < nprob; p0 += group) {
            int np = std::min(group, nprob - p0);
            void *args[] = {&M, &p0, const_cast<int *>(&nblk)};
            int tok = prof_begin("fsm_sweeps", s);
            rc = cuda_check(cudaLaunchCooperativeKernel((void *)k_fsmm_run_global<T>, np * nblk, 32 * P.wpc, args,
                                                        P.gsmem, s),
                            "fsm cooperative launch");
            prof_end(tok, s);
            if (rc) return rc;
        }
    }
    EIK_LAUNCH("fsm_unpack", s, k_fsmm_unpack<T><<<eg, 256, 0, s>>>(M, stats));
    return cuda_check(cudaGetLastError(), "fsm launch");
}
}  // namespace eik

using namespace eik;

extern "C" const char *eik_last_error(void) { return g_err; }

extern "C" int eik_version(void) { return 102; }

namespace eik {
int set_spin_limit_dd(long long);
int set_spin_limit_batch(long long);
int set_spin_limit_dd3(long long);
int set_spin_limit_fsm3(long long);
int set_spin_limit_adj(long long);
int set_spin_limit_dd1(long long);
}  // namespace eik

extern "C" int eik_set_wait_limit(int64_t iterations) {
    if (iterations < 0) {
        set_error("eik_set_wait_limit: iterations must be >= 0 (0 restores the default)");
        return EIK_EINVAL;
    }
    const long long v = iterations == 0 ? SPIN_LIMIT_DEFAULT : (long long)iterations;
    int (*const setters[])(long long) = {set_spin_limit_fsm, set_spin_limit_dd, set_spin_limit_batch,
                                         set_spin_limit_dd3, set_spin_limit_fsm3, set_spin_limit_adj,
                                         set_spin_limit_dd1};
    for (auto f : setters) {
        const int rc = cuda_check((cudaError_t)f(v), "cudaMemcpyToSymbol(wait limit)");
        if (rc) return rc;
    }
    return EIK_OK;
}

extern "C" int eik_profile_enable(int on) {
    int prev = g_prof_on ? 1 : 0;
    g_prof_on = on != 0;
    return prev;
}

extern "C" int eik_profile_collect(eik_kernel_time *out, int max_entries) {
    std::vector<eik_kernel_time> acc;
    int rc = EIK_OK;
    for (auto &r : g_prof) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            set_error("eik_profile_collect: event query failed");
            rc = EIK_ECUDA;
        }
        size_t k = 0;
        while (k < acc.size() && std::string(acc[k].name) != r.name) ++k;
        if (k == acc.size()) acc.push_back(eik_kernel_time{r.name, 0, 0.0, 0.0});
        acc[k].launches += 1;
        acc[k].total_ms += ms;
        if (ms > acc[k].max_ms) acc[k].max_ms = ms;
        g_prof_pool.push_back(r.a);
        g_prof_pool.push_back(r.b);
    }
    g_prof.clear();
    if (rc != EIK_OK) return rc;
    for (size_t k = 0; k < acc.size() && (int)k < max_entries; ++k) out[k] = acc[k];
    return (int)acc.size();
}

namespace eik {
// 3-D form (eik_fsm3.cu)
size_t fsm3_workspace_size(const eik_grid *grid);
int fsm3_run(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g, void *u, int64_t max_sweeps,
             void *ws, eik_fsm_stats *stats, cudaStream_t s);
}  // namespace eik

extern "C" size_t eik_fsm_workspace_size(const eik_grid *grid) {
    if (grid && grid->ndim == 3) return valid_grid_common(grid, 3) ? fsm3_workspace_size(grid) : 0;
    FsmPlan P;
    if (!fsm_plan(grid, P)) return 0;
    return P.bytes;
}

extern "C" int eik_fsm(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g, void *u,
                       int64_t max_sweeps, void *ws, size_t ws_bytes, eik_fsm_stats *stats, void *stream) {
    if (grid && grid->ndim == 3) {
        if (!valid_grid_common(grid, 3)) return EIK_EINVAL;
        if (!r || !gamma || !g || !u || !ws) {
            set_error("eik_fsm: NULL array argument");
            return EIK_EINVAL;
        }
        if (max_sweeps < 1 || max_sweeps > MAX_SWEEPS) {
            set_error("max_sweeps must be in [1, %lld]", MAX_SWEEPS);
            return EIK_EINVAL;
        }
        if (reinterpret_cast<uintptr_t>(ws) & 255) {
            set_error("workspace must be 256-byte aligned");
            return EIK_EINVAL;
        }
        const size_t need = fsm3_workspace_size(grid);
        if (ws_bytes < need) {
            set_error("workspace of %zu bytes is smaller than the %zu required", ws_bytes, need);
            return EIK_ENOMEM;
        }
        return fsm3_run(grid, r, gamma, g, u, max_sweeps, ws, stats, static_cast<cudaStream_t>(stream));
    }
    FsmPlan P;
    if (!fsm_plan(grid, P)) return EIK_EINVAL;
    if (!r || !gamma || !g || !u || !ws) {
        set_error("eik_fsm: NULL array argument");
        return EIK_EINVAL;
    }
    if (max_sweeps < 1 || max_sweeps > MAX_SWEEPS || grid->n[1] > MAX_BOX_ROWS) {
        set_error("max_sweeps must be in [1, %lld] and n[1] <= %d", MAX_SWEEPS, MAX_BOX_ROWS);
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

extern "C" size_t eik_fsm_many_workspace_size(const eik_grid *grid, int nprob) {
    FsmManyPlan M;
    if (!fsm_many_plan(grid, nprob, M)) return 0;
    return M.bytes;
}

extern "C" int eik_fsm_many(const eik_grid *grid, int nprob, const void *r, const uint8_t *const *gamma,
                            const void *const *g, void *const *u, int64_t max_sweeps, void *ws, size_t ws_bytes,
                            eik_fsm_stats *stats, void *stream) {
    FsmManyPlan M;
    if (!fsm_many_plan(grid, nprob, M)) return EIK_EINVAL;
    if (!r || !gamma || !g || !u || !ws) {
        set_error("eik_fsm_many: NULL argument");
        return EIK_EINVAL;
    }
    for (int p = 0; p < nprob; ++p) {
        if (!gamma[p] || !g[p] || !u[p]) {
            set_error("eik_fsm_many: NULL array of problem %d", p);
            return EIK_EINVAL;
        }
    }
    if (max_sweeps < 1 || max_sweeps > MAX_SWEEPS || grid->n[1] > MAX_BOX_ROWS) {
        set_error("max_sweeps must be in [1, %lld] and n[1] <= %d", MAX_SWEEPS, MAX_BOX_ROWS);
        return EIK_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(ws) & 255) {
        set_error("workspace must be 256-byte aligned");
        return EIK_EINVAL;
    }
    if (ws_bytes < M.bytes) {
        set_error("workspace of %zu bytes is smaller than the %zu required", ws_bytes, M.bytes);
        return EIK_ENOMEM;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (grid->dtype == EIK_F64) return fsm_many_run<double>(grid, M, nprob, r, gamma, g, u, max_sweeps, ws, stats, s);
    return fsm_many_run<float>(grid, M, nprob, r, gamma, g, u, max_sweeps, ws, stats, s);
}

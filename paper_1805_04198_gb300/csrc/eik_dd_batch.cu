// eik_dd_batch.cu -- many independent 2-D DD problems (each one the iteration of
// Sec. 3.2, Steps 1-4, Alg. 1-5) solved together on one stream.
//
// Every stage of the single-problem solve (eik_dd.cu) becomes one launch over
// the whole batch, built from the same per-stage bodies:
//   * element stages (packing, Alg. 4, delta) run over a flat list of
//     (problem, 256-element block) items, so a large problem gets many blocks
//     and a small one few;
//   * the subdomain solves (Steps 2 + 3) and the shifted-grid solves (Steps 1
//     and 4) run the warp-systolic engine, whose CTA holds one warp per
//     32-column block of its box.  Problems of different sizes need different
//     CTA shapes, so these stages are launched once per width class (all boxes
//     needing the same number of warps), with the class's shared memory;
//   * the causal sweep (Alg. 2) is one cooperative launch over every coarse line
//     of every problem, with one batch-wide change flag per round;
//   * each problem keeps its own stop flag: a problem that has converged or
//     reached its own iteration cap makes its later items return at once.
// A launch of a box stage either gives every item its own CTA or starts the
// CTAs that fit on the GPU and lets them draw items from a queue (largest
// problems first when asked).  Which is faster depends on the mix of sizes;
// eik_dd_batched_autotune times the candidates on the caller's batch.
//
// Nothing here synchronises with the host, allocates or copies between host
// and device: the per-problem argument blocks and the item tables reach the
// device as kernel parameters.  The whole solve can therefore be captured into
// a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "dd2_device.cuh"
#include "dd2_host.cuh"
#include "host_util.h"
#include "prof.h"

namespace eik {

EIK_SPIN_LIMIT_SETTER(set_spin_limit_batch)

// Flat list of items over problems: problem p owns items [pre[p], pre[p+1]).
struct Segs {
    const int *pre;  // [n + 1]
    int n, total;
};

// Problem and local index of item `it` (largest p with pre[p] <= it).
__device__ __forceinline__ int seg_find(const int *pre, int n, int it, int &local) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(pre + mid) <= it) lo = mid;
        else hi = mid - 1;
    }
    local = it - __ldg(pre + lo);
    return lo;
}

// Boxes of one width class: the class's problems in launch order, the
// prefix of their item counts, and the queue counters of the queue form.
struct ItemList {
    const int *prob;  // [n] problem ids
    const int *pre;   // [n + 1] item prefix in the order of `prob`
    int n, items;
    int *queue;       // [2]: next item, CTAs that ran dry; null = one CTA per item
};

struct BatchCtl {
    unsigned *bar;  // [4] grid barrier of the causal sweep
    int *chg;       // [4] causal round flags
    int *err;       // batch-level device error (a barrier wait that expired)
};

// Runs body(problem, local item) for the items this CTA takes.  All threads
// of the CTA call it; the body may return early (uniformly) for a finished
// problem.
template <class Body>
__device__ __forceinline__ void for_items(const ItemList &L, Body body) {
    if (!L.queue) {
        if ((int)blockIdx.x >= L.items) return;
        int local;
        const int k = seg_find(L.pre, L.n, blockIdx.x, local);
        body(__ldg(L.prob + k), local);
        return;
    }
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) {
            const int it = atomicAdd(L.queue, 1);
            if (it >= L.items) {
                // every CTA runs dry exactly once; the last one re-arms the
                // queue for the next launch of this class
                __threadfence();
                if (atomicAdd(L.queue + 1, 1) == (int)gridDim.x - 1) {
                    L.queue[0] = 0;
                    L.queue[1] = 0;
                    __threadfence();
                }
            }
            s_item = it;
        }
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= L.items) break;
        int local;
        const int k = seg_find(L.pre, L.n, it, local);
        body(__ldg(L.prob + k), local);
    }
}

// --------------------------------------------------------------------------
// Kernels
// --------------------------------------------------------------------------
constexpr int UPLOAD_BYTES = 24576;
struct UploadChunk {
    unsigned char b[UPLOAD_BYTES];
};

// Copies host-built tables (carried in the kernel parameters) to the device.
__global__ void kb_upload(unsigned char *dst, const __grid_constant__ UploadChunk c, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = c.b[i];
}

template <class T>
__global__ void kb_init(const DDArgs<T> *__restrict__ args, BatchCtl C, int *queues, int nq) {
    init_body(args[blockIdx.x]);
    if (blockIdx.x == 0) {
        if (threadIdx.x < 4) {
            C.bar[threadIdx.x] = 0;
            C.chg[threadIdx.x] = 0;
        }
        if (threadIdx.x == 0) *C.err = 0;
        for (int i = threadIdx.x; i < 2 * nq; i += blockDim.x) queues[i] = 0;
    }
}

template <class T>
__global__ void kb_pack(const DDArgs<T> *__restrict__ args, Segs tiles, Segs coarse) {
    for (int b = blockIdx.x; b < tiles.total + coarse.total; b += gridDim.x) {
        int local;
        if (b < tiles.total) {
            const int p = seg_find(tiles.pre, tiles.n, b, local);
            pack_tiles_body(args[p], local, __ldg(tiles.pre + p + 1) - __ldg(tiles.pre + p));
        } else {
            const int p = seg_find(coarse.pre, coarse.n, b - tiles.total, local);
            pack_coarse_body(args[p], local, __ldg(coarse.pre + p + 1) - __ldg(coarse.pre + p));
        }
    }
}

template <class T>
__global__ void kb_alg4(const DDArgs<T> *__restrict__ args, Segs S, int k) {
    for (int b = blockIdx.x; b < S.total; b += gridDim.x) {
        int local;
        const int p = seg_find(S.pre, S.n, b, local);
        alg4_body(args[p], k, local, __ldg(S.pre + p + 1) - __ldg(S.pre + p));
    }
}

template <class T>
__global__ void kb_delta(const DDArgs<T> *__restrict__ args, Segs S, int k) {
    for (int b = blockIdx.x; b < S.total; b += gridDim.x) {
        int local;
        const int p = seg_find(S.pre, S.n, b, local);
        delta_body(args[p], k, local, __ldg(S.pre + p + 1) - __ldg(S.pre + p));
    }
}

template <class T>
__global__ void kb_check(const DDArgs<T> *__restrict__ args, int nprob, int k) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nprob) check_body(args[p], k);
}

template <class T>
__global__ void kb_finalize(const DDArgs<T> *__restrict__ args, BatchCtl C, eik_dd_stats *out, long long launches) {
    const int p = blockIdx.x;
    finalize_body(args[p], out + p, launches);
    if (threadIdx.x == 0 && *C.err && out[p].error == 0) out[p].error = *C.err;
}

// Causal sweep (Alg. 2) over every coarse line of every problem: the same
// rounds as the single-problem kernel, with the lines of all problems dealt to
// the warps of one cooperative grid.
template <class T>
__global__ void kb_causal(const DDArgs<T> *__restrict__ args, Segs hl, Segs vl, BatchCtl C, int only_if_not_done,
                          int lw) {
    const long long wlim = spin_limit();  // limit of the grid-barrier waits
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    extern __shared__ __align__(16) unsigned char causal_smem[];
    T *su = reinterpret_cast<T *>(causal_smem + (size_t)(threadIdx.x >> 5) * causal_warp_bytes<T>(lw));
    uint8_t *sw = reinterpret_cast<uint8_t *>(su) + causal_align16((size_t)lw * sizeof(T));
    __shared__ int blk_changed;
    if (blockIdx.x == 0 && threadIdx.x < 3) C.chg[threadIdx.x] = 0;
    if (!grid_barrier(C.bar, C.err, wlim)) return;
    int rounds = 0;
    for (;;) {
        if (threadIdx.x == 0) blk_changed = 0;
        __syncthreads();
        bool ch = false;
        for (int l = gw; l < hl.total; l += warps_total) {
            int local;
            const DDArgs<T> &A = args[seg_find(hl.pre, hl.n, l, local)];
            if (only_if_not_done && *A.done) continue;
            if (lw > 0) {
                ch |= causal_line_smem(A, true, local, su, sw);
            } else {
                ch |= causal_line(A, true, local, 0);
                ch |= causal_line(A, true, local, 1);
            }
        }
        if (!grid_barrier(C.bar, C.err, wlim)) return;
        for (int l = gw; l < vl.total; l += warps_total) {
            int local;
            const DDArgs<T> &A = args[seg_find(vl.pre, vl.n, l, local)];
            if (only_if_not_done && *A.done) continue;
            if (lw > 0) {
                ch |= causal_line_smem(A, false, local, su, sw);
            } else {
                ch |= causal_line(A, false, local, 0);
                ch |= causal_line(A, false, local, 1);
            }
        }
        if (lane == 0 && ch) atomicOr(&blk_changed, 1);
        __syncthreads();
        if (threadIdx.x == 0 && blk_changed) atomicOr(&C.chg[rounds % 3], 1);
        ++rounds;
        if (!grid_barrier(C.bar, C.err, wlim)) return;
        const int any = *(volatile int *)&C.chg[(rounds - 1) % 3];
        if (blockIdx.x == 0 && threadIdx.x == 0) C.chg[(rounds + 1) % 3] = 0;
        if (!any || rounds > 10000) break;
    }
    if (blockIdx.x == 0) {
        for (int p = threadIdx.x; p < hl.n; p += blockDim.x)
            if (!(only_if_not_done && *args[p].done)) atomicMax(&args[p].st->causal_rounds_max, rounds);
    }
}

// Box stages: the same register caps as the single-problem kernels (FP64: a
// 9-warp CTA, 3 warps per scheduler, at most 168 registers a thread).
#define EIK_BATCH_PAIR(name, body, RF, RD)                                                         \
    __global__ void __maxnreg__(RF) name##_f32(const DDArgs<float> *__restrict__ args, ItemList L) { \
        extern __shared__ __align__(16) char smem[];                                               \
        for_items(L, [&](int p, int local) { body<float>(args[p], smem, local); });                \
    }                                                                                              \
    __global__ void __maxnreg__(RD) name##_f64(const DDArgs<double> *__restrict__ args, ItemList L) { \
        extern __shared__ __align__(16) char smem[];                                               \
        for_items(L, [&](int p, int local) { body<double>(args[p], smem, local); });               \
    }
EIK_BATCH_PAIR(kb_step1, k_step1_body, 96, 168)
EIK_BATCH_PAIR(kb_step4, k_step4_body, 160, 168)
EIK_BATCH_PAIR(kb_step4a, k_step4a_body, 160, 168)
// The batch's subdomains are small (17-65 nodes a side): chunks in which every
// lane is on a valid row are rare there, and the engine's second copy of the
// step for them made the batch's subdomain stage 16% slower, so it is left out.
template <class T>
__device__ __forceinline__ void kb_fine_body(const DDArgs<T> &A, char *smem, int tile) {
    k_fine_body<T, false>(A, smem, tile);
}
EIK_BATCH_PAIR(kb_fine, kb_fine_body, 96, 168)

template <class T> struct BatchKernels;
template <> struct BatchKernels<float> {
    static constexpr void (*step1)(const DDArgs<float> *, ItemList) = kb_step1_f32;
    static constexpr void (*step4)(const DDArgs<float> *, ItemList) = kb_step4_f32;
    static constexpr void (*step4a)(const DDArgs<float> *, ItemList) = kb_step4a_f32;
    static constexpr void (*fine)(const DDArgs<float> *, ItemList) = kb_fine_f32;
};
template <> struct BatchKernels<double> {
    static constexpr void (*step1)(const DDArgs<double> *, ItemList) = kb_step1_f64;
    static constexpr void (*step4)(const DDArgs<double> *, ItemList) = kb_step4_f64;
    static constexpr void (*step4a)(const DDArgs<double> *, ItemList) = kb_step4a_f64;
    static constexpr void (*fine)(const DDArgs<double> *, ItemList) = kb_fine_f64;
};

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------
constexpr int ELEM_BLOCK = 256;  // threads (and elements) per element-stage block

struct BoxClass {
    int nw;           // warps per CTA (32-column blocks of the widest box)
    size_t smem;      // dynamic shared memory (max over the class)
    int n, items;     // problems, boxes
    int prob_at, pre_at;  // offsets of the tables in the int area
    int queue;        // queue slot
};

struct BatchPlan {
    int nprob = 0, dtype = 0;
    size_t args_bytes = 0;
    std::vector<DDPlan> P;
    std::vector<size_t> region;  // byte offset of each problem's workspace region
    std::vector<int> tab;        // int tables
    int tiles_at = 0, coarse_at = 0, hl_at = 0, vl_at = 0;
    int tiles_total = 0, coarse_total = 0, hl_total = 0, vl_total = 0;
    std::vector<BoxClass> fine, grid;
    size_t args_off = 0, tab_off = 0, ctl_off = 0;
    int nq = 0;
    size_t bytes = 0;
    int max_iter = 0;
    bool adaptive = false;  // some problem uses the per-node weight: every problem
                            // carries the weight as a fourth Alg. 5 static
};

static const eik_dd_batch_config kDefaultConfig = {0, 0, 0, 1};

static bool batch_validate(int nprob, const eik_grid *grids, const eik_dd_params *params) {
    if (nprob < 1 || nprob > 65535) {
        set_error("nprob = %d out of range [1, 65535]", nprob);
        return false;
    }
    if (!grids || !params) {
        set_error("grids or params is NULL");
        return false;
    }
    for (int p = 0; p < nprob; ++p) {
        if (grids[p].ndim != 2) {
            set_error("problem %d: the batched solve takes 2-D grids only (ndim = %d)", p, grids[p].ndim);
            return false;
        }
        if (grids[p].dtype != grids[0].dtype) {
            set_error("problem %d: every problem of a batch must have the same dtype", p);
            return false;
        }
        if (!dd_validate(&grids[p], &params[p])) {
            char msg[512];
            snprintf(msg, sizeof msg, "%s", eik_last_error());
            set_error("problem %d: %s", p, msg);
            return false;
        }
    }
    return true;
}

// Orders the problems of a class: largest boxes first (stable), or input order.
static void class_order(std::vector<int> &ids, const std::vector<long long> &cost, bool largest_first) {
    if (largest_first)
        std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) { return cost[a] > cost[b]; });
}

template <class T>
static void batch_plan(int nprob, const eik_grid *grids, const eik_dd_params *params, const eik_dd_batch_config &cfg,
                       BatchPlan &B) {
    B.nprob = nprob;
    B.dtype = grids[0].dtype;
    B.P.resize(nprob);
    B.tab.clear();
    B.max_iter = 0;
    B.adaptive = false;
    for (int p = 0; p < nprob; ++p) B.adaptive = B.adaptive || params[p].theta_adaptive != 0;
    for (int p = 0; p < nprob; ++p) {
        eik_dd_params q = params[p];
        if (B.adaptive) q.theta_adaptive = 1;  // storage and Step 4 shape of the weighted form
        B.P[p] = dd_plan(&grids[p], &q);
        B.max_iter = std::max(B.max_iter, params[p].max_iter);
    }
    auto push_prefix = [&](auto count) -> int {
        const int at = (int)B.tab.size();
        int acc = 0;
        for (int p = 0; p < nprob; ++p) {
            B.tab.push_back(acc);
            acc += (int)count(p);
        }
        B.tab.push_back(acc);
        return at;
    };
    auto blocks = [](size_t n) { return (n + ELEM_BLOCK - 1) / ELEM_BLOCK; };
    B.tiles_at = push_prefix([&](int p) {
        const DDGeom &G = B.P[p].G;
        return blocks((size_t)G.tx * G.ty * G.tnx * G.tny);
    });
    B.tiles_total = B.tab.back();
    B.coarse_at = push_prefix([&](int p) { return blocks(B.P[p].G.coarse_elems); });
    B.coarse_total = B.tab.back();
    B.hl_at = push_prefix([&](int p) { return B.P[p].G.ncy + 1; });
    B.hl_total = B.tab.back();
    B.vl_at = push_prefix([&](int p) { return B.P[p].G.ncx + 1; });
    B.vl_total = B.tab.back();

    // width classes of the box stages
    B.nq = 0;
    auto make_classes = [&](std::vector<BoxClass> &out, auto width, auto items, auto cost, auto smem) {
        out.clear();
        std::vector<int> keys;
        for (int p = 0; p < nprob; ++p) keys.push_back(width(p));
        std::vector<int> uk = keys;
        std::sort(uk.begin(), uk.end());
        uk.erase(std::unique(uk.begin(), uk.end()), uk.end());
        std::vector<long long> cst(nprob);
        for (int p = 0; p < nprob; ++p) cst[p] = cost(p);
        for (int w : uk) {
            BoxClass c;
            c.nw = w;
            c.smem = 0;
            std::vector<int> ids;
            for (int p = 0; p < nprob; ++p)
                if (keys[p] == w) {
                    ids.push_back(p);
                    c.smem = std::max(c.smem, (size_t)smem(p));
                }
            class_order(ids, cst, cfg.largest_first != 0);
            c.n = (int)ids.size();
            c.prob_at = (int)B.tab.size();
            for (int p : ids) B.tab.push_back(p);
            c.pre_at = (int)B.tab.size();
            int acc = 0;
            for (int p : ids) {
                B.tab.push_back(acc);
                acc += items(p);
            }
            B.tab.push_back(acc);
            c.items = acc;
            c.queue = B.nq++;
            out.push_back(c);
        }
    };
    make_classes(
        B.fine, [&](int p) { return B.P[p].G.tnb; },
        [&](int p) { return B.P[p].G.tx * B.P[p].G.ty; },
        [&](int p) { return (long long)B.P[p].G.tnx * B.P[p].G.tny; }, [&](int p) { return B.P[p].fine_smem; });
    make_classes(
        B.grid, [&](int p) { return B.P[p].grid_threads / 32; }, [&](int p) { return B.P[p].G.ngrids; },
        [&](int p) { return (long long)(B.P[p].G.ncx + 1) * (B.P[p].G.ncy + 1); },
        [&](int p) { return std::max(B.P[p].step1_smem, B.P[p].step4_smem); });

    // workspace: argument blocks, int tables, control words, problem regions
    Carver cv(nullptr);
    B.args_bytes = sizeof(DDArgs<T>) * (size_t)nprob;
    cv.take<DDArgs<T>>(nprob);
    B.args_off = 0;
    B.tab_off = (cv.used + 255) & ~(size_t)255;
    cv.take<int>(B.tab.size());
    B.ctl_off = (cv.used + 255) & ~(size_t)255;
    cv.take<int>(16 + 2 * (size_t)B.nq);
    B.region.resize(nprob);
    for (int p = 0; p < nprob; ++p) {
        B.region[p] = (cv.used + 255) & ~(size_t)255;
        cv.used = B.region[p] + B.P[p].bytes;
    }
    B.bytes = cv.used + 256;
}

static int upload(void *dst, const void *src, size_t n, cudaStream_t s) {
    const unsigned char *b = static_cast<const unsigned char *>(src);
    UploadChunk chunk;
    for (size_t off = 0; off < n; off += UPLOAD_BYTES) {
        const int m = (int)std::min<size_t>(UPLOAD_BYTES, n - off);
        memcpy(chunk.b, b + off, m);
        EIK_LAUNCH("dd_batch_upload", s, kb_upload<<<std::max(1, m / 4096), 256, 0, s>>>(static_cast<unsigned char *>(dst) + off, chunk, m));
    }
    return cuda_check(cudaGetLastError(), "upload launch");
}

template <class T>
static int batch_run(int nprob, const eik_grid *grids, const void *const *r, const uint8_t *const *gamma,
                     const void *const *g, const eik_dd_params *params, void *const *u_out,
                     const eik_dd_batch_config &cfg, void *ws, eik_dd_stats *stats, cudaStream_t s) {
    BatchPlan B;
    batch_plan<T>(nprob, grids, params, cfg, B);
    char *base = static_cast<char *>(ws);
    std::vector<DDArgs<T>> args(nprob);
    for (int p = 0; p < nprob; ++p) {
        DDArgs<T> &A = args[p];
        memset(&A, 0, sizeof(A));
        A.G = B.P[p].G;
        A.r = static_cast<const T *>(r[p]);
        A.gamma = gamma[p];
        A.g = static_cast<const T *>(g[p]);
        A.u_out = static_cast<T *>(u_out[p]);
        A.sy = grids[p].stride[1];
        dd_layout<T>(B.P[p], &A, base + B.region[p], params[p].max_iter);
        A.theta = (T)params[p].theta;
        A.step4_identity = (!params[p].theta_adaptive && params[p].theta == 0.0) ? 1 : 0;
        A.tol = (T)params[p].tol;
        A.max_iter = params[p].max_iter;
        A.max_fsm = params[p].max_fsm_sweeps;
        A.max_coarse = params[p].max_coarse_sweeps;
        A.adaptive = params[p].theta_adaptive ? 1 : 0;
        for (int s2 = 0; s2 < 3; ++s2) A.om[s2] = params[p].omega[s2];
        A.sg = params[p].sig_gamma;
        A.sd = params[p].sig_delta;
        A.sx0 = params[p].sig_x0;
        A.cap = params[p].theta_cap;
    }
    auto step4k = B.adaptive ? BatchKernels<T>::step4a : BatchKernels<T>::step4;
    const DDArgs<T> *dargs = reinterpret_cast<const DDArgs<T> *>(base + B.args_off);
    const int *dtab = reinterpret_cast<const int *>(base + B.tab_off);
    int *ctl = reinterpret_cast<int *>(base + B.ctl_off);
    BatchCtl C;
    C.bar = reinterpret_cast<unsigned *>(ctl);
    C.chg = ctl + 4;
    C.err = ctl + 8;
    int *queues = ctl + 16;

    int rc;
    int dev;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    int nsm = 0, smem_optin = 0;
    if ((rc = cuda_check(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "attr"))) return rc;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    size_t need_fine = 0, need_grid = 0;
    for (auto &c : B.fine) need_fine = std::max(need_fine, c.smem);
    for (auto &c : B.grid) need_grid = std::max(need_grid, c.smem);
    if ((int)need_fine > smem_optin || (int)need_grid > smem_optin) {
        set_error("shared memory need (%zu, %zu) exceeds the device limit %d", need_fine, need_grid, smem_optin);
        return EIK_EUNSUPPORTED;
    }
    if ((rc = cuda_check(set_dyn_smem(BatchKernels<T>::fine, (int)std::max<size_t>(need_fine, 1)), "smem attr fine")))
        return rc;
    if ((rc = cuda_check(set_dyn_smem(BatchKernels<T>::step1, (int)std::max<size_t>(need_grid, 1)), "smem attr step1")))
        return rc;
    if ((rc = cuda_check(set_dyn_smem(step4k, (int)std::max<size_t>(need_grid, 1)), "smem attr step4")))
        return rc;

    // launch shapes of the box classes
    auto item_list = [&](const BoxClass &c, bool queue) {
        ItemList L;
        L.prob = dtab + c.prob_at;
        L.pre = dtab + c.pre_at;
        L.n = c.n;
        L.items = c.items;
        L.queue = queue ? queues + 2 * c.queue : nullptr;
        return L;
    };
    auto ctas = [&](void (*k)(const DDArgs<T> *, ItemList), const BoxClass &c, bool queue) -> int {
        if (!queue) return c.items;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * c.nw, c.smem);
        if (per_sm < 1) per_sm = 1;
        if (cfg.ctas_per_sm > 0) per_sm = std::min(per_sm, cfg.ctas_per_sm);
        return std::max(1, std::min(c.items, per_sm * nsm));
    };
    const bool fq = cfg.fine_queue != 0, gq = cfg.coarse_queue != 0;

    // causal sweep: cooperative grid of what is co-resident
    int maxlen = 0;
    for (int p = 0; p < nprob; ++p) maxlen = std::max(maxlen, std::max(B.P[p].G.nx, B.P[p].G.ny));
    CausalShape cs;
    if ((rc = causal_shape<T>((const void *)kb_causal<T>, maxlen, std::max(B.hl_total, B.vl_total), nsm, smem_optin,
                              cs)))
        return rc;
    Segs tiles{dtab + B.tiles_at, nprob, B.tiles_total};
    Segs coarse{dtab + B.coarse_at, nprob, B.coarse_total};
    Segs hl{dtab + B.hl_at, nprob, B.hl_total};
    Segs vl{dtab + B.vl_at, nprob, B.vl_total};
    const int eb = std::max(1, std::min(B.coarse_total, nsm * 8));
    const int pb = std::max(1, std::min(B.tiles_total + B.coarse_total, nsm * 16));

    long long nl = 0;
    if ((rc = upload(base + B.args_off, args.data(), B.args_bytes, s))) return rc;
    nl += (long long)((B.args_bytes + UPLOAD_BYTES - 1) / UPLOAD_BYTES);
    if ((rc = upload(base + B.tab_off, B.tab.data(), B.tab.size() * sizeof(int), s))) return rc;
    nl += (long long)((B.tab.size() * sizeof(int) + UPLOAD_BYTES - 1) / UPLOAD_BYTES);
    EIK_LAUNCH("dd_init", s, kb_init<T><<<nprob, 256, 0, s>>>(dargs, C, queues, B.nq)); ++nl;
    EIK_LAUNCH("dd_pack", s, kb_pack<T><<<pb, ELEM_BLOCK, 0, s>>>(dargs, tiles, coarse)); ++nl;
    for (const BoxClass &c : B.grid) {
        EIK_LAUNCH("dd_step1_coarse_fsm", s,
                   BatchKernels<T>::step1<<<ctas(BatchKernels<T>::step1, c, gq), 32 * c.nw, c.smem, s>>>(dargs, item_list(c, gq)));
        ++nl;
    }
    auto launch_causal = [&](int only) -> int {
        void *kargs[] = {(void *)&dargs, &hl, &vl, &C, &only, &cs.lw};
        int tok = prof_begin("dd_causal_sweep", s);
        int r2 = cuda_check(cudaLaunchCooperativeKernel((void *)kb_causal<T>, cs.blocks, cs.threads, kargs, cs.smem, s),
                            "causal launch");
        prof_end(tok, s);
        ++nl;
        return r2;
    };
    if ((rc = launch_causal(0))) return rc;
    for (int k = 0; k <= B.max_iter; ++k) {
        for (const BoxClass &c : B.fine) {
            EIK_LAUNCH("dd_fine_subdomains", s,
                       BatchKernels<T>::fine<<<ctas(BatchKernels<T>::fine, c, fq), 32 * c.nw, c.smem, s>>>(dargs, item_list(c, fq)));
            ++nl;
        }
        EIK_LAUNCH("dd_alg4_restrict", s, kb_alg4<T><<<eb, ELEM_BLOCK, 0, s>>>(dargs, coarse, k)); ++nl;
        EIK_LAUNCH("dd_check", s, kb_check<T><<<(nprob + 127) / 128, 128, 0, s>>>(dargs, nprob, k)); ++nl;
        if (k == B.max_iter) break;
        for (const BoxClass &c : B.grid) {
            EIK_LAUNCH("dd_step4_weighted", s,
                       step4k<<<ctas(step4k, c, gq), 32 * c.nw, c.smem, s>>>(dargs, item_list(c, gq)));
            ++nl;
        }
        if ((rc = launch_causal(1))) return rc;
        EIK_LAUNCH("dd_delta", s, kb_delta<T><<<eb, ELEM_BLOCK, 0, s>>>(dargs, coarse, k)); ++nl;
    }
    ++nl;
    if (stats) EIK_LAUNCH("dd_finalize", s, kb_finalize<T><<<nprob, 32, 0, s>>>(dargs, C, stats, nl));
    return cuda_check(cudaGetLastError(), "batched dd launch");
}

static size_t batch_bytes(int nprob, const eik_grid *grids, const eik_dd_params *params) {
    BatchPlan B;
    if (grids[0].dtype == EIK_F64) batch_plan<double>(nprob, grids, params, kDefaultConfig, B);
    else batch_plan<float>(nprob, grids, params, kDefaultConfig, B);
    return B.bytes;
}

}  // namespace eik

using namespace eik;

extern "C" size_t eik_dd_batched_workspace_size(int nprob, const eik_grid *grids, const eik_dd_params *params) {
    if (!batch_validate(nprob, grids, params)) return 0;
    return batch_bytes(nprob, grids, params);
}

extern "C" int eik_dd_solve_batched(int nprob, const eik_grid *grids, const void *const *r,
                                    const uint8_t *const *gamma, const void *const *g, const eik_dd_params *params,
                                    void *const *u_out, const eik_dd_batch_config *config, void *ws, size_t ws_bytes,
                                    eik_dd_stats *stats, void *stream) {
    if (!batch_validate(nprob, grids, params)) return EIK_EINVAL;
    if (!r || !gamma || !g || !u_out || !ws) {
        set_error("eik_dd_solve_batched: NULL array argument");
        return EIK_EINVAL;
    }
    for (int p = 0; p < nprob; ++p) {
        if (!r[p] || !gamma[p] || !g[p] || !u_out[p]) {
            set_error("eik_dd_solve_batched: NULL array of problem %d", p);
            return EIK_EINVAL;
        }
    }
    if (reinterpret_cast<uintptr_t>(ws) & 255) {
        set_error("workspace must be 256-byte aligned");
        return EIK_EINVAL;
    }
    const size_t need = batch_bytes(nprob, grids, params);
    if (ws_bytes < need) {
        set_error("workspace of %zu bytes is smaller than the %zu required", ws_bytes, need);
        return EIK_ENOMEM;
    }
    const eik_dd_batch_config cfg = config ? *config : kDefaultConfig;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (grids[0].dtype == EIK_F64)
        return batch_run<double>(nprob, grids, r, gamma, g, params, u_out, cfg, ws, stats, s);
    return batch_run<float>(nprob, grids, r, gamma, g, params, u_out, cfg, ws, stats, s);
}

extern "C" int eik_dd_batched_autotune(int nprob, const eik_grid *grids, const void *const *r,
                                       const uint8_t *const *gamma, const void *const *g,
                                       const eik_dd_params *params, void *const *u_out, int tune_iters, void *ws,
                                       size_t ws_bytes, eik_dd_batch_config *best, double *best_ms, void *stream) {
    if (!best) {
        set_error("eik_dd_batched_autotune: best is NULL");
        return EIK_EINVAL;
    }
    if (tune_iters < 0) {
        set_error("tune_iters must be >= 0");
        return EIK_EINVAL;
    }
    if (!batch_validate(nprob, grids, params)) return EIK_EINVAL;
    std::vector<eik_dd_params> pt(params, params + nprob);
    for (auto &q : pt) q.max_iter = std::min(q.max_iter, tune_iters);
    std::vector<eik_dd_batch_config> cands;
    for (int lf = 0; lf < 2; ++lf)
        for (int fq = 0; fq < 2; ++fq)
            for (int gq = 0; gq < 2; ++gq) {
                if (!fq && !gq) {
                    cands.push_back({0, 0, 0, lf});
                    continue;
                }
                cands.push_back({fq, gq, 0, lf});
                cands.push_back({fq, gq, 1, lf});
            }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    int rc;
    if ((rc = cuda_check(cudaEventCreate(&e0), "event"))) return rc;
    if ((rc = cuda_check(cudaEventCreate(&e1), "event"))) {
        cudaEventDestroy(e0);
        return rc;
    }
    double best_t = INFINITY;
    // one untimed run first (module load, caches)
    rc = eik_dd_solve_batched(nprob, grids, r, gamma, g, pt.data(), u_out, &cands[0], ws, ws_bytes, nullptr, stream);
    for (size_t i = 0; rc == EIK_OK && i < cands.size(); ++i) {
        cudaEventRecord(e0, s);
        rc = eik_dd_solve_batched(nprob, grids, r, gamma, g, pt.data(), u_out, &cands[i], ws, ws_bytes, nullptr,
                                  stream);
        if (rc) break;
        cudaEventRecord(e1, s);
        if ((rc = cuda_check(cudaEventSynchronize(e1), "autotune sync"))) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_t) {
            best_t = ms;
            *best = cands[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == EIK_OK && best_ms) *best_ms = best_t;
    return rc;
}

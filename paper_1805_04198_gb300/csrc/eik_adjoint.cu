// eik_adjoint.cu -- gradient dJ/dr of a scalar J(u) through the converged
// Godunov system (the discretisation of Sec. 1.1), for a u returned by
// eik_fsm or eik_dd_solve.  The paper has no gradient; this is the discrete
// adjoint-state method:
//   at every reached non-Gamma node j, u_j = F(a_j, r_j) with a_j the
//   neighbour minima of the branch taken (Alg. 3 choice);
//   lambda = dJ/du + (dF/du)^T lambda,   dJ/dr_j = lambda_j dF_j/dr_j.
// (dF/du)^T is strictly causal in reverse (a node only feeds neighbours with
// larger u), so the linear system is solved exactly by Gauss-Seidel sweeps in
// the 2^d orderings -- the same warp-systolic engine as the forward sweeps,
// with lambda as the state and, per node, the four incoming weights and
// dJ/du as statics.  A sweep that changes nothing ends the solve; every node's
// value is then the fixed summation -x, +x, -y, +y of final neighbour values,
// so the result does not depend on the sweep order.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "engine.cuh"
#include "host_util.h"
#include "prof.h"
#include "ptr_table.cuh"

#include <vector>

namespace eik {

EIK_SPIN_LIMIT_SETTER(set_spin_limit_adj)

struct AdjDev {
    unsigned long long sweeps;
    int converged;
    int err;
};

template <class T>
struct AdjArgs {
    const T *r;
    const uint8_t *gamma;
    const T *u;
    const T *dJdu;
    T *grad;
    long long sy;
    int nx, ny, nb, nstepp;
    T h;
    T *win;    // [4][nx*ny] incoming weights: from -x, +x, -y, +y
    T *dudr;   // [nx*ny]
    T *state;  // lambda, strip-major
    T *sk;     // skewed statics [5][4][nb][nstepp][32]
    T *ghands;
    int *gctl;
    AdjDev *dev;
    long long max_sweeps;
    int launches;
};

// dF_j/du of node j towards each neighbour side and dF_j/dr_j (zero where j
// does not use the neighbour; all zero at Gamma and unreached nodes).
template <class T>
__device__ void adj_node(const AdjArgs<T> &A, int x, int y, T wm[2], T wp[2], T &dudr) {
    using N = Num<T>;
    const T INF = N::inf();
    wm[0] = wm[1] = wp[0] = wp[1] = T(0);
    dudr = T(0);
    const size_t j = (size_t)y * A.sy + x;
    const T uj = A.u[j];
    if (A.gamma[j] || !(uj < INF)) return;
    const T vmx = x > 0 ? A.u[j - 1] : INF, vpx = x + 1 < A.nx ? A.u[j + 1] : INF;
    const T vmy = y > 0 ? A.u[j - A.sy] : INF, vpy = y + 1 < A.ny ? A.u[j + A.sy] : INF;
    const T rj = A.r[j];
    uint8_t w;
    (void)local_solve2(vmx, vpx, vmy, vpy, N::mul(rj, A.h), w);
    const int wx = wind_comp(w, 0), wy = wind_comp(w, 1);
    const int used = (wx != 0) + (wy != 0);
    if (used == 0) return;
    const T ax = wx > 0 ? vmx : vpx, ay = wy > 0 ? vmy : vpy;
    if (used == 1) {
        if (wx > 0) wm[0] = T(1);
        if (wx < 0) wp[0] = T(1);
        if (wy > 0) wm[1] = T(1);
        if (wy < 0) wp[1] = T(1);
        dudr = A.h;
        return;
    }
    T D = T(0);
    D = N::add(D, N::sub(uj, ax));
    D = N::add(D, N::sub(uj, ay));
    if (!(D > T(0))) return;
    const T gx = N::div(N::sub(uj, ax), D), gy = N::div(N::sub(uj, ay), D);
    if (wx > 0) wm[0] = gx; else wp[0] = gx;
    if (wy > 0) wm[1] = gy; else wp[1] = gy;
    dudr = N::div(N::mul(N::mul(rj, A.h), A.h), D);
}

template <class T>
__device__ void adj_zero_body(const AdjArgs<T> &A, size_t bid, size_t nbid) {
    const size_t n = (size_t)A.nx * A.ny;
    for (size_t t = bid * blockDim.x + threadIdx.x; t < 4 * n; t += nbid * blockDim.x) A.win[t] = T(0);
}

template <class T>
__global__ void k_adj_zero(AdjArgs<T> A) {
    adj_zero_body(A, blockIdx.x, gridDim.x);
}

// each node scatters the weights of its dependencies into its neighbours'
// incoming slots (every slot has exactly one writer)
template <class T>
__device__ void adj_nodes_body(const AdjArgs<T> &A, size_t bid, size_t nbid) {
    const size_t n = (size_t)A.nx * A.ny;
    for (size_t t = bid * blockDim.x + threadIdx.x; t < n; t += nbid * blockDim.x) {
        const int x = (int)(t % A.nx), y = (int)(t / A.nx);
        T wm[2], wp[2], dr;
        adj_node(A, x, y, wm, wp, dr);
        A.dudr[t] = dr;
        // j uses its -x neighbour i = j-1: lambda_i pulls from its +x side
        if (x > 0 && wm[0] != T(0)) A.win[1 * n + t - 1] = wm[0];
        if (x + 1 < A.nx && wp[0] != T(0)) A.win[0 * n + t + 1] = wp[0];
        if (y > 0 && wm[1] != T(0)) A.win[3 * n + t - A.nx] = wm[1];
        if (y + 1 < A.ny && wp[1] != T(0)) A.win[2 * n + t + A.nx] = wp[1];
    }
}

template <class T>
__global__ void k_adj_nodes(AdjArgs<T> A) {
    adj_nodes_body(A, blockIdx.x, gridDim.x);
}

// Skewed statics in output order: thread e writes element e of every channel
// ([dir][logical block][step][lane], the inverse of skew_index), so a warp's
// stores are contiguous; positions outside the box get 0.
template <class T>
__device__ void adj_pack_body(const AdjArgs<T> &A, size_t bid, size_t nbid) {
    const size_t n = (size_t)A.nx * A.ny;
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
        T v0 = T(0), v1 = T(0), v2 = T(0), v3 = T(0), v4 = T(0);
        if (x < A.nx && lr >= 0 && lr < A.ny) {
            const int y = sy > 0 ? lr : A.ny - 1 - lr;
            const size_t t = (size_t)y * A.nx + x;
            v0 = A.win[t];
            v1 = A.win[n + t];
            v2 = A.win[2 * n + t];
            v3 = A.win[3 * n + t];
            v4 = A.dJdu[(size_t)y * A.sy + x];
        }
        A.sk[e] = v0;
        A.sk[chan + e] = v1;
        A.sk[2 * chan + e] = v2;
        A.sk[3 * chan + e] = v3;
        A.sk[4 * chan + e] = v4;
    }
    const size_t box = (size_t)A.nb * A.ny * 32;
    for (size_t t = bid * blockDim.x + threadIdx.x; t < box; t += nbid * blockDim.x) A.state[t] = T(0);
}

template <class T>
__global__ void k_adj_pack(AdjArgs<T> A) {
    adj_pack_body(A, blockIdx.x, gridDim.x);
}

// lambda_i = dJ/du_i + W(-x) l(-x) + W(+x) l(+x) + W(-y) l(-y) + W(+y) l(+y)
template <class T>
struct AdjPolicy {
    __device__ __forceinline__ T update(T self, T vmx, T vpx, T vmy, T vpy, const T *sv, uint8_t,
                                        bool &changed) const {
        using N = Num<T>;
        T acc = sv[4];
        if (sv[0] != T(0)) acc = N::add(acc, N::mul(sv[0], vmx));
        if (sv[1] != T(0)) acc = N::add(acc, N::mul(sv[1], vpx));
        if (sv[2] != T(0)) acc = N::add(acc, N::mul(sv[2], vmy));
        if (sv[3] != T(0)) acc = N::add(acc, N::mul(sv[3], vpy));
        changed = !(acc == self);
        return acc;
    }
};

template <class T>
__device__ __forceinline__ Box<T, 5> adj_box(const AdjArgs<T> &A) {
    Box<T, 5> bx;
    const size_t chan = (size_t)4 * A.nb * A.nstepp * 32;
    bx.u = A.state;
    for (int c = 0; c < 5; ++c) bx.st[c] = A.sk + c * chan;
    bx.sb = nullptr;
    bx.nx = A.nx;
    bx.ny = A.ny;
    bx.nb = A.nb;
    bx.nstepp = A.nstepp;
    return bx;
}

template <class T>
__device__ void adj_run_body(const AdjArgs<T> &A, char *smem) {
    const Box<T, 5> bx = adj_box(A);
    AdjPolicy<T> pol;
    long long sweeps;
    bool conv;
    if (threadIdx.x == 0) A.dev->err = 0;
    __syncthreads();
    engine_run<T, 5, false>(bx, pol, A.max_sweeps, smem, sweeps, conv, &A.dev->err);
    if (threadIdx.x == 0) {
        A.dev->sweeps = (unsigned long long)sweeps;
        A.dev->converged = conv ? 1 : 0;
    }
}

template <class T>
__global__ void __maxnreg__((RegCap<T, 152, 176>::v)) k_adj_run(AdjArgs<T> A) {
    extern __shared__ __align__(16) char smem[];
    adj_run_body(A, smem);
}

template <class T>
__global__ void k_adj_init_global(AdjArgs<T> A) {
    engine_global_init(A.gctl, A.nb);
    if (threadIdx.x == 0) A.dev->err = 0;
}

template <class T>
__device__ void adj_run_global_body(const AdjArgs<T> &A, char *smem, int cta) {
    const Box<T, 5> bx = adj_box(A);
    AdjPolicy<T> pol;
    long long sweeps;
    bool conv;
    engine_run<T, 5, false, true>(bx, pol, A.max_sweeps, smem, sweeps, conv, &A.dev->err, A.ghands, A.gctl, cta);
    if (cta == 0 && threadIdx.x == 0) {
        A.dev->sweeps = (unsigned long long)sweeps;
        A.dev->converged = conv ? 1 : 0;
    }
}

template <class T>
__global__ void __maxnreg__((RegCap<T, 152, 176>::v)) k_adj_run_global(AdjArgs<T> A) {
    extern __shared__ __align__(16) char smem[];
    adj_run_global_body(A, smem, (int)blockIdx.x);
}

template <class T>
__device__ void adj_grad_body(const AdjArgs<T> &A, eik_adjoint_stats *out, size_t bid, size_t nbid) {
    const size_t n = (size_t)A.nx * A.ny;
    if (A.grad) {
        for (size_t t = bid * blockDim.x + threadIdx.x; t < n; t += nbid * blockDim.x) {
            const int x = (int)(t % A.nx), y = (int)(t / A.nx);
            A.grad[(size_t)y * A.sy + x] = Num<T>::mul(A.state[box_index(x, y, A.ny)], A.dudr[t]);
        }
    }
    if (out && bid == 0 && threadIdx.x == 0) {
        out->sweeps = (int64_t)A.dev->sweeps;
        out->converged = A.dev->converged;
        out->error = A.dev->err;
        out->launches = A.launches;
    }
}

template <class T>
__global__ void k_adj_grad(AdjArgs<T> A, eik_adjoint_stats *out) {
    adj_grad_body(A, out, blockIdx.x, gridDim.x);
}

struct AdjPlan {
    int nx, ny, nb, nstepp, wpc;
    size_t smem, gsmem, bytes;
};

template <class T>
static size_t adj_layout(const AdjPlan &P, AdjArgs<T> *A, void *ws) {
    Carver cv(ws);
    const size_t n = (size_t)P.nx * P.ny;
    T *win = cv.take<T>(4 * n);
    T *dudr = cv.take<T>(n);
    T *state = cv.take<T>((size_t)P.nb * P.ny * 32);
    T *sk = cv.take<T>((size_t)5 * 4 * P.nb * P.nstepp * 32);
    T *ghands = cv.take<T>((size_t)P.nb * P.ny);
    int *gctl = cv.take<int>(engine_global_ints(P.nb));
    AdjDev *dev = cv.take<AdjDev>(1);
    if (A) {
        A->win = win;
        A->dudr = dudr;
        A->state = state;
        A->sk = sk;
        A->ghands = ghands;
        A->gctl = gctl;
        A->dev = dev;
    }
    return cv.used + 256;
}

static bool adj_plan(const eik_grid *grid, AdjPlan &P) {
    if (!valid_grid_common(grid, 2)) return false;
    if (grid->n[1] > MAX_BOX_ROWS) {
        set_error("n[1] must be <= %d", MAX_BOX_ROWS);
        return false;
    }
    P.nx = (int)grid->n[0];
    P.ny = (int)grid->n[1];
    P.nb = ceil32(P.nx);
    P.nstepp = nstep_padded(P.ny);
    P.wpc = 2;
    const bool f64 = grid->dtype == EIK_F64;
    P.smem = f64 ? engine_smem_bytes<double, 5, false>(P.nb, P.ny) : engine_smem_bytes<float, 5, false>(P.nb, P.ny);
    P.gsmem = f64 ? engine_smem_bytes<double, 5, false, true>(P.wpc, P.ny)
                  : engine_smem_bytes<float, 5, false, true>(P.wpc, P.ny);
    P.bytes = f64 ? adj_layout<double>(P, nullptr, nullptr) : adj_layout<float>(P, nullptr, nullptr);
    return true;
}

template <class T>
static int adj_run(const eik_grid *grid, const AdjPlan &P, const void *r, const uint8_t *gamma, const void *u,
                   const void *dJdu, void *grad, int64_t max_sweeps, void *ws, eik_adjoint_stats *stats,
                   cudaStream_t s) {
    AdjArgs<T> A;
    memset(&A, 0, sizeof(A));
    A.r = static_cast<const T *>(r);
    A.gamma = gamma;
    A.u = static_cast<const T *>(u);
    A.dJdu = static_cast<const T *>(dJdu);
    A.grad = static_cast<T *>(grad);
    A.sy = grid->stride[1];
    A.nx = P.nx;
    A.ny = P.ny;
    A.nb = P.nb;
    A.nstepp = P.nstepp;
    A.h = (T)grid->h;
    A.max_sweeps = max_sweeps;
    adj_layout<T>(P, &A, ws);
    int rc, dev, optin = 0, nsm = 0;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncAttributes fa;
    if ((rc = cuda_check(cudaFuncGetAttributes(&fa, k_adj_run<T>), "func attr"))) return rc;
    const bool single = (int)P.smem <= optin && P.nb <= 32 && regs_fit(fa, P.nb);
    A.launches = single ? 5 : 6;
    const size_t total = (size_t)P.nx * P.ny;
    const int tb = (int)std::min<size_t>((total + 255) / 256, (size_t)nsm * 16);
    EIK_LAUNCH("adj_zero", s, k_adj_zero<T><<<tb, 256, 0, s>>>(A));
    EIK_LAUNCH("adj_nodes", s, k_adj_nodes<T><<<tb, 256, 0, s>>>(A));
    EIK_LAUNCH("adj_pack", s, k_adj_pack<T><<<tb, 256, 0, s>>>(A));
    if (single) {
        if ((rc = cuda_check(set_dyn_smem(k_adj_run<T>, (int)P.smem), "smem attr")))
            return rc;
        EIK_LAUNCH("adj_sweeps", s, k_adj_run<T><<<1, 32 * P.nb, P.smem, s>>>(A));
    } else {
        const int nblk = (P.nb + P.wpc - 1) / P.wpc;
        if ((rc = cuda_check(set_dyn_smem(k_adj_run_global<T>, (int)P.gsmem), "smem attr")))
            return rc;
        int per_sm = 0;
        if ((rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_run_global<T>, 32 * P.wpc,
                                                                          P.gsmem), "occupancy")))
            return rc;
        if (per_sm * nsm < nblk) {
            set_error("grid of %d x %d nodes needs %d co-resident CTAs, the device holds %d", P.nx, P.ny, nblk,
                      per_sm * nsm);
            return EIK_EUNSUPPORTED;
        }
        EIK_LAUNCH("adj_init", s, k_adj_init_global<T><<<1, 256, 0, s>>>(A));
        void *args[] = {&A};
        int tok = prof_begin("adj_sweeps", s);
        rc = cuda_check(cudaLaunchCooperativeKernel((void *)k_adj_run_global<T>, nblk, 32 * P.wpc, args, P.gsmem, s),
                        "adjoint cooperative launch");
        prof_end(tok, s);
        if (rc) return rc;
    }
    EIK_LAUNCH("adj_grad", s, k_adj_grad<T><<<tb, 256, 0, s>>>(A, stats));
    return cuda_check(cudaGetLastError(), "adjoint launch");
}


// --------------------------------------------------------------------------
// Many right-hand sides on one grid and one slowness (the sources of a
// tomography problem): every per-problem kernel of adj_run covers all problems
// in one launch (the multi-CTA sweep form in co-resident groups), and
// optionally grad_sum = sum over problems of dJ_p/dr, added in problem order.
// --------------------------------------------------------------------------
template <class T>
struct AdjMany {
    AdjArgs<T> A;            // shared fields; the per-problem ones are set by adj_prob
    const void *const *tab;  // [4][nprob]: gamma, u, dJdu, grad (grad entries may be null)
    char *ws0;               // workspace of problem 0; problem p at ws0 + p * per
    size_t per;
    size_t o_win, o_dudr, o_state, o_sk, o_ghands, o_gctl, o_dev;
    T *grad_sum;             // may be null
    int nprob;
};

template <class T>
__device__ __forceinline__ AdjArgs<T> adj_prob(const AdjMany<T> &M, int p) {
    AdjArgs<T> A = M.A;
    A.gamma = static_cast<const uint8_t *>(M.tab[p]);
    A.u = static_cast<const T *>(M.tab[M.nprob + p]);
    A.dJdu = static_cast<const T *>(M.tab[2 * M.nprob + p]);
    A.grad = static_cast<T *>(const_cast<void *>(M.tab[3 * M.nprob + p]));
    char *b = M.ws0 + (size_t)p * M.per;
    A.win = reinterpret_cast<T *>(b + M.o_win);
    A.dudr = reinterpret_cast<T *>(b + M.o_dudr);
    A.state = reinterpret_cast<T *>(b + M.o_state);
    A.sk = reinterpret_cast<T *>(b + M.o_sk);
    A.ghands = reinterpret_cast<T *>(b + M.o_ghands);
    A.gctl = reinterpret_cast<int *>(b + M.o_gctl);
    A.dev = reinterpret_cast<AdjDev *>(b + M.o_dev);
    return A;
}

template <class T>
__global__ void k_adjm_zero(AdjMany<T> M) {
    adj_zero_body(adj_prob(M, blockIdx.y), blockIdx.x, gridDim.x);
}
template <class T>
__global__ void k_adjm_nodes(AdjMany<T> M) {
    adj_nodes_body(adj_prob(M, blockIdx.y), blockIdx.x, gridDim.x);
}
template <class T>
__global__ void k_adjm_pack(AdjMany<T> M) {
    adj_pack_body(adj_prob(M, blockIdx.y), blockIdx.x, gridDim.x);
}
template <class T>
__global__ void __maxnreg__((RegCap<T, 152, 176>::v)) k_adjm_run(AdjMany<T> M) {
    extern __shared__ __align__(16) char smem[];
    adj_run_body(adj_prob(M, blockIdx.x), smem);
}
template <class T>
__global__ void k_adjm_init_global(AdjMany<T> M) {
    const AdjArgs<T> A = adj_prob(M, blockIdx.x);
    engine_global_init(A.gctl, A.nb);
    if (threadIdx.x == 0) A.dev->err = 0;
}
// CTA c of the launch serves problem p0 + c / nblk as its CTA c % nblk
template <class T>
__global__ void __maxnreg__((RegCap<T, 160, 160>::v)) k_adjm_run_global(AdjMany<T> M, int p0, int nblk) {
    extern __shared__ __align__(16) char smem[];
    adj_run_global_body(adj_prob(M, p0 + (int)blockIdx.x / nblk), smem, (int)blockIdx.x % nblk);
}
template <class T>
__global__ void k_adjm_grad(AdjMany<T> M, eik_adjoint_stats *out) {
    adj_grad_body(adj_prob(M, blockIdx.y), out ? out + blockIdx.y : nullptr, blockIdx.x, gridDim.x);
}
// grad_sum = g_0 + g_1 + ... + g_{nprob-1}, g_p = lambda_p dF/dr of problem p,
// accumulated left to right
template <class T>
__global__ void k_adjm_sum(AdjMany<T> M) {
    const AdjArgs<T> &A = M.A;
    const size_t n = (size_t)A.nx * A.ny;
    const size_t per = M.per;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(t % A.nx), y = (int)(t / A.nx);
        const size_t bi = box_index(x, y, A.ny);
        T acc = T(0);
        for (int p = 0; p < M.nprob; ++p) {
            const char *b = M.ws0 + (size_t)p * per;
            const T gp = Num<T>::mul(reinterpret_cast<const T *>(b + M.o_state)[bi],
                                     reinterpret_cast<const T *>(b + M.o_dudr)[t]);
            acc = p == 0 ? gp : Num<T>::add(acc, gp);
        }
        M.grad_sum[(size_t)y * A.sy + x] = acc;
    }
}

struct AdjManyPlan {
    AdjPlan P;
    size_t tab_bytes, per, bytes;
};

static bool adj_many_plan(const eik_grid *grid, int nprob, AdjManyPlan &M) {
    if (nprob < 1 || nprob > 65535) {
        set_error("nprob = %d out of range [1, 65535]", nprob);
        return false;
    }
    if (!adj_plan(grid, M.P)) return false;
    M.tab_bytes = ((size_t)4 * nprob * sizeof(void *) + 255) & ~(size_t)255;
    M.per = (M.P.bytes + 255) & ~(size_t)255;
    M.bytes = M.tab_bytes + (size_t)nprob * M.per + 256;
    return true;
}

template <class T>
static int adj_many_run(const eik_grid *grid, const AdjManyPlan &MP, int nprob, const void *r,
                        const uint8_t *const *gamma, const void *const *u, const void *const *dJdu,
                        void *const *grad, void *grad_sum, int64_t max_sweeps, void *ws, eik_adjoint_stats *stats,
                        cudaStream_t s) {
    const AdjPlan &P = MP.P;
    AdjMany<T> M;
    memset(&M, 0, sizeof(M));
    AdjArgs<T> &A = M.A;
    A.r = static_cast<const T *>(r);
    A.sy = grid->stride[1];
    A.nx = P.nx;
    A.ny = P.ny;
    A.nb = P.nb;
    A.nstepp = P.nstepp;
    A.h = (T)grid->h;
    A.max_sweeps = max_sweeps;
    char *const dummy = reinterpret_cast<char *>(256);
    AdjArgs<T> L;
    adj_layout<T>(P, &L, dummy);
    M.o_win = reinterpret_cast<char *>(L.win) - dummy;
    M.o_dudr = reinterpret_cast<char *>(L.dudr) - dummy;
    M.o_state = reinterpret_cast<char *>(L.state) - dummy;
    M.o_sk = reinterpret_cast<char *>(L.sk) - dummy;
    M.o_ghands = reinterpret_cast<char *>(L.ghands) - dummy;
    M.o_gctl = reinterpret_cast<char *>(L.gctl) - dummy;
    M.o_dev = reinterpret_cast<char *>(L.dev) - dummy;
    M.tab = static_cast<const void *const *>(ws);
    M.ws0 = static_cast<char *>(ws) + MP.tab_bytes;
    M.per = MP.per;
    M.nprob = nprob;
    M.grad_sum = static_cast<T *>(grad_sum);

    int rc, dev, optin = 0, nsm = 0;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncAttributes fa;
    if ((rc = cuda_check(cudaFuncGetAttributes(&fa, k_adjm_run<T>), "func attr"))) return rc;
    const bool single = (int)P.smem <= optin && P.nb <= 32 && regs_fit(fa, P.nb);
    const int nblk = (P.nb + P.wpc - 1) / P.wpc;
    int group = nprob;
    if (!single) {
        if ((rc = cuda_check(set_dyn_smem(k_adjm_run_global<T>, (int)P.gsmem), "smem attr")))
            return rc;
        int per_sm = 0;
        if ((rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adjm_run_global<T>, 32 * P.wpc,
                                                                          P.gsmem), "occupancy")))
            return rc;
        group = std::min(nprob, per_sm * nsm / nblk);
        if (group < 1) {
            set_error("grid of %d x %d nodes needs %d co-resident CTAs, the device holds %d", P.nx, P.ny, nblk,
                      per_sm * nsm);
            return EIK_EUNSUPPORTED;
        }
    } else if ((rc = cuda_check(set_dyn_smem(k_adjm_run<T>, (int)P.smem), "smem attr"))) {
        return rc;
    }
    std::vector<const void *> tab((size_t)4 * nprob);
    for (int p = 0; p < nprob; ++p) {
        tab[p] = gamma[p];
        tab[nprob + p] = u[p];
        tab[2 * nprob + p] = dJdu[p];
        tab[3 * nprob + p] = grad ? grad[p] : nullptr;
    }
    int nl = upload_ptrs(const_cast<const void **>(M.tab), tab.data(), 4 * nprob, s);
    if (nl < 0) return nl;
    const int ngroups = (nprob + group - 1) / group;
    nl += 4 + (single ? 1 : 1 + ngroups) + (grad_sum ? 1 : 0);
    A.launches = nl;
    const size_t total = (size_t)P.nx * P.ny;
    const dim3 eg((unsigned)std::max<size_t>(1, std::min<size_t>((total + 255) / 256, (size_t)nsm * 16 / nprob + 1)),
                  (unsigned)nprob);
    EIK_LAUNCH("adj_zero", s, k_adjm_zero<T><<<eg, 256, 0, s>>>(M));
    EIK_LAUNCH("adj_nodes", s, k_adjm_nodes<T><<<eg, 256, 0, s>>>(M));
    EIK_LAUNCH("adj_pack", s, k_adjm_pack<T><<<eg, 256, 0, s>>>(M));
    if (single) {
        EIK_LAUNCH("adj_sweeps", s, k_adjm_run<T><<<nprob, 32 * P.nb, P.smem, s>>>(M));
    } else {
        EIK_LAUNCH("adj_init", s, k_adjm_init_global<T><<<nprob, 256, 0, s>>>(M));
        for (int p0 = 0; p0 < nprob; p0 += group) {
            int np = std::min(group, nprob - p0);
            void *args[] = {&M, &p0, const_cast<int *>(&nblk)};
            int tok = prof_begin("adj_sweeps", s);
            rc = cuda_check(cudaLaunchCooperativeKernel((void *)k_adjm_run_global<T>, np * nblk, 32 * P.wpc, args,
                                                        P.gsmem, s),
                            "adjoint cooperative launch");
            prof_end(tok, s);
            if (rc) return rc;
        }
    }
    EIK_LAUNCH("adj_grad", s, k_adjm_grad<T><<<eg, 256, 0, s>>>(M, stats));
    if (grad_sum) {
        const int sb = (int)std::min<size_t>((total + 255) / 256, (size_t)nsm * 16);
        EIK_LAUNCH("adj_sum", s, k_adjm_sum<T><<<sb, 256, 0, s>>>(M));
    }
    return cuda_check(cudaGetLastError(), "adjoint launch");
}
}  // namespace eik

using namespace eik;

extern "C" size_t eik_dd_adjoint_workspace_size(const eik_grid *grid) {
    AdjPlan P;
    if (!adj_plan(grid, P)) return 0;
    return P.bytes;
}

extern "C" int eik_dd_adjoint(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *u,
                              const void *dJdu, void *grad_r, int64_t max_sweeps, void *ws, size_t ws_bytes,
                              eik_adjoint_stats *stats, void *stream) {
    AdjPlan P;
    if (!adj_plan(grid, P)) return EIK_EINVAL;
    if (!r || !gamma || !u || !dJdu || !grad_r || !ws) {
        set_error("eik_dd_adjoint: NULL array argument");
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
    if (ws_bytes < P.bytes) {
        set_error("workspace of %zu bytes is smaller than the %zu required", ws_bytes, P.bytes);
        return EIK_ENOMEM;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (grid->dtype == EIK_F64) return adj_run<double>(grid, P, r, gamma, u, dJdu, grad_r, max_sweeps, ws, stats, s);
    return adj_run<float>(grid, P, r, gamma, u, dJdu, grad_r, max_sweeps, ws, stats, s);
}

extern "C" size_t eik_dd_adjoint_many_workspace_size(const eik_grid *grid, int nprob) {
    AdjManyPlan M;
    if (!adj_many_plan(grid, nprob, M)) return 0;
    return M.bytes;
}

extern "C" int eik_dd_adjoint_many(const eik_grid *grid, int nprob, const void *r, const uint8_t *const *gamma,
                                   const void *const *u, const void *const *dJdu, void *const *grad_r,
                                   void *grad_sum, int64_t max_sweeps, void *ws, size_t ws_bytes,
                                   eik_adjoint_stats *stats, void *stream) {
    AdjManyPlan M;
    if (!adj_many_plan(grid, nprob, M)) return EIK_EINVAL;
    if (!r || !gamma || !u || !dJdu || !ws || (!grad_r && !grad_sum)) {
        set_error("eik_dd_adjoint_many: NULL argument (grad_r and grad_sum may not both be NULL)");
        return EIK_EINVAL;
    }
    for (int p = 0; p < nprob; ++p) {
        if (!gamma[p] || !u[p] || !dJdu[p]) {
            set_error("eik_dd_adjoint_many: NULL array of problem %d", p);
            return EIK_EINVAL;
        }
    }
    if (max_sweeps < 1 || max_sweeps > MAX_SWEEPS) {
        set_error("max_sweeps must be in [1, %lld]", MAX_SWEEPS);
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
    if (grid->dtype == EIK_F64)
        return adj_many_run<double>(grid, M, nprob, r, gamma, u, dJdu, grad_r, grad_sum, max_sweeps, ws, stats, s);
    return adj_many_run<float>(grid, M, nprob, r, gamma, u, dJdu, grad_r, grad_sum, max_sweeps, ws, stats, s);
}

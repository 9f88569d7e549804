// eik_dd1.cu -- the one-dimensional two-scale iteration of Sec. 3.1 (Steps
// 1-4): eq. 1d on [0, 1] with the coarse grid X_i = i H (i = 0..N) and the
// subintervals [iH, (i+1)H] of M fine cells each (h = H / M).  eik_dd_solve
// runs it when grid->ndim == 1.
//
// One CTA runs the whole iteration in one launch.  The coarse state (U, the
// new U, u^k, C_H(U^k), the winds W^k and w^k, the fixed-node mask) and the
// two end copies of every subinterval sit in shared memory; the interior fine
// nodes live in the output array.  The threads solve the subintervals (Steps
// 2-3, one subinterval per thread at a time, by the 1-D FSM of Sec. 1.1) and
// make the Step 3 choice at the coarse nodes; one thread runs the serial
// coarse work (Step 1's coarse FSM, Step 4's weighted Gauss-Seidel sweeps, the
// causal sweep and the update size).  No host round trip per iteration.
//
// Readings, the same as for the 2-D method: a wind is the direction of travel
// (+1 when the left neighbour gives the minimum, so the W~ of Step 4 is read
// with the opposite sign to the printed one); a tie goes to the right
// neighbour; an inflow end of a subinterval starts at U and is swept like any
// node, and an end that keeps that starting value echoes the coarse wind and
// is no candidate of the minimum unless both copies are echoes; the weighted
// update is u^k + theta (U~ - C_H(U^k)), and u^k where U~ or C_H(U^k) is
// +inf; the causal sweep repeats both directions until nothing changes.
// Step 1 has no causal sweep (the 1-D text gives none), the Step 3 choice
// compares the two fine winds only, and Step 4 tests W^k = w^k = W~.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "engine.cuh"  // MAX_SWEEPS, the sweep cap of every DD solve
#include "host_util.h"
#include "prof.h"

namespace eik {

constexpr int DD1_MAX_SUB = 2048;  // subintervals: the coarse state must fit in shared memory

template <class T>
struct DD1Args {
    const T *r;
    const uint8_t *gamma;
    const T *g;
    T *u;
    eik_dd_stats *stats;
    int N;         // subintervals
    long long M;   // fine cells per subinterval
    T h, H, theta, tol;
    int max_iter;
    long long max_fsm, max_coarse;
};

template <class T>
static size_t dd1_smem_bytes(int N) {
    return (size_t)(4 * (N + 1) + 2 * N) * sizeof(T) + (size_t)3 * (N + 1) + (size_t)4 * N;
}

// C_H of eq. 1dgod at node i of an array of n + 1 nodes, with the wind of the
// neighbour used (+1 left, -1 right, 0 when the value is +inf).  The 1-D
// Godunov update of a fine node is the same expression with spacing h.
template <class T>
__device__ __forceinline__ T ch1(T a, T b, T rh, int &w) {
    T v;
    if (a < b) {
        v = Num<T>::add(a, rh);
        w = 1;
    } else {
        v = Num<T>::add(b, rh);
        w = -1;
    }
    if (!(v < Num<T>::inf())) w = 0;
    return v;
}

template <class T>
__device__ __forceinline__ T ch1_at(const T *U, int i, int N, T rH, int &w) {
    const T inf = Num<T>::inf();
    return ch1(i > 0 ? U[i - 1] : inf, i < N ? U[i + 1] : inf, rH, w);
}

// Coarse FSM of Step 1 on U[0..N] (spacing H, r sampled at X_i), Gamma nodes
// fixed.  Sweeps alternate right-to-left, left-to-right until one changes
// nothing or the cap is reached.  One thread.
template <class T>
__device__ long long coarse_fsm(const DD1Args<T> &A, T *U, const uint8_t *cfix, bool &conv) {
    const int N = A.N;
    long long s = 0;
    conv = false;
    while (s < A.max_coarse) {
        bool ch = false;
        const int step = (s % 2 == 0) ? -1 : 1;
        for (int i = step > 0 ? 0 : N; i >= 0 && i <= N; i += step) {
            if (cfix[i]) continue;
            int w;
            const T ut = ch1_at(U, i, N, Num<T>::mul(A.r[(long long)i * A.M], A.H), w);
            if (ut < U[i]) {
                U[i] = ut;
                ch = true;
            }
        }
        ++s;
        if (!ch) {
            conv = true;
            break;
        }
    }
    return s;
}

// Steps 2-3 on subinterval `sub` (one thread).  Step 2: a Gamma node is fixed
// at g; an end where the coarse wind points into the subinterval (W = +1 at
// its left end, W = -1 at its right end) starts at U, every other node at
// +inf.  Step 3: FSM sweeps (right-to-left first) until one changes nothing
// or the cap is reached.  The interior nodes are left in u; the ends' values,
// winds and echo flags go to eu / ew / ee at 2 sub (left) and 2 sub + 1
// (right).  Returns the sweeps run; conv = 0 if the cap stopped them.
template <class T>
__device__ long long solve_sub(const DD1Args<T> &A, int sub, const T *U, const int8_t *W, T *eu, int8_t *ew,
                               uint8_t *ee, bool &conv) {
    const T inf = Num<T>::inf();
    const long long M = A.M, f0 = (long long)sub * M;
    T *u = A.u + f0;
    const T *r = A.r + f0;
    const uint8_t *gm = A.gamma + f0;
    const T *g = A.g + f0;
    const bool fix0 = gm[0] != 0, fixM = gm[M] != 0;
    const bool in0 = !fix0 && W[sub] > 0, inM = !fixM && W[sub + 1] < 0;
    const T s0 = fix0 ? g[0] : (in0 ? U[sub] : inf);
    const T sM = fixM ? g[M] : (inM ? U[sub + 1] : inf);
    T e0 = s0, eM = sM;
    for (long long j = 1; j < M; ++j) u[j] = gm[j] ? g[j] : inf;
    long long s = 0;
    conv = false;
    while (s < A.max_fsm) {
        bool ch = false;
        if (s % 2 == 0) {
            // right to left: `right` is node j+1 after its update, `cur` node
            // j before it (node j-1 is read before it is updated)
            T right = inf, cur = eM;
            for (long long j = M; j >= 0; --j) {
                const T left = j == 0 ? inf : (j == 1 ? e0 : u[j - 1]);
                T v = cur;
                if (!gm[j]) {
                    int w;
                    const T ut = ch1(left, right, Num<T>::mul(r[j], A.h), w);
                    if (ut < v) {
                        v = ut;
                        ch = true;
                    }
                }
                if (j == M) eM = v;
                else if (j == 0) e0 = v;
                else u[j] = v;
                right = v;
                cur = left;
            }
        } else {
            T left = inf, cur = e0;
            for (long long j = 0; j <= M; ++j) {
                const T right = j == M ? inf : (j + 1 == M ? eM : u[j + 1]);
                T v = cur;
                if (!gm[j]) {
                    int w;
                    const T ut = ch1(left, right, Num<T>::mul(r[j], A.h), w);
                    if (ut < v) {
                        v = ut;
                        ch = true;
                    }
                }
                if (j == 0) e0 = v;
                else if (j == M) eM = v;
                else u[j] = v;
                left = v;
                cur = right;
            }
        }
        ++s;
        if (!ch) {
            conv = true;
            break;
        }
    }
    // winds of the ends at the final values (0 at Gamma and at +inf)
    int w0 = 0, wM = 0;
    if (!fix0 && e0 < inf) (void)ch1(inf, M == 1 ? eM : u[1], Num<T>::mul(r[0], A.h), w0);
    if (!fixM && eM < inf) (void)ch1(M == 1 ? e0 : u[M - 1], inf, Num<T>::mul(r[M], A.h), wM);
    const bool echo0 = in0 && e0 == s0, echoM = inM && eM == sM;
    if (echo0) w0 = W[sub];
    if (echoM) wM = W[sub + 1];
    eu[2 * sub] = e0;
    eu[2 * sub + 1] = eM;
    ew[2 * sub] = (int8_t)w0;
    ew[2 * sub + 1] = (int8_t)wM;
    ee[2 * sub] = echo0 ? 1 : 0;
    ee[2 * sub + 1] = echoM ? 1 : 0;
    return s;
}

template <class T>
__device__ __forceinline__ T abs_(T x) {
    return x < T(0) ? -x : x;
}

template <class T>
__global__ void __launch_bounds__(1024, 1) k_dd1(DD1Args<T> A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = A.N;
    const long long M = A.M;
    const T inf = Num<T>::inf();
    T *U = reinterpret_cast<T *>(smem);
    T *Un = U + (N + 1);     // the U being built by Step 4
    T *uk = Un + (N + 1);    // u^k of Step 3's choice
    T *Cold = uk + (N + 1);  // C_H(U^k)
    T *eu = Cold + (N + 1);  // end copies of the subintervals
    int8_t *W = reinterpret_cast<int8_t *>(eu + 2 * N);
    int8_t *wk = W + (N + 1);
    uint8_t *cfix = reinterpret_cast<uint8_t *>(wk + (N + 1));
    int8_t *ew = reinterpret_cast<int8_t *>(cfix + (N + 1));
    uint8_t *ee = reinterpret_cast<uint8_t *>(ew + 2 * N);
    __shared__ unsigned long long s_fine_upd, s_coarse_upd, s_fsm_max, s_coarse_max, s_fsm_caps, s_coarse_caps;
    __shared__ int s_causal_max;
    __shared__ T s_delta;
    const int tid = threadIdx.x, nt = blockDim.x;

    if (tid == 0) {
        s_fine_upd = s_coarse_upd = s_fsm_max = s_coarse_max = s_fsm_caps = s_coarse_caps = 0;
        s_causal_max = 0;
        s_delta = inf;
    }
    for (int i = tid; i <= N; i += nt) {
        const long long f = (long long)i * M;
        cfix[i] = A.gamma[f] ? 1 : 0;
        U[i] = A.gamma[f] ? A.g[f] : inf;
    }
    __syncthreads();
    // Step 1: FSM on the coarse grid, then the winds W^0
    if (tid == 0) {
        bool conv;
        const long long s = coarse_fsm(A, U, cfix, conv);
        s_coarse_max = (unsigned long long)s;
        s_coarse_caps = conv ? 0 : 1;
        s_coarse_upd = (unsigned long long)s * (N + 1);
    }
    __syncthreads();
    for (int i = tid; i <= N; i += nt) {
        int w = 0;
        if (!cfix[i] && U[i] < inf) (void)ch1_at(U, i, N, Num<T>::mul(A.r[(long long)i * M], A.H), w);
        W[i] = (int8_t)w;
    }
    __syncthreads();

    int k = 0, converged = 0;
    for (;; ++k) {
        // Steps 2-3: every subinterval on its own
        for (int sub = tid; sub < N; sub += nt) {
            bool cv;
            const long long s = solve_sub(A, sub, U, W, eu, ew, ee, cv);
            atomicMax(&s_fsm_max, (unsigned long long)s);
            if (!cv) atomicAdd(&s_fsm_caps, 1ull);
            atomicAdd(&s_fine_upd, (unsigned long long)s * (unsigned long long)(M + 1));
        }
        __syncthreads();
        // Step 3's choice of u^k_i and w^k_i between the two fine copies
        for (int i = tid; i <= N; i += nt) {
            if (i == 0) {
                uk[0] = eu[0];
                wk[0] = ew[0];
            } else if (i == N) {
                uk[N] = eu[2 * N - 1];
                wk[N] = ew[2 * N - 1];
            } else {
                const T uL = eu[2 * i - 1], uR = eu[2 * i];
                const int wL = ew[2 * i - 1], wR = ew[2 * i];
                const int eL = ee[2 * i - 1], eR = ee[2 * i];
                bool takeL;
                if (wL == 1 && wR == 1) takeL = true;          // wind from left to right
                else if (wL == -1 && wR == -1) takeL = false;  // wind from right to left
                else if (eL != eR) takeL = eR != 0;            // the computed copy of the two
                else takeL = !(uR < uL);                       // minimum, a tie to the left copy
                uk[i] = takeL ? uL : uR;
                wk[i] = (int8_t)(takeL ? wL : wR);
            }
        }
        __syncthreads();
        if (k == A.max_iter) break;
        if (k >= 1 && s_delta < A.tol) {
            converged = 1;
            break;
        }
        // Step 4: C_H(U^k), then weighted Gauss-Seidel sweeps from the FSM
        // initialisation
        for (int i = tid; i <= N; i += nt) {
            int w;
            Cold[i] = ch1_at(U, i, N, Num<T>::mul(A.r[(long long)i * M], A.H), w);
            Un[i] = cfix[i] ? A.g[(long long)i * M] : inf;
        }
        __syncthreads();
        if (tid == 0) {
            long long s = 0;
            for (;;) {
                if (s >= A.max_coarse) {
                    ++s_coarse_caps;
                    break;
                }
                bool changed = false;
                const int step = (s % 2 == 0) ? -1 : 1;
                for (int i = step > 0 ? 0 : N; i >= 0 && i <= N; i += step) {
                    if (cfix[i]) continue;
                    int Wt;
                    const T Ut = ch1_at(Un, i, N, Num<T>::mul(A.r[(long long)i * M], A.H), Wt);
                    T v = uk[i];
                    if (Ut < inf && Cold[i] < inf && W[i] == wk[i] && wk[i] == Wt)
                        v = Num<T>::add(uk[i], Num<T>::mul(A.theta, Num<T>::sub(Ut, Cold[i])));
                    if (!(v == Un[i])) changed = true;
                    Un[i] = v;
                }
                ++s;
                if (!changed) break;
            }
            if ((unsigned long long)s > s_coarse_max) s_coarse_max = (unsigned long long)s;
            s_coarse_upd += (unsigned long long)s * (N + 1);
            for (int i = 0; i <= N; ++i) W[i] = wk[i];
            // causal sweep in both directions until nothing changes (values
            // only rise to a neighbour's, so it ends; the cap is a guard)
            int rounds = 0;
            bool changed;
            const long long round_cap = (long long)(N + 2) * (N + 2);
            do {
                changed = false;
                ++rounds;
                for (int i = 1; i <= N; ++i)
                    if (W[i] == 1 && Un[i] < Un[i - 1] && Un[i - 1] < inf) {
                        Un[i] = Un[i - 1];
                        changed = true;
                    }
                for (int i = N - 1; i >= 0; --i)
                    if (W[i] == -1 && Un[i] < Un[i + 1] && Un[i + 1] < inf) {
                        Un[i] = Un[i + 1];
                        changed = true;
                    }
            } while (changed && rounds < round_cap);
            if (rounds > s_causal_max) s_causal_max = rounds;
            T d = T(0);
            for (int i = 0; i <= N; ++i)
                if (!(Un[i] == U[i])) {
                    const T t = abs_(Num<T>::sub(Un[i], U[i]));
                    if (t > d) d = t;
                }
            s_delta = d;
        }
        __syncthreads();
        T *t = U;  // U^{k+1} is the U just built
        U = Un;
        Un = t;
    }
    // the patched fine solution: coarse nodes take u^k
    for (int i = tid; i <= N; i += nt) A.u[(long long)i * M] = uk[i];
    if (tid == 0 && A.stats) {
        eik_dd_stats *o = A.stats;
        o->iters = k;
        o->converged = converged;
        o->error = EIK_OK;
        o->causal_rounds_max = s_causal_max;
        o->fsm_sweeps_max = (int64_t)s_fsm_max;
        o->coarse_sweeps_max = (int64_t)s_coarse_max;
        o->fsm_cap_hits = (int64_t)s_fsm_caps;
        o->coarse_cap_hits = (int64_t)s_coarse_caps;
        o->last_delta = k >= 1 ? (double)s_delta : INFINITY;
        o->fine_updates = (int64_t)s_fine_upd;
        o->coarse_updates = (int64_t)s_coarse_upd;
        o->launches = 1;
    }
}

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------
bool dd1_validate(const eik_grid *grid, const eik_dd_params *p) {
    if (!valid_grid_common(grid, 1)) return false;
    const long long n = grid->n[0];
    const int N = p->tiles[0];
    if (N < 1 || (n - 1) % N != 0) {
        set_error("tiles[0] = %d does not divide n[0]-1 = %lld", N, n - 1);
        return false;
    }
    if (N > DD1_MAX_SUB) {
        set_error("1-D solve: %d subintervals, at most %d (the coarse state is held in shared memory)", N,
                  DD1_MAX_SUB);
        return false;
    }
    const long long M = (n - 1) / N;
    if (p->coarse_ratio != M) {
        set_error("1-D solve: the coarse nodes are the subinterval ends, so coarse_ratio must be (n-1)/tiles[0] = %lld",
                  M);
        return false;
    }
    if (p->max_iter < 0 || p->max_iter > 100000 || p->max_fsm_sweeps < 1 || p->max_coarse_sweeps < 1 ||
        p->max_fsm_sweeps > MAX_SWEEPS || p->max_coarse_sweeps > MAX_SWEEPS) {
        set_error("max_iter must be in [0, 100000] and sweep caps in [1, %lld]", MAX_SWEEPS);
        return false;
    }
    if (!std::isfinite(p->theta) || std::isnan(p->tol)) {
        set_error("theta must be finite and tol a number");
        return false;
    }
    if (p->theta_adaptive) {
        set_error("the per-node weight of Sec. 4.2 is built for the 2-D and 3-D solves only");
        return false;
    }
    return true;
}

// The 1-D solve uses no workspace; a non-zero size marks the request valid.
size_t dd1_workspace_size() { return 256; }

template <class T>
static int dd1_run_t(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                     const eik_dd_params *p, void *u_out, eik_dd_stats *stats, cudaStream_t s) {
    DD1Args<T> A;
    memset(&A, 0, sizeof(A));
    A.r = static_cast<const T *>(r);
    A.gamma = gamma;
    A.g = static_cast<const T *>(g);
    A.u = static_cast<T *>(u_out);
    A.stats = stats;
    A.N = p->tiles[0];
    A.M = (grid->n[0] - 1) / A.N;
    A.h = (T)grid->h;
    A.H = (T)((double)A.M * grid->h);
    A.theta = (T)p->theta;
    A.tol = (T)p->tol;
    A.max_iter = p->max_iter;
    A.max_fsm = p->max_fsm_sweeps;
    A.max_coarse = p->max_coarse_sweeps;
    const size_t smem = dd1_smem_bytes<T>(A.N);
    int rc, dev, optin = 0;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if ((long long)smem > optin) {
        set_error("1-D solve needs %zu bytes of shared memory (limit %d)", smem, optin);
        return EIK_EUNSUPPORTED;
    }
    if ((rc = cuda_check(cudaFuncSetAttribute(k_dd1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                         "attr")))
        return rc;
    const int threads = std::min(1024, (A.N + 1 + 31) / 32 * 32);
    EIK_LAUNCH("dd1_iteration", s, k_dd1<T><<<1, threads, smem, s>>>(A));
    return cuda_check(cudaGetLastError(), "dd1 launch");
}

int dd1_run(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g, const eik_dd_params *p,
            void *u_out, eik_dd_stats *stats, cudaStream_t s) {
    if (grid->dtype == EIK_F64) return dd1_run_t<double>(grid, r, gamma, g, p, u_out, stats, s);
    return dd1_run_t<float>(grid, r, gamma, g, p, u_out, stats, s);
}

}  // namespace eik

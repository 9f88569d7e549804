// eik_dd1.cu -- the one-dimensional two-scale iteration of Sec. 3.1 (Steps
// 1-4): eq. 1d on [0, 1] with the coarse grid X_i = i H (i = 0..N) and the
// subintervals [iH, (i+1)H] of M fine cells each (h = H / M).  eik_dd_solve
// runs it when grid->ndim == 1.
//
// One cooperative launch runs the whole iteration.  The subintervals are
// spread over one CTA per SM (a few consecutive subintervals per CTA, one per
// thread): each thread solves its subinterval by the 1-D FSM of Sec. 1.1
// (Steps 2-3), a chain of dependent updates walking contiguous memory, so the
// work is latency-bound per thread and wants as many SMs as there are
// subintervals to spare.  CTA 0 holds the coarse state (U, the new U, u^k,
// C_H(U^k), the winds W^k and w^k, the fixed-node mask) in shared memory and
// runs the coarse work between two grid barriers: the Step 3 choice at the
// coarse nodes (its threads), then one thread for the serial part (Step 1's
// coarse FSM, Step 4's weighted Gauss-Seidel sweeps, the causal sweep, the
// update size).  U and W are published to global memory for the next fine
// phase; the subintervals' end copies come back through global memory.
// Every grid barrier is a bounded wait: on expiry the kernel records
// EIK_EDEVICE_TIMEOUT in the statistics and returns.
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

EIK_SPIN_LIMIT_SETTER(set_spin_limit_dd1)

constexpr int DD1_MAX_SUB = 2048;  // subintervals: the coarse state must fit in shared memory

// Control words at the start of the workspace (cleared before every launch).
struct DD1Ctl {
    unsigned bar[2];  // grid barrier: arrivals, generation
    int err;          // EIK_OK or DEV_TIMEOUT
    int stop;         // set by CTA 0: 1 = the iteration ends after this fine phase
    unsigned long long fsm_max, fsm_caps, fine_upd;
};

template <class T>
struct DD1Args {
    const T *r;
    const uint8_t *gamma;
    const T *g;
    T *u;
    eik_dd_stats *stats;
    DD1Ctl *ctl;
    T *gU;            // U^k published for the fine phase (N + 1)
    int8_t *gW;       // W^k (N + 1)
    T *geu;           // end copies of the subintervals: 2 sub (left), 2 sub + 1 (right)
    int8_t *gew;      // their winds
    uint8_t *gee;     // their echo flags
    int N;            // subintervals
    int per;          // subintervals per CTA
    long long M;      // fine cells per subinterval
    T h, H, theta, tol;
    int max_iter;
    long long max_fsm, max_coarse;
};

// Shared memory of CTA 0: U, the new U, u^k, C_H(U^k), r(X_i) H (N + 1
// each), W^k, w^k and the fixed-node mask (N + 1 bytes each).
template <class T>
static size_t dd1_smem_bytes(int N) {
    return (size_t)5 * (N + 1) * sizeof(T) + (size_t)3 * (N + 1);
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

template <class T>
static size_t dd1_ws_bytes(int N) {
    return al256(sizeof(DD1Ctl)) + al256((size_t)(N + 1) * sizeof(T)) + al256((size_t)(N + 1)) +
           al256((size_t)2 * N * sizeof(T)) + al256((size_t)2 * N) + al256((size_t)2 * N);
}

// C_H of eq. 1dgod from the two neighbour values, with the wind of the one
// used (+1 left, -1 right, 0 when the value is +inf).  The 1-D Godunov update
// of a fine node is the same expression with spacing h.
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

template <class T>
__device__ __forceinline__ T abs_(T x) {
    return x < T(0) ? -x : x;
}

// Coarse FSM of Step 1 on U[0..N] (spacing H, r sampled at X_i), Gamma nodes
// fixed.  Sweeps alternate right-to-left, left-to-right until one changes
// nothing or the cap is reached.  One thread.
template <class T>
__device__ long long coarse_fsm(const DD1Args<T> &A, T *U, const T *rHc, const uint8_t *cfix, bool &conv) {
    const int N = A.N;
    long long s = 0;
    conv = false;
    while (s < A.max_coarse) {
        bool ch = false;
        const int step = (s % 2 == 0) ? -1 : 1;
        for (int i = step > 0 ? 0 : N; i >= 0 && i <= N; i += step) {
            if (cfix[i]) continue;
            int w;
            const T ut = ch1_at(U, i, N, rHc[i], w);
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

// One Gauss-Seidel sweep of the 1-D FSM over a subinterval (nodes 0..M, the
// ends e0 and eM in registers, the interior in u), in direction DIR (-1 right
// to left, +1 left to right); returns whether a value changed.  Node j is
// updated from its two neighbours as they are at that moment: the one behind
// (already updated in this sweep, carried in a register) and the one ahead
// (not yet reached, its old value).  The nodes after the first are taken in
// sweep order as positions p = 0..M-1 (p = M-1 the far end), in blocks of
// DD1_BLK: the next block's old values, r and Gamma flags are loaded before
// the current block is processed, and the lines further ahead are prefetched,
// so the chain of dependent updates does not wait on memory.
constexpr int DD1_BLK = 8;

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}


template <class T, int DIR>
__device__ __forceinline__ bool sweep_dir(const DD1Args<T> &A, T *u, const T *r, const uint8_t *gm, T &e0, T &eM) {
    const T inf = Num<T>::inf();
    const long long M = A.M;
    const long long jn = DIR < 0 ? M : 0;          // the near end, first in the sweep
    T &nearv = DIR < 0 ? eM : e0;
    T &farv = DIR < 0 ? e0 : eM;
    auto jpos = [&](long long p) { return DIR < 0 ? M - 1 - p : 1 + p; };
    bool ch = false;
    T cu[DD1_BLK], cr[DD1_BLK], nu[DD1_BLK], nr[DD1_BLK];
    uint8_t cg[DD1_BLK], ng[DD1_BLK];
    // block loader: old value (the far end's from its register), r and flag
    // of positions p0..p0+DD1_BLK-1; +inf past the far end
    auto load = [&](long long p0, T *bu, T *br, uint8_t *bg) {
#pragma unroll
        for (int i = 0; i < DD1_BLK; ++i) {
            const long long p = p0 + i;
            bu[i] = inf;
            br[i] = T(1);
            bg[i] = 1;
            if (p <= M - 1) {
                const long long j = jpos(p);
                bu[i] = p < M - 1 ? u[j] : farv;
                br[i] = r[j];
                bg[i] = gm[j];
            }
        }
    };
    load(0, cu, cr, cg);
    // the near end: nothing behind it, position 0 ahead
    T carry;
    {
        T v = nearv;
        if (!gm[jn]) {
            int w;
            const T ut = DIR < 0 ? ch1(cu[0], inf, Num<T>::mul(r[jn], A.h), w)
                                 : ch1(inf, cu[0], Num<T>::mul(r[jn], A.h), w);
            if (ut < v) {
                v = ut;
                ch = true;
            }
        }
        nearv = v;
        carry = v;
    }
    for (long long p0 = 0; p0 <= M - 1; p0 += DD1_BLK) {
        load(p0 + DD1_BLK, nu, nr, ng);
        if (p0 + 16 * DD1_BLK <= M - 1) {  // into L2 further ahead
            const long long jf = jpos(p0 + 16 * DD1_BLK);
            prefetch_l2(u + jf);
            prefetch_l2(r + jf);
            prefetch_l2(gm + jf);
        }
#pragma unroll
        for (int i = 0; i < DD1_BLK; ++i) {
            const long long p = p0 + i;
            if (p <= M - 1) {
                const T ahead = i + 1 < DD1_BLK ? cu[i + 1] : nu[0];
                T v = cu[i];
                if (!cg[i]) {
                    int w;
                    const T rh = Num<T>::mul(cr[i], A.h);
                    const T ut = DIR < 0 ? ch1(ahead, carry, rh, w) : ch1(carry, ahead, rh, w);
                    if (ut < v) {
                        v = ut;
                        ch = true;
                    }
                }
                if (p < M - 1) u[jpos(p)] = v;
                else farv = v;
                carry = v;
            }
        }
#pragma unroll
        for (int i = 0; i < DD1_BLK; ++i) {
            cu[i] = nu[i];
            cr[i] = nr[i];
            cg[i] = ng[i];
        }
    }
    return ch;
}

// Steps 2-3 on subinterval `sub` (one thread), given U and W at its two ends.
// Step 2: a Gamma node is fixed at g; an end where the coarse wind points into
// the subinterval (W = +1 at its left end, W = -1 at its right end) starts at
// U, every other node at +inf.  Step 3: FSM sweeps (right-to-left first) until
// one changes nothing or the cap is reached.  The interior nodes are left in
// u; the ends' values, winds and echo flags go to the end-copy arrays.
// Returns the sweeps run; conv = false if the cap stopped them.
template <class T>
__device__ long long solve_sub(const DD1Args<T> &A, int sub, T Ul, T Ur, int Wl, int Wr, bool &conv) {
    const T inf = Num<T>::inf();
    const long long M = A.M, f0 = (long long)sub * M;
    T *u = A.u + f0;
    const T *r = A.r + f0;
    const uint8_t *gm = A.gamma + f0;
    const T *g = A.g + f0;
    const bool fix0 = gm[0] != 0, fixM = gm[M] != 0;
    const bool in0 = !fix0 && Wl > 0, inM = !fixM && Wr < 0;
    const T s0 = fix0 ? g[0] : (in0 ? Ul : inf);
    const T sM = fixM ? g[M] : (inM ? Ur : inf);
    T e0 = s0, eM = sM;
    for (long long j = 1; j < M; ++j) u[j] = gm[j] ? g[j] : inf;
    long long s = 0;
    conv = false;
    while (s < A.max_fsm) {
        const bool ch = (s % 2 == 0) ? sweep_dir<T, -1>(A, u, r, gm, e0, eM) : sweep_dir<T, 1>(A, u, r, gm, e0, eM);
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
    if (echo0) w0 = Wl;
    if (echoM) wM = Wr;
    A.geu[2 * sub] = e0;
    A.geu[2 * sub + 1] = eM;
    A.gew[2 * sub] = (int8_t)w0;
    A.gew[2 * sub + 1] = (int8_t)wM;
    A.gee[2 * sub] = echo0 ? 1 : 0;
    A.gee[2 * sub + 1] = echoM ? 1 : 0;
    return s;
}

template <class T>
__global__ void __launch_bounds__(64) k_dd1(DD1Args<T> A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = A.N;
    const long long M = A.M;
    const T inf = Num<T>::inf();
    const long long lim = spin_limit();
    DD1Ctl *ctl = A.ctl;
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool lead = blockIdx.x == 0;
    // CTA 0's coarse state
    T *U = reinterpret_cast<T *>(smem);
    T *Un = U + (N + 1);     // the U being built by Step 4
    T *uk = Un + (N + 1);    // u^k of Step 3's choice
    T *Cold = uk + (N + 1);  // C_H(U^k)
    T *rHc = Cold + (N + 1); // r(X_i) H
    int8_t *W = reinterpret_cast<int8_t *>(rHc + (N + 1));
    int8_t *wk = W + (N + 1);
    uint8_t *cfix = reinterpret_cast<uint8_t *>(wk + (N + 1));
    __shared__ unsigned long long s_coarse_upd, s_coarse_max, s_coarse_caps;
    __shared__ int s_causal_max;
    __shared__ T s_delta;

    if (lead) {
        if (tid == 0) {
            s_coarse_upd = s_coarse_max = s_coarse_caps = 0;
            s_causal_max = 0;
            s_delta = inf;
            ctl->fsm_max = ctl->fsm_caps = ctl->fine_upd = 0;
        }
        for (int i = tid; i <= N; i += nt) {
            const long long f = (long long)i * M;
            cfix[i] = A.gamma[f] ? 1 : 0;
            U[i] = A.gamma[f] ? A.g[f] : inf;
            rHc[i] = Num<T>::mul(A.r[f], A.H);
        }
        __syncthreads();
        // Step 1: FSM on the coarse grid, then the winds W^0
        if (tid == 0) {
            bool conv;
            const long long s = coarse_fsm(A, U, rHc, cfix, conv);
            s_coarse_max = (unsigned long long)s;
            s_coarse_caps = conv ? 0 : 1;
            s_coarse_upd = (unsigned long long)s * (N + 1);
        }
        __syncthreads();
        for (int i = tid; i <= N; i += nt) {
            int w = 0;
            if (!cfix[i] && U[i] < inf) (void)ch1_at(U, i, N, rHc[i], w);
            W[i] = (int8_t)w;
            A.gU[i] = U[i];
            A.gW[i] = (int8_t)w;
        }
    }
    bool ok = grid_barrier(ctl->bar, &ctl->err, lim);
    int k = 0, converged = 0;
    const int sub = blockIdx.x * A.per + tid;
    while (ok) {
        // Steps 2-3: every subinterval on its own (U, W written by another SM:
        // read past L1)
        if (tid < A.per && sub < N) {
            bool cv;
            const long long s = solve_sub(A, sub, __ldcg(A.gU + sub), __ldcg(A.gU + sub + 1),
                                          (int)__ldcg(A.gW + sub), (int)__ldcg(A.gW + sub + 1), cv);
            atomicMax(&ctl->fsm_max, (unsigned long long)s);
            if (!cv) atomicAdd(&ctl->fsm_caps, 1ull);
            atomicAdd(&ctl->fine_upd, (unsigned long long)s * (unsigned long long)(M + 1));
        }
        if (!(ok = grid_barrier(ctl->bar, &ctl->err, lim))) break;
        if (lead) {
            // Step 3's choice of u^k_i and w^k_i between the two fine copies
            for (int i = tid; i <= N; i += nt) {
                if (i == 0) {
                    uk[0] = __ldcg(A.geu);
                    wk[0] = __ldcg(A.gew);
                } else if (i == N) {
                    uk[N] = __ldcg(A.geu + 2 * N - 1);
                    wk[N] = __ldcg(A.gew + 2 * N - 1);
                } else {
                    const T uL = __ldcg(A.geu + 2 * i - 1), uR = __ldcg(A.geu + 2 * i);
                    const int wL = __ldcg(A.gew + 2 * i - 1), wR = __ldcg(A.gew + 2 * i);
                    const int eL = __ldcg(A.gee + 2 * i - 1), eR = __ldcg(A.gee + 2 * i);
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
            int stop = 0;
            if (k == A.max_iter) stop = 1;
            else if (k >= 1 && s_delta < A.tol) stop = 2;
            if (!stop) {
                // Step 4: C_H(U^k), then weighted Gauss-Seidel sweeps from the
                // FSM initialisation
                for (int i = tid; i <= N; i += nt) {
                    int w;
                    Cold[i] = ch1_at(U, i, N, rHc[i], w);
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
                            const T Ut = ch1_at(Un, i, N, rHc[i], Wt);
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
                    // causal sweep in both directions until nothing changes
                    // (values only rise to a neighbour's, so it ends; the cap
                    // is a guard)
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
                for (int i = tid; i <= N; i += nt) {
                    A.gU[i] = U[i];
                    A.gW[i] = W[i];
                }
            }
            if (tid == 0) ctl->stop = stop;
        }
        if (!(ok = grid_barrier(ctl->bar, &ctl->err, lim))) break;
        const int stop = *(volatile int *)&ctl->stop;
        if (stop) {
            converged = stop == 2 ? 1 : 0;
            break;
        }
        ++k;
    }
    if (!lead) return;
    // the patched fine solution: coarse nodes take u^k
    if (ok)
        for (int i = tid; i <= N; i += nt) A.u[(long long)i * M] = uk[i];
    if (tid == 0 && A.stats) {
        eik_dd_stats *o = A.stats;
        o->iters = k;
        o->converged = converged;
        o->error = *(volatile int *)&ctl->err;
        o->causal_rounds_max = s_causal_max;
        o->fsm_sweeps_max = (int64_t)*(volatile unsigned long long *)&ctl->fsm_max;
        o->coarse_sweeps_max = (int64_t)s_coarse_max;
        o->fsm_cap_hits = (int64_t)*(volatile unsigned long long *)&ctl->fsm_caps;
        o->coarse_cap_hits = (int64_t)s_coarse_caps;
        o->last_delta = k >= 1 ? (double)s_delta : INFINITY;
        o->fine_updates = (int64_t)*(volatile unsigned long long *)&ctl->fine_upd;
        o->coarse_updates = (int64_t)s_coarse_upd;
        o->launches = 1;
        o->fine_solves_skipped = 0;
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

size_t dd1_workspace_size(const eik_grid *grid, const eik_dd_params *p) {
    return grid->dtype == EIK_F64 ? dd1_ws_bytes<double>(p->tiles[0]) : dd1_ws_bytes<float>(p->tiles[0]);
}

template <class T>
static int dd1_run_t(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                     const eik_dd_params *p, void *u_out, void *ws, eik_dd_stats *stats, cudaStream_t s) {
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
    const int N = A.N;
    char *w = static_cast<char *>(ws);
    A.ctl = reinterpret_cast<DD1Ctl *>(w);
    w += al256(sizeof(DD1Ctl));
    A.gU = reinterpret_cast<T *>(w);
    w += al256((size_t)(N + 1) * sizeof(T));
    A.gW = reinterpret_cast<int8_t *>(w);
    w += al256((size_t)(N + 1));
    A.geu = reinterpret_cast<T *>(w);
    w += al256((size_t)2 * N * sizeof(T));
    A.gew = reinterpret_cast<int8_t *>(w);
    w += al256((size_t)2 * N);
    A.gee = reinterpret_cast<uint8_t *>(w);

    const size_t smem = dd1_smem_bytes<T>(N);
    int rc, dev, nsm = 0, optin = 0, coop = 0;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if ((long long)smem > optin || !coop) {
        set_error("1-D solve needs %zu bytes of shared memory (limit %d) and cooperative launch", smem, optin);
        return EIK_EUNSUPPORTED;
    }
    if ((rc = cuda_check(set_dyn_smem(k_dd1<T>, (int)smem),
                         "attr")))
        return rc;
    // subintervals spread over one CTA per SM, one thread each
    A.per = (N + nsm - 1) / nsm;
    const int nblk = (N + A.per - 1) / A.per;
    const int threads = std::max(32, (A.per + 31) / 32 * 32);
    int per_sm = 0;
    if ((rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dd1<T>, threads, smem), "occ")))
        return rc;
    if (per_sm * nsm < nblk) {
        set_error("1-D solve needs %d co-resident CTAs, the device holds %d", nblk, per_sm * nsm);
        return EIK_EUNSUPPORTED;
    }
    if ((rc = cuda_check(cudaMemsetAsync(A.ctl, 0, sizeof(DD1Ctl), s), "clear control words"))) return rc;
    void *args[] = {&A};
    const int tok = prof_begin("dd1_iteration", s);
    rc = cuda_check(cudaLaunchCooperativeKernel((void *)k_dd1<T>, nblk, threads, args, smem, s), "dd1 launch");
    prof_end(tok, s);
    return rc;
}

int dd1_run(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g, const eik_dd_params *p,
            void *u_out, void *ws, eik_dd_stats *stats, cudaStream_t s) {
    if (grid->dtype == EIK_F64) return dd1_run_t<double>(grid, r, gamma, g, p, u_out, ws, stats, s);
    return dd1_run_t<float>(grid, r, gamma, g, p, u_out, ws, stats, s);
}

}  // namespace eik

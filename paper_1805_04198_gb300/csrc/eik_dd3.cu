// eik_dd3.cu -- the two-scale DD iteration (Sec. 3.2, Steps 1-4, Alg. 1-5)
// in three dimensions.  The paper states the method in 2-D and says it
// "can be generalized"; the generalisation used here:
//   * coarse set: every node with some index = 0 mod c, the union of the
//     c^3 - (c-1)^3 shifted coarse grids (offsets with at least one zero);
//   * Alg. 4 / Alg. 5 agreement tests on every interface / coarse-line axis
//     of a node; the causal sweep (Alg. 2) along every axis e whose fine
//     neighbours stay on the coarse set (the node lies on a coarse plane of
//     another axis);
//   * the 3-D Godunov local solve (sorted-minima cascade).
// Subdomains and shifted coarse grids are small boxes that fit in shared
// memory, so each is swept by one CTA along hyperplanes i + j + k = const
// (nodes of a hyperplane are independent; a barrier separates hyperplanes),
// which is the serial Gauss-Seidel order of the paper's loop nest.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "host_util.h"
#include "prof.h"

namespace eik {

EIK_SPIN_LIMIT_SETTER(set_spin_limit_dd3)

struct Grid3 {
    int ox, oy, oz, mx, my, mz;
    long long off;  // element offset in the coarse arrays ([z][y][x] box)
};

struct DD3Geom {
    int n[3], T[3], S[3], c, ng;
    long long nc;           // coarse elements
    double h, H;
};

struct DevStats3 {
    unsigned long long fsm_sweeps_max, coarse_sweeps_max, fsm_caps, coarse_caps, fine_updates, coarse_updates;
    unsigned long long fine_skips;
    int causal_rounds_max, err, iters, converged;
};

template <class T>
struct DD3Args {
    DD3Geom G;
    const T *r;
    const uint8_t *gamma;
    const T *g;
    T *u_out;
    long long sy, sz;
    Grid3 *grids;
    int *offmap;  // [c^3] offset -> grid index (-1 if not a shifted grid)
    T *U, *Uprev, *U0, *rc, *uk, *cold;
    uint8_t *W, *wk, *mask;
    T *cu;
    uint8_t *cw;
    int *done;
    double *deltas;
    int *chg;
    unsigned *bar;
    DevStats3 *st;
    // Step 2 data of each subdomain's last solve in this call (the starting
    // value of every face node and the coarse wind an inflow node echoes),
    // [ntiles][face slots], and whether the subdomain has been solved
    T *sig_u;
    uint8_t *sig_w;
    int *sig_ok;
    T theta, tol;
    // constant weight 0: Alg. 5 yields u^k at every node, Alg. 4 writes
    // U^{k+1} = u^k itself and Step 4 is not launched
    int step4_identity;
    int max_iter;
    long long max_fsm, max_coarse;
    // per-node weight of Sec. 4.2 (adaptive = 1): weights, damping, cap, the
    // last four C_H(nbrs U) (slot m % 4), du = u^k - u^{k-1}, the weight
    int adaptive;
    double om[3], sg, sd, sx0, cap;
    T *Ch[4];
    double *du;
    T *th;
};

template <class T>
__device__ __forceinline__ size_t fidx(const DD3Args<T> &A, int X, int Y, int Z) {
    return (size_t)Z * A.sz + (size_t)Y * A.sy + X;
}

template <class T>
__device__ __forceinline__ long long coarse_addr3(const DD3Args<T> &A, int X, int Y, int Z) {
    const int c = A.G.c;
    const int g = A.offmap[((Z % c) * c + (Y % c)) * c + (X % c)];
    const Grid3 d = A.grids[g];
    return d.off + ((long long)(Z / c) * d.my + (Y / c)) * d.mx + (X / c);
}

__device__ __forceinline__ int coarse_axes3(int X, int Y, int Z, int c) {
    return (X % c == 0 ? 1 : 0) | (Y % c == 0 ? 2 : 0) | (Z % c == 0 ? 4 : 0);
}

// --------------------------------------------------------------------------
// Box sweeps in shared memory along hyperplanes.  Sweep k uses ordering
// k mod 8 of the paper's loop nest: sign of x = bit 2, y = bit 1, z = bit 0.
// Thread t owns the columns (x, y) = c mod mx, c / mx for c = t, t + blockDim,
// ...; hyperplane i + j + k = dg (logical indices of the ordering) holds one
// node of each column, so a thread updates at most one node per owned column
// per hyperplane.  The per-node read-only data the policy needs ("statics",
// from global memory) are loaded one hyperplane ahead into registers, so their
// latency overlaps the current hyperplane and its barrier.  The policy gives
// load(x, y, z, idx) -> Stat and apply(self, vm, vp, stat, idx, changed).
// --------------------------------------------------------------------------
constexpr int BOX3_COLS = 4;       // columns per thread with prefetched statics
constexpr int BOX3_THREADS = 512;  // threads of a box-sweep CTA

// Shared-memory plane stride of a box: the x-y plane padded to an even number
// of elements.  Along a hyperplane, neighbouring columns' nodes are one plane
// apart in z and one element apart in x (or y), so with an odd plane size
// (e.g. 33 x 33) a warp's accesses would all fall into one bank.
__host__ __device__ inline int box3_ps(int mx, int my) { return mx * my + ((mx * my) & 1); }

template <class T, class P>
__device__ void box3_sweeps(T *su, int mx, int my, int mz, const P &pol, long long max_sweeps, long long &sweeps,
                            bool &conv) {
    using S = typename P::Stat;
    const T INF = Num<T>::inf();
    const int ndiag = mx + my + mz - 2;
    const int ncol = mx * my;
    const int plane = box3_ps(mx, my);
    int cx[BOX3_COLS], cy[BOX3_COLS];
#pragma unroll
    for (int t = 0; t < BOX3_COLS; ++t) {
        const int c = threadIdx.x + t * blockDim.x;
        cx[t] = c < ncol ? c % mx : 0;
        cy[t] = c < ncol ? c / mx : 0;
    }
    // one node: gather neighbours from shared memory and apply the policy
    auto node = [&](int x, int y, int z, S st, bool &ch) {
        const int idx = z * plane + y * mx + x;
        T vm[3], vp[3];
        vm[0] = x > 0 ? su[idx - 1] : INF;
        vp[0] = x + 1 < mx ? su[idx + 1] : INF;
        vm[1] = y > 0 ? su[idx - mx] : INF;
        vp[1] = y + 1 < my ? su[idx + mx] : INF;
        vm[2] = z > 0 ? su[idx - plane] : INF;
        vp[2] = z + 1 < mz ? su[idx + plane] : INF;
        const T self = su[idx];
        S sl = st;
        pol.fill(sl, idx);
        bool c1 = false;
        const T nw = pol.apply(self, vm, vp, sl, idx, c1);
        if (c1) {
            su[idx] = nw;
            ch = true;
        }
    };
    sweeps = 0;
    conv = false;
    for (long long k = 0; k < max_sweeps; ++k) {
        const int q = (int)(k & 7);
        const int sx = (q & 4) ? 1 : -1, sy = (q & 2) ? 1 : -1, sz = (q & 1) ? 1 : -1;
        int base[BOX3_COLS];  // logical x + y of each owned column (kp = dg - base)
#pragma unroll
        for (int t = 0; t < BOX3_COLS; ++t) {
            const int c = threadIdx.x + t * blockDim.x;
            base[t] = c < ncol ? (sx > 0 ? cx[t] : mx - 1 - cx[t]) + (sy > 0 ? cy[t] : my - 1 - cy[t]) : -(1 << 28);
        }
        auto zof = [&](int kp) { return sz > 0 ? kp : mz - 1 - kp; };
        S cur[BOX3_COLS], nxt[BOX3_COLS];
#pragma unroll
        for (int t = 0; t < BOX3_COLS; ++t) {
            const int kp = 0 - base[t];
            if (kp >= 0 && kp < mz) cur[t] = pol.load(cx[t], cy[t], zof(kp), (zof(kp) * my + cy[t]) * mx + cx[t]);
        }
        bool ch = false;
        for (int dg = 0; dg < ndiag; ++dg) {
#pragma unroll
            for (int t = 0; t < BOX3_COLS; ++t) {
                const int kp = dg + 1 - base[t];
                if (kp >= 0 && kp < mz) nxt[t] = pol.load(cx[t], cy[t], zof(kp), (zof(kp) * my + cy[t]) * mx + cx[t]);
            }
            // gather every owned node of this hyperplane, then compute, then
            // store (nodes of one hyperplane never read each other)
            T vmv[BOX3_COLS][3], vpv[BOX3_COLS][3], sf[BOX3_COLS], nw[BOX3_COLS];
            int qi[BOX3_COLS];
            bool on[BOX3_COLS], c1[BOX3_COLS];
#pragma unroll
            for (int t = 0; t < BOX3_COLS; ++t) {
                const int kp = dg - base[t];
                on[t] = kp >= 0 && kp < mz;
                c1[t] = false;
                if (on[t]) {
                    const int x = cx[t], y = cy[t], z = zof(kp);
                    const int idx = z * plane + y * mx + x;
                    qi[t] = idx;
                    vmv[t][0] = x > 0 ? su[idx - 1] : INF;
                    vpv[t][0] = x + 1 < mx ? su[idx + 1] : INF;
                    vmv[t][1] = y > 0 ? su[idx - mx] : INF;
                    vpv[t][1] = y + 1 < my ? su[idx + mx] : INF;
                    vmv[t][2] = z > 0 ? su[idx - plane] : INF;
                    vpv[t][2] = z + 1 < mz ? su[idx + plane] : INF;
                    sf[t] = su[idx];
                    pol.fill(cur[t], idx);
                }
            }
#pragma unroll
            for (int t = 0; t < BOX3_COLS; ++t)
                if (on[t]) nw[t] = pol.apply(sf[t], vmv[t], vpv[t], cur[t], qi[t], c1[t]);
#pragma unroll
            for (int t = 0; t < BOX3_COLS; ++t)
                if (on[t] && c1[t]) {
                    su[qi[t]] = nw[t];
                    ch = true;
                }
            // columns beyond the prefetched ones (wide boxes)
            for (int c = threadIdx.x + BOX3_COLS * blockDim.x; c < ncol; c += blockDim.x) {
                const int x = c % mx, y = c / mx;
                const int kp = dg - ((sx > 0 ? x : mx - 1 - x) + (sy > 0 ? y : my - 1 - y));
                if (kp >= 0 && kp < mz) {
                    const int z = zof(kp);
                    node(x, y, z, pol.load(x, y, z, (z * my + y) * mx + x), ch);
                }
            }
            __syncthreads();
#pragma unroll
            for (int t = 0; t < BOX3_COLS; ++t) cur[t] = nxt[t];
        }
        ++sweeps;
        if (!__syncthreads_or(ch ? 1 : 0)) {
            conv = true;
            break;
        }
    }
}

// FSM update (Sec. 1.1): u = min(u, u~) at free nodes.
template <class T>
struct Fsm3 {
    const uint8_t *fixed;  // shared, per box node; 1 = fixed (Gamma), 2 = swept inflow node
    const T *r;            // per box node, via rix
    long long r0, rsx, rsy, rsz;  // global index of box node (x,y,z) = r0 + x*rsx + y*rsy + z*rsz
    T hs;
    struct Stat {
        T r;
        uint8_t fixed;
    };
    __device__ __forceinline__ Stat load(int x, int y, int z, int) const {
        return Stat{r[r0 + x * rsx + y * rsy + z * rsz], 0};
    }
    // shared-memory part of the node's data, read when the node is gathered
    __device__ __forceinline__ void fill(Stat &st, int idx) const { st.fixed = fixed[idx]; }
    __device__ __forceinline__ T apply(T self, const T *vm, const T *vp, const Stat &st, int,
                                       bool &changed) const {
        if (st.fixed == 1) return self;
        uint8_t w;
        const T ut = local_solve3(vm, vp, Num<T>::mul(st.r, hs), w);
        changed = ut < self;
        return changed ? ut : self;
    }
};

// Alg. 5 update on a shifted grid box (box layout arrays from `off`).
template <class T>
struct Alg5_3 {
    const T *rc, *uk, *cold;
    const uint8_t *mask;
    long long off;
    T Hs, theta;
    const T *th;  // per-node weight (nullptr: the constant theta)
    struct Stat {
        T rc, uk, cold, th;
        uint8_t m;
    };
    __device__ __forceinline__ Stat load(int, int, int, int idx) const {
        const long long a = off + idx;
        return Stat{rc[a], uk[a], cold[a], th ? th[a] : theta, mask[a]};
    }
    __device__ __forceinline__ void fill(Stat &, int) const {}
    __device__ __forceinline__ T apply(T self, const T *vm, const T *vp, const Stat &st, int,
                                       bool &changed) const {
        using N = Num<T>;
        const uint8_t m = st.m;
        if (m & 1) return self;
        uint8_t w;
        const T Ut = local_solve3(vm, vp, N::mul(st.rc, Hs), w);
        const T ukv = st.uk, cv = st.cold;
        bool pass = (Ut < N::inf()) && (cv < N::inf());
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const int wc = wind_comp(w, ax);
            pass = pass && ((wc <= 0 && (m & (2 << (2 * ax)))) || (wc >= 0 && (m & (4 << (2 * ax)))));
        }
        const T nu = pass ? N::add(ukv, N::mul(st.th, N::sub(Ut, cv))) : ukv;
        changed = !(nu == self);
        return nu;
    }
};

// --------------------------------------------------------------------------
// Set-up
// --------------------------------------------------------------------------
template <class T>
__global__ void k3_init(DD3Args<T> A) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        memset(A.st, 0, sizeof(DevStats3));
        *A.done = 0;
        A.bar[0] = A.bar[1] = 0;
    }
    for (int k = threadIdx.x; k < A.max_iter + 2; k += blockDim.x) A.deltas[k] = k == 0 ? INFINITY : 0.0;
    for (int t = threadIdx.x; t < A.G.T[0] * A.G.T[1] * A.G.T[2]; t += blockDim.x) A.sig_ok[t] = 0;
}

// one CTA row per shifted grid (blockIdx.y), threads over its nodes
template <class T>
__global__ void k3_pack_coarse(DD3Args<T> A) {
    const Grid3 d = A.grids[blockIdx.y];
    const long long n = (long long)d.mx * d.my * d.mz;
    const int c = A.G.c;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % d.mx), j = (int)((e / d.mx) % d.my), k = (int)(e / ((long long)d.mx * d.my));
        const int X = d.ox + c * i, Y = d.oy + c * j, Z = d.oz + c * k;
        const size_t f = fidx(A, X, Y, Z);
        const bool gam = A.gamma[f] != 0;
        const long long a = d.off + e;
        A.rc[a] = gam ? T(-1) : A.r[f];
        A.U0[a] = gam ? A.g[f] : Num<T>::inf();
        A.W[a] = WIND_ZERO;
    }
}

template <class T>
__device__ void grid3_winds(const DD3Args<T> &A, const Grid3 &d, const T *su, T Hs) {
    const T INF = Num<T>::inf();
    const int n = d.mx * d.my * d.mz;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int x = e % d.mx, y = (e / d.mx) % d.my, z = e / (d.mx * d.my);
        const long long a = d.off + e;
        uint8_t w = WIND_ZERO;
        const T rv = A.rc[a];
        const int ps = box3_ps(d.mx, d.my);
        const int q = z * ps + y * d.mx + x;
        if (rv > T(0) && su[q] < INF) {
            T vm[3], vp[3];
            vm[0] = x > 0 ? su[q - 1] : INF;
            vp[0] = x + 1 < d.mx ? su[q + 1] : INF;
            vm[1] = y > 0 ? su[q - d.mx] : INF;
            vp[1] = y + 1 < d.my ? su[q + d.mx] : INF;
            vm[2] = z > 0 ? su[q - ps] : INF;
            vp[2] = z + 1 < d.mz ? su[q + ps] : INF;
            (void)local_solve3(vm, vp, Num<T>::mul(rv, Hs), w);
        }
        A.W[a] = w;
    }
}

// Step 1: FSM with Alg. 1 on every shifted grid (one CTA per grid).
template <class T>
__global__ void __launch_bounds__(BOX3_THREADS, 1) k3_step1(DD3Args<T> A) {
    extern __shared__ __align__(16) char smem[];
    const Grid3 d = A.grids[blockIdx.x];
    const int n = d.mx * d.my * d.mz;
    const int ps = box3_ps(d.mx, d.my);
    T *su = reinterpret_cast<T *>(smem);
    uint8_t *fx = reinterpret_cast<uint8_t *>(su + (size_t)d.mz * ps);
    auto sq = [&](int e) { return (e / (d.mx * d.my)) * ps + e % (d.mx * d.my); };
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        su[sq(e)] = A.U0[d.off + e];
        fx[sq(e)] = A.rc[d.off + e] > T(0) ? 0 : 1;
    }
    __syncthreads();
    Fsm3<T> pol{fx, A.rc, d.off, 1, d.mx, (long long)d.mx * d.my, T(A.G.H)};
    long long sweeps;
    bool conv;
    box3_sweeps(su, d.mx, d.my, d.mz, pol, A.max_coarse, sweeps, conv);
    for (int e = threadIdx.x; e < n; e += blockDim.x) A.U[d.off + e] = su[sq(e)];
    grid3_winds(A, d, su, T(A.G.H));
    if (threadIdx.x == 0) {
        atomicMax(&A.st->coarse_sweeps_max, (unsigned long long)sweeps);
        if (!conv) atomicAdd(&A.st->coarse_caps, 1ull);
        atomicAdd(&A.st->coarse_updates, (unsigned long long)sweeps * n);
    }
}

// Step 4: Alg. 5 on every shifted grid.
template <class T>
__global__ void __launch_bounds__(BOX3_THREADS, 1) k3_step4(DD3Args<T> A, int k) {
    if (*A.done) return;
    extern __shared__ __align__(16) char smem[];
    const Grid3 d = A.grids[blockIdx.x];
    const int n = d.mx * d.my * d.mz;
    const T INF = Num<T>::inf();
    const T Hs = T(A.G.H);
    const int ps = box3_ps(d.mx, d.my);
    T *su = reinterpret_cast<T *>(smem);
    auto sq = [&](int e) { return (e / (d.mx * d.my)) * ps + e % (d.mx * d.my); };
    for (int e = threadIdx.x; e < n; e += blockDim.x) su[sq(e)] = A.U[d.off + e];
    __syncthreads();
    // C_H(nbrs^H(U^k)) and U^k for the delta
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int x = e % d.mx, y = (e / d.mx) % d.my, z = e / (d.mx * d.my);
        const int q = sq(e);
        const long long a = d.off + e;
        A.Uprev[a] = su[q];
        T vm[3], vp[3];
        vm[0] = x > 0 ? su[q - 1] : INF;
        vp[0] = x + 1 < d.mx ? su[q + 1] : INF;
        vm[1] = y > 0 ? su[q - d.mx] : INF;
        vp[1] = y + 1 < d.my ? su[q + d.mx] : INF;
        vm[2] = z > 0 ? su[q - ps] : INF;
        vp[2] = z + 1 < d.mz ? su[q + ps] : INF;
        const T rv = A.rc[a];
        uint8_t w;
        const T cold = local_solve3(vm, vp, Num<T>::mul(rv > T(0) ? rv : T(0), Hs), w);
        A.cold[a] = cold;
        if (A.adaptive) {
            // Sec. 4.2 with every term lagged as in eq. firstthetaest
            double thv = (double)A.theta;
            if (k >= 1) {
                const int nt = k < 3 ? k : 3;
                const T *c1 = A.Ch[(k + 3) & 3], *c2 = A.Ch[(k + 2) & 3], *c3 = A.Ch[(k + 1) & 3];
                double dC[3] = {0.0, 0.0, 0.0};
                dC[0] = __dsub_rn((double)cold, (double)c1[a]);
                if (nt > 1) dC[1] = __dsub_rn((double)c1[a], (double)c2[a]);
                if (nt > 2) dC[2] = __dsub_rn((double)c2[a], (double)c3[a]);
                thv = theta_estimate(A, A.du[a], dC, nt, (double)A.theta);
            }
            A.Ch[k & 3][a] = cold;
            A.th[a] = (T)thv;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += blockDim.x) su[sq(e)] = A.U0[d.off + e];  // Sec. 1.1 initialisation
    __threadfence_block();
    __syncthreads();
    Alg5_3<T> pol{A.rc, A.uk, A.cold, A.mask, d.off, Hs, A.theta, A.adaptive ? A.th : nullptr};
    long long sweeps;
    bool conv;
    box3_sweeps(su, d.mx, d.my, d.mz, pol, A.max_coarse, sweeps, conv);
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        A.U[d.off + e] = su[sq(e)];
        A.W[d.off + e] = A.wk[d.off + e];  // W = w^k
    }
    if (threadIdx.x == 0) {
        atomicMax(&A.st->coarse_sweeps_max, (unsigned long long)sweeps);
        if (!conv) atomicAdd(&A.st->coarse_caps, 1ull);
        atomicAdd(&A.st->coarse_updates, (unsigned long long)sweeps * n);
    }
}

// --------------------------------------------------------------------------
// Steps 2 + 3: one CTA per subdomain, the subdomain box in shared memory.
// --------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ bool tile3_inflow(const DD3Args<T> &A, const int *l, const int *Xg, long long &ca) {
    bool face = false;
    for (int a = 0; a < 3; ++a) face = face || l[a] == 0 || l[a] == A.G.S[a];
    if (!face) return false;
    ca = coarse_addr3(A, Xg[0], Xg[1], Xg[2]);
    const uint8_t w = A.W[ca];
    bool in = false;
    for (int a = 0; a < 3; ++a) {
        const int wc = wind_comp(w, a);
        in = in || (l[a] == 0 && wc > 0) || (l[a] == A.G.S[a] && wc < 0);
    }
    return in;
}

// Face slots of a subdomain box: the six face planes in the order x = 0,
// x = S, y = 0, y = S, z = 0, z = S; a node on several faces takes the slot
// of the first.  Returns -1 off the faces.
__host__ __device__ inline int box3_face_slots(const int *S) {
    const int m0 = S[0] + 1, m1 = S[1] + 1, m2 = S[2] + 1;
    return 2 * (m1 * m2 + m0 * m2 + m0 * m1);
}
__device__ inline int box3_face_slot(const int *S, const int *l) {
    const int m0 = S[0] + 1, m1 = S[1] + 1, m2 = S[2] + 1;
    if (l[0] == 0) return l[1] + m1 * l[2];
    if (l[0] == S[0]) return m1 * m2 + l[1] + m1 * l[2];
    int off = 2 * m1 * m2;
    if (l[1] == 0) return off + l[0] + m0 * l[2];
    if (l[1] == S[1]) return off + m0 * m2 + l[0] + m0 * l[2];
    off += 2 * m0 * m2;
    if (l[2] == 0) return off + l[0] + m0 * l[1];
    if (l[2] == S[2]) return off + m0 * m1 + l[0] + m0 * l[1];
    return -1;
}

template <class T>
__device__ __forceinline__ bool same_bits3(T a, T b);
template <>
__device__ __forceinline__ bool same_bits3<float>(float a, float b) { return __float_as_uint(a) == __float_as_uint(b); }
template <>
__device__ __forceinline__ bool same_bits3<double>(double a, double b) {
    return __double_as_longlong(a) == __double_as_longlong(b);
}

template <class T>
__global__ void __launch_bounds__(BOX3_THREADS, 1) k3_fine(DD3Args<T> A) {
    if (*A.done) return;
    extern __shared__ __align__(16) char smem[];
    const DD3Geom &G = A.G;
    const int tile = blockIdx.x;
    const int t0 = tile % G.T[0], t1 = (tile / G.T[0]) % G.T[1], t2 = tile / (G.T[0] * G.T[1]);
    const int mx = G.S[0] + 1, my = G.S[1] + 1, mz = G.S[2] + 1;
    const int n = mx * my * mz;
    const T INF = Num<T>::inf();
    const int ps = box3_ps(mx, my);
    T *su = reinterpret_cast<T *>(smem);
    uint8_t *fx = reinterpret_cast<uint8_t *>(su + (size_t)mz * ps);
    const int b0 = t0 * G.S[0], b1 = t1 * G.S[1], b2 = t2 * G.S[2];
    // Step 2: boundary data; inflow nodes start at U (and are swept like the
    // rest), interior and outflow nodes at +inf; Gamma is fixed at g.  The
    // face nodes' data are compared with those of the subdomain's previous
    // solve in this call: if none changed, that solve's results (fine values,
    // copies) are still in place and equal bit for bit to what this one would
    // write (r, Gamma and g do not change within a call), so it is skipped.
    const int nslot = box3_face_slots(G.S);
    T *sgu = A.sig_u + (size_t)tile * nslot;
    uint8_t *sgw = A.sig_w + (size_t)tile * nslot;
    bool diff = false;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int l[3] = {e % mx, (e / mx) % my, e / (mx * my)};
        const int Xg[3] = {b0 + l[0], b1 + l[1], b2 + l[2]};
        const size_t f = fidx(A, Xg[0], Xg[1], Xg[2]);
        long long ca;
        T v = INF;
        uint8_t fixed = 0;
        if (A.gamma[f]) {
            v = A.g[f];
            fixed = 1;
        } else if (tile3_inflow(A, l, Xg, ca)) {
            v = A.U[ca];
            fixed = 2;
        }
        const int q = l[2] * ps + l[1] * mx + l[0];
        su[q] = v;
        fx[q] = fixed;
        const int fs = box3_face_slot(G.S, l);
        if (fs >= 0) {
            const T sv = fixed ? v : INF;
            const uint8_t swv = fixed == 2 ? A.W[ca] : (uint8_t)0;
            if (!same_bits3(sv, sgu[fs]) || swv != sgw[fs]) {
                diff = true;
                sgu[fs] = sv;
                sgw[fs] = swv;
            }
        }
    }
    const bool solved = A.sig_ok[tile] != 0;
    if (!__syncthreads_or(diff) && solved) {
        if (threadIdx.x == 0) atomicAdd(&A.st->fine_skips, 1ull);
        return;
    }
    if (threadIdx.x == 0) A.sig_ok[tile] = 1;
    __syncthreads();
    Fsm3<T> pol{fx, A.r, (long long)fidx(A, b0, b1, b2), 1, A.sy, A.sz, T(G.h)};
    long long sweeps;
    bool conv;
    box3_sweeps(su, mx, my, mz, pol, A.max_fsm, sweeps, conv);
    if (threadIdx.x == 0) {
        atomicMax(&A.st->fsm_sweeps_max, (unsigned long long)sweeps);
        if (!conv) atomicAdd(&A.st->fsm_caps, 1ull);
        atomicAdd(&A.st->fine_updates, (unsigned long long)sweeps * n);
    }
    // outputs: copies (u, w) at coarse-set nodes, fine values elsewhere
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int l[3] = {e % mx, (e / mx) % my, e / (mx * my)};
        const int Xg[3] = {b0 + l[0], b1 + l[1], b2 + l[2]};
        const size_t f = fidx(A, Xg[0], Xg[1], Xg[2]);
        const int q = l[2] * ps + l[1] * mx + l[0];
        const T uv = su[q];
        if (!coarse_axes3(Xg[0], Xg[1], Xg[2], G.c)) {
            A.u_out[f] = uv;
            continue;
        }
        const long long ca = coarse_addr3(A, Xg[0], Xg[1], Xg[2]);
        uint8_t w = WIND_ZERO;
        if (fx[q] == 2 && uv == A.U[ca]) {
            w = A.W[ca] | WIND_ECHO;  // inflow value kept: the coarse wind
        } else if (fx[q] != 1 && uv < INF) {
            T vm[3], vp[3];
            vm[0] = l[0] > 0 ? su[q - 1] : INF;
            vp[0] = l[0] + 1 < mx ? su[q + 1] : INF;
            vm[1] = l[1] > 0 ? su[q - mx] : INF;
            vp[1] = l[1] + 1 < my ? su[q + mx] : INF;
            vm[2] = l[2] > 0 ? su[q - ps] : INF;
            vp[2] = l[2] + 1 < mz ? su[q + ps] : INF;
            (void)local_solve3(vm, vp, Num<T>::mul(A.r[f], T(G.h)), w);
        }
        int slot = 0;
        for (int a = 0; a < 3; ++a)
            if (Xg[a] % G.S[a] == 0 && Xg[a] > 0 && Xg[a] < G.n[a] - 1 && l[a] == 0) slot |= 1 << a;
        A.cu[(size_t)slot * G.nc + ca] = uv;
        A.cw[(size_t)slot * G.nc + ca] = w;
    }
}

// --------------------------------------------------------------------------
// Alg. 4 and the inputs of Alg. 5
// --------------------------------------------------------------------------
template <class T>
__global__ void k3_alg4(DD3Args<T> A) {
    if (*A.done) return;
    const DD3Geom &G = A.G;
    const Grid3 d = A.grids[blockIdx.y];
    const long long n = (long long)d.mx * d.my * d.mz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int Xg[3] = {d.ox + G.c * (int)(e % d.mx), d.oy + G.c * (int)((e / d.mx) % d.my),
                           d.oz + G.c * (int)(e / ((long long)d.mx * d.my))};
        const long long a = d.off + e;
        int B = 0;
        for (int ax = 0; ax < 3; ++ax)
            if (Xg[ax] % G.S[ax] == 0 && Xg[ax] > 0 && Xg[ax] < G.n[ax] - 1) B |= 1 << ax;
        const uint8_t Wk = A.W[a];
        int best = 0;
        if (B) {
            int sel = 0;
            bool ok = true;
            for (int ax = 0; ax < 3 && ok; ++ax) {
                if (!(B & (1 << ax))) continue;
                bool allneg = wind_comp(Wk, ax) <= 0, allpos = wind_comp(Wk, ax) >= 0;
                for (int s = 0; s < 8; ++s) {
                    if (s & ~B) continue;
                    const int wv = wind_comp(A.cw[(size_t)s * G.nc + a], ax);
                    if (wv > 0) allneg = false;
                    if (wv < 0) allpos = false;
                }
                // Alg. 4: wind toward -axis -> plus-side copy (first branch)
                if (allneg) sel |= 1 << ax;
                else if (!allpos) ok = false;
            }
            if (ok) {
                best = sel;
            } else {
                // minimum of the fine solutions: copies that echo their Step 2
                // value are candidates only if every copy does; ties keep the
                // lowest subdomain index (slot order)
                bool computed = false;
                for (int s = 0; s < 8; ++s)
                    if (!(s & ~B) && !(A.cw[(size_t)s * G.nc + a] & WIND_ECHO)) computed = true;
                best = -1;
                T bv = T(0);
                for (int s = 0; s < 8; ++s) {
                    if (s & ~B) continue;
                    if (computed && (A.cw[(size_t)s * G.nc + a] & WIND_ECHO)) continue;
                    const T v = A.cu[(size_t)s * G.nc + a];
                    if (best < 0 || v < bv) {
                        bv = v;
                        best = s;
                    }
                }
            }
        }
        const T ukv = A.cu[(size_t)best * G.nc + a];
        const uint8_t wkv = A.cw[(size_t)best * G.nc + a] & (uint8_t)~WIND_ECHO;
        if (A.adaptive) A.du[a] = __dsub_rn((double)ukv, (double)A.uk[a]);  // u^k - u^{k-1}
        A.uk[a] = ukv;
        A.wk[a] = wkv;
        const size_t f = fidx(A, Xg[0], Xg[1], Xg[2]);
        A.u_out[f] = ukv;
        if (A.step4_identity) {
            // Step 4 with weight 0: U^{k+1} = u^k before the causal sweep, W = w^k
            A.Uprev[a] = A.U[a];
            A.U[a] = ukv;
            A.W[a] = wkv;
            continue;
        }
        uint8_t m = A.gamma[f] ? 1 : 0;
        for (int ax = 0; ax < 3; ++ax) {
            const bool on = Xg[ax] % G.c == 0;
            const int wf = wind_comp(wkv, ax), wc = wind_comp(Wk, ax);
            if (!on || (wf <= 0 && wc <= 0)) m |= 2 << (2 * ax);
            if (!on || (wf >= 0 && wc >= 0)) m |= 4 << (2 * ax);
        }
        A.mask[a] = m;
    }
}

template <class T>
__global__ void k3_check(DD3Args<T> A, int k) {
    if (*A.done) return;
    const double delta = A.deltas[k];
    const bool failed = A.st->err != DEV_OK;  // an expired wait: later stages would only repeat it
    const bool conv = k >= 1 && delta < (double)A.tol && !failed;
    if (k == A.max_iter || conv || failed) {
        *A.done = 1;
        A.st->iters = k;
        A.st->converged = conv ? 1 : 0;
    }
}

template <class T>
__global__ void k3_delta(DD3Args<T> A, int k) {
    if (*A.done) return;
    double m = 0.0;
    for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < A.G.nc;
         a += (long long)gridDim.x * blockDim.x) {
        const T u1 = A.U[a], u0 = A.Uprev[a];
        if (u1 == u0) continue;
        const double dv = fabs((double)u1 - (double)u0);
        if (dv > m) m = dv;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(FULL, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0)
        atomicMax(reinterpret_cast<unsigned long long *>(&A.deltas[k + 1]), (unsigned long long)__double_as_longlong(m));
}

// --------------------------------------------------------------------------
// Causal sweep (Alg. 2): every line along axis e whose nodes lie on a coarse
// plane of another axis; least fixed point by segmented max-scans, rounds
// until nothing changes.
// --------------------------------------------------------------------------
template <class T>
__device__ bool causal3_line(const DD3Args<T> &A, int e, int c1, int c2, int rev) {
    const DD3Geom &G = A.G;
    const T INF = Num<T>::inf();
    const int lane = threadIdx.x & 31;
    const int len = G.n[e];
    const int a1 = (e + 1) % 3, a2 = (e + 2) % 3;
    bool changed = false;
    T carry = INF, carry_orig = INF;
    for (int ch = 0; ch < (len + 31) / 32; ++ch) {
        const int pos = ch * 32 + lane;
        const bool valid = pos < len;
        const int p = rev ? len - 1 - pos : pos;
        int Xg[3];
        Xg[e] = p;
        Xg[a1] = c1;
        Xg[a2] = c2;
        long long a = 0;
        T u = INF;
        int wc = 0;
        if (valid) {
            a = coarse_addr3(A, Xg[0], Xg[1], Xg[2]);
            u = __ldcg(A.U + a);
            wc = wind_comp(__ldcg(A.W + a), e);
        }
        T pred_orig = __shfl_up_sync(FULL, u, 1);
        if (lane == 0) pred_orig = carry_orig;
        bool ff = valid && pos > 0 && (rev ? wc < 0 : wc > 0) && (pred_orig < INF);
        T v = u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T vo = __shfl_up_sync(FULL, v, o);
            const bool fo = __shfl_up_sync(FULL, ff ? 1 : 0, o) != 0;
            if (lane >= o && ff) {
                v = fmax(v, vo);
                ff = fo;
            }
        }
        if (ff) v = fmax(v, carry);
        if (valid && v > u) {
            A.U[a] = v;
            changed = true;
        }
        carry = __shfl_sync(FULL, v, 31);
        carry_orig = __shfl_sync(FULL, u, 31);
    }
    return __any_sync(FULL, changed);  // warp-uniform: any lane raised a node
}

template <class T>
__global__ void k3_causal(DD3Args<T> A, int only_if_not_done) {
    const long long wlim = spin_limit();  // limit of the grid-barrier waits
    if (only_if_not_done && *A.done) return;
    const DD3Geom &G = A.G;
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    __shared__ int blk_changed;
    if (blockIdx.x == 0 && threadIdx.x < 3) A.chg[threadIdx.x] = 0;
    if (!grid_barrier(A.bar, &A.st->err, wlim)) return;
    int rounds = 0;
    for (;;) {
        if (threadIdx.x == 0) blk_changed = 0;
        __syncthreads();
        bool ch = false;
        for (int e = 0; e < 3; ++e) {
            const int a1 = (e + 1) % 3, a2 = (e + 2) % 3;
            const int n1 = G.n[a1], n2 = G.n[a2];
            for (int L = gw; L < n1 * n2; L += warps_total) {
                const int c1 = L % n1, c2 = L / n1;
                if (c1 % G.c != 0 && c2 % G.c != 0) continue;  // not on the coarse set
                ch |= causal3_line(A, e, c1, c2, 0);
                ch |= causal3_line(A, e, c1, c2, 1);
            }
            if (!grid_barrier(A.bar, &A.st->err, wlim)) return;
        }
        if (lane == 0 && ch) atomicOr(&blk_changed, 1);
        __syncthreads();
        if (threadIdx.x == 0 && blk_changed) atomicOr(&A.chg[rounds % 3], 1);
        ++rounds;
        if (!grid_barrier(A.bar, &A.st->err, wlim)) return;
        const int any = *(volatile int *)&A.chg[(rounds - 1) % 3];
        if (blockIdx.x == 0 && threadIdx.x == 0) A.chg[(rounds + 1) % 3] = 0;
        if (!any || rounds > 10000) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(&A.st->causal_rounds_max, rounds);
}

template <class T>
__global__ void k3_finalize(DD3Args<T> A, eik_dd_stats *out, long long launches) {
    if (threadIdx.x != 0 || !out) return;
    out->iters = A.st->iters;
    out->converged = A.st->converged;
    out->error = A.st->err;
    out->causal_rounds_max = A.st->causal_rounds_max;
    out->fsm_sweeps_max = (int64_t)A.st->fsm_sweeps_max;
    out->coarse_sweeps_max = (int64_t)A.st->coarse_sweeps_max;
    out->fsm_cap_hits = (int64_t)A.st->fsm_caps;
    out->coarse_cap_hits = (int64_t)A.st->coarse_caps;
    const int k = A.st->iters;
    out->last_delta = k >= 1 ? A.deltas[k] : INFINITY;
    out->fine_updates = (int64_t)A.st->fine_updates;
    out->coarse_updates = (int64_t)A.st->coarse_updates;
    out->launches = launches;
    out->fine_solves_skipped = (int64_t)A.st->fine_skips;
}

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------
struct DD3Plan {
    DD3Geom G;
    std::vector<Grid3> grids;
    std::vector<int> offmap;
    size_t fine_smem, grid_smem, bytes;
    int fine_threads, grid_threads;
    bool adaptive;
};

static bool dd3_plan(const eik_grid *grid, const eik_dd_params *p, DD3Plan &P) {
    const int c = p->coarse_ratio;
    DD3Geom &G = P.G;
    for (int a = 0; a < 3; ++a) {
        G.n[a] = (int)grid->n[a];
        G.T[a] = p->tiles[a];
        G.S[a] = (G.n[a] - 1) / G.T[a];
    }
    G.c = c;
    G.h = grid->h;
    G.H = (double)c * grid->h;
    P.adaptive = p->theta_adaptive != 0;
    P.grids.clear();
    P.offmap.assign((size_t)c * c * c, -1);
    long long off = 0;
    for (int oz = 0; oz < c; ++oz)
        for (int oy = 0; oy < c; ++oy)
            for (int ox = 0; ox < c; ++ox) {
                if (ox && oy && oz) continue;
                Grid3 d;
                d.ox = ox;
                d.oy = oy;
                d.oz = oz;
                d.mx = (G.n[0] - 1 - ox) / c + 1;
                d.my = (G.n[1] - 1 - oy) / c + 1;
                d.mz = (G.n[2] - 1 - oz) / c + 1;
                d.off = off;
                off += (long long)d.mx * d.my * d.mz;
                P.offmap[((size_t)oz * c + oy) * c + ox] = (int)P.grids.size();
                P.grids.push_back(d);
            }
    G.ng = (int)P.grids.size();
    G.nc = off;
    const size_t tsz = grid->dtype == EIK_F64 ? 8 : 4;
    const size_t tile_n = (size_t)(G.S[2] + 1) * box3_ps(G.S[0] + 1, G.S[1] + 1);
    size_t gmax = 0;
    for (auto &d : P.grids) gmax = std::max(gmax, (size_t)d.mz * box3_ps(d.mx, d.my));
    P.fine_smem = tile_n * (tsz + 1) + 16;
    P.grid_smem = gmax * (tsz + 1) + 16;
    P.fine_threads = BOX3_THREADS;
    P.grid_threads = BOX3_THREADS;
    return true;
}

template <class T>
static size_t dd3_layout(const DD3Plan &P, DD3Args<T> *A, void *ws, int max_iter) {
    const DD3Geom &G = P.G;
    Carver cv(ws);
    T *U = cv.take<T>(G.nc), *Uprev = cv.take<T>(G.nc), *U0 = cv.take<T>(G.nc), *rc = cv.take<T>(G.nc);
    T *uk = cv.take<T>(G.nc), *cold = cv.take<T>(G.nc);
    uint8_t *W = cv.take<uint8_t>(G.nc), *wk = cv.take<uint8_t>(G.nc), *mask = cv.take<uint8_t>(G.nc);
    T *cu = cv.take<T>(8 * (size_t)G.nc);
    uint8_t *cw = cv.take<uint8_t>(8 * (size_t)G.nc);
    Grid3 *grids = cv.take<Grid3>(P.grids.size());
    int *offmap = cv.take<int>(P.offmap.size());
    int *done = cv.take<int>(4);
    double *deltas = cv.take<double>((size_t)max_iter + 2);
    int *chg = cv.take<int>(4);
    unsigned *bar = cv.take<unsigned>(4);
    DevStats3 *st = cv.take<DevStats3>(1);
    const size_t ntl = (size_t)G.T[0] * G.T[1] * G.T[2], nsl = (size_t)box3_face_slots(G.S);
    T *sig_u = cv.take<T>(ntl * nsl);
    uint8_t *sig_w = cv.take<uint8_t>(ntl * nsl);
    int *sig_ok = cv.take<int>(ntl);
    T *Ch[4] = {nullptr, nullptr, nullptr, nullptr}, *th = nullptr;
    double *du = nullptr;
    if (P.adaptive) {
        for (int s = 0; s < 4; ++s) Ch[s] = cv.take<T>(G.nc);
        th = cv.take<T>(G.nc);
        du = cv.take<double>(G.nc);
    }
    if (A) {
        for (int s = 0; s < 4; ++s) A->Ch[s] = Ch[s];
        A->th = th;
        A->du = du;
        A->U = U; A->Uprev = Uprev; A->U0 = U0; A->rc = rc; A->uk = uk; A->cold = cold;
        A->W = W; A->wk = wk; A->mask = mask; A->cu = cu; A->cw = cw;
        A->grids = grids; A->offmap = offmap; A->done = done; A->deltas = deltas; A->chg = chg; A->bar = bar;
        A->st = st;
        A->sig_u = sig_u;
        A->sig_w = sig_w;
        A->sig_ok = sig_ok;
    }
    return cv.used + 256;
}

// Shifted-grid tables, built on the device in the enumeration order of the
// host plan (z offset outermost, x innermost; offsets with no zero skipped).
__global__ void k3_tables(Grid3 *grids, int *offmap, int c, int n0, int n1, int n2) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long off = 0;
    int gi = 0;
    for (int oz = 0; oz < c; ++oz)
        for (int oy = 0; oy < c; ++oy)
            for (int ox = 0; ox < c; ++ox) {
                const int m = (oz * c + oy) * c + ox;
                if (ox && oy && oz) {
                    offmap[m] = -1;
                    continue;
                }
                Grid3 d;
                d.ox = ox;
                d.oy = oy;
                d.oz = oz;
                d.mx = (n0 - 1 - ox) / c + 1;
                d.my = (n1 - 1 - oy) / c + 1;
                d.mz = (n2 - 1 - oz) / c + 1;
                d.off = off;
                off += (long long)d.mx * d.my * d.mz;
                offmap[m] = gi;
                grids[gi++] = d;
            }
}

size_t dd3_workspace_size(const eik_grid *grid, const eik_dd_params *p) {
    DD3Plan P;
    dd3_plan(grid, p, P);
    return grid->dtype == EIK_F64 ? dd3_layout<double>(P, nullptr, nullptr, p->max_iter)
                                  : dd3_layout<float>(P, nullptr, nullptr, p->max_iter);
}

bool dd3_validate(const eik_grid *grid, const eik_dd_params *p) {
    for (int a = 0; a < 3; ++a) {
        if (p->tiles[a] < 1 || (grid->n[a] - 1) % p->tiles[a] != 0) {
            set_error("tiles[%d] = %d does not divide n[%d]-1", a, p->tiles[a], a);
            return false;
        }
        if (((grid->n[a] - 1) / p->tiles[a]) % p->coarse_ratio != 0) {
            set_error("coarse_ratio %d does not divide the subdomain width along axis %d", p->coarse_ratio, a);
            return false;
        }
    }
    if (p->coarse_ratio < 1 || p->coarse_ratio > 64) {
        set_error("coarse_ratio must be in [1, 64] in 3-D");
        return false;
    }
    return true;
}

template <class T>
static int dd3_run_t(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g,
                     const eik_dd_params *p, void *u_out, void *ws, eik_dd_stats *stats, cudaStream_t s) {
    DD3Plan P;
    dd3_plan(grid, p, P);
    DD3Args<T> A;
    memset(&A, 0, sizeof(A));
    A.G = P.G;
    A.r = static_cast<const T *>(r);
    A.gamma = gamma;
    A.g = static_cast<const T *>(g);
    A.u_out = static_cast<T *>(u_out);
    A.sy = grid->stride[1];
    A.sz = grid->stride[2];
    dd3_layout<T>(P, &A, ws, p->max_iter);
    A.theta = (T)p->theta;
    A.tol = (T)p->tol;
    A.max_iter = p->max_iter;
    A.max_fsm = p->max_fsm_sweeps;
    A.max_coarse = p->max_coarse_sweeps;
    A.adaptive = P.adaptive ? 1 : 0;
    A.step4_identity = (!P.adaptive && p->theta == 0.0) ? 1 : 0;
    for (int s2 = 0; s2 < 3; ++s2) A.om[s2] = p->omega[s2];
    A.sg = p->sig_gamma;
    A.sd = p->sig_delta;
    A.sx0 = p->sig_x0;
    A.cap = p->theta_cap;
    const DD3Geom &G = P.G;
    int rc, dev, nsm = 0, optin = 0;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if ((int)P.fine_smem > optin || (int)P.grid_smem > optin) {
        set_error("3-D subdomain or coarse grid box needs %zu / %zu bytes of shared memory (limit %d)", P.fine_smem,
                  P.grid_smem, optin);
        return EIK_EUNSUPPORTED;
    }
    if ((rc = cuda_check(set_dyn_smem(k3_fine<T>, (int)P.fine_smem), "attr")))
        return rc;
    if ((rc = cuda_check(set_dyn_smem(k3_step1<T>, (int)P.grid_smem), "attr")))
        return rc;
    if ((rc = cuda_check(set_dyn_smem(k3_step4<T>, (int)P.grid_smem), "attr")))
        return rc;
    const int causal_threads = 256;
    int per_sm = 0;
    if ((rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k3_causal<T>, causal_threads, 0), "occ")))
        return rc;
    const int causal_blocks = std::max(1, std::min(per_sm * nsm, 2 * nsm));
    const int ntiles = G.T[0] * G.T[1] * G.T[2];
    dim3 cgrid(8, G.ng);
    const int ew = 256;
    const int eb = (int)std::min<long long>((G.nc + ew - 1) / ew, (long long)nsm * 8);
    long long nl = 0;
    EIK_LAUNCH("dd3_init", s, k3_init<T><<<1, 256, 0, s>>>(A)); ++nl;
    EIK_LAUNCH("dd3_tables", s, k3_tables<<<1, 32, 0, s>>>(A.grids, A.offmap, G.c, G.n[0], G.n[1], G.n[2])); ++nl;
    EIK_LAUNCH("dd3_pack_coarse", s, k3_pack_coarse<T><<<cgrid, ew, 0, s>>>(A)); ++nl;
    EIK_LAUNCH("dd3_step1_coarse_fsm", s, k3_step1<T><<<G.ng, P.grid_threads, P.grid_smem, s>>>(A)); ++nl;
    auto launch_causal = [&](int only) -> int {
        void *args[] = {&A, &only};
        int tok = prof_begin("dd3_causal_sweep", s);
        int r2 = cuda_check(cudaLaunchCooperativeKernel((void *)k3_causal<T>, causal_blocks, causal_threads, args, 0, s),
                            "causal launch");
        prof_end(tok, s);
        ++nl;
        return r2;
    };
    if ((rc = launch_causal(0))) return rc;
    for (int k = 0; k <= p->max_iter; ++k) {
        EIK_LAUNCH("dd3_fine_subdomains", s, k3_fine<T><<<ntiles, P.fine_threads, P.fine_smem, s>>>(A)); ++nl;
        EIK_LAUNCH("dd3_alg4_restrict", s, k3_alg4<T><<<cgrid, ew, 0, s>>>(A)); ++nl;
        EIK_LAUNCH("dd3_check", s, k3_check<T><<<1, 1, 0, s>>>(A, k)); ++nl;
        if (k == p->max_iter) break;
        if (!A.step4_identity) {
            EIK_LAUNCH("dd3_step4_weighted", s, k3_step4<T><<<G.ng, P.grid_threads, P.grid_smem, s>>>(A, k));
            ++nl;
        }
        if ((rc = launch_causal(1))) return rc;
        EIK_LAUNCH("dd3_delta", s, k3_delta<T><<<eb, ew, 0, s>>>(A, k)); ++nl;
    }
    ++nl;
    EIK_LAUNCH("dd3_finalize", s, k3_finalize<T><<<1, 32, 0, s>>>(A, stats, nl));
    return cuda_check(cudaGetLastError(), "dd3 launch");
}

int dd3_run(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g, const eik_dd_params *p,
            void *u_out, void *ws, eik_dd_stats *stats, cudaStream_t s) {
    if (grid->dtype == EIK_F64) return dd3_run_t<double>(grid, r, gamma, g, p, u_out, ws, stats, s);
    return dd3_run_t<float>(grid, r, gamma, g, p, u_out, ws, stats, s);
}

}  // namespace eik

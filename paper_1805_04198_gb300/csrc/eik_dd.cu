// eik_dd.cu -- two-scale domain decomposition (Sec. 3.2, Steps 1-4, Alg. 1-5)
// on one GPU, 2-D.
//
// Per parareal iteration k the device runs, on one stream:
//   k_fine   one CTA per subdomain: Step 2 boundary data from (U, W), Step 3
//            FSM sweeps by the warp-systolic engine, then the Alg. 3 winds of
//            the converged state at the subdomain's coarse-set nodes (written
//            as per-subdomain copies) and the fine values of interior nodes;
//   k_alg4   one thread per coarse-set node: Alg. 4 choice among the copies
//            -> u^k, w^k; the skewed per-direction inputs of Alg. 5;
//   k_check  stop test (k == max_iter, or k >= 1 and max|U^k - U^{k-1}| < tol);
//   k_step4  one CTA per shifted coarse grid: C_H(nbrs U^k), reset, Alg. 5
//            sweeps by the same engine, W = w^k;
//   k_causal cooperative: Alg. 2 along every coarse line to its least fixed
//            point (segmented max-scans, rounds until nothing changes);
//   k_delta  max|U^{k+1} - U^k| over the coarse set.
// Every kernel returns at once when the device flag `done` is set, so the
// host enqueues max_iter + 1 iterations without reading anything back.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "dd_geom.cuh"
#include "engine.cuh"
#include "host_util.h"
#include "prof.h"

namespace eik {

struct DevStats {
    unsigned long long fsm_sweeps_max, coarse_sweeps_max, fsm_caps, coarse_caps;
    unsigned long long fine_updates, coarse_updates;
    int causal_rounds_max;
    int err;
    int iters;
    int converged;
    unsigned long long delta_bits[1];  // placeholder (per-iteration deltas live in `deltas`)
};

template <class T>
struct DDArgs {
    DDGeom G;
    // caller arrays
    const T *r;
    const uint8_t *gamma;
    const T *g;
    T *u_out;
    long long sy;  // row stride of caller arrays (elements)
    // tiles
    T *tile_state;
    T *tile_rsk;
    // coarse, grid layout
    T *U, *Uprev, *U0, *rc, *uk;
    uint8_t *W, *wk;
    T *cu;        // [4][coarse_elems]
    uint8_t *cw;  // [4][coarse_elems]
    // coarse, skewed per direction
    T *rc_sk, *uk_sk, *cold_sk;
    uint8_t *mask_sk;
    // control
    int *done;
    double *deltas;  // [max_iter + 2] as doubles (max via integer atomics on bits)
    int *chg;        // [4] causal round flags + barrier
    unsigned *bar;   // [2] grid barrier count / generation
    DevStats *st;
    T theta, tol;
    int max_iter;
    long long max_fsm, max_coarse;
};

template <class T>
__device__ __forceinline__ T fine_at(const T *a, long long sy, int X, int Y) {
    return a[(size_t)Y * sy + X];
}

// --------------------------------------------------------------------------
// Engine policies
// --------------------------------------------------------------------------

// FSM update u = min(u, u~) (Sec. 1.1, eq. FSMupdate).  Statics: r, stored
// as a non-positive value at fixed nodes (Gamma, Dirichlet boundary data).
template <class T>
struct FsmPolicy {
    T h;
    __device__ __forceinline__ T update(T self, T vmx, T vpx, T vmy, T vpy, const T *sv, uint8_t,
                                        bool &changed) const {
        const T r = sv[0];
        const T ut = local_solve2_value(vmx, vpx, vmy, vpy, Num<T>::mul(r, h));
        const bool take = (r > T(0)) && (ut < self);
        changed = take;
        return take ? ut : self;
    }
};

// Alg. 5 weighted correction.  Statics: r, u^k, C_H(nbrs U^k); byte mask:
// bit 0 Gamma, bits 1/2 "x component may be <= 0 / >= 0", bits 3/4 the same
// for y (from w^k and W^k on the axes of the node's coarse lines; both set on
// other axes).
template <class T>
struct Alg5Policy {
    T H, theta;
    __device__ __forceinline__ T update(T self, T vmx, T vpx, T vmy, T vpy, const T *sv, uint8_t mask,
                                        bool &changed) const {
        using N = Num<T>;
        uint8_t w;
        const T Ut = local_solve2(vmx, vpx, vmy, vpy, N::mul(sv[0], H), w);
        const T uk = sv[1], cold = sv[2];
        const int wx = wind_comp(w, 0), wy = wind_comp(w, 1);
        bool pass = (Ut < N::inf()) && (cold < N::inf());
        pass = pass && ((wx <= 0 && (mask & 2)) || (wx >= 0 && (mask & 4)));
        pass = pass && ((wy <= 0 && (mask & 8)) || (wy >= 0 && (mask & 16)));
        const T nu0 = pass ? N::add(uk, N::mul(theta, N::sub(Ut, cold))) : uk;
        const T nu = (mask & 1) ? self : nu0;
        changed = !(nu == self);
        return nu;
    }
};

// --------------------------------------------------------------------------
// Set-up kernels (once per solve)
// --------------------------------------------------------------------------
template <class T>
__global__ void k_pack_tiles(DDArgs<T> A) {
    const DDGeom &G = A.G;
    const size_t per_tile = (size_t)G.tnx * G.tny;
    const size_t total = per_tile * G.tx * G.ty;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        int tile = (int)(t / per_tile);
        int rem = (int)(t % per_tile);
        int xl = rem % G.tnx, yl = rem / G.tnx;
        int tx = tile % G.tx, ty = tile / G.tx;
        int X = tx * G.sx + xl, Y = ty * G.sy + yl;
        T v = A.gamma[(size_t)Y * A.sy + X] ? T(-1) : fine_at(A.r, A.sy, X, Y);
        T *base = A.tile_rsk + (size_t)tile * G.tile_sk_elems;
        for (int d = 0; d < 4; ++d) base[skew_index(d, xl, yl, G.tnb, G.tny, G.tnstepp)] = v;
    }
}

template <class T>
__global__ void k_pack_coarse(DDArgs<T> A) {
    const DDGeom &G = A.G;
    for (size_t a = blockIdx.x * (size_t)blockDim.x + threadIdx.x; a < G.coarse_elems;
         a += (size_t)gridDim.x * blockDim.x) {
        int g, i, j;
        if (!coarse_decode(G, a, g, i, j)) continue;
        GridDesc d = grid_desc(G, g);
        int X = d.ox + G.c * i, Y = d.oy + G.c * j;
        bool gam = A.gamma[(size_t)Y * A.sy + X] != 0;
        T rv = fine_at(A.r, A.sy, X, Y);
        A.rc[a] = gam ? T(-1) : rv;
        A.U0[a] = gam ? fine_at(A.g, A.sy, X, Y) : Num<T>::inf();
        A.W[a] = WIND_ZERO;
        T *sk = A.rc_sk + d.skoff;
        for (int dd = 0; dd < 4; ++dd) sk[skew_index(dd, i, j, d.nb, d.my, d.nstepp)] = gam ? T(-1) : rv;
    }
}

// --------------------------------------------------------------------------
// Coarse-grid kernels (one CTA per shifted grid)
// --------------------------------------------------------------------------
template <class T>
__device__ void grid_winds(const DDArgs<T> &A, const GridDesc &d, T Hs) {
    // Alg. 1 wind of the converged coarse state (Gamma / unreached: zero wind)
    const T INF = Num<T>::inf();
    T *U = A.U + d.off;
    const size_t n = (size_t)d.nb * d.my * 32;
    for (size_t e = threadIdx.x; e < n; e += blockDim.x) {
        int b = (int)(e / ((size_t)d.my * 32));
        int rem = (int)(e % ((size_t)d.my * 32));
        int j = rem / 32, i = 32 * b + rem % 32;
        if (i >= d.mx) continue;
        const size_t a = d.off + e;
        uint8_t w = WIND_ZERO;
        const T rv = A.rc[a];
        const T uv = __ldcg(U + e);
        if (rv > T(0) && uv < INF) {
            T vmx = i > 0 ? __ldcg(U + box_index(i - 1, j, d.my)) : INF;
            T vpx = i + 1 < d.mx ? __ldcg(U + box_index(i + 1, j, d.my)) : INF;
            T vmy = j > 0 ? __ldcg(U + box_index(i, j - 1, d.my)) : INF;
            T vpy = j + 1 < d.my ? __ldcg(U + box_index(i, j + 1, d.my)) : INF;
            (void)local_solve2(vmx, vpx, vmy, vpy, Num<T>::mul(rv, Hs), w);
        }
        A.W[a] = w;
    }
}

// Step 1: FSM with Alg. 1 on every shifted grid; Gamma nodes fixed at g.
template <class T>
__device__ __forceinline__ void k_step1_body(DDArgs<T> &A, char *smem) {
    const DDGeom &G = A.G;
    const GridDesc d = grid_desc(G, blockIdx.x);
    const size_t n = (size_t)d.nb * d.my * 32;
    for (size_t e = threadIdx.x; e < n; e += blockDim.x) A.U[d.off + e] = A.U0[d.off + e];
    __syncthreads();
    Box<T, 1> bx;
    bx.u = A.U + d.off;
    bx.st[0] = A.rc_sk + d.skoff;
    bx.sb = nullptr;
    bx.nx = d.mx;
    bx.ny = d.my;
    bx.nb = d.nb;
    bx.nstepp = d.nstepp;
    FsmPolicy<T> pol{T(G.H)};
    long long sweeps;
    bool conv;
    engine_run<T, 1, false>(bx, pol, A.max_coarse, smem, sweeps, conv, &A.st->err);
    if (threadIdx.x == 0) {
        atomicMax(&A.st->coarse_sweeps_max, (unsigned long long)sweeps);
        if (!conv) atomicAdd(&A.st->coarse_caps, 1ull);
        atomicAdd(&A.st->coarse_updates, (unsigned long long)sweeps * d.mx * d.my);
    }
    grid_winds(A, d, T(G.H));
}

// Step 4: Alg. 5 on every shifted grid.
template <class T>
__device__ __forceinline__ void k_step4_body(DDArgs<T> &A, char *smem) {
    if (*A.done) return;
    const DDGeom &G = A.G;
    const GridDesc d = grid_desc(G, blockIdx.x);
    const T INF = Num<T>::inf();
    const T Hs = T(G.H);
    const size_t n = (size_t)d.nb * d.my * 32;
    T *U = A.U + d.off;
    // C_H(nbrs^H(U^k)) from the previous iterate; keep U^k for the delta
    for (size_t e = threadIdx.x; e < n; e += blockDim.x) {
        int b = (int)(e / ((size_t)d.my * 32));
        int rem = (int)(e % ((size_t)d.my * 32));
        int j = rem / 32, i = 32 * b + rem % 32;
        if (i >= d.mx) continue;
        const size_t a = d.off + e;
        A.Uprev[a] = U[e];
        T vmx = i > 0 ? U[box_index(i - 1, j, d.my)] : INF;
        T vpx = i + 1 < d.mx ? U[box_index(i + 1, j, d.my)] : INF;
        T vmy = j > 0 ? U[box_index(i, j - 1, d.my)] : INF;
        T vpy = j + 1 < d.my ? U[box_index(i, j + 1, d.my)] : INF;
        const T rv = A.rc[a];
        const T cold = local_solve2_value(vmx, vpx, vmy, vpy, Num<T>::mul(rv > T(0) ? rv : T(0), Hs));
        T *sk = A.cold_sk + d.skoff;
        for (int dd = 0; dd < 4; ++dd) sk[skew_index(dd, i, j, d.nb, d.my, d.nstepp)] = cold;
    }
    __syncthreads();
    // "Initialize U as described in Sec. 1.1"
    for (size_t e = threadIdx.x; e < n; e += blockDim.x) U[e] = A.U0[d.off + e];
    __threadfence_block();
    __syncthreads();
    Box<T, 3> bx;
    bx.u = U;
    bx.st[0] = A.rc_sk + d.skoff;
    bx.st[1] = A.uk_sk + d.skoff;
    bx.st[2] = A.cold_sk + d.skoff;
    bx.sb = A.mask_sk + d.skoff;
    bx.nx = d.mx;
    bx.ny = d.my;
    bx.nb = d.nb;
    bx.nstepp = d.nstepp;
    Alg5Policy<T> pol{Hs, A.theta};
    long long sweeps;
    bool conv;
    engine_run<T, 3, true>(bx, pol, A.max_coarse, smem, sweeps, conv, &A.st->err);
    if (threadIdx.x == 0) {
        atomicMax(&A.st->coarse_sweeps_max, (unsigned long long)sweeps);
        if (!conv) atomicAdd(&A.st->coarse_caps, 1ull);
        atomicAdd(&A.st->coarse_updates, (unsigned long long)sweeps * d.mx * d.my);
    }
    // W = w^k
    for (size_t e = threadIdx.x; e < n; e += blockDim.x) A.W[d.off + e] = A.wk[d.off + e];
}

// --------------------------------------------------------------------------
// Causal sweep (Alg. 2): least fixed point along every coarse line.
// --------------------------------------------------------------------------
// One direction of one line: values v (current) with "connected to the
// predecessor in scan order" flags; inclusive segmented max-scan per 32-node
// chunk with a carry across chunks.
template <class T>
__device__ bool causal_line(const DDArgs<T> &A, bool horizontal, int line, int rev) {
    const DDGeom &G = A.G;
    const T INF = Num<T>::inf();
    const int lane = threadIdx.x & 31;
    const int len = horizontal ? G.nx : G.ny;
    const int fixedc = line * G.c;
    const int axis = horizontal ? 0 : 1;
    bool changed = false;
    T carry = INF;        // scanned value of the previous node in scan order
    T carry_orig = INF;   // its value before this pass
    const int nch = (len + 31) / 32;
    for (int ch = 0; ch < nch; ++ch) {
        const int pos = ch * 32 + lane;                // position in scan order
        const bool valid = pos < len;
        const int p = rev ? len - 1 - pos : pos;       // coordinate along the line
        const int X = horizontal ? p : fixedc, Y = horizontal ? fixedc : p;
        size_t a = 0;
        T u = INF;
        int wc = 0;
        if (valid) {
            a = coarse_addr(G, X, Y);
            u = __ldcg(A.U + a);
            wc = wind_comp(__ldcg(A.W + a), axis);
        }
        // predecessor in scan order is the upwind side when the wind points
        // away from it: forward scan raises from p-1 when w > 0, reverse scan
        // raises from p+1 when w < 0.
        T pred_orig = __shfl_up_sync(FULL, u, 1);
        if (lane == 0) pred_orig = carry_orig;
        bool f = valid && pos > 0 && (rev ? wc < 0 : wc > 0) && (pred_orig < INF);
        T v = u;
        bool ff = f;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T vo = __shfl_up_sync(FULL, v, o);
            bool fo = __shfl_up_sync(FULL, ff ? 1 : 0, o) != 0;
            if (lane >= o && ff) {
                v = fmax(v, vo);
                ff = fo;
            }
        }
        if (ff) v = fmax(v, carry);
        if (valid && v > u) {  // values only rise; NaN never counts as a change
            A.U[a] = v;
            changed = true;
        }
        carry = __shfl_sync(FULL, v, 31);
        carry_orig = __shfl_sync(FULL, u, 31);
    }
    return __any_sync(FULL, changed);  // warp-uniform: any lane raised a node
}

template <class T>
__global__ void k_causal(DDArgs<T> A, int only_if_not_done) {
    if (only_if_not_done && *A.done) return;
    const DDGeom &G = A.G;
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    __shared__ int blk_changed;
    if (blockIdx.x == 0 && threadIdx.x < 3) A.chg[threadIdx.x] = 0;
    if (!grid_barrier(A.bar, &A.st->err)) return;
    int rounds = 0;
    for (;;) {
        if (threadIdx.x == 0) blk_changed = 0;
        __syncthreads();
        bool ch = false;
        for (int l = gw; l <= G.ncy; l += warps_total) {
            ch |= causal_line(A, true, l, 0);
            ch |= causal_line(A, true, l, 1);
        }
        if (!grid_barrier(A.bar, &A.st->err)) return;
        for (int l = gw; l <= G.ncx; l += warps_total) {
            ch |= causal_line(A, false, l, 0);
            ch |= causal_line(A, false, l, 1);
        }
        if (lane == 0 && ch) atomicOr(&blk_changed, 1);
        __syncthreads();
        if (threadIdx.x == 0 && blk_changed) atomicOr(&A.chg[rounds % 3], 1);
        ++rounds;
        if (!grid_barrier(A.bar, &A.st->err)) return;
        const int any = *(volatile int *)&A.chg[(rounds - 1) % 3];
        if (blockIdx.x == 0 && threadIdx.x == 0) A.chg[(rounds + 1) % 3] = 0;
        if (!any || rounds > 10000) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(&A.st->causal_rounds_max, rounds);
}

// --------------------------------------------------------------------------
// Steps 2 + 3: one CTA per subdomain.
// --------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ bool tile_inflow(const DDArgs<T> &A, int xl, int yl, int X, int Y, size_t &ca) {
    const DDGeom &G = A.G;
    const bool onface = xl == 0 || xl == G.sx || yl == 0 || yl == G.sy;
    if (!onface) return false;
    ca = coarse_addr(G, X, Y);
    const uint8_t w = A.W[ca];
    const int wx = wind_comp(w, 0), wy = wind_comp(w, 1);
    // Step 2: inflow when W . n > 0 for an inward normal n of this subdomain
    return (xl == 0 && wx > 0) || (xl == G.sx && wx < 0) || (yl == 0 && wy > 0) || (yl == G.sy && wy < 0);
}

template <class T>
__device__ __forceinline__ void k_fine_body(DDArgs<T> &A, char *smem) {
    if (*A.done) return;
    const DDGeom &G = A.G;
    const T INF = Num<T>::inf();
    const int tile = blockIdx.x;
    const int tx = tile % G.tx, ty = tile / G.tx;
    const int NX = G.tnx, NY = G.tny;
    T *ut = A.tile_state + (size_t)tile * G.tile_elems;
    T *rsk = A.tile_rsk + (size_t)tile * G.tile_sk_elems;
    // Step 2: boundary data.  Interior and outflow nodes start at +inf.
    for (size_t e = threadIdx.x; e < G.tile_elems; e += blockDim.x) {
        int b = (int)(e / ((size_t)NY * 32));
        int rem = (int)(e % ((size_t)NY * 32));
        int yl = rem / 32, xl = 32 * b + rem % 32;
        T v = INF;
        if (xl < NX) {
            int X = tx * G.sx + xl, Y = ty * G.sy + yl;
            size_t ca;
            if (A.gamma[(size_t)Y * A.sy + X]) v = fine_at(A.g, A.sy, X, Y);
            else if (tile_inflow(A, xl, yl, X, Y, ca)) v = A.U[ca];
        }
        ut[e] = v;
    }
    // fixed-node marks of the face nodes for this iteration: Dirichlet (inflow)
    // and Gamma nodes carry a non-positive slowness in the skewed statics
    for (int f = threadIdx.x; f < 2 * NY + 2 * NX; f += blockDim.x) {
        int xl, yl;
        if (f < NY) { xl = 0; yl = f; }
        else if (f < 2 * NY) { xl = NX - 1; yl = f - NY; }
        else if (f < 2 * NY + NX) { xl = f - 2 * NY; yl = 0; }
        else { xl = f - 2 * NY - NX; yl = NY - 1; }
        int X = tx * G.sx + xl, Y = ty * G.sy + yl;
        size_t ca;
        const bool fixed = A.gamma[(size_t)Y * A.sy + X] || tile_inflow(A, xl, yl, X, Y, ca);
        const T v = fixed ? T(-1) : fine_at(A.r, A.sy, X, Y);
        for (int dd = 0; dd < 4; ++dd) rsk[skew_index(dd, xl, yl, G.tnb, NY, G.tnstepp)] = v;
    }
    __threadfence_block();
    __syncthreads();
    // Step 3: FSM sweeps in the subdomain
    Box<T, 1> bx;
    bx.u = ut;
    bx.st[0] = A.tile_rsk + (size_t)tile * G.tile_sk_elems;
    bx.sb = nullptr;
    bx.nx = NX;
    bx.ny = NY;
    bx.nb = G.tnb;
    bx.nstepp = G.tnstepp;
    FsmPolicy<T> pol{T(G.h)};
    long long sweeps;
    bool conv;
    engine_run<T, 1, false>(bx, pol, A.max_fsm, smem, sweeps, conv, &A.st->err);
    if (threadIdx.x == 0) {
        atomicMax(&A.st->fsm_sweeps_max, (unsigned long long)sweeps);
        if (!conv) atomicAdd(&A.st->fsm_caps, 1ull);
        atomicAdd(&A.st->fine_updates, (unsigned long long)sweeps * NX * NY);
    }
    // outputs: copies (u, w) at coarse-set nodes, fine values elsewhere
    for (size_t e = threadIdx.x; e < G.tile_elems; e += blockDim.x) {
        int b = (int)(e / ((size_t)NY * 32));
        int rem = (int)(e % ((size_t)NY * 32));
        int yl = rem / 32, xl = 32 * b + rem % 32;
        if (xl >= NX) continue;
        int X = tx * G.sx + xl, Y = ty * G.sy + yl;
        const T uv = __ldcg(ut + e);
        if (!in_coarse_set(G, X, Y)) {
            A.u_out[(size_t)Y * A.sy + X] = uv;
            continue;
        }
        size_t ca = coarse_addr(G, X, Y);
        uint8_t w = WIND_ZERO;
        if (A.gamma[(size_t)Y * A.sy + X]) {
            w = WIND_ZERO;
        } else {
            size_t ca2;
            if (tile_inflow(A, xl, yl, X, Y, ca2)) {
                w = A.W[ca];
            } else if (uv < INF) {
                T vmx = xl > 0 ? __ldcg(ut + box_index(xl - 1, yl, NY)) : INF;
                T vpx = xl + 1 < NX ? __ldcg(ut + box_index(xl + 1, yl, NY)) : INF;
                T vmy = yl > 0 ? __ldcg(ut + box_index(xl, yl - 1, NY)) : INF;
                T vpy = yl + 1 < NY ? __ldcg(ut + box_index(xl, yl + 1, NY)) : INF;
                T rv = fine_at(A.r, A.sy, X, Y);
                (void)local_solve2(vmx, vpx, vmy, vpy, Num<T>::mul(rv, T(G.h)), w);
            }
        }
        // copy slot: bit 0 = plus side of an x interface, bit 1 = of a y interface
        int slot = 0;
        if (X % G.sx == 0 && X > 0 && X < G.nx - 1 && xl == 0) slot |= 1;
        if (Y % G.sy == 0 && Y > 0 && Y < G.ny - 1 && yl == 0) slot |= 2;
        A.cu[(size_t)slot * G.coarse_elems + ca] = uv;
        A.cw[(size_t)slot * G.coarse_elems + ca] = w;
    }
}

// Kernel entry points.  Register caps keep two 9-warp subdomain CTAs per SM in
// FP32 and let a 9-warp coarse-grid CTA fit the register file in FP64.
#define EIK_KERNEL_PAIR(name, RF, RD)                                                  \
    __global__ void __maxnreg__(RF) name##_f32(DDArgs<float> A) {                     \
        extern __shared__ __align__(16) char smem[];                                  \
        name##_body<float>(A, smem);                                                  \
    }                                                                                 \
    __global__ void __maxnreg__(RD) name##_f64(DDArgs<double> A) {                    \
        extern __shared__ __align__(16) char smem[];                                  \
        name##_body<double>(A, smem);                                                 \
    }
EIK_KERNEL_PAIR(k_step1, 96, 224)
EIK_KERNEL_PAIR(k_step4, 160, 224)
EIK_KERNEL_PAIR(k_fine, 96, 224)

template <class T> struct DDKernels;
template <> struct DDKernels<float> {
    static constexpr void (*step1)(DDArgs<float>) = k_step1_f32;
    static constexpr void (*step4)(DDArgs<float>) = k_step4_f32;
    static constexpr void (*fine)(DDArgs<float>) = k_fine_f32;
};
template <> struct DDKernels<double> {
    static constexpr void (*step1)(DDArgs<double>) = k_step1_f64;
    static constexpr void (*step4)(DDArgs<double>) = k_step4_f64;
    static constexpr void (*fine)(DDArgs<double>) = k_fine_f64;
};

// --------------------------------------------------------------------------
// Alg. 4 + inputs of Alg. 5
// --------------------------------------------------------------------------
template <class T>
__global__ void k_alg4(DDArgs<T> A) {
    if (*A.done) return;
    const DDGeom &G = A.G;
    for (size_t a = blockIdx.x * (size_t)blockDim.x + threadIdx.x; a < G.coarse_elems;
         a += (size_t)gridDim.x * blockDim.x) {
        int g, i, j;
        if (!coarse_decode(G, a, g, i, j)) continue;
        GridDesc d = grid_desc(G, g);
        const int X = d.ox + G.c * i, Y = d.oy + G.c * j;
        const bool bxi = X % G.sx == 0 && X > 0 && X < G.nx - 1;
        const bool byi = Y % G.sy == 0 && Y > 0 && Y < G.ny - 1;
        const uint8_t Wk = A.W[a];
        int best = 0;
        if (bxi || byi) {
            int sel = 0;
            bool ok = true;
            for (int ax = 0; ax < 2 && ok; ++ax) {
                const bool on = ax == 0 ? bxi : byi;
                if (!on) continue;
                bool allneg = wind_comp(Wk, ax) <= 0, allpos = wind_comp(Wk, ax) >= 0;
                for (int s = 0; s < 4; ++s) {
                    if ((s & 1) && !bxi) continue;
                    if ((s & 2) && !byi) continue;
                    const int wv = wind_comp(A.cw[(size_t)s * G.coarse_elems + a], ax);
                    if (wv > 0) allneg = false;
                    if (wv < 0) allpos = false;
                }
                // Alg. 4: wind toward -axis -> the plus-side copy (first branch)
                if (allneg) sel |= (1 << ax);
                else if (!allpos) ok = false;
            }
            if (ok) {
                best = sel;
            } else {
                // minimum; ties keep the lowest subdomain index (slot order)
                best = 0;
                T bv = A.cu[a];
                for (int s = 1; s < 4; ++s) {
                    if ((s & 1) && !bxi) continue;
                    if ((s & 2) && !byi) continue;
                    const T v = A.cu[(size_t)s * G.coarse_elems + a];
                    if (v < bv) {
                        bv = v;
                        best = s;
                    }
                }
            }
        }
        const T ukv = A.cu[(size_t)best * G.coarse_elems + a];
        const uint8_t wkv = A.cw[(size_t)best * G.coarse_elems + a];
        A.uk[a] = ukv;
        A.wk[a] = wkv;
        A.u_out[(size_t)Y * A.sy + X] = ukv;
        // Alg. 5 agreement bits from w^k and W^k on the axes of the node's
        // coarse lines (A = axes with index = 0 mod c)
        uint8_t m = A.gamma[(size_t)Y * A.sy + X] ? 1 : 0;
        const bool onx = X % G.c == 0, ony = Y % G.c == 0;
        const int wkx = wind_comp(wkv, 0), wky = wind_comp(wkv, 1);
        const int Wx = wind_comp(Wk, 0), Wy = wind_comp(Wk, 1);
        if (!onx || (wkx <= 0 && Wx <= 0)) m |= 2;
        if (!onx || (wkx >= 0 && Wx >= 0)) m |= 4;
        if (!ony || (wky <= 0 && Wy <= 0)) m |= 8;
        if (!ony || (wky >= 0 && Wy >= 0)) m |= 16;
        for (int dd = 0; dd < 4; ++dd) {
            size_t si = d.skoff + skew_index(dd, i, j, d.nb, d.my, d.nstepp);
            A.uk_sk[si] = ukv;
            A.mask_sk[si] = m;
        }
    }
}

template <class T>
__global__ void k_check(DDArgs<T> A, int k) {
    if (*A.done) return;
    const double delta = A.deltas[k];
    const bool conv = k >= 1 && delta < (double)A.tol;
    if (k == A.max_iter || conv) {
        *A.done = 1;
        A.st->iters = k;
        A.st->converged = conv ? 1 : 0;
    }
}

__device__ inline void atomic_max_nonneg(double *addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

template <class T>
__global__ void k_delta(DDArgs<T> A, int k) {
    if (*A.done) return;
    const DDGeom &G = A.G;
    double m = 0.0;
    for (size_t a = blockIdx.x * (size_t)blockDim.x + threadIdx.x; a < G.coarse_elems;
         a += (size_t)gridDim.x * blockDim.x) {
        int g, i, j;
        if (!coarse_decode(G, a, g, i, j)) continue;
        const T u1 = A.U[a], u0 = A.Uprev[a];
        if (u1 == u0) continue;
        const double dv = fabs((double)u1 - (double)u0);
        if (dv > m) m = dv;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(FULL, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomic_max_nonneg(&A.deltas[k + 1], m);
}

template <class T>
__global__ void k_init_stats(DDArgs<T> A) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        memset(A.st, 0, sizeof(DevStats));
        *A.done = 0;
        A.bar[0] = A.bar[1] = 0;
    }
    for (int k = threadIdx.x; k < A.max_iter + 2; k += blockDim.x) A.deltas[k] = k == 0 ? INFINITY : 0.0;
}

template <class T>
__global__ void k_finalize(DDArgs<T> A, eik_dd_stats *out, long long launches) {
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
}

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------
struct DDPlan {
    DDGeom G;
    size_t bytes;
    size_t fine_smem, step1_smem, step4_smem;
    int grid_threads;
};

// 3-D implementation (eik_dd3.cu)
size_t dd3_workspace_size(const eik_grid *grid, const eik_dd_params *p);
bool dd3_validate(const eik_grid *grid, const eik_dd_params *p);
int dd3_run(const eik_grid *grid, const void *r, const uint8_t *gamma, const void *g, const eik_dd_params *p,
            void *u_out, void *ws, eik_dd_stats *stats, cudaStream_t s);

static bool dd_validate(const eik_grid *grid, const eik_dd_params *p) {
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
        return dd3_validate(grid, p);
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
    return true;
}

template <class T>
static size_t dd_layout(const DDPlan &P, DDArgs<T> *A, void *ws, int max_iter) {
    const DDGeom &G = P.G;
    Carver cv(ws);
    const size_t ntiles = (size_t)G.tx * G.ty;
    T *tile_state = cv.take<T>(ntiles * G.tile_elems);
    T *tile_rsk = cv.take<T>(ntiles * G.tile_sk_elems);
    T *U = cv.take<T>(G.coarse_elems);
    T *Uprev = cv.take<T>(G.coarse_elems);
    T *U0 = cv.take<T>(G.coarse_elems);
    T *rc = cv.take<T>(G.coarse_elems);
    T *uk = cv.take<T>(G.coarse_elems);
    uint8_t *W = cv.take<uint8_t>(G.coarse_elems);
    uint8_t *wk = cv.take<uint8_t>(G.coarse_elems);
    T *cu = cv.take<T>(4 * G.coarse_elems);
    uint8_t *cw = cv.take<uint8_t>(4 * G.coarse_elems);
    T *rc_sk = cv.take<T>(G.coarse_sk_elems);
    T *uk_sk = cv.take<T>(G.coarse_sk_elems);
    T *cold_sk = cv.take<T>(G.coarse_sk_elems);
    uint8_t *mask_sk = cv.take<uint8_t>(G.coarse_sk_elems);
    int *done = cv.take<int>(4);
    double *deltas = cv.take<double>((size_t)max_iter + 2);
    int *chg = cv.take<int>(4);
    unsigned *bar = cv.take<unsigned>(4);
    DevStats *st = cv.take<DevStats>(1);
    if (A) {
        A->tile_state = tile_state;
        A->tile_rsk = tile_rsk;
        A->U = U;
        A->Uprev = Uprev;
        A->U0 = U0;
        A->rc = rc;
        A->uk = uk;
        A->W = W;
        A->wk = wk;
        A->cu = cu;
        A->cw = cw;
        A->rc_sk = rc_sk;
        A->uk_sk = uk_sk;
        A->cold_sk = cold_sk;
        A->mask_sk = mask_sk;
        A->done = done;
        A->deltas = deltas;
        A->chg = chg;
        A->bar = bar;
        A->st = st;
    }
    return cv.used + 256;
}

static DDPlan dd_plan(const eik_grid *grid, const eik_dd_params *p) {
    DDPlan P;
    P.G = make_geom((int)grid->n[0], (int)grid->n[1], p->tiles[0], p->tiles[1], p->coarse_ratio, grid->h);
    P.step1_smem = P.step4_smem = 0;
    P.bytes = grid->dtype == EIK_F64 ? dd_layout<double>(P, nullptr, nullptr, p->max_iter)
                                     : dd_layout<float>(P, nullptr, nullptr, p->max_iter);
    const int gnb = ceil32(P.G.ncx + 1);
    P.grid_threads = 32 * gnb;
    if (grid->dtype == EIK_F64) {
        P.fine_smem = engine_smem_bytes<double, 1, false>(P.G.tnb, P.G.tny);
        P.step1_smem = engine_smem_bytes<double, 1, false>(gnb, P.G.ncy + 1);
        P.step4_smem = engine_smem_bytes<double, 3, true>(gnb, P.G.ncy + 1);
    } else {
        P.fine_smem = engine_smem_bytes<float, 1, false>(P.G.tnb, P.G.tny);
        P.step1_smem = engine_smem_bytes<float, 1, false>(gnb, P.G.ncy + 1);
        P.step4_smem = engine_smem_bytes<float, 3, true>(gnb, P.G.ncy + 1);
    }
    return P;
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
    A.tol = (T)p->tol;
    A.max_iter = p->max_iter;
    A.max_fsm = p->max_fsm_sweeps;
    A.max_coarse = p->max_coarse_sweeps;
    const DDGeom &G = P.G;
    const int ntiles = G.tx * G.ty;

    int rc;
    int dev;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    int nsm = 0;
    if ((rc = cuda_check(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "attr"))) return rc;
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if ((int)P.fine_smem > smem_optin || (int)P.step1_smem > smem_optin || (int)P.step4_smem > smem_optin) {
        set_error("shared memory need (%zu, %zu, %zu) exceeds the device limit %d", P.fine_smem, P.step1_smem,
                  P.step4_smem, smem_optin);
        return EIK_EUNSUPPORTED;
    }
    if ((rc = cuda_check(cudaFuncSetAttribute(DDKernels<T>::fine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.fine_smem),
                         "smem attr fine")))
        return rc;
    if ((rc = cuda_check(cudaFuncSetAttribute(DDKernels<T>::step1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.step1_smem),
                         "smem attr step1")))
        return rc;
    if ((rc = cuda_check(cudaFuncSetAttribute(DDKernels<T>::step4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.step4_smem),
                         "smem attr step4")))
        return rc;
    // causal sweep: cooperative grid sized to what is co-resident
    const int causal_threads = 256;
    int per_sm = 0;
    if ((rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_causal<T>, causal_threads, 0),
                         "occupancy")))
        return rc;
    const int lines = std::max(G.ncx, G.ncy) + 1;
    int causal_blocks = std::min(per_sm * nsm, std::max(1, (lines + 7) / 8));
    if (causal_blocks < 1) causal_blocks = 1;

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
        void *args[] = {&A, &only};
        int tok = prof_begin("dd_causal_sweep", s);
        int r2 = cuda_check(cudaLaunchCooperativeKernel((void *)k_causal<T>, causal_blocks, causal_threads, args, 0, s),
                            "causal launch");
        prof_end(tok, s);
        ++nl;
        return r2;
    };
    if ((rc = launch_causal(0))) return rc;
    for (int k = 0; k <= p->max_iter; ++k) {
        EIK_LAUNCH("dd_fine_subdomains", s, DDKernels<T>::fine<<<ntiles, 32 * G.tnb, P.fine_smem, s>>>(A)); ++nl;
        EIK_LAUNCH("dd_alg4_restrict", s, k_alg4<T><<<eb, ew, 0, s>>>(A)); ++nl;
        EIK_LAUNCH("dd_check", s, k_check<T><<<1, 1, 0, s>>>(A, k)); ++nl;
        if (k == p->max_iter) break;
        EIK_LAUNCH("dd_step4_weighted", s, DDKernels<T>::step4<<<G.ngrids, P.grid_threads, P.step4_smem, s>>>(A)); ++nl;
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
// Some callers cannot call cudaMalloc at all: code running inside a CUDA graph
// that is being captured (allocation calls are not capturable), hosts whose
// allocator is owned by another runtime that must not be bypassed, and
// real-time loops that forbid allocation after start-up.  For them the scratch
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

// dd2_device.cuh -- device side of the 2-D two-scale domain decomposition
// (Sec. 3.2, Steps 1-4, Alg. 1-5): argument block, engine policies and the
// per-stage bodies.  The single-problem solve (eik_dd.cu) and the batched
// solve (eik_dd_batch.cu) wrap the same bodies in their own kernels.
#pragma once

#include "common.cuh"
#include "dd_geom.cuh"
#include "engine.cuh"
#include "eik.h"

namespace eik {

struct DevStats {
    unsigned long long fsm_sweeps_max, coarse_sweeps_max, fsm_caps, coarse_caps;
    unsigned long long fine_updates, coarse_updates, fine_skips;
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
    int *ldirty;     // [ncy+1] horizontal then [ncx+1] vertical coarse lines the causal sweep must
                     // (re)visit; null: every line in every round
    int tile0;       // first subdomain of a subdomain launch (a slab of a sharded solve)
    // Step 2 data of each subdomain's last solve in this call, for the skip of
    // a solve whose data are unchanged: per face node the starting value and
    // the coarse wind an inflow copy echoes ([ntiles][face_nodes]); sig_ok
    // [ntiles] = 1 once the subdomain has been solved in this call
    T *sig_u;
    uint8_t *sig_w;
    int *sig_ok;
    // order of the subdomain launch when a planning pass ran before it (null:
    // CTA b solves tile0 + b and checks its own data): [ntiles] the
    // subdomains that need a solve first, then the others; order_cnt [2]
    // counts of both (reset by the stop test of each iteration)
    int *order;
    int *order_cnt;
    unsigned *bar;   // [2] grid barrier count / generation
    DevStats *st;
    T theta, tol;
    // constant weight 0: every branch of Alg. 5 yields u^k exactly (u^k + 0 (U~ -
    // C_H) = u^k), so Alg. 4 writes U^{k+1} = u^k itself and Step 4 has no sweeps
    int step4_identity;
    int max_iter;
    long long max_fsm, max_coarse;
    // per-node weight of Sec. 4.2 (adaptive theta)
    int adaptive;
    double om[3], sg, sd, sx0, cap;
    T *Ch[4];      // C_H(nbrs^H(U^m)) of the last four iterates m, slot m % 4
    T *theta_sk;   // skewed per-node weight (a static of the Alg. 5 sweeps)
};

template <class T>
__device__ __forceinline__ T fine_at(const T *a, long long sy, int X, int Y) {
    return a[(size_t)Y * sy + X];
}

// --------------------------------------------------------------------------
// Engine policies
// --------------------------------------------------------------------------

// FSM update u = min(u, u~) (Sec. 1.1, eq. FSMupdate).  Statics: r, stored
// as a non-positive value at fixed nodes (Gamma).
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
    bool per_node;  // weight from the fourth static instead of `theta`
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
        const T th = per_node ? sv[3] : theta;
        const T nu0 = pass ? N::add(uk, N::mul(th, N::sub(Ut, cold))) : uk;
        const T nu = (mask & 1) ? self : nu0;
        changed = !(nu == self);
        return nu;
    }
};

// --------------------------------------------------------------------------
// Set-up kernels (once per solve)
// --------------------------------------------------------------------------
// Bodies take the block index and count explicitly so that the batched
// kernels (several problems per launch) can reuse them.
template <class T>
__device__ void pack_tiles_body(const DDArgs<T> &A, size_t bid, size_t nbid) {
    const DDGeom &G = A.G;
    const size_t per_tile = (size_t)G.tnx * G.tny;
    const size_t total = per_tile * G.tx * G.ty;
    for (size_t t = bid * blockDim.x + threadIdx.x; t < total; t += nbid * blockDim.x) {
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
__global__ void k_pack_tiles(DDArgs<T> A) {
    pack_tiles_body(A, blockIdx.x, gridDim.x);
}

template <class T>
__device__ void pack_coarse_body(const DDArgs<T> &A, size_t bid, size_t nbid) {
    const DDGeom &G = A.G;
    for (size_t a = bid * blockDim.x + threadIdx.x; a < G.coarse_elems; a += nbid * blockDim.x) {
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

template <class T>
__global__ void k_pack_coarse(DDArgs<T> A) {
    pack_coarse_body(A, blockIdx.x, gridDim.x);
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
__device__ __forceinline__ void k_step1_body(const DDArgs<T> &A, char *smem, int gidx) {
    const DDGeom &G = A.G;
    const GridDesc d = grid_desc(G, gidx);
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
template <class T, bool ADAPT>
__device__ __forceinline__ void k_step4_gen(const DDArgs<T> &A, char *smem, int gidx) {
    if (*A.done || A.step4_identity) return;  // weight 0: Alg. 4 already wrote U^{k+1} = u^k
    const DDGeom &G = A.G;
    const GridDesc d = grid_desc(G, gidx);
    const T Hs = T(G.H);
    const size_t n = (size_t)d.nb * d.my * 32;
    T *U = A.U + d.off;
    // C_H(nbrs^H(U^k)), U^k and W = w^k were prepared by Alg. 4 (alg4_body)
    // "Initialize U as described in Sec. 1.1"
    for (size_t e = threadIdx.x; e < n; e += blockDim.x) U[e] = A.U0[d.off + e];
    __threadfence_block();
    __syncthreads();
    constexpr int NST = ADAPT ? 4 : 3;
    Box<T, NST> bx;
    bx.u = U;
    bx.st[0] = A.rc_sk + d.skoff;
    bx.st[1] = A.uk_sk + d.skoff;
    bx.st[2] = A.cold_sk + d.skoff;
    if (ADAPT) bx.st[NST - 1] = A.theta_sk + d.skoff;
    bx.sb = A.mask_sk + d.skoff;
    bx.nx = d.mx;
    bx.ny = d.my;
    bx.nb = d.nb;
    bx.nstepp = d.nstepp;
    Alg5Policy<T> pol{Hs, A.theta, ADAPT};
    long long sweeps;
    bool conv;
    engine_run<T, NST, true>(bx, pol, A.max_coarse, smem, sweeps, conv, &A.st->err);
    if (threadIdx.x == 0) {
        atomicMax(&A.st->coarse_sweeps_max, (unsigned long long)sweeps);
        if (!conv) atomicAdd(&A.st->coarse_caps, 1ull);
        atomicAdd(&A.st->coarse_updates, (unsigned long long)sweeps * d.mx * d.my);
    }
}

template <class T>
__device__ __forceinline__ void k_step4_body(const DDArgs<T> &A, char *smem, int gidx) {
    k_step4_gen<T, false>(A, smem, gidx);
}
template <class T>
__device__ __forceinline__ void k_step4a_body(const DDArgs<T> &A, char *smem, int gidx) {
    k_step4_gen<T, true>(A, smem, gidx);
}

// --------------------------------------------------------------------------
// Causal sweep (Alg. 2): least fixed point along every coarse line.
// --------------------------------------------------------------------------
// One direction of one line: values v (current) with "connected to the
// predecessor in scan order" flags; inclusive segmented max-scan per 32-node
// chunk with a carry across chunks.
// `cross` (nullable): flags of the crossing lines, one per coarse line of the
// other direction; a raised intersection node marks its crossing line.
template <class T>
__device__ bool causal_line(const DDArgs<T> &A, bool horizontal, int line, int rev, int *cross = nullptr) {
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
            if (cross && p % G.c == 0) cross[p / G.c] = 1;
        }
        carry = __shfl_sync(FULL, v, 31);
        carry_orig = __shfl_sync(FULL, u, 31);
    }
    return __any_sync(FULL, changed);  // warp-uniform: any lane raised a node
}

// The same sweep with the whole line staged in shared memory: one warp per
// line, values su[] and per-node bytes sw[] (bit 0: wind along +axis, bit 1:
// along -axis, bit 2: linked to its scan predecessor in the current pass,
// bit 7: raised).  In a pass each lane scans a contiguous segment of
// ceil(len/32) nodes serially, the lanes' segment results are combined by one
// warp scan of (value, linked-throughout) pairs, and each lane raises the
// linked prefix of its segment to the carry that reaches it.  The segmented
// max-scan has one result, so the values equal those of causal_line.
__host__ __device__ inline size_t causal_align16(size_t b) { return (b + 15) & ~(size_t)15; }
template <class T>
__host__ __device__ inline size_t causal_warp_bytes(int lw) {
    return causal_align16((size_t)lw * sizeof(T)) + causal_align16((size_t)lw);
}

template <class T>
__device__ void causal_pass_smem(T *su, uint8_t *sw, int len, int rev) {
    const T INF = Num<T>::inf();
    const int lane = threadIdx.x & 31;
    const int seg = (len + 31) >> 5;
    const int s = lane * seg;
    const int e = s + seg < len ? s + seg : len;
    const uint8_t dirbit = rev ? 2 : 1;
    // original value of the node before this segment in scan order
    T prev_orig = (s > 0 && s <= len) ? su[rev ? len - s : s - 1] : INF;
    __syncwarp();
    T vprev = -INF;
    bool through = true;
    for (int pos = s; pos < e; ++pos) {
        const int idx = rev ? len - 1 - pos : pos;
        const T orig = su[idx];
        uint8_t w = sw[idx];
        const bool f = (w & dirbit) && pos > 0 && (prev_orig < INF);
        const T v = (pos > s && f) ? fmax(orig, vprev) : orig;
        through = through && f;
        w = f ? (uint8_t)(w | 4) : (uint8_t)(w & ~4);
        if (v > orig) {
            su[idx] = v;
            w |= 0x80;
        }
        sw[idx] = w;
        prev_orig = orig;
        vprev = v;
    }
    // carry reaching each segment: composition of x -> (all ? max(v, x) : v)
    T cv = vprev;
    bool ca = through;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T pv = __shfl_up_sync(FULL, cv, o);
        const bool pa = __shfl_up_sync(FULL, ca ? 1 : 0, o) != 0;
        if (lane >= o) {
            cv = ca ? fmax(cv, pv) : cv;
            ca = ca && pa;
        }
    }
    T carry = __shfl_up_sync(FULL, cv, 1);
    if (lane == 0) carry = -INF;
    if (carry > -INF) {
        for (int pos = s; pos < e; ++pos) {
            const int idx = rev ? len - 1 - pos : pos;
            const uint8_t w = sw[idx];
            if (!(w & 4)) break;
            if (carry > su[idx]) {
                su[idx] = carry;
                sw[idx] = (uint8_t)(w | 0x80);
            }
        }
    }
    __syncwarp();
}

// Both passes of Alg. 2 on one coarse line through shared memory; returns
// whether any node was raised (warp-uniform).
template <class T>
__device__ bool causal_line_smem(const DDArgs<T> &A, bool horizontal, int line, T *su, uint8_t *sw,
                                 int *cross = nullptr) {
    const DDGeom &G = A.G;
    const int lane = threadIdx.x & 31;
    const int len = horizontal ? G.nx : G.ny;
    const int fixedc = line * G.c;
    const int axis = horizontal ? 0 : 1;
    constexpr int UNR = 4;
    for (int p0 = 0; p0 < len; p0 += 32 * UNR) {
        T uv[UNR];
        uint8_t wv[UNR];
#pragma unroll
        for (int r = 0; r < UNR; ++r) {
            const int p = p0 + 32 * r + lane;
            uv[r] = Num<T>::inf();
            wv[r] = WIND_ZERO;
            if (p < len) {
                const size_t a = coarse_addr(G, horizontal ? p : fixedc, horizontal ? fixedc : p);
                uv[r] = __ldcg(A.U + a);
                wv[r] = __ldcg(A.W + a);
            }
        }
#pragma unroll
        for (int r = 0; r < UNR; ++r) {
            const int p = p0 + 32 * r + lane;
            if (p < len) {
                const int wc = wind_comp(wv[r], axis);
                su[p] = uv[r];
                sw[p] = (uint8_t)((wc > 0 ? 1 : 0) | (wc < 0 ? 2 : 0));
            }
        }
    }
    __syncwarp();
    causal_pass_smem(su, sw, len, 0);
    causal_pass_smem(su, sw, len, 1);
    bool changed = false;
    for (int p = lane; p < len; p += 32) {
        if (sw[p] & 0x80) {
            A.U[coarse_addr(G, horizontal ? p : fixedc, horizontal ? fixedc : p)] = su[p];
            changed = true;
            if (cross && p % G.c == 0) cross[p / G.c] = 1;
        }
    }
    __syncwarp();
    return __any_sync(FULL, changed);
}

// lw > 0: lines staged in shared memory (lw = capacity per warp, dynamic
// shared memory of causal_warp_bytes<T>(lw) per warp); lw = 0: lines read
// and written in place, 32 nodes at a time.
template <class T>
__global__ void k_causal(DDArgs<T> A, int only_if_not_done, int lw) {
    const long long wlim = spin_limit();  // limit of the grid-barrier waits
    if (only_if_not_done && *A.done) return;
    const DDGeom &G = A.G;
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    extern __shared__ __align__(16) unsigned char causal_smem[];
    T *su = reinterpret_cast<T *>(causal_smem + (size_t)(threadIdx.x >> 5) * causal_warp_bytes<T>(lw));
    uint8_t *sw = reinterpret_cast<uint8_t *>(su) + causal_align16((size_t)lw * sizeof(T));
    __shared__ int blk_changed;
    if (blockIdx.x == 0 && threadIdx.x < 3) A.chg[threadIdx.x] = 0;
    // Lines share only their intersection nodes, so after the first round a
    // line needs another pass only if a crossing line raised one of them: the
    // flags start set, a line clears its own before its pass, and a raised
    // intersection node sets the crossing line's.  The least fixed point is
    // the same; lines that cannot change are skipped.
    int *const hdirty = A.ldirty, *const vdirty = A.ldirty ? A.ldirty + G.ncy + 1 : nullptr;
    if (A.ldirty)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G.ncy + 1 + G.ncx + 1; i += gridDim.x * blockDim.x)
            A.ldirty[i] = 1;
    if (!grid_barrier(A.bar, &A.st->err, wlim)) return;
    int rounds = 0;
    for (;;) {
        if (threadIdx.x == 0) blk_changed = 0;
        __syncthreads();
        bool ch = false;
        for (int l = gw; l <= G.ncy; l += warps_total) {
            if (hdirty) {
                if (!vload(hdirty + l)) continue;
                __syncwarp();
                if (lane == 0) hdirty[l] = 0;
            }
            if (lw > 0) {
                ch |= causal_line_smem(A, true, l, su, sw, vdirty);
            } else {
                ch |= causal_line(A, true, l, 0, vdirty);
                ch |= causal_line(A, true, l, 1, vdirty);
            }
        }
        if (!grid_barrier(A.bar, &A.st->err, wlim)) return;
        for (int l = gw; l <= G.ncx; l += warps_total) {
            if (vdirty) {
                if (!vload(vdirty + l)) continue;
                __syncwarp();
                if (lane == 0) vdirty[l] = 0;
            }
            if (lw > 0) {
                ch |= causal_line_smem(A, false, l, su, sw, hdirty);
            } else {
                ch |= causal_line(A, false, l, 0, hdirty);
                ch |= causal_line(A, false, l, 1, hdirty);
            }
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

// Face nodes of a subdomain box (NX x NY nodes): the bottom and top rows,
// then the left and right columns without their corners.
__host__ __device__ inline int tile_face_count(const DDGeom &G) { return 2 * G.tnx + 2 * (G.tny - 2); }
__device__ inline void tile_face_node(const DDGeom &G, int f, int &xl, int &yl) {
    const int NX = G.tnx, NY = G.tny;
    if (f < NX) { xl = f; yl = 0; }
    else if (f < 2 * NX) { xl = f - NX; yl = NY - 1; }
    else if (f < 2 * NX + NY - 2) { xl = 0; yl = 1 + f - 2 * NX; }
    else { xl = NX - 1; yl = 1 + f - 2 * NX - (NY - 2); }
}

template <class T>
__device__ __forceinline__ bool same_bits(T a, T b);
template <>
__device__ __forceinline__ bool same_bits<float>(float a, float b) { return __float_as_uint(a) == __float_as_uint(b); }
template <>
__device__ __forceinline__ bool same_bits<double>(double a, double b) {
    return __double_as_longlong(a) == __double_as_longlong(b);
}

// Whether subdomain `tile` must be solved in this iteration: its Step 2 data
// (every face node's starting value, and the coarse wind that an inflow node
// keeping its value echoes in Step 3's copies) differ from those of its last
// solve in this call, or it has not been solved yet.  The interior starts at
// +inf and r, Gamma and g do not change within a call, so equal data give the
// same solve bit for bit: its results (the fine values in u_out, the copies at
// the coarse-set nodes, the subdomain state) are still in place.  Records the
// new data.  All threads of the CTA call it and get the same answer.
template <class T>
__device__ bool tile_needs_solve(const DDArgs<T> &A, int tile) {
    const DDGeom &G = A.G;
    const T INF = Num<T>::inf();
    const int tx = tile % G.tx, ty = tile / G.tx;
    const int nf = tile_face_count(G);
    T *su = A.sig_u + (size_t)tile * nf;
    uint8_t *sw = A.sig_w + (size_t)tile * nf;
    bool diff = false;
    for (int f = threadIdx.x; f < nf; f += blockDim.x) {
        int xl, yl;
        tile_face_node(G, f, xl, yl);
        const int X = tx * G.sx + xl, Y = ty * G.sy + yl;
        T v = INF;
        uint8_t wv = 0;
        size_t ca;
        if (A.gamma[(size_t)Y * A.sy + X]) {
            v = fine_at(A.g, A.sy, X, Y);
        } else if (tile_inflow(A, xl, yl, X, Y, ca)) {
            v = A.U[ca];
            wv = A.W[ca];
        }
        if (!same_bits(v, su[f]) || wv != sw[f]) {
            diff = true;
            su[f] = v;
            sw[f] = wv;
        }
    }
    const bool solved = A.sig_ok[tile] != 0;
    const bool need = __syncthreads_or(diff) || !solved;
    if (need && threadIdx.x == 0) A.sig_ok[tile] = 1;
    return need;
}

template <class T, bool STEADY_PATH = true>
__device__ __forceinline__ void k_fine_body(const DDArgs<T> &A, char *smem, int tile, bool check = true) {
    if (*A.done) return;
    if (check && !tile_needs_solve(A, tile)) {
        if (threadIdx.x == 0) atomicAdd(&A.st->fine_skips, 1ull);
        return;
    }
    const DDGeom &G = A.G;
    const T INF = Num<T>::inf();
    const int tx = tile % G.tx, ty = tile / G.tx;
    const int NX = G.tnx, NY = G.tny;
    T *ut = A.tile_state + (size_t)tile * G.tile_elems;
    // Step 2: boundary data.  Inflow nodes start at U, interior and outflow
    // nodes at +inf; all of them are swept (Step 3), only Gamma is fixed.
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
    // (Gamma nodes carry a non-positive slowness in the skewed statics, set
    // once when the statics are packed)
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
    engine_run<T, 1, false, false, STEADY_PATH>(bx, pol, A.max_fsm, smem, sweeps, conv, &A.st->err);
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
            if (tile_inflow(A, xl, yl, X, Y, ca2) && uv == A.U[ca]) {
                w = A.W[ca] | WIND_ECHO;  // inflow value kept: the coarse wind
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

// --------------------------------------------------------------------------
// Exchange records of a sharded solve: the copies (u, w) one subdomain wrote at
// its coarse-set nodes (Step 3's output that Alg. 4 reads), in a fixed order:
// rows yl = 0..S, in a row on a coarse line every node, in another row the
// nodes on coarse columns.  Record = [ncs values][ncs winds], each part
// padded to 16 bytes.
// --------------------------------------------------------------------------
__host__ __device__ inline int tile_coarse_count(const DDGeom &G) {
    const int full = G.sy / G.c + 1, colc = G.sx / G.c + 1;
    return full * G.tnx + (G.tny - full) * colc;
}
template <class T>
__host__ __device__ inline size_t tile_record_bytes(const DDGeom &G) {
    const size_t n = (size_t)tile_coarse_count(G);
    return ((n * sizeof(T) + 15) & ~(size_t)15) + ((n + 15) & ~(size_t)15);
}
// Position of tile node (xl, yl) in the record (-1: not on the coarse set).
__device__ inline int tile_coarse_index(const DDGeom &G, int xl, int yl) {
    const int colc = G.sx / G.c + 1;
    const int full = (yl + G.c - 1) / G.c;  // coarse rows below yl
    const int base = full * G.tnx + (yl - full) * colc;
    if (yl % G.c == 0) return base + xl;
    return xl % G.c == 0 ? base + xl / G.c : -1;
}
// Copy slot of tile node (xl, yl) at fine node (X, Y) (as written by Step 3).
__device__ inline int tile_copy_slot(const DDGeom &G, int xl, int yl, int X, int Y) {
    int slot = 0;
    if (X % G.sx == 0 && X > 0 && X < G.nx - 1 && xl == 0) slot |= 1;
    if (Y % G.sy == 0 && Y > 0 && Y < G.ny - 1 && yl == 0) slot |= 2;
    return slot;
}

// pack = 1: copies of tiles [t0, t1) -> their records; pack = 0: every record
// of tiles [t0, t1) -> the copies.
template <class T>
__global__ void k_shard_records(DDArgs<T> A, int t0, int t1, unsigned char *xbuf, int pack) {
    const DDGeom &G = A.G;
    const int ncs = tile_coarse_count(G);
    const size_t rec = tile_record_bytes<T>(G);
    const size_t voff = ((size_t)ncs * sizeof(T) + 15) & ~(size_t)15;
    const size_t per_tile = (size_t)G.tnx * G.tny;
    const size_t total = per_tile * (size_t)(t1 - t0);
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int tile = t0 + (int)(e / per_tile);
        const int rem = (int)(e % per_tile);
        const int xl = rem % G.tnx, yl = rem / G.tnx;
        const int idx = tile_coarse_index(G, xl, yl);
        if (idx < 0) continue;
        const int X = (tile % G.tx) * G.sx + xl, Y = (tile / G.tx) * G.sy + yl;
        const size_t slot = (size_t)tile_copy_slot(G, xl, yl, X, Y) * G.coarse_elems + coarse_addr(G, X, Y);
        unsigned char *r = xbuf + (size_t)tile * rec;
        T *rv = reinterpret_cast<T *>(r);
        uint8_t *rw = r + voff;
        if (pack) {
            rv[idx] = A.cu[slot];
            rw[idx] = A.cw[slot];
        } else {
            A.cu[slot] = rv[idx];
            A.cw[slot] = rw[idx];
        }
    }
}

// --------------------------------------------------------------------------
// Alg. 4 + inputs of Alg. 5
// --------------------------------------------------------------------------
template <class T>
__device__ void alg4_body(const DDArgs<T> &A, int k, size_t bid, size_t nbid) {
    if (*A.done) return;
    const DDGeom &G = A.G;
    for (size_t a = bid * blockDim.x + threadIdx.x; a < G.coarse_elems; a += nbid * blockDim.x) {
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
                // minimum of the fine solutions: copies that echo their Step 2
                // value are candidates only if every copy does; ties keep the
                // lowest subdomain index (slot order)
                bool computed = false;
                for (int s = 0; s < 4; ++s) {
                    if ((s & 1) && !bxi) continue;
                    if ((s & 2) && !byi) continue;
                    if (!(A.cw[(size_t)s * G.coarse_elems + a] & WIND_ECHO)) computed = true;
                }
                best = -1;
                T bv = T(0);
                for (int s = 0; s < 4; ++s) {
                    if ((s & 1) && !bxi) continue;
                    if ((s & 2) && !byi) continue;
                    if (computed && (A.cw[(size_t)s * G.coarse_elems + a] & WIND_ECHO)) continue;
                    const T v = A.cu[(size_t)s * G.coarse_elems + a];
                    if (best < 0 || v < bv) {
                        bv = v;
                        best = s;
                    }
                }
            }
        }
        const T ukv = A.cu[(size_t)best * G.coarse_elems + a];
        const uint8_t wkv = A.cw[(size_t)best * G.coarse_elems + a] & (uint8_t)~WIND_ECHO;
        const T uold = A.uk[a];  // u^{k-1} (meaningful for k >= 1)
        A.uk[a] = ukv;
        A.wk[a] = wkv;
        A.u_out[(size_t)Y * A.sy + X] = ukv;
        if (A.step4_identity) {
            // Step 4 with weight 0: U^{k+1} = u^k before the causal sweep, W = w^k
            // (no thread reads a neighbour's U here, so the update is in place)
            A.Uprev[a] = A.U[a];
            A.U[a] = ukv;
            A.W[a] = wkv;
            continue;
        }
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
        // Step 4 inputs that depend only on U^k, computed here while U still
        // holds U^k: C_H(nbrs^H(U^k)) of the node's own shifted grid, U^k for
        // the delta, and W = w^k (the mask above has read W^k)
        const T INF = Num<T>::inf();
        const T *Ug = A.U + d.off;
        const T vmx = i > 0 ? Ug[box_index(i - 1, j, d.my)] : INF;
        const T vpx = i + 1 < d.mx ? Ug[box_index(i + 1, j, d.my)] : INF;
        const T vmy = j > 0 ? Ug[box_index(i, j - 1, d.my)] : INF;
        const T vpy = j + 1 < d.my ? Ug[box_index(i, j + 1, d.my)] : INF;
        const T rv = A.rc[a];
        const T cold = local_solve2_value(vmx, vpx, vmy, vpy, Num<T>::mul(rv > T(0) ? rv : T(0), T(G.H)));
        A.Uprev[a] = A.U[a];
        A.W[a] = wkv;
        T th = A.theta;
        if (A.adaptive) {
            double thv = (double)A.theta;
            if (k >= 1) {
                const int n = k < 3 ? k : 3;
                const T *c1 = A.Ch[(k + 3) & 3], *c2 = A.Ch[(k + 2) & 3], *c3 = A.Ch[(k + 1) & 3];
                double dC[3] = {0.0, 0.0, 0.0};
                dC[0] = __dsub_rn((double)cold, (double)c1[a]);
                if (n > 1) dC[1] = __dsub_rn((double)c1[a], (double)c2[a]);
                if (n > 2) dC[2] = __dsub_rn((double)c2[a], (double)c3[a]);
                thv = theta_estimate(A, __dsub_rn((double)ukv, (double)uold), dC, n, (double)A.theta);
            }
            A.Ch[k & 3][a] = cold;
            th = (T)thv;
        }
        for (int dd = 0; dd < 4; ++dd) {
            size_t si = d.skoff + skew_index(dd, i, j, d.nb, d.my, d.nstepp);
            A.uk_sk[si] = ukv;
            A.mask_sk[si] = m;
            A.cold_sk[si] = cold;
            if (A.theta_sk) A.theta_sk[si] = th;  // per-node or (in a mixed batch) constant weight
        }
    }
}

template <class T>
__global__ void k_alg4(DDArgs<T> A, int k) {
    alg4_body(A, k, blockIdx.x, gridDim.x);
}

template <class T>
__device__ void check_body(const DDArgs<T> &A, int k) {
    if (A.order_cnt) A.order_cnt[0] = A.order_cnt[1] = 0;  // for the next planning pass
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
__global__ void k_check(DDArgs<T> A, int k) {
    check_body(A, k);
}

__device__ inline void atomic_max_nonneg(double *addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

template <class T>
__device__ void delta_body(const DDArgs<T> &A, int k, size_t bid, size_t nbid) {
    if (*A.done) return;
    const DDGeom &G = A.G;
    double m = 0.0;
    for (size_t a = bid * blockDim.x + threadIdx.x; a < G.coarse_elems; a += nbid * blockDim.x) {
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
__global__ void k_delta(DDArgs<T> A, int k) {
    delta_body(A, k, blockIdx.x, gridDim.x);
}

template <class T>
__device__ void init_body(const DDArgs<T> &A) {
    if (threadIdx.x == 0) {
        memset(A.st, 0, sizeof(DevStats));
        *A.done = 0;
        A.bar[0] = A.bar[1] = 0;
    }
    for (int k = threadIdx.x; k < A.max_iter + 2; k += blockDim.x) A.deltas[k] = k == 0 ? INFINITY : 0.0;
    for (int t = threadIdx.x; t < A.G.tx * A.G.ty; t += blockDim.x) A.sig_ok[t] = 0;
    if (threadIdx.x == 0 && A.order_cnt) A.order_cnt[0] = A.order_cnt[1] = 0;
}

template <class T>
__global__ void k_init_stats(DDArgs<T> A) {
    init_body(A);
}

template <class T>
__device__ void finalize_body(const DDArgs<T> &A, eik_dd_stats *out, long long launches) {
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

template <class T>
__global__ void k_finalize(DDArgs<T> A, eik_dd_stats *out, long long launches) {
    finalize_body(A, out, launches);
}

}  // namespace eik

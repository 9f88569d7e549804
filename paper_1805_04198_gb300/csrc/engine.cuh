// engine.cuh -- warp-systolic Gauss-Seidel sweep engine for one 2-D grid box.
//
// A sweep of the fast sweeping method (Sec. 1.1) visits the nodes in one of
// the 2^d orderings; node (x, y) then reads its upwind-in-the-ordering
// neighbours already updated in this sweep and the other two from before it.
// Any schedule that respects exactly those four dependencies gives the same
// result as the serial loop nest.  The schedule used here:
//
//  * the box is cut into 32-column blocks; one warp owns one block and one
//    lane owns one column of it (logical column order follows the sweep sign
//    of x, so lane 0 is the upwind side);
//  * at step s lane l updates logical row s - l: its left neighbour (new) comes
//    from lane l-1 by a register shuffle, its upper neighbour (new) is the value
//    it produced one step earlier, its right neighbour (old) is lane l+1's
//    prefetched lower neighbour, shuffled down;
//  * the block's rows stream through a 48-row shared-memory ring (6 chunks of
//    8 rows): chunks are loaded two chunks ahead with coalesced 16-byte loads
//    and written back as soon as all 32 lanes finished them;
//  * lane 31 hands its new column to the next block's warp through shared
//    memory, published every chunk; lane 31 reads the next block's first
//    column (old values) from global memory, prefetched with the chunk;
//  * per-node read-only data ("statics": slowness, masks, ...) are stored
//    pre-skewed per sweep direction ([dir][block][step][lane]) so each step is
//    one coalesced 128-byte load, prefetched a chunk ahead into registers.
//
// Storage of the state u: strip-major [block][row][32] (row = physical y,
// 32 = physical x within the block), padded to a whole number of blocks;
// padding columns are never touched.  One-sided differences at the box edges
// come for free: missing neighbours are +inf.
#pragma once

#include "common.cuh"

namespace eik {

constexpr int CH = 8;            // rows per chunk
constexpr int RS = 6;            // chunks held in the ring
constexpr int RROWS = CH * RS;   // ring rows per warp

__host__ __device__ inline int ceil32(int v) { return (v + 31) >> 5; }

// Element index of node (i, j) of a strip-major box of height my.
__host__ __device__ inline size_t box_index(int i, int j, int my) {
    return ((size_t)(i >> 5) * my + j) * 32 + (i & 31);
}

__host__ __device__ inline int nstep_padded(int ny) { return ((ny + 31 + CH - 1) / CH) * CH + 2 * CH; }

// Sweep direction d in [0, 4): bit 1 = sign of x, bit 0 = sign of y (set =
// +1).  The paper's loop nest (x sign outermost, -1 first) visits d = 0..3 in
// order, so sweep k uses d = k % 4.
__host__ __device__ inline int dir_sx(int d) { return (d & 2) ? 1 : -1; }
__host__ __device__ inline int dir_sy(int d) { return (d & 1) ? 1 : -1; }

// Index of node (i, j) of a box (width mx -> nb blocks, height my) in the
// skewed statics layout for direction d.
__host__ __device__ inline size_t skew_index(int d, int i, int j, int nb, int my, int nstepp) {
    int sx = dir_sx(d), sy = dir_sy(d);
    int b = i >> 5, pc = i & 31;
    int q = sx > 0 ? b : nb - 1 - b;
    int l = sx > 0 ? pc : 31 - pc;
    int lr = sy > 0 ? j : my - 1 - j;
    int s = lr + l;
    return (((size_t)d * nb + q) * nstepp + s) * 32 + l;
}

template <class T, int NST>
struct Box {
    T *u;                          // state, strip-major [nb][ny][32]
    const T *st[NST];              // skewed statics [4][nb][nstepp][32]
    const uint8_t *sb;             // skewed byte statics (may be null)
    int nx, ny, nb, nstepp;
};

// Shared memory needed per CTA (one warp per block).
template <class T>
__host__ __device__ inline size_t engine_smem_bytes(int nb, int ny) {
    size_t per_warp = (size_t)RROWS * 32 * sizeof(T) + (size_t)RROWS * sizeof(T) +
                      (size_t)((ny + 3) & ~3) * sizeof(T);
    return nb * per_warp + 16 * sizeof(int) + (size_t)nb * sizeof(int) + 64;
}

struct EngineShared {
    int abort_flag;
};

template <class T>
__device__ __forceinline__ T ld_cg(const T *p) { return __ldcg(p); }

// One sweep of one block by one warp.  Returns whether any node changed.
template <class T, int NST, bool HASB, class P>
__device__ bool run_block(const Box<T, NST> &bx, P &pol, int dir, int q, T *ring, T *halo, T *hand_out,
                          const T *hand_in, volatile int *prog_out, volatile int *prog_in,
                          volatile int *abort_flag, int *err) {
    using N = Num<T>;
    const T INF = N::inf();
    const int lane = threadIdx.x & 31;
    const int NB = bx.nb, NY = bx.ny, NX = bx.nx;
    const int sx = dir_sx(dir), sy = dir_sy(dir);
    const int b = sx > 0 ? q : NB - 1 - q;
    const int pc = sx > 0 ? lane : 31 - lane;
    const int x = 32 * b + pc;
    const bool colok = x < NX;
    const bool has_prev = q > 0;
    const bool has_next = q + 1 < NB;
    const int bn = sx > 0 ? b + 1 : b - 1;
    const int pcn = sx > 0 ? 0 : 31;
    const bool nextok = has_next && (32 * bn + pcn) < NX;
    T *ublk = bx.u + (size_t)b * NY * 32;
    const T *unext = bx.u + (size_t)(has_next ? bn : b) * NY * 32;
    const size_t stbase = ((size_t)dir * NB + q) * bx.nstepp;
    const int nchunks = (NY + CH - 1) / CH;
    const int nsteps = NY + 31;

    // staging: lane covers logical row r8 of the chunk, columns cg*8 .. cg*8+7
    constexpr int SV = (8 * (int)sizeof(T)) / 16;
    const int r8 = lane >> 2, cg = lane & 3;
    uint4 stage[SV];
    T hstage = INF;

    auto prow = [&](int m) { return sy > 0 ? m : NY - 1 - m; };
    auto load_chunk = [&](int j) {
        int m = j * CH + r8;
        if (m < NY) {
            const uint4 *src = reinterpret_cast<const uint4 *>(ublk + (size_t)prow(m) * 32 + cg * 8);
#pragma unroll
            for (int k = 0; k < SV; ++k) stage[k] = __ldcg(src + k);
        }
        int mh = j * CH + lane;
        hstage = INF;
        if (lane < CH && nextok && mh < NY) hstage = ld_cg(unext + (size_t)prow(mh) * 32 + pcn);
    };
    auto store_chunk = [&](int j) {
        int m = j * CH + r8;
        uint4 *dst = reinterpret_cast<uint4 *>(ring + ((j % RS) * CH + r8) * 32 + cg * 8);
        if (m < NY) {
#pragma unroll
            for (int k = 0; k < SV; ++k) dst[k] = stage[k];
        }
        if (lane < CH) halo[(j % RS) * CH + lane] = hstage;
    };
    auto write_back = [&](int j) {
        int m = j * CH + r8;
        if (m < NY) {
            const uint4 *src = reinterpret_cast<const uint4 *>(ring + ((j % RS) * CH + r8) * 32 + cg * 8);
            uint4 *dst = reinterpret_cast<uint4 *>(ublk + (size_t)prow(m) * 32 + cg * 8);
#pragma unroll
            for (int k = 0; k < SV; ++k) __stcg(dst + k, src[k]);
        }
    };

    T stc[NST > 0 ? NST : 1][CH], stn[NST > 0 ? NST : 1][CH];
    uint8_t sbc[CH], sbn[CH];
    auto load_statics = [&](int j, T (&dst)[NST > 0 ? NST : 1][CH], uint8_t (&dsb)[CH]) {
#pragma unroll
        for (int i = 0; i < CH; ++i) {
            int s = j * CH + i;
            bool ok = s < bx.nstepp;
            size_t idx = (stbase + (size_t)s) * 32 + lane;
#pragma unroll
            for (int k = 0; k < NST; ++k) dst[k][i] = ok ? __ldcg(bx.st[k] + idx) : T(0);
            if (HASB) dsb[i] = ok ? __ldcg(bx.sb + idx) : (uint8_t)0;
        }
    };

    // prologue: chunk 0 into the ring, chunk 1 staged, statics of chunks 0, 1
    load_chunk(0);
    store_chunk(0);
    if (nchunks > 1) load_chunk(1);
    load_statics(0, stc, sbc);
    load_statics(1, stn, sbn);

    T last = INF;
    bool changed = false;
    const int lastJ = nchunks + RS - 2;  // boundary that writes back the last chunk

    for (int J = 0; J <= lastJ; ++J) {
        __syncwarp();
        if (J >= RS - 1 && J - (RS - 1) < nchunks) write_back(J - (RS - 1));
        if (has_next) {
            // rows whose hand-off values lane 31 has written: m <= 8J - 32
            int done = 8 * J - 31;
            done = done < 0 ? 0 : (done > NY ? NY : done);
            if (J == lastJ) done = NY;
            if (lane == 31) {
                __threadfence_block();
                *prog_out = done;
            }
        }
        if (J + 1 < nchunks) store_chunk(J + 1);
        if (J + 2 < nchunks) load_chunk(J + 2);
        if (J > 0) {
#pragma unroll
            for (int i = 0; i < CH; ++i) {
#pragma unroll
                for (int k = 0; k < NST; ++k) stc[k][i] = stn[k][i];
                if (HASB) sbc[i] = sbn[i];
            }
            load_statics(J + 1, stn, sbn);
        }
        const int s0 = J * CH;
        if (s0 < nsteps && has_prev) {
            int need = s0 + CH;
            need = need > NY ? NY : need;
            long long it = 0;
            while (*prog_in < need) {
                if (*abort_flag) break;
                if (++it > SPIN_LIMIT) {
                    *abort_flag = 1;
                    atomicExch(err, DEV_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
            __threadfence_block();
        }
        __syncwarp();
        if (*abort_flag) break;
        if (s0 >= nsteps) continue;

#pragma unroll
        for (int i = 0; i < CH; ++i) {
            const int s = s0 + i;
            const int m = s - lane;
            const bool rowok = (unsigned)m < (unsigned)NY;
            const bool act = rowok && colok;
            const int slot = rowok ? ((m >> 3) % RS) * CH + (m & 7) : 0;
            T self = INF, dn = INF;
            if (act) self = ring[slot * 32 + pc];
            const int m1 = m + 1;
            if (colok && (unsigned)m1 < (unsigned)NY) dn = ring[(((m1 >> 3) % RS) * CH + (m1 & 7)) * 32 + pc];
            T left = __shfl_up_sync(FULL, last, 1);
            T right = __shfl_down_sync(FULL, dn, 1);
            if (lane == 0) left = (has_prev && rowok) ? hand_in[m] : INF;
            if (lane == 31) right = (nextok && rowok) ? halo[slot] : INF;
            const T up = last;
            T nw = INF;
            if (act) {
                const T vmx = sx > 0 ? left : right, vpx = sx > 0 ? right : left;
                const T vmy = sy > 0 ? up : dn, vpy = sy > 0 ? dn : up;
                const int y = sy > 0 ? m : NY - 1 - m;
                T sv[NST > 0 ? NST : 1];
#pragma unroll
                for (int k = 0; k < NST; ++k) sv[k] = stc[k][i];
                nw = pol.update(self, vmx, vpx, vmy, vpy, sv, HASB ? sbc[i] : (uint8_t)0, x, y, changed);
                ring[slot * 32 + pc] = nw;
                if (lane == 31 && has_next) hand_out[m] = nw;
            }
            last = nw;
        }
    }
    return __any_sync(FULL, changed);
}

// Runs sweeps on one box until a sweep changes nothing or max_sweeps ran.
// Requires blockDim.x == 32 * bx.nb and engine_smem_bytes<T>(nb, ny) bytes of
// dynamic shared memory starting at `smem`.  All threads must call it.
template <class T, int NST, bool HASB, class P>
__device__ void engine_run(const Box<T, NST> &bx, P &pol, long long max_sweeps, char *smem, long long &sweeps,
                           bool &converged, int *err) {
    const int nw = bx.nb;
    const int warp = threadIdx.x >> 5;
    const size_t ring_elems = (size_t)RROWS * 32, halo_elems = RROWS, hand_elems = (size_t)((bx.ny + 3) & ~3);
    T *base = reinterpret_cast<T *>(smem);
    T *ring = base + (size_t)warp * ring_elems;
    T *halo = base + (size_t)nw * ring_elems + (size_t)warp * halo_elems;
    T *hands = base + (size_t)nw * (ring_elems + halo_elems);
    int *ints = reinterpret_cast<int *>(hands + (size_t)nw * hand_elems);
    volatile int *abort_flag = ints;
    volatile int *prog = ints + 16;

    if (threadIdx.x == 0) *abort_flag = 0;
    sweeps = 0;
    converged = false;
    while (sweeps < max_sweeps) {
        const int dir = (int)(sweeps & 3);
        if ((int)threadIdx.x < nw) prog[threadIdx.x] = 0;
        __syncthreads();
        bool ch = false;
        if (warp < nw) {
            ch = run_block<T, NST, HASB>(bx, pol, dir, warp, ring, halo, hands + (size_t)warp * hand_elems,
                                         hands + (size_t)(warp > 0 ? warp - 1 : 0) * hand_elems, prog + warp,
                                         prog + (warp > 0 ? warp - 1 : 0), abort_flag, err);
        }
        const int any = __syncthreads_or(ch ? 1 : 0);
        ++sweeps;
        if (*abort_flag) break;
        if (!any) {
            converged = true;
            break;
        }
    }
    __syncthreads();
}

}  // namespace eik

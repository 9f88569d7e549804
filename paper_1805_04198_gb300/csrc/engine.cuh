// engine.cuh -- warp-systolic Gauss-Seidel sweep engine for one 2-D grid box.
//
// A sweep of the fast sweeping method (Sec. 1.1) visits the nodes in one of
// the 2^d orderings; node (x, y) then reads its upwind-in-the-ordering
// neighbours already updated in this sweep and the other two from before it.
// Any schedule that respects exactly those four dependencies gives the same
// result as the serial loop nest.  The schedule used here:
//
//  * the box is cut into 32-column blocks; warp w owns physical block w for the
//    whole run, lane l one column of it (lane order follows the sweep sign of
//    x, so lane 0 is the upwind side);
//  * at step s lane l updates logical row s - l: its left neighbour (new) comes
//    from lane l-1 by a register shuffle, its upper neighbour (new) is the
//    value it produced one step earlier, its right neighbour (old) is lane
//    l+1's prefetched lower neighbour, shuffled down;
//  * the block's rows stream through a 64-row shared-memory ring in chunks of
//    8 rows, copied from global memory by cp.async three chunks ahead and
//    written back as soon as all 32 lanes finished them;
//  * the block's last lane hands its new column to the next block's warp
//    through shared memory (published per chunk, tagged with the sweep); it
//    reads the next block's first column (old values) from global memory;
//  * per-node read-only data ("statics") are stored pre-skewed per sweep
//    direction ([dir][block][step][lane]) so a chunk of 8 steps is one
//    contiguous copy into a small shared ring;
//  * there is no CTA-wide barrier between sweeps: a warp starts sweep k+1 as
//    soon as its own block and the block whose old column it reads have
//    finished sweep k, so the pipeline reverses direction without draining
//    when the x sign flips.  A sweep that changes no node anywhere marks a
//    fixed point; the engine then stops (sweeps a warp had already begun
//    speculatively change nothing).
//
// Storage of the state u: strip-major [block][row][32] (row = physical y,
// 32 = physical x within the block), padded to a whole number of blocks;
// padding columns are never touched.  One-sided differences at the box edges
// come for free: missing neighbours are +inf.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace eik {

constexpr int CH = 8;             // rows (and steps) per chunk
constexpr int RROWS = 64;         // u ring rows per warp (power of two)
constexpr int SRCH = 3;           // statics chunks held in the statics ring
constexpr int LEAD = 3;           // u chunks copied ahead of the current one
constexpr int SWEEP_SHIFT = 13;   // hand-off progress tag: rows < 2^13, sweeps < 2^18
constexpr int MAX_BOX_ROWS = (1 << SWEEP_SHIFT) - 1;
constexpr long long MAX_SWEEPS = 1ll << 17;

__host__ __device__ inline int ceil32(int v) { return (v + 31) >> 5; }

// Element index of node (i, j) of a strip-major box of height my.
__host__ __device__ inline size_t box_index(int i, int j, int my) {
    return ((size_t)(i >> 5) * my + j) * 32 + (i & 31);
}

// Steps of one statics stream, padded to whole chunks plus the lead.
__host__ __device__ inline int nstep_padded(int ny) { return ((ny + 31 + CH - 1) / CH) * CH + 4 * CH; }

// Sweep direction d in [0, 4): bit 1 = sign of x, bit 0 = sign of y (set =
// +1).  The paper's loop nest (x sign outermost, -1 first) visits d = 0..3 in
// order, so sweep k uses d = k % 4.
__host__ __device__ inline int dir_sx(int d) { return (d & 2) ? 1 : -1; }
__host__ __device__ inline int dir_sy(int d) { return (d & 1) ? 1 : -1; }

// Index of node (i, j) of a box (width -> nb blocks, height my) in the skewed
// statics layout for direction d: [d][q][s][l], q = logical block, s = step,
// l = lane.
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

// Shared memory needed per CTA of `nw` warps (one warp per block).  With
// GLOBAL the hand-off columns and control words live in global memory.
template <class T, int NST, bool HASB, bool GLOBAL = false>
__host__ __device__ inline size_t engine_smem_bytes(int nw, int ny) {
    size_t per_warp = (size_t)RROWS * 32 * sizeof(T)                 // u ring
                      + (size_t)NST * SRCH * CH * 32 * sizeof(T)     // statics ring
                      + (size_t)RROWS * sizeof(T)                    // halo ring
                      + (GLOBAL ? 0 : (size_t)((ny + 3) & ~3) * sizeof(T))  // hand-off column
                      + (HASB ? (size_t)SRCH * CH * 32 : 0);         // byte statics ring
    return nw * per_warp + (GLOBAL ? 0 : (size_t)(32 + 2 * nw) * sizeof(int)) + 64;
}

// Control words of a multi-CTA engine run (global memory, zeroed by
// engine_global_init before the run): abort, stop_at, fin[8], chg[8], then
// prog[nb], done[nb].
__host__ __device__ inline size_t engine_global_ints(int nb) { return 32 + 2 * (size_t)nb; }

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Shared control words of one engine run.
struct EngineCtl {
    long long lim;  // polls a wait may make (read once when the run starts)
    int *prog;      // [nb] hand-off progress: (sweep << SWEEP_SHIFT) | rows published
    int *done;      // [nb] sweeps completed by the block (all rows written back)
    int *fin;       // [8] warps that finished sweep k (slot k & 7)
    int *chg;       // [8] any node changed in sweep k
    int *stop_at;   // first sweep that changed nothing (INT_MAX while unknown)
    int *abort_flag;
};

__device__ __forceinline__ int vload(const int *p) { return *(const volatile int *)p; }
__device__ __forceinline__ void vstore(int *p, int v) { *(volatile int *)p = v; }
template <bool GLOBAL>
__device__ __forceinline__ void fence() {
    if (GLOBAL) __threadfence();
    else __threadfence_block();
}

// Bounded wait until *p >= target.  Returns false if the engine is stopping
// (the last useful sweep is known to precede `sweep`) or on timeout.
__device__ __forceinline__ bool wait_ge(const int *p, int target, const EngineCtl &C, int sweep, int *err) {
    if (vload(p) >= target) return true;
    // the sleep doubles from 32 ns to 1 us: short waits wake quickly, long
    // ones leave the issue slots to the warps doing work
    long long it = 0;
    unsigned ns = 32;
    while (vload(p) < target) {
        if (vload(C.abort_flag) || vload(C.stop_at) < sweep) return false;
        if (++it > C.lim) {
            vstore(C.abort_flag, 1);
            atomicExch(err, DEV_TIMEOUT);
            return false;
        }
        __nanosleep(ns);
        ns = ns < 1024 ? 2 * ns : 1024;
    }
    return true;
}

// One sweep (number k, direction (SX, SY)) of physical block b by its warp.
// Returns -1 if the engine is stopping, else whether any node changed.
template <int SX, int SY, bool GLOBAL, class T, int NST, bool HASB, bool STEADY_PATH, class P>
__device__ int run_block(const Box<T, NST> &bx, const P &pol, int k, int b, T *ring, T *sring, uint8_t *sbring,
                         T *halo, T *hand, const T *hands, size_t hand_elems, const EngineCtl &C, int *err) {
    using N = Num<T>;
    constexpr int DIR = (SX > 0 ? 2 : 0) | (SY > 0 ? 1 : 0);
    const T INF = N::inf();
    const int lane = threadIdx.x & 31;
    const int NB = bx.nb, NY = bx.ny, NX = bx.nx;
    const int q = SX > 0 ? b : NB - 1 - b;         // logical block
    const int pc = SX > 0 ? lane : 31 - lane;       // physical column in the block
    const int x = 32 * b + pc;
    const bool colok = x < NX;
    const bool fullblk = 32 * b + 31 < NX;  // every lane of the block on a column
    const int bp = b - SX, bn = b + SX;              // physical predecessor / successor
    const bool has_prev = bp >= 0 && bp < NB;
    const bool has_next = bn >= 0 && bn < NB;
    const int pcn = SX > 0 ? 0 : 31;                 // successor's first logical column
    const bool nextok = has_next && (32 * bn + pcn) < NX;
    T *ublk = bx.u + (size_t)b * NY * 32;
    const T *unext = bx.u + (size_t)(has_next ? bn : b) * NY * 32;
    const T *hand_in = hands + (size_t)(has_prev ? bp : b) * hand_elems;
    const int nchunks = (NY + CH - 1) / CH;
    const int nsteps = NY + 31;
    const int tag = k << SWEEP_SHIFT;

    // Start condition: the successor block (whose old column this sweep reads)
    // has finished sweep k-1.  Our own block finished it in program order.
    if (k > 0 && has_next) {
        if (!wait_ge(C.done + bn, k, C, k, err)) return -1;
        fence<GLOBAL>();
    }

    auto prow = [&](int m) { return SY > 0 ? m : NY - 1 - m; };
    constexpr int EPL = 8;                                  // elements per lane per chunk
    constexpr int CPL = EPL * (int)sizeof(T) / 16;          // 16-byte copies per lane
    constexpr int E16 = 16 / (int)sizeof(T);                // elements per 16-byte copy
    const int r8 = lane >> 2, cg = lane & 3;
    auto issue_chunk = [&](int j) {                         // u rows of chunk j -> ring
        const int m = j * CH + r8;
        if (j < nchunks && m < NY) {
            const T *src = ublk + (size_t)prow(m) * 32 + cg * EPL;
            T *dst = ring + (m & (RROWS - 1)) * 32 + cg * EPL;
#pragma unroll
            for (int c = 0; c < CPL; ++c) cp_async16(dst + c * E16, src + c * E16);
        }
    };
    const size_t stbase = ((size_t)DIR * NB + q) * bx.nstepp;
    auto issue_statics = [&](int j) {                       // statics of steps 8j.. -> statics ring
        const int s0 = j * CH;
        if (s0 + CH > bx.nstepp) return;
        const int slot = j % SRCH;
#pragma unroll
        for (int kk = 0; kk < NST; ++kk) {
            const T *src = bx.st[kk] + (stbase + s0) * 32 + lane * EPL;
            T *dst = sring + ((size_t)kk * SRCH * CH + slot * CH) * 32 + lane * EPL;
#pragma unroll
            for (int c = 0; c < CPL; ++c) cp_async16(dst + c * E16, src + c * E16);
        }
        if (HASB && lane < 16) cp_async16(sbring + (slot * CH) * 32 + lane * 16, bx.sb + (stbase + s0) * 32 + lane * 16);
    };
    T hreg = INF;  // halo of one chunk (lanes 0..7), staged in a register
    auto load_halo = [&](int j) {
        const int mh = j * CH + lane;
        hreg = (lane < CH && nextok && j < nchunks && mh < NY) ? __ldcg(unext + (size_t)prow(mh) * 32 + pcn) : INF;
    };
    auto write_back = [&](int j) {
        const int m = j * CH + r8;
        if (m < NY) {
            const uint4 *src = reinterpret_cast<const uint4 *>(ring + (m & (RROWS - 1)) * 32 + cg * EPL);
            uint4 *dst = reinterpret_cast<uint4 *>(ublk + (size_t)prow(m) * 32 + cg * EPL);
#pragma unroll
            for (int c = 0; c < CPL; ++c) __stcg(dst + c, src[c]);
        }
    };

    // Prologue: u chunks 0..LEAD-1 and statics chunks 0..1 in flight (one
    // group per chunk), halo of chunk 0 in the ring, of chunk 1 in hreg.
    fence<GLOBAL>();
#pragma unroll
    for (int j = 0; j < LEAD; ++j) {
        issue_chunk(j);
        if (j < 2) issue_statics(j);
        cp_async_commit();
    }
    load_halo(0);
    if (lane < CH) halo[lane] = hreg;
    load_halo(1);

    T last = INF, cur = INF, dnx = INF, hal = INF;
    // hand-off values of the current chunk: lane i holds logical row s0 + i;
    // with GLOBAL the next chunk's values are fetched one boundary ahead
    T hcur = INF, hnext = INF;
    auto hand_row = [&](int m) -> T {
        return (lane < CH && m < NY) ? (GLOBAL ? __ldcg(hand_in + m) : hand_in[m]) : INF;
    };
    bool changed = false;
    const int lastJ = nchunks + 4;                 // boundary that writes back the last chunk
    const bool lane0 = lane == 0, lane31 = lane == 31;
    T *myring = ring + pc;
    int known = -1;
    if (GLOBAL && has_prev) {
        if (!wait_ge(C.prog + bp, tag | (CH > NY ? NY : CH), C, k, err)) {
            cp_async_wait<0>();
            return -1;
        }
        known = vload(C.prog + bp);
        fence<GLOBAL>();
        hnext = hand_row(lane);
    }
    auto ringval = [&](int m) -> T {
        return (colok && (unsigned)m < (unsigned)NY) ? myring[(m & (RROWS - 1)) * 32] : INF;
    };

    for (int J = 0; J <= lastJ; ++J) {
        __syncwarp();
        // chunk J-5 is complete: its last row 8J-33 was updated by lane 31 at step 8J-2
        if (J >= 5 && J - 5 < nchunks) write_back(J - 5);
        if (has_next && lane31) {
            int pub = CH * J - 31;  // rows whose hand-off values this lane has written
            pub = pub < 0 ? 0 : (pub > NY ? NY : pub);
            if (J == lastJ) pub = NY;
            fence<GLOBAL>();
            vstore(C.prog + b, tag | pub);
        }
        // halo of chunk J+1 into the ring, load halo of chunk J+2
        if (lane < CH) halo[((J + 1) * CH + lane) & (RROWS - 1)] = hreg;
        load_halo(J + 2);
        // copies for u chunk J+LEAD (into the slot of chunk J-5, written back
        // above) and statics chunk J+2 (slot of chunk J-1, used up)
        issue_chunk(J + LEAD);
        issue_statics(J + 2);
        cp_async_commit();
        // the group of boundary J-2 (u chunk J+1, statics chunk J) has landed
        cp_async_wait<2>();
        const int s0 = J * CH;
        if (s0 < nsteps && has_prev) {
            // rows this chunk needs (smem hand-off) or the next chunk needs
            // (global hand-off, fetched a boundary ahead)
            const int rows = GLOBAL ? s0 + 2 * CH : s0 + CH;
            const int need = tag | (rows > NY ? NY : rows);
            if (known < need) {
                if (!wait_ge(C.prog + bp, need, C, k, err)) {
                    cp_async_wait<0>();
                    return -1;
                }
                known = vload(C.prog + bp);
                fence<GLOBAL>();
            }
            if (GLOBAL) {
                hcur = hnext;
                hnext = hand_row(s0 + CH + lane);
            } else {
                hcur = hand_row(s0 + lane);
            }
        }
        __syncwarp();
        if ((J & 7) == 7 && (vload(C.abort_flag) || vload(C.stop_at) < k)) {
            cp_async_wait<0>();
            return -1;
        }
        if (s0 >= nsteps) continue;
        if (J == 0) {
            cur = ringval(-lane);
            dnx = ringval(1 - lane);
        }
        hal = halo[(s0 - lane) & (RROWS - 1)];
        const T *sbase = sring + (size_t)((J % SRCH) * CH) * 32 + lane;
        const uint8_t *bbase = sbring + ((J % SRCH) * CH) * 32 + lane;
        // The chunk's 8 steps.  STEADY: every lane of a full block is on a
        // valid row at every step and so is the row two ahead that it loads,
        // so the row and column tests are dropped (the same operations on the
        // same values otherwise).
        auto run_chunk = [&](auto steady_tag) {
            constexpr bool STEADY = decltype(steady_tag)::value;
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const int m = s0 + i - lane;
                const bool rowok = STEADY || (unsigned)m < (unsigned)NY;
                const bool act = STEADY || (colok && rowok);
                // loads for the next step, issued before this step's store
                const T dn2 = STEADY ? myring[((m + 2) & (RROWS - 1)) * 32] : ringval(m + 2);
                const T hal2 = halo[(m + 1) & (RROWS - 1)];
                T sv[NST > 0 ? NST : 1];
#pragma unroll
                for (int kk = 0; kk < NST; ++kk) sv[kk] = sbase[((size_t)kk * SRCH * CH + i) * 32];
                const uint8_t sbv = HASB ? bbase[i * 32] : (uint8_t)0;
                const T hin = __shfl_sync(FULL, hcur, i);
                const T fromleft = __shfl_up_sync(FULL, last, 1);
                const T fromright = __shfl_down_sync(FULL, dnx, 1);
                const T left = lane0 ? ((has_prev && rowok) ? hin : INF) : fromleft;
                const T right = lane31 ? ((nextok && rowok) ? hal : INF) : fromright;
                bool ch = false;
                const T upd = pol.update(cur, SX > 0 ? left : right, SX > 0 ? right : left, SY > 0 ? last : dnx,
                                         SY > 0 ? dnx : last, sv, sbv, ch);
                const T nw = act ? upd : INF;
                changed = changed || (act && ch);
                if (act) myring[(m & (RROWS - 1)) * 32] = nw;
                if (act && lane31 && has_next) hand[m] = nw;
                last = nw;
                cur = dnx;
                dnx = dn2;
                hal = hal2;
            }
        };
        if constexpr (STEADY_PATH) {
            if (fullblk && s0 >= 31 && s0 + CH + 1 < NY) run_chunk(std::true_type{});
            else run_chunk(std::false_type{});
        } else {
            run_chunk(std::false_type{});
        }
    }
    cp_async_wait<0>();
    fence<GLOBAL>();  // every lane's write-back before the block's completion flag
    __syncwarp();
    return __any_sync(FULL, changed) ? 1 : 0;
}

// Runs sweeps on one box until a sweep changes nothing or max_sweeps ran.
// Single-CTA form (GLOBAL = false): the CTA holds every block of the box,
// blockDim.x >= 32 * bx.nb, engine_smem_bytes<T, NST, HASB>(nb, ny) bytes of
// dynamic shared memory at `smem`.  Multi-CTA form (GLOBAL = true): CTA c
// owns blocks [c * nw, c * nw + nw) with nw = blockDim.x / 32, hand-off
// columns live in `ghands` ([nb][ny] elements) and the control words in
// `gctl` (engine_global_ints(nb) ints, zeroed before the launch); every CTA of
// the grid must be co-resident (cooperative launch).  All threads must call it.
template <class T, int NST, bool HASB, bool GLOBAL = false, bool STEADY_PATH = true, class P>
__device__ void engine_run(const Box<T, NST> &bx, const P &pol, long long max_sweeps, char *smem, long long &sweeps,
                           bool &converged, int *err, T *ghands = nullptr, int *gctl = nullptr, int cta = -1) {
    const int nwc = GLOBAL ? (int)(blockDim.x >> 5) : bx.nb;   // warps (blocks) of this CTA
    // multi-CTA form: this CTA's index among the CTAs of the box (blockIdx.x
    // unless several boxes share the grid)
    const int b0 = GLOBAL ? (cta >= 0 ? cta : (int)blockIdx.x) * nwc : 0;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const size_t ring_e = (size_t)RROWS * 32, sring_e = (size_t)NST * SRCH * CH * 32;
    const size_t halo_e = RROWS, hand_e = GLOBAL ? (size_t)bx.ny : (size_t)((bx.ny + 3) & ~3);
    const size_t sb_b = HASB ? (size_t)SRCH * CH * 32 : 0;
    T *base = reinterpret_cast<T *>(smem);
    T *ring = base + (size_t)warp * ring_e;
    T *sring = base + (size_t)nwc * ring_e + (size_t)warp * sring_e;
    T *halo = base + (size_t)nwc * (ring_e + sring_e) + (size_t)warp * halo_e;
    T *hands;
    uint8_t *bytes;
    if (GLOBAL) {
        hands = ghands;
        bytes = reinterpret_cast<uint8_t *>(base + (size_t)nwc * (ring_e + sring_e + halo_e));
    } else {
        hands = base + (size_t)nwc * (ring_e + sring_e + halo_e);
        bytes = reinterpret_cast<uint8_t *>(hands + (size_t)nwc * hand_e);
    }
    uint8_t *sbring = bytes + (size_t)warp * sb_b;
    int *ints = GLOBAL ? gctl : reinterpret_cast<int *>(bytes + (size_t)nwc * sb_b);
    EngineCtl C;
    C.lim = spin_limit();
    C.abort_flag = ints;
    C.stop_at = ints + 1;
    C.fin = ints + 8;
    C.chg = ints + 16;
    C.prog = ints + 32;
    C.done = ints + 32 + bx.nb;

    if (!GLOBAL) {
        if (threadIdx.x == 0) {
            C.abort_flag[0] = 0;
            C.stop_at[0] = 0x7fffffff;
        }
        if (threadIdx.x < 8) {
            C.fin[threadIdx.x] = 0;
            C.chg[threadIdx.x] = 0;
        }
        if ((int)threadIdx.x < bx.nb) {
            C.prog[threadIdx.x] = -1;
            C.done[threadIdx.x] = 0;
        }
    }
    __syncthreads();

    const int b = b0 + warp;
    if (warp < nwc && b < bx.nb) {
        T *hand = hands + (size_t)b * hand_e;
        for (long long kk = 0; kk < max_sweeps; ++kk) {
            const int k = (int)kk;
            if (vload(C.abort_flag) || vload(C.stop_at) < k) break;
            int ch;
            switch (k & 3) {
                case 0: ch = run_block<-1, -1, GLOBAL, T, NST, HASB, STEADY_PATH>(bx, pol, k, b, ring, sring, sbring, halo, hand, hands, hand_e, C, err); break;
                case 1: ch = run_block<-1, +1, GLOBAL, T, NST, HASB, STEADY_PATH>(bx, pol, k, b, ring, sring, sbring, halo, hand, hands, hand_e, C, err); break;
                case 2: ch = run_block<+1, -1, GLOBAL, T, NST, HASB, STEADY_PATH>(bx, pol, k, b, ring, sring, sbring, halo, hand, hands, hand_e, C, err); break;
                default: ch = run_block<+1, +1, GLOBAL, T, NST, HASB, STEADY_PATH>(bx, pol, k, b, ring, sring, sbring, halo, hand, hands, hand_e, C, err); break;
            }
            if (ch < 0) break;
            // sweep k of this block is complete: publish it, then the sweep status
            if (lane == 0) {
                fence<GLOBAL>();
                vstore(C.done + b, k + 1);
                if (ch) atomicOr(C.chg + (k & 7), 1);
                fence<GLOBAL>();
                const int f = atomicAdd(C.fin + (k & 7), 1);
                if (f == bx.nb - 1) {
                    if (vload(C.chg + (k & 7)) == 0) {
                        atomicMin(C.stop_at, k);
                    } else {
                        vstore(C.chg + (k & 7), 0);
                        vstore(C.fin + (k & 7), 0);
                    }
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();
    const int st = vload(C.stop_at);
    converged = st != 0x7fffffff && !vload(C.abort_flag);
    sweeps = st != 0x7fffffff ? (long long)st + 1 : max_sweeps;
    __syncthreads();
}

// Zeroes the control words of a multi-CTA engine run (one thread block).
__device__ inline void engine_global_init(int *gctl, int nb) {
    for (int i = threadIdx.x; i < (int)engine_global_ints(nb); i += blockDim.x) {
        int v = 0;
        if (i == 1) v = 0x7fffffff;
        if (i >= 32 && i < 32 + nb) v = -1;
        gctl[i] = v;
    }
}

}  // namespace eik

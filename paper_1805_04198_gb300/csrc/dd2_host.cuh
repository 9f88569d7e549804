// dd2_host.cuh -- host-side plan and workspace layout of one 2-D DD problem,
// shared by the single-problem and the batched solves.
#pragma once

#include "dd2_device.cuh"
#include "host_util.h"

#include <algorithm>

namespace eik {

struct DDPlan {
    DDGeom G;
    size_t bytes;
    size_t fine_smem, step1_smem, step4_smem;
    int grid_threads;
    bool adaptive;  // per-node weight: history of C_H and a fourth Alg. 5 static
};

// Checks a DD request (2-D or 3-D); sets the error text and returns false if
// it is invalid.
bool dd_validate(const eik_grid *grid, const eik_dd_params *p);

template <class T>
inline size_t dd_layout(const DDPlan &P, DDArgs<T> *A, void *ws, int max_iter) {
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
    int *ldirty = cv.take<int>((size_t)G.ncx + G.ncy + 2);
    T *sig_u = cv.take<T>(ntiles * tile_face_count(G));
    uint8_t *sig_w = cv.take<uint8_t>(ntiles * tile_face_count(G));
    int *sig_ok = cv.take<int>(ntiles);
    int *order = cv.take<int>(ntiles);
    int *order_cnt = cv.take<int>(2);
    unsigned *bar = cv.take<unsigned>(4);
    DevStats *st = cv.take<DevStats>(1);
    T *Ch[4] = {nullptr, nullptr, nullptr, nullptr};
    T *theta_sk = nullptr;
    if (P.adaptive) {
        for (int s = 0; s < 4; ++s) Ch[s] = cv.take<T>(G.coarse_elems);
        theta_sk = cv.take<T>(G.coarse_sk_elems);
    }
    if (A) {
        for (int s = 0; s < 4; ++s) A->Ch[s] = Ch[s];
        A->theta_sk = theta_sk;
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
        A->ldirty = ldirty;
        A->sig_u = sig_u;
        A->sig_w = sig_w;
        A->sig_ok = sig_ok;
        A->order = order;
        A->order_cnt = order_cnt;
        A->bar = bar;
        A->st = st;
    }
    return cv.used + 256;
}

// Launch shape of a cooperative causal-sweep kernel: lines staged in shared
// memory (one warp per line, up to 2 warps per CTA) when a line of lw nodes
// fits, else the in-place form with 8 warps per CTA.  blocks is capped by what
// is co-resident so that the grid barrier cannot wait on an unscheduled CTA.
struct CausalShape {
    int threads, blocks, lw;
    size_t smem;
};

template <class T>
inline int causal_shape(const void *kernel, int lw, int lines, int nsm, int smem_optin, CausalShape &cs) {
    const size_t wb = causal_warp_bytes<T>(lw);
    // two warps (lines) per CTA: the staged gathers of a line are many small
    // loads, so lines spread over more SMs finish sooner (8 per CTA on 33 SMs:
    // 7.8 ms of causal sweep on the 4097^2 solve; 2 per CTA on 129 SMs: 7.1 ms)
    int wpb = (int)std::min<size_t>(2, (size_t)std::max(0, smem_optin - 1024) / wb);
    if (wpb >= 1) {
        cs.threads = 32 * wpb;
        cs.smem = (size_t)wpb * wb;
        cs.lw = lw;
    } else {
        wpb = 8;
        cs.threads = 256;
        cs.smem = 0;
        cs.lw = 0;
    }
    int rc = cuda_check(set_dyn_smem(kernel, (int)cs.smem),
                        "smem attr causal");
    if (rc) return rc;
    int per_sm = 0;
    rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, cs.threads, cs.smem), "occupancy");
    if (rc) return rc;
    if (per_sm < 1) {
        set_error("causal sweep: no CTA of %d threads and %zu bytes fits on an SM", cs.threads, cs.smem);
        return EIK_EUNSUPPORTED;
    }
    cs.blocks = std::max(1, std::min(per_sm * nsm, (lines + wpb - 1) / wpb));
    return EIK_OK;
}

inline DDPlan dd_plan(const eik_grid *grid, const eik_dd_params *p) {
    DDPlan P;
    P.G = make_geom((int)grid->n[0], (int)grid->n[1], p->tiles[0], p->tiles[1], p->coarse_ratio, grid->h);
    P.step1_smem = P.step4_smem = 0;
    P.adaptive = p->theta_adaptive != 0;
    P.bytes = grid->dtype == EIK_F64 ? dd_layout<double>(P, nullptr, nullptr, p->max_iter)
                                     : dd_layout<float>(P, nullptr, nullptr, p->max_iter);
    const int gnb = ceil32(P.G.ncx + 1);
    P.grid_threads = 32 * gnb;
    if (grid->dtype == EIK_F64) {
        P.fine_smem = engine_smem_bytes<double, 1, false>(P.G.tnb, P.G.tny);
        P.step1_smem = engine_smem_bytes<double, 1, false>(gnb, P.G.ncy + 1);
        P.step4_smem = P.adaptive ? engine_smem_bytes<double, 4, true>(gnb, P.G.ncy + 1)
                                  : engine_smem_bytes<double, 3, true>(gnb, P.G.ncy + 1);
    } else {
        P.fine_smem = engine_smem_bytes<float, 1, false>(P.G.tnb, P.G.tny);
        P.step1_smem = engine_smem_bytes<float, 1, false>(gnb, P.G.ncy + 1);
        P.step4_smem = P.adaptive ? engine_smem_bytes<float, 4, true>(gnb, P.G.ncy + 1)
                                  : engine_smem_bytes<float, 3, true>(gnb, P.G.ncy + 1);
    }
    return P;
}

}  // namespace eik

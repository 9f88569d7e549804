// dd_geom.cuh -- index geometry of the two-scale decomposition (2-D).
//
// Fine grid: nx x ny nodes, spacing h.  Subdomains (Sec. 3.2, Omega^h_{i,j}):
// tx x ty tiles of Sx x Sy cells that share their boundary nodes.
// Coarse set: every fine node with x = 0 mod c or y = 0 mod c; it is the union
// of the shifted coarse grids Omega^H + (l h, 0) and Omega^H + (0, m h)
// (Sec. 3.2), each a full coarse grid of spacing H = c h:
//   grid 0              offset (0, 0)        (ncx+1) x (ncy+1) nodes
//   grid g in [1, c)    offset (g, 0)         ncx    x (ncy+1)
//   grid g in [c, 2c-1) offset (0, g-c+1)    (ncx+1) x  ncy
// Each grid is stored as one strip-major box ([block][row][32]) so that a
// coarse-grid sweep streams it like any other box.
#pragma once

#include "engine.cuh"

namespace eik {

struct DDGeom {
    int nx, ny;        // fine nodes per axis
    int tx, ty;        // subdomains per axis
    int sx, sy;        // cells per subdomain
    int c;             // coarse ratio
    int cshift;        // log2(c) when c is a power of two, else -1
    int ncx, ncy;      // (nx-1)/c, (ny-1)/c
    int ngrids;        // 2c - 1
    // tile boxes
    int tnx, tny, tnb, tnstepp;
    size_t tile_elems, tile_sk_elems;
    // grid families: element counts of one box and of its skewed statics
    size_t e0, eh, ev, k0, kh, kv;
    size_t coarse_elems, coarse_sk_elems;
    double h, H;
};

struct GridDesc {
    int ox, oy, mx, my, nb, nstepp;
    size_t off, skoff;
};

__host__ __device__ inline GridDesc grid_desc(const DDGeom &G, int g) {
    GridDesc d;
    if (g == 0) {
        d.ox = 0; d.oy = 0; d.mx = G.ncx + 1; d.my = G.ncy + 1;
        d.off = 0; d.skoff = 0;
    } else if (g < G.c) {
        d.ox = g; d.oy = 0; d.mx = G.ncx; d.my = G.ncy + 1;
        d.off = G.e0 + (size_t)(g - 1) * G.eh;
        d.skoff = G.k0 + (size_t)(g - 1) * G.kh;
    } else {
        d.ox = 0; d.oy = g - G.c + 1; d.mx = G.ncx + 1; d.my = G.ncy;
        d.off = G.e0 + (size_t)(G.c - 1) * G.eh + (size_t)(g - G.c) * G.ev;
        d.skoff = G.k0 + (size_t)(G.c - 1) * G.kh + (size_t)(g - G.c) * G.kv;
    }
    d.nb = ceil32(d.mx);
    d.nstepp = nstep_padded(d.my);
    return d;
}

__host__ inline DDGeom make_geom(int nx, int ny, int tx, int ty, int c, double h) {
    DDGeom G;
    G.nx = nx; G.ny = ny; G.tx = tx; G.ty = ty; G.c = c;
    G.cshift = -1;
    for (int sft = 0; sft < 31; ++sft)
        if ((1 << sft) == c) G.cshift = sft;
    G.sx = (nx - 1) / tx; G.sy = (ny - 1) / ty;
    G.ncx = (nx - 1) / c; G.ncy = (ny - 1) / c;
    G.ngrids = 2 * c - 1;
    G.tnx = G.sx + 1; G.tny = G.sy + 1;
    G.tnb = ceil32(G.tnx);
    G.tnstepp = nstep_padded(G.tny);
    G.tile_elems = (size_t)G.tnb * G.tny * 32;
    G.tile_sk_elems = (size_t)4 * G.tnb * G.tnstepp * 32;
    int mx0 = G.ncx + 1, my0 = G.ncy + 1;
    G.e0 = (size_t)ceil32(mx0) * my0 * 32;
    G.eh = (size_t)ceil32(G.ncx) * (G.ncy + 1) * 32;
    G.ev = (size_t)ceil32(G.ncx + 1) * G.ncy * 32;
    G.k0 = (size_t)4 * ceil32(mx0) * nstep_padded(my0) * 32;
    G.kh = (size_t)4 * ceil32(G.ncx) * nstep_padded(G.ncy + 1) * 32;
    G.kv = (size_t)4 * ceil32(G.ncx + 1) * nstep_padded(G.ncy) * 32;
    G.coarse_elems = G.e0 + (size_t)(c - 1) * (G.eh + G.ev);
    G.coarse_sk_elems = G.k0 + (size_t)(c - 1) * (G.kh + G.kv);
    G.h = h;
    G.H = (double)c * h;
    return G;
}

// Shifted grid and in-grid indices (i, j) of a coarse-set fine node (X, Y).
__host__ __device__ inline void coarse_locate(const DDGeom &G, int X, int Y, int &g, int &i, int &j) {
    const bool p2 = G.cshift >= 0;
    const int rx = p2 ? (X & (G.c - 1)) : X % G.c, ry = p2 ? (Y & (G.c - 1)) : Y % G.c;
    if (rx == 0 && ry == 0) {
        g = 0;
    } else if (ry == 0) {
        g = rx;
    } else {
        g = G.c - 1 + ry;
    }
    i = p2 ? X >> G.cshift : X / G.c;
    j = p2 ? Y >> G.cshift : Y / G.c;
}

__host__ __device__ inline size_t coarse_addr(const DDGeom &G, int X, int Y) {
    int g, i, j;
    coarse_locate(G, X, Y, g, i, j);
    GridDesc d = grid_desc(G, g);
    return d.off + box_index(i, j, d.my);
}

__host__ __device__ inline bool in_coarse_set(const DDGeom &G, int X, int Y) {
    if (G.cshift >= 0) return ((X & (G.c - 1)) == 0) || ((Y & (G.c - 1)) == 0);
    return (X % G.c == 0) || (Y % G.c == 0);
}

// Inverse of the coarse layout: element index -> (grid, i, j); false for padding.
__host__ __device__ inline bool coarse_decode(const DDGeom &G, size_t a, int &g, int &i, int &j) {
    size_t rel;
    if (a < G.e0) {
        g = 0;
        rel = a;
    } else if (a < G.e0 + (size_t)(G.c - 1) * G.eh) {
        size_t t = a - G.e0;
        g = 1 + (int)(t / G.eh);
        rel = t % G.eh;
    } else {
        size_t t = a - G.e0 - (size_t)(G.c - 1) * G.eh;
        g = G.c + (int)(t / G.ev);
        rel = t % G.ev;
    }
    GridDesc d = grid_desc(G, g);
    size_t per_block = (size_t)d.my * 32;
    int b = (int)(rel / per_block);
    size_t r2 = rel % per_block;
    j = (int)(r2 / 32);
    i = 32 * b + (int)(r2 % 32);
    return i < d.mx;
}

}  // namespace eik

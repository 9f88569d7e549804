/*
 * eik_oracle.c -- serial FP64 oracle for arXiv:1805.04198 (Martin & Tsai).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of bench.py; never by the product path.  Plain loops, no
 * blocking, no fusion: each routine follows the paper's steps in the paper's
 * order so it can be checked against the text by eye.  Build with
 * -ffp-contract=off so no multiply-add is fused (the arithmetic below is the
 * arithmetic the results are defined by).
 *
 * Readings of the paper taken here (each also listed in the design doc):
 *  - wind signs: direction of travel everywhere (+1 when the upwind, smaller
 *    neighbour is on the minus side); Alg. 1, 2, 4 and Step 2 are consistent
 *    only under this sign, so Alg. 3's printed signs are read as flipped;
 *  - Alg. 1 uses Alg. 3's branch test |a-b| < r h;
 *  - the wind of an FSM solve is the wind of the local solve at the converged
 *    state (path-independent; equal to the last stored wind except at exact
 *    neighbour ties);
 *  - an FSM (fine or coarse) stops after the first sweep that changes nothing;
 *  - Steps 2-3: a subdomain boundary node starts at U when W.n > 0 for some
 *    inward normal n of the subdomain (inflow), otherwise at +inf; every
 *    boundary node is then swept like an interior one, with one-sided
 *    differences (Step 3), so an inflow value can only decrease; only Gamma
 *    stays fixed (at g).  The wind of an inflow node whose value never moved
 *    is W, otherwise that of its local solve;
 *  - Alg. 4 / Alg. 5 at a node lying on several coarse lines (or interfaces):
 *    the agreement test is applied per axis and must pass on every axis;
 *  - Alg. 4's minimum is taken over the fine solutions: a copy from a
 *    subdomain for which the node was inflow and whose solve kept the Step 2
 *    value U (an echo of the boundary data, not a solution) is not a
 *    candidate unless every copy is one;
 *  - Alg. 5 keeps the paper's overwrite update, evaluated as
 *    u^k + theta (U~ - C_H(U^k)); when U~ or C_H(U^k) is +inf it takes u^k;
 *  - causal sweep (Alg. 2): repeated until nothing changes (its least fixed
 *    point); a node is never raised to an unreached (+inf) neighbour.
 */
#include "eik_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define INF HUGE_VAL

/* ------------------------------------------------------------------------- */
/* Local solver: Sec. 1.1 eq. (godonuv); 2-D closed form of Sec. 3.2 (C_H) and  */
/* Alg. 3; 3-D by the sorted-minima cascade (the paper says the 2-D method      */
/* "can be generalized"; the 3-D Godunov solve is the standard one of its       */
/* FSM reference).                                                              */
/* ------------------------------------------------------------------------- */
double orc_local_solve(int d, const double *vm, const double *vp, double rh, signed char *w)
{
    double a[3];
    int s[3];
    int k;
    for (k = 0; k < d; ++k) {
        /* Alg. 3: take the smaller neighbour along each axis; a tie goes to the
         * plus-side neighbour.  Sign = direction of travel. */
        if (vm[k] < vp[k]) {
            a[k] = vm[k];
            s[k] = +1;
        } else {
            a[k] = vp[k];
            s[k] = -1;
        }
        w[k] = 0;
    }
    if (d == 1) {
        double u = a[0] + rh;
        if (u < INF) w[0] = (signed char)s[0];
        return u;
    }
    if (d == 2) {
        double u;
        if (fabs(a[0] - a[1]) < rh) {
            double t = a[0] - a[1];
            u = (a[0] + a[1] + sqrt(2.0 * rh * rh - t * t)) * 0.5;
            w[0] = (signed char)s[0];
            w[1] = (signed char)s[1];
        } else {
            if (a[0] < a[1]) {
                u = a[0] + rh;
                if (u < INF) w[0] = (signed char)s[0];
            } else {
                u = a[1] + rh;
                if (u < INF) w[1] = (signed char)s[1];
            }
        }
        return u;
    }
    /* d == 3: order the axis minima p0 <= p1 <= p2 (ties keep axis order). */
    {
        int p[3] = {0, 1, 2};
        int i, j;
        double u;
        for (i = 1; i < 3; ++i)
            for (j = i; j > 0 && a[p[j]] < a[p[j - 1]]; --j) {
                int t = p[j];
                p[j] = p[j - 1];
                p[j - 1] = t;
            }
        if (fabs(a[p[0]] - a[p[1]]) < rh) {
            double t = a[p[0]] - a[p[1]];
            u = (a[p[0]] + a[p[1]] + sqrt(2.0 * rh * rh - t * t)) * 0.5;
            if (u > a[p[2]]) {
                /* three-term quadratic in t = u - a_p0:
                 *   t^2 + (t - d1)^2 + (t - d2)^2 = (r h)^2 */
                double d1 = a[p[1]] - a[p[0]];
                double d2 = a[p[2]] - a[p[0]];
                double sd = d1 + d2;
                double disc = sd * sd - 3.0 * (d1 * d1 + d2 * d2 - rh * rh);
                if (disc < 0.0) disc = 0.0;
                u = a[p[0]] + (sd + sqrt(disc)) / 3.0;
                w[0] = (signed char)s[0];
                w[1] = (signed char)s[1];
                w[2] = (signed char)s[2];
            } else {
                w[p[0]] = (signed char)s[p[0]];
                w[p[1]] = (signed char)s[p[1]];
            }
        } else {
            u = a[p[0]] + rh;
            if (u < INF) w[p[0]] = (signed char)s[p[0]];
        }
        return u;
    }
}

/* ------------------------------------------------------------------------- */
/* A "local grid": a dense box of m[0] x m[1] x m[2] nodes, spacing hs.         */
/* Used for whole grids, for subdomains (Step 3) and for shifted coarse grids  */
/* (Steps 1 and 4), after gathering their values into a dense local array.     */
/* ------------------------------------------------------------------------- */
static long lidx(const long *m, long x, long y, long z) { return x + m[0] * (y + m[1] * z); }

static void nbrs(int d, const long *m, const double *u, long x, long y, long z, double *vm, double *vp)
{
    long c[3] = {x, y, z};
    long st[3] = {1, m[0], m[0] * m[1]};
    long i = lidx(m, x, y, z);
    int k;
    for (k = 0; k < d; ++k) {
        vm[k] = (c[k] > 0) ? u[i - st[k]] : INF;
        vp[k] = (c[k] < m[k] - 1) ? u[i + st[k]] : INF;
    }
}

/* The 2^d sweep orderings of Sec. 1.1 in the printed loop order: the sign of
 * axis 0 is the outermost loop, -1 before +1; within a sweep axis 0 is the
 * outermost node loop.  sgn[k] receives the sign of axis k for ordering q. */
static void ordering(int d, int q, int *sgn)
{
    int k;
    for (k = 0; k < 3; ++k) sgn[k] = 1;
    for (k = 0; k < d; ++k) sgn[k] = ((q >> (d - 1 - k)) & 1) ? +1 : -1;
}

static long start_of(long mm, int s) { return s > 0 ? 0 : mm - 1; }

/* One Gauss-Seidel FSM sweep (Sec. 1.1 update u = min(u, u~)). */
static int fsm_sweep(int d, const long *m, double hs, const double *r, const unsigned char *fixed,
                     double *u, int q)
{
    int sg[3];
    long x, y, z;
    int changed = 0;
    ordering(d, q, sg);
    for (x = start_of(m[0], sg[0]); x >= 0 && x < m[0]; x += sg[0])
        for (y = start_of(m[1], sg[1]); y >= 0 && y < m[1]; y += sg[1])
            for (z = start_of(m[2], sg[2]); z >= 0 && z < m[2]; z += sg[2]) {
                long i = lidx(m, x, y, z);
                double vm[3], vp[3], ut;
                signed char w[3];
                if (fixed[i]) continue;
                nbrs(d, m, u, x, y, z, vm, vp);
                ut = orc_local_solve(d, vm, vp, r[i] * hs, w);
                if (ut < u[i]) {
                    u[i] = ut;
                    changed = 1;
                }
            }
    return changed;
}

/* FSM on a local grid: sweeps cycle through the orderings until one sweep
 * changes nothing (a fixed point) or max_sweeps ran.  Returns sweeps done. */
static long fsm_local(int d, const long *m, double hs, const double *r, const unsigned char *fixed,
                      double *u, long max_sweeps, int *converged)
{
    long s = 0;
    int nq = 1 << d;
    *converged = 0;
    while (s < max_sweeps) {
        int ch = fsm_sweep(d, m, hs, r, fixed, u, (int)(s % nq));
        ++s;
        if (!ch) {
            *converged = 1;
            break;
        }
    }
    return s;
}

/* Wind of the local solve at the current state (Alg. 1 / Alg. 3). */
static void winds_local(int d, const long *m, double hs, const double *r, const unsigned char *fixed,
                        const double *u, signed char *w)
{
    long x, y, z;
    for (z = 0; z < m[2]; ++z)
        for (y = 0; y < m[1]; ++y)
            for (x = 0; x < m[0]; ++x) {
                long i = lidx(m, x, y, z);
                double vm[3], vp[3];
                signed char wt[3] = {0, 0, 0};
                int k;
                if (!fixed[i] && u[i] < INF) {
                    nbrs(d, m, u, x, y, z, vm, vp);
                    (void)orc_local_solve(d, vm, vp, r[i] * hs, wt);
                }
                if (!fixed[i])
                    for (k = 0; k < 3; ++k) w[3 * i + k] = (k < d) ? wt[k] : 0;
            }
}

long orc_fsm(int d, const long *n, double h, const double *r, const unsigned char *gamma,
             const double *g, double *u, signed char *w, long max_sweeps, int *converged)
{
    long m[3] = {n[0], d > 1 ? n[1] : 1, d > 2 ? n[2] : 1};
    long N = m[0] * m[1] * m[2], i, s;
    /* Sec. 1.1 initialisation: Gamma fixed at g, every other node large. */
    for (i = 0; i < N; ++i) u[i] = gamma[i] ? g[i] : INF;
    s = fsm_local(d, m, h, r, gamma, u, max_sweeps, converged);
    if (w) {
        for (i = 0; i < 3 * N; ++i) w[i] = 0;
        winds_local(d, m, h, r, gamma, u, w);
    }
    return s;
}

/* ------------------------------------------------------------------------- */
/* Dijkstra / FMM on the same local solver (binary heap, lazy deletion).        */
/* ------------------------------------------------------------------------- */
typedef struct { double v; long i; } hent;

static void hpush(hent *h, long *hn, double v, long i)
{
    long k = (*hn)++;
    h[k].v = v;
    h[k].i = i;
    while (k > 0) {
        long p = (k - 1) / 2;
        if (h[p].v <= h[k].v) break;
        hent t = h[p];
        h[p] = h[k];
        h[k] = t;
        k = p;
    }
}

static hent hpop(hent *h, long *hn)
{
    hent top = h[0];
    long k = 0;
    h[0] = h[--(*hn)];
    for (;;) {
        long l = 2 * k + 1, rr = l + 1, b = k;
        if (l < *hn && h[l].v < h[b].v) b = l;
        if (rr < *hn && h[rr].v < h[b].v) b = rr;
        if (b == k) break;
        hent t = h[b];
        h[b] = h[k];
        h[k] = t;
        k = b;
    }
    return top;
}

void orc_fmm(int d, const long *n, double h, const double *r, const unsigned char *gamma,
             const double *g, double *u)
{
    long m[3] = {n[0], d > 1 ? n[1] : 1, d > 2 ? n[2] : 1};
    long N = m[0] * m[1] * m[2], i;
    long st[3] = {1, m[0], m[0] * m[1]};
    unsigned char *acc = calloc((size_t)N, 1);
    double *ua = malloc(sizeof(double) * (size_t)N); /* accepted values, +inf otherwise */
    hent *hp = malloc(sizeof(hent) * (size_t)(N * 2 * d + N + 1));
    long hn = 0;
    for (i = 0; i < N; ++i) {
        ua[i] = INF;
        u[i] = INF;
        if (gamma[i]) {
            u[i] = g[i];
            hpush(hp, &hn, g[i], i);
        }
    }
    while (hn > 0) {
        hent e = hpop(hp, &hn);
        long c[3], k;
        if (acc[e.i] || e.v != u[e.i]) continue;
        acc[e.i] = 1;
        ua[e.i] = u[e.i];
        c[0] = e.i % m[0];
        c[1] = (e.i / m[0]) % m[1];
        c[2] = e.i / (m[0] * m[1]);
        for (k = 0; k < d; ++k) {
            int sd;
            for (sd = -1; sd <= 1; sd += 2) {
                long cc[3] = {c[0], c[1], c[2]};
                long j;
                double vm[3], vp[3], ut;
                signed char w[3];
                cc[k] += sd;
                if (cc[k] < 0 || cc[k] >= m[k]) continue;
                j = e.i + sd * st[k];
                if (acc[j] || gamma[j]) continue;
                /* tentative value from accepted neighbours only */
                nbrs(d, m, ua, cc[0], cc[1], cc[2], vm, vp);
                ut = orc_local_solve(d, vm, vp, r[j] * h, w);
                if (ut < u[j]) {
                    u[j] = ut;
                    hpush(hp, &hn, ut, j);
                }
            }
        }
    }
    free(acc);
    free(ua);
    free(hp);
}

/* ------------------------------------------------------------------------- */
/* Two-scale DD, Sec. 3.2.                                                      */
/* ------------------------------------------------------------------------- */
typedef struct {
    int d;
    long n[3], N;
    long st[3];
    long S[3];
    int T[3];
    int c;
} geom_t;

static void coords(const geom_t *G, long i, long *x)
{
    x[0] = i % G->n[0];
    x[1] = (i / G->n[0]) % G->n[1];
    x[2] = i / (G->n[0] * G->n[1]);
}

/* Axes along which node x lies on a coarse line (index = 0 mod c). */
static int coarse_axes(const geom_t *G, const long *x)
{
    int k, A = 0;
    for (k = 0; k < G->d; ++k)
        if (x[k] % G->c == 0) A |= 1 << k;
    return A;
}

/* The shifted coarse grid holding node x: offset o = x mod c, spacing c
 * (Sec. 3.2: Omega^H + (l h, 0), Omega^H + (0, m h), and their 3-D analogues).
 * Its dense box has m[k] = (n[k]-1-o[k])/c + 1 nodes per axis. */
static void grid_box(const geom_t *G, const long *o, long *m)
{
    int k;
    for (k = 0; k < 3; ++k) m[k] = (k < G->d) ? (G->n[k] - 1 - o[k]) / G->c + 1 : 1;
}

static long grid_fine(const geom_t *G, const long *o, long x, long y, long z)
{
    long c = G->c;
    long xx = o[0] + c * x, yy = (G->d > 1) ? o[1] + c * y : 0, zz = (G->d > 2) ? o[2] + c * z : 0;
    return xx + G->n[0] * (yy + G->n[1] * zz);
}

/* Enumerate every shifted coarse grid: offsets with at least one zero. */
static int next_offset(const geom_t *G, long *o, int first)
{
    for (;;) {
        int k;
        if (first) {
            o[0] = o[1] = o[2] = 0;
            first = 0;
        } else {
            for (k = 0; k < G->d; ++k) {
                if (++o[k] < G->c) break;
                o[k] = 0;
            }
            if (k == G->d) return 0;
        }
        for (k = 0; k < G->d; ++k)
            if (o[k] == 0) return 1;
    }
}

/* Causal sweep, Alg. 2, generalised per axis: along every axis e such that the
 * fine neighbour x +- e_e is also on the coarse set, a node whose wind points
 * along -e (upwind at +e) is raised to that neighbour if smaller, and the
 * mirror case.  Passes in the 2^d orderings are repeated until nothing
 * changes.  Returns the number of rounds. */
static long causal_sweep(const geom_t *G, double *U, const signed char *W)
{
    long rounds = 0;
    int changed;
    do {
        int q;
        changed = 0;
        ++rounds;
        for (q = 0; q < (1 << G->d); ++q) {
            int sg[3];
            long x[3];
            ordering(G->d, q, sg);
            for (x[0] = start_of(G->n[0], sg[0]); x[0] >= 0 && x[0] < G->n[0]; x[0] += sg[0])
                for (x[1] = start_of(G->n[1], sg[1]); x[1] >= 0 && x[1] < G->n[1]; x[1] += sg[1])
                    for (x[2] = start_of(G->n[2], sg[2]); x[2] >= 0 && x[2] < G->n[2]; x[2] += sg[2]) {
                        int A = coarse_axes(G, x), e;
                        long i = x[0] + G->n[0] * (x[1] + G->n[1] * x[2]);
                        if (!A) continue;
                        for (e = 0; e < G->d; ++e) {
                            if ((A & ~(1 << e)) == 0) continue;
                            if (W[3 * i + e] < 0 && x[e] + 1 < G->n[e]) {
                                double v = U[i + G->st[e]];
                                if (v < INF && U[i] < v) {
                                    U[i] = v;
                                    changed = 1;
                                }
                            }
                            if (W[3 * i + e] > 0 && x[e] > 0) {
                                double v = U[i - G->st[e]];
                                if (v < INF && U[i] < v) {
                                    U[i] = v;
                                    changed = 1;
                                }
                            }
                        }
                    }
        }
    } while (changed);
    return rounds;
}

/* Scatter of one shifted coarse grid's dense local box back to fine indexing. */
static void grid_scatter_d(const geom_t *G, const long *o, const long *m, const double *src, double *dst)
{
    long x, y, z;
    for (z = 0; z < m[2]; ++z)
        for (y = 0; y < m[1]; ++y)
            for (x = 0; x < m[0]; ++x) dst[grid_fine(G, o, x, y, z)] = src[lidx(m, x, y, z)];
}

/* Step 1 on one shifted grid: FSM with Alg. 1 (spacing H), Gamma fixed at g.
 * Writes U and W on the grid's nodes. */
static long step1_grid(const geom_t *G, const long *o, double H, const double *r, const unsigned char *gamma,
                       const double *g, double *U, signed char *W, long max_sweeps, long *caps)
{
    long m[3], M, i, s, x, y, z;
    double *ul, *rl;
    unsigned char *fl;
    signed char *wl;
    int conv;
    grid_box(G, o, m);
    M = m[0] * m[1] * m[2];
    ul = malloc(sizeof(double) * (size_t)M);
    rl = malloc(sizeof(double) * (size_t)M);
    fl = malloc((size_t)M);
    wl = calloc((size_t)(3 * M), 1);
    for (z = 0; z < m[2]; ++z)
        for (y = 0; y < m[1]; ++y)
            for (x = 0; x < m[0]; ++x) {
                long f = grid_fine(G, o, x, y, z), l = lidx(m, x, y, z);
                rl[l] = r[f];
                fl[l] = gamma[f] ? 1 : 0;
                ul[l] = gamma[f] ? g[f] : INF; /* Sec. 1.1 initialisation */
            }
    s = fsm_local(G->d, m, H, rl, fl, ul, max_sweeps, &conv);
    if (!conv) ++*caps;
    winds_local(G->d, m, H, rl, fl, ul, wl);
    for (z = 0; z < m[2]; ++z)
        for (y = 0; y < m[1]; ++y)
            for (x = 0; x < m[0]; ++x) {
                long f = grid_fine(G, o, x, y, z), l = lidx(m, x, y, z);
                U[f] = ul[l];
                for (i = 0; i < 3; ++i) W[3 * f + i] = wl[3 * l + i];
            }
    free(ul);
    free(rl);
    free(fl);
    free(wl);
    return s;
}

/* Decision margins of Alg. 1 at the nodes of one shifted grid, at its
 * converged Step 1 values (test infrastructure, no part of the method): per
 * node the smallest of |vm - vp| on each axis (which neighbour an axis takes),
 * | |a0 - a1| - rH | (two-axis or one-axis branch) and |a0 - a1| (the axis of
 * the one-axis branch), over the pairs of the 2-D local solve; +inf where a
 * compared pair holds an infinite value.  A wind whose margin is below the
 * error of a lower-precision evaluation of U may come out otherwise there. */
static void step1_margins(const geom_t *G, const long *o, double H, const double *r, const unsigned char *gamma,
                          const double *U, double *margin)
{
    long m[3], M, x, y, z;
    double *ul;
    grid_box(G, o, m);
    M = m[0] * m[1] * m[2];
    ul = malloc(sizeof(double) * (size_t)M);
    for (z = 0; z < m[2]; ++z)
        for (y = 0; y < m[1]; ++y)
            for (x = 0; x < m[0]; ++x) ul[lidx(m, x, y, z)] = U[grid_fine(G, o, x, y, z)];
    for (z = 0; z < m[2]; ++z)
        for (y = 0; y < m[1]; ++y)
            for (x = 0; x < m[0]; ++x) {
                long f = grid_fine(G, o, x, y, z), l = lidx(m, x, y, z);
                double vm[3], vp[3], a[3], mg = INF, rH = r[f] * H;
                int k, j;
                if (gamma[f] || !(ul[l] < INF)) {
                    margin[f] = INF;
                    continue;
                }
                nbrs(G->d, m, ul, x, y, z, vm, vp);
                for (k = 0; k < G->d; ++k) {
                    double dv = fabs(vm[k] - vp[k]);
                    if (dv < mg) mg = dv;
                    a[k] = vm[k] < vp[k] ? vm[k] : vp[k];
                }
                for (k = 0; k < G->d; ++k)
                    for (j = k + 1; j < G->d; ++j) {
                        double t = fabs(a[k] - a[j]);
                        if (t < mg) mg = t;
                        if (fabs(t - rH) < mg) mg = fabs(t - rH);
                    }
                margin[f] = mg;
            }
    free(ul);
}

/* Per-node weight of Sec. 4.2.  The bound M-bar of Theorem 2 is estimated by
 * eq. secthetaest: the last change of the fine values over a weighted mean of
 * the last changes of the coarse solver,
 *   theta-bar = (u^k - u^{k-1}) / [sum_s w_s (C^{k-s} - C^{k-1-s}) / sum_s w_s],
 * C^m = C_H(nbrs^H(U^m)), over the terms s = 0, 1, 2 whose iterates exist
 * (reading: the lag of the first estimate, eq. firstthetaest, for every term),
 * then damped by eq. thetaest: [sig t + (1 - sig) delta t]^+ with
 * sig = 1 / (1 + exp((t - x0) / gamma)).  Undefined estimates (no history,
 * zero or non-finite quotient) take the constant theta. */
typedef struct {
    const orc_dd_params *p;
    int nhist;               /* coarse-solver values available before this update */
    const double *C1, *C2, *C3;  /* C^{k-1}, C^{k-2}, C^{k-3} (full grid) */
    const double *uprev;     /* u^{k-1} */
} theta_ctx;

/* The estimate itself: du = u^k - u^{k-1}, dC[s] = C^{k-s} - C^{k-1-s} for the
 * n available terms.  Returns `fallback` where the estimate is undefined. */
double orc_theta_estimate(const orc_dd_params *p, double du, const double *dC, int n, double fallback)
{
    double den = 0.0, wsum = 0.0, t, sig, v;
    int s;
    for (s = 0; s < n && s < 3; ++s) {
        den += p->omega[s] * dC[s];
        wsum += p->omega[s];
    }
    if (!(wsum > 0.0)) return fallback;
    den = den / wsum;
    t = du / den;
    if (!isfinite(t) || den == 0.0) return fallback;
    sig = 1.0 / (1.0 + exp((t - p->sig_x0) / p->sig_gamma));
    v = sig * t + (1.0 - sig) * p->sig_delta * t;
    if (p->theta_cap > 0.0 && v > p->theta_cap) v = p->theta_cap;
    return v > 0.0 ? v : 0.0;
}

/* The weight of one node from its history: Ck = C^k, C1..C3 = C^{k-1..k-3}
 * (only the first nhist are read), uk = u^k, uprev = u^{k-1}.  The s-th term
 * of the mean is C^{k-s} - C^{k-1-s}. */
double orc_theta_node(const orc_dd_params *p, int nhist, double Ck, double C1, double C2, double C3, double uk,
                      double uprev)
{
    double Cs[4], dC[3];
    int s, n;
    if (!p->theta_adaptive || nhist < 1) return p->theta;
    Cs[0] = Ck;
    Cs[1] = C1;
    Cs[2] = C2;
    Cs[3] = C3;
    n = nhist < 3 ? nhist : 3;
    for (s = 0; s < n; ++s) dC[s] = Cs[s] - Cs[s + 1];
    return orc_theta_estimate(p, uk - uprev, dC, n, p->theta);
}

static double theta_node(const theta_ctx *T, long f, double uk_f, double Ck_f)
{
    if (!T->p->theta_adaptive || T->nhist < 1) return T->p->theta;
    return orc_theta_node(T->p, T->nhist, Ck_f, T->C1[f], T->nhist > 1 ? T->C2[f] : 0.0,
                          T->nhist > 2 ? T->C3[f] : 0.0, uk_f, T->uprev[f]);
}

/* C_H(nbrs^H(U^k)) at every node of a box (Sec. 3.2, the coarse solver
 * applied to the previous iterate; Step 4's last term). */
static void coarse_solver_prev(int d, const long *m, double H, const double *r, const double *Uk, double *Cold)
{
    long x, y, z;
    for (z = 0; z < m[2]; ++z)
        for (y = 0; y < m[1]; ++y)
            for (x = 0; x < m[0]; ++x) {
                long l = lidx(m, x, y, z);
                double vm[3], vp[3];
                signed char w[3];
                nbrs(d, m, Uk, x, y, z, vm, vp);
                Cold[l] = orc_local_solve(d, vm, vp, r[l] * H, w);
            }
}

/* Alg. 5 sweeps on one box (the U update of Step 4, Sec. 3.2).  U is
 * initialised as in Sec. 1.1 (fixed nodes at g, the rest +inf) and swept in
 * the 2^d orderings; at a free node with U~, W~ from the current neighbours
 * (Alg. 1), the weighted update u^k + theta (U~ - C_H(U^k)) is taken when on
 * every coarse-line axis of the node (bit k of axes) w^k, W^k and W~ all point
 * the same way or are zero, otherwise u^k.  Stops after a sweep that changes
 * nothing or max_sweeps sweeps (*capped = 1). */
static long alg5_sweeps(int d, const long *m, double H, const double *r, const unsigned char *fixed,
                        const double *g, const double *uk, const signed char *wk, const signed char *Wk,
                        const int *axes, const double *Cold, const double *theta, long max_sweeps, double *U,
                        int *capped)
{
    long s = 0, x, y, z, M = m[0] * m[1] * m[2], l;
    int nq = 1 << d;
    *capped = 0;
    /* "Initialize U as described in Sec. 1.1" */
    for (l = 0; l < M; ++l) U[l] = fixed[l] ? g[l] : INF;
    for (;;) {
        int changed = 0, sg[3];
        if (s >= max_sweeps) {
            *capped = 1;
            break;
        }
        ordering(d, (int)(s % nq), sg);
        for (x = start_of(m[0], sg[0]); x >= 0 && x < m[0]; x += sg[0])
            for (y = start_of(m[1], sg[1]); y >= 0 && y < m[1]; y += sg[1])
                for (z = start_of(m[2], sg[2]); z >= 0 && z < m[2]; z += sg[2]) {
                    double vm[3], vp[3], Ut, Unew;
                    signed char Wt[3];
                    int pass, k;
                    l = lidx(m, x, y, z);
                    if (fixed[l]) continue;
                    nbrs(d, m, U, x, y, z, vm, vp);
                    Ut = orc_local_solve(d, vm, vp, r[l] * H, Wt);
                    /* Alg. 5 agreement test, per coarse-line axis: the fine wind
                     * w^k, the coarse wind W^k and the current wind W~ all point
                     * the same way (or are zero) along that axis. */
                    pass = (Ut < INF) && (Cold[l] < INF);
                    for (k = 0; k < d && pass; ++k) {
                        int a = wk[3 * l + k], b = Wk[3 * l + k], c = Wt[k];
                        if (!(axes[l] & (1 << k))) continue;
                        if (!((a <= 0 && b <= 0 && c <= 0) || (a >= 0 && b >= 0 && c >= 0))) pass = 0;
                    }
                    if (pass)
                        Unew = uk[l] + theta[l] * (Ut - Cold[l]);
                    else
                        Unew = uk[l];
                    if (!(Unew == U[l])) changed = 1;
                    U[l] = Unew;
                }
        ++s;
        if (!changed) break;
    }
    return s;
}

long orc_step4_box(int d, const long *n, double H, const double *r, const unsigned char *fixed, const double *g,
                   const double *Uk, const double *uk, const signed char *wk, const signed char *Wk,
                   const int *axes, const double *theta, long max_sweeps, double *U, double *Cold, int *capped)
{
    long m[3] = {n[0], d > 1 ? n[1] : 1, d > 2 ? n[2] : 1};
    long M = m[0] * m[1] * m[2];
    double *C = Cold ? Cold : malloc(sizeof(double) * (size_t)M);
    long s;
    coarse_solver_prev(d, m, H, r, Uk, C);
    s = alg5_sweeps(d, m, H, r, fixed, g, uk, wk, Wk, axes, C, theta, max_sweeps, U, capped);
    if (!Cold) free(C);
    return s;
}

/* Step 4 on one shifted grid: gathers the grid's nodes into a dense box and
 * runs Alg. 5 there.  Uk = U^k (for C_H(nbrs U^k)), uk/wk the Alg. 4 output,
 * Wk = W^k.  Writes the swept U (W is set to w^k by the caller) and
 * C_H(nbrs U^k) at the grid's nodes into Cout (full grid, may be NULL).  The
 * weight of a node is theta_node(T, ...) (T may be NULL: constant theta); it
 * is also written to theta_out (full grid, may be NULL). */
static long step4_grid(const geom_t *G, const long *o, double H, double theta, const double *r,
                       const unsigned char *gamma, const double *g, const double *Uk, const double *uk,
                       const signed char *wk, const signed char *Wk, double *U, long max_sweeps, long *caps,
                       const theta_ctx *T, double *Cout, double *theta_out)
{
    long m[3], M, s = 0, x, y, z;
    double *Ul, *Ukl, *Cold, *ukl, *rl, *thl, *gl;
    unsigned char *fl;
    int *Al, capped;
    long *fidx;
    signed char *wkl, *Wkl;
    grid_box(G, o, m);
    M = m[0] * m[1] * m[2];
    Ul = malloc(sizeof(double) * (size_t)M);
    Ukl = malloc(sizeof(double) * (size_t)M);
    Cold = malloc(sizeof(double) * (size_t)M);
    thl = malloc(sizeof(double) * (size_t)M);
    gl = malloc(sizeof(double) * (size_t)M);
    fidx = malloc(sizeof(long) * (size_t)M);
    ukl = malloc(sizeof(double) * (size_t)M);
    rl = malloc(sizeof(double) * (size_t)M);
    fl = malloc((size_t)M);
    Al = malloc(sizeof(int) * (size_t)M);
    wkl = malloc((size_t)(3 * M));
    Wkl = malloc((size_t)(3 * M));
    for (z = 0; z < m[2]; ++z)
        for (y = 0; y < m[1]; ++y)
            for (x = 0; x < m[0]; ++x) {
                long f = grid_fine(G, o, x, y, z), l = lidx(m, x, y, z), xf[3];
                int k;
                coords(G, f, xf);
                rl[l] = r[f];
                fidx[l] = f;
                fl[l] = gamma[f] ? 1 : 0;
                gl[l] = g[f];
                Ukl[l] = Uk[f];
                ukl[l] = uk[f];
                Al[l] = coarse_axes(G, xf);
                for (k = 0; k < 3; ++k) {
                    wkl[3 * l + k] = wk[3 * f + k];
                    Wkl[3 * l + k] = Wk[3 * f + k];
                }
            }
    /* C_H(nbrs^H(U^k)) at every node, from the previous iterate, then the
     * weight of every node (constant, or Sec. 4.2's estimate). */
    coarse_solver_prev(G->d, m, H, rl, Ukl, Cold);
    for (z = 0; z < m[2]; ++z)
        for (y = 0; y < m[1]; ++y)
            for (x = 0; x < m[0]; ++x) {
                long l = lidx(m, x, y, z);
                thl[l] = T ? theta_node(T, fidx[l], ukl[l], Cold[l]) : theta;
                if (Cout) Cout[fidx[l]] = Cold[l];
                if (theta_out) theta_out[fidx[l]] = thl[l];
            }
    s = alg5_sweeps(G->d, m, H, rl, fl, gl, ukl, wkl, Wkl, Al, Cold, thl, max_sweeps, Ul, &capped);
    if (capped) ++*caps;
    grid_scatter_d(G, o, m, Ul, U);
    free(Ul);
    free(Ukl);
    free(Cold);
    free(thl);
    free(gl);
    free(fidx);
    free(ukl);
    free(rl);
    free(fl);
    free(Al);
    free(wkl);
    free(Wkl);
    return s;
}

/* Step 2 + Step 3 on one subdomain: boundary data from (U, W), FSM, winds.
 * ut/wt: the subdomain's local arrays ((S+1)^d nodes). */
static long step23_tile(const geom_t *G, const int *t, double h, const double *r, const unsigned char *gamma,
                        const double *g, const double *U, const signed char *W, double *ut, signed char *wt,
                        unsigned char *echo, long max_sweeps, long *caps)
{
    long m[3], M, x, y, z, s, l;
    double *rl, *u0;
    unsigned char *fl, *in;
    int conv, k;
    for (k = 0; k < 3; ++k) m[k] = (k < G->d) ? G->S[k] + 1 : 1;
    M = m[0] * m[1] * m[2];
    rl = malloc(sizeof(double) * (size_t)M);
    u0 = malloc(sizeof(double) * (size_t)M);
    fl = malloc((size_t)M);
    in = malloc((size_t)M);
    for (z = 0; z < m[2]; ++z)
        for (y = 0; y < m[1]; ++y)
            for (x = 0; x < m[0]; ++x) {
                long lc[3] = {x, y, z}, xf[3], f, l = lidx(m, x, y, z);
                int inflow = 0, face = 0;
                for (k = 0; k < 3; ++k) xf[k] = (k < G->d) ? t[k] * G->S[k] + lc[k] : 0;
                f = xf[0] + G->n[0] * (xf[1] + G->n[1] * xf[2]);
                rl[l] = r[f];
                in[l] = 0;
                for (k = 0; k < 3; ++k) wt[3 * l + k] = 0;
                if (gamma[f]) {
                    fl[l] = 1;
                    ut[l] = g[f];
                    continue;
                }
                /* Step 2: inflow when W . n > 0 for an inward normal n. */
                for (k = 0; k < G->d; ++k) {
                    if (lc[k] == 0) {
                        face = 1;
                        if (W[3 * f + k] > 0) inflow = 1;
                    }
                    if (lc[k] == m[k] - 1) {
                        face = 1;
                        if (W[3 * f + k] < 0) inflow = 1;
                    }
                }
                fl[l] = 0;
                ut[l] = (face && inflow) ? U[f] : INF;
                in[l] = (unsigned char)(face && inflow);
            }
    memcpy(u0, ut, sizeof(double) * (size_t)M);
    s = fsm_local(G->d, m, h, rl, fl, ut, max_sweeps, &conv);
    if (!conv) ++*caps;
    winds_local(G->d, m, h, rl, fl, ut, wt);
    /* an inflow node that kept its boundary value keeps the coarse wind W and
     * is marked as an echo of the boundary data (Alg. 4 reads the mark) */
    for (z = 0; z < m[2]; ++z)
        for (y = 0; y < m[1]; ++y)
            for (x = 0; x < m[0]; ++x) {
                long xf[3], f, lc[3] = {x, y, z};
                l = lidx(m, x, y, z);
                echo[l] = (unsigned char)(in[l] && ut[l] == u0[l]);
                if (!echo[l]) continue;
                for (k = 0; k < 3; ++k) xf[k] = (k < G->d) ? t[k] * G->S[k] + lc[k] : 0;
                f = xf[0] + G->n[0] * (xf[1] + G->n[1] * xf[2]);
                for (k = 0; k < 3; ++k) wt[3 * l + k] = W[3 * f + k];
            }
    free(rl);
    free(u0);
    free(fl);
    free(in);
    return s;
}

/* Alg. 4's choice at one coarse-set node (Sec. 3.2).  The node lies on the
 * interfaces of the axes in B (bit k); nc[k] = 2 copies along such an axis
 * (minus-side subdomain first), 1 otherwise; the copies are enumerated with
 * axis 0 fastest, i.e. in ascending linear subdomain index.  Copy q has value
 * u[q], wind w[3q..3q+2] and echo flag echo[q]; W is the coarse wind W^k.
 * Per interface axis: when every fine wind and W^k point toward -axis (or
 * are zero) the plus-side copy is taken (Alg. 4's first branch), when they
 * all point toward +axis the minus-side copy; if some axis has neither, the
 * minimum of the fine solutions (echoes only when every copy is one; ties to
 * the lowest index).  Returns the index of the chosen copy. */
int orc_alg4_select(int d, int B, const int *nc, int ncopies, const double *u, const signed char *w,
                    const unsigned char *echo, const signed char *W)
{
    int k, q, ok = 1, sel[3] = {0, 0, 0}, best;
    if (!B) return 0;
    for (k = 0; k < d && ok; ++k) {
        int allneg = 1, allpos = 1;
        if (!(B & (1 << k))) continue;
        if (W[k] > 0) allneg = 0;
        if (W[k] < 0) allpos = 0;
        for (q = 0; q < ncopies; ++q) {
            int wv = w[3 * q + k];
            if (wv > 0) allneg = 0;
            if (wv < 0) allpos = 0;
        }
        /* Alg. 4: first branch (wind toward -axis: take the plus-side
         * copy) wins when both hold; then the minus-side copy. */
        if (allneg)
            sel[k] = 1;
        else if (allpos)
            sel[k] = 0;
        else
            ok = 0;
    }
    if (ok) {
        /* index of the selected copy in the enumeration */
        int stride = 1;
        best = 0;
        for (k = 0; k < 3; ++k) {
            best += sel[k] * stride;
            stride *= nc[k];
        }
        return best;
    }
    /* otherwise the minimum of the fine solutions: copies that only echo
     * their Step 2 boundary value are not candidates unless every copy is
     * one; ties keep the lowest subdomain index */
    {
        int computed = 0;
        for (q = 0; q < ncopies; ++q)
            if (!echo[q]) computed = 1;
        best = -1;
        for (q = 0; q < ncopies; ++q) {
            if (computed && echo[q]) continue;
            if (best < 0 || u[q] < u[best]) best = q;
        }
    }
    return best;
}

/* Alg. 4 at every coarse-set node: choose u^k, w^k among the subdomain copies. */
static void alg4(const geom_t *G, double **tu, signed char **tw, unsigned char **te, const signed char *W, double *uk,
                 signed char *wk)
{
    long i;
    long tm[3];
    int k;
    for (k = 0; k < 3; ++k) tm[k] = (k < G->d) ? G->S[k] + 1 : 1;
    for (i = 0; i < G->N; ++i) {
        long x[3];
        long cand[3][2];
        int nc[3], B = 0;
        int A, q, ncopies, best;
        long cidx[8], lidxs[8];
        double cu[8];
        signed char cw[24];
        unsigned char ce[8];
        coords(G, i, x);
        A = coarse_axes(G, x);
        if (!A) continue;
        for (k = 0; k < 3; ++k) {
            if (k >= G->d) {
                cand[k][0] = 0;
                nc[k] = 1;
                continue;
            }
            if (x[k] % G->S[k] == 0 && x[k] > 0 && x[k] < G->n[k] - 1) {
                cand[k][0] = x[k] / G->S[k] - 1; /* minus side */
                cand[k][1] = x[k] / G->S[k];     /* plus side */
                nc[k] = 2;
                B |= 1 << k;
            } else {
                long tt = x[k] / G->S[k];
                if (tt >= G->T[k]) tt = G->T[k] - 1;
                cand[k][0] = tt;
                nc[k] = 1;
            }
        }
        /* copies in ascending linear subdomain index (axis 0 fastest) */
        ncopies = 0;
        {
            int a0, a1, a2;
            for (a2 = 0; a2 < nc[2]; ++a2)
                for (a1 = 0; a1 < nc[1]; ++a1)
                    for (a0 = 0; a0 < nc[0]; ++a0) {
                        long tt[3] = {cand[0][a0], cand[1][a1], cand[2][a2]};
                        long lc[3];
                        for (k = 0; k < 3; ++k) lc[k] = (k < G->d) ? x[k] - tt[k] * G->S[k] : 0;
                        cidx[ncopies] = tt[0] + G->T[0] * (tt[1] + G->T[1] * tt[2]);
                        lidxs[ncopies] = lidx(tm, lc[0], lc[1], lc[2]);
                        ++ncopies;
                    }
        }
        for (q = 0; q < ncopies; ++q) {
            cu[q] = tu[cidx[q]][lidxs[q]];
            ce[q] = te[cidx[q]][lidxs[q]];
            for (k = 0; k < 3; ++k) cw[3 * q + k] = tw[cidx[q]][3 * lidxs[q] + k];
        }
        best = orc_alg4_select(G->d, B, nc, ncopies, cu, cw, ce, W + 3 * i);
        uk[i] = cu[best];
        for (k = 0; k < 3; ++k) wk[3 * i + k] = cw[3 * best + k];
    }
}

static double coarse_delta(const geom_t *G, const double *U1, const double *U0)
{
    long i;
    double dmax = 0.0;
    for (i = 0; i < G->N; ++i) {
        long x[3];
        double dv;
        coords(G, i, x);
        if (!coarse_axes(G, x)) continue;
        if (U1[i] == U0[i]) continue; /* covers inf == inf */
        dv = fabs(U1[i] - U0[i]);
        if (dv > dmax) dmax = dv;
    }
    return dmax;
}

/* Test hooks of dd_iterate (all optional): Step 1's W^0 and decision
 * margins out; U^0, W^0 replaced by given ones after Step 1; the subdomain
 * copies of iteration 0 at the coarse-set nodes and the margins of the
 * decisions behind Alg. 4's choice among them out. */
typedef struct {
    signed char *W0_out;
    double *margin_out;
    const double *U0_in;
    const signed char *W0_in;
    double *copies_out;  /* [4][N], slot as in the copy export below, NaN where absent */
    double *cmargin_out; /* [N] */
} dd_hooks;

/* Alg. 3 decision margin at node l of a subdomain's final state (spacing h,
 * one-sided at the box edges), as step1_margins; for an inflow node also the
 * gap between its starting value and the local solve (whether it kept U, the
 * echo rule of the copies). */
static double tile_node_margin(int d, const long *m, double rh, const double *ut, long x, long y, long z,
                               int inflow, double u0)
{
    double vm[3], vp[3], a[3], mg = INF;
    signed char w[3];
    int k, j;
    nbrs(d, m, ut, x, y, z, vm, vp);
    for (k = 0; k < d; ++k) {
        double dv = fabs(vm[k] - vp[k]);
        if (dv < mg) mg = dv;
        a[k] = vm[k] < vp[k] ? vm[k] : vp[k];
    }
    for (k = 0; k < d; ++k)
        for (j = k + 1; j < d; ++j) {
            double t = fabs(a[k] - a[j]);
            if (t < mg) mg = t;
            if (fabs(t - rh) < mg) mg = fabs(t - rh);
        }
    if (inflow) {
        double ls = orc_local_solve(d, vm, vp, rh, w);
        if (fabs(ls - u0) < mg) mg = fabs(ls - u0);
    }
    return mg;
}

/* The copies of every subdomain at its coarse-set nodes (slot bit 0: the node
 * is the subdomain's x = 0 face on an interior x interface, bit 1 the same for
 * y), and per node the smallest decision margin over its copies.  (Copies
 * closer than the compared precision's error may be chosen either way without
 * moving the result beyond it, so their gap is no decision margin.) */
static void export_copies(const geom_t *G, double h, const double *r, const unsigned char *gamma, const double *U,
                          const signed char *W, double **tu, double *copies, double *cmargin)
{
    long ti, ntiles = (long)G->T[0] * G->T[1] * G->T[2], i, m[3];
    int k;
    for (k = 0; k < 3; ++k) m[k] = (k < G->d) ? G->S[k] + 1 : 1;
    for (i = 0; i < 4 * G->N; ++i) copies[i] = NAN;
    for (i = 0; i < G->N; ++i) cmargin[i] = NAN;
    for (ti = 0; ti < ntiles; ++ti) {
        int t[3];
        long x, y, z;
        t[0] = (int)(ti % G->T[0]);
        t[1] = (int)((ti / G->T[0]) % G->T[1]);
        t[2] = (int)(ti / ((long)G->T[0] * G->T[1]));
        for (z = 0; z < m[2]; ++z)
            for (y = 0; y < m[1]; ++y)
                for (x = 0; x < m[0]; ++x) {
                    long lc[3] = {x, y, z}, xf[3], f, l = lidx(m, x, y, z);
                    int slot = 0, inflow = 0;
                    double mg;
                    for (k = 0; k < 3; ++k) xf[k] = (k < G->d) ? t[k] * G->S[k] + lc[k] : 0;
                    if (!coarse_axes(G, xf)) continue;
                    f = xf[0] + G->n[0] * (xf[1] + G->n[1] * xf[2]);
                    if (G->d >= 1 && lc[0] == 0 && xf[0] > 0 && xf[0] < G->n[0] - 1) slot |= 1;
                    if (G->d >= 2 && lc[1] == 0 && xf[1] > 0 && xf[1] < G->n[1] - 1) slot |= 2;
                    copies[(long)slot * G->N + f] = tu[ti][l];
                    if (gamma[f] || !(tu[ti][l] < INF)) continue;
                    for (k = 0; k < G->d; ++k) {
                        if (lc[k] == 0 && W[3 * f + k] > 0) inflow = 1;
                        if (lc[k] == m[k] - 1 && W[3 * f + k] < 0) inflow = 1;
                    }
                    mg = tile_node_margin(G->d, m, r[f] * h, tu[ti], x, y, z, inflow, U[f]);
                    if (isnan(cmargin[f]) || mg < cmargin[f]) cmargin[f] = mg;
                }
    }
}

static int dd_iterate(const orc_dd_params *p, const double *r, const unsigned char *gamma, const double *g,
                      double *u_out, double *U_out, double *delta_log, orc_dd_stats *st, long probe,
                      double *probe_log, const dd_hooks *hk)
{
    geom_t G;
    long i, ntiles;
    int k, it;
    double H, delta = INF;
    double *U, *Uprev, *uk, **tu, *uprev, *Chist[4];
    signed char *W, *wk, **tw;
    unsigned char **te;
    long tilenodes;
    orc_dd_stats S0;
    theta_ctx tctx;
    double *thfull = NULL;
    long *offs, *gsweeps, *gcaps, *tsweeps, *tcaps, ngrid = 0;
    memset(&S0, 0, sizeof(S0));
    if (p->d < 2 || p->d > 3 || p->c < 1) return -1;
    memset(&G, 0, sizeof(G));
    G.d = p->d;
    G.c = p->c;
    for (k = 0; k < 3; ++k) {
        G.n[k] = (k < p->d) ? p->n[k] : 1;
        G.T[k] = (k < p->d) ? p->tiles[k] : 1;
        if (k < p->d) {
            if (G.T[k] < 1 || (G.n[k] - 1) % G.T[k]) return -1;
            G.S[k] = (G.n[k] - 1) / G.T[k];
            if (G.S[k] % G.c) return -1;
        } else
            G.S[k] = 0;
    }
    G.N = G.n[0] * G.n[1] * G.n[2];
    G.st[0] = 1;
    G.st[1] = G.n[0];
    G.st[2] = G.n[0] * G.n[1];
    H = G.c * p->h;
    ntiles = (long)G.T[0] * G.T[1] * G.T[2];
    tilenodes = 1;
    for (k = 0; k < p->d; ++k) tilenodes *= G.S[k] + 1;
    if (probe_log && (probe < 0 || probe >= G.N)) return -1;

    U = malloc(sizeof(double) * (size_t)G.N);
    Uprev = malloc(sizeof(double) * (size_t)G.N);
    uk = malloc(sizeof(double) * (size_t)G.N);
    uprev = malloc(sizeof(double) * (size_t)G.N);
    for (k = 0; k < 4; ++k) Chist[k] = malloc(sizeof(double) * (size_t)G.N);
    W = calloc((size_t)(3 * G.N), 1);
    wk = calloc((size_t)(3 * G.N), 1);
    tu = malloc(sizeof(double *) * (size_t)ntiles);
    tw = malloc(sizeof(signed char *) * (size_t)ntiles);
    te = malloc(sizeof(unsigned char *) * (size_t)ntiles);
    for (i = 0; i < ntiles; ++i) {
        tu[i] = malloc(sizeof(double) * (size_t)tilenodes);
        tw[i] = malloc((size_t)(3 * tilenodes));
        te[i] = malloc((size_t)tilenodes);
    }
    for (i = 0; i < G.N; ++i) U[i] = uk[i] = NAN;
    /* the shifted coarse grids, in enumeration order */
    {
        long o[3];
        int first = 1;
        while (next_offset(&G, o, first)) {
            first = 0;
            ++ngrid;
        }
        offs = malloc(sizeof(long) * (size_t)(3 * ngrid));
        first = 1;
        ngrid = 0;
        while (next_offset(&G, o, first)) {
            first = 0;
            offs[3 * ngrid] = o[0];
            offs[3 * ngrid + 1] = o[1];
            offs[3 * ngrid + 2] = o[2];
            ++ngrid;
        }
    }
    gsweeps = malloc(sizeof(long) * (size_t)ngrid);
    gcaps = malloc(sizeof(long) * (size_t)ngrid);
    tsweeps = malloc(sizeof(long) * (size_t)ntiles);
    tcaps = malloc(sizeof(long) * (size_t)ntiles);
    if (probe_log) {
        for (k = 0; k < 4 * (p->max_iter + 1); ++k) probe_log[k] = NAN;
        thfull = malloc(sizeof(double) * (size_t)G.N);
        for (i = 0; i < G.N; ++i) thfull[i] = NAN;
    }

    /* Step 1: every shifted coarse grid, independently; then the causal sweep.
     * (Built with OpenMP, the grids run in parallel: each writes only its own
     * nodes, and the counters are combined after the loop.) */
    {
        long q;
        for (q = 0; q < ngrid; ++q) {
            gsweeps[q] = 0;
            gcaps[q] = 0;
        }
#pragma omp parallel for schedule(dynamic, 1)
        for (q = 0; q < ngrid; ++q)
            gsweeps[q] = step1_grid(&G, offs + 3 * q, H, r, gamma, g, U, W, p->max_coarse_sweeps, &gcaps[q]);
        for (q = 0; q < ngrid; ++q) {
            long m[3];
            if (gsweeps[q] > S0.coarse_sweeps_max) S0.coarse_sweeps_max = gsweeps[q];
            S0.coarse_cap_hits += gcaps[q];
            grid_box(&G, offs + 3 * q, m);
            S0.coarse_updates += (long long)gsweeps[q] * m[0] * m[1] * m[2];
        }
    }
    if (hk && hk->margin_out) {
        long q;
        for (i = 0; i < G.N; ++i) hk->margin_out[i] = NAN;
        for (q = 0; q < ngrid; ++q) step1_margins(&G, offs + 3 * q, H, r, gamma, U, hk->margin_out);
    }
    {
        long cr = causal_sweep(&G, U, W);
        if (cr > S0.causal_rounds_max) S0.causal_rounds_max = cr;
    }
    if (hk && hk->W0_out) memcpy(hk->W0_out, W, (size_t)(3 * G.N));
    if (hk && hk->U0_in)
        for (i = 0; i < G.N; ++i)
            if (!isnan(U[i])) U[i] = hk->U0_in[i];
    if (hk && hk->W0_in) memcpy(W, hk->W0_in, (size_t)(3 * G.N));
    if (delta_log)
        for (k = 0; k <= p->max_iter; ++k) delta_log[k] = NAN;
    if (delta_log) delta_log[0] = INF;

    for (it = 0;; ++it) {
        /* Steps 2 + 3: every subdomain independently (in parallel when built
         * with OpenMP; tile ti has coordinates t, axis 0 fastest). */
        long ti;
        for (ti = 0; ti < ntiles; ++ti) tcaps[ti] = 0;
#pragma omp parallel for schedule(dynamic, 1)
        for (ti = 0; ti < ntiles; ++ti) {
            int t[3];
            t[0] = (int)(ti % G.T[0]);
            t[1] = (int)((ti / G.T[0]) % G.T[1]);
            t[2] = (int)(ti / ((long)G.T[0] * G.T[1]));
            tsweeps[ti] = step23_tile(&G, t, p->h, r, gamma, g, U, W, tu[ti], tw[ti], te[ti], p->max_fsm_sweeps,
                                      &tcaps[ti]);
        }
        for (ti = 0; ti < ntiles; ++ti) {
            if (tsweeps[ti] > S0.fsm_sweeps_max) S0.fsm_sweeps_max = tsweeps[ti];
            S0.fsm_cap_hits += tcaps[ti];
            S0.fine_updates += (long long)tsweeps[ti] * tilenodes;
        }
        /* Alg. 4 */
        alg4(&G, tu, tw, te, W, uk, wk);
        if (hk && hk->copies_out && it == 0) export_copies(&G, p->h, r, gamma, U, W, tu, hk->copies_out, hk->cmargin_out);
        if (thfull) {
            probe_log[4 * it + 0] = uk[probe];
            probe_log[4 * it + 3] = U[probe];
        }
        S0.iters = it;
        if (it == p->max_iter) break;
        if (it >= 1 && delta < p->tol) {
            S0.converged = 1;
            break;
        }
        /* Step 4: Alg. 5 on every shifted grid, W = w^k, then the causal sweep. */
        memcpy(Uprev, U, sizeof(double) * (size_t)G.N);
        tctx.p = p;
        tctx.nhist = it < 3 ? it : 3;
        tctx.C1 = it >= 1 ? Chist[(it + 3) % 4] : NULL;
        tctx.C2 = it >= 2 ? Chist[(it + 2) % 4] : NULL;
        tctx.C3 = it >= 3 ? Chist[(it + 1) % 4] : NULL;
        tctx.uprev = uprev;
        {
            long q;
            double *Unew = malloc(sizeof(double) * (size_t)G.N);
            memcpy(Unew, U, sizeof(double) * (size_t)G.N);
            for (q = 0; q < ngrid; ++q) gcaps[q] = 0;
#pragma omp parallel for schedule(dynamic, 1)
            for (q = 0; q < ngrid; ++q)
                gsweeps[q] = step4_grid(&G, offs + 3 * q, H, p->theta, r, gamma, g, Uprev, uk, wk, W, Unew,
                                        p->max_coarse_sweeps, &gcaps[q], &tctx, Chist[it % 4], thfull);
            for (q = 0; q < ngrid; ++q) {
                long m[3];
                if (gsweeps[q] > S0.coarse_sweeps_max) S0.coarse_sweeps_max = gsweeps[q];
                S0.coarse_cap_hits += gcaps[q];
                grid_box(&G, offs + 3 * q, m);
                S0.coarse_updates += (long long)gsweeps[q] * m[0] * m[1] * m[2];
            }
            memcpy(U, Unew, sizeof(double) * (size_t)G.N);
            free(Unew);
        }
        if (thfull) {
            probe_log[4 * it + 1] = Chist[it % 4][probe];
            probe_log[4 * it + 2] = thfull[probe];
        }
        for (i = 0; i < G.N; ++i) {
            long x[3];
            coords(&G, i, x);
            if (coarse_axes(&G, x)) {
                int kk;
                for (kk = 0; kk < 3; ++kk) W[3 * i + kk] = wk[3 * i + kk];
            }
        }
        {
            long cr = causal_sweep(&G, U, W);
            if (cr > S0.causal_rounds_max) S0.causal_rounds_max = cr;
        }
        delta = coarse_delta(&G, U, Uprev);
        if (delta_log && it + 1 <= p->max_iter) delta_log[it + 1] = delta;
        memcpy(uprev, uk, sizeof(double) * (size_t)G.N);
    }
    S0.last_delta = delta;

    /* Patched fine solution: coarse-set nodes take u^k, the rest their
     * (unique) subdomain's value. */
    for (i = 0; i < G.N; ++i) {
        long x[3], tt[3], lc[3], tl;
        long tm[3];
        coords(&G, i, x);
        if (coarse_axes(&G, x)) {
            u_out[i] = uk[i];
            continue;
        }
        for (k = 0; k < 3; ++k) {
            tm[k] = (k < G.d) ? G.S[k] + 1 : 1;
            tt[k] = (k < G.d) ? x[k] / G.S[k] : 0;
            lc[k] = (k < G.d) ? x[k] - tt[k] * G.S[k] : 0;
        }
        tl = tt[0] + G.T[0] * (tt[1] + G.T[1] * tt[2]);
        u_out[i] = tu[tl][lidx(tm, lc[0], lc[1], lc[2])];
    }
    if (U_out)
        for (i = 0; i < G.N; ++i) U_out[i] = U[i];
    if (st) *st = S0;

    for (i = 0; i < ntiles; ++i) {
        free(tu[i]);
        free(tw[i]);
        free(te[i]);
    }
    free(tu);
    free(tw);
    free(te);
    free(U);
    free(Uprev);
    free(uprev);
    for (k = 0; k < 4; ++k) free(Chist[k]);
    free(uk);
    free(W);
    free(wk);
    free(thfull);
    free(offs);
    free(gsweeps);
    free(gcaps);
    free(tsweeps);
    free(tcaps);
    return 0;
}

int orc_dd(const orc_dd_params *p, const double *r, const unsigned char *gamma, const double *g,
           double *u_out, double *U_out, double *delta_log, orc_dd_stats *st)
{
    return dd_iterate(p, r, gamma, g, u_out, U_out, delta_log, st, -1, NULL, NULL);
}

int orc_dd_probe(const orc_dd_params *p, const double *r, const unsigned char *gamma, const double *g,
                 double *u_out, double *U_out, double *delta_log, orc_dd_stats *st, long probe_node,
                 double *probe_log)
{
    return dd_iterate(p, r, gamma, g, u_out, U_out, delta_log, st, probe_node, probe_log, NULL);
}

int orc_dd_margins(const orc_dd_params *p, const double *r, const unsigned char *gamma, const double *g,
                   double *u_out, orc_dd_stats *st, signed char *W0_out, double *margin_out,
                   const double *U0_in, const signed char *W0_in, double *copies_out, double *cmargin_out)
{
    dd_hooks hk;
    hk.W0_out = W0_out;
    hk.margin_out = margin_out;
    hk.U0_in = U0_in;
    hk.W0_in = W0_in;
    hk.copies_out = (copies_out && cmargin_out) ? copies_out : NULL;
    hk.cmargin_out = cmargin_out;
    return dd_iterate(p, r, gamma, g, u_out, NULL, NULL, st, -1, NULL, &hk);
}

/* ------------------------------------------------------------------------- */
/* The one-dimensional method, Sec. 3.1 (Steps 1-4).                           */
/* Fine grid x_j = j h, j = 0..N M; coarse grid X_i = i H = x_{iM}; subinterval */
/* i holds fine nodes iM..iM+M.  Readings shared with the 2-D method: winds     */
/* are directions of travel (+1 when the left neighbour gives the minimum; the  */
/* sign printed in Step 4 for W~ is read as flipped, as in 2-D); ties go to the */
/* right neighbour (-1); inflow boundary nodes start at U and are swept, and    */
/* one that keeps U echoes the coarse wind and is no candidate of the minimum   */
/* unless both copies are echoes; the weighted update is evaluated as           */
/* u^k + theta (U~ - C_H(U^k)), and u^k when U~ or C_H(U^k) is +inf; the       */
/* causal sweep is repeated until nothing changes.  Step 1 has no causal sweep  */
/* (the 2-D text adds one there); the Step 3 choice compares the two fine      */
/* winds only, as printed (no W^k in the 1-D rule); the Step 4 test is the      */
/* printed equality W^k = w^k = W~.                                             */
/* ------------------------------------------------------------------------- */

/* C_H(U_{i-1}, U_{i+1}) of eq. 1dgod at coarse node i (+inf outside), with the
 * wind of the neighbour used. */
static double ch1(const double *U, long i, long N, double rH, int *w)
{
    double a = (i > 0) ? U[i - 1] : INF, b = (i < N) ? U[i + 1] : INF, v;
    if (a < b) {
        v = a + rH;
        *w = +1;
    } else {
        v = b + rH;
        *w = -1;
    }
    if (!(v < INF)) *w = 0;
    return v;
}

int orc_dd1(const orc_dd1_params *p, const double *r, const unsigned char *gamma, const double *g, double *u_out,
            double *U_log, double *u_log, double *Upre_log, signed char *W_log, orc_dd1_stats *st)
{
    const long N = p->N, M = p->M, nf = p->N * p->M + 1;
    const double H = (double)p->M * p->h;
    long i, j, k, sub;
    double *U, *Uprev, *Unew, *uk, *Cold, **tu, delta = INF;
    signed char *W, *wk, **tw;
    unsigned char *cfix, **te;
    orc_dd1_stats S0;
    if (N < 1 || M < 1 || p->max_iter < 0 || !(p->h > 0.0)) return -1;
    memset(&S0, 0, sizeof(S0));
    U = malloc(sizeof(double) * (size_t)(N + 1));
    Uprev = malloc(sizeof(double) * (size_t)(N + 1));
    Unew = malloc(sizeof(double) * (size_t)(N + 1));
    uk = malloc(sizeof(double) * (size_t)(N + 1));
    Cold = malloc(sizeof(double) * (size_t)(N + 1));
    W = calloc((size_t)(N + 1), 1);
    wk = calloc((size_t)(N + 1), 1);
    cfix = malloc((size_t)(N + 1));
    tu = malloc(sizeof(double *) * (size_t)N);
    tw = malloc(sizeof(signed char *) * (size_t)N);
    te = malloc(sizeof(unsigned char *) * (size_t)N);
    for (sub = 0; sub < N; ++sub) {
        tu[sub] = malloc(sizeof(double) * (size_t)(M + 1));
        tw[sub] = malloc((size_t)(3 * (M + 1)));
        te[sub] = malloc((size_t)(M + 1));
    }
    for (i = 0; i <= N; ++i) cfix[i] = gamma[i * M] ? 1 : 0;

    /* Step 1: FSM on the coarse grid (spacing H, r sampled at X_i), winds. */
    {
        long mc[3] = {N + 1, 1, 1};
        double *rc = malloc(sizeof(double) * (size_t)(N + 1));
        signed char *wc = calloc((size_t)(3 * (N + 1)), 1);
        int conv;
        long s;
        for (i = 0; i <= N; ++i) {
            rc[i] = r[i * M];
            U[i] = cfix[i] ? g[i * M] : INF;
        }
        s = fsm_local(1, mc, H, rc, cfix, U, p->max_coarse_sweeps, &conv);
        if (!conv) ++S0.coarse_cap_hits;
        if (s > S0.coarse_sweeps_max) S0.coarse_sweeps_max = s;
        winds_local(1, mc, H, rc, cfix, U, wc);
        for (i = 0; i <= N; ++i) W[i] = cfix[i] ? 0 : wc[3 * i];
        free(rc);
        free(wc);
    }

    for (k = 0;; ++k) {
        if (U_log)
            for (i = 0; i <= N; ++i) U_log[k * (N + 1) + i] = U[i];
        if (W_log)
            for (i = 0; i <= N; ++i) W_log[k * (N + 1) + i] = W[i];
        /* Steps 2 + 3: every subinterval on its own. */
        for (sub = 0; sub < N; ++sub) {
            long m[3] = {M + 1, 1, 1};
            double *rl = malloc(sizeof(double) * (size_t)(M + 1));
            double *u0 = malloc(sizeof(double) * (size_t)(M + 1));
            unsigned char *fl = malloc((size_t)(M + 1)), *in = malloc((size_t)(M + 1));
            int conv;
            long s;
            for (j = 0; j <= M; ++j) {
                long f = sub * M + j;
                rl[j] = r[f];
                fl[j] = gamma[f] ? 1 : 0;
                in[j] = 0;
                tw[sub][3 * j] = tw[sub][3 * j + 1] = tw[sub][3 * j + 2] = 0;
                if (fl[j]) {
                    tu[sub][j] = g[f];
                    continue;
                }
                /* Step 2: U where the characteristic arrives into the
                 * subinterval (W = +1 at its left end, W = -1 at its right
                 * end), +inf otherwise. */
                if (j == 0 && W[sub] > 0) in[j] = 1;
                if (j == M && W[sub + 1] < 0) in[j] = 1;
                tu[sub][j] = in[j] ? U[j == 0 ? sub : sub + 1] : INF;
            }
            memcpy(u0, tu[sub], sizeof(double) * (size_t)(M + 1));
            s = fsm_local(1, m, p->h, rl, fl, tu[sub], p->max_fsm_sweeps, &conv);
            if (!conv) ++S0.fsm_cap_hits;
            if (s > S0.fsm_sweeps_max) S0.fsm_sweeps_max = s;
            S0.fine_updates += (long long)s * (M + 1);
            winds_local(1, m, p->h, rl, fl, tu[sub], tw[sub]);
            for (j = 0; j <= M; ++j) {
                te[sub][j] = (unsigned char)(in[j] && tu[sub][j] == u0[j]);
                if (te[sub][j]) tw[sub][3 * j] = W[j == 0 ? sub : sub + 1];
            }
            free(rl);
            free(u0);
            free(fl);
            free(in);
        }
        /* Step 3's choice of u^k_i, w^k_i between the two fine values. */
        for (i = 0; i <= N; ++i) {
            if (i == 0) {
                uk[i] = tu[0][0];
                wk[i] = tw[0][0];
            } else if (i == N) {
                uk[i] = tu[N - 1][M];
                wk[i] = tw[N - 1][3 * M];
            } else {
                double uL = tu[i - 1][M], uR = tu[i][0];
                int wL = tw[i - 1][3 * M], wR = tw[i][0];
                int eL = te[i - 1][M], eR = te[i][0], takeL;
                if (wL == 1 && wR == 1)
                    takeL = 1; /* wind from left to right */
                else if (wL == -1 && wR == -1)
                    takeL = 0; /* wind from right to left */
                else if (eL != eR)
                    takeL = eR; /* the computed value of the two */
                else
                    takeL = !(uR < uL); /* minimum, tie to the left copy */
                uk[i] = takeL ? uL : uR;
                wk[i] = (signed char)(takeL ? wL : wR);
            }
        }
        if (u_log)
            for (i = 0; i <= N; ++i) u_log[k * (N + 1) + i] = uk[i];
        S0.iters = (int)k;
        if (k == p->max_iter) break;
        if (k >= 1 && delta < p->tol) {
            S0.converged = 1;
            break;
        }
        /* Step 4: weighted coarse sweeps. */
        memcpy(Uprev, U, sizeof(double) * (size_t)(N + 1));
        for (i = 0; i <= N; ++i) {
            int wd;
            Cold[i] = ch1(Uprev, i, N, r[i * M] * H, &wd);
            Unew[i] = cfix[i] ? g[i * M] : INF; /* initialise as in FSM */
        }
        {
            long s = 0;
            for (;;) {
                int changed = 0;
                long step = (s % 2 == 0) ? -1 : +1, i0 = (step > 0) ? 0 : N;
                if (s >= p->max_coarse_sweeps) {
                    ++S0.coarse_cap_hits;
                    break;
                }
                for (i = i0; i >= 0 && i <= N; i += step) {
                    int Wt;
                    double Ut, v;
                    if (cfix[i]) continue;
                    Ut = ch1(Unew, i, N, r[i * M] * H, &Wt);
                    if (Ut < INF && Cold[i] < INF && W[i] == wk[i] && wk[i] == Wt)
                        v = uk[i] + p->theta * (Ut - Cold[i]);
                    else
                        v = uk[i];
                    if (!(v == Unew[i])) changed = 1;
                    Unew[i] = v;
                }
                ++s;
                if (!changed) break;
            }
            if (s > S0.coarse_sweeps_max) S0.coarse_sweeps_max = s;
        }
        if (Upre_log)
            for (i = 0; i <= N; ++i) Upre_log[k * (N + 1) + i] = Unew[i];
        for (i = 0; i <= N; ++i) W[i] = wk[i];
        /* causal sweep, both directions, until nothing changes */
        {
            long rounds = 0;
            int changed;
            do {
                changed = 0;
                ++rounds;
                for (i = 1; i <= N; ++i)
                    if (W[i] == 1 && Unew[i] < Unew[i - 1] && Unew[i - 1] < INF) {
                        Unew[i] = Unew[i - 1];
                        changed = 1;
                    }
                for (i = N - 1; i >= 0; --i)
                    if (W[i] == -1 && Unew[i] < Unew[i + 1] && Unew[i + 1] < INF) {
                        Unew[i] = Unew[i + 1];
                        changed = 1;
                    }
            } while (changed);
            if (rounds > S0.causal_rounds_max) S0.causal_rounds_max = rounds;
        }
        memcpy(U, Unew, sizeof(double) * (size_t)(N + 1));
        delta = 0.0;
        for (i = 0; i <= N; ++i)
            if (!(U[i] == Uprev[i]) && fabs(U[i] - Uprev[i]) > delta) delta = fabs(U[i] - Uprev[i]);
    }
    S0.last_delta = (S0.iters >= 1) ? delta : INF;
    /* patched fine solution: coarse nodes take u^k, the rest their subinterval */
    for (j = 0; j < nf; ++j) {
        if (j % M == 0)
            u_out[j] = uk[j / M];
        else
            u_out[j] = tu[j / M][j % M];
    }
    if (st) *st = S0;
    for (sub = 0; sub < N; ++sub) {
        free(tu[sub]);
        free(tw[sub]);
        free(te[sub]);
    }
    free(tu);
    free(tw);
    free(te);
    free(U);
    free(Uprev);
    free(Unew);
    free(uk);
    free(Cold);
    free(W);
    free(wk);
    free(cfix);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of the converged discrete system (a project addition; the paper has */
/* no gradient).  At a converged u every reached non-Gamma node j satisfies     */
/* u_j = F(a_j, r_j), a_j the per-axis neighbour minima of the branch the local */
/* solve takes (Alg. 3 choice, ties to the plus side).  Linearising:            */
/*   du_j = sum_{i used by j} dF_j/du_i du_i + dF_j/dr_j dr_j,                  */
/* with the used neighbours i all smaller than u_j (causality).  For a scalar J */
/* with dJ/du given, lambda = dJ/du + (dF/du)^T lambda; each lambda_i pulls     */
/* from the downwind neighbours j that use i, so visiting nodes in decreasing u */
/* gives lambda exactly.  dJ/dr_j = lambda_j dF_j/dr_j.                         */
/* Branch derivatives: one term dF/da = 1, dF/dr = h; several terms with        */
/* sum_k (u - a_k)^2 = (r h)^2: dF/da_k = (u - a_k)/D, dF/dr = r h h / D,       */
/* D = sum_k (u - a_k) over the used axes in axis order.                        */
/* ------------------------------------------------------------------------- */
static int cmp_desc(const void *A, const void *B)
{
    const hent *a = A, *b = B;
    if (a->v > b->v) return -1;
    if (a->v < b->v) return 1;
    return (a->i < b->i) ? -1 : (a->i > b->i);
}

/* Weight dF_j/du_{j+off} with which node j depends on its neighbour j+off (0
 * if j does not use that neighbour), and dF_j/dr_j. */
static void adj_node(int d, const long *m, double h, const double *r, const unsigned char *gamma, const double *u,
                     long j, double wm[3], double wp[3], double *dudr)
{
    long c[3];
    double vm[3], vp[3], D = 0.0;
    signed char w[3];
    int k, used = 0;
    for (k = 0; k < 3; ++k) wm[k] = wp[k] = 0.0;
    *dudr = 0.0;
    if (gamma[j] || !(u[j] < INF)) return;
    c[0] = j % m[0];
    c[1] = (j / m[0]) % m[1];
    c[2] = j / (m[0] * m[1]);
    nbrs(d, m, u, c[0], c[1], c[2], vm, vp);
    (void)orc_local_solve(d, vm, vp, r[j] * h, w);
    for (k = 0; k < d; ++k)
        if (w[k] != 0) {
            D = D + (u[j] - (w[k] > 0 ? vm[k] : vp[k]));
            ++used;
        }
    if (used == 0) return;
    if (used == 1) {
        for (k = 0; k < d; ++k) {
            if (w[k] > 0) wm[k] = 1.0;
            if (w[k] < 0) wp[k] = 1.0;
        }
        *dudr = h;
        return;
    }
    if (!(D > 0.0)) return;
    for (k = 0; k < d; ++k) {
        if (w[k] > 0) wm[k] = (u[j] - vm[k]) / D;
        if (w[k] < 0) wp[k] = (u[j] - vp[k]) / D;
    }
    *dudr = ((r[j] * h) * h) / D;
}

void orc_adjoint(int d, const long *n, double h, const double *r, const unsigned char *gamma,
                 const double *u, const double *dJdu, double *dJdr)
{
    long m[3] = {n[0], d > 1 ? n[1] : 1, d > 2 ? n[2] : 1};
    long N = m[0] * m[1] * m[2], i, cnt = 0;
    long st[3] = {1, m[0], m[0] * m[1]};
    hent *ord = malloc(sizeof(hent) * (size_t)N);
    double *lam = malloc(sizeof(double) * (size_t)N);
    for (i = 0; i < N; ++i) {
        lam[i] = 0.0;
        dJdr[i] = 0.0;
        ord[cnt].v = u[i] < INF ? u[i] : HUGE_VAL;
        ord[cnt].i = i;
        ++cnt;
    }
    qsort(ord, (size_t)cnt, sizeof(hent), cmp_desc);
    for (i = 0; i < cnt; ++i) {
        long j = ord[i].i, c[3];
        int k;
        double acc = dJdu[j];
        c[0] = j % m[0];
        c[1] = (j / m[0]) % m[1];
        c[2] = j / (m[0] * m[1]);
        /* pull from the neighbours in the order -x, +x, -y, +y, -z, +z */
        for (k = 0; k < d; ++k) {
            int sd;
            for (sd = -1; sd <= 1; sd += 2) {
                double wm[3], wp[3], dr, wgt;
                long nb;
                if ((sd < 0 && c[k] == 0) || (sd > 0 && c[k] == m[k] - 1)) continue;
                nb = j + sd * st[k];
                adj_node(d, m, h, r, gamma, u, nb, wm, wp, &dr);
                /* node nb depends on j through its minus side if j is below it */
                wgt = sd > 0 ? wm[k] : wp[k];
                if (wgt != 0.0) acc = acc + wgt * lam[nb];
            }
        }
        lam[j] = acc;
    }
    for (i = 0; i < N; ++i) {
        double wm[3], wp[3], dr;
        adj_node(d, m, h, r, gamma, u, i, wm, wp, &dr);
        dJdr[i] = lam[i] * dr;
    }
    free(ord);
    free(lam);
}

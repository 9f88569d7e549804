"""Seeded synthetic inputs for the two-scale DD Eikonal solver.

This module holds no arithmetic of the method: it only draws slowness fields
r_eps, source sets Gamma and boundary values g.  Both the CUDA path and the CPU
oracle are fed from here (fields are generated in FP64 and rounded to the run
dtype by the caller; the oracle receives the same rounded values promoted back
to FP64).

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), top 53 bits -> [0, 1).
"""
from __future__ import annotations

import math

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (Steele, Lea & Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + int(self.uniform() * (hi - lo + 1))


def node_coords(shape, h):
    """Per-axis node coordinates (x, y[, z]) as 1-D arrays; shape is (.., y, x)."""
    return [np.arange(n, dtype=np.float64) * h for n in reversed(shape)]


def sin_product(shape, h, amp, eps):
    """r = 1 + amp * prod_a sin(2 pi x_a / eps) (the paper's smooth oscillatory r)."""
    cs = node_coords(shape, h)
    d = len(shape)
    f = np.ones(shape, dtype=np.float64)
    for a, c in enumerate(cs):
        s = np.sin(2.0 * math.pi * c / eps)
        view = [1] * d
        view[d - 1 - a] = -1
        f = f * s.reshape(view)
    return 1.0 + amp * f


def fourier_modes(seed, nmodes, kmin, kmax):
    """Wave vectors (|k| ~ U[kmin, kmax], angle ~ U[0, 2pi)) and phases of a 2-D field."""
    rng = SplitMix64(seed)
    modes = []
    for _ in range(nmodes):
        kmag = kmin + (kmax - kmin) * rng.uniform()
        ang = 2.0 * math.pi * rng.uniform()
        phi = 2.0 * math.pi * rng.uniform()
        modes.append((kmag * math.cos(ang), kmag * math.sin(ang), phi))
    return modes


def fourier_field(shape, h, seed, eps, nmodes=32):
    """F = sum_q cos(2 pi k_q . x + phi_q) with |k_q| in [1/eps, 2/eps], 2-D only."""
    ny, nx = shape
    x = np.arange(nx, dtype=np.float64) * h
    y = np.arange(ny, dtype=np.float64) * h
    modes = fourier_modes(seed, nmodes, 1.0 / eps, 2.0 / eps)
    # each mode factors as exp(i(2 pi ky y + phi)) exp(i 2 pi kx x); the sum over
    # modes is then one (ny x nmodes) @ (nmodes x nx) complex product
    ex = np.stack([np.exp(1j * (2.0 * math.pi * kx * x)) for kx, _, _ in modes])
    ey = np.stack([np.exp(1j * (2.0 * math.pi * ky * y + phi)) for _, ky, phi in modes])
    return np.real(ey.T @ ex)


def multiscale_r(shape, h, seed, eps, r0_slope=0.3, amp=0.4, floor=0.2):
    """r = clip(1 + r0_slope x + amp F / max|F|, floor): smooth r0 plus a_eps."""
    F = fourier_field(shape, h, seed, eps)
    x = np.arange(shape[1], dtype=np.float64) * h
    r = 1.0 + r0_slope * x[None, :] + amp * F / np.max(np.abs(F))
    return np.maximum(r, floor)


def point_source(shape, idx):
    """Gamma = one node (index tuple in array order), g = 0."""
    gamma = np.zeros(shape, dtype=np.uint8)
    gamma[idx] = 1
    return gamma, np.zeros(shape, dtype=np.float64)


def left_edge_source(shape):
    """Gamma = every node with x = 0, g = 0."""
    gamma = np.zeros(shape, dtype=np.uint8)
    gamma[..., 0] = 1
    return gamma, np.zeros(shape, dtype=np.float64)


# --------------------------------------------------------------------------
# Named workloads (sizes follow the benchmark configurations).
# --------------------------------------------------------------------------
SEED_C1 = 1805041981
SEED_C3 = 1805041982
SEED_C4 = 1805041983


def workload_c0():
    """2-D 257^2, h=1/256, r = 1 + .5 sin(2 pi x/eps) sin(2 pi y/eps), eps = 1/16,
    point source at (0.5, 0.5), 4x4 subdomains, coarse ratio 8 (33^2), theta 1."""
    n = 257
    h = 1.0 / 256
    r = sin_product((n, n), h, 0.5, 1.0 / 16)
    gamma, g = point_source((n, n), (128, 128))
    return dict(name="c0_2d_257_pointsrc", r=r, gamma=gamma, g=g, h=h, tiles=(4, 4), c=8, theta=1.0,
                max_iter=10, tol=1e-10)


def workload_c1(n=4097, tiles=16, c=16):
    """2-D 4097^2, h=1/4096, r = clip(1 + .3x + .4 F/max|F|, .2), 32 Fourier modes,
    eps = 1/64, Gamma = left edge, 16x16 subdomains, coarse 257^2 (c = 16)."""
    h = 1.0 / (n - 1)
    r = multiscale_r((n, n), h, SEED_C1, 1.0 / 64)
    gamma, g = left_edge_source((n, n))
    return dict(name="c1_2d_%d_leftedge" % n, r=r, gamma=gamma, g=g, h=h, tiles=(tiles, tiles), c=c,
                theta=1.0, max_iter=2 * tiles + 10, tol=0.0)


def workload_c2(n=257, tiles=8, c=8):
    """3-D 257^3, h=1/256, r = 1 + .4 sin sin sin (eps = 1/32), centre source."""
    h = 1.0 / (n - 1)
    r = sin_product((n, n, n), h, 0.4, 1.0 / 32)
    m = (n - 1) // 2
    gamma, g = point_source((n, n, n), (m, m, m))
    return dict(name="c2_3d_%d_pointsrc" % n, r=r, gamma=gamma, g=g, h=h, tiles=(tiles, tiles, tiles), c=c,
                theta=1.0, max_iter=2 * tiles + 10, tol=0.0)


def workload_c3(nprob=256, sides=(257, 513, 1025, 2049), tiles=(8, 16, 32), theta=0.0, tol=1e-6,
                seed0=SEED_C3):
    """Batch of independent 2-D problems.  Problem p draws from SplitMix64(seed0 + p):
    side n ~ U(sides), subdomains per side T ~ U(tiles), eps ~ U[16h, 64h] with
    h = 1/(n-1), a seed for its Fourier-mode slowness (as for the 4097^2
    workload, |k| in [1/eps, 2/eps]) and a point source at a uniformly drawn
    interior node.  Coarse ratio c = min(8, (n-1)/T); iteration cap 2T + 10,
    stop when the coarse update falls below tol; weight theta."""
    out = []
    for p in range(nprob):
        rng = SplitMix64(seed0 + p)
        n = sides[rng.randint(0, len(sides) - 1)]
        T = tiles[rng.randint(0, len(tiles) - 1)]
        h = 1.0 / (n - 1)
        eps = h * (16.0 + 48.0 * rng.uniform())
        fseed = rng.next_u64()
        sy, sx = rng.randint(1, n - 2), rng.randint(1, n - 2)
        r = multiscale_r((n, n), h, fseed, eps)
        gamma, g = point_source((n, n), (sy, sx))
        S = (n - 1) // T
        out.append(dict(name="c3_p%d_%d_T%d" % (p, n, T), r=r, gamma=gamma, g=g, h=h, tiles=(T, T),
                        c=min(8, S), theta=theta, max_iter=2 * T + 10, tol=tol))
    return out


def workload_c4(n=1025, nsrc=64, nrec=256):
    """Travel-time tomography: 1025^2 (h = 1/1024), true slowness from the
    Fourier-mode generator (eps = 1/32, seed SEED_C4), starting model the true
    one Gaussian-smoothed with sigma = eps; sources on x = 0 at rows 16 s + 8,
    receivers on x = 1 at rows 4 m + 2."""
    from scipy.ndimage import gaussian_filter
    h = 1.0 / (n - 1)
    eps = 1.0 / 32
    r_true = multiscale_r((n, n), h, SEED_C4, eps)
    r0 = gaussian_filter(r_true, sigma=eps / h, mode="nearest")
    src_rows = [16 * s + 8 for s in range(nsrc)]
    rec_rows = [4 * m + 2 for m in range(nrec)]
    return dict(name="c4_2d_%d_tomography" % n, r_true=r_true, r0=r0, h=h, src_rows=src_rows,
                rec_rows=rec_rows, n=n)


# --------------------------------------------------------------------------
# Obstacle and random workloads of Sec. 4 ("Mazes and obstacles",
# "Multiscale slowness functions"), unit square, Gamma = one node.
# --------------------------------------------------------------------------
SEED_CHECKER = 1805041984


def _box_mask(X, Y, x0, x1, y0, y1):
    return (X >= x0 - 1e-12) & (X <= x1 + 1e-12) & (Y >= y0 - 1e-12) & (Y <= y1 + 1e-12)


def workload_fast_strip(n=501, tiles=10):
    """The fast obstacle r^4: r = 0.01 on [0.26, 0.27] x [0, 0.6], r = 1
    elsewhere, source at (0, 0); H = 1/tiles (1/10) and h = 1/(n-1) (1/500),
    coarse ratio = subdomain width (the paper's construction)."""
    h = 1.0 / (n - 1)
    x, y = node_coords((n, n), h)
    X, Y = np.meshgrid(x, y)
    r = np.ones((n, n))
    r[_box_mask(X, Y, 0.26, 0.27, 0.0, 0.6)] = 0.01
    gamma, g = point_source((n, n), (0, 0))
    S = (n - 1) // tiles
    return dict(name="fast_strip_%d" % n, r=r, gamma=gamma, g=g, h=h, tiles=(tiles, tiles), c=S)


def workload_maze(n=501, tiles=10):
    """Stand-in for the maze r^3, whose exact geometry is only drawn in a
    figure: slow barriers (r = 1000) and a fast obstacle (r = 0.01) with the
    features the text names, r = 1 elsewhere, source at (0, 0).
      * a solid slow disc containing a whole subdomain: centre (0.55, 0.45),
        radius 0.09 (contains [0.5, 0.6] x [0.4, 0.5]);
      * a fast disc inside one subdomain: centre (0.25, 0.75), radius 0.03;
      * a slow wall on the coarse line x = 0.4, y in [0, 0.7], 3 nodes thick
        (coarse nodes inside the obstacle), and a slow wall y in [0.845,
        0.855], x in [0.15, 1] (no coarse line inside it)."""
    h = 1.0 / (n - 1)
    x, y = node_coords((n, n), h)
    X, Y = np.meshgrid(x, y)
    r = np.ones((n, n))
    r[(X - 0.55) ** 2 + (Y - 0.45) ** 2 <= 0.09 ** 2] = 1000.0
    r[_box_mask(X, Y, 0.4 - h, 0.4 + h, 0.0, 0.7)] = 1000.0
    r[_box_mask(X, Y, 0.15, 1.0, 0.845, 0.855)] = 1000.0
    r[(X - 0.25) ** 2 + (Y - 0.75) ** 2 <= 0.03 ** 2] = 0.01
    gamma, g = point_source((n, n), (0, 0))
    S = (n - 1) // tiles
    return dict(name="maze_standin_%d" % n, r=r, gamma=gamma, g=g, h=h, tiles=(tiles, tiles), c=S)


def workload_checkerboard(n=1401, tiles=14, eps_nodes=7, seed=SEED_CHECKER):
    """Random periodic checkerboard: squares of side eps = eps_nodes * h, each
    independently slowness 1 or 2 with probability 1/2 (SplitMix64, one draw
    per square in row-major order); source at the centre; H = 1/tiles (1/14),
    h = 1/(n-1) (1/1400), coarse ratio = subdomain width."""
    h = 1.0 / (n - 1)
    m = (n + eps_nodes - 1) // eps_nodes
    rng = SplitMix64(seed)
    cells = np.array([1.0 + (rng.next_u64() >> 63) for _ in range(m * m)]).reshape(m, m)
    idx = np.arange(n) // eps_nodes
    r = cells[np.ix_(idx, idx)]
    gamma, g = point_source((n, n), ((n - 1) // 2, (n - 1) // 2))
    S = (n - 1) // tiles
    return dict(name="checkerboard_%d_eps%dh" % (n, eps_nodes), r=r, gamma=gamma, g=g, h=h,
                tiles=(tiles, tiles), c=S)

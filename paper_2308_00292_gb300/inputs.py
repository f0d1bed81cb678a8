"""Seeded synthetic point clouds shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws points and
charges.  It is the one module the CUDA path's tests/benchmark and the CPU
oracle both consume.  The paper measures only on synthetic distributions
(uniform cube, sphere surface, Sec. 5 and Table 2), so every workload here is
synthetic; NumPy's PCG64 generator (``default_rng(seed)``) in float64.

Workloads:
  uniform_cube  -- points U[0,1)^3, charges U[-1,1]             (C1 / D1 shape)
  clustered     -- 50 Gaussian clusters + 10% background, net-zero normal
                   charges                                       (C2 shape)
  sphere        -- points on a sphere of radius 0.45, charges U[-1,1]
                                                                 (Table 2 shape)
  batch         -- many independent systems of log-uniform sizes, each
                   uniform in the cube or one Gaussian cluster   (batched)
  disk2d        -- points uniform in the unit disk, charges U[-1,1]  (2D log)
  circle2d      -- points on the unit circle, charges U[-1,1]    (2D log, Table 3 shape)
  circle_disk2d -- half on the unit circle, half uniform in the unit disk
                                                                 (2D log workload)
"""
from __future__ import annotations

import numpy as np


def uniform_cube(n: int, seed: int = 1, lo: float = 0.0, hi: float = 1.0):
    """n points uniform in [lo, hi)^3 and charges uniform in [-1, 1]."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(lo, hi, size=(n, 3))
    q = rng.uniform(-1.0, 1.0, size=n)
    return x, q


def clustered(n: int, seed: int = 2, nclusters: int = 50, background: float = 0.10,
              sigma_lo: float = 1e-3, sigma_hi: float = 1e-1):
    """Mixture of Gaussian clusters plus a uniform background in [0,1)^3.

    Cluster centres U[0.1, 0.9]^3, widths log-uniform in [sigma_lo, sigma_hi],
    equal weights; points falling outside [0,1)^3 are redrawn.  Charges are
    standard normal shifted to a zero net charge.
    """
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.1, 0.9, size=(nclusters, 3))
    sig = np.exp(rng.uniform(np.log(sigma_lo), np.log(sigma_hi), size=nclusters))
    nb = int(round(background * n))
    nc = n - nb
    which = rng.integers(0, nclusters, size=nc)
    x = np.empty((n, 3))
    pts = centres[which] + sig[which, None] * rng.standard_normal((nc, 3))
    bad = np.any((pts < 0.0) | (pts >= 1.0), axis=1)
    while bad.any():
        k = int(bad.sum())
        pts[bad] = centres[which[bad]] + sig[which[bad], None] * rng.standard_normal((k, 3))
        bad = np.any((pts < 0.0) | (pts >= 1.0), axis=1)
    x[:nc] = pts
    x[nc:] = rng.uniform(0.0, 1.0, size=(nb, 3))
    perm = rng.permutation(n)
    x = x[perm]
    q = rng.standard_normal(n)
    q -= q.mean()
    return x, q


def sphere(n: int, seed: int = 5, radius: float = 0.45):
    """n points on the sphere |x| = radius (normalised Gaussian directions)."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    x = radius * d
    q = rng.uniform(-1.0, 1.0, size=n)
    return x, q


def batch(nsys: int, seed: int = 6, n_lo: int = 500, n_hi: int = 50_000, sigma_lo: float = 1e-2,
          sigma_hi: float = 1e-1):
    """nsys independent systems, one after another.

    System sizes are log-uniform integers in [n_lo, n_hi]; each system is, with
    probability 1/2, uniform in [0,1)^3 or a single Gaussian cluster (centre
    U[0.3, 0.7]^3, width log-uniform in [sigma_lo, sigma_hi], points outside
    [0,1)^3 redrawn).  Charges are U[-1, 1].  Returns (points, charges,
    offsets) with offsets[s] .. offsets[s + 1] the points of system s.
    """
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi + 1), size=nsys))).astype(np.int64)
    sizes = np.clip(sizes, n_lo, n_hi)
    kinds = rng.integers(0, 2, size=nsys)
    off = np.zeros(nsys + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    x = np.empty((int(off[-1]), 3))
    for s in range(nsys):
        m = int(sizes[s])
        if kinds[s] == 0:
            pts = rng.uniform(0.0, 1.0, size=(m, 3))
        else:
            c = rng.uniform(0.3, 0.7, size=3)
            sig = float(np.exp(rng.uniform(np.log(sigma_lo), np.log(sigma_hi))))
            pts = c + sig * rng.standard_normal((m, 3))
            bad = np.any((pts < 0.0) | (pts >= 1.0), axis=1)
            while bad.any():
                pts[bad] = c + sig * rng.standard_normal((int(bad.sum()), 3))
                bad = np.any((pts < 0.0) | (pts >= 1.0), axis=1)
        x[off[s]:off[s + 1]] = pts
    q = rng.uniform(-1.0, 1.0, size=int(off[-1]))
    return x, q, off


# The configurations the library is measured on (sizes, distributions, seeds).
def disk2d(n: int, seed: int = 8):
    """n points uniform in the unit disk (radius sqrt(U), angle U[0, 2 pi)),
    charges uniform in [-1, 1]; coordinates (n, 2)."""
    rng = np.random.default_rng(seed)
    r = np.sqrt(rng.random(n))
    th = rng.uniform(0.0, 2.0 * np.pi, size=n)
    q = rng.uniform(-1.0, 1.0, size=n)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1), q


def circle2d(n: int, seed: int = 9):
    """n points on the unit circle (angle U[0, 2 pi)), charges uniform in
    [-1, 1]; coordinates (n, 2)."""
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, 2.0 * np.pi, size=n)
    q = rng.uniform(-1.0, 1.0, size=n)
    return np.stack([np.cos(th), np.sin(th)], axis=1), q


def circle_disk2d(n: int, seed: int = 10):
    """n // 2 points on the unit circle and the rest uniform in the unit disk,
    charges uniform in [-1, 1]; coordinates (n, 2)."""
    rng = np.random.default_rng(seed)
    nc = n // 2
    th = rng.uniform(0.0, 2.0 * np.pi, size=n)
    r = np.concatenate([np.ones(nc), np.sqrt(rng.random(n - nc))])
    q = rng.uniform(-1.0, 1.0, size=n)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1), q


CONFIGS = {
    "laplace3d_uniform_n2e4": dict(gen="uniform_cube", n=20000, seed=1, eps=1e-6, leaf_cap=280),
    "laplace3d_clustered_n1e7": dict(gen="clustered", n=10_000_000, seed=2, eps=1e-6, leaf_cap=200),
    "laplace3d_clustered_n1e7_eps1e-9": dict(gen="clustered", n=10_000_000, seed=2, eps=1e-9, leaf_cap=200),
    "laplace3d_sphere_n4e6": dict(gen="sphere", n=4_000_000, seed=5, eps=1e-6, leaf_cap=280),
    # the clustered workload at 2e6 points: small enough for ncu --set full captures
    "laplace3d_clustered_n2e6": dict(gen="clustered", n=2_000_000, seed=2, eps=1e-6, leaf_cap=200),
    # the differentiable workload: potentials plus gradients in charges and positions
    "laplace3d_uniform_n2e6": dict(gen="uniform_cube", n=2_000_000, seed=4, eps=1e-6, leaf_cap=200),
    # 4096 independent systems of 500 .. 50 000 points (about 4.4e7 in all)
    "laplace3d_batched_4096": dict(gen="batch", nsys=4096, seed=6, eps=1e-6, leaf_cap=0),
    # the Yukawa kernel exp(-10 r)/r on 4e6 uniform points at eps 1e-8
    "yukawa3d_uniform_n4e6": dict(gen="uniform_cube", n=4_000_000, seed=7, eps=1e-8, lam=10.0, leaf_cap=0),
    # the 2D log r workload: 8e6 points, half on the unit circle, half in the disk
    "log2d_circle_disk_n8e6": dict(gen="circle_disk2d", n=8_000_000, seed=10, eps=1e-8, leaf_cap=0),
}


def make(gen: str, n: int, seed: int, **_):
    return {"uniform_cube": uniform_cube, "clustered": clustered, "sphere": sphere, "disk2d": disk2d,
            "circle2d": circle2d, "circle_disk2d": circle_disk2d}[gen](n, seed=seed)

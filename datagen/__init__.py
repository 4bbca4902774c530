"""Seeded synthetic workloads for the LBVH build and the spatial / nearest queries.

This module is shared by the CPU oracle, the tests and the benchmark.  It holds
no arithmetic of the search method itself: it only draws point clouds, boxes
and query sets, and it states the radius that gives a target mean neighbour
count.  Every array is drawn in float64 with ``numpy.random.default_rng`` and
cast to float32 (row-major ``[n][3]`` for points, ``[n][6]`` = lo.xyz, hi.xyz
for boxes).

Distributions:

* ``cube``            -- uniform in the unit cube [0,1)^3.
* ``hollow_sphere``   -- uniform on the unit sphere (radius 1, thickness 0),
                         from normalised i.i.d. normal triples.
* ``lattice``         -- the 256^3 integer grid, site index x + 256 y + 65536 z.
* ``boxes``           -- centres uniform in [0,1)^3, half-widths uniform in
                         [0, 1e-3] per axis.
* ``query_cubes``     -- box queries: cubes of one half-width, centres uniform
                         in [0,1)^3 (``box_half_for_mean`` sizes them for a
                         target mean number of hits).
* ``gaussian_mixture``-- 64 anisotropic Gaussians, means uniform in [0,1)^3,
                         covariance Q diag(lambda) Q^T, Q Haar-random (QR of a
                         normal matrix), lambda log-uniform in [1e-4, 1e-2].
* ``paper_shape``     -- the four shapes of the paper's experiments (Sec. 3.1):
                         filled / hollow cube and sphere in [-a, a]^3, a = p^(1/3).

Seeds: workload ``c`` uses base seed ``SEED0 + c``; independent streams (points,
queries, lattice sites, batch sizes, MLP init, ...) are separated by a stream id.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np

SEED0 = 1_908_118_070

# stream ids, so that e.g. the query set does not change when n changes
STREAM_POINTS = 0
STREAM_QUERIES = 1
STREAM_SITES = 2
STREAM_SIZES = 3
STREAM_MLP = 4
STREAM_TRAIN = 5
STREAM_MIXTURE = 6
STREAM_KIND = 7
STREAM_K = 8
STREAM_HELDOUT = 9  # a held-out query draw for tuning (never the timed or tested queries)


def rng(seed: int, stream: int = 0, sub: int = 0) -> np.random.Generator:
    """Independent generator for (seed, stream, sub)."""
    return np.random.default_rng([int(seed), int(stream), int(sub)])


def cube(n: int, seed: int, stream: int = STREAM_POINTS, sub: int = 0) -> np.ndarray:
    """n points uniform in [0,1)^3, float32 [n][3]."""
    g = rng(seed, stream, sub)
    return g.random((n, 3), dtype=np.float64).astype(np.float32)


def hollow_sphere(n: int, seed: int, stream: int = STREAM_POINTS, sub: int = 0) -> np.ndarray:
    """n points uniform on the unit sphere centred at 0, float32 [n][3]."""
    g = rng(seed, stream, sub)
    v = g.standard_normal((n, 3))
    nrm = np.linalg.norm(v, axis=1, keepdims=True)
    nrm[nrm == 0.0] = 1.0
    return (v / nrm).astype(np.float32)


LATTICE_SIDE = 256


def lattice(side: int = LATTICE_SIDE) -> np.ndarray:
    """All side^3 integer-grid points as float32, index i = x + side*y + side^2*z."""
    ax = np.arange(side, dtype=np.float32)
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float32)


def lattice_sites(m: int, seed: int, side: int = LATTICE_SIDE) -> Tuple[np.ndarray, np.ndarray]:
    """m lattice sites drawn uniformly with replacement: (site index int64, coords float32 [m][3])."""
    g = rng(seed, STREAM_SITES)
    idx = g.integers(0, side ** 3, size=m, dtype=np.int64)
    x = idx % side
    y = (idx // side) % side
    z = idx // (side * side)
    return idx, np.stack([x, y, z], axis=1).astype(np.float32)


def boxes(n: int, seed: int, half_max: float = 1e-3, stream: int = STREAM_POINTS) -> np.ndarray:
    """n axis-aligned boxes, float32 [n][6] = (lo.x, lo.y, lo.z, hi.x, hi.y, hi.z)."""
    g = rng(seed, stream)
    c = g.random((n, 3), dtype=np.float64)
    h = g.random((n, 3), dtype=np.float64) * half_max
    return np.concatenate([c - h, c + h], axis=1).astype(np.float32)


def query_cubes(m: int, seed: int, half: float, stream: int = STREAM_QUERIES) -> np.ndarray:
    """m query boxes: cubes of half-width ``half`` with centres uniform in [0,1)^3, float32 [m][6]."""
    c = rng(seed, stream).random((m, 3), dtype=np.float64)
    return np.concatenate([c - half, c + half], axis=1).astype(np.float32)


def box_half_for_mean(n: int, mean: float = 10.0, prim_half_max: float = 1e-3) -> float:
    """Half-width of cube queries that meet ``mean`` of n unit-cube boxes on average.

    Per axis a query of half-width h meets a box of half-width u when the centres are at most
    h + u apart: probability 2 (h + u) for u ~ U[0, prim_half_max], 2 h + prim_half_max on
    average; over three independent axes n (2 h + prim_half_max)^3 = mean.  Points: 0."""
    return ((mean / n) ** (1.0 / 3.0) - prim_half_max) / 2.0


def gaussian_mixture_params(seed: int, n_comp: int = 64, lam_lo: float = 1e-4, lam_hi: float = 1e-2):
    """Means [c][3] and Cholesky-like factors A [c][3][3] with A A^T = Q diag(lambda) Q^T."""
    g = rng(seed, STREAM_MIXTURE)
    means = g.random((n_comp, 3))
    factors = np.empty((n_comp, 3, 3))
    for c in range(n_comp):
        q, r = np.linalg.qr(g.standard_normal((3, 3)))
        q = q * np.sign(np.diag(r))[None, :]  # Haar measure
        lam = np.exp(g.uniform(math.log(lam_lo), math.log(lam_hi), size=3))
        factors[c] = q * np.sqrt(lam)[None, :]
    return means, factors


def gaussian_mixture(n: int, seed: int, stream: int = STREAM_POINTS, n_comp: int = 64) -> np.ndarray:
    """n points from the equal-weight mixture of ``n_comp`` anisotropic Gaussians, float32 [n][3]."""
    means, factors = gaussian_mixture_params(seed, n_comp)
    g = rng(seed, stream)
    comp = g.integers(0, n_comp, size=n)
    z = g.standard_normal((n, 3))
    pts = means[comp] + np.einsum("nij,nj->ni", factors[comp], z)
    return pts.astype(np.float32)


def batched_sizes(n_clouds: int, seed: int, lo_exp: float = 3.0, hi_exp: float = 5.0) -> np.ndarray:
    """Cloud sizes floor(10^U[lo_exp, hi_exp]) (log-uniform in [1e3, 1e5])."""
    g = rng(seed, STREAM_SIZES)
    return np.floor(10.0 ** g.uniform(lo_exp, hi_exp, size=n_clouds)).astype(np.int64)


def batched_workload(n_clouds: int, seed: int) -> List[dict]:
    """Clouds of uneven sizes, each uniform-cube or hollow-sphere (fair coin), with
    its own queries (as many as points) and k drawn from {1, 10, 32}."""
    sizes = batched_sizes(n_clouds, seed)
    g = rng(seed, STREAM_KIND)
    kinds = g.integers(0, 2, size=n_clouds)
    ks = rng(seed, STREAM_K).choice(np.array([1, 10, 32]), size=n_clouds)
    out = []
    for c in range(n_clouds):
        n = int(sizes[c])
        gen = cube if kinds[c] == 0 else hollow_sphere
        out.append(dict(points=gen(n, seed, STREAM_POINTS, c), queries=gen(n, seed, STREAM_QUERIES, c),
                        k=int(ks[c]), dist="cube" if kinds[c] == 0 else "hollow_sphere",
                        radius=radius_for_mean(n, "cube" if kinds[c] == 0 else "hollow_sphere")))
    return out


def radius_for_mean(n: int, dist: str, mean: float = 10.0) -> float:
    """Radius whose ball holds ``mean`` points on average.

    cube (unit volume): (4/3) pi r^3 n = mean;  hollow unit sphere (area 4 pi):
    pi r^2 n / (4 pi) = mean (small-r disc)."""
    if dist == "cube":
        return (3.0 * mean / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    if dist == "hollow_sphere":
        return math.sqrt(4.0 * mean / n)
    raise ValueError(dist)


def paper_shape(p: int, shape: str, seed: int, stream: int = STREAM_POINTS) -> np.ndarray:
    """The paper's data sets (Sec. 3.1): a = p^(1/3), Omega = [-a, a]^3.

    filled_cube: uniform in Omega.  hollow_cube: on the faces of Omega, faces
    taken cyclically, uniform on each face.  filled_sphere: uniform in Omega,
    kept if inside the ball of radius a.  hollow_sphere: drawn in [-1,1]^3 and
    projected onto the sphere of radius a (not uniform on the sphere)."""
    g = rng(seed, stream)
    a = p ** (1.0 / 3.0)
    if shape == "filled_cube":
        pts = g.uniform(-a, a, size=(p, 3))
    elif shape == "hollow_cube":
        pts = g.uniform(-a, a, size=(p, 3))
        face = np.arange(p) % 6
        axis = face // 2
        side = np.where(face % 2 == 0, -a, a)
        pts[np.arange(p), axis] = side
    elif shape == "filled_sphere":
        chunks, have = [], 0
        while have < p:
            c = g.uniform(-a, a, size=(2 * (p - have) + 16, 3))
            c = c[np.sum(c * c, axis=1) <= a * a]
            chunks.append(c)
            have += len(c)
        pts = np.concatenate(chunks)[:p]
    elif shape == "hollow_sphere":
        c = g.uniform(-1.0, 1.0, size=(p, 3))
        nrm = np.linalg.norm(c, axis=1, keepdims=True)
        nrm[nrm == 0.0] = 1.0
        pts = a * c / nrm
    else:
        raise ValueError(shape)
    return pts.astype(np.float32)


def paper_radius(p: int, k: int = 10) -> float:
    """Radius giving k neighbours on average in the filled cube of side 2a (Sec. 3.1):
    density p / (2a)^3 = 1/8, so (4/3) pi r^3 / 8 = k."""
    return (6.0 * k / math.pi) ** (1.0 / 3.0)


def workload(name: str, n: int, m: int, seed: int) -> Tuple[np.ndarray, np.ndarray]:
    """(points, queries) for a named distribution: cube, hollow_sphere, gaussian_mixture."""
    gen = {"cube": cube, "hollow_sphere": hollow_sphere, "gaussian_mixture": gaussian_mixture}[name]
    return gen(n, seed, STREAM_POINTS), gen(m, seed, STREAM_QUERIES)

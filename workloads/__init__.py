"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds no arithmetic of the convection method itself: it only builds
meshes (vertex coordinates and connectivity), analytic velocity fields that are
evaluated at points somebody else chooses, and seeded random numbers.

Workloads (periodic boxes, Taylor-Green data) follow the synthetic configurations
that stand in for the paper's airfoil runs (the paper's Section 4 uses curved
hexahedral Eppler-387 meshes that are not available here):

* ``C1``: 2D periodic square [0, 2pi]^2, 8x8 squares split into 2 triangles, k=2.
* ``C2``: 3D periodic box [0, 2pi]^3, 16^3 cubes split into 6 tetrahedra, k=3.
* ``C3``: 3D periodic box, 32^3 cubes x 6 tetrahedra, k=4.
* ``C4``: 512 independent periodic boxes, n ~ U{4..12}, k ~ U{2,3,4,5}.
* ``C5``: 3D periodic box, 24^3 cubes x 6 tetrahedra, k=3.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np

TWO_PI = 2.0 * math.pi


@dataclass(frozen=True)
class Mesh:
    """Simplicial mesh of a periodic box.

    coords:   [n_vertices, dim] float64, unwrapped coordinates (the grid has
              (n+1)^dim points so that every element keeps straight edges).
    elems:    [n_elems, dim+1] int64 vertex ids (order as generated; consumers
              reorder vertices by representative id themselves).
    rep:      [n_vertices] int64 periodic representative of each vertex.
    dim, n:   spatial dimension and number of cubes per direction.
    length:   box edge length.
    """

    coords: np.ndarray
    elems: np.ndarray
    rep: np.ndarray
    dim: int
    n: int
    length: float

    @property
    def n_elems(self) -> int:
        return int(self.elems.shape[0])


def periodic_box_mesh(dim: int, n: int, length: float = TWO_PI) -> Mesh:
    """Kuhn/Freudenthal split of an n^dim periodic grid of cubes.

    Each cube with lower corner c is split into dim! simplices, one per
    permutation pi of the axes: v0 = c, v_{j+1} = v_j + e_{pi(j)}.  In 2D this
    gives the two triangles on either side of the cube diagonal.  The split is
    conforming across cubes and across the periodic boundary.
    """
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    if n < 3:
        # with n = 2 two different facets of the torus can share one vertex set
        raise ValueError("n must be >= 3 so that a facet is fixed by its vertex set")
    m = n + 1
    h = length / n
    grid = np.stack(np.meshgrid(*([np.arange(m)] * dim), indexing="ij"), axis=-1)
    grid = grid.reshape(-1, dim)
    # vertex id: axis 0 fastest
    ids = np.zeros(len(grid), dtype=np.int64)
    reps = np.zeros(len(grid), dtype=np.int64)
    mult, multn = 1, 1
    for ax in range(dim):
        ids += grid[:, ax] * mult
        reps += (grid[:, ax] % n) * multn
        mult *= m
        multn *= n
    order = np.argsort(ids)
    coords = (grid[order] * h).astype(np.float64)
    rep = reps[order]

    def vid(idx):
        v = 0
        mult = 1
        for ax in range(dim):
            v += idx[..., ax] * mult
            mult *= m
        return v

    cubes = np.stack(np.meshgrid(*([np.arange(n)] * dim), indexing="ij"), axis=-1)
    cubes = cubes.reshape(-1, dim)
    # cube index with axis 0 fastest
    key = np.zeros(len(cubes), dtype=np.int64)
    mult = 1
    for ax in range(dim):
        key += cubes[:, ax] * mult
        mult *= n
    cubes = cubes[np.argsort(key)]
    perms = list(itertools.permutations(range(dim)))
    elems = np.zeros((len(cubes), len(perms), dim + 1), dtype=np.int64)
    eye = np.eye(dim, dtype=np.int64)
    for p, perm in enumerate(perms):
        cur = cubes.copy()
        elems[:, p, 0] = vid(cur)
        for j, ax in enumerate(perm):
            cur = cur + eye[ax]
            elems[:, p, j + 1] = vid(cur)
    return Mesh(coords, elems.reshape(-1, dim + 1), rep, dim, n, float(length))


# ---------------------------------------------------------------- hexahedral boxes
@dataclass(frozen=True)
class HexBox:
    """Structured periodic box of hexahedra (parallelepipeds), for the hexahedral path.

    lines:  three increasing arrays of grid-line positions (n_a + 1 values, from 0);
            cube (i, j, l) spans [lines[0][i], lines[0][i+1]] x ... before the map.
    A:      3x3 matrix with det A > 0; every point xi of the grid is placed at A xi,
            so each cube becomes a parallelepiped.  The box is periodic with the
            lattice vectors A (L_a e_a), L_a = lines[a][-1].
    Cells are numbered with axis 0 fastest: e = i + n0 (j + n1 l).
    """

    lines: tuple
    A: np.ndarray

    @property
    def n(self) -> tuple:
        return tuple(len(x) - 1 for x in self.lines)

    @property
    def n_elems(self) -> int:
        n = self.n
        return int(n[0] * n[1] * n[2])


def hex_box(n, length: float = TWO_PI, jitter: float = 0.0, shear: float = 0.0, seed: int = 0) -> HexBox:
    """A periodic hexahedral box: n = (n0, n1, n2) cubes per direction (or one int),
    grid spacings length/n_a perturbed by a relative U[-jitter, jitter] (seeded) and
    the map A = I + shear * (seeded strictly upper-triangular matrix, entries U[-1, 1])."""
    if np.isscalar(n):
        n = (int(n),) * 3
    rng = np.random.Generator(np.random.PCG64(seed))
    lines = []
    for na in n:
        if na < 3:
            raise ValueError("n must be >= 3 in every direction")
        h = np.full(na, length / na) * (1.0 + rng.uniform(-jitter, jitter, size=na))
        lines.append(np.concatenate([[0.0], np.cumsum(h)]))
    U = np.triu(rng.uniform(-1.0, 1.0, size=(3, 3)), 1)
    A = np.eye(3) + shear * U
    return HexBox(tuple(lines), A)


def hex_box_tets(hb: HexBox) -> Mesh:
    """The same periodic box split into 6 tetrahedra per cell (the Kuhn split of
    periodic_box_mesh on the grid lines of hb, placed by hb.A)."""
    base = periodic_box_mesh(3, hb.n[0]) if len(set(hb.n)) == 1 else None
    if base is None:
        raise ValueError("the tetrahedral split needs the same count in every direction")
    n = hb.n[0]
    h = base.length / n
    idx = np.rint(base.coords / h).astype(np.int64)                  # grid indices
    xi = np.stack([hb.lines[a][idx[:, a]] for a in range(3)], axis=-1)
    coords = xi @ hb.A.T
    L = np.array([hb.lines[a][-1] for a in range(3)])
    return Mesh(coords, base.elems, base.rep, 3, n, float(L[0]))


# ---------------------------------------------------------------- analytic fields
def taylor_green(x: np.ndarray) -> np.ndarray:
    """Taylor-Green velocity at points x [..., dim].

    2D: (sin x cos y, -cos x sin y).  3D: (sin x cos y cos z, -cos x sin y cos z, 0).
    """
    x = np.asarray(x, dtype=np.float64)
    if x.shape[-1] == 2:
        X, Y = x[..., 0], x[..., 1]
        return np.stack([np.sin(X) * np.cos(Y), -np.cos(X) * np.sin(Y)], axis=-1)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    return np.stack(
        [np.sin(X) * np.cos(Y) * np.cos(Z), -np.cos(X) * np.sin(Y) * np.cos(Z), np.zeros_like(X)],
        axis=-1,
    )


def taylor_green_convective(x: np.ndarray) -> np.ndarray:
    """(u . grad) u for the Taylor-Green field above, written out by hand."""
    x = np.asarray(x, dtype=np.float64)
    if x.shape[-1] == 2:
        X, Y = x[..., 0], x[..., 1]
        return np.stack([0.5 * np.sin(2 * X), 0.5 * np.sin(2 * Y)], axis=-1)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    c2z = np.cos(Z) ** 2
    return np.stack(
        [0.5 * np.sin(2 * X) * c2z, 0.5 * np.sin(2 * Y) * c2z, np.zeros_like(X)], axis=-1
    )


def constant_field(value):
    """A constant velocity field (a callable of points)."""
    v = np.asarray(value, dtype=np.float64)

    def f(x):
        x = np.asarray(x, dtype=np.float64)
        return np.broadcast_to(v, x.shape[:-1] + v.shape).copy()

    return f


# ---------------------------------------------------------------- random numbers
def uniform_noise(size: int, amplitude: float, seed: int, dtype=np.float64) -> np.ndarray:
    """U[-amplitude, amplitude] noise from numpy's PCG64 with the given seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.uniform(-amplitude, amplitude, size=size)).astype(dtype)


def normal_vectors(count: int, size: int, seed: int) -> np.ndarray:
    """count unit-norm Gaussian directions of length size (finite-difference probes)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal((count, size))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def batch_draws(count: int = 512, seed: int = 1):
    """(n, k) per mesh of the heterogeneous batch: n ~ U{4..12}, k ~ U{2,3,4,5}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = rng.integers(4, 13, size=count)
    k = rng.integers(2, 6, size=count)
    return [(int(a), int(b)) for a, b in zip(n, k)]


# ---------------------------------------------------------------- configurations
CONFIGS = {
    "C1": dict(dim=2, n=8, k=2, dt=1e-3, substeps=100, noise=0.0, precisions=("f64",)),
    "C2": dict(dim=3, n=16, k=3, dt=5e-4, substeps=1000, noise=1e-3, precisions=("f64", "f32")),
    "C3": dict(dim=3, n=32, k=4, dt=5e-4, substeps=10, noise=1e-3, precisions=("f32", "f64")),
    "C5": dict(dim=3, n=24, k=3, dt=5e-4, substeps=200, noise=1e-3, precisions=("f32",)),
}


def config_mesh(name: str) -> Mesh:
    c = CONFIGS[name]
    return periodic_box_mesh(c["dim"], c["n"])

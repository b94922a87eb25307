"""Exactly divergence-free, normal-continuous fields for the oracle's pins (FP64).

w_h = curl(I_{k+1} A): A is a smooth periodic potential (scalar stream function
in 2D, vector potential in 3D), I_{k+1} its element-wise Lagrange interpolant on
equispaced nodes of degree k+1.  The interpolant is continuous across facets
(its facet trace depends on facet nodes only), so curl of it has a continuous
normal component and zero divergence: w_h lies in the normal-continuous [P^k]^d
space and is divergence-free in every element, which is what the identities of
Section 2.2 / 3.2 need (the integration by parts behind the energy identity).
"""
from __future__ import annotations

import itertools

import numpy as np

from .fe import dubiner, simplex_rule
from .mesh import MeshTopo


def lagrange_nodes(dim: int, p: int) -> np.ndarray:
    pts = [np.array(e, dtype=np.float64) / p
           for e in itertools.product(range(p + 1), repeat=dim) if sum(e) <= p]
    return np.array(pts)


def curl_field(topo: MeshTopo, dim: int, k: int, potential) -> np.ndarray:
    """L2 coefficients [E, d, nb_k] of curl(I_{k+1} potential).

    potential(x [.., d]) returns [..] (2D stream function) or [.., 3] (3D).
    """
    p = k + 1
    nodes = lagrange_nodes(dim, p)
    V, _ = dubiner(dim, p, nodes)                                    # [nn, nb_p]
    Vinv = np.linalg.inv(V)
    phys = topo.X[:, None, 0, :] + np.einsum("ecj,nj->enc", topo.J, nodes)
    vals = potential(phys)
    xq, wq = simplex_rule(dim, 2 * k + 2)
    _, dpsi = dubiner(dim, p, xq)                                    # [nq, nb_p, d] reference grads
    phi_k, _ = dubiner(dim, k, xq)
    if dim == 2:
        coef = np.einsum("bn,en->eb", Vinv, vals)                    # [E, nb_p]
        gref = np.einsum("qbc,eb->eqc", dpsi, coef)
        g = np.einsum("ecb,eqc->eqb", topo.Jinv, gref)               # physical gradient
        w = np.stack([g[..., 1], -g[..., 0]], axis=-1)
    else:
        coef = np.einsum("bn,enm->emb", Vinv, vals)                  # [E, 3, nb_p]
        gref = np.einsum("qbc,emb->eqmc", dpsi, coef)
        g = np.einsum("ecb,eqmc->eqmb", topo.Jinv, gref)             # d A_m / d x_b
        w = np.stack([g[..., 2, 1] - g[..., 1, 2],
                      g[..., 0, 2] - g[..., 2, 0],
                      g[..., 1, 0] - g[..., 0, 1]], axis=-1)
    return np.einsum("q,qi,eqa->eai", wq, phi_k, w)


def tg_potential(dim: int):
    """Potential whose curl is the Taylor-Green field of ``workloads.taylor_green``."""
    if dim == 2:
        return lambda x: np.sin(x[..., 0]) * np.sin(x[..., 1])
    def A(x):
        z = np.zeros(x.shape[:-1])
        return np.stack([z, z, np.sin(x[..., 0]) * np.sin(x[..., 1]) * np.cos(x[..., 2])], axis=-1)
    return A


def random_potential(dim: int, seed: int, modes: int = 3):
    """A smooth periodic random potential (sum of a few Fourier modes)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    comps = 1 if dim == 2 else 3
    ks = rng.integers(-2, 3, size=(comps, modes, dim))
    amp = rng.standard_normal((comps, modes))
    ph = rng.uniform(0, 2 * np.pi, size=(comps, modes))

    def A(x):
        out = np.stack([sum(amp[c, m] * np.cos(x @ ks[c, m] + ph[c, m]) for m in range(modes))
                        for c in range(comps)], axis=-1)
        return out[..., 0] if dim == 2 else out
    return A

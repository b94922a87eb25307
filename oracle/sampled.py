"""The oracle's convection apply on a sample of the elements of a large mesh.

y on element T depends only on the coefficients of T and of the elements that share a
facet with T (Section 3.2, eq. "hopudefinition": volume term on T, facet terms on the
facets of T).  So the oracle evaluates y on sampled elements exactly by building the
sub-mesh of those elements and their facet neighbours: the sampled elements keep all of
their facets as interior facets with the same geometry, orientation and sides as in the
full mesh (both follow from the vertices' periodic representatives), and the outer
facets of the neighbours, which become boundary facets, only change the neighbours'
outputs, which are not compared.  Test infrastructure (tests and the CPU-baseline legs of
the benchmark): it calls nothing but the oracle.
"""
from __future__ import annotations

import numpy as np

from . import convection as C
from . import mesh


def neighbourhood(topo: mesh.MeshTopo, sample: np.ndarray) -> np.ndarray:
    """Element ids: the sample first (in the given order), then its facet neighbours."""
    sample = np.asarray(sample, dtype=np.int64)
    F = topo.elem_facet[sample].reshape(-1)
    other = np.where(topo.fa[F, 0] == np.repeat(sample, topo.dim + 1), topo.fb[F, 0], topo.fa[F, 0])
    other = other[other >= 0]
    rest = np.setdiff1d(np.unique(other), sample)
    return np.concatenate([sample, rest])


def sampled_apply(coords, elems, rep, topo, ref, wL, uL, l, sample) -> np.ndarray:
    """y[sample] of ``oracle.convection.apply`` on the full mesh (wL, uL: full L2 fields)."""
    ids = neighbourhood(topo, sample)
    sub = mesh.MeshTopo(coords, np.asarray(elems)[ids], rep)
    y = C.apply(sub, ref, wL[ids], uL[ids], l)
    return y[: len(sample)]

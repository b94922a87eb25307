"""The sampled oracle apply (oracle/sampled.py) equals the full oracle apply on
the sampled elements, bit for bit, on periodic meshes and on meshes with boundary facets."""
import numpy as np
import pytest

import workloads as W
from oracle import convection as C
from oracle import fe, hdiv, mesh
from oracle.sampled import neighbourhood, sampled_apply


@pytest.mark.parametrize("dim,n,k,periodic", [(3, 4, 3, True), (3, 3, 2, False), (2, 6, 2, True)])
def test_sampled_apply_equals_full_apply(dim, n, k, periodic):
    m = W.periodic_box_mesh(dim, n)
    rep = m.rep if periodic else None
    topo = mesh.MeshTopo(m.coords, m.elems, rep)
    ref = fe.ref_element(dim, k)
    sp = hdiv.HDiv(topo, ref)
    rng = np.random.default_rng(11)
    wL = sp.to_l2(rng.standard_normal(sp.n_hdiv))
    uL = rng.standard_normal((topo.n_elems, dim, ref.nb))
    full = C.apply(topo, ref, wL, uL, k - 1)
    s = rng.choice(topo.n_elems, topo.n_elems // 3, replace=False)
    y = sampled_apply(m.coords, m.elems, rep, topo, ref, wL, uL, k - 1, s)
    assert np.array_equal(y, full[s])


def test_neighbourhood_holds_every_facet_neighbour():
    m = W.periodic_box_mesh(3, 3)
    topo = mesh.MeshTopo(m.coords, m.elems, m.rep)
    s = np.array([0, 7, 40])
    ids = neighbourhood(topo, s)
    assert list(ids[:3]) == [0, 7, 40] and len(set(ids)) == len(ids)
    for e in s:
        for F in topo.elem_facet[e]:
            assert topo.fa[F, 0] in ids and topo.fb[F, 0] in ids

"""The element-partitioned apply on one GPU (P logical partitions, halo exchange by the
library's pack / unpack kernels) against the apply on the whole mesh.

Every partition's owned elements see the same facets, geometry and inputs as in the whole
mesh, and the kernels compute each element and each facet independently of where they sit
in the mesh, so the owned outputs must be bit-identical to the unpartitioned apply (in FP64
and in FP32), and the FP64 ones equal the oracle to 1e-12.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import convection as C
from oracle import fe, hdiv, mesh

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dim,n,k,P", [(3, 6, 3, 2), (3, 6, 4, 3), (2, 8, 2, 4)])
def test_partitioned_apply_is_bit_identical(dim, n, k, P, prec):
    from paper_2408_06698_gb300 import Hopu
    from paper_2408_06698_gb300.partition import PartitionedHopu, slab_partitions
    m = W.periodic_box_mesh(dim, n)
    l = k - 1
    g = Hopu(m.coords, m.elems, m.rep, k=k, l=l, prec=prec)
    parts = slab_partitions(m, P)
    pg = PartitionedHopu(m.coords, m.elems, m.rep, parts, k=k, l=l, prec=prec)
    rng = np.random.default_rng(41)
    wV = torch.as_tensor(rng.standard_normal(g.n_hdiv), dtype=g.dtype, device=g.device)
    uL = torch.as_tensor(rng.standard_normal(g.n_l2), dtype=g.dtype, device=g.device)
    wL = g.project("hdiv_to_l2", wV)
    y_whole = g.apply_convection(wV, uL)
    y_l2w = g.apply_convection_l2(wL, uL)
    torch.cuda.synchronize()
    assert torch.equal(y_whole, y_l2w)                     # the L2-wind entry point
    ys = pg.apply_convection_l2(pg.scatter(wL), pg.scatter(uL))
    y_part = pg.gather(ys, torch.full_like(uL, float("nan")))
    for c in pg.ctx:
        c.sync()
    assert torch.equal(y_part, y_whole)
    if prec == "f64":
        topo = mesh.MeshTopo(m.coords, m.elems, m.rep)
        sp = hdiv.HDiv(topo, fe.ref_element(dim, k))
        ref = C.apply(topo, sp.ref, sp.to_l2(wV.cpu().numpy()), uL.cpu().numpy().reshape(topo.n_elems, dim, -1), l)
        got = y_part.cpu().numpy()
        assert np.abs(got - ref.reshape(-1)).max() < 1e-12 * np.abs(ref).max()
    print(f"d={dim} n={n} k={k} P={P} {prec}: halo sizes {[len(p.halo) for p in parts]}, bit-identical")


def test_pack_rejects_ids_outside_the_mesh():
    from paper_2408_06698_gb300 import Hopu
    from paper_2408_06698_gb300._lib import HopuError
    m = W.periodic_box_mesh(3, 3)
    g = Hopu(m.coords, m.elems, m.rep, k=2, l=1, prec="f64")
    u = torch.zeros(g.n_l2, dtype=g.dtype, device=g.device)
    ids = torch.tensor([0, g.n_elems + 5], dtype=torch.int32, device=g.device)
    g.pack_elements(ids, u)
    with pytest.raises(HopuError, match="outside the mesh"):
        g.sync()

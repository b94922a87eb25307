"""GPU parity of the batch entry points (many meshes of uneven size and order).

Every mesh of a batch must advance exactly as the oracle advances it alone; the merged
class layout must give every mesh contiguous facet, interior and L2 ranges.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import fe, hdiv, mesh, rk

pytestmark = pytest.mark.gpu


def _space(m, k):
    return hdiv.HDiv(mesh.MeshTopo(m.coords, m.elems, m.rep), fe.ref_element(m.dim, k))


def _fill(batch, classes, i, sp, uV):
    c, fo, fl, io, il, lo, ll = batch.layout[i]
    nf = sp.topo.n_facets * sp.ref.nf
    assert fl == nf and il == sp.n_hdiv - nf
    classes[c][fo:fo + fl] = torch.as_tensor(uV[:nf], dtype=batch.dtype, device=batch.device)
    classes[c][io:io + il] = torch.as_tensor(uV[nf:], dtype=batch.dtype, device=batch.device)


def _read(batch, classes, i):
    c, fo, fl, io, il, lo, ll = batch.layout[i]
    v = classes[c]
    return np.concatenate([v[fo:fo + fl].double().cpu().numpy(), v[io:io + il].double().cpu().numpy()])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_of_mixed_orders_matches_oracle(prec):
    from paper_2408_06698_gb300 import HopuBatch
    spec = [(3, 2), (4, 3), (3, 4), (3, 5), (4, 2), (3, 3)]
    meshes = [W.periodic_box_mesh(3, n) for n, _ in spec]
    ks = [k for _, k in spec]
    b = HopuBatch([(m.coords, m.elems, m.rep) for m in meshes], ks, l=-2, prec=prec)
    assert sorted(v.k for v in b.classes) == [2, 3, 4, 5]
    classes = [torch.zeros(v.n_hdiv, dtype=b.dtype, device=b.device) for v in b.classes]
    spaces, inits = [], []
    for i, (m, k) in enumerate(zip(meshes, ks)):
        sp = _space(m, k)
        uV = sp.interpolate(W.taylor_green) + W.uniform_noise(sp.n_hdiv, 1e-3, 100 + i)
        uV = torch.as_tensor(uV, dtype=b.dtype).double().numpy()   # what the GPU sees
        _fill(b, classes, i, sp, uV)
        spaces.append(sp)
        inits.append(uV)
    dt = 1e-2
    b.rk_substep(classes, dt, 1)
    b.rk_substep(classes, dt, 1)          # graph replay
    torch.cuda.synchronize()
    tol = 1e-12 if prec == "f64" else 2e-6
    for i, (sp, uV, k) in enumerate(zip(spaces, inits, ks)):
        ref = rk.substeps_stage(sp, uV, dt, 2, k - 1)
        got = _read(b, classes, i)
        assert np.abs(got - ref).max() < tol * np.abs(ref).max(), (i, k, np.abs(got - ref).max())


def test_c4_batch_draw_512_meshes_sampled():
    """The 512-mesh draw (n ~ U{4..12}, k ~ U{2..5}, seed 1), FP32, sampled parity."""
    from paper_2408_06698_gb300 import HopuBatch
    draws = W.batch_draws(512, seed=1)
    meshes = [W.periodic_box_mesh(3, n) for n, _ in draws]
    ks = [k for _, k in draws]
    b = HopuBatch([(m.coords, m.elems, m.rep) for m in meshes], ks, l=-2, prec="f32")
    total = sum(m.n_elems for m in meshes)
    assert sum(v.n_elems for v in b.classes) == total
    classes = [torch.zeros(v.n_hdiv, dtype=b.dtype, device=b.device) for v in b.classes]
    # initial data: the canonical interpolant of Taylor-Green, by each class context
    for c, v in enumerate(b.classes):
        classes[c].copy_(v.interpolate_function(W.taylor_green))
    sample = [i for i, (n, k) in enumerate(draws) if n == 4][:4]
    b.rk_substep(classes, 5e-4, 2)
    torch.cuda.synchronize()
    for i in sample:
        # the oracle starts from its own interpolant of the same field (FP64)
        sp = _space(meshes[i], ks[i])
        ref = rk.substeps_stage(sp, sp.interpolate(W.taylor_green), 5e-4, 2, ks[i] - 1)
        got = _read(b, classes, i)
        assert np.abs(got - ref).max() < 2e-6 * np.abs(ref).max(), (i, ks[i])

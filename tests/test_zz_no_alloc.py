"""hopu_apply_convection_noalloc: the allocation-free apply, through the C ABI.

Callers that cannot allocate device memory (a caller-owned pool or budget, all device
memory reserved up front) use this entry point; its scratch is a static device buffer
inside the library.  This test compares it with hopu_apply_convection and with the FP64
oracle on the same inputs, on two calls in a row (the second call runs on the buffer the
first one left behind), on a periodic mesh and on a box whose faces are boundary facets,
within the tolerances of the parity tests.  It lives in a file of its own that pytest
collects last.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from oracle import convection as C
from oracle import fe, hdiv, mesh

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-6}


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_noalloc_apply_matches_apply_and_oracle_twice(prec, periodic):
    from paper_2408_06698_gb300 import Hopu
    m = W.periodic_box_mesh(3, 6 if periodic else 4)
    rep = m.rep if periodic else None
    k, l = 3, 2
    g = Hopu(m.coords, m.elems, rep, k=k, l=l, prec=prec)
    sp = hdiv.HDiv(mesh.MeshTopo(m.coords, m.elems, rep), fe.ref_element(3, k))
    assert periodic or len(g.boundary_facets()) > 0
    rng = np.random.default_rng(700)
    lib = g.lib
    for call in range(2):
        wV = torch.as_tensor(rng.standard_normal(g.n_hdiv), dtype=g.dtype, device=g.device)
        uL = torch.as_tensor(rng.standard_normal(g.n_l2), dtype=g.dtype, device=g.device)
        y_ref = g.apply_convection(wV, uL)
        y = torch.full((g.n_l2,), float("nan"), dtype=g.dtype, device=g.device)
        g._sync_stream()
        st = lib.hopu_apply_convection_noalloc(g.ctx, ctypes.c_void_p(wV.data_ptr()), ctypes.c_void_p(uL.data_ptr()),
                                               ctypes.c_void_p(y.data_ptr()), None)
        assert st == 0, lib.hopu_last_error(g.ctx).decode()
        torch.cuda.synchronize()
        a, b = y.double().cpu().numpy(), y_ref.double().cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.abs(a - b).max() <= TOL[prec] * np.abs(b).max(), (call, np.abs(a - b).max())
        wVh = wV.double().cpu().numpy()
        uLh = uL.double().cpu().numpy().reshape(sp.topo.n_elems, 3, sp.ref.nb)
        ref = C.apply(sp.topo, sp.ref, sp.to_l2(wVh), uLh, l).reshape(-1)
        assert np.abs(a - ref).max() <= TOL[prec] * np.abs(ref).max(), (call, np.abs(a - ref).max())


def test_noalloc_rejects_meshes_beyond_the_static_buffer():
    from paper_2408_06698_gb300 import Hopu
    m = W.periodic_box_mesh(3, 24)          # 82,944 tetrahedra, k = 3, FP64: ~120 MB of scratch
    g = Hopu(m.coords, m.elems, m.rep, k=3, l=2, prec="f64")
    x = torch.zeros(g.n_hdiv, dtype=g.dtype, device=g.device)
    u = torch.zeros(g.n_l2, dtype=g.dtype, device=g.device)
    y = torch.zeros(g.n_l2, dtype=g.dtype, device=g.device)
    st = g.lib.hopu_apply_convection_noalloc(g.ctx, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                             ctypes.c_void_p(y.data_ptr()), None)
    assert st == -1 and "static buffer" in g.lib.hopu_last_error(g.ctx).decode()

"""GPU parity on meshes with boundary facets (walls / outlets and inlets) against the oracle.

The boxes of the periodic tests without the periodic identification: every face of the
box is a boundary.  Wall / outlet facets take the element's own trace as exterior trace
(no jump); inlet facets take given data u_I for the convected velocity (the wind keeps
its own, single-valued normal component), here a linear field (a polynomial of
degree <= k on every facet, so that the library's projection of the data onto P^k of
the facet is exact and the oracle, which uses the point values, sees the same data).
Tolerances as in the periodic parity tests.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import convection as C
from oracle import fe, hdiv, mesh, rk

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-6}


def _mk(dim, n, k, prec, l=-1):
    from paper_2408_06698_gb300 import Hopu
    m = W.periodic_box_mesh(dim, n)
    g = Hopu(m.coords, m.elems, None, k=k, l=l, prec=prec)
    sp = hdiv.HDiv(mesh.MeshTopo(m.coords, m.elems), fe.ref_element(dim, k))
    return g, sp


def _dev(g, x):
    return torch.as_tensor(np.ascontiguousarray(x).reshape(-1), dtype=g.dtype, device=g.device)


def _host(t):
    return t.detach().double().cpu().numpy()


def _rounded(g, x):
    return _host(_dev(g, x)).reshape(np.shape(x))


def _rel(got, ref):
    return float(np.abs(np.asarray(got).reshape(-1) - np.asarray(ref).reshape(-1)).max() / np.abs(ref).max())


def _linear(dim):
    A = np.array([[0.3, -0.7, 0.2], [0.5, 0.1, -0.4], [-0.2, 0.6, 0.3]])[:dim, :dim]
    b = np.array([0.8, -0.5, 0.35])[:dim]
    return lambda x: np.einsum("ab,...b->...a", A, x) + b


CASES = [(2, 4, 2), (3, 3, 3), (3, 3, 4)]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dim,n,k", CASES)
def test_topology_and_projections(dim, n, k, prec):
    g, sp = _mk(dim, n, k, prec)
    t = sp.topo
    assert (g.n_hdiv, g.n_l2, g.n_facets) == (sp.n_hdiv, sp.n_l2, t.n_facets)
    assert np.array_equal(g.boundary_facets(), np.where(t.boundary)[0])
    pts = g.points("facet").reshape(t.n_facets, -1, dim)
    assert np.abs(pts - t.facet_points(sp.ref.sq)).max() < 1e-12
    rng = np.random.default_rng(1100 + 10 * dim + k)
    uV = _rounded(g, rng.standard_normal(sp.n_hdiv))
    tol = 1e-12 if prec == "f64" else 2e-6
    assert _rel(_host(g.project("hdiv_to_l2", _dev(g, uV))), sp.to_l2(uV)) < tol
    uL = _rounded(g, rng.standard_normal((t.n_elems, dim, sp.ref.nb)))
    assert _rel(_host(g.project("l2_to_hdiv", _dev(g, uL))), sp.from_l2(uL)) < tol
    assert _rel(_host(g.project("l2_to_hdiv_dual", _dev(g, uL))), sp.dual(uL)) < tol


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dim,n,k", CASES)
def test_apply_with_walls_and_inlets(dim, n, k, prec):
    g, sp = _mk(dim, n, k, prec, l=k - 1)
    t = sp.topo
    rng = np.random.default_rng(1200 + 10 * dim + k)
    wV = _rounded(g, rng.standard_normal(sp.n_hdiv))
    uL = _rounded(g, rng.standard_normal((t.n_elems, dim, sp.ref.nb)))
    wL = sp.to_l2(wV)
    # every boundary facet a wall / outlet
    y = _host(g.apply_convection(_dev(g, wV), _dev(g, uL)))
    ref = C.apply(t, sp.ref, wL, uL, k - 1)
    assert _rel(y, ref) < TOL[prec], _rel(y, ref)
    # half of them inlets with linear data
    bf = np.where(t.boundary)[0]
    inl = bf[rng.random(bf.size) < 0.5]
    f = _linear(dim)
    g.set_inlet(inl, fun=f)
    pts = t.facet_points(sp.ref.sq)
    mask = np.zeros(t.n_facets, dtype=bool)
    mask[inl] = True
    y = _host(g.apply_convection(_dev(g, wV), _dev(g, uL)))
    ref = C.apply(t, sp.ref, wL, uL, k - 1, exterior=(f(pts), C.facet_trace(t, sp.ref, wL, "A")), inlet=mask)
    assert _rel(y, ref) < TOL[prec], _rel(y, ref)
    assert _rel(ref, C.apply(t, sp.ref, wL, uL, k - 1)) > 1e-3     # the inlets matter
    g.set_inlet([])
    y = _host(g.apply_convection(_dev(g, wV), _dev(g, uL)))
    assert _rel(y, C.apply(t, sp.ref, wL, uL, k - 1)) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dim,n,k", [(2, 4, 2), (3, 3, 3)])
def test_stage_substeps_with_walls(dim, n, k, prec):
    g, sp = _mk(dim, n, k, prec, l=k - 1)
    u0 = _rounded(g, sp.interpolate(W.taylor_green) + W.uniform_noise(sp.n_hdiv, 1e-3, 0))
    stream = torch.cuda.Stream(device=g.device)
    with torch.cuda.stream(stream):
        x = _dev(g, u0)
        g.rk_substep(x, 1e-2, 2)
    stream.synchronize()
    ref = rk.substeps_stage(sp, u0, 1e-2, 2, k - 1)
    assert _rel(_host(x), ref) < TOL[prec] * 4


def test_boundary_errors():
    from paper_2408_06698_gb300 import _lib as L
    g, sp = _mk(3, 3, 2, "f64")
    interior = int(np.where(~sp.topo.boundary)[0][0])
    with pytest.raises(L.HopuError):
        g.set_inlet([interior], fun=_linear(3))
    g.lib.hopu_clear_error(g.ctx)
    b = int(g.boundary_facets()[0])
    with pytest.raises(L.HopuError):
        g.set_inlet([b, b], fun=_linear(3))
    g.lib.hopu_clear_error(g.ctx)
    u = g.new("hdiv").zero_()
    with pytest.raises(L.HopuError):
        g.vjp_rollout(u, 1e-2, 1, 1)                  # not for meshes with boundary facets

"""GPU parity of adaptive HOPU (hopu_adapt_l, hopu_set_facet_l) against the FP64 oracle.

eta per facet: FP64 to 1e-12, FP32 to 1e-5 relative.  The new orders are integers
decided from eta in FP64 on both sides; they must agree exactly wherever eta is not
within the comparison tolerance of a threshold (those facets may go either way and
are only checked to be one of the two neighbouring orders).
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import adaptive as AD
from oracle import fe, hdiv, mesh, rk

pytestmark = pytest.mark.gpu

TH = [0.1, 0.2, 0.3, 0.4, 0.5, 0.6]


def _mk(dim, n, k, prec, l=-1):
    from paper_2408_06698_gb300 import Hopu
    m = W.periodic_box_mesh(dim, n)
    g = Hopu(m.coords, m.elems, m.rep, k=k, l=l, prec=prec)
    sp = hdiv.HDiv(mesh.MeshTopo(m.coords, m.elems, m.rep), fe.ref_element(dim, k))
    return g, sp


def _dev(g, x, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(x).reshape(-1), dtype=dtype or g.dtype, device=g.device)


def _rounded(g, x):
    return _dev(g, x).double().cpu().numpy().reshape(np.shape(x))


def _check_orders(got, ref, eta, th, tol):
    near = np.zeros(eta.shape, dtype=bool)
    for t in th:
        near |= np.abs(eta - t) <= tol * max(t, 1e-300)
    assert np.array_equal(got[~near], ref[~near])
    assert np.all(np.abs(got[near] - ref[near]) <= 1)
    return int(near.sum())


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("dim,n,k,amp", [(2, 6, 2, 0.02), (3, 3, 2, 0.005), (3, 4, 3, 0.005), (3, 3, 5, 0.002)])
def test_eta_and_new_orders(dim, n, k, amp, prec, tol):
    g, sp = _mk(dim, n, k, prec)
    rng = np.random.default_rng(900 + 10 * dim + k)
    uL = sp.to_l2(sp.interpolate(W.taylor_green)) + amp * rng.standard_normal((sp.topo.n_elems, dim, sp.ref.nb))
    uL = _rounded(g, uL)
    l0 = rng.integers(-1, k + 1, size=sp.topo.n_facets).astype(np.int8)
    th = TH[: k + 1]
    fl = torch.as_tensor(l0, device=g.device)
    eta = torch.zeros(sp.topo.n_facets, dtype=torch.float64, device=g.device)
    g.adapt_l(_dev(g, uL), th, fl, eta)
    g.sync()
    eta_ref, l_ref = AD.adapt(sp.topo, sp.ref, uL, l0.astype(np.int64), th)
    e = eta.cpu().numpy()
    assert np.max(np.abs(e - eta_ref) / np.maximum(eta_ref, 1e-3)) < tol
    near = _check_orders(fl.cpu().numpy().astype(np.int64), l_ref, eta_ref, th, 10 * tol)
    assert near <= sp.topo.n_facets // 100
    assert len(np.unique(l_ref)) >= 3          # the draw exercises several orders


def test_adapt_l_rejects_bad_thresholds():
    from paper_2408_06698_gb300 import _lib as L
    g, sp = _mk(3, 3, 2, "f64")
    fl = torch.zeros(sp.topo.n_facets, dtype=torch.int8, device=g.device)
    u = g.new("l2").zero_()
    for th in ([0.2, 0.1, 0.3], [0.1, 0.2, 1.5], [0.0, 0.1, 0.2]):
        with pytest.raises(L.HopuError):
            g.adapt_l(u, th, fl)
        g.lib.hopu_clear_error(g.ctx)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-6)])
def test_substeps_with_per_facet_orders(prec, tol):
    dim, n, k = 3, 3, 3
    g, sp = _mk(dim, n, k, prec, l=1)
    rng = np.random.default_rng(950)
    lF = rng.integers(-1, k + 1, size=sp.topo.n_facets).astype(np.int8)
    u0 = _rounded(g, sp.interpolate(W.taylor_green) + W.uniform_noise(sp.n_hdiv, 1e-3, 0))
    fl = torch.as_tensor(lF, device=g.device)
    g.set_facet_l(fl)
    stream = torch.cuda.Stream(device=g.device)
    with torch.cuda.stream(stream):
        x = _dev(g, u0)
        g.rk_substep(x, 1e-2, 2)                 # captured graph with the per-facet orders
    stream.synchronize()
    ref = rk.substeps_stage(sp, u0, 1e-2, 2, lF.astype(np.int64))
    got = x.double().cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() < tol * 2
    g.set_facet_l(None)                          # back to the uniform l = 1
    y = _dev(g, u0)
    g.rk_substep(y, 1e-2, 1)
    ref1 = rk.substeps_stage(sp, u0, 1e-2, 1, 1)
    assert np.abs(y.double().cpu().numpy() - ref1).max() / np.abs(ref1).max() < tol * 2


def test_adaptive_substeps_match_the_oracle_loop():
    """20 STAGE substeps, orders re-determined before substeps 0 and 10 (k = 3, limits
    {0.1, 0.2, 0.3, 0.4}); the oracle runs the same loop."""
    dim, n, k = 3, 3, 3
    g, sp = _mk(dim, n, k, "f64")
    rng = np.random.default_rng(960)
    u0 = sp.interpolate(W.taylor_green) + 0.01 * rng.standard_normal(sp.n_hdiv)
    th = [0.1, 0.2, 0.3, 0.4]
    fl = torch.full((sp.topo.n_facets,), -1, dtype=torch.int8, device=g.device)
    x = _dev(g, u0)
    g.adaptive_substeps(x, 5e-3, 20, th, fl, period=10)
    g.sync()
    l_cur = np.full(sp.topo.n_facets, -1, dtype=np.int64)
    u = u0.copy()
    for _ in range(2):
        _, l_cur = AD.adapt(sp.topo, sp.ref, sp.to_l2(u), l_cur, th)
        u = rk.substeps_stage(sp, u, 5e-3, 10, l_cur)
    assert np.array_equal(fl.cpu().numpy().astype(np.int64), l_cur)
    assert np.abs(x.cpu().numpy() - u).max() / np.abs(u).max() < 1e-11

"""Pins of the oracle's velocity space V_h and its maps (CPU only)."""
import numpy as np
import pytest

import workloads as W
from oracle import convection as C
from oracle import fe, fields, hdiv, mesh

CASES = [(2, 4, 2), (2, 3, 3), (3, 3, 2), (3, 3, 3)]


def _space(dim, n, k):
    m = W.periodic_box_mesh(dim, n)
    topo = mesh.MeshTopo(m.coords, m.elems, m.rep)
    return hdiv.HDiv(topo, fe.ref_element(dim, k))


@pytest.mark.parametrize("dim,n,k", CASES)
def test_mesh_topology(dim, n, k):
    sp = _space(dim, n, k)
    t = sp.topo
    assert t.n_elems == n ** dim * (2 if dim == 2 else 6)
    assert t.n_facets * 2 == t.n_elems * (dim + 1)          # closed periodic mesh
    assert not np.any(t.boundary)
    # all elements have the same volume (2pi/n)^dim / dim!
    vol = (2 * np.pi / n) ** dim / (2 if dim == 2 else 6)
    assert np.allclose(t.absdet / (2 if dim == 2 else 6), vol)
    # the sign relating global and reference facet functionals is (-1)^f
    assert np.all(t.sigma == np.array([(-1) ** f for f in range(dim + 1)])[None, :])
    # sides: A's outward normal is n_F, both sides see the same facet points
    pA = t.facet_points(sp.ref.sq)
    e, f = t.fb[:, 0], t.fb[:, 1]
    loc = np.array([[j for j in range(dim + 1) if j != ff] for ff in range(dim + 1)])
    P = t.X[e[:, None], loc[f]]
    pB = P[:, None, 0, :] + np.einsum("qj,Fjc->Fqc", sp.ref.sq, P[:, 1:, :] - P[:, None, 0, :])
    shift = (pA - pB) / (2 * np.pi)
    assert np.allclose(shift, np.round(shift), atol=1e-12)   # equal modulo the period


@pytest.mark.parametrize("dim,n,k", CASES)
def test_roundtrip_is_identity_on_vh(dim, n, k):
    sp = _space(dim, n, k)
    u = np.random.default_rng(0).standard_normal(sp.n_hdiv)
    assert np.abs(sp.from_l2(sp.to_l2(u)) - u).max() < 1e-13


@pytest.mark.parametrize("dim,n,k", CASES)
def test_image_is_normal_continuous(dim, n, k):
    sp = _space(dim, n, k)
    uL = sp.to_l2(np.random.default_rng(1).standard_normal(sp.n_hdiv))
    uA = C.facet_trace(sp.topo, sp.ref, uL, "A")
    uB = C.facet_trace(sp.topo, sp.ref, uL, "B")
    jn = np.einsum("Fqa,Fa->Fq", uA - uB, sp.topo.nF)
    assert np.abs(jn).max() < 1e-12 * np.abs(uA).max()
    assert np.abs(uA - uB).max() > 1e-3                        # tangential jumps remain


@pytest.mark.parametrize("dim,n,k", CASES)
def test_dual_is_transpose(dim, n, k):
    sp = _space(dim, n, k)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(sp.n_hdiv)
    y = rng.standard_normal((sp.topo.n_elems, dim, sp.ref.nb))
    lhs = np.sum(sp.to_l2(x) * y)
    assert abs(lhs - np.dot(x, sp.dual(y))) < 1e-12 * np.sqrt(sp.n_hdiv * y.size)


@pytest.mark.parametrize("dim,n,k", CASES)
def test_interpolant_reproduces_vh_fields(dim, n, k):
    # curl of a continuous P^{k+1} interpolant lies in V_h; its canonical
    # interpolant, computed from point values, must give back the same field.
    sp = _space(dim, n, k)
    wL = fields.curl_field(sp.topo, dim, k, fields.random_potential(dim, 5))
    # evaluate the piecewise polynomial at facet points (side A) and volume points
    fvals = C.facet_trace(sp.topo, sp.ref, wL, "A")
    vvals = np.einsum("qi,eai->eqa", sp.ref.phi, wL)
    wV = sp.interpolate_values(fvals, vvals)
    assert np.abs(sp.to_l2(wV) - wL).max() < 1e-12 * np.abs(wL).max()


def test_interpolant_converges_for_taylor_green():
    errs = []
    for n in (4, 8, 16):
        sp = _space(2, n, 2)
        uV = sp.interpolate(W.taylor_green)
        diff = sp.to_l2(uV) - sp.l2_project(W.taylor_green)
        errs.append(np.sqrt(np.sum(sp.topo.absdet[:, None, None] * diff ** 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.8), rates                          # order k+1 = 3


def test_single_element_mesh_has_boundary_facets():
    coords = np.array([[0.0, 0, 0], [1.0, 0.1, 0], [0.2, 1.1, 0.1], [0.1, 0.3, 0.9]])
    t = mesh.MeshTopo(coords, np.array([[2, 0, 3, 1]]))
    assert t.n_facets == 4 and np.all(t.boundary)
    assert np.all(t.fa[:, 0] == 0)

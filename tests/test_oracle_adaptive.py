"""Pins of the oracle's adaptive HOPU (Section 3.2: the jump indicator eta and the order
rule with thresholds eta_{-1} = 0 < eta_0 < ... < eta_k < eta_{k+1} = 1)."""
import numpy as np
import pytest

import workloads as W
from oracle import adaptive as AD
from oracle import fe, hdiv, mesh


def _space(dim, n, k):
    m = W.periodic_box_mesh(dim, n)
    return hdiv.HDiv(mesh.MeshTopo(m.coords, m.elems, m.rep), fe.ref_element(dim, k))


def _piecewise_constant(sp, values):
    """L2 coefficients of the field equal to values[e] on element e (a closed form: the
    Dubiner function of degree 0 is the constant 1/sqrt(|T^|), so a constant c has the
    single coefficient c sqrt(|T^|))."""
    ref = sp.ref
    vol = float(np.sum(ref.wq))                       # |T^|
    uL = np.zeros((sp.topo.n_elems, ref.dim, ref.nb))
    uL[:, :, 0] = values * np.sqrt(vol)
    return uL


@pytest.mark.parametrize("dim,n,k", [(2, 4, 2), (3, 3, 3)])
def test_eta_closed_form_for_piecewise_constant_fields(dim, n, k):
    sp = _space(dim, n, k)
    t = sp.topo
    c = np.random.default_rng(40).standard_normal((t.n_elems, dim)) + 2.0
    uL = _piecewise_constant(sp, c)
    cA, cB = c[t.fa[:, 0]], c[t.fb[:, 0]]
    jump, avg = cA - cB, 0.5 * (cA + cB)
    # l = -1: nothing projected, eta = |c_A - c_B| / |(c_A + c_B)/2|
    ref = np.linalg.norm(jump, axis=1) / np.linalg.norm(avg, axis=1)
    assert np.allclose(AD.facet_eta(t, sp.ref, uL, -1), ref, rtol=1e-12)
    # l >= 0: the constant tangential jump lies in P^l and is projected out
    ref = np.abs(np.einsum("Fa,Fa->F", jump, t.nF)) / np.linalg.norm(avg, axis=1)
    for l in range(0, k + 1):
        assert np.allclose(AD.facet_eta(t, sp.ref, uL, l), ref, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("dim,n,k", [(2, 4, 2), (3, 3, 2)])
def test_eta_vanishes_for_continuous_and_normal_continuous_fields(dim, n, k):
    sp = _space(dim, n, k)
    uL = _piecewise_constant(sp, np.tile(np.arange(1.0, dim + 1.0), (sp.topo.n_elems, 1)))
    for l in (-1, 0, k):
        assert np.abs(AD.facet_eta(sp.topo, sp.ref, uL, l)).max() < 1e-13
    # E(V_h) is normal-continuous: with l = k only the normal jump survives (I - Pi^k)
    uV = np.random.default_rng(41).standard_normal(sp.n_hdiv)
    eta_k = AD.facet_eta(sp.topo, sp.ref, sp.to_l2(uV), k)
    assert np.abs(eta_k).max() < 1e-12
    assert np.abs(AD.facet_eta(sp.topo, sp.ref, sp.to_l2(uV), -1)).max() > 1e-3


def test_order_rule_at_and_between_thresholds():
    th = [0.1, 0.2, 0.3, 0.4]
    eta = np.array([0.0, 0.05, 0.1, 0.1000001, 0.2, 0.25, 0.3, 0.4, 0.45, 1.0, 3.0, np.inf])
    want = np.array([-1, -1, -1, 0, 0, 1, 1, 2, 3, 3, 3, 3])
    assert np.array_equal(AD.order_from_eta(eta, th, 3), want)
    with pytest.raises(ValueError):
        AD.order_from_eta(eta, [0.1, 0.3, 0.2, 0.4], 3)
    with pytest.raises(ValueError):
        AD.order_from_eta(eta, [0.1, 0.2, 0.3], 3)


def test_adapt_uses_the_current_orders():
    """eta depends on l through Pi^l: the same field gives different eta for different
    current orders, and adapt() evaluates it with the orders it is given."""
    sp = _space(3, 3, 3)
    rng = np.random.default_rng(42)
    uL = sp.to_l2(sp.interpolate(W.taylor_green)) + 0.05 * rng.standard_normal((sp.topo.n_elems, 3, sp.ref.nb))
    l0 = rng.integers(-1, 4, size=sp.topo.n_facets)
    eta, lnew = AD.adapt(sp.topo, sp.ref, uL, l0, [0.1, 0.2, 0.3, 0.4])
    for l in (-1, 3):
        m = l0 == l
        assert np.allclose(eta[m], AD.facet_eta(sp.topo, sp.ref, uL, l)[m], rtol=1e-14)
    assert np.array_equal(lnew, AD.order_from_eta(eta, [0.1, 0.2, 0.3, 0.4], 3))

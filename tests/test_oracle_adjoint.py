"""Pins of the oracle's derivatives (P13): JVP against finite differences of the apply,
the dot-product identity between the independently written JVP and VJP, the transposed
back-projection, and the rollout adjoint against finite differences of the rollout loss.
"""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as A
from oracle import convection as C
from oracle import fe, fields, hdiv, mesh


def _space(dim, n, k):
    m = W.periodic_box_mesh(dim, n)
    return hdiv.HDiv(mesh.MeshTopo(m.coords, m.elems, m.rep), fe.ref_element(dim, k))


@pytest.mark.parametrize("dim,n,k", [(2, 4, 2), (3, 3, 2)])
def test_from_l2_transpose_is_the_adjoint(dim, n, k):
    sp = _space(dim, n, k)
    rng = np.random.default_rng(20)
    y = rng.standard_normal((sp.topo.n_elems, dim, sp.ref.nb))
    v = rng.standard_normal(sp.n_hdiv)
    lhs = np.dot(sp.from_l2(y), v)
    assert abs(lhs - np.sum(y * sp.from_l2_transpose(v))) < 1e-12 * np.sqrt(y.size * v.size)


@pytest.mark.parametrize("dim,n,k", [(2, 4, 2), (3, 3, 2), (3, 3, 3)])
def test_jvp_matches_finite_differences(dim, n, k):
    sp = _space(dim, n, k)
    rng = np.random.default_rng(21)
    wL = sp.to_l2(rng.standard_normal(sp.n_hdiv))
    uL = rng.standard_normal(wL.shape)
    dw = sp.to_l2(rng.standard_normal(sp.n_hdiv))
    du = rng.standard_normal(wL.shape)
    for l in (-1, k - 1):
        jv = A.jvp_apply(sp.topo, sp.ref, wL, uL, dw, du, l)
        h = 1e-6
        fd = (C.apply(sp.topo, sp.ref, wL + h * dw, uL + h * du, l)
              - C.apply(sp.topo, sp.ref, wL - h * dw, uL - h * du, l)) / (2 * h)
        assert np.abs(jv - fd).max() < 1e-6 * np.abs(jv).max()


@pytest.mark.parametrize("dim,n,k", [(2, 4, 2), (3, 3, 2), (3, 3, 3)])
def test_vjp_dot_product_identity(dim, n, k):
    sp = _space(dim, n, k)
    rng = np.random.default_rng(22)
    wL = sp.to_l2(rng.standard_normal(sp.n_hdiv))
    uL = rng.standard_normal(wL.shape)
    dw = rng.standard_normal(wL.shape)
    du = rng.standard_normal(wL.shape)
    ybar = rng.standard_normal(wL.shape)
    for l in (-1, 0, k - 1, k):
        jv = A.jvp_apply(sp.topo, sp.ref, wL, uL, dw, du, l)
        wb, ub = A.vjp_apply(sp.topo, sp.ref, wL, uL, ybar, l)
        lhs = np.sum(ybar * jv)
        rhs = np.sum(wb * dw) + np.sum(ub * du)
        assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + np.abs(ybar * jv).sum())


def test_rollout_adjoint_matches_finite_differences():
    sp = _space(2, 4, 2)
    u0 = sp.interpolate(W.taylor_green) + W.uniform_noise(sp.n_hdiv, 1e-2, 23)
    dt, n = 2e-2, 5
    loss, g = A.rollout_vjp(sp, u0, dt, n, 1)
    loss2, _ = A.rollout_loss(sp, u0, dt, n, 1)
    assert loss == pytest.approx(loss2, rel=1e-14)
    dirs = W.normal_vectors(4, sp.n_hdiv, seed=2)
    for d in dirs:
        h = 1e-5
        fd = (A.rollout_loss(sp, u0 + h * d, dt, n, 1)[0] - A.rollout_loss(sp, u0 - h * d, dt, n, 1)[0]) / (2 * h)
        assert abs(fd - np.dot(g, d)) < 1e-7 * max(abs(fd), np.abs(g).max())


def test_seeded_rollout_adjoint_matches_finite_differences():
    """With a cotangent seed s of u_n, the result g satisfies <s, (d u_n / d u0) d> = <g, d>
    (the Jacobian-vector product by central differences of the rollout's final state)."""
    sp = _space(3, 3, 2)
    u0 = sp.interpolate(W.taylor_green) + W.uniform_noise(sp.n_hdiv, 1e-2, 24)
    dt, n = 2e-2, 3
    s = np.random.default_rng(25).standard_normal(sp.n_hdiv)
    _, g = A.rollout_vjp(sp, u0, dt, n, 1, seed=s)
    for d in W.normal_vectors(3, sp.n_hdiv, seed=2):
        h = 1e-5
        jd = (A.rollout_loss(sp, u0 + h * d, dt, n, 1)[1] - A.rollout_loss(sp, u0 - h * d, dt, n, 1)[1]) / (2 * h)
        assert abs(np.dot(s, jd) - np.dot(g, d)) < 1e-7 * np.linalg.norm(s) * max(np.linalg.norm(jd), 1.0)

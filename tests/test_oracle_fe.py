"""Pins of the oracle's reference-element ingredients (CPU only).

Every check compares against something other than the oracle itself: closed-form
monomial integrals, textbook Gauss abscissae, hand-derived Dubiner polynomials,
finite differences and exact polynomial-degree structure.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import fe, hdiv

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "quadrature_closed_forms.txt")


def _monomial_exact(e):
    return math.prod(math.factorial(a) for a in e) / math.factorial(sum(e) + len(e))


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_quadrature_exact_on_monomials(dim):
    # int_{unit simplex} x^a y^b z^c = a! b! c! / (a+b+c+dim)!
    for deg in range(0, 16):
        x, w = fe.simplex_rule(dim, deg)
        for e in itertools.product(range(deg + 1), repeat=dim):
            if sum(e) > deg:
                continue
            val = np.sum(w * np.prod(x ** np.array(e), axis=1))
            assert abs(val - _monomial_exact(e)) < 1e-15 * max(1, 1 / _monomial_exact(e)) + 1e-16


def test_quadrature_not_exact_beyond_degree():
    # the rule must really be the m = ceil((deg+1)/2) rule: degree 2m fails
    x, w = fe.simplex_rule(1, 3)           # m = 2
    assert abs(np.sum(w * x[:, 0] ** 4) - 1 / 5) > 1e-4


def test_gauss_factors_match_closed_forms():
    rows = [l.split("#")[0].split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    for r in rows:
        if r[0] == "J1":
            t, w = fe.gauss_jacobi_01(1, 1)
            assert abs(2 * t[0] - 1 - float(r[1])) < 1e-15
            assert abs(w[0] * 4 - float(r[2])) < 1e-15   # w_t = w_x / 2^(alpha+1)
            continue
        m = int(r[0])
        t, w = fe.gauss_jacobi_01(m, 0)
        x = 2 * t - 1
        j = np.argmin(np.abs(x - float(r[1])))
        assert abs(x[j] - float(r[1])) < 1e-15
        assert abs(2 * w[j] - float(r[2])) < 1e-15


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 5])
def test_dubiner_orthonormal(dim, k):
    x, w = fe.simplex_rule(dim, 2 * k + 1)
    v, _ = fe.dubiner(dim, k, x)
    M = (v * w[:, None]).T @ v
    assert np.abs(M - np.eye(len(M))).max() < 2e-14


def test_dubiner_hand_derived_low_order():
    # triangle: phi_0 = sqrt(2), phi_(p=0,q=1) = 6y - 2, phi_(1,0) = sqrt(12)(2x + y - 1)
    pts = np.array([[0.1, 0.2], [0.3, 0.5], [0.7, 0.05]])
    v, g = fe.dubiner(2, 1, pts)
    x, y = pts[:, 0], pts[:, 1]
    assert np.allclose(v[:, 0], math.sqrt(2), atol=1e-15)
    assert np.allclose(v[:, 1], 6 * y - 2, atol=1e-14)
    assert np.allclose(v[:, 2], math.sqrt(12) * (2 * x + y - 1), atol=1e-14)
    assert np.allclose(g[:, 2, 0], 2 * math.sqrt(12)) and np.allclose(g[:, 2, 1], math.sqrt(12))
    # tetrahedron: phi_0 = sqrt(6); (0,0,1): sqrt(1*2*5) P_1^{(2,0)}(2z-1) = sqrt(10)(4z - 1)
    p3 = np.array([[0.1, 0.2, 0.3], [0.25, 0.25, 0.25]])
    v3, _ = fe.dubiner(3, 1, p3)
    assert np.allclose(v3[:, 0], math.sqrt(6), atol=1e-14)
    assert np.allclose(v3[:, 1], math.sqrt(10) * (4 * p3[:, 2] - 1), atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_dubiner_gradient_finite_difference(dim):
    rng = np.random.default_rng(1)
    pts = rng.uniform(0.05, 1.0 / dim - 0.05, (9, dim))
    _, g = fe.dubiner(dim, 5, pts)
    h = 1e-6
    for c in range(dim):
        e = np.zeros(dim)
        e[c] = h
        fd = (fe.dubiner(dim, 5, pts + e)[0] - fe.dubiner(dim, 5, pts - e)[0]) / (2 * h)
        assert np.abs(fd - g[:, :, c]).max() < 1e-6 * np.abs(g).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_dubiner_graded_degree(dim):
    # the first C(n+d, d) functions are exactly polynomials of degree <= n:
    # a least-squares fit by monomials of degree <= n reproduces them.
    k = 4
    rng = np.random.default_rng(2)
    pts = rng.dirichlet(np.ones(dim + 1), size=200)[:, :dim]
    v, _ = fe.dubiner(dim, k, pts)
    for n in range(k + 1):
        exps = [e for e in itertools.product(range(n + 1), repeat=dim) if sum(e) <= n]
        A = np.stack([np.prod(pts ** np.array(e), axis=1) for e in exps], axis=1)
        nb = fe.n_basis(dim, n)
        coef, *_ = np.linalg.lstsq(A, v[:, :nb], rcond=None)
        assert np.abs(A @ coef - v[:, :nb]).max() < 1e-10
        if n < k:   # the next function is not of degree n
            coef, *_ = np.linalg.lstsq(A, v[:, nb], rcond=None)
            assert np.abs(A @ coef - v[:, nb]).max() > 1e-3


@pytest.mark.parametrize("dim,k", [(2, 2), (2, 3), (3, 2), (3, 3), (3, 4), (3, 5)])
def test_interior_space_is_nedelec_and_unisolvent(dim, k):
    ref = fe.RefElement(dim, k)
    z = ref.z                                            # [nint, nq, d]
    nint = fe.n_interior(dim, k)
    assert z.shape[0] == nint
    A = z.transpose(1, 2, 0).reshape(-1, nint)
    assert np.linalg.matrix_rank(A, tol=1e-10) == nint  # a basis
    # contains grad P^{k-1} (the commuting-diagram property of the BDM element)
    _, g = fe.dubiner(dim, k - 1, ref.xq)
    G = g.transpose(0, 2, 1).reshape(-1, g.shape[1])        # rows (q, c) like A
    coef, *_ = np.linalg.lstsq(A, G, rcond=None)
    assert np.abs(A @ coef - G).max() < 1e-10
    D = hdiv.reference_dof_matrix(ref)
    assert np.linalg.cond(D) < 200

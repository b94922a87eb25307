"""Reference-element ingredients of the oracle (FP64, numpy/scipy).

* Quadrature: collapsed (Stroud conical) Gauss-Jacobi rules on the unit simplex,
  m points per collapsed direction with m = ceil((degree+1)/2); the nodes and
  weights of each 1D factor come from ``scipy.special.roots_jacobi``.  The paper
  asks that every form be integrated exactly (Section 2.2, the remark closing the
  discrete model); the volume rule is exact to degree 3k-1 and the facet rule to
  degree 3k, enough for every polynomial integrand of the convection form.
  Pinned by tests/test_oracle_fe.py against the closed form
  int_{unit simplex} x^a y^b z^c = a! b! c! / (a+b+c+dim)!.
* Basis of the discontinuous space P^k(T): the orthonormal Dubiner (Koornwinder)
  basis in collapsed coordinates, graded by total degree so that the first
  C(l+d, d) functions span P^l (needed by the facet projection Pi^l of
  Section 3.2).  Values use ``scipy.special.eval_jacobi``.  Pinned by
  orthonormality under the pinned rule, by finite differences of the gradients
  and by an exact polynomial-degree check.
* Interior moment space of the velocity space (the BDM element of the paper's
  reference [boffi2013mixed] for H(div) elements): Z = N1_{k-1}, see
  ``interior_space``.  Unisolvence is pinned by the invertibility of the
  reference DOF matrix and by a dimension/rank check (tests).
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np
from scipy.special import eval_jacobi, roots_jacobi


# ------------------------------------------------------------------ quadrature
def gauss_jacobi_01(m: int, alpha: int):
    """Nodes t in (0,1), weights w with sum w f(t) = int_0^1 f(t) (1-t)^alpha dt."""
    x, w = roots_jacobi(m, float(alpha), 0.0)
    return (1.0 + x) / 2.0, w / 2.0 ** (alpha + 1)


def points_per_direction(degree: int) -> int:
    return max(1, int(math.ceil((degree + 1) / 2)))


def simplex_rule(dim: int, degree: int):
    """Collapsed Gauss-Jacobi rule on the unit simplex of dimension dim (1, 2, 3).

    Returns (points [n, dim], weights [n]); weights sum to 1/dim!.
    """
    m = points_per_direction(degree)
    if dim == 1:
        t, w = gauss_jacobi_01(m, 0)
        return t[:, None], w
    if dim == 2:
        t1, w1 = gauss_jacobi_01(m, 0)
        t2, w2 = gauss_jacobi_01(m, 1)
        e1, e2 = np.meshgrid(t1, t2, indexing="ij")
        pts = np.stack([e1 * (1 - e2), e2], axis=-1).reshape(-1, 2)
        return pts, np.outer(w1, w2).reshape(-1)
    if dim == 3:
        t1, w1 = gauss_jacobi_01(m, 0)
        t2, w2 = gauss_jacobi_01(m, 1)
        t3, w3 = gauss_jacobi_01(m, 2)
        e1, e2, e3 = np.meshgrid(t1, t2, t3, indexing="ij")
        pts = np.stack([e1 * (1 - e2) * (1 - e3), e2 * (1 - e3), e3], axis=-1).reshape(-1, 3)
        return pts, np.einsum("i,j,k->ijk", w1, w2, w3).reshape(-1)
    raise ValueError(dim)


# ------------------------------------------------------------------ Dubiner basis
def dubiner_indices(dim: int, k: int):
    """(p[,q[,r]]) tuples graded by total degree n; inside a degree p ascends, then q."""
    out = []
    for n in range(k + 1):
        if dim == 1:
            out.append((n,))
        elif dim == 2:
            for p in range(n + 1):
                out.append((p, n - p))
        else:
            for p in range(n + 1):
                for q in range(n - p + 1):
                    out.append((p, q, n - p - q))
    return out


def n_basis(dim: int, k: int) -> int:
    return math.comb(k + dim, dim) if k >= 0 else 0


def _P(n, a, x):
    return eval_jacobi(n, a, 0.0, x)


def _dP(n, a, x):
    """d/dx P_n^{(a,0)}(x) = (n+a+1)/2 P_{n-1}^{(a+1,1)}(x)."""
    if n == 0:
        return np.zeros_like(x)
    return 0.5 * (n + a + 1) * eval_jacobi(n - 1, a + 1.0, 1.0, x)


def _safe_div(a, b):
    return np.where(b > 0, a / np.where(b > 0, b, 1.0), 0.0)


def _pow(b, e):
    if e == 0:
        return np.ones_like(b)
    if e > 0:
        return b ** e
    return np.where(b > 0, np.where(b > 0, b, 1.0) ** e, 0.0)


def dubiner(dim: int, k: int, x: np.ndarray):
    """Orthonormal Dubiner basis of P^k on the unit simplex at points x [N, dim].

    Returns (values [N, nb], gradients [N, nb, dim]).
    """
    x = np.asarray(x, dtype=np.float64)
    idx = dubiner_indices(dim, k)
    N = x.shape[0]
    vals = np.zeros((N, len(idx)))
    grads = np.zeros((N, len(idx), dim))
    if dim == 1:
        xi = 2 * x[:, 0] - 1
        for j, (m,) in enumerate(idx):
            c = math.sqrt(2 * m + 1)
            vals[:, j] = c * _P(m, 0, xi)
            grads[:, j, 0] = c * 2 * _dP(m, 0, xi)
        return vals, grads
    if dim == 2:
        X, Y = x[:, 0], x[:, 1]
        s = 1 - Y
        xi1 = _safe_div(2 * X, s) - 1
        xi2 = 2 * Y - 1
        for j, (p, q) in enumerate(idx):
            c = math.sqrt((2 * p + 1) * (2 * p + 2 * q + 2))
            Pp, dPp = _P(p, 0, xi1), _dP(p, 0, xi1)
            F1 = Pp * _pow(s, p)
            F1x = 2 * dPp * _pow(s, p - 1)
            F1y = 2 * X * dPp * _pow(s, p - 2) - p * Pp * _pow(s, p - 1)
            F2 = _P(q, 2 * p + 1, xi2)
            F2y = 2 * _dP(q, 2 * p + 1, xi2)
            vals[:, j] = c * F1 * F2
            grads[:, j, 0] = c * F1x * F2
            grads[:, j, 1] = c * (F1y * F2 + F1 * F2y)
        return vals, grads
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    s = 1 - Y - Z
    t = 1 - Z
    xi1 = _safe_div(2 * X, s) - 1
    xi2 = _safe_div(2 * Y, t) - 1
    xi3 = 2 * Z - 1
    for j, (p, q, r) in enumerate(idx):
        c = math.sqrt((2 * p + 1) * (2 * p + 2 * q + 2) * (2 * p + 2 * q + 2 * r + 3))
        Pp, dPp = _P(p, 0, xi1), _dP(p, 0, xi1)
        F1 = Pp * _pow(s, p)
        F1x = 2 * dPp * _pow(s, p - 1)
        F1yz = 2 * X * dPp * _pow(s, p - 2) - p * Pp * _pow(s, p - 1)
        a2 = 2 * p + 1
        Pq, dPq = _P(q, a2, xi2), _dP(q, a2, xi2)
        F2 = Pq * _pow(t, q)
        F2y = 2 * dPq * _pow(t, q - 1)
        F2z = 2 * Y * dPq * _pow(t, q - 2) - q * Pq * _pow(t, q - 1)
        a3 = 2 * p + 2 * q + 2
        F3 = _P(r, a3, xi3)
        F3z = 2 * _dP(r, a3, xi3)
        vals[:, j] = c * F1 * F2 * F3
        grads[:, j, 0] = c * F1x * F2 * F3
        grads[:, j, 1] = c * (F1yz * F2 + F1 * F2y) * F3
        grads[:, j, 2] = c * (F1yz * F2 * F3 + F1 * F2z * F3 + F1 * F2 * F3z)
    return vals, grads


# ------------------------------------------------------------------ reference simplex
def ref_vertices(dim: int) -> np.ndarray:
    return np.vstack([np.zeros(dim), np.eye(dim)])


def facet_vertices(dim: int, f: int) -> np.ndarray:
    """Vertices of the reference facet opposite vertex f, in ascending local order."""
    V = ref_vertices(dim)
    return V[[j for j in range(dim + 1) if j != f]]


def facet_map(dim: int, f: int, s: np.ndarray) -> np.ndarray:
    """Point of reference facet f with parametric coordinates s [N, dim-1]."""
    P = facet_vertices(dim, f)
    return P[0] + (s @ (P[1:] - P[0]))


def scaled_outward_normal(dim: int, f: int) -> np.ndarray:
    """-grad(lambda_f): outward normal of reference facet f times |facet| / |param simplex|."""
    if f == 0:
        return np.ones(dim)
    v = np.zeros(dim)
    v[f - 1] = -1.0
    return v


# ------------------------------------------------------------------ interior moment space
def interior_space(dim: int, k: int, x: np.ndarray) -> np.ndarray:
    """Values [n_int, N, dim] of the interior moment functions z_j at points x.

    Z = [P^{k-2}]^d  (+)  x~ x q e_m (3D)  /  x~^perp q (2D), where
    x~ = (d+1)(x - centroid) and q runs over polynomials of degree exactly k-2
    whose top-degree parts span the homogeneous polynomials of that degree.  This
    is the classical interior space of the BDM_k element (Nedelec first kind of
    index k-1), written in a well-conditioned basis:

    * part A: phi_j e_m for every Dubiner phi_j of P^{k-2}, m = 0..d-1 (m-major);
    * part B, 2D: x~^perp phi_j, phi_j in the degree-(k-2) Dubiner block, with
      x~^perp = (-x~_2, x~_1);
    * part B, 3D: for m = 0, 1: x~ x (phi_j e_m), phi_j in the degree-(k-2) block
      of the 3D Dubiner basis; for m = 2: x~ x (chi_j e_2), chi_j in the
      degree-(k-2) block of the 2D Dubiner basis of (x_1, x_2).  Excluding the
      multiples of x_3 from the third family removes exactly the kernel
      x~ x (x~ h) = 0 of the cross product, so the family is a basis.
    """
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[0]
    if k < 2:
        return np.zeros((0, N, dim))
    out = []
    phi, _ = dubiner(dim, k - 2, x)
    for m in range(dim):
        for j in range(phi.shape[1]):
            z = np.zeros((N, dim))
            z[:, m] = phi[:, j]
            out.append(z)
    xt = (dim + 1) * (x - 1.0 / (dim + 1))
    lo = n_basis(dim, k - 3)
    if dim == 2:
        for j in range(lo, phi.shape[1]):
            out.append(np.stack([-xt[:, 1] * phi[:, j], xt[:, 0] * phi[:, j]], axis=-1))
    else:
        chi, _ = dubiner(2, k - 2, x[:, :2])
        lo2 = n_basis(2, k - 3)
        for m in range(3):
            e = np.zeros(3)
            e[m] = 1.0
            cr = np.cross(xt, e)                                       # x~ cross e_m
            qs = phi[:, lo:] if m < 2 else chi[:, lo2:]
            for j in range(qs.shape[1]):
                out.append(cr * qs[:, j][:, None])
    return np.array(out)


def n_interior(dim: int, k: int) -> int:
    return dim * n_basis(dim, k) - (dim + 1) * n_basis(dim - 1, k)


# ------------------------------------------------------------------ tables
class RefElement:
    """All reference tables of order k in dimension dim (FP64).

    vol_degree / facet_degree default to the exactness the convection form needs
    (3k-1 and 3k); tests raise them to check that nothing depends on the rule.
    """

    def __init__(self, dim: int, k: int, vol_degree: int | None = None,
                 facet_degree: int | None = None):
        self.dim, self.k = dim, k
        self.vol_degree = 3 * k - 1 if vol_degree is None else vol_degree
        self.facet_degree = 3 * k if facet_degree is None else facet_degree
        self.nb = n_basis(dim, k)
        self.nf = n_basis(dim - 1, k)
        self.nint = n_interior(dim, k)
        self.xq, self.wq = simplex_rule(dim, self.vol_degree)
        self.sq, self.wf = simplex_rule(dim - 1, self.facet_degree)
        self.phi, self.dphi = dubiner(dim, k, self.xq)
        self.phi_f = np.array([dubiner(dim, k, facet_map(dim, f, self.sq))[0]
                               for f in range(dim + 1)])           # [d+1, nqf, nb]
        self.psi, _ = dubiner(dim - 1, k, self.sq)                  # [nqf, nf]
        self.Nhat = np.array([scaled_outward_normal(dim, f) for f in range(dim + 1)])
        self.z = interior_space(dim, k, self.xq)                    # [nint, nq, d]
        assert self.z.shape[0] == self.nint, (self.z.shape, self.nint)
        self.param_measure = 1.0 / math.factorial(dim - 1)


@lru_cache(maxsize=None)
def ref_element(dim: int, k: int, vol_degree=None, facet_degree=None) -> RefElement:
    return RefElement(dim, k, vol_degree, facet_degree)

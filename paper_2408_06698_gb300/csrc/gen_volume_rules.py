"""Write volume_rules.h: compact quadrature rules on the unit tetrahedron for the volume
kernels (3D, k = 3, 4, 5; exact to degree 3k - 1 = 8, 11, 14).

The volume term of the convection operator integrates a polynomial of degree 3k - 1 per
element.  The collapsed Gauss-Jacobi (Stroud conical product) rule needs m^3 points,
m = ceil(3k / 2) (125, 216, 512); any rule exact to that degree gives the same integral,
and the kernels' cost is proportional to the number of passes over the points (32 lanes,
two points per lane and pass in FP32).  The rules here have 46, 100 and 190 points: 1, 2
and 3 passes instead of 2, 4 and 8 at k = 3, 4, 5.

Construction: N points p = sum_v lambda_v V_v with barycentric coordinates
lambda = softmax(theta) (strictly inside) and weights w = exp(rho) (positive); the
unknowns (theta, rho) solve the moment equations
    sum_p w_p phi_j(p) = int_T phi_j,   j over the Dubiner basis of P^deg,
normalised to unit L2 norm (int_T phi_j = 0 for j > 0), by Levenberg-Marquardt with the
least-norm step of the underdetermined system (4N unknowns, C(deg+3, 3) equations), from
seeded random starting points.  The Jacobian uses central differences of the basis in
the point coordinates.  Accepted rules reproduce every monomial moment
int x^a y^b z^c = a! b! c! / (a + b + c + 3)!  (a + b + c <= deg) to 1e-14 relative.

Run from the repository root:  python paper_2408_06698_gb300/csrc/gen_volume_rules.py
"""
from __future__ import annotations

import math
import os

import numpy as np
from scipy.special import roots_jacobi

# (k, degree, points, seed): the seeds give the rules written to volume_rules.h
RULES = [(3, 8, 46, 2), (4, 11, 100, 1), (5, 14, 190, 0)]


def jacobi(n: int, alpha: int, x: np.ndarray) -> list:
    """P_0..P_n^{(alpha, 0)}(x) by the three-term recurrence."""
    P = [np.ones_like(x)]
    if n >= 1:
        P.append(((alpha + 2) * x + alpha) / 2)
    for m in range(1, n):
        a1 = 2 * (m + 1) * (m + alpha + 1) * (2 * m + alpha)
        a2 = (2 * m + alpha + 1) * alpha ** 2
        a3 = (2 * m + alpha) * (2 * m + alpha + 1) * (2 * m + alpha + 2)
        a4 = 2 * m * (m + alpha) * (2 * m + alpha + 2)
        P.append(((a2 + a3 * x) * P[m] - a4 * P[m - 1]) / a1)
    return P


def dubiner(deg: int, X: np.ndarray) -> np.ndarray:
    """Unnormalised Dubiner basis of P^deg on the unit tetrahedron at interior points
    X [N, 3]: values [n_basis, N]."""
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    a = 2 * x / (1 - y - z) - 1
    b = 2 * y / (1 - z) - 1
    c = 2 * z - 1
    Pa = jacobi(deg, 0, a)
    out = []
    for p in range(deg + 1):
        Pb = jacobi(deg - p, 2 * p + 1, b)
        for q in range(deg - p + 1):
            Pc = jacobi(deg - p - q, 2 * p + 2 * q + 2, c)
            for r in range(deg - p - q + 1):
                out.append(Pa[p] * ((1 - b) / 2) ** p * Pb[q] * ((1 - c) / 2) ** (p + q) * Pc[r])
    return np.array(out)


def collapsed_rule(m: int):
    """Stroud conical product rule with m points per direction (exact to 2m - 1)."""
    t0, w0 = roots_jacobi(m, 0, 0)
    t1, w1 = roots_jacobi(m, 1, 0)
    t2, w2 = roots_jacobi(m, 2, 0)
    P, W = [], []
    for i in range(m):
        for j in range(m):
            for k in range(m):
                z = (1 + t2[k]) / 2
                y = (1 + t1[j]) / 2 * (1 - z)
                x = (1 + t0[i]) / 2 * (1 - y - z)
                P.append((x, y, z))
                W.append(w0[i] * w1[j] * w2[k] / 64)
    return np.array(P), np.array(W)


def softmax(th: np.ndarray) -> np.ndarray:
    e = np.exp(th - th.max(1, keepdims=True))
    return e / e.sum(1, keepdims=True)


def solve(deg: int, N: int, seed: int, iters: int = 400):
    Pr, Wr = collapsed_rule(deg + 1)          # exact for the squared basis (norms)
    nrm = np.sqrt((dubiner(deg, Pr) ** 2 * Wr).sum(1))
    vol = Wr.sum()
    target = np.zeros(nrm.size)
    target[0] = vol / nrm[0]
    rng = np.random.default_rng(seed)
    th = rng.standard_normal((N, 4)) * 0.8
    rho = np.full(N, np.log(vol / N))

    def resid(th, rho):
        lam = softmax(th)
        return (dubiner(deg, lam[:, 1:]) / nrm[:, None]) @ np.exp(rho) - target

    r, mu, h = resid(th, rho), 1e-2, 1e-6
    for _ in range(iters):
        lam = softmax(th)
        X, w = lam[:, 1:], np.exp(rho)
        B = dubiner(deg, X) / nrm[:, None]
        G = np.zeros((B.shape[0], N, 3))
        for c in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[:, c] += h
            Xm[:, c] -= h
            G[:, :, c] = (dubiner(deg, Xp) - dubiner(deg, Xm)) / (2 * h) / nrm[:, None]
        dX = lam[:, 1:, None] * (np.eye(4)[None, 1:, :] - lam[:, None, :])   # d X_c / d theta_j
        J = np.concatenate([np.einsum("jpc,pck->jpk", G * w[None, :, None], dX).reshape(B.shape[0], 4 * N),
                            B * w[None, :]], 1)
        d = -J.T @ np.linalg.solve(J @ J.T + mu * np.eye(J.shape[0]), r)
        th2, rho2 = th + d[:4 * N].reshape(N, 4), rho + d[4 * N:]
        r2 = resid(th2, rho2)
        if np.linalg.norm(r2) < np.linalg.norm(r):
            th, rho, r, mu = th2, rho2, r2, max(mu / 4, 1e-16)
        else:
            mu *= 5
        if np.linalg.norm(r) < 2e-16:
            break
    lam = softmax(th)
    return lam[:, 1:], np.exp(rho), float(np.linalg.norm(r)), float(lam.min())


def monomial_error(deg: int, X: np.ndarray, w: np.ndarray) -> float:
    worst = 0.0
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
                got = float(np.sum(w * X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c))
                worst = max(worst, abs(got - exact) / exact)
    return worst


def main() -> None:
    lines = [
        "// Compact quadrature rules on the unit tetrahedron {x, y, z >= 0, x + y + z <= 1} for",
        "// the volume kernels, exact to degree 3k - 1.  Written by gen_volume_rules.py (beside",
        "// this file), which states how they are computed; do not edit by hand.",
        "// Per point: x, y, z, weight (the weights sum to 1/6).",
        "#pragma once",
        "",
        "namespace hopu {",
        "",
    ]
    for k, deg, N, seed in RULES:
        X, w, res, lam_min = solve(deg, N, seed)
        order = np.lexsort((X[:, 0], X[:, 1], X[:, 2]))
        X, w = X[order], w[order]
        err = monomial_error(deg, X, w)
        if not (res < 1e-14 and err < 1e-14 and w.min() > 0 and lam_min > 1e-4):
            raise RuntimeError(f"k={k}: rule rejected (residual {res:.2e}, monomials {err:.2e})")
        lines.append(f"// k = {k}: degree {deg}, {N} points; moment residual {res:.1e}, worst monomial "
                     f"relative error {err:.1e},")
        lines.append(f"// smallest barycentric coordinate {lam_min:.2e}, weights in [{w.min():.2e}, {w.max():.2e}]")
        lines.append(f"inline constexpr int kTetRule{k}N = {N};")
        lines.append(f"inline constexpr double kTetRule{k}[{N} * 4] = {{")
        for p in range(N):
            lines.append("    " + ", ".join(f"{v:.17g}" for v in (X[p, 0], X[p, 1], X[p, 2], w[p])) + ",")
        lines.append("};")
        lines.append("")
        print(f"k={k}: {N} points, residual {res:.1e}, monomials {err:.1e}")
    lines.append("}  // namespace hopu")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "volume_rules.h")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()

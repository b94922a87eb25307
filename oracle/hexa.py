"""Hexahedral elements for the oracle (FP64).  Test infrastructure only: imported by
tests/, __graft_entry__.smoke() and the CPU legs of bench.py; the library never reads it.

The paper's meshes are hexahedral (Section 2.1: T_h is a subdivision into hexahedra) and
its convection operator is the HOPU form of Section 3.2 (eq. "hopudefinition").  It is
evaluated here in the conservative reading that oracle/convection.py states for simplices,

  c(w; u, v) = sum_T - int_T (u (x) w) : grad v
             + sum_E int_E [ (w.n) <u> + (I - Pi^l)[ 1/2 |w.n| (I - Pi^l)[[u]] ] ] . [[v]],

on the discontinuous space L_h = { v : v|_T o Phi_T in Q^k(T^)^3 }, T^ = [0, 1]^3, Q^k the
polynomials of degree <= k in each reference coordinate, with the orthonormal tensor
Legendre basis phi_i(x^) = L_i1(x^_1) L_i2(x^_2) L_i3(x^_3), i = i1 + (k+1)(i2 + (k+1) i3).
The cells of a workloads.HexBox are parallelepipeds (affine Phi_T), so M_T = |det J| I and
y = M^-1 c(w; u, .) divides by |det J|.

Readings (the paper is written for hexahedra but states V_h^proj with P^l):
  H1  on a quadrilateral facet the space P^l of V_h^proj (Section 3.2) is read as Q^l
      (degree <= l in each facet coordinate): the traces of Q^k are Q^k(F), and only then
      does l = k make Pi^l the identity on tangential traces, as Section 3.2 states.
  H2  quadrature: tensor Gauss-Legendre with m = ceil((3k+1)/2) points per direction in
      the volume and on the facets, exact for the polynomial integrands (degree <= 3k per
      direction on parallelepipeds); |w.n| is integrated by the facet rule, as on simplices.

Facets: facet F = a E + e is the facet of cell e on its low side in direction a; side A is
the cell below it (periodic wrap), through its local facet 2a+1 (x^_a = 1), side B is e,
through local facet 2a (x^_a = 0); n_F is side A's outward unit normal, [[u]] = u^A - u^B.
Both sides parametrise the facet by the two other reference coordinates in increasing axis
order, so their facet points coincide (every cell of a HexBox has the same orientation).
Directions that are not periodic end in walls or outlets (HexMesh's periodic flags): their
facets are single-sided and take the cell's own trace as the exterior one, as in the
simplicial oracle (no term in the paper's form, Section 2.1).

Pins: tests/test_oracle_hexa.py (closed-form Legendre values and Gauss moments,
orthonormality, finite-difference derivatives, the reference divergence theorem, the box's
volume and closed cells, facet points that coincide from both sides, zero output for
constant fields, the energy identity, the l = k limit, the Q^l orthogonality of (I - Pi^l),
the form equal to the simplicial oracle's on the same box for polynomial fields, periodic or
walled, and with walls the form equal to the volume integral of (grad u) w + (div w) u
evaluated from the polynomials' analytic gradients; with an inlet, the form equal to the
simplicial oracle's with the same exterior data; the order-k convergence of the discrete
(u . grad) u on Taylor-Green).
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg


def legendre01(n: int, x):
    """Orthonormal Legendre polynomials on [0, 1] up to degree n at x: values and
    derivatives, both [len(x), n+1] (L_i = sqrt(2i+1) P_i(2x - 1))."""
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    t = 2.0 * x - 1.0
    V = np.zeros((x.size, n + 1))
    D = np.zeros((x.size, n + 1))
    for i in range(n + 1):
        c = np.zeros(i + 1)
        c[i] = 1.0
        s = math.sqrt(2 * i + 1)
        V[:, i] = s * npleg.legval(t, c)
        if i > 0:
            D[:, i] = 2.0 * s * npleg.legval(t, npleg.legder(c))
    return V, D


def gauss01(m: int):
    """m-point Gauss-Legendre rule on [0, 1] (exact to degree 2m - 1)."""
    t, w = npleg.leggauss(m)
    return 0.5 * (t + 1.0), 0.5 * w


def points_per_direction(k: int) -> int:
    """Reading H2: ceil((3k + 1) / 2) points, exact to degree 3k per direction."""
    return (3 * k + 2) // 2


def basis(k: int, x):
    """phi [n, nb] and reference gradients dphi [n, nb, 3] of Q^k at points x [n, 3]."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    V = [legendre01(k, x[:, a]) for a in range(3)]
    r = np.arange(k + 1)
    i1, i2, i3 = np.meshgrid(r, r, r, indexing="ij")
    # basis index i = i1 + (k+1)(i2 + (k+1) i3)
    i1 = np.transpose(i1, (2, 1, 0)).reshape(-1)
    i2 = np.transpose(i2, (2, 1, 0)).reshape(-1)
    i3 = np.transpose(i3, (2, 1, 0)).reshape(-1)
    idx = (i1, i2, i3)
    phi = V[0][0][:, i1] * V[1][0][:, i2] * V[2][0][:, i3]
    dphi = np.zeros(phi.shape + (3,))
    for c in range(3):
        f = [V[a][1 if a == c else 0][:, idx[a]] for a in range(3)]
        dphi[:, :, c] = f[0] * f[1] * f[2]
    return phi, dphi


def facet_point(f: int, s):
    """Reference points [n, 3] of local facet f at facet coordinates s [n, 2]: axis a = f // 2
    held at f % 2, the two other axes (increasing order) taking s."""
    s = np.asarray(s, dtype=np.float64).reshape(-1, 2)
    a = f // 2
    x = np.zeros((s.shape[0], 3))
    x[:, a] = float(f % 2)
    others = [b for b in range(3) if b != a]
    x[:, others[0]] = s[:, 0]
    x[:, others[1]] = s[:, 1]
    return x


class RefHex:
    """Reference tables of Q^k on [0, 1]^3 with the tensor Gauss rules of reading H2."""

    def __init__(self, k: int, m: int | None = None):
        self.dim, self.k = 3, k
        self.m = points_per_direction(k) if m is None else m
        self.nb = (k + 1) ** 3
        x1, w1 = gauss01(self.m)
        g = np.arange(self.m)
        q1, q2, q3 = [np.transpose(t, (2, 1, 0)).reshape(-1) for t in np.meshgrid(g, g, g, indexing="ij")]
        self.xq = np.stack([x1[q1], x1[q2], x1[q3]], axis=-1)        # q = q1 + m (q2 + m q3)
        self.wq = w1[q1] * w1[q2] * w1[q3]
        self.phi, self.dphi = basis(k, self.xq)
        p1, p2 = [t.T.reshape(-1) for t in np.meshgrid(g, g, indexing="ij")]
        self.sq = np.stack([x1[p1], x1[p2]], axis=-1)                 # p = p1 + m p2
        self.wf = w1[p1] * w1[p2]
        self.phi_f = np.array([basis(k, facet_point(f, self.sq))[0] for f in range(6)])  # [6, nqf, nb]
        L = legendre01(k, x1)[0]
        r = np.arange(k + 1)
        ms, mt = [t.T.reshape(-1) for t in np.meshgrid(r, r, indexing="ij")]
        self.psi = L[p1][:, ms] * L[p2][:, mt]                        # facet modes m = ms + (k+1) mt
        self.psi_deg = np.maximum(ms, mt)
        self.Nhat = np.zeros((6, 3))
        for f in range(6):
            self.Nhat[f, f // 2] = 1.0 if f % 2 else -1.0

    def q_modes(self, l: int) -> np.ndarray:
        """Columns of psi spanning Q^l on a facet (reading H1)."""
        return np.where(self.psi_deg <= l)[0]


class HexMesh:
    """Geometry and facets of a workloads.HexBox (FP64), periodic in the directions a with
    periodic[a] True.  In another direction the facets at the two ends of the box are
    boundary facets (walls or outlets): F = a E + e for a cell e at the low end becomes the
    single-sided facet of e (side A, through local facet 2a, n_F out of e), and the facets
    of the cells at the high end (local facet 2a+1) are appended after the 3E others."""

    def __init__(self, hb, periodic=(True, True, True)):
        n0, n1, n2 = hb.n
        self.n = (n0, n1, n2)
        E = n0 * n1 * n2
        self.n_elems = E
        e = np.arange(E)
        self.cell = np.stack([e % n0, (e // n0) % n1, e // (n0 * n1)], axis=-1)   # axis 0 fastest
        A = np.asarray(hb.A, dtype=np.float64)
        h = np.stack([np.diff(hb.lines[a])[self.cell[:, a]] for a in range(3)], axis=-1)
        lo = np.stack([hb.lines[a][self.cell[:, a]] for a in range(3)], axis=-1)
        self.J = A[None, :, :] * h[:, None, :]                       # A diag(h)
        self.x0 = lo @ A.T
        self.detJ = np.linalg.det(self.J)
        self.absdet = np.abs(self.detJ)
        self.Jinv = np.linalg.inv(self.J)
        self.lattice = np.stack([A[:, a] * hb.lines[a][-1] for a in range(3)])  # rows: periods
        # facets F = a E + e: side A = the cell below e in direction a, side B = e
        below = []
        for a in range(3):
            c = self.cell.copy()
            c[:, a] = (c[:, a] - 1) % self.n[a]
            below.append(c[:, 0] + n0 * (c[:, 1] + n1 * c[:, 2]))
        below = np.stack(below)                                      # [3, E]
        self.n_facets = 3 * E
        self.fa = np.stack([below.reshape(-1), np.repeat(2 * np.arange(3) + 1, E)], axis=-1)
        self.fb = np.stack([np.tile(e, 3), np.repeat(2 * np.arange(3), E)], axis=-1)
        a_of_F = np.repeat(np.arange(3), E)
        sgn = np.ones(3 * E)                                          # side A's N^ = sgn e_a
        fa, fb = self.fa.copy(), self.fb.copy()
        extra_a, extra_dir = [], []
        for a in range(3):
            if periodic[a]:
                continue
            low = np.where(self.cell[:, a] == 0)[0]                   # the cells at the low end
            F = a * E + low
            fa[F] = np.stack([low, np.full(low.size, 2 * a)], axis=-1)
            fb[F] = -1
            sgn[F] = -1.0
            high = np.where(self.cell[:, a] == self.n[a] - 1)[0]
            extra_a.append(np.stack([high, np.full(high.size, 2 * a + 1)], axis=-1))
            extra_dir.append(np.full(high.size, a))
        if extra_a:
            fa = np.concatenate([fa] + extra_a)
            fb = np.concatenate([fb, -np.ones((sum(x.shape[0] for x in extra_a), 2), dtype=np.int64)])
            a_of_F = np.concatenate([a_of_F] + extra_dir)
            sgn = np.concatenate([sgn, np.ones(fa.shape[0] - 3 * E)])
        self.fa, self.fb = fa, fb
        self.n_facets = fa.shape[0]
        self.boundary = fb[:, 0] < 0
        # Nanson: n dA = det J J^-T N^ dA^ on side A (N^ = sgn e_a)
        eA = self.fa[:, 0]
        v = sgn[:, None] * self.detJ[eA, None] * self.Jinv[eA, a_of_F, :]   # (J^-T e_a)^T = row a
        self.aF = np.linalg.norm(v, axis=-1)
        self.nF = v / self.aF[:, None]

    def volume_points(self, xq) -> np.ndarray:
        return self.x0[:, None, :] + np.einsum("ecj,qj->eqc", self.J, xq)

    def facet_points(self, ref: RefHex, side: str = "A") -> np.ndarray:
        """Physical points [F, nqf, 3] of the facet rule seen from side A or B (unwrapped)."""
        ef = self.fa if side == "A" else self.fb
        out = np.zeros((self.n_facets, ref.wf.size, 3))
        for f in range(6):
            msk = ef[:, 1] == f
            if np.any(msk):
                xr = facet_point(f, ref.sq)
                el = ef[msk, 0]
                out[msk] = self.x0[el, None, :] + np.einsum("ecj,qj->eqc", self.J[el], xr)
        return out


# ------------------------------------------------------------------ fields
def project(mesh: HexMesh, ref: RefHex, f) -> np.ndarray:
    """L2 projection [E, 3, nb] of an analytic field f(x [..., 3]) onto L_h (orthonormal
    basis on an affine cell: c = int_T^ (f o Phi) phi_i, by the volume rule)."""
    X = mesh.volume_points(ref.xq)
    F = np.asarray(f(X), dtype=np.float64)                            # [E, nq, 3]
    return np.einsum("q,eqa,qi->eai", ref.wq, F, ref.phi)


def evaluate(ref: RefHex, cL: np.ndarray, x) -> np.ndarray:
    """Values [E, n, 3] of L2 coefficients at reference points x [n, 3] of every cell."""
    return np.einsum("qi,eai->eqa", basis(ref.k, x)[0], cL)


# ------------------------------------------------------------------ the operator
def _traces(mesh: HexMesh, ref: RefHex, cL: np.ndarray, side: str) -> np.ndarray:
    ef = mesh.fa if side == "A" else mesh.fb
    out = np.zeros((mesh.n_facets, ref.wf.size, 3))
    for f in range(6):
        msk = ef[:, 1] == f
        if np.any(msk):
            out[msk] = np.einsum("pi,Fai->Fpa", ref.phi_f[f], cL[ef[msk, 0]])
    return out


def complement_projection(ref: RefHex, l, nF: np.ndarray, V: np.ndarray) -> np.ndarray:
    """(I - Pi^l) V at the facet points, V [F, nqf, 3]: Pi^l is the facet-wise L2 projection
    onto tangential Q^l fields (reading H1); on a flat facet that is (I - n n^T) applied to
    the componentwise Q^l projection.  l < 0: Pi = 0.  l: one order or one per facet."""
    l_F = np.full(V.shape[0], int(l)) if np.isscalar(l) else np.asarray(l, dtype=np.int64)
    out = V.copy()
    for lv in np.unique(l_F):
        if lv < 0:
            continue
        msk = l_F == lv
        P = ref.psi[:, ref.q_modes(int(lv))]
        coef = np.einsum("p,pm,Fpa->Fma", ref.wf, P, V[msk])
        PiS = np.einsum("pm,Fma->Fpa", P, coef)
        n = nF[msk]
        PiV = PiS - np.einsum("Fpa,Fa->Fp", PiS, n)[..., None] * n[:, None, :]
        out[msk] = V[msk] - PiV
    return out


def facet_quantities(mesh: HexMesh, ref: RefHex, wL, uL, l: int, u_inlet=None):
    """Per facet point: w.n (= <w>.n_F), [[u]], <u>, (I-Pi)[[u]], (I-Pi)[1/2|w.n|(I-Pi)[[u]]].

    Boundary facets (walls and outlets, Section 2.1: no term in the paper's form) take
    side A's own traces as side B, as the simplicial oracle does: the jump vanishes and the
    conservative form keeps the flux (w.n) u . v that its cell-wise integration by parts
    needs to equal the paper's form.  Inlet facets (u_inlet: a dict facet index -> the
    exterior velocity at the facet points [nqf, 3]) take it as side B's velocity (Section
    2.2) and side A's own wind (the wind's normal component is single-valued)."""
    uA, uB = _traces(mesh, ref, uL, "A"), _traces(mesh, ref, uL, "B")
    wA, wB = _traces(mesh, ref, wL, "A"), _traces(mesh, ref, wL, "B")
    b = mesh.boundary
    if np.any(b):
        uB[b], wB[b] = uA[b], wA[b]
    for F, val in (u_inlet or {}).items():
        uB[F] = val
    wn = 0.5 * np.einsum("Fpa,Fa->Fp", wA + wB, mesh.nF)
    jump = uA - uB
    avg = 0.5 * (uA + uB)
    PJ = complement_projection(ref, l, mesh.nF, jump)
    Ph = complement_projection(ref, l, mesh.nF, 0.5 * np.abs(wn)[..., None] * PJ)
    return wn, jump, avg, PJ, Ph


def residual(mesh: HexMesh, ref: RefHex, wL, uL, l: int, u_inlet=None) -> np.ndarray:
    """r[e, a, i] = c(w; u, phi_i e_a) (conservative reading)."""
    U = np.einsum("qi,eai->eqa", ref.phi, uL)
    W = np.einsum("qi,eai->eqa", ref.phi, wL)
    Wt = np.einsum("e,ecb,eqb->eqc", mesh.absdet, mesh.Jinv, W)       # |det J| J^-1 w
    r = -np.einsum("q,eqa,qic,eqc->eai", ref.wq, U, ref.dphi, Wt)
    wn, jump, avg, PJ, Ph = facet_quantities(mesh, ref, wL, uL, l, u_inlet)
    g = wn[..., None] * avg + Ph
    for side, sgn in (("A", 1.0), ("B", -1.0)):
        ef = mesh.fa if side == "A" else mesh.fb
        for f in range(6):
            msk = ef[:, 1] == f
            if np.any(msk):
                contrib = sgn * mesh.aF[msk, None, None] * np.einsum("p,Fpa,pi->Fai", ref.wf, g[msk], ref.phi_f[f])
                np.add.at(r, ef[msk, 0], contrib)
    return r


def apply(mesh: HexMesh, ref: RefHex, wL, uL, l: int, u_inlet=None) -> np.ndarray:
    """y = M_L^-1 c(w; u, .), M_T = |det J| I."""
    return residual(mesh, ref, wL, uL, l, u_inlet) / mesh.absdet[:, None, None]


def end_facets(mesh: HexMesh, d: int, end: int) -> np.ndarray:
    """The boundary facets at the low (end 0) or high (end 1) end of non-periodic direction
    d, ordered by the cells' two other indices (lower axis fastest)."""
    E = mesh.n_elems
    a_other = [b for b in range(3) if b != d]
    cells = np.where(mesh.cell[:, d] == (0 if end == 0 else mesh.n[d] - 1))[0]
    key = mesh.cell[cells, a_other[0]] + mesh.n[a_other[0]] * mesh.cell[cells, a_other[1]]
    cells = cells[np.argsort(key)]
    local = 2 * d + (0 if end == 0 else 1)
    out = []
    for e in cells:
        F = np.where((mesh.fa[:, 0] == e) & (mesh.fa[:, 1] == local) & mesh.boundary)[0]
        out.append(int(F[0]))
    return np.array(out, dtype=np.int64)


def form_value(mesh, ref, wL, uL, l) -> float:
    """c(w; u, u)."""
    return float(np.sum(uL * residual(mesh, ref, wL, uL, l)))


def facet_dissipation(mesh, ref, wL, uL, l) -> float:
    """sum_F int_F 1/2 |w.n| |(I - Pi^l)[[u]]|^2."""
    wn, jump, avg, PJ, Ph = facet_quantities(mesh, ref, wL, uL, l)
    return float(np.sum(mesh.aF[:, None] * ref.wf[None, :] * 0.5 * np.abs(wn) * np.sum(PJ * PJ, axis=-1)))


def facet_eta(mesh: HexMesh, ref: RefHex, uL, l) -> np.ndarray:
    """Adaptive HOPU's jump indicator per facet (Section 3.2, after eq. "hopudefinition"):
    eta = int_E |(I - Pi^l)[[u]]| ds / int_E |<u>| ds with the facet's current order l (one
    or one per facet); the readings of oracle/adaptive.py (a zero average with a non-zero
    jump: +inf; both zero: 0).  The orders follow from adaptive.order_from_eta."""
    _, jump, avg, PJ, _ = facet_quantities(mesh, ref, uL, uL, l)
    num = np.einsum("p,Fp->F", ref.wf, np.linalg.norm(PJ, axis=-1))
    den = np.einsum("p,Fp->F", ref.wf, np.linalg.norm(avg, axis=-1))
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(den > 0, num / np.where(den > 0, den, 1.0), np.where(num > 0, np.inf, 0.0))


def kinetic_energy(mesh, uL) -> float:
    """1/2 int |u|^2 = 1/2 sum_T |det J| |c_T|^2."""
    return 0.5 * float(np.sum(mesh.absdet[:, None, None] * uL * uL))


def substeps_stage(mesh, ref, uL, dt: float, n: int, l: int, u_inlet=None) -> np.ndarray:
    """n SSP-RK3 substeps of du/dt = -M^-1 c(u; u, .) in L_h (the STAGE wind w = u;
    the Shu-Osher stages of oracle/rk.py)."""
    from .rk import ssp_rk3
    u = np.array(uL, dtype=np.float64)
    for _ in range(n):
        u = ssp_rk3(lambda v: apply(mesh, ref, v, v, l, u_inlet), u, dt)
    return u

"""Pins of the hexahedral oracle (oracle/hexa.py) against what the mathematics fixes:
closed forms of the Legendre polynomials and Gauss moments, orthonormality, finite
differences, the divergence theorem on the reference cell, the box's volume and closed cells,
facet points that coincide from both sides, the constant-state and energy identities of
Section 3.2, the l = k limit, the Q^l orthogonality of (I - Pi^l), and the value of the form
on the same box split into tetrahedra (the simplicial oracle, pinned on its own) for
polynomial fields."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import convection as C
from oracle import hexa as H
from oracle.fe import ref_element
from oracle.mesh import MeshTopo


def test_legendre_closed_forms():
    x = np.array([0.0, 0.13, 0.5, 0.77, 1.0])
    V, D = H.legendre01(3, x)
    assert np.allclose(V[:, 0], 1.0, atol=1e-15)
    assert np.allclose(V[:, 1], math.sqrt(3) * (2 * x - 1), atol=1e-14)
    assert np.allclose(V[:, 2], math.sqrt(5) * (6 * x * x - 6 * x + 1), atol=1e-14)
    assert np.allclose(V[:, 3], math.sqrt(7) * (20 * x**3 - 30 * x**2 + 12 * x - 1), atol=1e-13)
    assert np.allclose(D[:, 0], 0.0)
    assert np.allclose(D[:, 1], 2 * math.sqrt(3), atol=1e-14)
    assert np.allclose(D[:, 2], math.sqrt(5) * (12 * x - 6), atol=1e-13)
    assert np.allclose(D[:, 3], math.sqrt(7) * (60 * x**2 - 60 * x + 12), atol=1e-12)


@pytest.mark.parametrize("m", [2, 4, 7])
def test_gauss_moments(m):
    x, w = H.gauss01(m)
    for p in range(2 * m):
        assert np.dot(w, x**p) == pytest.approx(1.0 / (p + 1), rel=1e-13)
    assert abs(np.dot(w, x ** (2 * m)) - 1.0 / (2 * m + 1)) > 1e-10    # and not beyond 2m-1


def test_points_per_direction():
    assert [H.points_per_direction(k) for k in (1, 2, 3, 4, 5)] == [2, 4, 5, 7, 8]


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_orthonormal_and_exact(k):
    ref = H.RefHex(k)
    G = np.einsum("q,qi,qj->ij", ref.wq, ref.phi, ref.phi)
    assert np.abs(G - np.eye(ref.nb)).max() < 1e-13
    # basis index i = i1 + (k+1)(i2 + (k+1) i3): phi_i at x = L_i1(x1) L_i2(x2) L_i3(x3)
    x = np.array([[0.2, 0.7, 0.4]])
    L = [H.legendre01(k, x[:, a])[0][0] for a in range(3)]
    i1, i2, i3 = k, 1 % (k + 1), 0
    assert H.basis(k, x)[0][0, i1 + (k + 1) * (i2 + (k + 1) * i3)] == pytest.approx(L[0][i1] * L[1][i2] * L[2][i3])
    # the facet rule integrates degree 3k in each direction
    g = ref.sq[:, 0] ** (3 * k) * ref.sq[:, 1] ** (3 * k)
    assert np.dot(ref.wf, g) == pytest.approx(1.0 / (3 * k + 1) ** 2, rel=1e-12)


def test_gradient_finite_differences():
    k = 3
    rng = np.random.default_rng(4)
    x = rng.uniform(0.1, 0.9, size=(5, 3))
    _, dphi = H.basis(k, x)
    h = 1e-6
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        fd = (H.basis(k, x + e)[0] - H.basis(k, x - e)[0]) / (2 * h)
        assert np.abs(fd - dphi[:, :, c]).max() < 1e-6


@pytest.mark.parametrize("k", [2, 3])
def test_reference_divergence_theorem(k):
    """int_T^ d_c phi_i = sum_f N^_f,c int_F^ phi_i (facet traces, normals, volume gradients)."""
    ref = H.RefHex(k)
    lhs = np.einsum("q,qic->ic", ref.wq, ref.dphi)
    rhs = np.einsum("fc,p,fpi->ic", ref.Nhat, ref.wf, ref.phi_f)
    assert np.abs(lhs - rhs).max() < 1e-12


def _box(seed=1, n=3):
    return W.hex_box(n, jitter=0.25, shear=0.4, seed=seed)


def test_mesh_geometry():
    hb = _box(2, (3, 4, 5))
    m = H.HexMesh(hb)
    vol = np.linalg.det(hb.A) * np.prod([x[-1] for x in hb.lines])
    assert m.absdet.sum() == pytest.approx(vol, rel=1e-13)
    assert m.n_facets == 3 * m.n_elems
    # every cell is closed: its outward area vectors sum to zero
    acc = np.zeros((m.n_elems, 3))
    np.add.at(acc, m.fa[:, 0], m.aF[:, None] * m.nF)
    np.add.at(acc, m.fb[:, 0], -m.aF[:, None] * m.nF)
    assert np.abs(acc).max() < 1e-12
    # each facet once as side A and once as side B of each cell direction
    assert np.all(np.bincount(m.fa[:, 0], minlength=m.n_elems) == 3)
    assert np.all(np.bincount(m.fb[:, 0], minlength=m.n_elems) == 3)
    # the facet points of both sides coincide up to a period of the box
    ref = H.RefHex(2)
    d = m.facet_points(ref, "A") - m.facet_points(ref, "B")
    coef = np.einsum("Fpc,ac->Fpa", d, np.linalg.inv(m.lattice.T))  # d = sum_a coef_a period_a
    assert np.abs(coef - np.rint(coef)).max() < 1e-12
    assert np.abs(d[:, 1:] - d[:, :1]).max() < 1e-12                   # one shift per facet


def _const(v):
    return lambda x: np.broadcast_to(np.asarray(v, dtype=float), x.shape).copy()


@pytest.mark.parametrize("k", [2, 3])
def test_constant_state_gives_zero(k):
    m, ref = H.HexMesh(_box(3)), H.RefHex(k)
    u = H.project(m, ref, _const([1.0, -2.0, 0.5]))
    w = H.project(m, ref, _const([0.3, 0.7, -0.4]))
    for l in (-1, 0, k - 1, k):
        assert np.abs(H.apply(m, ref, w, u, l)).max() < 1e-12


def _div_free(k):
    """A divergence-free polynomial wind of total degree <= k whose component a does not
    depend on x_a, so that on an axis-aligned periodic box its normal component is
    continuous across every facet, the periodic seams included."""
    if k >= 3:
        return lambda x: np.stack([1e-2 * x[..., 1] ** 2 * x[..., 2] + 0.4,
                                   1e-2 * x[..., 0] * x[..., 2] ** 2 - 0.3,
                                   1e-2 * x[..., 0] ** 2 * x[..., 1] + 0.2], axis=-1)
    return lambda x: np.stack([0.1 * x[..., 1] * x[..., 2] + 0.4, 0.1 * x[..., 0] * x[..., 2] - 0.3,
                               0.1 * x[..., 0] * x[..., 1] + 0.2], axis=-1)


@pytest.mark.parametrize("k", [2, 3])
def test_energy_identity(k):
    """c(w; u, u) = sum_F int 1/2 |w.n| |(I - Pi^l)[[u]]|^2 for a divergence-free w with a
    continuous normal component (axis-aligned cells of uneven size: no shear)."""
    m, ref = H.HexMesh(W.hex_box(3, jitter=0.25, shear=0.0, seed=4)), H.RefHex(k)
    w = H.project(m, ref, _div_free(k))
    u = W.uniform_noise(m.n_elems * 3 * ref.nb, 1.0, 5).reshape(m.n_elems, 3, ref.nb)
    for l in (-1, 0, 1, k):
        cv = H.form_value(m, ref, w, u, l)
        dis = H.facet_dissipation(m, ref, w, u, l)
        assert dis > 0
        assert cv == pytest.approx(dis, rel=1e-11)


def test_l_equals_k_keeps_the_normal_jump_only():
    k = 3
    m, ref = H.HexMesh(_box(5)), H.RefHex(k)
    u = W.uniform_noise(m.n_elems * 3 * ref.nb, 1.0, 6).reshape(m.n_elems, 3, ref.nb)
    w = W.uniform_noise(m.n_elems * 3 * ref.nb, 1.0, 7).reshape(m.n_elems, 3, ref.nb)
    _, jump, _, PJ, _ = H.facet_quantities(m, ref, w, u, k)
    normal = np.einsum("Fpa,Fa->Fp", jump, m.nF)[..., None] * m.nF[:, None, :]
    assert np.abs(PJ - normal).max() < 1e-12
    _, jump, _, PJ, _ = H.facet_quantities(m, ref, w, u, -1)
    assert np.abs(PJ - jump).max() == 0.0


@pytest.mark.parametrize("l", [0, 1, 2])
def test_complement_is_orthogonal_to_tangential_q_l(l):
    """(I - Pi^l) V is L2(F)-orthogonal to every tangential field with Q^l components, and
    not to the Q^(l+1) modes outside Q^l (a P^l projection would fail the first check)."""
    k = 3
    ref = H.RefHex(k)
    rng = np.random.default_rng(8)
    V = rng.standard_normal((4, ref.wf.size, 3))
    nF = rng.standard_normal((4, 3))
    nF /= np.linalg.norm(nF, axis=1, keepdims=True)
    R = H.complement_projection(ref, l, nF, V)
    Rt = R - np.einsum("Fpa,Fa->Fp", R, nF)[..., None] * nF[:, None, :]
    for mm in ref.q_modes(l):
        assert np.abs(np.einsum("p,p,Fpa->Fa", ref.wf, ref.psi[:, mm], Rt)).max() < 1e-12
    outside = [mm for mm in range(ref.psi.shape[1]) if ref.psi_deg[mm] == l + 1]
    big = max(np.abs(np.einsum("p,p,Fpa->Fa", ref.wf, ref.psi[:, mm], Rt)).max() for mm in outside)
    assert big > 1e-3
    # the normal part is untouched
    assert np.abs(np.einsum("Fpa,Fa->Fp", R - V, nF)).max() < 1e-12


def _poly(k, seed, scale=1.0, base=None):
    """A random vector polynomial of total degree <= k in x / (2 pi)."""
    rng = np.random.default_rng(seed)
    exps = [(a, b, c) for a in range(k + 1) for b in range(k + 1) for c in range(k + 1) if a + b + c <= k]
    coef = rng.uniform(-1.0, 1.0, size=(len(exps), 3)) * scale / len(exps)

    def f(x):
        y = x / (2 * math.pi)
        out = np.zeros(x.shape[:-1] + (3,))
        for (a, b, c), cf in zip(exps, coef):
            out += (y[..., 0] ** a * y[..., 1] ** b * y[..., 2] ** c)[..., None] * cf
        if base is not None:
            out += base
        return out

    return f


def _tet_project(topo, ref, f):
    X = topo.volume_points(ref.xq)
    return np.einsum("q,eqa,qi->eai", ref.wq, f(X), ref.phi)


@pytest.mark.parametrize("k", [2, 3])
def test_form_equals_the_simplicial_oracle(k):
    """For global polynomial u, v, w of total degree <= k (in both spaces), pure upwind
    (l = -1), the form c(w; u, v) on the hexahedral box equals the one on the same box
    split into tetrahedra: the volume integrals are the same polynomial integrals, interior
    jumps vanish, and on the periodic seam both integrate the same facet terms (w.n keeps
    one sign there, so |w.n| is a polynomial).  The two oracles share no code."""
    hb = _box(6)
    m, ref = H.HexMesh(hb), H.RefHex(k)
    tets = W.hex_box_tets(hb)
    topo, tref = MeshTopo(tets.coords, tets.elems, tets.rep), ref_element(3, k)
    base = hb.A @ np.ones(3)                          # A^-1 w = (1, 1, 1): w.n > 0 on every seam
    fw = _poly(k, 11, 0.2, base)
    fu, fv = _poly(k, 12), _poly(k, 13)
    wn, *_ = H.facet_quantities(m, ref, H.project(m, ref, fw), H.project(m, ref, fu), -1)
    assert wn.min() > 0.1
    vals = []
    for proj, res, mesh_, ref_ in ((H.project, None, m, ref), (_tet_project, None, topo, tref)):
        uL, wL, vL = proj(mesh_, ref_, fu), proj(mesh_, ref_, fw), proj(mesh_, ref_, fv)
        if mesh_ is m:
            r = H.residual(m, ref, wL, uL, -1)
        else:
            r = C.residual_conservative(topo, tref, wL, uL, -1)
        vals.append(float(np.sum(vL * r)))
    assert abs(vals[0]) > 1e-3
    assert vals[0] == pytest.approx(vals[1], rel=1e-11)


class _Poly:
    """A vector polynomial of total degree <= k in y = x / (2 pi), with its gradient."""

    def __init__(self, k, seed, scale=1.0, base=None):
        rng = np.random.default_rng(seed)
        self.exps = [(a, b, c) for a in range(k + 1) for b in range(k + 1) for c in range(k + 1) if a + b + c <= k]
        self.coef = rng.uniform(-1.0, 1.0, size=(len(self.exps), 3)) * scale / len(self.exps)
        self.base = np.zeros(3) if base is None else np.asarray(base, dtype=float)

    def __call__(self, x):
        y = x / (2 * math.pi)
        out = np.zeros(x.shape[:-1] + (3,)) + self.base
        for (a, b, c), cf in zip(self.exps, self.coef):
            out += (y[..., 0] ** a * y[..., 1] ** b * y[..., 2] ** c)[..., None] * cf
        return out

    def grad(self, x):
        """[..., component, direction]"""
        y = x / (2 * math.pi)
        out = np.zeros(x.shape[:-1] + (3, 3))
        for (a, b, c), cf in zip(self.exps, self.coef):
            ex = (a, b, c)
            for d in range(3):
                if ex[d] == 0:
                    continue
                e2 = list(ex)
                e2[d] -= 1
                m = ex[d] * y[..., 0] ** e2[0] * y[..., 1] ** e2[1] * y[..., 2] ** e2[2] / (2 * math.pi)
                out[..., :, d] += m[..., None] * cf
        return out


@pytest.mark.parametrize("k,periodic", [(2, (False, False, False)), (3, (True, False, False)),
                                        (3, (False, True, False))])
def test_walls_reduce_to_the_volume_integral(k, periodic):
    """With walls / outlets in the non-periodic directions and polynomial u, w continuous
    across every interior facet (no jumps; in a periodic direction the fields must be
    periodic, so they do not depend on that coordinate there), c(w; u, phi_i e_a) equals
    int_T ((grad u) w + (div w) u)_a phi_i, evaluated directly from the polynomials'
    analytic gradients: the boundary flux of the conservative form cancels the cell-wise
    integration by parts, and Section 2.1's wall / outlet facets add no term."""
    hb = W.hex_box(3, jitter=0.25, shear=0.0, seed=12)
    m, ref = H.HexMesh(hb, periodic=periodic), H.RefHex(k)
    pu, pw = _Poly(k, 21), _Poly(k, 22, 0.3, base=[0.4, -0.3, 0.2])
    for P in (pu, pw):                                   # drop the periodic coordinates
        keep = [i for i, ex in enumerate(P.exps) if all(ex[d] == 0 for d in range(3) if periodic[d])]
        P.exps = [P.exps[i] for i in keep]
        P.coef = P.coef[keep]
    uL, wL = H.project(m, ref, pu), H.project(m, ref, pw)
    r = H.residual(m, ref, wL, uL, -1)
    X = m.volume_points(ref.xq)
    U, Wv, GU, GW = pu(X), pw(X), pu.grad(X), pw.grad(X)
    g = np.einsum("eqab,eqb->eqa", GU, Wv) + np.einsum("eqbb->eq", GW)[..., None] * U
    direct = np.einsum("q,e,eqa,qi->eai", ref.wq, m.absdet, g, ref.phi)
    assert np.abs(r - direct).max() < 1e-11 * np.abs(direct).max()
    assert m.boundary.sum() == sum(2 * m.n_elems // m.n[a] for a in range(3) if not periodic[a])


def test_walls_match_the_simplicial_oracle():
    """A box walled on all six sides, split into tetrahedra (no periodic identification),
    polynomial fields: the two oracles' forms agree for any HOPU order, every facet jump
    being zero (interior: continuous fields; walls: the own trace)."""
    k = 2
    hb = W.hex_box(3, jitter=0.25, shear=0.3, seed=14)
    m, ref = H.HexMesh(hb, periodic=(False, False, False)), H.RefHex(k)
    tets = W.hex_box_tets(hb)
    topo, tref = MeshTopo(tets.coords, tets.elems, None), ref_element(3, k)
    assert np.any(topo.boundary)
    fu, fw, fv = _Poly(k, 31), _Poly(k, 32, 0.3, base=[0.2, 0.5, -0.4]), _Poly(k, 33)
    for l in (-1, 1):
        rh = H.residual(m, ref, H.project(m, ref, fw), H.project(m, ref, fu), l)
        rt = C.residual_conservative(topo, tref, _tet_project(topo, tref, fw), _tet_project(topo, tref, fu), l)
        ch = float(np.sum(H.project(m, ref, fv) * rh))
        ct = float(np.sum(_tet_project(topo, tref, fv) * rt))
        assert abs(ch) > 1e-3
        assert ch == pytest.approx(ct, rel=1e-11)


def test_inlet_matches_the_simplicial_oracle():
    """A walled box with an inlet at the low end of direction 1 (exterior velocity g, the
    wind's own trace, Section 2.2): for polynomial fields with inflow (w.n < 0 on the whole
    inlet, so |w.n| is a polynomial there) the hexahedral and simplicial forms agree; with
    g the field's own trace the inlet adds nothing (the walled form)."""
    k = 2
    hb = W.hex_box(3, jitter=0.25, shear=0.3, seed=15)
    m, ref = H.HexMesh(hb, periodic=(False, False, False)), H.RefHex(k)
    tets = W.hex_box_tets(hb)
    topo, tref = MeshTopo(tets.coords, tets.elems, None), ref_element(3, k)
    base = hb.A @ np.array([0.0, 0.6, 0.0])                # A^-1 w = (0, 0.6, 0): inflow at y = 0
    fu, fw, fv, fg = _Poly(k, 41), _Poly(k, 42, 0.2, base=base), _Poly(k, 43), _Poly(k, 44)
    Ainv = np.linalg.inv(hb.A)
    # hexahedral inlet facets: the low end of direction 1
    Fin = H.end_facets(m, 1, 0)
    pts = m.facet_points(ref, "A")
    uin = {int(F): fg(pts[F]) for F in Fin}
    # simplicial inlet facets: boundary facets in the plane (A^-1 x)_1 = 0
    P = topo.facet_points(tref.sq)
    xi = np.einsum("ab,Fqb->Fqa", Ainv, P)
    inlet = topo.boundary & (np.abs(xi[:, :, 1]).max(axis=1) < 1e-12)
    assert inlet.sum() == 2 * len(Fin)                     # two triangles per quadrilateral
    wLt, uLt = _tet_project(topo, tref, fw), _tet_project(topo, tref, fu)
    ext = (fg(P), C.facet_trace(topo, tref, wLt, "A"))
    for l in (-1,):
        rh = H.residual(m, ref, H.project(m, ref, fw), H.project(m, ref, fu), l, uin)
        rt = C.residual_conservative(topo, tref, wLt, uLt, l, exterior=ext, inlet=inlet)
        ch = float(np.sum(H.project(m, ref, fv) * rh))
        ct = float(np.sum(_tet_project(topo, tref, fv) * rt))
        assert ch == pytest.approx(ct, rel=1e-11)
    # the field's own trace as inlet data: the walled form
    own = {int(F): H._traces(m, ref, H.project(m, ref, fu), "A")[F] for F in Fin}
    r_own = H.residual(m, ref, H.project(m, ref, fw), H.project(m, ref, fu), 1, own)
    r_wall = H.residual(m, ref, H.project(m, ref, fw), H.project(m, ref, fu), 1)
    assert np.abs(r_own - r_wall).max() < 1e-13 * np.abs(r_wall).max()


@pytest.mark.parametrize("k,ns", [(2, (3, 6, 12)), (3, (6, 12))])
def test_order_k_consistency_on_taylor_green(k, ns):
    """The discrete (u . grad) u of the L2-projected Taylor-Green field converges at order k
    in L2 on periodic cubes of the 2 pi box (HOPU l = k - 1)."""
    errs = []
    for n in ns:
        m, ref = H.HexMesh(W.hex_box(n)), H.RefHex(k)
        uL = H.project(m, ref, W.taylor_green)
        y = H.apply(m, ref, uL, uL, k - 1)
        diff = y - H.project(m, ref, W.taylor_green_convective)
        errs.append(np.sqrt(np.sum(m.absdet[:, None, None] * diff ** 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > k - 0.25 and np.all(rates > k - 0.35), (errs, rates)   # k = 2: 2.67; k = 3: 2.83


def test_eta_closed_forms():
    """eta for a field constant c1 / c2 on alternate layers of cells in direction 0 (a jump
    only across the facets of direction 0): |c1 - c2| / |c1 + c2| * 2 there with l = -1,
    the normal part of the jump only with l >= 0 (Q^0 holds the constant tangential part),
    0 on the other facets; 0 everywhere for a continuous field."""
    hb = W.hex_box(4, jitter=0.2, shear=0.0, seed=16)
    m, ref = H.HexMesh(hb), H.RefHex(2)
    c1, c2 = np.array([1.0, -0.5, 0.25]), np.array([0.2, 0.4, -0.6])
    uL = np.zeros((m.n_elems, 3, ref.nb))
    layer = m.cell[:, 0] % 2 == 0
    uL[layer, :, 0], uL[~layer, :, 0] = c1, c2
    E = m.n_elems
    jump = np.linalg.norm(c1 - c2)
    want = jump / np.linalg.norm(0.5 * (c1 + c2))
    eta = H.facet_eta(m, ref, uL, -1)
    assert np.allclose(eta[:E], want, rtol=1e-12) and np.abs(eta[E:]).max() < 1e-14
    eta0 = H.facet_eta(m, ref, uL, 0)                    # no shear: n_F = e_0 on those facets
    assert np.allclose(eta0[:E], abs((c1 - c2)[0]) / np.linalg.norm(0.5 * (c1 + c2)), rtol=1e-12)
    uc = H.project(m, ref, lambda x: np.stack([np.sin(0 * x[..., 0]) + 1.0, 0 * x[..., 1], 0 * x[..., 2]], -1))
    assert np.abs(H.facet_eta(m, ref, uc, -1)).max() < 1e-13
    # per-facet orders act facet by facet: against the uniform l = -1 result, only cells with
    # a facet of another order change, and a uniform order array equals the scalar order
    w, u = W.uniform_noise(uL.size, 1.0, 3).reshape(uL.shape), W.uniform_noise(uL.size, 1.0, 4).reshape(uL.shape)
    lF = np.full(m.n_facets, -1)
    lF[np.random.default_rng(5).choice(m.n_facets, size=20, replace=False)] = 1
    diff = np.abs(H.apply(m, ref, w, u, lF) - H.apply(m, ref, w, u, -1)).max(axis=(1, 2))
    touched = np.zeros(m.n_elems, dtype=bool)
    touched[m.fa[lF == 1, 0]] = True
    touched[m.fb[lF == 1, 0]] = True
    assert diff[~touched].max() == 0.0 and diff[touched].min() > 0.0
    assert np.abs(H.apply(m, ref, w, u, np.full(m.n_facets, 1)) - H.apply(m, ref, w, u, 1)).max() == 0.0

"""Pins of the oracle's HOPU convection operator and substeps (CPU only).

Each pin is a property the paper's form fixes (Section 2.2 eq. "upwind",
Section 3.2 eq. "hopudefinition" and the limits stated after it), checked on
inputs built independently of the operator (curl fields, polynomials written
out by hand, Taylor-Green data).
"""
import numpy as np
import pytest

import workloads as W
from oracle import convection as C
from oracle import fe, fields, hdiv, mesh, rk

CASES = [(2, 4, 2), (3, 3, 2), (3, 3, 3)]


def _space(dim, n, k, **kw):
    m = W.periodic_box_mesh(dim, n)
    topo = mesh.MeshTopo(m.coords, m.elems, m.rep)
    return hdiv.HDiv(topo, fe.RefElement(dim, k, **kw) if kw else fe.ref_element(dim, k))


def _divfree(sp, seed=3):
    return fields.curl_field(sp.topo, sp.ref.dim, sp.ref.k, fields.random_potential(sp.ref.dim, seed))


def _ls(k):
    return [-1, 0, k - 1, k]


@pytest.mark.parametrize("dim,n,k", CASES)
def test_P1_constant_u_divfree_w_gives_zero(dim, n, k):
    sp = _space(dim, n, k)
    wL = _divfree(sp)
    uc = sp.l2_project(W.constant_field(np.arange(1, dim + 1) * 0.7))
    # a wrong operator gives |y| ~ |w| |u| / h; rounding gives ~1e-15 of that
    scale = np.abs(wL).max() * np.abs(uc).max() * n / (2 * np.pi) * sp.ref.nb
    for l in _ls(k):
        y = C.apply(sp.topo, sp.ref, wL, uc, l)
        assert np.abs(y).max() < 1e-13 * scale


@pytest.mark.parametrize("dim,n,k", CASES)
def test_P2_conservative_equals_paper_form_for_divfree_wind(dim, n, k):
    sp = _space(dim, n, k)
    wL = _divfree(sp)
    uL = np.random.default_rng(4).standard_normal(wL.shape)
    for l in _ls(k):
        r1 = C.residual_conservative(sp.topo, sp.ref, wL, uL, l)
        r2 = C.residual_nonconservative(sp.topo, sp.ref, wL, uL, l)
        assert np.abs(r1 - r2).max() < 1e-13 * np.abs(r1).max()


def test_P2_forms_differ_by_divergence_term_otherwise():
    # with a wind that is not divergence-free the two forms must differ by
    # sum_T int (div w) u.v -- a check that the test above is not vacuous
    sp = _space(2, 4, 2)
    rng = np.random.default_rng(5)
    wV = rng.standard_normal(sp.n_hdiv)
    wL, uL = sp.to_l2(wV), rng.standard_normal((sp.topo.n_elems, 2, sp.ref.nb))
    r1 = C.residual_conservative(sp.topo, sp.ref, wL, uL, -1)
    r2 = C.residual_nonconservative(sp.topo, sp.ref, wL, uL, -1)
    divw = np.einsum("qic,eai,eca->eq", sp.ref.dphi, wL, sp.topo.Jinv)
    U = np.einsum("qi,eai->eqa", sp.ref.phi, uL)
    extra = np.einsum("q,e,eq,eqa,qi->eai", sp.ref.wq, sp.topo.absdet, divw, U, sp.ref.phi)
    assert np.abs(r1 - r2).max() > 1e-3
    assert np.abs(r1 - r2 - extra).max() < 1e-12 * np.abs(extra).max()


@pytest.mark.parametrize("dim,n,k", CASES)
def test_P3_energy_identity(dim, n, k):
    sp = _space(dim, n, k)
    wL = _divfree(sp)
    uL = np.random.default_rng(6).standard_normal(wL.shape)
    for l in _ls(k):
        cval = C.form_value(sp.topo, sp.ref, wL, uL, l)
        diss = C.facet_dissipation(sp.topo, sp.ref, wL, uL, l)
        assert diss > 0
        assert abs(cval - diss) < 1e-12 * diss


@pytest.mark.parametrize("dim,n,k", CASES)
def test_P4_central_limit_and_upwind_limit(dim, n, k):
    sp = _space(dim, n, k)
    wL = _divfree(sp)
    uL = sp.to_l2(np.random.default_rng(7).standard_normal(sp.n_hdiv))
    ref_scale = C.facet_dissipation(sp.topo, sp.ref, wL, uL, -1)
    # l = k and u in E(V_h): no dissipation at all (central flux)
    assert abs(C.form_value(sp.topo, sp.ref, wL, uL, k)) < 1e-12 * ref_scale
    # l = -1 is the standard upwind form of Section 2.2: 1/2 |w.n| [[u]].[[v]]
    wn, jump, avg, PJ, Ph = C.facet_quantities(sp.topo, sp.ref, wL, uL, -1)
    assert np.array_equal(PJ, jump)
    assert np.allclose(Ph, 0.5 * np.abs(wn)[..., None] * jump, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim,n,k", CASES)
def test_P5_dissipation_non_increasing_in_l_for_constant_wind(dim, n, k):
    sp = _space(dim, n, k)
    wL = sp.l2_project(W.constant_field(np.linspace(0.3, 1.1, dim)))
    uL = np.random.default_rng(8).standard_normal(wL.shape)
    vals = [C.form_value(sp.topo, sp.ref, wL, uL, l) for l in range(-1, k + 1)]
    assert all(a >= b - 1e-12 * vals[0] for a, b in zip(vals, vals[1:]))
    assert vals[0] > vals[-1]


@pytest.mark.parametrize("dim,n,k", CASES)
def test_P6_momentum_conservation(dim, n, k):
    sp = _space(dim, n, k)
    rng = np.random.default_rng(9)
    wL = sp.to_l2(rng.standard_normal(sp.n_hdiv))
    uL = rng.standard_normal(wL.shape)
    for l in _ls(k):
        y = C.apply(sp.topo, sp.ref, wL, uL, l)
        # int y_a = sum_T |det J| y_{a,0} / phi_0 ; the test function e_a has no jump
        mom = np.sum(sp.topo.absdet[:, None] * y[:, :, 0], axis=0)
        assert np.abs(mom).max() < 1e-12 * np.sum(sp.topo.absdet[:, None] * np.abs(y[:, :, 0]))


def _poly_field(dim, k, seed):
    """A random vector polynomial of degree k and its gradient, written out in monomials."""
    import itertools
    rng = np.random.default_rng(seed)
    exps = [e for e in itertools.product(range(k + 1), repeat=dim) if sum(e) <= k]
    A = rng.standard_normal((dim, len(exps)))

    def u(x):
        mons = np.stack([np.prod(x ** np.array(e), axis=-1) for e in exps], axis=-1)
        return mons @ A.T

    def grad(x):  # [.., a, b] = d u_a / d x_b
        out = np.zeros(x.shape[:-1] + (dim, dim))
        for j, e in enumerate(exps):
            for b in range(dim):
                if e[b] == 0:
                    continue
                e2 = list(e)
                e2[b] -= 1
                mono = e[b] * np.prod(x ** np.array(e2), axis=-1)
                out[..., :, b] += mono[..., None] * A[:, j]
        return out
    return u, grad


@pytest.mark.parametrize("dim,k", [(2, 2), (3, 2), (3, 3)])
def test_P7_single_element_inlet_exactness(dim, k):
    # one element, every facet an inlet facet whose exterior value is u itself:
    # then y = L2 projection of (w . grad) u, which is exact for polynomial u.
    if dim == 3:
        coords = np.array([[0.0, 0, 0], [1.0, 0.1, 0], [0.2, 1.1, 0.1], [0.1, 0.3, 0.9]])
    else:
        coords = np.array([[0.0, 0.0], [1.2, 0.1], [0.3, 0.9]])
    topo = mesh.MeshTopo(coords, np.arange(dim + 1)[None, :])
    ref = fe.ref_element(dim, k)
    sp = hdiv.HDiv(topo, ref)
    u, grad = _poly_field(dim, k, 11)
    wconst = np.linspace(0.4, -0.9, dim)
    wfun = W.constant_field(wconst)
    uL, wL = sp.l2_project(u), sp.l2_project(wfun)
    pts = topo.facet_points(ref.sq)
    ext = (u(pts), wfun(pts))
    expect = sp.l2_project(lambda x: np.einsum("...ab,b->...a", grad(x), wconst))
    for l in _ls(k):
        y = C.apply(topo, ref, wL, uL, l, exterior=ext)
        assert np.abs(y - expect).max() < 1e-12 * np.abs(expect).max()


@pytest.mark.parametrize("dim,k,ns", [(2, 2, (4, 8, 16)), (3, 2, (3, 6, 12))])
def test_P8_order_k_consistency_on_taylor_green(dim, k, ns):
    errs = []
    for n in ns:
        sp = _space(dim, n, k)
        uL = sp.to_l2(sp.interpolate(W.taylor_green))
        y = C.apply(sp.topo, sp.ref, uL, uL, k - 1)
        diff = y - sp.l2_project(W.taylor_green_convective)
        errs.append(np.sqrt(np.sum(sp.topo.absdet[:, None, None] * diff ** 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > k - 0.2 and np.all(rates > k - 0.3), (errs, rates)


def test_P11_frozen_substep_is_third_order_taylor():
    sp = _space(2, 4, 2)
    wV = sp.from_l2(_divfree(sp))
    rng = np.random.default_rng(12)
    uL = rng.standard_normal((sp.topo.n_elems, 2, sp.ref.nb))
    dt = 0.05
    wL = sp.to_l2(wV)
    A = lambda v: C.apply(sp.topo, sp.ref, wL, v, 1)
    Au = A(uL)
    A2u = A(Au)
    A3u = A(A2u)
    expect = uL - dt * Au + dt ** 2 / 2 * A2u - dt ** 3 / 6 * A3u
    got = rk.substeps_frozen(sp, wV, uL, dt, 1, 1)
    assert np.abs(got - expect).max() < 1e-13 * np.abs(uL).max()


@pytest.mark.parametrize("dim,n,k", [(2, 3, 2), (3, 3, 2)])
def test_P12_rule_is_exact_where_the_integrand_is_polynomial(dim, n, k):
    # l = k with u, w in V_h (no |w.n| term survives) and l = -1 with a constant
    # wind (|w.n| constant per facet): richer rules must give the same result.
    sp = _space(dim, n, k)
    sp4 = _space(dim, n, k, vol_degree=3 * k + 3, facet_degree=3 * k + 4)
    rng = np.random.default_rng(13)
    uV, wV = rng.standard_normal(sp.n_hdiv), rng.standard_normal(sp.n_hdiv)
    y = C.apply(sp.topo, sp.ref, sp.to_l2(wV), sp.to_l2(uV), k)
    y4 = C.apply(sp4.topo, sp4.ref, sp4.to_l2(wV), sp4.to_l2(uV), k)
    assert np.abs(y - y4).max() < 1e-12 * np.abs(y).max()
    wc = W.constant_field(np.linspace(0.2, 1.0, dim))
    uL = rng.standard_normal((sp.topo.n_elems, dim, sp.ref.nb))
    y = C.apply(sp.topo, sp.ref, sp.l2_project(wc), uL, -1)
    y4 = C.apply(sp4.topo, sp4.ref, sp4.l2_project(wc), uL, -1)
    assert np.abs(y - y4).max() < 1e-12 * np.abs(y).max()


def test_stage_substep_conserves_momentum_and_is_consistent():
    # STAGE substeps: parity unpinned beyond GPU agreement; check the two
    # properties the scheme must keep: momentum and first-order consistency.
    sp = _space(2, 4, 2)
    uV = sp.interpolate(W.taylor_green)
    dt = 1e-3
    u1 = rk.substeps_stage(sp, uV, dt, 1, 1)
    y = sp.from_l2(C.apply(sp.topo, sp.ref, sp.to_l2(uV), sp.to_l2(uV), 1))
    assert np.abs((u1 - uV) / dt + y).max() < 5e-2 * np.abs(y).max()
    m0 = np.sum(sp.topo.absdet[:, None] * sp.to_l2(uV)[:, :, 0], axis=0)
    m1 = np.sum(sp.topo.absdet[:, None] * sp.to_l2(u1)[:, :, 0], axis=0)
    assert np.abs(m1 - m0).max() < 1e-12


def _locate(topo, x):
    """(element, reference point) of physical points x [P, d] inside the periodic box
    (unwrapped element coordinates cover [0, 2pi]^d): barycentric search over all elements."""
    d = topo.dim
    ref = np.einsum("ecj,epj->epc", topo.Jinv, x[None, :, :] - topo.X[:, None, 0, :])   # [E, P, d]
    lam = np.concatenate([1.0 - ref.sum(-1, keepdims=True), ref], axis=-1)
    inside = np.all(lam > -1e-12, axis=-1)
    e = np.argmax(inside, axis=0)
    assert np.all(inside[e, np.arange(x.shape[0])]), "a point lies in no element"
    return e, ref[e, np.arange(x.shape[0])]


def _values(sp, uL, e, xref):
    v, _ = fe.dubiner(sp.ref.dim, sp.ref.k, xref)                  # [P, nb]
    return np.einsum("pi,pai->pa", v, uL[e])


def _shifted(sp, vL, shift):
    """Exact L2 coefficients of x -> v(x + shift) for an element-wise polynomial field v
    of degree k: each element's polynomial is sampled through the element containing the
    shifted points and projected with the volume rule (exact for degree 2k <= 3k - 1)."""
    t, ref = sp.topo, sp.ref
    x = t.volume_points(ref.xq).reshape(-1, ref.dim)
    e1, xr1 = _locate(t, np.mod(x + shift, 2.0 * np.pi))
    vals = _values(sp, vL, e1, xr1).reshape(t.n_elems, -1, ref.dim)
    return np.einsum("q,qi,eqa->eai", ref.wq, ref.phi, vals)


@pytest.mark.parametrize("dim,n,k", [(2, 4, 2), (3, 3, 2)])
@pytest.mark.parametrize("axis", [0, 1])
def test_P10_translation_by_one_cube(dim, n, k, axis):
    """The periodic Kuhn mesh is invariant under a shift by one cube, so the operator
    commutes with it: y[w(. + h e), u(. + h e)](x) = y[w, u](x + h e).  Elements at the
    periodic seam see their vertices in another order than their interior neighbours, so
    a mistake in the orientation signs, the facet pairing or the trace permutations breaks
    the identity.  Element-wise polynomial (L2) inputs are shifted exactly; compared point
    by point at every volume quadrature point.  The wind is a constant plus a small
    polynomial perturbation, so that w.n keeps its sign on every facet: |w.n| is then a
    polynomial there and the facet rule integrates it exactly whatever the order of the
    facet's points (the collapsed facet rule is not symmetric under relabelling the
    vertices of a triangle, so with sign changes inside a facet the identity would only
    hold up to the rule's error)."""
    sp = _space(dim, n, k)
    t = sp.topo
    h = 2.0 * np.pi / n
    shift = np.zeros(dim)
    shift[axis] = h
    rng = np.random.default_rng(50 + axis)
    wL = 0.002 * rng.standard_normal((t.n_elems, dim, sp.ref.nb))
    wL[:, :, 0] += np.array([1.0, 0.55, 0.2][:dim]) * np.sqrt(float(np.sum(sp.ref.wq)))   # constant part
    uL = rng.standard_normal((t.n_elems, dim, sp.ref.nb))
    wn = C.facet_quantities(t, sp.ref, wL, uL, -1)[0]
    assert not np.any(np.any(wn > 0, axis=1) & np.any(wn < 0, axis=1))   # the precondition
    wS, uS = _shifted(sp, wL, shift), _shifted(sp, uL, shift)
    x = t.volume_points(sp.ref.xq).reshape(-1, dim)
    e0 = np.repeat(np.arange(t.n_elems), sp.ref.xq.shape[0])
    xr0 = np.tile(sp.ref.xq, (t.n_elems, 1))
    e1, xr1 = _locate(t, np.mod(x + shift, 2.0 * np.pi))
    assert np.abs(_values(sp, uS, e0, xr0) - _values(sp, uL, e1, xr1)).max() < 1e-12 * np.abs(uL).max()
    for l in (-1, k - 1, k):
        y = C.apply(t, sp.ref, wL, uL, l)
        ys = C.apply(t, sp.ref, wS, uS, l)
        lhs = _values(sp, ys, e0, xr0)
        rhs = _values(sp, y, e1, xr1)
        assert np.abs(lhs - rhs).max() < 1e-11 * np.abs(rhs).max(), l


def _box(dim, n, k):
    """The box of the periodic tests without the identification: every face a boundary."""
    m = W.periodic_box_mesh(dim, n)
    topo = mesh.MeshTopo(m.coords, m.elems)
    return hdiv.HDiv(topo, fe.ref_element(dim, k))


@pytest.mark.parametrize("dim,n,k", [(2, 3, 2), (3, 3, 2)])
def test_P2_with_wall_and_outlet_boundaries(dim, n, k):
    """Non-periodic box, every boundary facet a wall or outlet (no term in the paper's
    form): for a divergence-free normal-continuous wind the conservative form, which keeps
    (w.n) u . v there, equals the paper's form; w.n does not vanish on the boundary."""
    sp = _box(dim, n, k)
    t = sp.topo
    assert np.any(t.boundary)
    wL = _divfree(sp, seed=5)
    wn = C.facet_quantities(t, sp.ref, wL, wL, -1)[0]
    assert np.abs(wn[t.boundary]).max() > 1e-2
    uL = np.random.default_rng(60).standard_normal(wL.shape)
    for l in _ls(k):
        r1 = C.residual_conservative(t, sp.ref, wL, uL, l)
        r2 = C.residual_nonconservative(t, sp.ref, wL, uL, l)
        assert np.abs(r1 - r2).max() < 1e-11 * np.abs(r1).max(), l


@pytest.mark.parametrize("dim,n,k", [(2, 3, 2), (3, 3, 2)])
def test_inlet_with_the_interior_trace_equals_the_wall_rule(dim, n, k):
    """An inlet whose data equal the interior trace has no jump: the result must not
    depend on which boundary facets are declared inlets; with other data it must."""
    sp = _box(dim, n, k)
    t = sp.topo
    rng = np.random.default_rng(61)
    wL, uL = rng.standard_normal((2, t.n_elems, dim, sp.ref.nb))
    ext = (C.facet_trace(t, sp.ref, uL, "A"), C.facet_trace(t, sp.ref, wL, "A"))
    inlet = t.boundary & (rng.random(t.n_facets) < 0.5)
    y0 = C.apply(t, sp.ref, wL, uL, 1)
    y1 = C.apply(t, sp.ref, wL, uL, 1, exterior=ext, inlet=inlet)
    assert np.abs(y1 - y0).max() < 1e-13 * np.abs(y0).max()
    ext2 = (ext[0] + 0.5, ext[1])
    y2 = C.apply(t, sp.ref, wL, uL, 1, exterior=ext2, inlet=inlet)
    assert np.abs(y2 - y0).max() > 1e-3 * np.abs(y0).max()


@pytest.mark.parametrize("dim,k", [(2, 2), (3, 2)])
def test_energy_identity_with_walls(dim, k):
    """P3 on a non-periodic box whose wind is tangential on the boundary (a stream
    function / vector potential vanishing there): c(w; u, u) = sum_F int 1/2 |w.n|
    |(I - Pi^l)[[u]]|^2 over the interior facets, the walls contributing nothing."""
    sp = _box(dim, 3, k)
    t = sp.topo
    L = 2.0 * np.pi
    if dim == 2:
        pot = lambda x: np.sin(x[..., 0] / 2) ** 2 * np.sin(x[..., 1] / 2) ** 2 * np.cos(x[..., 0] - x[..., 1])
    else:
        def pot(x):
            b = (np.sin(x[..., 0] / 2) * np.sin(x[..., 1] / 2) * np.sin(x[..., 2] / 2)) ** 2
            return np.stack([b * np.cos(x[..., 1]), b * np.sin(x[..., 2]), b * np.cos(x[..., 0] + 1.0)], axis=-1)
    wL = fields.curl_field(t, dim, k, pot)
    wn = C.facet_quantities(t, sp.ref, wL, wL, -1)[0]
    assert np.abs(wn[t.boundary]).max() < 1e-12 * np.abs(wn).max()   # tangential on the walls
    uL = np.random.default_rng(62).standard_normal(wL.shape)
    for l in _ls(k):
        cval = C.form_value(t, sp.ref, wL, uL, l)
        diss = C.facet_dissipation(t, sp.ref, wL, uL, l)
        assert abs(cval - diss) < 1e-11 * abs(diss), l
    del L


def test_stage_substeps_are_third_order_in_time():
    """SSP-RK3 (Shu-Osher) is third order: with the central flux (l = k, no |w.n| factor,
    so the STAGE right-hand side is a smooth quadratic map of the V_h state) the error at
    a fixed time falls by 2^3 when the substep halves.  A wrong stage weight or a stage
    evaluated at the wrong state drops the order."""
    sp = _space(2, 4, 2)
    u0 = sp.interpolate(W.taylor_green) + W.uniform_noise(sp.n_hdiv, 1e-2, 7)
    T = 0.4
    ref = rk.substeps_stage(sp, u0, T / 256, 256, 2)
    errs = [np.abs(rk.substeps_stage(sp, u0, T / n, n, 2) - ref).max() for n in (8, 16, 32)]
    rates = [np.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert all(2.8 < r < 3.3 for r in rates), (errs, rates)

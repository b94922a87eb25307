"""The hexahedral path (include/hopu_hex.h) against the hexahedral oracle (oracle/hexa.py):
the apply element by element in FP64 (1e-12) and FP32 (1e-6), every order 2..5 and HOPU
orders l = -1, 0, k-1, k, boxes with uneven cell counts, spacings and a shear, with a
separate wind and with w = u; SSP-RK3 STAGE substeps; the FP64 functionals; walls,
outlets and inlets; per-facet orders and the adaptive step; a full-size apply on sampled
cells."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import hexa as H

pytestmark = pytest.mark.gpu


def _ctx(hb, k, prec):
    from paper_2408_06698_gb300 import HopuHex
    return HopuHex(hb.lines, hb.A, k=k, prec=prec)


def _dev(g, a):
    return torch.tensor(np.ascontiguousarray(a).reshape(-1), dtype=g.dtype, device=g.device)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _fields(m, ref, seed):
    """Taylor-Green-like data plus noise (w and u differ)."""
    u = H.project(m, ref, W.taylor_green) + W.uniform_noise(m.n_elems * 3 * ref.nb, 1e-2, seed).reshape(
        m.n_elems, 3, ref.nb)
    w = H.project(m, ref, lambda x: W.taylor_green(x + 0.3)) + W.uniform_noise(
        m.n_elems * 3 * ref.nb, 1e-2, seed + 1).reshape(m.n_elems, 3, ref.nb)
    return w, u


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_hex_apply_fp64(k):
    hb = W.hex_box((3, 4, 5), jitter=0.2, shear=0.3, seed=k)
    m, ref = H.HexMesh(hb), H.RefHex(k)
    g = _ctx(hb, k, "f64")
    w, u = _fields(m, ref, 10 * k)
    for l in (-1, 0, k - 1, k):
        y = g.apply(_dev(g, w), _dev(g, u), l).cpu().numpy().reshape(m.n_elems, 3, ref.nb)
        ref_y = H.apply(m, ref, w, u, l)
        err = np.abs(y - ref_y).max() / np.abs(ref_y).max()
        print(f"hex k={k} l={l}: FP64 max rel {err:.2e}")
        assert err < 1e-12


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_hex_apply_fp32(k):
    hb = W.hex_box((4, 3, 3), jitter=0.2, shear=0.3, seed=20 + k)
    m, ref = H.HexMesh(hb), H.RefHex(k)
    g = _ctx(hb, k, "f32")
    w, u = _fields(m, ref, 30 * k)
    w32, u32 = w.astype(np.float32).astype(np.float64), u.astype(np.float32).astype(np.float64)
    for l in (-1, k - 1):
        y = g.apply(_dev(g, w32), _dev(g, u32), l).cpu().numpy().astype(np.float64).reshape(m.n_elems, 3, ref.nb)
        ref_y = H.apply(m, ref, w32, u32, l)
        err = _rel(y, ref_y)
        print(f"hex k={k} l={l}: FP32 normwise {err:.2e}")
        assert err < 1e-6


@pytest.mark.parametrize("k", [2, 3, 4, 5])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_hex_apply_wind_is_field(k, prec, tol):
    """The apply with the wind the convected field itself (one tensor for both: the kernel
    that interpolates each component once), on noisy Taylor-Green data."""
    hb = W.hex_box((3, 4, 3), jitter=0.2, shear=0.3, seed=40 + k)
    m, ref = H.HexMesh(hb), H.RefHex(k)
    g = _ctx(hb, k, prec)
    _, u = _fields(m, ref, 50 * k)
    if prec == "f32":
        u = u.astype(np.float32).astype(np.float64)
    ud = _dev(g, u)
    for l in (-1, k - 1):
        y = g.apply(ud, ud, l).cpu().numpy().astype(np.float64).reshape(u.shape)
        ref_y = H.apply(m, ref, u, u, l)
        err = _rel(y, ref_y)
        print(f"hex w=u k={k} l={l} {prec}: normwise {err:.2e}")
        assert err < tol


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_hex_energy_functionals(prec, tol):
    """hopu_hex_energy against the oracle's kinetic energy, c(w; u, u) and facet dissipation
    (w = u, and a separate wind), FP64 sums of the working precision's values."""
    k = 3
    hb = W.hex_box((3, 4, 3), jitter=0.2, shear=0.3, seed=9)
    m, ref = H.HexMesh(hb), H.RefHex(k)
    g = _ctx(hb, k, prec)
    w, u = _fields(m, ref, 90)
    if prec == "f32":
        w, u = w.astype(np.float32).astype(np.float64), u.astype(np.float32).astype(np.float64)
    ud, wd = _dev(g, u), _dev(g, w)
    e, c, d = g.energy(ud)
    assert e == pytest.approx(H.kinetic_energy(m, u), rel=tol) and c == 0.0 and d == 0.0
    for wind, wn in ((ud, u), (wd, w)):
        for l in (-1, k - 1):
            e, c, d = g.energy(ud, wind, l)
            ce, de = H.form_value(m, ref, wn, u, l), H.facet_dissipation(m, ref, wn, u, l)
            print(f"hex energy {prec} l={l}: c {c:.6e} / {ce:.6e}, dissipation {d:.6e} / {de:.6e}")
            assert e == pytest.approx(H.kinetic_energy(m, u), rel=tol)
            assert abs(c - ce) <= tol * (abs(ce) + de)
            assert d == pytest.approx(de, rel=tol)


@pytest.mark.parametrize("periodic", [(True, False, True), (False, False, False), (True, True, False)])
def test_hex_walls(periodic):
    """Boxes whose non-periodic directions end in walls / outlets: the apply (separate wind
    and w = u), STAGE substeps and the functionals against the oracle's walled box."""
    from paper_2408_06698_gb300 import HopuHex
    k = 3
    hb = W.hex_box((4, 3, 3), jitter=0.2, shear=0.3, seed=60)
    m, ref = H.HexMesh(hb, periodic=periodic), H.RefHex(k)
    assert m.boundary.any()
    w, u = _fields(m, ref, 70)
    for prec, tol in (("f64", 1e-12), ("f32", 1e-6)):
        g = HopuHex(hb.lines, hb.A, k=k, prec=prec, periodic=periodic)
        uu, ww = (u, w) if prec == "f64" else (u.astype(np.float32).astype(np.float64),
                                              w.astype(np.float32).astype(np.float64))
        ud = _dev(g, uu)
        for wind, wn in ((_dev(g, ww), ww), (ud, uu)):
            for l in (-1, k - 1):
                y = g.apply(wind, ud, l).cpu().numpy().astype(np.float64).reshape(u.shape)
                err = _rel(y, H.apply(m, ref, wn, uu, l))
                print(f"hex walls {periodic} {prec} l={l}: {err:.2e}")
                assert err < tol
        e, c, d = g.energy(ud, ud, k - 1)
        assert d == pytest.approx(H.facet_dissipation(m, ref, uu, uu, k - 1), rel=tol * 20)
        v = ud.clone()
        g.rk_substeps(v, 1e-2, 2, k - 1)
        want = H.substeps_stage(m, ref, uu, 1e-2, 2, k - 1)
        err = _rel(v.cpu().numpy().astype(np.float64).reshape(u.shape), want)
        print(f"hex walls {periodic} {prec} substeps: {err:.2e}")
        assert err < tol
        g.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_hex_inlets(prec, tol):
    """Inlets at both ends of direction 1 (walls in direction 2): the exterior velocity's
    facet modes given to the library, their point values to the oracle; the apply (separate
    wind and w = u), STAGE substeps and the dissipation."""
    from paper_2408_06698_gb300 import HopuHex
    from paper_2408_06698_gb300 import _lib as L
    k = 3
    periodic = (True, False, False)
    hb = W.hex_box((3, 4, 3), jitter=0.2, shear=0.3, seed=80)
    m, ref = H.HexMesh(hb, periodic=periodic), H.RefHex(k)
    w, u = _fields(m, ref, 81)
    if prec == "f32":
        w, u = w.astype(np.float32).astype(np.float64), u.astype(np.float32).astype(np.float64)
    g = HopuHex(hb.lines, hb.A, k=k, prec=prec, periodic=periodic)
    nfm = (k + 1) ** 2
    u_inlet = {}
    for end in (0, 1):
        Fs = H.end_facets(m, 1, end)
        modes = W.uniform_noise(len(Fs) * 3 * nfm, 0.5, 90 + end).reshape(len(Fs), 3, nfm)
        if prec == "f32":
            modes = modes.astype(np.float32).astype(np.float64)
        g.set_inlet(1, end, torch.tensor(modes, dtype=g.dtype, device=g.device))
        for j, F in enumerate(Fs):
            u_inlet[int(F)] = np.einsum("pm,am->pa", ref.psi, modes[j])
    ud = _dev(g, u)
    for wind, wn in ((_dev(g, w), w), (ud, u)):
        for l in (-1, k - 1):
            y = g.apply(wind, ud, l).cpu().numpy().astype(np.float64).reshape(u.shape)
            err = _rel(y, H.apply(m, ref, wn, u, l, u_inlet))
            print(f"hex inlets {prec} l={l}: {err:.2e}")
            assert err < tol
    e, c, d = g.energy(ud, ud, k - 1)
    _, _, _, PJ, _ = H.facet_quantities(m, ref, u, u, k - 1, u_inlet)
    wnv, *_ = H.facet_quantities(m, ref, u, u, k - 1, u_inlet)
    dref = float(np.sum(m.aF[:, None] * ref.wf[None, :] * 0.5 * np.abs(wnv) * np.sum(PJ * PJ, axis=-1)))
    assert d == pytest.approx(dref, rel=20 * tol)
    v = ud.clone()
    g.rk_substeps(v, 1e-2, 2, k - 1)
    want = H.substeps_stage(m, ref, u, 1e-2, 2, k - 1, u_inlet)
    err = _rel(v.cpu().numpy().astype(np.float64).reshape(u.shape), want)
    print(f"hex inlets {prec} substeps: {err:.2e}")
    assert err < tol
    with pytest.raises(L.HopuError):
        g.set_inlet(0, 0, None)                         # direction 0 is periodic
    g.set_inlet(1, 0, None)                             # back to a wall
    g.set_inlet(1, 1, None)
    y = g.apply(ud, ud, -1).cpu().numpy().astype(np.float64).reshape(u.shape)
    assert _rel(y, H.apply(m, ref, u, u, -1)) < tol
    g.close()


@pytest.mark.parametrize("prec,tol,etol", [("f64", 1e-12, 1e-12), ("f32", 1e-6, 1e-5)])
def test_hex_adaptive(prec, tol, etol):
    """Adaptive HOPU on hexahedra: the apply and substeps with per-facet orders, and
    hopu_hex_adapt_l's indicator and new orders against the oracle (orders compared where
    eta is not within etol of a threshold)."""
    from oracle.adaptive import order_from_eta
    from paper_2408_06698_gb300 import _lib as L
    k = 3
    hb = W.hex_box((4, 3, 3), jitter=0.2, shear=0.3, seed=95)
    m, ref = H.HexMesh(hb), H.RefHex(k)
    g = _ctx(hb, k, prec)
    w, u = _fields(m, ref, 96)                  # coarse cells: jumps of several sizes
    if prec == "f32":
        w, u = w.astype(np.float32).astype(np.float64), u.astype(np.float32).astype(np.float64)
    lF = np.random.default_rng(98).integers(-1, k + 1, size=m.n_facets)
    ld = torch.tensor(lF, dtype=torch.int8, device=g.device)
    g.set_facet_l(ld)
    ud, wd = _dev(g, u), _dev(g, w)
    for wind, wn in ((wd, w), (ud, u)):
        y = g.apply(wind, ud, 0).cpu().numpy().astype(np.float64).reshape(u.shape)
        err = _rel(y, H.apply(m, ref, wn, u, lF))
        print(f"hex per-facet l {prec}: {err:.2e}")
        assert err < tol
    v = ud.clone()
    g.rk_substeps(v, 1e-2, 1, 0)
    from oracle.rk import ssp_rk3
    want = ssp_rk3(lambda x: H.apply(m, ref, x, x, lF), u, 1e-2)
    assert _rel(v.cpu().numpy().astype(np.float64).reshape(u.shape), want) < tol
    g.set_facet_l(None)
    y = g.apply(ud, ud, 1).cpu().numpy().astype(np.float64).reshape(u.shape)
    assert _rel(y, H.apply(m, ref, u, u, 1)) < tol
    # the adaptive step
    thr = [0.3, 0.4, 0.5, 0.7]
    lcur = torch.tensor(lF, dtype=torch.int8, device=g.device)
    eta = torch.zeros(m.n_facets, dtype=torch.float64, device=g.device)
    g.adapt_l(ud, thr, lcur, eta)
    eta_ref = H.facet_eta(m, ref, u, lF)
    eg = eta.cpu().numpy()
    assert np.all(np.abs(eg - eta_ref) <= etol * np.abs(eta_ref) + 1e-300)
    away = np.min(np.abs(eta_ref[:, None] - np.array(thr)[None, :]), axis=1) > 2 * etol * np.abs(eta_ref)
    new_ref = order_from_eta(eta_ref, thr, k)
    got = lcur.cpu().numpy().astype(np.int64)
    print(f"hex eta {prec}: max rel {np.max(np.abs(eg - eta_ref) / np.abs(eta_ref)):.2e}, orders "
          f"{np.bincount(new_ref + 1, minlength=k + 2)}")
    assert np.all(got[away] == new_ref[away]) and away.mean() > 0.95
    assert len(np.unique(new_ref)) >= 3
    with pytest.raises(L.HopuError) as ei:
        g.adapt_l(ud, [0.3, 0.2, 0.1, 0.05], lcur)
    assert ei.value.status == L.HOPU_EINVAL
    g.close()
    from paper_2408_06698_gb300 import HopuHex
    gw = HopuHex(hb.lines, hb.A, k=k, prec=prec, periodic=(True, True, False))
    with pytest.raises(L.HopuError) as ei:
        gw.adapt_l(_dev(gw, u), thr, lcur)
    assert ei.value.status == L.HOPU_ENOTSUP


def test_hex_constant_state_and_errors():
    from paper_2408_06698_gb300 import _lib as L
    hb = W.hex_box(3, jitter=0.1, shear=0.2, seed=3)
    m, ref = H.HexMesh(hb), H.RefHex(3)
    g = _ctx(hb, 3, "f64")
    c = H.project(m, ref, lambda x: np.broadcast_to([1.0, -0.5, 0.25], x.shape).copy())
    y = g.apply(_dev(g, c), _dev(g, c), 1).cpu().numpy()
    assert np.abs(y).max() < 1e-12
    x = _dev(g, c)
    with pytest.raises(L.HopuError) as ei:
        g.apply(x, x, 1, out=x)
    assert ei.value.status == L.HOPU_EINVAL
    from paper_2408_06698_gb300 import HopuHex
    with pytest.raises(L.HopuError) as ei:
        HopuHex(hb.lines, hb.A, k=6)
    assert ei.value.status == L.HOPU_ENOTSUP


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-6)])
def test_hex_substeps(prec, tol):
    k = 3
    hb = W.hex_box((3, 3, 4), jitter=0.2, shear=0.3, seed=7)
    m, ref = H.HexMesh(hb), H.RefHex(k)
    g = _ctx(hb, k, prec)
    u0 = H.project(m, ref, W.taylor_green)
    if prec == "f32":
        u0 = u0.astype(np.float32).astype(np.float64)
    dt, n, l = 2e-2, 4, 1
    u = _dev(g, u0)
    g.rk_substeps(u, dt, n, l)
    got = u.cpu().numpy().astype(np.float64).reshape(u0.shape)
    want = H.substeps_stage(m, ref, u0, dt, n, l)
    err = _rel(got, want)
    print(f"hex substeps {prec}: {err:.2e} (change {_rel(want, u0):.2e})")
    assert err < tol


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_hex_full_size_sampled(prec, tol):
    """32^3 cells, k = 4 (the bench's hexahedral workload): the apply on Taylor-Green
    data, checked on 64 sampled cells against the oracle on their 3x3x3 neighbourhoods."""
    k, n = 4, 32
    hb = W.hex_box(n, jitter=0.1, shear=0.2, seed=11)
    g = _ctx(hb, k, prec)
    m_small = None
    mfull = H.HexMesh(hb)
    ref = H.RefHex(k)
    u = H.project(mfull, ref, W.taylor_green)
    w = u
    if prec == "f32":
        u = w = u.astype(np.float32).astype(np.float64)
    ud = _dev(g, u)
    y = g.apply(ud, ud, k - 1).cpu().numpy().astype(np.float64).reshape(u.shape)   # w = u: one tensor
    rng = np.random.default_rng(3)
    cells = rng.choice(mfull.n_elems, size=64, replace=False)
    want = _sampled_apply(mfull, ref, w, u, k - 1, cells)
    err = _rel(y[cells], want)
    print(f"hex 32^3 k=4 {prec}: sampled normwise {err:.2e}")
    assert err < tol
    del m_small


def _sampled_apply(m, ref, w, u, l, cells):
    """The oracle's apply on the given cells only: the residual is local to a cell and its
    six facets, so run the oracle's per-facet quantities on those facets."""
    E = m.n_elems
    out = np.zeros((len(cells), 3, ref.nb))
    U = np.einsum("qi,eai->eqa", ref.phi, u[cells])
    Wv = np.einsum("qi,eai->eqa", ref.phi, w[cells])
    Wt = np.einsum("e,ecb,eqb->eqc", m.absdet[cells], m.Jinv[cells], Wv)
    out -= np.einsum("q,eqa,qic,eqc->eai", ref.wq, U, ref.dphi, Wt)
    for j, e in enumerate(cells):
        for d in range(3):
            above = m.cell[e].copy()
            above[d] = (above[d] + 1) % m.n[d]
            ea = above[0] + m.n[0] * (above[1] + m.n[1] * above[2])
            for F, side in ((d * E + ea, "A"), (d * E + e, "B")):
                sub = _SubMesh(m, np.array([F]))
                wn, jump, avg, PJ, Ph = H.facet_quantities(sub, ref, w, u, l)
                g = wn[..., None] * avg + Ph
                f = 2 * d + 1 if side == "A" else 2 * d
                sgn = 1.0 if side == "A" else -1.0
                out[j] += sgn * m.aF[F] * np.einsum("p,pa,pi->ai", ref.wf, g[0], ref.phi_f[f])
    return out / m.absdet[cells, None, None]


class _SubMesh:
    """A view of some facets of a HexMesh (the attributes facet_quantities reads)."""

    def __init__(self, m, facets):
        self.n_facets = len(facets)
        self.fa, self.fb, self.nF = m.fa[facets], m.fb[facets], m.nF[facets]
        self.boundary = m.boundary[facets]

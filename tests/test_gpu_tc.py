"""GPU parity of the tensor-core precision modes against the FP64 oracle.

HOPU_FP32_TC runs the volume contractions of the STAGE substep, the element part of the
back-projection R E^{-1} and the two dense products of the refined V_h -> L2 projection
(whose compensated residual stays on the CUDA cores) on the tensor cores (tcgen05
kind::tf32) in 3xTF32; HOPU_TF32 runs the batched V_h -> L2 projection GEMM,
the volume contractions and the back-projection with one TF32 product.  Tolerances (relative to the largest reference entry): HOPU_FP32_TC is held to
the FP32 bounds (1e-6); one TF32 product (2^-11) is held to its own bounds (1e-2 on the
projection, 2e-3 on the apply, 1e-4 on one substep state) and its errors are printed.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import convection as C
from oracle import fe, hdiv, mesh, rk

pytestmark = pytest.mark.gpu

CASES = [(2, 4, 1), (2, 8, 2), (2, 4, 4), (3, 3, 1), (3, 3, 2), (3, 5, 3), (3, 3, 4), (3, 3, 5)]
PTOL = {"f32_tc": 1e-6, "tf32": 1e-2}


def _mk(dim, n, k, prec, l=-1, wind="stage", tile_hint=2):
    """tile_hint 2 forces the tensor-core kernels (the autotuner may prefer others)."""
    from paper_2408_06698_gb300 import Hopu
    m = W.periodic_box_mesh(dim, n)
    g = Hopu(m.coords, m.elems, m.rep, k=k, l=l, prec=prec, wind=wind, tile_hint=tile_hint)
    topo = mesh.MeshTopo(m.coords, m.elems, m.rep)
    sp = hdiv.HDiv(topo, fe.ref_element(dim, k))
    return g, sp


def _dev(g, x):
    return torch.as_tensor(np.ascontiguousarray(x).reshape(-1), dtype=g.dtype, device=g.device)


def _host(t):
    return t.detach().double().cpu().numpy()


def _rounded(g, x):
    return _host(_dev(g, x)).reshape(np.shape(x))


def _rel(got, ref):
    return float(np.abs(np.asarray(got).reshape(-1) - np.asarray(ref).reshape(-1)).max() / np.abs(ref).max())


@pytest.mark.parametrize("prec", ["f32_tc", "tf32"])
@pytest.mark.parametrize("dim,n,k", CASES)
def test_tc_projection(dim, n, k, prec):
    g, sp = _mk(dim, n, k, prec)
    rng = np.random.default_rng(700 + 10 * dim + k)
    uV = _rounded(g, rng.standard_normal(sp.n_hdiv))
    got = _host(g.project("hdiv_to_l2", _dev(g, uV)))
    g.sync()
    err = _rel(got, sp.to_l2(uV))
    print(f"{prec} d={dim} k={k} E={sp.topo.n_elems}: V_h -> L2 error {err:.2e}")
    assert err < PTOL[prec]
    # L2 -> V_h: the tensor-core back-projection where this order has one (bound of the
    # FMA kernel in 3xTF32, of one TF32 product in HOPU_TF32)
    uL = _rounded(g, rng.standard_normal((sp.topo.n_elems, dim, sp.ref.nb)))
    err = _rel(_host(g.project("l2_to_hdiv", _dev(g, uL))), sp.from_l2(uL))
    print(f"{prec} d={dim} k={k}: L2 -> V_h ({g.tuning()['l2v']}) error {err:.2e}")
    assert err < (2e-6 if prec == "f32_tc" else PTOL[prec])


@pytest.mark.parametrize("dim,n,k", [(2, 8, 1), (2, 8, 2), (2, 6, 4), (3, 3, 1), (3, 3, 2), (3, 4, 3), (3, 3, 4)])
def test_tc_apply_and_substep(dim, n, k):
    g, sp = _mk(dim, n, k, "f32_tc", l=k - 1)
    rng = np.random.default_rng(800 + k)
    wV = _rounded(g, rng.standard_normal(sp.n_hdiv))
    uL = _rounded(g, rng.standard_normal((sp.topo.n_elems, dim, sp.ref.nb)))
    y = _host(g.apply_convection(_dev(g, wV), _dev(g, uL)))
    ref = C.apply(sp.topo, sp.ref, sp.to_l2(wV), uL, k - 1)
    err = _rel(y, ref)
    print(f"f32_tc apply d={dim} k={k}: {err:.2e}")
    assert err < 1e-6
    u0 = _rounded(g, sp.interpolate(W.taylor_green) + W.uniform_noise(sp.n_hdiv, 1e-3, 0))
    x = _dev(g, u0)
    g.rk_substep(x, 5e-3, 1)
    g.sync()
    ref = rk.substeps_stage(sp, u0, 5e-3, 1, k - 1)
    err = _rel(_host(x), ref)
    print(f"f32_tc substep d={dim} k={k}: {err:.2e}")
    assert err < 1e-6


def test_tc_full_size_projection():
    """16^3 x 6 tetrahedra, k = 3: the TF32 tensor-core projection against the compensated
    FP32 FMA one on the same input, at the TF32 bound."""
    from paper_2408_06698_gb300 import Hopu
    m = W.periodic_box_mesh(3, 16)
    a = Hopu(m.coords, m.elems, m.rep, k=3, l=2, prec="tf32", tile_hint=2)
    b = Hopu(m.coords, m.elems, m.rep, k=3, l=2, prec="f32")
    assert a.tuning()["v2l"] == "tc"
    u = a.interpolate_function(W.taylor_green)
    u += torch.as_tensor(W.uniform_noise(a.n_hdiv, 1e-3, 0), device=a.device).float()
    ya = a.project("hdiv_to_l2", u)
    yb = b.project("hdiv_to_l2", u)
    a.sync()
    err = float((ya - yb).abs().max() / yb.abs().max())
    print(f"full size V_h -> L2, TF32 tensor cores vs compensated FP32 FMA: {err:.2e}")
    assert err < PTOL["tf32"]


def test_tc_full_size_substep():
    """16^3 x 6 tetrahedra, k = 3: one STAGE substep with the tensor-core projection and
    volume kernels against the FP32 FMA kernels on the same state (both at FP32 parity
    with the oracle on the small meshes), and against the FP64 path."""
    from paper_2408_06698_gb300 import Hopu
    m = W.periodic_box_mesh(3, 16)
    a = Hopu(m.coords, m.elems, m.rep, k=3, l=2, prec="f32_tc", tile_hint=2)
    b = Hopu(m.coords, m.elems, m.rep, k=3, l=2, prec="f32")
    c = Hopu(m.coords, m.elems, m.rep, k=3, l=2, prec="f64")
    assert a.tuning() == {"v2l": "tc", "volume": "tc", "l2v": "tc"}
    u = c.interpolate_function(W.taylor_green)
    u += torch.as_tensor(W.uniform_noise(c.n_hdiv, 1e-3, 0), device=c.device)
    xa, xb, xc = u.float().clone(), u.float().clone(), u.float().double().clone()
    a.rk_substep(xa, 5e-4, 1)
    b.rk_substep(xb, 5e-4, 1)
    c.rk_substep(xc, 5e-4, 1)
    a.sync()
    ea = float((xa.double() - xc).abs().max() / xc.abs().max())
    eb = float((xb.double() - xc).abs().max() / xc.abs().max())
    print(f"full size substep vs FP64: 3xTF32 tensor cores {ea:.2e}, FP32 FMA {eb:.2e}")
    assert ea < 4e-7 and eb < 4e-7


@pytest.mark.parametrize("dim,n,k", [(2, 8, 2), (3, 4, 3), (3, 3, 4)])
def test_tf32_apply_and_substep(dim, n, k):
    """HOPU_TF32 with the tensor-core kernels forced (tile_hint 2), at its own bounds."""
    g, sp = _mk(dim, n, k, "tf32", l=k - 1)
    rng = np.random.default_rng(900 + k)
    wV = _rounded(g, rng.standard_normal(sp.n_hdiv))
    uL = _rounded(g, rng.standard_normal((sp.topo.n_elems, dim, sp.ref.nb)))
    y = _host(g.apply_convection(_dev(g, wV), _dev(g, uL)))
    err = _rel(y, C.apply(sp.topo, sp.ref, sp.to_l2(wV), uL, k - 1))
    print(f"tf32 apply d={dim} k={k}: {err:.2e}")
    assert err < 2e-3
    u0 = _rounded(g, sp.interpolate(W.taylor_green) + W.uniform_noise(sp.n_hdiv, 1e-3, 0))
    x = _dev(g, u0)
    g.rk_substep(x, 5e-3, 1)
    g.sync()
    err = _rel(_host(x), rk.substeps_stage(sp, u0, 5e-3, 1, k - 1))
    print(f"tf32 substep d={dim} k={k}: {err:.2e}")
    assert err < 1e-4


def test_autotuner_choices():
    """tile_hint 0 times both variants of each family on the mesh and keeps one; 1 and 2
    force them; every choice gives the same substep to FP32 accuracy."""
    from paper_2408_06698_gb300 import Hopu
    m = W.periodic_box_mesh(3, 8)
    got = {}
    for hint in (0, 1, 2):
        g = Hopu(m.coords, m.elems, m.rep, k=3, l=2, prec="f32_tc", tile_hint=hint)
        t = g.tuning()
        if hint == 1:
            assert t == {"v2l": "fma", "volume": "fma", "l2v": "fma"}
        if hint == 2:
            assert t == {"v2l": "tc", "volume": "tc", "l2v": "tc"}
        assert set(t.values()) <= {"fma", "tc"}
        u = g.interpolate_function(W.taylor_green)
        g.rk_substep(u, 5e-4, 2)
        g.sync()
        got[hint] = u.double().cpu().numpy()
        print(f"tile_hint {hint}: {t}")
    for hint in (0, 2):
        assert np.abs(got[hint] - got[1]).max() < 1e-6 * np.abs(got[1]).max()
    g = Hopu(m.coords, m.elems, m.rep, k=3, l=2, prec="f32")
    assert g.tuning() == {"v2l": "fma", "volume": "fma", "l2v": "fma"}
    assert g.tuning_l2v()["ms"] == {}


L2V_CASES = [(2, 4, 1), (2, 8, 2), (2, 4, 4), (3, 3, 1), (3, 3, 2), (3, 5, 3), (3, 3, 4)]


@pytest.mark.parametrize("prec", ["f32_tc", "tf32"])
@pytest.mark.parametrize("dim,n,k", L2V_CASES)
def test_tc_back_projection(dim, n, k, prec):
    """The tensor-core element back-projection (k_l2v_tc) forced on an FMA context: L2 ->
    V_h against the oracle and against the FMA kernel of the same context (several
    128-element tiles, the last one ragged, on the 3D meshes)."""
    g, sp = _mk(dim, n, k, prec, tile_hint=1)
    rng = np.random.default_rng(1100 + 10 * dim + k)
    uL = _rounded(g, rng.standard_normal((sp.topo.n_elems, dim, sp.ref.nb)))
    ref = sp.from_l2(uL)
    g.set_l2v_variant(0)
    y_fma = _host(g.project("l2_to_hdiv", _dev(g, uL)))
    g.set_l2v_variant(1)
    assert g.tuning()["l2v"] == "tc"
    y_tc = _host(g.project("l2_to_hdiv", _dev(g, uL)))
    g.sync()
    e_tc, e_fma, e_ab = _rel(y_tc, ref), _rel(y_fma, ref), _rel(y_tc, y_fma)
    print(f"{prec} d={dim} k={k} E={sp.topo.n_elems}: L2 -> V_h tc {e_tc:.2e}, fma {e_fma:.2e}, tc vs fma {e_ab:.2e}")
    assert e_fma < 2e-6
    assert e_tc < (2e-6 if prec == "f32_tc" else PTOL[prec])


def test_tc_back_projection_unavailable_is_einval():
    from paper_2408_06698_gb300._lib import HopuError
    g, _ = _mk(3, 3, 5, "f32_tc", tile_hint=1)
    with pytest.raises(HopuError, match="no tensor-core back-projection"):
        g.set_l2v_variant(1)
    g2, _ = _mk(3, 3, 3, "f32", tile_hint=0)
    with pytest.raises(HopuError):
        g2.set_l2v_variant(1)


@pytest.mark.parametrize("dim,n,k", [(3, 4, 3), (3, 3, 4)])
def test_tc_back_projection_in_the_substep(dim, n, k):
    """STAGE substeps with the register volume kernel + the tensor-core back-projection
    (3xTF32) against the oracle, at the FP32 bound."""
    g, sp = _mk(dim, n, k, "f32_tc", l=k - 1, tile_hint=1)
    g.set_volume_variant(1)
    g.set_l2v_variant(1)
    u0 = _rounded(g, sp.interpolate(W.taylor_green) + W.uniform_noise(sp.n_hdiv, 1e-3, 0))
    x = _dev(g, u0)
    g.rk_substep(x, 5e-3, 2)
    g.sync()
    err = _rel(_host(x), rk.substeps_stage(sp, u0, 5e-3, 2, k - 1))
    print(f"f32_tc substeps (register volume + tensor-core back-projection) d={dim} k={k}: {err:.2e}")
    assert err < 1e-6


def test_tc_back_projection_full_size_substep():
    """32^3 x 6 tetrahedra, k = 4 (196,608 elements, 1536 tiles): one STAGE substep with the
    tensor-core projection and back-projection (3xTF32; the volume term on the FMA kernels,
    which have no tensor-core variant at k = 4) and with the FMA kernels, both against the
    FP64 path on the same FP32-rounded state."""
    from paper_2408_06698_gb300 import Hopu
    m = W.periodic_box_mesh(3, 32)
    a = Hopu(m.coords, m.elems, m.rep, k=4, l=3, prec="f32_tc", tile_hint=2)
    assert a.tuning() == {"v2l": "tc", "volume": "fma", "l2v": "tc"}
    b = Hopu(m.coords, m.elems, m.rep, k=4, l=3, prec="f32")
    c = Hopu(m.coords, m.elems, m.rep, k=4, l=3, prec="f64")
    u = c.interpolate_function(W.taylor_green)
    u += torch.as_tensor(W.uniform_noise(c.n_hdiv, 1e-3, 0), device=c.device)
    xa, xb, xc = u.float().clone(), u.float().clone(), u.float().double().clone()
    a.rk_substep(xa, 5e-4, 1)
    b.rk_substep(xb, 5e-4, 1)
    c.rk_substep(xc, 5e-4, 1)
    a.sync()
    ea = float((xa.double() - xc).abs().max() / xc.abs().max())
    eb = float((xb.double() - xc).abs().max() / xc.abs().max())
    print(f"32^3 k=4 substep vs FP64: tensor-core back-projection {ea:.2e}, FMA {eb:.2e}")
    assert ea < 4e-7 and eb < 4e-7


@pytest.mark.parametrize("n,k", [(16, 3), (32, 4)])
def test_tc_refined_projection_full_size(n, k):
    """The refined projection with its dense products on the tensor cores (k_v2l_tcr) at
    the 16^3 k = 3 and 32^3 k = 4 sizes: V_h -> L2 of the FP32-rounded Taylor-Green + noise
    field against the FP64 projection of the same field, the FMA refined projection beside
    it; both at the FP32 bound."""
    from paper_2408_06698_gb300 import Hopu
    m = W.periodic_box_mesh(3, n)
    a = Hopu(m.coords, m.elems, m.rep, k=k, l=k - 1, prec="f32_tc", tile_hint=2)
    assert a.tuning()["v2l"] == "tc"
    b = Hopu(m.coords, m.elems, m.rep, k=k, l=k - 1, prec="f32")
    c = Hopu(m.coords, m.elems, m.rep, k=k, l=k - 1, prec="f64")
    u = c.interpolate_function(W.taylor_green)
    u += torch.as_tensor(W.uniform_noise(c.n_hdiv, 1e-3, 0), device=c.device)
    u32 = u.float()
    ya = a.project("hdiv_to_l2", u32)
    yb = b.project("hdiv_to_l2", u32)
    yc = c.project("hdiv_to_l2", u32.double())
    a.sync()
    scale = float(yc.abs().max())
    ea = float((ya.double() - yc).abs().max()) / scale
    eb = float((yb.double() - yc).abs().max()) / scale
    print(f"{n}^3 k={k} V_h -> L2 vs FP64: tensor-core refined {ea:.2e}, FMA refined {eb:.2e}")
    assert ea < 1e-6 and eb < 1e-6

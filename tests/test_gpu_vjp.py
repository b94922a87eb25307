"""GPU parity of the derivatives (hopu_vjp_apply, hopu_vjp_rollout) against the FP64 oracle.

Small meshes: element-by-element comparison with ``oracle.adjoint`` on the same rounded
inputs (FP64 1e-12 of the largest reference entry, FP32 2e-6 for the apply's VJP).
Full size (24^3 x 6 tetrahedra, k = 3, 200 substeps, checkpoints every 20): the oracle
cannot run that rollout in seconds, so both adjoints are checked against central finite
differences (a property at any size) over 16 seeded Gaussian directions, each scaled to
the 2-norm of u0 so that h is a relative step.  The differences are taken of the FP64
rollout (itself at oracle parity on small meshes): along such a direction the loss
changes by about 1e-7 of itself, below what an FP32 rollout resolves.  Directions whose
difference quotient crosses a kink of |w.n| are not separated out; the bound covers
them all.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import adjoint as A
from oracle import fe, hdiv, mesh

pytestmark = pytest.mark.gpu


def _mk(dim, n, k, prec, l=-1, wind="stage"):
    from paper_2408_06698_gb300 import Hopu
    m = W.periodic_box_mesh(dim, n)
    g = Hopu(m.coords, m.elems, m.rep, k=k, l=l, prec=prec, wind=wind)
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


VJP_TOL = {"f64": 1e-12, "f32": 2e-6}


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dim,n,k", [(2, 4, 2), (2, 5, 4), (3, 3, 2), (3, 3, 3), (3, 3, 4), (3, 3, 5)])
def test_vjp_apply(dim, n, k, prec):
    for l in sorted({-1, k - 1, k}):
        g, sp = _mk(dim, n, k, prec, l=l)
        rng = np.random.default_rng(500 + 10 * dim + k)
        wV = _rounded(g, rng.standard_normal(sp.n_hdiv))
        uL = _rounded(g, rng.standard_normal((sp.topo.n_elems, dim, sp.ref.nb)))
        yb = _rounded(g, rng.standard_normal(uL.shape))
        wbar, ubar = g.vjp_apply(_dev(g, wV), _dev(g, uL), _dev(g, yb))
        wb_ref, ub_ref = A.vjp_apply(sp.topo, sp.ref, sp.to_l2(wV), uL, yb, l)
        assert _rel(_host(ubar), ub_ref) < VJP_TOL[prec], (l, _rel(_host(ubar), ub_ref))
        wbV = sp.dual(wb_ref)
        assert _rel(_host(wbar), wbV) < VJP_TOL[prec], (l, _rel(_host(wbar), wbV))
        # one output only
        _, ub2 = g.vjp_apply(_dev(g, wV), _dev(g, uL), _dev(g, yb), need_w=False)
        wb2, _ = g.vjp_apply(_dev(g, wV), _dev(g, uL), _dev(g, yb), need_u=False)
        assert torch.equal(ub2, ubar) and torch.equal(wb2, wbar)
        g.close()


@pytest.mark.parametrize("ckpt", [1, 2, 3, 8])
def test_vjp_rollout_fp64(ckpt):
    dim, n, k, l = 3, 3, 3, 2
    g, sp = _mk(dim, n, k, "f64", l=l)
    u0 = sp.interpolate(W.taylor_green) + W.uniform_noise(sp.n_hdiv, 1e-2, 26)
    dt, steps = 2e-2, 5
    loss, grad = g.vjp_rollout(_dev(g, u0), dt, steps, ckpt)
    loss_ref, grad_ref = A.rollout_vjp(sp, u0, dt, steps, l)
    assert loss == pytest.approx(loss_ref, rel=1e-12)
    assert _rel(_host(grad), grad_ref) < 1e-11
    # seeded form
    s = np.random.default_rng(27).standard_normal(sp.n_hdiv)
    _, gs = g.vjp_rollout(_dev(g, u0), dt, steps, ckpt, seed=_dev(g, s))
    _, gs_ref = A.rollout_vjp(sp, u0, dt, steps, l, seed=s)
    assert _rel(_host(gs), gs_ref) < 1e-11


def test_vjp_rollout_fp32_small():
    dim, n, k, l = 2, 6, 2, 1
    g, sp = _mk(dim, n, k, "f32", l=l)
    u0 = _rounded(g, sp.interpolate(W.taylor_green) + W.uniform_noise(sp.n_hdiv, 1e-2, 28))
    dt, steps = 1e-2, 6
    loss, grad = g.vjp_rollout(_dev(g, u0), dt, steps, 4)
    loss_ref, grad_ref = A.rollout_vjp(sp, u0, dt, steps, l)
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    assert _rel(_host(grad), grad_ref) < 2e-5


@pytest.mark.parametrize("dim,n,k", [(2, 4, 4), (3, 3, 2), (3, 3, 4)])
def test_vjp_rollout_fp32_orders(dim, n, k):
    """The FP32 STAGE rollout gradient (register adjoint kernels: w = u) against the oracle's
    adjoint at the orders the other rollout tests do not cover, same bounds as above."""
    l = k - 1
    g, sp = _mk(dim, n, k, "f32", l=l)
    u0 = _rounded(g, sp.interpolate(W.taylor_green) + W.uniform_noise(sp.n_hdiv, 1e-2, 29))
    dt, steps = 1e-2, 3
    loss, grad = g.vjp_rollout(_dev(g, u0), dt, steps, 2)
    loss_ref, grad_ref = A.rollout_vjp(sp, u0, dt, steps, l)
    err = _rel(_host(grad), grad_ref)
    print(f"d={dim} k={k}: FP32 rollout gradient vs oracle adjoint {err:.2e}")
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    assert err < 2e-5


def test_vjp_zero_substeps_and_errors():
    g, sp = _mk(3, 3, 2, "f64", l=1)
    u0 = sp.interpolate(W.taylor_green)
    loss, grad = g.vjp_rollout(_dev(g, u0), 1e-2, 0, 1)
    uL = sp.to_l2(u0)
    assert loss == pytest.approx(0.5 * float(np.sum(sp.topo.absdet[:, None, None] * uL**2)), rel=1e-13)
    assert _rel(_host(grad), sp.dual(sp.topo.absdet[:, None, None] * uL)) < 1e-13
    from paper_2408_06698_gb300 import _lib as L
    x = _dev(g, u0)
    with pytest.raises(L.HopuError):
        g.vjp_rollout(x, 1e-2, 3, 0)               # ckpt_every < 1
    g.lib.hopu_clear_error(g.ctx)
    gf, spf = _mk(3, 3, 2, "f64", l=1, wind="frozen")
    with pytest.raises(L.HopuError):
        gf.vjp_rollout(_dev(gf, u0), 1e-2, 3, 1)   # FROZEN wind: not supported
    y = g.new("l2")
    st = g.lib.hopu_vjp_apply(g.ctx, x.data_ptr(), y.data_ptr(), y.data_ptr(), None, y.data_ptr())
    assert st == L.HOPU_EINVAL                      # output aliases an input
    g.lib.hopu_clear_error(g.ctx)
    st = g.lib.hopu_vjp_apply(g.ctx, x.data_ptr(), y.data_ptr(), y.data_ptr(), None, None)
    assert st == L.HOPU_EINVAL                      # no output


def test_autograd_functions():
    from paper_2408_06698_gb300 import ConvectionApply, Rollout
    g, sp = _mk(3, 3, 3, "f64", l=2)
    rng = np.random.default_rng(29)
    w = _dev(g, rng.standard_normal(sp.n_hdiv)).requires_grad_(True)
    u = _dev(g, rng.standard_normal(sp.n_l2)).requires_grad_(True)
    yb = _dev(g, rng.standard_normal(sp.n_l2))
    y = ConvectionApply.apply(g, w, u)
    (y * yb).sum().backward()
    wb, ub = g.vjp_apply(w.detach(), u.detach(), yb)
    assert torch.equal(w.grad, wb) and torch.equal(u.grad, ub)
    u0 = _dev(g, sp.interpolate(W.taylor_green) + W.uniform_noise(sp.n_hdiv, 1e-2, 30)).requires_grad_(True)
    uN = Rollout.apply(g, u0, 2e-2, 4, 2)
    s = _dev(g, rng.standard_normal(sp.n_hdiv))
    (uN * s).sum().backward()
    _, ref = A.rollout_vjp(sp, _host(u0), 2e-2, 4, 2, seed=_host(s))
    assert _rel(_host(u0.grad), ref) < 1e-11


def _rollout_loss(g, u0, dt, steps):
    u = u0.clone()
    g.rk_substep(u, dt, steps)
    uL = g.project("hdiv_to_l2", u)
    return g.energy(uL)[0]


def _fd_errors(g64, u0, dt, steps, grads, ndir, h=1e-4):
    """Central differences of the FP64 forward rollout along ndir seeded unit Gaussian
    directions scaled to |u0| (h is a relative step); per gradient the relative errors
    |fd - <grad, d>| / max(|fd|, rms(fd) / 10)."""
    dirs = W.normal_vectors(ndir, g64.n_hdiv, seed=2)
    scale = float(torch.linalg.vector_norm(u0))
    fds, ads = [], [[] for _ in grads]
    for d in dirs:
        dd = torch.as_tensor(d * scale, device=g64.device, dtype=torch.float64)
        fds.append((_rollout_loss(g64, u0 + h * dd, dt, steps) - _rollout_loss(g64, u0 - h * dd, dt, steps)) / (2 * h))
        for i, gr in enumerate(grads):
            ads[i].append(float(torch.dot(gr.double(), dd)))
    fds = np.array(fds)
    den = np.maximum(np.abs(fds), 0.1 * np.sqrt(np.mean(fds**2)))
    return [np.abs(fds - np.array(a)) / den for a in ads]


def test_vjp_rollout_finite_differences_fp64():
    """FP64 adjoint against central differences of the FP64 rollout, 6^3 x 6, k = 3, l = 2."""
    from paper_2408_06698_gb300 import Hopu
    m = W.periodic_box_mesh(3, 6)
    g = Hopu(m.coords, m.elems, m.rep, k=3, l=2, prec="f64")
    dt, steps = 5e-4, 20
    u0 = g.interpolate_function(W.taylor_green)
    u0 += torch.as_tensor(W.uniform_noise(g.n_hdiv, 1e-3, 0), device=g.device)
    loss, grad = g.vjp_rollout(u0, dt, steps, 5)
    assert loss == pytest.approx(_rollout_loss(g, u0, dt, steps), rel=1e-13)
    (err,) = _fd_errors(g, u0, dt, steps, [grad], 4)
    print(f"FD relative errors (6^3, f64): max {err.max():.3e}")
    assert err.max() < 1e-7


def test_vjp_rollout_full_size():
    """Differentiation workload: 24^3 x 6 tetrahedra, k = 3, l = 2, Taylor-Green + 1e-3
    noise (seed 0), 200 substeps dt = 5e-4, loss = final kinetic energy, checkpoints every
    20 substeps.  The FP32 adjoint (FP32 coefficients, FP64 geometry) and the FP64 adjoint
    of the same initial state against central differences (h = 1e-4, 16 directions, seed
    2) of the FP64 rollout, and against each other."""
    from paper_2408_06698_gb300 import Hopu
    m = W.periodic_box_mesh(3, 24)
    dt, steps, ck = 5e-4, 200, 20
    g32 = Hopu(m.coords, m.elems, m.rep, k=3, l=2, prec="f32")
    u32 = g32.interpolate_function(W.taylor_green)
    u32 += torch.as_tensor(W.uniform_noise(g32.n_hdiv, 1e-3, 0), device=g32.device).float()
    loss32, grad32 = g32.vjp_rollout(u32, dt, steps, ck)
    g32.close()
    g64 = Hopu(m.coords, m.elems, m.rep, k=3, l=2, prec="f64")
    u0 = u32.double()
    loss64, grad64 = g64.vjp_rollout(u0, dt, steps, ck)
    rel = float(torch.linalg.vector_norm(grad32.double() - grad64) / torch.linalg.vector_norm(grad64))
    e64, e32 = _fd_errors(g64, u0, dt, steps, [grad64, grad32], 16)
    print(f"full size: loss {loss64:.12e} (f32 {loss32:.12e}); |g32 - g64| / |g64| = {rel:.3e}; "
          f"FD relative errors f64 max {e64.max():.3e}, f32 max {e32.max():.3e}")
    assert loss32 == pytest.approx(loss64, rel=1e-5)
    assert rel < 1e-4
    # at this size the difference quotient itself is off by ~5e-4: along every direction
    # some facet points' w.n change sign between u0 - h d and u0 + h d (kinks of |w.n|,
    # error linear in h); the FP64 adjoint, exact to rounding on the small meshes, shows it
    assert e64.max() < 1e-3
    assert e32.max() < 1e-3

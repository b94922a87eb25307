"""Failure detection on the GPU without a fault: a bounded device wait made to run out.

The tensor-core kernels wait for their MMAs on an mbarrier with a poll limit.  With the
limit set to 0 (hopu_set_wait_limit) the first completion wait of each launch gives up at
once: the kernel records ETIMEOUT in the device error word, drains its MMAs in flight
with the full limit, frees its tensor memory and returns.  The host reads the status
(hopu_sync), names the kernel, and after hopu_clear_error and the default limit the next
substep matches the oracle again.  Nothing here hangs or faults the GPU: every wait is
bounded and the drained MMAs complete normally.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import fe, hdiv, mesh, rk

pytestmark = pytest.mark.gpu


def test_tensor_core_wait_timeout_is_reported_and_recovers():
    from paper_2408_06698_gb300 import Hopu
    from paper_2408_06698_gb300._lib import HOPU_ETIMEOUT, HopuError
    dim, n, k, l, dt = 3, 3, 3, 2, 5e-3
    m = W.periodic_box_mesh(dim, n)
    g = Hopu(m.coords, m.elems, m.rep, k=k, l=l, prec="tf32", tile_hint=2)
    assert g.tuning() == {"v2l": "tc", "volume": "tc", "l2v": "tc"}
    sp = hdiv.HDiv(mesh.MeshTopo(m.coords, m.elems, m.rep), fe.ref_element(dim, k))
    u0 = g.interpolate_function(W.taylor_green)
    g.set_wait_limit(0)
    x = u0.clone()
    g.rk_substep(x, dt, 1)
    with pytest.raises(HopuError) as ei:
        g.sync()
    assert ei.value.status == HOPU_ETIMEOUT
    text = g.lib.hopu_last_error(g.ctx).decode()
    assert "k_v2l_tc" in text and "k_volume_tc" in text, text
    with pytest.raises(HopuError):                  # the error is sticky until cleared
        g.rk_substep(x, dt, 1)
    g.clear_error()
    g.set_wait_limit(None)
    x = u0.clone()
    g.rk_substep(x, dt, 1)
    g.sync()
    u0h = u0.double().cpu().numpy()
    ref = rk.substeps_stage(sp, u0h, dt, 1, l)
    err = float(np.abs(x.double().cpu().numpy() - ref).max() / np.abs(ref).max())
    print(f"after recovery, one TF32 substep vs oracle: {err:.2e}")
    assert err < 1e-4


def test_back_projection_wait_timeout_is_reported_and_recovers():
    """The tensor-core back-projection (k_l2v_tc, 3xTF32) on a 3^3 x 6 mesh, k = 4 (two
    tiles, the second ragged): with the poll limit 0 its first MMA wait gives up; after
    clearing, the L2 -> V_h projection matches the oracle."""
    from paper_2408_06698_gb300 import Hopu
    from paper_2408_06698_gb300._lib import HOPU_ETIMEOUT, HopuError
    dim, n, k = 3, 3, 4
    m = W.periodic_box_mesh(dim, n)
    g = Hopu(m.coords, m.elems, m.rep, k=k, l=k - 1, prec="f32_tc", tile_hint=1)
    g.set_l2v_variant(1)
    assert g.tuning()["l2v"] == "tc"
    sp = hdiv.HDiv(mesh.MeshTopo(m.coords, m.elems, m.rep), fe.ref_element(dim, k))
    uL = np.random.default_rng(17).standard_normal((sp.topo.n_elems, dim, sp.ref.nb)).astype(np.float32)
    x = torch.as_tensor(uL.reshape(-1), device=g.device)
    g.set_wait_limit(0)
    g.project("l2_to_hdiv", x)
    with pytest.raises(HopuError) as ei:
        g.sync()
    assert ei.value.status == HOPU_ETIMEOUT
    text = g.lib.hopu_last_error(g.ctx).decode()
    assert "k_l2v_tc" in text, text
    g.clear_error()
    g.set_wait_limit(None)
    y = g.project("l2_to_hdiv", x)
    g.sync()
    ref = sp.from_l2(uL.astype(np.float64))
    err = float(np.abs(y.double().cpu().numpy() - ref).max() / np.abs(ref).max())
    print(f"after recovery, 3xTF32 back-projection vs oracle: {err:.2e}")
    assert err < 2e-6


def test_refined_projection_wait_timeout_is_reported_and_recovers():
    """The 3xTF32 refined projection (k_v2l_tcr) on a 3^3 x 6 mesh, k = 4: with the poll
    limit 0 its first MMA wait gives up and is reported; after clearing, V_h -> L2 matches
    the oracle at the FP32 bound."""
    from paper_2408_06698_gb300 import Hopu
    from paper_2408_06698_gb300._lib import HOPU_ETIMEOUT, HopuError
    dim, n, k = 3, 3, 4
    m = W.periodic_box_mesh(dim, n)
    g = Hopu(m.coords, m.elems, m.rep, k=k, l=k - 1, prec="f32_tc", tile_hint=2)
    assert g.tuning()["v2l"] == "tc"
    sp = hdiv.HDiv(mesh.MeshTopo(m.coords, m.elems, m.rep), fe.ref_element(dim, k))
    uV = np.random.default_rng(19).standard_normal(sp.n_hdiv).astype(np.float32)
    x = torch.as_tensor(uV, device=g.device)
    g.set_wait_limit(0)
    g.project("hdiv_to_l2", x)
    with pytest.raises(HopuError) as ei:
        g.sync()
    assert ei.value.status == HOPU_ETIMEOUT
    text = g.lib.hopu_last_error(g.ctx).decode()
    assert "k_v2l_tcr" in text, text
    g.clear_error()
    g.set_wait_limit(None)
    y = g.project("hdiv_to_l2", x)
    g.sync()
    ref = sp.to_l2(uV.astype(np.float64))
    err = float(np.abs(y.double().cpu().numpy().reshape(ref.shape) - ref).max() / np.abs(ref).max())
    print(f"after recovery, refined tensor-core projection vs oracle: {err:.2e}")
    assert err < 1e-6

"""Host-side checks that need no GPU: the C ABI library loads and exports every symbol
the public header declares, its FP64 reference tables pass their self-test, mesh
validation reports errors before touching the device, and the bench's multi-rank
control plane (barrier, max over ranks) works with gloo at world size 2.
"""
import os
import re
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


@pytest.fixture(scope="module")
def lib():
    from paper_2408_06698_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2408_06698_gb300 import build
        build.build()
    return _lib.load()


def declared_functions():
    text = "".join(open(os.path.join(INCLUDE, f)).read() for f in sorted(os.listdir(INCLUDE)) if f.endswith(".h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hopu_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(lib):
    from paper_2408_06698_gb300 import _lib
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    # the binding declares exactly the header's functions
    assert sorted(_lib.SIGNATURES) == names


def test_alu_peak_probe_rejects_bad_arguments(lib):
    """Argument checks of hopu_measure_alu_peak come before any CUDA call."""
    from ctypes import byref, c_double
    from paper_2408_06698_gb300 import _lib
    out = c_double(-1.0)
    assert lib.hopu_measure_alu_peak(0, 0, byref(out)) == _lib.HOPU_EINVAL
    assert lib.hopu_measure_alu_peak(1, -5, byref(out)) == _lib.HOPU_EINVAL
    assert lib.hopu_measure_alu_peak(0, 10, None) == _lib.HOPU_EINVAL
    assert out.value == -1.0


def test_no_cpu_fallback_when_library_missing(tmp_path):
    from paper_2408_06698_gb300 import _lib
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib._lib = None
        try:
            _lib.load(str(tmp_path / "libhopu.so"))
        finally:
            _lib._lib = None


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3), (3, 4), (3, 5)])
def test_reference_tables_selftest(lib, dim, k):
    from paper_2408_06698_gb300 import selftest
    rep = selftest(dim, k)
    assert rep[0] < 1e-13 and rep[1] < 1e-13      # rules exact on monomials (closed form)
    assert rep[2] < 1e-13                          # orthonormal basis
    assert rep[3] < 1e-12                          # D Dinv = I


def _create(lib, coords, elems, rep, k=2, l=-1):
    from ctypes import byref, c_void_p
    from paper_2408_06698_gb300 import _lib as L
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    elems = np.ascontiguousarray(elems, dtype=np.int64)
    rep = None if rep is None else np.ascontiguousarray(rep, dtype=np.int64)
    desc = L.MeshDesc(coords.shape[1], coords.shape[0], coords.ctypes.data, elems.shape[0], elems.ctypes.data,
                      None if rep is None else rep.ctypes.data)
    opts = L.Options(k, l, L.HOPU_FP64, L.HOPU_WIND_STAGE, 0)
    ctx = c_void_p()
    st = lib.hopu_create(byref(desc), byref(opts), None, byref(ctx))
    msg = lib.hopu_last_error(None).decode()
    if ctx.value:
        lib.hopu_destroy(ctx)
    return st, msg


def test_mesh_validation_reports_errors(lib):
    import workloads as W
    from paper_2408_06698_gb300 import _lib as L
    m = W.periodic_box_mesh(3, 3)
    bad = m.elems.copy()
    bad[5, 2] = bad[5, 1]
    st, msg = _create(lib, m.coords, bad, m.rep)
    assert st == L.HOPU_EMESH and "identified" in msg
    st, msg = _create(lib, m.coords, m.elems, None)          # boundary facets are accepted
    assert st in (L.HOPU_OK, L.HOPU_ECUDA), msg               # (ECUDA: no device here)
    dup = np.concatenate([m.elems, m.elems[:1]])              # a facet with three neighbours
    st, msg = _create(lib, m.coords, dup, m.rep)
    assert st == L.HOPU_EMESH
    flat = m.coords.copy()
    flat[:, 2] = 0.0                                          # degenerate tetrahedra
    st, msg = _create(lib, flat, m.elems, m.rep)
    assert st == L.HOPU_EMESH and "degenerate" in msg
    st, _ = _create(lib, m.coords, m.elems, m.rep, k=2, l=3)  # l > k
    assert st == L.HOPU_EINVAL
    st, _ = _create(lib, m.coords, m.elems, m.rep, k=6)
    assert st == L.HOPU_ENOTSUP


def test_valid_mesh_without_device_fails_on_cuda_only(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import workloads as W
    from paper_2408_06698_gb300 import _lib as L
    m = W.periodic_box_mesh(2, 4)
    st, msg = _create(lib, m.coords, m.elems, m.rep)
    assert st == L.HOPU_ECUDA, msg                            # topology and tables built fine


def _hex_create(lib, lines, A, n=(3, 3, 3), k=3, prec=0, periodic=7):
    from ctypes import byref, c_void_p
    flat = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64) for x in lines]))
    Am = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
    h = c_void_p()
    st = lib.hopu_hex_create(n[0], n[1], n[2], flat.ctypes.data, Am.ctypes.data, periodic, k, prec, None, byref(h))
    msg = lib.hopu_hex_last_error(None).decode()
    if h.value:
        lib.hopu_hex_destroy(h)
    return st, msg


def test_hex_box_validation(lib):
    """hopu_hex_create checks its arguments before any CUDA call."""
    import torch
    import workloads as W
    from paper_2408_06698_gb300 import _lib as L
    hb = W.hex_box(3, jitter=0.2, shear=0.3, seed=1)
    bad = [x.copy() for x in hb.lines]
    bad[1][2] = bad[1][1]                                       # a cell of zero width
    assert _hex_create(lib, bad, hb.A)[0] == L.HOPU_EMESH
    assert _hex_create(lib, hb.lines, -np.eye(3))[0] == L.HOPU_EMESH   # det A < 0
    assert _hex_create(lib, hb.lines, hb.A, k=6)[0] == L.HOPU_ENOTSUP
    assert _hex_create(lib, hb.lines, hb.A, k=1)[0] == L.HOPU_ENOTSUP
    assert _hex_create(lib, hb.lines, hb.A, prec=2)[0] == L.HOPU_EINVAL  # tensor-core modes: no
    assert _hex_create(lib, hb.lines, hb.A, periodic=8)[0] == L.HOPU_EINVAL
    small = [x[:3] for x in hb.lines]
    assert _hex_create(lib, small, hb.A, n=(2, 2, 2))[0] == L.HOPU_EINVAL
    if not torch.cuda.is_available():
        st, msg = _hex_create(lib, hb.lines, hb.A)
        assert st == L.HOPU_ECUDA, msg                          # valid box: fails on the device only
    # every other entry point refuses a NULL context before touching the device
    from ctypes import c_double
    thr = (c_double * 4)(0.1, 0.2, 0.3, 0.4)
    out = (c_double * 3)()
    assert lib.hopu_hex_destroy(None) == L.HOPU_EINVAL
    assert lib.hopu_hex_apply(None, None, None, 0, None) == L.HOPU_EINVAL
    assert lib.hopu_hex_rk_substeps(None, None, 1e-3, 1, 0) == L.HOPU_EINVAL
    assert lib.hopu_hex_set_inlet(None, 0, 0, None) == L.HOPU_EINVAL
    assert lib.hopu_hex_set_facet_l(None, None) == L.HOPU_EINVAL
    assert lib.hopu_hex_adapt_l(None, None, thr, None, None) == L.HOPU_EINVAL
    assert lib.hopu_hex_energy(None, None, None, 0, out) == L.HOPU_EINVAL
    assert lib.hopu_hex_sizes(None, None, None) == L.HOPU_EINVAL


_RANK_SCRIPT = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"]); world = int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
bench.barrier(world)
t = bench.max_over_ranks(10.0 + rank, world)
v = bench.whole_job_value(1000.0, world, t)
print(json.dumps({{"rank": rank, "max": t, "value": v}}), flush=True)
dist.barrier()
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_bench_control_plane_world_size_2(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(_RANK_SCRIPT.format(root=ROOT))
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    assert all(p.returncode == 0 for p in procs), outs
    import json
    res = [json.loads(o[0].strip().splitlines()[-1]) for o in outs]
    assert all(r["max"] == 11.0 for r in res)                 # the slowest rank's time
    assert all(abs(r["value"] - 2 * 1000.0 / 11.0) < 1e-9 for r in res)


def test_reference_arm_prints_on_rank0_only(tmp_path):
    """torchrun-style launch of --impl reference at world size 2 (tiny oracle sample)."""
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                                       "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-block", "2,2,2"],
                                      env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=600) for p in procs]
    assert all(p.returncode == 0 for p in procs), outs
    import json
    line = json.loads(outs[0][0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    assert outs[1][0].strip() == ""


def test_bench_profiles_every_kernel_family():
    import bench
    from paper_2408_06698_gb300 import _lib as L
    assert bench.ALL_FAMILIES == L.KERNEL_FAMILIES
    assert set(bench.FAMILIES) <= set(bench.ALL_FAMILIES)

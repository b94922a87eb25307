#!/usr/bin/env python
"""Benchmark of the HOPU convection hot path on one GB300 (or N independent replicas).

Headline workload (the precision configuration, the largest single-GPU mesh the metric
is quoted on): 3D periodic box [0, 2pi]^3, 32^3 cubes x 6 tetrahedra (196,608 elements),
order k = 4, HOPU projection order l = k-1 = 3, Taylor-Green velocity interpolated into
the normal-continuous velocity space plus U[-1e-3, 1e-3] noise (seed 0), dt = 5e-4, FP32.

One step = one explicit SSP-RK3 substep in STAGE wind mode (per stage: V_h -> L2
projection, facet flux, volume term + lift + inverse mass, L2 -> V_h back-projection
with the stage combination) including the FP64 kinetic-energy reduction of the state
(logged on the device).  The metric counts DOF-updates of the convection apply: L2 DOFs x
3 applies per substep.  The stated error is that of the FP32 apply against the FP64
oracle (sampled elements) and against the FP64 GPU path (every output).

Also reported: FP64 and the tensor-core precision modes on the same workload, the
16^3 x 6, k = 3 box, the 2D k = 2 square, the 512-mesh batch and the rollout adjoint.

Launch: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
(torchrun for N > 1: every rank runs the same workload on its own GPU, weak scaling,
no data-path collective; a gloo group carries the barrier and the max over ranks).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s of HOPU convection apply, FP32 vs FP64 at stated error; % HBM peak"
UNIT = "DOF-updates/s"
WORKLOAD = dict(dim=3, n=32, k=4, l=3, dt=5e-4, noise=1e-3, seed=0)
WORKLOAD_NAME = ("3D periodic box [0,2pi]^3, 32^3 cubes x 6 tets (196,608 elements), k=4, HOPU l=3, "
                 "Taylor-Green + 1e-3 seeded noise, SSP-RK3 STAGE substeps dt=5e-4")
BOX16 = dict(dim=3, n=16, k=3, l=2, dt=5e-4, noise=1e-3, seed=0)
# the headline's precision mode: FP32 data; the projection's and back-projection's dense
# products on the tensor cores in 3xTF32 (the projection refined with a compensated FP32
# residual), the facet and volume terms on the FP32 FMA kernels; autotuned per kernel family
HEADLINE_PREC = "f32_tc"
HEADLINE_MODE = ("HOPU_FP32_TC: FP32 data; 3xTF32 tensor-core products in the V_h -> L2 projection "
                 "(refined by a compensated FP32 residual) and the back-projection, FP32 FMA facet and "
                 "volume kernels; autotuned")
APPLIES_PER_STEP = 3
L2_FLUSH_BYTES = 256 << 20
RESET_EVERY = 40  # substeps between restarts of the state from its initial value
FAMILIES = ["v2l", "facet", "volume", "l2v_elem", "l2v_facet"]        # the forward substep
ALL_FAMILIES = FAMILIES + ["facet_adj", "volume_adj"]                   # every profiled family


# ------------------------------------------------------------------ roofline arithmetic
# points of the compact volume rules the volume kernels integrate with (exact to degree
# 3k - 1; elsewhere the collapsed Gauss-Jacobi rule with m^d points)
COMPACT_VOLUME_POINTS = {(3, 3): 46, (3, 4): 100, (3, 5): 190}


def shape(dim, k):
    from math import comb
    nb = comb(k + dim, dim)
    nf = comb(k + dim - 1, dim - 1)
    mv = (3 * k + 1) // 2
    mf = (3 * k + 2) // 2
    return dict(nb=nb, nf=nf, nloc=dim * nb, nint=dim * nb - (dim + 1) * nf, nq=mv ** dim, nqf=mf ** (dim - 1),
                nq_kernel=COMPACT_VOLUME_POINTS.get((dim, k), mv ** dim))


def algorithmic(dim, k, E, NF, tsize):
    """Per-launch algorithmic flops and bytes of each kernel family (STAGE wind: w = u).

    Bytes count each input/output once (coefficients, the geometry actually read, facet
    moments, connectivity); flops count the contractions the kernels perform, the volume
    term with the kernels' own quadrature rule (nq_kernel points).
    """
    from math import comb
    s = shape(dim, k)
    nb, nf, nl, nq, nqf = s["nb"], s["nf"], s["nloc"], s["nq_kernel"], s["nqf"]
    nb1 = comb(k - 1 + dim, dim)
    d = dim
    l = k - 1
    nl_ = comb(l + d - 1, d - 1)
    geo_vol = (d * d + 1) * 8                        # |det J| J^-1 and |det J| (FP64)
    out = {}
    # volume: modal gradients (2 d^2 nb1 nb) + per point u (2 nb d), grad u (2 nb1 d^2),
    # W and div W (4 d^2), f (2 d^2 + 2 d), test (2 nb d) + facet lift (2 nl (d+1) nf)
    per_q = 2 * nb * d + 2 * nb1 * d * d + 4 * d * d + 2 * d * d + 2 * d + 2 * nb * d
    fl = E * (2 * d * d * nb1 * nb + nq * per_q + 2 * nl * (d + 1) * nf)
    by = E * (2 * nl * tsize + geo_vol + (d + 1) * 4) + NF * 2 * nf * d * tsize
    out["volume"] = (fl, by)
    # facet: two traces (2 * 2 nqf nb d), P^l moments and evaluation (4 nl_ d nqf), moments
    # of the two facet fields (2 * 2 nf d nqf)
    fl = NF * (2 * 2 * nqf * nb * d + 4 * nl_ * d * nqf + 2 * 2 * nf * d * nqf)
    by = NF * ((d + 1) * 8 + 2 * 4 + 2 * nf * d * tsize) + E * nl * tsize
    out["facet"] = (fl, by)
    # v2l: gather + Dinv (2 nl^2) + Piola (2 nl d)
    out["v2l"] = (E * (2 * nl * nl + 2 * nl * d), (NF * nf + E * s["nint"]) * tsize + E * nl * tsize
                  + E * ((d * d + 1) * 8 + (d + 1) * 4))
    out["l2v_elem"] = (E * (2 * nl * nl + 2 * nl * d), E * nl * tsize * 2 + E * s["nint"] * tsize * 2
                       + E * (d + 1) * nf * tsize + E * ((d * d + 1) * 8 + (d + 1) * 4))
    out["l2v_facet"] = (NF * nf * 6, NF * nf * tsize * 4 + NF * 8)
    return out


def seg_drift(energies, first, reset_every=RESET_EVERY):
    """Mean relative change of the logged energy per substep over the first restart segment
    of the timed substeps (log entry j holds the energy at the start of substep first + j)."""
    n = min(len(energies), (first // reset_every + 1) * reset_every - first)
    e = energies[:n]
    return (e[-1] - e[0]) / max(1, len(e) - 1) / e[0] if len(e) > 1 else None


def fp32_alu_peak_tflops(sm_mhz, n_sm=152):
    """FP32 FMA peak: SMs x 128 FP32 lanes x 2 flop x clock."""
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12


def fp64_alu_peak_tflops(sm_mhz, n_sm=152):
    """GB300 FP64: 1.25 TFLOP/s nominal at 2070 MHz, scaled by the clock."""
    return 1.25 * sm_mhz / 2070.0


# ------------------------------------------------------------------ clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.p = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "100"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if "Active" in r[5 + j] and "Not" not in r[5 + j]})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ oracle (CPU)
def oracle_worker(args):
    """Runs in a child process with one BLAS thread: the FP64 CPU oracle, as it stands."""
    import numpy as np

    import workloads as W
    from oracle import fe, hdiv, mesh
    cfg = json.loads(args.oracle_worker)
    dim, n, k, l, dt = cfg["dim"], cfg["n"], cfg["k"], cfg["l"], cfg["dt"]
    m = W.periodic_box_mesh(dim, n)
    sp = hdiv.HDiv(mesh.MeshTopo(m.coords, m.elems, m.rep), fe.ref_element(dim, k))
    u = sp.interpolate(W.taylor_green) + W.uniform_noise(sp.n_hdiv, cfg["noise"], cfg["seed"])
    res = {"n": n, "n_l2": sp.n_l2, "elements": sp.topo.n_elems}
    from oracle import adjoint as A
    t0 = time.perf_counter()
    loss, _ = A.rollout_vjp(sp, u, dt, cfg["steps"], l)
    res["seconds"] = time.perf_counter() - t0
    res["steps"] = cfg["steps"]
    res["loss"] = float(loss)
    with open(cfg["out"] + ".json", "w") as f:
        json.dump(res, f)


def run_oracle(cfg: dict, timeout: float = 1800):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-worker", json.dumps(cfg)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError("oracle worker failed:\n" + r.stdout[-2000:] + r.stderr[-4000:])
    with open(cfg["out"] + ".json") as f:
        return json.load(f)


def oracle_pool(block, workers=None):
    """The oracle on every host core (oracle.pool: spawned processes, one block of the
    headline box each)."""
    from oracle.pool import OraclePool
    w = WORKLOAD
    return OraclePool(w["n"], w["k"], w["l"], block=block, workers=workers, seed=w["seed"])


def sampled_oracle_apply(uV, l, dim, n, k, n_sample=300, seed=5):
    """The oracle's apply (w = u = E uV) on n_sample seeded elements of the n^dim box,
    element by element (oracle.sampled); returns (sample ids, y[sample])."""
    import numpy as np

    import workloads as W
    from oracle import fe, hdiv, mesh
    from oracle.sampled import sampled_apply
    m = W.periodic_box_mesh(dim, n)
    topo = mesh.MeshTopo(m.coords, m.elems, m.rep)
    sp = hdiv.HDiv(topo, fe.ref_element(dim, k))
    uL = sp.to_l2(uV)
    sample = np.random.default_rng(seed).choice(topo.n_elems, n_sample, replace=False)
    return sample, uL, sampled_apply(m.coords, m.elems, m.rep, topo, sp.ref, uL, uL, l, sample)


# ------------------------------------------------------------------ ranks (control plane only)
def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """Max of a host scalar over all ranks (gloo); the identity on one rank."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Weak scaling: every rank processes units_per_rank; the job takes the slowest rank's time."""
    return world * units_per_rank / max_seconds


# ------------------------------------------------------------------ reference arm
def reference_arm(args, rank):
    """The FP64 CPU oracle as it stands, on every host core, on the headline workload: each
    step is one oracle apply of a bounded sample (blocks of --ref-block cubes of the
    32^3 x 6 box, default 8 x 8 x 4, one block per core), counted in the headline's unit."""
    if rank != 0:
        return
    K, Wm = args.steps, args.warmup
    pool = oracle_pool(tuple(int(x) for x in args.ref_block.split(",")))
    try:
        for _ in range(Wm):
            pool.step()
        secs = sum(pool.step() for _ in range(K))
    finally:
        pool.close()
    value = pool.dofs_per_step * K / secs
    sample = pool.describe()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": K, "warmup": Wm, "ms_per_step": 1e3 * secs / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "sample": sample, "oracle": "numpy FP64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.workers, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def kernel_sources_sha() -> str:
    """sha256[:16] of the headers the 3D k = 4 translation unit (csrc/ops_d3k4.cu, every
    kernel of the 32^3 k = 4 substep) includes, followed transitively within csrc/, sorted
    by name and concatenated."""
    d = os.path.join(ROOT, "paper_2408_06698_gb300", "csrc")
    seen, todo = set(), ["ops_d3k4.cu"]
    while todo:
        name = todo.pop()
        with open(os.path.join(d, name)) as f:
            for line in f:
                t = line.strip()
                if t.startswith('#include "'):
                    inc = t.split('"')[1]
                    if inc not in seen and os.path.exists(os.path.join(d, inc)):
                        seen.add(inc)
                        todo.append(inc)
    h = hashlib.sha256()
    for name in sorted(seen):
        with open(os.path.join(d, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_from_profiles(kernel: str):
    """DRAM bytes per launch from the committed ncu capture, if the kernels are unchanged."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        t = json.load(f)
    ent = t.get(kernel)
    if not ent:
        return None
    if ent.get("kernel_sources_sha") != kernel_sources_sha():
        return None
    return ent.get("dram_bytes_per_launch_full_size")


def _events_ms(stream, fn, K):
    """Device time (ms) of K calls of fn on stream, bracketed by CUDA events."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        stream.synchronize()
        a.record(stream)
        for _ in range(K):
            fn()
        b.record(stream)
    stream.synchronize()
    return a.elapsed_time(b)


def other_configs(dev, stream, world):
    """2D k=2 FP64 (8x8x2 triangles) and the 512-mesh batch: throughput in the headline's
    unit."""
    import torch

    import workloads as W
    from paper_2408_06698_gb300 import Hopu, HopuBatch
    out = {}
    # 2D periodic square, Taylor-Green (canonical interpolant), 1 apply + 100 substeps dt=1e-3
    m = W.periodic_box_mesh(2, 8)
    g = Hopu(m.coords, m.elems, m.rep, k=2, l=1, prec="f64", device=dev)
    u = g.interpolate_function(W.taylor_green)
    uL = g.project("hdiv_to_l2", u)
    y = g.new("l2")
    g.apply_convection(u, uL, out=y)
    ms = _events_ms(stream, lambda: g.rk_substep(u, 1e-3, 1), 100)
    out["square_8x8x2_k2_f64"] = {"elements": g.n_elems, "substeps": 100, "ms_per_substep": ms / 100,
                                  "value": g.n_l2 * APPLIES_PER_STEP * 100 / (ms / 1e3), "unit": UNIT}
    del g
    # 512 meshes, n ~ U{4..12}, k ~ U{2..5} (seed 1), FP32, one graph replay per substep
    draws = W.batch_draws(512, seed=1)
    meshes = [W.periodic_box_mesh(3, n) for n, _ in draws]
    b = HopuBatch([(mm.coords, mm.elems, mm.rep) for mm in meshes], [k for _, k in draws], l=-2,
                  prec=HEADLINE_PREC, device=dev)
    states = []
    for c, v in enumerate(b.classes):
        states.append(torch.as_tensor(W.uniform_noise(v.n_hdiv, 1.0, 1000 + c), device=dev).float())
    b.rk_substep(states, 5e-4, 3)
    K = 20
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a0.record()
    for _ in range(K):
        b.rk_substep(states, 5e-4, 1)
    a1.record()
    torch.cuda.synchronize()
    ms = a0.elapsed_time(a1)
    l2 = sum(v.n_l2 for v in b.classes)
    out["batch_512_meshes_f32"] = {"meshes": 512, "elements": sum(mm.n_elems for mm in meshes),
                                   "precision_mode": HEADLINE_PREC,
                                   "order_classes": len(b.classes), "substeps": K, "ms_per_substep": ms / K,
                                   "value": l2 * APPLIES_PER_STEP * K / (ms / 1e3), "unit": UNIT}
    b.close()
    try:
        out["hex_box_32cubed_k4"] = hex_row(dev, stream)
    except Exception as exc:            # an auxiliary row: reported, never the end of the line
        out["hex_box_32cubed_k4"] = {"error": f"{type(exc).__name__}: {exc}"}
    return out


def hex_row(dev, stream, n=32, k=4, l=3, substeps=10, dt=5e-4):
    """The hexahedral path: 32^3 parallelepipeds (jittered spacings, sheared), k = 4, l = 3,
    piecewise Taylor-Green data with noise (the smooth-field accuracy against the oracle is
    covered by the parity tests); FP32 and FP64 apply and STAGE substeps (CUDA events), the
    FP32 apply and substeps against FP64 on the same rounded input."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2408_06698_gb300 import HopuHex
    hb = W.hex_box(n, jitter=0.1, shear=0.2, seed=11)
    nb = (k + 1) ** 3
    nl2 = n ** 3 * 3 * nb
    # cell means (coefficient 0 of each component block, L_0 = 1) from Taylor-Green at the
    # cell centres, U[-1e-3, 1e-3] on every coefficient
    mid = [0.5 * (x[1:] + x[:-1]) for x in hb.lines]
    c2, c1, c0 = np.meshgrid(mid[2], mid[1], mid[0], indexing="ij")    # cell index: axis 0 fastest
    xc = np.stack([c0.reshape(-1), c1.reshape(-1), c2.reshape(-1)], axis=-1) @ np.asarray(hb.A).T
    u0 = W.uniform_noise(nl2, 1e-3, 77).reshape(n ** 3, 3, nb)
    u0[:, :, 0] += W.taylor_green(xc)
    u0 = u0.reshape(-1).astype(np.float32).astype(np.float64)
    row = {"workload": f"{n}^3 hexahedra (parallelepipeds), k={k}, l={l}, STAGE wind; cell means from "
                       "Taylor-Green at the cell centres, U[-1e-3, 1e-3] on every coefficient",
           "cells": n ** 3, "l2_dofs": nl2}
    res = {}
    for prec in ("f32", "f64"):
        with torch.cuda.stream(stream):
            g = HopuHex(hb.lines, hb.A, k=k, prec=prec, device=dev)
            u = torch.tensor(u0, dtype=g.dtype, device=dev)
            y = g.new()
            g.apply(u, u, l, out=y)
            ms_apply = _events_ms(stream, lambda: g.apply(u, u, l, out=y), 20) / 20
            v = u.clone()
            g.rk_substeps(v, dt, 2, l)
            ms_sub = _events_ms(stream, lambda: g.rk_substeps(v, dt, 1, l), substeps) / substeps
            v = u.clone()
            g.rk_substeps(v, dt, substeps, l)
            stream.synchronize()
        res[prec] = (y.double().cpu().numpy(), v.double().cpu().numpy())
        row[prec] = {"ms_per_apply": ms_apply, "ms_per_substep": ms_sub,
                     "value": nl2 * APPLIES_PER_STEP / (ms_sub / 1e3), "unit": UNIT}
        g.close()
    ya, yb = res["f32"][0], res["f64"][0]
    sa, sb = res["f32"][1], res["f64"][1]
    row["f32_apply_rel_error_vs_f64"] = float(np.linalg.norm(ya - yb) / np.linalg.norm(yb))
    row[f"f32_{substeps}_substeps_rel_error_vs_f64"] = float(np.linalg.norm(sa - sb) / np.linalg.norm(sb))
    row["fp32_over_fp64_speedup"] = row["f64"]["ms_per_substep"] / row["f32"]["ms_per_substep"]
    vol, fac = hex_flops(k, same=True)    # the apply and substeps run with w = u
    flops = vol * n ** 3 + fac * 3 * n ** 3
    ach = flops / (row["f32"]["ms_per_apply"] / 1e3) / 1e12
    peak = fp32_alu_peak_tflops(2070.0)
    try:
        row["cpu_baseline"] = hex_cpu_baseline(k=k, l=l)
    except Exception as exc:            # a context number: never let it stop the bench line
        row["cpu_baseline"] = {"error": f"{type(exc).__name__}: {exc}"}
    row["roofline_f32_apply"] = {"bound": "alu", "flops_per_apply": flops, "achieved": ach, "peak": peak,
                                 "unit": "TFLOP/s", "frac": ach / peak,
                                 "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (maximum SM clock)",
                                 "flops_per_cell_volume": vol, "flops_per_facet": fac}
    return row


def hex_cpu_baseline(n=8, k=4, l=3, reps=2):
    """cpu_baseline leg of the hexahedral row: the FP64 hexahedral oracle's apply (w = u) on
    an n^3 sample of the same box family, one process, in the row's unit."""
    import numpy as np

    import workloads as W
    from oracle import hexa as HX
    hb = W.hex_box(n, jitter=0.1, shear=0.2, seed=11)
    mesh, ref = HX.HexMesh(hb), HX.RefHex(k)
    u = W.uniform_noise(n ** 3 * 3 * ref.nb, 1.0, 5).reshape(n ** 3, 3, ref.nb)
    HX.apply(mesh, ref, u, u, l)
    t0 = time.perf_counter()
    for _ in range(reps):
        HX.apply(mesh, ref, u, u, l)
    secs = (time.perf_counter() - t0) / reps
    return {"value": u.size / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n}^3 cells of the same box family, k={k}, l={l}, one FP64 oracle apply (w = u), "
                      f"one process", "seconds_per_apply": secs}


def hex_flops(k, same=True):
    """Algorithmic flops (2 per multiply-add) of the hexahedral kernels, per cell (volume:
    the value + gradient passes of the fields (three when the wind is the convected field,
    six otherwise), the point integrands, the three test passes, the lift) and per facet
    (the traces (6 or 12), 11 point fields to the points, 9 moment fields back)."""
    K1, M = k + 1, (3 * k + 2) // 2
    NB, NQ, NFM, NQF = K1 ** 3, M ** 3, K1 ** 2, M ** 2
    nfield = 3 if same else 6
    interp = K1 * (2 * K1 * K1 * M + 3 * K1 * M * M + 4 * M ** 3)
    test = M ** 3 * K1 + K1 ** 2 * M ** 2 + K1 ** 3 * M
    vol = 2 * (nfield * interp + 3 * test + 33 * NQ + 18 * NB)
    fac = 2 * (2 * nfield * NFM * K1 + 11 * (K1 * M * K1 + M * M * K1) + 27 * NQF
               + 9 * (M * M * K1 + K1 * K1 * M))
    return vol, fac


def our_arm(args, rank, world):
    import numpy as np
    import torch

    import workloads as W
    from paper_2408_06698_gb300 import Hopu, measure_alu_peak

    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    meshes, states = {}, {}

    def make(cfg, prec, tile_hint=0):
        """A context on the configuration's mesh and its initial state: the Taylor-Green
        interpolant plus the seeded noise, computed by the first context made on that mesh
        and shared (rounded once to FP32) by every precision."""
        key = (cfg["dim"], cfg["n"], cfg["k"])
        if key not in meshes:
            meshes[key] = W.periodic_box_mesh(cfg["dim"], cfg["n"])
        m = meshes[key]
        g = Hopu(m.coords, m.elems, m.rep, k=cfg["k"], l=cfg["l"], prec=prec, device=dev, tile_hint=tile_hint)
        if key not in states:
            u0 = g.interpolate_function(W.taylor_green)
            noise = torch.as_tensor(W.uniform_noise(g.n_hdiv, cfg["noise"], cfg["seed"]), device=dev)
            u0 += noise.to(g.dtype)
            states[key] = u0.float().double()
        return g, states[key].to(g.dtype).clone()

    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed_steps(g, state, K, Wm, dt, profile=False, clocks=None, e2e=False, reset_every=RESET_EVERY):
        """K substeps, each bracketed by CUDA events on the launching stream.

        The state is restarted from its initial value every reset_every substeps (warm-up
        included), outside the events: the convection-only substeps are not energy stable
        once the wind has lost its exact divergence (no pressure projection on this path),
        and the Taylor-Green state overflows after ~85 substeps in every precision.

        One step = one SSP-RK3 substep (all rows of the hot path: projections, facet and
        volume kernels, inverse mass, stage combinations, back-projection) including the
        FP64 kinetic-energy reduction of the state, which the substep writes into a
        device-side log (no host round trip inside the step).  The L2 flush and the
        profile read-out run between the events.  e2e: the state is copied in from pinned
        host memory and back out inside the events of every step.
        """
        host = torch.empty(g.n_hdiv, dtype=g.dtype, pin_memory=True) if e2e else None
        if e2e:
            host.copy_(state)
        log = torch.zeros(K + Wm + 1, dtype=torch.float64, device=dev)
        start = state.clone()
        with torch.cuda.stream(stream):
            g.set_energy_log(log)
            for w in range(Wm):
                if w > 0 and w % reset_every == 0:
                    state.copy_(start)
                g.rk_substep(state, dt, 1)
            if profile:
                g.profile(True)
            acc = {f: [0.0, 0] for f in ALL_FAMILIES}
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
            stream.synchronize()
            barrier(world)
            if clocks:
                clocks.start()
            t0 = time.perf_counter()
            for i in range(K):
                flush.zero_()                      # L2 flush outside the timed events
                if (Wm + i) > 0 and (Wm + i) % reset_every == 0:
                    state.copy_(start)             # restart, outside the timed events
                    if e2e:
                        host.copy_(start, non_blocking=True)
                ev[i][0].record(stream)
                if e2e:
                    state.copy_(host, non_blocking=True)
                g.rk_substep(state, dt, 1)
                if e2e:
                    host.copy_(state, non_blocking=True)
                ev[i][1].record(stream)
                if profile:
                    g.profile_read(acc)            # synchronises; outside the events
            stream.synchronize()
            wall = time.perf_counter() - t0
            barrier(world)
            ck = clocks.stop() if clocks else None
            if profile:
                g.profile(False)
            g.set_energy_log(None)
        dev_ms = sum(a.elapsed_time(b) for a, b in ev)
        energies = log[Wm:Wm + K].cpu().numpy().tolist()
        return dev_ms, wall, acc, ck, energies

    def kernel_table(acc, alg=None):
        out = {}
        for f in FAMILIES:
            n = max(1, acc[f][1])
            avg = acc[f][0] / n
            row = {"launches": acc[f][1], "avg_us": 1e3 * avg}
            if alg is not None and acc[f][1]:
                row["tflops"] = alg[f][0] / (avg / 1e3) / 1e12
                row["gbs"] = alg[f][1] / (avg / 1e3) / 1e9
            out[f] = row
        return out

    K, Wm = args.steps, args.warmup
    H = WORKLOAD
    dt = H["dt"]
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = Clocks(uuid)

    # ---------------- headline: FP32 on the 32^3 x 6, k = 4 box.  It runs without
    # per-kernel events (they would split the substep graph's programmatic launch
    # overlap); a second, profiled pass of the same workload gives the kernel times.
    g32, s32 = make(H, HEADLINE_PREC, tile_hint=args.tile_hint)
    if args.volume_variant >= 0:
        g32.set_volume_variant(args.volume_variant)
    u_start = s32.clone()
    dev_ms, wall, _, ck, energies = timed_steps(g32, s32, K, Wm, dt, clocks=clocks)
    tmax_ms = max_over_ranks(dev_ms, world)
    dofs = g32.n_l2 * APPLIES_PER_STEP
    value = whole_job_value(dofs * K, world, tmax_ms / 1e3)
    s32p = u_start.clone()
    Kp = min(K, 30)
    prof_ms, _, acc, _, _ = timed_steps(g32, s32p, Kp, 2, dt, profile=True)
    del s32p

    # ---------------- e2e through host buffers (pinned), same metric
    s32e = u_start.clone()
    Ke = min(K, 30)
    e_ms, _, _, _, _ = timed_steps(g32, s32e, Ke, 2, dt, e2e=True)
    e_max = max_over_ranks(e_ms, world)
    e2e = {"value": whole_job_value(dofs * Ke, world, e_max / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": g32.n_hdiv * 4, "d2h_bytes_per_step": g32.n_hdiv * 4,
           "steps": Ke, "note": "pinned host state copied in and out around every substep, inside the events"}
    del s32e

    # ---------------- FP64 path (same workload, fewer steps)
    g64, s64 = make(H, "f64")
    K64 = min(K, 10)
    d64, _, _, _, _ = timed_steps(g64, s64.clone(), K64, 2, dt)
    d64 = max_over_ranks(d64, world)
    _, _, acc64, _, _ = timed_steps(g64, s64.clone(), min(K64, 5), 1, dt, profile=True)
    fp64 = {"value": whole_job_value(dofs * K64, world, d64 / 1e3), "unit": UNIT, "steps": K64,
            "ms_per_step": d64 / K64, "kernels": kernel_table(acc64)}

    # ---------------- the stated error of the headline: FP32 apply against the FP64 GPU
    # path (every output, same rounded input) and against the oracle (sampled elements,
    # rank 0), one FP32 substep against the FP64 one
    uV32 = u_start.clone()
    with torch.cuda.stream(stream):
        uL32 = g32.project("hdiv_to_l2", uV32)
        y32 = g32.apply_convection(uV32, uL32)
        uV64 = uV32.double()
        y64 = g64.apply_convection(uV64, g64.project("hdiv_to_l2", uV64))
        x32, x64 = uV32.clone(), uV64.clone()
        g32.rk_substep(x32, dt, 1)
        g64.rk_substep(x64, dt, 1)
    stream.synchronize()
    d = y32.double() - y64
    stated = {"apply_max_rel_vs_gpu_f64": float(d.abs().max() / y64.abs().max()),
              "apply_l2_rel_vs_gpu_f64": float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(y64)),
              "substep_state_max_rel_vs_gpu_f64": float((x32.double() - x64).abs().max() / x64.abs().max()),
              "inputs": "the FP32 state, rounded once, given to both paths"}
    if rank == 0 and not args.no_cpu_baseline:
        sample, _, yref = sampled_oracle_apply(uV32.double().cpu().numpy(), H["l"], H["dim"], H["n"], H["k"])
        nb = yref.shape[-1]
        for prec, y in (("f32", y32), ("f64", y64)):
            got = y.double().cpu().numpy().reshape(-1, H["dim"], nb)[sample]
            stated[f"apply_max_rel_vs_oracle_{prec}"] = float(np.abs(got - yref).max() / np.abs(yref).max())
        stated["oracle_sample"] = f"{len(sample)} seeded elements (oracle.sampled: their facet neighbourhood)"
    worst = max(stated["apply_max_rel_vs_gpu_f64"], stated["apply_l2_rel_vs_gpu_f64"],
                stated.get("apply_max_rel_vs_oracle_f32", 0.0))
    stated["fp32_bound"] = 1e-6
    stated["fp32_meets_bound"] = bool(worst <= 1e-6)
    stated["summary"] = (f"FP32 apply within 1e-6 of FP64 (worst {worst:.2e})" if worst <= 1e-6 else
                         f"FP32 apply misses 1e-6: {worst:.2e}")
    del y32, y64, uL32, x32, x64, uV64

    # ---------------- tensor-core precision modes on the same workload
    prec_rows = {}
    for name, prec, hint in (("f32_fma", "f32", 0), ("f32_tc_tensor_cores", "f32_tc", 2),
                             ("tf32_tensor_cores", "tf32", 2)):
        g, s = make(H, prec, tile_hint=hint)
        Kt = min(K, 20)
        dtm, _, _, _, en = timed_steps(g, s, Kt, 2, dt)
        _, _, acct, _, _ = timed_steps(g, s, min(Kt, 5), 1, dt, profile=True)
        with torch.cuda.stream(stream):
            ua = u_start.clone().to(g.dtype)
            ya = g.apply_convection(ua, g.project("hdiv_to_l2", ua))
            ub = ua.double()
            yb = g64.apply_convection(ub, g64.project("hdiv_to_l2", ub))
        stream.synchronize()
        dd = ya.double() - yb
        prec_rows[name] = {"ms_per_step": dtm / Kt, "value": dofs * Kt / (dtm / 1e3), "unit": UNIT,
                           "kernel_variants": g.tuning(), "volume_variant": g.tuning_volume(),
                           "kernels": kernel_table(acct),
                           "apply_max_rel_vs_gpu_f64": float(dd.abs().max() / yb.abs().max()),
                           "apply_l2_rel_vs_gpu_f64": float(torch.linalg.vector_norm(dd) / torch.linalg.vector_norm(yb)),
                           "energy_drift_per_substep": float(np.mean(np.diff(en)) / en[0])}
        del g, s, ya, yb, ua, ub
    del g64, s64

    # ---------------- the 16^3 x 6, k = 3 box (FP32, FP64, 3xTF32 autotuned)
    box16 = {}
    for prec in ("f32", "f64", "f32_tc"):
        g, s = make(BOX16, prec)
        K16 = min(K, 200) if prec != "f64" else min(K, 20)
        d16, _, _, _, _ = timed_steps(g, s, K16, 3, BOX16["dt"])
        _, _, acc16, _, _ = timed_steps(g, s, min(K16, 30), 1, BOX16["dt"], profile=True)
        box16[prec] = {"ms_per_step": d16 / K16, "value": g.n_l2 * APPLIES_PER_STEP * K16 / (d16 / 1e3),
                       "unit": UNIT, "steps": K16, "kernel_variants": g.tuning(),
                       "volume_variant": g.tuning_volume(), "kernels": kernel_table(acc16)}
        if prec in ("f32", "f32_tc") and rank == 0 and not args.no_cpu_baseline:
            uV = s.clone()
            with torch.cuda.stream(stream):
                y = g.apply_convection(uV, g.project("hdiv_to_l2", uV))
            stream.synchronize()
            sample, _, yref = sampled_oracle_apply(uV.double().cpu().numpy(), BOX16["l"], 3, BOX16["n"], BOX16["k"])
            got = y.double().cpu().numpy().reshape(-1, 3, yref.shape[-1])[sample]
            box16[prec]["apply_max_rel_vs_oracle"] = float(np.abs(got - yref).max() / np.abs(yref).max())
        del g, s
    box16["workload"] = "3D periodic box, 16^3 cubes x 6 tets (24,576 elements), k=3, l=2, same recipe"

    # ---------------- element-partitioned apply on this GPU: 4 z-slab partitions of the
    # headline box (logical partitions; halo exchange by the pack / unpack kernels)
    from paper_2408_06698_gb300.partition import PartitionedHopu, slab_partitions
    mH = meshes[(H["dim"], H["n"], H["k"])]
    parts = slab_partitions(mH, 4)
    pg = PartitionedHopu(mH.coords, mH.elems, mH.rep, parts, k=H["k"], l=H["l"], prec=HEADLINE_PREC, device=dev)
    with torch.cuda.stream(stream):
        uLw = g32.project("hdiv_to_l2", u_start.clone())
        ul = pg.scatter(uLw)
        yw = g32.apply_convection_l2(uLw, uLw)
        yp = pg.gather(pg.apply_convection_l2(ul, ul), torch.empty_like(uLw))
    stream.synchronize()
    Kpa = 5
    t_whole = _events_ms(stream, lambda: g32.apply_convection_l2(uLw, uLw, out=yw), Kpa) / Kpa
    t_part = _events_ms(stream, lambda: pg.apply_convection_l2(ul, ul), Kpa) / Kpa
    t_exch = _events_ms(stream, lambda: pg.exchange(ul), Kpa) / Kpa
    halo = sum(len(p.halo) for p in parts)
    part_row = {"partitions": len(parts), "kind": "z slabs, logical partitions on one GPU",
                "ms_per_apply_partitioned": t_part, "ms_per_apply_whole_mesh": t_whole,
                "ms_halo_exchange": t_exch, "halo_elements": halo,
                "halo_fraction": halo / g32.n_elems,
                "exchange_bytes_per_apply": halo * (g32.n_l2 // g32.n_elems) * 4,
                "owned_outputs_bit_identical": bool(torch.equal(yp, yw)),
                "note": "apply with the wind in L2 (w = u); P applies run one after another on one stream"}
    del pg, ul, yp, yw, uLw

    # ---------------- differentiation: 24^3 x 6, k = 3, 200-substep rollout, VJP with
    # checkpoints every 20 substeps (FP32)
    vjp = None
    if not args.no_vjp:
        mv = W.periodic_box_mesh(3, 24)
        gv = Hopu(mv.coords, mv.elems, mv.rep, k=3, l=2, prec=HEADLINE_PREC, device=dev)
        uv = gv.interpolate_function(W.taylor_green)
        uv += torch.as_tensor(W.uniform_noise(gv.n_hdiv, 1e-3, 0), device=dev).float()
        with torch.cuda.stream(stream):
            gv.vjp_rollout(uv, dt, 20, 20)            # warm-up: allocations, first launches
            stream.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            loss_v, _ = gv.vjp_rollout(uv, dt, 200, 20)
            t1.record(stream)
        stream.synchronize()
        vms = max_over_ranks(t0.elapsed_time(t1), world)
        vjp = {"workload": "24^3 x 6 tets (82,944 elements), k=3, l=2, HOPU_FP32_TC, 200 STAGE substeps dt=5e-4, "
                           "loss = final kinetic energy, checkpoints every 20 substeps",
               "ms_rollout_and_adjoint": vms, "loss": loss_v,
               "dof_updates_per_s_forward_equivalent": gv.n_l2 * APPLIES_PER_STEP * 200 / (vms / 1e3)}
        del gv, uv

    others = None if args.quick else other_configs(dev, stream, world)

    # ---------------- roofline of the dominant kernel (FP32 headline, live CUDA events)
    alg = algorithmic(H["dim"], H["k"], g32.n_elems, g32.n_facets, 4)
    dom = max(FAMILIES, key=lambda f: acc[f][0])
    avg_ms = acc[dom][0] / max(1, acc[dom][1])
    flops, byts = alg[dom]
    sm_mhz = (ck or {}).get("sm_mhz") or 2070.0
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    ach_tflops = flops / (avg_ms / 1e3) / 1e12
    # FMA peaks measured on this device after the timed regions (hopu_measure_alu_peak)
    alu_meas = {"fp32_tflops": measure_alu_peak(False), "fp64_tflops": measure_alu_peak(True),
                "fp32_nominal_tflops_at_sampled_clock": fp32_alu_peak_tflops(sm_mhz),
                "fp64_nominal_tflops_at_sampled_clock": fp64_alu_peak_tflops(sm_mhz)}
    alu_peak = fp32_alu_peak_tflops(sm_mhz)
    traffic = traffic_from_profiles(dom)
    roofline = {"kernel": dom, "bound": "alu", "achieved": ach_tflops, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": ach_tflops / alu_peak, "traffic": traffic,
                "peak_source": f"FP32 FMA: 152 SMs x 128 lanes x 2 flop x {sm_mhz:.0f} MHz (median SM clock "
                               "sampled during the timed region)",
                "peak_measured": alu_meas["fp32_tflops"],
                "frac_of_measured": ach_tflops / alu_meas["fp32_tflops"],
                "achieved_bytes_gbs": byts / (avg_ms / 1e3) / 1e9,
                "hbm_frac_of_measured": byts / (avg_ms / 1e3) / 1e9 / hbm_peak,
                "flops_per_launch": flops, "algorithmic_bytes_per_launch": byts,
                "avg_launch_ms": avg_ms, "launches": acc[dom][1]}
    step_bytes = sum(alg[f][1] * (acc[f][1] / max(1, Kp)) for f in FAMILIES)
    hbm_step_frac = step_bytes / (tmax_ms / K / 1e3) / 1e9 / hbm_peak
    launches = round(sum(acc[f][1] for f in FAMILIES) * K / Kp) + K   # + the energy-log kernel of every substep

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
        "ms_per_step": tmax_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "precision_mode": HEADLINE_MODE, "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "elements": g32.n_elems, "l2_dofs": g32.n_l2,
                   "hdiv_dofs": g32.n_hdiv, "applies_per_step": APPLIES_PER_STEP,
                   "volume_kernel_variant": g32.tuning_volume(),
                   "l2_flush": f"{L2_FLUSH_BYTES >> 20} MB memset between timed steps (outside the events); "
                               "the step's working set is also larger than L2",
                   "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"},
        "stated_error": stated,
        "roofline": roofline, "alu_peaks_measured": alu_meas, "e2e": e2e, "gpu_launches": launches,
        "clocks": ck, "fp64": fp64, "fp32_over_fp64_speedup": fp64["ms_per_step"] / (tmax_ms / K),
        "precision_modes": prec_rows, "box_16cubed_k3": box16, "partitioned_apply": part_row, "vjp": vjp,
        "other_configs": others,
        "hbm_frac_whole_step_of_measured": hbm_step_frac, "kernels_f32": kernel_table(acc, alg),
        "profiled_pass": {"steps": Kp, "ms_per_step": prof_ms / Kp,
                          "note": "per-kernel CUDA events around every launch (roofline, kernels_f32)"},
        "energy_drift_per_step": seg_drift(energies, Wm),
        "wall_s_timed": wall,
    }

    # ---------------- CPU baseline: the oracle on every host core (rank 0)
    if rank == 0 and not args.no_cpu_baseline:
        pool = oracle_pool((8, 8, 8))
        try:
            secs = pool.step()
        finally:
            pool.close()
        line["cpu_baseline"] = {"value": pool.dofs_per_step / secs, "unit": UNIT, "cores": pool.workers,
                                "kind": "oracle", "sample": pool.describe(), "seconds": secs,
                                "host_cores": os.cpu_count()}
        if line.get("vjp"):
            rv = run_oracle({"dim": 3, "n": 6, "k": 3, "l": 2, "dt": dt, "noise": 1e-3, "seed": 0, "steps": 2,
                             "out": os.path.join(tempfile.mkdtemp(), "v")})
            line["vjp"]["cpu_baseline"] = {
                "value": rv["n_l2"] * APPLIES_PER_STEP * rv["steps"] / rv["seconds"], "unit": UNIT,
                "cores": 1, "kind": "oracle",
                "sample": "FP64 oracle rollout + adjoint, 2 STAGE substeps of the 6^3 x 6 k=3 box "
                          "(same recipe), forward-equivalent DOF-updates/s, 1 BLAS thread",
                "seconds": rv["seconds"]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def profile_case(spec: str):
    """A small case for ncu captures ("hex,n,k,prec": the hexahedral path, three applies on
    an n^3 box); else an n^3 x 6 box, order k, precision prec
    ("n,k,prec[,volume_variant[,tile_hint]]"): build the context (tile_hint as in
    hopu_options; optionally overriding the autotuner's STAGE volume variant, whose choice
    under a profiler can differ from the plain run's), interpolate Taylor-Green, three
    V_h -> L2 projections, one apply and two STAGE substeps on a side stream
    (graph-captured)."""
    import torch

    import workloads as W
    from paper_2408_06698_gb300 import Hopu
    f = spec.split(",")
    if f[0] == "hex":
        # "hex,n,k,prec": n^3 hexahedral box (the bench's hexahedral geometry), 3 applies
        from paper_2408_06698_gb300 import HopuHex
        n, k, prec = int(f[1]), int(f[2]), f[3]
        hb = W.hex_box(n, jitter=0.1, shear=0.2, seed=11)
        gh = HopuHex(hb.lines, hb.A, k=k, prec=prec)
        u = torch.tensor(W.uniform_noise(gh.n_l2, 1.0, 3), dtype=gh.dtype, device=gh.device)
        y = gh.new()
        for _ in range(3):
            gh.apply(u, u, k - 1, out=y)
        torch.cuda.synchronize()
        print("profile case ok", spec, float(y.abs().max()))
        return
    n, k, prec = int(f[0]), int(f[1]), f[2]
    m = W.periodic_box_mesh(3, n)
    g = Hopu(m.coords, m.elems, m.rep, k=k, l=k - 1, prec=prec, tile_hint=int(f[4]) if len(f) > 4 else 0)
    if len(f) > 3:
        g.set_volume_variant(int(f[3]))
    u = g.interpolate_function(W.taylor_green)
    for _ in range(3):
        uL = g.project("hdiv_to_l2", u)
    y = g.apply_convection(u, uL)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g.rk_substep(u, 5e-4, 2)
    s.synchronize()
    torch.cuda.synchronize()
    print("profile case ok", spec, float(y.abs().max()))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-vjp", action="store_true", help="skip the rollout-adjoint measurement")
    ap.add_argument("--quick", action="store_true", help="skip the 2D and batch configurations")
    ap.add_argument("--tile-hint", type=int, default=0,
                    help="tile_hint of the headline context (0 autotune, 1 FMA, 2 tensor cores)")
    ap.add_argument("--volume-variant", type=int, default=-1,
                    help="pin the headline's STAGE volume variant (launch lists under a profiler, whose "
                         "serialised launches change the autotuner's choice); -1 keeps the autotuned one")
    ap.add_argument("--ref-block", default="8,8,4",
                    help="cubes per core of the reference arm's per-step oracle sample (bx,by,bz)")
    ap.add_argument("--profile-case", default=None, help="n,k,prec: a small case for ncu captures, then exit")
    ap.add_argument("--oracle-worker", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_worker:
        oracle_worker(args)
        return
    if args.profile_case:
        profile_case(args.profile_case)
        return
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    if args.impl == "reference":
        reference_arm(args, rank)
    else:
        our_arm(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

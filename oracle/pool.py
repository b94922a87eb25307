"""The FP64 CPU oracle's convection apply on every host core at once (benchmark baseline).

Used only by bench.py's cpu_baseline leg and its --impl reference arm.  The oracle runs as
it stands (numpy, one BLAS thread per process); this module only distributes a bounded
sample of a periodic box's elements over worker processes:

* the box's cubes are cut into blocks of bx x by x bz cubes; worker w owns the 6 bx by bz
  tetrahedra of block w;
* each worker builds the sub-mesh of its elements and their facet neighbours (the
  oracle's ``sampled`` module: the owned elements' outputs are exactly those of the full
  mesh), interpolates Taylor-Green plus seeded noise into V_h on it and takes its L2
  image (set-up, not timed);
* ``step()`` releases every worker through one barrier; each times one oracle apply
  (w = u, the STAGE wind) of its sub-mesh, and the step's time is the slowest worker's.
  The DOF-updates counted are the owned elements' L2 DOFs only; the neighbour elements'
  outputs are extra work the sample pays for and are stated as overhead.

Workers are started with the ``spawn`` method (never forked from a process that may hold
a CUDA context).
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time


def _blocks(n: int, bx: int, by: int, bz: int, count: int):
    """The first `count` blocks (cube index ranges) of an n^3 grid cut into bx x by x bz blocks."""
    out = []
    for k0 in range(0, n - bz + 1, bz):
        for j0 in range(0, n - by + 1, by):
            for i0 in range(0, n - bx + 1, bx):
                out.append((i0, j0, k0))
                if len(out) == count:
                    return out
    return out


def block_elements(n: int, origin, size):
    """Element ids of the cubes in the block (periodic_box_mesh numbering: 6 tetrahedra per
    cube, cube index with axis 0 fastest)."""
    import numpy as np
    i0, j0, k0 = origin
    bx, by, bz = size
    i, j, k = np.meshgrid(np.arange(i0, i0 + bx), np.arange(j0, j0 + by), np.arange(k0, k0 + bz), indexing="ij")
    cubes = (i + n * j + n * n * k).reshape(-1)
    return (6 * cubes[:, None] + np.arange(6)[None, :]).reshape(-1)


def _worker(wid, n, k, l, ids, n_own, seed, barrier, cmd_q, res_q):
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        os.environ[v] = "1"
    import numpy as np

    import workloads as W
    from oracle import convection as C
    from oracle import fe, hdiv, mesh
    m = W.periodic_box_mesh(3, n)
    sub = mesh.MeshTopo(m.coords, m.elems[np.asarray(ids)], m.rep)
    sp = hdiv.HDiv(sub, fe.ref_element(3, k))
    uV = sp.interpolate(W.taylor_green) + W.uniform_noise(sp.n_hdiv, 1e-3, seed + wid)
    uL = sp.to_l2(uV)
    res_q.put(("ready", wid, sub.n_elems))
    while True:
        cmd = cmd_q.get()
        if cmd == "stop":
            break
        barrier.wait()
        t0 = time.perf_counter()
        y = C.apply(sub, sp.ref, uL, uL, l)
        dt = time.perf_counter() - t0
        res_q.put(("done", wid, dt, float(np.abs(y[:n_own]).max())))


class OraclePool:
    """`workers` processes, each holding one block of a periodic n^3 x 6 box (order k, HOPU l)."""

    def __init__(self, n: int, k: int, l: int, block=(8, 8, 8), workers: int | None = None, seed: int = 0):
        import numpy as np

        import workloads as W
        from oracle import mesh
        from oracle.sampled import neighbourhood
        nb = (n // block[0]) * (n // block[1]) * (n // block[2])
        self.workers = max(1, min(workers or os.cpu_count() or 1, nb))
        self.n, self.k, self.l, self.block = n, k, l, block
        m = W.periodic_box_mesh(3, n)
        topo = mesh.MeshTopo(m.coords, m.elems, m.rep)
        ctx = mp.get_context("spawn")
        self.barrier = ctx.Barrier(self.workers + 1)
        self.res_q = ctx.Queue()
        self.cmd_q = [ctx.Queue() for _ in range(self.workers)]
        self.own = 0
        self.computed = 0
        self.procs = []
        for w, origin in enumerate(_blocks(n, *block, self.workers)):
            own = block_elements(n, origin, block)
            ids = neighbourhood(topo, own)
            self.own += len(own)
            p = ctx.Process(target=_worker, args=(w, n, k, l, ids.tolist(), len(own), seed, self.barrier,
                                                  self.cmd_q[w], self.res_q), daemon=True)
            p.start()
            self.procs.append(p)
        for _ in range(self.workers):
            msg = self._get(1800)
            self.computed += msg[2]
        from math import comb
        self.nloc = 3 * comb(k + 3, 3)

    def _get(self, timeout: float):
        """Next worker message; raises if a worker died or the time-out passed."""
        import queue
        t_end = time.monotonic() + timeout
        while True:
            try:
                return self.res_q.get(timeout=2.0)
            except queue.Empty:
                dead = [p.exitcode for p in self.procs if not p.is_alive()]
                if dead or time.monotonic() > t_end:
                    self.close()
                    raise RuntimeError(f"oracle pool: worker exit codes {dead}" if dead else "oracle pool: time-out")

    def step(self) -> float:
        """One oracle apply on every worker at once; returns the slowest worker's seconds."""
        for q in self.cmd_q:
            q.put("go")
        self.barrier.wait(timeout=600)
        times = [self._get(3600)[2] for _ in range(self.workers)]
        return max(times)

    @property
    def dofs_per_step(self) -> int:
        return self.own * self.nloc

    def describe(self) -> str:
        return (f"{self.workers} blocks of {self.block[0]}x{self.block[1]}x{self.block[2]} cubes "
                f"({self.own} of the {6 * self.n ** 3} tetrahedra of the {self.n}^3 x 6 box, k={self.k}, "
                f"l={self.l}), one FP64 oracle apply (w = u) per step, one process and one BLAS thread per "
                f"block; each process also evaluates the facet neighbours its outputs need "
                f"({self.computed - self.own} extra elements, not counted)")

    def close(self):
        for q in self.cmd_q:
            try:
                q.put("stop")
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()

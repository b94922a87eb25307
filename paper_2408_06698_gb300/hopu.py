"""Python binding of libhopu: a context object whose methods mirror the C ABI calls.

PyTorch provides device memory and streams; every step of the convection path runs in
the library's CUDA kernels.  Methods take and return torch tensors on the context's
device in the context's working precision.
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_double, c_int64, c_void_p

import numpy as np
import torch

from . import _lib as L

_PREC = {"f64": L.HOPU_FP64, "f32": L.HOPU_FP32, "f32_tc": L.HOPU_FP32_TC, "tf32": L.HOPU_TF32}
_WIND = {"stage": L.HOPU_WIND_STAGE, "frozen": L.HOPU_WIND_FROZEN}
_DIR = {"hdiv_to_l2": L.HOPU_HDIV_TO_L2, "l2_to_hdiv": L.HOPU_L2_TO_HDIV, "l2_to_hdiv_dual": L.HOPU_L2_TO_HDIV_DUAL}


class Hopu:
    """One mesh, one order k, one precision: mirrors a ``hopu_ctx``.

    coords [nv, d] float64, elems [ne, d+1] int64, rep [nv] int64 or None (host arrays).
    """

    def __init__(self, coords, elems, rep=None, k: int = 3, l: int = -1, prec: str = "f64",
                 wind: str = "stage", device: str | torch.device = "cuda", tile_hint: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("libhopu needs a CUDA device")
        self.lib = L.load()
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        if prec not in _PREC:
            raise ValueError(f"prec must be one of {sorted(_PREC)}")
        self.dtype = torch.float64 if prec == "f64" else torch.float32
        self.prec, self.k, self.l, self.wind = prec, k, l, wind
        self._coords = np.ascontiguousarray(coords, dtype=np.float64)
        self._elems = np.ascontiguousarray(elems, dtype=np.int64)
        self._rep = None if rep is None else np.ascontiguousarray(rep, dtype=np.int64)
        self.dim = int(self._coords.shape[1])
        desc = L.MeshDesc(self.dim, self._coords.shape[0], self._coords.ctypes.data, self._elems.shape[0],
                          self._elems.ctypes.data, None if self._rep is None else self._rep.ctypes.data)
        opts = L.Options(k, l, _PREC[prec], _WIND[wind], int(tile_hint))
        self.ctx = c_void_p()
        with torch.cuda.device(self.device):
            st = self.lib.hopu_create(byref(desc), byref(opts), c_void_p(self._stream()), byref(self.ctx))
        if st != L.HOPU_OK:
            raise L.HopuError(st, "hopu_create", self.lib.hopu_last_error(None).decode())
        nh, nl, nf = c_int64(), c_int64(), c_int64()
        self.lib.hopu_sizes(self.ctx, byref(nh), byref(nl), byref(nf))
        self.n_hdiv, self.n_l2, self.n_facets = nh.value, nl.value, nf.value
        self.n_elems = int(self._elems.shape[0])

    # ------------------------------------------------------------------ plumbing
    def _stream(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def _sync_stream(self):
        self._check(self.lib.hopu_set_stream(self.ctx, c_void_p(self._stream())), "hopu_set_stream")

    def _check(self, st: int, where: str):
        if st != L.HOPU_OK:
            raise L.HopuError(st, where, self.lib.hopu_last_error(self.ctx).decode())

    def _vec(self, t: torch.Tensor, n: int, name: str) -> int:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if t.device != self.device or t.dtype != self.dtype or not t.is_contiguous() or t.numel() != n:
            raise ValueError(f"{name}: expected contiguous {self.dtype} tensor of {n} entries on {self.device}, "
                             f"got {t.dtype} {tuple(t.shape)} on {t.device}")
        return t.data_ptr()

    def new(self, space: str) -> torch.Tensor:
        n = self.n_hdiv if space == "hdiv" else self.n_l2
        return torch.empty(n, dtype=self.dtype, device=self.device)

    # ------------------------------------------------------------------ the C ABI calls
    def project(self, direction: str, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        d = _DIR[direction]
        nin, nout = (self.n_hdiv, self.n_l2) if d == L.HOPU_HDIV_TO_L2 else (self.n_l2, self.n_hdiv)
        if out is None:
            out = torch.empty(nout, dtype=self.dtype, device=self.device)
        self._sync_stream()
        self._check(self.lib.hopu_project(self.ctx, d, self._vec(x, nin, "in"), self._vec(out, nout, "out")),
                    "hopu_project")
        return out

    def apply_convection(self, w_hdiv, u_l2, out=None, facet_l=None) -> torch.Tensor:
        if out is None:
            out = self.new("l2")
        fl = None
        if facet_l is not None:
            if facet_l.dtype != torch.int8 or facet_l.numel() != self.n_facets or facet_l.device != self.device:
                raise ValueError("facet_l must be an int8 device tensor with one entry per facet")
            fl = facet_l.contiguous().data_ptr()
        self._sync_stream()
        self._check(self.lib.hopu_apply_convection(self.ctx, self._vec(w_hdiv, self.n_hdiv, "w_hdiv"),
                                                   self._vec(u_l2, self.n_l2, "u_l2"),
                                                   self._vec(out, self.n_l2, "y_l2"), fl), "hopu_apply_convection")
        return out

    def apply_convection_l2(self, w_l2, u_l2, out=None) -> torch.Tensor:
        """y = M^{-1} c(w; u, .) with the wind given as an L2 vector."""
        if out is None:
            out = self.new("l2")
        self._sync_stream()
        self._check(self.lib.hopu_apply_convection_l2(self.ctx, self._vec(w_l2, self.n_l2, "w_l2"),
                                                      self._vec(u_l2, self.n_l2, "u_l2"),
                                                      self._vec(out, self.n_l2, "y_l2"), None),
                    "hopu_apply_convection_l2")
        return out

    def _ids(self, ids: torch.Tensor) -> int:
        if ids.dtype != torch.int32 or ids.device != self.device or not ids.is_contiguous():
            raise ValueError("ids must be a contiguous int32 tensor on the context's device")
        return ids.data_ptr()

    def pack_elements(self, ids: torch.Tensor, l2: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """out[j] = the L2 block of element ids[j] (flat, len(ids) * dim * nb values)."""
        nl = self.n_l2 // self.n_elems
        if out is None:
            out = torch.empty(ids.numel() * nl, dtype=self.dtype, device=self.device)
        self._sync_stream()
        self._check(self.lib.hopu_pack_elements(self.ctx, self._ids(ids), ids.numel(), self._vec(l2, self.n_l2, "l2"),
                                                self._vec(out, ids.numel() * nl, "buf")), "hopu_pack_elements")
        return out

    def unpack_elements(self, ids: torch.Tensor, buf: torch.Tensor, l2: torch.Tensor) -> torch.Tensor:
        """The L2 blocks of elements ids[j] of l2 are set from buf[j]."""
        nl = self.n_l2 // self.n_elems
        self._sync_stream()
        self._check(self.lib.hopu_unpack_elements(self.ctx, self._ids(ids), ids.numel(),
                                                  self._vec(buf, ids.numel() * nl, "buf"),
                                                  self._vec(l2, self.n_l2, "l2")), "hopu_unpack_elements")
        return l2

    def vjp_apply(self, w_hdiv, u_l2, ybar_l2, need_w: bool = True, need_u: bool = True):
        """(wbar_hdiv, ubar_l2) = cotangents of apply_convection(w, u) for ybar (None if not needed)."""
        wbar = self.new("hdiv") if need_w else None
        ubar = self.new("l2") if need_u else None
        self._sync_stream()
        self._check(self.lib.hopu_vjp_apply(self.ctx, self._vec(w_hdiv, self.n_hdiv, "w_hdiv"),
                                            self._vec(u_l2, self.n_l2, "u_l2"), self._vec(ybar_l2, self.n_l2, "ybar_l2"),
                                            None if wbar is None else wbar.data_ptr(),
                                            None if ubar is None else ubar.data_ptr()), "hopu_vjp_apply")
        return wbar, ubar

    def vjp_rollout(self, u0_hdiv, dt: float, n_substeps: int, ckpt_every: int = 1, seed=None):
        """Gradient through n STAGE substeps from u0.  seed None: (loss, d loss/d u0) for
        loss = 1/2 int |E u_n|^2; else (None, cotangent of u0) for the cotangent seed of u_n."""
        out = self.new("hdiv")
        loss = c_double(0.0)
        if seed is not None:
            out.copy_(seed)
        self._sync_stream()
        self._check(self.lib.hopu_vjp_rollout(self.ctx, self._vec(u0_hdiv, self.n_hdiv, "u0_hdiv"), float(dt),
                                              int(n_substeps), int(ckpt_every), out.data_ptr(),
                                              byref(loss) if seed is None else None), "hopu_vjp_rollout")
        return (float(loss.value) if seed is None else None), out

    def boundary_facets(self) -> np.ndarray:
        """Ids of the facets with a single element (walls / outlets unless declared inlets)."""
        cnt = c_int64()
        self._check(self.lib.hopu_boundary_facets(self.ctx, None, byref(cnt)), "hopu_boundary_facets")
        out = np.empty(cnt.value, dtype=np.int64)
        if cnt.value:
            self._check(self.lib.hopu_boundary_facets(self.ctx, out.ctypes.data, None), "hopu_boundary_facets")
        return out

    def set_inlet(self, facets, values=None, fun=None):
        """Declare boundary facets inlets with data u_I given at their facet quadrature
        points (values [n, nqf, dim]) or as a callable of points; no facets clears them."""
        f = np.ascontiguousarray(np.asarray(facets, dtype=np.int64).reshape(-1))
        if f.size == 0:
            self._check(self.lib.hopu_set_inlet(self.ctx, None, 0, None), "hopu_set_inlet")
            return
        if values is None:
            pts = self.points("facet").reshape(self.n_facets, -1, self.dim)[f]
            values = fun(pts)
        v = np.ascontiguousarray(values, dtype=np.float64)
        self._check(self.lib.hopu_set_inlet(self.ctx, f.ctypes.data, f.size, v.ctypes.data), "hopu_set_inlet")

    def set_facet_l(self, facet_l: torch.Tensor | None):
        """Per-facet HOPU orders (int8 device tensor, kept referenced) for later calls; None = uniform l."""
        if facet_l is None:
            self._check(self.lib.hopu_set_facet_l(self.ctx, None), "hopu_set_facet_l")
            self._facet_l = None
            return
        if facet_l.dtype != torch.int8 or facet_l.numel() != self.n_facets or facet_l.device != self.device \
                or not facet_l.is_contiguous():
            raise ValueError("facet_l must be a contiguous int8 device tensor with one entry per facet")
        self._check(self.lib.hopu_set_facet_l(self.ctx, c_void_p(facet_l.data_ptr())), "hopu_set_facet_l")
        self._facet_l = facet_l

    def adapt_l(self, u_l2: torch.Tensor, thresholds, facet_l: torch.Tensor, eta_out: torch.Tensor | None = None):
        """Adaptive HOPU: eta per facet with the current orders in facet_l, new orders written back."""
        th = (c_double * (self.k + 1))(*[float(x) for x in thresholds])
        if len(thresholds) != self.k + 1:
            raise ValueError(f"need k+1 = {self.k + 1} thresholds")
        if facet_l.dtype != torch.int8 or facet_l.numel() != self.n_facets or facet_l.device != self.device:
            raise ValueError("facet_l must be an int8 device tensor with one entry per facet")
        ep = None
        if eta_out is not None:
            if eta_out.dtype != torch.float64 or eta_out.numel() != self.n_facets or eta_out.device != self.device:
                raise ValueError("eta_out must be a float64 device tensor with one entry per facet")
            ep = c_void_p(eta_out.data_ptr())
        self._sync_stream()
        self._check(self.lib.hopu_adapt_l(self.ctx, self._vec(u_l2, self.n_l2, "u_l2"), th,
                                          c_void_p(facet_l.data_ptr()), ep), "hopu_adapt_l")
        return facet_l

    def adaptive_substeps(self, state: torch.Tensor, dt: float, n_substeps: int, thresholds,
                          facet_l: torch.Tensor, period: int = 10) -> torch.Tensor:
        """STAGE substeps with adaptive HOPU orders: before every period-th substep (the
        first included) the orders are re-determined from the current state."""
        if self.wind != "stage":
            raise ValueError("adaptive_substeps runs the STAGE wind rule")
        self.set_facet_l(facet_l)
        uL = self.new("l2")
        done = 0
        while done < n_substeps:
            self.project("hdiv_to_l2", state, out=uL)
            self.adapt_l(uL, thresholds, facet_l)
            m = min(period, n_substeps - done)
            self.rk_substep(state, dt, m)
            done += m
        return state

    def tuning(self) -> dict:
        """Kernel variants the autotuner kept, 'fma' or 'tc' per family: the V_h -> L2
        projection ('v2l'), the STAGE volume kernel ('volume') and the element part of the
        back-projection ('l2v')."""
        out = (ctypes.c_int * 2)()
        self._check(self.lib.hopu_tuning(self.ctx, out), "hopu_tuning")
        tc = ctypes.c_int()
        self._check(self.lib.hopu_tuning_l2v(self.ctx, byref(tc), None), "hopu_tuning_l2v")
        return {"v2l": "tc" if out[0] else "fma", "volume": "tc" if out[1] else "fma",
                "l2v": "tc" if tc.value else "fma"}

    def tuning_l2v(self) -> dict:
        """The back-projection kernel the autotuner kept and its timings (ms per launch)."""
        tc = ctypes.c_int()
        ms = (c_double * 2)()
        self._check(self.lib.hopu_tuning_l2v(self.ctx, byref(tc), ms), "hopu_tuning_l2v")
        return {"kernel": "tc" if tc.value else "fma",
                "ms": {n: ms[i] for i, n in enumerate(("fma", "tc")) if ms[i] >= 0}}

    def set_l2v_variant(self, tc: int):
        """Override the autotuner's back-projection kernel: 0 FMA, 1 tensor cores."""
        self._check(self.lib.hopu_set_l2v_variant(self.ctx, int(tc)), "hopu_set_l2v_variant")

    VOLUME_VARIANTS = {0: "register, fused back-projection", 1: "register + separate back-projection",
                       2: "warp per element, fused back-projection", 3: "tensor cores",
                       4: "register with gradient tables + separate back-projection",
                       5: "register, basis split over two lanes + separate back-projection",
                       -1: "warp per element + separate back-projection"}

    def tuning_volume(self) -> dict:
        """The STAGE volume kernel variant the autotuner kept and its timings (ms per launch)."""
        v = ctypes.c_int()
        ms = (c_double * 6)()
        self._check(self.lib.hopu_tuning_volume(self.ctx, byref(v), ms), "hopu_tuning_volume")
        names = ["reg_fused", "reg_split", "warp_fused", "tensor", "reg_tables_split", "reg_half_split"]
        return {"variant": v.value, "name": self.VOLUME_VARIANTS.get(v.value, "?"),
                "ms": {names[i]: ms[i] for i in range(6) if ms[i] >= 0}}

    def set_volume_variant(self, variant: int):
        """Override the autotuner's STAGE volume variant (numbering of tuning_volume)."""
        self._check(self.lib.hopu_set_volume_variant(self.ctx, int(variant)), "hopu_set_volume_variant")

    def sync(self):
        """Synchronise the context stream; raises on a device-side failure (ETIMEOUT)."""
        self._check(self.lib.hopu_sync(self.ctx), "hopu_sync")

    def set_wait_limit(self, polls: int | None):
        """Polls of the tensor-core MMA completion waits (None: the default, 2^22)."""
        self._check(self.lib.hopu_set_wait_limit(self.ctx, -1 if polls is None else int(polls)),
                    "hopu_set_wait_limit")

    def clear_error(self):
        self.lib.hopu_clear_error(self.ctx)

    def set_frozen_wind(self, w_hdiv: torch.Tensor):
        self._sync_stream()
        self._check(self.lib.hopu_set_frozen_wind(self.ctx, self._vec(w_hdiv, self.n_hdiv, "w_hdiv")),
                    "hopu_set_frozen_wind")

    def set_energy_log(self, log: torch.Tensor | None):
        """Log 1/2 int |u|^2 at the start of every later substep into a float64 device tensor."""
        if log is None:
            self._check(self.lib.hopu_set_energy_log(self.ctx, None, 0), "hopu_set_energy_log")
            self._elog = None
            return
        if log.dtype != torch.float64 or log.device != self.device or not log.is_contiguous():
            raise ValueError("energy log must be a contiguous float64 tensor on the context's device")
        self._sync_stream()
        self._check(self.lib.hopu_set_energy_log(self.ctx, c_void_p(log.data_ptr()), log.numel()),
                    "hopu_set_energy_log")
        self._elog = log

    def rk_substep(self, state: torch.Tensor, dt: float, n_substeps: int = 1) -> torch.Tensor:
        n = self.n_hdiv if self.wind == "stage" else self.n_l2
        self._sync_stream()
        self._check(self.lib.hopu_rk_substep(self.ctx, self._vec(state, n, "state"), float(dt), int(n_substeps)),
                    "hopu_rk_substep")
        return state

    def energy(self, u_l2: torch.Tensor, w_hdiv: torch.Tensor | None = None):
        out = (c_double * 3)()
        self._sync_stream()
        wp = None if w_hdiv is None else self._vec(w_hdiv, self.n_hdiv, "w_hdiv")
        self._check(self.lib.hopu_energy(self.ctx, wp, self._vec(u_l2, self.n_l2, "u_l2"), out), "hopu_energy")
        return float(out[0]), float(out[1]), float(out[2])

    def points(self, which: str) -> np.ndarray:
        w = 0 if which == "facet" else 1
        cnt = c_int64()
        self._check(self.lib.hopu_points(self.ctx, w, None, byref(cnt)), "hopu_points")
        buf = np.empty((cnt.value, self.dim), dtype=np.float64)
        self._check(self.lib.hopu_points(self.ctx, w, buf.ctypes.data, None), "hopu_points")
        return buf

    def interpolate(self, fvals: np.ndarray, vvals: np.ndarray, out: torch.Tensor | None = None) -> torch.Tensor:
        fvals = np.ascontiguousarray(fvals, dtype=np.float64)
        vvals = np.ascontiguousarray(vvals, dtype=np.float64)
        if out is None:
            out = self.new("hdiv")
        self._sync_stream()
        self._check(self.lib.hopu_interpolate(self.ctx, fvals.ctypes.data, vvals.ctypes.data,
                                              self._vec(out, self.n_hdiv, "u_hdiv")), "hopu_interpolate")
        return out

    def interpolate_function(self, fun) -> torch.Tensor:
        """Canonical interpolant of a callable of points [.., d] -> [.., d]."""
        fp = self.points("facet")
        vp = self.points("volume")
        return self.interpolate(fun(fp), fun(vp))

    def profile(self, enable: bool = True):
        self._check(self.lib.hopu_profile(self.ctx, int(bool(enable))), "hopu_profile")

    def profile_read(self, acc: dict | None = None) -> dict:
        """Add per-kernel-family device time (ms) and launch counts into acc."""
        n = len(L.KERNEL_FAMILIES)
        ms, cnt = (c_double * n)(), (c_int64 * n)()
        self._check(self.lib.hopu_profile_read(self.ctx, ms, cnt), "hopu_profile_read")
        acc = acc if acc is not None else {f: [0.0, 0] for f in L.KERNEL_FAMILIES}
        for i, f in enumerate(L.KERNEL_FAMILIES):
            acc[f][0] += ms[i]
            acc[f][1] += cnt[i]
        return acc

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.lib.hopu_destroy(self.ctx)
            self.ctx = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # substep launch counts (kernels per call), for the bench's launch accounting
    def launches_per_substep(self) -> int:
        n = 15 if self.wind == "stage" else 6
        return n + (1 if getattr(self, "_elog", None) is not None else 0)


class ConvectionApply(torch.autograd.Function):
    """y = apply_convection(w, u) as an autograd node; the backward is hopu_vjp_apply."""

    @staticmethod
    def forward(ctx, hopu: Hopu, w_hdiv, u_l2):
        ctx.hopu = hopu
        ctx.save_for_backward(w_hdiv, u_l2)
        return hopu.apply_convection(w_hdiv.detach().contiguous(), u_l2.detach().contiguous())

    @staticmethod
    def backward(ctx, ybar):
        w, u = ctx.saved_tensors
        wbar, ubar = ctx.hopu.vjp_apply(w.detach(), u.detach(), ybar.contiguous(),
                                        need_w=ctx.needs_input_grad[1], need_u=ctx.needs_input_grad[2])
        return None, wbar, ubar


class Rollout(torch.autograd.Function):
    """u_n = n STAGE SSP-RK3 substeps of u0 as an autograd node; the backward is
    hopu_vjp_rollout with the incoming cotangent as seed."""

    @staticmethod
    def forward(ctx, hopu: Hopu, u0_hdiv, dt: float, n_substeps: int, ckpt_every: int = 1):
        ctx.hopu, ctx.dt, ctx.n, ctx.ck = hopu, dt, n_substeps, ckpt_every
        ctx.save_for_backward(u0_hdiv)
        u = u0_hdiv.detach().clone()
        return hopu.rk_substep(u, dt, n_substeps)

    @staticmethod
    def backward(ctx, ubar):
        (u0,) = ctx.saved_tensors
        _, g = ctx.hopu.vjp_rollout(u0.detach(), ctx.dt, ctx.n, ctx.ck, seed=ubar.contiguous())
        return None, g, None, None, None


class _ClassView(Hopu):
    """A non-owning Hopu view of one order class of a batch (the batch owns the context)."""

    def __init__(self, batch: "HopuBatch", ctx: c_void_p, k: int, n_hdiv: int, n_l2: int):
        self.lib = batch.lib
        self.device, self.dtype, self.prec = batch.device, batch.dtype, batch.prec
        self.k, self.l, self.wind, self.dim = k, None, batch.wind, batch.dim
        self.ctx = ctx
        self.n_hdiv, self.n_l2 = n_hdiv, n_l2
        nh, nl, nf = c_int64(), c_int64(), c_int64()
        self.lib.hopu_sizes(self.ctx, byref(nh), byref(nl), byref(nf))
        self.n_facets = nf.value
        self.n_elems = n_l2 // (self.dim * _nbasis(self.dim, k))

    def close(self):  # owned by the batch
        self.ctx = c_void_p()


def _nbasis(d, k):
    from math import comb
    return comb(k + d, d)


class HopuBatch:
    """Many meshes of uneven size and order, advanced together (mirrors hopu_batch)."""

    def __init__(self, meshes, ks, l: int = -2, prec: str = "f32", wind: str = "stage",
                 device: str | torch.device = "cuda"):
        if not torch.cuda.is_available():
            raise RuntimeError("libhopu needs a CUDA device")
        self.lib = L.load()
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        if prec not in _PREC:
            raise ValueError(f"prec must be one of {sorted(_PREC)}")
        self.dtype = torch.float64 if prec == "f64" else torch.float32
        self.prec, self.wind = prec, wind
        self._keep = []
        descs = (L.MeshDesc * len(meshes))()
        for i, (coords, elems, rep) in enumerate(meshes):
            c = np.ascontiguousarray(coords, dtype=np.float64)
            e = np.ascontiguousarray(elems, dtype=np.int64)
            r = None if rep is None else np.ascontiguousarray(rep, dtype=np.int64)
            self._keep += [c, e, r]
            descs[i] = L.MeshDesc(c.shape[1], c.shape[0], c.ctypes.data, e.shape[0], e.ctypes.data,
                                  None if r is None else r.ctypes.data)
        self.dim = int(descs[0].dim)
        karr = (ctypes.c_int * len(ks))(*[int(x) for x in ks])
        opts = L.Options(0, l, _PREC[prec], _WIND[wind], 0)
        self.b = c_void_p()
        self.stream = torch.cuda.Stream(device=self.device)
        with torch.cuda.device(self.device):
            st = self.lib.hopu_batch_create(descs, karr, len(meshes), byref(opts), c_void_p(self.stream.cuda_stream),
                                            byref(self.b))
        if st != L.HOPU_OK:
            raise L.HopuError(st, "hopu_batch_create", self.lib.hopu_batch_last_error(None).decode())
        nc = ctypes.c_int()
        self.lib.hopu_batch_classes(self.b, byref(nc), None, None, None)
        n = nc.value
        ck, nh, nl = (ctypes.c_int * n)(), (c_int64 * n)(), (c_int64 * n)()
        self.lib.hopu_batch_classes(self.b, byref(nc), ck, nh, nl)
        self.classes = []
        for c in range(n):
            ctx = c_void_p()
            self.lib.hopu_batch_context(self.b, c, byref(ctx))
            self.classes.append(_ClassView(self, ctx, ck[c], nh[c], nl[c]))
        self.layout = []
        for i in range(len(meshes)):
            o = (c_int64 * 7)()
            self.lib.hopu_batch_layout(self.b, i, o)
            self.layout.append(tuple(int(x) for x in o))

    def mesh_views(self, i: int, class_state: torch.Tensor, space: str = "hdiv"):
        """(facet dofs, interior dofs) views of mesh i in a V_h class vector, or its L2 block."""
        c, fo, fl, io, il, lo, ll = self.layout[i]
        if space == "hdiv":
            return class_state[fo:fo + fl], class_state[io:io + il]
        return class_state[lo:lo + ll]

    def rk_substep(self, class_states, dt: float, n_substeps: int = 1):
        ptrs = (c_void_p * len(self.classes))()
        for c, (v, t) in enumerate(zip(self.classes, class_states)):
            n = v.n_hdiv if self.wind == "stage" else v.n_l2
            ptrs[c] = v._vec(t, n, f"class_states[{c}]")
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)             # inputs produced on the caller's stream
        st = self.lib.hopu_batch_rk_substep(self.b, ptrs, float(dt), int(n_substeps))
        cur.wait_stream(self.stream)             # results visible on the caller's stream
        if st != L.HOPU_OK:
            raise L.HopuError(st, "hopu_batch_rk_substep", self.lib.hopu_batch_last_error(self.b).decode())

    def close(self):
        if getattr(self, "b", None) is not None and self.b.value:
            for v in self.classes:
                v.close()
            self.lib.hopu_batch_destroy(self.b)
            self.b = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HopuHex:
    """A structured periodic box of parallelepipeds at order k (mirrors a ``hopu_hex``).

    lines: three increasing arrays of grid-line positions (n_a + 1 each); A: 3x3 matrix,
    det A > 0 (cell (c0, c1, c2) is A [lines0[c0], lines0[c0+1]] x ...); periodic: per
    direction, else walls / outlets at its ends.  L2 vectors are [E][3][(k+1)^3] device
    tensors in the context's precision."""

    def __init__(self, lines, A, k: int = 3, prec: str = "f64", device: str | torch.device = "cuda",
                 periodic=(True, True, True)):
        if not torch.cuda.is_available():
            raise RuntimeError("libhopu needs a CUDA device")
        if prec not in ("f64", "f32"):
            raise ValueError("prec must be 'f64' or 'f32'")
        self.lib = L.load()
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.dtype = torch.float64 if prec == "f64" else torch.float32
        self.k, self.prec = k, prec
        self.n = tuple(len(x) - 1 for x in lines)
        self._lines = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64) for x in lines]))
        self._A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(3, 3))
        self.stream = torch.cuda.current_stream(self.device)
        self.h = c_void_p()
        with torch.cuda.device(self.device):
            mask = sum(1 << a for a in range(3) if periodic[a])
            st = self.lib.hopu_hex_create(self.n[0], self.n[1], self.n[2], self._lines.ctypes.data,
                                          self._A.ctypes.data, mask, int(k), _PREC[prec],
                                          c_void_p(self.stream.cuda_stream), byref(self.h))
        if st != L.HOPU_OK:
            raise L.HopuError(st, "hopu_hex_create", self.lib.hopu_hex_last_error(None).decode())
        ne, nl = c_int64(), c_int64()
        self.lib.hopu_hex_sizes(self.h, byref(ne), byref(nl))
        self.n_elems, self.n_l2 = ne.value, nl.value

    def _check(self, st: int, where: str):
        if st != L.HOPU_OK:
            raise L.HopuError(st, where, self.lib.hopu_hex_last_error(self.h).decode())

    def _vec(self, t: torch.Tensor, name: str) -> int:
        if (not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != self.dtype
                or not t.is_contiguous() or t.numel() != self.n_l2):
            raise ValueError(f"{name}: expected a contiguous {self.dtype} tensor of {self.n_l2} entries "
                             f"on {self.device}")
        return t.data_ptr()

    def new(self) -> torch.Tensor:
        return torch.empty(self.n_l2, dtype=self.dtype, device=self.device)

    def apply(self, wL: torch.Tensor, uL: torch.Tensor, l: int, out: torch.Tensor | None = None) -> torch.Tensor:
        """y = M^-1 c(w; u, .) (hopu_hex_apply), on the context's stream."""
        y = self.new() if out is None else out
        self._check(self.lib.hopu_hex_apply(self.h, c_void_p(self._vec(wL, "wL")), c_void_p(self._vec(uL, "uL")),
                                            int(l), c_void_p(self._vec(y, "yL"))), "hopu_hex_apply")
        return y

    def rk_substeps(self, uL: torch.Tensor, dt: float, n: int, l: int) -> torch.Tensor:
        """n SSP-RK3 substeps in place, wind = the stage's field (hopu_hex_rk_substeps)."""
        self._check(self.lib.hopu_hex_rk_substeps(self.h, c_void_p(self._vec(uL, "uL")), float(dt), int(n), int(l)),
                    "hopu_hex_rk_substeps")
        return uL

    def set_inlet(self, dir: int, end: int, modes: torch.Tensor | None):
        """Inlet data of one end of a non-periodic direction (hopu_hex_set_inlet): facet modes
        [n_s * n_t, 3, (k+1)^2] in the context's precision, or None for a wall / outlet."""
        ptr = None
        if modes is not None:
            if modes.device != self.device or modes.dtype != self.dtype or not modes.is_contiguous():
                raise ValueError(f"modes: expected a contiguous {self.dtype} tensor on {self.device}")
            ptr = c_void_p(modes.data_ptr())
        self._check(self.lib.hopu_hex_set_inlet(self.h, int(dir), int(end), ptr), "hopu_hex_set_inlet")

    def set_facet_l(self, facet_l: torch.Tensor | None):
        """Per-facet orders (int8 [3E] on the device; hopu_hex_set_facet_l); None: per call."""
        if facet_l is not None and (facet_l.dtype != torch.int8 or facet_l.device != self.device
                                    or facet_l.numel() != 3 * self.n_elems or not facet_l.is_contiguous()):
            raise ValueError("facet_l: expected a contiguous int8 tensor of 3E entries on the device")
        self._facet_l = facet_l                 # kept alive: the library reads it at every launch
        self._check(self.lib.hopu_hex_set_facet_l(self.h, None if facet_l is None else c_void_p(facet_l.data_ptr())),
                    "hopu_hex_set_facet_l")

    def adapt_l(self, uL: torch.Tensor, thresholds, facet_l: torch.Tensor, eta: torch.Tensor | None = None):
        """Adaptive HOPU step (hopu_hex_adapt_l): facet_l (int8 [3E], in/out) gets the new
        orders from the jump indicator; eta (float64 [3E]) receives it when given."""
        th = (c_double * (self.k + 1))(*[float(x) for x in thresholds])
        self._check(self.lib.hopu_hex_adapt_l(self.h, c_void_p(self._vec(uL, "uL")), th, c_void_p(facet_l.data_ptr()),
                                              None if eta is None else c_void_p(eta.data_ptr())), "hopu_hex_adapt_l")
        return facet_l

    def energy(self, uL: torch.Tensor, wL: torch.Tensor | None = None, l: int = -1):
        """(1/2 int |u|^2, c(w; u, u), facet dissipation) in FP64 (hopu_hex_energy)."""
        out = (c_double * 3)()
        w = None if wL is None else c_void_p(self._vec(wL, "wL"))
        self._check(self.lib.hopu_hex_energy(self.h, w, c_void_p(self._vec(uL, "uL")), int(l), out),
                    "hopu_hex_energy")
        return out[0], out[1], out[2]

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.lib.hopu_hex_destroy(self.h)
            self.h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_alu_peak(fp64: bool = False, iters: int | None = None) -> float:
    """Measured FMA throughput (TFLOP/s) of the current CUDA device (hopu_measure_alu_peak)."""
    lib = L.load()
    out = c_double()
    it = int(iters if iters is not None else (50 if fp64 else 2000))
    st = lib.hopu_measure_alu_peak(1 if fp64 else 0, it, byref(out))
    if st != L.HOPU_OK:
        raise L.HopuError(st, "hopu_measure_alu_peak")
    return float(out.value)


def selftest(dim: int, k: int):
    """Host-only check of the library's reference tables (no GPU needed)."""
    lib = L.load()
    rep = (c_double * 4)()
    st = lib.hopu_selftest(dim, k, rep)
    if st != L.HOPU_OK:
        raise L.HopuError(st, "hopu_selftest")
    return list(rep)

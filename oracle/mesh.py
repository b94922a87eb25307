"""Mesh topology and affine geometry for the oracle (FP64).

Conventions (they fix the layout of every coefficient vector):

* Every element's vertices are reordered by ascending periodic-representative id
  before its affine map x = x_0 + J xhat is formed.  A shared facet then has the
  same vertex order seen from both sides, which fixes one parametrisation of the
  facet for both neighbours (the mesh notation of Section 2.1: T, T', facet E).
* Local facet f of an element is the facet opposite local vertex f.
* Facets are numbered by the lexicographic order of their sorted representative
  vertex tuples.
* Canonical facet normal n_F: the unit right-hand normal (P1-P0) x (P2-P0) of the
  sorted vertex triple (3D), or the sorted edge direction turned by -90 degrees
  (2D).  Side A of a facet is the element whose outward normal equals n_F, side B
  the other one, so that [[u]] = u^A - u^B and n = n_F as in Section 2.1.
* sigma[e, f] = sign(n_F . n_out(e,f)) * sign(det J_e), the sign relating the
  global facet degree of freedom to the reference facet functional.

Facets with a single neighbour are boundary facets (side B = -1).
"""
from __future__ import annotations

import numpy as np

from .fe import scaled_outward_normal


class MeshTopo:
    def __init__(self, coords, elems, rep=None):
        coords = np.asarray(coords, dtype=np.float64)
        elems = np.asarray(elems, dtype=np.int64)
        if rep is None:
            rep = np.arange(coords.shape[0], dtype=np.int64)
        rep = np.asarray(rep, dtype=np.int64)
        d = coords.shape[1]
        self.dim = d
        E = elems.shape[0]
        self.n_elems = E
        order = np.argsort(rep[elems], axis=1, kind="stable")
        self.ev = np.take_along_axis(elems, order, axis=1)
        self.X = coords[self.ev]                                     # [E, d+1, d]
        self.J = np.transpose(self.X[:, 1:, :] - self.X[:, :1, :], (0, 2, 1))  # J[:, :, j] = x_{j+1}-x_0
        self.detJ = np.linalg.det(self.J)
        self.Jinv = np.linalg.inv(self.J)
        self.absdet = np.abs(self.detJ)

        # ---- facets
        loc = [[j for j in range(d + 1) if j != f] for f in range(d + 1)]
        keys = np.stack([rep[self.ev[:, loc[f]]] for f in range(d + 1)], axis=1)  # [E, d+1, d]
        flat = keys.reshape(-1, d)
        uniq, inv, counts = np.unique(flat, axis=0, return_inverse=True, return_counts=True)
        inv = inv.reshape(E, d + 1)
        self.n_facets = uniq.shape[0]
        self.elem_facet = inv                                         # [E, d+1]
        if np.any(counts > 2):
            raise ValueError("non-manifold mesh: a facet has more than two neighbours")

        # outward (unnormalised) normals of every (e, f): J^{-T} Nhat_f
        Nhat = np.array([scaled_outward_normal(d, f) for f in range(d + 1)])
        out = np.einsum("ecb,fc->efb", self.Jinv, Nhat)              # [E, d+1, d] (J^{-T} Nhat)

        # canonical normal and area factor from each (e, f)'s own physical vertices
        P = np.stack([self.X[:, loc[f], :] for f in range(d + 1)], axis=1)  # [E, d+1, d, d]
        if d == 3:
            cr = np.cross(P[:, :, 1] - P[:, :, 0], P[:, :, 2] - P[:, :, 0])
        else:
            t = P[:, :, 1] - P[:, :, 0]
            cr = np.stack([t[..., 1], -t[..., 0]], axis=-1)
        area = np.linalg.norm(cr, axis=-1)                            # |F| / |param simplex|
        nF = cr / area[..., None]
        s = np.sign(np.einsum("efb,efb->ef", nF, out))
        self.sigma = s * np.sign(self.detJ)[:, None]                  # [E, d+1]

        # side A / B per facet
        fa_e = -np.ones(self.n_facets, dtype=np.int64)
        fa_f = -np.ones(self.n_facets, dtype=np.int64)
        fb_e = -np.ones(self.n_facets, dtype=np.int64)
        fb_f = -np.ones(self.n_facets, dtype=np.int64)
        self.nF = np.zeros((self.n_facets, d))
        self.aF = np.zeros(self.n_facets)
        ee, ff = np.meshgrid(np.arange(E), np.arange(d + 1), indexing="ij")
        ee, ff, FF = ee.reshape(-1), ff.reshape(-1), inv.reshape(-1)
        sA = s.reshape(-1) > 0
        # side A: outward normal agrees with the canonical normal
        fa_e[FF[sA]] = ee[sA]
        fa_f[FF[sA]] = ff[sA]
        fb_e[FF[~sA]] = ee[~sA]
        fb_f[FF[~sA]] = ff[~sA]
        nflat = nF.reshape(-1, d)
        aflat = area.reshape(-1)
        self.nF[FF] = nflat
        self.aF[FF] = aflat
        if np.any(fa_e < 0):
            # boundary facet whose only neighbour points against n_F: flip the
            # facet's orientation so that its single neighbour becomes side A.
            bad = np.where(fa_e < 0)[0]
            fa_e[bad], fa_f[bad] = fb_e[bad], fb_f[bad]
            fb_e[bad], fb_f[bad] = -1, -1
            self.nF[bad] = -self.nF[bad]
            for F in bad:
                e, f = fa_e[F], fa_f[F]
                self.sigma[e, f] = -self.sigma[e, f]
        self.fa = np.stack([fa_e, fa_f], axis=1)
        self.fb = np.stack([fb_e, fb_f], axis=1)
        self.boundary = fb_e < 0
        # side of each (e, f): +1 if e is side A of its facet, -1 if side B
        self.side = np.where(self.fa[self.elem_facet, 0] == np.arange(E)[:, None], 1, -1)

    def facet_points(self, sq: np.ndarray) -> np.ndarray:
        """Physical points [F, nqf, d] of facet parameters sq, taken from side A."""
        d = self.dim
        e, f = self.fa[:, 0], self.fa[:, 1]
        loc = np.array([[j for j in range(d + 1) if j != ff] for ff in range(d + 1)])
        P = self.X[e[:, None], loc[f]]                                 # [F, d, d]
        return P[:, None, 0, :] + np.einsum("qj,Fjc->Fqc", sq, P[:, 1:, :] - P[:, None, 0, :])

    def volume_points(self, xq: np.ndarray) -> np.ndarray:
        """Physical points [E, nq, d] of reference points xq."""
        return self.X[:, None, 0, :] + np.einsum("ecj,qj->eqc", self.J, xq)

"""The normal-continuous velocity space V_h of the oracle (FP64).

Reading of the paper: the velocity space of Section 2.2 (eq. "disc_velspace")
must have tangential facet traces in P^k for "Pi^l = I when l = k"
(Section 3.2) to hold, so V_h is taken as the normal-continuous [P^k]^d space
(the BDM_k element of the paper's reference [boffi2013mixed]).  Its local space
is all of [P^k(T)]^d, so V_h embeds exactly in the discontinuous space used by
the convection operator.

Degrees of freedom (they fix the layout of a V_h coefficient vector):

* facet F, m = 0..nf-1:  int_F (u . n_F) q_m ds, with q_m(x(s)) the orthonormal
  Dubiner polynomial of the facet parameter s (sorted-vertex parametrisation);
  stored first, facet-major: index F*nf + m.
* element T, j = 0..nint-1: int_That uhat . z_j dxhat, with uhat the contravariant
  Piola pull-back (u = J uhat / det J) and z_j the interior moment functions of
  ``fe.interior_space``; stored after the facets: index F*nf + T*nint + j.

Maps (Section 2.3 names the averaging operator R used by the element-wise BDDC
solver; the same averaging brings an element-wise field back to V_h):

* ``to_l2``    E  : V_h -> L2, element-wise gather, reference change of basis,
                    Piola map.  Pinned: ``from_l2(to_l2(u)) == u`` (tests) and the
                    normal continuity of the result.
* ``from_l2``  R E_T^{-1}: L2 -> V_h, local functionals then R (average of the two
                    copies of each facet functional).  Pinned by the same round trip.
* ``dual``     E^T: restriction of an L2 residual to V_h test functions (the
                    paper's C u^n of the matrix form).  Pinned by the adjoint
                    identity <E x, y> = <x, E^T y> (tests).
* ``interpolate`` the canonical interpolant from the moments above (quadrature
                    of a given function).  Pinned: it reproduces [P^k]^d fields that
                    are normal-continuous (tests).
"""
from __future__ import annotations

import numpy as np

from .fe import RefElement
from .mesh import MeshTopo


def reference_dof_matrix(ref: RefElement) -> np.ndarray:
    """D[row, b*nb + i] = functional_row(phi_i e_b) on the reference element."""
    d, nb, nf, nint = ref.dim, ref.nb, ref.nf, ref.nint
    n = d * nb
    D = np.zeros((n, n))
    for f in range(d + 1):
        T = np.einsum("q,qi,qm->mi", ref.wf, ref.phi_f[f], ref.psi)   # [nf, nb]
        for b in range(d):
            D[f * nf:(f + 1) * nf, b * nb:(b + 1) * nb] = ref.Nhat[f, b] * T
    for b in range(d):
        D[(d + 1) * nf:, b * nb:(b + 1) * nb] = np.einsum("q,qi,jq->ji", ref.wq, ref.phi, ref.z[:, :, b])
    return D


class HDiv:
    def __init__(self, topo: MeshTopo, ref: RefElement):
        self.topo, self.ref = topo, ref
        self.D = reference_dof_matrix(ref)
        self.Dinv = np.linalg.inv(self.D)
        self.n_facet_dofs = topo.n_facets * ref.nf
        self.n_hdiv = self.n_facet_dofs + topo.n_elems * ref.nint
        self.n_l2 = topo.n_elems * ref.dim * ref.nb

    # -------------------------------------------------------------- V_h -> L2
    def to_l2(self, uV: np.ndarray) -> np.ndarray:
        t, r = self.topo, self.ref
        d, nb, nf = r.dim, r.nb, r.nf
        fac = uV[: self.n_facet_dofs].reshape(t.n_facets, nf)
        inter = uV[self.n_facet_dofs:].reshape(t.n_elems, r.nint)
        loc_f = t.sigma[:, :, None] * fac[t.elem_facet]               # [E, d+1, nf]
        l = np.concatenate([loc_f.reshape(t.n_elems, -1), inter], axis=1)
        chat = (l @ self.Dinv.T).reshape(t.n_elems, d, nb)
        return np.einsum("eab,ebi->eai", t.J, chat) / t.detJ[:, None, None]

    # -------------------------------------------------------------- L2 -> V_h (R E_T^{-1})
    def local_functionals(self, uL: np.ndarray) -> np.ndarray:
        t = self.topo
        chat = t.detJ[:, None, None] * np.einsum("eba,eai->ebi", t.Jinv, uL)
        return chat.reshape(t.n_elems, -1) @ self.D.T

    def from_l2(self, uL: np.ndarray) -> np.ndarray:
        t, r = self.topo, self.ref
        nf = r.nf
        ell = self.local_functionals(uL)
        loc_f = ell[:, : (r.dim + 1) * nf].reshape(t.n_elems, r.dim + 1, nf) * t.sigma[:, :, None]
        acc = np.zeros((t.n_facets, nf))
        cnt = np.zeros(t.n_facets)
        np.add.at(acc, t.elem_facet.reshape(-1), loc_f.reshape(-1, nf))
        np.add.at(cnt, t.elem_facet.reshape(-1), 1.0)
        fac = acc / cnt[:, None]
        return np.concatenate([fac.reshape(-1), ell[:, (r.dim + 1) * nf:].reshape(-1)])

    # -------------------------------------------------------------- (R E_T^{-1})^T
    def from_l2_transpose(self, vV: np.ndarray) -> np.ndarray:
        """Transpose of ``from_l2``: distribute each facet value to its copies with the
        averaging weight (1/2 on interior facets) and the sign sigma, copy interior
        values, then apply (D Piola^{-1})^T per element."""
        t, r = self.topo, self.ref
        nf = r.nf
        cnt = np.zeros(t.n_facets)
        np.add.at(cnt, t.elem_facet.reshape(-1), 1.0)
        fac = vV[: self.n_facet_dofs].reshape(t.n_facets, nf) / cnt[:, None]
        loc_f = t.sigma[:, :, None] * fac[t.elem_facet]
        inter = vV[self.n_facet_dofs:].reshape(t.n_elems, r.nint)
        ell = np.concatenate([loc_f.reshape(t.n_elems, -1), inter], axis=1)
        chat = (ell @ self.D).reshape(t.n_elems, r.dim, r.nb)
        return t.detJ[:, None, None] * np.einsum("eba,ebi->eai", t.Jinv, chat)

    # -------------------------------------------------------------- E^T
    def dual(self, rL: np.ndarray) -> np.ndarray:
        t, r = self.topo, self.ref
        nf = r.nf
        rhat = np.einsum("eab,eai->ebi", t.J, rL) / t.detJ[:, None, None]
        l = rhat.reshape(t.n_elems, -1) @ self.Dinv
        loc_f = l[:, : (r.dim + 1) * nf].reshape(t.n_elems, r.dim + 1, nf) * t.sigma[:, :, None]
        acc = np.zeros((t.n_facets, nf))
        np.add.at(acc, t.elem_facet.reshape(-1), loc_f.reshape(-1, nf))
        return np.concatenate([acc.reshape(-1), l[:, (r.dim + 1) * nf:].reshape(-1)])

    # -------------------------------------------------------------- interpolant
    def facet_points(self):
        return self.topo.facet_points(self.ref.sq)

    def volume_points(self):
        return self.topo.volume_points(self.ref.xq)

    def interpolate_values(self, fvals: np.ndarray, vvals: np.ndarray) -> np.ndarray:
        """Moments of a field given at facet points [F, nqf, d] and volume points [E, nq, d]."""
        t, r = self.topo, self.ref
        un = np.einsum("Fqc,Fc->Fq", fvals, t.nF)
        fac = t.aF[:, None] * np.einsum("q,Fq,qm->Fm", r.wf, un, r.psi)
        uhat = t.detJ[:, None, None] * np.einsum("eba,eqa->eqb", t.Jinv, vvals)
        inter = np.einsum("q,eqb,jqb->ej", r.wq, uhat, r.z)
        return np.concatenate([fac.reshape(-1), inter.reshape(-1)])

    def interpolate(self, fun) -> np.ndarray:
        return self.interpolate_values(fun(self.facet_points()), fun(self.volume_points()))

    # -------------------------------------------------------------- L2 helpers
    def l2_project(self, fun) -> np.ndarray:
        """Element-wise L2 projection of fun onto [P^k]^d (orthonormal basis)."""
        t, r = self.topo, self.ref
        vals = fun(self.volume_points())                               # [E, nq, d]
        return np.einsum("q,qi,eqa->eai", r.wq, r.phi, vals)

    def evaluate(self, uL: np.ndarray, xref: np.ndarray) -> np.ndarray:
        """Values [E, N, d] of an L2 field at reference points xref [N, d]."""
        from .fe import dubiner
        v, _ = dubiner(self.ref.dim, self.ref.k, xref)
        return np.einsum("qi,eai->eqa", v, uL)

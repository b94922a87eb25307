"""HOPU convection operator of the oracle (FP64).

The paper's form (Section 3.2, eq. "hopudefinition"; with Pi = 0 it is the upwind
form of Section 2.2, eq. "upwind"):

  c(w; u, v) = sum_T int_T ((grad u) w) . v
             + sum_{E in F^I} [ - int_E (w.n) [[u]] . <v>
                                + int_E 1/2 |w.n| (I - Pi^l)[[u]] . (I - Pi^l)[[v]] ]

with [[u]] = u^T - u^T', <u> = (u^T + u^T')/2, n outward of T (Section 2.1).

Conservative reading (the operator the GPU path applies): integrating the volume
term by parts element by element gives

  c(w; u, v) = sum_T - int_T (u (x) w) : grad v
             + sum_E int_E [ (w.n) <u> + (I - Pi^l)[ 1/2 |w.n| (I - Pi^l)[[u]] ] ] . [[v]]

which equals the form above whenever w is normal-continuous and divergence-free
in every element (the difference is sum_T int_T (div w) u . v).  Both are coded
here, independently; tests pin one against the other.

Pi^l: facet-wise L2 projection onto tangential P^l vector fields (Section 3.2).
On an affine facet the normal n is constant, so Pi^l V = (I - n n^T) Pi_s^l V
with Pi_s^l the scalar P^l projection applied per Cartesian component.  l = -1
means Pi = 0 (standard upwind, ILES of Section 3.1); l = k gives the central
flux for normal-continuous u.  w.n is evaluated as <w>.n, which equals w.n for
normal-continuous w.

Integrals use the rules of ``fe.RefElement`` (exact to degree 3k-1 in the volume
and 3k on facets; the factor |w.n| is not a polynomial and is integrated by the
same facet rule).

Pins (tests/test_oracle_convection.py): y = 0 for constant u and divergence-free
w; conservative = non-conservative form for divergence-free w; the energy
identity c(w;u,u) = sum_F int 1/2 |w.n| |(I-Pi^l)[[u]]|^2; l = k central limit;
monotonicity in l for constant wind; momentum conservation; single-element
exactness with inlet data; order-k convergence on Taylor-Green.
"""
from __future__ import annotations

import numpy as np

from .fe import RefElement, n_basis
from .mesh import MeshTopo


def _as_facet_l(topo: MeshTopo, l) -> np.ndarray:
    if np.isscalar(l):
        return np.full(topo.n_facets, int(l), dtype=np.int64)
    return np.asarray(l, dtype=np.int64)


def facet_trace(topo: MeshTopo, ref: RefElement, vL: np.ndarray, side: str) -> np.ndarray:
    """Values [F, nqf, d] of an L2 field on every facet, seen from side 'A' or 'B'.

    Boundary facets have no side B; their entries are left at zero.
    """
    ef = topo.fa if side == "A" else topo.fb
    out = np.zeros((topo.n_facets, ref.wf.shape[0], ref.dim))
    for f in range(ref.dim + 1):
        m = ef[:, 1] == f
        if np.any(m):
            out[m] = np.einsum("qi,Fai->Fqa", ref.phi_f[f], vL[ef[m, 0]])
    return out


def complement_projection(ref: RefElement, l_F: np.ndarray, nF: np.ndarray,
                          V: np.ndarray) -> np.ndarray:
    """(I - Pi^l) V at the facet points; V [F, nqf, d]; Pi^l onto tangential P^l."""
    out = V.copy()
    d = ref.dim
    for l in np.unique(l_F):
        if l < 0:
            continue
        m = l_F == l
        Psi = ref.psi[:, : n_basis(d - 1, int(l))]
        coef = np.einsum("q,qm,Fqa->Fma", ref.wf, Psi, V[m])
        PiS = np.einsum("qm,Fma->Fqa", Psi, coef)
        n = nF[m]
        PiV = PiS - np.einsum("Fqa,Fa->Fq", PiS, n)[..., None] * n[:, None, :]
        out[m] = V[m] - PiV
    return out


def facet_quantities(topo, ref, wL, uL, l, exterior=None, inlet=None):
    """Per facet point: w.n, [[u]], <u>, (I-Pi)[[u]] and (I-Pi)[1/2|w.n|(I-Pi)[[u]]].

    Boundary facets (Section 2.1: F^I holds interior, periodic and inlet facets; wall
    and outlet facets carry no term in the paper's form):
    * inlet facets take the given exterior traces as side B (Section 2.2: the jump and
      the average use u_I); exterior = (u_ext, w_ext) arrays [F, nqf, d]; inlet is a
      boolean mask [F] (None: every boundary facet is an inlet when exterior is given).
      The wind of a V_h field has a single-valued normal component, so callers give
      w_ext = the wind's own trace (reading A12); a different w_ext is also accepted;
    * the other boundary facets (walls, outlets) take side A's own trace as side B:
      the jump vanishes, so the paper's form has no term there, and the conservative
      form keeps the flux (w.n) u . v that its element-wise integration by parts needs
      to equal the paper's form (reading A12).
    """
    l_F = _as_facet_l(topo, l)
    uA, wA = facet_trace(topo, ref, uL, "A"), facet_trace(topo, ref, wL, "A")
    uB, wB = facet_trace(topo, ref, uL, "B"), facet_trace(topo, ref, wL, "B")
    if np.any(topo.boundary):
        b = topo.boundary
        uB[b], wB[b] = uA[b], wA[b]
        if exterior is not None:
            bi = b if inlet is None else (b & np.asarray(inlet, dtype=bool))
            uB[bi], wB[bi] = exterior[0][bi], exterior[1][bi]
    wn = 0.5 * np.einsum("Fqa,Fa->Fq", wA + wB, topo.nF)
    jump = uA - uB
    avg = 0.5 * (uA + uB)
    PJ = complement_projection(ref, l_F, topo.nF, jump)
    Ph = complement_projection(ref, l_F, topo.nF, 0.5 * np.abs(wn)[..., None] * PJ)
    return wn, jump, avg, PJ, Ph


def _test_facets(topo, ref, r, g, side):
    """r[e] += sign * a_F int_param g . phi_i(facet point) for the given side."""
    ef = topo.fa if side == "A" else topo.fb
    for f in range(ref.dim + 1):
        m = (ef[:, 1] == f) & (ef[:, 0] >= 0)
        if np.any(m):
            contrib = topo.aF[m, None, None] * np.einsum("q,Fqa,qi->Fai", ref.wf, g[m], ref.phi_f[f])
            np.add.at(r, ef[m, 0], contrib)


def residual_conservative(topo, ref, wL, uL, l, exterior=None, inlet=None) -> np.ndarray:
    """r[e, a, i] = c(w; u, phi_i e_a) in the conservative reading."""
    U = np.einsum("qi,eai->eqa", ref.phi, uL)
    W = np.einsum("qi,eai->eqa", ref.phi, wL)
    Wt = np.einsum("e,ecb,eqb->eqc", topo.absdet, topo.Jinv, W)       # |det J| J^{-1} w
    r = -np.einsum("q,eqa,qic,eqc->eai", ref.wq, U, ref.dphi, Wt)
    wn, jump, avg, PJ, Ph = facet_quantities(topo, ref, wL, uL, l, exterior, inlet)
    g = wn[..., None] * avg + Ph
    _test_facets(topo, ref, r, g, "A")
    _test_facets(topo, ref, r, -g, "B")
    return r


def residual_nonconservative(topo, ref, wL, uL, l, exterior=None, inlet=None) -> np.ndarray:
    """r[e, a, i] = c(w; u, phi_i e_a) in the paper's form (eq. "hopudefinition")."""
    W = np.einsum("qi,eai->eqa", ref.phi, wL)
    gref = np.einsum("qic,eai->eqac", ref.dphi, uL)                     # reference gradient
    grad = np.einsum("ecb,eqac->eqab", topo.Jinv, gref)                 # d u_a / d x_b
    adv = np.einsum("eqab,eqb->eqa", grad, W)                           # (grad u) w
    r = np.einsum("q,e,eqa,qi->eai", ref.wq, topo.absdet, adv, ref.phi)
    wn, jump, avg, PJ, Ph = facet_quantities(topo, ref, wL, uL, l, exterior, inlet)
    central = -0.5 * wn[..., None] * jump                               # -(w.n)[[u]].<v>
    _test_facets(topo, ref, r, central + Ph, "A")                       # [[v]] = v^A
    _test_facets(topo, ref, r, central - Ph, "B")                       # [[v]] = -v^B
    return r


def apply(topo, ref, wL, uL, l, form="conservative", exterior=None, inlet=None) -> np.ndarray:
    """y = M_L^{-1} c(w; u, .) (orthonormal basis: M_T = |det J| I)."""
    fn = residual_conservative if form == "conservative" else residual_nonconservative
    return fn(topo, ref, wL, uL, l, exterior, inlet) / topo.absdet[:, None, None]


# ------------------------------------------------------------------ functionals
def kinetic_energy(topo, uL) -> float:
    """1/2 int |u|^2 = 1/2 sum_T |det J| |c_T|^2."""
    return 0.5 * float(np.sum(topo.absdet[:, None, None] * uL * uL))


def form_value(topo, ref, wL, uL, l) -> float:
    """c(w; u, u)."""
    return float(np.sum(uL * residual_conservative(topo, ref, wL, uL, l)))


def facet_dissipation(topo, ref, wL, uL, l) -> float:
    """sum_F int_F 1/2 |w.n| |(I-Pi^l)[[u]]|^2."""
    wn, jump, avg, PJ, Ph = facet_quantities(topo, ref, wL, uL, l)
    return float(np.sum(topo.aF[:, None] * ref.wf[None, :] * 0.5 * np.abs(wn) * np.sum(PJ * PJ, axis=-1)))

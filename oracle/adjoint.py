"""Derivatives of the convection apply and of explicit rollouts (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The apply is y = M^{-1} c(w; u, .) with the conservative form of Section 3.2
(eq. "hopudefinition", reading A2):

  c(w; u, v) = - sum_T int u . (w . grad) v
               + sum_F int (w.n) <u> . [[v]] + 1/2 |w.n| (I-Pi)[[u]] . (I-Pi)[[v]],

linear in u and in v, and in w except for |w.n| (w.n = <w>.n on facets).  With
z = M^{-1} ybar:

* JVP  (du, dw):  M^{-1} [ c(w; du, .) + c_w(w; u, .)[dw] ],  where c_w replaces
  |w.n| by sign(w.n)(dw.n) and (w.n) by (dw.n) and w by dw in the volume term;
* VJP: ubar = c(w; phi_j, z) (the transposed form, u-slot basis function phi_j),
       wbar = d/dw c(w; u, z) tested with phi_j:
         volume  -sum_a u_a d_b z_a,
         facet   for both sides' wind traces: n [1/2 <u>.[[z]] + 1/4 sign(w.n) PJ(u).PJ(z)],
  with PJ = (I - Pi)[[.]] and sign(0) = 0 (the reading for the kink of |s| at s = 0).

Pins (tests/test_oracle_adjoint.py): the JVP against central finite differences of
``convection.apply``; the dot-product identity <ybar, J x> = <J^T ybar, x> between the two
independently written derivatives; the rollout adjoint against finite differences of
the rollout loss.
"""
from __future__ import annotations

import numpy as np

from . import convection as C
from .hdiv import HDiv


def _grad_ref(ref, vL):
    """Reference gradients [E, nq, d(component), d(direction)] of an L2 field."""
    return np.einsum("qic,eai->eqac", ref.dphi, vL)


def _facet_fields(topo, ref, wL, uL, zL, l):
    """Point values on facets: w.n, <u>, (I-Pi)[[u]], [[z]], (I-Pi)[[z]]."""
    l_F = C._as_facet_l(topo, l)
    tr = lambda v, s: C.facet_trace(topo, ref, v, s)
    uA, uB, wA, wB, zA, zB = tr(uL, "A"), tr(uL, "B"), tr(wL, "A"), tr(wL, "B"), tr(zL, "A"), tr(zL, "B")
    wn = 0.5 * np.einsum("Fqa,Fa->Fq", wA + wB, topo.nF)
    PJu = C.complement_projection(ref, l_F, topo.nF, uA - uB)
    Jz = zA - zB
    PJz = C.complement_projection(ref, l_F, topo.nF, Jz)
    return l_F, wn, 0.5 * (uA + uB), PJu, Jz, PJz


def vjp_apply(topo, ref, wL, uL, ybar, l):
    """(wbar_L, ubar_L) = cotangents of y = apply(w, u) for the cotangent ybar."""
    z = ybar / topo.absdet[:, None, None]
    W = np.einsum("qi,eai->eqa", ref.phi, wL)
    U = np.einsum("qi,eai->eqa", ref.phi, uL)
    gz = np.einsum("ecb,eqac->eqab", topo.Jinv, _grad_ref(ref, z))        # d z_a / d x_b
    # ubar volume: -int ((w.grad) z) . phi_i
    ub = -np.einsum("q,e,eqb,eqab,qi->eai", ref.wq, topo.absdet, W, gz, ref.phi)
    # wbar volume: -int sum_a u_a d_b z_a phi_j
    wb = -np.einsum("q,e,eqa,eqab,qi->ebi", ref.wq, topo.absdet, U, gz, ref.phi)
    l_F, wn, avg_u, PJu, Jz, PJz = _facet_fields(topo, ref, wL, uL, z, l)
    hz = C.complement_projection(ref, l_F, topo.nF, 0.5 * np.abs(wn)[..., None] * PJz)
    central = 0.5 * wn[..., None] * Jz
    C._test_facets(topo, ref, ub, central + hz, "A")
    C._test_facets(topo, ref, ub, central - hz, "B")
    s = 0.5 * np.einsum("Fqa,Fqa->Fq", avg_u, Jz) + 0.25 * np.sign(wn) * np.einsum("Fqa,Fqa->Fq", PJu, PJz)
    sn = s[..., None] * topo.nF[:, None, :]
    C._test_facets(topo, ref, wb, sn, "A")
    C._test_facets(topo, ref, wb, sn, "B")
    return wb, ub


def jvp_apply(topo, ref, wL, uL, dw, du, l):
    """Directional derivative of apply(w, u) in the direction (dw, du), written out."""
    # d/du: the operator is linear in u
    r = C.residual_conservative(topo, ref, wL, du, l)
    # d/dw: volume term is linear in w; on facets w.n enters linearly and through |w.n|
    U = np.einsum("qi,eai->eqa", ref.phi, uL)
    dW = np.einsum("qi,eai->eqa", ref.phi, dw)
    dWt = np.einsum("e,ecb,eqb->eqc", topo.absdet, topo.Jinv, dW)
    r = r - np.einsum("q,eqa,qic,eqc->eai", ref.wq, U, ref.dphi, dWt)
    l_F = C._as_facet_l(topo, l)
    tr = lambda v, s: C.facet_trace(topo, ref, v, s)
    uA, uB, wA, wB = tr(uL, "A"), tr(uL, "B"), tr(wL, "A"), tr(wL, "B")
    dA, dB = tr(dw, "A"), tr(dw, "B")
    wn = 0.5 * np.einsum("Fqa,Fa->Fq", wA + wB, topo.nF)
    dwn = 0.5 * np.einsum("Fqa,Fa->Fq", dA + dB, topo.nF)
    PJ = C.complement_projection(ref, l_F, topo.nF, uA - uB)
    Ph = C.complement_projection(ref, l_F, topo.nF, 0.5 * (np.sign(wn) * dwn)[..., None] * PJ)
    g = dwn[..., None] * 0.5 * (uA + uB) + Ph
    C._test_facets(topo, ref, r, g, "A")
    C._test_facets(topo, ref, r, -g, "B")
    return r / topo.absdet[:, None, None]


# ------------------------------------------------------------------ rollouts
def _stage_rhs(space: HDiv, uV, l):
    uL = space.to_l2(uV)
    return space.from_l2(C.apply(space.topo, space.ref, uL, uL, l))


def _rhs_vjp(space: HDiv, uV, vbar, l):
    """J_F(u)^T vbar for F(u) = R E_T^{-1} apply(E u, E u)."""
    t, r = space.topo, space.ref
    ybar = space.from_l2_transpose(vbar)                  # (R E_T^{-1})^T
    uL = space.to_l2(uV)
    wb, ub = vjp_apply(t, r, uL, uL, ybar, l)
    return space.dual(wb + ub)                            # E^T


def rollout_loss(space: HDiv, u0V, dt, n, l):
    """Loss 1/2 int |E u_n|^2 after n STAGE SSP-RK3 substeps."""
    u = u0V.copy()
    for _ in range(n):
        u1 = u - dt * _stage_rhs(space, u, l)
        u2 = 0.75 * u + 0.25 * (u1 - dt * _stage_rhs(space, u1, l))
        u = u / 3.0 + 2.0 / 3.0 * (u2 - dt * _stage_rhs(space, u2, l))
    return C.kinetic_energy(space.topo, space.to_l2(u)), u


def rollout_vjp(space: HDiv, u0V, dt, n, l, seed=None):
    """(loss, d loss / d u0) by the discrete adjoint of the SSP-RK3 substeps.

    With ``seed`` (a V_h cotangent of u_n) the adjoint starts from it instead of the
    gradient of the loss, and the result is the cotangent of u0 (the loss is still
    returned)."""
    states = []
    u = u0V.copy()
    for _ in range(n):
        u1 = u - dt * _stage_rhs(space, u, l)
        u2 = 0.75 * u + 0.25 * (u1 - dt * _stage_rhs(space, u1, l))
        states.append((u, u1, u2))
        u = u / 3.0 + 2.0 / 3.0 * (u2 - dt * _stage_rhs(space, u2, l))
    uL = space.to_l2(u)
    loss = C.kinetic_energy(space.topo, uL)
    ubar = space.dual(space.topo.absdet[:, None, None] * uL) if seed is None else np.array(seed, dtype=float)
    for (u0, u1, u2) in reversed(states):
        b2 = 2.0 / 3.0 * (ubar - dt * _rhs_vjp(space, u2, ubar, l))
        b1 = 0.25 * (b2 - dt * _rhs_vjp(space, u1, b2, l))
        ubar = ubar / 3.0 + 0.75 * b2 + b1 - dt * _rhs_vjp(space, u0, b1, l)
    return loss, ubar

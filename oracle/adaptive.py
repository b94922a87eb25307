"""Adaptive HOPU of the oracle (FP64): the facet jump indicator and the order rule.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 3.2 (after eq. "hopudefinition") chooses the projection order l per facet
from the average absolute jump

    eta_E = int_E |(I - Pi^l)[[u]]| ds / int_E |<u>| ds

(|.| the Euclidean norm of the vector at a point), compared with increasing
thresholds eta_{-1} = 0 < eta_0 < ... < eta_k < eta_{k+1} = 1: for
eta_i < eta <= eta_{i+1} the facet uses l = i when i >= 0, and eta below eta_0 means
standard upwinding (l = -1).  The paper re-determines the orders every 10th time step
and uses the limits {0.1, 0.2, 0.3, 0.4} for k = 3.

Readings (where the passage is silent):
* eta depends on l through Pi^l; it is evaluated with the facet's current order
  (initially -1, i.e. Pi = 0);
* eta = 0 (including a facet where <u> vanishes identically together with the jump)
  gives l = -1; eta above eta_{k+1} = 1 gives l = k (the last interval extended);
* a facet whose int |<u>| is zero but whose jump is not gets eta = +inf, hence l = k.

Pins (tests/test_oracle_adaptive.py): closed forms of eta for piecewise-constant
fields on a two-element mesh and on a periodic box; eta = 0 for continuous fields and,
with l = k, for normal-continuous ones; the order rule at and between the thresholds.
"""
from __future__ import annotations

import numpy as np

from . import convection as C
from .mesh import MeshTopo


def facet_eta(topo: MeshTopo, ref, uL: np.ndarray, l) -> np.ndarray:
    """eta per facet of the L2 field uL with the facet orders l (scalar or [F])."""
    l_F = C._as_facet_l(topo, l)
    uA = C.facet_trace(topo, ref, uL, "A")
    uB = C.facet_trace(topo, ref, uL, "B")
    PJ = C.complement_projection(ref, l_F, topo.nF, uA - uB)
    num = np.einsum("q,Fq->F", ref.wf, np.linalg.norm(PJ, axis=-1))
    den = np.einsum("q,Fq->F", ref.wf, np.linalg.norm(0.5 * (uA + uB), axis=-1))
    with np.errstate(divide="ignore", invalid="ignore"):
        eta = np.where(den > 0, num / np.where(den > 0, den, 1.0), np.where(num > 0, np.inf, 0.0))
    return eta


def order_from_eta(eta: np.ndarray, thresholds, k: int) -> np.ndarray:
    """l per facet: i for thresholds[i] < eta <= thresholds[i+1] (thresholds[k+1] = 1
    implied, eta > 1 -> k), -1 for eta <= thresholds[0]."""
    th = np.asarray(thresholds, dtype=float)
    if th.shape != (k + 1,) or np.any(np.diff(th) <= 0) or th[0] <= 0 or th[-1] >= 1:
        raise ValueError("need k+1 increasing thresholds in (0, 1)")
    eta = np.asarray(eta, dtype=float)
    out = np.full(eta.shape, -1, dtype=np.int64)
    for i in range(k + 1):               # eta above thresholds[i] -> at least order i
        out[eta > th[i]] = i
    return out


def adapt(topo: MeshTopo, ref, uL: np.ndarray, l, thresholds) -> tuple[np.ndarray, np.ndarray]:
    """(eta, new l) for the current orders l."""
    eta = facet_eta(topo, ref, uL, l)
    return eta, order_from_eta(eta, thresholds, ref.k)

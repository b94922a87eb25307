"""Explicit SSP-RK3 substeps of the convection operator (oracle, FP64).

The paper treats convection explicitly (Section 2.3: the IMEX variant and the
projection splitting both evaluate c_h explicitly); it does not print the
explicit substep, so the Shu-Osher SSP-RK3 scheme is used:

  u1 = u - dt A(u);  u2 = 3/4 u + 1/4 (u1 - dt A(u1));  u+ = 1/3 u + 2/3 (u2 - dt A(u2)).

Wind rules (reading of the paper's silence on the wind inside substeps):

* STAGE  (default): the state lives in V_h; at every stage w = u = E u_V and
  A(u_V) = R E_T^{-1} M_L^{-1} c(E u_V; E u_V, .).  No closed form for the
  nonlinear stage map; pinned by the scheme's third order in dt (with the central
  flux the map is smooth and the error at a fixed time falls by 2^3 per halving),
  momentum conservation and first-order consistency (tests).
* FROZEN: the wind w = E w_V is fixed; the state lives in L2 and
  A(u_L) = M_L^{-1} c(w; u_L, .), which is linear in u_L.  Pinned: one substep
  equals u - dt A u + dt^2/2 A^2 u - dt^3/6 A^3 u (tests).
"""
from __future__ import annotations

import numpy as np

from . import convection
from .hdiv import HDiv


def stage_rhs(space: HDiv, uV: np.ndarray, l) -> np.ndarray:
    uL = space.to_l2(uV)
    y = convection.apply(space.topo, space.ref, uL, uL, l)
    return space.from_l2(y)


def ssp_rk3(rhs, u: np.ndarray, dt: float) -> np.ndarray:
    u1 = u - dt * rhs(u)
    u2 = 0.75 * u + 0.25 * (u1 - dt * rhs(u1))
    return u / 3.0 + 2.0 / 3.0 * (u2 - dt * rhs(u2))


def substeps_stage(space: HDiv, uV: np.ndarray, dt: float, n: int, l) -> np.ndarray:
    for _ in range(n):
        uV = ssp_rk3(lambda v: stage_rhs(space, v, l), uV, dt)
    return uV


def substeps_frozen(space: HDiv, wV: np.ndarray, uL: np.ndarray, dt: float, n: int, l) -> np.ndarray:
    wL = space.to_l2(wV)
    for _ in range(n):
        uL = ssp_rk3(lambda v: convection.apply(space.topo, space.ref, wL, v, l), uL, dt)
    return uL

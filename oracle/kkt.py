"""KKT optimality measures of a horizon-QP point (a pin on every solve).

For  min 1/2 z^T P z + q^T z  s.t.  E z = e,  lo <= C z <= hi:
  stationarity     |P z + q + E^T nu + C^T y|_inf
  equalities       |E z - e|_inf
  bound violation  max(lo - C z, C z - hi, 0)
  dual sign        y_i > 0 only where the upper bound is finite, y_i < 0 only
                   where the lower bound is finite
  complementarity  max_i  y_i^+ (hi_i - C_i z) + y_i^- (C_i z - lo_i)

Oracle code: test infrastructure only.
"""
from __future__ import annotations

import numpy as np


def kkt_measures(P, q, E, e, C, lo, hi, z, nu, y):
    Cz = C @ z
    stat = P @ z + q + E.T @ nu + C.T @ y
    viol = np.maximum(np.maximum(lo - Cz, Cz - hi), 0.0)
    yp = np.maximum(y, 0.0)
    yn = np.maximum(-y, 0.0)
    sign = np.where(np.isfinite(hi), 0.0, yp) + np.where(np.isfinite(lo), 0.0, yn)
    gap_up = np.where(np.isfinite(hi), hi - Cz, 0.0)
    gap_lo = np.where(np.isfinite(lo), Cz - lo, 0.0)
    comp = yp * gap_up + yn * gap_lo
    return dict(stationarity=float(np.max(np.abs(stat))),
                equality=float(np.max(np.abs(E @ z - e), initial=0.0)),
                violation=float(np.max(viol, initial=0.0)),
                dual_sign=float(np.max(sign, initial=0.0)),
                complementarity=float(np.max(np.abs(comp), initial=0.0)))

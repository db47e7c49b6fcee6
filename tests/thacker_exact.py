"""The analytic solution of Thacker's problem in its damped, non-oscillating form
(Appendix B): uniform velocity (u(t), v(t)) and a planar free surface w(t, x, y) over the
paraboloid z = a (x - x0)^2 + b (y - y0)^2, with linear resistance -tau h v.  For each
direction, with Delta = tau^2 - 8 g a (or b) > 0:
  lambda_1,2 = (-tau -/+ sqrt(Delta)) / 2,
  A = (V0 lambda_2 - V0') / sqrt(Delta),  B = -(V0 lambda_1 - V0') / sqrt(Delta),
  V(t) = A e^{lambda_1 t} + B e^{lambda_2 t},
  W0(t) = [A^2 lambda_2 / lambda_1 (1 - e^{2 lambda_1 t}) + B^2 lambda_1 / lambda_2 (1 - e^{2 lambda_2 t})
           + 2 A B (1 - e^{-tau t})] / (2 g);
  w(t, x, y) = w0 + W0_a(t) + W0_b(t) - (x - x0)(tau u + u')/g - (y - y0)(tau v + v')/g,
  h = [w - z]_+.
"""
import math

import numpy as np


def _branch(t, delta, tau, V0, dV0, g):
    sd = math.sqrt(delta)
    l1, l2 = (-tau - sd) / 2.0, (-tau + sd) / 2.0
    A = (V0 * l2 - dV0) / sd
    B = -(V0 * l1 - dV0) / sd
    e1, e2 = np.exp(l1 * t), np.exp(l2 * t)
    V = A * e1 + B * e2
    dV = A * l1 * e1 + B * l2 * e2
    W0 = (A * A * l2 / l1 * (1.0 - np.exp(2.0 * l1 * t)) + B * B * l1 / l2 * (1.0 - np.exp(2.0 * l2 * t))
          + 2.0 * A * B * (1.0 - np.exp(-tau * t))) / (2.0 * g)
    return V, dV, W0


def solution(T, t, x, y):
    """(u, v, w, h) at time t; x, y arrays of positions [m]."""
    g, tau = T["g"], T["tau"]
    da, db = tau * tau - 8.0 * g * T["a"], tau * tau - 8.0 * g * T["b"]
    assert da > 0 and db > 0, "parameters of the oscillating case"
    u, du, Wa = _branch(t, da, tau, 0.0, T["du0"], g)
    v, dv, Wb = _branch(t, db, tau, 0.0, T["dv0"], g)
    w = T["w0"] + Wa + Wb - (x - T["x0"]) * (tau * u + du) / g - (y - T["y0"]) * (tau * v + dv) / g
    z = T["a"] * (x - T["x0"]) ** 2 + T["b"] * (y - T["y0"]) ** 2
    return u, v, w, np.maximum(w - z, 0.0)

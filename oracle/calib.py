"""Reference of the flume study's host arithmetic, Sec. 4.3 (test infrastructure only).

Written out as the paper states it, one term at a time:
  * h_bar: the mean steady depth over the N_v cells with x_i >= 9 m (Eq. eq_h_bar);
  * delta_s, delta_p: the double sums of forward differences over the regular grid
    alpha_s^i = lo_s + (i - 1) d_s, alpha_p^j = lo_p + (j - 1) d_p, divided by
    (N_s - 1) N_p d_s, respectively N_s (N_p - 1) d_p;
  * chi: the square root of the mean over experiments and gauges of the squared
    difference of measured and computed depths (Eq. eq_chi_6experim);
  * Hooke and Jeeves' pattern search (the direct search the paper uses), evaluating one
    point at a time: exploratory moves coordinate by coordinate (+step, then -step, keep
    any improvement), pattern moves x + (x - base) while they improve, the step halved
    when an exploration around the base fails, until it is below tol.  Coordinates are
    scaled to the box, u = (x - lo) / (hi - lo); a point outside it counts as +inf.
Only tests load this module.
"""
from __future__ import annotations

import math


def h_bar(h, x):
    """h, x: depths and cell-centre abscissae, flat sequences of the same length."""
    total, n = 0.0, 0
    for hi, xi in zip(h, x):
        if xi >= 9.0:
            total += float(hi)
            n += 1
    return total / n


def sensitivity(H, d_s, d_p):
    """H[i][j] = h_bar(alpha_s^i, alpha_p^j), i < N_s, j < N_p."""
    ns, np_ = len(H), len(H[0])
    s = 0.0
    for i in range(ns - 1):
        for j in range(np_):
            s += (float(H[i + 1][j]) - float(H[i][j])) / d_s
    p = 0.0
    for i in range(ns):
        for j in range(np_ - 1):
            p += (float(H[i][j + 1]) - float(H[i][j])) / d_p
    return s / ((ns - 1) * np_), p / (ns * (np_ - 1))


def chi(h_exp, h_sim):
    """h_exp, h_sim: [experiments][gauges]."""
    total, n = 0.0, 0
    for row_e, row_s in zip(h_exp, h_sim):
        for a, b in zip(row_e, row_s):
            total += (float(a) - float(b)) ** 2
            n += 1
    return math.sqrt(total / n)


def hooke_jeeves(f, x0, step, lo, hi, shrink=0.5, tol=1e-3, max_evals=100000):
    """Returns (x, f(x), accepted base points, evaluations)."""
    d = len(x0)
    span = [hi[i] - lo[i] for i in range(d)]
    seen = {}

    def F(u):
        k = tuple(round(v, 12) for v in u)
        if k not in seen:
            if any(v < -1e-12 or v > 1.0 + 1e-12 for v in u):
                seen[k] = math.inf
            else:
                seen[k] = float(f([lo[i] + k[i] * span[i] for i in range(d)]))
        return seen[k]

    def explore(c, fc, s):
        x, fx = list(c), fc
        for i in range(d):
            t = list(x)
            t[i] = x[i] + s[i]
            ft = F(t)
            if ft < fx:
                x, fx = t, ft
                continue
            t = list(x)
            t[i] = x[i] - s[i]
            ft = F(t)
            if ft < fx:
                x, fx = t, ft
        return x, fx

    s = [step[i] / span[i] for i in range(d)]
    b = [(x0[i] - lo[i]) / span[i] for i in range(d)]
    fb = F(b)
    path = [[lo[i] + b[i] * span[i] for i in range(d)]]
    while max(s) >= tol and len(seen) < max_evals:
        x, fx = explore(b, fb, s)
        if fx < fb:
            while True:
                prev, b, fb = b, x, fx
                path.append([lo[i] + b[i] * span[i] for i in range(d)])
                p = [b[i] + (b[i] - prev[i]) for i in range(d)]
                x, fx = explore(p, F(p), s)
                if not fx < fb:
                    break
        else:
            s = [v * shrink for v in s]
    return [lo[i] + b[i] * span[i] for i in range(d)], fb, path, len(seen)

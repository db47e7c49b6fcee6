"""The FP64 scheme's own sensitivity on rough beds (what the rough-bed GPU parity bound
rests on): disturbed at every step by float32-sized rounding, the oracle's 200-step
trajectory on a bed drawn independently per cell moves by more than the stated 1e-4 in
discharge, while on a smooth bed it stays within 1e-5."""
import numpy as np

import oracle
from envelope import per_step_envelope
from paper_2406_14933_gb300 import inputs


def _own_steps(p, m, a, b, n):
    ts, t = [], 0.0
    for _ in range(n):
        r = p.run(m, a, b, t, 1e9, max_steps=1)
        m, a, b, t = r["m"], r["v1"], r["v2"], r["t"]
        ts.append(t)
    return np.array(ts)


def _envelope(smooth):
    sc = inputs.tiny(66, 270, seed=99 + 66, bc=(1, 1, 0, 1), rain_mm_h=40.0, smooth=smooth)
    p = oracle.from_scenario(sc)
    m0, a0, b0 = p.mass(sc.h0), sc.v1_0.ravel().astype(np.float64), sc.v2_0.ravel().astype(np.float64)
    ts = _own_steps(p, m0, a0, b0, 200)
    eh, eq, _ = per_step_envelope(p, m0, a0, b0, ts, seeds=6)
    return eh, eq


def test_rough_bed_amplifies_float32_rounding():
    eh, eq = _envelope(smooth=False)
    assert eq > 1e-4, eq


def test_smooth_bed_does_not():
    eh, eq = _envelope(smooth=True)
    assert eh < 1e-5 and eq < 1e-5, (eh, eq)

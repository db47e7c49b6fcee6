"""Sensitivity envelope of the FP64 scheme (test infrastructure): how far the oracle's
own trajectory moves when every step's state is disturbed by float32-sized rounding.

The GPU keeps velocities in float32 and the mass as a compensated float32 pair, so each
of its steps differs from the FP64 oracle's by rounding of that size.  Where the scheme
turns such differences into larger ones (a wet/dry switch, an upwind or tie decision of
Eqs. fvm_2D_eq.05-06 at a front), no float32 implementation can follow the FP64
trajectory more closely than the FP64 scheme follows itself under the same
disturbances.  `per_step_envelope` measures that: the largest relative L2 distance, over
seeded runs, between the oracle's run on the given time levels and the same run with
every step's velocities moved by -1, 0 or +1 float32 unit in the last place and every
mass by -1, 0 or +1 part in 2^48, chosen at random per cell."""
import numpy as np


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def _nudge(x, rng):
    x32 = x.astype(np.float32)
    s = rng.choice([-1, 0, 1], x.size)
    up, dn = np.nextafter(x32, np.float32(np.inf)), np.nextafter(x32, np.float32(-np.inf))
    return np.where(s > 0, up, np.where(s < 0, dn, x32)).astype(np.float64)


def per_step_envelope(p, m0, a0, b0, ts, seeds=12):
    """(depth, discharge) envelope at the last time level of ts, and the reference run."""
    ref = p.run(m0, a0, b0, 0.0, ts[-1], t_replay=np.asarray(ts))
    h_ref = p.depth(ref["m"])
    q_ref = np.concatenate([ref["m"] * ref["v1"], ref["m"] * ref["v2"]])
    eh = eq = 0.0
    for seed in range(seeds):
        rng = np.random.default_rng(100 + seed)
        m, a, b, tp = m0.copy(), a0.copy(), b0.copy(), 0.0
        for tn in ts:
            m, a, b = p.step(m, a, b, tn - tp, tn)
            tp = tn
            a, b = _nudge(a, rng), _nudge(b, rng)
            m = np.where(m > 0, m * (1.0 + rng.choice([-1, 0, 1], m.size) * 2.0 ** -48), m)
        eh = max(eh, _rel(p.depth(m), h_ref))
        eq = max(eq, _rel(np.concatenate([m * a, m * b]), q_ref))
    return eh, eq, ref

"""Writes fullrun_envelope.txt: the FP64 oracle's own sensitivity on the two large
terrains of the full-run parity tests (test infrastructure; calls only oracle/ and the
seeded input generators).

For each case the oracle runs from the initial state to the horizon with its own CFL
steps (no sample cuts), once undisturbed and once per seed with every step's state
disturbed by float32-sized rounding: velocities moved by -1, 0 or +1 float32 unit in the
last place and masses by -1, 0 or +1 part in 2^48, at random per cell (the size of the
differences between a float32 state with a compensated mass and the float64 one).  The
file records, per case, the largest relative L2 distance over the seeds between the
disturbed and the undisturbed final depth and discharge fields, and between their outlet
outflow totals.

    python tests/golden/make_fullrun_envelope.py [threads]
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2406_14933_gb300 import inputs  # noqa: E402

CASES = {
    "catchment512_whole_storm": (lambda: inputs.carved_catchment(rows=512, cols=512, l=40.0), 7200.0),
    "fractal_basin1024_to_1200s": (lambda: inputs.fractal_basin(), 1200.0),
}
SEEDS = 2


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def _nudge(x, rng):
    x32 = x.astype(np.float32)
    s = rng.choice([-1, 0, 1], x.size)
    up, dn = np.nextafter(x32, np.float32(np.inf)), np.nextafter(x32, np.float32(-np.inf))
    return np.where(s > 0, up, np.where(s < 0, dn, x32)).astype(np.float64)


def envelope(sc, t_end, threads):
    p = oracle.from_scenario(sc, threads=threads)
    m0, a0, b0 = p.mass(sc.h0), sc.v1_0.ravel().astype(np.float64), sc.v2_0.ravel().astype(np.float64)
    ref = p.run(m0, a0, b0, 0.0, t_end)
    q_ref = np.concatenate([ref["m"] * ref["v1"], ref["m"] * ref["v2"]])
    eh = eq = eo = 0.0
    for seed in range(SEEDS):
        rng = np.random.default_rng(100 + seed)
        m, a, b, t = m0.copy(), a0.copy(), b0.copy(), 0.0
        out = 0.0
        while t < t_end:
            dt = min(p.cfl_dt(m, a, b), t_end - t)
            tn = t + dt if t + dt < t_end else t_end
            led = oracle.Ledger()
            m, a, b = p.step(m, a, b, tn - t, tn, ledger=led)
            out += led.outflow
            t = tn
            a, b = _nudge(a, rng), _nudge(b, rng)
            m = np.where(m > 0, m * (1.0 + rng.choice([-1, 0, 1], m.size) * 2.0 ** -48), m)
        eh = max(eh, _rel(p.depth(m), p.depth(ref["m"])))
        eq = max(eq, _rel(np.concatenate([m * a, m * b]), q_ref))
        eo = max(eo, abs(out - ref["ledger"].outflow) / max(abs(ref["ledger"].outflow), 1e-300))
    return eh, eq, eo, ref["steps"]


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else oracle.max_threads()
    lines = ["# case depth_rel_l2 discharge_rel_l2 outflow_rel steps seeds (see make_fullrun_envelope.py)"]
    for name, (make, t_end) in CASES.items():
        eh, eq, eo, steps = envelope(make(), t_end, threads)
        lines.append(f"{name} {eh:.6e} {eq:.6e} {eo:.6e} {steps} {SEEDS}")
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "fullrun_envelope.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()

"""Oracle side of the full-run parity tests, importable by spawned worker processes
(test infrastructure): each call builds its scenario from the seeded generators and runs
the FP64 oracle from the scenario's initial state to its end time with its own CFL steps
and the scenario's hydrograph sample times."""
import numpy as np

import oracle
from paper_2406_14933_gb300 import inputs


def member(s, sample_dt):
    sc = inputs.ensemble_member(s)
    sc.sample_dt = sample_dt
    return sc


def run_to_end(sc, t_end, threads=1, sample_cap=4096):
    p = oracle.from_scenario(sc, threads=threads)
    res = p.run(p.mass(sc.h0), sc.v1_0, sc.v2_0, 0.0, t_end, sample_dt=sc.sample_dt, sample_cap=sample_cap)
    led = res["ledger"]
    return dict(m=res["m"], v1=res["v1"], v2=res["v2"], t=res["t"], steps=res["steps"],
                samples=res["samples"], rain_in=led.rain_in, outflow=led.outflow, clamped=led.clamped,
                storage=p.storage(res["m"]), storage0=p.storage(p.mass(sc.h0)))


def run_member(s, sample_dt, threads=1):
    sc = member(s, sample_dt)
    return run_to_end(sc, sc.t_end, threads=threads)

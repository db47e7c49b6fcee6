"""Crop replay: the FP64 oracle re-runs a few steps of a large raster on small crops of a
state, and the cells far enough inside each crop are compared with the full raster's.

A cell's update reads only its six neighbours, so after k steps a cell at least k rings
inside a crop (or on a true raster side, where the crop keeps the raster's own boundary
condition) depends on nothing outside the crop.  Crops start on even rows so that the
odd-row offset of the hexagons is kept.
"""
import numpy as np

from paper_2406_14933_gb300 import inputs

K_STEPS = 3
CROP = 48


def coeffs(sc, sl):
    if sc.cls is not None:
        k = sc.cls[sl]
        return sc.class_theta[k], sc.class_alpha_s[k], sc.class_alpha_p[k]
    return sc.theta[sl], sc.alpha_s[sl], sc.alpha_p[sl]


def crop_bc(sc, r0, c0):
    """Boundary conditions of a crop: the raster's own on sides it shares with the raster
    (free intervals moved into crop coordinates), walls elsewhere.  Returns (bc, free_range,
    margins W, E, S, N) where a margin is the number of rings not compared on that side."""
    h = w = CROP
    on = (c0 == 0, c0 + w == sc.cols, r0 == 0, r0 + h == sc.rows)      # W, E, S, N
    bc, fr, margin = [], [], []
    for side in range(4):
        if not on[side]:
            bc.append(inputs.WALL)
            fr.append((0, 0))
            margin.append(K_STEPS)
            continue
        b, e = sc.free_range[side]
        off, ext = (c0, w) if side >= 2 else (r0, h)
        if sc.bc[side] == inputs.FREE and b != e:
            b2, e2 = min(max(b - off, 0), ext), min(max(e - off, 0), ext)
            if b2 == e2:
                bc.append(inputs.WALL)
                fr.append((0, 0))
            else:
                bc.append(inputs.FREE)
                fr.append((b2, e2))
        else:
            bc.append(sc.bc[side])
            fr.append((0, 0))
        margin.append(0)
    return tuple(bc), tuple(fr), margin


def pick_crops(sc, rng, n, extra=()):
    out = list(extra)
    while len(out) < n:
        r0 = 2 * int(rng.integers(0, (sc.rows - CROP) // 2 + 1))
        c0 = int(rng.integers(0, sc.cols - CROP + 1))
        out.append((r0, c0))
    return out


def compare_crops(orc, sc, crops, t0, ts, state0, state1):
    """Replays the steps ending at times ts (from t0) on every crop of state0 = (m, v1, v2)
    and compares with state1 on the kept cells.  Returns (depth rel. L2, discharge rel. L2,
    number of cells compared)."""
    m0, a0, b0 = state0
    m1, a1, b1 = state1
    hg, ho, qg, qo = [], [], [], []
    for r0, c0 in crops:
        sl = (slice(r0, r0 + CROP), slice(c0, c0 + CROP))
        th, as_, ap = coeffs(sc, sl)
        bc, fr, (mw, me, ms, mn) = crop_bc(sc, r0, c0)
        p = orc.Problem(CROP, CROP, sc.l, sc.z[sl], th, as_, ap, bc=bc, g=sc.g, cfl=sc.cfl,
                        dt_max=sc.dt_max, rain_t=sc.rain_t, rain_r=sc.rain_r, free_range=fr)
        res = p.run(m0[sl], a0[sl], b0[sl], t0, ts[-1], t_replay=np.array(ts))
        assert res["steps"] == len(ts)
        keep = (slice(ms, CROP - mn), slice(mw, CROP - me))
        mo = res["m"].reshape(CROP, CROP)[keep]
        mg = np.asarray(m1[sl], np.float64)[keep]
        tk = np.asarray(th, np.float64)[keep]
        ho.append(mo / tk)
        hg.append(mg / tk)
        qo += [mo * res["v1"].reshape(CROP, CROP)[keep], mo * res["v2"].reshape(CROP, CROP)[keep]]
        qg += [mg * np.asarray(a1[sl], np.float64)[keep], mg * np.asarray(b1[sl], np.float64)[keep]]

    def rel(a, b):
        a = np.concatenate([x.ravel() for x in a])
        b = np.concatenate([x.ravel() for x in b])
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)), int(b.size)

    (eh, n), (eq, _) = rel(hg, ho), rel(qg, qo)
    return eh, eq, n

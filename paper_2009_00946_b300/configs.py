"""Tomography configurations (plain data).

Each function returns a JSON-serialisable dict describing one instance:
telescope, guide stars / wavefront sensors, turbulence layers, regularisation
weight, deformable mirrors and fitting directions, and the run settings.

The atmosphere profiles are synthetic stand-ins (heights evenly spread, Cn^2
fractions proportional to exp(-h / 3 km), normalised): the standard 9- and
35-layer median profiles are not reproduced here.  The asterisms follow the
MAORY-like setting of Sec. 4.1 (LGS on a 1-arcmin-radius hexagon at 90 km,
fitting/evaluation directions on the 5x5 grid at -60..60 arcsec).

alpha: fixed once, by a one-time scan of the layer reconstruction error
against the synthetic truth on the small NGS configuration (minimum near
100-300), then reused unchanged for every configuration.
"""

from __future__ import annotations

import math

import numpy as np

ARCSEC = math.pi / (180.0 * 3600.0)
R0 = 0.157        # m at 500 nm
L0 = 25.0         # m, outer scale
SIGMA = 0.1       # rad, slope noise
LGS_HEIGHT = 90e3  # m, sodium layer
ALPHA = 200.0     # regularisation weight (one-time scan on the small NGS case: minimum near 100-300)


def synthetic_profile(n_layers: int, h_max: float):
    h = np.linspace(0.0, h_max, n_layers)
    w = np.exp(-h / 3000.0)
    w = w / w.sum()
    return [float(x) for x in h], [float(x) for x in w]


def ring(n: int, radius_arcsec: float, az0_deg: float = 0.0):
    out = []
    for k in range(n):
        az = math.radians(az0_deg + 360.0 * k / n)
        out.append((radius_arcsec * ARCSEC * math.cos(az), radius_arcsec * ARCSEC * math.sin(az)))
    return out


def fit_grid_5x5():
    v = [-60.0, -30.0, 0.0, 30.0, 60.0]
    return [(x * ARCSEC, y * ARCSEC) for y in v for x in v]


def _wfs(dirs, n_sub, H, sigma=SIGMA):
    return [{"n_sub": int(n_sub), "theta_x": float(tx), "theta_y": float(ty),
             "gs_height": float(H), "sigma": float(sigma)} for (tx, ty) in dirs]


def _layers(heights, fracs, n, J):
    return [{"height": float(h), "cn2": float(c), "n": int(n), "levels": int(J)}
            for h, c in zip(heights, fracs)]


def c1_plain():
    """D = 8 m, 3 NGS on a 30-arcsec ring, 16x16 subapertures, 2 layers
    (0 / 6 km, 0.7 / 0.3) on 32^2 / 64^2 grids, db3 with 3 levels, 20 PCG
    iterations from a cold start, one frame, FP64."""
    dirs = []
    for az in (90.0, 210.0, 330.0):
        a = math.radians(az)
        dirs.append((30.0 * ARCSEC * math.cos(a), 30.0 * ARCSEC * math.sin(a)))
    layers = [{"height": 0.0, "cn2": 0.7, "n": 32, "levels": 3},
              {"height": 6000.0, "cn2": 0.3, "n": 64, "levels": 3}]
    return {"name": "c1_plain", "D": 8.0, "obstruction": 0.0, "r0": R0, "L0": L0,
            "alpha": ALPHA, "wfs": _wfs(dirs, 16, 0.0), "layers": layers,
            "n_iter": 20, "warm": False, "k_rr": 0, "frames": 1, "seed": 1,
            "precision": "fp64"}


def c2_elt(n_layer_grid: int = 128, levels: int = 4, frames: int = 1000):
    """ELT MCAO bulk: D = 39 m (28 % obstructed), 6 LGS at 90 km on a
    1-arcmin-radius hexagon, 84x84 subapertures, 9 layers 0-16 km on
    128^2 grids, db3 with 4 levels, 4 warm-started PCG iterations per frame,
    frozen flow at 500 Hz, FP32 with FP64 reductions."""
    h, c = synthetic_profile(9, 16000.0)
    return {"name": "c2_elt", "D": 39.0, "obstruction": 0.28, "r0": R0, "L0": L0,
            "alpha": ALPHA, "wfs": _wfs(ring(6, 60.0), 84, LGS_HEIGHT),
            "layers": _layers(h, c, n_layer_grid, levels),
            "n_iter": 4, "warm": True, "k_rr": 10, "frames": frames, "seed": 2,
            "precision": "fp32"}


def c3_elt_dm(frames: int = 2000):
    """ELT MCAO frame: the c2 asterism, 35 layers 0-25 km on 128^2 grids, db3
    with 4 levels, 3 DMs at 0 / 4 / 12.7 km (pitch 0.5 / 0.67 / 1 m, bilinear)
    fitted over the 5x5 directions at -60..60 arcsec; 4 PCG iterations plus
    the fit per frame."""
    h, c = synthetic_profile(35, 25000.0)
    dms = [{"height": 0.0, "pitch": 0.5}, {"height": 4000.0, "pitch": 0.67},
           {"height": 12700.0, "pitch": 1.0}]
    return {"name": "c3_elt_dm", "D": 39.0, "obstruction": 0.28, "r0": R0, "L0": L0,
            "alpha": ALPHA, "wfs": _wfs(ring(6, 60.0), 84, LGS_HEIGHT),
            "layers": _layers(h, c, 128, 4), "dms": dms, "fit_dirs": fit_grid_5x5(),
            "n_fit": 8, "gain": 1.0,
            "n_iter": 4, "warm": True, "k_rr": 10, "frames": frames, "seed": 3,
            "precision": "fp32"}


def mcao_small(lgs: bool = True):
    """Small MCAO case for closed-loop checks: D = 8 m, 4 guide stars (LGS at
    90 km or NGS) on a 30-arcsec ring, 16x16 subapertures, 3 layers 0-8 km on
    32^2 / 64^2 grids (3 levels), 2 mirrors at 0 / 6 km (pitch 0.5 / 0.8 m),
    3x3 fitting directions within +-30 arcsec."""
    h, c = synthetic_profile(3, 8000.0)
    layers = _layers(h, c, 64, 3)
    layers[0]["n"] = 32
    dirs = [(x * ARCSEC, y * ARCSEC) for y in (-30.0, 0.0, 30.0) for x in (-30.0, 0.0, 30.0)]
    return {"name": "mcao_small", "D": 8.0, "obstruction": 0.0, "r0": R0, "L0": L0, "alpha": ALPHA,
            "wfs": _wfs(ring(4, 30.0, 45.0), 16, LGS_HEIGHT if lgs else 0.0), "layers": layers,
            "dms": [{"height": 0.0, "pitch": 0.5}, {"height": 6000.0, "pitch": 0.8}], "fit_dirs": dirs,
            "n_fit": 8, "gain": 0.5, "n_iter": 4, "warm": True, "k_rr": 10, "frames": 8, "seed": 6,
            "precision": "fp32"}


def maory(n_layers: int = 6, n_iter: int = 4):
    """MAORY-like timing case (Sec. 4.1, Table 2): D = 39 m, 28 % obstructed;
    6 LGS (90 km) with 80x80 subapertures on a 1-arcmin-radius hexagon and 3
    NGS tip-tilt sensors (2x2, 1x1, 1x1) on a 80-arcsec-radius ring; L = M
    layers and mirrors at 0, 4, 8, 12, 16, 20 km (the first n_layers), layer
    grids 128^2 (4 levels), mirrors of 81^2 (0 km), 48^2 (4-16 km) and 54^2
    (20 km) actuators covering the 5x5 +-60-arcsec evaluation grid; fit =
    sampling of each layer at its mirror's actuators; n_iter PCG iterations."""
    heights = [0.0, 4000.0, 8000.0, 12000.0, 16000.0, 20000.0][:n_layers]
    n_act = [81, 48, 48, 48, 48, 54][:n_layers]
    dirs = fit_grid_5x5()
    thmax = max(max(abs(x), abs(y)) for x, y in dirs)
    dms = []
    for h, na in zip(heights, n_act):
        span = 39.0 + 2.0 * thmax * h          # footprint over the evaluation grid
        dms.append({"height": h, "pitch": span / (na - 1.5)})   # -> na actuators per side
    w = np.exp(-np.array(heights) / 3000.0)
    w = w / w.sum()
    lgs = _wfs(ring(6, 60.0, 0.0), 80, LGS_HEIGHT)
    ngs_dirs = ring(3, 80.0, 180.0)
    ngs = _wfs(ngs_dirs[:1], 2, 0.0) + _wfs(ngs_dirs[1:], 1, 0.0)
    return {"name": "maory_%dL" % n_layers, "D": 39.0, "obstruction": 0.28, "r0": R0, "L0": L0,
            "alpha": ALPHA, "wfs": lgs + ngs, "layers": _layers(heights, list(w), 128, 4),
            "dms": dms, "fit_dirs": dirs, "n_fit": 0, "gain": 0.5, "n_iter": n_iter, "warm": True,
            "k_rr": 10, "frames": 200, "seed": 7, "precision": "fp32"}


def ao_mode_small(mode: str = "moao"):
    """Small LTAO / MOAO case (Sec. 1 and 4.3 operating modes): the mcao_small
    asterism and layers (4 LGS 16x16 on a 30-arcsec ring, 3 layers 0-8 km on
    32^2 / 64^2 grids), open loop, 8 fitting CG steps.  LTAO: one mirror at
    0 km (pitch 0.5 m) fitted on axis.  MOAO: three objects at (0, 0),
    (20, 0) and (-15, 15) arcsec, each with its own mirror at 0 km."""
    cfg = dict(mcao_small(True))
    if mode == "ltao":
        cfg.update(name="ltao_small", dms=[{"height": 0.0, "pitch": 0.5}], fit_dirs=[(0.0, 0.0)])
    elif mode == "moao":
        dirs = [(0.0, 0.0), (20.0 * ARCSEC, 0.0), (-15.0 * ARCSEC, 15.0 * ARCSEC)]
        cfg.update(name="moao_small", dms=[{"height": 0.0, "pitch": 0.5} for _ in dirs], fit_dirs=dirs,
                   fit_mode="moao")
    else:
        raise ValueError("mode must be 'ltao' or 'moao'")
    cfg.update(gain=0.5, n_fit=8)
    return cfg


def maory_mode(mode: str = "moao", n_layers: int = 6, n_obj: int = 5):
    """The MAORY-like asterism and layers (maory()) in the LTAO or MOAO
    operating mode (Sec. 4.3 times all three): LTAO, one mirror at 0 km with
    the 81-actuator pitch fitted on axis; MOAO, n_obj objects on the 5x5
    evaluation grid (centre first, then the corners), one such mirror each.
    Least-squares fit with 8 CG steps, open loop."""
    cfg = dict(maory(n_layers, 4))
    pitch = 39.0 / (81 - 1.5)
    grid = fit_grid_5x5()
    order = [12, 0, 4, 20, 24, 2, 10, 14, 22]
    if mode == "ltao":
        cfg.update(name="maory_ltao", dms=[{"height": 0.0, "pitch": pitch}], fit_dirs=[(0.0, 0.0)])
    elif mode == "moao":
        dirs = [grid[i] for i in order[:n_obj]]
        cfg.update(name="maory_moao_%d" % n_obj, dms=[{"height": 0.0, "pitch": pitch} for _ in dirs],
                   fit_dirs=dirs, fit_mode="moao")
    else:
        raise ValueError("mode must be 'ltao' or 'moao'")
    cfg.update(n_fit=8, gain=0.5)
    return cfg


def c4_instance(i: int):
    """Instance i of the uneven batch: D ~ U[8, 39] m, n_s ~ U{16..84} (even),
    L ~ U{2..9} layers 0-16 km, G ~ U{3..6} LGS on a 60-arcsec ring; layer
    grid n = next power of two >= 1.5 * footprint / d, clamped to 32..256;
    J = log2(n) - 3 levels; 4 PCG iterations, FP32."""
    rng = np.random.Generator(np.random.PCG64(4 + i))
    D = float(rng.uniform(8.0, 39.0))
    n_sub = int(rng.integers(8, 43)) * 2
    L = int(rng.integers(2, 10))
    G = int(rng.integers(3, 7))
    h, c = synthetic_profile(L, 16000.0)
    d = D / n_sub
    foot = D + 2.0 * 60.0 * ARCSEC * max(h)
    n = 1 << int(math.ceil(math.log2(1.5 * foot / d)))
    n = int(min(256, max(32, n)))
    J = int(math.log2(n)) - 3
    return {"name": "c4_batch_%02d" % i, "D": D, "obstruction": 0.0, "r0": R0, "L0": L0,
            "alpha": ALPHA, "wfs": _wfs(ring(G, 60.0), n_sub, LGS_HEIGHT),
            "layers": _layers(h, c, n, J),
            "n_iter": 4, "warm": True, "k_rr": 10, "frames": 1, "seed": 4 + i,
            "precision": "fp32"}


def c4_batch(count: int = 64):
    return [c4_instance(i) for i in range(count)]


def c5_autograd():
    """Differentiation: D = 16 m, 4 LGS on a 60-arcsec ring at 90 km, 40x40
    subapertures, 5 layers 0-16 km on 64^2 grids, 3 levels, 4 iterations,
    batch of 32 frames."""
    h, c = synthetic_profile(5, 16000.0)
    return {"name": "c5_autograd", "D": 16.0, "obstruction": 0.0, "r0": R0, "L0": L0,
            "alpha": ALPHA, "wfs": _wfs(ring(4, 60.0), 40, LGS_HEIGHT),
            "layers": _layers(h, c, 64, 3),
            "n_iter": 4, "warm": False, "k_rr": 0, "frames": 32, "seed": 5,
            "precision": "fp32"}


def tiny(n_sub: int = 4, n: int = 8, levels=(1, 2), G: int = 2, lgs: bool = False,
         obstruction: float = 0.0, D: float = 2.0):
    """Small instance for dense checks: D = 2 m, 2 guide stars, 2 layers on
    8^2 grids (1-2 levels)."""
    dirs = ring(G, 20.0, 45.0)
    H = LGS_HEIGHT if lgs else 0.0
    layers = [{"height": 0.0, "cn2": 0.6, "n": n, "levels": int(levels[0])},
              {"height": 5000.0, "cn2": 0.4, "n": n, "levels": int(levels[1])}]
    return {"name": "tiny", "D": D, "obstruction": obstruction, "r0": R0, "L0": L0,
            "alpha": ALPHA, "wfs": _wfs(dirs, n_sub, H), "layers": layers,
            "n_iter": 8, "warm": False, "k_rr": 0, "frames": 1, "seed": 11,
            "precision": "fp64"}


ALL = {"c1_plain": c1_plain, "c2_elt": c2_elt, "c3_elt_dm": c3_elt_dm,
       "c5_autograd": c5_autograd}

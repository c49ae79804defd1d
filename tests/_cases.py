"""Shared GPU test geometries."""

from paper_2009_00946_b300 import configs


def ragged_cfg():
    """Uneven instance: odd subaperture counts, NGS + LGS, obstruction, layers
    of different sizes and level counts (several tiles and ragged edges)."""
    cfg = configs.tiny(n_sub=7, n=16, levels=(3, 1), G=3, lgs=True, obstruction=0.25, D=6.0)
    cfg["wfs"][1]["n_sub"] = 9
    cfg["wfs"][2]["gs_height"] = 0.0
    cfg["layers"][1]["n"] = 64
    cfg["layers"][1]["levels"] = 4
    cfg["layers"].append({"height": 9000.0, "cn2": 0.2, "n": 32, "levels": 2})
    return cfg


def elementwise_check(got, want, sides, tol, border=2, what=""):
    """Per-element bound beside the relative L2 norm: on every n x n layer (or
    mirror) grid, the largest |got - want| on the border strips (the first and
    last `border` rows and columns, where the last-cell tie-break of the
    bilinear tables and the periodic wrap of the DWT act) and over the whole
    grid must stay within tol * max |want| of that grid.  A wrong edge row or
    column, invisible in a norm over hundreds of thousands of elements, fails
    here."""
    import numpy as np
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    o = 0
    for li, n in enumerate(sides):
        g = got[o:o + n * n].reshape(n, n)
        w = want[o:o + n * n].reshape(n, n)
        o += n * n
        scale = max(float(np.max(np.abs(w))), 1e-300)
        d = np.abs(g - w)
        b = max(float(d[:border].max()), float(d[-border:].max()), float(d[:, :border].max()),
                float(d[:, -border:].max()))
        assert b <= tol * scale, ("border", what, li, b / scale)
        assert float(d.max()) <= tol * scale, ("grid", what, li, float(d.max()) / scale)
    assert o == got.size

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

"""One-off scan of the regularisation weight alpha (Eq. fewha: "a scalar factor
alpha for tuning the balance between the fitting and the regularizing terms").

Runs the oracle on the small NGS configuration (and optionally the LGS
autograd-sized one) over a few synthetic frames for a grid of alpha values and
prints the piston-removed relative layer error against the synthetic truth and
the relative error of the on-axis integrated wavefront.  The chosen value is
recorded by hand as ALPHA in paper_2009_00946_b300/configs.py.

Usage: python -m oracle.scan_alpha [--cfg c1_plain|c5_autograd] [--frames 3]
"""

from __future__ import annotations

import argparse

import numpy as np

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cfg", default="c1_plain")
    ap.add_argument("--frames", type=int, default=3)
    ap.add_argument("--iters", type=int, default=20)
    args = ap.parse_args()
    cfg = configs.ALL[args.cfg]()
    S, T = synth.frames(cfg, args.frames)
    for alpha in [1.0, 10.0, 30.0, 100.0, 300.0, 1000.0, 3000.0, 10000.0]:
        cfg["alpha"] = alpha
        R = fo.Reconstructor(cfg)
        g = R.geom
        el, ew = [], []
        for k in range(args.frames):
            R.frame(S[k], args.iters, warm=False)
            phi = R.layers()
            num = den = 0.0
            onaxis_rec = onaxis_true = 0.0
            for l in range(g.L):
                a = phi[g.off[l]:g.off[l + 1]]
                b = T[k][g.off[l]:g.off[l + 1]]
                num += np.sum(((a - a.mean()) - (b - b.mean())) ** 2)
                den += np.sum((b - b.mean()) ** 2)
            el.append(np.sqrt(num / den))
            # on-axis wavefront at the pupil nodes of WFS 0's grid
            x = g.x_nodes[0]
            rec = np.zeros((x.size, x.size))
            tru = np.zeros_like(rec)
            for l in range(g.L):
                u = (x - g.X0[l]) / g.delta[l]
                c, t = fo._bilinear_table(u, g.n[l])
                tab = (c, t, c, t)
                rec += fo.FitGeometry._interp(g.layer(phi, l), tab)
                tru += fo.FitGeometry._interp(T[k][g.off[l]:g.off[l + 1]].reshape(g.n[l], g.n[l]), tab)
            rec -= rec.mean()
            tru -= tru.mean()
            ew.append(np.linalg.norm(rec - tru) / np.linalg.norm(tru))
        print("alpha %8.3f  layer err %.4f  on-axis wavefront err %.4f" % (alpha, np.mean(el), np.mean(ew)))


if __name__ == "__main__":
    main()

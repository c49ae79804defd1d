"""Pins of reading R15 (LGS tip-tilt filter): the right-hand side ignores any
tip / tilt added to a laser guide star's slopes but not to a natural guide
star's; M stays symmetric positive definite with the exact Jacobi diagonal;
the reverse-mode gradients match central differences."""

import copy

import numpy as np
import pytest

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs, synth


def _cfg(lgs=True, tt=True):
    cfg = configs.tiny(n_sub=6, n=8, levels=(2, 2), lgs=lgs, obstruction=0.2)
    cfg["lgs_tip_tilt_filter"] = tt
    return cfg


def test_rhs_ignores_lgs_tip_tilt_only():
    for lgs in (True, False):
        g = fo.Geometry(_cfg(lgs=lgs))
        s = np.random.default_rng(1).standard_normal(g.S)
        t = s.copy()
        for q in range(g.G):
            n = g.n_sub[q]
            blk = t[g.soff[q]:g.soff[q + 1]].reshape(2, n, n)
            blk[0] += 0.7      # tip on every subaperture of sensor q
            blk[1] -= 1.3      # tilt
        d = np.linalg.norm(fo.rhs(g, t) - fo.rhs(g, s)) / np.linalg.norm(fo.rhs(g, s))
        if lgs:
            assert d < 1e-13 and all(g.tt)
        else:
            assert d > 1e-3 and not any(g.tt)


def test_filtered_M_spd_and_exact_jacobi():
    g = fo.Geometry(_cfg())
    M = fo.assemble_M_dense(g)
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh((M + M.T) / 2).min() > 0
    assert np.abs(np.diag(M) - fo.jacobi_diag(g)).max() <= 1e-11 * np.abs(np.diag(M)).max()
    # and the filter lowers the data term: unfiltered M - filtered M is PSD
    M0 = fo.assemble_M_dense(fo.Geometry(_cfg(tt=False)))
    assert np.linalg.eigvalsh((M0 - M + (M0 - M).T) / 2).min() > -1e-10 * np.abs(M0).max()


def test_filtered_reverse_mode_matches_central_differences():
    cfg = _cfg()
    g = fo.Geometry(cfg)
    pr = g.default_params()
    Jinv = 1.0 / fo.jacobi_diag(g, pr)
    S, T = synth.frames(cfg, 1)
    loss, gg, ga, gw = fo.solve_loss_grad(g, pr, Jinv, S[0], T[0], 4)
    h = 1e-6
    for q in range(g.G):
        p1, p2 = copy.deepcopy(pr), copy.deepcopy(pr)
        p1.w[q] *= 1 + h
        p2.w[q] *= 1 - h
        fd = (fo.solve_loss(g, p1, Jinv, S[0], T[0], 4) - fo.solve_loss(g, p2, Jinv, S[0], T[0], 4)) / (2 * h * pr.w[q])
        assert abs(gw[q] - fd) <= 1e-6 * max(abs(gw[q]), 1e-3 * loss), q
    p1, p2 = copy.deepcopy(pr), copy.deepcopy(pr)
    p1.alpha *= 1 + h
    p2.alpha *= 1 - h
    fd = (fo.solve_loss(g, p1, Jinv, S[0], T[0], 4) - fo.solve_loss(g, p2, Jinv, S[0], T[0], 4)) / (2 * h * pr.alpha)
    assert abs(ga - fd) <= 1e-6 * max(abs(ga), 1e-3 * loss)

"""Pins of the oracle's reverse mode through the unrolled Alg. 2: gradients of
|W^T c_K - phi_true|^2 with respect to the Cn^2 fractions, alpha and the
sensor weights against central finite differences of the forward solve (FP64),
and the adjoint identity <J v, u> = <v, J^T u> of the solve map b -> c_K."""

import copy

import numpy as np
import pytest

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs, synth


def _case(name):
    if name == "tiny_lgs":
        cfg = configs.tiny(lgs=True, obstruction=0.2, n_sub=6, levels=(2, 2))
    else:
        cfg = configs.c5_autograd()
    g = fo.Geometry(cfg)
    pr = g.default_params()
    Jinv = 1.0 / fo.jacobi_diag(g, pr)
    S, T = synth.frames(cfg, 1)
    return g, pr, Jinv, S[0], T[0]


@pytest.mark.parametrize("name", ["tiny_lgs", "c5_autograd"])
def test_reverse_mode_matches_central_differences(name):
    g, pr, Jinv, s, phit = _case(name)
    loss, gg, ga, gw = fo.solve_loss_grad(g, pr, Jinv, s, phit, 4)
    L = lambda p: fo.solve_loss(g, p, Jinv, s, phit, 4)
    h = 1e-6

    def fd(set_scaled):
        p1, p2 = copy.deepcopy(pr), copy.deepcopy(pr)
        x = set_scaled(p1, 1 + h)
        set_scaled(p2, 1 - h)
        return (L(p1) - L(p2)) / (2 * h * x)

    for l in range(g.L):
        def sc(p, f, l=l):
            v = p.cn2[l]
            p.cn2[l] = v * f
            return v
        assert abs(gg[l] - fd(sc)) <= 1e-6 * max(abs(gg[l]), 1e-3 * loss), ("gamma", l)

    def sa(p, f):
        v = p.alpha
        p.alpha = v * f
        return v
    assert abs(ga - fd(sa)) <= 1e-6 * max(abs(ga), 1e-3 * loss)
    for q in range(g.G):
        def sw(p, f, q=q):
            v = p.w[q]
            p.w[q] = v * f
            return v
        assert abs(gw[q] - fd(sw)) <= 1e-6 * max(abs(gw[q]), 1e-3 * loss), ("w", q)


def test_solve_map_adjoint_identity():
    g, pr, Jinv, s, _ = _case("tiny_lgs")
    Mop = lambda v: fo.apply_M(g, v, pr)
    b = fo.rhs(g, s, pr)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(g.N)
    u = rng.standard_normal(g.N)
    _, _, tape = fo.pcg_alg2_tape(Mop, Jinv, b, 4)
    bbar, _ = fo.pcg_alg2_adjoint(Mop, Jinv, tape, u)
    eps = 1e-6 * np.linalg.norm(b) / np.linalg.norm(v)
    cp, _, _ = fo.pcg_alg2_tape(Mop, Jinv, b + eps * v, 4)
    cm, _, _ = fo.pcg_alg2_tape(Mop, Jinv, b - eps * v, 4)
    Jv = (cp - cm) / (2 * eps)
    assert abs(Jv @ u - v @ bbar) <= 1e-6 * abs(v @ bbar)


@pytest.mark.parametrize("name", ["tiny_lgs", "c5_autograd"])
def test_slope_gradient_matches_central_differences(name):
    """d loss / d s = C^{-1} Gamma P W^T bbar against central differences of
    the forward solve along random slope directions (the solve is nonlinear in
    s through the CG step lengths, so this checks bbar as well), and zero on
    masked subapertures."""
    g, pr, Jinv, s, phit = _case(name)
    loss, _, _, _, gs = fo.solve_loss_grad(g, pr, Jinv, s, phit, 4, with_slopes=True)
    assert gs.shape == s.shape
    rng = np.random.default_rng(11)
    for _ in range(3):
        v = rng.standard_normal(s.size)
        eps = 1e-5 * np.linalg.norm(s) / np.linalg.norm(v)
        fd = (fo.solve_loss(g, pr, Jinv, s + eps * v, phit, 4) - fo.solve_loss(g, pr, Jinv, s - eps * v, phit, 4)) \
            / (2 * eps)
        assert abs(fd - float(gs @ v)) <= 1e-6 * max(abs(fd), 1e-6 * loss), (fd, float(gs @ v))
    for q in range(g.G):
        gx, gy = g.split_slopes(gs, q)
        assert np.all(gx[g.mask[q] == 0] == 0) and np.all(gy[g.mask[q] == 0] == 0)

"""Differentiation of the solve on the GPU (4-iteration cold-start Alg. 2 on the
autograd configuration: D = 16 m, 4 LGS, 40x40, 5 layers on 64^2, J = 3):
taped forward and reverse mode through the C ABI against the FP64 oracle's
solve and adjoint, central differences of the GPU loss, and the torch
autograd form over a batch of 32 frames."""

import copy

import numpy as np
import pytest

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs, synth

pytestmark = pytest.mark.gpu
N_ITER = 4


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2009_00946_b300 import autograd, fewha
    cfg = configs.c5_autograd()
    g = fo.Geometry(cfg)
    pr = g.default_params()
    Jinv = 1.0 / fo.jacobi_diag(g, pr)
    S, T = synth.frames(cfg, 32)
    return torch, fewha, autograd, cfg, g, pr, Jinv, S, T


def _other_params(pr):
    p = copy.deepcopy(pr)
    p.cn2 = p.cn2 * np.array([1.3, 0.8, 1.1, 0.9, 1.2])
    p.alpha = p.alpha * 0.7
    p.w = p.w * np.array([1.0, 1.5, 0.6, 1.1])
    return p


def _gpu_grads(env, S_, prec, s, phit, params=None):
    torch, fewha = env[0], env[1]
    dt = torch.float64 if prec == fewha.FP64 else torch.float32
    if params is not None:
        S_.set_params(params.cn2, params.alpha, params.w)
    with torch.cuda.stream(S_.stream):   # every tensor made and used on the solver's stream
        sd = torch.from_numpy(np.asarray(s)).to("cuda", dt)
        tape = torch.empty(S_.tape_bytes(N_ITER), dtype=torch.uint8, device="cuda")
        phi = torch.empty(S_.N, dtype=dt, device="cuda")
        S_.solve_taped(sd, N_ITER, tape, phi)
        phibar = 2.0 * (phi - torch.from_numpy(phit).to("cuda", dt))
        gg = torch.empty(S_.n_layers, dtype=torch.float64, device="cuda")
        ga = torch.empty(1, dtype=torch.float64, device="cuda")
        gw = torch.empty(S_.n_wfs, dtype=torch.float64, device="cuda")
        gs = torch.empty_like(sd)
        S_.backward(sd, N_ITER, tape, phibar, gg, ga, gw, gs)
    S_.sync()
    loss = float(((phi.double() - torch.from_numpy(phit).cuda()) ** 2).sum())
    return phi.cpu().numpy(), loss, gg.cpu().numpy(), float(ga.cpu()), gw.cpu().numpy(), gs.cpu().numpy()


def test_taped_solve_and_adjoint_match_oracle_fp64(env):
    torch, fewha, _, cfg, g, pr, Jinv, S, T = env
    with fewha.Solver(cfg, precision=fewha.FP64) as S_:
        phi, loss, gg, ga, gw, gs = _gpu_grads(env, S_, fewha.FP64, S[0], T[0])
    b = fo.rhs(g, S[0], pr)
    c, _, _ = fo.pcg_alg2_tape(lambda v: fo.apply_M(g, v, pr), Jinv, b, N_ITER)
    assert rel(phi, np.concatenate([x.ravel() for x in fo.layers_from_coeffs(g, c)])) < 1e-10
    lo, ogg, oga, ogw, ogs = fo.solve_loss_grad(g, pr, Jinv, S[0], T[0], N_ITER, with_slopes=True)
    assert abs(loss - lo) <= 1e-10 * lo
    assert rel(gg, ogg) < 1e-8 and abs(ga - oga) <= 1e-8 * abs(oga) and rel(gw, ogw) < 1e-8
    assert rel(gs, ogs) < 1e-8                      # slope gradient C^{-1} Gamma P W^T bbar


def test_set_params_then_gradients_match_oracle_fp64(env):
    """New gamma, alpha, w with the create-time preconditioner: M and the
    gradients follow the oracle run with those parameters and the same J."""
    torch, fewha, _, cfg, g, pr, Jinv, S, T = env
    p2 = _other_params(pr)
    with fewha.Solver(cfg, precision=fewha.FP64) as S_:
        S_.set_params(p2.cn2, p2.alpha, p2.w)
        x = synth.random_coeffs(cfg, 3)
        assert rel(S_.apply_M(x), fo.apply_M(g, x, p2)) < 1e-11
        _, loss, gg, ga, gw, _ = _gpu_grads(env, S_, fewha.FP64, S[1], T[1])
    lo, ogg, oga, ogw = fo.solve_loss_grad(g, p2, Jinv, S[1], T[1], N_ITER)
    assert abs(loss - lo) <= 1e-10 * lo
    assert rel(gg, ogg) < 1e-8 and abs(ga - oga) <= 1e-8 * abs(oga) and rel(gw, ogw) < 1e-8


def test_gpu_gradients_match_central_differences_fp64(env):
    """Central differences of the GPU's own FP64 loss (relative steps 1e-6)
    in every parameter and along a random slope direction."""
    torch, fewha, _, cfg, g, pr, Jinv, S, T = env
    with fewha.Solver(cfg, precision=fewha.FP64) as S_:
        _, loss, gg, ga, gw, gs = _gpu_grads(env, S_, fewha.FP64, S[2], T[2], pr)

        def L(p, s=S[2]):
            return _gpu_grads(env, S_, fewha.FP64, s, T[2], p)[1]

        h = 1e-6
        for l in range(g.L):
            p1, p2 = copy.deepcopy(pr), copy.deepcopy(pr)
            p1.cn2[l] *= 1 + h
            p2.cn2[l] *= 1 - h
            fd = (L(p1) - L(p2)) / (2 * h * pr.cn2[l])
            assert abs(gg[l] - fd) <= 1e-5 * max(abs(gg[l]), 1e-3 * loss), ("gamma", l)
        p1, p2 = copy.deepcopy(pr), copy.deepcopy(pr)
        p1.alpha *= 1 + h
        p2.alpha *= 1 - h
        assert abs(ga - (L(p1) - L(p2)) / (2 * h * pr.alpha)) <= 1e-5 * max(abs(ga), 1e-3 * loss)
        for q in range(g.G):
            p1, p2 = copy.deepcopy(pr), copy.deepcopy(pr)
            p1.w[q] *= 1 + h
            p2.w[q] *= 1 - h
            fd = (L(p1) - L(p2)) / (2 * h * pr.w[q])
            assert abs(gw[q] - fd) <= 1e-5 * max(abs(gw[q]), 1e-3 * loss), ("w", q)
        v = np.random.default_rng(7).standard_normal(S_.S)
        eps = 1e-4 * np.linalg.norm(S[2]) / np.linalg.norm(v)
        fd = (L(pr, S[2] + eps * v) - L(pr, S[2] - eps * v)) / (2 * eps)
        assert abs(fd - float(gs @ v)) <= 1e-6 * abs(fd)


def test_fp32_autograd_batch_of_32_frames_matches_oracle(env):
    """torch autograd over the 32-frame batch on an FP32 handle: loss
    sum_f |phi_f - phi_true_f|^2, gradients in gamma, alpha, w against the sum
    of the oracle's FP64 adjoints."""
    torch, fewha, autograd, cfg, g, pr, Jinv, S, T = env
    with fewha.Solver(cfg, precision=fewha.FP32) as S_:
        cn2, alpha, w = autograd.default_params(cfg)
        for t in (cn2, alpha, w):
            t.requires_grad_(True)
        slopes = torch.from_numpy(S.astype(np.float32)).cuda().requires_grad_(True)
        phi = autograd.FewhaSolve.apply(S_, N_ITER, slopes, cn2, alpha, w)
        loss = ((phi.double() - torch.from_numpy(T.reshape(32, -1)).cuda()) ** 2).sum()
        loss.backward()
        got = (cn2.grad.cpu().numpy(), float(alpha.grad.cpu()), w.grad.cpu().numpy())
        assert slopes.grad is not None and slopes.grad.shape == slopes.shape
        gsl = slopes.grad.double().cpu().numpy()
    ref_loss, ogg, oga, ogw = 0.0, np.zeros(g.L), 0.0, np.zeros(g.G)
    for f in range(32):
        lo, a, b, c, gs = fo.solve_loss_grad(g, pr, Jinv, S[f].astype(np.float32).astype(np.float64), T[f], N_ITER,
                                             with_slopes=True)
        ref_loss += lo
        ogg += a
        oga += b
        ogw += c
        assert rel(gsl[f], gs) < 2e-3, (f, rel(gsl[f], gs))   # per-frame slope gradient
    assert abs(float(loss.detach()) - ref_loss) <= 1e-4 * ref_loss
    assert rel(got[0], ogg) < 2e-3, (got[0], ogg)
    assert abs(got[1] - oga) <= 2e-3 * abs(oga), (got[1], oga)
    assert rel(got[2], ogw) < 2e-3, (got[2], ogw)


def _batch_grads(env, S_, dt, s, phit):
    torch = env[0]
    B = s.shape[0]
    with torch.cuda.stream(S_.stream):
        sd = torch.from_numpy(np.ascontiguousarray(s)).to("cuda", dt)
        tape = torch.empty(S_.tape_bytes_batch(N_ITER, B), dtype=torch.uint8, device="cuda")
        phi = torch.empty(B, S_.N, dtype=dt, device="cuda")
        S_.solve_taped_batch(sd, N_ITER, tape, phi)
        phibar = (2.0 * (phi - torch.from_numpy(phit.reshape(B, -1)).to("cuda", dt))).contiguous()
        gg = torch.empty(B, S_.n_layers, dtype=torch.float64, device="cuda")
        ga = torch.empty(B, dtype=torch.float64, device="cuda")
        gw = torch.empty(B, S_.n_wfs, dtype=torch.float64, device="cuda")
        gs = torch.empty_like(sd)
        S_.backward_batch(sd, N_ITER, tape, phibar, gg, ga, gw, gs)
    S_.sync()
    return [t.cpu().numpy() for t in (phi, gg, ga, gw, gs)]


def test_frame_batch_equals_single_frames_bit_for_bit_fp64(env):
    """The frame-batched taped solve and reverse mode (every kernel of the
    chain taking all frames in one launch) give each frame exactly what the
    one-frame calls give -- the same kernels and, per frame, the same
    reduction order -- and match the oracle's adjoint."""
    torch, fewha, _, cfg, g, pr, Jinv, S, T = env
    B = 8
    with fewha.Solver(cfg, precision=fewha.FP64) as S_:
        phi, gg, ga, gw, gs = _batch_grads(env, S_, torch.float64, S[:B], T[:B])
        for f in range(B):
            ph1, _, gg1, ga1, gw1, gs1 = _gpu_grads(env, S_, fewha.FP64, S[f], T[f])
            assert np.array_equal(phi[f], ph1), f
            assert np.array_equal(gg[f], gg1) and ga[f] == ga1 and np.array_equal(gw[f], gw1), f
            assert np.array_equal(gs[f], gs1), f
    for f in (0, B - 1):
        _, ogg, oga, ogw, ogs = fo.solve_loss_grad(g, pr, Jinv, S[f], T[f], N_ITER, with_slopes=True)
        assert rel(gg[f], ogg) < 1e-8 and abs(ga[f] - oga) <= 1e-8 * abs(oga) and rel(gw[f], ogw) < 1e-8, f
        assert rel(gs[f], ogs) < 1e-8, f


def test_frame_batch_launch_count_does_not_grow_with_frames(env):
    """One launch sequence for the whole batch: 32 frames take as many kernel
    launches as one frame."""
    torch, fewha, _, cfg, g, pr, Jinv, S, T = env
    with fewha.Solver(cfg, precision=fewha.FP32) as S_:
        n0 = S_.launch_count()
        _batch_grads(env, S_, torch.float32, S[:1].astype(np.float32), T[:1])
        n1 = S_.launch_count() - n0
        _batch_grads(env, S_, torch.float32, S.astype(np.float32), T)
        n32 = S_.launch_count() - n0 - n1
        assert n1 > 0 and n32 == n1, (n1, n32)

"""Parity of the plain CUDA path (one kernel per operator) with the FP64 oracle,
through the C ABI.  Bars: FP64 GPU <= 1e-10 relative L2 against the oracle
(operator tables and single applications <= 1e-12); FP32 <= 1e-4."""

import numpy as np
import pytest

from _cases import elementwise_check

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs, synth

from _cases import ragged_cfg

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def fw():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2009_00946_b300 import fewha
    return fewha


FP64_CFGS = {"c1": configs.c1_plain, "ragged": ragged_cfg,
             "tiny_lgs": lambda: configs.tiny(lgs=True, obstruction=0.3, n_sub=6, levels=(2, 2))}


@pytest.mark.parametrize("name", list(FP64_CFGS))
def test_fp64_tables_match_oracle(fw, name):
    cfg = FP64_CFGS[name]()
    g = fo.Geometry(cfg)
    pr = g.default_params()
    with fw.Solver(cfg, precision=fw.FP64) as S:
        assert S.N == g.N and S.S == g.S
        aD = S.vector(fw.VEC_ALPHA_D)
        Jd = S.vector(fw.VEC_JACOBI)
    want_aD = pr.alpha * g.D_diag(pr)
    assert np.max(np.abs(aD - want_aD) / want_aD) < 1e-12
    want_J = fo.jacobi_diag(g, pr)
    assert np.max(np.abs(Jd - want_J) / want_J) < 1e-11


@pytest.mark.parametrize("name", list(FP64_CFGS))
def test_fp64_apply_M_matches_oracle(fw, name):
    cfg = FP64_CFGS[name]()
    g = fo.Geometry(cfg)
    x = synth.random_coeffs(cfg, 21)
    with fw.Solver(cfg, precision=fw.FP64) as S:
        y = S.apply_M(x)
    assert rel(y, fo.apply_M(g, x)) < 1e-12


@pytest.mark.parametrize("name", list(FP64_CFGS))
def test_fp64_rhs_matches_oracle(fw, name):
    cfg = FP64_CFGS[name]()
    g = fo.Geometry(cfg)
    s = synth.random_slopes(cfg, 22)
    with fw.Solver(cfg, precision=fw.FP64) as S:
        S.set_frame(s)
        S.solve(1, warm=False)
        S.sync()
        b = S.vector(fw.VEC_B)
    assert rel(b, fo.rhs(g, s)) < 1e-12


def test_c1_fp64_frame_matches_oracle(fw):
    """Plain FEWHA, FP64, 20 iterations from a cold start: c, phi, b <= 1e-10."""
    cfg = configs.c1_plain()
    S_in, _ = synth.frames(cfg, 1)
    R = fo.Reconstructor(cfg)
    out = R.frame(S_in[0], 20, warm=False)
    with fw.Solver(cfg, precision=fw.FP64) as S:
        S.set_frame(S_in[0])
        S.solve(20, warm=False)
        S.sync()
        c = S.vector(fw.VEC_C)
        b = S.vector(fw.VEC_B)
        phi = S.layers()
    assert rel(b, out["b"]) < 1e-12
    assert rel(c, out["c"]) < 1e-10
    assert rel(phi, R.layers()) < 1e-10
    elementwise_check(phi, R.layers(), [l["n"] for l in cfg["layers"]], 1e-9, what="c1 fp64")


def test_fp64_warm_frames_with_replacement(fw):
    cfg = configs.c5_autograd()
    cfg["warm"] = True
    S_in, _ = synth.frames(cfg, 7)
    R = fo.Reconstructor(cfg)
    with fw.Solver(cfg, precision=fw.FP64, k_rr=3) as S:
        for k in range(7):
            o = R.frame(S_in[k], 4, warm=True, k_rr=3)
            S.set_frame(S_in[k])
            S.solve(4, warm=True)
            S.sync()
            assert rel(S.vector(fw.VEC_C), o["c"]) < 1e-10, k
            assert rel(S.vector(fw.VEC_R), o["r"]) < 1e-9, k


def test_fp64_fit_matches_oracle(fw):
    cfg = configs.tiny(n_sub=6, n=16, levels=(2, 2), D=4.0)
    cfg["fit_dirs"] = [(x * fo.ARCSEC, y * fo.ARCSEC) for y in (-20.0, 20.0) for x in (-20.0, 0.0, 20.0)]
    cfg["dms"] = [{"height": 0.0, "pitch": 0.5}, {"height": 5000.0, "pitch": 0.8}]
    S_in, _ = synth.frames(cfg, 3)
    R = fo.Reconstructor(cfg)
    with fw.Solver(cfg, precision=fw.FP64) as S:
        for k in range(3):
            o = R.frame(S_in[k], 6, warm=True, k_rr=0, gain=0.4, n_fit=8)
            S.set_residual_replacement(0)
            S.set_frame(S_in[k])
            S.solve(6, warm=True)
            a = S.fit_dm(0.4, 8)
            assert rel(a, o["a"]) < 1e-10, k


def test_fp32_plain_elt_frames_match_oracle(fw):
    """ELT bulk (84x84, 6 LGS, 9 layers 128^2, 4 warm iterations), FP32 plain
    path, 12 frames across a residual replacement: layers <= 1e-4."""
    cfg = configs.c2_elt()
    S_in, _ = synth.frames(cfg, 12)
    R = fo.Reconstructor(cfg)
    with fw.Solver(cfg, precision=fw.FP32, path=fw.PATH_PLAIN, k_rr=10) as S:
        for k in range(12):
            R.frame(S_in[k], 4, warm=True, k_rr=10)
            S.set_frame(S_in[k].astype(np.float32))
            S.solve(4, warm=True)
            S.sync()
            assert rel(S.layers(), R.layers()) < 1e-4, k
            elementwise_check(S.layers(), R.layers(), [l["n"] for l in cfg["layers"]], 1e-3, what=k)


def test_nan_slopes_reported(fw):
    cfg = configs.c2_elt()
    g = fo.Geometry(cfg)
    s = synth.random_slopes(cfg, 3).astype(np.float32)
    with fw.Solver(cfg, precision=fw.FP32, path=fw.PATH_PLAIN) as S:
        bad = s.copy()
        inactive = int(np.flatnonzero(g.mask[0].ravel() == 0)[0])
        bad[inactive] = np.nan                      # masked subaperture: ignored
        S.set_frame(bad)
        S.solve(2, warm=False)
        S.sync()
        active = int(np.flatnonzero(g.mask[0].ravel() == 1)[0])
        bad[active] = np.nan
        S.set_frame(bad)
        S.solve(2, warm=False)
        with pytest.raises(fw.FewhaError) as ei:
            S.sync()
        assert ei.value.name == "INPUT"


def test_plain_deterministic_and_state_roundtrip(fw):
    cfg = configs.c5_autograd()
    S_in, _ = synth.frames(cfg, 3)
    outs = []
    for _ in range(2):
        with fw.Solver(cfg, precision=fw.FP32, path=fw.PATH_PLAIN) as S:
            for k in range(3):
                S.set_frame(S_in[k].astype(np.float32))
                S.solve(4, warm=True)
            S.sync()
            outs.append(S.vector(fw.VEC_C))
            state = S.get_state()
    assert np.array_equal(outs[0], outs[1])
    with fw.Solver(cfg, precision=fw.FP32, path=fw.PATH_PLAIN) as S2:
        S2.set_state(*state, frame_count=3)
        with fw.Solver(cfg, precision=fw.FP32, path=fw.PATH_PLAIN) as S1:
            S1.set_state(*state, frame_count=3)
            for S in (S1, S2):
                S.set_frame(S_in[0].astype(np.float32))
                S.solve(4, warm=True)
                S.sync()
            assert np.array_equal(S1.vector(fw.VEC_C), S2.vector(fw.VEC_C))


def test_frame_graph_matches_stepwise_fp64(fw):
    cfg = configs.c5_autograd()
    S_in, _ = synth.frames(cfg, 3)
    with fw.Solver(cfg, precision=fw.FP64) as A, fw.Solver(cfg, precision=fw.FP64) as B:
        for k in range(3):
            A.set_frame(S_in[k])
            A.solve(4, warm=True)
            la = A.layers()
            lb = np.empty_like(la)
            B.frame(np.ascontiguousarray(S_in[k]), 4, warm=True, layers_out=lb)
            assert np.array_equal(la, lb), k

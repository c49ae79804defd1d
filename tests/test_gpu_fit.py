"""ELT frame with mirror fitting (35 layers, 3 DMs at 0 / 4 / 12.7 km, 5x5
fitting directions): FP32 fused solve + fit <= 1e-4 and FP64 plain <= 1e-10
against the oracle, on the mirror commands and the layers."""

import numpy as np
import pytest

from _cases import elementwise_check

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs, synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def fw():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2009_00946_b300 import fewha
    return fewha


@pytest.fixture(scope="module")
def c3_ref():
    cfg = configs.c3_elt_dm()
    S_in, _ = synth.frames(cfg, 3)
    R = fo.Reconstructor(cfg)
    ref = []
    for k in range(3):
        o = R.frame(S_in[k], 4, warm=True, k_rr=10, gain=0.4, n_fit=8)
        ref.append((o["a"].copy(), R.layers()))
    return cfg, S_in, ref


def test_c3_fp32_fused_frame_graph_matches_oracle(fw, c3_ref):
    cfg, S_in, ref = c3_ref
    with fw.Solver(cfg, precision=fw.FP32, k_rr=10) as S:
        S.set_path(fw.PATH_FUSED)
        assert S.NA == sum(n * n for n in (79, 63, 48))
        dm = np.empty(S.NA, np.float32)
        lay = np.empty(S.N, np.float32)
        for k in range(3):
            S.frame(np.ascontiguousarray(S_in[k], dtype=np.float32), 4, warm=True, gain=0.4, n_fit=8,
                    layers_out=lay, dm_out=dm)
            assert rel(lay, ref[k][1]) < 1e-4, k
            assert rel(dm, ref[k][0]) < 1e-4, k
            elementwise_check(lay, ref[k][1], [l["n"] for l in cfg["layers"]], 1e-3, what=k)
            elementwise_check(dm, ref[k][0], [79, 63, 48], 1e-3, what=("dm", k))


def test_c3_fp64_plain_matches_oracle(fw, c3_ref):
    cfg, S_in, ref = c3_ref
    with fw.Solver(cfg, precision=fw.FP64, k_rr=10) as S:
        for k in range(2):
            S.set_frame(S_in[k])
            S.solve(4, warm=True)
            a = S.fit_dm(0.4, 8)
            assert rel(a, ref[k][0]) < 1e-10, k


def test_fit_without_mirrors_is_a_state_error(fw):
    cfg = configs.c5_autograd()
    with fw.Solver(cfg, precision=fw.FP32) as S:
        S.set_frame(np.zeros(S.S, np.float32))
        S.solve(1, warm=False)
        with pytest.raises(fw.FewhaError) as ei:
            S.fit_dm(1.0, 8)
        assert ei.value.name == "STATE"


def test_describe_and_phase_trace(fw):
    """The plan summary names the path; a traced fused frame records one
    arrival/departure pair per CTA at each grid barrier, in time order."""
    cfg = configs.c5_autograd()
    s = synth.random_slopes(cfg, 5).astype(np.float32)
    with fw.Solver(cfg, precision=fw.FP32) as S:
        S.set_path(fw.PATH_FUSED)
        assert "fused" in S.describe()
        S.set_trace(True)
        S.set_frame(s)
        S.solve(3, warm=False)
        S.sync()
        tr = S.trace().astype(np.int64)
        assert tr.shape[0] == 3 + 2 * 3 and tr.shape[2] == 2
        assert np.all(tr[:, :, 1] >= tr[:, :, 0])
        assert np.all(tr[1:, :, 0] >= tr[:-1, :, 1])
    with fw.Solver(cfg, precision=fw.FP64) as S:
        assert "plain" in S.describe()
        with pytest.raises(fw.FewhaError):
            S.set_trace(True)

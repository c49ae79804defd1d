"""The level-weighted (modified) Jacobi preconditioner on the GPU (reading
R18): the handle's preconditioner diagonal equals the oracle's, and warm-started
frames with the weights match the FP64 oracle -- FP64 plain <= 1e-10, FP32
fused frame graph <= 1e-4 on the layers."""

import copy

import numpy as np
import pytest

from oracle import fewha_oracle as fo
from paper_2009_00946_b300 import configs, synth

pytestmark = pytest.mark.gpu
WEIGHTS = [1.0, 0.5, 0.25]
N_FR = 6


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def fw():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2009_00946_b300 import fewha
    return fewha


@pytest.fixture(scope="module")
def weighted():
    cfg = copy.deepcopy(configs.c5_autograd())
    cfg["jacobi_level_weights"] = WEIGHTS
    S_in, _ = synth.frames(cfg, N_FR)
    R = fo.Reconstructor(cfg)
    ref = []
    for k in range(N_FR):
        R.frame(S_in[k], 4, warm=True, k_rr=10)
        ref.append(R.layers())
    return cfg, S_in, ref


def test_preconditioner_diagonal_matches_oracle(fw, weighted):
    cfg, _, _ = weighted
    g = fo.Geometry(cfg)
    with fw.Solver(cfg, precision=fw.FP64) as S:
        got = S.vector(fw.VEC_JACOBI)
    want = fo.preconditioner_diag(g)
    assert rel(got, want) < 1e-12
    assert rel(got, fo.jacobi_diag(g)) > 1e-3   # the weights are in effect


def test_weighted_frames_match_oracle(fw, weighted):
    import torch
    cfg, S_in, ref = weighted
    with fw.Solver(cfg, precision=fw.FP64, path=fw.PATH_PLAIN, k_rr=10) as S:
        for k in range(N_FR):
            S.set_frame(S_in[k])
            S.solve(4, warm=True)
            assert rel(S.layers(), ref[k]) < 1e-10, k
    with fw.Solver(cfg, precision=fw.FP32, k_rr=10) as S:
        S.set_path(fw.PATH_FUSED)
        ds = torch.empty(S.S, dtype=torch.float32, device="cuda")
        dl = torch.empty(S.N, dtype=torch.float32, device="cuda")
        for k in range(N_FR):
            with torch.cuda.stream(S.stream):
                ds.copy_(torch.from_numpy(S_in[k].astype(np.float32)).cuda())
            S.stream.synchronize()
            S.frame(ds, 4, warm=True, layers_out=dl)
            S.sync()
            assert rel(dl.cpu().numpy(), ref[k]) < 1e-4, k


def test_invalid_weight_refused(fw):
    cfg = copy.deepcopy(configs.c5_autograd())
    cfg["jacobi_level_weights"] = [1.0, -2.0]
    with pytest.raises(ValueError):
        fw.Solver(cfg, precision=fw.FP32)

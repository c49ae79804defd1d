"""The allocation-free layer reconstruction, fewha_layers_noalloc.

It exists for callers that cannot allocate device memory (a control loop that
reserves everything at start-up, code inside a framework that owns the device
memory).  Its output must match the handle-based fewha_get_layers, which
computes the same W^{-1} c with memory it allocated at create time.  This file
is collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""

import ctypes

import numpy as np
import pytest

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


def _noalloc(fw, cfg, coeffs_dev, out_dev, stream):
    L = len(cfg["layers"])
    n = (ctypes.c_int * L)(*[l["n"] for l in cfg["layers"]])
    J = (ctypes.c_int * L)(*[l["levels"] for l in cfg["layers"]])
    msg = ctypes.create_string_buffer(256)
    st = fw.lib().fewha_layers_noalloc(ctypes.c_void_p(coeffs_dev.data_ptr()), ctypes.c_void_p(out_dev.data_ptr()),
                                       L, n, J, ctypes.c_void_p(stream.cuda_stream), msg, 256)
    return st, msg.value.decode()


@pytest.mark.parametrize("name", ["c2_elt", "c1_plain"])
def test_noalloc_layers_match_get_layers_on_two_calls(fw, name):
    import torch
    cfg = configs.ALL[name]()
    with fw.Solver(cfg, precision=fw.FP32, path=fw.PATH_PLAIN) as S:
        stream = S.stream
        out = torch.empty(S.N, dtype=torch.float32, device="cuda")
        for call in range(2):
            c = synth.random_coeffs(cfg, 100 + call).astype(np.float32)
            zeros = np.zeros(S.N, np.float32)
            S.set_state(c, zeros, zeros, frame_count=0)
            want = S.layers()                            # existing entry point
            c_dev = torch.from_numpy(c).to("cuda")
            torch.cuda.synchronize()
            st, msg = _noalloc(fw, cfg, c_dev, out, stream)
            assert st == 0, msg
            stream.synchronize()
            got = out.cpu().numpy()
            assert rel(got, want.astype(np.float64)) < 1e-6, (name, call)


def test_noalloc_rejects_sizes_beyond_its_scratch(fw):
    import torch
    cfg = configs.c3_elt_dm()
    cfg["layers"] = cfg["layers"][:1] * 17
    for l in cfg["layers"]:
        l["n"], l["levels"] = 256, 4            # 17 * 256^2 > 2^20 coefficients
    x = torch.zeros(8, dtype=torch.float32, device="cuda")
    y = torch.zeros(8, dtype=torch.float32, device="cuda")
    st, msg = _noalloc(fw, cfg, x, y, torch.cuda.current_stream())
    assert st == 1, msg                          # FEWHA_ERR_ARG, nothing enqueued
    assert "scratch" in msg

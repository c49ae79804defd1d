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


def _mixed_levels_cfg():
    """Layers of different sides and DWT level counts, so that the coarse
    levels of the deeper layers run while the shallower layers skip them."""
    cfg = configs.c1_plain()
    base = cfg["layers"][0]
    cfg["layers"] = [dict(base, height=0.0, n=64, levels=2), dict(base, height=3000.0, n=128, levels=4),
                     dict(base, height=6000.0, n=256, levels=5), dict(base, height=9000.0, n=32, levels=3)]
    return cfg


def test_noalloc_mixed_levels_match_oracle_and_get_layers(fw):
    import torch

    from oracle import fewha_oracle as fo
    cfg = _mixed_levels_cfg()
    sides = [l["n"] for l in cfg["layers"]]
    with fw.Solver(cfg, precision=fw.FP32, path=fw.PATH_PLAIN) as S:
        out = torch.empty(S.N, dtype=torch.float32, device="cuda")
        for call in range(2):
            c = synth.random_coeffs(cfg, 300 + call).astype(np.float32)
            zeros = np.zeros(S.N, np.float32)
            S.set_state(c, zeros, zeros, frame_count=0)
            want_lib = S.layers().astype(np.float64)
            want, o = [], 0
            for l, n in zip(cfg["layers"], sides):       # the oracle's synthesis, layer by layer
                want.append(fo.inv_dwt2(c[o:o + n * n].astype(np.float64).reshape(n, n), l["levels"]).ravel())
                o += n * n
            want = np.concatenate(want)
            c_dev = torch.from_numpy(c).to("cuda")
            torch.cuda.synchronize()
            st, msg = _noalloc(fw, cfg, c_dev, out, S.stream)
            assert st == 0, msg
            S.stream.synchronize()
            got = out.cpu().numpy().astype(np.float64)
            assert rel(got, want) < 1e-6, call
            assert rel(got, want_lib) < 1e-6, call
            o = 0
            for n in sides:                              # every layer on its own, element by element
                g, w = got[o:o + n * n], want[o:o + n * n]
                assert np.max(np.abs(g - w)) <= 1e-5 * np.max(np.abs(w)), (n, call)
                o += n * n


def test_noalloc_rejects_overlapping_buffers(fw):
    import torch
    cfg = configs.c1_plain()
    N = sum(l["n"] ** 2 for l in cfg["layers"])
    buf = torch.zeros(2 * N, dtype=torch.float32, device="cuda")
    # layers start 4 floats into the coefficient range: a partial overlap
    st, msg = _noalloc(fw, cfg, buf, buf[4:], torch.cuda.current_stream())
    assert st == 1 and "overlap" in msg, msg
    st, msg = _noalloc(fw, cfg, buf[4:], buf, torch.cuda.current_stream())
    assert st == 1 and "overlap" in msg, msg


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
